// explicit.cu -- plain Levenberg-Marquardt over the full vector (shape, alpha, beta), the
// comparison method of the paper's claim that implicit amplitudes need fewer iterations
// (Results and Discussion). Model h_i = alpha f_i + beta (Eq. 10 for f), per-pixel Jacobian
// (alpha df_i/dp_j, f_i, 1) (Eq. 11 for df/dp), normal equations J^T J and J^T (g - h)
// (Eq. 12), the damped solve of Eq. 14 and the damping schedule and stop tests of the
// implicit fit (the Fit2DGaussian listing): lambda = 10^k from k = -2, accept -> k - 1,
// reject -> k + 1 and solve again while k < 4, stop on MAX_ERROR, MIN_DELTA, MIN_STEP (on the
// shape parameters), NO_DECREASE, NOT_CONVERGED or the iteration budget. alpha and beta are
// not boxed; the shape parameters are (limit() box). Start amplitudes: alpha0 = max g - min g,
// beta0 = min g.
//
// One warp per spot, lanes over the pixels (row-major, 32 apart, in registers for the whole
// fit). FP32; pixels enter shifted by the integer nearest min g (exact for integer pixels),
// and residuals are formed as g' - fma(alpha, e, beta'). The 5 or 6 unknowns are solved by a
// Cholesky factorisation of the Jacobi-scaled damped matrix, unrolled in registers; the
// isotropic model fills the sigma_y slot with an identity row.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fitspots.h"

namespace {

constexpr int kExThreads = 128;
constexpr int kQ = 6;                      // (x0, y0, sx, sy, alpha, beta)
constexpr int kNA = kQ * (kQ + 1) / 2;     // packed upper triangle of J^T J

struct ExArgs {
  const void *images;
  int dtype;
  int64_t image_elems;
  const int64_t *offsets;
  const int32_t *dims;
  const float *init;
  const uint8_t *model;
  int32_t n;
  int max_iter;
  float max_error, min_delta, min_step;
  float *out_params, *out_alpha, *out_beta, *out_chi2;
  int32_t *out_state, *out_iters, *out_evals;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int tri(int j, int k) {  // packed index of (j, k), j <= k
  return j * kQ - j * (j - 1) / 2 + (k - j);
}

// (A + lambda diag A) d = b for the 6 unknowns, A packed; false if not positive definite or
// the step is not finite.
__device__ __forceinline__ bool solve6(const float (&A)[kNA], const float (&b)[kQ], float lam,
                                       float (&d)[kQ]) {
  float s[kQ], L[kQ][kQ], y[kQ];
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    const float a = A[tri(j, j)];
    if (!(a > 0.f)) return false;
    s[j] = rsqrtf(a);
  }
  const float dg = 1.f + lam;
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
#pragma unroll
    for (int k = 0; k <= j; ++k) {
      float t = (j == k) ? dg : A[tri(k, j)] * s[j] * s[k];
#pragma unroll
      for (int m = 0; m < k; ++m) t -= L[j][m] * L[k][m];
      if (j == k) {
        if (!(t > 0.f)) return false;
        L[j][j] = sqrtf(t);
      } else {
        L[j][k] = t / L[k][k];
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    float t = b[j] * s[j];
#pragma unroll
    for (int k = 0; k < j; ++k) t -= L[j][k] * y[k];
    y[j] = t / L[j][j];
  }
#pragma unroll
  for (int j = kQ - 1; j >= 0; --j) {
    float t = y[j];
#pragma unroll
    for (int k = j + 1; k < kQ; ++k) t -= L[k][j] * d[k];
    d[j] = t / L[j][j];
  }
  bool ok = true;
#pragma unroll
  for (int j = 0; j < kQ; ++j) {
    d[j] *= s[j];
    ok = ok && isfinite(d[j]);
  }
  return ok;
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) {
  v = (v < lo) ? lo : v;
  return (v > hi) ? hi : v;
}

template <typename T>
__global__ void __launch_bounds__(kExThreads) explicit_kernel(ExArgs a) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (kExThreads / 32);
  for (int s = blockIdx.x * (kExThreads / 32) + (threadIdx.x >> 5); s < a.n; s += warps) {
    const int W = a.dims[2 * s], H = a.dims[2 * s + 1], m = a.model[s];
    const int64_t off = a.offsets[s];
    const bool iso = m == FS_MODEL_ISO;
    const int P = iso ? 3 : 4, N = W * H;
    if (!((m == FS_MODEL_ISO || m == FS_MODEL_ELLIPTIC) && W >= 3 && H >= 3 && W <= 32 &&
          H <= 32 && N > P + 2 && off >= 0 && off + N <= a.image_elems)) {
      if (lane == 0) {
        for (int j = 0; j < 4; ++j) a.out_params[4 * s + j] = a.init[4 * s + j];
        a.out_alpha[s] = a.out_beta[s] = a.out_chi2[s] = __int_as_float(0x7fc00000);
        a.out_state[s] = FS_STATE_INVALID_ROI;
        a.out_iters[s] = 0;
        if (a.out_evals) a.out_evals[s] = 0;
      }
      continue;
    }
    // pixels of this lane: i = lane + 32 k
    const T *const img = static_cast<const T *>(a.images) + off;
    float g[32];
    float lo = INFINITY, hi = -INFINITY;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int i = lane + 32 * k;
      g[k] = i < N ? (float)__ldg(img + i) : 0.f;
      if (i < N) {
        lo = fminf(lo, g[k]);
        hi = fmaxf(hi, g[k]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const float sh = rintf(lo);
#pragma unroll
    for (int k = 0; k < 32; ++k) g[k] = (lane + 32 * k < N) ? g[k] - sh : 0.f;
    const int sy = 32 / W, sx = 32 - sy * W;
    const int x_start = lane % W, y_start = lane / W;
    const float smax = (float)max(W, H);
    auto limit = [&](float (&q)[kQ]) {
      q[0] = clampf(q[0], -0.5f, (float)W - 0.5f);
      q[1] = clampf(q[1], -0.5f, (float)H - 0.5f);
      q[2] = clampf(q[2], 0.25f, smax);
      q[3] = iso ? q[2] : clampf(q[3], 0.25f, smax);
    };
    // chi^2 and, with grad, J^T J and J^T r at q (all lanes get the totals)
    auto evaluate = [&](const float (&q)[kQ], bool grad, float (&A)[kNA], float (&b)[kQ]) -> float {
      const float ivx = 1.f / (q[2] * q[2]), ivy = 1.f / (q[3] * q[3]);
      const float cx = ivx / q[2], cy = ivy / q[3];
      float c2 = 0.f, acc[kNA + kQ];
#pragma unroll
      for (int j = 0; j < kNA + kQ; ++j) acc[j] = 0.f;
      int x = x_start, y = y_start;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if (lane + 32 * k < N) {
          const float dx = (float)x - q[0], dy = (float)y - q[1];
          const float e = __expf(-0.5f * (dx * dx * ivx + dy * dy * ivy));
          const float r = g[k] - fmaf(q[4], e, q[5]);
          c2 = fmaf(r, r, c2);
          if (grad) {
            const float ae = q[4] * e;
            float J[kQ];
            J[0] = ae * dx * ivx;
            J[1] = ae * dy * ivy;
            if (iso) {
              J[2] = ae * (dx * dx + dy * dy) * cx;
              J[3] = 0.f;
            } else {
              J[2] = ae * dx * dx * cx;
              J[3] = ae * dy * dy * cy;
            }
            J[4] = e;
            J[5] = 1.f;
#pragma unroll
            for (int j = 0; j < kQ; ++j) {
              acc[kNA + j] = fmaf(J[j], r, acc[kNA + j]);
#pragma unroll
              for (int l = j; l < kQ; ++l) acc[tri(j, l)] = fmaf(J[j], J[l], acc[tri(j, l)]);
            }
          }
        }
        x += sx;
        y += sy;
        if (x >= W) {
          x -= W;
          ++y;
        }
      }
      c2 = warp_sum(c2);
      if (grad) {
#pragma unroll
        for (int j = 0; j < kNA; ++j) A[j] = warp_sum(acc[j]);
#pragma unroll
        for (int j = 0; j < kQ; ++j) b[j] = warp_sum(acc[kNA + j]);
        if (iso) {  // the sigma_y slot: an identity row and a zero right-hand side
#pragma unroll
          for (int j = 0; j < kQ; ++j) A[j <= 3 ? tri(j, 3) : tri(3, j)] = 0.f;
          A[tri(3, 3)] = 1.f;
          b[3] = 0.f;
        }
      }
      return isfinite(c2) ? c2 : __int_as_float(0x7fc00000);
    };
    auto all_small = [&](const float (&d)[kQ], const float (&p)[kQ]) {
      bool sm = true;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < P) sm = sm && fabsf(d[j]) < a.min_step * fabsf(p[j]);
      return sm;
    };

    float q[kQ];
#pragma unroll
    for (int j = 0; j < 4; ++j) q[j] = a.init[4 * s + j];
    if (iso) q[3] = q[2];
    limit(q);
    q[4] = hi - lo;
    q[5] = lo - sh;
    float A[kNA], b[kQ], best[kQ], dl[kQ], qt[kQ];
    int klam = -2, it = 0, evals = 0, state = FS_STATE_MAX_ITER;
    while (it < a.max_iter) {
      ++it;
      ++evals;
      const float chi = evaluate(q, true, A, b);
      if (isnan(chi)) {
        state = FS_STATE_NOT_CONVERGED;
        break;
      }
      if (chi < a.max_error) {
        state = FS_STATE_MAX_ERROR;
        break;
      }
#pragma unroll
      for (int j = 0; j < kQ; ++j) best[j] = q[j];
      auto trial = [&]() -> float {
#pragma unroll
        for (int j = 0; j < kQ; ++j) qt[j] = best[j] + dl[j];
        limit(qt);
        float Ad[kNA], bd[kQ];
        return evaluate(qt, false, Ad, bd);
      };
      if (!solve6(A, b, exp10f((float)klam), dl)) {
        state = FS_STATE_NOT_CONVERGED;
        break;
      }
      ++evals;
      float Chi = trial();
      if (chi > Chi) --klam;
      bool failed = false;
      while (!all_small(dl, best) && chi < Chi && klam < 4) {
        ++klam;
        if (!solve6(A, b, exp10f((float)klam), dl)) {
          failed = true;
          break;
        }
        ++evals;
        Chi = trial();
      }
      if (failed) {
        state = FS_STATE_NOT_CONVERGED;
        break;
      }
      if (chi < Chi || isnan(Chi)) {
        state = (all_small(dl, best) && !isnan(Chi)) ? FS_STATE_NO_DECREASE
                                                     : FS_STATE_NOT_CONVERGED;
        break;
      }
#pragma unroll
      for (int j = 0; j < kQ; ++j) q[j] = qt[j];
      if (Chi < a.max_error) {
        state = FS_STATE_MAX_ERROR;
        break;
      }
      if (chi * (1.f - a.min_delta) < Chi) {
        state = FS_STATE_MIN_DELTA;
        break;
      }
      if (all_small(dl, best)) {
        state = FS_STATE_MIN_STEP;
        break;
      }
    }
    float Ad[kNA], bd[kQ];
    const float chi = evaluate(q, false, Ad, bd);
    if (lane == 0) {
      a.out_params[4 * s] = q[0];
      a.out_params[4 * s + 1] = q[1];
      a.out_params[4 * s + 2] = q[2];
      a.out_params[4 * s + 3] = iso ? q[2] : q[3];
      a.out_alpha[s] = q[4];
      a.out_beta[s] = q[5] + sh;
      a.out_chi2[s] = chi / (float)(N - P - 2);
      a.out_state[s] = state;
      a.out_iters[s] = it;
      if (a.out_evals) a.out_evals[s] = evals;
    }
  }
}

}  // namespace

extern "C" int fit_spots_explicit(const void *images, int dtype, int64_t image_elems,
                                  const int64_t *offsets, const int32_t *roi_dims,
                                  const float *init_params, const uint8_t *model, int64_t n,
                                  int max_iter, double max_error, double min_delta,
                                  double min_step, float *out_params, float *out_alpha,
                                  float *out_beta, float *out_chi2, int32_t *out_state,
                                  int32_t *out_iters, int32_t *out_evals, void *stream) {
  if (n < 0 || n > FS_MAX_SPOTS || image_elems < 0) return FS_ERR_SIZE;
  if (dtype != FS_U16 && dtype != FS_F32) return FS_ERR_DTYPE;
  if (max_iter < 1 || max_iter > 1000) return FS_ERR_MAX_ITER;
  if (!(max_error >= 0.0) || !isfinite(max_error) || !(min_delta >= 0.0) || !(min_delta < 1.0) ||
      !(min_step >= 0.0) || !isfinite(min_step))
    return FS_ERR_TOL;
  if (n == 0) return FS_OK;
  if (!images || !offsets || !roi_dims || !init_params || !model || !out_params || !out_alpha ||
      !out_beta || !out_chi2 || !out_state || !out_iters)
    return FS_ERR_NULL;
  ExArgs a;
  a.images = images;
  a.dtype = dtype;
  a.image_elems = image_elems;
  a.offsets = offsets;
  a.dims = roi_dims;
  a.init = init_params;
  a.model = model;
  a.n = (int32_t)n;
  a.max_iter = max_iter;
  a.max_error = (float)max_error;
  a.min_delta = (float)min_delta;
  a.min_step = (float)min_step;
  a.out_params = out_params;
  a.out_alpha = out_alpha;
  a.out_beta = out_beta;
  a.out_chi2 = out_chi2;
  a.out_state = out_state;
  a.out_iters = out_iters;
  a.out_evals = out_evals;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return FS_ERR_CUDA;
  const int per_block = kExThreads / 32;
  int64_t blocks = (n + per_block - 1) / per_block;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  if (dtype == FS_U16)
    explicit_kernel<unsigned short>
        <<<(int)blocks, kExThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  else
    explicit_kernel<float><<<(int)blocks, kExThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
