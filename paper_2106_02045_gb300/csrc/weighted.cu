// weighted.cu -- variance-weighted implicit-amplitude fit (sm_103a).
//
// The paper's fit minimises the unweighted chi^2 (Eq. 2) and notes that its residuals are
// not weighted; this variant minimises chi^2_w = sum w_i (g_i - alpha f_i - beta)^2 with
// w_i = 1 / max(g_i, 1), the Poisson variance estimated from the data. The implicit
// amplitudes solve the weighted form of Eq. 5-6,
//   [Sff Sf; Sf Sw] (alpha, beta) = (Sfg, Sg)   (Sw = sum w, Sf = sum w f, Sff = sum w f^2,
//                                                Sg = sum w g, Sfg = sum w f g),
// their derivatives the same equations differentiated in p (Eq. 7-8 with weights), the
// per-pixel Jacobian is J_ij = dalpha_j f_i + alpha df_i/dp_j + dbeta_j (Eq. 9), and the LM
// step solves (J^T W J + lambda diag) delta = J^T W (g - h) (Eq. 12, 14) with the damping
// schedule, limit() box and stop tests of the unweighted fit. With all weights 1 it is the
// unweighted fit.
//
// One warp per spot, lanes over the pixels (in registers for the whole fit). The weights
// break the separability the unweighted kernels use, so every evaluation makes two
// per-pixel passes: the amplitude sums and their derivatives, then the residuals, chi^2_w,
// J^T W J and J^T W r. FP32; pixels enter shifted by the integer nearest min g (the weights
// use the unshifted values).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fitspots.h"
#include "warp_lm.cuh"

namespace {

using namespace fs_warp;

constexpr int kWThreads = 128;

struct WArgs {
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

template <typename T>
__global__ void __launch_bounds__(kWThreads) weighted_kernel(WArgs a) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (kWThreads / 32);
  for (int s = blockIdx.x * (kWThreads / 32) + (threadIdx.x >> 5); s < a.n; s += warps) {
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
    const T *const img = static_cast<const T *>(a.images) + off;
    float g[32];
    float lo = INFINITY;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int i = lane + 32 * k;
      g[k] = i < N ? (float)__ldg(img + i) : 0.f;
      if (i < N) lo = fminf(lo, g[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    const float sh = rintf(lo);
#pragma unroll
    for (int k = 0; k < 32; ++k) g[k] = (lane + 32 * k < N) ? g[k] - sh : 0.f;
    const int stepy = 32 / W, stepx = 32 - stepy * W;
    const int x_start = lane % W, y_start = lane / W;
    const float smax = (float)max(W, H);
    auto limit = [&](float (&p)[4]) {
      p[0] = clampf(p[0], -0.5f, (float)W - 0.5f);
      p[1] = clampf(p[1], -0.5f, (float)H - 0.5f);
      p[2] = clampf(p[2], 0.25f, smax);
      p[3] = iso ? p[2] : clampf(p[3], 0.25f, smax);
    };
    // chi^2_w at p, and with grad the normal equations (isotropic: width slot 3 an identity
    // row); alpha and beta (relative to the shift) are returned as well
    auto evaluate = [&](const float (&p)[4], bool grad, float &alpha, float &beta, float (&A)[10],
                        float (&b)[4]) -> float {
      const float ivx = 1.f / (p[2] * p[2]), ivy = 1.f / (p[3] * p[3]);
      const float cx = ivx / p[2], cy = ivy / p[3];
      // pass 1: weighted amplitude sums and their derivatives
      float S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // Sw Sf Sff Sg Sfg
      float dS[3][4];                           // dSf dSff dSfg per shape parameter
#pragma unroll
      for (int j = 0; j < 4; ++j) dS[0][j] = dS[1][j] = dS[2][j] = 0.f;
      {
        int x = x_start, y = y_start;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          if (lane + 32 * k < N) {
            const float dx = (float)x - p[0], dy = (float)y - p[1];
            const float e = __expf(-0.5f * (dx * dx * ivx + dy * dy * ivy));
            const float w = 1.f / fmaxf(g[k] + sh, 1.f);
            const float we = w * e;
            S[0] += w;
            S[1] += we;
            S[2] = fmaf(we, e, S[2]);
            S[3] = fmaf(w, g[k], S[3]);
            S[4] = fmaf(we, g[k], S[4]);
            if (grad) {
              float ph[4];
              ph[0] = dx * ivx;
              ph[1] = dy * ivy;
              ph[2] = iso ? (dx * dx + dy * dy) * cx : dx * dx * cx;
              ph[3] = iso ? 0.f : dy * dy * cy;
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float wd = we * ph[j];  // w df/dp_j
                dS[0][j] += wd;
                dS[1][j] = fmaf(2.f * wd, e, dS[1][j]);
                dS[2][j] = fmaf(wd, g[k], dS[2][j]);
              }
            }
          }
          x += stepx;
          y += stepy;
          if (x >= W) {
            x -= W;
            ++y;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 5; ++j) S[j] = warp_sum(S[j]);
      const float D = fmaf(S[0], S[2], -S[1] * S[1]);
      if (!(D > 0.f) || !isfinite(D)) return __int_as_float(0x7fc00000);
      const float iD = 1.f / D;
      alpha = (S[0] * S[4] - S[1] * S[3]) * iD;
      beta = (S[2] * S[3] - S[1] * S[4]) * iD;
      float da[4] = {0.f, 0.f, 0.f, 0.f}, db[4] = {0.f, 0.f, 0.f, 0.f};
      if (grad) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float dSf = warp_sum(dS[0][j]), dSff = warp_sum(dS[1][j]);
          const float dSfg = warp_sum(dS[2][j]);
          // Sff a + Sf b = Sfg and Sf a + Sw b = Sg, differentiated in p_j
          const float r1 = dSfg - dSff * alpha - dSf * beta, r2 = -dSf * alpha;
          da[j] = (S[0] * r1 - S[1] * r2) * iD;
          db[j] = (S[2] * r2 - S[1] * r1) * iD;
        }
      }
      // pass 2: residuals, chi^2_w and the normal equations
      float c2 = 0.f, acc[14];
#pragma unroll
      for (int j = 0; j < 14; ++j) acc[j] = 0.f;
      {
        int x = x_start, y = y_start;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          if (lane + 32 * k < N) {
            const float dx = (float)x - p[0], dy = (float)y - p[1];
            const float e = __expf(-0.5f * (dx * dx * ivx + dy * dy * ivy));
            const float w = 1.f / fmaxf(g[k] + sh, 1.f);
            const float r = g[k] - fmaf(alpha, e, beta);
            const float wr = w * r;
            c2 = fmaf(wr, r, c2);
            if (grad) {
              const float ae = alpha * e;
              float J[4];
              J[0] = fmaf(ae, dx * ivx, fmaf(da[0], e, db[0]));
              J[1] = fmaf(ae, dy * ivy, fmaf(da[1], e, db[1]));
              J[2] = fmaf(ae, iso ? (dx * dx + dy * dy) * cx : dx * dx * cx, fmaf(da[2], e, db[2]));
              J[3] = iso ? 0.f : fmaf(ae, dy * dy * cy, fmaf(da[3], e, db[3]));
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                acc[10 + j] = fmaf(J[j], wr, acc[10 + j]);
                const float wj = w * J[j];
#pragma unroll
                for (int l = j; l < 4; ++l) acc[tri4(j, l)] = fmaf(wj, J[l], acc[tri4(j, l)]);
              }
            }
          }
          x += stepx;
          y += stepy;
          if (x >= W) {
            x -= W;
            ++y;
          }
        }
      }
      c2 = warp_sum(c2);
      if (grad) {
#pragma unroll
        for (int j = 0; j < 10; ++j) A[j] = warp_sum(acc[j]);
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = warp_sum(acc[10 + j]);
        if (iso) {
          A[tri4(0, 3)] = A[tri4(1, 3)] = A[tri4(2, 3)] = 0.f;
          A[tri4(3, 3)] = 1.f;
          b[3] = 0.f;
        }
      }
      return isfinite(c2) ? c2 : __int_as_float(0x7fc00000);
    };
    float p[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = a.init[4 * s + j];
    if (iso) p[3] = p[2];
    limit(p);
    const LmResult lm = lm_drive(p, iso, P, a.max_iter, a.max_error, a.min_delta, a.min_step,
                                 evaluate, limit);
    float al, be;
    float Ad[10], bd[4];
    const float chi = evaluate(p, false, al, be, Ad, bd);
    if (lane == 0) {
      a.out_params[4 * s] = p[0];
      a.out_params[4 * s + 1] = p[1];
      a.out_params[4 * s + 2] = p[2];
      a.out_params[4 * s + 3] = iso ? p[2] : p[3];
      a.out_alpha[s] = al;
      a.out_beta[s] = be + sh;
      a.out_chi2[s] = chi / (float)(N - P - 2);
      a.out_state[s] = lm.state;
      a.out_iters[s] = lm.iters;
      if (a.out_evals) a.out_evals[s] = lm.evals;
    }
  }
}

}  // namespace

extern "C" int fit_spots_weighted(const void *images, int dtype, int64_t image_elems,
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
  WArgs a;
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
  const int per_block = kWThreads / 32;
  int64_t blocks = (n + per_block - 1) / per_block;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  if (dtype == FS_U16)
    weighted_kernel<unsigned short>
        <<<(int)blocks, kWThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  else
    weighted_kernel<float><<<(int)blocks, kWThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
