// poisson.cu -- Poisson-likelihood implicit-amplitude fit (sm_103a).
//
// The paper's fit minimises the unweighted chi^2 (Eq. 2) of photon-counting images. This
// variant maximises the Poisson likelihood of the counts instead: the objective is the
// deviance D(p) = 2 sum [h - g + g ln(g / h)] of the model h = alpha f(p) + beta, and alpha,
// beta are implicit as in Eq. 5-6 -- at every evaluated p they are the likelihood's optimum
// for the profile f(p), the root of the score equations sum (g/h - 1) (f, 1) = 0. That root
// is found by iteratively reweighted least squares: the weighted Eq. 5-6 with weights 1/h at
// the current means, written as the correction
//   [Sff Sf; Sf Sw] (dalpha, dbeta) = (sum (g/h - 1) f, sum (g/h - 1)),   Sxy = sum x y / h,
// started from the amplitudes of the previously evaluated point (the unweighted amplitudes of
// Eq. 6 at the first point, or where the previous ones give a mean <= 0; a flat model at the
// mean count where those do too), each correction halved while it would make a mean <= 0.
// The log-likelihood is strictly concave in (alpha, beta), so the root is unique and its
// value does not depend on the path to it.
//
// The LM step (Eq. 12, 14) uses the deviance's own gradient and Fisher information: by the
// envelope theorem -1/2 dD/dp_j = sum (g/h - 1) alpha df/dp_j, and the normal matrix is
// sum J J^T / h over the part J = alpha df/dp - (c f + e) of alpha df/dp that the amplitudes
// cannot absorb ((c, e) its least squares on (f, 1) with weights 1/h). Damping schedule,
// limit() box and stop tests are the unweighted fit's, applied to D.
//
// One warp per spot, lanes over the pixels: counts and profile values in registers for the
// whole fit (ROIs up to 32 x 32). FP32; negative pixel values count as 0.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fitspots.h"
#include "warp_lm.cuh"

namespace {

using namespace fs_warp;

constexpr int kPThreads = 128;
constexpr int kIrlsMax = 40;        // amplitude iterations per evaluated point
constexpr float kIrlsTol = 1e-6f;   // stop once a correction is below this x (|alpha| + |beta|)
// deviance changes within this fraction of the deviance of 0 or of the min_delta threshold are
// recomputed from the parameter difference (the FP32 model values leave D about 1e-7 relative)
constexpr float kTieWindow = 1e-6f;

struct PArgs {
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

// 1/x on the MUFU unit (about 1 ulp); x is a positive normal number here
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One pixel's deviance term h - g + g ln(g / h) (h > 0). With s = (h - g) / (h + g) and
// ln(g / h) = -2 atanh(s), it is (h - g) s - 2 g (s^3/3 + s^5/5 + ...): for |s| <= 0.2 that
// series (to s^13, truncation below 3e-10 of the term) keeps full relative precision where h
// is close to g and the direct form would cancel.
__device__ __forceinline__ float deviance_term(float g, float h) {
  if (!(g > 0.f)) return h;
  const float r = h - g, s = r * rcp_approx(h + g);
  if (fabsf(s) <= 0.2f) {
    const float s2 = s * s;
    float q = fmaf(s2, 1.f / 13.f, 1.f / 11.f);
    q = fmaf(s2, q, 1.f / 9.f);
    q = fmaf(s2, q, 1.f / 7.f);
    q = fmaf(s2, q, 1.f / 5.f);
    q = fmaf(s2, q, 1.f / 3.f);
    return fmaf(r, s, -2.f * g * s * s2 * q);
  }
  const float u = r * rcp_approx(g);
  return g * (u - log1pf(u));
}

template <typename T>
__global__ void __launch_bounds__(kPThreads) poisson_kernel(PArgs a) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (kPThreads / 32);
  for (int s = blockIdx.x * (kPThreads / 32) + (threadIdx.x >> 5); s < a.n; s += warps) {
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
    float G = 0.f;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int i = lane + 32 * k;
      g[k] = i < N ? fmaxf((float)__ldg(img + i), 0.f) : 0.f;
      G += g[k];
    }
    const float flat = fmaxf(warp_sum(G) / (float)N, 1e-3f);
    const int stepy = 32 / W, stepx = 32 - stepy * W;
    const int x_start = lane % W, y_start = lane / W;
    const float smax = (float)max(W, H);
    // amplitudes of the last evaluated point: the next point's start (the optimum it reaches
    // does not depend on the start); NaN until the first evaluation
    float warm_a = __int_as_float(0x7fc00000), warm_b = 0.f;
    auto limit = [&](float (&p)[4]) {
      p[0] = clampf(p[0], -0.5f, (float)W - 0.5f);
      p[1] = clampf(p[1], -0.5f, (float)H - 0.5f);
      p[2] = clampf(p[2], 0.25f, smax);
      p[3] = iso ? p[2] : clampf(p[3], 0.25f, smax);
    };
    // the deviance at p, the amplitudes there and, with grad, the Fisher normal equations
    auto evaluate = [&](const float (&p)[4], bool grad, float &alpha, float &beta, float (&A)[10],
                        float (&b)[4]) -> double {
      const float ivx = 1.f / (p[2] * p[2]), ivy = 1.f / (p[3] * p[3]);
      const float cx = ivx / p[2], cy = ivy / p[3];
      // the profile and its range
      float e[32];
      float fmin = INFINITY, fmax = 0.f;
      {
        int x = x_start, y = y_start;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          e[k] = 0.f;
          if (lane + 32 * k < N) {
            const float dx = (float)x - p[0], dy = (float)y - p[1];
            e[k] = __expf(-0.5f * (dx * dx * ivx + dy * dy * ivy));
            fmin = fminf(fmin, e[k]);
            fmax = fmaxf(fmax, e[k]);
          }
          x += stepx;
          y += stepy;
          if (x >= W) {
            x -= W;
            ++y;
          }
        }
      }
      fmin = warp_min(fmin);
      fmax = warp_max(fmax);
      // smallest mean of alpha f + beta over the ROI (f spans [fmin, fmax])
      auto low = [&](float al, float be) { return be + fminf(al * fmin, al * fmax); };
      float al = warm_a, be = warm_b;
      if (!(low(al, be) > 0.f)) {
        // the unweighted amplitudes of Eq. 6, else a flat model at the mean count
        float S1 = 0.f, S2 = 0.f, Sg = 0.f, Seg = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          S1 += e[k];
          S2 = fmaf(e[k], e[k], S2);
          Sg += g[k];
          Seg = fmaf(e[k], g[k], Seg);
        }
        S1 = warp_sum(S1);
        S2 = warp_sum(S2);
        Sg = warp_sum(Sg);
        Seg = warp_sum(Seg);
        const float Nf = (float)N, Du = fmaf(Nf, S2, -S1 * S1);
        al = (Nf * Seg - S1 * Sg) / Du;
        be = (S2 * Sg - S1 * Seg) / Du;
        if (!(Du > 0.f) || !(low(al, be) > 0.f)) {
          al = 0.f;
          be = flat;
        }
      }
      // amplitudes: reweighted least squares on the score equations
      for (int it = 0; it < kIrlsMax; ++it) {
        float Sw = 0.f, Sf = 0.f, Sff = 0.f, s1 = 0.f, s0 = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          if (lane + 32 * k < N) {
            const float w = rcp_approx(fmaf(al, e[k], be));
            const float we = w * e[k], r = fmaf(g[k], w, -1.f);
            Sw += w;
            Sf += we;
            Sff = fmaf(we, e[k], Sff);
            s1 = fmaf(r, e[k], s1);
            s0 += r;
          }
        }
        Sw = warp_sum(Sw);
        Sf = warp_sum(Sf);
        Sff = warp_sum(Sff);
        s1 = warp_sum(s1);
        s0 = warp_sum(s0);
        const float Dt = fmaf(Sff, Sw, -Sf * Sf);
        if (!(Dt > 0.f) || !isfinite(Dt)) return (double)NAN;
        const float da = (Sw * s1 - Sf * s0) / Dt, db = (Sff * s0 - Sf * s1) / Dt;
        float t = 1.f;
        while (t > 1e-6f && !(low(al + t * da, be + t * db) > 0.f)) t *= 0.5f;
        if (!(low(al + t * da, be + t * db) > 0.f)) break;
        al += t * da;
        be += t * db;
        const float scale = kIrlsTol * (fabsf(al) + fabsf(be));
        if (fabsf(t * da) <= scale && fabsf(t * db) <= scale) break;
      }
      alpha = warm_a = al;
      beta = warm_b = be;
      // the deviance (compensated sums in each lane, FP64 across the warp: the LM compares
      // deviances that differ in their eighth digit); with grad the weighted moments of
      // alpha df/dp
      float Dv = 0.f, Dc = 0.f, Sw = 0.f, Sf = 0.f, Sff = 0.f, vf[4], v1[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) vf[j] = v1[j] = 0.f;
      {
        int x = x_start, y = y_start;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          if (lane + 32 * k < N) {
            const float h = fmaf(al, e[k], be);
            const float dterm = deviance_term(g[k], h) - Dc, dsum = Dv + dterm;
            Dc = (dsum - Dv) - dterm;
            Dv = dsum;
            if (grad) {
              const float w = rcp_approx(h), we = w * e[k];
              Sw += w;
              Sf += we;
              Sff = fmaf(we, e[k], Sff);
              const float dx = (float)x - p[0], dy = (float)y - p[1], ae = al * e[k];
              float ad[4];
              ad[0] = ae * (dx * ivx);
              ad[1] = ae * (dy * ivy);
              ad[2] = ae * (iso ? (dx * dx + dy * dy) * cx : dx * dx * cx);
              ad[3] = iso ? 0.f : ae * (dy * dy * cy);
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                vf[j] = fmaf(we, ad[j], vf[j]);
                v1[j] = fmaf(w, ad[j], v1[j]);
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
      const double Dev = 2.0 * warp_sum((double)Dv - (double)Dc);
      if (!isfinite(Dev)) return (double)NAN;
      if (!grad) return Dev;
      Sw = warp_sum(Sw);
      Sf = warp_sum(Sf);
      Sff = warp_sum(Sff);
      const float Dt = fmaf(Sff, Sw, -Sf * Sf);
      if (!(Dt > 0.f) || !isfinite(Dt)) return (double)NAN;
      const float iD = 1.f / Dt;
      float c[4], c0[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float f1 = warp_sum(vf[j]), u1 = warp_sum(v1[j]);
        c[j] = (Sw * f1 - Sf * u1) * iD;
        c0[j] = (Sff * u1 - Sf * f1) * iD;
      }
      // the score in p and the Fisher matrix of the part of alpha df/dp that the amplitudes
      // cannot absorb
      float acc[14];
#pragma unroll
      for (int j = 0; j < 14; ++j) acc[j] = 0.f;
      {
        int x = x_start, y = y_start;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          if (lane + 32 * k < N) {
            const float w = rcp_approx(fmaf(al, e[k], be)), r = fmaf(g[k], w, -1.f);
            const float dx = (float)x - p[0], dy = (float)y - p[1], ae = al * e[k];
            float ad[4], J[4];
            ad[0] = ae * (dx * ivx);
            ad[1] = ae * (dy * ivy);
            ad[2] = ae * (iso ? (dx * dx + dy * dy) * cx : dx * dx * cx);
            ad[3] = iso ? 0.f : ae * (dy * dy * cy);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              J[j] = ad[j] - fmaf(c[j], e[k], c0[j]);
              acc[10 + j] = fmaf(r, ad[j], acc[10 + j]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float wj = w * J[j];
#pragma unroll
              for (int l = j; l < 4; ++l) acc[tri4(j, l)] = fmaf(wj, J[l], acc[tri4(j, l)]);
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
      for (int j = 0; j < 10; ++j) A[j] = warp_sum(acc[j]);
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = warp_sum(acc[10 + j]);
      if (iso) {
        A[tri4(0, 3)] = A[tri4(1, 3)] = A[tri4(2, 3)] = 0.f;
        A[tri4(3, 3)] = 1.f;
        b[3] = 0.f;
      }
      return Dev;
    };

    // The deviance change D(t) - D(b) between the best point b and a trial t, for decisions
    // near a tie: per pixel 2 [dh - g log1p(dh / h_b)], dh = h_t - h_b formed from the
    // parameter difference (the exponent difference in closed form, expm1 of it), so the
    // change keeps its relative precision where D(t) and D(b) agree in their leading digits.
    auto refine = [&](const float (&pb)[4], float ab, float bb, const float (&pt)[4], float at,
                      float bt) -> double {
      const float ivxb = 1.f / (pb[2] * pb[2]), ivyb = 1.f / (pb[3] * pb[3]);
      const float ivxt = 1.f / (pt[2] * pt[2]), ivyt = 1.f / (pt[3] * pt[3]);
      const float d0 = pt[0] - pb[0], d1 = pt[1] - pb[1];
      // ivx_b - ivx_t = (s_t - s_b)(s_t + s_b) ivx_t ivx_b, likewise for y
      const float kx = (pt[2] - pb[2]) * (pt[2] + pb[2]) * ivxt * ivxb;
      const float ky = (pt[3] - pb[3]) * (pt[3] + pb[3]) * ivyt * ivyb;
      const float dal = at - ab, dbe = bt - bb;
      float acc = 0.f;
      int x = x_start, y = y_start;
#pragma unroll 4
      for (int k = 0; k < 32; ++k) {
        if (lane + 32 * k < N) {
          const float dxb = (float)x - pb[0], dyb = (float)y - pb[1];
          const float dxt = dxb - d0, dyt = dyb - d1;
          // exponent at t minus exponent at b
          const float da = 0.5f * (d0 * (dxt + dxb) * ivxt + dxb * dxb * kx +
                                   d1 * (dyt + dyb) * ivyt + dyb * dyb * ky);
          const float eb = __expf(-0.5f * (dxb * dxb * ivxb + dyb * dyb * ivyb));
          const float dh = fmaf(at * eb, expm1f(da), fmaf(dal, eb, dbe));
          const float hb = fmaf(ab, eb, bb);
          const float gk = g[k];
          acc += gk > 0.f ? dh - gk * log1pf(dh / hb) : dh;
        }
        x += stepx;
        y += stepy;
        if (x >= W) {
          x -= W;
          ++y;
        }
      }
      return 2.0 * warp_sum((double)acc);
    };

    float p[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = a.init[4 * s + j];
    if (iso) p[3] = p[2];
    limit(p);
    const LmResult lm = lm_drive(p, iso, P, a.max_iter, a.max_error, a.min_delta, a.min_step,
                                 evaluate, limit, refine, kTieWindow);
    float al, be, Ad[10], bd[4];
    const double dv = evaluate(p, false, al, be, Ad, bd);
    if (lane == 0) {
      a.out_params[4 * s] = p[0];
      a.out_params[4 * s + 1] = p[1];
      a.out_params[4 * s + 2] = p[2];
      a.out_params[4 * s + 3] = iso ? p[2] : p[3];
      a.out_alpha[s] = al;
      a.out_beta[s] = be;
      a.out_chi2[s] = (float)(dv / (double)(N - P - 2));
      a.out_state[s] = lm.state;
      a.out_iters[s] = lm.iters;
      if (a.out_evals) a.out_evals[s] = lm.evals;
    }
  }
}

}  // namespace

extern "C" int fit_spots_poisson(const void *images, int dtype, int64_t image_elems,
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
  PArgs a;
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
  const int per_block = kPThreads / 32;
  int64_t blocks = (n + per_block - 1) / per_block;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  if (dtype == FS_U16)
    poisson_kernel<unsigned short>
        <<<(int)blocks, kPThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  else
    poisson_kernel<float><<<(int)blocks, kPThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
