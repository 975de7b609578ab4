// warp_lm.cuh -- pieces shared by the one-warp-per-spot comparison fits (weighted.cu,
// poisson.cu): warp reductions, the damped 4 x 4 solve and the Levenberg-Marquardt driver
// with the paper's damping schedule, limit() box and stop tests (Sec. 2, Eq. 12-14).
//
// The driver is generic in the objective: `evaluate(p, grad, alpha, beta, A, b)` returns the
// objective at p (NaN where it is undefined; float or double, compared in that type) and, with grad, the normal matrix A (packed upper
// triangle of a 4 x 4; the isotropic model's slot 3 an identity row) and the right-hand side b
// of the step A delta = b. Every lane of the warp calls it with the same p and gets the same
// warp-reduced results, so the driver's branches are warp-uniform.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "fitspots.h"

namespace fs_warp {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ int tri4(int j, int k) {  // packed (j, k), j <= k, of a 4 x 4
  return j * 4 - j * (j - 1) / 2 + (k - j);
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) {
  v = (v < lo) ? lo : v;
  return (v > hi) ? hi : v;
}

// (A + lambda diag A) d = b, 4 unknowns, A packed; Jacobi-scaled Cholesky.
__device__ __forceinline__ bool solve4(const float (&A)[10], const float (&b)[4], float lam,
                                       float (&d)[4]) {
  float s[4], L[4][4], y[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float a = A[tri4(j, j)];
    if (!(a > 0.f)) return false;
    s[j] = rsqrtf(a);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
#pragma unroll
    for (int k = 0; k <= j; ++k) {
      float t = (j == k) ? 1.f + lam : A[tri4(k, j)] * s[j] * s[k];
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
  for (int j = 0; j < 4; ++j) {
    float t = b[j] * s[j];
#pragma unroll
    for (int k = 0; k < j; ++k) t -= L[j][k] * y[k];
    y[j] = t / L[j][j];
  }
#pragma unroll
  for (int j = 3; j >= 0; --j) {
    float t = y[j];
#pragma unroll
    for (int k = j + 1; k < 4; ++k) t -= L[k][j] * d[k];
    d[j] = t / L[j][j];
  }
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    d[j] *= s[j];
    ok = ok && isfinite(d[j]);
  }
  return ok;
}

struct LmResult {
  int iters, evals, state;
};

// The LM loop of the fit: lambda = 10^klam from 10^-2, lowered after an accepted first trial,
// raised (up to 10^4) while the trial does not decrease the objective and the step is not
// below min_step; stop on max_error, min_delta (relative decrease), min_step, no decrease or a
// failed evaluation / a solve that fails up to the damping cap. p is updated in place (the
// accepted point).
//
// Ties: where the change of the objective from the best point to the trial lies within
// tie_window * (objective) of 0 or of the min_delta threshold, the difference of two rounded
// objectives decides nothing, and `refine(best, alpha_b, beta_b, trial, alpha_t, beta_t)` is
// asked for the change itself, computed from the parameter difference with relative
// precision (NaN: keep the plain difference). The decisions then use that change.
template <typename Eval, typename Limit, typename Refine>
__device__ __forceinline__ LmResult lm_drive(float (&p)[4], bool iso, int P, int max_iter,
                                             float max_error, float min_delta, float min_step,
                                             Eval &&evaluate, Limit &&limit, Refine &&refine,
                                             float tie_window) {
  auto all_small = [&](const float (&d)[4], const float (&q)[4]) {
    bool sm = true;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < P) sm = sm && fabsf(d[j]) < min_step * fabsf(q[j]);
    return sm;
  };
  float A[10], b[4], best[4], dl[4], pt[4];
  float al = 0.f, be = 0.f, at = 0.f, bt = 0.f;
  int klam = -2;
  // Eq. 14 at lambda = 10^klam, raising klam tenfold (up to 10^4) while the damped system is
  // not positive definite: with a positive diagonal that only happens through the FP32
  // rounding of a nearly singular normal matrix, and more damping is the step the exact
  // system would allow, as for a rejected trial.
  auto solve_raising = [&]() {
    while (!solve4(A, b, exp10f((float)klam), dl)) {
      if (klam >= 4) return false;
      ++klam;
    }
    return true;
  };
  using Obj = decltype(evaluate(p, true, al, be, A, b));
  int it = 0, evals = 0, state = FS_STATE_MAX_ITER;
  while (it < max_iter) {
    ++it;
    ++evals;
    const Obj chi = evaluate(p, true, al, be, A, b);
    if (isnan(chi)) {
      state = FS_STATE_NOT_CONVERGED;
      break;
    }
    if (chi < max_error) {
      state = FS_STATE_MAX_ERROR;
      break;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) best[j] = p[j];
    auto trial = [&]() -> Obj {
#pragma unroll
      for (int j = 0; j < 4; ++j) pt[j] = best[j] + dl[j];
      limit(pt);
      float Ad[10], bd[4];
      return evaluate(pt, false, at, bt, Ad, bd);
    };
    // the change chi_t - chi of a trial, refined near the two decision thresholds
    bool refined = false;
    auto change = [&](Obj Chi) -> Obj {
      Obj d = Chi - chi;
      refined = false;
      const Obj win = Obj(tie_window) * chi;
      if (isfinite(d) && (fabs(d) <= win || fabs(d + Obj(min_delta) * chi) <= win)) {
        const Obj r = Obj(refine(best, al, be, pt, at, bt));
        if (isfinite(r)) {
          d = r;
          refined = true;
        }
      }
      return d;
    };
    if (!solve_raising()) {
      state = FS_STATE_NOT_CONVERGED;
      break;
    }
    if (iso) dl[3] = dl[2];
    ++evals;
    Obj Chi = trial();
    Obj dC = change(Chi);
    if (dC < Obj(0)) --klam;
    bool failed = false;
    while (!all_small(dl, best) && dC > Obj(0) && klam < 4) {
      ++klam;
      if (!solve_raising()) {
        failed = true;
        break;
      }
      if (iso) dl[3] = dl[2];
      ++evals;
      Chi = trial();
      dC = change(Chi);
    }
    if (failed) {
      state = FS_STATE_NOT_CONVERGED;
      break;
    }
    if (dC > Obj(0) || isnan(Chi)) {
      state = (all_small(dl, best) && !isnan(Chi)) ? FS_STATE_NO_DECREASE : FS_STATE_NOT_CONVERGED;
      break;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = pt[j];
    if (Chi < max_error) {
      state = FS_STATE_MAX_ERROR;
      break;
    }
    if (refined ? dC > -Obj(min_delta) * chi : chi * (Obj(1) - Obj(min_delta)) < Chi) {
      state = FS_STATE_MIN_DELTA;
      break;
    }
    if (all_small(dl, best)) {
      state = FS_STATE_MIN_STEP;
      break;
    }
  }
  return {it, evals, state};
}

// The driver without tie refinement (the plain difference of two objectives decides).
template <typename Eval, typename Limit>
__device__ __forceinline__ LmResult lm_drive(float (&p)[4], bool iso, int P, int max_iter,
                                             float max_error, float min_delta, float min_step,
                                             Eval &&evaluate, Limit &&limit) {
  auto none = [](const float (&)[4], float, float, const float (&)[4], float, float) {
    return (double)NAN;
  };
  return lm_drive(p, iso, P, max_iter, max_error, min_delta, min_step, evaluate, limit, none,
                  0.f);
}

}  // namespace fs_warp
