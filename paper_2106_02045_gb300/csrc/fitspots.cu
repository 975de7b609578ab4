// fitspots.cu -- sm_103a kernels and C ABI for batched implicit-amplitude LM fitting of
// 2-D Gaussian spots (Leutenegger & Weber, arXiv 2106.02045).
//
// Work mapping. A spot is held by a group of L threads (L = 4, 8, 16 or 32; 32/L groups
// per warp). Thread t of a group owns the ROI columns x = t, t+L, ... (C of them) over
// R rows, with the pixel values in registers for the whole fit. The Gaussian profile of
// both models separates, f(x, y) = e_x(x) e_y(y) (Eq. 10 and its elliptic extension),
// so a model evaluation needs W + H exponentials (SFU __expf) instead of W*H, and every
// per-spot sum of the method is either a product of 1-D moments
// (F, F(bold), sum d_j, sum f d_j, sum d_j d_k of Eq. 5, 7 and of J^T J) or a bilinear
// form e_x^T M e_y of a pixel matrix M (the cross-sums with the data). Per pixel and
// evaluated point that costs 7 FP32 operations:
//   pass 1 (for Eq. 6):      s(x)  += e_y g'                                    (1)
//   pass 2 (Eq. 2, 9, 13):   u = g' - (alpha e_x) e_y;  chi += u u;  w = e_y u;
//                            t0 += w;  t1 += y w;  t2 += y^2 w                  (6)
// where g' = g - s is the pixel value minus an integer per-spot shift s (kept close to
// beta^ so that chi^2 = sum (u - beta')^2 does not cancel). Per-thread partial sums are
// combined with a pairwise tree through shared memory (no atomics, fixed order, so a
// spot's result does not depend on its neighbours). The LM bookkeeping (Eq. 6 2x2
// solve, J^T J assembly, diagonally scaled Cholesky of Eq. 14, damping, stop tests) runs
// in FP32; the 2x2 amplitude solve is redone in FP64 where its determinant cancels by a
// factor above 1024, the damped solve where the FP32 factorisation fails (FP64 runs at about
// 1/74 of the FP32 rate on this GPU, so it is kept to those systems), and a damped system
// that rounding leaves not positive definite gets more damping instead of ending the fit.
//
// Gradient. With alpha^, beta^ at their optimum, sum_i r_i = sum_i r_i f_i = 0 (Eq. 4), so
// J^T r = alpha^ sum_i r_i df_i/dp_j (the other two terms of Eq. 9 vanish), and
//   J^T J = a R^T + alpha (Fd a^T + D1 b^T) + alpha^2 Ddd
// with a = d alpha^/dp, b = d beta^/dp (Eq. 8 solved through the 2x2 normal matrix),
// R_j = sum r df/dp_j, Fd_j = sum f df/dp_j, D1_j = sum df/dp_j, Ddd = sum df df^T.
//
// Decisions near a tie. An FP32 chi^2 of ~10^3 terms carries 1e-7..1e-6 relative
// rounding noise, the order of the stop threshold min_delta (1e-6). When the FP32 change
// chi_t^2 - chi_b^2 falls within that noise of 0 or of -min_delta * chi_b^2, the
// group recomputes the change directly as sum dh (dh - 2 r_b) with dh = h_t - h_b formed
// from the exact parameter difference (expm1 of the exponent difference), so the
// accept/reject and minimum-decrease tests of the Fit2DGaussian listing are taken on a
// difference that has relative, not absolute, FP32 error.
//
// Scheduling. A prepass sorts spot indices into 16 size classes (ceil(W/8), ceil(H/8)) and
// a seventeenth for ROIs with a side above 32 (at most 1024 pixels, the paper's bound on
// one fit). fit_spots then fits every class of W, H <= 32 in ONE persistent launch of a
// generic batched kernel (each ROI oriented with its longer side along the lanes, rows in
// compile-time blocks of 8/16/24/32), largest classes first, and the elongated class in a
// second launch (row blocks); warps pull spots from per-class atomic cursors and refill a
// slot as soon as its spot finishes. fit_spots_per_class keeps one launch per class with
// the configuration the autotuned table assigns. fit_spots_uniform skips the prepass for
// batches of equal-size, contiguous spots (the paper's own layout).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "fitspots.h"

namespace {

constexpr int kMaxPixels = 1024;  // pixels per spot (Sec. "Implementation")
constexpr int kMaxSide = 32;      // sides of the 16 size classes held in registers
constexpr int kElongClass = 16;   // ROIs with a side above 32 (and at most 1024 pixels)
constexpr int kNumClasses = 17;
constexpr int kElongBlocks = 11;  // 32-row blocks of the longest side, 1024 / 3 = 341 rows
constexpr int kWarpsPerBlock = 4;
constexpr int K1 = 17;    // first reduction: FG' + 16 one-dimensional moments
constexpr int K2 = 6;     // second reduction: chi_u, Tf, Tx, Txx, Ty1, Ty2
constexpr int kTot = 32;  // totals: first (20 slots), second (8), tie refinement (4)
constexpr float kTieWindow = 5e-7f;

struct FitArgs {
  const void *images;
  int dtype;
  int64_t image_elems;
  const int64_t *offsets;
  const int32_t *dims;
  const float *init;
  const uint8_t *model;
  int32_t n;
  int max_iter;
  float max_error;
  float min_delta;
  float min_step;
  float *out_params;
  float *out_alpha;
  float *out_beta;
  float *out_chi2;
  int32_t *out_state;
  int32_t *out_iters;
  int32_t *out_evals;
  // equal-size contiguous batch: spot s is at s*uw*uh, no offsets/dims/model arrays
  int uniform, uw, uh, umodel;
  // schedule (workspace)
  int32_t *counts;   // [16] spots per class
  int32_t *starts;   // [16] first slot of each class in perm
  int32_t *cursors;  // [16] next unclaimed item per class
  int32_t *fill;     // [16] scatter cursors
  int32_t *perm;     // [n]
};

// 10^k for the damping factor lambda = 10^k (k = -2 initially); k < -45 gives 0.
__constant__ float kPow10[50] = {
    1e-45f, 1e-44f, 1e-43f, 1e-42f, 1e-41f, 1e-40f, 1e-39f, 1e-38f, 1e-37f, 1e-36f,
    1e-35f, 1e-34f, 1e-33f, 1e-32f, 1e-31f, 1e-30f, 1e-29f, 1e-28f, 1e-27f, 1e-26f,
    1e-25f, 1e-24f, 1e-23f, 1e-22f, 1e-21f, 1e-20f, 1e-19f, 1e-18f, 1e-17f, 1e-16f,
    1e-15f, 1e-14f, 1e-13f, 1e-12f, 1e-11f, 1e-10f, 1e-9f,  1e-8f,  1e-7f,  1e-6f,
    1e-5f,  1e-4f,  1e-3f,  1e-2f,  1e-1f,  1e0f,   1e1f,   1e2f,   1e3f,   1e4f};

__device__ __forceinline__ float pow10i(int k) { return k < -45 ? 0.f : kPow10[min(k, 4) + 45]; }

// ------------------------------------------------------------------ small helpers
__host__ __device__ __forceinline__ int size_class(int W, int H) {
  if (W > kMaxSide || H > kMaxSide) return kElongClass;
  return ((W + 7) / 8 - 1) * 4 + ((H + 7) / 8 - 1);
}

// A fittable ROI: both sides at least 3, at most 1024 pixels and more pixels than unknowns.
__host__ __device__ __forceinline__ bool roi_ok(int W, int H, int P) {
  return W >= 3 && H >= 3 && W <= kMaxPixels / 3 && H <= kMaxPixels / 3 && W * H <= kMaxPixels &&
         W * H > P + 2;
}

__device__ __forceinline__ bool spot_valid(const FitArgs &a, int s, int &W, int &H, int &m) {
  W = a.dims[2 * s];
  H = a.dims[2 * s + 1];
  m = a.model[s];
  const int64_t off = a.offsets[s];
  const int P = (m == FS_MODEL_ISO) ? 3 : 4;
  return (m == FS_MODEL_ISO || m == FS_MODEL_ELLIPTIC) && roi_ok(W, H, P) && off >= 0 &&
         off + (int64_t)W * H <= a.image_elems;
}

__device__ void write_invalid(const FitArgs &a, int s) {
  for (int j = 0; j < 4; ++j) a.out_params[4 * s + j] = a.init[4 * s + j];
  a.out_alpha[s] = __int_as_float(0x7fc00000);
  a.out_beta[s] = __int_as_float(0x7fc00000);
  a.out_chi2[s] = __int_as_float(0x7fc00000);
  a.out_state[s] = FS_STATE_INVALID_ROI;
  a.out_iters[s] = 0;
  if (a.out_evals) a.out_evals[s] = 0;
}

// limit(): the box read into the unspecified clamp of the Fit2DGaussian listing,
// x0 in [-0.5, W-0.5], y0 in [-0.5, H-0.5], each sigma in [0.25, max(W, H)]. Plain
// comparisons, so a NaN stays NaN (and the spot then reports NOT_CONVERGED).
__device__ __forceinline__ float clampf(float v, float lo, float hi) {
  v = (v < lo) ? lo : v;
  return (v > hi) ? hi : v;
}
__device__ __forceinline__ void limit_params(float (&q)[4], int W, int H, bool iso) {
  const float smax = (float)max(W, H);
  q[0] = clampf(q[0], -0.5f, (float)W - 0.5f);
  q[1] = clampf(q[1], -0.5f, (float)H - 0.5f);
  q[2] = clampf(q[2], 0.25f, smax);
  q[3] = iso ? q[2] : clampf(q[3], 0.25f, smax);
}

// e^x - 1 without cancellation: Taylor series through x^5 for |x| < 1/16 (truncation below
// 3e-8 relative), e^x - 1 beyond (relative error below 4e-6 there).
__device__ __forceinline__ float expm1_small(float x) {
  float t = fmaf(x, 1.f / 120.f, 1.f / 24.f);
  t = fmaf(x, t, 1.f / 6.f);
  t = fmaf(x, t, 0.5f);
  t = fmaf(x, t, 1.f);
  return fabsf(x) < 0.0625f ? x * t : __expf(x) - 1.f;
}

// 1/s^2, computed the same way wherever a profile is (re)built
__device__ __forceinline__ float inv_sq(float s) { return __fdividef(1.f, s * s); }

// 1/x in FP64 for x in the FP32 normal range: the FP32 reciprocal as the start value and
// one Newton step, relative error below 1e-13 (the start is good to 2^-23, the step squares
// the error). Cheaper on the FP64 pipe than a full-precision division.
__device__ __forceinline__ double rcp64(double x) {
  const double r = (double)__frcp_rn((float)x);
  return fma(r, fma(-x, r, 1.0), r);
}

// Eq. 6 at an evaluated point, as the LM step uses it: the amplitude alpha^, beta^ - shift and
// the 2 x 2 normal matrix's entries F, F(bold) and 1 / (N F(bold) - F^2), plus the difference
// between alpha^ and the FP32 alpha the pixel passes used (their residuals are moved by it).
struct Amp {
  float F, FF, iD, al, bp, dal;
};

// The amplitude system of the pixel passes in FP32: its cancellation ratio N F(bold) / D (the
// digits that D = N F(bold) - F^2 loses; large when the profile is nearly flat).
__device__ __forceinline__ float amplitude_cancellation(float Nf, float X01, float X02, float Y01,
                                                        float Y02) {
  const float F = X01 * Y01, FF = X02 * Y02;
  return __fdividef(Nf * FF, fmaf(Nf, FF, -F * F));
}

// Eq. 6 in FP64: the 2 x 2 normal equations of the amplitudes, combined and solved in double
// precision from the evaluation's FP32 sums, for systems where N F(bold) - F^2 cancels. FG
// and Gs are the sums of the shifted pixels g' = g - shift, so bp is beta^ - shift. Returns
// false when the system has no unique solution.
__device__ __forceinline__ bool amplitudes64(float Nf, float X01, float X02, float Y01, float Y02,
                                             float FG, float Gs, double &al, double &bp,
                                             Amp &r) {
  const double F = (double)X01 * (double)Y01, FF = (double)X02 * (double)Y02;
  const double N = (double)Nf, D = fma(N, FF, -F * F);
  if (!(D > 1e-30) || !(D < 1e30)) return false;
  const double iD = rcp64(D);
  al = fma(N, (double)FG, -F * (double)Gs) * iD;
  bp = fma((double)Gs, FF, -F * (double)FG) * iD;
  r.F = (float)F;
  r.FF = (float)FF;
  r.iD = (float)iD;
  return true;
}

// Above this cancellation ratio the amplitudes are solved again in FP64 (10 bits of the FP32
// determinant lost). FP64 runs at about 1/64 of the FP32 rate on this GPU and the LM step runs
// one slot per lane, so a warp pays for the FP64 path whenever any of its 16 slots takes it;
// a lower ratio (64) cost 16 % of the 32 x 32 fit time with no measurable change in the fits.
constexpr float kAmpCancel64 = 1024.f;

// Eq. 14 in FP32: the same scaling, Cholesky with reciprocal-square-root pivots. piv receives
// the smallest pivot relative to 1 + lambda (the scaled matrix's unit diagonal): the fraction
// of the diagonal that survives the elimination, small when the system is nearly singular.
__device__ __forceinline__ bool solve_damped32(const float (&A)[10], const float (&b)[4], float lam,
                                               float (&d)[4], float &piv) {
  piv = 0.f;
  if (!(A[0] > 0.f) || !(A[4] > 0.f) || !(A[7] > 0.f) || !(A[9] > 0.f)) return false;
  const float s0 = rsqrtf(A[0]), s1 = rsqrtf(A[4]), s2 = rsqrtf(A[7]), s3 = rsqrtf(A[9]);
  const float dg = 1.f + lam;
  const float m01 = A[1] * s0 * s1, m02 = A[2] * s0 * s2, m03 = A[3] * s0 * s3;
  const float m12 = A[5] * s1 * s2, m13 = A[6] * s1 * s3, m23 = A[8] * s2 * s3;
  const float r00 = rsqrtf(dg);
  const float l10 = m01 * r00, l20 = m02 * r00, l30 = m03 * r00;
  const float p1 = dg - l10 * l10;
  if (!(p1 > 0.f)) return false;
  const float r11 = rsqrtf(p1);
  const float l21 = (m12 - l20 * l10) * r11, l31 = (m13 - l30 * l10) * r11;
  const float p2 = dg - l20 * l20 - l21 * l21;
  if (!(p2 > 0.f)) return false;
  const float r22 = rsqrtf(p2);
  const float l32 = (m23 - l30 * l20 - l31 * l21) * r22;
  const float p3 = dg - l30 * l30 - l31 * l31 - l32 * l32;
  if (!(p3 > 0.f)) return false;
  const float r33 = rsqrtf(p3);
  piv = __fdividef(fminf(p1, fminf(p2, p3)), dg);
  const float z0 = b[0] * s0 * r00;
  const float z1 = (b[1] * s1 - l10 * z0) * r11;
  const float z2 = (b[2] * s2 - l20 * z0 - l21 * z1) * r22;
  const float z3 = (b[3] * s3 - l30 * z0 - l31 * z1 - l32 * z2) * r33;
  const float y3 = z3 * r33;
  const float y2 = (z2 - l32 * y3) * r22;
  const float y1 = (z1 - l21 * y2 - l31 * y3) * r11;
  const float y0 = (z0 - l10 * y1 - l20 * y2 - l30 * y3) * r00;
  d[0] = y0 * s0;
  d[1] = y1 * s1;
  d[2] = y2 * s2;
  d[3] = y3 * s3;
  return isfinite(d[0]) && isfinite(d[1]) && isfinite(d[2]) && isfinite(d[3]);
}

// Eq. 14 with the diagonal scaling that makes the damping scale-invariant: M = S A S has a
// unit diagonal, (M + lambda I) y = S b, delta = S y. A is packed upper-triangular:
// A00 A01 A02 A03 A11 A12 A13 A22 A23 A33 (the isotropic model passes A33 = 1 and zeros in
// its row and column). The scaling S = diag(A)^-1/2 and the scaled entries are formed in
// FP32; the elimination (the pivots of L D L^T) and both substitutions run in FP64. Called
// only where the FP32 factorisation failed, so it is written for size, not speed: plain
// loops over a 4 x 4 array that lives in local memory (L1), keeping the hot loop's code
// small. Returns false when the damped matrix is not positive definite or the step is not
// finite.
__device__ __forceinline__ bool solve_damped64(const float (&A)[10], const float (&b)[4],
                                               float lam, float (&d)[4]) {
  if (!(A[0] > 0.f) || !(A[4] > 0.f) || !(A[7] > 0.f) || !(A[9] > 0.f)) return false;
  const float s0 = rsqrtf(A[0]), s1 = rsqrtf(A[4]), s2 = rsqrtf(A[7]), s3 = rsqrtf(A[9]);
  const double dg = 1.0 + (double)lam;
  double m[16], z[4];
  m[0] = m[5] = m[10] = m[15] = dg;
  m[1] = m[4] = A[1] * s0 * s1;
  m[2] = m[8] = A[2] * s0 * s2;
  m[3] = m[12] = A[3] * s0 * s3;
  m[6] = m[9] = A[5] * s1 * s2;
  m[7] = m[13] = A[6] * s1 * s3;
  m[11] = m[14] = A[8] * s2 * s3;
  z[0] = (double)(b[0] * s0);
  z[1] = (double)(b[1] * s1);
  z[2] = (double)(b[2] * s2);
  z[3] = (double)(b[3] * s3);
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {  // forward elimination; m[5k] is the k-th pivot
    const double piv = m[5 * k];
    if (!(piv > 1e-30)) return false;
    const double ip = rcp64(piv);
#pragma unroll 1
    for (int i = k + 1; i < 4; ++i) {
      const double f = m[4 * i + k] * ip;
#pragma unroll 1
      for (int j = k + 1; j < 4; ++j) m[4 * i + j] = fma(-f, m[4 * k + j], m[4 * i + j]);
      z[i] = fma(-f, z[k], z[i]);
    }
  }
#pragma unroll 1
  for (int k = 3; k >= 0; --k) {  // back substitution
    double t = z[k];
#pragma unroll 1
    for (int j = k + 1; j < 4; ++j) t = fma(-m[4 * k + j], z[j], t);
    z[k] = t * rcp64(m[5 * k]);
  }
  d[0] = (float)z[0] * s0;
  d[1] = (float)z[1] * s1;
  d[2] = (float)z[2] * s2;
  d[3] = (float)z[3] * s3;
  return isfinite(d[0]) && isfinite(d[1]) && isfinite(d[2]) && isfinite(d[3]);
}

// Eq. 14: FP32, redone in FP64 where the FP32 factorisation fails (the rounding of a nearly
// singular system). A low FP32 pivot alone does not call for FP64: the step is then
// imprecise in a direction along which chi^2 hardly changes, and the LM iteration corrects
// it; measured on GB300, taking FP64 there too (pivot below 1/1024 or 1/32) moved no parity
// figure and cost 1 % and 6 % of the 32 x 32 fit time.
__device__ __forceinline__ bool solve_damped(const float (&A)[10], const float (&b)[4], float lam,
                                             float (&d)[4]) {
  float piv;
  if (solve_damped32(A, b, lam, d, piv)) return true;
  return solve_damped64(A, b, lam, d);
}

// Eq. 14 at lambda = 10^klam, raising klam tenfold at a time (up to the 10^4 cap) while the
// damped system is not positive definite. With a positive diagonal, J^T J + lambda diag(J^T J)
// is positive definite for every lambda > 0, so a failed factorisation comes from the rounding
// of a nearly singular FP32 normal matrix; more damping is the step the exact system would
// allow, as for a rejected trial. False when no lambda up to the cap gives a step. The
// per-spot kernels use this loop; the batched ones raise lambda by one decade per round
// instead (kResolve), which keeps the loop out of their hot code.
__device__ __forceinline__ bool solve_damped_raising(const float (&A)[10], const float (&b)[4],
                                                     int &klam, float (&d)[4]) {
  for (;;) {  // one inlined copy of the solve
    if (solve_damped(A, b, pow10i(klam), d)) return true;
    if (klam >= 4) return false;
    ++klam;
  }
}

// Normal equations A = J^T J and b = J^T r at an evaluated point (Eq. 9, 12 and 13) from the
// evaluation's sums, in the reduced separable form:
//   J^T r = alpha^ R,   J^T J = a R^T + alpha^ (Fd a^T + D1 b^T) + alpha^2 Ddd
// with R_j = sum r df/dp_j, Fd_j = sum f df/dp_j, D1_j = sum df/dp_j, Ddd = sum df df^T and
// a = d alpha^/dp, b = d beta^/dp (Eq. 8 through the 2 x 2 normal matrix of Eq. 6).
//   xm  column moments X01 X02 X11 X21 X12 X22 X32 X42 (X_mn = sum_x dx^m e_x^n)
//   ym  row moments, the same for the rows
//   tr  residual sums Tf Tx Txx Ty1 Ty2 of pass 2, taken with the group's FP32 alpha32 and
//       row weights y - yc0 (eta = y0 - yc0)
//   am  the amplitude solve; R is moved from the pixel passes' FP32 alpha to alpha^ (a shift
//       of the residual by am.dal f) so that every term refers to one point
// The isotropic model folds the two width columns into one and pads with an identity row.
__device__ __forceinline__ void normal_equations(const float (&xm)[8], const float (&ym)[8],
                                                 const float (&tr)[5], float Nf, const Amp &am,
                                                 float sx, float sy, float eta, bool iso,
                                                 float (&A)[10], float (&bv)[4]) {
  const float X01 = xm[0], X02 = xm[1], X11 = xm[2], X21 = xm[3], X12 = xm[4], X22 = xm[5],
              X32 = xm[6], X42 = xm[7];
  const float Y01 = ym[0], Y02 = ym[1], Y11 = ym[2], Y21 = ym[3], Y12 = ym[4], Y22 = ym[5],
              Y32 = ym[6], Y42 = ym[7];
  const float Tf = tr[0], Tx = tr[1], Txx = tr[2], Ty1 = tr[3], Ty2 = tr[4];
  const float alpha = am.al, bp = am.bp, F = am.F, FF = am.FF, iD = am.iD, dal = am.dal;
  const float ivx = inv_sq(sx), ivy = inv_sq(sy);
  const float cx = __fdividef(ivx, sx), cy = __fdividef(ivy, sy);
  const float Sfdy = fmaf(-eta, Tf, Ty1);
  const float Sfdy2 = Ty2 - 2.f * eta * Ty1 + eta * eta * Tf;
  float Rd[4], D1[4], Fd[4], aa[4], bb[4];
  D1[0] = X11 * Y01 * ivx;
  D1[1] = X01 * Y11 * ivy;
  D1[2] = X21 * Y01 * cx;
  D1[3] = X01 * Y21 * cy;
  Fd[0] = X12 * Y02 * ivx;
  Fd[1] = X02 * Y12 * ivy;
  Fd[2] = X22 * Y02 * cx;
  Fd[3] = X02 * Y22 * cy;
  Rd[0] = fmaf(-dal, Fd[0], ivx * fmaf(-bp * X11, Y01, Tx));    // sum r df/dx0
  Rd[1] = fmaf(-dal, Fd[1], ivy * fmaf(-bp * X01, Y11, Sfdy));  // sum r df/dy0
  Rd[2] = fmaf(-dal, Fd[2], cx * fmaf(-bp * X21, Y01, Txx));    // sum r df/dsx
  Rd[3] = fmaf(-dal, Fd[3], cy * fmaf(-bp * X01, Y21, Sfdy2));  // sum r df/dsy
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    aa[j] = (Nf * Rd[j] - alpha * (Nf * Fd[j] - F * D1[j])) * iD;  // d alpha^/dp_j
    bb[j] = (alpha * (F * Fd[j] - FF * D1[j]) - F * Rd[j]) * iD;   // d beta^/dp_j
  }
  const float a2 = alpha * alpha;
  float Dd[10];
  Dd[0] = X22 * Y02 * ivx * ivx;
  Dd[1] = X12 * Y12 * ivx * ivy;
  Dd[2] = X32 * Y02 * ivx * cx;
  Dd[3] = X12 * Y22 * ivx * cy;
  Dd[4] = X02 * Y22 * ivy * ivy;
  Dd[5] = X22 * Y12 * ivy * cx;
  Dd[6] = X02 * Y32 * ivy * cy;
  Dd[7] = X42 * Y02 * cx * cx;
  Dd[8] = X22 * Y22 * cx * cy;
  Dd[9] = X02 * Y42 * cy * cy;
  float M[10];
  int idx = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = j; k < 4; ++k, ++idx)
      M[idx] = fmaf(aa[j], Rd[k], alpha * (Fd[j] * aa[k] + D1[j] * bb[k])) + a2 * Dd[idx];
  if (iso) {  // sigma_x = sigma_y = sigma: fold the two width columns into one
    A[0] = M[0];
    A[1] = M[1];
    A[2] = M[2] + M[3];
    A[3] = 0.f;
    A[4] = M[4];
    A[5] = M[5] + M[6];
    A[6] = 0.f;
    A[7] = M[7] + 2.f * M[8] + M[9];
    A[8] = 0.f;
    A[9] = 1.f;
    bv[0] = alpha * Rd[0];
    bv[1] = alpha * Rd[1];
    bv[2] = alpha * (Rd[2] + Rd[3]);
    bv[3] = 0.f;
  } else {
#pragma unroll
    for (int k = 0; k < 10; ++k) A[k] = M[k];
#pragma unroll
    for (int j = 0; j < 4; ++j) bv[j] = alpha * Rd[j];
  }
}

// ------------------------------------------------------------------ group reductions
// Shared memory of one group: partials red[k*RS + lane] (RS = L + 4 keeps the float4 row
// reads of a quarter-warp on distinct banks), then kTot totals. The group stride is
// congruent to L mod 32 so that the groups of a warp write to distinct banks.
__host__ __device__ constexpr int round_up(int v, int m) { return (v + m - 1) / m * m; }
__host__ __device__ constexpr int red_stride(int L) { return L + 4; }
__host__ __device__ constexpr int group_stride(int L) {
  return round_up(K1 * red_stride(L) + kTot, 32) + L;
}
// per warp: row tables (R + 1 per group), refinement tables (2R + 2 per group), reductions
__host__ __device__ constexpr int tab_floats(int L, int R) { return round_up((32 / L) * (R + 1), 4); }
__host__ __device__ constexpr int rtab_floats(int L, int R) { return round_up((32 / L) * (2 * R + 2), 4); }
__host__ __device__ constexpr int warp_smem_floats(int L, int R) {
  return round_up(tab_floats(L, R) + rtab_floats(L, R) + (32 / L) * group_stride(L), 32);
}

// Pairwise sum of L consecutive floats (16-byte aligned).
template <int L>
__device__ __forceinline__ float sum_row(const float *row) {
  constexpr int Q = L / 4;
  float s[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float4 v = reinterpret_cast<const float4 *>(row)[i];
    s[i] = (v.x + v.y) + (v.z + v.w);
  }
#pragma unroll
  for (int step = 1; step < Q; step *= 2)
#pragma unroll
    for (int i = 0; i + step < Q; i += 2 * step) s[i] += s[i + step];
  return s[0];
}

// Sum K per-thread partials (already stored at red[k*RS + lane]) over the L threads of
// a group into tot[0..K); on return every thread of the group can read the totals.
template <int L, int K>
__device__ __forceinline__ void group_reduce(const float *red, float *tot, int lg, unsigned gmask) {
  constexpr int RS = red_stride(L);
  __syncwarp(gmask);
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += L) {
    const int k = k0 + lg;
    if (k < K) tot[k] = sum_row<L>(red + k * RS);
  }
  __syncwarp(gmask);
}

template <int L>
__device__ __forceinline__ float group_sum_shfl(float v, unsigned gmask) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o);
  return v;
}

// ------------------------------------------------------------------ the fit loop
struct ClassList {
  int8_t cls[kNumClasses];
  int8_t count;
};

// Persistent kernel for one configuration: L threads per spot, C columns per thread,
// R rows per thread. It drains the size classes of `cl` in order (or the whole batch of
// a uniform call).
template <int L, int C, int R>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) fit_kernel(FitArgs a, ClassList cl) {
  constexpr int S = 32 / L;
  constexpr int NR = (R + L - 1) / L;
  constexpr int TS = R + 1;
  constexpr int TS2 = 2 * R + 2;
  constexpr int RS = red_stride(L);
  constexpr float yc0 = 0.5f * (float)R;  // origin of the row weights y~ = y - R/2
  constexpr int kChunk = L < 8 ? L : 8;   // items a group claims per atomic
  static_assert(S * L == 32, "lane groups must tile a warp");
  extern __shared__ float4 smem4[];
  float *sw = reinterpret_cast<float *>(smem4) + (threadIdx.x >> 5) * warp_smem_floats(L, R);
  const int lane = threadIdx.x & 31;
  const int gi = lane / L, lg = lane % L;
  const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (gi * L));
  float *tab = sw + gi * TS;
  float2 *rtab = reinterpret_cast<float2 *>(sw + tab_floats(L, R) + gi * TS2);
  float *red = sw + tab_floats(L, R) + rtab_floats(L, R) + gi * group_stride(L);
  float *tot1 = red + K1 * RS;  // totals of the first reduction (17 used)
  float *tot2 = tot1 + 20;      // totals of the second reduction (6 used)
  float *tot3 = tot2 + 8;       // total of the tie refinement

  for (int ci = 0; ci < cl.count; ++ci) {
    const int cls = cl.cls[ci];
    const int cnt = a.uniform ? a.n : a.counts[cls];
    const int beg = a.uniform ? 0 : a.starts[cls];

    float g[C][R];
    bool active = false, idle = cnt == 0;
    int cbase = 0, cnext = 0, cend = 0;  // the group's claimed chunk of items
    int cspot = 0, cwh = 0, cmod = 0;    // schedule entry held by thread j of the chunk
    int64_t coff = 0;
    int spot = 0, W = 0, H = 0, P = 4;
    bool iso = false;
    float Nf = 0.f, Gs = 0.f, shift = 0.f;
    float p[4] = {0.f, 0.f, 1.f, 1.f}, pe[4] = {0.f, 0.f, 1.f, 1.f}, dl[4] = {0.f, 0.f, 0.f, 0.f};
    float A[10], bv[4];
    float chib = 0.f, alb = 0.f, bpb = 0.f, noiseb = 0.f;
    float ral = 0.f, rbl = 0.f;  // FP64-solved amplitude and background at p, as reported
    int klam = -2, it = 0, evals = 0;
    bool first_eval = false, first_trial = false;
#pragma unroll
    for (int k = 0; k < 10; ++k) A[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) bv[k] = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int y = 0; y < R; ++y) g[c][y] = 0.f;

    while (true) {
      // -------------------------------------------------------------- refill the slot
      if (!active && !idle) {
        if (cnext >= cend) {
          // claim the next kChunk items of this class; thread j of the group keeps the
          // schedule entry of item j (spot, offset, size, model)
          int base = 0;
          if (lg == 0) base = atomicAdd(a.cursors + cls, kChunk);
          base = __shfl_sync(gmask, base, gi * L);
          cbase = base;
          cnext = base;
          cend = min(base + kChunk, cnt);
          if (lg < kChunk && base + lg < cnt) {
            const int it_ = base + lg;
            if (a.uniform) {
              cspot = it_;
              coff = (int64_t)it_ * (a.uw * a.uh);
              cwh = (a.uw << 8) | a.uh;
              cmod = a.umodel;
            } else {
              cspot = a.perm[beg + it_];
              coff = a.offsets[cspot];
              cwh = (a.dims[2 * cspot] << 8) | a.dims[2 * cspot + 1];
              cmod = a.model[cspot];
            }
          }
        }
        if (cnext >= cnt) {
          idle = true;
        } else {
          const int src = gi * L + (cnext - cbase);
          spot = __shfl_sync(gmask, cspot, src);
          const int64_t off = __shfl_sync(gmask, coff, src);
          const int wh = __shfl_sync(gmask, cwh, src);
          W = wh >> 8;
          H = wh & 255;
          iso = __shfl_sync(gmask, cmod, src) == FS_MODEL_ISO;
          ++cnext;
          if (cnext < cend) {
            // warm L2 with the next spot of the chunk (pixels and start values)
            const int nsrc = gi * L + (cnext - cbase);
            const int nspot = __shfl_sync(gmask, cspot, nsrc);
            const int64_t noff = __shfl_sync(gmask, coff, nsrc);
            const int nwh = __shfl_sync(gmask, cwh, nsrc);
            const int esz = a.dtype == FS_U16 ? 2 : 4;
            const char *nb = static_cast<const char *>(a.images) + noff * esz;
            const int nbytes = (nwh >> 8) * (nwh & 255) * esz;
            for (int line = lg; line * 128 < nbytes; line += L)  // addresses inside the spot
              asm volatile("prefetch.global.L2 [%0];" ::"l"(nb + line * 128));
            if (lg == 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.init + 4 * nspot));
          }
          P = iso ? 3 : 4;
          if (a.dtype == FS_U16) {
            const unsigned short *img = static_cast<const unsigned short *>(a.images) + off;
#pragma unroll
            for (int c = 0; c < C; ++c) {
              const int x = lg + L * c;
#pragma unroll
              for (int y = 0; y < R; ++y)
                g[c][y] = (x < W && y < H) ? (float)__ldg(img + y * W + x) : 0.f;
            }
          } else {
            const float *img = static_cast<const float *>(a.images) + off;
#pragma unroll
            for (int c = 0; c < C; ++c) {
              const int x = lg + L * c;
#pragma unroll
              for (int y = 0; y < R; ++y) g[c][y] = (x < W && y < H) ? __ldg(img + y * W + x) : 0.f;
            }
          }
          // integer shift = corner pixel (a background estimate); refined after pass 1
          shift = rintf(__shfl_sync(gmask, g[0][0], gi * L));
          float part = 0.f;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const int x = lg + L * c;
#pragma unroll
            for (int y = 0; y < R; ++y) {
              g[c][y] = (x < W && y < H) ? g[c][y] - shift : 0.f;
              part += g[c][y];
            }
          }
          Gs = group_sum_shfl<L>(part, gmask);
          Nf = (float)(W * H);
#pragma unroll
          for (int j = 0; j < 4; ++j) pe[j] = a.init[4 * spot + j];
          limit_params(pe, W, H, iso);
          klam = -2;
          it = 0;
          evals = 0;
          first_eval = true;
          active = true;
        }
      }
      if (!__any_sync(0xffffffffu, active)) break;
      if (!active) continue;

      // -------------------------------------------------------------- evaluate at pe
      const float sx = pe[2], sy = iso ? pe[2] : pe[3];
      const float ivx = inv_sq(sx), ivy = inv_sq(sy);
      const float nhx = -0.5f * ivx, nhy = -0.5f * ivy;
      float ex[C], dxv[C];
      {
        // column profile e_x and the column moments sum dx^m e_x^n
        float m[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int x = lg + L * c;
          const float d = (float)x - pe[0];
          const float e = (x < W) ? __expf(d * d * nhx) : 0.f;
          ex[c] = e;
          dxv[c] = d;
          const float e2 = e * e, de = d * e, de2 = d * e2;
          m[0] += e;
          m[1] += e2;
          m[2] += de;
          m[3] = fmaf(d, de, m[3]);
          m[4] += de2;
          m[5] = fmaf(d, de2, m[5]);
          m[6] = fmaf(d * d, de2, m[6]);
          m[7] = fmaf(d * d * d, de2, m[7]);
        }
        // slots: 1 X01, 2 X02, 5 X11, 6 X21, 7 X12, 8 X22, 9 X32, 10 X42
        red[1 * RS + lg] = m[0];
        red[2 * RS + lg] = m[1];
#pragma unroll
        for (int k = 0; k < 6; ++k) red[(5 + k) * RS + lg] = m[2 + k];
      }
      {
        // row profile e_y into the group's table, and the row moments
        float m[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          const int y = lg + L * k;
          if (y < R) {
            const float d = (float)y - pe[1];
            const float e = (y < H) ? __expf(d * d * nhy) : 0.f;
            tab[y] = e;
            const float e2 = e * e, de = d * e, de2 = d * e2;
            m[0] += e;
            m[1] += e2;
            m[2] += de;
            m[3] = fmaf(d, de, m[3]);
            m[4] += de2;
            m[5] = fmaf(d, de2, m[5]);
            m[6] = fmaf(d * d, de2, m[6]);
            m[7] = fmaf(d * d * d, de2, m[7]);
          }
        }
        // slots: 3 Y01, 4 Y02, 11 Y11, 12 Y21, 13 Y12, 14 Y22, 15 Y32, 16 Y42
        red[3 * RS + lg] = m[0];
        red[4 * RS + lg] = m[1];
#pragma unroll
        for (int k = 0; k < 6; ++k) red[(11 + k) * RS + lg] = m[2 + k];
      }
      __syncwarp(gmask);
      // pass 1: s(x) = sum_y e_y g'(x, y);  FG' partial = sum_x e_x s(x)
      {
        float s0[C];
#pragma unroll
        for (int c = 0; c < C; ++c) s0[c] = 0.f;
#pragma unroll
        for (int y = 0; y < R; ++y) {
          const float e = tab[y];
#pragma unroll
          for (int c = 0; c < C; ++c) s0[c] = fmaf(e, g[c][y], s0[c]);
        }
        float fg = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) fg = fmaf(ex[c], s0[c], fg);
        red[lg] = fg;
      }
      group_reduce<L, K1>(red, tot1, lg, gmask);
      const float4 t1a = reinterpret_cast<const float4 *>(tot1)[0];
      const float FG = t1a.x, X01 = t1a.y, X02 = t1a.z, Y01 = t1a.w, Y02 = tot1[4];
      const float F = X01 * Y01, FF = X02 * Y02;
      const float D = fmaf(Nf, FF, -F * F);
      const bool okD = D > 0.f && isfinite(D);
      const float iD = __fdividef(1.f, D);
      const float alpha = (Nf * FG - F * Gs) * iD;  // Eq. 6, for the pixel passes
      float bp = (Gs * FF - F * FG) * iD;           // beta^ - shift
      // Eq. 6 as reported and assembled: FP32, or FP64 where N F(bold) - F^2 cancels
      Amp am{F, FF, iD, alpha, bp, 0.f};
      bool ok64 = true, amp64 = false;
      double al64 = 0.0, bp64 = 0.0;
      if (okD && __fdividef(Nf * FF, D) > kAmpCancel64) {
        amp64 = true;
        ok64 = amplitudes64(Nf, X01, X02, Y01, Y02, FG, Gs, al64, bp64, am);
        am.al = (float)al64;
        am.dal = (float)(al64 - (double)alpha);
      }
      if (first_eval && okD) {
        // move the shift to the integer nearest beta^ (exact for integer pixel values)
        const float dl0 = rintf(bp);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int x = lg + L * c;
#pragma unroll
          for (int y = 0; y < R; ++y) g[c][y] = (x < W && y < H) ? g[c][y] - dl0 : 0.f;
        }
        Gs = fmaf(-Nf, dl0, Gs);
        shift += dl0;
        bp -= dl0;
        bp64 -= (double)dl0;
      }
      am.bp = amp64 ? (float)bp64 : bp;
      // pass 2: u = g' - alpha e_x e_y; chi_u = sum u^2; row-weighted sums of e_y u
      {
        float ca[C], ch0[C], ch1[C], t0[C], t1[C], t2[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          ca[c] = -alpha * ex[c];
          ch0[c] = ch1[c] = t0[c] = t1[c] = t2[c] = 0.f;
        }
#pragma unroll
        for (int y = 0; y < R; ++y) {
          const float e = tab[y];
          const float yy = (float)y - yc0;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const float u = fmaf(ca[c], e, g[c][y]);
            if (y & 1) ch1[c] = fmaf(u, u, ch1[c]);
            else ch0[c] = fmaf(u, u, ch0[c]);
            const float w = e * u;
            t0[c] += w;
            t1[c] = fmaf(yy, w, t1[c]);
            t2[c] = fmaf(yy * yy, w, t2[c]);
          }
        }
        float v2[K2] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float e = ex[c], d = dxv[c];
          const float et0 = e * t0[c];
          v2[0] += ch0[c] + ch1[c];
          v2[1] += et0;
          v2[2] = fmaf(d, et0, v2[2]);
          v2[3] = fmaf(d * d, et0, v2[3]);
          v2[4] = fmaf(e, t1[c], v2[4]);
          v2[5] = fmaf(e, t2[c], v2[5]);
        }
#pragma unroll
        for (int k = 0; k < K2; ++k) red[k * RS + lg] = v2[k];
      }
      group_reduce<L, K2>(red, tot2, lg, gmask);
      const float chiu = tot2[0];
      const float Su = fmaf(-alpha, F, Gs);             // sum u = G' - alpha F
      float chi = chiu - 2.f * bp * Su + Nf * bp * bp;  // Eq. 2: sum (u - beta')^2
      if (!okD || !ok64 || !isfinite(alpha)) chi = __int_as_float(0x7fc00000);
      ++evals;

      // -------------------------------------------------------------- chi^2 change
      // delta = chi_t^2 - chi_b^2, refined near the two decision thresholds. The window
      // covers the FP32 error of each chi^2: rounding alpha f and the profile in every
      // residual u gives errors of ~eps |alpha| f per pixel, i.e. a chi^2 error of about
      // 6 eps |alpha| sqrt(chi^2 F(bold) / N); the window takes four times that per point.
      const float noise =
          24.f * 5.9604645e-8f * fabsf(alpha) * sqrtf(fmaxf(chi, 0.f) * FF * __fdividef(1.f, Nf));
      float delta = chi - chib;
      const float win = kTieWindow * chib + noise + noiseb;
      if (!first_eval && isfinite(chi) && isfinite(chib) && delta >= -a.min_delta * chib - win &&
          delta <= win) {
        const float sbx = p[2], sby = iso ? p[2] : p[3];
        const float ivbx = inv_sq(sbx), ivby = inv_sq(sby);
        const float nhbx = -0.5f * ivbx, nhby = -0.5f * ivby;
        const float dsx = sx - sbx, dsy = sy - sby;
        const float d0 = pe[0] - p[0], d1 = pe[1] - p[1];
        const float kx = dsx * (sx + sbx) * ivx * ivbx, ky = dsy * (sy + sby) * ivy * ivby;
        float mx[C], omx[C], exb[C], cab[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int x = lg + L * c;
          const float db = (float)x - p[0], dt = dxv[c];
          // exponent difference x_t - x_b, from the parameter differences
          const float dxe = 0.5f * fmaf(d0 * (dt + db), ivx, db * db * kx);
          mx[c] = (x < W) ? expm1_small(dxe) : 0.f;
          omx[c] = 1.f + mx[c];
          exb[c] = (x < W) ? __expf(db * db * nhbx) : 0.f;
          cab[c] = -alb * exb[c];
        }
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          const int y = lg + L * k;
          if (y < R) {
            const float db = (float)y - p[1], dt = (float)y - pe[1];
            const float dye = 0.5f * fmaf(d1 * (dt + db), ivy, db * db * ky);
            rtab[y] = (y < H) ? make_float2(expm1_small(dye), __expf(db * db * nhby))
                              : make_float2(0.f, 0.f);
          }
        }
        __syncwarp(gmask);
        const float dal = alpha - alb, dbp = bp - bpb;
        float acc = 0.f;
#pragma unroll
        for (int y = 0; y < R; ++y) {
          if (y < H) {  // padding rows and columns are not part of the spot
            const float2 q = rtab[y];  // (e_y,t / e_y,b - 1, e_y,b)
#pragma unroll
            for (int c = 0; c < C; ++c) {
              if (lg + L * c < W) {
                const float fb = exb[c] * q.y;
                const float tt = fmaf(q.x, omx[c], mx[c]);             // f_t / f_b - 1
                const float dh = fmaf(fb, fmaf(alpha, tt, dal), dbp);  // h_t - h_b
                const float rb = fmaf(cab[c], q.y, g[c][y]) - bpb;     // g - h_b
                acc = fmaf(dh, fmaf(-2.f, rb, dh), acc);
              }
            }
          }
        }
        red[lg] = acc;
        group_reduce<L, 1>(red, tot3, lg, gmask);
        delta = tot3[0];
      }

      // -------------------------------------------------------------- LM step
      const float ra_t = am.al, rb_t = amp64 ? (float)(bp64 + (double)shift) : bp + shift;
      bool finish = false, need_grad = false, need_solve = false;
      int state = FS_STATE_MAX_ITER;
      float ra = ra_t, rb = rb_t, rc = chi;  // values reported on finish
      if (first_eval) {
        first_eval = false;
        it = 1;
#pragma unroll
        for (int j = 0; j < 4; ++j) p[j] = pe[j];
        if (isnan(chi)) {
          finish = true;
          state = FS_STATE_NOT_CONVERGED;
        } else if (chi < a.max_error) {
          finish = true;
          state = FS_STATE_MAX_ERROR;
        } else {
          chib = chi;
          alb = alpha;
          bpb = bp;
          noiseb = noise;
          ral = ra_t;
          rbl = rb_t;
          need_grad = true;
        }
      } else {
        const float Chi = chi;
        const bool nan_t = isnan(Chi);
        if (first_trial && !nan_t && delta < 0.f) --klam;  // error decreased: lambda / 10
        first_trial = false;
        const float ms = a.min_step;
        const bool small = fabsf(dl[0]) < ms * fabsf(p[0]) && fabsf(dl[1]) < ms * fabsf(p[1]) &&
                           fabsf(dl[2]) < ms * fabsf(p[2]) &&
                           (iso || fabsf(dl[3]) < ms * fabsf(p[3]));
        if (!small && !nan_t && delta > 0.f && klam < 4) {
          ++klam;  // reject: lambda * 10, same normal equations
          need_solve = true;
        } else if (nan_t || delta > 0.f) {
          finish = true;  // keep the best point
          state = (small && !nan_t) ? FS_STATE_NO_DECREASE : FS_STATE_NOT_CONVERGED;
          ra = ral;
          rb = rbl;
          rc = chib;
        } else {
          const float chi_prev = chib;
#pragma unroll
          for (int j = 0; j < 4; ++j) p[j] = pe[j];
          chib = Chi;
          alb = alpha;
          bpb = bp;
          noiseb = noise;
          ral = ra_t;
          rbl = rb_t;
          if (Chi < a.max_error) {
            finish = true;
            state = FS_STATE_MAX_ERROR;
          } else if (delta > -a.min_delta * chi_prev) {
            finish = true;
            state = FS_STATE_MIN_DELTA;
          } else if (small) {
            finish = true;
            state = FS_STATE_MIN_STEP;
          } else if (it >= a.max_iter) {
            finish = true;
            state = FS_STATE_MAX_ITER;
          } else {
            ++it;
            need_grad = true;
          }
        }
      }

      if (need_grad) {
        // normal equations at p (= pe) from this evaluation's sums
        const float xm[8] = {X01, X02, tot1[5], tot1[6], tot1[7], tot1[8], tot1[9], tot1[10]};
        const float ym[8] = {Y01, Y02, tot1[11], tot1[12], tot1[13], tot1[14], tot1[15], tot1[16]};
        const float tr[5] = {tot2[1], tot2[2], tot2[3], tot2[4], tot2[5]};
        normal_equations(xm, ym, tr, Nf, am, sx, sy, pe[1] - yc0, iso, A, bv);
        first_trial = true;
        need_solve = true;
      }
      if (need_solve) {
        float d[4];
        if (solve_damped_raising(A, bv, klam, d)) {
          if (iso) d[3] = d[2];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            dl[j] = d[j];
            pe[j] = p[j] + d[j];
          }
          limit_params(pe, W, H, iso);
        } else {
          finish = true;
          state = FS_STATE_NOT_CONVERGED;
          ra = ral;
          rb = rbl;
          rc = chib;
        }
      }

      if (finish) {
        if (lg == 0) {
          a.out_params[4 * spot + 0] = p[0];
          a.out_params[4 * spot + 1] = p[1];
          a.out_params[4 * spot + 2] = p[2];
          a.out_params[4 * spot + 3] = iso ? p[2] : p[3];
          a.out_alpha[spot] = ra;
          a.out_beta[spot] = rb;
          a.out_chi2[spot] = rc / (Nf - (float)(P + 2));
          a.out_state[spot] = state;
          a.out_iters[spot] = it;
          if (a.out_evals) a.out_evals[spot] = evals;
        }
        active = false;
      }
    }
  }
}

// ------------------------------------------------------------------ batched fit loop
// Batched configurations (L, C, R, NB): one lane per spot for the LM step, lane groups for the
// pixel passes. A warp keeps kSlots spots in flight. Each round its 32 / L lane groups
// evaluate the active spots at their trial points, 32 / L at a time (each group as one spot of
// the per-spot kernel with the same geometry), then lane j runs the LM step of slot j from
// that evaluation's sums and refills the slot when its spot finishes. The scalar LM work thus
// runs once per spot instead of once per lane of a group. Pixels are re-read from global
// memory (mostly L2) at each evaluation; slot state and evaluation results live in shared
// memory. NB > 1 is the generic geometry that serves every size class, the elongated one (a
// side above 32, at most 1024 pixels) included: each ROI is oriented with its longer side
// along the 32 lanes when that side is at most 32, else with its shorter side there; a lane
// holds R rows of its column at a time and the passes walk the spot's blocks of R rows. An
// oriented ROI is the transpose of the caller's (the separable sums and the limit() box are
// symmetric in x and y); its parameters are swapped on the way in and out.
constexpr int kSlots = 16;
// slot state (floats; integer fields stored as bits)
enum : int {
  SP = 0,        // best point p[4]
  SPE = 4,       // trial point pe[4]
  SDL = 8,       // last step dl[4]
  SA = 12,       // normal matrix A[10]
  SBV = 22,      // gradient b[4]
  SCHIB = 26,    // chi^2 at p
  SALB = 27,     // alpha at p (the pixel passes' FP32 value, for the tie refinement)
  SBPB = 28,     // beta - shift at p (likewise)
  SNOISEB = 29,  // chi^2 error estimate at p
  SSH0 = 30,     // integer pixel shift (corner pixel, then moved to the nearest of beta)
  SGS = 31,      // sum of shifted pixels
  SKLAM = 32, SIT = 33, SEVALS = 34, SSPOT = 35, SOFFLO = 36, SOFFHI = 37,
  SFLAGS = 38,   // W | H << 9 | iso, transposed, first_eval, first_trial, active bits
  SRA = 39,      // alpha^ at p from the FP64 solve of Eq. 6 (reported)
  SRB = 40,      // beta^ at p, likewise
  kSlotFields = 41
};
// evaluation results handed from the warp to the slot's lane: amplitudes and chi^2 of the
// pixel passes, the tie-refined change, the pixel sum and shift the amplitude sums were taken
// with, the 17 moments and FG' of the first reduction and the 6 residual sums of the second
enum : int {
  RALPHA = 0, RBP, RCHI, RNOISE, RDELTA, RGS1, RSH1, RT1, RT2 = RT1 + K1,
  kResFields = RT2 + K2
};
constexpr int kIsoBit = 1 << 18, kTransBit = 1 << 19, kFirstEval = 1 << 20,
              kFirstTrial = 1 << 21, kActive = 1 << 22,
              kResolve = 1 << 23;  // the damped solve failed: raised lambda, solve next round
__device__ __forceinline__ int flag_w(int f) { return f & 511; }
__device__ __forceinline__ int flag_h(int f) { return (f >> 9) & 511; }

// Shared memory of one warp: slot state and results, then the pass area (row tables of the
// 32 / L groups, RT = NB R rows each, then the groups' reduction areas). The tie refinement's
// table lives in rows 1.. of the group's reduction area, which hold nothing at that point.
__host__ __device__ constexpr int batched_warp_floats(int L, int RT) {
  return round_up((kSlotFields + kResFields) * kSlots, 32) +
         round_up(tab_floats(L, RT) + (32 / L) * group_stride(L), 32);
}

// Rows row0 .. row0 + R - 1 of one spot minus a shift, columns lg + L c of this lane; element
// (x, y) sits at off + x cs + y rs. Exact for uint16 pixels (the value is built as 2^23 + g in
// the float's mantissa, then 2^23 + shift is subtracted; both are integers below 2^24);
// padding rows and columns are 0. `full` (W = L C, H = R, row0 = 0, cs = 1, rs = W) skips the
// padding tests.
template <int L, int C, int R>
__device__ __forceinline__ void load_rows(const FitArgs &a, int64_t off, int cs, int rs, int W,
                                          int H, int lg, int row0, bool full, float shift,
                                          float (&g)[C][R]) {
  if (a.dtype == FS_U16) {
    const unsigned short *img = static_cast<const unsigned short *>(a.images) + off;
    const float k = 8388608.f + shift;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int x = lg + L * c;
      if (full) {
#pragma unroll
        for (int y = 0; y < R; ++y)
          g[c][y] = __int_as_float(0x4b000000 | (int)__ldg(img + y * (L * C) + x)) - k;
      } else {
#pragma unroll
        for (int y = 0; y < R; ++y) {
          const int yy = row0 + y;
          g[c][y] = (x < W && yy < H)
                        ? __int_as_float(0x4b000000 | (int)__ldg(img + x * cs + yy * rs)) - k
                        : 0.f;
        }
      }
    }
  } else {
    const float *img = static_cast<const float *>(a.images) + off;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int x = lg + L * c;
      if (full) {
#pragma unroll
        for (int y = 0; y < R; ++y) g[c][y] = __ldg(img + y * (L * C) + x) - shift;
      } else {
#pragma unroll
        for (int y = 0; y < R; ++y) {
          const int yy = row0 + y;
          g[c][y] = (x < W && yy < H) ? __ldg(img + x * cs + yy * rs) - shift : 0.f;
        }
      }
    }
  }
}

// Resident blocks per SM the batched kernels are compiled for: the kernel waits on L2 for
// the pixels of every evaluation, so occupancy pays until the register file runs out; C R
// registers hold a lane's pixels.
__host__ __device__ constexpr int batched_min_blocks(int C, int R) {
  return C * R <= 32 ? 6 : C * R <= 64 ? 4 : 3;
}

// Column moments sum dx^m e^n of this lane's columns (or rows), in the slot order of the
// first reduction: e, e^2, d e, d^2 e, d e^2, d^2 e^2, d^3 e^2, d^4 e^2.
__device__ __forceinline__ void moment_terms(float d, float e, float (&m)[8]) {
  const float e2 = e * e, de = d * e, de2 = d * e2;
  m[0] += e;
  m[1] += e2;
  m[2] += de;
  m[3] = fmaf(d, de, m[3]);
  m[4] += de2;
  m[5] = fmaf(d, de2, m[5]);
  m[6] = fmaf(d * d, de2, m[6]);
  m[7] = fmaf(d * d * d, de2, m[7]);
}

#define ST(f, j) st[(f) * kSlots + (j)]
#define STI(f, j) (*reinterpret_cast<int *>(&st[(f) * kSlots + (j)]))
#define RES(f, j) res[(f) * kSlots + (j)]

// the block's dynamic shared memory (every fit kernel's per-warp areas)
extern __shared__ float4 g_smem4[];

// The LM step of slot j (Eq. 6 in FP64, accept / reject and the damping schedule, the stop
// tests, the normal equations of Eq. 12-13 and the damped solve of Eq. 14 in FP64) on the
// slot's own lane, from the evaluation results the warp left in shared memory.
// wf is the warp's stride in the block's shared memory, yc0 the row-weight origin of the
// geometry; origin selects the row-weight origin of the slot's evaluation (0: yc0, 1: half
// its rows rounded up to 8, 2: half its rows).
// Returns whether the slot is still active.
__device__ __forceinline__ bool lm_step(const FitArgs &a, const int wf, const int j, const float yc0,
                                     const int origin) {
  float *const st = reinterpret_cast<float *>(g_smem4) + (threadIdx.x >> 5) * wf;
  const float *const res = st + kSlotFields * kSlots;
  bool active = true;
    int flags = STI(SFLAGS, j);
    const int W = flag_w(flags), H = flag_h(flags);
    const bool iso = flags & kIsoBit, trans = flags & kTransBit;
    bool first_eval = flags & kFirstEval, first_trial = flags & kFirstTrial;
    // a round without an evaluation: only the damped solve, at the lambda the last round raised
    bool resolve = flags & kResolve;
    const int P = iso ? 3 : 4;
    const float Nf = (float)(W * H);
    // origin of the row weights, as the slot's evaluation took it: the geometry's fixed R / 2,
    // half the rows rounded up to 8 (generic geometry) or half the rows (row blocks)
    const float yc = origin == 0 ? yc0 : origin == 1 ? (float)(((H + 7) >> 3) << 2) : 0.5f * (float)H;
    const int spot = STI(SSPOT, j);
    float p[4], pe[4], dl[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      p[k] = ST(SP + k, j);
      pe[k] = ST(SPE + k, j);
      dl[k] = ST(SDL + k, j);
    }
    int klam = STI(SKLAM, j), it = STI(SIT, j), evals = STI(SEVALS, j) + (resolve ? 0 : 1);
    float chib = ST(SCHIB, j), alb = ST(SALB, j), bpb = ST(SBPB, j), noiseb = ST(SNOISEB, j);
    float rab = ST(SRA, j), rbb = ST(SRB, j);
    const float shift = ST(SSH0, j);
    const float alpha = RES(RALPHA, j), bp = RES(RBP, j);
    float chi = RES(RCHI, j);
    const float noise = RES(RNOISE, j), delta = RES(RDELTA, j);
    // Eq. 6 as reported and assembled: the pixel passes' FP32 solution, or the FP64 one (from
    // this evaluation's sums, moved to the slot's current shift) where N F(bold) - F^2 cancels
    const float X01 = RES(RT1 + 1, j), X02 = RES(RT1 + 2, j), Y01 = RES(RT1 + 3, j),
                Y02 = RES(RT1 + 4, j);
    Amp am;
    am.F = X01 * Y01;
    am.FF = X02 * Y02;
    am.iD = __fdividef(1.f, fmaf(Nf, am.FF, -am.F * am.F));
    am.al = alpha;
    am.bp = bp;
    am.dal = 0.f;
    float rb_t = bp + shift;
    if (amplitude_cancellation(Nf, X01, X02, Y01, Y02) > kAmpCancel64 && isfinite(chi)) {
      double al64, bp64;
      if (amplitudes64(Nf, X01, X02, Y01, Y02, RES(RT1 + 0, j), RES(RGS1, j), al64, bp64, am)) {
        bp64 += (double)RES(RSH1, j) - (double)shift;
        am.al = (float)al64;
        am.bp = (float)bp64;
        am.dal = (float)(al64 - (double)alpha);
        rb_t = (float)(bp64 + (double)shift);
      } else {
        chi = __int_as_float(0x7fc00000);
      }
    }
    const float ra_t = am.al;

    bool finish = false, need_grad = false, need_solve = false;
    int state = FS_STATE_MAX_ITER;
    float ra = ra_t, rb = rb_t, rc = chi;  // values reported on finish
    if (resolve) {
      need_solve = true;
    } else if (first_eval) {
      first_eval = false;
      it = 1;
#pragma unroll
      for (int k = 0; k < 4; ++k) p[k] = pe[k];
      if (isnan(chi)) {
        finish = true;
        state = FS_STATE_NOT_CONVERGED;
      } else if (chi < a.max_error) {
        finish = true;
        state = FS_STATE_MAX_ERROR;
      } else {
        chib = chi;
        alb = alpha;
        bpb = bp;
        noiseb = noise;
        rab = ra_t;
        rbb = rb_t;
        need_grad = true;
      }
    } else {
      const float Chi = chi;
      const bool nan_t = isnan(Chi);
      if (first_trial && !nan_t && delta < 0.f) --klam;  // error decreased: lambda / 10
      first_trial = false;
      const float ms = a.min_step;
      const bool small = fabsf(dl[0]) < ms * fabsf(p[0]) && fabsf(dl[1]) < ms * fabsf(p[1]) &&
                         fabsf(dl[2]) < ms * fabsf(p[2]) &&
                         (iso || fabsf(dl[3]) < ms * fabsf(p[3]));
      if (!small && !nan_t && delta > 0.f && klam < 4) {
        ++klam;  // reject: lambda * 10, same normal equations
        need_solve = true;
      } else if (nan_t || delta > 0.f) {
        finish = true;  // keep the best point
        state = (small && !nan_t) ? FS_STATE_NO_DECREASE : FS_STATE_NOT_CONVERGED;
        ra = rab;
        rb = rbb;
        rc = chib;
      } else {
        const float chi_prev = chib;
#pragma unroll
        for (int k = 0; k < 4; ++k) p[k] = pe[k];
        chib = Chi;
        alb = alpha;
        bpb = bp;
        noiseb = noise;
        rab = ra_t;
        rbb = rb_t;
        if (Chi < a.max_error) {
          finish = true;
          state = FS_STATE_MAX_ERROR;
        } else if (delta > -a.min_delta * chi_prev) {
          finish = true;
          state = FS_STATE_MIN_DELTA;
        } else if (small) {
          finish = true;
          state = FS_STATE_MIN_STEP;
        } else if (it >= a.max_iter) {
          finish = true;
          state = FS_STATE_MAX_ITER;
        } else {
          ++it;
          need_grad = true;
        }
      }
    }

    float A[10], bv[4];
    if (need_grad) {
      // normal equations at p (= pe) from this evaluation's sums
      const float xm[8] = {RES(RT1 + 1, j), RES(RT1 + 2, j), RES(RT1 + 5, j), RES(RT1 + 6, j),
                           RES(RT1 + 7, j), RES(RT1 + 8, j), RES(RT1 + 9, j), RES(RT1 + 10, j)};
      const float ym[8] = {RES(RT1 + 3, j),  RES(RT1 + 4, j),  RES(RT1 + 11, j),
                           RES(RT1 + 12, j), RES(RT1 + 13, j), RES(RT1 + 14, j),
                           RES(RT1 + 15, j), RES(RT1 + 16, j)};
      const float tr[5] = {RES(RT2 + 1, j), RES(RT2 + 2, j), RES(RT2 + 3, j), RES(RT2 + 4, j),
                           RES(RT2 + 5, j)};
      normal_equations(xm, ym, tr, Nf, am, pe[2], iso ? pe[2] : pe[3], pe[1] - yc, iso, A, bv);
#pragma unroll
      for (int k = 0; k < 10; ++k) ST(SA + k, j) = A[k];
#pragma unroll
      for (int k = 0; k < 4; ++k) ST(SBV + k, j) = bv[k];
      first_trial = true;
      need_solve = true;
    } else if (need_solve) {
#pragma unroll
      for (int k = 0; k < 10; ++k) A[k] = ST(SA + k, j);
#pragma unroll
      for (int k = 0; k < 4; ++k) bv[k] = ST(SBV + k, j);
    }
    if (need_solve) {
      float d[4];
      resolve = false;
      if (solve_damped(A, bv, pow10i(klam), d)) {
        if (iso) d[3] = d[2];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          dl[k] = d[k];
          pe[k] = p[k] + d[k];
        }
        limit_params(pe, W, H, iso);
      } else if (klam < 4) {
        // not positive definite at this lambda (FP32 rounding of a nearly singular J^T J):
        // tenfold damping, solved in the slot's next round, which evaluates nothing
        ++klam;
        resolve = true;
      } else {
        finish = true;
        state = FS_STATE_NOT_CONVERGED;
        ra = rab;
        rb = rbb;
        rc = chib;
      }
    }
    if (finish) {
      // a transposed spot's parameters go back to the caller's orientation
      const float sxo = p[2], syo = iso ? p[2] : p[3];
      a.out_params[4 * spot + 0] = trans ? p[1] : p[0];
      a.out_params[4 * spot + 1] = trans ? p[0] : p[1];
      a.out_params[4 * spot + 2] = trans ? syo : sxo;
      a.out_params[4 * spot + 3] = trans ? sxo : syo;
      a.out_alpha[spot] = ra;
      a.out_beta[spot] = rb;
      a.out_chi2[spot] = rc / (Nf - (float)(P + 2));
      a.out_state[spot] = state;
      a.out_iters[spot] = it;
      if (a.out_evals) a.out_evals[spot] = evals;
      active = false;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ST(SP + k, j) = p[k];
      ST(SPE + k, j) = pe[k];
      ST(SDL + k, j) = dl[k];
    }
    STI(SKLAM, j) = klam;
    STI(SIT, j) = it;
    STI(SEVALS, j) = evals;
    ST(SCHIB, j) = chib;
    ST(SALB, j) = alb;
    ST(SBPB, j) = bpb;
    ST(SNOISEB, j) = noiseb;
    ST(SRA, j) = rab;
    ST(SRB, j) = rbb;
    flags = (flags & (kFirstEval - 1)) | (first_eval ? kFirstEval : 0) |
            (first_trial ? kFirstTrial : 0) | (active ? kActive : 0) |
            (resolve && active ? kResolve : 0);
    STI(SFLAGS, j) = flags;
  return active;
}

// One evaluation of slot j with one column per lane (L = 32, C = 1): profile, pass 1, the
// amplitude solve, pass 2, chi^2 and its refinement, the results handed to the slot's lane.
// kTrans: the slot's ROI is the transpose of the caller's (element (x, y) at x H + y);
// kMulti: rows in more than one block of R (the elongated class: the block loop runs at run
// time, rows past the spot are skipped and the row weights take the spot's centre H / 2 as
// origin). Otherwise the loops are fully unrolled over R rows, padding rows holding zeros.
template <int R, int NB, bool kMulti, bool kTrans>
__device__ __forceinline__ void eval_one_column(const FitArgs &a, float *const st,
                                                float *const res, float *const tab,
                                                float *const red, float2 *const rtab,
                                                float *const racc, float *const tot1,
                                                float *const tot2, float *const tot3,
                                                const int j, const int lane, const bool rtrans) {
  constexpr int L = 32, RT = NB * R, NR = (RT + L - 1) / L, RS = red_stride(L);
  constexpr int NRE = kMulti ? NR : 1;  // row-table passes this path needs
  constexpr float yc0 = 0.5f * (float)RT;
  constexpr bool kElong = kMulti;
  constexpr unsigned full = 0xffffffffu;
  const int lg = lane;
    const int flags = STI(SFLAGS, j);
    const int W = flag_w(flags), H = flag_h(flags);
    const bool iso = flags & kIsoBit, first_eval = flags & kFirstEval;
    const bool trans = kMulti ? rtrans : kTrans;  // one row-block path for both orientations
    const int64_t off =
        (int64_t)(((uint64_t)(uint32_t)STI(SOFFHI, j) << 32) | (uint32_t)STI(SOFFLO, j));
    // element strides of a step along the lanes' axis and along the rows
    const int cs = trans ? H : 1, rs = trans ? 1 : W;
    const int nb = kMulti ? (H + R - 1) / R : 1;  // row blocks of this spot
    const bool fullroi = !kElong && !kTrans && W == 32 && H == R;
    const float Nf = (float)(W * H);
    const float yc = kElong ? 0.5f * (float)H : yc0;  // origin of the row weights
    float pe[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) pe[k] = ST(SPE + k, j);
    const int x = lg;
    float g2[1][R];
    float (&g)[R] = g2[0];
    float shift, Gs;
    if (first_eval) {
      // integer shift = corner pixel (a background estimate); refined after pass 1
      float part = 0.f;
      shift = 0.f;
      for (int b = 0; b < nb; ++b) {
        load_rows<32, 1, R>(a, off, cs, rs, W, H, x, b * R, fullroi, shift, g2);
        if (b == 0) {
          shift = rintf(__shfl_sync(full, g[0], 0));
#pragma unroll
          for (int y = 0; y < R; ++y) g[y] = (x < W && y < H) ? g[y] - shift : 0.f;
        }
#pragma unroll
        for (int y = 0; y < R; ++y) part += g[y];
      }
      Gs = group_sum_shfl<L>(part, full);
    } else {
      shift = ST(SSH0, j);
      Gs = ST(SGS, j);
      load_rows<32, 1, R>(a, off, cs, rs, W, H, x, (nb - 1) * R, fullroi, shift, g2);
    }
    const float gs1 = Gs, sh1 = shift;  // the pixel sum and shift of the amplitude sums
    // the registers hold the spot's last row block

    const float sx = pe[2], sy = iso ? pe[2] : pe[3];
    const float ivx = inv_sq(sx), ivy = inv_sq(sy);
    const float nhx = -0.5f * ivx, nhy = -0.5f * ivy;
    float ex, dxv;
    {
      // column profile e_x and the column moments sum dx^m e_x^n
      float m[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const float d = (float)x - pe[0];
      const float e = (x < W) ? __expf(d * d * nhx) : 0.f;
      ex = e;
      dxv = d;
      moment_terms(d, e, m);
      red[1 * RS + lg] = m[0];
      red[2 * RS + lg] = m[1];
#pragma unroll
      for (int k = 0; k < 6; ++k) red[(5 + k) * RS + lg] = m[2 + k];
    }
    {
      // row profile e_y into the table, and the row moments
      float m[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < NRE; ++k) {
        const int y = lg + 32 * k;
        if (y < RT && (!kElong || 32 * k < H)) {  // rows past the spot are never read
          const float d = (float)y - pe[1];
          const float e = (y < H) ? __expf(d * d * nhy) : 0.f;
          tab[y] = e;
          moment_terms(d, e, m);
        }
      }
      red[3 * RS + lg] = m[0];
      red[4 * RS + lg] = m[1];
#pragma unroll
      for (int k = 0; k < 6; ++k) red[(11 + k) * RS + lg] = m[2 + k];
    }
    __syncwarp();
    // pass 1: s(x) = sum_y e_y g'(x, y);  FG' partial = e_x s(x); blocks last to first
    {
      float s0 = 0.f;
      for (int b = nb - 1; b >= 0; --b) {
        if (b != nb - 1) load_rows<32, 1, R>(a, off, cs, rs, W, H, x, b * R, false, shift, g2);
        if constexpr (kElong) {
#pragma unroll
          for (int y = 0; y < R; ++y)
            if (b * R + y < H) s0 = fmaf(tab[b * R + y], g[y], s0);  // rows of the spot
        } else {
          // four rows of the table per 16-byte broadcast read
          const float4 *const t4 = reinterpret_cast<const float4 *>(tab);
#pragma unroll
          for (int q = 0; q < R / 4; ++q) {
            const float4 e = t4[q];
            s0 = fmaf(e.x, g[4 * q], s0);
            s0 = fmaf(e.y, g[4 * q + 1], s0);
            s0 = fmaf(e.z, g[4 * q + 2], s0);
            s0 = fmaf(e.w, g[4 * q + 3], s0);
          }
        }
      }
      red[lg] = ex * s0;
    }
    // the registers hold the first row block
    group_reduce<L, K1>(red, tot1, lg, full);
    const float4 t1a = reinterpret_cast<const float4 *>(tot1)[0];
    const float FG = t1a.x, X01 = t1a.y, X02 = t1a.z, Y01 = t1a.w, Y02 = tot1[4];
    const float F = X01 * Y01, FF = X02 * Y02;
    const float D = fmaf(Nf, FF, -F * F);
    const bool okD = D > 0.f && isfinite(D);
    const float iD = __fdividef(1.f, D);
    const float alpha = (Nf * FG - F * Gs) * iD;  // Eq. 6, for the pixel passes
    float bp = (Gs * FF - F * FG) * iD;           // beta^ - shift
    if (first_eval && okD) {
      // move the shift to the integer nearest beta^ (exact for integer pixel values)
      const float dl0 = rintf(bp);
#pragma unroll
      for (int y = 0; y < R; ++y) g[y] = (x < W && y < H) ? g[y] - dl0 : 0.f;
      Gs = fmaf(-Nf, dl0, Gs);
      shift += dl0;
      bp -= dl0;
    }
    // pass 2: u = g' - alpha e_x e_y; chi_u = sum u^2; row-weighted sums of e_y u;
    // blocks first to last
    {
      const float ca = -alpha * ex;
      float ch0 = 0.f, ch1 = 0.f, t0 = 0.f, t1 = 0.f, t2 = 0.f;
      for (int b = 0; b < nb; ++b) {
        if (b != 0) load_rows<32, 1, R>(a, off, cs, rs, W, H, x, b * R, false, shift, g2);
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
          // four rows of the table per 16-byte broadcast read (one row at a time in row blocks)
          const float4 e4 = kElong ? make_float4(0.f, 0.f, 0.f, 0.f)
                                   : reinterpret_cast<const float4 *>(tab)[q];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int y = 4 * q + r;
            if (!kElong || b * R + y < H) {  // padding rows hold zeros
              const float e = kElong ? tab[b * R + y] : r == 0 ? e4.x : r == 1 ? e4.y : r == 2 ? e4.z : e4.w;
              const float yy = (float)(b * R + y) - yc;
              const float u = fmaf(ca, e, g[y]);
              if (y & 1) ch1 = fmaf(u, u, ch1);
              else ch0 = fmaf(u, u, ch0);
              const float w = e * u;
              t0 += w;
              t1 = fmaf(yy, w, t1);
              t2 = fmaf(yy * yy, w, t2);
            }
          }
        }
      }
      const float e = ex, d = dxv;
      const float et0 = e * t0;
      red[0 * RS + lg] = ch0 + ch1;
      red[1 * RS + lg] = et0;
      red[2 * RS + lg] = d * et0;
      red[3 * RS + lg] = d * d * et0;
      red[4 * RS + lg] = e * t1;
      red[5 * RS + lg] = e * t2;
    }
    // the registers hold the last row block
    group_reduce<L, K2>(red, tot2, lg, full);
    const float chiu = tot2[0];
    const float Su = fmaf(-alpha, F, Gs);             // sum u = G' - alpha F
    float chi = chiu - 2.f * bp * Su + Nf * bp * bp;  // Eq. 2: sum (u - beta')^2
    if (!okD || !isfinite(alpha)) chi = __int_as_float(0x7fc00000);

    // chi^2 change, refined near the decision thresholds (as in the per-spot kernel)
    const float noise =
        24.f * 5.9604645e-8f * fabsf(alpha) * sqrtf(fmaxf(chi, 0.f) * FF * __fdividef(1.f, Nf));
    const float chib = ST(SCHIB, j), noiseb = ST(SNOISEB, j);
    float delta = chi - chib;
    const float win = kTieWindow * chib + noise + noiseb;
    if (!first_eval && isfinite(chi) && isfinite(chib) && delta >= -a.min_delta * chib - win &&
        delta <= win) {
      float p[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) p[k] = ST(SP + k, j);
      const float alb = ST(SALB, j), bpb = ST(SBPB, j);
      const float sbx = p[2], sby = iso ? p[2] : p[3];
      const float ivbx = inv_sq(sbx), ivby = inv_sq(sby);
      const float nhbx = -0.5f * ivbx, nhby = -0.5f * ivby;
      const float dsx = sx - sbx, dsy = sy - sby;
      const float d0 = pe[0] - p[0], d1 = pe[1] - p[1];
      const float kx = dsx * (sx + sbx) * ivx * ivbx, ky = dsy * (sy + sby) * ivy * ivby;
      float mx, omx, exb, cab;
      {
        const float db = (float)x - p[0], dt = dxv;
        const float dxe = 0.5f * fmaf(d0 * (dt + db), ivx, db * db * kx);
        mx = (x < W) ? expm1_small(dxe) : 0.f;
        omx = 1.f + mx;
        exb = (x < W) ? __expf(db * db * nhbx) : 0.f;
        cab = -alb * exb;
      }
      __syncwarp();  // the elongated table replaces the row table
#pragma unroll
      for (int k = 0; k < NRE; ++k) {
        const int y = lg + 32 * k;
        if (y < RT && (!kElong || 32 * k < H)) {
          const float db = (float)y - p[1], dt = (float)y - pe[1];
          const float dye = 0.5f * fmaf(d1 * (dt + db), ivy, db * db * ky);
          rtab[y] = (y < H) ? make_float2(expm1_small(dye), __expf(db * db * nhby))
                            : make_float2(0.f, 0.f);
        }
      }
      __syncwarp();
      const float dal = alpha - alb, dbp = bp - bpb;
      float acc = 0.f;
      for (int b = nb - 1; b >= 0; --b) {
        if (b != nb - 1) load_rows<32, 1, R>(a, off, cs, rs, W, H, x, b * R, false, shift, g2);
#pragma unroll
        for (int y = 0; y < R; ++y) {
          const int row = b * R + y;
          if (row < H && x < W) {
            const float2 q = rtab[row];
            const float fb = exb * q.y;
            const float tt = fmaf(q.x, omx, mx);
            const float dh = fmaf(fb, fmaf(alpha, tt, dal), dbp);
            const float rb = fmaf(cab, q.y, g[y]) - bpb;
            acc = fmaf(dh, fmaf(-2.f, rb, dh), acc);
          }
        }
      }
      racc[lg] = acc;
      group_reduce<L, 1>(racc, tot3, lg, full);
      delta = tot3[0];
    }
    // hand the results to the slot's lane
    if (lane < 7) {
      const float v = lane == 0   ? alpha
                      : lane == 1 ? bp
                      : lane == 2 ? chi
                      : lane == 3 ? noise
                      : lane == 4 ? delta
                      : lane == 5 ? gs1
                                  : sh1;
      RES(lane, j) = v;
    }
    if (lane < K1) RES(RT1 + lane, j) = tot1[lane];
    if (lane < K2) RES(RT2 + lane, j) = tot2[lane];
    if (first_eval && lane == 0) {
      ST(SSH0, j) = shift;
      ST(SGS, j) = Gs;
    }
    __syncwarp();
}

// One size class, drained by one warp: slots are refilled from the class's queue until it
// runs dry and every slot has finished. (L, C, R) is the evaluation geometry. NB > 1 only with
// L = 32, C = 1: the generic geometry (any ROI of at most 1024 pixels), rows in blocks of R,
// at most NB of them.
template <int L, int C, int R, int NB, bool G>
__device__ __forceinline__ void batched_drain(const FitArgs &a, const int cls, const int wf) {
  constexpr int S = 32 / L;
  constexpr int RT = NB * R;          // rows of the row table
  constexpr int NR = (RT + L - 1) / L;
  constexpr int RS = red_stride(L);
  constexpr float yc0 = 0.5f * (float)RT;
  constexpr bool kElong = NB > 1;  // row blocks: the elongated class (per-spot row origin)
  constexpr unsigned full = 0xffffffffu;
  static_assert(S * L == 32, "lane groups must tile a warp");
  static_assert(!G || (L == 32 && C == 1), "the generic geometry has one column per lane");
  static_assert(NB == 1 || G, "row blocks need the generic geometry");
  static_assert(kElong || 2 * RT + 2 <= (K1 - 1) * RS, "refinement table fits the reduction rows");
  static_assert(!kElong || 2 * RT + 2 <= round_up(RT + 1, 4) + (K1 - 1) * RS,
                "refinement table fits the row table and the reduction rows");
  float *const sw = reinterpret_cast<float *>(g_smem4) + (threadIdx.x >> 5) * wf;
  float *const st = sw;                          // [kSlotFields][kSlots]
  float *const res = sw + kSlotFields * kSlots;  // [kResFields][kSlots]
  float *const pw = sw + round_up((kSlotFields + kResFields) * kSlots, 32);  // pass area
  const int lane = threadIdx.x & 31;
  const int gi = lane / L, lg = lane % L;
  const unsigned gmask = (L == 32) ? full : (((1u << L) - 1u) << (gi * L));
  float *const tab = pw + gi * (RT + 1);
  float *const red = pw + tab_floats(L, RT) + gi * group_stride(L);
  // tie-refinement table: free reduction rows (one group per warp for the elongated class,
  // whose table also takes the row table's place) and the row of its own reduction
  float2 *const rtab = reinterpret_cast<float2 *>(kElong ? tab : red + RS);
  float *const racc = kElong ? red + (K1 - 1) * RS : red;
  float *const tot1 = red + K1 * RS;
  float *const tot2 = tot1 + 20;
  float *const tot3 = tot2 + 8;

  const int cnt = a.uniform ? a.n : a.counts[cls];
  const int beg = a.uniform ? 0 : a.starts[cls];
  // lane j < kSlots owns slot j: its activity and whether the class has run dry for it
  bool active = false, idle = lane >= kSlots || cnt == 0;
  if (lane < kSlots) STI(SFLAGS, lane) = 0;
  __syncwarp();
  while (true) {
    // -------------------------------------------------------------- refill free slots
    {
      const bool need = !active && !idle;
      const unsigned m = __ballot_sync(full, need);
      if (m) {
        const int leader = __ffs(m) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(a.cursors + cls, __popc(m));
        base = __shfl_sync(full, base, leader);
        if (need) {
          const int item = base + __popc(m & ((1u << lane) - 1u));
          if (item >= cnt) {
            idle = true;
          } else {
            int spot, W, H, mod;
            int64_t off;
            if (a.uniform) {
              spot = item;
              off = (int64_t)item * (a.uw * a.uh);
              W = a.uw;
              H = a.uh;
              mod = a.umodel;
            } else {
              spot = a.perm[beg + item];
              off = a.offsets[spot];
              W = a.dims[2 * spot];
              H = a.dims[2 * spot + 1];
              mod = a.model[spot];
            }
            const bool iso = mod == FS_MODEL_ISO;
            // row-block geometry: the longer side along the lanes when it fits them (fewer
            // row blocks, more lanes busy), else the shorter one (the long side in rows)
            const bool trans = G && (W > kMaxSide || (H <= kMaxSide && H > W));
            float q[4], pe[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = a.init[4 * spot + k];
            if (trans) {
              pe[0] = q[1];
              pe[1] = q[0];
              pe[2] = iso ? q[2] : q[3];
              pe[3] = q[2];
              const int t = W;
              W = H;
              H = t;
            } else {
#pragma unroll
              for (int k = 0; k < 4; ++k) pe[k] = q[k];
            }
            limit_params(pe, W, H, iso);
#pragma unroll
            for (int k = 0; k < 4; ++k) ST(SPE + k, lane) = pe[k];
            STI(SKLAM, lane) = -2;
            STI(SIT, lane) = 0;
            STI(SEVALS, lane) = 0;
            STI(SSPOT, lane) = spot;
            STI(SOFFLO, lane) = (int)(off & 0xffffffff);
            STI(SOFFHI, lane) = (int)(off >> 32);
            STI(SFLAGS, lane) = W | (H << 9) | (iso ? kIsoBit : 0) | (trans ? kTransBit : 0) |
                                kFirstEval | kActive;
            active = true;
          }
        }
      }
    }
    if (!__ballot_sync(full, active)) break;
    // slots to evaluate now: the active ones without a pending re-solve
    const unsigned amask =
        __ballot_sync(full, active && lane < kSlots && !(STI(SFLAGS, lane) & kResolve));
    __syncwarp();

    if constexpr (L == 32 && C == 1) {
      // one spot per warp, one column per lane (80 registers, 6 blocks per SM)
      for (unsigned rem = amask; rem; rem &= rem - 1) {
        const int j = __ffs(rem) - 1;
        const bool tr = G && (STI(SFLAGS, j) & kTransBit);  // warp-uniform
        if constexpr (NB > 1) {
          eval_one_column<R, NB, true, false>(a, st, res, tab, red, rtab, racc, tot1, tot2, tot3, j,
                                              lane, tr);
        } else if constexpr (G) {
          // the oriented ROI's rows rounded up to 8: its pixels in 8, 16, 24 or 32 registers
          const int rb = (flag_h(STI(SFLAGS, j)) + 7) >> 3;
#define FS_GEN_EVAL(RB)                                                                          \
  if (tr)                                                                                        \
    eval_one_column<RB, 1, false, true>(a, st, res, tab, red, rtab, racc, tot1, tot2, tot3, j,   \
                                        lane, true);                                             \
  else                                                                                           \
    eval_one_column<RB, 1, false, false>(a, st, res, tab, red, rtab, racc, tot1, tot2, tot3, j,  \
                                         lane, false);
          if (rb == 1) {
            FS_GEN_EVAL(8)
          } else if (rb == 2) {
            FS_GEN_EVAL(16)
          } else if (rb == 3) {
            FS_GEN_EVAL(24)
          } else {
            FS_GEN_EVAL(32)
          }
#undef FS_GEN_EVAL
        } else {
          eval_one_column<R, NB, false, false>(a, st, res, tab, red, rtab, racc, tot1, tot2, tot3, j,
                                               lane, false);
        }
      }
    } else {
      // -------------------------------------------------------------- evaluate the slots,
      // S at a time (group gi takes the gi-th remaining active slot)
      for (unsigned rem = amask; rem;) {
        unsigned r = rem;
#pragma unroll
        for (int k = 0; k < S - 1; ++k)
          if (k < gi) r &= r - 1;
#pragma unroll
        for (int k = 0; k < S; ++k) rem &= rem - 1;
        if (r) {
          const int j = __ffs(r) - 1;
          const int flags = STI(SFLAGS, j);
          const int W = flag_w(flags), H = flag_h(flags);
          const bool iso = flags & kIsoBit;
          const bool first_eval = flags & kFirstEval;
          const int64_t off =
              (int64_t)(((uint64_t)(uint32_t)STI(SOFFHI, j) << 32) | (uint32_t)STI(SOFFLO, j));
          const float Nf = (float)(W * H);
          float pe[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) pe[k] = ST(SPE + k, j);
          float g[C][R];
          float shift, Gs;
          if (first_eval) {
            // integer shift = corner pixel (a background estimate); refined after pass 1
            load_rows<L, C, R>(a, off, 1, W, W, H, lg, 0, false, 0.f, g);
            shift = rintf(__shfl_sync(gmask, g[0][0], gi * L));
            float part = 0.f;
#pragma unroll
            for (int c = 0; c < C; ++c) {
              const int x = lg + L * c;
#pragma unroll
              for (int y = 0; y < R; ++y) {
                g[c][y] = (x < W && y < H) ? g[c][y] - shift : 0.f;
                part += g[c][y];
              }
            }
            Gs = group_sum_shfl<L>(part, gmask);
          } else {
            shift = ST(SSH0, j);
            Gs = ST(SGS, j);
            load_rows<L, C, R>(a, off, 1, W, W, H, lg, 0, W == L * C && H == R, shift, g);
          }
          const float gs1 = Gs, sh1 = shift;  // the pixel sum and shift of the amplitude sums
          const float sx = pe[2], sy = iso ? pe[2] : pe[3];
          const float ivx = inv_sq(sx), ivy = inv_sq(sy);
          const float nhx = -0.5f * ivx, nhy = -0.5f * ivy;
          float ex[C], dxv[C];
          {
            // column profile e_x and the column moments sum dx^m e_x^n
            float m[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < C; ++c) {
              const int x = lg + L * c;
              const float d = (float)x - pe[0];
              const float e = (x < W) ? __expf(d * d * nhx) : 0.f;
              ex[c] = e;
              dxv[c] = d;
              moment_terms(d, e, m);
            }
            // slots: 1 X01, 2 X02, 5 X11, 6 X21, 7 X12, 8 X22, 9 X32, 10 X42
            red[1 * RS + lg] = m[0];
            red[2 * RS + lg] = m[1];
#pragma unroll
            for (int k = 0; k < 6; ++k) red[(5 + k) * RS + lg] = m[2 + k];
          }
          {
            // row profile e_y into the group's table, and the row moments
            float m[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < NR; ++k) {
              const int y = lg + L * k;
              if (y < R) {
                const float d = (float)y - pe[1];
                const float e = (y < H) ? __expf(d * d * nhy) : 0.f;
                tab[y] = e;
                moment_terms(d, e, m);
              }
            }
            // slots: 3 Y01, 4 Y02, 11 Y11, 12 Y21, 13 Y12, 14 Y22, 15 Y32, 16 Y42
            red[3 * RS + lg] = m[0];
            red[4 * RS + lg] = m[1];
#pragma unroll
            for (int k = 0; k < 6; ++k) red[(11 + k) * RS + lg] = m[2 + k];
          }
          __syncwarp(gmask);
          // pass 1: s(x) = sum_y e_y g'(x, y);  FG' partial = sum_x e_x s(x)
          {
            float s0[C];
#pragma unroll
            for (int c = 0; c < C; ++c) s0[c] = 0.f;
#pragma unroll
            for (int y = 0; y < R; ++y) {
              const float e = tab[y];
#pragma unroll
              for (int c = 0; c < C; ++c) s0[c] = fmaf(e, g[c][y], s0[c]);
            }
            float fg = 0.f;
#pragma unroll
            for (int c = 0; c < C; ++c) fg = fmaf(ex[c], s0[c], fg);
            red[lg] = fg;
          }
          group_reduce<L, K1>(red, tot1, lg, gmask);
          const float4 t1a = reinterpret_cast<const float4 *>(tot1)[0];
          const float FG = t1a.x, X01 = t1a.y, X02 = t1a.z, Y01 = t1a.w, Y02 = tot1[4];
          const float F = X01 * Y01, FF = X02 * Y02;
          const float D = fmaf(Nf, FF, -F * F);
          const bool okD = D > 0.f && isfinite(D);
          const float iD = __fdividef(1.f, D);
          const float alpha = (Nf * FG - F * Gs) * iD;  // Eq. 6, for the pixel passes
          float bp = (Gs * FF - F * FG) * iD;           // beta^ - shift
          if (first_eval && okD) {
            // move the shift to the integer nearest beta^ (exact for integer pixel values)
            const float dl0 = rintf(bp);
#pragma unroll
            for (int c = 0; c < C; ++c) {
              const int x = lg + L * c;
#pragma unroll
              for (int y = 0; y < R; ++y) g[c][y] = (x < W && y < H) ? g[c][y] - dl0 : 0.f;
            }
            Gs = fmaf(-Nf, dl0, Gs);
            shift += dl0;
            bp -= dl0;
          }
          // pass 2: u = g' - alpha e_x e_y; chi_u = sum u^2; row-weighted sums of e_y u
          {
            float ca[C], ch0[C], ch1[C], t0[C], t1[C], t2[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
              ca[c] = -alpha * ex[c];
              ch0[c] = ch1[c] = t0[c] = t1[c] = t2[c] = 0.f;
            }
#pragma unroll
            for (int y = 0; y < R; ++y) {
              const float e = tab[y];
              const float yy = (float)y - yc0;
#pragma unroll
              for (int c = 0; c < C; ++c) {
                const float u = fmaf(ca[c], e, g[c][y]);
                if (y & 1) ch1[c] = fmaf(u, u, ch1[c]);
                else ch0[c] = fmaf(u, u, ch0[c]);
                const float w = e * u;
                t0[c] += w;
                t1[c] = fmaf(yy, w, t1[c]);
                t2[c] = fmaf(yy * yy, w, t2[c]);
              }
            }
            float v2[K2] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < C; ++c) {
              const float e = ex[c], d = dxv[c];
              const float et0 = e * t0[c];
              v2[0] += ch0[c] + ch1[c];
              v2[1] += et0;
              v2[2] = fmaf(d, et0, v2[2]);
              v2[3] = fmaf(d * d, et0, v2[3]);
              v2[4] = fmaf(e, t1[c], v2[4]);
              v2[5] = fmaf(e, t2[c], v2[5]);
            }
#pragma unroll
            for (int k = 0; k < K2; ++k) red[k * RS + lg] = v2[k];
          }
          group_reduce<L, K2>(red, tot2, lg, gmask);
          const float chiu = tot2[0];
          const float Su = fmaf(-alpha, F, Gs);             // sum u = G' - alpha F
          float chi = chiu - 2.f * bp * Su + Nf * bp * bp;  // Eq. 2: sum (u - beta')^2
          if (!okD || !isfinite(alpha)) chi = __int_as_float(0x7fc00000);

          // ------------------------------------------------------------ chi^2 change
          // delta = chi_t^2 - chi_b^2, refined near the two decision thresholds. The window
          // covers the FP32 error of each chi^2: rounding alpha f and the profile in every
          // residual u gives errors of ~eps |alpha| f per pixel, i.e. a chi^2 error of about
          // 6 eps |alpha| sqrt(chi^2 F(bold) / N); the window takes four times that per point.
          const float chib = ST(SCHIB, j), noiseb = ST(SNOISEB, j);
          const float noise =
              24.f * 5.9604645e-8f * fabsf(alpha) * sqrtf(fmaxf(chi, 0.f) * FF * __fdividef(1.f, Nf));
          float delta = chi - chib;
          const float win = kTieWindow * chib + noise + noiseb;
          if (!first_eval && isfinite(chi) && isfinite(chib) && delta >= -a.min_delta * chib - win &&
              delta <= win) {
            float p[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) p[k] = ST(SP + k, j);
            const float alb = ST(SALB, j), bpb = ST(SBPB, j);
            const float sbx = p[2], sby = iso ? p[2] : p[3];
            const float ivbx = inv_sq(sbx), ivby = inv_sq(sby);
            const float nhbx = -0.5f * ivbx, nhby = -0.5f * ivby;
            const float dsx = sx - sbx, dsy = sy - sby;
            const float d0 = pe[0] - p[0], d1 = pe[1] - p[1];
            const float kx = dsx * (sx + sbx) * ivx * ivbx, ky = dsy * (sy + sby) * ivy * ivby;
            float mx[C], omx[C], exb[C], cab[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
              const int x = lg + L * c;
              const float db = (float)x - p[0], dt = dxv[c];
              // exponent difference x_t - x_b, from the parameter differences
              const float dxe = 0.5f * fmaf(d0 * (dt + db), ivx, db * db * kx);
              mx[c] = (x < W) ? expm1_small(dxe) : 0.f;
              omx[c] = 1.f + mx[c];
              exb[c] = (x < W) ? __expf(db * db * nhbx) : 0.f;
              cab[c] = -alb * exb[c];
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) {
              const int y = lg + L * k;
              if (y < R) {
                const float db = (float)y - p[1], dt = (float)y - pe[1];
                const float dye = 0.5f * fmaf(d1 * (dt + db), ivy, db * db * ky);
                rtab[y] = (y < H) ? make_float2(expm1_small(dye), __expf(db * db * nhby))
                                  : make_float2(0.f, 0.f);
              }
            }
            __syncwarp(gmask);
            const float dal = alpha - alb, dbp = bp - bpb;
            float acc = 0.f;
#pragma unroll
            for (int y = 0; y < R; ++y) {
              if (y < H) {  // padding rows and columns are not part of the spot
                const float2 q = rtab[y];  // (e_y,t / e_y,b - 1, e_y,b)
#pragma unroll
                for (int c = 0; c < C; ++c) {
                  if (lg + L * c < W) {
                    const float fb = exb[c] * q.y;
                    const float tt = fmaf(q.x, omx[c], mx[c]);             // f_t / f_b - 1
                    const float dh = fmaf(fb, fmaf(alpha, tt, dal), dbp);  // h_t - h_b
                    const float rb = fmaf(cab[c], q.y, g[c][y]) - bpb;     // g - h_b
                    acc = fmaf(dh, fmaf(-2.f, rb, dh), acc);
                  }
                }
              }
            }
            racc[lg] = acc;
            group_reduce<L, 1>(racc, tot3, lg, gmask);
            delta = tot3[0];
          }

          // hand the results to the slot's lane
          if (lg < 7) {
            const float v = lg == 0   ? alpha
                            : lg == 1 ? bp
                            : lg == 2 ? chi
                            : lg == 3 ? noise
                            : lg == 4 ? delta
                            : lg == 5 ? gs1
                                      : sh1;
            RES(lg, j) = v;
          }
#pragma unroll
          for (int k0 = 0; k0 < K1; k0 += L)
            if (k0 + lg < K1) RES(RT1 + k0 + lg, j) = tot1[k0 + lg];
          if (lg < K2) RES(RT2 + lg, j) = tot2[lg];
          if (first_eval && lg == 0) {
            ST(SSH0, j) = shift;
            ST(SGS, j) = Gs;
          }
        }
        __syncwarp();
      }
    }

    // -------------------------------------------------------------- LM step, lane per slot
    if (active) active = lm_step(a, wf, lane, yc0, NB > 1 ? 2 : G ? 1 : 0);
    __syncwarp();
  }
}
#undef ST
#undef STI
#undef RES

// The classes of ROIs with both sides at most 16: the single mixed launch drains them with
// the 16-lane batched geometry (two spots per warp evaluation) instead of the generic
// 32-lane one, which would leave half of its lanes or more without a column.
__host__ __device__ constexpr bool small_class(int cls) {
  return cls == 0 || cls == 1 || cls == 4 || cls == 5;
}
constexpr int kSmallL = 16, kSmallR = 16;

// A batched configuration as a kernel of its own: drains the classes of `cl` in order. The
// generic configuration (G, one row block) takes the small classes with the 16-lane
// geometry, so that one launch still serves every class.
template <int L, int C, int R, int NB, bool G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, NB > 1 ? 5 : batched_min_blocks(C, R))
    fit_kernel_batched(FitArgs a, ClassList cl) {
  // per-warp stride of the block's shared memory: one for both geometries, since the warps
  // of a block can be in different classes at the same time
  constexpr int wf = G && NB == 1 ? (batched_warp_floats(L, R) > batched_warp_floats(kSmallL, kSmallR)
                                         ? batched_warp_floats(L, R)
                                         : batched_warp_floats(kSmallL, kSmallR))
                                  : batched_warp_floats(L, NB * R);
  for (int ci = 0; ci < cl.count; ++ci) {
    if constexpr (G && NB == 1) {
      if (small_class(cl.cls[ci])) {
        batched_drain<kSmallL, 1, kSmallR, 1, false>(a, cl.cls[ci], wf);
        continue;
      }
    }
    batched_drain<L, C, R, NB, G>(a, cl.cls[ci], wf);
  }
}

// ------------------------------------------------------------------ configurations
// id -> (L, C, R, NB); one kernel instantiation each. Per-spot configurations 0..35: for
// every row bound R, the width bound 8 has (4,2) (8,1); 16 has (4,4) (8,2) (16,1); 24 has
// (8,3); 32 has (8,4) (16,2) (32,1). Batched ones 36..55 (same geometry per evaluation, one
// lane per spot for the LM step): for every row bound, (32, 1) (16, 2) (8, 3) (16, 1) (8, 1).
// Last, the two generic configurations, one column per lane with each ROI oriented (see
// batched_drain): (32, 1, 32) for every class of W, H <= 32, the single launch of a mixed
// batch, and (32, 1, 32) with up to kElongBlocks row blocks, the elongated class's only one.
struct CfgDesc {
  int L, C, R, batched, NB, generic;
};
#define FS_CONFIGS_R(X, b, R)                                                                 \
  X(b + 0, 4, 2, R) X(b + 1, 8, 1, R) X(b + 2, 4, 4, R) X(b + 3, 8, 2, R) X(b + 4, 16, 1, R) \
  X(b + 5, 8, 3, R) X(b + 6, 8, 4, R) X(b + 7, 16, 2, R) X(b + 8, 32, 1, R)
#define FS_CONFIGS(X) \
  FS_CONFIGS_R(X, 0, 8) FS_CONFIGS_R(X, 9, 16) FS_CONFIGS_R(X, 18, 24) FS_CONFIGS_R(X, 27, 32)
#define FS_BATCHED_R(X, R) X(32, 1, R) X(16, 2, R) X(8, 3, R) X(16, 1, R) X(8, 1, R)
#define FS_BATCHED(X) FS_BATCHED_R(X, 8) FS_BATCHED_R(X, 16) FS_BATCHED_R(X, 24) FS_BATCHED_R(X, 32)

#define FS_DESC(id, L, C, R) {L, C, R, 0, 1, 0},
#define FS_BDESC(L, C, R) {L, C, R, 1, 1, 0},
constexpr CfgDesc kConfigs[] = {FS_CONFIGS(FS_DESC) FS_BATCHED(FS_BDESC){32, 1, 32, 1, 1, 1},
                                {32, 1, 32, 1, kElongBlocks, 1}};
#undef FS_DESC
#undef FS_BDESC
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);
constexpr int kGenericConfig = kNumConfigs - 2;  // every class of W, H <= 32, one launch
constexpr int kElongConfig = kNumConfigs - 1;    // the elongated class

typedef void (*FitKernelFn)(FitArgs, ClassList);
#define FS_PTR(id, L, C, R) &fit_kernel<L, C, R>,
#define FS_BPTR(L, C, R) &fit_kernel_batched<L, C, R, 1, false>,
const FitKernelFn kKernels[] = {FS_CONFIGS(FS_PTR) FS_BATCHED(FS_BPTR)
                                     &fit_kernel_batched<32, 1, 32, 1, true>,
                                 &fit_kernel_batched<32, 1, 32, kElongBlocks, true>};
#undef FS_PTR
#undef FS_BPTR
static_assert(sizeof(kKernels) / sizeof(kKernels[0]) == kNumConfigs, "one kernel per configuration");

size_t config_smem_bytes(int cfg) {
  const CfgDesc &c = kConfigs[cfg];
  int per_warp = c.batched ? batched_warp_floats(c.L, c.NB * c.R) : warp_smem_floats(c.L, c.R);
  if (c.generic && c.NB == 1)  // also drains the small classes with the 16-lane geometry
    per_warp = std::max(per_warp, batched_warp_floats(kSmallL, kSmallR));
  return (size_t)kWarpsPerBlock * per_warp * sizeof(float);
}

// ------------------------------------------------------------------ schedule prepass
constexpr int kPrepassThreads = 256;
constexpr int kPrepassChunk = 2048;

__global__ void __launch_bounds__(kPrepassThreads) classify_count_kernel(FitArgs a) {
  __shared__ int h[kNumClasses];
  if (threadIdx.x < kNumClasses) h[threadIdx.x] = 0;
  __syncthreads();
  const int lo = blockIdx.x * kPrepassChunk;
  const int hi = min(a.n, lo + kPrepassChunk);
  for (int s = lo + threadIdx.x; s < hi; s += kPrepassThreads) {
    int W, H, m;
    if (spot_valid(a, s, W, H, m)) atomicAdd(&h[size_class(W, H)], 1);
    else write_invalid(a, s);
  }
  __syncthreads();
  if (threadIdx.x < kNumClasses && h[threadIdx.x]) atomicAdd(&a.counts[threadIdx.x], h[threadIdx.x]);
}

__global__ void classify_scan_kernel(FitArgs a) {
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int c = 0; c < kNumClasses; ++c) {
      a.starts[c] = acc;
      acc += a.counts[c];
    }
  }
}

__global__ void __launch_bounds__(kPrepassThreads) classify_scatter_kernel(FitArgs a) {
  __shared__ int h[kNumClasses], base[kNumClasses];
  if (threadIdx.x < kNumClasses) h[threadIdx.x] = 0;
  __syncthreads();
  const int lo = blockIdx.x * kPrepassChunk;
  const int hi = min(a.n, lo + kPrepassChunk);
  for (int s = lo + threadIdx.x; s < hi; s += kPrepassThreads) {
    int W, H, m;
    if (spot_valid(a, s, W, H, m)) atomicAdd(&h[size_class(W, H)], 1);
  }
  __syncthreads();
  if (threadIdx.x < kNumClasses) {
    base[threadIdx.x] =
        h[threadIdx.x] ? a.starts[threadIdx.x] + atomicAdd(&a.fill[threadIdx.x], h[threadIdx.x]) : 0;
    h[threadIdx.x] = 0;
  }
  __syncthreads();
  for (int s = lo + threadIdx.x; s < hi; s += kPrepassThreads) {
    int W, H, m;
    if (spot_valid(a, s, W, H, m)) {
      const int c = size_class(W, H);
      a.perm[base[c] + atomicAdd(&h[c], 1)] = s;
    }
  }
}

// ------------------------------------------------------------------ host state
constexpr size_t kSchedHeaderBytes = 4 * kNumClasses * sizeof(int32_t);  // counts starts cursors fill

int8_t g_class_cfg[kNumClasses];
std::once_flag g_init_once;
std::mutex g_cfg_mutex;
thread_local int g_last_cuda_error = 0;

int config_for(int L, int C, int R, int batched) {
  for (int i = 0; i < kNumConfigs; ++i)
    if (kConfigs[i].L == L && kConfigs[i].C == C && kConfigs[i].R == R &&
        kConfigs[i].batched == batched && kConfigs[i].NB == 1)
      return i;
  return -1;
}

// A configuration serves a class when its columns cover the class's width bound and its
// rows equal the class's row bound; the elongated class has a configuration of its own.
bool config_fits(int cfg, int cls) {
  if (cfg < 0 || cfg >= kNumConfigs || cls < 0 || cls >= kNumClasses) return false;
  if (cls == kElongClass || cfg == kElongConfig) return cls == kElongClass && cfg == kElongConfig;
  if (cfg == kGenericConfig) return true;  // the generic geometry takes any ROI up to 32 x 32
  const int wmax = (cls / 4 + 1) * 8, hmax = (cls % 4 + 1) * 8;
  const int cols = kConfigs[cfg].L * kConfigs[cfg].C;
  return cols >= wmax && kConfigs[cfg].R == hmax;
}

// Built-in choice per size class (lanes, cols, batched) for a class that runs alone
// (fit_spots_uniform, fit_spots_per_class), from timing every usable configuration on
// 131,072-spot samples at each class's bound size on a GB300 (the autotuner's choice): the
// batched kernels win except at 24 x 24, where the per-spot one-column kernel does; for
// widths 17..24 with more than 8 rows the one-column 32-lane kernels beat three columns per
// lane, whose larger LM step and register needs leave too few resident warps.
constexpr int kDefaultCfg[kNumClasses - 1][3] = {
    {8, 1, 1},  {8, 1, 1},  {8, 1, 1},  {8, 1, 1},    // width bound 8, rows 8..32
    {16, 1, 1}, {16, 1, 1}, {16, 1, 1}, {16, 1, 1},   // 16
    {8, 3, 1},  {32, 1, 1}, {32, 1, 0}, {32, 1, 1},   // 24
    {16, 2, 1}, {32, 1, 1}, {32, 1, 1}, {32, 1, 1}};  // 32

int default_config(int cls) {
  if (cls == kElongClass) return kElongConfig;
  return config_for(kDefaultCfg[cls][0], kDefaultCfg[cls][1], (cls % 4 + 1) * 8, kDefaultCfg[cls][2]);
}

void init_defaults() {
  for (int cls = 0; cls < kNumClasses; ++cls) g_class_cfg[cls] = (int8_t)default_config(cls);
}

struct ClassTable {
  int8_t cfg[kNumClasses];    // configuration per size class
  int8_t order[kNumClasses];  // processing order (largest first)
};

ClassTable current_table() {
  std::call_once(g_init_once, init_defaults);
  ClassTable t;
  std::lock_guard<std::mutex> lk(g_cfg_mutex);
  for (int c = 0; c < kNumClasses; ++c) t.cfg[c] = g_class_cfg[c];
  // largest classes first: the elongated class (up to 1024 pixels, the longest fits), then
  // by pixel bound (W bound * H bound), descending
  int k = 0;
  t.order[k++] = (int8_t)kElongClass;
  for (int area = 32 * 32; area > 0; area -= 64)
    for (int c = 0; c < kNumClasses; ++c)
      if (c != kElongClass && ((c / 4 + 1) * 8) * ((c % 4 + 1) * 8) == area) t.order[k++] = (int8_t)c;
  return t;
}

// Per device: SM count and, per configuration, resident blocks per SM (lazily filled).
struct DeviceInfo {
  int sms = 0;
  int blocks_per_sm[kNumConfigs] = {};
};
DeviceInfo g_dev_info[64];
std::mutex g_dev_mutex;

int set_cuda_error(cudaError_t e) {
  g_last_cuda_error = (int)e;
  return FS_ERR_CUDA;
}

// Grid size of configuration `which` on the current device: one wave of resident blocks.
int persistent_grid(int which, int *grid) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (dev < 0 || dev >= 64) return FS_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_dev_mutex);
  DeviceInfo &d = g_dev_info[dev];
  if (d.sms == 0) {
    if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return set_cuda_error(e);
  }
  int &slot = d.blocks_per_sm[which];
  if (slot == 0) {
    const void *fn = reinterpret_cast<const void *>(kKernels[which]);
    const size_t smem = config_smem_bytes(which);
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return set_cuda_error(e);
    int b = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kWarpsPerBlock * 32, smem)) !=
        cudaSuccess)
      return set_cuda_error(e);
    slot = b < 1 ? 1 : b;
  }
  *grid = d.sms * slot;
  return FS_OK;
}
int config_grid(int cfg, int *grid) { return persistent_grid(cfg, grid); }

int check_common(int dtype, int64_t n, int max_iter, double max_error, double min_delta,
                 double min_step) {
  // the work cursors are 32-bit and run past the count before every warp sees the end
  if (n < 0 || n > FS_MAX_SPOTS) return FS_ERR_SIZE;
  if (dtype != FS_U16 && dtype != FS_F32) return FS_ERR_DTYPE;
  if (max_iter < 1 || max_iter > 1000) return FS_ERR_MAX_ITER;
  if (!(max_error >= 0.0) || !isfinite(max_error) || !(min_delta >= 0.0) || !(min_delta < 1.0) ||
      !(min_step >= 0.0) || !isfinite(min_step))
    return FS_ERR_TOL;
  return FS_OK;
}

void fill_common(FitArgs &a, const void *images, int dtype, int64_t image_elems,
                 const float *init, int64_t n, int max_iter, double max_error, double min_delta,
                 double min_step, float *out_params, float *out_alpha, float *out_beta,
                 float *out_chi2, int32_t *out_state, int32_t *out_iters, int32_t *out_evals,
                 void *workspace) {
  a.images = images;
  a.dtype = dtype;
  a.image_elems = image_elems;
  a.offsets = nullptr;
  a.dims = nullptr;
  a.model = nullptr;
  a.init = init;
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
  a.uniform = 0;
  a.uw = a.uh = a.umodel = 0;
  int32_t *ws = static_cast<int32_t *>(workspace);
  a.counts = ws;
  a.starts = ws + kNumClasses;
  a.cursors = ws + 2 * kNumClasses;
  a.fill = ws + 3 * kNumClasses;
  a.perm = ws + 4 * kNumClasses;
}

// ------------------------------------------------------------------ built-in scratch
// Schedule scratch for fit_spots_noalloc: the same layout fit_spots keeps in the caller's
// workspace (class counts, starts, cursors, scatter cursors, then the spot permutation),
// sized for kStaticMaxSpots spots. It lives in every GPU that loads the library until the
// process exits. Host code must not pass g_static_ws itself to a kernel (on the host it
// names a stand-in, not device memory); its device address is looked up once per device.
constexpr int64_t kStaticMaxSpots = 1 << 20;
constexpr size_t kStaticWsBytes = kSchedHeaderBytes + (size_t)kStaticMaxSpots * sizeof(int32_t);
static __device__ __align__(256) int32_t g_static_ws[kStaticWsBytes / sizeof(int32_t)];

void *g_static_ws_addr[64];
std::mutex g_static_mutex;

// Device address of g_static_ws on the current device, looked up with cudaGetSymbolAddress.
// Outside stream capture the lookup is repeated on every call (it is cheap), so that a
// context that was reset and created again never gets a stale address; inside a capture the
// address of the last lookup is used (a capture region may not call it), so the first call on
// a device must come before any capture.
int static_workspace(cudaStream_t stream, void **ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (dev < 0 || dev >= 64) return FS_ERR_ARG;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(stream, &cap)) != cudaSuccess) return set_cuda_error(e);
  std::lock_guard<std::mutex> lk(g_static_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess || !p) return set_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    g_static_ws_addr[dev] = p;
  } else if (!g_static_ws_addr[dev]) {
    return set_cuda_error(cudaErrorStreamCaptureUnsupported);
  }
  *ptr = g_static_ws_addr[dev];
  return FS_OK;
}

// ------------------------------------------------------------------ host-buffer pipeline
// One chunk buffer in the device workspace of fit_spots_uniform_host: images, start values,
// the seven outputs and the schedule header, each 256-byte aligned.
struct ChunkLayout {
  size_t images, init, params, alpha, beta, chi2, state, iters, evals, sched, bytes;
};

ChunkLayout chunk_layout(int64_t chunk, int width, int height, int dtype) {
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t esz = dtype == FS_U16 ? 2 : 4, c = (size_t)chunk;
  ChunkLayout l;
  size_t o = 0;
  l.images = o; o += up(c * width * height * esz);
  l.init = o; o += up(c * 16);
  l.params = o; o += up(c * 16);
  l.alpha = o; o += up(c * 4);
  l.beta = o; o += up(c * 4);
  l.chi2 = o; o += up(c * 4);
  l.state = o; o += up(c * 4);
  l.iters = o; o += up(c * 4);
  l.evals = o; o += up(c * 4);
  l.sched = o; o += up(kSchedHeaderBytes);
  l.bytes = o;
  return l;
}

// Per device: the copy stream, a second fit stream and the events that order the two chunk
// buffers, created once (std::call_once) and kept for the life of the process.
struct HostPipe {
  cudaStream_t copy = nullptr;
  cudaStream_t fit2 = nullptr;                    // odd chunks are fitted here
  cudaEvent_t in_ready[2] = {nullptr, nullptr};   // chunk's inputs on the device
  cudaEvent_t fitted[2] = {nullptr, nullptr};     // chunk's fit done
  cudaEvent_t drained = nullptr;                  // last results copied back
  cudaError_t init_error = cudaSuccess;
  std::once_flag once;
  std::mutex mu;                                  // one caller enqueues at a time
};
HostPipe g_pipe[64];

int host_pipe(HostPipe **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (dev < 0 || dev >= 64) return FS_ERR_ARG;
  HostPipe &p = g_pipe[dev];
  std::call_once(p.once, [&p] {
    cudaError_t x = cudaStreamCreateWithFlags(&p.copy, cudaStreamNonBlocking);
    if (x == cudaSuccess) x = cudaStreamCreateWithFlags(&p.fit2, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && x == cudaSuccess; ++b) {
      x = cudaEventCreateWithFlags(&p.in_ready[b], cudaEventDisableTiming);
      if (x == cudaSuccess) x = cudaEventCreateWithFlags(&p.fitted[b], cudaEventDisableTiming);
    }
    if (x == cudaSuccess) x = cudaEventCreateWithFlags(&p.drained, cudaEventDisableTiming);
    p.init_error = x;
  });
  if (p.init_error != cudaSuccess) return set_cuda_error(p.init_error);
  *out = &p;
  return FS_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

size_t fit_spots_workspace(int64_t n) {
  if (n <= 0) return 0;
  return kSchedHeaderBytes + (size_t)n * sizeof(int32_t);
}

size_t fit_spots_uniform_workspace(void) { return kSchedHeaderBytes; }

const char *fit_spots_strerror(int code) {
  switch (code) {
    case FS_OK: return "ok";
    case FS_ERR_NULL: return "a required pointer is NULL";
    case FS_ERR_SIZE: return "spot count or image size out of range";
    case FS_ERR_DTYPE: return "unknown pixel type";
    case FS_ERR_MAX_ITER: return "max_iter outside [1, 1000]";
    case FS_ERR_TOL: return "tolerance negative, not finite, or min_delta >= 1";
    case FS_ERR_WORKSPACE: return "workspace too small or misaligned";
    case FS_ERR_CUDA: return "CUDA error";
    case FS_ERR_ARG: return "argument out of range";
    case FS_ERR_FULL: return "frame queue full, frame rejected";
    default: return "unknown error code";
  }
}

int fit_spots_last_cuda_error(void) { return g_last_cuda_error; }

int fit_spots_num_classes(void) { return kNumClasses; }
int fit_spots_num_configs(void) { return kNumConfigs; }

int fit_spots_config_info(int config, int *lanes, int *cols, int *rows) {
  if (config < 0 || config >= kNumConfigs) return FS_ERR_ARG;
  if (lanes) *lanes = kConfigs[config].L;
  if (cols) *cols = kConfigs[config].C;
  if (rows) *rows = kConfigs[config].R;
  return FS_OK;
}

int fit_spots_default_config(int size_class) {
  if (size_class < 0 || size_class >= kNumClasses) return FS_ERR_ARG;
  return default_config(size_class);
}

int fit_spots_config_batched(int config) {
  if (config < 0 || config >= kNumConfigs) return FS_ERR_ARG;
  return kConfigs[config].batched;
}

int fit_spots_config_generic(int config) {
  if (config < 0 || config >= kNumConfigs) return FS_ERR_ARG;
  return kConfigs[config].generic;
}

int fit_spots_config_fits(int size_class, int config) {
  return config_fits(config, size_class) ? 1 : 0;
}

int fit_spots_get_config(int size_class) {
  if (size_class < 0 || size_class >= kNumClasses) return FS_ERR_ARG;
  std::call_once(g_init_once, init_defaults);
  std::lock_guard<std::mutex> lk(g_cfg_mutex);
  return g_class_cfg[size_class];
}

int fit_spots_set_config(int size_class, int config) {
  if (!config_fits(config, size_class)) return FS_ERR_ARG;
  std::call_once(g_init_once, init_defaults);
  std::lock_guard<std::mutex> lk(g_cfg_mutex);
  g_class_cfg[size_class] = (int8_t)config;
  return FS_OK;
}

}  // extern "C"

namespace {
// fit_spots and fit_spots_per_class: the prepass, then either one launch of the generic
// configuration's kernel for all size classes, or one persistent launch per size class with
// the configuration the table assigns to it.
int fit_spots_impl(const void *images, int dtype, int64_t image_elems, const int64_t *offsets,
                   const int32_t *roi_dims, const float *init_params, const uint8_t *model,
                   int64_t n, int max_iter, double max_error, double min_delta, double min_step,
                   float *out_params, float *out_alpha, float *out_beta, float *out_chi2,
                   int32_t *out_state, int32_t *out_iters, int32_t *out_evals, void *workspace,
                   size_t ws_bytes, void *stream, bool per_class) {
  int rc = check_common(dtype, n, max_iter, max_error, min_delta, min_step);
  if (rc) return rc;
  if (image_elems < 0) return FS_ERR_SIZE;
  if (n == 0) return FS_OK;
  if (!images || !offsets || !roi_dims || !init_params || !model || !out_params || !out_alpha ||
      !out_beta || !out_chi2 || !out_state || !out_iters || !workspace)
    return FS_ERR_NULL;
  if (ws_bytes < fit_spots_workspace(n) || (reinterpret_cast<uintptr_t>(workspace) & 15))
    return FS_ERR_WORKSPACE;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FitArgs a;
  fill_common(a, images, dtype, image_elems, init_params, n, max_iter, max_error, min_delta,
              min_step, out_params, out_alpha, out_beta, out_chi2, out_state, out_iters, out_evals,
              workspace);
  a.offsets = offsets;
  a.dims = roi_dims;
  a.model = model;

  cudaError_t e = cudaMemsetAsync(workspace, 0, kSchedHeaderBytes, st);
  if (e != cudaSuccess) return set_cuda_error(e);
  const int pblocks = (int)((n + kPrepassChunk - 1) / kPrepassChunk);
  classify_count_kernel<<<pblocks, kPrepassThreads, 0, st>>>(a);
  classify_scan_kernel<<<1, 32, 0, st>>>(a);
  classify_scatter_kernel<<<pblocks, kPrepassThreads, 0, st>>>(a);
  if (!per_class) {
    // every size class of W, H <= 32, largest first, in one persistent launch of the generic
    // configuration; then the elongated class (a launch that finds no work if it is empty)
    const ClassTable ct = current_table();
    ClassList cl;
    cl.count = 0;
    for (int oi = 0; oi < kNumClasses; ++oi)
      if (ct.order[oi] != kElongClass) cl.cls[cl.count++] = ct.order[oi];
    int grid = 0;
    if ((rc = persistent_grid(kGenericConfig, &grid))) return rc;
    kKernels[kGenericConfig]<<<grid, kWarpsPerBlock * 32, config_smem_bytes(kGenericConfig), st>>>(
        a, cl);
    ClassList ce;
    ce.count = 1;
    ce.cls[0] = (int8_t)kElongClass;
    if ((rc = persistent_grid(kElongConfig, &grid))) return rc;
    kKernels[kElongConfig]<<<grid, kWarpsPerBlock * 32, config_smem_bytes(kElongConfig), st>>>(
        a, ce);
  } else {
    // one persistent launch per size class, each with the configuration the table assigns
    const ClassTable ct = current_table();
    for (int oi = 0; oi < kNumClasses; ++oi) {
      const int cls = ct.order[oi], cfg = ct.cfg[cls];
      if (cfg < 0 || cfg >= kNumConfigs) continue;
      ClassList cl;
      cl.count = 1;
      cl.cls[0] = (int8_t)cls;
      int grid = 0;
      if ((rc = persistent_grid(cfg, &grid))) return rc;
      kKernels[cfg]<<<grid, kWarpsPerBlock * 32, config_smem_bytes(cfg), st>>>(a, cl);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_cuda_error(e);
  return FS_OK;
}
}  // namespace

extern "C" {

int fit_spots(const void *images, int dtype, int64_t image_elems, const int64_t *offsets,
              const int32_t *roi_dims, const float *init_params, const uint8_t *model, int64_t n,
              int max_iter, double max_error, double min_delta, double min_step,
              float *out_params, float *out_alpha, float *out_beta, float *out_chi2,
              int32_t *out_state, int32_t *out_iters, int32_t *out_evals, void *workspace,
              size_t ws_bytes, void *stream) {
  return fit_spots_impl(images, dtype, image_elems, offsets, roi_dims, init_params, model, n,
                        max_iter, max_error, min_delta, min_step, out_params, out_alpha,
                        out_beta, out_chi2, out_state, out_iters, out_evals, workspace, ws_bytes,
                        stream, false);
}

int fit_spots_per_class(const void *images, int dtype, int64_t image_elems,
                        const int64_t *offsets, const int32_t *roi_dims,
                        const float *init_params, const uint8_t *model, int64_t n, int max_iter,
                        double max_error, double min_delta, double min_step, float *out_params,
                        float *out_alpha, float *out_beta, float *out_chi2, int32_t *out_state,
                        int32_t *out_iters, int32_t *out_evals, void *workspace,
                        size_t ws_bytes, void *stream) {
  return fit_spots_impl(images, dtype, image_elems, offsets, roi_dims, init_params, model, n,
                        max_iter, max_error, min_delta, min_step, out_params, out_alpha,
                        out_beta, out_chi2, out_state, out_iters, out_evals, workspace, ws_bytes,
                        stream, true);
}

int fit_spots_uniform(const void *images, int dtype, int width, int height, int model_id,
                      const float *init_params, int64_t n, int max_iter, double max_error,
                      double min_delta, double min_step, float *out_params, float *out_alpha,
                      float *out_beta, float *out_chi2, int32_t *out_state, int32_t *out_iters,
                      int32_t *out_evals, void *workspace, size_t ws_bytes, void *stream) {
  int rc = check_common(dtype, n, max_iter, max_error, min_delta, min_step);
  if (rc) return rc;
  const int P = model_id == FS_MODEL_ISO ? 3 : 4;
  if ((model_id != FS_MODEL_ISO && model_id != FS_MODEL_ELLIPTIC) || !roi_ok(width, height, P))
    return FS_ERR_ARG;
  if (n == 0) return FS_OK;
  if (!images || !init_params || !out_params || !out_alpha || !out_beta || !out_chi2 ||
      !out_state || !out_iters || !workspace)
    return FS_ERR_NULL;
  if (ws_bytes < fit_spots_uniform_workspace() || (reinterpret_cast<uintptr_t>(workspace) & 15))
    return FS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FitArgs a;
  fill_common(a, images, dtype, n * width * height, init_params, n, max_iter, max_error,
              min_delta, min_step, out_params, out_alpha, out_beta, out_chi2, out_state,
              out_iters, out_evals, workspace);
  a.uniform = 1;
  a.uw = width;
  a.uh = height;
  a.umodel = model_id;
  a.perm = nullptr;
  const int cls = size_class(width, height);
  const ClassTable ct = current_table();
  const int cfg = ct.cfg[cls];
  ClassList cl;
  cl.count = 1;
  cl.cls[0] = (int8_t)cls;
  int grid = 0;
  rc = config_grid(cfg, &grid);
  if (rc) return rc;
  cudaError_t e = cudaMemsetAsync(workspace, 0, kSchedHeaderBytes, st);
  if (e != cudaSuccess) return set_cuda_error(e);
  kKernels[cfg]<<<grid, kWarpsPerBlock * 32, config_smem_bytes(cfg), st>>>(a, cl);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_cuda_error(e);
  return FS_OK;
}

size_t fit_spots_uniform_host_workspace(int64_t chunk, int width, int height, int dtype) {
  if (chunk < 1 || !roi_ok(width, height, 0) || (dtype != FS_U16 && dtype != FS_F32)) return 0;
  return 2 * chunk_layout(chunk, width, height, dtype).bytes;
}

int fit_spots_uniform_host(const void *images, int dtype, int width, int height, int model_id,
                           const float *init_params, int64_t n, int max_iter, double max_error,
                           double min_delta, double min_step, float *out_params,
                           float *out_alpha, float *out_beta, float *out_chi2,
                           int32_t *out_state, int32_t *out_iters, int32_t *out_evals,
                           int64_t chunk, void *workspace, size_t ws_bytes, void *stream) {
  int rc = check_common(dtype, n, max_iter, max_error, min_delta, min_step);
  if (rc) return rc;
  const int P = model_id == FS_MODEL_ISO ? 3 : 4;
  if ((model_id != FS_MODEL_ISO && model_id != FS_MODEL_ELLIPTIC) || !roi_ok(width, height, P) ||
      chunk < 1 || chunk > INT32_MAX)
    return FS_ERR_ARG;
  if (n == 0) return FS_OK;
  if (!images || !init_params || !out_params || !out_alpha || !out_beta || !out_chi2 ||
      !out_state || !out_iters || !workspace)
    return FS_ERR_NULL;
  if (chunk > n) chunk = n;
  const ChunkLayout l = chunk_layout(chunk, width, height, dtype);
  if (ws_bytes < 2 * l.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return FS_ERR_WORKSPACE;
  HostPipe *pp = nullptr;
  if ((rc = host_pipe(&pp))) return rc;
  std::lock_guard<std::mutex> lk(pp->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream), cp = pp->copy;
  const size_t esz = dtype == FS_U16 ? 2 : 4, px = (size_t)width * height;
  const int64_t nchunks = (n + chunk - 1) / chunk;
  char *ws = static_cast<char *>(workspace);
  cudaError_t e = cudaSuccess;
  // the copy stream and the second fit stream start after whatever the caller queued on
  // `stream` before this call
  if ((e = cudaEventRecord(pp->drained, st)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(cp, pp->drained, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(pp->fit2, pp->drained, 0)) != cudaSuccess)
    return set_cuda_error(e);
  auto upload = [&](int64_t k) -> cudaError_t {
    char *b = ws + (k & 1) * l.bytes;
    const int64_t s0 = k * chunk, m = std::min<int64_t>(chunk, n - s0);
    cudaError_t x = cudaMemcpyAsync(b + l.images, static_cast<const char *>(images) + s0 * px * esz,
                                    m * px * esz, cudaMemcpyHostToDevice, cp);
    if (x == cudaSuccess)
      x = cudaMemcpyAsync(b + l.init, init_params + 4 * s0, m * 16, cudaMemcpyHostToDevice, cp);
    if (x == cudaSuccess) x = cudaEventRecord(pp->in_ready[k & 1], cp);
    return x;
  };
  if ((e = upload(0)) != cudaSuccess) return set_cuda_error(e);
  for (int64_t k = 0; k < nchunks; ++k) {
    // chunk k+1 goes up while chunk k is fitted (its buffer was drained, in copy-stream
    // order, by chunk k-1's download). Even chunks are fitted on `stream`, odd ones on the
    // second fit stream, so that chunk k+1's blocks take the SMs that chunk k's last fits
    // leave idle at the end of its persistent launch.
    if (k + 1 < nchunks && (e = upload(k + 1)) != cudaSuccess) return set_cuda_error(e);
    char *b = ws + (k & 1) * l.bytes;
    const int64_t s0 = k * chunk, m = std::min<int64_t>(chunk, n - s0);
    cudaStream_t fs = (k & 1) ? pp->fit2 : st;
    if ((e = cudaStreamWaitEvent(fs, pp->in_ready[k & 1], 0)) != cudaSuccess)
      return set_cuda_error(e);
    rc = fit_spots_uniform(b + l.images, dtype, width, height, model_id,
                           reinterpret_cast<const float *>(b + l.init), m, max_iter, max_error,
                           min_delta, min_step, reinterpret_cast<float *>(b + l.params),
                           reinterpret_cast<float *>(b + l.alpha),
                           reinterpret_cast<float *>(b + l.beta),
                           reinterpret_cast<float *>(b + l.chi2),
                           reinterpret_cast<int32_t *>(b + l.state),
                           reinterpret_cast<int32_t *>(b + l.iters),
                           out_evals ? reinterpret_cast<int32_t *>(b + l.evals) : nullptr,
                           b + l.sched, kSchedHeaderBytes, fs);
    if (rc) return rc;
    if ((e = cudaEventRecord(pp->fitted[k & 1], fs)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(cp, pp->fitted[k & 1], 0)) != cudaSuccess)
      return set_cuda_error(e);
    struct { void *dst; size_t off, sz; } outs[7] = {
        {out_params + 4 * s0, l.params, 16}, {out_alpha + s0, l.alpha, 4},
        {out_beta + s0, l.beta, 4},          {out_chi2 + s0, l.chi2, 4},
        {out_state + s0, l.state, 4},        {out_iters + s0, l.iters, 4},
        {out_evals ? out_evals + s0 : nullptr, l.evals, 4}};
    for (auto &o : outs)
      if (o.dst && (e = cudaMemcpyAsync(o.dst, b + o.off, m * o.sz, cudaMemcpyDeviceToHost, cp)) !=
                       cudaSuccess)
        return set_cuda_error(e);
  }
  // `stream` completes only after the last results are on the host (every download waited
  // for its chunk's fit, so this covers the second fit stream too)
  if ((e = cudaEventRecord(pp->drained, cp)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(st, pp->drained, 0)) != cudaSuccess)
    return set_cuda_error(e);
  return FS_OK;
}

int64_t fit_spots_noalloc_max_spots(void) { return kStaticMaxSpots; }

int fit_spots_noalloc(const void *images, int dtype, int64_t image_elems, const int64_t *offsets,
                      const int32_t *roi_dims, const float *init_params, const uint8_t *model,
                      int64_t n, int max_iter, double max_error, double min_delta,
                      double min_step, float *out_params, float *out_alpha, float *out_beta,
                      float *out_chi2, int32_t *out_state, int32_t *out_iters, int32_t *out_evals,
                      void *stream) {
  int rc = check_common(dtype, n, max_iter, max_error, min_delta, min_step);
  if (rc) return rc;
  if (n > kStaticMaxSpots) return FS_ERR_SIZE;
  if (n == 0) return FS_OK;
  void *ws = nullptr;
  rc = static_workspace(static_cast<cudaStream_t>(stream), &ws);
  if (rc) return rc;
  // fit_spots clears the schedule header on the stream before use; the permutation is
  // rewritten in full by the prepass, so nothing from an earlier call leaks through.
  return fit_spots(images, dtype, image_elems, offsets, roi_dims, init_params, model, n,
                   max_iter, max_error, min_delta, min_step, out_params, out_alpha, out_beta,
                   out_chi2, out_state, out_iters, out_evals, ws, kStaticWsBytes, stream);
}

}  // extern "C"
