// backward.cu -- implicit-function-theorem gradient of the spot fits (sm_103a).
//
// At a minimum of chi^2 (Eq. 2) over the full vector q = (p, alpha, beta) the gradient
// -sum_i r_i K_i vanishes, K_i = dh_i/dq = (alpha df_i/dp, f_i, 1), r = g - h. Its
// derivative in g_i gives dq/dg_i = M^-1 K_i with
//   M = sum_i K_i K_i^T - sum_i r_i d^2 h_i/dq^2,
// d^2 h/dp^2 = alpha d^2 f/dp^2 and d^2 h/dp dalpha = df/dp (Eq. 10 and its derivatives,
// Eq. 11, differentiated once more). For an upstream gradient u of the outputs the
// vector-Jacobian product is grad_g_i = (M^-1 u) . K_i, plus u_chi * 2 r_i / (N - P - 2)
// for the normalised chi^2 (its g-derivative at the minimum). The start parameters do
// not move the minimum, so their gradient is zero.
//
// Every sum that builds M separates (f = e_x e_y, and the derivatives are e_x e_y times
// polynomials of degree <= 4 in dx, dy): the pixel sums are the 13 bilinear forms
// G_ab = sum g' e_x dx^a e_y dy^b and the rest are products of 1-D moments
// E_m = sum_x e_x dx^m, P_m = sum_x e_x^2 dx^m (F_m, Q_m over y). Pixel values enter as
// g' = g - rint(beta), which keeps the sums free of the background's magnitude.
//
// Mapping: a warp takes a group of 32 consecutive spots in three phases.
//   A (warp per spot, each spot in turn): row-weighted column sums c_b(x) =
//     sum_y g' e_y dy^b (5 FMA per pixel), then G_ab = sum_x e_x dx^a c_b(x) reduced
//     across the columns into a per-group table.
//   S (lane per spot): the 1-D moments, M, and the Jacobi-scaled 6x6 solve by Gaussian
//     elimination with partial pivoting, unrolled in registers.
//   B (warp per spot): grad_g = e_x e_y (alpha (A(x) + B(y)) + v_alpha) + v_beta
//     + u_chi2 term, A and B the 1-D parts of v . K; the pixels come back from L2.
// The next group's pixels are prefetched into L2 while a group runs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fitspots.h"

namespace {

constexpr int kBwdThreads = 128;
constexpr int kBwdWarps = kBwdThreads / 32;
constexpr int kGroup = 16;   // spots per warp group: lane j and lane j + 16 serve spot j in phase S
constexpr int kAhead = 3;    // spots prefetched into L2 ahead of phase A
constexpr int kNG = 13;      // bilinear data sums G_ab
constexpr int kGStride = kGroup + 1;
constexpr int kChunk = 8;    // pixel rows a lane loads before it computes on them
constexpr int kRec = 20;     // per-spot record (floats)
// Pixel passes take one spot per warp (32 lanes) or, when two consecutive spots are both at
// most 16 wide, one spot per half-warp. Reduction rows: [13][36] for one spot, [2][13][20]
// for a pair (stride chosen so a quarter-warp's float4 rows fall on distinct banks).
constexpr int kRedStride1 = 36, kRedStride2 = 20;
constexpr int kRedFloats = 2 * kNG * kRedStride2 > kNG * kRedStride1 ? 2 * kNG * kRedStride2
                                                                     : kNG * kRedStride1;
// per warp: phase A row tables [64] float4 + [64] float and the reduction rows, which phase B
// reuses for its row table [64] float2; group table [kNG][kGStride]; spot records
// [kGroup][kRec]; next-group pixel ranges [kGroup] int4
constexpr int kPassFloats = 64 * 4 + 64 + kRedFloats;
constexpr int kGTabFloats = (kNG * kGStride + 3) / 4 * 4;
constexpr int kBwdWarpFloats = kPassFloats + kGTabFloats + kGroup * kRec + kGroup * 4;
static_assert(kPassFloats >= 64 * 2, "phase B row table");

struct BwdArgs {
  const void *images;
  int dtype;
  int64_t image_elems;
  const int64_t *offsets;
  const int32_t *dims;
  const uint8_t *model;
  int32_t n;
  const float *params, *alpha, *beta;
  const int32_t *state;
  const float *gp, *ga, *gb, *gc;  // upstream gradients (any may be null = 0)
  float *grad;
};

// L2 policies: a group's pixels are read in phase A and again in phase B; phase A and the
// prefetch mark them evict-last, phase B's second read and the gradient stores evict-first,
// so that the write stream does not push out pixels still waiting for phase B.
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float ldpix(const float *p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ldpix(const unsigned short *p, uint64_t pol) {
  unsigned short v;
  asm("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
  return (float)v;
}
__device__ __forceinline__ void stgrad(float *q, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(q), "f"(v), "l"(pol) : "memory");
}

// bilinear data sums G_ab (slot: (a, b))
enum : int { G00 = 0, G10, G01, G20, G02, G11, G30, G03, G12, G21, G40, G22, G04 };

// Column C of Gaussian elimination with partial pivoting on a 6x6 system; the row swap
// is a select per element so that M and v stay in registers.
template <int C>
__device__ __forceinline__ void elim_step(float (&M)[6][6], float (&v)[6], bool &ok) {
  int piv = C;
  float best = fabsf(M[C][C]);
#pragma unroll
  for (int r = C + 1; r < 6; ++r)
    if (fabsf(M[r][C]) > best) {
      best = fabsf(M[r][C]);
      piv = r;
    }
  ok = ok && best > 1e-30f;
#pragma unroll
  for (int r = C + 1; r < 6; ++r) {
    const bool sw = piv == r;
#pragma unroll
    for (int k = C; k < 6; ++k) {
      const float t = M[C][k];
      M[C][k] = sw ? M[r][k] : t;
      M[r][k] = sw ? t : M[r][k];
    }
    const float t = v[C];
    v[C] = sw ? v[r] : t;
    v[r] = sw ? t : v[r];
  }
  const float inv = 1.f / M[C][C];
#pragma unroll
  for (int r = C + 1; r < 6; ++r) {
    const float f = M[r][C] * inv;
#pragma unroll
    for (int k = C; k < 6; ++k) M[r][k] -= f * M[C][k];
    v[r] -= f * v[C];
  }
}

template <int R>
__device__ __forceinline__ void back_step(const float (&M)[6][6], float (&v)[6]) {
  float t = v[R];
#pragma unroll
  for (int k = R + 1; k < 6; ++k) t -= M[R][k] * v[k];
  v[R] = t / M[R][R];
}

// Prefetch into L2 the pixel range [off, off + npx) of a spot with one bulk prefetch, the
// range widened to 16-byte boundaries (which stay inside the pages the range touches).
template <typename T>
__device__ __forceinline__ void prefetch_range(const T *img, int64_t off, int npx, uint64_t pol) {
  if (npx <= 0) return;
  const uintptr_t lo = reinterpret_cast<uintptr_t>(img + off) & ~uintptr_t(15);
  const uintptr_t hi = (reinterpret_cast<uintptr_t>(img + off + npx) + 15) & ~uintptr_t(15);
  asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(lo),
               "r"((uint32_t)(hi - lo)), "l"(pol)
               : "memory");
}

// Phase A rows of one lane: c_b += g' e_y dy^b over kChunk rows starting at p (pixels) and
// row r0 of the row tables, rows `step` pixels (kStep if nonzero) and `rs` table rows apart;
// with kPred only the first `nleft` rows count.
template <typename T, bool kPred, int kStep>
__device__ __forceinline__ void rows_a(const T *p, int step, const float4 *t4, const float *t1,
                                       int rs, int nleft, float sh, uint64_t pol,
                                       float (&c)[5]) {
  const int st = kStep ? kStep : step;
  float gv[kChunk];
#pragma unroll
  for (int u = 0; u < kChunk; ++u)
    gv[u] = !kPred || u < nleft ? ldpix(p + u * st, pol) - sh : 0.f;
#pragma unroll
  for (int u = 0; u < kChunk; ++u) {
    const int r = (kPred ? min(u, max(nleft - 1, 0)) : u) * rs;
    const float4 r4 = t4[r];
    const float r5 = t1[r];
    c[0] = fmaf(gv[u], r4.x, c[0]);
    c[1] = fmaf(gv[u], r4.y, c[1]);
    c[2] = fmaf(gv[u], r4.z, c[2]);
    c[3] = fmaf(gv[u], r4.w, c[3]);
    c[4] = fmaf(gv[u], r5, c[4]);
  }
}

// Phase B rows of one lane: grad = e_x e_y (K1 + alpha B(y)) + u_chi g + K2 with the row
// table rb = (e_y, alpha B(y)); same row addressing as rows_a.
// kChi: the upstream gradient of the normalised chi^2 is given, so the gradient has a term in
// the pixels themselves and they are read again; without it phase B reads no pixels.
template <typename T, bool kPred, int kStep, bool kChi>
__device__ __forceinline__ void rows_b(const T *p, float *q, int step, const float2 *rb, int rs,
                                       int nleft, float ex, float K1, float cc, float K2,
                                       uint64_t pol) {
  const int st = kStep ? kStep : step;
  float gv[kChunk];
#pragma unroll
  for (int u = 0; u < kChunk; ++u)
    gv[u] = kChi && (!kPred || u < nleft) ? ldpix(p + u * st, pol) : 0.f;
#pragma unroll
  for (int u = 0; u < kChunk; ++u)
    if (!kPred || u < nleft) {
      const float2 eb = rb[u * rs];
      stgrad(q + u * st, fmaf(ex * eb.x, K1 + eb.y, kChi ? fmaf(cc, gv[u], K2) : K2), pol);
    }
}

// The rows of one lane in a pixel pass: a warp-uniform fast path when every lane has the same
// number of rows a full row step apart (step = lanes per spot), else per-lane predication.
struct LaneRows {
  int nv;      // this lane's rows
  int nmax;    // most rows of any lane of the warp
  bool fast;   // every lane: nv == nmax, step == lanes per spot
};

// The spot's record: geometry and profile (phase A), solution coefficients (phase B).
struct SpotRec {
  float x0, y0, ivx, ivy;
  float sh, rW, al, bp;
  float vx, vy, vsx, vsy;   // v . K coefficients of the 1-D parts (already times 1/s^2, 1/s^3)
  float va, vb, cchi, pad;
  int off_lo, off_hi;
  int whr;   // W | H << 8 | (32 / W) << 16 | (16 / W) << 24: rows per step for 32 and 16 lanes
  int nrow;  // row steps for 32 lanes | for 16 lanes << 8 | full for 32 << 16 | full for 16 << 17
};
static_assert(sizeof(SpotRec) == kRec * 4, "record size");

// M for q = (x0, y0, sx, sy, alpha, beta) from the 13 data sums and the 1-D moments, the
// isotropic fold, and the Jacobi-scaled solve M v = u. Returns false for a singular or
// non-finite system.
__device__ __forceinline__ bool solve_spot(const float (&G)[kNG], const float (&Ex)[5],
                                           const float (&Px)[5], const float (&Fy)[5],
                                           const float (&Qy)[5], float ivx, float ivy, float cx,
                                           float cy, float al, float bp, int N, bool iso,
                                           float (&v)[6]) {
  const float E0 = Ex[0], E1 = Ex[1], E2 = Ex[2], E3 = Ex[3], E4 = Ex[4];
  const float P0 = Px[0], P1 = Px[1], P2 = Px[2], P3 = Px[3], P4 = Px[4];
  const float F0 = Fy[0], F1 = Fy[1], F2 = Fy[2], F3 = Fy[3], F4 = Fy[4];
  const float Q0 = Qy[0], Q1 = Qy[1], Q2 = Qy[2], Q3 = Qy[3], Q4 = Qy[4];
  // sum d_j d_k (= sum f^2 phi_j phi_k), sum f d_j, sum d_j, sum g' d_j, sum g' h_jk,
  // sum f h_jk, sum h_jk with phi = (ivx dx, ivy dy, cx dx^2, cy dy^2)
  float DD[10], FD[4], SD[4], GD[4], GH[10], FH[10], SH[10];
  DD[0] = ivx * ivx * P2 * Q0;
  DD[1] = ivx * ivy * P1 * Q1;
  DD[2] = ivx * cx * P3 * Q0;
  DD[3] = ivx * cy * P1 * Q2;
  DD[4] = ivy * ivy * P0 * Q2;
  DD[5] = ivy * cx * P2 * Q1;
  DD[6] = ivy * cy * P0 * Q3;
  DD[7] = cx * cx * P4 * Q0;
  DD[8] = cx * cy * P2 * Q2;
  DD[9] = cy * cy * P0 * Q4;
  FD[0] = ivx * P1 * Q0;
  FD[1] = ivy * P0 * Q1;
  FD[2] = cx * P2 * Q0;
  FD[3] = cy * P0 * Q2;
  SD[0] = ivx * E1 * F0;
  SD[1] = ivy * E0 * F1;
  SD[2] = cx * E2 * F0;
  SD[3] = cy * E0 * F2;
  GD[0] = ivx * G[G10];
  GD[1] = ivy * G[G01];
  GD[2] = cx * G[G20];
  GD[3] = cy * G[G02];
  GH[0] = ivx * ivx * G[G20] - ivx * G[G00];
  FH[0] = ivx * ivx * P2 * Q0 - ivx * P0 * Q0;
  SH[0] = ivx * ivx * E2 * F0 - ivx * E0 * F0;
  GH[1] = ivx * ivy * G[G11];
  FH[1] = ivx * ivy * P1 * Q1;
  SH[1] = ivx * ivy * E1 * F1;
  GH[2] = ivx * cx * G[G30] - 2.f * cx * G[G10];
  FH[2] = ivx * cx * P3 * Q0 - 2.f * cx * P1 * Q0;
  SH[2] = ivx * cx * E3 * F0 - 2.f * cx * E1 * F0;
  GH[3] = ivx * cy * G[G12];
  FH[3] = ivx * cy * P1 * Q2;
  SH[3] = ivx * cy * E1 * F2;
  GH[4] = ivy * ivy * G[G02] - ivy * G[G00];
  FH[4] = ivy * ivy * P0 * Q2 - ivy * P0 * Q0;
  SH[4] = ivy * ivy * E0 * F2 - ivy * E0 * F0;
  GH[5] = ivy * cx * G[G21];
  FH[5] = ivy * cx * P2 * Q1;
  SH[5] = ivy * cx * E2 * F1;
  GH[6] = ivy * cy * G[G03] - 2.f * cy * G[G01];
  FH[6] = ivy * cy * P0 * Q3 - 2.f * cy * P0 * Q1;
  SH[6] = ivy * cy * E0 * F3 - 2.f * cy * E0 * F1;
  GH[7] = cx * cx * G[G40] - 3.f * ivx * ivx * G[G20];
  FH[7] = cx * cx * P4 * Q0 - 3.f * ivx * ivx * P2 * Q0;
  SH[7] = cx * cx * E4 * F0 - 3.f * ivx * ivx * E2 * F0;
  GH[8] = cx * cy * G[G22];
  FH[8] = cx * cy * P2 * Q2;
  SH[8] = cx * cy * E2 * F2;
  GH[9] = cy * cy * G[G04] - 3.f * ivy * ivy * G[G02];
  FH[9] = cy * cy * P0 * Q4 - 3.f * ivy * ivy * P0 * Q2;
  SH[9] = cy * cy * E0 * F4 - 3.f * ivy * ivy * E0 * F2;
  float M[6][6];
  {
    int t = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = j; k < 4; ++k, ++t) {
        const float rh = GH[t] - al * FH[t] - bp * SH[t];  // sum r h_jk
        M[j][k] = M[k][j] = al * (al * DD[t] - rh);
      }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float rd = GD[j] - al * FD[j] - bp * SD[j];  // sum r d_j
      M[j][4] = M[4][j] = al * FD[j] - rd;
      M[j][5] = M[5][j] = al * SD[j];
    }
  }
  M[4][4] = P0 * Q0;
  M[4][5] = M[5][4] = E0 * F0;
  M[5][5] = (float)N;
  if (iso) {  // sigma_x = sigma_y = sigma: merge row/column 3 into 2, leave 3 as identity
#pragma unroll
    for (int k = 0; k < 6; ++k) M[2][k] += M[3][k];
#pragma unroll
    for (int k = 0; k < 6; ++k) M[k][2] += M[k][3];
    v[2] += v[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) M[3][k] = M[k][3] = 0.f;
    M[3][3] = 1.f;
    v[3] = 0.f;
  }
  // Jacobi scaling, then Gaussian elimination with partial pivoting
  bool ok = true;
  float sc[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    ok = ok && M[j][j] > 0.f;
    sc[j] = M[j][j] > 0.f ? rsqrtf(M[j][j]) : 1.f;
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) {
#pragma unroll
    for (int k = 0; k < 6; ++k) M[j][k] *= sc[j] * sc[k];
    v[j] *= sc[j];
  }
  elim_step<0>(M, v, ok);
  elim_step<1>(M, v, ok);
  elim_step<2>(M, v, ok);
  elim_step<3>(M, v, ok);
  elim_step<4>(M, v, ok);
  elim_step<5>(M, v, ok);
  back_step<5>(M, v);
  back_step<4>(M, v);
  back_step<3>(M, v);
  back_step<2>(M, v);
  back_step<1>(M, v);
  back_step<0>(M, v);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    v[j] *= sc[j];
    ok = ok && isfinite(v[j]);
  }
  return ok;
}

template <typename T, bool kChi>
__global__ void __launch_bounds__(kBwdThreads, 8) backward_kernel(BwdArgs a) {
  __shared__ float4 sm4[kBwdWarps * kBwdWarpFloats / 4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T *const img = static_cast<const T *>(a.images);
  const uint64_t keep = policy_evict_last(), drop = policy_evict_first();
  float *const wbase = reinterpret_cast<float *>(sm4) + warp * kBwdWarpFloats;
  float4 *const rowt4 = reinterpret_cast<float4 *>(wbase);                // [2][32]: e_y dy^0..3
  float *const rowt1 = wbase + 64 * 4;                                     // [2][32]: e_y dy^4
  float *const red = rowt1 + 64;                                           // reduction rows
  float2 *const rowb = reinterpret_cast<float2 *>(wbase);                  // phase B [2][32]
  float *const gtab = wbase + kPassFloats;                                 // [kNG][17]
  SpotRec *const rec = reinterpret_cast<SpotRec *>(gtab + kGTabFloats);    // [kGroup]
  int4 *const nxt = reinterpret_cast<int4 *>(rec + kGroup);  // next group: offset, pixels
  const int ngroups = (a.n + kGroup - 1) / kGroup;
  const int gstride = gridDim.x * kBwdWarps;
  const int jl = lane & (kGroup - 1);  // the group spot this lane serves in phases 0 and S
  const bool ylane = lane >= kGroup;    // phase S: the y moments of spot jl
  int g = blockIdx.x * kBwdWarps + warp;
  if (g < ngroups && lane < kAhead && g * kGroup + lane < a.n) {
    const int s = g * kGroup + lane;
    const int W = a.dims[2 * s], H = a.dims[2 * s + 1];
    const int64_t off = a.offsets[s];
    if (W >= 1 && H >= 1 && W <= 32 && H <= 32 && off >= 0 &&
        off + (int64_t)W * H <= a.image_elems)
      prefetch_range(img, off, W * H, keep);
  }
  for (; g < ngroups; g += gstride) {
    const int s0 = g * kGroup;
    const int ns = min(kGroup, a.n - s0);
    // ---- phase 0: lanes j and j + 16 read spot s0 + j; lanes 16.. also read the pixel range
    // of spot j of this warp's next group (for the prefetch)
    const int s = s0 + jl;
    const bool have = jl < ns;
    const int W = have ? a.dims[2 * s] : 0, H = have ? a.dims[2 * s + 1] : 0;
    const int m = have ? a.model[s] : -1;
    const int64_t off = have ? a.offsets[s] : 0;
    const bool iso = m == FS_MODEL_ISO;
    const int P = iso ? 3 : 4;
    const bool valid = have && (m == FS_MODEL_ISO || m == FS_MODEL_ELLIPTIC) && W >= 3 &&
                       H >= 3 && W <= 32 && H <= 32 && W * H > P + 2 && off >= 0 &&
                       off + (int64_t)W * H <= a.image_elems;
    const int st = valid ? a.state[s] : FS_STATE_INVALID_ROI;
    const bool conv = valid && (st == FS_STATE_MIN_DELTA || st == FS_STATE_MIN_STEP ||
                                st == FS_STATE_MAX_ERROR || st == FS_STATE_NO_DECREASE);
    float x0 = 0.f, y0 = 0.f, sx = 1.f, sy = 1.f, al = 0.f, be = 0.f;
    if (valid) {
      x0 = a.params[4 * s];
      y0 = a.params[4 * s + 1];
      sx = a.params[4 * s + 2];
      sy = iso ? sx : a.params[4 * s + 3];
      al = a.alpha[s];
      be = a.beta[s];
    }
    const float ivx = 1.f / (sx * sx), ivy = 1.f / (sy * sy);
    const float sh = rintf(be), bp = be - sh;
    // rows per step for 32 and for 16 lanes per spot; a layout is full when a row step covers
    // all its lanes and H is a multiple of it (every lane then has the same rows)
    const int rps = valid ? 32 / W : 1, rps2 = valid ? max(16 / W, 1) : 1;
    const bool full = valid && rps * W == 32 && H % rps == 0;
    const bool full2 = valid && W <= 16 && rps2 * W == 16 && H % rps2 == 0;
    if (!ylane) {
      SpotRec &r = rec[jl];
      *reinterpret_cast<float4 *>(&r.x0) = make_float4(x0, y0, ivx, ivy);
      *reinterpret_cast<float4 *>(&r.sh) = make_float4(sh, valid ? 1.f / (float)W : 1.f, al, bp);
      *reinterpret_cast<int4 *>(&r.off_lo) =
          make_int4((int)(off & 0xffffffff), (int)(off >> 32),
                    W | (H << 8) | (rps << 16) | (rps2 << 24),
                    valid ? ((H + rps - 1) / rps) | (((H + rps2 - 1) / rps2) << 8) |
                                ((int)full << 16) | ((int)full2 << 17)
                          : 0);
    } else {
      int4 rng = make_int4(0, 0, 0, 0);
      if (g + gstride < ngroups) {
        const int sn = (g + gstride) * kGroup + jl;
        if (sn < a.n) {
          const int Wn = a.dims[2 * sn], Hn = a.dims[2 * sn + 1];
          const int64_t on = a.offsets[sn];
          if (Wn >= 1 && Hn >= 1 && Wn <= 32 && Hn <= 32 && on >= 0 &&
              on + (int64_t)Wn * Hn <= a.image_elems)
            rng = make_int4((int)(on & 0xffffffff), (int)(on >> 32), Wn * Hn, 0);
        }
      }
      nxt[jl] = rng;
    }
    const unsigned conv_mask = __ballot_sync(0xffffffffu, conv) & 0xffffu;
    const unsigned valid_mask = __ballot_sync(0xffffffffu, valid) & 0xffffu;
    __syncwarp();

    // ---- phase A: G_ab of each converged spot into gtab[k][j]
    for (int j = 0; j < ns;) {
      if (lane < 2) {  // prefetch spot j + kAhead + lane (this group's, else the next group's)
        const int t = j + kAhead + lane;
        if (t < ns) {
          const int4 o = *reinterpret_cast<const int4 *>(&rec[t].off_lo);
          const int64_t ot = (int64_t)(((uint64_t)(uint32_t)o.y << 32) | (uint32_t)o.x);
          if ((valid_mask >> t) & 1u)
            prefetch_range(img, ot, (o.z & 0xff) * ((o.z >> 8) & 0xff), keep);
        } else if (t - kGroup >= 0 && t - kGroup < kGroup) {
          const int4 r4 = nxt[t - kGroup];
          prefetch_range(img, (int64_t)(((uint64_t)(uint32_t)r4.y << 32) | (uint32_t)r4.x), r4.z,
                         keep);
        }
      }
      if (!((conv_mask >> j) & 1u)) {
        ++j;
        continue;
      }
      const bool pair = j + 1 < ns && ((conv_mask >> (j + 1)) & 1u) &&
                        (rec[j].whr & 0xff) <= 16 && (rec[j + 1].whr & 0xff) <= 16;
      const int L = pair ? 16 : 32;
      const int h = pair ? lane >> 4 : 0;  // which spot of the step this lane serves
      const int ln = lane & (L - 1);       // lane within the spot
      const int js = j + h;
      const float4 ra = *reinterpret_cast<const float4 *>(&rec[js].x0);
      const float4 rb = *reinterpret_cast<const float4 *>(&rec[js].sh);
      const int4 rc = *reinterpret_cast<const int4 *>(&rec[js].off_lo);
      const float x0j = ra.x, y0j = ra.y, ivxj = ra.z, ivyj = ra.w, shj = rb.x, rWj = rb.y;
      const int Wj = rc.z & 0xff, Hj = (rc.z >> 8) & 0xff;
      const int rpsj = pair ? rc.z >> 24 : (rc.z >> 16) & 0xff;
      const int nrj = pair ? (rc.w >> 8) & 0xff : rc.w & 0xff;
      const bool fullj = (rc.w >> (pair ? 17 : 16)) & 1;
      const T *const pj = img + (int64_t)(((uint64_t)(uint32_t)rc.y << 32) | (uint32_t)rc.x);
      float4 *const t4 = rowt4 + h * 32;
      float *const t1 = rowt1 + h * 32;
      // row table: e_y dy^b, b = 0..4 (zero beyond the ROI)
      for (int r = ln; r < 32; r += L) {
        const float dy = (float)r - y0j;
        const float e = r < Hj ? __expf(-0.5f * dy * dy * ivyj) : 0.f;
        const float e1 = e * dy, e2 = e1 * dy, e3 = e2 * dy;
        t4[r] = make_float4(e, e1, e2, e3);
        t1[r] = e3 * dy;
      }
      __syncwarp();
      const int yo = (int)(((float)ln + 0.5f) * rWj);
      const int xl = ln - yo * Wj;
      const bool plane = yo < rpsj;
      // this lane's rows yo, yo + rps, ...: nv of them
      const int nv = plane && yo < Hj ? (int)(((float)(Hj - yo - 1) + 0.5f) / (float)rpsj) + 1 : 0;
      const int nmax = pair ? max(nrj, __shfl_xor_sync(0xffffffffu, nrj, 16)) : nrj;
      const bool fast = __all_sync(0xffffffffu, fullj && nrj == nmax);
      float c[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      {
        const int step = rpsj * Wj;
        const T *p = pj + (yo * Wj + xl);
        const float4 *r4 = t4 + yo;
        const float *r1 = t1 + yo;
        int t0 = 0;
        if (fast) {
          if (pair)
            for (; t0 + kChunk <= nmax; t0 += kChunk)
              rows_a<T, false, 16>(p + t0 * 16, 16, r4 + t0 * rpsj, r1 + t0 * rpsj, rpsj, 0, shj,
                                   keep, c);
          else
            for (; t0 + kChunk <= nmax; t0 += kChunk)
              rows_a<T, false, 32>(p + t0 * 32, 32, r4 + t0 * rpsj, r1 + t0 * rpsj, rpsj, 0, shj,
                                   keep, c);
        }
        for (; t0 < nmax; t0 += kChunk)
          rows_a<T, true, 0>(p + t0 * step, step, r4 + t0 * rpsj, r1 + t0 * rpsj, rpsj, nv - t0,
                             shj, keep, c);
      }
      // column x collects the partial sums of lanes x + t W, t < rps, of its own spot
      float c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3], c4 = c[4];
      const int rmax = pair ? max(rpsj, __shfl_xor_sync(0xffffffffu, rpsj, 16)) : rpsj;
      for (int t = 1; t < rmax; ++t) {
        const int d = t < rpsj ? t * Wj : 0;
        const float z0 = __shfl_down_sync(0xffffffffu, c[0], d, L);
        const float z1 = __shfl_down_sync(0xffffffffu, c[1], d, L);
        const float z2 = __shfl_down_sync(0xffffffffu, c[2], d, L);
        const float z3 = __shfl_down_sync(0xffffffffu, c[3], d, L);
        const float z4 = __shfl_down_sync(0xffffffffu, c[4], d, L);
        if (t < rpsj) {
          c0 += z0;
          c1 += z1;
          c2 += z2;
          c3 += z3;
          c4 += z4;
        }
      }
      {
        const int RS = pair ? kRedStride2 : kRedStride1;
        float *const rr = red + h * kNG * RS + ln;
        const float dx = (float)ln - x0j;
        const float p0 = ln < Wj ? __expf(-0.5f * dx * dx * ivxj) : 0.f;
        const float p1 = p0 * dx, p2 = p1 * dx, p3 = p2 * dx, p4 = p3 * dx;
        rr[G00 * RS] = p0 * c0;
        rr[G10 * RS] = p1 * c0;
        rr[G01 * RS] = p0 * c1;
        rr[G20 * RS] = p2 * c0;
        rr[G02 * RS] = p0 * c2;
        rr[G11 * RS] = p1 * c1;
        rr[G30 * RS] = p3 * c0;
        rr[G03 * RS] = p0 * c3;
        rr[G12 * RS] = p1 * c2;
        rr[G21 * RS] = p2 * c1;
        rr[G40 * RS] = p4 * c0;
        rr[G22 * RS] = p2 * c2;
        rr[G04 * RS] = p0 * c4;
        __syncwarp();
        if (lane < (pair ? 2 * kNG : kNG)) {
          const int hh = lane >= kNG, k = lane - hh * kNG;
          const float4 *r = reinterpret_cast<const float4 *>(red + (hh * kNG + k) * RS);
          const int nq = ((rec[j + hh].whr & 0xff) + 3) >> 2;
          float q0 = 0.f, q1 = 0.f;
          int i = 0;
          for (; i + 1 < nq; i += 2) {
            const float4 w0 = r[i], w1 = r[i + 1];
            q0 += (w0.x + w0.y) + (w0.z + w0.w);
            q1 += (w1.x + w1.y) + (w1.z + w1.w);
          }
          if (i < nq) {
            const float4 w0 = r[i];
            q0 += (w0.x + w0.y) + (w0.z + w0.w);
          }
          gtab[k * kGStride + j + hh] = q0 + q1;
        }
      }
      __syncwarp();
      j += pair ? 2 : 1;
    }

    // ---- phase S: lane j (x moments, the solve) and lane j + 16 (y moments) for spot j
    float vx = 0.f, vy = 0.f, vsx = 0.f, vsy = 0.f, va = 0.f, vb = 0.f, cchi = 0.f;
    bool ok = false;
    {
      const int nA = ylane ? H : W;
      const float cA = ylane ? y0 : x0, ivA = ylane ? ivy : ivx;
      float Ex[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, Px[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      if (conv)
        for (int x = 0; x < nA; ++x) {
          const float d = (float)x - cA;
          const float e = __expf(-0.5f * d * d * ivA), ee = e * e;
          const float d2 = d * d;
          Ex[0] += e;
          Ex[1] = fmaf(e, d, Ex[1]);
          Ex[2] = fmaf(e, d2, Ex[2]);
          Ex[3] = fmaf(e * d, d2, Ex[3]);
          Ex[4] = fmaf(e * d2, d2, Ex[4]);
          Px[0] += ee;
          Px[1] = fmaf(ee, d, Px[1]);
          Px[2] = fmaf(ee, d2, Px[2]);
          Px[3] = fmaf(ee * d, d2, Px[3]);
          Px[4] = fmaf(ee * d2, d2, Px[4]);
        }
      float Fy[5], Qy[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        Fy[k] = __shfl_down_sync(0xffffffffu, Ex[k], kGroup);
        Qy[k] = __shfl_down_sync(0xffffffffu, Px[k], kGroup);
      }
      if (conv && !ylane) {
        float G[kNG];
#pragma unroll
        for (int k = 0; k < kNG; ++k) G[k] = gtab[k * kGStride + jl];
        const float cx = ivx / sx, cy = ivy / sy;
        float v[6];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = a.gp ? a.gp[4 * s + k] : 0.f;
        v[4] = a.ga ? a.ga[s] : 0.f;
        v[5] = a.gb ? a.gb[s] : 0.f;
        const float uc = a.gc ? a.gc[s] : 0.f;
        ok = solve_spot(G, Ex, Px, Fy, Qy, ivx, ivy, cx, cy, al, bp, W * H, iso, v);
        // (vx, vy, vsx, vsy, va, vb) as coefficients of the 1-D parts; the isotropic sigma
        // moves both widths
        if (ok) {
          vx = v[0] * ivx;
          vy = v[1] * ivy;
          vsx = v[2] * cx;
          vsy = (iso ? v[2] : v[3]) * cy;
          va = v[4];
          vb = v[5];
          cchi = 2.f * uc / (float)(W * H - P - 2);
        }
      }
    }
    if (!ylane) {
      SpotRec &r = rec[jl];
      *reinterpret_cast<float4 *>(&r.vx) = make_float4(vx, vy, vsx, vsy);
      *reinterpret_cast<float4 *>(&r.va) = make_float4(va, vb, cchi, 0.f);
    }
    const unsigned ok_mask = __ballot_sync(0xffffffffu, ok) & 0xffffu;
    __syncwarp();

    // ---- phase B: grad_g = e_x e_y (alpha (A(x) + B(y)) + va) + vb + cchi (g' - alpha f - bp)
    for (int j = 0; j < ns;) {
      if (!((valid_mask >> j) & 1u)) {
        ++j;
        continue;
      }
      if (!((ok_mask >> j) & 1u)) {  // no gradient through fits that did not converge
        const int4 rc = *reinterpret_cast<const int4 *>(&rec[j].off_lo);
        const int Wj = rc.z & 0xff, Hj = (rc.z >> 8) & 0xff;
        float *const gj = a.grad + (int64_t)(((uint64_t)(uint32_t)rc.y << 32) | (uint32_t)rc.x);
        for (int i = lane; i < Wj * Hj; i += 32) stgrad(gj + i, 0.f, drop);
        ++j;
        continue;
      }
      const bool pair = j + 1 < ns && ((ok_mask >> (j + 1)) & 1u) &&
                        (rec[j].whr & 0xff) <= 16 && (rec[j + 1].whr & 0xff) <= 16;
      const int L = pair ? 16 : 32;
      const int h = pair ? lane >> 4 : 0;
      const int ln = lane & (L - 1);
      const int js = j + h;
      const int4 rc = *reinterpret_cast<const int4 *>(&rec[js].off_lo);
      const float4 rb = *reinterpret_cast<const float4 *>(&rec[js].sh);
      const float4 ra = *reinterpret_cast<const float4 *>(&rec[js].x0);
      const float4 rv = *reinterpret_cast<const float4 *>(&rec[js].vx);
      const float4 rw = *reinterpret_cast<const float4 *>(&rec[js].va);
      const int Wj = rc.z & 0xff, Hj = (rc.z >> 8) & 0xff;
      const int rpsj = pair ? rc.z >> 24 : (rc.z >> 16) & 0xff;
      const int nrj = pair ? (rc.w >> 8) & 0xff : rc.w & 0xff;
      const bool fullj = (rc.w >> (pair ? 17 : 16)) & 1;
      const int64_t offj = (int64_t)(((uint64_t)(uint32_t)rc.y << 32) | (uint32_t)rc.x);
      const T *const pj = img + offj;
      float *const gj = a.grad + offj;
      const float alj = rb.z, betaj = rb.x + rb.w;
      const float vaj = rw.x, vbj = rw.y, ccj = rw.z;
      // grad = f (alpha (A(x) + B(y)) + va) + vb + cchi (g - alpha f - beta)
      //      = e_x e_y (K1 + alpha B(y)) + cchi g + K2
      float2 *const tb = rowb + h * 32;
      for (int r = ln; r < 32; r += L) {
        const float dy = (float)r - ra.y;
        const float e = r < Hj ? __expf(-0.5f * dy * dy * ra.w) : 0.f;
        tb[r] = make_float2(e, alj * dy * fmaf(rv.w, dy, rv.y));
      }
      __syncwarp();
      const int yo = (int)(((float)ln + 0.5f) * rb.y);
      const int xl = ln - yo * Wj;
      const bool plane = yo < rpsj;
      const int nv = plane && yo < Hj ? (int)(((float)(Hj - yo - 1) + 0.5f) / (float)rpsj) + 1 : 0;
      const int nmax = pair ? max(nrj, __shfl_xor_sync(0xffffffffu, nrj, 16)) : nrj;
      const bool fast = __all_sync(0xffffffffu, fullj && nrj == nmax);
      const float dx = (float)xl - ra.x;
      const float ex = __expf(-0.5f * dx * dx * ra.z);
      const float K1 = fmaf(alj, dx * fmaf(rv.z, dx, rv.x), vaj) - ccj * alj;
      const float K2 = fmaf(-ccj, betaj, vbj);
      {
        const int step = rpsj * Wj;
        const T *p = pj + (yo * Wj + xl);
        float *q = gj + (yo * Wj + xl);
        const float2 *rt = tb + yo;
        int t0 = 0;
        if (fast) {
          if (pair)
            for (; t0 + kChunk <= nmax; t0 += kChunk)
              rows_b<T, false, 16, kChi>(p + t0 * 16, q + t0 * 16, 16, rt + t0 * rpsj, rpsj, 0, ex, K1,
                                   ccj, K2, drop);
          else
            for (; t0 + kChunk <= nmax; t0 += kChunk)
              rows_b<T, false, 32, kChi>(p + t0 * 32, q + t0 * 32, 32, rt + t0 * rpsj, rpsj, 0, ex, K1,
                                   ccj, K2, drop);
        }
        for (; t0 < nmax; t0 += kChunk)
          rows_b<T, true, 0, kChi>(p + t0 * step, q + t0 * step, step, rt + t0 * rpsj, rpsj, nv - t0,
                             ex, K1, ccj, K2, drop);
      }
      __syncwarp();
      j += pair ? 2 : 1;
    }
    __syncwarp();
  }
}

}  // namespace

extern "C" int fit_spots_backward(const void *images, int dtype, int64_t image_elems,
                                  const int64_t *offsets, const int32_t *roi_dims,
                                  const uint8_t *model, int64_t n, const float *params,
                                  const float *alpha, const float *beta, const int32_t *state,
                                  const float *grad_params, const float *grad_alpha,
                                  const float *grad_beta, const float *grad_chi2,
                                  float *grad_images, void *stream) {
  if (n < 0 || n > FS_MAX_SPOTS || image_elems < 0) return FS_ERR_SIZE;
  if (dtype != FS_U16 && dtype != FS_F32) return FS_ERR_DTYPE;
  if (n == 0) return FS_OK;
  if (!images || !offsets || !roi_dims || !model || !params || !alpha || !beta || !state ||
      !grad_images)
    return FS_ERR_NULL;
  BwdArgs a;
  a.images = images;
  a.dtype = dtype;
  a.image_elems = image_elems;
  a.offsets = offsets;
  a.dims = roi_dims;
  a.model = model;
  a.n = (int32_t)n;
  a.params = params;
  a.alpha = alpha;
  a.beta = beta;
  a.state = state;
  a.gp = grad_params;
  a.ga = grad_alpha;
  a.gb = grad_beta;
  a.gc = grad_chi2;
  a.grad = grad_images;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return FS_ERR_CUDA;
  const int warps_per_block = kBwdThreads / 32;
  const int64_t groups = (n + kGroup - 1) / kGroup;
  int64_t blocks = (groups + warps_per_block - 1) / warps_per_block;
  // without an upstream gradient of the normalised chi^2 the second pixel pass reads no pixels
  const bool chi = grad_chi2 != nullptr;
  const void *fn = dtype == FS_U16
                       ? (chi ? reinterpret_cast<const void *>(backward_kernel<unsigned short, true>)
                              : reinterpret_cast<const void *>(backward_kernel<unsigned short, false>))
                       : (chi ? reinterpret_cast<const void *>(backward_kernel<float, true>)
                              : reinterpret_cast<const void *>(backward_kernel<float, false>));
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBwdThreads, 0);
  if (e != cudaSuccess) return FS_ERR_CUDA;
  const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  if (blocks > cap) blocks = cap;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == FS_U16) {
    if (chi) backward_kernel<unsigned short, true><<<(int)blocks, kBwdThreads, 0, st>>>(a);
    else backward_kernel<unsigned short, false><<<(int)blocks, kBwdThreads, 0, st>>>(a);
  } else {
    if (chi) backward_kernel<float, true><<<(int)blocks, kBwdThreads, 0, st>>>(a);
    else backward_kernel<float, false><<<(int)blocks, kBwdThreads, 0, st>>>(a);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
