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
constexpr int kGroup = 32;   // spots per warp group (one per lane in phase S)
constexpr int kNG = 13;      // bilinear data sums G_ab
constexpr int kGStride = kGroup + 1;
constexpr int kChunk = 8;    // pixel rows a lane loads before it computes on them
// per warp: row table [32][8], reduction rows [kNG][32], group table [kNG][kGStride],
// pass-B row table [32] float2
constexpr int kGTabFloats = (kNG * kGStride + 1) / 2 * 2;
constexpr int kBwdWarpFloats = (32 * 8 + kNG * 32 + kGTabFloats + 32 * 2 + 3) / 4 * 4;

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

__device__ __forceinline__ float pix(const BwdArgs &a, int64_t idx) {
  return a.dtype == FS_U16 ? (float)static_cast<const unsigned short *>(a.images)[idx]
                           : static_cast<const float *>(a.images)[idx];
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

__device__ __forceinline__ float shfl(float v, int j) { return __shfl_sync(0xffffffffu, v, j); }
__device__ __forceinline__ int shfl(int v, int j) { return __shfl_sync(0xffffffffu, v, j); }

// Prefetch into L2 the pixel range of a spot (whole 128-byte lines; the range is in bounds
// and every touched line overlaps it).
__device__ __forceinline__ void prefetch_spot(const BwdArgs &a, int s) {
  const int W = a.dims[2 * s], H = a.dims[2 * s + 1];
  const int64_t off = a.offsets[s];
  if (W < 1 || H < 1 || W > 32 || H > 32 || off < 0 || off + (int64_t)W * H > a.image_elems)
    return;
  const int esz = a.dtype == FS_U16 ? 2 : 4;
  const char *base = static_cast<const char *>(a.images);
  const uintptr_t lo = reinterpret_cast<uintptr_t>(base + off * esz) & ~uintptr_t(127);
  const uintptr_t hi = reinterpret_cast<uintptr_t>(base + (off + (int64_t)W * H) * esz);
  for (uintptr_t p = lo; p < hi; p += 128)
    asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(p));
}

__global__ void __launch_bounds__(kBwdThreads) backward_kernel(BwdArgs a) {
  __shared__ float4 sm4[kBwdWarps * kBwdWarpFloats / 4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *const rowt = reinterpret_cast<float *>(sm4) + warp * kBwdWarpFloats;  // [32][8]
  float *const red = rowt + 32 * 8;                        // [kNG][32]
  float *const gtab = red + kNG * 32;                      // [kNG][kGStride]
  float2 *const rowb = reinterpret_cast<float2 *>(gtab + kGTabFloats);  // [32]
  const int ngroups = (a.n + kGroup - 1) / kGroup;
  const int gstride = gridDim.x * kBwdWarps;
  int g = blockIdx.x * kBwdWarps + warp;
  if (g < ngroups && g * kGroup + lane < a.n) prefetch_spot(a, g * kGroup + lane);
  for (; g < ngroups; g += gstride) {
    const int s0 = g * kGroup;
    const int ns = min(kGroup, a.n - s0);
    {
      const int sn = (g + gstride) * kGroup + lane;
      if (g + gstride < ngroups && sn < a.n) prefetch_spot(a, sn);
    }
    // ---- lane j holds spot s0 + j
    const int s = s0 + lane;
    const bool have = lane < ns;
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
    const int rps = valid ? 32 / W : 1;
    const float rW = valid ? 1.f / (float)W : 1.f;
    const int nrow = valid ? (H + rps - 1) / rps : 0;  // row steps of the pixel passes
    const unsigned conv_mask = __ballot_sync(0xffffffffu, conv);
    const unsigned valid_mask = __ballot_sync(0xffffffffu, valid);

    // ---- phase A: G_ab of each converged spot into gtab[k][j]
    for (int j = 0; j < ns; ++j) {
      if (!((conv_mask >> j) & 1u)) continue;
      const int Wj = shfl(W, j), Hj = shfl(H, j), rpsj = shfl(rps, j), nrj = shfl(nrow, j);
      const int olo = shfl((int)(off & 0xffffffff), j), ohi = shfl((int)(off >> 32), j);
      const int64_t offj = (int64_t)(((uint64_t)(uint32_t)ohi << 32) | (uint32_t)olo);
      const float x0j = shfl(x0, j), y0j = shfl(y0, j), ivxj = shfl(ivx, j), ivyj = shfl(ivy, j);
      const float shj = shfl(sh, j), rWj = shfl(rW, j);
      // row table: e_y dy^b, b = 0..4 (zero beyond the ROI)
      {
        const float dy = (float)lane - y0j;
        const float e = lane < Hj ? __expf(-0.5f * dy * dy * ivyj) : 0.f;
        const float e1 = e * dy, e2 = e1 * dy, e3 = e2 * dy;
        *reinterpret_cast<float4 *>(rowt + lane * 8) = make_float4(e, e1, e2, e3);
        rowt[lane * 8 + 4] = e3 * dy;
      }
      __syncwarp();
      const int yo = (int)(((float)lane + 0.5f) * rWj);
      const int xl = lane - yo * Wj;
      const bool plane = yo < rpsj;
      float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f, c4 = 0.f;
      for (int t0 = 0; t0 < nrj; t0 += kChunk) {
        float gv[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int y = yo + (t0 + u) * rpsj;
          gv[u] = plane && y < Hj ? pix(a, offj + (int64_t)y * Wj + xl) - shj : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int y = min(yo + (t0 + u) * rpsj, 31);
          const float4 r4 = *reinterpret_cast<const float4 *>(rowt + y * 8);
          const float r5 = rowt[y * 8 + 4];
          c0 = fmaf(gv[u], r4.x, c0);
          c1 = fmaf(gv[u], r4.y, c1);
          c2 = fmaf(gv[u], r4.z, c2);
          c3 = fmaf(gv[u], r4.w, c3);
          c4 = fmaf(gv[u], r5, c4);
        }
      }
      for (int t = 1; t < rpsj; ++t) {
        const int d = t * Wj;
        c0 += __shfl_down_sync(0xffffffffu, c0, d);
        c1 += __shfl_down_sync(0xffffffffu, c1, d);
        c2 += __shfl_down_sync(0xffffffffu, c2, d);
        c3 += __shfl_down_sync(0xffffffffu, c3, d);
        c4 += __shfl_down_sync(0xffffffffu, c4, d);
      }
      {
        const float dx = (float)lane - x0j;
        const float p0 = lane < Wj ? __expf(-0.5f * dx * dx * ivxj) : 0.f;
        const float p1 = p0 * dx, p2 = p1 * dx, p3 = p2 * dx, p4 = p3 * dx;
        red[G00 * 32 + lane] = p0 * c0;
        red[G10 * 32 + lane] = p1 * c0;
        red[G01 * 32 + lane] = p0 * c1;
        red[G20 * 32 + lane] = p2 * c0;
        red[G02 * 32 + lane] = p0 * c2;
        red[G11 * 32 + lane] = p1 * c1;
        red[G30 * 32 + lane] = p3 * c0;
        red[G03 * 32 + lane] = p0 * c3;
        red[G12 * 32 + lane] = p1 * c2;
        red[G21 * 32 + lane] = p2 * c1;
        red[G40 * 32 + lane] = p4 * c0;
        red[G22 * 32 + lane] = p2 * c2;
        red[G04 * 32 + lane] = p0 * c4;
      }
      __syncwarp();
      if (lane < kNG) {
        const float4 *r = reinterpret_cast<const float4 *>(red + lane * 32);
        float q[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float4 w = r[i];
          q[i] = (w.x + w.y) + (w.z + w.w);
        }
        gtab[lane * kGStride + j] =
            ((q[0] + q[1]) + (q[2] + q[3])) + ((q[4] + q[5]) + (q[6] + q[7]));
      }
      __syncwarp();
    }

    // ---- phase S: lane j builds M for its spot and solves M v = u
    float vx = 0.f, vy = 0.f, vsx = 0.f, vsy = 0.f, va = 0.f, vb = 0.f, cchi = 0.f;
    bool ok = false;
    if (conv) {
      const float cx = ivx / sx, cy = ivy / sy;
      float E0 = 0.f, E1 = 0.f, E2 = 0.f, E3 = 0.f, E4 = 0.f;
      float P0 = 0.f, P1 = 0.f, P2 = 0.f, P3 = 0.f, P4 = 0.f;
      for (int x = 0; x < W; ++x) {
        const float d = (float)x - x0;
        const float e = __expf(-0.5f * d * d * ivx), ee = e * e;
        const float d2 = d * d;
        E0 += e;
        E1 = fmaf(e, d, E1);
        E2 = fmaf(e, d2, E2);
        E3 = fmaf(e * d, d2, E3);
        E4 = fmaf(e * d2, d2, E4);
        P0 += ee;
        P1 = fmaf(ee, d, P1);
        P2 = fmaf(ee, d2, P2);
        P3 = fmaf(ee * d, d2, P3);
        P4 = fmaf(ee * d2, d2, P4);
      }
      float F0 = 0.f, F1 = 0.f, F2 = 0.f, F3 = 0.f, F4 = 0.f;
      float Q0 = 0.f, Q1 = 0.f, Q2 = 0.f, Q3 = 0.f, Q4 = 0.f;
      for (int y = 0; y < H; ++y) {
        const float d = (float)y - y0;
        const float e = __expf(-0.5f * d * d * ivy), ee = e * e;
        const float d2 = d * d;
        F0 += e;
        F1 = fmaf(e, d, F1);
        F2 = fmaf(e, d2, F2);
        F3 = fmaf(e * d, d2, F3);
        F4 = fmaf(e * d2, d2, F4);
        Q0 += ee;
        Q1 = fmaf(ee, d, Q1);
        Q2 = fmaf(ee, d2, Q2);
        Q3 = fmaf(ee * d, d2, Q3);
        Q4 = fmaf(ee * d2, d2, Q4);
      }
      float G[kNG];
#pragma unroll
      for (int k = 0; k < kNG; ++k) G[k] = gtab[k * kGStride + lane];
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
      float M[6][6], v[6];
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
      M[5][5] = (float)(W * H);
      // upstream in (x0, y0, sx, sy, alpha, beta) order; the isotropic sigma is reported in
      // slots 2 and 3, so both feed its gradient
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = a.gp ? a.gp[4 * s + j] : 0.f;
      v[4] = a.ga ? a.ga[s] : 0.f;
      v[5] = a.gb ? a.gb[s] : 0.f;
      const float uc = a.gc ? a.gc[s] : 0.f;
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
      ok = true;
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
    const unsigned ok_mask = __ballot_sync(0xffffffffu, ok);

    // ---- phase B: grad_g = e_x e_y (alpha (A(x) + B(y)) + va) + vb + cchi (g' - alpha f - bp)
    for (int j = 0; j < ns; ++j) {
      if (!((valid_mask >> j) & 1u)) continue;
      const bool okj = (ok_mask >> j) & 1u;
      const int Wj = shfl(W, j), Hj = shfl(H, j), rpsj = shfl(rps, j), nrj = shfl(nrow, j);
      const int olo = shfl((int)(off & 0xffffffff), j), ohi = shfl((int)(off >> 32), j);
      const int64_t offj = (int64_t)(((uint64_t)(uint32_t)ohi << 32) | (uint32_t)olo);
      const float rWj = shfl(rW, j);
      const int yo = (int)(((float)lane + 0.5f) * rWj);
      const int xl = lane - yo * Wj;
      const bool plane = yo < rpsj;
      if (!okj) {  // no gradient through fits that did not converge
        if (plane)
          for (int y = yo; y < Hj; y += rpsj) a.grad[offj + (int64_t)y * Wj + xl] = 0.f;
        continue;
      }
      const float x0j = shfl(x0, j), y0j = shfl(y0, j), ivxj = shfl(ivx, j), ivyj = shfl(ivy, j);
      const float alj = shfl(al, j), shj = shfl(sh, j), bpj = shfl(bp, j);
      const float vxj = shfl(vx, j), vyj = shfl(vy, j), vsxj = shfl(vsx, j), vsyj = shfl(vsy, j);
      const float vaj = shfl(va, j), vbj = shfl(vb, j), ccj = shfl(cchi, j);
      {
        const float dy = (float)lane - y0j;
        const float e = lane < Hj ? __expf(-0.5f * dy * dy * ivyj) : 0.f;
        rowb[lane] = make_float2(e, dy * fmaf(vsyj, dy, vyj));
      }
      __syncwarp();
      const float dx = (float)xl - x0j;
      const float ex = __expf(-0.5f * dx * dx * ivxj);
      const float Ax = dx * fmaf(vsxj, dx, vxj);
      for (int t0 = 0; t0 < nrj; t0 += kChunk) {
        float gv[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int y = yo + (t0 + u) * rpsj;
          gv[u] = plane && y < Hj ? pix(a, offj + (int64_t)y * Wj + xl) - shj : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int y = yo + (t0 + u) * rpsj;
          if (plane && y < Hj) {
            const float2 eb = rowb[y];
            const float f = ex * eb.x;
            const float r = gv[u] - fmaf(alj, f, bpj);
            a.grad[offj + (int64_t)y * Wj + xl] = fmaf(f, fmaf(alj, Ax + eb.y, vaj), vbj) + ccj * r;
          }
        }
      }
      __syncwarp();
    }
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
  if (n < 0 || n > INT32_MAX || image_elems < 0) return FS_ERR_SIZE;
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
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, backward_kernel, kBwdThreads, 0);
  if (e != cudaSuccess) return FS_ERR_CUDA;
  const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  if (blocks > cap) blocks = cap;
  backward_kernel<<<(int)blocks, kBwdThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
