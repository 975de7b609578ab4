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
// Mapping: one spot per warp. Every sum that builds M separates (f = e_x e_y, and
// the derivatives are e_x e_y times polynomials of degree <= 4 in dx, dy): the pixel sums
// are the 13 bilinear forms G_ab = sum g' e_x dx^a e_y dy^b (a + b <= 4, as needed) and
// the rest are products of 1-D moments E_m = sum e_x dx^m, P_m = sum e_x^2 dx^m (and F_m,
// Q_m over y). Pass A therefore costs 5 FMA per pixel (row-weighted column sums); the 6x6
// system is Jacobi-scaled and solved by Gaussian elimination with partial pivoting,
// unrolled in registers; pass B writes grad_g = e_x e_y (alpha (A(x) + B(y)) + v_alpha)
// + v_beta + u_chi2 term, with A, B the 1-D parts of v . K. Pixel values enter as
// g' = g - rint(beta), which keeps the sums free of the background's magnitude.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fitspots.h"

namespace {

constexpr int kBwdThreads = 128;
constexpr int kBwdWarps = kBwdThreads / 32;
constexpr int kNSum = 33;  // 13 bilinear data sums, E0..4, P0..4, F0..4, Q0..4
constexpr int kBwdWarpFloats = 32 * 8 + 32 * 2 + kNSum * 32 + 36;

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
constexpr int kE = 13, kP = 18, kF = 23, kQ = 28;

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

__global__ void __launch_bounds__(kBwdThreads) backward_kernel(BwdArgs a) {
  __shared__ float4 sm4[kBwdWarps * kBwdWarpFloats / 4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *const rowt = reinterpret_cast<float *>(sm4) + warp * kBwdWarpFloats;  // [32][8]
  float2 *const rowb = reinterpret_cast<float2 *>(rowt + 32 * 8);           // [32]
  float *const red = rowt + 32 * 8 + 32 * 2;                                // [kNSum][32]
  float *const tot = red + kNSum * 32;                                      // [kNSum]
  const int warps = gridDim.x * kBwdWarps;
  for (int s = blockIdx.x * kBwdWarps + warp; s < a.n; s += warps) {
    const int W = a.dims[2 * s], H = a.dims[2 * s + 1], m = a.model[s];
    const int64_t off = a.offsets[s];
    const bool iso = m == FS_MODEL_ISO;
    const int P = iso ? 3 : 4;
    const bool valid = (m == FS_MODEL_ISO || m == FS_MODEL_ELLIPTIC) && W >= 3 && H >= 3 &&
                       W <= 32 && H <= 32 && W * H > P + 2 && off >= 0 &&
                       off + (int64_t)W * H <= a.image_elems;
    if (!valid) continue;
    const int N = W * H;
    const int st = a.state[s];
    const bool conv = st == FS_STATE_MIN_DELTA || st == FS_STATE_MIN_STEP ||
                      st == FS_STATE_MAX_ERROR || st == FS_STATE_NO_DECREASE;
    const float x0 = a.params[4 * s], y0 = a.params[4 * s + 1], sx = a.params[4 * s + 2];
    const float sy = iso ? sx : a.params[4 * s + 3];
    const float al = a.alpha[s], be = a.beta[s];
    const float ivx = 1.f / (sx * sx), ivy = 1.f / (sy * sy);
    const float cx = ivx / sx, cy = ivy / sy;
    const float sh = rintf(be), bp = be - sh;  // pixels enter as g - sh
    // pixel mapping: rps rows per step, lane l -> column l % W, first row l / W
    const int rps = 32 / W;
    const int xl = lane % W, yo = lane / W;
    const bool plane = yo < rps;

    // ---- 1-D profiles: column `lane` and row `lane`, and the row table e_y dy^b
    const float dxl = (float)lane - x0, dyl = (float)lane - y0;
    const float exl = lane < W ? __expf(-0.5f * dxl * dxl * ivx) : 0.f;
    const float eyl = lane < H ? __expf(-0.5f * dyl * dyl * ivy) : 0.f;
    {
      float t = eyl;
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        rowt[lane * 8 + b] = t;
        t *= dyl;
      }
    }
    __syncwarp();

    // ---- pass A: c_b(x) = sum_y g' e_y dy^b over this lane's rows
    float c[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (conv && plane) {
      for (int y = yo; y < H; y += rps) {
        const float g = pix(a, off + (int64_t)y * W + xl) - sh;
        const float4 r4 = *reinterpret_cast<const float4 *>(rowt + y * 8);
        const float r5 = rowt[y * 8 + 4];
        c[0] = fmaf(g, r4.x, c[0]);
        c[1] = fmaf(g, r4.y, c[1]);
        c[2] = fmaf(g, r4.z, c[2]);
        c[3] = fmaf(g, r4.w, c[3]);
        c[4] = fmaf(g, r5, c[4]);
      }
    }
    for (int t = 1; t < rps; ++t)
#pragma unroll
      for (int b = 0; b < 5; ++b) c[b] += __shfl_down_sync(0xffffffffu, c[b], t * W);
    // ---- partial sums: lanes < W hold column `lane` (G_ab, E, P), lanes < H row `lane`
    {
      float v[kNSum];
#pragma unroll
      for (int k = 0; k < kNSum; ++k) v[k] = 0.f;
      if (lane < W) {
        const float p0 = exl, p1 = p0 * dxl, p2 = p1 * dxl, p3 = p2 * dxl, p4 = p3 * dxl;
        v[G00] = p0 * c[0];
        v[G10] = p1 * c[0];
        v[G01] = p0 * c[1];
        v[G20] = p2 * c[0];
        v[G02] = p0 * c[2];
        v[G11] = p1 * c[1];
        v[G30] = p3 * c[0];
        v[G03] = p0 * c[3];
        v[G12] = p1 * c[2];
        v[G21] = p2 * c[1];
        v[G40] = p4 * c[0];
        v[G22] = p2 * c[2];
        v[G04] = p0 * c[4];
        v[kE + 0] = p0;
        v[kE + 1] = p1;
        v[kE + 2] = p2;
        v[kE + 3] = p3;
        v[kE + 4] = p4;
        v[kP + 0] = p0 * exl;
        v[kP + 1] = p1 * exl;
        v[kP + 2] = p2 * exl;
        v[kP + 3] = p3 * exl;
        v[kP + 4] = p4 * exl;
      }
      if (lane < H) {
        const float q0 = eyl, q1 = q0 * dyl, q2 = q1 * dyl, q3 = q2 * dyl, q4 = q3 * dyl;
        v[kF + 0] = q0;
        v[kF + 1] = q1;
        v[kF + 2] = q2;
        v[kF + 3] = q3;
        v[kF + 4] = q4;
        v[kQ + 0] = q0 * eyl;
        v[kQ + 1] = q1 * eyl;
        v[kQ + 2] = q2 * eyl;
        v[kQ + 3] = q3 * eyl;
        v[kQ + 4] = q4 * eyl;
      }
#pragma unroll
      for (int k = 0; k < kNSum; ++k) red[k * 32 + lane] = v[k];
    }
    __syncwarp();
    for (int k = lane; k < kNSum; k += 32) {
      const float4 *r = reinterpret_cast<const float4 *>(red + k * 32);
      float q[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float4 w = r[i];
        q[i] = (w.x + w.y) + (w.z + w.w);
      }
      tot[k] = ((q[0] + q[1]) + (q[2] + q[3])) + ((q[4] + q[5]) + (q[6] + q[7]));
    }
    __syncwarp();

    // ---- M for q = (x0, y0, sx, sy, alpha, beta)
    const float E0 = tot[kE], E1 = tot[kE + 1], E2 = tot[kE + 2], E3 = tot[kE + 3], E4 = tot[kE + 4];
    const float P0 = tot[kP], P1 = tot[kP + 1], P2 = tot[kP + 2], P3 = tot[kP + 3], P4 = tot[kP + 4];
    const float F0 = tot[kF], F1 = tot[kF + 1], F2 = tot[kF + 2], F3 = tot[kF + 3], F4 = tot[kF + 4];
    const float Q0 = tot[kQ], Q1 = tot[kQ + 1], Q2 = tot[kQ + 2], Q3 = tot[kQ + 3], Q4 = tot[kQ + 4];
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
    GD[0] = ivx * tot[G10];
    GD[1] = ivy * tot[G01];
    GD[2] = cx * tot[G20];
    GD[3] = cy * tot[G02];
    GH[0] = ivx * ivx * tot[G20] - ivx * tot[G00];
    FH[0] = ivx * ivx * P2 * Q0 - ivx * P0 * Q0;
    SH[0] = ivx * ivx * E2 * F0 - ivx * E0 * F0;
    GH[1] = ivx * ivy * tot[G11];
    FH[1] = ivx * ivy * P1 * Q1;
    SH[1] = ivx * ivy * E1 * F1;
    GH[2] = ivx * cx * tot[G30] - 2.f * cx * tot[G10];
    FH[2] = ivx * cx * P3 * Q0 - 2.f * cx * P1 * Q0;
    SH[2] = ivx * cx * E3 * F0 - 2.f * cx * E1 * F0;
    GH[3] = ivx * cy * tot[G12];
    FH[3] = ivx * cy * P1 * Q2;
    SH[3] = ivx * cy * E1 * F2;
    GH[4] = ivy * ivy * tot[G02] - ivy * tot[G00];
    FH[4] = ivy * ivy * P0 * Q2 - ivy * P0 * Q0;
    SH[4] = ivy * ivy * E0 * F2 - ivy * E0 * F0;
    GH[5] = ivy * cx * tot[G21];
    FH[5] = ivy * cx * P2 * Q1;
    SH[5] = ivy * cx * E2 * F1;
    GH[6] = ivy * cy * tot[G03] - 2.f * cy * tot[G01];
    FH[6] = ivy * cy * P0 * Q3 - 2.f * cy * P0 * Q1;
    SH[6] = ivy * cy * E0 * F3 - 2.f * cy * E0 * F1;
    GH[7] = cx * cx * tot[G40] - 3.f * ivx * ivx * tot[G20];
    FH[7] = cx * cx * P4 * Q0 - 3.f * ivx * ivx * P2 * Q0;
    SH[7] = cx * cx * E4 * F0 - 3.f * ivx * ivx * E2 * F0;
    GH[8] = cx * cy * tot[G22];
    FH[8] = cx * cy * P2 * Q2;
    SH[8] = cx * cy * E2 * F2;
    GH[9] = cy * cy * tot[G04] - 3.f * ivy * ivy * tot[G02];
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
    M[5][5] = (float)N;
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
    // Jacobi scaling, then Gaussian elimination with partial pivoting (row swaps by select)
    bool ok = conv;
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
    // (vx, vy, vsx, vsy, va, vb); the isotropic sigma moves both widths
    float vx = 0.f, vy = 0.f, vsx = 0.f, vsy = 0.f, va = 0.f, vb = 0.f;
    if (ok) {
      vx = v[0];
      vy = v[1];
      vsx = v[2];
      vsy = iso ? v[2] : v[3];
      va = v[4];
      vb = v[5];
    }
    const float cchi = ok ? 2.f * uc / (float)(N - P - 2) : 0.f;
    // ---- pass B: grad_g = e_x e_y (alpha (A(x) + B(y)) + va) + vb + cchi (g' - alpha f - bp)
    rowb[lane] = make_float2(eyl, fmaf(vy * ivy, dyl, vsy * cy * dyl * dyl));
    __syncwarp();
    if (plane) {
      const float dxc = (float)xl - x0;
      const float exc = __expf(-0.5f * dxc * dxc * ivx);
      const float Ax = fmaf(vx * ivx, dxc, vsx * cx * dxc * dxc);
      for (int y = yo; y < H; y += rps) {
        const int64_t idx = off + (int64_t)y * W + xl;
        float gval = 0.f;
        if (ok) {
          const float2 eb = rowb[y];
          const float f = exc * eb.x;
          const float r = pix(a, idx) - sh - fmaf(al, f, bp);
          gval = fmaf(f, fmaf(al, Ax + eb.y, va), vb) + cchi * r;
        }
        a.grad[idx] = gval;
      }
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
  int64_t blocks = (n + warps_per_block - 1) / warps_per_block;
  const int64_t cap = (int64_t)sms * 16;
  if (blocks > cap) blocks = cap;
  backward_kernel<<<(int)blocks, kBwdThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
