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
// Mapping: one spot per warp, pixel i handled by lane i mod 32. Pass A accumulates the
// 34 sums that build M (FP32, per lane, then a butterfly over the warp); M is diagonally
// scaled and solved by Gaussian elimination with partial pivoting (FP32, replicated in the
// lanes); pass B recomputes the profile and writes grad_g. The kernel is bound by the two
// reads of the pixels and the write of the gradient.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fitspots.h"

namespace {

constexpr int kBwdThreads = 128;
constexpr int kNSum = 34;

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

// Profile, first and second derivatives of the 4-parameter (x0, y0, sx, sy) profile at
// offsets (dx, dy): f, d[4], h[10] (upper triangle, row-major over j <= k).
__device__ __forceinline__ void derivs(float dx, float dy, float sx, float sy, float ivx,
                                       float ivy, float &f, float (&d)[4], float (&h)[10]) {
  f = __expf(-0.5f * (dx * dx * ivx + dy * dy * ivy));
  const float ax = dx * ivx, ay = dy * ivy;                          // d ln f / d x0, y0
  const float bx = dx * dx * ivx / sx, by = dy * dy * ivy / sy;      // d ln f / d sx, sy
  d[0] = ax * f;
  d[1] = ay * f;
  d[2] = bx * f;
  d[3] = by * f;
  h[0] = (ax * ax - ivx) * f;                       // x0 x0
  h[1] = ax * ay * f;                               // x0 y0
  h[2] = (ax * bx - 2.f * dx * ivx / sx) * f;       // x0 sx
  h[3] = ax * by * f;                               // x0 sy
  h[4] = (ay * ay - ivy) * f;                       // y0 y0
  h[5] = ay * bx * f;                               // y0 sx
  h[6] = (ay * by - 2.f * dy * ivy / sy) * f;       // y0 sy
  h[7] = (bx * bx - 3.f * dx * dx * ivx * ivx) * f; // sx sx
  h[8] = bx * by * f;                               // sx sy
  h[9] = (by * by - 3.f * dy * dy * ivy * ivy) * f; // sy sy
}

__device__ __forceinline__ int tri(int j, int k) {  // index of (j, k), j <= k, in a 4x4 triangle
  const int lo = j < k ? j : k, hi = j < k ? k : j;
  return lo * 4 - lo * (lo - 1) / 2 + (hi - lo);
}

__global__ void __launch_bounds__(kBwdThreads) backward_kernel(BwdArgs a) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (kBwdThreads / 32);
  for (int s = blockIdx.x * (kBwdThreads / 32) + (threadIdx.x >> 5); s < a.n; s += warps) {
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
    // upstream in (x0, y0, sx, sy, alpha, beta) order; the isotropic sigma is reported in
    // slots 2 and 3, so both feed its gradient
    float u[6];
    for (int j = 0; j < 4; ++j) u[j] = a.gp ? a.gp[4 * s + j] : 0.f;
    u[4] = a.ga ? a.ga[s] : 0.f;
    u[5] = a.gb ? a.gb[s] : 0.f;
    const float uc = a.gc ? a.gc[s] : 0.f;

    // pass A: the sums that build M
    float acc[kNSum];
#pragma unroll
    for (int k = 0; k < kNSum; ++k) acc[k] = 0.f;
    if (conv) {
      for (int i = lane; i < N; i += 32) {
        const int x = i % W, y = i / W;
        float f, d[4], h[10];
        derivs((float)x - x0, (float)y - y0, sx, sy, ivx, ivy, f, d, h);
        const float r = pix(a, off + i) - fmaf(al, f, be);
        int t = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int k = j; k < 4; ++k, ++t) acc[t] = fmaf(d[j], d[k], acc[t]);  // 0..9   d d^T
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[10 + j] = fmaf(f, d[j], acc[10 + j]);                              // 10..13 f d
          acc[14 + j] += d[j];                                                   // 14..17 d
          acc[18 + j] = fmaf(r, d[j], acc[18 + j]);                              // 18..21 r d
        }
        acc[22] = fmaf(f, f, acc[22]);                                           // 22 f f
        acc[23] += f;                                                            // 23 f
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[24 + k] = fmaf(r, h[k], acc[24 + k]);  // 24..33 r h
      }
#pragma unroll
      for (int k = 0; k < kNSum; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    }

    // M for q = (x0, y0, sx, sy, alpha, beta), then folded for the isotropic model
    float M[6][6], v[6];
    for (int j = 0; j < 4; ++j) {
      for (int k = 0; k < 4; ++k) M[j][k] = al * (al * acc[tri(j, k)] - acc[24 + tri(j, k)]);
      M[j][4] = M[4][j] = al * acc[10 + j] - acc[18 + j];
      M[j][5] = M[5][j] = al * acc[14 + j];
      v[j] = u[j];
    }
    M[4][4] = acc[22];
    M[4][5] = M[5][4] = acc[23];
    M[5][5] = (float)N;
    v[4] = u[4];
    v[5] = u[5];
    int Q = 6;
    if (iso) {  // sigma_x = sigma_y = sigma: merge rows/columns 2 and 3
      for (int k = 0; k < 6; ++k) M[2][k] += M[3][k];
      for (int k = 0; k < 6; ++k) M[k][2] += M[k][3];
      v[2] += v[3];
      for (int r = 3; r < 5; ++r) {
        for (int k = 0; k < 6; ++k) M[r][k] = M[r + 1][k];
        v[r] = v[r + 1];
      }
      for (int r = 0; r < 5; ++r)
        for (int k = 3; k < 5; ++k) M[r][k] = M[r][k + 1];
      Q = 5;
    }
    // Jacobi scaling, then Gaussian elimination with partial pivoting
    float sc[6];
    bool ok = conv;
    for (int j = 0; j < Q; ++j) {
      ok = ok && M[j][j] > 0.f;
      sc[j] = M[j][j] > 0.f ? rsqrtf(M[j][j]) : 1.f;
    }
    for (int j = 0; j < Q; ++j) {
      for (int k = 0; k < Q; ++k) M[j][k] *= sc[j] * sc[k];
      v[j] *= sc[j];
    }
    for (int c = 0; c < Q && ok; ++c) {
      int piv = c;
      for (int r = c + 1; r < Q; ++r)
        if (fabsf(M[r][c]) > fabsf(M[piv][c])) piv = r;
      if (!(fabsf(M[piv][c]) > 1e-30f)) {
        ok = false;
        break;
      }
      if (piv != c) {
        for (int k = 0; k < Q; ++k) {
          const float t = M[c][k];
          M[c][k] = M[piv][k];
          M[piv][k] = t;
        }
        const float t = v[c];
        v[c] = v[piv];
        v[piv] = t;
      }
      const float inv = 1.f / M[c][c];
      for (int r = c + 1; r < Q; ++r) {
        const float f = M[r][c] * inv;
        for (int k = c; k < Q; ++k) M[r][k] -= f * M[c][k];
        v[r] -= f * v[c];
      }
    }
    if (ok) {
      for (int r = Q - 1; r >= 0; --r) {
        float t = v[r];
        for (int k = r + 1; k < Q; ++k) t -= M[r][k] * v[k];
        v[r] = t / M[r][r];
      }
      for (int j = 0; j < Q; ++j) v[j] *= sc[j];
      for (int j = 0; j < 6; ++j) ok = ok && isfinite(v[j < Q ? j : 0]);
    }
    // back to (x0, y0, sx, sy, alpha, beta): the isotropic sigma moves both widths
    float vx = 0.f, vy = 0.f, vsx = 0.f, vsy = 0.f, va = 0.f, vb = 0.f;
    if (ok) {
      vx = v[0];
      vy = v[1];
      vsx = v[2];
      vsy = iso ? v[2] : v[3];
      va = iso ? v[3] : v[4];
      vb = iso ? v[4] : v[5];
    }
    const float cchi = ok ? 2.f * uc / (float)(N - P - 2) : 0.f;
    // pass B: grad_g_i = v . K_i (+ chi^2 term); zero for fits that did not converge
    for (int i = lane; i < N; i += 32) {
      float gval = 0.f;
      if (ok) {
        const int x = i % W, y = i / W;
        const float dx = (float)x - x0, dy = (float)y - y0;
        const float f = __expf(-0.5f * (dx * dx * ivx + dy * dy * ivy));
        float lin;
        if (iso) {
          lin = vx * dx * ivx + vy * dy * ivy + vsx * (dx * dx + dy * dy) * ivx / sx;
        } else {
          lin = vx * dx * ivx + vy * dy * ivy + vsx * dx * dx * ivx / sx + vsy * dy * dy * ivy / sy;
        }
        const float r = pix(a, off + i) - fmaf(al, f, be);
        gval = fmaf(f, fmaf(al, lin, va), vb) + cchi * r;
      }
      a.grad[off + i] = gval;
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
  int64_t blocks = (n + warps_per_block - 1) / warps_per_block;
  const int64_t cap = (int64_t)sms * 16;
  if (blocks > cap) blocks = cap;
  backward_kernel<<<(int)blocks, kBwdThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
