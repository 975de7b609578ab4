// background.cu -- local background pre-subtraction (sm_103a).
//
// The fit assumes a uniform background beta in each ROI (Sec. "Implicit-amplitudes
// least-squares fitting"), where the paper also allows a locally varying background to be
// estimated and subtracted beforehand without fixing a method. This pass fits the plane
// b(x, y) = c0 + cx (x - xc) + cy (y - yc), xc = (W - 1) / 2, yc = (H - 1) / 2, by least
// squares to the ROI's border ring (pixels within `border` of an edge) and subtracts its
// tilt cx (x - xc) + cy (y - yc) from every pixel; c0 stays for the fit's beta.
//
// The ring is symmetric under x -> W - 1 - x and under y -> H - 1 - y, so over the ring
// sum (x - xc) = sum (y - yc) = sum (x - xc)(y - yc) = 0 and the 3 x 3 normal equations are
// diagonal: c0 = mean of the ring, cx = sum (x - xc) g / sum (x - xc)^2, likewise cy.
// Coordinates enter doubled (2x - W + 1, an integer), so for uint16 pixels every sum is an
// exact integer (split into two 32-bit halves for the warp reduction) and the coefficients
// are rounded only by the final FP32 conversions and divisions; float32 pixels are summed in
// FP32. No FP64: on this part a warp-wide FP64 instruction costs as much as 64 FP32 ones.
//
// The pass is bound by HBM traffic, N (sizeof(pixel) + 4) bytes per ROI, and needs many
// bytes in flight. A CTA takes 16 consecutive ROIs at a time; when their pixels lie in one
// span that fits the shared-memory stage (packed batches), all 256 threads copy the span
// with 16-byte vector loads (element loads for the unaligned head and tail), then each warp
// takes two ROIs from shared memory: ring sums, coefficients, and the subtracted pixels
// stored straight to global memory (coalesced FP32). Any other group (scattered or
// overlapping ROIs, bad offsets) is processed from global memory, one warp per ROI.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "fitspots.h"

namespace {

constexpr int kBgThreads = 256;
constexpr int kBgWarps = kBgThreads / 32;
constexpr int kBgGroup = 16;                    // ROIs per CTA step, two per warp
constexpr int kBgMaxPixels = 1024;
constexpr int kBgMaxBorder = 8;
constexpr int kBgStageElems = kBgGroup * (kBgMaxPixels + 8);   // room for 16 padded ROIs

template <typename T>
constexpr size_t stage_bytes() {
  return (size_t)kBgStageElems * sizeof(T) + 16;
}

struct BgArgs {
  const void *images;
  int64_t image_elems;
  const int64_t *offsets;
  const int32_t *dims;
  int32_t n;
  int border;
  float *out_images;
  float *out_plane;
};

__device__ __forceinline__ bool bg_roi_ok(int W, int H, int64_t off, int64_t elems) {
  return W >= 3 && H >= 3 && W <= kBgMaxPixels / 3 && H <= kBgMaxPixels / 3 &&
         W * H <= kBgMaxPixels && off >= 0 && off + (int64_t)W * H <= elems;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// warp total of 32-bit lane sums that may exceed 32 bits in total (exact)
__device__ __forceinline__ long long warp_sum_wide(int v) {
  const int hi = __reduce_add_sync(0xffffffffu, v >> 15);
  const unsigned lo = __reduce_add_sync(0xffffffffu, (unsigned)(v & 0x7fff));
  return (long long)hi * 32768 + (long long)lo;
}

// One ROI by one warp: ring sums, plane, subtracted pixels. `src` points at the ROI's first
// pixel, in shared or global memory (the caller's inlined pointer keeps the state space).
template <typename T>
__device__ __forceinline__ void bg_roi(const BgArgs &a, int s, int W, int H, int64_t off,
                                       const T *src, int lane) {
  const int N = W * H, bd = a.border;
  const int stepy = 32 / W, stepx = 32 - stepy * W;
  int cnt = 0, xx = 0, yy = 0;          // ring size, sum (2x - W + 1)^2, sum (2y - H + 1)^2
  int is0 = 0, isx = 0, isy = 0;        // uint16: exact lane sums
  float fs0 = 0.f, fsx = 0.f, fsy = 0.f;  // float32 lane sums
  int x = lane % W, y = lane / W;
  for (int i = lane; i < N; i += 32) {
    if (x < bd || x >= W - bd || y < bd || y >= H - bd) {
      const int dx = 2 * x - W + 1, dy = 2 * y - H + 1;
      ++cnt;
      xx += dx * dx;
      yy += dy * dy;
      if constexpr (sizeof(T) == 2) {
        const int gv = (int)src[i];
        is0 += gv;
        isx += dx * gv;
        isy += dy * gv;
      } else {
        const float gv = (float)src[i];
        fs0 += gv;
        fsx = fmaf((float)dx, gv, fsx);
        fsy = fmaf((float)dy, gv, fsy);
      }
    }
    x += stepx;
    y += stepy;
    if (x >= W) {
      x -= W;
      ++y;
    }
  }
  const float C = (float)__reduce_add_sync(0xffffffffu, cnt);
  const float XX = (float)__reduce_add_sync(0xffffffffu, xx);
  const float YY = (float)__reduce_add_sync(0xffffffffu, yy);
  float S0, SX, SY;
  if constexpr (sizeof(T) == 2) {
    S0 = (float)__reduce_add_sync(0xffffffffu, is0);
    SX = __ll2float_rn(warp_sum_wide(isx));
    SY = __ll2float_rn(warp_sum_wide(isy));
  } else {
    S0 = warp_sum_f(fs0);
    SX = warp_sum_f(fsx);
    SY = warp_sum_f(fsy);
  }
  // doubled coordinates: cx = (sum dx g / 2) / (sum dx^2 / 4) = 2 sum dx g / sum dx^2
  const float c0 = __fdiv_rn(S0, C), fx = __fdiv_rn(2.f * SX, XX), fy = __fdiv_rn(2.f * SY, YY);
  const float hx = 0.5f * (float)(W - 1), hy = 0.5f * (float)(H - 1);
  float *const out = a.out_images + off;
  x = lane % W;
  y = lane / W;
  for (int i = lane; i < N; i += 32) {
    out[i] = (float)src[i] - fmaf(fx, (float)x - hx, fy * ((float)y - hy));
    x += stepx;
    y += stepy;
    if (x >= W) {
      x -= W;
      ++y;
    }
  }
  if (lane == 0 && a.out_plane) {
    a.out_plane[3 * s] = c0;
    a.out_plane[3 * s + 1] = fx;
    a.out_plane[3 * s + 2] = fy;
  }
}

__device__ __forceinline__ void bg_invalid(const BgArgs &a, int s, int lane) {
  if (lane == 0 && a.out_plane)
    a.out_plane[3 * s] = a.out_plane[3 * s + 1] = a.out_plane[3 * s + 2] =
        __int_as_float(0x7fc00000);
}

extern __shared__ __align__(16) unsigned char g_bg_stage[];

template <typename T>
__global__ void __launch_bounds__(kBgThreads) background_kernel(BgArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int groups = (a.n + kBgGroup - 1) / kBgGroup;
  const T *const images = static_cast<const T *>(a.images);
  __shared__ int64_t s_first, s_end;
  for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const int r0 = grp * kBgGroup, r1 = min(r0 + kBgGroup, a.n);
    // the group's span, and whether every ROI of it is valid and inside the span
    bool in = true;
    if (threadIdx.x < kBgGroup) {
      const int r = r0 + threadIdx.x;
      if (r < r1) {
        const int W = a.dims[2 * r], H = a.dims[2 * r + 1];
        const int64_t off = a.offsets[r];
        in = bg_roi_ok(W, H, off, a.image_elems);
        if (threadIdx.x == 0) s_first = off;
        if (r == r1 - 1) s_end = off + (int64_t)W * H;
      }
    }
    __syncthreads();
    const int64_t first = s_first, end = s_end;
    if (threadIdx.x < kBgGroup && r0 + (int)threadIdx.x < r1) {
      const int64_t off = a.offsets[r0 + threadIdx.x];
      const int N = a.dims[2 * (r0 + threadIdx.x)] * a.dims[2 * (r0 + threadIdx.x) + 1];
      in = in && off >= first && off + N <= end;
    }
    const bool staged = __syncthreads_and(in) && end - first <= kBgStageElems;
    if (staged) {
      // bytes [base, base + nb) of the image buffer to the stage, so that the 16-byte
      // aligned middle lands 16-byte aligned in shared memory
      const unsigned char *base = reinterpret_cast<const unsigned char *>(images + first);
      const int64_t nb = (end - first) * (int64_t)sizeof(T);
      const uintptr_t b0 = reinterpret_cast<uintptr_t>(base);
      const uintptr_t a0 = (b0 + 15) & ~(uintptr_t)15, a1 = (b0 + nb) & ~(uintptr_t)15;
      const int shift = (int)(a0 - b0), pad = (16 - shift) & 15;
      unsigned char *stage = g_bg_stage + pad;   // stage[p] holds base[p]
      if (a1 > a0) {
        const int nv = (int)((a1 - a0) >> 4);
        const uint4 *src = reinterpret_cast<const uint4 *>(a0);
        uint4 *dst = reinterpret_cast<uint4 *>(stage + shift);
        for (int v = threadIdx.x; v < nv; v += kBgThreads) dst[v] = __ldg(src + v);
        // head and tail elements outside the aligned middle
        const int head = shift / (int)sizeof(T);
        const int tail0 = (int)((a1 - b0) / sizeof(T)), tot = (int)(end - first);
        const T *eg = images + first;
        T *es = reinterpret_cast<T *>(stage);
        if ((int)threadIdx.x < head) es[threadIdx.x] = __ldg(eg + threadIdx.x);
        if (tail0 + (int)threadIdx.x < tot) es[tail0 + threadIdx.x] = __ldg(eg + tail0 + threadIdx.x);
      } else {
        const T *eg = images + first;
        T *es = reinterpret_cast<T *>(stage);
        for (int e = threadIdx.x; e < (int)(end - first); e += kBgThreads) es[e] = __ldg(eg + e);
      }
      __syncthreads();
      const T *es = reinterpret_cast<const T *>(stage);
      for (int r = r0 + warp; r < r1; r += kBgWarps) {
        const int W = a.dims[2 * r], H = a.dims[2 * r + 1];
        const int64_t off = a.offsets[r];
        bg_roi<T>(a, r, W, H, off, es + (off - first), lane);
      }
    } else {
      for (int r = r0 + warp; r < r1; r += kBgWarps) {
        const int W = a.dims[2 * r], H = a.dims[2 * r + 1];
        const int64_t off = a.offsets[r];
        if (bg_roi_ok(W, H, off, a.image_elems))
          bg_roi<T>(a, r, W, H, off, images + off, lane);
        else
          bg_invalid(a, r, lane);
      }
    }
    __syncthreads();   // the stage and s_first / s_end are reused by the next group
  }
}

}  // namespace

extern "C" int fit_spots_subtract_background(const void *images, int dtype, int64_t image_elems,
                                             const int64_t *offsets, const int32_t *roi_dims,
                                             int64_t n, int border, float *out_images,
                                             float *out_plane, void *stream) {
  if (n < 0 || n > FS_MAX_SPOTS || image_elems < 0) return FS_ERR_SIZE;
  if (dtype != FS_U16 && dtype != FS_F32) return FS_ERR_DTYPE;
  if (border < 1 || border > kBgMaxBorder) return FS_ERR_ARG;
  if (n == 0) return FS_OK;
  if (!images || !offsets || !roi_dims || !out_images) return FS_ERR_NULL;
  BgArgs a;
  a.images = images;
  a.image_elems = image_elems;
  a.offsets = offsets;
  a.dims = roi_dims;
  a.n = (int32_t)n;
  a.border = border;
  a.out_images = out_images;
  a.out_plane = out_plane;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return FS_ERR_CUDA;
  auto launch = [&](auto kernel, size_t smem) -> cudaError_t {
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    int per_sm = 0;
    if (err == cudaSuccess)
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBgThreads, smem);
    if (err != cudaSuccess) return err;
    const int64_t groups = (n + kBgGroup - 1) / kBgGroup;
    const int64_t blocks = std::min<int64_t>(groups, (int64_t)sms * std::max(per_sm, 1));
    kernel<<<(int)blocks, kBgThreads, smem, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError();
  };
  e = dtype == FS_U16 ? launch(background_kernel<unsigned short>, stage_bytes<unsigned short>())
                      : launch(background_kernel<float>, stage_bytes<float>());
  return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
