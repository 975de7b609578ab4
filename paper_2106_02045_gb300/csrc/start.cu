// start.cu -- start values of the fit computed on the device (sm_103a).
//
// The fit starts from (x0, y0, s0, s0) estimated from the ROI's own pixels, so a caller with
// pixels on the device needs no host pass (the Results section of the paper estimates start
// values from the image before fitting). Two rules:
//   FS_START_CENTROID  background b0 = min g, amplitude a0 = max g - b0, centre = centroid of
//                      max(g - b0, 0) (the ROI centre if that weight is zero everywhere)
//   FS_START_PAPER     centre = the pixel whose in-ROI 3 x 3 neighbourhood has the largest
//                      mean (ties: the lowest row-major index)
// and in both, s0 = sqrt(max(M, 1) / pi) with M = #{g > a0 e^(-1/2) + b0}: the pixels above the
// level a Gaussian reaches at one sigma, counted as the disc they cover.
//
// Decisions are taken in FP32 on quantities that are exact for integer-valued pixels below
// 2^21 (uint16 data, photon counts): a0 and the threshold are formed as fl(fl(a0 c) + b0)
// with c = fl(e^(-1/2)); two neighbourhood means S_i / c_i and S_j / c_j are compared as
// S_i c_j against S_j c_i. S is separable: the in-ROI row sums of three (left, centre, right,
// added in that order) of the rows above, at and below (added in that order). One warp per
// spot, lanes over the pixels (row-major, 32 apart); the ROI and its row sums are staged in
// shared memory once and both passes and the windows read them there.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fitspots.h"

namespace {

constexpr int kStartThreads = 128;
// e^(-1/2) and pi rounded to FP32 (bit patterns, so that every implementation of the rule
// uses the same constants)
constexpr unsigned kOneSigmaBits = 0x3f1b4598u, kPiBits = 0x40490fdbu;

struct StartArgs {
  const void *images;
  int dtype;
  int64_t image_elems;
  const int64_t *offsets;
  const int32_t *dims;
  int32_t n;
  int rule;
  float *out;
};

template <typename T>
__device__ __forceinline__ float px(const T *p, int i) {
  return (float)__ldg(p + i);
}

// per warp: one ROI of <= 32 x 32 pixels, and for the 3 x 3 rule its row sums of three
__host__ __device__ constexpr int start_warp_floats(int rule) {
  return rule == FS_START_PAPER ? 2 * 1024 : 1024;
}

// candidate (mean numerator S, neighbour count c, pixel index i) of the 3 x 3 rule: does a
// beat b? Larger S / c, ties to the lower index.
__device__ __forceinline__ bool beats(float Sa, float ca, int ia, float Sb, float cb, int ib) {
  const float l = __fmul_rn(Sa, cb), r = __fmul_rn(Sb, ca);
  return l > r || (l == r && ia < ib);
}

template <typename T>
__global__ void __launch_bounds__(kStartThreads) start_kernel(StartArgs a) {
  extern __shared__ float sm_all[];
  float *const sg = sm_all + (threadIdx.x >> 5) * start_warp_floats(a.rule);  // the warp's ROI
  float *const sr = sg + 1024;  // its row sums of three (3 x 3 rule only)
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (kStartThreads / 32);
  const T *const img = static_cast<const T *>(a.images);
  for (int s = blockIdx.x * (kStartThreads / 32) + (threadIdx.x >> 5); s < a.n; s += warps) {
    const int W = a.dims[2 * s], H = a.dims[2 * s + 1];
    const int64_t off = a.offsets[s];
    if (W < 1 || H < 1 || W > 32 || H > 32 || off < 0 || off + (int64_t)W * H > a.image_elems) {
      if (lane < 4) a.out[4 * s + lane] = __int_as_float(0x7fc00000);
      continue;
    }
    const T *const g = img + off;
    const int N = W * H;
    // the ROI into shared memory (read once, coalesced), min and max on the way
    __syncwarp();
    float lo = INFINITY, hi = -INFINITY;
    for (int i = lane; i < N; i += 32) {
      const float v = px(g, i);
      sg[i] = v;
      lo = fminf(lo, v);
      hi = fmaxf(hi, v);
    }
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const float b0 = lo, a0 = __fsub_rn(hi, lo);
    const float thr = __fadd_rn(__fmul_rn(a0, __uint_as_float(kOneSigmaBits)), b0);
    // pixels above the one-sigma level, weighted centroid, and the 3 x 3 candidate
    int M = 0;
    float sw = 0.f, swx = 0.f, swy = 0.f;
    float bS = -INFINITY, bc = 1.f;
    int bi = N;
    // (x, y) of pixel i = lane + 32 k, stepped without divisions
    const int sy = 32 / W, sx = 32 - sy * W;
    const int x_start = lane - (lane / W) * W, y_start = lane / W;
    if (a.rule == FS_START_PAPER) {
      int x = x_start;
      for (int i = lane; i < N; i += 32) {
        float r = 0.f;
        if (x > 0) r = __fadd_rn(r, sg[i - 1]);
        r = __fadd_rn(r, sg[i]);
        if (x < W - 1) r = __fadd_rn(r, sg[i + 1]);
        sr[i] = r;
        x += sx;
        if (x >= W) x -= W;
      }
      __syncwarp();
    }
    int y = y_start, x = x_start;
    for (int i = lane; i < N; i += 32) {
      const float v = sg[i];
      M += v > thr;
      const float w = fmaxf(v - b0, 0.f);
      sw += w;
      swx = fmaf(w, (float)x, swx);
      swy = fmaf(w, (float)y, swy);
      if (a.rule == FS_START_PAPER) {
        float S = 0.f;
        if (y > 0) S = __fadd_rn(S, sr[i - W]);
        S = __fadd_rn(S, sr[i]);
        if (y < H - 1) S = __fadd_rn(S, sr[i + W]);
        const int c = (1 + (x > 0) + (x < W - 1)) * (1 + (y > 0) + (y < H - 1));
        if (beats(S, (float)c, i, bS, bc, bi)) {
          bS = S;
          bc = (float)c;
          bi = i;
        }
      }
      x += sx;
      y += sy;
      if (x >= W) {
        x -= W;
        ++y;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      M += __shfl_xor_sync(0xffffffffu, M, o);
      sw += __shfl_xor_sync(0xffffffffu, sw, o);
      swx += __shfl_xor_sync(0xffffffffu, swx, o);
      swy += __shfl_xor_sync(0xffffffffu, swy, o);
      const float oS = __shfl_xor_sync(0xffffffffu, bS, o);
      const float oc = __shfl_xor_sync(0xffffffffu, bc, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (beats(oS, oc, oi, bS, bc, bi)) {
        bS = oS;
        bc = oc;
        bi = oi;
      }
    }
    float x0, y0;
    if (a.rule == FS_START_PAPER) {
      y0 = (float)(bi / W);
      x0 = (float)(bi % W);
    } else if (sw > 0.f) {
      x0 = swx / sw;
      y0 = swy / sw;
    } else {
      x0 = 0.5f * (float)(W - 1);
      y0 = 0.5f * (float)(H - 1);
    }
    const float s0 = __fsqrt_rn(__fdiv_rn((float)max(M, 1), __uint_as_float(kPiBits)));
    if (lane == 0) {
      a.out[4 * s] = x0;
      a.out[4 * s + 1] = y0;
      a.out[4 * s + 2] = s0;
      a.out[4 * s + 3] = s0;
    }
  }
}

}  // namespace

extern "C" int fit_spots_start(const void *images, int dtype, int64_t image_elems,
                               const int64_t *offsets, const int32_t *roi_dims, int64_t n,
                               int rule, float *out_init, void *stream) {
  if (n < 0 || n > FS_MAX_SPOTS || image_elems < 0) return FS_ERR_SIZE;
  if (dtype != FS_U16 && dtype != FS_F32) return FS_ERR_DTYPE;
  if (rule != FS_START_CENTROID && rule != FS_START_PAPER) return FS_ERR_ARG;
  if (n == 0) return FS_OK;
  if (!images || !offsets || !roi_dims || !out_init) return FS_ERR_NULL;
  StartArgs a;
  a.images = images;
  a.dtype = dtype;
  a.image_elems = image_elems;
  a.offsets = offsets;
  a.dims = roi_dims;
  a.n = (int32_t)n;
  a.rule = rule;
  a.out = out_init;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return FS_ERR_CUDA;
  const int per_block = kStartThreads / 32;
  int64_t blocks = (n + per_block - 1) / per_block;
  if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
  const size_t smem = (size_t)per_block * start_warp_floats(rule) * sizeof(float);
  if (dtype == FS_U16)
    start_kernel<unsigned short>
        <<<(int)blocks, kStartThreads, smem, static_cast<cudaStream_t>(stream)>>>(a);
  else
    start_kernel<float><<<(int)blocks, kStartThreads, smem, static_cast<cudaStream_t>(stream)>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
