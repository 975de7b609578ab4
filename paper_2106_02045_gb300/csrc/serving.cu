// serving.cu -- device side of the real-time tracking loop (sm_103a).
//
// Fiducial markers are tracked frame to frame (the paper's motivation: stabilising a
// sample at millisecond time scales by following sparse fiducial spots). Per frame and
// marker the ROI of side R is placed at the rounded previous centre, cut from the frame
// on the device, fitted with the previous fit as the start point (fit_spots_uniform), and
// the marker state is advanced from the fit. Marker state never leaves the device on the
// hot path; only the small per-frame results are copied back.
//
// A batch covers up to kMaxBatch frames of different sessions (continuous batching): the
// descriptor desc = [count, slot_0, session_0, slot_1, session_1, ...] lives in device
// memory, so one captured graph serves any batch of a given size whatever its slots and
// sessions are. Every marker's work depends only on its own session's state and frame,
// never on the other frames in the batch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fitspots.h"

namespace {

constexpr int kCutThreads = 128;

struct CutArgs {
  const uint16_t *frames;  // device frame slots, slot s at frames + s * fw * fh
  int fw, fh, roi, markers;
  const int32_t *desc;     // [1 + 2 * kMaxBatch]
  const float *state;      // [sessions][markers][4] (x, y, sx, sy) in frame coordinates
  uint16_t *rois;          // [batch * markers][roi * roi]
  float *init;             // [batch * markers][4] in ROI coordinates
  int32_t *origin;         // [batch * markers][2]
};

__global__ void __launch_bounds__(kCutThreads) roi_cut_kernel(CutArgs a) {
  const int count = a.desc[0];
  const int b = blockIdx.y, m = blockIdx.x;
  if (b >= count || m >= a.markers) return;
  const int slot = a.desc[1 + 2 * b], sess = a.desc[2 + 2 * b];
  const float *st = a.state + ((int64_t)sess * a.markers + m) * 4;
  const int R = a.roi;
  // ROI at the rounded previous centre, kept inside the frame
  int ox = (int)rintf(st[0]) - R / 2, oy = (int)rintf(st[1]) - R / 2;
  ox = min(max(ox, 0), a.fw - R);
  oy = min(max(oy, 0), a.fh - R);
  const int64_t k = (int64_t)b * a.markers + m;
  const uint16_t *src = a.frames + (int64_t)slot * a.fw * a.fh;
  uint16_t *dst = a.rois + k * R * R;
  for (int i = threadIdx.x; i < R * R; i += kCutThreads) {
    const int y = i / R, x = i - y * R;
    dst[i] = src[(int64_t)(oy + y) * a.fw + ox + x];
  }
  if (threadIdx.x == 0) {
    a.init[4 * k + 0] = st[0] - (float)ox;
    a.init[4 * k + 1] = st[1] - (float)oy;
    a.init[4 * k + 2] = st[2];
    a.init[4 * k + 3] = st[3];
    a.origin[2 * k] = ox;
    a.origin[2 * k + 1] = oy;
  }
}

struct UpdArgs {
  const int32_t *desc;
  int markers;
  const float *params, *alpha, *beta, *chi2;
  const int32_t *fstate, *origin;
  float *state;    // [sessions][markers][4], updated in place
  float *results;  // [batch * markers][8]: x, y, sx, sy (frame coordinates), alpha, beta, chi2, state
};

__global__ void state_update_kernel(UpdArgs a) {
  const int count = a.desc[0];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count * a.markers) return;
  const int b = k / a.markers, m = k - b * a.markers;
  const int sess = a.desc[2 + 2 * b];
  float *st = a.state + ((int64_t)sess * a.markers + m) * 4;
  const int fs = a.fstate[k];
  const float x = a.params[4 * k] + (float)a.origin[2 * k];
  const float y = a.params[4 * k + 1] + (float)a.origin[2 * k + 1];
  const float sx = a.params[4 * k + 2], sy = a.params[4 * k + 3];
  const bool conv = (fs == FS_STATE_MIN_DELTA || fs == FS_STATE_MIN_STEP ||
                     fs == FS_STATE_MAX_ERROR || fs == FS_STATE_NO_DECREASE) &&
                    isfinite(x) && isfinite(y) && isfinite(sx) && isfinite(sy);
  if (conv) {  // a lost marker keeps its last position
    st[0] = x;
    st[1] = y;
    st[2] = sx;
    st[3] = sy;
  }
  float *r = a.results + 8 * (int64_t)k;
  r[0] = x;
  r[1] = y;
  r[2] = sx;
  r[3] = sy;
  r[4] = a.alpha[k];
  r[5] = a.beta[k];
  r[6] = a.chi2[k];
  r[7] = (float)fs;
}

}  // namespace

extern "C" {

int fs_serve_roi_cut(const uint16_t *frames, int frame_w, int frame_h, int roi, int markers,
                     const int32_t *desc, int max_batch, const float *state, uint16_t *rois,
                     float *init, int32_t *origin, void *stream) {
  if (!frames || !desc || !state || !rois || !init || !origin) return FS_ERR_NULL;
  if (roi < 3 || roi > 32 || frame_w < roi || frame_h < roi || markers < 1 || max_batch < 1 ||
      markers > 65535 || max_batch > 65535)
    return FS_ERR_ARG;
  CutArgs a{frames, frame_w, frame_h, roi, markers, desc, state, rois, init, origin};
  roi_cut_kernel<<<dim3(markers, max_batch), kCutThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}

int fs_serve_update(const int32_t *desc, int max_batch, int markers, const float *params,
                    const float *alpha, const float *beta, const float *chi2,
                    const int32_t *fit_state, const int32_t *origin, float *state,
                    float *results, void *stream) {
  if (!desc || !params || !alpha || !beta || !chi2 || !fit_state || !origin || !state || !results)
    return FS_ERR_NULL;
  if (markers < 1 || max_batch < 1 || markers > 65535 || max_batch > 65535) return FS_ERR_ARG;
  UpdArgs a{desc, markers, params, alpha, beta, chi2, fit_state, origin, state, results};
  const int total = markers * max_batch;
  state_update_kernel<<<(total + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}

}  // extern "C"
