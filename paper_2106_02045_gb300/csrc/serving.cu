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
  const float *params, *alpha, *beta, *chi2, *init;
  const int32_t *fstate, *iters, *origin;
  float *state;    // [sessions][markers][4], updated in place
  float *results;  // [batch * markers][kResultFloats]
};

__global__ void state_update_kernel(UpdArgs a) {
  const int count = a.desc[0];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count * a.markers) return;
  const int b = k / a.markers, m = k - b * a.markers;
  const int sess = a.desc[2 + 2 * b];
  float *st = a.state + ((int64_t)sess * a.markers + m) * 4;
  const int fs = a.fstate[k];
  const float ox = (float)a.origin[2 * k], oy = (float)a.origin[2 * k + 1];
  const float x = a.params[4 * k] + ox;
  const float y = a.params[4 * k + 1] + oy;
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
  float *r = a.results + FS_SERVE_RESULT_FLOATS * (int64_t)k;
  r[0] = x;
  r[1] = y;
  r[2] = sx;
  r[3] = sy;
  r[4] = a.alpha[k];
  r[5] = a.beta[k];
  r[6] = a.chi2[k];
  r[7] = (float)fs;
  r[8] = ox;
  r[9] = oy;
#pragma unroll
  for (int j = 0; j < 4; ++j) r[10 + j] = a.init[4 * k + j];
  r[14] = (float)a.iters[k];
  r[15] = 0.f;
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
                    const int32_t *fit_state, const int32_t *fit_iters, const float *init,
                    const int32_t *origin, float *state, float *results, void *stream) {
  if (!desc || !params || !alpha || !beta || !chi2 || !fit_state || !fit_iters || !init ||
      !origin || !state || !results)
    return FS_ERR_NULL;
  if (markers < 1 || max_batch < 1 || markers > 65535 || max_batch > 65535) return FS_ERR_ARG;
  UpdArgs a{desc, markers, params, alpha, beta, chi2, init, fit_state, fit_iters, origin, state,
            results};
  const int total = markers * max_batch;
  state_update_kernel<<<(total + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}

}  // extern "C"

// ====================================================================== sessions (host side)
// A session serves `streams` camera streams of one frame size with continuous batching:
// frames arrive through fs_session_submit_frame (host pointers, ideally pinned), wait in a
// bounded queue for a device frame slot (the memory budget), are copied in on a copy stream,
// and join the next batch (at most one frame per stream, since a stream's next ROI placement
// needs its previous fit) while earlier batches may still run. Each batch is one launch of a
// CUDA graph captured at creation for its size: ROI cut, warm-started fit, state update.
// fs_session_poll admits, launches and retires; a retired frame's results and its arrival
// and completion stamps (fs_session_clock) go to the caller. One host thread per session.
#include <algorithm>
#include <chrono>
#include <deque>
#include <new>
#include <vector>

struct fs_session {
  fs_session_config cfg{};
  cudaStream_t compute = nullptr, copy = nullptr;
  // device buffers
  uint16_t *frames = nullptr, *rois = nullptr;
  float *state = nullptr, *init = nullptr, *results = nullptr;
  float *fparams = nullptr, *falpha = nullptr, *fbeta = nullptr, *fchi2 = nullptr;
  int32_t *origin = nullptr, *fstate = nullptr, *fiters = nullptr, *desc = nullptr;
  void *ws = nullptr;
  // pinned host staging, one buffer per batch in flight
  int32_t *h_desc = nullptr;
  float *h_results = nullptr;
  std::vector<cudaGraphExec_t> graphs;  // batch size k at k - 1
  std::vector<cudaEvent_t> slot_ready, buf_done;
  struct Frame {
    int stream;
    int64_t index;
    double t_arrival;
    const uint16_t *host;
    int slot;
  };
  struct Batch {
    std::vector<Frame> frames;
    int buf;
  };
  std::deque<Frame> pending;  // waiting for a frame slot
  std::vector<Frame> landed;  // copied in, or copying
  std::deque<Batch> inflight;
  std::deque<int> free_slots, free_bufs;
  std::vector<char> busy;  // a stream with a frame in a batch on the device
  int64_t dropped = 0, served = 0, batches = 0;
  cudaError_t err = cudaSuccess;
};

namespace {

size_t frame_elems(const fs_session_config &c) { return (size_t)c.frame_w * c.frame_h; }
size_t batch_spots(const fs_session_config &c) { return (size_t)c.max_batch * c.markers; }

// The device work of a batch of k frames (the descriptor already in s->desc).
int session_step(fs_session *s, int k) {
  const fs_session_config &c = s->cfg;
  int rc = fs_serve_roi_cut(s->frames, c.frame_w, c.frame_h, c.roi, c.markers, s->desc, k,
                            s->state, s->rois, s->init, s->origin, s->compute);
  if (rc) return rc;
  const int64_t n = (int64_t)k * c.markers;
  rc = fit_spots_uniform(s->rois, FS_U16, c.roi, c.roi, FS_MODEL_ISO, s->init, n, c.max_iter, 0.0,
                         c.min_delta, c.min_step, s->fparams, s->falpha, s->fbeta, s->fchi2,
                         s->fstate, s->fiters, nullptr, s->ws, fit_spots_uniform_workspace(),
                         s->compute);
  if (rc) return rc;
  return fs_serve_update(s->desc, k, c.markers, s->fparams, s->falpha, s->fbeta, s->fchi2,
                         s->fstate, s->fiters, s->init, s->origin, s->state, s->results,
                         s->compute);
}

void session_free(fs_session *s) {
  if (!s) return;
  if (s->compute) cudaStreamSynchronize(s->compute);
  if (s->copy) cudaStreamSynchronize(s->copy);
  for (auto g : s->graphs)
    if (g) cudaGraphExecDestroy(g);
  for (auto e : s->slot_ready)
    if (e) cudaEventDestroy(e);
  for (auto e : s->buf_done)
    if (e) cudaEventDestroy(e);
  void *dev[] = {s->frames, s->rois,   s->state,  s->init,   s->results, s->fparams, s->falpha,
                 s->fbeta,  s->fchi2,  s->origin, s->fstate, s->fiters,  s->desc,    s->ws};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (s->h_desc) cudaFreeHost(s->h_desc);
  if (s->h_results) cudaFreeHost(s->h_results);
  if (s->compute) cudaStreamDestroy(s->compute);
  if (s->copy) cudaStreamDestroy(s->copy);
  delete s;
}

int cuda_fail(fs_session *s, cudaError_t e) {
  if (s) s->err = e;
  return FS_ERR_CUDA;
}

}  // namespace

extern "C" {

double fs_session_clock(void) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int fs_session_create(const fs_session_config *cfg, fs_session **out) {
  if (!cfg || !out) return FS_ERR_NULL;
  const fs_session_config c = *cfg;
  if (c.roi < 3 || c.roi > 32 || c.frame_w < c.roi || c.frame_h < c.roi || c.frame_w > 65536 ||
      c.frame_h > 65536 || c.markers < 1 || c.markers > 65535 || c.streams < 1 ||
      c.streams > 65535 || c.max_batch < 1 || c.max_batch > 64 || c.max_batch > c.streams ||
      c.frame_slots < 1 || c.frame_slots > 4096 || c.queue_limit < 0 || c.max_inflight < 1 ||
      c.max_inflight > 64 || c.max_iter < 1 || c.max_iter > 1000 || !(c.min_delta >= 0.0) ||
      !(c.min_delta < 1.0) || !(c.min_step >= 0.0))
    return FS_ERR_ARG;
  *out = nullptr;
  fs_session *s = new (std::nothrow) fs_session;
  if (!s) return FS_ERR_ARG;
  s->cfg = c;
  const size_t nb = batch_spots(c), R2 = (size_t)c.roi * c.roi;
  cudaError_t e = cudaSuccess;
  auto dalloc = [&](auto **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
  };
  dalloc(&s->frames, (size_t)c.frame_slots * frame_elems(c) * sizeof(uint16_t));
  dalloc(&s->state, (size_t)c.streams * c.markers * 4 * sizeof(float));
  dalloc(&s->rois, nb * R2 * sizeof(uint16_t));
  dalloc(&s->init, nb * 4 * sizeof(float));
  dalloc(&s->origin, nb * 2 * sizeof(int32_t));
  dalloc(&s->fparams, nb * 4 * sizeof(float));
  dalloc(&s->falpha, nb * sizeof(float));
  dalloc(&s->fbeta, nb * sizeof(float));
  dalloc(&s->fchi2, nb * sizeof(float));
  dalloc(&s->fstate, nb * sizeof(int32_t));
  dalloc(&s->fiters, nb * sizeof(int32_t));
  dalloc(&s->results, nb * FS_SERVE_RESULT_FLOATS * sizeof(float));
  dalloc(&s->desc, (1 + 2 * (size_t)c.max_batch) * sizeof(int32_t));
  dalloc(&s->ws, fit_spots_uniform_workspace());
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void **>(&s->h_desc),
                      (size_t)c.max_inflight * (1 + 2 * c.max_batch) * sizeof(int32_t), 0);
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void **>(&s->h_results),
                      (size_t)c.max_inflight * nb * FS_SERVE_RESULT_FLOATS * sizeof(float), 0);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
  s->slot_ready.assign(c.frame_slots, nullptr);
  s->buf_done.assign(c.max_inflight, nullptr);
  for (auto &ev : s->slot_ready)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  for (auto &ev : s->buf_done)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->state, 0, (size_t)c.streams * c.markers * 16, s->compute);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(s->desc, 0, (1 + 2 * (size_t)c.max_batch) * sizeof(int32_t), s->compute);
  int rc = FS_OK;
  // warm-up outside capture (the fit's one-time attribute set-up), then one graph per size;
  // a zero descriptor count makes every kernel of the warm-up return at once
  for (int k = 1; k <= c.max_batch && e == cudaSuccess && rc == FS_OK; ++k) rc = session_step(s, k);
  if (e == cudaSuccess && rc == FS_OK) e = cudaStreamSynchronize(s->compute);
  s->graphs.assign(c.max_batch, nullptr);
  for (int k = 1; k <= c.max_batch && e == cudaSuccess && rc == FS_OK; ++k) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(s->compute, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    rc = session_step(s, k);
    const cudaError_t e2 = cudaStreamEndCapture(s->compute, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && rc == FS_OK) e = cudaGraphInstantiate(&s->graphs[k - 1], g, 0);
    if (g) cudaGraphDestroy(g);
  }
  if (e != cudaSuccess || rc != FS_OK) {
    session_free(s);
    return e != cudaSuccess ? FS_ERR_CUDA : rc;
  }
  for (int i = 0; i < c.frame_slots; ++i) s->free_slots.push_back(i);
  for (int i = 0; i < c.max_inflight; ++i) s->free_bufs.push_back(i);
  s->busy.assign(c.streams, 0);
  *out = s;
  return FS_OK;
}

int fs_session_destroy(fs_session *s) {
  if (!s) return FS_ERR_NULL;
  session_free(s);
  return FS_OK;
}

int fs_session_add_markers(fs_session *s, int stream, const float *host_state) {
  if (!s || !host_state) return FS_ERR_NULL;
  if (stream < 0 || stream >= s->cfg.streams) return FS_ERR_ARG;
  const size_t bytes = (size_t)s->cfg.markers * 4 * sizeof(float);
  cudaError_t e = cudaMemcpyAsync(s->state + (size_t)stream * s->cfg.markers * 4, host_state, bytes,
                                  cudaMemcpyHostToDevice, s->compute);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->compute);
  return e == cudaSuccess ? FS_OK : cuda_fail(s, e);
}

int fs_session_get_markers(fs_session *s, int stream, float *host_state) {
  if (!s || !host_state) return FS_ERR_NULL;
  if (stream < 0 || stream >= s->cfg.streams) return FS_ERR_ARG;
  const size_t bytes = (size_t)s->cfg.markers * 4 * sizeof(float);
  cudaError_t e = cudaMemcpyAsync(host_state, s->state + (size_t)stream * s->cfg.markers * 4, bytes,
                                  cudaMemcpyDeviceToHost, s->compute);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->compute);
  return e == cudaSuccess ? FS_OK : cuda_fail(s, e);
}

int fs_session_submit_frame(fs_session *s, int stream, int64_t index, const uint16_t *host_frame,
                            double t_arrival) {
  if (!s || !host_frame) return FS_ERR_NULL;
  if (stream < 0 || stream >= s->cfg.streams) return FS_ERR_ARG;
  if ((int64_t)s->pending.size() >= s->cfg.queue_limit) {
    ++s->dropped;
    return FS_ERR_FULL;
  }
  s->pending.push_back({stream, index, t_arrival, host_frame, -1});
  return FS_OK;
}

int fs_session_poll(fs_session *s, fs_frame_done *done, float *results, int max_frames,
                    int *n_done) {
  if (!s || !n_done || (max_frames > 0 && (!done || !results))) return FS_ERR_NULL;
  if (max_frames < 0) return FS_ERR_ARG;
  *n_done = 0;
  const fs_session_config &c = s->cfg;
  const size_t fbytes = frame_elems(c) * sizeof(uint16_t);
  const size_t nb = batch_spots(c);
  cudaError_t e = cudaSuccess;
  // 1. admission: free frame slots (the memory budget) take waiting frames
  while (!s->pending.empty() && !s->free_slots.empty()) {
    auto fr = s->pending.front();
    s->pending.pop_front();
    fr.slot = s->free_slots.front();
    s->free_slots.pop_front();
    if ((e = cudaMemcpyAsync(s->frames + (size_t)fr.slot * frame_elems(c), fr.host, fbytes,
                             cudaMemcpyHostToDevice, s->copy)) != cudaSuccess ||
        (e = cudaEventRecord(s->slot_ready[fr.slot], s->copy)) != cudaSuccess)
      return cuda_fail(s, e);
    s->landed.push_back(fr);
  }
  // 2. launch: one frame per stream, oldest first, among frames already on the device
  if (!s->landed.empty() && !s->free_bufs.empty()) {
    fs_session::Batch b;
    std::vector<size_t> take;
    std::vector<char> chosen(c.streams, 0);
    for (size_t i = 0; i < s->landed.size() && (int)take.size() < c.max_batch; ++i) {
      const auto &fr = s->landed[i];
      if (chosen[fr.stream] || s->busy[fr.stream]) continue;
      const cudaError_t q = cudaEventQuery(s->slot_ready[fr.slot]);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return cuda_fail(s, q);
      chosen[fr.stream] = 1;
      take.push_back(i);
    }
    if (!take.empty()) {
      const int k = (int)take.size();
      b.buf = s->free_bufs.front();
      s->free_bufs.pop_front();
      int32_t *hd = s->h_desc + (size_t)b.buf * (1 + 2 * c.max_batch);
      hd[0] = k;
      for (int j = 0; j < k; ++j) {
        const auto &fr = s->landed[take[j]];
        hd[1 + 2 * j] = fr.slot;
        hd[2 + 2 * j] = fr.stream;
        b.frames.push_back(fr);
        s->busy[fr.stream] = 1;
        if ((e = cudaStreamWaitEvent(s->compute, s->slot_ready[fr.slot], 0)) != cudaSuccess)
          return cuda_fail(s, e);
      }
      for (int j = k - 1; j >= 0; --j) s->landed.erase(s->landed.begin() + take[j]);
      float *hr = s->h_results + (size_t)b.buf * nb * FS_SERVE_RESULT_FLOATS;
      if ((e = cudaMemcpyAsync(s->desc, hd, (1 + 2 * (size_t)c.max_batch) * sizeof(int32_t),
                               cudaMemcpyHostToDevice, s->compute)) != cudaSuccess ||
          (e = cudaGraphLaunch(s->graphs[k - 1], s->compute)) != cudaSuccess ||
          (e = cudaMemcpyAsync(hr, s->results, (size_t)k * c.markers * FS_SERVE_RESULT_FLOATS *
                                                   sizeof(float),
                               cudaMemcpyDeviceToHost, s->compute)) != cudaSuccess ||
          (e = cudaEventRecord(s->buf_done[b.buf], s->compute)) != cudaSuccess)
        return cuda_fail(s, e);
      s->inflight.push_back(std::move(b));
      ++s->batches;
    }
  }
  // 3. retire finished batches, oldest first, while the caller's arrays have room
  while (!s->inflight.empty()) {
    auto &b = s->inflight.front();
    if (*n_done + (int)b.frames.size() > max_frames) break;
    const cudaError_t q = cudaEventQuery(s->buf_done[b.buf]);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) return cuda_fail(s, q);
    const double t = fs_session_clock();
    const float *hr = s->h_results + (size_t)b.buf * nb * FS_SERVE_RESULT_FLOATS;
    const size_t per = (size_t)c.markers * FS_SERVE_RESULT_FLOATS;
    for (size_t j = 0; j < b.frames.size(); ++j) {
      const auto &fr = b.frames[j];
      fs_frame_done &d = done[*n_done];
      d.stream = fr.stream;
      d.reserved = 0;
      d.index = fr.index;
      d.t_arrival = fr.t_arrival;
      d.t_done = t;
      std::copy(hr + j * per, hr + (j + 1) * per, results + (size_t)(*n_done) * per);
      ++*n_done;
      s->free_slots.push_back(fr.slot);
      s->busy[fr.stream] = 0;
      ++s->served;
    }
    s->free_bufs.push_back(b.buf);
    s->inflight.pop_front();
  }
  return FS_OK;
}

int fs_session_pending(const fs_session *s) {
  if (!s) return FS_ERR_NULL;
  size_t n = s->pending.size() + s->landed.size();
  for (const auto &b : s->inflight) n += b.frames.size();
  return (int)n;
}

int fs_session_stats(const fs_session *s, int64_t *dropped, int64_t *served, int64_t *batches) {
  if (!s) return FS_ERR_NULL;
  if (dropped) *dropped = s->dropped;
  if (served) *served = s->served;
  if (batches) *batches = s->batches;
  return FS_OK;
}

}  // extern "C"
