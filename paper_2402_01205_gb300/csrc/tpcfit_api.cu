// C-ABI runtime of the batched TPC Kalman track fit: handles, device scratch
// pools, streams and events, the blocking and asynchronous fit paths, and the
// chunked host-frame pipeline (host->device copy, fit and device->host copy of
// consecutive chunks overlapped on three streams).
//
// Declarations and contracts: include/tpcfit.h.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "tpcfit.h"
#include "tpcfit_internal.h"

using namespace tpcfit;

// ----------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------
static thread_local char g_errmsg[512] = "";

static int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_errmsg, sizeof(g_errmsg), fmt, ap);
  va_end(ap);
  return code;
}

#define CU(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return fail(TPCFIT_E_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                         \
  } while (0)

extern "C" const char *tpcfit_strerror(int code) {
  switch (code) {
    case TPCFIT_OK: return "ok";
    case TPCFIT_E_INVAL: return "invalid argument or malformed frame";
    case TPCFIT_E_NOMEM: return "out of device memory or over the HBM budget";
    case TPCFIT_E_CUDA: return "CUDA runtime error";
    case TPCFIT_E_TIMEOUT: return "timed out";
    case TPCFIT_E_BUSY: return "busy";
    case TPCFIT_E_NOTFOUND: return "unknown ticket";
    case TPCFIT_E_NODEV: return "no usable CUDA device (sm_103 required)";
    default: return "unknown error";
  }
}

extern "C" const char *tpcfit_last_error_message(void) { return g_errmsg; }

namespace tpcfit {
int set_error_message(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace tpcfit

extern "C" double tpcfit_now(void) {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// ----------------------------------------------------------------------------
// device buffers
// ----------------------------------------------------------------------------
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  // grow to at least `bytes`; the caller guarantees no work in flight uses it
  int ensure(size_t bytes) {
    if (bytes <= cap) return TPCFIT_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = bytes + bytes / 8 + 4096;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return fail(TPCFIT_E_NOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    cap = want;
    return TPCFIT_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <class T> T *as(size_t byte_off = 0) const { return reinterpret_cast<T *>((char *)p + byte_off); }
};

static inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Scratch of one launch sequence: seed, permutation, histogram/cursors, work
// counter and frame-error word, carved from one allocation.
struct Scratch {
  DevBuf buf;
  DevBuf pred;  // the smoother's forward predictions (allocated on its first use)
  float *seed = nullptr;
  int32_t *perm = nullptr;
  uint32_t *hist = nullptr;  // 2*kKeyBins
  unsigned long long *work = nullptr;
  int32_t *err = nullptr;
  size_t small_bytes = 0;  // hist+work+err (zeroed per launch sequence)
  static size_t small_size() { return align256(2 * kKeyBins * sizeof(uint32_t) + 16 + 16); }
  static size_t bytes_for(int64_t nt) {
    return small_size() + align256((size_t)nt * 5 * sizeof(float)) + align256((size_t)nt * sizeof(int32_t));
  }
  // point the fields into `base` (at least bytes_for(nt) bytes)
  void layout(char *base, int64_t nt) {
    hist = reinterpret_cast<uint32_t *>(base);
    work = reinterpret_cast<unsigned long long *>(base + 2 * kKeyBins * sizeof(uint32_t));
    err = reinterpret_cast<int32_t *>(base + 2 * kKeyBins * sizeof(uint32_t) + 16);
    small_bytes = small_size();
    seed = reinterpret_cast<float *>(base + small_bytes);
    perm = reinterpret_cast<int32_t *>(base + small_bytes + align256((size_t)nt * 5 * sizeof(float)));
  }
  int ensure(int64_t nt) {
    int rc = buf.ensure(bytes_for(nt));
    if (rc) return rc;
    layout(buf.as<char>(), nt);
    return TPCFIT_OK;
  }
};

// Device copy of one chunk of a host frame (inputs and results).
struct Stage {
  DevBuf buf;
  int64_t *off = nullptr;
  float *x = nullptr, *y = nullptr, *z = nullptr, *sy2 = nullptr, *sz2 = nullptr;
  uint8_t *row = nullptr;
  float *state = nullptr, *cov = nullptr, *xref = nullptr;
  double *chi2 = nullptr;
  int32_t *ndf = nullptr, *status = nullptr;
  uint8_t *accept = nullptr;
  int16_t *res_y = nullptr, *res_z = nullptr;
  cudaEvent_t free_ev = nullptr;  // recorded after the results left this stage
  int ensure(int64_t nt, int64_t nc) {
    size_t o = 0;
    size_t off_o = o; o += align256((size_t)(nt + 1) * 8);
    size_t x_o = o; o += align256((size_t)nc * 4);
    size_t y_o = o; o += align256((size_t)nc * 4);
    size_t z_o = o; o += align256((size_t)nc * 4);
    size_t sy_o = o; o += align256((size_t)nc * 4);
    size_t sz_o = o; o += align256((size_t)nc * 4);
    size_t row_o = o; o += align256((size_t)nc);
    size_t st_o = o; o += align256((size_t)nt * 20);
    size_t cv_o = o; o += align256((size_t)nt * 60);
    size_t xr_o = o; o += align256((size_t)nt * 4);
    size_t c2_o = o; o += align256((size_t)nt * 8);
    size_t nd_o = o; o += align256((size_t)nt * 4);
    size_t ss_o = o; o += align256((size_t)nt * 4);
    size_t ac_o = o; o += align256((size_t)nc);
    size_t ry_o = o; o += align256((size_t)nc * 2);
    size_t rz_o = o; o += align256((size_t)nc * 2);
    int rc = buf.ensure(o);
    if (rc) return rc;
    off = buf.as<int64_t>(off_o);
    x = buf.as<float>(x_o); y = buf.as<float>(y_o); z = buf.as<float>(z_o);
    sy2 = buf.as<float>(sy_o); sz2 = buf.as<float>(sz_o); row = buf.as<uint8_t>(row_o);
    state = buf.as<float>(st_o); cov = buf.as<float>(cv_o); xref = buf.as<float>(xr_o);
    chi2 = buf.as<double>(c2_o); ndf = buf.as<int32_t>(nd_o); status = buf.as<int32_t>(ss_o);
    accept = buf.as<uint8_t>(ac_o);
    res_y = buf.as<int16_t>(ry_o);
    res_z = buf.as<int16_t>(rz_o);
    return TPCFIT_OK;
  }
};

// ----------------------------------------------------------------------------
// serving state (declared here, implemented in tpcfit_serve.cu)
// ----------------------------------------------------------------------------
struct ServeState;
int serve_start(tpcfit_handle *h);
void serve_stop(tpcfit_handle *h);
int serve_submit(tpcfit_handle *h, const tpcfit_frame *f, tpcfit_result *r, uint64_t *ticket);
int serve_poll(tpcfit_handle *h, uint64_t ticket, int *state, double *t_done, double timeout_s, bool wait);
int serve_stats(tpcfit_handle *h, tpcfit_serve_stats *out);

struct tpcfit_handle {
  tpcfit_config cfg;
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;  // fit kernels
  cudaStream_t h2d = nullptr, d2h = nullptr;
  float *d_rowx = nullptr;
  Scratch scratch;
  Stage stage[2];
  DevBuf rans_buf;           // rANS codec scratch
  DevBuf follow_buf;         // track-following scratch (cell grid)
  int32_t *h_err = nullptr;  // pinned
  // ring of event quadruples around prepare / sort / fit of timed calls
  static constexpr int kRing = 64;
  struct TimedCall {
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool pending = false;
    int launches = 0;
  } ring[kRing];
  int ring_pos = 0;
  int last_slot = -1;
  int fit_regs = 0;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_fit[2] = {nullptr, nullptr};
  int last_launches = 0;
  tpcfit_timing timing{};
  int fit_grid = 0, fit_block = 128;
  int64_t chunk_clusters = 16 << 20;
  ServeState *serve = nullptr;
  std::mutex mu;  // serialises fit paths with the serving worker
};

// exposed to the serving runtime
FitArgs make_args(tpcfit_handle *h, const tpcfit_frame *f, const tpcfit_result *r, Scratch &s, int64_t off_base);
int run_sequence(tpcfit_handle *h, const FitArgs &a, cudaStream_t st, Scratch &s, bool timed, int *launches);
cudaStream_t handle_stream(tpcfit_handle *h) { return h->stream; }
int64_t handle_chunk_clusters(tpcfit_handle *h) { return h->chunk_clusters; }
size_t serve_scratch_bytes(int64_t n_tracks) { return Scratch::bytes_for(n_tracks); }
int serve_prepare_frame(tpcfit_handle *h, const tpcfit_frame *f, tpcfit_result *r, void *scratch_base,
                        int64_t off_base, cudaStream_t st, FitArgs *args, const int32_t **err_dev);
int handle_device(tpcfit_handle *h) { return h->device; }
// exposed to the rANS codec (tpcfit_rans.cu)
int handle_rans_scratch(tpcfit_handle *h, size_t bytes, void **p) {
  int rc = h->rans_buf.ensure(bytes);
  if (rc) return rc;
  *p = h->rans_buf.p;
  return TPCFIT_OK;
}
int handle_follow_scratch(tpcfit_handle *h, size_t bytes, void **p) {
  if (bytes > h->follow_buf.cap) CU(cudaDeviceSynchronize());  // growing frees the old buffer
  int rc = h->follow_buf.ensure(bytes);
  if (rc) return rc;
  *p = h->follow_buf.p;
  return TPCFIT_OK;
}
int32_t *handle_pinned_word(tpcfit_handle *h) { return h->h_err; }
int report_error(int code, const char *msg) { return fail(code, "%s", msg); }
const tpcfit_config &handle_config(tpcfit_handle *h) { return h->cfg; }
ServeState *&handle_serve(tpcfit_handle *h) { return h->serve; }
std::mutex &handle_mutex(tpcfit_handle *h) { return h->mu; }
int handle_fit_grid(tpcfit_handle *h) { return h->fit_grid; }
int handle_fit_block(tpcfit_handle *h) { return h->fit_block; }
const float *handle_rowx(tpcfit_handle *h) { return h->d_rowx; }

// ----------------------------------------------------------------------------
// config and handle
// ----------------------------------------------------------------------------
extern "C" void tpcfit_default_config(tpcfit_config *c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->bz_tesla = 0.5f;
  c->chi2_max = 16.0f;
  c->xx0_per_row = 5e-4f;
  c->mass_gev = 0.13957f;
  c->snp_max = 0.999f;
  c->seed_cov[0] = 1.0f;
  c->seed_cov[1] = 1.0f;
  c->seed_cov[2] = 0.01f;
  c->seed_cov[3] = 0.01f;
  c->seed_cov[4] = 1.0f;
  c->restart_scale = 100.0f;
  c->reseed_pct = 50;
  c->min_clusters = 10;
  c->n_rows = 152;
  c->row_x0_cm = 85.0f;
  c->row_pitch_cm = (float)(162.0 / 151.0);
  c->hbm_budget_bytes = 120ull << 30;
  c->max_slots = 8;
  c->device = 0;
  c->block_threads = 0;
  c->blocks_per_sm = 0;
  c->sort_tracks = 1;
  c->res_step_y_cm = 0.01f;
  c->res_step_z_cm = 0.01f;
  c->host_chunk_clusters = (int64_t)16 << 20;
}

static int check_config(const tpcfit_config &c) {
  if (!(c.bz_tesla != 0.0f) || !(c.chi2_max > 0.0f) || !(c.xx0_per_row >= 0.0f) || !(c.mass_gev >= 0.0f) ||
      !(c.snp_max > 0.0f && c.snp_max < 1.0f) || !(c.restart_scale > 0.0f))
    return fail(TPCFIT_E_INVAL, "fit parameter out of range");
  for (int i = 0; i < 5; ++i)
    if (!(c.seed_cov[i] > 0.0f)) return fail(TPCFIT_E_INVAL, "seed_cov[%d] must be > 0", i);
  if (c.n_rows < 1 || c.n_rows > kMaxRows) return fail(TPCFIT_E_INVAL, "n_rows must be in [1, %d]", kMaxRows);
  if (c.min_clusters < 0) return fail(TPCFIT_E_INVAL, "min_clusters < 0");
  if (c.max_slots < 1 || c.max_slots > 64) return fail(TPCFIT_E_INVAL, "max_slots must be in [1, 64]");
  if (c.block_threads != 0 && c.block_threads != 128 && c.block_threads != 256)
    return fail(TPCFIT_E_INVAL, "block_threads must be 0, 128 or 256");
  if (c.blocks_per_sm < 0) return fail(TPCFIT_E_INVAL, "blocks_per_sm < 0");
  if (!(c.res_step_y_cm > 0.0f) || !(c.res_step_z_cm > 0.0f)) return fail(TPCFIT_E_INVAL, "residual steps must be > 0");
  if (const char *why = check_variant_params(c)) return fail(TPCFIT_E_INVAL, "%s", why);
  return TPCFIT_OK;
}

extern "C" int tpcfit_create(const tpcfit_config *cfg_in, tpcfit_handle **out) {
  if (!out) return fail(TPCFIT_E_INVAL, "out is NULL");
  tpcfit_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else tpcfit_default_config(&cfg);
  int rc = check_config(cfg);
  if (rc) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= cfg.device || cfg.device < 0) {
    cudaGetLastError();
    return fail(TPCFIT_E_NODEV, "CUDA device %d not available", cfg.device);
  }
  cudaDeviceProp prop;
  CU(cudaGetDeviceProperties(&prop, cfg.device));
  if (prop.major != 10 || prop.minor != 3)
    return fail(TPCFIT_E_NODEV, "device %d is sm_%d%d; this library is built for sm_103a", cfg.device, prop.major,
                prop.minor);
  CU(cudaSetDevice(cfg.device));
  tpcfit_handle *h = new tpcfit_handle();
  h->cfg = cfg;
  h->device = cfg.device;
  h->sms = prop.multiProcessorCount;
  auto cleanup = [&](int code) {
    tpcfit_destroy(h);
    return code;
  };
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking) != cudaSuccess)
    return cleanup(fail(TPCFIT_E_CUDA, "stream creation failed"));
  for (auto &tc : h->ring)
    for (auto &e : tc.ev)
      if (cudaEventCreate(&e) != cudaSuccess) return cleanup(fail(TPCFIT_E_CUDA, "event creation failed"));
  for (int i = 0; i < 2; ++i) {
    if (cudaEventCreateWithFlags(&h->ev_in[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fit[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->stage[i].free_ev, cudaEventDisableTiming) != cudaSuccess)
      return cleanup(fail(TPCFIT_E_CUDA, "event creation failed"));
  }
  if (cudaMallocHost(&h->h_err, sizeof(int32_t)) != cudaSuccess) return cleanup(fail(TPCFIT_E_CUDA, "pinned alloc"));
  // pad-row plane positions, float-rounded from double like the frames store them
  float rowx[kMaxRows];
  for (int r = 0; r < kMaxRows; ++r)
    rowx[r] = (float)((double)cfg.row_x0_cm + (double)r * (double)cfg.row_pitch_cm);
  if (cfg.row_x0_cm == 85.0f && cfg.row_pitch_cm == (float)(162.0 / 151.0))
    for (int r = 0; r < kMaxRows; ++r) rowx[r] = (float)(85.0 + (double)r * (162.0 / 151.0));
  if (cudaMalloc(&h->d_rowx, sizeof(rowx)) != cudaSuccess ||
      cudaMemcpy(h->d_rowx, rowx, sizeof(rowx), cudaMemcpyHostToDevice) != cudaSuccess)
    return cleanup(fail(TPCFIT_E_NOMEM, "row table allocation failed"));
  // default shape: 128 threads x 5 blocks per SM for the plain fit (640 tracks
  // per SM; 2 % faster than 4 blocks on the Pb-Pb frame, 6.70 against 6.84 ms),
  // 4 for the variant; 128 x 4 was 0.8 % faster than 256 x 2
  h->fit_block = cfg.block_threads ? cfg.block_threads : 128;
  const bool variant = cfg.xrho_per_row > 0.0f || cfg.fit_iterations > 0;
  const int bps = cfg.blocks_per_sm > 0 ? cfg.blocks_per_sm : fit_default_blocks_per_sm(h->fit_block, variant);
  h->fit_grid = h->sms * bps;
  h->fit_regs = fit_regs_per_thread(h->fit_block, variant, bps);
  h->chunk_clusters = cfg.host_chunk_clusters > 0 ? cfg.host_chunk_clusters : (int64_t)16 << 20;
  *out = h;
  return TPCFIT_OK;
}

extern "C" int tpcfit_destroy(tpcfit_handle *h) {
  if (!h) return fail(TPCFIT_E_INVAL, "handle is NULL");
  cudaSetDevice(h->device);
  if (h->serve) serve_stop(h);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->h2d) cudaStreamSynchronize(h->h2d);
  if (h->d2h) cudaStreamSynchronize(h->d2h);
  h->scratch.buf.release();
  h->scratch.pred.release();
  h->rans_buf.release();
  h->follow_buf.release();
  for (auto &s : h->stage) {
    s.buf.release();
    if (s.free_ev) cudaEventDestroy(s.free_ev);
  }
  for (auto &tc : h->ring)
    for (auto &e : tc.ev)
      if (e) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i) {
    if (h->ev_in[i]) cudaEventDestroy(h->ev_in[i]);
    if (h->ev_fit[i]) cudaEventDestroy(h->ev_fit[i]);
  }
  if (h->d_rowx) cudaFree(h->d_rowx);
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->stream) cudaStreamDestroy(h->stream);
  if (h->h2d) cudaStreamDestroy(h->h2d);
  if (h->d2h) cudaStreamDestroy(h->d2h);
  delete h;
  return TPCFIT_OK;
}

// ----------------------------------------------------------------------------
// one launch sequence
// ----------------------------------------------------------------------------
FitArgs make_args(tpcfit_handle *h, const tpcfit_frame *f, const tpcfit_result *r, Scratch &s, int64_t off_base) {
  FitArgs a;
  std::memset(&a, 0, sizeof(a));
  const tpcfit_config &c = h->cfg;
  a.n_tracks = f->n_tracks;
  a.n_clusters = f->n_clusters;
  a.off = f->track_offsets;
  a.off_base = off_base;
  a.x = f->x; a.y = f->y; a.z = f->z; a.sy2 = f->sy2; a.sz2 = f->sz2; a.row = f->row;
  a.state = r->state; a.cov = r->cov; a.x_ref = r->x_ref; a.chi2 = r->chi2;
  a.ndf = r->ndf; a.status = r->status; a.accept = r->accept;
  a.chi2_out_c = r->chi2_out_cluster;
  a.chi2_in_c = r->chi2_in_cluster;
  a.restart_state = r->restart_state;
  a.sm_state = r->smoothed_state;
  a.sm_cov = r->smoothed_cov;
  a.res_y = r->res_y;
  a.res_z = r->res_z;
  a.res_inv_step_y = 1.0f / c.res_step_y_cm;
  a.res_inv_step_z = 1.0f / c.res_step_z_cm;
  a.seed = s.seed;
  a.perm = c.sort_tracks ? s.perm : nullptr;
  a.hist = s.hist;
  a.work = s.work;
  a.frame_error = s.err;
  a.row_x = h->d_rowx;
  fit_params(a, c);
  return a;
}

// Fold a completed timed call into the timing record.
static void fold_timing(tpcfit_handle *h, int slot) {
  auto &tc = h->ring[slot];
  if (!tc.pending) return;
  cudaEventSynchronize(tc.ev[3]);
  float a = 0, b = 0, c = 0, t = 0;
  cudaEventElapsedTime(&a, tc.ev[0], tc.ev[1]);
  cudaEventElapsedTime(&b, tc.ev[1], tc.ev[2]);
  cudaEventElapsedTime(&c, tc.ev[2], tc.ev[3]);
  cudaEventElapsedTime(&t, tc.ev[0], tc.ev[3]);
  cudaGetLastError();
  tc.pending = false;
  tpcfit_timing &T = h->timing;
  if (slot == h->last_slot) {
    T.prepare_ms = a;
    T.sort_ms = b;
    T.fit_ms = c;
    T.total_ms = t;
    T.kernel_launches = tc.launches;
  }
  T.prepare_ms_sum += a;
  T.sort_ms_sum += b;
  T.fit_ms_sum += c;
  T.total_ms_sum += t;
  T.n_timed += 1;
  T.fit_grid = h->fit_grid;
  T.fit_block = h->fit_block;
  T.fit_regs = h->fit_regs;
}

// Enqueue prepare, sort and fit of one frame on `st`.  The scratch's small
// region (histogram, work counter, error word) must be zeroed by the caller.
int run_sequence(tpcfit_handle *h, const FitArgs &a, cudaStream_t st, Scratch &s, bool timed, int *launches) {
  (void)s;
  int slot = -1;
  if (timed) {
    slot = h->ring_pos;
    h->ring_pos = (h->ring_pos + 1) % tpcfit_handle::kRing;
    fold_timing(h, slot);  // a call 64 timed calls old: long complete
    h->last_slot = slot;
    CU(cudaEventRecord(h->ring[slot].ev[0], st));
  }
  int l = 0;
  CU(launch_prepare(a, st));
  l += 1;
  if (timed) CU(cudaEventRecord(h->ring[slot].ev[1], st));
  CU(launch_sort(a, st, &l));
  if (timed) CU(cudaEventRecord(h->ring[slot].ev[2], st));
  if (a.sm_state) CU(launch_smooth(a, smooth_grid(), st));
  else CU(launch_fit(a, h->fit_grid, h->fit_block, st));
  l += 1;
  if (a.res_y || a.res_z) {
    CU(launch_residuals(a, st));
    l += 1;
  }
  if (timed) {
    CU(cudaEventRecord(h->ring[slot].ev[3], st));
    h->ring[slot].pending = true;
    h->ring[slot].launches = l;
  }
  if (launches) *launches += l;
  return TPCFIT_OK;
}

// Fit of one resident serving frame (or part of a frame, whose offsets start
// at off_base) on a slot stream; scratch lives in the slot's allocation.
// Serving: the checks, seeds and sort of one resident part on `st`; *args
// receives the part's fit arguments for the serving engine's launch.
int serve_prepare_frame(tpcfit_handle *h, const tpcfit_frame *f, tpcfit_result *r, void *scratch_base,
                        int64_t off_base, cudaStream_t st, FitArgs *args, const int32_t **err_dev) {
  Scratch s;
  s.layout((char *)scratch_base, f->n_tracks);
  CU(cudaMemsetAsync(s.hist, 0, s.small_bytes, st));
  FitArgs a = make_args(h, f, r, s, off_base);
  CU(launch_prepare(a, st));
  CU(launch_sort(a, st, nullptr));
  *args = fit_args_for_launch(a);
  *err_dev = s.err;
  return TPCFIT_OK;
}

static int check_frame_shape(const tpcfit_frame *f, const tpcfit_result *r) {
  if (!f || !r) return fail(TPCFIT_E_INVAL, "frame or result is NULL");
  if (f->n_tracks < 0 || f->n_clusters < 0) return fail(TPCFIT_E_INVAL, "negative size");
  if (f->n_tracks > (int64_t)INT32_MAX - 64) return fail(TPCFIT_E_INVAL, "n_tracks above 2^31-64");
  if (!f->track_offsets) return fail(TPCFIT_E_INVAL, "track_offsets is NULL");
  if (f->n_clusters > 0 && (!f->y || !f->z || !f->sy2 || !f->sz2 || !f->row))
    return fail(TPCFIT_E_INVAL, "cluster array is NULL");
  if (f->n_clusters > 0 && !f->x && f->mem != TPCFIT_MEM_HOST)
    return fail(TPCFIT_E_INVAL, "x may be NULL only in a host frame (clusters on their pad-row planes)");
  if (f->n_tracks > 0 && (!r->state || !r->cov || !r->x_ref || !r->chi2 || !r->ndf || !r->status))
    return fail(TPCFIT_E_INVAL, "result array is NULL");
  if (f->n_clusters > 0 && !r->accept) return fail(TPCFIT_E_INVAL, "accept is NULL");
  if ((f->mem != TPCFIT_MEM_HOST && f->mem != TPCFIT_MEM_DEVICE) ||
      (r->mem != TPCFIT_MEM_HOST && r->mem != TPCFIT_MEM_DEVICE))
    return fail(TPCFIT_E_INVAL, "mem must be TPCFIT_MEM_HOST or TPCFIT_MEM_DEVICE");
  if (!r->smoothed_state != !r->smoothed_cov)
    return fail(TPCFIT_E_INVAL, "the smoother writes both smoothed_state and smoothed_cov");
  return TPCFIT_OK;
}

// The smoother variant (smoothed outputs requested) takes neither energy loss
// nor seed iteration.
static int check_smoother(const tpcfit_handle *h, const tpcfit_result *r) {
  if (r->smoothed_state && (h->cfg.xrho_per_row > 0.0f || h->cfg.fit_iterations > 0))
    return fail(TPCFIT_E_INVAL, "the smoother takes neither energy loss nor seed iteration");
  return TPCFIT_OK;
}

static int wait_stream(cudaStream_t s, double timeout_s) {
  if (timeout_s < 0) {
    CU(cudaStreamSynchronize(s));
    return TPCFIT_OK;
  }
  const double t0 = tpcfit_now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) return TPCFIT_OK;
    if (e != cudaErrorNotReady) return fail(TPCFIT_E_CUDA, "stream: %s", cudaGetErrorString(e));
    if (tpcfit_now() - t0 > timeout_s) return fail(TPCFIT_E_TIMEOUT, "stream wait exceeded %.3f s", timeout_s);
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// The smoother's prediction scratch of `s` (sized by the smoother's grid and
// the handle's pad rows, fixed per handle: allocated once) into a.sm_pred.
static int smoother_scratch(tpcfit_handle *h, Scratch &s, FitArgs &a) {
  const int grid = smooth_grid();
  if (grid <= 0) return fail(TPCFIT_E_CUDA, "smoother grid");
  int rc = s.pred.ensure(smooth_pred_bytes(grid, h->cfg.n_rows));
  if (rc) return rc;
  a.sm_pred = s.pred.as<float>();
  return TPCFIT_OK;
}

// device frame -> device results on stream st
static int fit_device(tpcfit_handle *h, const tpcfit_frame *f, tpcfit_result *r, cudaStream_t st) {
  int rc = h->scratch.ensure(f->n_tracks);
  if (rc) return rc;
  CU(cudaMemsetAsync(h->scratch.hist, 0, h->scratch.small_bytes, st));
  FitArgs a = make_args(h, f, r, h->scratch, 0);
  if (a.sm_state && (rc = smoother_scratch(h, h->scratch, a))) return rc;
  int launches = 0;
  rc = run_sequence(h, a, st, h->scratch, true, &launches);
  if (rc) return rc;
  CU(cudaMemcpyAsync(h->h_err, h->scratch.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  h->last_launches = launches;
  return TPCFIT_OK;
}

// ----------------------------------------------------------------------------
// batched events: one captured launch sequence, replayed
// ----------------------------------------------------------------------------
struct tpcfit_batch {
  tpcfit_handle *h = nullptr;
  int device = 0;
  Scratch scratch;
  cudaStream_t stream = nullptr;  // capture stream and default replay stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;  // recorded after the latest replay
  int32_t *h_err = nullptr;    // pinned; the latest replay's frame-error word
  int launches = 0;            // kernels per replay
};

static void batch_free(tpcfit_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->done) cudaEventDestroy(b->done);
  if (b->stream) cudaStreamDestroy(b->stream);
  if (b->h_err) cudaFreeHost(b->h_err);
  b->scratch.buf.release();
  b->scratch.pred.release();
  delete b;
}

extern "C" int tpcfit_batch_create(tpcfit_handle *h, const tpcfit_frame *f, tpcfit_result *r, tpcfit_batch **out) {
  if (!h || !out) return fail(TPCFIT_E_INVAL, "handle or out is NULL");
  int rc = check_frame_shape(f, r);
  if (rc) return rc;
  if ((rc = check_smoother(h, r))) return rc;
  if (f->mem != TPCFIT_MEM_DEVICE || r->mem != TPCFIT_MEM_DEVICE)
    return fail(TPCFIT_E_INVAL, "a batch takes a device frame and device results");
  CU(cudaSetDevice(h->device));
  tpcfit_batch *b = new tpcfit_batch();
  b->h = h;
  b->device = h->device;
  auto bail = [&](int code) {
    if (b->stream) {
      cudaStreamCaptureStatus cs;
      if (cudaStreamIsCapturing(b->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(b->stream, &g);
        if (g) cudaGraphDestroy(g);
      }
    }
    cudaGetLastError();
    batch_free(b);
    return code;
  };
  if ((rc = b->scratch.ensure(std::max<int64_t>(f->n_tracks, 1)))) return bail(rc);
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&b->h_err, sizeof(int32_t)) != cudaSuccess)
    return bail(fail(TPCFIT_E_CUDA, "batch stream, event or pinned word"));
  *b->h_err = 0;
  // set the kernel attributes before capture (no such calls inside it)
  FitArgs a = make_args(h, f, r, b->scratch, 0);
  if (a.sm_state && (rc = smoother_scratch(h, b->scratch, a))) return bail(rc);
  if (fit_set_attributes(a, h->fit_block) != cudaSuccess) return bail(fail(TPCFIT_E_CUDA, "fit kernel attributes"));
  const int sgrid = a.sm_state ? smooth_grid() : 0;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bail(fail(TPCFIT_E_CUDA, "begin capture: %s", cudaGetErrorString(e)));
  int l = 0;
  if ((e = cudaMemsetAsync(b->scratch.hist, 0, b->scratch.small_bytes, b->stream)) != cudaSuccess ||
      (e = launch_prepare(a, b->stream)) != cudaSuccess || (e = launch_sort(a, b->stream, &l)) != cudaSuccess ||
      (e = (a.sm_state ? launch_smooth(a, sgrid, b->stream) : launch_fit(a, h->fit_grid, h->fit_block, b->stream))) !=
          cudaSuccess ||
      (e = launch_residuals(a, b->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b->h_err, b->scratch.err, sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream)) !=
          cudaSuccess)
    return bail(fail(TPCFIT_E_CUDA, "capture: %s", cudaGetErrorString(e)));
  if (f->n_tracks > 0) l += 2 + ((r->res_y || r->res_z) ? 1 : 0);  // prepare, fit, residuals
  if ((e = cudaStreamEndCapture(b->stream, &b->graph)) != cudaSuccess)
    return bail(fail(TPCFIT_E_CUDA, "end capture: %s", cudaGetErrorString(e)));
  if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
    return bail(fail(TPCFIT_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e)));
  b->launches = l;
  *out = b;
  return TPCFIT_OK;
}

extern "C" int tpcfit_batch_launch(tpcfit_batch *b, void *stream) {
  if (!b) return fail(TPCFIT_E_INVAL, "batch is NULL");
  CU(cudaSetDevice(b->device));
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : b->stream;
  CU(cudaGraphLaunch(b->exec, st));
  CU(cudaEventRecord(b->done, st));
  return TPCFIT_OK;
}

extern "C" int tpcfit_batch_sync(tpcfit_batch *b, double timeout_s) {
  if (!b) return fail(TPCFIT_E_INVAL, "batch is NULL");
  CU(cudaSetDevice(b->device));
  const double t0 = tpcfit_now();
  for (;;) {
    cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return fail(TPCFIT_E_CUDA, "batch: %s", cudaGetErrorString(e));
    if (timeout_s >= 0 && tpcfit_now() - t0 > timeout_s)
      return fail(TPCFIT_E_TIMEOUT, "batch wait exceeded %.3f s", timeout_s);
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  if (*b->h_err) return fail(TPCFIT_E_INVAL, "malformed track offsets in the batch frame");
  return TPCFIT_OK;
}

extern "C" int tpcfit_batch_destroy(tpcfit_batch *b) {
  if (!b) return fail(TPCFIT_E_INVAL, "batch is NULL");
  cudaSetDevice(b->device);
  cudaEventSynchronize(b->done);
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  return TPCFIT_OK;
}

static int validate_host_offsets(const tpcfit_frame *f) {
  const int64_t *o = f->track_offsets;
  if (o[0] != 0 || o[f->n_tracks] != f->n_clusters) return fail(TPCFIT_E_INVAL, "offsets do not span [0, n_clusters]");
  for (int64_t t = 0; t < f->n_tracks; ++t)
    if (o[t + 1] < o[t]) return fail(TPCFIT_E_INVAL, "offsets decrease at track %lld", (long long)t);
  return TPCFIT_OK;
}

// x of clusters on their pad-row planes: x[i] = row_x[row[i]] (host frames
// whose x is NULL; the row table has kMaxRows entries, so every row byte
// indexes it).
__global__ void k_x_from_rows(const uint8_t *__restrict__ row, int64_t n, const float *__restrict__ row_x,
                              float *__restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = row_x[row[i]];
}

cudaError_t tpcfit::launch_x_from_rows(const uint8_t *row, int64_t n, const float *row_x, float *x, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_x_from_rows<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(row, n, row_x, x);
  return cudaGetLastError();
}

// Chunk schedule of a host frame (host path and serving).  A call costs the
// host->device copy of every input byte (the link is the bound) plus what no
// copy overlaps: the fit and the result copy of the last chunk, and a setup
// cost per copy (7 per chunk).  So the chunks grow from C/4 clusters at the
// end of the frame by a factor 1.4 per chunk towards its start, up to 4C
// (C = host_chunk_clusters): each chunk's copy still outlasts the fit and
// result copy of the chunk before it (the copy moves about 0.10 ms per M
// clusters, fit and results take about 0.06), so the copies run back to back.
// Cut points (track indices, 0 first, nt last, whole tracks per chunk) come
// from a binary search on the offsets; returns -1, or the track at which the
// offsets decrease or leave [0, n_clusters] (the offsets inside a chunk are
// the caller's to check).
int64_t tpcfit::chunk_cuts(const int64_t *off, int64_t nt, int64_t nc_all, int64_t C, std::vector<int64_t> &cuts) {
  std::vector<int64_t> sizes;  // planned chunk sizes in clusters, the last chunk first
  int64_t planned = 0;
  for (double sz = std::max(1.0, (double)C / 4.0); planned < nc_all || sizes.empty();
       sz = std::min(sz * 1.4, 4.0 * (double)C)) {
    sizes.push_back(std::max<int64_t>(1, (int64_t)sz));
    planned += sizes.back();
  }
  if (sizes.size() > 1 && planned - sizes.back() / 4 * 3 >= nc_all) {
    // the first chunk would hold under a quarter of its planned size: the next one takes it
    planned -= sizes.back();
    sizes.pop_back();
  }
  cuts.assign(1, 0);
  int64_t after = planned - sizes.back();  // clusters planned after the current chunk
  for (size_t k = sizes.size(); k-- > 0 && cuts.back() < nt;) {
    const int64_t t0 = cuts.back();
    int64_t t1 = nt;  // the last chunk ends with the frame
    if (k > 0) {
      const int64_t target = nc_all - after;  // first t1 in (t0, nt] with off[t1] >= target, or nt
      int64_t lo = t0 + 1, hi = nt;
      while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (off[mid] >= target) hi = mid;
        else lo = mid + 1;
      }
      t1 = lo;
      after -= sizes[k - 1];
    }
    if (off[t1] < off[t0] || off[t1] > nc_all) return t1;
    cuts.push_back(t1);
  }
  return -1;
}

// host frame (and host or device results): chunks of tracks, copies and fits
// of consecutive chunks overlapped (two staging buffers).
static int fit_host(tpcfit_handle *h, const tpcfit_frame *f, tpcfit_result *r) {
  if (r->chi2_out_cluster || r->chi2_in_cluster || r->restart_state)
    return fail(TPCFIT_E_INVAL, "diagnostic outputs need a device frame and device results");
  if (r->smoothed_state || r->smoothed_cov)
    return fail(TPCFIT_E_INVAL, "smoothed outputs need a device frame and device results");
  const int64_t *off = f->track_offsets;
  const int64_t nt = f->n_tracks;
  int rc = TPCFIT_OK;
  if (off[0] != 0 || off[nt] != f->n_clusters) return fail(TPCFIT_E_INVAL, "offsets do not span [0, n_clusters]");
  std::vector<int64_t> cuts;
  const int64_t bad = chunk_cuts(off, nt, f->n_clusters, h->chunk_clusters, cuts);
  if (bad >= 0)
    return fail(TPCFIT_E_INVAL, "offsets decrease or leave [0, n_clusters] before track %lld", (long long)bad);
  int64_t max_nt = 0, max_nc = 0;
  for (size_t i = 0; i + 1 < cuts.size(); ++i) {
    max_nt = std::max(max_nt, cuts[i + 1] - cuts[i]);
    max_nc = std::max(max_nc, off[cuts[i + 1]] - off[cuts[i]] + 2 * kCopyPad);
  }
  if ((rc = h->scratch.ensure(max_nt))) return rc;
  for (int i = 0; i < 2; ++i)
    if ((rc = h->stage[i].ensure(max_nt, max_nc))) return rc;
  CU(cudaMemsetAsync(h->scratch.err, 0, sizeof(int32_t), h->stream));
  const cudaMemcpyKind dk = (r->mem == TPCFIT_MEM_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  int launches = 0;
  const size_t nchunks = cuts.size() - 1;
  for (size_t ci = 0; ci < nchunks; ++ci) {
    Stage &S = h->stage[ci & 1];
    const int64_t t0 = cuts[ci], t1 = cuts[ci + 1];
    const int64_t c0 = off[t0], c1 = off[t1];
    const int64_t cnt = t1 - t0, ncl = c1 - c0;
    // inputs: wait until this stage's previous results have been copied out;
    // the copies read [c0, c1) of the inputs, inside [0, n_clusters] (checked above)
    CU(cudaStreamWaitEvent(h->h2d, S.free_ev, 0));
    CU(cudaMemcpyAsync(S.off, off + t0, (size_t)(cnt + 1) * 8, cudaMemcpyHostToDevice, h->h2d));
    tpcfit_frame cf = *f;
    XFill xfill;  // a frame without x: its x is filled on the fit stream, after the copies
    CU(copy_clusters_in(*f, c0, c1, ClusterArrays{S.x, S.y, S.z, S.sy2, S.sz2, S.row}, h->d_rowx, cf, h->h2d,
                        &xfill));
    CU(cudaEventRecord(h->ev_in[ci & 1], h->h2d));
    // fit
    CU(cudaStreamWaitEvent(h->stream, h->ev_in[ci & 1], 0));
    if (xfill.n > 0) CU(launch_x_from_rows(xfill.row, xfill.n, h->d_rowx, xfill.x, h->stream));
    CU(cudaMemsetAsync(h->scratch.hist, 0, 2 * kKeyBins * sizeof(uint32_t) + 16, h->stream));
    cf.n_tracks = cnt;
    cf.track_offsets = S.off;
    tpcfit_result cr = *r;
    cr.chi2_out_cluster = cr.chi2_in_cluster = nullptr;
    cr.restart_state = nullptr;
    cr.state = S.state; cr.cov = S.cov; cr.x_ref = S.xref; cr.chi2 = S.chi2; cr.ndf = S.ndf;
    cr.status = S.status; cr.accept = S.accept;
    cr.res_y = r->res_y ? S.res_y : nullptr;
    cr.res_z = r->res_z ? S.res_z : nullptr;
    FitArgs a = make_args(h, &cf, &cr, h->scratch, c0);
    if ((rc = run_sequence(h, a, h->stream, h->scratch, nchunks == 1, &launches))) return rc;
    CU(cudaEventRecord(h->ev_fit[ci & 1], h->stream));
    // results out
    CU(cudaStreamWaitEvent(h->d2h, h->ev_fit[ci & 1], 0));
    CU(cudaMemcpyAsync(r->state + 5 * t0, S.state, (size_t)cnt * 20, dk, h->d2h));
    CU(cudaMemcpyAsync(r->cov + 15 * t0, S.cov, (size_t)cnt * 60, dk, h->d2h));
    CU(cudaMemcpyAsync(r->x_ref + t0, S.xref, (size_t)cnt * 4, dk, h->d2h));
    CU(cudaMemcpyAsync(r->chi2 + t0, S.chi2, (size_t)cnt * 8, dk, h->d2h));
    CU(cudaMemcpyAsync(r->ndf + t0, S.ndf, (size_t)cnt * 4, dk, h->d2h));
    CU(cudaMemcpyAsync(r->status + t0, S.status, (size_t)cnt * 4, dk, h->d2h));
    if (ncl > 0) CU(cudaMemcpyAsync(r->accept + c0, S.accept, (size_t)ncl, dk, h->d2h));
    if (ncl > 0 && r->res_y) CU(cudaMemcpyAsync(r->res_y + c0, S.res_y, (size_t)ncl * 2, dk, h->d2h));
    if (ncl > 0 && r->res_z) CU(cudaMemcpyAsync(r->res_z + c0, S.res_z, (size_t)ncl * 2, dk, h->d2h));
    CU(cudaEventRecord(S.free_ev, h->d2h));
  }
  CU(cudaMemcpyAsync(h->h_err, h->scratch.err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  // the offsets inside the chunks, checked while the device works (everything
  // is enqueued first, so a stalled host thread does not idle the link): the
  // kernels reject such tracks on their own (k_prepare touches nothing of a
  // track whose offsets leave its chunk); this names the first one
  int64_t bad_track = -1;
  for (int64_t t = 0; t < nt && bad_track < 0; ++t)
    if (off[t + 1] < off[t]) bad_track = t;
  if ((rc = wait_stream(h->stream, -1))) return rc;
  if ((rc = wait_stream(h->d2h, -1))) return rc;
  h->last_launches = launches;
  if (bad_track >= 0) return fail(TPCFIT_E_INVAL, "offsets decrease at track %lld", (long long)bad_track);
  if (*h->h_err) return fail(TPCFIT_E_INVAL, "malformed track offsets");
  return TPCFIT_OK;
}

extern "C" int tpcfit_fit(tpcfit_handle *h, const tpcfit_frame *f, tpcfit_result *r) {
  if (!h) return fail(TPCFIT_E_INVAL, "handle is NULL");
  int rc = check_frame_shape(f, r);
  if (rc) return rc;
  if ((rc = check_smoother(h, r))) return rc;
  std::lock_guard<std::mutex> lk(h->mu);
  CU(cudaSetDevice(h->device));
  if (f->n_tracks == 0) return TPCFIT_OK;
  if (f->mem == TPCFIT_MEM_HOST) return fit_host(h, f, r);
  if (r->mem != TPCFIT_MEM_DEVICE) return fail(TPCFIT_E_INVAL, "device frames need device results");
  if ((rc = fit_device(h, f, r, h->stream))) return rc;
  if ((rc = wait_stream(h->stream, -1))) return rc;
  if (*h->h_err) return fail(TPCFIT_E_INVAL, "malformed track offsets");
  return TPCFIT_OK;
}

extern "C" int tpcfit_fit_async(tpcfit_handle *h, const tpcfit_frame *f, tpcfit_result *r, void *stream) {
  if (!h) return fail(TPCFIT_E_INVAL, "handle is NULL");
  int rc = check_frame_shape(f, r);
  if (rc) return rc;
  if ((rc = check_smoother(h, r))) return rc;
  if (f->mem != TPCFIT_MEM_DEVICE || r->mem != TPCFIT_MEM_DEVICE)
    return fail(TPCFIT_E_INVAL, "tpcfit_fit_async takes device frames and device results");
  std::lock_guard<std::mutex> lk(h->mu);
  CU(cudaSetDevice(h->device));
  if (f->n_tracks == 0) return TPCFIT_OK;
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  if (h->scratch.buf.cap < (size_t)f->n_tracks * 24 + 8192) {
    // growing the pool frees the old buffer: let earlier work on any stream finish
    CU(cudaDeviceSynchronize());
  }
  if ((rc = fit_device(h, f, r, st))) return rc;
  return TPCFIT_OK;
}

extern "C" int tpcfit_sync(tpcfit_handle *h, double timeout_s) {
  if (!h) return fail(TPCFIT_E_INVAL, "handle is NULL");
  std::lock_guard<std::mutex> lk(h->mu);
  CU(cudaSetDevice(h->device));
  int rc;
  // work may have been enqueued on caller streams: wait for the device
  if (timeout_s < 0) {
    CU(cudaDeviceSynchronize());
  } else if ((rc = wait_stream(h->stream, timeout_s))) {
    return rc;
  } else {
    CU(cudaDeviceSynchronize());
  }
  if (h->scratch.err) {
    if (*h->h_err) {
      *h->h_err = 0;
      return fail(TPCFIT_E_INVAL, "malformed track offsets");
    }
  }
  return TPCFIT_OK;
}

extern "C" int tpcfit_last_timing(tpcfit_handle *h, tpcfit_timing *out) {
  if (!h || !out) return fail(TPCFIT_E_INVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(h->mu);
  CU(cudaSetDevice(h->device));
  for (int i = 0; i < tpcfit_handle::kRing; ++i) fold_timing(h, (h->ring_pos + i) % tpcfit_handle::kRing);
  if (h->timing.n_timed == 0) return fail(TPCFIT_E_INVAL, "no completed timed fit");
  *out = h->timing;
  return TPCFIT_OK;
}

extern "C" int tpcfit_reset_timing(tpcfit_handle *h) {
  if (!h) return fail(TPCFIT_E_INVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(h->mu);
  CU(cudaSetDevice(h->device));
  for (int i = 0; i < tpcfit_handle::kRing; ++i) fold_timing(h, i);
  tpcfit_timing &T = h->timing;
  T.n_timed = 0;
  T.prepare_ms_sum = T.sort_ms_sum = T.fit_ms_sum = T.total_ms_sum = 0.0;
  return TPCFIT_OK;
}

extern "C" int tpcfit_submit(tpcfit_handle *h, const tpcfit_frame *f, tpcfit_result *r, uint64_t *ticket) {
  if (!h || !ticket) return fail(TPCFIT_E_INVAL, "NULL argument");
  int rc = check_frame_shape(f, r);
  if (rc) return rc;
  if (f->mem != TPCFIT_MEM_HOST || r->mem != TPCFIT_MEM_HOST)
    return fail(TPCFIT_E_INVAL, "tpcfit_submit takes host frames and host results");
  if ((rc = validate_host_offsets(f))) return rc;
  if (!h->serve && (rc = serve_start(h))) return fail(rc, "serving start-up failed");
  rc = serve_submit(h, f, r, ticket);
  if (rc == TPCFIT_E_NOMEM) return fail(rc, "frame larger than the whole HBM budget");
  return rc;
}

extern "C" int tpcfit_poll(tpcfit_handle *h, uint64_t ticket, int *state, double *t_done_s) {
  if (!h || !state) return fail(TPCFIT_E_INVAL, "NULL argument");
  if (!h->serve) return fail(TPCFIT_E_NOTFOUND, "no ticket was issued");
  return serve_poll(h, ticket, state, t_done_s, 0.0, false);
}

extern "C" int tpcfit_wait(tpcfit_handle *h, uint64_t ticket, double timeout_s, int *state, double *t_done_s) {
  if (!h || !state) return fail(TPCFIT_E_INVAL, "NULL argument");
  if (!h->serve) return fail(TPCFIT_E_NOTFOUND, "no ticket was issued");
  return serve_poll(h, ticket, state, t_done_s, timeout_s, true);
}

extern "C" int tpcfit_get_serve_stats(tpcfit_handle *h, tpcfit_serve_stats *out) {
  if (!h || !out) return fail(TPCFIT_E_INVAL, "NULL argument");
  return serve_stats(h, out);
}
