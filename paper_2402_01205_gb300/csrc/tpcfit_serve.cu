// Serving runtime: time frames submitted from the host are admitted into
// resident device slots as slots and HBM budget free up, and their results
// copied back into the caller's buffers.  A frame is split into parts of
// about host_chunk_clusters clusters (tracks are independent), each admitted
// to a slot of its own; a ticket is done when all its parts are.
//
// A part moves through four phases.  Admission copies its clusters in on the
// slot's stream (one part's copies after the other's: the link is shared) and
// runs the checks, seeds and sort there.  The serving engine then fits every
// part prepared at that moment in ONE persistent launch on the engine stream:
// warps claim (part, 32-track group) descriptors from a device table with an
// atomic cursor, so the parts of different frames share the GPU instead of
// queueing as separate kernels; each part's completion counter reaches zero
// when its last group is fitted, and the warp that fitted it sets the part's
// flag in host-mapped memory.  The worker sees the flag and copies that part's
// results back (after its residual codes, if requested) on the slot's stream
// while the launch still fits the other parts.
//
// The paper's asynchronous reconstruction limits the number of time frames in
// flight and throttles their injection (Sec. 7) and processes several time
// frames at once ("horizontal" parallelism, Sec. 4); here that becomes
// admission by slot count and device-memory budget, and fitting the resident
// frames together.
//
// Admission is FIFO with bounded backfill: a later, smaller frame may overtake
// the head of the queue while the head does not fit, but only for
// kBackfillWindow seconds after the head first failed to fit, so a large frame
// cannot starve.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "tpcfit.h"
#include "tpcfit_internal.h"

using namespace tpcfit;

// from tpcfit_api.cu
struct ServeState;
struct Scratch;
cudaStream_t handle_stream(tpcfit_handle *h);
int handle_device(tpcfit_handle *h);
const tpcfit_config &handle_config(tpcfit_handle *h);
ServeState *&handle_serve(tpcfit_handle *h);
int serve_prepare_frame(tpcfit_handle *h, const tpcfit_frame *f, tpcfit_result *r, void *scratch_base,
                        int64_t off_base, cudaStream_t st, FitArgs *args, const int32_t **err_dev);
int64_t handle_chunk_clusters(tpcfit_handle *h);
const float *handle_rowx(tpcfit_handle *h);
int handle_fit_grid(tpcfit_handle *h);
int handle_fit_block(tpcfit_handle *h);
size_t serve_scratch_bytes(int64_t n_tracks);
void serve_stop(tpcfit_handle *h);

namespace {

bool debug_on() {
  static const bool on = std::getenv("TPCFIT_DEBUG") != nullptr;
  return on;
}

constexpr double kBackfillWindow = 0.050;  // seconds a blocked queue head may be overtaken
// The engine launch fills every SM, so parts admitted meanwhile are checked,
// seeded and sorted right after it ends, all at once.  An idle engine waits for
// the parts still being prepared, at most this long after the first part is
// ready, so that one launch takes them all.
constexpr double kGatherWindow = 0.0002;

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device bytes one resident frame occupies: inputs, results (with `n_res`
// residual code arrays), fit scratch.
size_t frame_bytes(int64_t nt, int64_t nc, int n_res) {
  return a256((size_t)(nt + 1) * 8) + 5 * a256((size_t)nc * 4) + 2 * a256((size_t)nc) + a256((size_t)nt * 20) +
         a256((size_t)nt * 60) + a256((size_t)nt * 4) + a256((size_t)nt * 8) + 2 * a256((size_t)nt * 4) +
         (size_t)n_res * a256((size_t)nc * 2) + serve_scratch_bytes(nt);
}

struct Request {
  tpcfit_frame frame;
  tpcfit_result res;
  size_t bytes = 0;  // the whole frame resident at once (admission limit)
  int state = TPCFIT_PENDING;
  double t_submit = 0, t_done = 0;
  int parts_left = 0;
  bool failed = false;
};

// Tracks [t0, t1) of a request, fitted as one resident frame.
struct Part {
  uint64_t ticket = 0;
  int64_t t0 = 0, t1 = 0;
  size_t bytes = 0;
};

enum Phase { kFree, kPreparing, kReady, kFitting, kFinishing };

struct Slot {
  Phase phase = kFree;
  Part part;
  cudaStream_t stream = nullptr;
  cudaEvent_t prepared = nullptr;  // recorded after the part's checks, seeds and sort
  cudaEvent_t done = nullptr;      // recorded after the part's result copies
  cudaEvent_t in_done = nullptr;   // recorded after this slot's input copies
  void *mem = nullptr;
  size_t bytes = 0;
  tpcfit_frame df;                 // the resident part (device arrays in mem)
  tpcfit_result dr;
  FitArgs args;                    // its fit arguments (valid from kReady)
  const int32_t *err_dev = nullptr;
  int pos = -1;                    // its index in the engine launch (kFitting)
  int32_t *h_err = nullptr;        // pinned
  bool failed = false;
};

}  // namespace

struct ServeState {
  tpcfit_handle *h = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Part> queue;
  std::map<uint64_t, Request> reqs;
  std::vector<Slot> slots;
  size_t used = 0, budget = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  double head_blocked_since = -1.0;
  cudaMemPool_t pool = nullptr;
  cudaEvent_t last_in = nullptr;  // input copies of the latest admitted part (the next part's copies wait for it)
  // the engine: one launch at a time over the prepared parts
  cudaStream_t engine = nullptr;
  cudaEvent_t engine_done = nullptr;
  bool engine_busy = false;
  double ready_since = -1.0;  // when the oldest part waiting for the idle engine became ready
  // its part table, built in pinned memory and copied to the device per launch:
  // FitArgs[n], then prefix u64[n+1], then remaining u32[n]
  size_t table_bytes = 0;
  char *h_table = nullptr, *d_table = nullptr;
  unsigned long long *d_cursor = nullptr;
  int32_t *h_flags = nullptr;  // host-mapped, one per part of a launch
  int32_t *d_flags = nullptr;
  tpcfit_serve_stats stats{};
};

// Carve one allocation into the frame and result arrays of a resident frame.
static void carve(void *mem, int64_t nt, int64_t nc, bool want_ry, bool want_rz, tpcfit_frame *df,
                  tpcfit_result *dr, void **scratch) {
  char *p = (char *)mem;
  auto take = [&](size_t b) {
    char *q = p;
    p += a256(b);
    return q;
  };
  df->track_offsets = (const int64_t *)take((size_t)(nt + 1) * 8);
  df->x = (const float *)take((size_t)nc * 4);
  df->y = (const float *)take((size_t)nc * 4);
  df->z = (const float *)take((size_t)nc * 4);
  df->sy2 = (const float *)take((size_t)nc * 4);
  df->sz2 = (const float *)take((size_t)nc * 4);
  df->row = (const uint8_t *)take((size_t)nc);
  df->sector = nullptr;
  df->n_tracks = nt;
  df->n_clusters = nc;
  df->mem = TPCFIT_MEM_DEVICE;
  dr->state = (float *)take((size_t)nt * 20);
  dr->cov = (float *)take((size_t)nt * 60);
  dr->x_ref = (float *)take((size_t)nt * 4);
  dr->chi2 = (double *)take((size_t)nt * 8);
  dr->ndf = (int32_t *)take((size_t)nt * 4);
  dr->status = (int32_t *)take((size_t)nt * 4);
  dr->accept = (uint8_t *)take((size_t)nc);
  dr->res_y = want_ry ? (int16_t *)take((size_t)nc * 2) : nullptr;
  dr->res_z = want_rz ? (int16_t *)take((size_t)nc * 2) : nullptr;
  dr->mem = TPCFIT_MEM_DEVICE;
  dr->chi2_out_cluster = dr->chi2_in_cluster = nullptr;
  dr->restart_state = nullptr;
  dr->smoothed_state = dr->smoothed_cov = nullptr;
  *scratch = p;
}

// Admit part P to slot `si` (lock held): allocation, input copies, then the
// part's checks, seeds and sort, all on the slot's stream.
static bool admit(ServeState *S, const Part &P, int si) {
  Request &R = S->reqs[P.ticket];
  Slot &L = S->slots[si];
  const tpcfit_frame &F = R.frame;
  const int64_t c0 = F.track_offsets[P.t0], c1 = F.track_offsets[P.t1];
  const int64_t nt = P.t1 - P.t0, nc = c1 - c0;
  if (cudaError_t e = cudaMallocFromPoolAsync(&L.mem, P.bytes, S->pool, L.stream); e != cudaSuccess) {
    cudaGetLastError();
    if (debug_on()) std::fprintf(stderr, "tpcfit serve: ticket %llu: pool allocation of %zu bytes failed: %s\n",
                                 (unsigned long long)P.ticket, P.bytes, cudaGetErrorString(e));
    return false;
  }
  L.bytes = P.bytes;
  L.part = P;
  L.failed = false;
  L.pos = -1;
  L.err_dev = nullptr;
  S->used += P.bytes;
  void *scratch = nullptr;
  carve(L.mem, nt, nc + 2 * kCopyPad, R.res.res_y != nullptr, R.res.res_z != nullptr, &L.df, &L.dr, &scratch);
  bool ok = true;
  // input copies in admission order, one part at a time: the link is shared, and a
  // part whose bytes arrive first can be fitted while the next one is copied
  if (S->last_in && cudaStreamWaitEvent(L.stream, S->last_in, 0) != cudaSuccess) ok = false;
  if (ok && cudaMemcpyAsync((void *)L.df.track_offsets, F.track_offsets + P.t0, (size_t)(nt + 1) * 8,
                            cudaMemcpyHostToDevice, L.stream) != cudaSuccess)
    ok = false;
  if (ok) {
    const ClusterArrays stage{const_cast<float *>(L.df.x), const_cast<float *>(L.df.y), const_cast<float *>(L.df.z),
                              const_cast<float *>(L.df.sy2), const_cast<float *>(L.df.sz2),
                              const_cast<uint8_t *>(L.df.row)};
    if (cudaError_t e = copy_clusters_in(F, c0, c1, stage, handle_rowx(S->h), L.df, L.stream); e != cudaSuccess) {
      ok = false;
      if (debug_on()) std::fprintf(stderr, "tpcfit serve: ticket %llu: input copy failed: %s\n",
                                   (unsigned long long)P.ticket, cudaGetErrorString(e));
    }
  }
  if (ok) {
    if (cudaEventRecord(L.in_done, L.stream) != cudaSuccess) ok = false;
    else S->last_in = L.in_done;
  }
  if (ok && serve_prepare_frame(S->h, &L.df, &L.dr, scratch, c0, L.stream, &L.args, &L.err_dev) != TPCFIT_OK)
    ok = false;
  if (ok && cudaEventRecord(L.prepared, L.stream) != cudaSuccess) ok = false;
  if (!ok) cudaGetLastError();
  L.failed = !ok;
  L.phase = kPreparing;
  return true;
}

// Copy part results back and release the slot's memory, on the slot's stream
// (lock held); the part must be fitted (or failed: nothing is copied).
static void finish(ServeState *S, int si) {
  Slot &L = S->slots[si];
  Request &R = S->reqs[L.part.ticket];
  const Part &P = L.part;
  const int64_t c0 = R.frame.track_offsets[P.t0];
  const int64_t nt = P.t1 - P.t0, nc = R.frame.track_offsets[P.t1] - c0;
  bool ok = !L.failed;
  auto cp = [&](void *dst, const void *src, size_t b) {
    if (!b || !ok) return;
    if (cudaError_t e = cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, L.stream); e != cudaSuccess) {
      ok = false;
      if (debug_on()) std::fprintf(stderr, "tpcfit serve: ticket %llu: copy of %zu bytes failed: %s\n",
                                   (unsigned long long)P.ticket, b, cudaGetErrorString(e));
    }
  };
  if (ok && nt > 0 && launch_residuals(L.args, L.stream) != cudaSuccess) ok = false;
  if (L.err_dev) cp(L.h_err, L.err_dev, sizeof(int32_t));
  const tpcfit_result &O = R.res;
  cp(O.state + 5 * P.t0, L.dr.state, (size_t)nt * 20);
  cp(O.cov + 15 * P.t0, L.dr.cov, (size_t)nt * 60);
  cp(O.x_ref + P.t0, L.dr.x_ref, (size_t)nt * 4);
  cp(O.chi2 + P.t0, L.dr.chi2, (size_t)nt * 8);
  cp(O.ndf + P.t0, L.dr.ndf, (size_t)nt * 4);
  cp(O.status + P.t0, L.dr.status, (size_t)nt * 4);
  cp(O.accept + c0, L.dr.accept, (size_t)nc);
  if (L.dr.res_y) cp(O.res_y + c0, L.dr.res_y, (size_t)nc * 2);
  if (L.dr.res_z) cp(O.res_z + c0, L.dr.res_z, (size_t)nc * 2);
  if (!ok) cudaGetLastError();
  L.failed = !ok;
  cudaFreeAsync(L.mem, L.stream);  // released in stream order after the copies
  cudaEventRecord(L.done, L.stream);
  L.phase = kFinishing;
}

// One part of a request has finished (lock held).
static void part_done(ServeState *S, uint64_t tk, bool failed) {
  Request &R = S->reqs[tk];
  R.failed |= failed;
  if (--R.parts_left == 0) {
    R.t_done = tpcfit_now();
    R.state = R.failed ? TPCFIT_FAILED : TPCFIT_DONE;
  }
}

// One engine launch over every prepared part (lock held, engine idle).
static void launch_engine(ServeState *S) {
  const int ns = (int)S->slots.size();
  FitArgs *parts = reinterpret_cast<FitArgs *>(S->h_table);
  unsigned long long *prefix = reinterpret_cast<unsigned long long *>(S->h_table + ns * sizeof(FitArgs));
  unsigned *remaining = reinterpret_cast<unsigned *>(S->h_table + ns * sizeof(FitArgs) + (ns + 1) * 8);
  int n = 0;
  unsigned long long groups = 0;
  for (int i = 0; i < ns; ++i) {
    Slot &L = S->slots[i];
    if (L.phase != kReady) continue;
    parts[n] = L.args;
    prefix[n] = groups;
    const unsigned g = (unsigned)((L.args.n_tracks + 31) / 32);
    remaining[n] = g;
    groups += g;
    S->h_flags[n] = 0;
    L.pos = n;
    L.phase = kFitting;
    ++n;
  }
  prefix[n] = groups;
  if (n == 0) return;
  const tpcfit_config &c = handle_config(S->h);
  PartsArgs pa;
  pa.parts = reinterpret_cast<const FitArgs *>(S->d_table);
  pa.prefix = reinterpret_cast<const unsigned long long *>(S->d_table + ns * sizeof(FitArgs));
  pa.remaining = reinterpret_cast<unsigned *>(S->d_table + ns * sizeof(FitArgs) + (ns + 1) * 8);
  pa.cursor = S->d_cursor;
  pa.done_flag = S->d_flags;
  pa.n_parts = n;
  bool ok = cudaMemcpyAsync(S->d_table, S->h_table, S->table_bytes, cudaMemcpyHostToDevice, S->engine) == cudaSuccess &&
            cudaMemsetAsync(S->d_cursor, 0, sizeof(unsigned long long), S->engine) == cudaSuccess &&
            launch_fit_parts(pa, c.xrho_per_row > 0.0f || c.fit_iterations > 0, handle_fit_grid(S->h),
                             handle_fit_block(S->h), S->engine) == cudaSuccess &&
            cudaEventRecord(S->engine_done, S->engine) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (debug_on()) std::fprintf(stderr, "tpcfit serve: engine launch over %d parts failed\n", n);
    for (int i = 0; i < ns; ++i)
      if (S->slots[i].phase == kFitting) {
        S->slots[i].failed = true;
        finish(S, i);
      }
    return;
  }
  S->engine_busy = true;
  S->stats.launches += 1;
  S->stats.parts += n;
  S->stats.max_parts_per_launch = std::max<int64_t>(S->stats.max_parts_per_launch, n);
}

static void worker_loop(ServeState *S) {
  cudaSetDevice(handle_device(S->h));
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    bool progress = false;
    for (size_t i = 0; i < S->slots.size(); ++i) {
      Slot &L = S->slots[i];
      if (L.phase == kFinishing) {  // results copied back
        cudaError_t q = cudaEventQuery(L.done);
        if (q == cudaErrorNotReady) continue;
        const bool failed = !(q == cudaSuccess && !L.failed && *L.h_err == 0);
        if (failed && debug_on())
          std::fprintf(stderr, "tpcfit serve: ticket %llu failed: event %s, enqueue %s, frame error word %d\n",
                       (unsigned long long)L.part.ticket, cudaGetErrorString(q), L.failed ? "failed" : "ok", *L.h_err);
        part_done(S, L.part.ticket, failed);
        if (q != cudaSuccess) cudaGetLastError();
        S->used -= L.bytes;
        L.phase = kFree;
        L.mem = nullptr;
        progress = true;
      } else if (L.phase == kPreparing) {  // checks, seeds and sort done?
        cudaError_t q = cudaEventQuery(L.prepared);
        if (L.failed) q = cudaErrorUnknown;
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess || L.args.n_tracks == 0) {  // nothing for the engine
          if (q != cudaSuccess) {
            cudaGetLastError();
            L.failed = true;
          }
          finish(S, (int)i);
        } else {
          L.phase = kReady;
        }
        progress = true;
      } else if (L.phase == kFitting && *(volatile int32_t *)(S->h_flags + L.pos) == 1) {  // fitted
        finish(S, (int)i);
        progress = true;
      }
    }
    if (progress) S->cv_done.notify_all();
    // the engine launch finished: every part it fitted has raised its flag,
    // unless the launch failed
    if (S->engine_busy && cudaEventQuery(S->engine_done) != cudaErrorNotReady) {
      const bool launch_ok = cudaEventQuery(S->engine_done) == cudaSuccess;
      if (!launch_ok) cudaGetLastError();
      for (size_t i = 0; i < S->slots.size(); ++i) {
        Slot &L = S->slots[i];
        if (L.phase != kFitting) continue;
        if (!(launch_ok && *(volatile int32_t *)(S->h_flags + L.pos) == 1)) L.failed = true;
        finish(S, (int)i);
      }
      S->engine_busy = false;
      progress = true;
    }
    if (!S->engine_busy) {
      bool ready = false, preparing = false;
      for (auto &L : S->slots) {
        ready |= L.phase == kReady;
        preparing |= L.phase == kPreparing;
      }
      if (!ready) {
        S->ready_since = -1.0;
      } else {
        const double t = tpcfit_now();
        if (S->ready_since < 0) S->ready_since = t;
        if (!preparing || t - S->ready_since > kGatherWindow) {
          launch_engine(S);
          S->ready_since = -1.0;
          progress = true;
        }
      }
    }
    // admissions
    const double now = tpcfit_now();
    for (auto it = S->queue.begin(); it != S->queue.end();) {
      int free_slot = -1;
      for (size_t i = 0; i < S->slots.size(); ++i)
        if (S->slots[i].phase == kFree) {
          free_slot = (int)i;
          break;
        }
      if (free_slot < 0) break;
      const Part P = *it;
      const bool is_head = (it == S->queue.begin());
      if (S->used + P.bytes <= S->budget) {
        if (!admit(S, P, free_slot)) {
          part_done(S, P.ticket, true);
          S->cv_done.notify_all();
        }
        if (is_head) S->head_blocked_since = -1.0;
        it = S->queue.erase(it);
        progress = true;
        continue;
      }
      if (is_head) {
        if (S->head_blocked_since < 0) S->head_blocked_since = now;
        if (now - S->head_blocked_since > kBackfillWindow) break;  // no more overtaking
      }
      ++it;
    }
    bool busy = S->engine_busy;
    for (auto &L : S->slots) busy |= L.phase != kFree;
    if (!progress) {
      if (busy) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      } else {
        S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      }
    }
  }
}

int serve_start(tpcfit_handle *h) {
  ServeState *S = new ServeState();
  S->h = h;
  const tpcfit_config &c = handle_config(h);
  S->budget = (size_t)c.hbm_budget_bytes;
  cudaSetDevice(handle_device(h));
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = handle_device(h);
  if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return TPCFIT_E_CUDA;
  }
  uint64_t keep = (uint64_t)S->budget;
  cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  const int ns = c.max_slots;
  S->slots.resize((size_t)ns);
  S->table_bytes = (size_t)ns * sizeof(FitArgs) + (size_t)(ns + 1) * 8 + (size_t)ns * 4;
  bool ok = cudaStreamCreateWithFlags(&S->engine, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&S->engine_done, cudaEventDisableTiming) == cudaSuccess &&
            cudaMallocHost(&S->h_table, S->table_bytes) == cudaSuccess &&
            cudaMalloc(&S->d_table, S->table_bytes) == cudaSuccess &&
            cudaMalloc(&S->d_cursor, sizeof(unsigned long long)) == cudaSuccess &&
            cudaHostAlloc(&S->h_flags, (size_t)ns * sizeof(int32_t), cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer(&S->d_flags, S->h_flags, 0) == cudaSuccess;
  for (auto &L : S->slots) {
    if (!ok) break;
    ok = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&L.prepared, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&L.in_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaMallocHost(&L.h_err, sizeof(int32_t)) == cudaSuccess;
    if (ok) *L.h_err = 0;
  }
  handle_serve(h) = S;
  if (!ok) {
    cudaGetLastError();
    serve_stop(h);
    return TPCFIT_E_CUDA;
  }
  for (int i = 0; i < ns; ++i) S->h_flags[i] = 0;
  S->worker = std::thread(worker_loop, S);
  return TPCFIT_OK;
}

void serve_stop(tpcfit_handle *h) {
  ServeState *S = handle_serve(h);
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  if (S->engine) cudaStreamSynchronize(S->engine);
  for (auto &L : S->slots) {
    if (L.stream) cudaStreamSynchronize(L.stream);
    if (L.prepared) cudaEventDestroy(L.prepared);
    if (L.done) cudaEventDestroy(L.done);
    if (L.in_done) cudaEventDestroy(L.in_done);
    if (L.stream) cudaStreamDestroy(L.stream);
    if (L.h_err) cudaFreeHost(L.h_err);
  }
  if (S->engine_done) cudaEventDestroy(S->engine_done);
  if (S->engine) cudaStreamDestroy(S->engine);
  if (S->h_table) cudaFreeHost(S->h_table);
  if (S->d_table) cudaFree(S->d_table);
  if (S->d_cursor) cudaFree(S->d_cursor);
  if (S->h_flags) cudaFreeHost(S->h_flags);
  if (S->pool) cudaMemPoolDestroy(S->pool);
  handle_serve(h) = nullptr;
  delete S;
}

int serve_stats(tpcfit_handle *h, tpcfit_serve_stats *out) {
  ServeState *S = handle_serve(h);
  std::memset(out, 0, sizeof(*out));
  if (!S) return TPCFIT_OK;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  return TPCFIT_OK;
}

int serve_submit(tpcfit_handle *h, const tpcfit_frame *f, tpcfit_result *r, uint64_t *ticket) {
  ServeState *S = handle_serve(h);
  const int n_res = (r->res_y ? 1 : 0) + (r->res_z ? 1 : 0);
  const size_t bytes = frame_bytes(f->n_tracks, f->n_clusters + 2 * kCopyPad, n_res);
  if (bytes > S->budget) return TPCFIT_E_NOMEM;
  // parts by the chunk schedule of the host path (offsets were checked by the caller)
  const int64_t *off = f->track_offsets;
  std::vector<int64_t> cuts;
  if (chunk_cuts(off, f->n_tracks, f->n_clusters, handle_chunk_clusters(h), cuts) >= 0) return TPCFIT_E_INVAL;
  std::vector<Part> parts;
  for (size_t i = 0; i + 1 < cuts.size(); ++i) {
    Part P;
    P.t0 = cuts[i];
    P.t1 = cuts[i + 1];
    P.bytes = frame_bytes(P.t1 - P.t0, off[P.t1] - off[P.t0] + 2 * kCopyPad, n_res);  // room for the widened copy
    parts.push_back(P);
  }
  std::lock_guard<std::mutex> lk(S->mu);
  const uint64_t tk = S->next_ticket++;
  Request &R = S->reqs[tk];
  R.frame = *f;
  R.res = *r;
  R.bytes = bytes;
  R.t_submit = tpcfit_now();
  R.parts_left = (int)parts.size();
  if (parts.empty()) {
    R.state = TPCFIT_DONE;
    R.t_done = R.t_submit;
  }
  for (Part &P : parts) {
    P.ticket = tk;
    S->queue.push_back(P);
  }
  *ticket = tk;
  S->cv_work.notify_one();
  return TPCFIT_OK;
}

int serve_poll(tpcfit_handle *h, uint64_t ticket, int *state, double *t_done, double timeout_s, bool wait) {
  ServeState *S = handle_serve(h);
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return TPCFIT_E_NOTFOUND;
  if (wait) {
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s);
    while (it->second.state == TPCFIT_PENDING) {
      if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second.state == TPCFIT_PENDING) {
        *state = TPCFIT_PENDING;
        return TPCFIT_E_TIMEOUT;
      }
      it = S->reqs.find(ticket);
      if (it == S->reqs.end()) return TPCFIT_E_NOTFOUND;
    }
  }
  *state = it->second.state;
  if (t_done) *t_done = it->second.t_done;
  if (it->second.state != TPCFIT_PENDING) S->reqs.erase(it);
  return TPCFIT_OK;
}
