// Serving runtime: time frames submitted from the host are admitted into
// resident device slots as slots and HBM budget free up, fitted on one stream
// per slot (so the copies and kernels of different frames overlap on the
// device), and their results copied back into the caller's buffers.  A frame
// is split into parts of about host_chunk_clusters clusters (tracks are
// independent), each admitted to a slot of its own, so that the copies of one
// part overlap the fit of the previous part of the same frame; a ticket is
// done when all its parts are.
//
// The paper's asynchronous reconstruction limits the number of time frames in
// flight and throttles their injection (Sec. 7) and processes several time
// frames at once ("horizontal" parallelism, Sec. 4); here that becomes
// admission by slot count and device-memory budget.
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
int serve_launch_frame(tpcfit_handle *h, const tpcfit_frame *dev_frame, tpcfit_result *dev_res, void *scratch_base,
                       int64_t off_base, cudaStream_t st, const int32_t **err_dev);
int64_t handle_chunk_clusters(tpcfit_handle *h);
const float *handle_rowx(tpcfit_handle *h);
size_t serve_scratch_bytes(int64_t n_tracks);
void serve_stop(tpcfit_handle *h);

namespace {

bool debug_on() {
  static const bool on = std::getenv("TPCFIT_DEBUG") != nullptr;
  return on;
}

constexpr double kBackfillWindow = 0.050;  // seconds a blocked queue head may be overtaken

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

struct Slot {
  bool busy = false;
  Part part;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t in_done = nullptr;  // recorded after this slot's input copies
  void *mem = nullptr;
  size_t bytes = 0;
  int32_t *h_err = nullptr;  // pinned
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
  cudaEvent_t last_in = nullptr;  // input copies of the latest launched part (the next part's copies wait for it)
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

// Enqueue copy-in, fit and copy-out of part P on slot `si` (lock held).
static bool launch(ServeState *S, const Part &P, int si) {
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
  L.busy = true;
  L.part = P;
  L.failed = false;
  S->used += P.bytes;
  tpcfit_frame df;
  tpcfit_result dr;
  void *scratch = nullptr;
  carve(L.mem, nt, nc + 2 * kCopyPad, R.res.res_y != nullptr, R.res.res_z != nullptr, &df, &dr, &scratch);
  bool ok = true;
  auto cp = [&](const void *dst, const void *src, size_t b, cudaMemcpyKind k) {
    if (!b || !ok) return;
    if (cudaError_t e = cudaMemcpyAsync((void *)dst, src, b, k, L.stream); e != cudaSuccess) {
      ok = false;
      if (debug_on()) std::fprintf(stderr, "tpcfit serve: ticket %llu: copy of %zu bytes failed: %s\n",
                                   (unsigned long long)P.ticket, b, cudaGetErrorString(e));
    }
  };
  // input copies in launch order, one part at a time: the link is shared, and a
  // part whose bytes arrive first can be fitted while the next one is copied
  if (S->last_in && cudaStreamWaitEvent(L.stream, S->last_in, 0) != cudaSuccess) ok = false;
  cp(df.track_offsets, F.track_offsets + P.t0, (size_t)(nt + 1) * 8, cudaMemcpyHostToDevice);
  if (ok) {
    const ClusterArrays stage{const_cast<float *>(df.x), const_cast<float *>(df.y), const_cast<float *>(df.z),
                              const_cast<float *>(df.sy2), const_cast<float *>(df.sz2), const_cast<uint8_t *>(df.row)};
    if (cudaError_t e = copy_clusters_in(F, c0, c1, stage, handle_rowx(S->h), df, L.stream); e != cudaSuccess) {
      ok = false;
      if (debug_on()) std::fprintf(stderr, "tpcfit serve: ticket %llu: input copy failed: %s\n",
                                   (unsigned long long)P.ticket, cudaGetErrorString(e));
    }
  }
  if (ok) {
    if (cudaError_t e = cudaEventRecord(L.in_done, L.stream); e != cudaSuccess) ok = false;
    else S->last_in = L.in_done;
  }
  const int32_t *err_dev = nullptr;
  if (ok && serve_launch_frame(S->h, &df, &dr, scratch, c0, L.stream, &err_dev) != TPCFIT_OK) ok = false;
  if (ok) cp(L.h_err, err_dev, sizeof(int32_t), cudaMemcpyDeviceToHost);
  const tpcfit_result &O = R.res;
  cp(O.state + 5 * P.t0, dr.state, (size_t)nt * 20, cudaMemcpyDeviceToHost);
  cp(O.cov + 15 * P.t0, dr.cov, (size_t)nt * 60, cudaMemcpyDeviceToHost);
  cp(O.x_ref + P.t0, dr.x_ref, (size_t)nt * 4, cudaMemcpyDeviceToHost);
  cp(O.chi2 + P.t0, dr.chi2, (size_t)nt * 8, cudaMemcpyDeviceToHost);
  cp(O.ndf + P.t0, dr.ndf, (size_t)nt * 4, cudaMemcpyDeviceToHost);
  cp(O.status + P.t0, dr.status, (size_t)nt * 4, cudaMemcpyDeviceToHost);
  cp(O.accept + c0, dr.accept, (size_t)nc, cudaMemcpyDeviceToHost);
  if (dr.res_y) cp(O.res_y + c0, dr.res_y, (size_t)nc * 2, cudaMemcpyDeviceToHost);
  if (dr.res_z) cp(O.res_z + c0, dr.res_z, (size_t)nc * 2, cudaMemcpyDeviceToHost);
  if (!ok) cudaGetLastError();
  L.failed = !ok;
  cudaFreeAsync(L.mem, L.stream);  // released in stream order after the copies
  cudaEventRecord(L.done, L.stream);
  return true;
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

static void worker_loop(ServeState *S) {
  cudaSetDevice(handle_device(S->h));
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    bool progress = false;
    // completions
    for (size_t i = 0; i < S->slots.size(); ++i) {
      Slot &L = S->slots[i];
      if (!L.busy) continue;
      cudaError_t q = cudaEventQuery(L.done);
      if (q == cudaErrorNotReady) continue;
      const bool failed = !(q == cudaSuccess && !L.failed && *L.h_err == 0);
      if (failed && debug_on())
        std::fprintf(stderr, "tpcfit serve: ticket %llu failed: event %s, enqueue %s, frame error word %d\n",
                     (unsigned long long)L.part.ticket, cudaGetErrorString(q), L.failed ? "failed" : "ok", *L.h_err);
      part_done(S, L.part.ticket, failed);
      if (q != cudaSuccess) cudaGetLastError();
      S->used -= L.bytes;
      L.busy = false;
      L.mem = nullptr;
      progress = true;
    }
    if (progress) S->cv_done.notify_all();
    // admissions
    const double now = tpcfit_now();
    for (auto it = S->queue.begin(); it != S->queue.end();) {
      int free_slot = -1;
      for (size_t i = 0; i < S->slots.size(); ++i)
        if (!S->slots[i].busy) {
          free_slot = (int)i;
          break;
        }
      if (free_slot < 0) break;
      const Part P = *it;
      const bool is_head = (it == S->queue.begin());
      if (S->used + P.bytes <= S->budget) {
        if (!launch(S, P, free_slot)) {
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
    bool busy = false;
    for (auto &L : S->slots) busy |= L.busy;
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
  S->slots.resize((size_t)c.max_slots);
  for (auto &L : S->slots) {
    if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&L.in_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&L.h_err, sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      handle_serve(h) = S;
      serve_stop(h);
      return TPCFIT_E_CUDA;
    }
    *L.h_err = 0;
  }
  handle_serve(h) = S;
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
  for (auto &L : S->slots) {
    if (L.stream) cudaStreamSynchronize(L.stream);
    if (L.done) cudaEventDestroy(L.done);
    if (L.in_done) cudaEventDestroy(L.in_done);
    if (L.stream) cudaStreamDestroy(L.stream);
    if (L.h_err) cudaFreeHost(L.h_err);
  }
  if (S->pool) cudaMemPoolDestroy(S->pool);
  handle_serve(h) = nullptr;
  delete S;
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
