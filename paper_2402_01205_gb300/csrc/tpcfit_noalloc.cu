// Allocation-free fit entry point (declared in include/tpcfit_noalloc.h).
//
// Some callers cannot call cudaMalloc while they fit: an application whose
// device memory is entirely reserved by another allocator (a framework's
// caching pool that already owns the HBM, where an extra cudaMalloc fails or
// fragments it), or a steady-state online loop that forbids allocation to keep
// its latency predictable.  This entry point serves them: the caller passes
// device-resident inputs and outputs, and every scratch buffer the fit needs
// (seeds, sort permutation and histogram, work counter, error word, pad-row
// table) lives in one file-scope device array of fixed size.  Nothing is
// allocated, neither here nor in any library routine it calls.
//
// Limits and sharing: frames of at most TPCFIT_NOALLOC_MAX_TRACKS tracks.  The
// array is shared by every call in the process on a given device and keeps the
// last call's contents; each call clears the parts that must start at zero.
// Calls that overlap on the GPU (two calls in flight at once, on any streams)
// race on the array and give wrong results.

#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "tpcfit.h"
#include "tpcfit_noalloc.h"
#include "tpcfit_internal.h"

using namespace tpcfit;

namespace {

constexpr size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// Layout of the static scratch (byte offsets).
constexpr size_t kHistOff = 0;                                                     // 2*kKeyBins uint32
constexpr size_t kWorkOff = a256(2 * kKeyBins * sizeof(uint32_t));                // u64 work counter
constexpr size_t kErrOff = kWorkOff + 16;                                          // int32 frame error
constexpr size_t kZeroBytes = kErrOff + 16;                                        // cleared per call
constexpr size_t kRowxOff = a256(kZeroBytes);                                      // kMaxRows floats
constexpr size_t kSeedOff = kRowxOff + a256(kMaxRows * sizeof(float));             // max_tracks*5 floats
constexpr size_t kPermOff = kSeedOff + a256((size_t)TPCFIT_NOALLOC_MAX_TRACKS * 5 * sizeof(float));
constexpr size_t kScratchBytes = kPermOff + a256((size_t)TPCFIT_NOALLOC_MAX_TRACKS * sizeof(int32_t));

}  // namespace

// The scratch array.  The CUDA runtime loads it with the library's device code
// on a device (at the first launch or symbol lookup there: lazily, by default)
// and keeps it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// The code, with `msg` as the thread's tpcfit_last_error_message.
int fail(int code, const char *msg) { return set_error_message(code, msg); }

// Pad-row plane positions, float-rounded from double, written into the
// scratch: the product and the sum each rounded on its own (no fused
// multiply-add), as the handle path computes the same table on the host.
__global__ void k_noalloc_rowx(float *rowx, double x0, double pitch) {
  const int r = threadIdx.x;
  if (r < kMaxRows) rowx[r] = (float)__dadd_rn(x0, __dmul_rn((double)r, pitch));
}

// Makes `device` current for the lifetime of the guard and gives the
// caller's thread its previous device back on every return.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    ok = cudaSetDevice(device) == cudaSuccess;
    if (!ok) cudaGetLastError();
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Per-device set-up, once per device with that device current: the host needs
// the array's device address to hand it to the kernels.
int setup(int device, void **addr) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (g_scratch_addr[device]) {
    *addr = g_scratch_addr[device];
    return TPCFIT_OK;
  }
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return fail(TPCFIT_E_CUDA, "cudaGetSymbolAddress of the static scratch failed");
  }
  g_scratch_addr[device] = p;
  *addr = p;
  return TPCFIT_OK;
}

}  // namespace

extern "C" int tpcfit_fit_noalloc(const tpcfit_config *cfg_in, const tpcfit_frame *f, tpcfit_result *r,
                                  void *stream) {
  tpcfit_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else tpcfit_default_config(&cfg);
  if (!f || !r) return fail(TPCFIT_E_INVAL, "frame or result is NULL");
  if (f->mem != TPCFIT_MEM_DEVICE || r->mem != TPCFIT_MEM_DEVICE)
    return fail(TPCFIT_E_INVAL, "tpcfit_fit_noalloc takes device frames and device results");
  if (f->n_tracks < 0 || f->n_clusters < 0 || !f->track_offsets)
    return fail(TPCFIT_E_INVAL, "bad frame sizes or NULL offsets");
  if (f->n_tracks > TPCFIT_NOALLOC_MAX_TRACKS)
    return fail(TPCFIT_E_INVAL, "frame has more tracks than TPCFIT_NOALLOC_MAX_TRACKS (65536); split it");
  if (f->n_clusters > 0 && (!f->x || !f->y || !f->z || !f->sy2 || !f->sz2 || !f->row || !r->accept))
    return fail(TPCFIT_E_INVAL, "NULL cluster or accept array");
  if (f->n_tracks > 0 && (!r->state || !r->cov || !r->x_ref || !r->chi2 || !r->ndf || !r->status))
    return fail(TPCFIT_E_INVAL, "NULL result array");
  if (cfg.n_rows < 1 || cfg.n_rows > kMaxRows || !(cfg.snp_max > 0.f && cfg.snp_max < 1.f) ||
      !(cfg.chi2_max > 0.f) || cfg.device < 0 || cfg.device >= kMaxDevices)
    return fail(TPCFIT_E_INVAL, "configuration out of range");
  if (const char *why = check_variant_params(cfg)) return fail(TPCFIT_E_INVAL, why);
  if (cfg.block_threads != 0 && cfg.block_threads != 128 && cfg.block_threads != 256)
    return fail(TPCFIT_E_INVAL, "block_threads must be 0, 128 or 256");
  if (cfg.blocks_per_sm < 0) return fail(TPCFIT_E_INVAL, "blocks_per_sm < 0");
  if (r->smoothed_state || r->smoothed_cov)
    return fail(TPCFIT_E_INVAL, "tpcfit_fit_noalloc does not run the smoother (use tpcfit_fit)");
  if ((r->res_y || r->res_z) && !(cfg.res_step_y_cm > 0.0f && cfg.res_step_z_cm > 0.0f))
    return fail(TPCFIT_E_INVAL, "residual steps must be > 0");
  DeviceGuard dev(cfg.device);
  if (!dev.ok) return fail(TPCFIT_E_NODEV, "cannot select the CUDA device");
  void *base = nullptr;
  int rc = setup(cfg.device, &base);
  if (rc) return rc;
  if (f->n_tracks == 0) return TPCFIT_OK;
  char *sc = static_cast<char *>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  FitArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_tracks = f->n_tracks;
  a.n_clusters = f->n_clusters;
  a.off = f->track_offsets;
  a.off_base = 0;
  a.x = f->x; a.y = f->y; a.z = f->z; a.sy2 = f->sy2; a.sz2 = f->sz2; a.row = f->row;
  a.state = r->state; a.cov = r->cov; a.x_ref = r->x_ref; a.chi2 = r->chi2;
  a.ndf = r->ndf; a.status = r->status; a.accept = r->accept;
  a.chi2_out_c = r->chi2_out_cluster;
  a.chi2_in_c = r->chi2_in_cluster;
  a.restart_state = r->restart_state;
  a.res_y = r->res_y;  // optional residual codes: one more kernel, no scratch
  a.res_z = r->res_z;
  a.res_inv_step_y = 1.0f / cfg.res_step_y_cm;
  a.res_inv_step_z = 1.0f / cfg.res_step_z_cm;
  a.hist = reinterpret_cast<uint32_t *>(sc + kHistOff);
  a.work = reinterpret_cast<unsigned long long *>(sc + kWorkOff);
  a.frame_error = reinterpret_cast<int32_t *>(sc + kErrOff);
  a.seed = reinterpret_cast<float *>(sc + kSeedOff);
  a.perm = cfg.sort_tracks ? reinterpret_cast<int32_t *>(sc + kPermOff) : nullptr;
  a.row_x = reinterpret_cast<const float *>(sc + kRowxOff);
  fit_params(a, cfg);

  // the row table as the handle-based path builds it (exact 162/151 pitch for the default geometry)
  double pitch = (double)cfg.row_pitch_cm;
  if (cfg.row_x0_cm == 85.0f && cfg.row_pitch_cm == (float)(162.0 / 151.0)) pitch = 162.0 / 151.0;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg.device);
  const int block = cfg.block_threads ? cfg.block_threads : 128;  // the handle path's default shape
  const int bps = cfg.blocks_per_sm > 0 ? cfg.blocks_per_sm
                                        : fit_default_blocks_per_sm(block, cfg.xrho_per_row > 0.0f || cfg.fit_iterations > 0);
  cudaError_t e;
  if ((e = cudaMemsetAsync(sc, 0, kZeroBytes, st)) != cudaSuccess) goto cuda_fail;
  k_noalloc_rowx<<<1, kMaxRows, 0, st>>>(reinterpret_cast<float *>(sc + kRowxOff), (double)cfg.row_x0_cm, pitch);
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_fail;
  if ((e = launch_prepare(a, st)) != cudaSuccess) goto cuda_fail;
  if ((e = launch_sort(a, st, nullptr)) != cudaSuccess) goto cuda_fail;
  if ((e = launch_fit(a, sms * bps, block, st)) != cudaSuccess) goto cuda_fail;
  if ((e = launch_residuals(a, st)) != cudaSuccess) goto cuda_fail;
  {
    int32_t err_host = 0;
    if ((e = cudaMemcpyAsync(&err_host, a.frame_error, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      goto cuda_fail;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto cuda_fail;
    if (err_host) return fail(TPCFIT_E_INVAL, "malformed track offsets");
  }
  return TPCFIT_OK;
cuda_fail:
  cudaGetLastError();
  if (e == cudaSuccess) return TPCFIT_OK;
  return fail(TPCFIT_E_CUDA, cudaGetErrorString(e));
}
