// Track following: cell grid of the clusters, launch of the follow kernel
// (fit_kernels.cu), and the gather of the followed tracks into a frame.
// Declarations and contracts: include/tpcfit_follow.h.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "tpcfit.h"
#include "tpcfit_follow.h"
#include "tpcfit_internal.h"

using namespace tpcfit;

// from tpcfit_api.cu
int handle_follow_scratch(tpcfit_handle *h, size_t bytes, void **p);
int32_t *handle_pinned_word(tpcfit_handle *h);
int report_error(int code, const char *msg);
cudaStream_t handle_stream(tpcfit_handle *h);
int handle_device(tpcfit_handle *h);
std::mutex &handle_mutex(tpcfit_handle *h);
const tpcfit_config &handle_config(tpcfit_handle *h);
const float *handle_rowx(tpcfit_handle *h);

namespace {

constexpr int kTile = 4096;  // exclusive-scan tile: 1024 threads x 4

// cell of every cluster (or 0xffffffff for clusters outside the grid's sectors/rows) and its rank in the cell
__global__ void k_cell_count(const float *__restrict__ y, const float *__restrict__ z, const uint8_t *__restrict__ row,
                             const uint8_t *__restrict__ sector, int64_t nc, int n_sectors, int n_rows, int ny,
                             int nz, float z_max, float tan_edge, const float *__restrict__ row_x,
                             uint32_t *__restrict__ cell_of, uint32_t *__restrict__ rank,
                             uint32_t *__restrict__ count) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += (int64_t)gridDim.x * blockDim.x) {
    const int r = row[k], s = sector[k];
    uint32_t cell = 0xffffffffu;
    if (r < n_rows && s < n_sectors) {
      const int iz = follow_zbin(z[k], z_max, nz), iy = follow_ybin(y[k], row_x[r], tan_edge, ny);
      cell = (uint32_t)((((int64_t)s * n_rows + r) * nz + iz) * ny + iy);
      rank[k] = atomicAdd(&count[cell], 1u);  // the cluster's place in its cell
    }
    cell_of[k] = cell;
  }
}

// exclusive scan of n uint32 in tiles (out may alias nothing)
__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t *__restrict__ in, int64_t n,
                                                     uint32_t *__restrict__ out, uint32_t *__restrict__ tile_sums) {
  __shared__ uint32_t s[1024];
  const int64_t t0 = (int64_t)blockIdx.x * kTile + 4 * threadIdx.x;
  uint32_t v[4], sum = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = (t0 + j < n) ? in[t0 + j] : 0u;
    sum += v[j];
  }
  s[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t x = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0u;
    __syncthreads();
    s[threadIdx.x] += x;
    __syncthreads();
  }
  uint32_t run = s[threadIdx.x] - sum;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (t0 + j < n) out[t0 + j] = run;
    run += v[j];
  }
  if (threadIdx.x == 1023) tile_sums[blockIdx.x] = s[1023];
}

// exclusive scan of the tile sums (one block), total into *total
__global__ void __launch_bounds__(1024) k_scan_sums(uint32_t *__restrict__ tile_sums, int64_t n_tiles,
                                                    uint32_t *__restrict__ total) {
  __shared__ uint32_t s[1024];
  const int64_t per = (n_tiles + 1023) / 1024;
  const int64_t a = threadIdx.x * per, b = (a + per < n_tiles) ? a + per : n_tiles;
  uint32_t sum = 0;
  for (int64_t i = a; i < b; ++i) sum += tile_sums[i];
  s[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t x = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0u;
    __syncthreads();
    s[threadIdx.x] += x;
    __syncthreads();
  }
  uint32_t run = s[threadIdx.x] - sum;
  for (int64_t i = a; i < b; ++i) {
    const uint32_t v = tile_sums[i];
    tile_sums[i] = run;
    run += v;
  }
  if (threadIdx.x == 1023) *total = s[1023];
}

__global__ void k_scan_add(uint32_t *__restrict__ out, int64_t n, const uint32_t *__restrict__ tile_sums,
                           const uint32_t *__restrict__ total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (i < n) ? out[i] + tile_sums[i / kTile] : *total;
}

__global__ void k_cell_fill(const float *__restrict__ y, const float *__restrict__ z, const float *__restrict__ sy2,
                            const float *__restrict__ sz2, int64_t nc, const uint32_t *__restrict__ cell_of,
                            const uint32_t *__restrict__ rank, const uint32_t *__restrict__ start,
                            float4 *__restrict__ crec, int32_t *__restrict__ cidx) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = cell_of[k];
    if (c == 0xffffffffu) continue;
    const uint32_t q = start[c] + rank[k];
    crec[q] = make_float4(y[k], z[k], sy2[k], sz2[k]);
    cidx[q] = (int32_t)k;
  }
}

__global__ void k_offsets64(const uint32_t *__restrict__ ex, int64_t n, int64_t *__restrict__ off) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    off[i] = (int64_t)ex[i];
}

// one warp per track: its attached clusters in row order
__global__ void __launch_bounds__(256) k_gather(const int32_t *__restrict__ att, int64_t n_seeds, int n_rows,
                                                const int64_t *__restrict__ off, const float *__restrict__ x,
                                                const float *__restrict__ y, const float *__restrict__ z,
                                                const float *__restrict__ sy2, const float *__restrict__ sz2,
                                                const uint8_t *__restrict__ row, int64_t nc, float *__restrict__ ox,
                                                float *__restrict__ oy, float *__restrict__ oz,
                                                float *__restrict__ osy2, float *__restrict__ osz2,
                                                uint8_t *__restrict__ orow) {
  const int lane = threadIdx.x & 31;
  uint32_t lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n_seeds; s += warps) {
    int64_t pos = off[s];
    const int64_t end = off[s + 1];
    for (int r0 = 0; r0 < n_rows; r0 += 32) {
      const int r = r0 + lane;
      const int32_t k = (r < n_rows) ? att[s * n_rows + r] : -1;
      const bool v = k >= 0 && k < nc;
      const uint32_t m = __ballot_sync(0xffffffffu, v);
      const int64_t q = pos + __popc(m & lt);
      if (v && q < end) {
        ox[q] = x[k];
        oy[q] = y[k];
        oz[q] = z[k];
        osy2[q] = sy2[k];
        osz2[q] = sz2[k];
        orow[q] = row[k];
      }
      pos += __popc(m);
    }
  }
}

__global__ void k_count_valid(const int32_t *__restrict__ att, const int32_t *__restrict__ n_att, int64_t n_seeds,
                              int n_rows, int64_t nc, uint32_t *__restrict__ len) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_seeds; s += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c = 0;
    for (int r = 0; r < n_rows; ++r) {
      const int32_t k = att[s * n_rows + r];
      c += (k >= 0 && k < nc) ? 1u : 0u;
    }
    len[s] = c;
  }
}

int cu_fail(cudaError_t e, const char *what) {
  cudaGetLastError();
  char msg[256];
  std::snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
  return report_error(TPCFIT_E_CUDA, msg);
}

#define FCU(call, what)                              \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cu_fail(e_, what); \
  } while (0)

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

int grid1d(int64_t n, int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)sms * 8;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

// exclusive scan of n uint32 (in) into out[0..n]; tile sums in `tiles`
int scan_u32(const uint32_t *in, int64_t n, uint32_t *out, uint32_t *tiles, uint32_t *total, int device,
             cudaStream_t st) {
  const int64_t n_tiles = (n + kTile - 1) / kTile;
  if (n_tiles > 0) {
    k_scan_tiles<<<(unsigned)n_tiles, 1024, 0, st>>>(in, n, out, tiles);
    FCU(cudaGetLastError(), "k_scan_tiles");
  }
  k_scan_sums<<<1, 1024, 0, st>>>(tiles, n_tiles, total);
  FCU(cudaGetLastError(), "k_scan_sums");
  k_scan_add<<<grid1d(n + 1, device), 256, 0, st>>>(out, n, tiles, total);
  FCU(cudaGetLastError(), "k_scan_add");
  return TPCFIT_OK;
}

}  // namespace

extern "C" void tpcfit_follow_default_config(tpcfit_follow_config *c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->window_sigma = 4.0f;
  c->nominal_v = 0.01f;
  c->max_miss = 4;
  c->tan_edge = (float)std::tan(10.0 * 3.14159265358979323846 / 180.0);
  c->z_max = 250.0f;
  const float sc[5] = {0.01f, 0.01f, 1e-4f, 1e-4f, 0.01f};
  for (int i = 0; i < 5; ++i) c->seed_cov[i] = sc[i];
  c->n_sectors = 36;
  c->n_ybins = 32;
  c->n_zbins = 50;
}

extern "C" int tpcfit_follow(tpcfit_handle *h, const tpcfit_follow_config *fc_in, const tpcfit_hits *hits,
                             const tpcfit_seeds *seeds, tpcfit_tracks *tr, void *stream) {
  if (!h || !hits || !seeds || !tr) return report_error(TPCFIT_E_INVAL, "NULL argument");
  tpcfit_follow_config fc;
  if (fc_in) fc = *fc_in;
  else tpcfit_follow_default_config(&fc);
  const tpcfit_config &cfg = handle_config(h);
  if (!(fc.window_sigma > 0.f) || !(fc.nominal_v >= 0.f) || fc.max_miss < 0 || !(fc.tan_edge > 0.f) ||
      !(fc.z_max > 0.f) || fc.n_sectors < 1 || fc.n_sectors > 256 || fc.n_ybins < 1 || fc.n_ybins > 4096 ||
      fc.n_zbins < 1 || fc.n_zbins > 4096)
    return report_error(TPCFIT_E_INVAL, "follow configuration out of range");
  for (int i = 0; i < 5; ++i)
    if (!(fc.seed_cov[i] > 0.f)) return report_error(TPCFIT_E_INVAL, "seed covariance must be > 0");
  const int64_t nc = hits->n_clusters, ns = seeds->n_seeds;
  if (nc < 0 || ns < 0 || nc > (int64_t)INT32_MAX || ns > (int64_t)INT32_MAX)
    return report_error(TPCFIT_E_INVAL, "bad sizes");
  if (nc > 0 && (!hits->y || !hits->z || !hits->sy2 || !hits->sz2 || !hits->row || !hits->sector))
    return report_error(TPCFIT_E_INVAL, "NULL cluster array");
  if (ns > 0 && (!seeds->state || !seeds->row || !seeds->sector || !tr->att || !tr->n_att || !tr->status))
    return report_error(TPCFIT_E_INVAL, "NULL seed or result array");
  const int nr = cfg.n_rows;
  const int64_t n_cells = (int64_t)fc.n_sectors * nr * fc.n_zbins * fc.n_ybins;
  if (n_cells >= (int64_t)UINT32_MAX || n_cells > (int64_t)kTile * 1024 * 16)
    return report_error(TPCFIT_E_INVAL, "too many grid cells");
  std::lock_guard<std::mutex> lk(handle_mutex(h));
  FCU(cudaSetDevice(handle_device(h)), "cudaSetDevice");
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : handle_stream(h);
  const int dev = handle_device(h);
  if (ns > 0) FCU(cudaMemsetAsync(tr->att, 0xff, (size_t)ns * nr * sizeof(int32_t), st), "memset att");
  if (ns == 0) return TPCFIT_OK;
  // scratch: count, start (n_cells+1), tiles, total, cell_of and rank (nc), cell arrays (nc)
  const int64_t n_tiles = (n_cells + kTile - 1) / kTile;
  const size_t o_cnt = 0, o_start = o_cnt + a256(4 * (size_t)n_cells);
  const size_t o_tiles = o_start + a256(4 * (size_t)(n_cells + 1)), o_tot = o_tiles + a256(4 * (size_t)n_tiles + 4);
  const size_t o_of = o_tot + 256, o_rank = o_of + a256(4 * (size_t)nc), o_rec = o_rank + a256(4 * (size_t)nc);
  const size_t o_idx = o_rec + a256(16 * (size_t)nc), bytes = o_idx + a256(4 * (size_t)nc);
  void *base = nullptr;
  int rc = handle_follow_scratch(h, bytes, &base);
  if (rc) return rc;
  char *sc = static_cast<char *>(base);
  auto U = [&](size_t o) { return reinterpret_cast<uint32_t *>(sc + o); };
  FCU(cudaMemsetAsync(sc, 0, o_start, st), "memset cells");
  if (nc > 0) {
    k_cell_count<<<grid1d(nc, dev), 256, 0, st>>>(hits->y, hits->z, hits->row, hits->sector, nc, fc.n_sectors, nr,
                                                  fc.n_ybins, fc.n_zbins, fc.z_max, fc.tan_edge, handle_rowx(h),
                                                  U(o_of), U(o_rank), U(o_cnt));
    FCU(cudaGetLastError(), "k_cell_count");
  }
  if ((rc = scan_u32(U(o_cnt), n_cells, U(o_start), U(o_tiles), U(o_tot), dev, st))) return rc;
  if (nc > 0) {
    k_cell_fill<<<grid1d(nc, dev), 256, 0, st>>>(hits->y, hits->z, hits->sy2, hits->sz2, nc, U(o_of), U(o_rank),
                                                 U(o_start), reinterpret_cast<float4 *>(sc + o_rec),
                                                 reinterpret_cast<int32_t *>(sc + o_idx));
    FCU(cudaGetLastError(), "k_cell_fill");
  }
  FollowArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_sectors = fc.n_sectors;
  a.n_rows = nr;
  a.ny = fc.n_ybins;
  a.nz = fc.n_zbins;
  a.z_max = fc.z_max;
  a.tan_edge = fc.tan_edge;
  a.cell_start = U(o_start);
  a.crec = reinterpret_cast<const float4 *>(sc + o_rec);
  a.cidx = reinterpret_cast<const int32_t *>(sc + o_idx);
  a.n_seeds = ns;
  a.seed_state = seeds->state;
  a.seed_row = seeds->row;
  a.seed_sector = seeds->sector;
  for (int i = 0; i < 5; ++i) a.seed_cov[i] = fc.seed_cov[i];
  a.att = tr->att;
  a.n_att = tr->n_att;
  a.status = tr->status;
  a.state_out = tr->state;
  a.row_x = handle_rowx(h);
  a.b = (float)(-0.299792458e-2 * (double)cfg.bz_tesla);
  a.chi2_max = cfg.chi2_max;
  a.chi2_max_d = (double)cfg.chi2_max;
  a.xx0 = cfg.xx0_per_row;
  a.mass2 = cfg.mass_gev * cfg.mass_gev;
  a.snp_max = cfg.snp_max;
  a.window_sigma = fc.window_sigma;
  a.nominal_v = fc.nominal_v;
  a.max_miss = fc.max_miss;
  FCU(launch_follow(a, st), "k_follow");
  return TPCFIT_OK;
}

extern "C" int tpcfit_gather_tracks(tpcfit_handle *h, const tpcfit_hits *hits, const tpcfit_tracks *tr,
                                    int64_t ns, int64_t *offsets, float *x, float *y, float *z, float *sy2,
                                    float *sz2, uint8_t *row, int64_t cap, int64_t *n_out, void *stream) {
  if (!h || !hits || !tr || !offsets || !n_out || ns < 0 || cap < 0) return report_error(TPCFIT_E_INVAL, "bad arguments");
  if (ns > 0 && (!tr->att || !tr->n_att)) return report_error(TPCFIT_E_INVAL, "NULL track arrays");
  if (hits->n_clusters > 0 && (!hits->x || !hits->y || !hits->z || !hits->sy2 || !hits->sz2 || !hits->row))
    return report_error(TPCFIT_E_INVAL, "NULL cluster array");
  if (cap > 0 && (!x || !y || !z || !sy2 || !sz2 || !row)) return report_error(TPCFIT_E_INVAL, "NULL output array");
  const int nr = handle_config(h).n_rows;
  std::lock_guard<std::mutex> lk(handle_mutex(h));
  FCU(cudaSetDevice(handle_device(h)), "cudaSetDevice");
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : handle_stream(h);
  const int dev = handle_device(h);
  const int64_t n_tiles = (ns + kTile - 1) / kTile;
  if (n_tiles > 4 * 1024 * 1024) return report_error(TPCFIT_E_INVAL, "too many seeds");
  const size_t o_len = 0, o_ex = a256(4 * (size_t)ns), o_tiles = o_ex + a256(4 * (size_t)(ns + 1));
  const size_t o_tot = o_tiles + a256(4 * (size_t)n_tiles + 4), bytes = o_tot + 256;
  void *base = nullptr;
  int rc = handle_follow_scratch(h, bytes, &base);
  if (rc) return rc;
  char *sc = static_cast<char *>(base);
  auto U = [&](size_t o) { return reinterpret_cast<uint32_t *>(sc + o); };
  if (ns > 0) {
    k_count_valid<<<grid1d(ns, dev), 256, 0, st>>>(tr->att, tr->n_att, ns, nr, hits->n_clusters, U(o_len));
    FCU(cudaGetLastError(), "k_count_valid");
  }
  if ((rc = scan_u32(U(o_len), ns, U(o_ex), U(o_tiles), U(o_tot), dev, st))) return rc;
  k_offsets64<<<grid1d(ns + 1, dev), 256, 0, st>>>(U(o_ex), ns, offsets);
  FCU(cudaGetLastError(), "k_offsets64");
  int32_t *hw = handle_pinned_word(h);
  FCU(cudaMemcpyAsync(hw, U(o_tot), sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy total");
  FCU(cudaStreamSynchronize(st), "gather");
  const int64_t total = (int64_t)(uint32_t)*hw;
  *n_out = total;
  if (total > cap) return report_error(TPCFIT_E_INVAL, "gathered clusters exceed the capacity");
  if (ns > 0) {
    const int64_t blocks = (ns + 7) / 8;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_gather<<<(unsigned)(blocks < sms * 8 ? blocks : sms * 8), 256, 0, st>>>(
        tr->att, ns, nr, offsets, hits->x, hits->y, hits->z, hits->sy2, hits->sz2, hits->row, hits->n_clusters, x, y,
        z, sy2, sz2, row);
    FCU(cudaGetLastError(), "k_gather");
  }
  FCU(cudaStreamSynchronize(st), "gather");
  return TPCFIT_OK;
}
