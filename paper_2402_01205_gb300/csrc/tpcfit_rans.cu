// rANS entropy coding of int16 codes (declared in include/tpcfit_rans.h).
//
// GPU layout: one warp codes one segment; lane l owns symbols l, l+32, ... of
// the segment (its own rANS state), so a warp step reads 32 consecutive codes
// (64 B) and the words the lanes emit or consume at a step are placed with a
// warp ballot (rank among the lanes that emit) in one contiguous block.
// Encoding writes each segment into a fixed-size slot of a scratch buffer
// (words backwards from the slot end, escapes forwards), a one-block scan
// turns the per-segment sizes into the container's offset tables, and a
// gather kernel packs the slots into the container.

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "tpcfit.h"
#include "tpcfit_rans.h"

// from tpcfit_api.cu
int handle_rans_scratch(tpcfit_handle *h, size_t bytes, void **p);
int32_t *handle_pinned_word(tpcfit_handle *h);
int report_error(int code, const char *msg);
cudaStream_t handle_stream(tpcfit_handle *h);
int handle_device(tpcfit_handle *h);
std::mutex &handle_mutex(tpcfit_handle *h);

namespace {

constexpr int kAlphabet = 512;
constexpr int kEscape = 511;
constexpr int kCodeRange = 255;
constexpr int kScaleBits = 12;
constexpr uint32_t kM = 1u << kScaleBits;
constexpr uint32_t kL = 1u << 16;
constexpr int kHeader = 64;
constexpr int kMaxSegment = 1 << 20;

struct Layout {
  int64_t n = 0;
  int32_t seg = 0;
  int64_t n_seg = 0;
  size_t freq_off = kHeader, segoff_off = 0, escoff_off = 0, payload_off = 0;
};

Layout layout_for(int64_t n, int32_t seg) {
  Layout L;
  L.n = n;
  L.seg = seg;
  L.n_seg = (n + seg - 1) / seg;
  L.segoff_off = L.freq_off + 2 * kAlphabet;
  L.escoff_off = L.segoff_off + 8 * (size_t)(L.n_seg + 1);
  L.payload_off = L.escoff_off + 8 * (size_t)(L.n_seg + 1);
  return L;
}

__device__ __forceinline__ int sym_of(int16_t c) {
  const int v = c;
  return (v >= -kCodeRange && v <= kCodeRange) ? v + kCodeRange : kEscape;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------------------
// encode
// ---------------------------------------------------------------------------
// Symbol counts: one sub-histogram per warp in shared memory.
__global__ void k_rans_hist(const int16_t *__restrict__ codes, int64_t n, unsigned long long *__restrict__ hist) {
  __shared__ uint32_t sh[8][kAlphabet];
  const int w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 8 * kAlphabet; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&sh[w][sym_of(codes[i])], 1u);
  __syncthreads();
  for (int s = threadIdx.x; s < kAlphabet; s += blockDim.x) {
    uint32_t t = 0;
    for (int k = 0; k < 8; ++k) t += sh[k][s];
    if (t) atomicAdd(&hist[s], (unsigned long long)t);
  }
}

// Normalisation of the counts to frequencies summing to 2^12 (one thread; the
// rule is sequential by definition), cumulative table, and the container's
// frequency table.  tab[s] = f | c << 16.
__global__ void k_rans_table(const unsigned long long *__restrict__ hist, uint32_t *__restrict__ tab,
                             uint16_t *__restrict__ freq_out) {
  __shared__ int f[kAlphabet];
  if (threadIdx.x == 0) {
    unsigned long long n = 0;
    for (int s = 0; s < kAlphabet; ++s) n += hist[s];
    int sum = 0;
    for (int s = 0; s < kAlphabet; ++s) {
      f[s] = 0;
      if (hist[s] > 0) {
        const unsigned long long q = (hist[s] * kM) / n;
        f[s] = q < 1 ? 1 : (int)q;
      }
      sum += f[s];
    }
    int d = n ? (int)kM - sum : 0;
    while (d != 0) {
      int best = 0;
      for (int s = 1; s < kAlphabet; ++s)
        if (f[s] > f[best]) best = s;
      if (d > 0) {
        f[best] += d;
        d = 0;
      } else {
        const int take = (-d < f[best] - 1) ? -d : f[best] - 1;
        f[best] -= take;
        d += take;
      }
    }
    int c = 0;
    for (int s = 0; s < kAlphabet; ++s) {
      tab[s] = (uint32_t)f[s] | ((uint32_t)c << 16);
      freq_out[s] = (uint16_t)f[s];
      c += f[s];
    }
  }
}

// One warp per segment (grid-stride over segments).  Slots: words (seg
// uint16) written backwards from the slot end, escapes (seg int16) forwards,
// 32 final states.
__global__ void __launch_bounds__(256) k_rans_encode(const int16_t *__restrict__ codes, int64_t n, int32_t seg,
                                                     int64_t n_seg, const uint32_t *__restrict__ tab,
                                                     uint16_t *__restrict__ wslot, int16_t *__restrict__ eslot,
                                                     uint32_t *__restrict__ states, uint32_t *__restrict__ wcnt,
                                                     uint32_t *__restrict__ ecnt, int32_t *__restrict__ err) {
  __shared__ uint32_t s_tab[kAlphabet];
  for (int s = threadIdx.x; s < kAlphabet; s += blockDim.x) s_tab[s] = tab[s];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n_seg; j += warps) {
    const int64_t s0 = j * seg;
    const int cnt = (int)((n - s0) < seg ? (n - s0) : seg);
    const int steps = (cnt + 31) >> 5;
    // escapes, in symbol order
    int16_t *es = eslot + s0;
    int ne = 0;
    for (int st = 0; st < steps; ++st) {
      const int i = st * 32 + lane;
      const bool act = i < cnt;
      const int16_t c = act ? codes[s0 + i] : (int16_t)0;
      const bool esc = act && sym_of(c) == kEscape;
      const uint32_t m = __ballot_sync(0xffffffffu, esc);
      if (esc) {
        const int k = ne + __popc(m & lt);
        if (k < seg) es[k] = c;
        else atomicOr(err, 32);
      }
      ne += __popc(m);
    }
    // rANS, last step first
    uint16_t *ws = wslot + s0;
    int wpos = seg;
    uint32_t x = kL;
    for (int st = steps - 1; st >= 0; --st) {
      const int i = st * 32 + lane;
      const bool act = i < cnt;
      uint32_t f = 1, c = 0;
      if (act) {
        const uint32_t t = s_tab[sym_of(codes[s0 + i])];
        f = t & 0xffffu;
        c = t >> 16;
      }
      const bool emit = act && (x >> (32 - kScaleBits)) >= f;  // x >= f 2^20, without the 2^32 overflow at f = M
      const uint32_t m = __ballot_sync(0xffffffffu, emit);
      const int k = __popc(m);
      if (emit) {
        const int q = wpos - k + __popc(m & lt);
        if (q >= 0 && q < seg) ws[q] = (uint16_t)(x & 0xffffu);
        else atomicOr(err, 64);
        x >>= 16;
      }
      wpos -= k;
      if (act) x = (x / f) * kM + (x % f) + c;
    }
    states[j * 32 + lane] = x;
    if (lane == 0) {
      wcnt[j] = (uint32_t)(seg - wpos);
      ecnt[j] = (uint32_t)ne;
    }
  }
}

// Offset tables of the container from the per-segment counts (one block):
// segment payload byte offsets (32 states + words each) and escape offsets;
// then the header.
__global__ void k_rans_scan(const uint32_t *__restrict__ wcnt, const uint32_t *__restrict__ ecnt, int64_t n_seg,
                            int64_t n, int32_t seg, uint8_t *__restrict__ out, size_t segoff_off,
                            size_t escoff_off, size_t out_cap, unsigned long long *__restrict__ totals,
                            int32_t *__restrict__ err) {
  if (escoff_off + 8 * (size_t)(n_seg + 1) > out_cap || segoff_off + 8 * (size_t)(n_seg + 1) > escoff_off) {
    if (threadIdx.x == 0) atomicOr(err, 128);
    return;
  }
  __shared__ unsigned long long s_p[1024], s_e[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  const int64_t per = (n_seg + nt - 1) / nt;
  const int64_t a = t * per, b = (a + per < n_seg) ? a + per : n_seg;
  unsigned long long sp = 0, se = 0;
  for (int64_t j = a; j < b; ++j) {
    sp += 128ull + 2ull * wcnt[j];
    se += ecnt[j];
  }
  s_p[t] = sp;
  s_e[t] = se;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {  // inclusive scan
    unsigned long long vp = 0, ve = 0;
    if (t >= o) {
      vp = s_p[t - o];
      ve = s_e[t - o];
    }
    __syncthreads();
    s_p[t] += vp;
    s_e[t] += ve;
    __syncthreads();
  }
  unsigned long long op = s_p[t] - sp, oe = s_e[t] - se;
  unsigned long long *so = reinterpret_cast<unsigned long long *>(out + segoff_off);
  unsigned long long *eo = reinterpret_cast<unsigned long long *>(out + escoff_off);
  for (int64_t j = a; j < b; ++j) {
    so[j] = op;
    eo[j] = oe;
    op += 128ull + 2ull * wcnt[j];
    oe += ecnt[j];
  }
  __syncthreads();
  if (t == nt - 1) {
    so[n_seg] = s_p[t];
    eo[n_seg] = s_e[t];
    totals[0] = s_p[t];
    totals[1] = s_e[t];
    uint8_t *h = out;
    h[0] = 'T'; h[1] = 'P'; h[2] = 'R'; h[3] = '1';
    *reinterpret_cast<uint32_t *>(h + 4) = 1u;
    *reinterpret_cast<long long *>(h + 8) = (long long)n;
    *reinterpret_cast<uint32_t *>(h + 16) = (uint32_t)seg;
    *reinterpret_cast<uint32_t *>(h + 20) = (uint32_t)n_seg;
    *reinterpret_cast<uint32_t *>(h + 24) = (uint32_t)kScaleBits;
    *reinterpret_cast<uint32_t *>(h + 28) = (uint32_t)kAlphabet;
    *reinterpret_cast<long long *>(h + 32) = (long long)s_e[t];
    *reinterpret_cast<long long *>(h + 40) = (long long)s_p[t];
    for (int k = 48; k < kHeader; ++k) h[k] = 0;
  }
}

// Pack the slots into the container (one warp per segment).  Segment payloads
// start at even byte offsets, so everything is moved as 16-bit words.
__global__ void __launch_bounds__(256) k_rans_gather(const uint16_t *__restrict__ wslot,
                                                     const int16_t *__restrict__ eslot,
                                                     const uint32_t *__restrict__ states,
                                                     const uint32_t *__restrict__ wcnt,
                                                     const uint32_t *__restrict__ ecnt, int64_t n_seg, int32_t seg,
                                                     uint8_t *__restrict__ out, size_t segoff_off, size_t escoff_off,
                                                     size_t payload_off, const unsigned long long *__restrict__ totals,
                                                     size_t out_cap, int32_t *__restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const unsigned long long *so = reinterpret_cast<const unsigned long long *>(out + segoff_off);
  const unsigned long long *eo = reinterpret_cast<const unsigned long long *>(out + escoff_off);
  uint16_t *pay = reinterpret_cast<uint16_t *>(out + payload_off);
  int16_t *esc = reinterpret_cast<int16_t *>(out + payload_off + totals[0]);
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n_seg; j += warps) {
    const int nw = (int)wcnt[j], ne = (int)ecnt[j];
    if (payload_off + so[j] + 128 + 2ull * nw > out_cap || nw > seg || ne > seg ||
        payload_off + totals[0] + 2ull * (eo[j] + ne) > out_cap) {
      if (lane == 0) atomicOr(err, 256);
      continue;
    }
    uint16_t *d = pay + so[j] / 2;
    const uint32_t x = states[j * 32 + lane];
    d[2 * lane] = (uint16_t)(x & 0xffffu);
    d[2 * lane + 1] = (uint16_t)(x >> 16);
    const uint16_t *src = wslot + j * (int64_t)seg + (seg - nw);
    for (int k = lane; k < nw; k += 32) d[64 + k] = src[k];
    const int16_t *es = eslot + j * (int64_t)seg;
    for (int k = lane; k < ne; k += 32) esc[eo[j] + k] = es[k];
  }
}

// ---------------------------------------------------------------------------
// decode
// ---------------------------------------------------------------------------
// err bits: 1 table, 2 offsets, 4 words, 8 escapes, 16 final states
__global__ void __launch_bounds__(256) k_rans_decode(const uint8_t *__restrict__ in, int64_t n, int32_t seg,
                                                     int64_t n_seg, size_t segoff_off, size_t escoff_off,
                                                     size_t payload_off, unsigned long long n_pay,
                                                     unsigned long long n_esc, int16_t *__restrict__ codes,
                                                     int32_t *__restrict__ err) {
  __shared__ uint16_t s_f[kAlphabet], s_c[kAlphabet];
  __shared__ uint16_t s_sym[kM];
  __shared__ int s_bad;
  const uint16_t *freq = reinterpret_cast<const uint16_t *>(in + kHeader);
  if (threadIdx.x == 0) {
    uint32_t c = 0;
    for (int s = 0; s < kAlphabet; ++s) {
      s_f[s] = freq[s];
      s_c[s] = (uint16_t)(c <= kM ? c : kM);  // cumulative frequency, at most 2^12 in a valid table
      c += freq[s];
    }
    s_bad = (c != kM);
  }
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) atomicOr(err, 1);
    return;
  }
  // slot -> symbol: the largest s with c_s <= slot (it has f_s > 0, since the
  // frequencies of a valid table sum to 2^12 and c is non-decreasing)
  for (int slot = threadIdx.x; slot < (int)kM; slot += blockDim.x) {
    int lo = 0, hi = kAlphabet - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_c[mid] <= slot) lo = mid;
      else hi = mid - 1;
    }
    s_sym[slot] = (uint16_t)lo;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const unsigned long long *so = reinterpret_cast<const unsigned long long *>(in + segoff_off);
  const unsigned long long *eo = reinterpret_cast<const unsigned long long *>(in + escoff_off);
  const uint16_t *pay = reinterpret_cast<const uint16_t *>(in + payload_off);
  const int16_t *esc = reinterpret_cast<const int16_t *>(in + payload_off + n_pay);
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n_seg; j += warps) {
    const unsigned long long p0 = so[j], p1 = so[j + 1], e0 = eo[j], e1 = eo[j + 1];
    if (p1 < p0 + 128 || p1 > n_pay || (p0 & 1) || ((p1 - p0) & 1) || e1 < e0 || e1 > n_esc) {
      if (lane == 0) atomicOr(err, 2);
      continue;
    }
    const uint16_t *d = pay + p0 / 2;
    uint32_t x = (uint32_t)d[2 * lane] | ((uint32_t)d[2 * lane + 1] << 16);
    const uint16_t *words = d + 64;
    const unsigned long long nw = (p1 - p0 - 128) / 2;
    unsigned long long wi = 0, ei = e0;
    const int64_t s0 = j * seg;
    const int cnt = (int)((n - s0) < seg ? (n - s0) : seg);
    const int steps = (cnt + 31) >> 5;
    int bad = 0;
    for (int st = 0; st < steps; ++st) {
      const int i = st * 32 + lane;
      const bool act = i < cnt;
      int s = 0;
      if (act) {
        const uint32_t slot = x & (kM - 1);
        s = s_sym[slot];
        x = (uint32_t)s_f[s] * (x >> kScaleBits) + slot - s_c[s];
      }
      const bool is_esc = act && s == kEscape;
      const uint32_t me = __ballot_sync(0xffffffffu, is_esc);
      int16_t code = (int16_t)(s - kCodeRange);
      if (is_esc) {
        const unsigned long long k = ei + __popc(me & lt);
        if (k < e1) code = esc[k];
        else bad |= 8, code = 0;
      }
      ei += __popc(me);
      const bool need = act && x < kL;
      const uint32_t mw = __ballot_sync(0xffffffffu, need);
      if (need) {
        const unsigned long long k = wi + __popc(mw & lt);
        if (k < nw) x = (x << 16) | words[k];
        else bad |= 4;
      }
      wi += __popc(mw);
      if (act) codes[s0 + i] = code;
    }
    if (wi != nw) bad |= 4;
    if (ei != e1) bad |= 8;
    if (lane < cnt && x != kL) bad |= 16;
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && lane == 0) atomicOr(err, bad);
  }
}

int cu_fail(cudaError_t e, const char *what) {
  cudaGetLastError();
  char msg[256];
  std::snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
  return report_error(TPCFIT_E_CUDA, msg);
}

#define RCU(call, what)                              \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cu_fail(e_, what); \
  } while (0)

int grid_for(int64_t n_seg, int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int64_t want = (n_seg + 7) / 8;  // 8 warps per block
  const int64_t cap = (int64_t)sms * 8;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

extern "C" int64_t tpcfit_rans_bound(int64_t n, int32_t seg) {
  if (seg == 0) seg = TPCFIT_RANS_SEGMENT_DEFAULT;
  if (n < 0 || seg < 32 || seg % 32 || seg > kMaxSegment) return -1;
  const Layout L = layout_for(n, seg);
  return (int64_t)L.payload_off + 128 * L.n_seg + 2 * n + 2 * n;  // at most one word and one escape per code
}

extern "C" int tpcfit_rans_encode(tpcfit_handle *h, const int16_t *codes, int64_t n, int32_t seg, uint8_t *out,
                                  int64_t out_cap, int64_t *out_size, void *stream) {
  if (!h || !out || !out_size || n < 0 || (n > 0 && !codes)) return report_error(TPCFIT_E_INVAL, "bad arguments");
  if (seg == 0) seg = TPCFIT_RANS_SEGMENT_DEFAULT;
  if (seg < 32 || seg % 32 || seg > kMaxSegment)
    return report_error(TPCFIT_E_INVAL, "segment_symbols must be a multiple of 32 in [32, 2^20]");
  if (reinterpret_cast<uintptr_t>(out) % 8 || reinterpret_cast<uintptr_t>(codes) % 2)
    return report_error(TPCFIT_E_INVAL, "out must be 8-byte aligned, codes 2-byte aligned");
  std::lock_guard<std::mutex> lk(handle_mutex(h));
  RCU(cudaSetDevice(handle_device(h)), "cudaSetDevice");
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : handle_stream(h);
  const Layout L = layout_for(n, seg);
  if (out_cap < (int64_t)L.payload_off) return report_error(TPCFIT_E_INVAL, "output capacity below the container");
  // scratch: hist (512 u64), totals (2 u64), tab (512 u32), wcnt, ecnt, states, word and escape slots
  auto a256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t o_hist = 0, o_tot = a256(8 * kAlphabet), o_tab = o_tot + 256, o_wc = o_tab + a256(4 * kAlphabet);
  const size_t o_ec = o_wc + a256(4 * (size_t)L.n_seg), o_st = o_ec + a256(4 * (size_t)L.n_seg);
  const size_t o_ws = o_st + a256(128 * (size_t)L.n_seg), o_es = o_ws + a256(2 * (size_t)L.n_seg * seg);
  const size_t bytes = o_es + a256(2 * (size_t)L.n_seg * seg);
  void *base = nullptr;
  int rc = handle_rans_scratch(h, bytes, &base);
  if (rc) return rc;
  char *sc = static_cast<char *>(base);
  auto *hist = reinterpret_cast<unsigned long long *>(sc + o_hist);
  auto *tot = reinterpret_cast<unsigned long long *>(sc + o_tot);
  auto *kerr = reinterpret_cast<int32_t *>(sc + o_tot + 64);  // zeroed with the histogram
  auto *tab = reinterpret_cast<uint32_t *>(sc + o_tab);
  auto *wc = reinterpret_cast<uint32_t *>(sc + o_wc);
  auto *ec = reinterpret_cast<uint32_t *>(sc + o_ec);
  auto *sts = reinterpret_cast<uint32_t *>(sc + o_st);
  auto *ws = reinterpret_cast<uint16_t *>(sc + o_ws);
  auto *es = reinterpret_cast<int16_t *>(sc + o_es);
  RCU(cudaMemsetAsync(hist, 0, o_tab, st), "memset");
  if (n > 0) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, handle_device(h));
    const int64_t hb = (n + 255) / 256;
    k_rans_hist<<<(unsigned)(hb < 4 * sms ? hb : 4 * sms), 256, 0, st>>>(codes, n, hist);
    RCU(cudaGetLastError(), "k_rans_hist");
  }
  k_rans_table<<<1, 32, 0, st>>>(hist, tab, reinterpret_cast<uint16_t *>(out + L.freq_off));
  RCU(cudaGetLastError(), "k_rans_table");
  if (L.n_seg > 0) {
    const int g = grid_for(L.n_seg, handle_device(h));
    k_rans_encode<<<g, 256, 0, st>>>(codes, n, seg, L.n_seg, tab, ws, es, sts, wc, ec, kerr);
    RCU(cudaGetLastError(), "k_rans_encode");
  }
  k_rans_scan<<<1, 1024, 0, st>>>(wc, ec, L.n_seg, n, seg, out, L.segoff_off, L.escoff_off, (size_t)out_cap, tot,
                                  kerr);
  RCU(cudaGetLastError(), "k_rans_scan");
  unsigned long long totals[2] = {0, 0};
  int32_t e_host = 0;
  RCU(cudaMemcpyAsync(totals, tot, sizeof(totals), cudaMemcpyDeviceToHost, st), "copy totals");
  RCU(cudaMemcpyAsync(&e_host, kerr, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy error word");
  RCU(cudaStreamSynchronize(st), "encode");
  if (e_host) {
    char msg[96];
    std::snprintf(msg, sizeof(msg), "rANS encoder bounds check failed (bits 0x%x)", e_host);
    return report_error(TPCFIT_E_CUDA, msg);
  }
  const int64_t size = (int64_t)L.payload_off + (int64_t)totals[0] + 2 * (int64_t)totals[1];
  *out_size = size;
  if (size > out_cap) return report_error(TPCFIT_E_INVAL, "output capacity below the container size");
  if (L.n_seg > 0) {
    const int g = grid_for(L.n_seg, handle_device(h));
    k_rans_gather<<<g, 256, 0, st>>>(ws, es, sts, wc, ec, L.n_seg, seg, out, L.segoff_off, L.escoff_off,
                                     L.payload_off, tot, (size_t)out_cap, kerr);
    RCU(cudaGetLastError(), "k_rans_gather");
  }
  RCU(cudaMemcpyAsync(&e_host, kerr, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy error word");
  RCU(cudaStreamSynchronize(st), "encode");
  if (e_host) {
    char msg[96];
    std::snprintf(msg, sizeof(msg), "rANS gather bounds check failed (bits 0x%x)", e_host);
    return report_error(TPCFIT_E_CUDA, msg);
  }
  return TPCFIT_OK;
}

extern "C" int tpcfit_rans_decode(tpcfit_handle *h, const uint8_t *in, int64_t in_size, int16_t *codes, int64_t n,
                                  void *stream) {
  if (!h || !in || n < 0 || (n > 0 && !codes)) return report_error(TPCFIT_E_INVAL, "bad arguments");
  if (in_size < kHeader + 2 * kAlphabet + 16) return report_error(TPCFIT_E_INVAL, "stream shorter than a container");
  if (reinterpret_cast<uintptr_t>(in) % 8 || reinterpret_cast<uintptr_t>(codes) % 2)
    return report_error(TPCFIT_E_INVAL, "in must be 8-byte aligned, codes 2-byte aligned");
  std::lock_guard<std::mutex> lk(handle_mutex(h));
  RCU(cudaSetDevice(handle_device(h)), "cudaSetDevice");
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : handle_stream(h);
  unsigned char hd[kHeader];
  RCU(cudaMemcpyAsync(hd, in, kHeader, cudaMemcpyDeviceToHost, st), "copy header");
  RCU(cudaStreamSynchronize(st), "copy header");
  uint32_t ver, seg, n_seg, k, a;
  long long hn, n_esc, n_pay;
  std::memcpy(&ver, hd + 4, 4);
  std::memcpy(&hn, hd + 8, 8);
  std::memcpy(&seg, hd + 16, 4);
  std::memcpy(&n_seg, hd + 20, 4);
  std::memcpy(&k, hd + 24, 4);
  std::memcpy(&a, hd + 28, 4);
  std::memcpy(&n_esc, hd + 32, 8);
  std::memcpy(&n_pay, hd + 40, 8);
  if (std::memcmp(hd, "TPR1", 4) || ver != 1 || k != (uint32_t)kScaleBits || a != (uint32_t)kAlphabet)
    return report_error(TPCFIT_E_INVAL, "not a TPR1 rANS container");
  if (hn != n) return report_error(TPCFIT_E_INVAL, "container holds a different number of codes");
  if (seg < 32 || seg % 32 || seg > (uint32_t)kMaxSegment || (int64_t)n_seg != (n + seg - 1) / seg || n_esc < 0 ||
      n_pay < 0 || (n_pay & 1))
    return report_error(TPCFIT_E_INVAL, "inconsistent container header");
  const Layout L = layout_for(n, (int32_t)seg);
  if ((int64_t)L.payload_off + n_pay + 2 * n_esc > in_size)
    return report_error(TPCFIT_E_INVAL, "container larger than the stream");
  int32_t *h_err = handle_pinned_word(h);
  void *base = nullptr;
  int rc = handle_rans_scratch(h, 256, &base);
  if (rc) return rc;
  int32_t *err = static_cast<int32_t *>(base);
  RCU(cudaMemsetAsync(err, 0, sizeof(int32_t), st), "memset");
  if (L.n_seg > 0) {
    const int g = grid_for(L.n_seg, handle_device(h));
    k_rans_decode<<<g, 256, 0, st>>>(in, n, (int32_t)seg, L.n_seg, L.segoff_off, L.escoff_off, L.payload_off,
                                     (unsigned long long)n_pay, (unsigned long long)n_esc, codes, err);
    RCU(cudaGetLastError(), "k_rans_decode");
  }
  RCU(cudaMemcpyAsync(h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy error word");
  RCU(cudaStreamSynchronize(st), "decode");
  if (*h_err) {
    char msg[128];
    std::snprintf(msg, sizeof(msg), "damaged rANS container (error bits 0x%x)", *h_err);
    return report_error(TPCFIT_E_INVAL, msg);
  }
  return TPCFIT_OK;
}
