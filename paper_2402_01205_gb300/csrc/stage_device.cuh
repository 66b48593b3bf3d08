// Staging of a track's clusters into shared memory with asynchronous copies,
// shared by the fit (fit_kernels.cu) and the smoother (smooth_kernels.cu):
// each lane copies its own track's clusters, in chunks of four consecutive
// cluster indices aligned to the arrays' 16-byte lines, into a ring of
// chunk buffers in its shared-memory column.
#pragma once

#include <cuda_runtime.h>

#include <stdint.h>

#include "tpcfit_internal.h"

namespace tpcfit {

constexpr int kChunk = 4;                 // clusters per staged chunk (per lane)
constexpr int kStageBufs = 3;             // chunk buffers per lane: a ring, chunk c in buffer c % 3
constexpr int kStageArrays = 5;           // x, y, z, sy2, sz2
// Shared memory of the staging over NCOL track columns: the pad-row table,
// the staged chunks ([buf][array][column] 16-byte entries) and their row
// words ([buf][word][column]).
constexpr size_t kSmemRowx = kMaxRows * sizeof(float);
template <int NCOL> __host__ __device__ constexpr size_t smem_f4() { return (size_t)kStageBufs * kStageArrays * NCOL * 16; }
template <int NCOL> __host__ __device__ constexpr size_t stage_smem() {
  return kSmemRowx + smem_f4<NCOL>() + (size_t)(kStageBufs * 2) * NCOL * sizeof(uint32_t);
}

// 4-byte asynchronous global->shared copy (zero-fill when !valid; the source
// address is then still a valid element and is not read).
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct Clu {
  float x, y, z, vy, vz;
  int r;
};

// Staging of one track's clusters.  The clusters [a, a+n) are read in chunks
// of four consecutive cluster indices aligned to the 16-byte boundaries of
// the cluster arrays: chunk c holds clusters g0+4c .. g0+4c+3 with
// g0 = a - lead, lead in [0, 3] (slots before a or past the track's end are
// don't-care).  Shared memory holds, per track column, a ring of kStageBufs
// chunk buffers: each array's four values of a chunk as one 16-byte entry
// ([buf][array][column] float4), then the chunk's row bytes as the two
// aligned 32-bit words that hold them ([buf][word][column]).
// Clusters in chunk c: slot (k + lead) & 3 of chunk (k + lead) >> 2.
__device__ __forceinline__ int chunk_lead(const FitArgs &A, int64_t a) {
  return (int)(((uint64_t)a + (reinterpret_cast<uintptr_t>(A.x) >> 2)) & 3u);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Issue the copies of chunk c of the track [a, e) into buffer `buf` (= c %
// kStageBufs) of its column; `f4` = the column's float4 entry of buffer 0,
// array 0 (as floats), `w` = its row word of buffer 0, word 0; NCOL columns.
// A chunk that lies inside the frame is copied as one 16-byte vector per
// array when the five arrays share their 16-byte phase (A.stage_vec), else
// cluster by cluster (only the track's own clusters, zero elsewhere).  A row
// word is copied only when it holds a byte of the track: an aligned word that
// holds a byte of an allocation lies inside it, allocations being at least
// 4-byte granular.
template <int NCOL>
__device__ __forceinline__ void stage_chunk(const FitArgs &A, int64_t a, int64_t e, int lead, uint32_t rsh, int c,
                                            int buf, float *f4, uint32_t *w) {
  const int64_t k0 = a - lead + 4 * (int64_t)c;
  float *dst = f4 + buf * (kStageArrays * NCOL * 4);
  const float *src[kStageArrays] = {A.x, A.y, A.z, A.sy2, A.sz2};
  if (A.stage_vec && k0 >= 0 && k0 + 4 <= A.n_clusters) {
#pragma unroll
    for (int j = 0; j < kStageArrays; ++j) cp_async16(dst + j * (NCOL * 4), src[j] + k0);
  } else {
#pragma unroll
    for (int s = 0; s < kChunk; ++s) {
      const int64_t k = k0 + s;
      const bool v = k >= a && k < e;
      const int64_t kk = v ? k : a;
#pragma unroll
      for (int j = 0; j < kStageArrays; ++j) cp_async4(dst + j * (NCOL * 4) + s, src[j] + kk, v);
    }
  }
  const uintptr_t ra = reinterpret_cast<uintptr_t>(A.row) + (uintptr_t)a;   // the track's first row byte
  const uintptr_t re = reinterpret_cast<uintptr_t>(A.row) + (uintptr_t)e;   // one past its last
  const uintptr_t w0 = (reinterpret_cast<uintptr_t>(A.row) + (uintptr_t)k0) & ~(uintptr_t)3;
  const uintptr_t wa = ra & ~(uintptr_t)3;  // a word that holds a byte of the track
  const bool v0 = w0 + 4 > ra;              // w0 < re: the chunk holds a cluster of the track
  const bool v1 = rsh != 0u && w0 + 4 < re;
  uint32_t *wd = w + buf * (2 * NCOL);
  cp_async4(wd, reinterpret_cast<const void *>(v0 ? w0 : wa), v0);
  cp_async4(wd + NCOL, reinterpret_cast<const void *>(v1 ? w0 + 4 : wa), v1);
  cp_async_commit();
}

// Rows of the chunk staged in buffer `buf`, one byte per slot.
template <int NCOL>
__device__ __forceinline__ uint32_t staged_rows(const uint32_t *w, int buf, uint32_t rsh) {
  const uint32_t *src = w + buf * (2 * NCOL);
  return __funnelshift_r(src[0], src[NCOL], 8u * rsh);
}

// Cluster in `slot` of the chunk staged in buffer `buf` (whose rows are rows_cur).
template <int NCOL>
__device__ __forceinline__ Clu read_staged(const float *f4, int slot, int buf, uint32_t rows_cur) {
  const float *src = f4 + buf * (kStageArrays * NCOL * 4) + slot;
  Clu c;
  c.x = src[0];
  c.y = src[NCOL * 4];
  c.z = src[2 * NCOL * 4];
  c.vy = src[3 * NCOL * 4];
  c.vz = src[4 * NCOL * 4];
  c.r = (rows_cur >> (8 * slot)) & 0xffu;
  return c;
}

}  // namespace tpcfit
