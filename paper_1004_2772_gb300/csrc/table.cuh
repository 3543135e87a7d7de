// find-or-put on the GPU (Alg. "find-or-put" with Alg. "Walking the (cache) line").
//
// One thread owns one key.  Memory-level parallelism, not warp cooperation, is
// what bounds a random-access table on HBM: a thread per key keeps one
// independent 32-byte bucket-sector request in flight per resident thread.
//
// Walk (Alg. "Walking the (cache) line", read as in its prose: the buckets of
// the aligned line that holds `index`, visited cyclically from `index`):
//   line  = index / L,  offset = index mod L,  walk = offset, offset+1, ...,
//   L-1, 0, ..., offset-1 inside the line.
// The line is read lazily one 32-byte sector (8 buckets) at a time, so a
// 128-byte line costs one sector when the key resolves in its first sector.
//
// Sequential semantics (Alg. "find-or-put"): the thread acts on the FIRST
// bucket in walk order that is empty or carries its memo:
//   empty      -> CAS(empty -> <memo, write>); on success write Data[i], publish
//                 <memo, done>, answer "new"; on failure re-evaluate the bucket
//                 with the value the CAS returned.
//   memo-equal -> wait (bounded) while the bucket is in the write state, then
//                 compare Data[i] with the key: equal answers "seen", otherwise
//                 the walk continues.
// Sector words read before a CAS may be stale, which is safe: the only change
// a bucket can undergo is empty -> write(memo) -> done(memo), so a stale
// non-empty word is still correct and a stale empty word is corrected by the
// CAS.  After the line: next line = (line + (2*memo + 1)) mod lines (double
// hashing with an odd step over a power-of-two line count, Section 3.2).
#pragma once

#include "common.cuh"

namespace vss {

// How a probe orders its read of a data row after the <memo, done> bucket
// word it observed (Section 3.3 memory-model requirement):
//   1 (default): bucket sectors are read with gpu-scope acquire loads, so
//                every later load of the thread is ordered after them;
//   0:           bucket sectors are read relaxed and an acquire fence is
//                issued before a data row is compared.
#ifndef VSS_ACQ_MODE
#define VSS_ACQ_MODE 1
#endif

// One 32-byte bucket sector in one instruction.
__device__ __forceinline__ void ld_sector(const uint32_t* p, uint4& a, uint4& b) {
#if VSS_ACQ_MODE == 1
  ld_acquire_v8(p, a, b);
#else
  ld_relaxed_v8(p, a, b);
#endif
}

struct LocalCounters {
  uint32_t busy_waits = 0;
  uint32_t rehashes = 0;
};

// Memory ordering of the publish step (Section 3.3: the data write must not be
// reordered before the claim, nor the done mark before the data write).  The
// writer orders data stores before <memo, done> with a gpu-scope fence; a
// reader that observed <memo, done> reads the data row only after an acquire
// (an acquire load of the bucket, or an acquire fence after a relaxed load).
// A CAS that returned <memo, done> is followed by the same fence.
// RT = true: the row width is the table's run-time t.nv (<= NV), for kernels
// that serve tables of several widths; otherwise it is exactly NV.
template <int NV, bool RT>
__device__ __forceinline__ bool data_equal_after_done(const TableView& t, uint32_t i,
                                                      const Vec<NV>& key, bool acquired) {
  if (!acquired) fence_acq_rel();
  Vec<NV> row;
  if (RT) load_row_rt<NV>(t.data + (size_t)i * t.nv, row, t.nv);
  else load_row<NV>(t.data + (size_t)i * NV, row);
  return vec_eq(row, key);
}

// Wait while bucket i is in the write state (bounded, with nanosleep backoff).
// Returns false on timeout (error latched).
__device__ __forceinline__ bool wait_done(const TableView& t, uint32_t i, uint32_t& b,
                                          LocalCounters& lc) {
  uint32_t spins = 0, ns = 16;
  lc.busy_waits++;
  while (!(b & kDone)) {
    if (++spins > t.max_spin) {
      latch_error(t.ctr, HT_ERR_TIMEOUT);
      return false;
    }
    __nanosleep(ns);
    ns = ns < 256 ? ns * 2 : ns;
    b = ld_acquire(t.buckets + i);
  }
  return true;
}

template <int NV, int L, bool RT = false>
__device__ __forceinline__ int find_or_put(const TableView& t, const Vec<NV>& key, uint64_t h,
                                        uint32_t& out_idx, LocalCounters& lc) {
  static_assert(L == 8 || L == 16 || L == 32, "line of 8, 16 or 32 buckets");
  constexpr int NS = L / kSectorBuckets;  // sectors per line
  const uint32_t memo = memo_of(h);
  const uint32_t index = (uint32_t)h & t.nb_mask;
  const uint32_t off = index & (L - 1);
  const uint32_t s0 = off >> 3;          // first sector of the walk
  const uint32_t p0 = off & 7;           // first position inside it
  const uint32_t step = (memo << 1) | 1u;
  uint32_t line = index / L;

  for (uint32_t r = 0; r <= t.max_rehash; ++r) {
    if (r) {
      lc.rehashes++;
      if ((r & 31) == 0 && ld_relaxed(&t.ctr->err) != 0) return FOP_ERR;  // another key failed
      line = (line + step) & t.lines_mask;
    }
    const uint32_t line_base = line * L;
    // A sector is kept as three 8-bit masks (empty / memo-equal / done), not
    // as its eight words: the walk only ever acts on empty or memo-equal
    // buckets, whose words the masks determine.  f_* hold sector s0 for the
    // wrap-around part of the walk (a longer line visits it twice).
    uint32_t f_emp = 0, f_mem = 0, f_dn = 0;
#pragma unroll 1
    for (int v = 0; v <= NS; ++v) {
      const uint32_t sec = (s0 + (uint32_t)v) & (NS - 1);
      const uint32_t base = line_base + sec * 8;
      uint32_t emp, mem, dn;
      if (v == 0 || v != NS) {
        uint4 a, b;
        ld_sector(t.buckets + base, a, b);
        const uint32_t wd[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        emp = 0;
        mem = 0;
        dn = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          emp |= (wd[k] == 0u ? 1u : 0u) << k;
          mem |= ((wd[k] & kMemoMask) == memo ? 1u : 0u) << k;
          dn |= (wd[k] >> 31) << k;
        }
        if (v == 0) {
          f_emp = emp;
          f_mem = mem;
          f_dn = dn;
        }
      } else {
        emp = f_emp;
        mem = f_mem;
        dn = f_dn;
      }
      // positions of this visit, in walk order = ascending inside the sector
      uint32_t todo = (v == 0) ? (0xFFu << p0) & 0xFFu : (v == NS) ? (1u << p0) - 1u : 0xFFu;
      while (todo) {
        const uint32_t cand = (emp | mem) & todo;
        if (!cand) break;
        const int pos = __ffs(cand) - 1;
        const uint32_t bit = 1u << pos;
        const uint32_t i = base + pos;
        bool acquired = (VSS_ACQ_MODE == 1);  // sector words came from acquire loads
        if (emp & bit) {
          const uint32_t old = atomicCAS(t.buckets + i, 0u, memo);  // <memo, write>
          if (old == 0u) {
            if (RT) store_row_rt<NV>(t.data + (size_t)i * t.nv, key, t.nv);
            else store_row<NV>(t.data + (size_t)i * NV, key);
            fence_acq_rel();                 // data before <memo, done>
            st_relaxed(t.buckets + i, memo | kDone);
            out_idx = i;
            return FOP_NEW;
          }
          // another thread claimed it first: re-evaluate with the word it wrote
          acquired = false;  // a relaxed CAS result: fence before reading the row
          emp &= ~bit;
          mem = ((old & kMemoMask) == memo) ? (mem | bit) : (mem & ~bit);
          dn = (old & kDone) ? (dn | bit) : (dn & ~bit);
        }
        if (mem & bit) {
          uint32_t b = memo | ((dn & bit) ? kDone : 0u);
          if (!(b & kDone)) {
            if (!wait_done(t, i, b, lc)) return FOP_ERR;
            acquired = true;
          }
          if (data_equal_after_done<NV, RT>(t, i, key, acquired)) {
            out_idx = i;
            return FOP_SEEN;
          }
        }
        todo &= ~((2u << pos) - 1u);  // this position is settled; continue the walk
      }
    }
  }
  latch_error(t.ctr, HT_ERR_FULL);
  return FOP_ERR;
}

}  // namespace vss
