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
// hashing with an odd step over a power-of-two line count, Section 3.2), or
// line + 1 when the table's rehash rule is the next line.
#pragma once

#include "common.cuh"

namespace vss {

// How a probe orders its read of a data row after the <memo, done> bucket
// word it observed (Section 3.3 memory-model requirement):
//   1 (default): bucket sectors are read with gpu-scope acquire loads, so
//                every later load of the thread is ordered after them;
//   0:           bucket sectors are read relaxed and an acquire fence is
//                issued before a data row is compared.
// Resident blocks of 256 threads per SM that the one-thread-per-key table
// kernels are compiled for (__launch_bounds__): five (48 registers; with
// 16-word rows about 120 bytes spill to L1) for rows of up to 16 words -- the
// extra threads keep more random accesses in flight, measured 2 % faster than
// four -- and four for wider rows, which would spill far more.
template <int NV>
constexpr int table_min_blocks() {
#ifdef VSS_TABLE_MINB
  return VSS_TABLE_MINB;  // a fixed count for every width (measurement builds)
#else
  return NV <= 4 ? 5 : 4;
#endif
}

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

// Bucket word formats (Section 3.2: memoised hash plus the write bit), by width.
// A 32-byte sector holds 8 buckets of 32 bits or 16 of 16 bits; `masks` turns
// one sector, read as eight 32-bit words, into per-bucket bit masks: empty,
// memo-equal (write or done) and done.
template <int BW>
struct Bucket;

template <>
struct Bucket<32> {
  static constexpr int kPerSector = 8;
  static constexpr uint32_t kDoneBit = kDone;
  static constexpr uint32_t kMemoBits = kMemoMask;
  __device__ static uint32_t memo(uint64_t h) { return memo_of(h); }
  __device__ static void masks(const uint32_t (&wd)[8], uint32_t memo, uint32_t& emp, uint32_t& mem,
                               uint32_t& dn) {
    emp = 0;
    mem = 0;
    dn = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      emp |= (wd[k] == 0u ? 1u : 0u) << k;
      mem |= ((wd[k] & kMemoMask) == memo ? 1u : 0u) << k;
      dn |= (wd[k] >> 31) << k;
    }
  }
  __device__ static uint32_t cas(uint32_t* buckets, uint32_t i, uint32_t val) {
    return atomicCAS(buckets + i, 0u, val);
  }
  __device__ static void publish(uint32_t* buckets, uint32_t i, uint32_t val) {
    st_relaxed(buckets + i, val);
  }
  __device__ static uint32_t load_acquire(const uint32_t* buckets, uint32_t i) {
    return ld_acquire(buckets + i);
  }
  __device__ static uint32_t load_relaxed(const uint32_t* buckets, uint64_t i) {
    return ld_relaxed(buckets + i);
  }
};

template <>
struct Bucket<16> {
  static constexpr int kPerSector = 16;
  static constexpr uint32_t kDoneBit = HT_BUCKET16_DONE;
  static constexpr uint32_t kMemoBits = HT_BUCKET16_MEMO;
  __device__ static uint32_t memo(uint64_t h) { return memo16_of(h); }
  __device__ static void masks(const uint32_t (&wd)[8], uint32_t memo, uint32_t& emp, uint32_t& mem,
                               uint32_t& dn) {
    // bucket 2k is the low half of word k, bucket 2k+1 the high half
    const uint32_t memo2 = memo * 0x10001u;
    emp = 0;
    mem = 0;
    dn = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t e = __vcmpeq2(wd[k], 0u);                      // 0xFFFF per empty half
      const uint32_t m = __vcmpeq2(wd[k] & 0x7FFF7FFFu, memo2);    // per memo-equal half
      emp |= ((e & 1u) | ((e >> 15) & 2u)) << (2 * k);
      mem |= ((m & 1u) | ((m >> 15) & 2u)) << (2 * k);
      dn |= (((wd[k] >> 15) & 1u) | ((wd[k] >> 30) & 2u)) << (2 * k);
    }
  }
  __device__ static uint32_t cas(uint32_t* buckets, uint32_t i, uint32_t val) {
    return atomicCAS(reinterpret_cast<unsigned short*>(buckets) + i, (unsigned short)0,
                     (unsigned short)val);
  }
  __device__ static void publish(uint32_t* buckets, uint32_t i, uint32_t val) {
    st_relaxed_u16(reinterpret_cast<uint16_t*>(buckets) + i, val);
  }
  __device__ static uint32_t load_acquire(const uint32_t* buckets, uint32_t i) {
    return ld_acquire_u16(reinterpret_cast<const uint16_t*>(buckets) + i);
  }
  __device__ static uint32_t load_relaxed(const uint32_t* buckets, uint64_t i) {
    return ld_relaxed_u16(reinterpret_cast<const uint16_t*>(buckets) + i);
  }
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
template <int BW>
__device__ __forceinline__ bool wait_done(const TableView& t, uint32_t i, uint32_t& b,
                                          LocalCounters& lc) {
  uint32_t spins = 0, ns = 16;
  lc.busy_waits++;
  while (!(b & Bucket<BW>::kDoneBit)) {
    if (++spins > t.max_spin) {
      latch_error(t.ctr, HT_ERR_TIMEOUT);
      return false;
    }
    __nanosleep(ns);
    ns = ns < 256 ? ns * 2 : ns;
    b = Bucket<BW>::load_acquire(t.buckets, i);
  }
  return true;
}

template <int NV, int L, bool RT = false, int BW = 32>
__device__ __forceinline__ int find_or_put(const TableView& t, const Vec<NV>& key, uint64_t h,
                                        uint32_t& out_idx, LocalCounters& lc) {
  using Bk = Bucket<BW>;
  constexpr int SB = Bk::kPerSector;      // buckets per 32-byte sector
  constexpr uint32_t kAll = (1u << SB) - 1u;
  static_assert(L % SB == 0 && L / SB >= 1 && L / SB <= 4, "line of 1, 2 or 4 sectors");
  constexpr int NS = L / SB;              // sectors per line
  const uint32_t memo = Bk::memo(h);
  const uint32_t off = (uint32_t)h & (L - 1);
  const uint32_t s0 = off / SB;           // first sector of the walk
  const uint32_t p0 = off % SB;           // first position inside it
  // line = (h / L) mod lines: a mask for power-of-two tables, otherwise a
  // division by the invariant line count (Section 3.1).  The rehash step is
  // odd for power-of-two line counts and in [1, lines - 1] otherwise (coprime
  // to a prime line count), so the line sequence visits every line.
  const bool pow2 = t.lines_div.m == 0;
  uint32_t line, step;
  if (pow2) {
    line = ((uint32_t)h & t.nb_mask) / L;
    step = (memo << 1) | 1u;
  } else {
    constexpr int kLog2L = L == 8 ? 3 : L == 16 ? 4 : L == 32 ? 5 : 6;
    line = div_r(t.lines_div, h >> kLog2L);
    constexpr int kMemoBits = BW == 32 ? 31 : 15;
    step = 1u + __umulhi(memo << (32 - kMemoBits), t.lines - 1u);
  }
  if (t.rehash_linear) step = 1u;  // ht_params.rehash = 1: the next line

  for (uint32_t r = 0; r <= t.max_rehash; ++r) {
    if (r) {
      lc.rehashes++;
      if ((r & 31) == 0 && ld_relaxed(&t.ctr->err) != 0) return FOP_ERR;  // another key failed
      if (pow2) {
        line = (line + step) & t.lines_mask;
      } else {
        line += step;
        line = line >= t.lines ? line - t.lines : line;
      }
    }
    const uint32_t line_base = line * L;
    // A sector is kept as three bit masks (empty / memo-equal / done), not
    // as its words: the walk only ever acts on empty or memo-equal buckets,
    // whose words the masks determine.  f_* hold sector s0 for the
    // wrap-around part of the walk (a longer line visits it twice).
    uint32_t f_emp = 0, f_mem = 0, f_dn = 0;
#pragma unroll 1
    for (int v = 0; v <= NS; ++v) {
      const uint32_t sec = (s0 + (uint32_t)v) & (NS - 1);
      const uint32_t base = line_base + sec * SB;
      uint32_t emp, mem, dn;
      if (v == 0 || v != NS) {
        uint4 a, b;
        // sector start in bytes: base * BW / 8, a multiple of 32
        ld_sector(t.buckets + (size_t)base * BW / 32, a, b);
        const uint32_t wd[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        Bk::masks(wd, memo, emp, mem, dn);
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
      uint32_t todo = (v == 0) ? (kAll << p0) & kAll : (v == NS) ? (1u << p0) - 1u : kAll;
      while (todo) {
        const uint32_t cand = (emp | mem) & todo;
        if (!cand) break;
        const int pos = __ffs(cand) - 1;
        const uint32_t bit = 1u << pos;
        const uint32_t i = base + pos;
        bool acquired = (VSS_ACQ_MODE == 1);  // sector words came from acquire loads
        if (emp & bit) {
          const uint32_t old = Bk::cas(t.buckets, i, memo);  // <memo, write>
          if (old == 0u) {
            if (RT) store_row_rt<NV>(t.data + (size_t)i * t.nv, key, t.nv);
            else store_row<NV>(t.data + (size_t)i * NV, key);
            fence_acq_rel();                 // data before <memo, done>
            Bk::publish(t.buckets, i, memo | Bk::kDoneBit);
            out_idx = i;
            return FOP_NEW;
          }
          // another thread claimed it first: re-evaluate with the word it wrote
          acquired = false;  // a relaxed CAS result: fence before reading the row
          emp &= ~bit;
          mem = ((old & Bk::kMemoBits) == memo) ? (mem | bit) : (mem & ~bit);
          dn = (old & Bk::kDoneBit) ? (dn | bit) : (dn & ~bit);
        }
        if (mem & bit) {
          uint32_t b = memo | ((dn & bit) ? Bk::kDoneBit : 0u);
          if (!(b & Bk::kDoneBit)) {
            if (!wait_done<BW>(t, i, b, lc)) return FOP_ERR;
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
