// Sub-warp cooperative find-or-put: G lanes own one key and read its whole
// line at once (Alg. "find-or-put" with Alg. "Walking the (cache) line").
//
// The line is 4*G buckets (G = 2, 4, 8: a 32-, 64- or 128-byte line); lane j
// of the group loads buckets 4j..4j+3 with one 16-byte acquire load, and the
// group ORs its lanes' bucket masks (empty / memo-equal / done) together with
// shuffles.  Rotating the masks by the key's offset puts them in walk order,
// so the group acts on the first empty-or-memo-equal bucket exactly as the
// one-thread walk in table.cuh does: the group leader claims an empty bucket
// with CAS; the lanes write or compare the data row in 16-byte chunks (lane j
// takes chunks j, j+G, ...).  Results, rehash sequence and line selection are
// those of find_or_put for a line of 4*G buckets.
//
// Memory ordering (Section 3.3): writer lanes store their chunks and fence,
// the group meets at __syncwarp (which orders memory among its lanes), and
// the leader publishes <memo, done>.  A reader group observed the done bit
// with an acquire load (or fences after a relaxed CAS result) in one lane and
// meets at __syncwarp before any lane reads the row.
#pragma once

#include "table.cuh"

namespace vss {

template <int G>
__device__ __forceinline__ uint32_t group_or(uint32_t x, unsigned gmask) {
#pragma unroll
  for (int s = 1; s < G; s <<= 1) x |= __shfl_xor_sync(gmask, x, s);
  return x;
}

// All lanes of the group call this with the same key and hash; all get the
// same result.  gl = lane index inside the group, gmask = the group's lanes.
template <int NV, int G>
__device__ __forceinline__ int find_or_put_group(const TableView& t, const Vec<NV>& key, uint64_t h,
                                                 uint32_t& out_idx, LocalCounters& lc, int gl,
                                                 unsigned gmask) {
  static_assert(G == 2 || G == 4 || G == 8, "groups of 2, 4 or 8 lanes");
  constexpr int L = 4 * G;
  constexpr uint32_t kAll = L == 32 ? 0xFFFFFFFFu : (1u << L) - 1u;
  const int leader = (int)(lane_id() & ~(unsigned)(G - 1));
  const uint32_t memo = memo_of(h);
  const uint32_t off = (uint32_t)h & (L - 1);
  const bool pow2 = t.lines_div.m == 0;
  uint32_t line, step;
  if (pow2) {
    line = ((uint32_t)h & t.nb_mask) / L;
    step = (memo << 1) | 1u;
  } else {
    constexpr int kLog2L = G == 2 ? 3 : G == 4 ? 4 : 5;
    line = div_r(t.lines_div, h >> kLog2L);
    step = 1u + __umulhi(memo << 1, t.lines - 1u);
  }
  if (t.rehash_linear) step = 1u;  // ht_params.rehash = 1: the next line
  // masks in walk order: bit p <-> bucket (off + p) mod L
  auto rot = [&](uint32_t m) -> uint32_t {
    return off ? ((m >> off) | (m << (L - off))) & kAll : m;
  };

  for (uint32_t r = 0; r <= t.max_rehash; ++r) {
    if (r) {
      if (gl == 0) lc.rehashes++;  // once per group
      if ((r & 31) == 0) {  // another key failed: the whole group leaves together
        const bool failed = ld_relaxed(&t.ctr->err) != 0;
        if (__any_sync(gmask, failed)) return FOP_ERR;
      }
      if (pow2) {
        line = (line + step) & t.lines_mask;
      } else {
        line += step;
        line = line >= t.lines ? line - t.lines : line;
      }
    }
    const uint32_t line_base = line * L;
    const uint4 w = ld_acquire_v4(t.buckets + line_base + 4 * gl);
    const uint32_t wd[4] = {w.x, w.y, w.z, w.w};
    uint32_t emp = 0, mem = 0, dn = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      emp |= (wd[k] == 0u ? 1u : 0u) << k;
      mem |= ((wd[k] & kMemoMask) == memo ? 1u : 0u) << k;
      dn |= (wd[k] >> 31) << k;
    }
    emp = group_or<G>(emp << (4 * gl), gmask);
    mem = group_or<G>(mem << (4 * gl), gmask);
    dn = group_or<G>(dn << (4 * gl), gmask);
    uint32_t todo = kAll;  // walk positions not yet settled
    while (true) {
      const uint32_t cand = rot(emp | mem) & todo;
      if (!cand) break;
      const int p = __ffs(cand) - 1;
      const uint32_t pos = (off + (uint32_t)p) & (L - 1);
      const uint32_t bit = 1u << pos;
      const uint32_t i = line_base + pos;
      bool acquired = true;
      if (emp & bit) {
        uint32_t old = 0;
        if ((int)lane_id() == leader) old = atomicCAS(t.buckets + i, 0u, memo);  // <memo, write>
        old = __shfl_sync(gmask, old, leader);
        if (old == 0u) {
          uint4* row = t.data + (size_t)i * NV;
#pragma unroll
          for (int j = 0; j < NV; ++j)
            if (j % G == gl) row[j] = key.c[j];
          fence_acq_rel();
          __syncwarp(gmask);
          if ((int)lane_id() == leader) {
            fence_acq_rel();               // every lane's chunk before <memo, done>
            st_relaxed(t.buckets + i, memo | kDone);
          }
          out_idx = i;
          return FOP_NEW;
        }
        acquired = false;
        emp &= ~bit;
        mem = ((old & kMemoMask) == memo) ? (mem | bit) : (mem & ~bit);
        dn = (old & kDone) ? (dn | bit) : (dn & ~bit);
      }
      if (mem & bit) {
        if (!(dn & bit)) {
          int ok = 1;
          if ((int)lane_id() == leader) {
            uint32_t b = memo;
            ok = wait_done<32>(t, i, b, lc) ? 1 : 0;
          }
          ok = __shfl_sync(gmask, ok, leader);
          if (!ok) return FOP_ERR;
          acquired = false;  // the leader acquired; the others order through it
        }
        if (!acquired) fence_acq_rel();
        __syncwarp(gmask);
        const uint4* row = t.data + (size_t)i * NV;
        bool same = true;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          if (j % G == gl) {
            const uint4 x = ld_relaxed_v4(row + j);
            const uint4 k = key.c[j];
            same = same && x.x == k.x && x.y == k.y && x.z == k.z && x.w == k.w;
          }
        }
        if (__all_sync(gmask, same)) {
          out_idx = i;
          return FOP_SEEN;
        }
      }
      todo &= ~((2u << p) - 1u);
    }
  }
  latch_error(t.ctr, HT_ERR_FULL);
  return FOP_ERR;
}

}  // namespace vss
