// Successor generation and one warp round of level expansion, shared by the
// single-model drivers (reach.cu) and the batched driver (batch.cu).
#pragma once

#include "coop.cuh"
#include "table.cuh"

namespace vss {

#ifndef VSS_DESC_CAP
#define VSS_DESC_CAP 960  // words per warp: with 16-word rows, four blocks of 8 warps fit in shared memory
#endif
// A successor descriptor is the 16-bit index of its edge in the device model
// (a model blob of at most 2^15 words holds fewer than 2^16 edges; the edge
// carries its process), so a warp's descriptor words hold two per word.
using desc_t = uint16_t;
constexpr int kDescCap = 2 * VSS_DESC_CAP;  // successor descriptors per warp and round

#ifndef VSS_WARP_DEDUP
#define VSS_WARP_DEDUP 0  // merge equal successors of one warp iteration before probing
#endif

template <int NV>
__host__ __device__ constexpr int row_stride() { return 4 * NV + 4; }  // padded: conflict-free 16 B reads

__host__ __device__ constexpr int warp_smem_words_nv(int nv) { return 32 * (4 * nv + 4) + VSS_DESC_CAP + 32; }

struct SModel {
  int P, S, W, crit_any, maxfan, spw_max;
  const int* base;
  const int* crit;
  const int* eb;
  const int4* edges;
  const int* uval;
};

// An edge of the device model: x = destination local state (bits 0-15) and
// its process (bits 16-30), y / z = guard variable / value, w = updated
// variable (-1 = none).
__device__ __forceinline__ int edge_dst(const int4& E) { return E.x & 0xFFFF; }
__device__ __forceinline__ int edge_proc(const int4& E) { return E.x >> 16; }

// Per-thread counters (a thread sees far fewer than 2^32 transitions between
// flushes); the digest needs all 64 bits.
struct Acc {
  uint32_t transitions = 0, deadlocks = 0, stored = 0;
  unsigned long long digest = 0;
};

// Counterexample support (Alg. "Reachability analysis": a state with no
// successor is a deadlock, "print trace").  With tracing on, frontiers carry
// each state's bucket index beside its row, every inserted state records the
// bucket of the predecessor that inserted it, and the deadlock of the lowest
// level (ties broken by fingerprint bits, then bucket) is kept in one word:
//   (level << 50) | (fingerprint >> 45) << 31 | bucket.
struct TraceDev {
  const uint32_t* cur_idx;
  uint32_t* next_idx;
  uint32_t* parent;
  unsigned long long* first_deadlock;
  uint32_t level;
};

template <int NV>
__device__ __forceinline__ void vec_set(Vec<NV>& v, int i, uint32_t x) {
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    v.c[j].x = (4 * j + 0 == i) ? x : v.c[j].x;
    v.c[j].y = (4 * j + 1 == i) ? x : v.c[j].y;
    v.c[j].z = (4 * j + 2 == i) ? x : v.c[j].z;
    v.c[j].w = (4 * j + 3 == i) ? x : v.c[j].w;
  }
}

// Phase 1 of a round, warp-cooperatively: the warp takes frontier rows
// [base, base + spw) (spw <= 32); lane i < spw reads state i's row, keeps it
// (and its hash sum) in shared memory, and lists the enabled edges of the
// state (next-state) as descriptors (16-bit edge indices) in its own slice of
// the warp's descriptor area; it counts the state's transitions and, when
// there are none, a deadlock.  A warp scan of the counts gives the round's T
// successors (returned; the inclusive prefix per lane stays in shared memory).
// RT: rows have the table's run-time width t.nv (<= NV) instead of NV.
// TR: record predecessors and the first deadlock (tr points to TraceDev).
template <int NV, bool RT, bool TR>
__device__ __forceinline__ uint32_t round_successors(const TableView& t, const SModel& m,
                                                     const uint4* cur, uint32_t n_cur, uint64_t base,
                                                     uint32_t spw, Acc& acc, uint32_t* wsm,
                                                     const TraceDev* tr) {
  constexpr int RS = row_stride<NV>();
  uint32_t* rows = wsm;
  desc_t* desc = reinterpret_cast<desc_t*>(wsm + 32 * RS);
  uint32_t* pref = wsm + 32 * RS + VSS_DESC_CAP;
  const unsigned lane = lane_id();
  const int P = m.P;
  const int maxfan = m.maxfan;
  const uint32_t nvr = RT ? t.nv : (uint32_t)NV;
  uint32_t c = 0;
  const uint64_t f = base + lane;
  if (lane < spw && f < n_cur) {
    uint4* r = reinterpret_cast<uint4*>(rows + lane * RS);
    Vec<NV> v;
    if (RT) load_row_cg_rt<NV>(cur + f * nvr, v, nvr);
    else load_row_cg<NV>(cur + f * NV, v);
#pragma unroll
    for (int j = 0; j < NV; ++j) r[j] = v.c[j];
    // the parent's hash sum, kept in the row's padding for its successors
    const uint64_t hs = hash_sum(v, t.state_words, t.seed);
    rows[lane * RS + 4 * NV] = (uint32_t)hs;
    rows[lane * RS + 4 * NV + 1] = (uint32_t)(hs >> 32);
    const int* rw = reinterpret_cast<const int*>(rows + lane * RS);
    int ncrit = 0;
    if (m.crit_any) {
      for (int p = 0; p < P; ++p) {
        const int cp = m.crit[p];
        ncrit += (cp >= 0 && rw[p] == cp) ? 1 : 0;
      }
    }
    desc_t* d = desc + lane * maxfan;
    for (int p = 0; p < P; ++p) {
      const int s = rw[p];
      const int b = m.base[p] + s;
      const int cp = m.crit[p];
      const int others = ncrit - ((cp >= 0 && s == cp) ? 1 : 0);
      const int e_end = m.eb[b + 1];
      for (int e = m.eb[b]; e < e_end; ++e) {
        const int4 E = m.edges[e];
        if (E.y >= 0 && rw[P + E.y] != E.z) continue;                  // guard
        if (cp >= 0 && edge_dst(E) == cp && others > 0) continue;     // mutex
        d[c++] = (desc_t)e;
      }
    }
    acc.transitions += c;
    if (c == 0) acc.deadlocks++;
    if (TR) {
      const uint32_t my = __ldcg(tr->cur_idx + f);
      rows[lane * RS + 4 * NV + 2] = my;
      if (c == 0) {
        const unsigned long long key = ((unsigned long long)tr->level << 50) |
                                       ((fingerprint(v, t.state_words) >> 45) << 31) | my;
        atomicMin(tr->first_deadlock, key);
      }
    }
  }
  uint32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += y;
  }
  pref[lane] = incl;
  const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();
  return T;
}

// Successor j (< T) of the round listed by round_successors: its vector w and
// table hash h, built from its owner's row and descriptor in shared memory
// (the successor's hash sum from the parent's: only words p and P + upd_var
// change); TR: the owner's bucket index too.
template <int NV, bool TR>
__device__ __forceinline__ void round_successor(const TableView& t, const SModel& m,
                                                const uint32_t* wsm, uint32_t j, Vec<NV>& w,
                                                uint64_t& h, uint32_t& parent_idx) {
  constexpr int RS = row_stride<NV>();
  const uint32_t* rows = wsm;
  const desc_t* desc = reinterpret_cast<const desc_t*>(wsm + 32 * RS);
  const uint32_t* pref = wsm + 32 * RS + VSS_DESC_CAP;
  const int P = m.P;
  uint32_t o = 0;  // owner = first lane whose inclusive prefix exceeds j
#pragma unroll
  for (uint32_t step = 16; step > 0; step >>= 1)
    if (pref[o + step - 1] <= j) o += step;
  const uint32_t k = j - (o ? pref[o - 1] : 0u);
  const int e = (int)desc[o * m.maxfan + k];
  const int4 E = m.edges[e];
  const int p = edge_proc(E);
  const uint32_t* ro = rows + o * RS;
  const uint4* r = reinterpret_cast<const uint4*>(ro);
#pragma unroll
  for (int q = 0; q < NV; ++q) w.c[q] = r[q];
  uint64_t hs = (uint64_t)ro[4 * NV] | ((uint64_t)ro[4 * NV + 1] << 32);
  const uint32_t dst = (uint32_t)edge_dst(E);
  hs += hash_term(t.seed, p, dst) - hash_term(t.seed, p, ro[p]);
  vec_set(w, p, dst);
  if (E.w >= 0) {
    const int q = P + E.w;
    const uint32_t uv = (uint32_t)m.uval[e];
    hs += hash_term(t.seed, q, uv) - hash_term(t.seed, q, ro[q]);
    vec_set(w, q, uv);
  }
  h = hash_final(hs, t.state_words);
  if (TR) parent_idx = ro[4 * NV + 2];
}

// One round of a level, warp-cooperatively and load-balanced over successors.
//
// Phase 1 (round_successors) lists the round's T successors as descriptors.
// Phase 2: lane j, j+32, ... builds successor j (round_successor) and runs
// find-or-put -- so no lane serialises a whole fan-out.  New states are
// appended to the next frontier (rows) with one atomicAdd per warp and
// iteration, straight from registers.
// G > 1 (cooperative probing, coop.cuh): the G lanes of a group build the
// same successor from shared memory and walk its line of 4G buckets together;
// an iteration then covers 32 / G successors and the group's first lane
// answers for it.
template <int NV, int L, bool RT, bool TR = false, int BW = 32, int G = 1>
__device__ __forceinline__ void expand_round(const TableView& t, const SModel& m, const uint4* cur,
                                             uint32_t n_cur, uint64_t base, uint32_t spw,
                                             uint4* next, uint32_t* next_count, uint32_t cap,
                                             Acc& acc, LocalCounters& lc, uint32_t* wsm,
                                             const TraceDev* tr = nullptr) {
  static_assert(G == 1 || ((G == 2 || G == 4 || G == 8) && L == 4 * G && BW == 32 && !RT && !TR &&
                            !VSS_WARP_DEDUP),
                "groups of 2, 4 or 8 lanes walk lines of 4G 32-bit buckets");
  constexpr uint32_t kPer = 32 / G;  // successors per iteration
  const unsigned lane = lane_id();
  const int gl = (int)(lane & (G - 1));
  const unsigned gmask = G == 1 ? 0xffffffffu : ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
  const uint32_t nvr = RT ? t.nv : (uint32_t)NV;
  const uint32_t T = round_successors<NV, RT, TR>(t, m, cur, n_cur, base, spw, acc, wsm, tr);
  const uint32_t iters = (T + kPer - 1) / kPer;
  for (uint32_t it = 0; it < iters; ++it) {
    const uint32_t j = it * kPer + lane / G;  // the same for the lanes of a group
    bool is_new = false;
    uint32_t new_idx = 0;
    Vec<NV> w;
    const bool valid = j < T;
    uint64_t h = 0;
    uint32_t parent_idx = 0;
    if (valid) round_successor<NV, TR>(t, m, wsm, j, w, h, parent_idx);
    // Siblings share successors (diamonds), so equal successors often meet in
    // one iteration: the lowest such lane probes, the others confirm equality
    // word by word and take its answer as "seen" instead of waiting on a
    // bucket in the write state.
    bool probe = valid;
#if VSS_WARP_DEDUP
    int lead = (int)lane;
    {
      const unsigned vmask = __ballot_sync(0xffffffffu, valid);
      const unsigned grp = __match_any_sync(0xffffffffu, h) & vmask;
      if (__any_sync(0xffffffffu, valid && __popc(grp) > 1)) {
        const int ld = valid ? __ffs(grp) - 1 : (int)lane;
        uint32_t diff = 0;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          diff |= __shfl_sync(0xffffffffu, w.c[q].x, ld) ^ w.c[q].x;
          diff |= __shfl_sync(0xffffffffu, w.c[q].y, ld) ^ w.c[q].y;
          diff |= __shfl_sync(0xffffffffu, w.c[q].z, ld) ^ w.c[q].z;
          diff |= __shfl_sync(0xffffffffu, w.c[q].w, ld) ^ w.c[q].w;
        }
        if (valid && ld != (int)lane && diff == 0) {
          probe = false;
          lead = ld;
        }
      }
    }
#endif
    int res = FOP_SEEN;
    uint32_t sidx = 0;
    if constexpr (G == 1) {
      if (probe) res = find_or_put<NV, L, RT, BW>(t, w, h, sidx, lc);
    } else {
      if (probe) {  // uniform over the group
        res = find_or_put_group<NV, G>(t, w, h, sidx, lc, gl, gmask);
        if (gl != 0) res = FOP_SEEN;  // the group's first lane answers
      }
    }
#if VSS_WARP_DEDUP
    {
      const int lres = __shfl_sync(0xffffffffu, res, lead);
      if (valid && !probe && lres == FOP_ERR) res = FOP_ERR;
    }
#endif
    if (valid && res == FOP_NEW) {
      is_new = true;
      acc.digest += fingerprint(w, t.state_words);
      acc.stored++;
      if (TR) {
        tr->parent[sidx] = parent_idx;
        new_idx = sidx;
      }
    }
    const unsigned nb = __ballot_sync(0xffffffffu, is_new);
    if (nb) {
      uint32_t wbase = 0;
      if (lane == 0) wbase = atomicAdd(next_count, (uint32_t)__popc(nb));
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (is_new) {
        const uint32_t pos = wbase + __popc(nb & ((1u << lane) - 1u));
        if (pos < cap) {
          if (RT) store_row_rt<NV>(next + (size_t)pos * nvr, w, nvr);
          else store_row<NV>(next + (size_t)pos * NV, w);
          if (TR) tr->next_idx[pos] = new_idx;
        } else {
          latch_error(t.ctr, HT_ERR_FULL);
        }
      }
    }
  }
  __syncwarp();  // the warp's shared rows/descriptors are rewritten next round
}

}  // namespace vss
