// Device side of level-synchronous reachability (Alg. "Reachability
// analysis"): per-level expansion, the device-wide level barrier and the two
// drivers' kernels.  The kernels are templates over the row chunks NV, the
// line length L and the bucket width BW; their instantiations are spread over
// several translation units (reach_k*.cu) so that they compile in parallel.
#pragma once

#include "expand.cuh"

namespace vss {

#ifndef VSS_ROUNDS_PER_WARP
#define VSS_ROUNDS_PER_WARP 1  // target rounds per warp and level (more measured slower)
#endif
#ifndef VSS_BARRIER_STATS
#define VSS_BARRIER_STATS 0  // measurement builds only: record barrier arrival spreads
#endif
// Resident blocks of 256 threads per SM that the expansion kernels are
// compiled for (__launch_bounds__): four (64 registers) for rows of up to 16
// words, where the shared memory of four blocks fits and the extra warps keep
// more random accesses in flight; three (80 registers) for wider rows, whose
// shared memory allows only three blocks anyway.
template <int NV>
constexpr int reach_min_blocks() {
#ifdef VSS_REACH_MINB
  return VSS_REACH_MINB;  // a fixed count for every width (measurement builds)
#else
  return NV <= 4 ? 4 : 3;
#endif
}
constexpr int kModelMaxWords = 1 << 15;    // model blob capacity (int32 words, 128 KiB)
constexpr int kHdr = 16;                   // blob header words

// Model blob (int32 words):
//   [0] P  [1] S  [2] W  [3] n_local_total  [4] E  [5] crit_any
//   [6] off_base [7] off_crit [8] off_eb [9] off_edges [10] off_uval [11] off_init
//   [12] smem_words (words copied to shared memory: everything before off_init)
//   [13] maxfan = sum over processes of the largest out-degree (bound on a state's successors)
//   [14] spw_max = states per warp round, min(32, kDescCap / maxfan)
// edges are int4 {dst, guard_var, guard_val, upd_var}; uval[e] = upd_val.
struct __align__(16) ReachTotals {
  unsigned long long transitions;
  unsigned long long deadlocks;
  unsigned long long digest;
  unsigned long long stored;
  uint32_t counts[4];   // frontier sizes, rotating over 3 levels
  uint32_t cursor[4];   // next unclaimed frontier row of a level, rotating over 3 levels
  uint32_t bar_count;   // grid-barrier arrivals since the run started (only grows)
  uint32_t bar_pad;
  uint32_t n_levels;
  uint32_t pad;
  unsigned long long first_deadlock;  // tracing: see TraceDev
};

struct ReachDev {
  const int* blob;
  int smem_words;
  uint4* frontier0;           // frontier rows (state vectors, nv chunks each)
  uint4* frontier1;
  uint32_t cap;               // rows per frontier array
  ReachTotals* tot;
  unsigned long long* level_sizes;
  unsigned long long* level_ns;   // globaltimer at the start of each level (persistent driver)
  uint32_t* idx0;                 // tracing: bucket index of each frontier row
  uint32_t* idx1;
  uint32_t* parent;               // tracing: bucket of the predecessor that inserted a state
  uint32_t max_levels;
  uint32_t bar_spin;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ SModel load_model_smem(const ReachDev& rd, int* sm) {
  for (int i = threadIdx.x; i < rd.smem_words; i += blockDim.x) sm[i] = __ldg(rd.blob + i);
  __syncthreads();
  SModel m;
  m.P = sm[0];
  m.S = sm[1];
  m.W = sm[2];
  m.crit_any = sm[5];
  m.maxfan = sm[13];
  m.spw_max = sm[14];
  m.base = sm + sm[6];
  m.crit = sm + sm[7];
  m.eb = sm + sm[8];
  m.edges = reinterpret_cast<const int4*>(sm + sm[9]);
  m.uval = sm + sm[10];
  return m;
}

// One level: a warp takes `spw` consecutive frontier states per round (spw
// shrinks on small levels so that every warp gets work) and expands them with
// expand_round.
template <int NV, int L, int BW, bool TR = false, int G = 1>
__device__ __forceinline__ void run_level(const TableView& t, const SModel& m, const uint4* cur,
                                          uint32_t n_cur, uint32_t* cursor, uint4* next,
                                          uint32_t* next_count, uint32_t cap, Acc& acc,
                                          LocalCounters& lc, uint32_t* wsm,
                                          const TraceDev* tr = nullptr) {
  const unsigned lane = lane_id();
  const uint32_t wpb = blockDim.x >> 5;
  const uint32_t warps = gridDim.x * wpb;
  // aim for several rounds per warp so that the dynamic claims balance the
  // level's end (a single static round leaves the level to its slowest warp)
  const uint32_t per = warps * (uint32_t)VSS_ROUNDS_PER_WARP;
  uint32_t spw = (n_cur + per - 1) / per;
  spw = spw < 1u ? 1u : (spw > (uint32_t)m.spw_max ? (uint32_t)m.spw_max : spw);
  const uint32_t warp_id = blockIdx.x * wpb + (threadIdx.x >> 5);
  const uint64_t static_rows = (uint64_t)warps * spw;
  for (bool first = true;; first = false) {
    // the first round is static (warp w takes rows w*spw ..); later rounds are
    // claimed from the level cursor, so warps that finish early take more,
    // and a level that fits in one round costs no atomic at all
    uint64_t base = (uint64_t)warp_id * spw;
    if (!first) {
      if (static_rows >= n_cur) break;
      uint32_t c0 = 0;
      if (lane == 0) c0 = atomicAdd(cursor, spw);
      base = static_rows + __shfl_sync(0xffffffffu, c0, 0);
    }
    if (base >= n_cur) {
      if (first) continue;
      break;
    }
    expand_round<NV, L, false, TR, BW, G>(t, m, cur, n_cur, base, spw, next, next_count, cap, acc, lc,
                                       wsm, tr);
  }
}

__device__ __forceinline__ void flush_acc(const TableView& t, const ReachDev& rd, Acc& acc,
                                          LocalCounters& lc) {
  const unsigned long long tr = warp_sum((unsigned long long)acc.transitions);
  const unsigned long long dl = warp_sum((unsigned long long)acc.deadlocks);
  const unsigned long long dg = warp_sum(acc.digest);
  const unsigned long long st = warp_sum((unsigned long long)acc.stored);
  const uint32_t bw = warp_sum(lc.busy_waits);
  const uint32_t rh = warp_sum(lc.rehashes);
  if (lane_id() == 0) {
    if (tr) atomicAdd(&rd.tot->transitions, tr);
    if (dl) atomicAdd(&rd.tot->deadlocks, dl);
    if (dg) atomicAdd(&rd.tot->digest, dg);
    if (st) atomicAdd(&t.ctr->stored, st);
    if (bw) atomicAdd(&t.ctr->busy_waits, (unsigned long long)bw);
    if (rh) atomicAdd(&t.ctr->rehashes, (unsigned long long)rh);
  }
  acc = Acc();
  lc = LocalCounters();
}

// Insert init (level 0).  Run by one thread.
template <int NV, int L, int BW>
__device__ void seed_init(const TableView& t, const ReachDev& rd, Acc& acc, LocalCounters& lc) {
  const int* init = rd.blob + rd.blob[11];
  Vec<NV> v;
#pragma unroll
  for (int j = 0; j < NV; ++j) v.c[j] = *reinterpret_cast<const uint4*>(init + 4 * j);
  const uint64_t h = table_hash(v, t.state_words, t.seed);
  uint32_t idx = 0;
  const int r = find_or_put<NV, L, false, BW>(t, v, h, idx, lc);
  rd.tot->counts[1] = 0;
  rd.tot->counts[2] = 0;
  if (r == FOP_NEW) {
#pragma unroll
    for (int j = 0; j < NV; ++j) rd.frontier0[j] = v.c[j];
    rd.tot->pad = idx;
    rd.tot->counts[0] = 1;
    rd.level_sizes[0] = 1;
    rd.tot->n_levels = 1;
    acc.digest += fingerprint(v, t.state_words);
    acc.stored++;
  } else {
    rd.tot->counts[0] = 0;
    if (r != FOP_ERR) latch_error(t.ctr, HT_ERR_INVALID);  // table was not empty
  }
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The
// arrival counter only grows: barrier number e completes when it reaches
// e * gridDim.x, so arriving is one release-add and waiting one acquire poll
// (no reset, no second flag).  The wait is bounded: after `bar_spin` polls the
// barrier latches HT_ERR_TIMEOUT and returns false; it also returns false as
// soon as any error is latched, so every block leaves the kernel instead of
// waiting for one that already left.
static __device__ bool grid_barrier(const ReachDev& rd, DevCounters* ctr, uint32_t& epoch) {
  __shared__ int ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    int good = 1;
#if VSS_BARRIER_STATS
    // measurement build: first and last block arrival of every barrier
    if (epoch < rd.max_levels) {
      const unsigned long long now = global_ns();
      atomicMin(&rd.level_ns[rd.max_levels / 2 + epoch], now);
      atomicMax(&rd.level_sizes[rd.max_levels / 2 + epoch], now);
    }
#endif
    const uint32_t target = epoch * gridDim.x;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&rd.tot->bar_count) : "memory");
    uint32_t spins = 0, ns = 32;
    while (ld_acquire(&rd.tot->bar_count) < target) {
      if (ld_relaxed(&ctr->err) != 0) { good = 0; break; }
      if (++spins > rd.bar_spin) { latch_error(ctr, HT_ERR_TIMEOUT); good = 0; break; }
      __nanosleep(ns);
      ns = ns < 256 ? ns * 2 : ns;
    }
    if (ld_relaxed(&ctr->err) != 0) good = 0;
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <int NV, int L, int BW, bool TR, int G = 1>
__global__ void __launch_bounds__(256, reach_min_blocks<NV>()) k_reach_persistent(TableView t, ReachDev rd) {
  extern __shared__ int smem[];
  const SModel m = load_model_smem(rd, smem);
  uint32_t* wsm = reinterpret_cast<uint32_t*>(smem + ((rd.smem_words + 3) & ~3)) +
                  (threadIdx.x >> 5) * warp_smem_words_nv(NV);
  Acc acc;
  LocalCounters lc;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    seed_init<NV, L, BW>(t, rd, acc, lc);
    rd.level_ns[0] = global_ns();
    if (TR) {
      rd.idx0[0] = rd.tot->pad;  // seed_init left init's bucket there
      rd.parent[rd.tot->pad] = 0xFFFFFFFFu;
    }
  }
  uint32_t epoch = 0;
  if (grid_barrier(rd, t.ctr, epoch)) {
    uint32_t k = 0;
    for (;;) {
      const uint32_t n_cur = ld_relaxed(&rd.tot->counts[k % 3]);
      const uint4* cur = (k & 1) ? rd.frontier1 : rd.frontier0;
      uint4* next = (k & 1) ? rd.frontier0 : rd.frontier1;
      TraceDev tr;
      if (TR) {
        tr.cur_idx = (k & 1) ? rd.idx1 : rd.idx0;
        tr.next_idx = (k & 1) ? rd.idx0 : rd.idx1;
        tr.parent = rd.parent;
        tr.first_deadlock = &rd.tot->first_deadlock;
        tr.level = k;
      }
      run_level<NV, L, BW, TR, G>(t, m, cur, n_cur, &rd.tot->cursor[k % 3], next,
                           &rd.tot->counts[(k + 1) % 3], rd.cap, acc, lc, wsm, &tr);
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st_relaxed(&rd.tot->counts[(k + 2) % 3], 0u);
        st_relaxed(&rd.tot->cursor[(k + 2) % 3], 0u);
      }
      if (!grid_barrier(rd, t.ctr, epoch)) break;
      const uint32_t n_next = ld_relaxed(&rd.tot->counts[(k + 1) % 3]);
      if (n_next == 0) break;
      ++k;
      if (k >= rd.max_levels) {
        if (threadIdx.x == 0) latch_error(t.ctr, HT_ERR_LEVELS);
        break;
      }
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        rd.level_sizes[k] = n_next;
        rd.level_ns[k] = global_ns();
        rd.tot->n_levels = k + 1;
      }
    }
  }
  flush_acc(t, rd, acc, lc);
}

template <int NV, int L, int BW>
__global__ void k_reach_seed(TableView t, ReachDev rd) {
  Acc acc;
  LocalCounters lc;
  seed_init<NV, L, BW>(t, rd, acc, lc);
  if (acc.digest) atomicAdd(&rd.tot->digest, acc.digest);
  if (acc.stored) atomicAdd(&t.ctr->stored, acc.stored);
}

template <int NV, int L, int BW, int G = 1>
__global__ void __launch_bounds__(256, reach_min_blocks<NV>()) k_reach_level(TableView t, ReachDev rd, uint32_t k) {
  extern __shared__ int smem[];
  const SModel m = load_model_smem(rd, smem);
  uint32_t* wsm = reinterpret_cast<uint32_t*>(smem + ((rd.smem_words + 3) & ~3)) +
                  (threadIdx.x >> 5) * warp_smem_words_nv(NV);
  Acc acc;
  LocalCounters lc;
  const uint32_t n_cur = rd.tot->counts[k % 3];
  const uint4* cur = (k & 1) ? rd.frontier1 : rd.frontier0;
  uint4* next = (k & 1) ? rd.frontier0 : rd.frontier1;
  run_level<NV, L, BW, false, G>(t, m, cur, n_cur, &rd.tot->cursor[k % 3], next,
                       &rd.tot->counts[(k + 1) % 3], rd.cap, acc, lc, wsm);
  flush_acc(t, rd, acc, lc);
}

// One level of the graph driver: a CUDA graph holds a fixed run of these, one
// per level, each preceded by zeroing the next level's count and this
// level's cursor.  A level whose frontier is empty (the search ended before
// it) or that comes after an error returns at once; an active level records
// its size before expanding.
template <int NV, int L, int BW, int G = 1>
__global__ void __launch_bounds__(256, reach_min_blocks<NV>()) k_reach_step(TableView t, ReachDev rd, uint32_t k) {
  const uint32_t n_cur = ld_relaxed(&rd.tot->counts[k % 3]);
  if (n_cur == 0 || ld_relaxed(&t.ctr->err) != 0) return;
  if (k >= rd.max_levels) {
    if (blockIdx.x == 0 && threadIdx.x == 0) latch_error(t.ctr, HT_ERR_LEVELS);
    return;
  }
  if (k > 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    rd.level_sizes[k] = n_cur;
    rd.tot->n_levels = k + 1;
  }
  extern __shared__ int smem[];
  const SModel m = load_model_smem(rd, smem);
  uint32_t* wsm = reinterpret_cast<uint32_t*>(smem + ((rd.smem_words + 3) & ~3)) +
                  (threadIdx.x >> 5) * warp_smem_words_nv(NV);
  Acc acc;
  LocalCounters lc;
  const uint4* cur = (k & 1) ? rd.frontier1 : rd.frontier0;
  uint4* next = (k & 1) ? rd.frontier0 : rd.frontier1;
  run_level<NV, L, BW, false, G>(t, m, cur, n_cur, &rd.tot->cursor[k % 3], next,
                       &rd.tot->counts[(k + 1) % 3], rd.cap, acc, lc, wsm);
  flush_acc(t, rd, acc, lc);
}

// ---------------------------------------------------------------------------
// Dispatch tables: each reach_k*.cu instantiates a share of the shapes.
// ---------------------------------------------------------------------------
struct ReachKernels {
  void (*persistent)(TableView, ReachDev);
  void (*persistent_trace)(TableView, ReachDev);  // nullptr: shape compiled without tracing
  void (*seed)(TableView, ReachDev);
  void (*level)(TableView, ReachDev, uint32_t);
  void (*step)(TableView, ReachDev, uint32_t);  // graph driver's level
};

template <int NV, int L, int BW, int G = 1>
static ReachKernels kernels_for() {
  // tracing is compiled for the default line of each bucket width only (32
  // buckets of 32 bits, 16 of 16 bits), with one lane per successor
  constexpr bool kTrace = G == 1 && (BW == 32 ? L == 32 : L == 16);
  return {k_reach_persistent<NV, L, BW, false, G>,
          kTrace ? k_reach_persistent<NV, L, BW, kTrace, G> : nullptr, k_reach_seed<NV, L, BW>,
          k_reach_level<NV, L, BW, G>, k_reach_step<NV, L, BW, G>};
}

// Cooperative probing (ht_params.group_lanes = G): lines of 4G 32-bit buckets.
template <int NV>
static ReachKernels kernels_group(int G) {
  switch (G) {
    case 2: return kernels_for<NV, 8, 32, 2>();
    case 4: return kernels_for<NV, 16, 32, 4>();
    default: return kernels_for<NV, 32, 32, 8>();
  }
}

template <int NV>
static ReachKernels kernels_w32(int L) {
  switch (L) {
    case 8: return kernels_for<NV, 8, 32>();
    case 16: return kernels_for<NV, 16, 32>();
    default: return kernels_for<NV, 32, 32>();
  }
}

template <int NV>
static ReachKernels kernels_w16(int L) {
  return L == 16 ? kernels_for<NV, 16, 16>() : kernels_for<NV, 32, 16>();
}

// Each returns false when the row-chunk count nv is not among its shapes.
bool reach_kernels_w32_lo(int nv, int L, ReachKernels* out);  // nv 1..4
bool reach_kernels_w32_hi(int nv, int L, ReachKernels* out);  // nv 5..8
bool reach_kernels_w16(int nv, int L, ReachKernels* out);     // nv 1..8
bool reach_kernels_group(int nv, int G, ReachKernels* out);   // nv 1..8, G 2 / 4 / 8

}  // namespace vss
