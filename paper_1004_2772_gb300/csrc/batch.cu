// Batched reachability: many independent models in one persistent kernel.
//
// Each model runs its own level-synchronous BFS (Alg. "Reachability analysis")
// on its own table.  There is no grid-wide barrier: a model's level is a set of
// work units (frontier rows) claimed by warps from a per-model 64-bit claim
// word; the warp that finishes the level's last unit advances that model alone
// (records the level size, swaps frontiers, publishes the next level), so the
// levels of different models overlap and a warp never waits while any model
// has unclaimed work.
//
// Tables start from the caller's size estimate and grow at a level boundary
// when the coming level could overflow them: a new table (and frontiers) is
// taken from a device memory pool by a bump allocator, cleared, and every done
// bucket of the old table is re-inserted -- each of these steps is again a set
// of units claimed by whichever warps are free.  The paper claims all memory up
// front and never resizes (Section 3.1); growing is what lets one launch serve
// models whose sizes are only estimated.
//
// Claim word: epoch (14 bits) | phase (2 bits) | units (24 bits) | claimed (24 bits).
// A warp that adds to `claimed` and finds it below `units` owns those units of
// that epoch; the epoch cannot advance until they are reported done, so the
// per-epoch fields it reads (double-buffered by epoch parity) stay valid.  An
// EXPAND unit is a group of grp[epoch & 1] frontier rows: one row while the
// level has at most kExpandUnitsMax rows, more for larger levels, so that a
// level of any size fits the 24-bit fields.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "batch.h"
#include "expand.cuh"
#include "internal.h"

namespace vss {

__device__ __forceinline__ unsigned long long pack_claim(uint32_t epoch, uint32_t phase,
                                                         uint32_t units, uint32_t claimed) {
  return ((unsigned long long)(epoch & 0x3FFFu) << 50) | ((unsigned long long)(phase & 3u) << 48) |
         ((unsigned long long)(units & kUnitsMax) << 24) | (claimed & kUnitsMax);
}
__device__ __forceinline__ uint32_t cl_epoch(unsigned long long w) { return (uint32_t)(w >> 50); }
__device__ __forceinline__ uint32_t cl_phase(unsigned long long w) { return (uint32_t)(w >> 48) & 3u; }
__device__ __forceinline__ uint32_t cl_units(unsigned long long w) { return (uint32_t)(w >> 24) & kUnitsMax; }
__device__ __forceinline__ uint32_t cl_claimed(unsigned long long w) { return (uint32_t)w & kUnitsMax; }

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long atom_add_acqrel64(unsigned long long* p,
                                                               unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

// Mutable fields of a model record are written by whichever thread advanced
// the model last, on any SM: read them through L2 (never a stale L1 line).
template <typename T>
__device__ __forceinline__ T ldm(const T& x) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte field");
  if (sizeof(T) == 4) {
    const uint32_t v = __ldcg(reinterpret_cast<const unsigned int*>(&x));
    T r;
    memcpy(&r, &v, 4);
    return r;
  } else {
    const unsigned long long v = __ldcg(reinterpret_cast<const unsigned long long*>(&x));
    T r;
    memcpy(&r, &v, 8);
    return r;
  }
}

__device__ __forceinline__ TableView model_table(const BatchModel& M, const BatchGlobal& g,
                                                 uint32_t* buckets, uint4* data, uint32_t log2,
                                                 uint32_t line_buckets) {
  TableView t;
  t.buckets = buckets;
  t.data = data;
  t.ctr = const_cast<DevCounters*>(&M.ctr);
  t.seed = g.seed;
  t.nb_mask = (uint32_t)((1ull << log2) - 1);
  const uint32_t lines = (uint32_t)((1ull << log2) / line_buckets);
  t.lines_mask = lines - 1;
  t.max_rehash = lines < 4096u ? lines : 4096u;
  t.max_spin = g.max_spin;
  t.state_words = M.W;
  t.nv = M.nv;
  t.bucket_bits = 32;
  t.lines = lines;
  t.rehash_linear = 0;
  t.lines_div = DivU64{0, 0, 0};  // power-of-two tables only
  return t;
}

__device__ __forceinline__ SModel model_view(const int* blob) {
  SModel m;
  m.P = blob[0];
  m.S = blob[1];
  m.W = blob[2];
  m.crit_any = blob[5];
  m.maxfan = blob[13];
  m.spw_max = blob[14];
  m.base = blob + blob[6];
  m.crit = blob + blob[7];
  m.eb = blob + blob[8];
  m.edges = reinterpret_cast<const int4*>(blob + blob[9]);
  m.uval = blob + blob[10];
  return m;
}

__device__ __forceinline__ uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

__device__ __forceinline__ unsigned long long ld_acquire_sys64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_acquire_sys32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_sys64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ void finish_model(BatchModel& M, const BatchGlobal& g, uint32_t epoch, uint32_t status) {
  if (status) latch_error(&M.ctr, status);
  M.finished = 1;
  __threadfence();
  atomicExch(&M.claim, pack_claim(epoch + 1, PH_DONE, 0, 0));
  if (!g.mb) {
    atomicAdd(&g.st->finished, 1u);
    return;
  }
  // serving: hand the result to the host through the slot's mapped mailbox
  const uint32_t s = (uint32_t)(&M - g.models);
  volatile ServeSlotOut* o = g.out + s;
  o->states = ldm(M.ctr.stored);
  o->transitions = ldm(M.transitions);
  o->deadlocks = ldm(M.deadlocks);
  o->digest = ldm(M.digest);
  o->busy_waits = ldm(M.ctr.busy_waits);
  o->rehashes = ldm(M.ctr.rehashes);
  o->n_levels = ldm(M.n_levels);
  o->status = ldm(M.ctr.err);
  o->grows = ldm(M.grows);
  __threadfence_system();
  st_release_sys64(&g.out[s].seq, ldm(g.accepted[s]));
  atomicSub(&g.st->active, 1u);
}

// Serving: take the jobs the host posted since the last scan into their slots.
// Run by one thread of a warp that found no work.  Returns whether it
// activated any job.
__device__ bool serve_accept(const BatchGlobal& g) {
  const unsigned long long db = ld_acquire_sys64(&g.mb->doorbell);
  if (db == ld_relaxed64(&g.st->seen_doorbell)) return false;
  if (atomicCAS(&g.st->scan_lock, 0u, 1u) != 0u) return false;
  const unsigned long long db2 = ld_acquire_sys64(&g.mb->doorbell);
  bool any = false;
  constexpr int kWords = sizeof(BatchModel) / 8;
  constexpr int kClaimWord = offsetof(BatchModel, claim) / 8;
  for (uint32_t s = 0; s < g.n_models; ++s) {
    const unsigned long long seq = ld_acquire_sys64(&g.in[s].seq);
    if (seq == ldm(g.accepted[s])) continue;
    // the host reuses a slot only after it saw the slot's last job finish
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&g.in[s].rec);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&g.models[s]);
    unsigned long long claim = 0;
    for (int i = 0; i < kWords; ++i) {
      const unsigned long long w = ld_relaxed_sys64(src + i);
      if (i == kClaimWord) claim = w;
      else dst[i] = w;
    }
    g.accepted[s] = seq;
    atomicAdd(&g.st->active, 1u);
    __threadfence();
    atomicExch(&g.models[s].claim, claim);
    any = true;
  }
  st_relaxed64(&g.st->seen_doorbell, db2);
  __threadfence();
  atomicExch(&g.st->scan_lock, 0u);
  return any;
}

__device__ void publish(BatchModel& M, uint32_t epoch, uint32_t phase, uint32_t units) {
  const uint32_t p = epoch & 1u;
  M.done[p] = 0;
  M.next_count[p] = 0;
  __threadfence();
  atomicExch(&M.claim, pack_claim(epoch, phase, units, 0));
}

// An EXPAND epoch over `rows` frontier rows: groups of rows as units when the
// level has more rows than kExpandUnitsMax.
__device__ void publish_expand(BatchModel& M, uint32_t epoch, uint32_t rows) {
  const uint32_t g = rows <= kExpandUnitsMax ? 1u : (rows + kExpandUnitsMax - 1) / kExpandUnitsMax;
  M.grp[epoch & 1u] = g;
  publish(M, epoch, PH_EXPAND, (rows + g - 1) / g);
}

// Set up the next epoch of model M after epoch e (phase ph) completed.  Run by
// one thread, the one that reported the epoch's last unit.
template <int L>
__device__ void advance(BatchModel& M, const BatchGlobal& g, uint32_t e, uint32_t ph) {
  __threadfence();
  if (ldm(M.ctr.err)) {
    finish_model(M, g, e, 0);
    return;
  }
  const uint32_t e1 = e + 1;
  if (ph == PH_CLEAR) {
    if (ldm(M.n_levels) == 0) {
      // the initial table is clear: insert init (level 0)
      const int* init = M.blob + M.blob[11];
      Vec<kBatchNV> v;
#pragma unroll
      for (int j = 0; j < kBatchNV; ++j)
        v.c[j] = j < (int)M.nv ? *reinterpret_cast<const uint4*>(init + 4 * j) : make_uint4(0, 0, 0, 0);
      const TableView t = model_table(M, g, ldm(M.buckets), ldm(M.data), ldm(M.log2_nb), L);
      LocalCounters lc;
      uint32_t idx = 0;
      const int r = find_or_put<kBatchNV, L, true>(t, v, table_hash(v, M.W, g.seed), idx, lc);
      if (r != FOP_NEW) {
        finish_model(M, g, e, HT_ERR_INVALID);
        return;
      }
      store_row_rt<kBatchNV>(ldm(M.fr[0]), v, M.nv);
      M.cur = 0;
      M.n_cur = 1;
      M.level = 0;
      M.level_sizes[0] = 1;
      M.n_levels = 1;
      atomicAdd(&M.digest, (unsigned long long)fingerprint(v, M.W));
      atomicAdd(&M.ctr.stored, 1ull);
      publish_expand(M, e1, 1);
    } else {
      // a grown table is clear: re-insert the old one and copy the frontier
      const uint32_t nrb = (uint32_t)(((1ull << ldm(M.log2_nb)) + kRehashUnit - 1) / kRehashUnit);
      M.n_rehash_b = nrb;
      const uint32_t units = nrb + (ldm(M.n_cur) + kCopyUnit - 1) / kCopyUnit;
      publish(M, e1, PH_REHASH, units);
    }
    return;
  }
  if (ph == PH_REHASH) {
    M.buckets = ldm(M.nbuckets);
    M.data = ldm(M.ndata);
    M.fr[0] = ldm(M.nfr[0]);
    M.fr[1] = ldm(M.nfr[1]);
    M.log2_nb = ldm(M.nlog2);
    publish_expand(M, e1, ldm(M.n_cur));
    return;
  }
  // PH_EXPAND done
  const uint32_t n_next = ldm(M.next_count[e & 1u]);
  if (n_next == 0) {
    finish_model(M, g, e, 0);
    return;
  }
  const uint32_t level = ldm(M.level) + 1;
  if (level >= M.max_levels) {
    finish_model(M, g, e, HT_ERR_LEVELS);
    return;
  }
  M.level = level;
  M.level_sizes[level] = n_next;
  M.n_levels = level + 1;
  M.cur = ldm(M.cur) ^ 1u;
  M.n_cur = n_next;
  // grow before a level that could push the table past grow_at (the coming
  // level adds at most n_next * maxfan states, and never more than the bound)
  const uint32_t lg = ldm(M.log2_nb);
  const double cap = (double)(1ull << lg);
  double need = (double)ldm(M.ctr.stored) + (double)n_next * (double)M.maxfan;
  const unsigned long long bound = M.states_bound;
  if (bound) need = fmin(need, (double)bound);
  if (need > g.grow_at * cap) {
    auto size_for = [&](double states) {
      uint32_t s = lg + 1;
      while (s < 31 && (double)(1ull << s) * g.grow_to < states) ++s;
      return s;
    };
    // a model that outgrows its first table and has a state bound grows once,
    // straight to the bound's size (if that fits the pool): its table then
    // ends at load grow_to instead of up to grow_at, and the states are
    // re-inserted once instead of at every doubling
    uint32_t nl = size_for(need);
    if (bound) {
      const uint32_t nlb = size_for((double)bound);
      if (nlb > nl && (1ull << nlb) / kClearUnit <= kUnitsMax &&
          ld_relaxed64(&g.st->pool_used) + generation_bytes(nlb, M.nv) <= g.pool_bytes)
        nl = nlb;
    }
    if ((1ull << nl) / kClearUnit <= kUnitsMax) {
      const uint64_t bytes = generation_bytes(nl, M.nv);
      const unsigned long long off = atomicAdd(&g.st->pool_used, (unsigned long long)bytes);
      if (off + bytes > g.pool_bytes) {
        finish_model(M, g, e, HT_ERR_OOM);
        return;
      }
      char* p = g.pool + off;
      const uint64_t nb = 1ull << nl;
      M.nbuckets = reinterpret_cast<uint32_t*>(p);
      p += align256(nb * 4);
      M.ndata = reinterpret_cast<uint4*>(p);
      p += align256(nb * 16 * M.nv);
      M.nfr[0] = reinterpret_cast<uint4*>(p);
      p += align256(nb * 16 * M.nv);
      M.nfr[1] = reinterpret_cast<uint4*>(p);
      M.nlog2 = nl;
      M.grows += 1;
      publish(M, e1, PH_CLEAR, (uint32_t)((nb + kClearUnit - 1) / kClearUnit));
      return;
    }
  }
  publish_expand(M, e1, n_next);
}

template <int L>
__global__ void __launch_bounds__(256, 2) k_reach_batch(BatchGlobal g) {
  extern __shared__ uint32_t smem[];
  uint32_t* wsm = smem + (threadIdx.x >> 5) * warp_smem_words_nv(kBatchNV);
  const unsigned lane = lane_id();
  const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint32_t n = g.n_models;
  uint32_t rot = gw * 2654435761u, idle = 0, nap = 64;
  unsigned long long idle_since = 0;
  for (;;) {
    if (ld_relaxed(&g.st->err)) break;
    if (!g.mb && ld_relaxed(&g.st->finished) >= n) break;
    // find a model with unclaimed units: 32 models per step, one per lane
    int m = -1;
    for (uint32_t b = 0; b < n && m < 0; b += 32) {
      const uint32_t k = b + lane;
      const uint32_t mi = (rot + k) % n;
      bool has = false;
      if (k < n) {
        const unsigned long long w = ld_relaxed64(&g.models[mi].claim);
        has = cl_phase(w) != PH_DONE && cl_claimed(w) < cl_units(w);
      }
      const unsigned ball = __ballot_sync(0xffffffffu, has);
      if (ball) m = (int)__shfl_sync(0xffffffffu, mi, __ffs(ball) - 1);
    }
    if (m < 0) {
      // no claimable work: back off (up to ~16 us between looks); every wait
      // here is bounded in time by idle_ns
      if (idle++ == 0) idle_since = global_ns();
      const bool idle_long = global_ns() - idle_since > g.idle_ns;
      if (g.mb) {
        // serving: look for newly posted jobs; leave when nothing is running
        // and the host asked to shut down or nothing arrived for idle_ns (the
        // host relaunches the kernel on its next submission)
        int took = 0, leave = 0;
        if (lane == 0) {
          // only the first warp of each block reads the host mailbox: reads of
          // host-mapped memory are slow, and every idle warp polling them
          // slowed the busy warps down (small jobs took 1.6x longer)
          took = (threadIdx.x < 32 && serve_accept(g)) ? 1 : 0;
          if (!took && ld_relaxed(&g.st->active) == 0) {
            const bool stop = ld_acquire_sys32(&g.mb->shutdown) != 0u;
            const bool posted = ld_acquire_sys64(&g.mb->doorbell) != ld_relaxed64(&g.st->seen_doorbell);
            leave = !posted && (stop || idle_long);
          } else if (!took && global_ns() - idle_since > g.stuck_ns) {
            atomicCAS(&g.st->err, 0u, (uint32_t)HT_ERR_TIMEOUT);
            leave = 1;
          }
        }
        took = __shfl_sync(0xffffffffu, took, 0);
        leave = __shfl_sync(0xffffffffu, leave, 0);
        if (leave) break;
        if (took) {
          idle = 0;
          nap = 64;
          continue;
        }
      } else if (global_ns() - idle_since > g.stuck_ns) {
        if (lane == 0) atomicCAS(&g.st->err, 0u, (uint32_t)HT_ERR_TIMEOUT);
        break;
      }
      __nanosleep(nap);
      nap = nap < 16384 ? nap * 2 : nap;
      continue;
    }
    idle = 0;
    nap = 64;
    rot = rot * 1664525u + 1013904223u;
    BatchModel& M = g.models[m];
    // claim: rows of an EXPAND level (several at a time), single units otherwise
    uint32_t e = 0, ph = PH_DONE, units = 0, u0 = 0, take = 1;
    if (lane == 0) {
      const unsigned long long w = ld_relaxed64(&M.claim);
      if (cl_phase(w) == PH_EXPAND) {
        // the model's fair share of the grid: its level spread over
        // warps / active models, so that a lone model's level takes one short
        // round on every warp while many models keep claims large (in units
        // of grp rows: at most one round of spw_max rows when grp is 1)
        const uint32_t warps = gridDim.x * (blockDim.x >> 5);
        uint32_t active = g.mb ? ld_relaxed(&g.st->active) : g.n_models - ld_relaxed(&g.st->finished);
        active = active < 1u ? 1u : active;
        const uint32_t gr = ldm(M.grp[cl_epoch(w) & 1u]);
        const uint32_t cap = gr >= M.spw_max ? 1u : M.spw_max / (gr ? gr : 1u);
        take = (uint32_t)(((uint64_t)cl_units(w) * active + warps - 1) / warps);
        take = take < 1u ? 1u : (take > cap ? cap : take);
      }
      const unsigned long long old = atom_add_acqrel64(&M.claim, take);
      e = cl_epoch(old);
      ph = cl_phase(old);
      units = cl_units(old);
      u0 = cl_claimed(old);
    }
    e = __shfl_sync(0xffffffffu, e, 0);
    ph = __shfl_sync(0xffffffffu, ph, 0);
    units = __shfl_sync(0xffffffffu, units, 0);
    u0 = __shfl_sync(0xffffffffu, u0, 0);
    take = __shfl_sync(0xffffffffu, take, 0);
    if (ph == PH_DONE || u0 >= units) continue;  // lost the race for this model
    const uint32_t cnt = min(take, units - u0);
    if (ph == PH_CLEAR) {
      const uint64_t nb = 1ull << ldm(M.nlog2);
      uint32_t* nbk = ldm(M.nbuckets);
      const uint4 z = make_uint4(0, 0, 0, 0);
      for (uint32_t q = 0; q < cnt; ++q) {
        const uint64_t b0 = (uint64_t)(u0 + q) * kClearUnit;
        for (uint32_t i = lane; i < kClearUnit / 8; i += 32) {
          const uint64_t b = b0 + (uint64_t)i * 8;
          if (b < nb) st_v8(nbk + b, z, z);
        }
      }
    } else if (ph == PH_EXPAND) {
      const uint32_t lg = ldm(M.log2_nb), cur = ldm(M.cur);
      const TableView t = model_table(M, g, ldm(M.buckets), ldm(M.data), lg, L);
      const SModel sm = model_view(M.blob);
      Acc acc;
      LocalCounters lc;
      // the claimed units' rows, in rounds of at most spw_max rows
      const uint32_t n_cur = ldm(M.n_cur), gr = ldm(M.grp[e & 1u]);
      const uint64_t lo = (uint64_t)u0 * gr;
      const uint64_t hi = min((uint64_t)(u0 + cnt) * gr, (uint64_t)n_cur);
      for (uint64_t b = lo; b < hi; b += M.spw_max) {
        const uint32_t spw = (uint32_t)min((uint64_t)M.spw_max, hi - b);
        expand_round<kBatchNV, L, true>(t, sm, ldm(M.fr[cur]), n_cur, b, spw, ldm(M.fr[cur ^ 1u]),
                                        &M.next_count[e & 1u], (uint32_t)(1ull << lg), acc, lc, wsm);
      }
      const unsigned long long tr = warp_sum((unsigned long long)acc.transitions);
      const unsigned long long dl = warp_sum((unsigned long long)acc.deadlocks);
      const unsigned long long dg = warp_sum(acc.digest);
      const unsigned long long st = warp_sum((unsigned long long)acc.stored);
      const uint32_t bw = warp_sum(lc.busy_waits), rh = warp_sum(lc.rehashes);
      if (lane == 0) {
        if (tr) atomicAdd(&M.transitions, tr);
        if (dl) atomicAdd(&M.deadlocks, dl);
        if (dg) atomicAdd(&M.digest, dg);
        if (st) atomicAdd(&M.ctr.stored, st);
        if (bw) atomicAdd(&M.ctr.busy_waits, (unsigned long long)bw);
        if (rh) atomicAdd(&M.ctr.rehashes, (unsigned long long)rh);
      }
    } else {  // PH_REHASH
      const TableView tn = model_table(M, g, ldm(M.nbuckets), ldm(M.ndata), ldm(M.nlog2), L);
      const uint64_t nb_old = 1ull << ldm(M.log2_nb);
      const uint32_t nrb = ldm(M.n_rehash_b), cur = ldm(M.cur), n_cur = ldm(M.n_cur);
      const uint32_t* obk = ldm(M.buckets);
      const uint4* odata = ldm(M.data);
      const uint4* ofr = ldm(M.fr[cur]);
      uint4* nfr = ldm(M.nfr[cur]);
      LocalCounters lc;
      for (uint32_t q = 0; q < cnt; ++q) {
        const uint32_t u = u0 + q;
        if (u < nrb) {
          for (uint32_t i = lane; i < kRehashUnit; i += 32) {
            const uint64_t b = (uint64_t)u * kRehashUnit + i;
            if (b >= nb_old) break;
            if (!(ld_relaxed(obk + b) & kDone)) continue;
            Vec<kBatchNV> v;
            load_row_rt<kBatchNV>(odata + b * M.nv, v, M.nv);
            uint32_t idx = 0;
            const int r = find_or_put<kBatchNV, L, true>(tn, v, table_hash(v, M.W, g.seed), idx, lc);
            if (r != FOP_NEW && r != FOP_ERR) latch_error(&M.ctr, HT_ERR_INVALID);  // a duplicate
          }
        } else {
          for (uint32_t i = lane; i < kCopyUnit; i += 32) {
            const uint64_t row = (uint64_t)(u - nrb) * kCopyUnit + i;
            if (row >= n_cur) break;
            Vec<kBatchNV> v;
            load_row_cg_rt<kBatchNV>(ofr + row * M.nv, v, M.nv);
            store_row_rt<kBatchNV>(nfr + row * M.nv, v, M.nv);
          }
        }
      }
    }
    // report the units; the warp that completes the epoch advances the model
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      const uint32_t d = atomicAdd(&M.done[e & 1u], cnt) + cnt;
      if (d == units) advance<L>(M, g, e, ph);
    }
    __syncwarp();
  }
}

BatchKernel batch_kernel(int L) {
  switch (L) {
    case 8: return k_reach_batch<8>;
    case 16: return k_reach_batch<16>;
    default: return k_reach_batch<32>;
  }
}

size_t batch_smem_bytes(int threads) {
  return (size_t)(threads / 32) * warp_smem_words_nv(kBatchNV) * 4;
}

static uint64_t up256(uint64_t x) { return (x + 255) & ~255ull; }

}  // namespace vss

using namespace vss;

struct reach_batch {
  int n_models = 0;
  uint32_t max_levels = 0;
  ht_params params{};
  void* owned = nullptr;
  BatchModel* models_dev = nullptr;
  BatchState* state_dev = nullptr;
  unsigned long long* levels_dev = nullptr;
  char* pool = nullptr;
  uint64_t pool_bytes = 0;
  uint64_t pool_initial = 0;
  BatchModel* init_pinned = nullptr;   // the models' initial records (pinned, graph-copyable)
  BatchState* state_init_pinned = nullptr;
  BatchModel* out_pinned = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int blocks = 0, threads = 256;
  size_t smem = 0;
  BatchKernel kernel = nullptr;
  BatchGlobal g{};
};

static uint64_t blob_words_total(const std::vector<std::vector<int>>& blobs) {
  uint64_t w = 0;
  for (auto& b : blobs) w += (b.size() + 63) & ~63ull;  // 256-byte aligned per model
  return w;
}

static uint64_t batch_layout_bytes(int n, uint64_t blob_words, uint32_t max_levels,
                                   uint64_t pool_bytes) {
  return up256((uint64_t)n * sizeof(BatchModel)) + up256(sizeof(BatchState)) + up256(blob_words * 4) +
         up256((uint64_t)n * max_levels * 8) + up256(pool_bytes);
}

static ht_status batch_pack(const reach_model* models, const int32_t* const* inits, int n,
                            std::vector<std::vector<int>>& blobs) {
  if (!models || !inits || n < 1) return HT_ERR_INVALID;
  blobs.resize(n);
  for (int i = 0; i < n; ++i) {
    ht_status st = pack_model(&models[i], inits[i], 32, blobs[i]);
    if (st != HT_OK) return st;
  }
  return HT_OK;
}

extern "C" {

ht_status reach_batch_bytes(const reach_model* models, const int32_t* const* inits, int n_models,
                            uint32_t max_levels, uint64_t pool_bytes, uint64_t* bytes) {
  if (!bytes || max_levels < 1) return HT_ERR_INVALID;
  std::vector<std::vector<int>> blobs;
  ht_status st = batch_pack(models, inits, n_models, blobs);
  if (st != HT_OK) return st;
  *bytes = batch_layout_bytes(n_models, blob_words_total(blobs), max_levels, pool_bytes);
  return HT_OK;
}

ht_status reach_batch_create_at(const reach_model* models, const int32_t* const* inits,
                                int n_models, const int32_t* log2_initial, uint32_t max_levels,
                                uint64_t pool_bytes, const ht_params* params, void* mem_dev,
                                uint64_t mem_bytes, reach_batch_t** out) {
  if (!out || max_levels < 1 || !mem_dev || (reinterpret_cast<uintptr_t>(mem_dev) & 255u))
    return HT_ERR_INVALID;
  *out = nullptr;
  std::vector<std::vector<int>> blobs;
  ht_status st = batch_pack(models, inits, n_models, blobs);
  if (st != HT_OK) return st;
  const uint64_t need = batch_layout_bytes(n_models, blob_words_total(blobs), max_levels, pool_bytes);
  if (mem_bytes < need) return HT_ERR_OOM;
  ht_params p{};
  st = resolve_params(params, 1u << 10, &p);
  if (st != HT_OK) return st;
  // batch tables use 32-bit buckets walked by one thread per key, double hashing
  if (p.bucket_bits != 32 || p.group_lanes != 1 || p.rehash != 0) return HT_ERR_INVALID;
  reach_batch_t* b = new (std::nothrow) reach_batch_t();
  if (!b) return HT_ERR_OOM;
  b->n_models = n_models;
  b->max_levels = max_levels;
  b->params = p;
  char* q = static_cast<char*>(mem_dev);
  b->models_dev = reinterpret_cast<BatchModel*>(q);
  q += up256((uint64_t)n_models * sizeof(BatchModel));
  b->state_dev = reinterpret_cast<BatchState*>(q);
  q += up256(sizeof(BatchState));
  int* blobs_dev = reinterpret_cast<int*>(q);
  q += up256(blob_words_total(blobs) * 4);
  b->levels_dev = reinterpret_cast<unsigned long long*>(q);
  q += up256((uint64_t)n_models * max_levels * 8);
  b->pool = q;
  b->pool_bytes = up256(pool_bytes);

  auto fail = [&](ht_status s) {
    if (b->init_pinned) cudaFreeHost(b->init_pinned);
    if (b->state_init_pinned) cudaFreeHost(b->state_init_pinned);
    if (b->out_pinned) cudaFreeHost(b->out_pinned);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    cudaGetLastError();
    delete b;
    return s;
  };
  if (cudaMallocHost(&b->init_pinned, sizeof(BatchModel) * n_models) != cudaSuccess ||
      cudaMallocHost(&b->out_pinned, sizeof(BatchModel) * n_models) != cudaSuccess ||
      cudaMallocHost(&b->state_init_pinned, sizeof(BatchState)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess)
    return fail(HT_ERR_CUDA);

  // upload the blobs; lay out the initial table generation of every model in the pool
  uint64_t bw = 0, pool_used = 0;
  for (int i = 0; i < n_models; ++i) {
    const std::vector<int>& bl = blobs[i];
    if (cudaMemcpy(blobs_dev + bw, bl.data(), bl.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(HT_ERR_CUDA);
    const reach_model& md = models[i];
    const uint32_t W = (uint32_t)md.state_words, nv = (W + 3) / 4;
    unsigned long long bound = 0;
    if (md.n_shared == 0) {
      long double pr = 1;
      for (int k = 0; k < md.n_procs; ++k) pr *= md.n_local[k];
      bound = pr > 1e15 ? 0 : (unsigned long long)pr;
    }
    int lg = log2_initial ? log2_initial[i] : 0;
    if (lg <= 0) {  // estimate: twice the bound, but start at most at 2^16 buckets
      lg = 10;
      while (lg < 16 && bound && (1ull << lg) < 2 * bound) ++lg;
      if (!bound) lg = 16;
    }
    if (lg < 10 || lg > 31) return fail(HT_ERR_INVALID);
    const uint64_t gen = generation_bytes((uint32_t)lg, nv);
    if (pool_used + gen > b->pool_bytes) return fail(HT_ERR_OOM);
    char* gp = b->pool + pool_used;
    pool_used += gen;
    BatchModel M;
    std::memset(&M, 0, sizeof(M));
    M.blob = blobs_dev + bw;
    M.level_sizes = b->levels_dev + (uint64_t)i * max_levels;
    M.W = W;
    M.nv = nv;
    M.maxfan = (uint32_t)bl[13];
    M.spw_max = (uint32_t)bl[14];
    M.max_levels = max_levels;
    M.log2_nb = (uint32_t)lg;
    const uint64_t nb = 1ull << lg;
    M.buckets = reinterpret_cast<uint32_t*>(gp);
    M.data = reinterpret_cast<uint4*>(gp + up256(nb * 4));
    M.fr[0] = reinterpret_cast<uint4*>(gp + up256(nb * 4) + up256(nb * 16 * nv));
    M.fr[1] = reinterpret_cast<uint4*>(gp + up256(nb * 4) + 2 * up256(nb * 16 * nv));
    M.nbuckets = M.buckets;  // the first CLEAR epoch clears the initial table
    M.nlog2 = M.log2_nb;
    M.states_bound = bound;
    const uint64_t clear_units = (nb + kClearUnit - 1) / kClearUnit;
    M.claim = ((unsigned long long)PH_CLEAR << 48) | (clear_units << 24);
    b->init_pinned[i] = M;
    bw += (bl.size() + 63) & ~63ull;
  }
  b->pool_initial = pool_used;
  std::memset(b->state_init_pinned, 0, sizeof(BatchState));
  b->state_init_pinned->pool_used = pool_used;

  b->kernel = batch_kernel((int)p.line_buckets);
  b->threads = 256;
  b->smem = batch_smem_bytes(b->threads);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(b->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b->kernel, b->threads, b->smem) != cudaSuccess ||
      per_sm < 1)
    return fail(HT_ERR_CUDA);
  b->blocks = per_sm * sms;
  b->g.models = b->models_dev;
  b->g.st = b->state_dev;
  b->g.pool = b->pool;
  b->g.pool_bytes = b->pool_bytes;
  b->g.seed = p.hash_seed;
  b->g.n_models = (uint32_t)n_models;
  b->g.max_spin = p.max_spin;
  b->g.idle_ns = 0;
  b->g.stuck_ns = 4000000000ull;  // 4 s with no claimable work while models are unfinished
  b->g.grow_at = 0.9f;
  b->g.grow_to = 0.5f;
  *out = b;
  return HT_OK;
}

ht_status reach_batch_create(const reach_model* models, const int32_t* const* inits, int n_models,
                             const int32_t* log2_initial, uint32_t max_levels, uint64_t pool_bytes,
                             const ht_params* params, reach_batch_t** out) {
  uint64_t bytes = 0;
  if (!out) return HT_ERR_INVALID;
  *out = nullptr;
  ht_status st = reach_batch_bytes(models, inits, n_models, max_levels, pool_bytes, &bytes);
  if (st != HT_OK) return st;
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return HT_ERR_OOM;
  }
  st = reach_batch_create_at(models, inits, n_models, log2_initial, max_levels, pool_bytes, params,
                             mem, bytes, out);
  if (st != HT_OK) {
    cudaFree(mem);
    return st;
  }
  (*out)->owned = mem;
  return HT_OK;
}

ht_status reach_batch_destroy(reach_batch_t* b) {
  if (!b) return HT_ERR_INVALID;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->init_pinned) cudaFreeHost(b->init_pinned);
  if (b->state_init_pinned) cudaFreeHost(b->state_init_pinned);
  if (b->out_pinned) cudaFreeHost(b->out_pinned);
  if (b->owned) cudaFree(b->owned);
  delete b;
  return HT_OK;
}

// The whole batch as one stream-ordered sequence: reset the model records and
// the pool, then one persistent launch.
static ht_status batch_enqueue(reach_batch_t* b, cudaStream_t s) {
  VSS_CUDA_TRY(cudaMemcpyAsync(b->models_dev, b->init_pinned, sizeof(BatchModel) * b->n_models,
                               cudaMemcpyHostToDevice, s));
  VSS_CUDA_TRY(cudaMemcpyAsync(b->state_dev, b->state_init_pinned, sizeof(BatchState),
                               cudaMemcpyHostToDevice, s));
  b->kernel<<<b->blocks, b->threads, b->smem, s>>>(b->g);
  VSS_CUDA_TRY(cudaGetLastError());
  return HT_OK;
}

ht_status reach_batch_run(reach_batch_t* b, int use_graph, void* stream) {
  if (!b) return HT_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!use_graph) {
    VSS_CUDA_TRY(cudaEventRecord(b->ev0, s));
    ht_status st = batch_enqueue(b, s);
    if (st != HT_OK) return st;
    VSS_CUDA_TRY(cudaEventRecord(b->ev1, s));
    return HT_OK;
  }
  if (!b->exec) {
    VSS_CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    ht_status st = batch_enqueue(b, b->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &g);
    if (st != HT_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return st != HT_OK ? st : HT_ERR_CUDA;
    }
    b->graph = g;
    VSS_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  VSS_CUDA_TRY(cudaEventRecord(b->ev0, s));
  VSS_CUDA_TRY(cudaGraphLaunch(b->exec, s));
  VSS_CUDA_TRY(cudaEventRecord(b->ev1, s));
  return HT_OK;
}

ht_status reach_batch_last_timing(reach_batch_t* b, float* ms) {
  if (!b || !ms) return HT_ERR_INVALID;
  VSS_CUDA_TRY(cudaEventSynchronize(b->ev1));
  VSS_CUDA_TRY(cudaEventElapsedTime(ms, b->ev0, b->ev1));
  return HT_OK;
}

ht_status reach_batch_results(reach_batch_t* b, void* stream, reach_result* outs,
                              uint64_t* level_sizes_host, uint32_t* grows) {
  if (!b || !outs) return HT_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BatchState st;
  VSS_CUDA_TRY(cudaMemcpyAsync(b->out_pinned, b->models_dev, sizeof(BatchModel) * b->n_models,
                               cudaMemcpyDeviceToHost, s));
  VSS_CUDA_TRY(cudaMemcpyAsync(&st, b->state_dev, sizeof(st), cudaMemcpyDeviceToHost, s));
  if (level_sizes_host)
    VSS_CUDA_TRY(cudaMemcpyAsync(level_sizes_host, b->levels_dev,
                                 (size_t)b->n_models * b->max_levels * 8, cudaMemcpyDeviceToHost, s));
  VSS_CUDA_TRY(cudaStreamSynchronize(s));
  ht_status worst = st.err ? (ht_status)st.err : HT_OK;
  for (int i = 0; i < b->n_models; ++i) {
    const BatchModel& M = b->out_pinned[i];
    reach_result& r = outs[i];
    std::memset(&r, 0, sizeof(r));
    r.states = M.ctr.stored;
    r.transitions = M.transitions;
    r.deadlocks = M.deadlocks;
    r.digest = M.digest;
    r.busy_waits = M.ctr.busy_waits;
    r.rehashes = M.ctr.rehashes;
    r.n_levels = M.n_levels;
    r.status = M.ctr.err ? (ht_status)M.ctr.err : (M.finished ? HT_OK : (st.err ? (ht_status)st.err : HT_ERR_TIMEOUT));
    if (grows) grows[i] = M.grows;
    if (r.status != HT_OK && worst == HT_OK) worst = r.status;
  }
  return worst;
}

}  // extern "C"
