// Owner-partitioned reachability: the static state-space partitioning of
// Sec. 4.1 (the design of Spin and DiVinE 2 that the paper compares its
// shared table with: a breadth-first exploration where a hash function assigns
// every successor to the queue of one worker, which checks it against its own
// state storage), as K owner partitions on one GPU.
//
// owner(v) = the top log2(K) bits of the state hash h(v).  Partition o owns a
// table (the store of Sec. 3, unchanged) and a frontier segment.  One BFS level
// (Alg. "Reachability analysis", level-synchronous) is, per chunk of the
// current frontier:
//   expand   every partition's frontier rows are expanded with the same
//            successor generator as the shared-table drivers (round_successors
//            / round_successor); each successor goes, with its hash, to the
//            outbox, and counts[source][owner] is incremented;
//   plan     the counts become inbox offsets: owner o's inbox is the
//            concatenation over sources s of the (s, o) segments -- the layout
//            an all-to-all exchange delivers (receive buffer ordered by source);
//   scatter  outbox entries move to their (source, owner) inbox segment;
//   insert   every owner runs find-or-put on its own table over its inbox and
//            appends new states to its next frontier segment.
// With K ranks instead of K partitions, "plan + scatter" is the all-to-all:
// the counts are exchanged first, then the rows.  Every owner sees exactly the
// successors it owns, so the visited set, the transitions (counted at
// expansion), the level sizes and the digest equal the shared-table run.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "reach_kernels.cuh"

namespace vss {

constexpr int kMaxParts = 16;

struct __align__(16) PartTotals {
  unsigned long long transitions;
  unsigned long long deadlocks;
  unsigned long long digest;
  unsigned long long exchanged;                 // successors whose owner is not their source
  unsigned long long busy_waits;
  unsigned long long rehashes;
  // zeroed before every chunk (one memset from out_count to the end of counts)
  uint32_t out_count;                           // outbox entries of the chunk
  uint32_t cursor;                              // rounds claimed in the chunk
  uint32_t counts[kMaxParts * kMaxParts];       // [source * K + owner]
  // written by the plan
  uint32_t seg_off[kMaxParts * kMaxParts];      // inbox offset of segment (source, owner)
  uint32_t fill[kMaxParts * kMaxParts];         // rows already placed in each segment
  uint32_t in_begin[kMaxParts + 1];             // owner o's inbox: [in_begin[o], in_begin[o + 1])
  uint32_t next_count[kMaxParts];               // rows in each next-frontier segment
};

struct PartDev {
  TableView tv[kMaxParts];
  int K;
  int log2K;
  const int* blob;
  int smem_words;
  uint4* cur;                       // frontier segments: partition p's rows start at row p * seg_rows
  uint4* next;
  uint64_t seg_rows;
  uint32_t ncur[kMaxParts];         // rows in each current segment
  uint32_t round_begin[kMaxParts + 1];  // first round of each partition in this level
  uint32_t spw;                     // frontier rows per warp round
  uint4* out_rows;
  unsigned long long* out_h;
  uint32_t* out_tag;                // source << 16 | owner
  uint4* in_rows;
  unsigned long long* in_h;
  uint32_t cap;                     // outbox and inbox rows
  PartTotals* tot;
};

__device__ __forceinline__ uint32_t owner_of(uint64_t h, int log2K) {
  return log2K ? (uint32_t)(h >> (64 - log2K)) : 0u;
}

__device__ __forceinline__ SModel part_model(const PartDev& pd, int* sm) {
  ReachDev rd{};
  rd.blob = pd.blob;
  rd.smem_words = pd.smem_words;
  return load_model_smem(rd, sm);
}

// Level 0: init goes to its owner's table and next-frontier segment.
template <int NV>
__global__ void k_part_seed(PartDev pd) {
  const int* init = pd.blob + pd.blob[11];
  Vec<NV> v;
#pragma unroll
  for (int j = 0; j < NV; ++j)
    v.c[j] = j < (int)pd.tv[0].nv ? *reinterpret_cast<const uint4*>(init + 4 * j) : make_uint4(0, 0, 0, 0);
  const TableView& t0 = pd.tv[0];
  const uint64_t h = table_hash(v, t0.state_words, t0.seed);
  const uint32_t o = owner_of(h, pd.log2K);
  LocalCounters lc;
  uint32_t idx = 0;
  const int r = find_or_put<NV, 32, true, 32>(pd.tv[o], v, h, idx, lc);
  if (r == FOP_NEW) {
    store_row_rt<NV>(pd.next + (size_t)o * pd.seg_rows * t0.nv, v, t0.nv);
    pd.tot->next_count[o] = 1;
    pd.tot->digest += fingerprint(v, t0.state_words);
    pd.tv[o].ctr->stored = 1;
  } else if (r != FOP_ERR) {
    latch_error(pd.tv[o].ctr, HT_ERR_INVALID);  // the table was not empty
  }
}

// Expansion of rounds [r0, r1) of the level: a warp claims a round (spw rows
// of one partition's segment), lists its successors and sends each to the
// outbox with its hash and (source, owner) tag.
template <int NV>
__global__ void __launch_bounds__(256) k_part_expand(PartDev pd, uint32_t r0, uint32_t r1) {
  extern __shared__ int smem[];
  const SModel m = part_model(pd, smem);
  uint32_t* wsm = reinterpret_cast<uint32_t*>(smem + ((pd.smem_words + 3) & ~3)) +
                  (threadIdx.x >> 5) * warp_smem_words_nv(NV);
  const TableView& t0 = pd.tv[0];
  const uint32_t nvr = t0.nv;
  const unsigned lane = lane_id();
  Acc acc;
  for (;;) {
    uint32_t r = 0;
    if (lane == 0) r = atomicAdd(&pd.tot->cursor, 1u) + r0;
    r = __shfl_sync(0xffffffffu, r, 0);
    if (r >= r1) break;
    int p = 0;
    while (p + 1 < pd.K && pd.round_begin[p + 1] <= r) ++p;
    const uint64_t base = (uint64_t)(r - pd.round_begin[p]) * pd.spw;
    const uint4* cur = pd.cur + (size_t)p * pd.seg_rows * nvr;
    const uint32_t T = round_successors<NV, true, false>(t0, m, cur, pd.ncur[p], base, pd.spw, acc,
                                                         wsm, nullptr);
    const uint32_t iters = (T + 31) / 32;
    for (uint32_t it = 0; it < iters; ++it) {
      const uint32_t j = it * 32 + lane;
      const bool valid = j < T;
      Vec<NV> w;
      uint64_t h = 0;
      uint32_t unused = 0;
      if (valid) round_successor<NV, false>(t0, m, wsm, j, w, h, unused);
      const uint32_t owner = valid ? owner_of(h, pd.log2K) : 0u;
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      uint32_t b = 0;
      if (lane == 0 && vm) b = atomicAdd(&pd.tot->out_count, (uint32_t)__popc(vm));
      b = __shfl_sync(0xffffffffu, b, 0);
      if (valid) {
        const uint32_t pos = b + __popc(vm & ((1u << lane) - 1u));
        if (pos < pd.cap) {
          store_row_rt<NV>(pd.out_rows + (size_t)pos * nvr, w, nvr);
          pd.out_h[pos] = h;
          pd.out_tag[pos] = ((uint32_t)p << 16) | owner;
        } else {
          latch_error(t0.ctr, HT_ERR_FULL);  // the host sizes chunks so that this cannot happen
        }
      }
      // per-(source, owner) counts: one atomic per owner present in the warp
      const unsigned grp = __match_any_sync(0xffffffffu, valid ? owner : 0xFFFFFFFFu);
      if (valid && (int)lane == __ffs(grp) - 1)
        atomicAdd(&pd.tot->counts[p * pd.K + (int)owner], (uint32_t)__popc(grp));
    }
    __syncwarp();  // the warp's shared rows/descriptors are rewritten next round
  }
  const unsigned long long tr = warp_sum((unsigned long long)acc.transitions);
  const unsigned long long dl = warp_sum((unsigned long long)acc.deadlocks);
  if (lane == 0) {
    if (tr) atomicAdd(&pd.tot->transitions, tr);
    if (dl) atomicAdd(&pd.tot->deadlocks, dl);
  }
}

// The exchange plan of the chunk (one thread): owner o's inbox holds the
// segments (0, o), (1, o), ..., (K-1, o) in that order.
__global__ void k_part_plan(PartDev pd) {
  PartTotals* t = pd.tot;
  const int K = pd.K;
  uint32_t run = 0;
  unsigned long long ex = 0;
  for (int o = 0; o < K; ++o) {
    t->in_begin[o] = run;
    for (int s = 0; s < K; ++s) {
      const uint32_t c = t->counts[s * K + o];
      t->seg_off[s * K + o] = run;
      t->fill[s * K + o] = 0;
      run += c;
      if (s != o) ex += c;
    }
  }
  t->in_begin[K] = run;
  t->exchanged += ex;
}

// Outbox -> inbox: each entry to its (source, owner) segment.
__global__ void __launch_bounds__(256) k_part_scatter(PartDev pd) {
  const uint32_t n = min(pd.tot->out_count, pd.cap);
  const uint32_t nvr = pd.tv[0].nv;
  const unsigned lane = lane_id();
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t base = warp * 32; base < n; base += nwarps * 32) {
    const uint64_t i = base + lane;
    const bool valid = i < n;
    const uint32_t tag = valid ? pd.out_tag[i] : 0xFFFFFFFFu;
    const unsigned grp = __match_any_sync(0xffffffffu, tag);
    const int leader = __ffs(grp) - 1;
    const uint32_t slot = (tag >> 16) * (uint32_t)pd.K + (tag & 0xFFFFu);
    uint32_t b = 0;
    if (valid && (int)lane == leader) b = atomicAdd(&pd.tot->fill[slot], (uint32_t)__popc(grp));
    b = __shfl_sync(0xffffffffu, b, leader);
    if (valid) {
      const uint32_t pos = pd.tot->seg_off[slot] + b + __popc(grp & ((1u << lane) - 1u));
      for (uint32_t j = 0; j < nvr; ++j) pd.in_rows[(size_t)pos * nvr + j] = pd.out_rows[i * nvr + j];
      pd.in_h[pos] = pd.out_h[i];
    }
  }
}

// Every owner's find-or-put over its inbox; new states go to its next segment.
template <int NV>
__global__ void __launch_bounds__(256) k_part_insert(PartDev pd) {
  const int K = pd.K;
  const uint32_t n = pd.tot->in_begin[K];
  const TableView& t0 = pd.tv[0];
  const uint32_t nvr = t0.nv;
  const unsigned lane = lane_id();
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  LocalCounters lc;
  unsigned long long digest = 0;
  for (uint64_t base = warp * 32; base < n; base += nwarps * 32) {
    const uint64_t i = base + lane;
    const bool valid = i < n;
    int o = 0;
    while (o + 1 < K && pd.tot->in_begin[o + 1] <= i) ++o;
    bool is_new = false;
    Vec<NV> w;
    if (valid) {
      load_row_rt<NV>(pd.in_rows + (size_t)i * nvr, w, nvr);
      const uint64_t h = pd.in_h[i];
      uint32_t idx = 0;
      is_new = find_or_put<NV, 32, true, 32>(pd.tv[o], w, h, idx, lc) == FOP_NEW;
      if (is_new) digest += fingerprint(w, t0.state_words);
    }
    const unsigned grp = __match_any_sync(0xffffffffu, is_new ? (uint32_t)o : 0xFFFFFFFFu);
    const int leader = __ffs(grp) - 1;
    uint32_t b = 0;
    if (is_new && (int)lane == leader) {
      b = atomicAdd(&pd.tot->next_count[o], (uint32_t)__popc(grp));
      atomicAdd(&pd.tv[o].ctr->stored, (unsigned long long)__popc(grp));
    }
    b = __shfl_sync(0xffffffffu, b, leader);
    if (is_new) {
      const uint32_t pos = b + __popc(grp & ((1u << lane) - 1u));
      if (pos < pd.seg_rows) store_row_rt<NV>(pd.next + ((size_t)o * pd.seg_rows + pos) * nvr, w, nvr);
      else latch_error(pd.tv[o].ctr, HT_ERR_FULL);
    }
  }
  const unsigned long long dg = warp_sum(digest);
  const uint32_t bw = warp_sum(lc.busy_waits);
  const uint32_t rh = warp_sum(lc.rehashes);
  if (lane == 0) {
    if (dg) atomicAdd(&pd.tot->digest, dg);
    if (bw) atomicAdd(&pd.tot->busy_waits, (unsigned long long)bw);
    if (rh) atomicAdd(&pd.tot->rehashes, (unsigned long long)rh);
  }
}

struct PartKernels {
  void (*seed)(PartDev);
  void (*expand)(PartDev, uint32_t, uint32_t);
  void (*insert)(PartDev);
  int nv;  // compiled row chunks (rows of up to 4 * nv words)
};

static PartKernels part_kernels(int nv) {
  if (nv <= 2) return {k_part_seed<2>, k_part_expand<2>, k_part_insert<2>, 2};
  if (nv <= 4) return {k_part_seed<4>, k_part_expand<4>, k_part_insert<4>, 4};
  return {k_part_seed<8>, k_part_expand<8>, k_part_insert<8>, 8};
}

static uint64_t up256(uint64_t x) { return (x + 255) / 256 * 256; }

}  // namespace vss

using namespace vss;

struct part_reach {
  int K = 0;
  int log2K = 0;
  uint64_t nbp = 0;  // buckets per partition
  int max_words = 0;
  uint64_t cap = 0;
  ht_t tables[kMaxParts];
  int* blob = nullptr;
  uint4* fr[2] = {nullptr, nullptr};
  uint4* out_rows = nullptr;
  unsigned long long* out_h = nullptr;
  uint32_t* out_tag = nullptr;
  uint4* in_rows = nullptr;
  unsigned long long* in_h = nullptr;
  PartTotals* tot = nullptr;
  PartTotals* host_tot = nullptr;  // pinned
  int num_sms = 0;
};

static bool part_shape_ok(int n_parts, int log2_buckets_part, int max_state_words, uint64_t exchange_rows) {
  return n_parts >= 1 && n_parts <= kMaxParts && (n_parts & (n_parts - 1)) == 0 && log2_buckets_part >= 10 &&
         log2_buckets_part <= 31 && max_state_words >= 1 && max_state_words <= 32 &&
         exchange_rows >= (uint64_t)VSS_DESC_CAP && exchange_rows <= (1ull << 31);
}

static uint64_t part_bytes(int K, int log2p, int words, uint64_t cap) {
  const uint64_t nbp = 1ull << log2p;
  const uint64_t nv = (uint64_t)((words + 3) / 4);
  return (uint64_t)K * up256(table_bytes(nbp, words)) + up256(kModelMaxWords * 4ull) +
         2 * up256((uint64_t)K * nbp * 16 * nv) + 2 * up256(cap * 16 * nv) + 2 * up256(cap * 8) +
         up256(cap * 4) + up256(sizeof(PartTotals));
}

extern "C" {

ht_status part_reach_bytes(int n_parts, int log2_buckets_part, int max_state_words, uint64_t exchange_rows,
                           uint64_t* bytes) {
  if (!bytes || !part_shape_ok(n_parts, log2_buckets_part, max_state_words, exchange_rows))
    return HT_ERR_INVALID;
  *bytes = part_bytes(n_parts, log2_buckets_part, max_state_words, exchange_rows);
  return HT_OK;
}

ht_status part_reach_create_at(int n_parts, int log2_buckets_part, int max_state_words,
                               uint64_t exchange_rows, const ht_params* params, void* mem_dev,
                               uint64_t mem_bytes, part_reach_t** out) {
  if (!out) return HT_ERR_INVALID;
  *out = nullptr;
  if (!part_shape_ok(n_parts, log2_buckets_part, max_state_words, exchange_rows)) return HT_ERR_INVALID;
  if (!mem_dev || (reinterpret_cast<uintptr_t>(mem_dev) & 255u)) return HT_ERR_INVALID;
  if (params && (params->bucket_bits > 32 || (params->bucket_bits && params->bucket_bits != 32) ||
                 (params->line_buckets && params->line_buckets != 32) ||
                 (params->group_lanes && params->group_lanes != 1)))
    return HT_ERR_INVALID;  // the partitioned kernels use the default walk: 32-bit buckets, 128-byte lines
  if (mem_bytes < part_bytes(n_parts, log2_buckets_part, max_state_words, exchange_rows)) return HT_ERR_OOM;
  part_reach_t* c = new (std::nothrow) part_reach_t();
  if (!c) return HT_ERR_OOM;
  c->K = n_parts;
  while ((1 << c->log2K) < n_parts) c->log2K++;
  c->nbp = 1ull << log2_buckets_part;
  c->max_words = max_state_words;
  c->cap = exchange_rows;
  const uint64_t nv = (uint64_t)((max_state_words + 3) / 4);
  char* p = static_cast<char*>(mem_dev);
  const uint64_t tb = up256(table_bytes(c->nbp, max_state_words));
  for (int k = 0; k < n_parts; ++k) {
    ht_status st = table_init_at(&c->tables[k], c->nbp, max_state_words, params, p, tb);
    if (st != HT_OK) {
      delete c;
      return st;
    }
    p += tb;
  }
  c->blob = reinterpret_cast<int*>(p);
  p += up256(kModelMaxWords * 4ull);
  for (int k = 0; k < 2; ++k) {
    c->fr[k] = reinterpret_cast<uint4*>(p);
    p += up256((uint64_t)n_parts * c->nbp * 16 * nv);
  }
  c->out_rows = reinterpret_cast<uint4*>(p);
  p += up256(exchange_rows * 16 * nv);
  c->in_rows = reinterpret_cast<uint4*>(p);
  p += up256(exchange_rows * 16 * nv);
  c->out_h = reinterpret_cast<unsigned long long*>(p);
  p += up256(exchange_rows * 8);
  c->in_h = reinterpret_cast<unsigned long long*>(p);
  p += up256(exchange_rows * 8);
  c->out_tag = reinterpret_cast<uint32_t*>(p);
  p += up256(exchange_rows * 4);
  c->tot = reinterpret_cast<PartTotals*>(p);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaMallocHost(&c->host_tot, sizeof(PartTotals)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return HT_ERR_CUDA;
  }
  *out = c;
  return HT_OK;
}

ht_status part_reach_destroy(part_reach_t* c) {
  if (!c) return HT_ERR_INVALID;
  if (c->host_tot) cudaFreeHost(c->host_tot);
  delete c;
  return HT_OK;
}

ht_status part_reach_run(part_reach_t* c, const reach_model* m, const int32_t* init_host, void* stream,
                         uint64_t* level_sizes_host, uint32_t max_levels, reach_result* out,
                         uint64_t* part_states_host, uint64_t* exchanged_host) {
  if (!c || !out || max_levels < 1) return HT_ERR_INVALID;
  std::memset(out, 0, sizeof(*out));
  std::vector<int> blob;
  ht_status st = pack_model(m, init_host, c->max_words, blob);
  if (st != HT_OK) return st;
  for (int k = 0; k < c->K; ++k) {
    st = table_set_words(&c->tables[k], m->state_words);
    if (st != HT_OK) return st;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nv = (m->state_words + 3) / 4;
  const PartKernels ks = part_kernels(nv);
  const int smem_words = blob[11];
  const size_t smem = (size_t)((smem_words + 3) & ~3) * 4 + (size_t)8 * warp_smem_words_nv(ks.nv) * 4;
  if (smem > 200 * 1024) return HT_ERR_INVALID;
  const uint32_t maxfan = (uint32_t)std::max(1, blob[13]);
  // a warp round's successors (spw states of at most maxfan each) fit one outbox chunk
  if (maxfan > c->cap) return HT_ERR_INVALID;
  const uint32_t spw = (uint32_t)std::min<uint64_t>((uint64_t)blob[14], c->cap / maxfan);
  VSS_CUDA_TRY(cudaMemcpyAsync(c->blob, blob.data(), blob.size() * 4, cudaMemcpyHostToDevice, s));
  for (int k = 0; k < c->K; ++k) {
    st = table_clear(&c->tables[k], s);
    if (st != HT_OK) return st;
  }
  VSS_CUDA_TRY(cudaMemsetAsync(c->tot, 0, sizeof(PartTotals), s));
  VSS_CUDA_TRY(cudaFuncSetAttribute(ks.expand, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  VSS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks.expand, 256, smem));
  if (per_sm < 1) return HT_ERR_INVALID;
  const int expand_blocks = per_sm * c->num_sms;
  const int move_blocks = 8 * c->num_sms;

  PartDev pd{};
  for (int k = 0; k < c->K; ++k) pd.tv[k] = c->tables[k].view;
  pd.K = c->K;
  pd.log2K = c->log2K;
  pd.blob = c->blob;
  pd.smem_words = smem_words;
  pd.seg_rows = c->nbp;
  pd.spw = spw;
  pd.out_rows = c->out_rows;
  pd.out_h = c->out_h;
  pd.out_tag = c->out_tag;
  pd.in_rows = c->in_rows;
  pd.in_h = c->in_h;
  pd.cap = (uint32_t)c->cap;
  pd.tot = c->tot;
  int cur = 0;
  pd.cur = c->fr[cur];
  pd.next = c->fr[1 - cur];
  ks.seed<<<1, 1, 0, s>>>(pd);
  VSS_CUDA_TRY(cudaGetLastError());
  // rounds per chunk: the chunk's successors (at most spw * maxfan per round) fit the outbox
  const uint32_t rpc = (uint32_t)std::max<uint64_t>(1, c->cap / ((uint64_t)spw * maxfan));
  std::vector<uint64_t> levels;
  const size_t zero_off = offsetof(PartTotals, out_count);
  const size_t zero_len = offsetof(PartTotals, seg_off) - zero_off;
  ht_status result = HT_OK;
  for (;;) {
    VSS_CUDA_TRY(cudaMemcpyAsync(c->host_tot, c->tot, sizeof(PartTotals), cudaMemcpyDeviceToHost, s));
    VSS_CUDA_TRY(cudaStreamSynchronize(s));
    uint32_t err = 0;
    for (int k = 0; k < c->K && !err; ++k) {
      DevCounters ctr;
      VSS_CUDA_TRY(cudaMemcpy(&ctr, c->tables[k].view.ctr, sizeof(ctr), cudaMemcpyDeviceToHost));
      err = ctr.err;
    }
    if (err) {
      result = (ht_status)err;
      break;
    }
    uint64_t n_next = 0;
    for (int k = 0; k < c->K; ++k) n_next += c->host_tot->next_count[k];
    if (n_next == 0) break;
    if (levels.size() >= max_levels) {
      result = HT_ERR_LEVELS;
      break;
    }
    levels.push_back(n_next);
    // the next level: the segments just filled become the current ones
    cur = 1 - cur;
    pd.cur = c->fr[cur];
    pd.next = c->fr[1 - cur];
    uint32_t rounds = 0;
    for (int k = 0; k < c->K; ++k) {
      pd.ncur[k] = c->host_tot->next_count[k];
      pd.round_begin[k] = rounds;
      rounds += (pd.ncur[k] + spw - 1) / spw;
    }
    pd.round_begin[c->K] = rounds;
    VSS_CUDA_TRY(cudaMemsetAsync(c->tot->next_count, 0, sizeof(c->tot->next_count), s));
    for (uint32_t r0 = 0; r0 < rounds; r0 += rpc) {
      const uint32_t r1 = std::min(rounds, r0 + rpc);
      VSS_CUDA_TRY(cudaMemsetAsync(reinterpret_cast<char*>(c->tot) + zero_off, 0, zero_len, s));
      ks.expand<<<expand_blocks, 256, smem, s>>>(pd, r0, r1);
      k_part_plan<<<1, 1, 0, s>>>(pd);
      k_part_scatter<<<move_blocks, 256, 0, s>>>(pd);
      ks.insert<<<move_blocks, 256, 0, s>>>(pd);
      VSS_CUDA_TRY(cudaGetLastError());
    }
  }
  // results
  VSS_CUDA_TRY(cudaMemcpyAsync(c->host_tot, c->tot, sizeof(PartTotals), cudaMemcpyDeviceToHost, s));
  VSS_CUDA_TRY(cudaStreamSynchronize(s));
  uint64_t states = 0;
  for (int k = 0; k < c->K; ++k) {
    DevCounters ctr;
    VSS_CUDA_TRY(cudaMemcpy(&ctr, c->tables[k].view.ctr, sizeof(ctr), cudaMemcpyDeviceToHost));
    states += ctr.stored;
    if (part_states_host) part_states_host[k] = ctr.stored;
    if (result == HT_OK && ctr.err) result = (ht_status)ctr.err;
  }
  const PartTotals& t = *c->host_tot;
  out->states = states;
  out->transitions = t.transitions;
  out->deadlocks = t.deadlocks;
  out->digest = t.digest;
  out->busy_waits = t.busy_waits;
  out->rehashes = t.rehashes;
  out->n_levels = (uint32_t)levels.size();
  out->status = result;
  if (exchanged_host) *exchanged_host = t.exchanged;
  if (level_sizes_host)
    for (uint32_t i = 0; i < out->n_levels && i < max_levels; ++i) level_sizes_host[i] = levels[i];
  return result;
}

ht_status part_reach_last_exchange(part_reach_t* c, uint32_t* counts_host, uint32_t* seg_off_host,
                                   uint32_t* in_begin_host) {
  if (!c || !counts_host || !seg_off_host || !in_begin_host) return HT_ERR_INVALID;
  PartTotals t;
  VSS_CUDA_TRY(cudaMemcpy(&t, c->tot, sizeof(t), cudaMemcpyDeviceToHost));
  const int K = c->K;
  for (int s = 0; s < K; ++s)
    for (int o = 0; o < K; ++o) {
      counts_host[s * K + o] = t.counts[s * K + o];
      seg_off_host[s * K + o] = t.seg_off[s * K + o];
    }
  for (int o = 0; o <= K; ++o) in_begin_host[o] = t.in_begin[o];
  return HT_OK;
}

}  // extern "C"
