// Level-synchronous reachability (Alg. "Reachability analysis") on the table.
//
// One thread expands one frontier state: it reads the state's row of the data
// array, enumerates the enabled edges of the model (next-state), and calls
// find-or-put on every successor.  A successor the table reports as new goes
// to the next frontier (the paper's enqueue-on-not-seen; Alg. "Reachability
// analysis" writes the test the other way round, but find-or-put answers
// "seen").  Frontiers hold the state vectors themselves, so a level reads its
// states with coalesced loads instead of a dependent gather through the data
// array; new states are appended with one atomicAdd per warp and iteration,
// so the next frontier is compacted without a separate pass.
//
// Two drivers share the expansion code:
//   persistent  one cooperative launch runs all levels; blocks meet at a
//               device-side barrier (bounded spin) between levels;
//   per-level   one launch per level; the host reads the next level's size.
//
// This file holds the host side (context layout, model packing, launches,
// results and the reach_* C ABI); the kernels are in reach_kernels.cuh.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "reach_kernels.cuh"

namespace vss {

// G > 1: cooperative probing by groups of G lanes (lines of 4G 32-bit buckets).
static ReachKernels pick_kernels(int nv, int L, int bw, int G = 1) {
  ReachKernels k{};
  bool ok;
  if (G > 1) ok = bw == 32 && L == 4 * G && reach_kernels_group(nv, G, &k);
  else ok = bw == 16 ? reach_kernels_w16(nv, L, &k)
                     : (reach_kernels_w32_lo(nv, L, &k) || reach_kernels_w32_hi(nv, L, &k));
  return ok ? k : ReachKernels{};
}

static uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

}  // namespace vss

using namespace vss;

constexpr int kTimingRing = 64;  // kernel timings kept per context
constexpr uint32_t kGraphLevels = 32;  // levels per graph of the graph driver

struct reach_ctx {
  ht_t table;
  uint64_t nb = 0;
  int max_words = 0;
  uint32_t max_levels = 0;
  void* owned = nullptr;
  int* blob = nullptr;                 // device
  uint4* frontier0 = nullptr;
  uint4* frontier1 = nullptr;
  ReachTotals* tot = nullptr;
  unsigned long long* level_sizes = nullptr;
  unsigned long long* level_ns = nullptr;
  uint32_t* idx0 = nullptr;
  uint32_t* idx1 = nullptr;
  uint32_t* parent = nullptr;
  bool traced = false;
  ReachTotals* host_tot = nullptr;     // pinned
  std::vector<int> host_blob;
  int smem_words = 0;
  bool loaded = false;
  int last_mode = -1;
  std::vector<unsigned long long> host_levels;  // per-level mode
  ht_status host_status = HT_OK;
  int coop = 0;
  // start / end events of the expansion kernels of the last kTimingRing runs
  cudaEvent_t ev[kTimingRing][2] = {};
  // graph driver: instantiated graphs of kGraphLevels levels each, chunk c
  // covering levels [c * kGraphLevels, (c + 1) * kGraphLevels); rebuilt after
  // every load (the kernels' arguments follow the loaded model)
  std::vector<cudaGraphExec_t> graphs;
  cudaStream_t capture_stream = nullptr;
  uint64_t runs = 0;  // runs started; run r uses slot r % kTimingRing
  uint32_t last_launches = 0;
};

static uint64_t frontier_bytes(uint64_t nb, int max_words) {
  return align_up(nb * 16ull * (uint64_t)((max_words + 3) / 4), 256);
}

static uint64_t ctx_bytes(uint64_t nb, int max_words, uint32_t max_levels) {
  return align_up(table_bytes(nb, max_words), 256) + align_up(kModelMaxWords * 4ull, 256) +
         2 * frontier_bytes(nb, max_words) + align_up(sizeof(ReachTotals), 256) +
         2 * align_up((uint64_t)max_levels * 8, 256) + 3 * align_up(nb * 4, 256);
}

namespace vss {
// successor descriptors are 16-bit edge indices: a full blob (5 words per
// edge) holds fewer than 2^16 edges
static_assert(kModelMaxWords / 5 < (1 << 16), "edge index must fit a 16-bit descriptor");

ht_status pack_model(const reach_model* m, const int32_t* init, int max_words,
                     std::vector<int>& blob) {
  if (!m || !init) return HT_ERR_INVALID;
  const int P = m->n_procs, S = m->n_shared, W = m->state_words, E = m->n_edges;
  if (P < 1 || S < 0 || W < P + S || W > max_words || E < 0) return HT_ERR_INVALID;
  if (!m->n_local || !m->crit || !m->edge_begin) return HT_ERR_INVALID;
  if (E > 0 && (!m->edge_dst || !m->guard_var || !m->guard_val || !m->upd_var || !m->upd_val))
    return HT_ERR_INVALID;
  long long nl_total = 0;
  for (int p = 0; p < P; ++p) {
    if (m->n_local[p] < 1 || m->n_local[p] > 65535) return HT_ERR_INVALID;
    if (m->crit[p] < -1 || m->crit[p] >= m->n_local[p]) return HT_ERR_INVALID;
    nl_total += m->n_local[p];
  }
  if (m->edge_begin[0] != 0 || m->edge_begin[nl_total] != E) return HT_ERR_INVALID;
  for (long long i = 0; i < nl_total; ++i)
    if (m->edge_begin[i + 1] < m->edge_begin[i]) return HT_ERR_INVALID;
  {
    long long b = 0;
    for (int p = 0; p < P; ++p)
      for (int s = 0; s < m->n_local[p]; ++s, ++b)
        for (int e = m->edge_begin[b]; e < m->edge_begin[b + 1]; ++e) {
          if (m->edge_dst[e] < 0 || m->edge_dst[e] >= m->n_local[p]) return HT_ERR_INVALID;
          if (m->guard_var[e] < -1 || m->guard_var[e] >= S) return HT_ERR_INVALID;
          if (m->upd_var[e] < -1 || m->upd_var[e] >= S) return HT_ERR_INVALID;
        }
  }
  for (int p = 0; p < P; ++p)
    if (init[p] < 0 || init[p] >= m->n_local[p]) return HT_ERR_INVALID;
  for (int w = P + S; w < W; ++w)
    if (init[w] != 0) return HT_ERR_INVALID;  // padding words stay 0
  auto up4 = [](long long x) { return (x + 3) & ~3LL; };
  const long long off_base = kHdr;
  const long long off_crit = off_base + P;
  const long long off_eb = off_crit + P;
  const long long off_edges = up4(off_eb + nl_total + 1);
  const long long off_uval = off_edges + 4LL * E;
  const long long off_init = up4(off_uval + E);
  const long long total = off_init + 4LL * ((W + 3) / 4);
  if (total > kModelMaxWords) return HT_ERR_INVALID;
  blob.assign((size_t)total, 0);
  int crit_any = 0;
  for (int p = 0; p < P; ++p) crit_any |= (m->crit[p] >= 0);
  long long maxfan = 0;
  {
    long long b = 0;
    for (int p = 0; p < P; ++p) {
      long long mp = 0;
      for (int s = 0; s < m->n_local[p]; ++s, ++b)
        mp = std::max<long long>(mp, m->edge_begin[b + 1] - m->edge_begin[b]);
      maxfan += mp;
    }
  }
  if (maxfan > kDescCap) return HT_ERR_INVALID;  // more successors per state than a warp round holds
  const int fan = (int)std::max<long long>(1, maxfan);
  const int spw_max = std::min(32, kDescCap / fan);
  int hdr[kHdr] = {P, S, W, (int)nl_total, E, crit_any, (int)off_base, (int)off_crit, (int)off_eb,
                   (int)off_edges, (int)off_uval, (int)off_init, (int)off_init, fan, spw_max, 0};
  std::memcpy(blob.data(), hdr, sizeof(hdr));
  long long acc = 0;
  for (int p = 0; p < P; ++p) {
    blob[off_base + p] = (int)acc;
    acc += m->n_local[p];
    blob[off_crit + p] = m->crit[p];
  }
  for (long long i = 0; i <= nl_total; ++i) blob[off_eb + i] = m->edge_begin[i];
  {
    // each edge carries its process above its destination (edge_dst / edge_proc)
    long long b = 0;
    for (int p = 0; p < P; ++p)
      for (int s = 0; s < m->n_local[p]; ++s, ++b)
        for (int e = m->edge_begin[b]; e < m->edge_begin[b + 1]; ++e)
          blob[off_edges + 4LL * e + 0] = m->edge_dst[e] | (p << 16);
  }
  for (int e = 0; e < E; ++e) {
    blob[off_edges + 4LL * e + 1] = m->guard_var[e];
    blob[off_edges + 4LL * e + 2] = m->guard_val[e];
    blob[off_edges + 4LL * e + 3] = m->upd_var[e];
    blob[off_uval + e] = m->upd_val[e];
  }
  for (int w = 0; w < W; ++w) blob[off_init + w] = init[w];
  return HT_OK;
}

}  // namespace vss

static ReachDev make_rd(reach_ctx_t* c) {
  ReachDev rd;
  rd.blob = c->blob;
  rd.smem_words = c->smem_words;
  rd.frontier0 = c->frontier0;
  rd.frontier1 = c->frontier1;
  rd.cap = (uint32_t)c->nb;
  rd.tot = c->tot;
  rd.level_sizes = c->level_sizes;
  rd.level_ns = c->level_ns;
  rd.idx0 = c->idx0;
  rd.idx1 = c->idx1;
  rd.parent = c->parent;
  rd.max_levels = c->max_levels;
  rd.bar_spin = 1u << 22;
  return rd;
}

// Blocks per SM for a single-model launch.  On tables of at most 2^20
// buckets the levels are short and latency-bound: the level barrier, whose
// cost grows with the number of blocks, weighs more than the memory-level
// parallelism of a third and fourth block per SM.
#ifndef VSS_SMALL_TABLE_BLOCKS
#define VSS_SMALL_TABLE_BLOCKS 2
#endif
static int blocks_per_sm(int occupancy, uint64_t nb) {
  if (VSS_SMALL_TABLE_BLOCKS > 0 && nb <= (1ull << 20) && occupancy > VSS_SMALL_TABLE_BLOCKS)
    return VSS_SMALL_TABLE_BLOCKS;
  return occupancy;
}

static size_t smem_bytes_for(reach_ctx_t* c, int threads) {
  return (size_t)((c->smem_words + 3) & ~3) * 4 +
         (size_t)(threads / 32) * warp_smem_words_nv((int)c->table.view.nv) * 4;
}

// Graph driver: capture chunk `chunk` (kGraphLevels levels, the seed first in
// chunk 0) once, then replay it.
static ht_status chunk_graph(reach_ctx_t* c, uint32_t chunk, const ReachKernels& ks, TableView tv,
                             ReachDev rd, int threads, size_t smem, cudaGraphExec_t* out) {
  if (chunk < c->graphs.size() && c->graphs[chunk]) {
    *out = c->graphs[chunk];
    return HT_OK;
  }
  if (!c->capture_stream)
    VSS_CUDA_TRY(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
  int per_sm = 0;
  VSS_CUDA_TRY(cudaFuncSetAttribute(ks.step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  VSS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks.step, threads, smem));
  if (per_sm < 1) return HT_ERR_INVALID;
  const int blocks = blocks_per_sm(per_sm, c->nb) * c->table.num_sms;
  cudaStream_t cs = c->capture_stream;
  cudaGraph_t graph = nullptr;
  VSS_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  if (chunk == 0) ks.seed<<<1, 1, 0, cs>>>(tv, rd);
  for (uint32_t i = 0; i < kGraphLevels; ++i) {
    const uint32_t k = chunk * kGraphLevels + i;
    cudaMemsetAsync(&c->tot->counts[(k + 1) % 3], 0, 4, cs);
    cudaMemsetAsync(&c->tot->cursor[k % 3], 0, 4, cs);
    ks.step<<<blocks, threads, smem, cs>>>(tv, rd, k);
  }
  const cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (e != cudaSuccess || !graph) {
    cudaGetLastError();
    return HT_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    return HT_ERR_CUDA;
  }
  if (c->graphs.size() <= chunk) c->graphs.resize(chunk + 1, nullptr);
  c->graphs[chunk] = exec;
  *out = exec;
  return HT_OK;
}

static ht_status run_graphs(reach_ctx_t* c, const ReachKernels& ks, TableView tv, ReachDev rd,
                            int threads, size_t smem, cudaStream_t s) {
  cudaEvent_t* ev = c->ev[c->runs % kTimingRing];
  c->runs++;
  VSS_CUDA_TRY(cudaEventRecord(ev[0], s));
  c->last_launches = 0;
  for (uint32_t chunk = 0;; ++chunk) {
    cudaGraphExec_t g = nullptr;
    ht_status st = chunk_graph(c, chunk, ks, tv, rd, threads, smem, &g);
    if (st != HT_OK) return st;
    VSS_CUDA_TRY(cudaGraphLaunch(g, s));
    VSS_CUDA_TRY(cudaEventRecord(ev[1], s));
    c->last_launches += kGraphLevels + (chunk == 0 ? 1 : 0);
    // the next chunk only if the search is still going at its first level
    const uint32_t k_next = (chunk + 1) * kGraphLevels;
    VSS_CUDA_TRY(cudaMemcpyAsync(c->host_tot, c->tot, sizeof(ReachTotals), cudaMemcpyDeviceToHost, s));
    VSS_CUDA_TRY(cudaMemcpyAsync(&c->host_tot->pad, &c->table.view.ctr->err, 4,
                                 cudaMemcpyDeviceToHost, s));
    VSS_CUDA_TRY(cudaStreamSynchronize(s));
    if (c->host_tot->pad) break;  // latched error: the result reports it
    if (c->host_tot->counts[k_next % 3] == 0) break;
    if (k_next >= c->max_levels) {  // the search goes on past the level capacity
      c->host_status = HT_ERR_LEVELS;
      break;
    }
  }
  return HT_OK;
}

extern "C" {

ht_status reach_ctx_bytes_n(uint64_t n_buckets, int max_state_words, uint32_t max_levels,
                            uint64_t* bytes) {
  if (!bytes || n_buckets < 16 || n_buckets > kMaxBuckets || max_state_words < 1 ||
      max_state_words > 32 || max_levels < 1)
    return HT_ERR_INVALID;
  *bytes = ctx_bytes(n_buckets, max_state_words, max_levels);
  return HT_OK;
}

ht_status reach_ctx_bytes(int log2_buckets, int max_state_words, uint32_t max_levels,
                          uint64_t* bytes) {
  if (log2_buckets < 4 || log2_buckets > 31) return HT_ERR_INVALID;
  return reach_ctx_bytes_n(1ull << log2_buckets, max_state_words, max_levels, bytes);
}

ht_status reach_ctx_buckets_for_bytes(uint64_t bytes, int max_state_words, uint32_t max_levels,
                                      const ht_params* params, uint64_t* n_buckets) {
  if (!n_buckets || max_state_words < 1 || max_state_words > 32 || max_levels < 1)
    return HT_ERR_INVALID;
  *n_buckets = 0;
  ht_params p{};
  ht_status st = resolve_params(params, 1u << 10, &p);
  if (st != HT_OK) return st;
  uint64_t lo = 0, hi = kMaxBuckets;  // ctx_bytes is increasing in nb
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo + 1) / 2;
    if (ctx_bytes(mid, max_state_words, max_levels) <= bytes) lo = mid;
    else hi = mid - 1;
  }
  const uint64_t nb = prime_line_buckets(lo, p.line_buckets);
  if (nb == 0) return HT_ERR_OOM;
  *n_buckets = nb;
  return HT_OK;
}

ht_status reach_ctx_create_n_at(uint64_t n_buckets, int max_state_words, uint32_t max_levels,
                                const ht_params* params, void* mem_dev, uint64_t mem_bytes,
                                reach_ctx_t** out) {
  if (!out) return HT_ERR_INVALID;
  *out = nullptr;
  uint64_t need = 0;
  ht_status st = reach_ctx_bytes_n(n_buckets, max_state_words, max_levels, &need);
  if (st != HT_OK) return st;
  if (!mem_dev || (reinterpret_cast<uintptr_t>(mem_dev) & 255u)) return HT_ERR_INVALID;
  if (mem_bytes < need) return HT_ERR_OOM;
  reach_ctx_t* c = new (std::nothrow) reach_ctx_t();
  if (!c) return HT_ERR_OOM;
  const uint64_t tb = align_up(table_bytes(n_buckets, max_state_words), 256);
  st = table_init_at(&c->table, n_buckets, max_state_words, params, mem_dev, tb);
  if (st != HT_OK) {
    delete c;
    return st;
  }
  char* p = static_cast<char*>(mem_dev) + tb;
  c->blob = reinterpret_cast<int*>(p);
  p += align_up(kModelMaxWords * 4ull, 256);
  const uint64_t fb = frontier_bytes(n_buckets, max_state_words);
  c->frontier0 = reinterpret_cast<uint4*>(p);
  p += fb;
  c->frontier1 = reinterpret_cast<uint4*>(p);
  p += fb;
  c->tot = reinterpret_cast<ReachTotals*>(p);
  p += align_up(sizeof(ReachTotals), 256);
  c->level_sizes = reinterpret_cast<unsigned long long*>(p);
  p += align_up((uint64_t)max_levels * 8, 256);
  c->level_ns = reinterpret_cast<unsigned long long*>(p);
  p += align_up((uint64_t)max_levels * 8, 256);
  const uint64_t ib = align_up(n_buckets * 4, 256);
  c->idx0 = reinterpret_cast<uint32_t*>(p);
  p += ib;
  c->idx1 = reinterpret_cast<uint32_t*>(p);
  p += ib;
  c->parent = reinterpret_cast<uint32_t*>(p);
  c->nb = n_buckets;
  c->max_words = max_state_words;
  c->max_levels = max_levels;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaMallocHost(&c->host_tot, sizeof(ReachTotals)) != cudaSuccess) {
    cudaGetLastError();
    reach_ctx_destroy(c);
    return HT_ERR_CUDA;
  }
  for (int i = 0; i < kTimingRing; ++i) {
    if (cudaEventCreate(&c->ev[i][0]) != cudaSuccess || cudaEventCreate(&c->ev[i][1]) != cudaSuccess) {
      cudaGetLastError();
      reach_ctx_destroy(c);
      return HT_ERR_CUDA;
    }
  }
  *out = c;
  return HT_OK;
}

ht_status reach_ctx_create_at(int log2_buckets, int max_state_words, uint32_t max_levels,
                              const ht_params* params, void* mem_dev, uint64_t mem_bytes,
                              reach_ctx_t** out) {
  if (log2_buckets < 4 || log2_buckets > 31) {
    if (out) *out = nullptr;
    return HT_ERR_INVALID;
  }
  return reach_ctx_create_n_at(1ull << log2_buckets, max_state_words, max_levels, params, mem_dev,
                               mem_bytes, out);
}

ht_status reach_ctx_create(int log2_buckets, int max_state_words, uint32_t max_levels,
                           const ht_params* params, reach_ctx_t** out) {
  uint64_t bytes = 0;
  if (!out) return HT_ERR_INVALID;
  *out = nullptr;
  ht_status st = reach_ctx_bytes(log2_buckets, max_state_words, max_levels, &bytes);
  if (st != HT_OK) return st;
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return HT_ERR_OOM;
  }
  st = reach_ctx_create_at(log2_buckets, max_state_words, max_levels, params, mem, bytes, out);
  if (st != HT_OK) {
    cudaFree(mem);
    return st;
  }
  (*out)->owned = mem;
  return HT_OK;
}

static void drop_graphs(reach_ctx_t* c) {
  for (cudaGraphExec_t g : c->graphs)
    if (g) cudaGraphExecDestroy(g);
  c->graphs.clear();
}

ht_status reach_ctx_destroy(reach_ctx_t* c) {
  if (!c) return HT_ERR_INVALID;
  drop_graphs(c);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  if (c->host_tot) cudaFreeHost(c->host_tot);
  for (int i = 0; i < kTimingRing; ++i)
    for (int j = 0; j < 2; ++j)
      if (c->ev[i][j]) cudaEventDestroy(c->ev[i][j]);
  if (c->owned) cudaFree(c->owned);
  delete c;
  return HT_OK;
}

ht_status reach_ctx_last_timing(reach_ctx_t* c, float* kernel_ms, uint32_t* launches) {
  if (!c || c->last_mode < 0 || c->runs == 0) return HT_ERR_INVALID;
  const int slot = (int)((c->runs - 1) % kTimingRing);
  VSS_CUDA_TRY(cudaEventSynchronize(c->ev[slot][1]));
  float ms = 0.f;
  VSS_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[slot][0], c->ev[slot][1]));
  if (kernel_ms) *kernel_ms = ms;
  if (launches) *launches = c->last_launches;
  return HT_OK;
}

ht_status reach_ctx_run_times(reach_ctx_t* c, uint32_t n, float* ms_host, uint32_t* got) {
  if (!c || (n && !ms_host)) return HT_ERR_INVALID;
  uint64_t avail = c->runs < (uint64_t)kTimingRing ? c->runs : (uint64_t)kTimingRing;
  const uint32_t k = (uint32_t)(avail < n ? avail : n);
  if (k) VSS_CUDA_TRY(cudaEventSynchronize(c->ev[(c->runs - 1) % kTimingRing][1]));
  for (uint32_t i = 0; i < k; ++i) {
    const int slot = (int)((c->runs - k + i) % kTimingRing);
    VSS_CUDA_TRY(cudaEventElapsedTime(&ms_host[i], c->ev[slot][0], c->ev[slot][1]));
  }
  if (got) *got = k;
  return HT_OK;
}

ht_status reach_ctx_level_ns(reach_ctx_t* c, void* stream, uint64_t* level_ns_host,
                             uint32_t max_levels, uint32_t* n_levels) {
  if (!c || !level_ns_host || c->last_mode != REACH_PERSISTENT) return HT_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  VSS_CUDA_TRY(cudaStreamSynchronize(s));
  uint32_t n = 0;
  VSS_CUDA_TRY(cudaMemcpy(&n, &c->tot->n_levels, 4, cudaMemcpyDeviceToHost));
  n = std::min(n, max_levels);
  if (n) VSS_CUDA_TRY(cudaMemcpy(level_ns_host, c->level_ns, (size_t)n * 8, cudaMemcpyDeviceToHost));
  if (n_levels) *n_levels = n;
  return HT_OK;
}

ht_status reach_ctx_deadlock_trace(reach_ctx_t* c, void* stream, int32_t* states_host,
                                   uint32_t max_len, uint32_t* len, uint32_t* level) {
  if (!c || !len || !c->traced) return HT_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  VSS_CUDA_TRY(cudaStreamSynchronize(s));
  unsigned long long key = 0;
  VSS_CUDA_TRY(cudaMemcpy(&key, &c->tot->first_deadlock, 8, cudaMemcpyDeviceToHost));
  *len = 0;
  if (key == ~0ull) return HT_OK;  // no deadlock
  const uint32_t lv = (uint32_t)(key >> 50);
  if (level) *level = lv;
  const uint32_t n = lv + 1;
  if (!states_host || max_len < n) return HT_ERR_INVALID;
  std::vector<uint32_t> path(n);
  uint32_t idx = (uint32_t)(key & 0x7FFFFFFFull);
  for (uint32_t k = n; k-- > 0;) {
    path[k] = idx;
    if (k) VSS_CUDA_TRY(cudaMemcpy(&idx, c->parent + idx, 4, cudaMemcpyDeviceToHost));
  }
  const uint32_t W = c->table.view.state_words, rw = 4 * c->table.view.nv;
  const int32_t* data = reinterpret_cast<const int32_t*>(c->table.view.data);
  for (uint32_t k = 0; k < n; ++k)
    VSS_CUDA_TRY(cudaMemcpy(states_host + (uint64_t)k * W, data + (uint64_t)path[k] * rw, W * 4,
                            cudaMemcpyDeviceToHost));
  *len = n;
  return HT_OK;
}

ht_status reach_ctx_table(reach_ctx_t* c, ht_t** table) {
  if (!c || !table) return HT_ERR_INVALID;
  *table = &c->table;
  return HT_OK;
}

ht_status reach_ctx_load(reach_ctx_t* c, const reach_model* m, const int32_t* init_host,
                         void* stream) {
  if (!c) return HT_ERR_INVALID;
  ht_status st = pack_model(m, init_host, c->max_words, c->host_blob);
  if (st != HT_OK) return st;
  st = table_set_words(&c->table, m->state_words);
  if (st != HT_OK) return st;
  c->smem_words = c->host_blob[11];
  if (smem_bytes_for(c, (int)c->table.params.block_threads) > 200 * 1024) return HT_ERR_INVALID;
  drop_graphs(c);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // synchronous w.r.t. the host buffer: the blob vector may change on the next load
  VSS_CUDA_TRY(cudaMemcpyAsync(c->blob, c->host_blob.data(), c->host_blob.size() * 4,
                               cudaMemcpyHostToDevice, s));
  VSS_CUDA_TRY(cudaStreamSynchronize(s));
  c->loaded = true;
  return HT_OK;
}

ht_status reach_ctx_run(reach_ctx_t* c, int mode, void* stream) {
  if (!c || !c->loaded) return HT_ERR_INVALID;
  const bool trace = (mode & REACH_TRACE) != 0;
  mode &= ~REACH_TRACE;
  if (mode != REACH_PERSISTENT && mode != REACH_PER_LEVEL && mode != REACH_GRAPH) return HT_ERR_INVALID;
  if (trace && mode != REACH_PERSISTENT) return HT_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ht_status st = table_clear(&c->table, s);
  if (st != HT_OK) return st;
  VSS_CUDA_TRY(cudaMemsetAsync(c->tot, 0, sizeof(ReachTotals), s));
  VSS_CUDA_TRY(cudaMemsetAsync(&c->tot->first_deadlock, 0xFF, sizeof(unsigned long long), s));
  const int threads = (int)c->table.params.block_threads;
  const size_t smem = smem_bytes_for(c, threads);
  const ReachKernels ks = pick_kernels((int)c->table.view.nv, (int)c->table.params.line_buckets,
                                         (int)c->table.view.bucket_bits, (int)c->table.params.group_lanes);
  if (!ks.persistent) return HT_ERR_INVALID;
  TableView tv = c->table.view;
  ReachDev rd = make_rd(c);
  c->last_mode = mode;
  c->traced = trace;
  c->host_status = HT_OK;
  if (mode == REACH_PERSISTENT) {
    if (!c->coop) return HT_ERR_CUDA;
    void (*kern)(TableView, ReachDev) = trace ? ks.persistent_trace : ks.persistent;
    if (!kern) return HT_ERR_INVALID;  // tracing is compiled for the default line length
    VSS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    VSS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return HT_ERR_INVALID;
    const int blocks = blocks_per_sm(per_sm, c->nb) * c->table.num_sms;
    void* args[] = {&tv, &rd};
    cudaEvent_t* ev = c->ev[c->runs % kTimingRing];
    VSS_CUDA_TRY(cudaEventRecord(ev[0], s));
    VSS_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kern), blocks, threads, args,
                                             smem, s));
    VSS_CUDA_TRY(cudaEventRecord(ev[1], s));
    c->runs++;
    c->last_launches = 1;
    return HT_OK;
  }
  if (mode == REACH_GRAPH) return run_graphs(c, ks, tv, rd, threads, smem, s);
  // per-level: one launch per level, the host reads each level's size
  VSS_CUDA_TRY(cudaFuncSetAttribute(ks.level, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  VSS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks.level, threads, smem));
  if (per_sm < 1) return HT_ERR_INVALID;
  cudaEvent_t* ev = c->ev[c->runs % kTimingRing];
  c->runs++;
  VSS_CUDA_TRY(cudaEventRecord(ev[0], s));
  ks.seed<<<1, 1, 0, s>>>(tv, rd);
  VSS_CUDA_TRY(cudaGetLastError());
  c->last_launches = 1;
  c->host_levels.assign(1, 1);
  uint32_t n_cur = 1;
  for (uint32_t k = 0;; ++k) {
    const uint64_t warps_needed = (n_cur + 31) / 32;
    const uint64_t want = (warps_needed * 32 + threads - 1) / threads;
    const uint64_t cap = (uint64_t)blocks_per_sm(per_sm, c->nb) * c->table.num_sms;
    const int blocks = (int)std::max<uint64_t>(1, std::min(want, cap));
    VSS_CUDA_TRY(cudaMemsetAsync(&c->tot->counts[(k + 1) % 3], 0, 4, s));
    VSS_CUDA_TRY(cudaMemsetAsync(&c->tot->cursor[k % 3], 0, 4, s));
    ks.level<<<blocks, threads, smem, s>>>(tv, rd, k);
    VSS_CUDA_TRY(cudaGetLastError());
    VSS_CUDA_TRY(cudaEventRecord(ev[1], s));
    c->last_launches++;
    VSS_CUDA_TRY(cudaMemcpyAsync(c->host_tot, c->tot, sizeof(ReachTotals), cudaMemcpyDeviceToHost, s));
    uint32_t err = 0;
    VSS_CUDA_TRY(cudaMemcpyAsync(&c->host_tot->pad, &c->table.view.ctr->err, 4,
                                 cudaMemcpyDeviceToHost, s));
    VSS_CUDA_TRY(cudaStreamSynchronize(s));
    err = c->host_tot->pad;
    if (err) {
      c->host_status = (ht_status)err;
      break;
    }
    const uint32_t n_next = c->host_tot->counts[(k + 1) % 3];
    if (n_next == 0) break;
    if (c->host_levels.size() >= c->max_levels) {
      c->host_status = HT_ERR_LEVELS;
      break;
    }
    c->host_levels.push_back(n_next);
    n_cur = n_next;
  }
  return HT_OK;
}

ht_status reach_ctx_result(reach_ctx_t* c, void* stream, uint64_t* level_sizes_host,
                           uint32_t max_levels, reach_result* out) {
  if (!c || !out) return HT_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::memset(out, 0, sizeof(*out));
  DevCounters ctr;
  VSS_CUDA_TRY(cudaMemcpyAsync(c->host_tot, c->tot, sizeof(ReachTotals), cudaMemcpyDeviceToHost, s));
  VSS_CUDA_TRY(cudaStreamSynchronize(s));
  VSS_CUDA_TRY(cudaMemcpy(&ctr, c->table.view.ctr, sizeof(ctr), cudaMemcpyDeviceToHost));
  const ReachTotals& t = *c->host_tot;
  out->transitions = t.transitions;
  out->deadlocks = t.deadlocks;
  out->digest = t.digest;
  out->states = ctr.stored;
  out->busy_waits = ctr.busy_waits;
  out->rehashes = ctr.rehashes;
  out->status = ctr.err ? (ht_status)ctr.err : c->host_status;
  if (c->last_mode == REACH_PER_LEVEL) {
    out->n_levels = (uint32_t)c->host_levels.size();
    if (level_sizes_host)
      for (uint32_t i = 0; i < out->n_levels && i < max_levels; ++i)
        level_sizes_host[i] = c->host_levels[i];
  } else {
    out->n_levels = t.n_levels;
    if (level_sizes_host && out->n_levels) {
      const uint32_t n = std::min(out->n_levels, max_levels);
      VSS_CUDA_TRY(cudaMemcpy(level_sizes_host, c->level_sizes, (size_t)n * 8, cudaMemcpyDeviceToHost));
    }
  }
  if (out->status == HT_OK && level_sizes_host && out->n_levels > max_levels) out->status = HT_ERR_LEVELS;
  return out->status;
}

ht_status reach(reach_ctx_t* c, const reach_model* m, const int32_t* init_host, int mode,
                void* stream, uint64_t* level_sizes_host, uint32_t max_levels, reach_result* out) {
  ht_status st = reach_ctx_load(c, m, init_host, stream);
  if (st != HT_OK) return st;
  st = reach_ctx_run(c, mode, stream);
  if (st != HT_OK) return st;
  return reach_ctx_result(c, stream, level_sizes_host, max_levels, out);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// reach_noalloc: reachability that allocates no device memory.
//
// For callers that cannot call cudaMalloc (a host process that must not grow
// its device footprint after start-up, code running where allocation is not
// allowed).  The table, the two frontiers and the counters live in one
// file-scope device array of kNoAllocScratchBytes, loaded with the library and
// held by every GPU that loads it until the process exits.  Host code cannot
// use the array's name as a device address: every call looks the address up
// with cudaGetSymbolAddress for the device (and context) current at the call.
// The lookup allocates nothing, and looking it up each time, rather than
// caching it per device, keeps a call correct after cudaDeviceReset (which
// reloads the module at a new address) and on a caller's own driver-API
// context (which holds its own copy of the module).
// ---------------------------------------------------------------------------
namespace vss {

constexpr uint64_t kNoAllocScratchBytes = 32ull << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static ht_status noalloc_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return HT_ERR_CUDA;
  }
  *out = p;
  return HT_OK;
}

}  // namespace vss

extern "C" ht_status reach_noalloc(const reach_model* m, const int32_t* init_host, int log2_buckets,
                                   const ht_params* params, void* stream,
                                   uint64_t* level_sizes_host, uint32_t max_levels,
                                   reach_result* out) {
  if (!m || !init_host || !out || max_levels < 1) return HT_ERR_INVALID;
  std::memset(out, 0, sizeof(*out));
  const int W = m->state_words;
  uint64_t need = 0;
  ht_status st = reach_ctx_bytes(log2_buckets, W, max_levels, &need);
  if (st != HT_OK) return st;
  if (need > kNoAllocScratchBytes) return HT_ERR_TOO_BIG;
  void* base = nullptr;
  st = noalloc_scratch(&base);
  if (st != HT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // carve the scratch array exactly like a context block
  ht_t table;
  const uint64_t nb = 1ull << log2_buckets;
  const uint64_t tb = align_up(table_bytes(nb, W), 256);
  st = table_init_at(&table, nb, W, params, base, tb);
  if (st != HT_OK) return st;
  char* p = static_cast<char*>(base) + tb;
  int* blob = reinterpret_cast<int*>(p);
  p += align_up(kModelMaxWords * 4ull, 256);
  const uint64_t fb = frontier_bytes(nb, W);
  uint4* f0 = reinterpret_cast<uint4*>(p);
  p += fb;
  uint4* f1 = reinterpret_cast<uint4*>(p);
  p += fb;
  ReachTotals* tot = reinterpret_cast<ReachTotals*>(p);
  p += align_up(sizeof(ReachTotals), 256);
  unsigned long long* lsz = reinterpret_cast<unsigned long long*>(p);
  p += align_up((uint64_t)max_levels * 8, 256);
  unsigned long long* lns = reinterpret_cast<unsigned long long*>(p);

  std::vector<int> host_blob;
  st = pack_model(m, init_host, W, host_blob);
  if (st != HT_OK) return st;
  const int threads = (int)table.params.block_threads;
  const int smem_words = host_blob[11];
  const size_t smem = (size_t)((smem_words + 3) & ~3) * 4 +
                      (size_t)(threads / 32) * warp_smem_words_nv((int)table.view.nv) * 4;
  if (smem > 200 * 1024) return HT_ERR_INVALID;
  int dev = 0, coop = 0;
  VSS_CUDA_TRY(cudaGetDevice(&dev));
  VSS_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return HT_ERR_CUDA;

  // everything that must start at zero is cleared: the previous call's table,
  // frontier counts, cursors and barrier words are still in the array
  VSS_CUDA_TRY(cudaMemcpyAsync(blob, host_blob.data(), host_blob.size() * 4,
                               cudaMemcpyHostToDevice, s));
  st = table_clear(&table, s);
  if (st != HT_OK) return st;
  VSS_CUDA_TRY(cudaMemsetAsync(tot, 0, sizeof(ReachTotals), s));

  const ReachKernels ks = pick_kernels((int)table.view.nv, (int)table.params.line_buckets,
                                         (int)table.view.bucket_bits, (int)table.params.group_lanes);
  if (!ks.persistent) return HT_ERR_INVALID;
  VSS_CUDA_TRY(cudaFuncSetAttribute(ks.persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int per_sm = 0;
  VSS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks.persistent, threads, smem));
  if (per_sm < 1) return HT_ERR_INVALID;
  TableView tv = table.view;
  ReachDev rd{};
  rd.blob = blob;
  rd.smem_words = smem_words;
  rd.frontier0 = f0;
  rd.frontier1 = f1;
  rd.cap = (uint32_t)nb;
  rd.tot = tot;
  rd.level_sizes = lsz;
  rd.level_ns = lns;
  rd.max_levels = max_levels;
  rd.bar_spin = 1u << 22;
  void* args[] = {&tv, &rd};
  VSS_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(ks.persistent),
                                           blocks_per_sm(per_sm, nb) * table.num_sms, threads, args,
                                           smem, s));

  ReachTotals t;
  DevCounters ctr;
  VSS_CUDA_TRY(cudaMemcpyAsync(&t, tot, sizeof(t), cudaMemcpyDeviceToHost, s));
  VSS_CUDA_TRY(cudaMemcpyAsync(&ctr, table.view.ctr, sizeof(ctr), cudaMemcpyDeviceToHost, s));
  VSS_CUDA_TRY(cudaStreamSynchronize(s));
  out->states = ctr.stored;
  out->transitions = t.transitions;
  out->deadlocks = t.deadlocks;
  out->digest = t.digest;
  out->busy_waits = ctr.busy_waits;
  out->rehashes = ctr.rehashes;
  out->n_levels = t.n_levels;
  out->status = (ht_status)ctr.err;
  if (level_sizes_host && out->n_levels) {
    const uint32_t n = std::min(out->n_levels, max_levels);
    VSS_CUDA_TRY(cudaMemcpyAsync(level_sizes_host, lsz, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    VSS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return out->status;
}

// ---------------------------------------------------------------------------
// One single-model run on device areas carved by the caller: the server runs a
// job that arrives at an idle GPU this way (the persistent single-model kernel
// has a shorter level path than the many-model kernel).
// ---------------------------------------------------------------------------
namespace vss {

uint64_t solo_totals_bytes() { return sizeof(ReachTotals); }

ht_status solo_launch(const SoloRun& r, int line_buckets, int threads, cudaStream_t s) {
  const uint32_t nv = r.tv.nv;
  const ReachKernels ks = pick_kernels((int)nv, line_buckets, (int)r.tv.bucket_bits);
  if (!ks.persistent || r.tv.lines_div.m != 0) return HT_ERR_INVALID;  // power-of-two tables
  const uint64_t nb = (uint64_t)r.tv.nb_mask + 1;
  VSS_CUDA_TRY(cudaMemsetAsync(r.tv.ctr, 0, sizeof(DevCounters), s));
  VSS_CUDA_TRY(cudaMemsetAsync(r.tv.buckets, 0, nb * (r.tv.bucket_bits / 8), s));
  ReachTotals* tot = static_cast<ReachTotals*>(r.tot_dev);
  VSS_CUDA_TRY(cudaMemsetAsync(tot, 0, sizeof(ReachTotals), s));
  VSS_CUDA_TRY(cudaMemsetAsync(&tot->first_deadlock, 0xFF, sizeof(unsigned long long), s));
  const size_t smem = (size_t)((r.smem_words + 3) & ~3) * 4 +
                      (size_t)(threads / 32) * warp_smem_words_nv((int)nv) * 4;
  if (smem > 200 * 1024) return HT_ERR_INVALID;
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  VSS_CUDA_TRY(cudaGetDevice(&dev));
  VSS_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  VSS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (!coop) return HT_ERR_CUDA;
  VSS_CUDA_TRY(cudaFuncSetAttribute(ks.persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  VSS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks.persistent, threads, smem));
  if (per_sm < 1) return HT_ERR_INVALID;
  TableView tv = r.tv;
  ReachDev rd{};
  rd.blob = r.blob_dev;
  rd.smem_words = r.smem_words;
  rd.frontier0 = r.fr0;
  rd.frontier1 = r.fr1;
  rd.cap = r.cap;
  rd.tot = tot;
  rd.level_sizes = r.level_sizes_dev;
  rd.level_ns = r.level_ns_dev;
  rd.max_levels = r.max_levels;
  rd.bar_spin = 1u << 22;
  void* args[] = {&tv, &rd};
  VSS_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(ks.persistent),
                                           blocks_per_sm(per_sm, nb) * sms, threads, args, smem, s));
  return HT_OK;
}

ht_status solo_result(const SoloRun& r, reach_result* out) {
  std::memset(out, 0, sizeof(*out));
  ReachTotals t;
  DevCounters ctr;
  VSS_CUDA_TRY(cudaMemcpy(&t, r.tot_dev, sizeof(t), cudaMemcpyDeviceToHost));
  VSS_CUDA_TRY(cudaMemcpy(&ctr, r.tv.ctr, sizeof(ctr), cudaMemcpyDeviceToHost));
  out->transitions = t.transitions;
  out->deadlocks = t.deadlocks;
  out->digest = t.digest;
  out->states = ctr.stored;
  out->busy_waits = ctr.busy_waits;
  out->rehashes = ctr.rehashes;
  out->n_levels = t.n_levels;
  out->status = (ht_status)ctr.err;
  return out->status;
}

}  // namespace vss
