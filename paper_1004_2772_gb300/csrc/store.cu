// The table: batched find-or-put, full-table scan, gather, and the ht_* C ABI.
#include <cstdlib>
#include <new>

#include "coop.cuh"
#include "internal.h"
#include "table.cuh"

namespace vss {

// Batched find-or-put: one thread per key, warp-uniform grid-stride loop.
// With DEDUP, lanes whose keys hash alike are merged first (__match_any_sync):
// the lowest such lane probes, the others compare their key with it through
// shuffles and take its answer as "seen" -- this removes write-busy waits on
// hot keys that arrive together.
template <int NV, int L, bool DEDUP, int BW>
__global__ void __launch_bounds__(256, table_min_blocks<NV>()) k_find_or_put(TableView t, const int32_t* __restrict__ keys,
                                                     uint64_t n, uint8_t* __restrict__ seen,
                                                     uint32_t* __restrict__ idx) {
  LocalCounters lc;
  uint32_t stored = 0;
  const uint32_t W = t.state_words;
  const unsigned lane = lane_id();
  const bool vec_ok = (W == 4u * NV) && ((reinterpret_cast<uintptr_t>(keys) & 15u) == 0);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n;
       base += stride) {
    const uint64_t k = base + lane;
    const bool valid = k < n;
    Vec<NV> key;
    if (valid && vec_ok) {
      const uint4* src = reinterpret_cast<const uint4*>(keys + k * W);
#pragma unroll
      for (int j = 0; j < NV; ++j) key.c[j] = __ldg(src + j);
    } else {
      const int32_t* src = keys + k * W;
      uint32_t w[4 * NV];
#pragma unroll
      for (int i = 0; i < 4 * NV; ++i) w[i] = (valid && i < (int)W) ? (uint32_t)__ldg(src + i) : 0u;
#pragma unroll
      for (int j = 0; j < NV; ++j) key.c[j] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
    }
    const uint64_t h = table_hash(key, W, t.seed);
    int res = FOP_ERR;
    uint32_t out = 0;
    bool probe = valid;
    int leader = (int)lane;
    if (DEDUP) {
      const unsigned vmask = __ballot_sync(0xffffffffu, valid);
      const unsigned grp = __match_any_sync(0xffffffffu, h) & vmask;
      if (__any_sync(0xffffffffu, valid && __popc(grp) > 1)) {
        const int lead = valid ? __ffs(grp) - 1 : (int)lane;
        uint32_t diff = 0;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          diff |= __shfl_sync(0xffffffffu, key.c[j].x, lead) ^ key.c[j].x;
          diff |= __shfl_sync(0xffffffffu, key.c[j].y, lead) ^ key.c[j].y;
          diff |= __shfl_sync(0xffffffffu, key.c[j].z, lead) ^ key.c[j].z;
          diff |= __shfl_sync(0xffffffffu, key.c[j].w, lead) ^ key.c[j].w;
        }
        if (valid && lead != (int)lane && diff == 0) {
          probe = false;
          leader = lead;
        }
      }
    }
    if (probe) res = find_or_put<NV, L, false, BW>(t, key, h, out, lc);
    if (DEDUP) {
      const int lres = __shfl_sync(0xffffffffu, res, leader);
      const uint32_t lout = __shfl_sync(0xffffffffu, out, leader);
      if (valid && !probe) {
        res = (lres == FOP_ERR) ? FOP_ERR : FOP_SEEN;
        out = lout;
      }
    }
    if (valid) {
      seen[k] = (uint8_t)res;
      if (idx) idx[k] = out;
      stored += (res == FOP_NEW);
    }
  }
  const uint32_t s = warp_sum(stored);
  const uint32_t bw = warp_sum(lc.busy_waits);
  const uint32_t rh = warp_sum(lc.rehashes);
  if (lane == 0) {
    if (s) atomicAdd(&t.ctr->stored, (unsigned long long)s);
    if (bw) atomicAdd(&t.ctr->busy_waits, (unsigned long long)bw);
    if (rh) atomicAdd(&t.ctr->rehashes, (unsigned long long)rh);
  }
}

// Batched find-or-put with G lanes per key (coop.cuh): the group loads its
// key (the same address in every lane), hashes it and probes whole lines.
template <int NV, int G>
__global__ void __launch_bounds__(256) k_find_or_put_group(TableView t, const int32_t* __restrict__ keys,
                                                           uint64_t n, uint8_t* __restrict__ seen,
                                                           uint32_t* __restrict__ idx) {
  LocalCounters lc;
  uint32_t stored = 0;
  const uint32_t W = t.state_words;
  const unsigned lane = lane_id();
  const int gl = (int)(lane & (G - 1));
  const unsigned gmask = ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
  const bool vec_ok = (W == 4u * NV) && ((reinterpret_cast<uintptr_t>(keys) & 15u) == 0);
  const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / G;
  for (uint64_t k = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; k < n; k += groups) {
    Vec<NV> key;
    if (vec_ok) {
      const uint4* src = reinterpret_cast<const uint4*>(keys + k * W);
#pragma unroll
      for (int j = 0; j < NV; ++j) key.c[j] = __ldg(src + j);
    } else {
      const int32_t* src = keys + k * W;
      uint32_t w[4 * NV];
#pragma unroll
      for (int i = 0; i < 4 * NV; ++i) w[i] = i < (int)W ? (uint32_t)__ldg(src + i) : 0u;
#pragma unroll
      for (int j = 0; j < NV; ++j) key.c[j] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
    }
    const uint64_t h = table_hash(key, W, t.seed);
    uint32_t out = 0;
    const int res = find_or_put_group<NV, G>(t, key, h, out, lc, gl, gmask);
    if (gl == 0) {
      seen[k] = (uint8_t)res;
      if (idx) idx[k] = out;
      stored += (res == FOP_NEW);
    }
  }
  const uint32_t s = warp_sum(stored);
  const uint32_t bw = warp_sum(lc.busy_waits);
  const uint32_t rh = warp_sum(lc.rehashes);
  if (lane == 0) {
    if (s) atomicAdd(&t.ctr->stored, (unsigned long long)s);
    if (bw) atomicAdd(&t.ctr->busy_waits, (unsigned long long)bw);
    if (rh) atomicAdd(&t.ctr->rehashes, (unsigned long long)rh);
  }
}

// Full scan: done / write-state bucket counts and the digest of done rows.
template <int NV>
__global__ void __launch_bounds__(256) k_scan(TableView t, uint64_t nb, unsigned long long* out) {
  unsigned long long done = 0, writing = 0, dig = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t b = t.bucket_bits == 16 ? Bucket<16>::load_relaxed(t.buckets, i)
                                           : Bucket<32>::load_relaxed(t.buckets, i);
    if (b & (t.bucket_bits == 16 ? Bucket<16>::kDoneBit : Bucket<32>::kDoneBit)) {
      Vec<NV> row;
      load_row<NV>(t.data + i * NV, row);
      dig += fingerprint(row, t.state_words);
      ++done;
    } else if (b) {
      ++writing;
    }
  }
  done = warp_sum(done);
  writing = warp_sum(writing);
  dig = warp_sum(dig);
  if (lane_id() == 0) {
    atomicAdd(out + 0, done);
    atomicAdd(out + 1, writing);
    atomicAdd(out + 2, dig);
  }
}

__global__ void k_gather(TableView t, const uint32_t* __restrict__ idx, uint64_t n,
                         int32_t* __restrict__ out) {
  const uint32_t W = t.state_words, rw = 4 * t.nv;
  const uint64_t total = n * W;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = e / W, w = e % W;
    const uint32_t* row = reinterpret_cast<const uint32_t*>(t.data) + (uint64_t)idx[k] * rw;
    out[e] = (int32_t)row[w];
  }
}

// ---------------------------------------------------------------------------
// Dispatch over the compile-time shape (row chunks NV, line buckets L).
// ---------------------------------------------------------------------------
using FopKernel = void (*)(TableView, const int32_t*, uint64_t, uint8_t*, uint32_t*);

template <int NV, int L, int BW>
static FopKernel pick_fop_l(bool dedup) {
  return dedup ? k_find_or_put<NV, L, true, BW> : k_find_or_put<NV, L, false, BW>;
}

template <int NV>
static FopKernel pick_fop_nv(int L, int bw, bool dedup) {
  if (bw == 16) return L == 16 ? pick_fop_l<NV, 16, 16>(dedup) : pick_fop_l<NV, 32, 16>(dedup);
  switch (L) {
    case 8: return pick_fop_l<NV, 8, 32>(dedup);
    case 16: return pick_fop_l<NV, 16, 32>(dedup);
    default: return pick_fop_l<NV, 32, 32>(dedup);
  }
}

template <int G>
static FopKernel pick_fop_group(int nv) {
  switch (nv) {
    case 1: return k_find_or_put_group<1, G>;
    case 2: return k_find_or_put_group<2, G>;
    case 3: return k_find_or_put_group<3, G>;
    case 4: return k_find_or_put_group<4, G>;
    case 5: return k_find_or_put_group<5, G>;
    case 6: return k_find_or_put_group<6, G>;
    case 7: return k_find_or_put_group<7, G>;
    default: return k_find_or_put_group<8, G>;
  }
}

static FopKernel pick_fop(int nv, int L, int bw, bool dedup, int group) {
  if (group == 2) return pick_fop_group<2>(nv);
  if (group == 4) return pick_fop_group<4>(nv);
  if (group == 8) return pick_fop_group<8>(nv);
  switch (nv) {
    case 1: return pick_fop_nv<1>(L, bw, dedup);
    case 2: return pick_fop_nv<2>(L, bw, dedup);
    case 3: return pick_fop_nv<3>(L, bw, dedup);
    case 4: return pick_fop_nv<4>(L, bw, dedup);
    case 5: return pick_fop_nv<5>(L, bw, dedup);
    case 6: return pick_fop_nv<6>(L, bw, dedup);
    case 7: return pick_fop_nv<7>(L, bw, dedup);
    default: return pick_fop_nv<8>(L, bw, dedup);
  }
}

using ScanKernel = void (*)(TableView, uint64_t, unsigned long long*);
static ScanKernel pick_scan(int nv) {
  switch (nv) {
    case 1: return k_scan<1>;
    case 2: return k_scan<2>;
    case 3: return k_scan<3>;
    case 4: return k_scan<4>;
    case 5: return k_scan<5>;
    case 6: return k_scan<6>;
    case 7: return k_scan<7>;
    default: return k_scan<8>;
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

uint64_t table_bytes(uint64_t nb, int max_words) {
  const uint64_t nv = (uint64_t)((max_words + 3) / 4);
  return align_up(sizeof(DevCounters), 256) + align_up(nb * 4, 256) + align_up(nb * 16 * nv, 256) +
         256;  // scan scratch
}

ht_status resolve_params(const ht_params* in, uint64_t nb, ht_params* out) {
  ht_params p{};
  if (in) p = *in;
  if (p.bucket_bits == 0) p.bucket_bits = 32;
  if (p.group_lanes == 0) p.group_lanes = 1;
  if (p.rehash > 1) return HT_ERR_INVALID;
  if (p.group_lanes != 1) {
    // a group of G lanes reads a line of 4G 32-bit buckets at once
    const uint32_t G = p.group_lanes;
    if ((G != 2 && G != 4 && G != 8) || p.bucket_bits != 32 || p.dedup) return HT_ERR_INVALID;
    if (p.line_buckets == 0) p.line_buckets = 4 * G;
    if (p.line_buckets != 4 * G) return HT_ERR_INVALID;
  }
  if (p.bucket_bits == 32) {
    if (p.line_buckets == 0) p.line_buckets = 32;
    if (p.line_buckets != 8 && p.line_buckets != 16 && p.line_buckets != 32) return HT_ERR_INVALID;
  } else if (p.bucket_bits == 16) {
    if (p.line_buckets == 0) p.line_buckets = 16;
    if (p.line_buckets != 16 && p.line_buckets != 32) return HT_ERR_INVALID;
  } else {
    return HT_ERR_INVALID;
  }
  if (nb < p.line_buckets || nb % p.line_buckets) return HT_ERR_INVALID;
  const uint64_t lines = nb / p.line_buckets;
  if (p.max_rehash == 0) p.max_rehash = (uint32_t)(lines < 4096 ? lines : 4096);
  if (p.max_spin == 0) p.max_spin = 1u << 18;
  if (p.block_threads == 0) p.block_threads = 256;
  if (p.block_threads % 32 || p.block_threads > 256) return HT_ERR_INVALID;
  if (p.hash_seed == 0) p.hash_seed = kDefaultSeed;
  *out = p;
  return HT_OK;
}

static bool valid_nb(uint64_t nb) { return nb >= 16 && nb <= kMaxBuckets; }

ht_status table_init_at(ht_t* h, uint64_t nb, int max_words, const ht_params* params, void* mem,
                        uint64_t mem_bytes) {
  if (!valid_nb(nb) || max_words < 1 || max_words > 32 || !mem) return HT_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(mem) & 255u) != 0) return HT_ERR_INVALID;
  ht_status st = resolve_params(params, nb, &h->params);
  if (st != HT_OK) return st;
  if (mem_bytes < table_bytes(nb, max_words)) return HT_ERR_OOM;
  const int nv = (max_words + 3) / 4;
  char* p = static_cast<char*>(mem);
  h->view.ctr = reinterpret_cast<DevCounters*>(p);
  p += align_up(sizeof(DevCounters), 256);
  h->view.buckets = reinterpret_cast<uint32_t*>(p);
  p += align_up(nb * 4, 256);
  h->view.data = reinterpret_cast<uint4*>(p);
  p += align_up(nb * 16 * (uint64_t)nv, 256);
  h->scan_scratch = reinterpret_cast<unsigned long long*>(p);
  const uint64_t lines = nb / h->params.line_buckets;
  const bool pow2 = (nb & (nb - 1)) == 0;
  h->view.seed = h->params.hash_seed;
  h->view.nb_mask = pow2 ? (uint32_t)(nb - 1) : 0u;
  h->view.lines_mask = pow2 ? (uint32_t)(lines - 1) : 0u;
  h->view.lines = (uint32_t)lines;
  h->view.lines_div = pow2 ? DivU64{0, 0, 0} : make_div((uint32_t)lines);
  h->view.max_rehash = h->params.max_rehash;
  h->view.max_spin = h->params.max_spin;
  h->view.state_words = (uint32_t)max_words;
  h->view.nv = (uint32_t)nv;
  h->view.bucket_bits = h->params.bucket_bits;
  h->view.rehash_linear = h->params.rehash;
  h->nb = nb;
  h->max_words = max_words;
  h->bytes = mem_bytes;
  int dev = 0;
  VSS_CUDA_TRY(cudaGetDevice(&dev));
  VSS_CUDA_TRY(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
  return HT_OK;
}

static bool is_prime(uint64_t n) {
  if (n < 2) return false;
  if (n % 2 == 0) return n == 2;
  for (uint64_t f = 3; f * f <= n; f += 2)
    if (n % f == 0) return false;
  return true;
}

uint64_t prime_line_buckets(uint64_t max_nb, uint32_t line_buckets) {
  if (max_nb > kMaxBuckets) max_nb = kMaxBuckets;
  if ((max_nb & (max_nb - 1)) == 0 && max_nb >= 16 && max_nb >= line_buckets) return max_nb;
  for (uint64_t lines = max_nb / line_buckets; lines >= 2; --lines)
    if (is_prime(lines) && lines * line_buckets >= 16) return lines * line_buckets;
  return 0;
}

ht_status table_set_words(ht_t* h, int words) {
  if (words < 1 || words > h->max_words) return HT_ERR_INVALID;
  h->view.state_words = (uint32_t)words;
  h->view.nv = (uint32_t)((words + 3) / 4);
  return HT_OK;
}

ht_status table_clear(ht_t* h, cudaStream_t s) {
  VSS_CUDA_TRY(cudaMemsetAsync(h->view.ctr, 0, sizeof(DevCounters), s));
  VSS_CUDA_TRY(cudaMemsetAsync(h->view.buckets, 0, (size_t)h->nb * (h->view.bucket_bits / 8), s));
  return HT_OK;
}

}  // namespace vss

using namespace vss;

extern "C" {

const char* ht_status_string(ht_status s) {
  switch (s) {
    case HT_OK: return "ok";
    case HT_ERR_INVALID: return "invalid argument";
    case HT_ERR_OOM: return "out of device memory";
    case HT_ERR_FULL: return "table full: no empty bucket within max_rehash lines";
    case HT_ERR_TIMEOUT: return "bounded wait ran out";
    case HT_ERR_CUDA: return "CUDA runtime error";
    case HT_ERR_LEVELS: return "more BFS levels than the level_sizes capacity";
    case HT_ERR_TOO_BIG: return "request exceeds the fixed scratch array of reach_noalloc";
    default: return "unknown status";
  }
}

ht_status ht_bytes_n(uint64_t n_buckets, int state_words, uint64_t* bytes) {
  if (!bytes || !valid_nb(n_buckets) || state_words < 1 || state_words > 32) return HT_ERR_INVALID;
  *bytes = table_bytes(n_buckets, state_words);
  return HT_OK;
}

ht_status ht_bytes(int log2_buckets, int state_words, uint64_t* bytes) {
  if (log2_buckets < 4 || log2_buckets > 31) return HT_ERR_INVALID;
  return ht_bytes_n(1ull << log2_buckets, state_words, bytes);
}

ht_status ht_create_n_at(uint64_t n_buckets, int state_words, const ht_params* params, void* mem_dev,
                         uint64_t mem_bytes, ht_t** out) {
  if (!out) return HT_ERR_INVALID;
  *out = nullptr;
  ht_t* h = new (std::nothrow) ht_t();
  if (!h) return HT_ERR_OOM;
  ht_status st = table_init_at(h, n_buckets, state_words, params, mem_dev, mem_bytes);
  if (st == HT_OK) st = table_clear(h, 0);
  if (st == HT_OK && cudaStreamSynchronize(0) != cudaSuccess) st = HT_ERR_CUDA;
  if (st != HT_OK) {
    delete h;
    return st;
  }
  *out = h;
  return HT_OK;
}

ht_status ht_create_at(int log2_buckets, int state_words, const ht_params* params, void* mem_dev,
                       uint64_t mem_bytes, ht_t** out) {
  if (log2_buckets < 4 || log2_buckets > 31) {
    if (out) *out = nullptr;
    return HT_ERR_INVALID;
  }
  return ht_create_n_at(1ull << log2_buckets, state_words, params, mem_dev, mem_bytes, out);
}

ht_status ht_create(int log2_buckets, int state_words, const ht_params* params, ht_t** out) {
  uint64_t bytes = 0;
  if (!out) return HT_ERR_INVALID;
  *out = nullptr;
  ht_status st = ht_bytes(log2_buckets, state_words, &bytes);
  if (st != HT_OK) return st;
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return HT_ERR_OOM;
  }
  st = ht_create_at(log2_buckets, state_words, params, mem, bytes, out);
  if (st != HT_OK) {
    cudaFree(mem);
    return st;
  }
  (*out)->owned = mem;
  return HT_OK;
}

ht_status ht_buckets_for_bytes(uint64_t bytes, int state_words, const ht_params* params,
                               uint64_t* n_buckets) {
  if (!n_buckets || state_words < 1 || state_words > 32) return HT_ERR_INVALID;
  *n_buckets = 0;
  ht_params p{};
  ht_status st = resolve_params(params, 1u << 10, &p);
  if (st != HT_OK) return st;
  // table_bytes is increasing in nb: the largest nb that fits, then round down
  uint64_t lo = 0, hi = kMaxBuckets;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo + 1) / 2;
    if (table_bytes(mid, state_words) <= bytes) lo = mid;
    else hi = mid - 1;
  }
  const uint64_t nb = prime_line_buckets(lo, p.line_buckets);
  if (nb == 0) return HT_ERR_OOM;
  *n_buckets = nb;
  return HT_OK;
}

ht_status vss_line_divide(uint32_t d, const uint64_t* n_host, uint64_t count, uint64_t* q_host,
                          uint32_t* r_host) {
  if (d == 0 || (count && (!n_host || !q_host || !r_host))) return HT_ERR_INVALID;
  const DivU64 v = make_div(d);
  for (uint64_t i = 0; i < count; ++i) {
    q_host[i] = div_q(v, n_host[i]);
    r_host[i] = div_r(v, n_host[i]);
  }
  return HT_OK;
}

ht_status ht_destroy(ht_t* h) {
  if (!h) return HT_ERR_INVALID;
  if (h->owned) cudaFree(h->owned);
  delete h;
  return HT_OK;
}

ht_status ht_clear(ht_t* h, void* stream) {
  if (!h) return HT_ERR_INVALID;
  return table_clear(h, static_cast<cudaStream_t>(stream));
}

ht_status ht_find_or_put(ht_t* h, const int32_t* keys_dev, uint64_t n, uint8_t* seen_dev,
                         uint32_t* idx_dev, void* stream) {
  if (!h || (n && (!keys_dev || !seen_dev))) return HT_ERR_INVALID;
  if (n == 0) return HT_OK;
  const int threads = (int)h->params.block_threads;
  const uint64_t want = (n * h->params.group_lanes + threads - 1) / threads;  // G lanes per key
  // 64 blocks per SM, run in waves: measured 6-26 % faster than 16 (the
  // grid-stride loop of fewer, longer-lived blocks ends unevenly)
  const uint64_t cap = (uint64_t)h->num_sms * 64;
  const int blocks = (int)(want < cap ? want : cap);
  FopKernel k = pick_fop((int)h->view.nv, (int)h->params.line_buckets, (int)h->view.bucket_bits,
                         h->params.dedup != 0, (int)h->params.group_lanes);
  k<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(h->view, keys_dev, n, seen_dev,
                                                                idx_dev);
  VSS_CUDA_TRY(cudaGetLastError());
  return HT_OK;
}

ht_status ht_sync(ht_t* h, void* stream) {
  if (!h) return HT_ERR_INVALID;
  VSS_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  uint32_t err = 0;
  VSS_CUDA_TRY(cudaMemcpy(&err, &h->view.ctr->err, 4, cudaMemcpyDeviceToHost));
  return (ht_status)err;
}

ht_status ht_stats(ht_t* h, void* stream, ht_stats_t* out) {
  if (!h || !out) return HT_ERR_INVALID;
  VSS_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  DevCounters c;
  VSS_CUDA_TRY(cudaMemcpy(&c, h->view.ctr, sizeof(c), cudaMemcpyDeviceToHost));
  out->stored = c.stored;
  out->busy_waits = c.busy_waits;
  out->rehashes = c.rehashes;
  out->capacity = h->nb;
  out->error = c.err;
  out->state_words = h->view.state_words;
  return HT_OK;
}

ht_status ht_scan(ht_t* h, void* stream, uint64_t* done, uint64_t* writing, uint64_t* digest) {
  if (!h) return HT_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  VSS_CUDA_TRY(cudaMemsetAsync(h->scan_scratch, 0, 3 * sizeof(unsigned long long), s));
  const uint64_t nb = h->nb;
  const uint64_t want = (nb + 255) / 256, cap = (uint64_t)h->num_sms * 8;
  pick_scan((int)h->view.nv)<<<(int)(want < cap ? want : cap), 256, 0, s>>>(h->view, nb,
                                                                            h->scan_scratch);
  VSS_CUDA_TRY(cudaGetLastError());
  unsigned long long r[3];
  VSS_CUDA_TRY(cudaMemcpyAsync(r, h->scan_scratch, sizeof(r), cudaMemcpyDeviceToHost, s));
  VSS_CUDA_TRY(cudaStreamSynchronize(s));
  if (done) *done = r[0];
  if (writing) *writing = r[1];
  if (digest) *digest = r[2];
  return HT_OK;
}

ht_status ht_gather(ht_t* h, const uint32_t* idx_dev, uint64_t n, int32_t* out_dev, void* stream) {
  if (!h || (n && (!idx_dev || !out_dev))) return HT_ERR_INVALID;
  if (n == 0) return HT_OK;
  const uint64_t total = n * h->view.state_words;
  const uint64_t want = (total + 255) / 256, cap = (uint64_t)h->num_sms * 8;
  k_gather<<<(int)(want < cap ? want : cap), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      h->view, idx_dev, n, out_dev);
  VSS_CUDA_TRY(cudaGetLastError());
  return HT_OK;
}

ht_status ht_arrays(ht_t* h, uint32_t** buckets_dev, int32_t** data_dev, uint32_t* row_words) {
  if (!h) return HT_ERR_INVALID;
  if (buckets_dev) *buckets_dev = h->view.buckets;
  if (data_dev) *data_dev = reinterpret_cast<int32_t*>(h->view.data);
  if (row_words) *row_words = 4 * h->view.nv;
  return HT_OK;
}

}  // extern "C"
