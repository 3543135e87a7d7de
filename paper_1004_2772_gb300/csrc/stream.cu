// Key streams for the hash-table benchmark, generated on the device.
//
// A fill of a table with n_ids distinct keys is a stream of 2 * n_ids calls:
// call 2i inserts key i; call 2i+1 repeats a key chosen from
// r = mix(c xor mix(seed)): uniformly among the earlier ids [0, i] as
// floor(r * (i + 1) / 2^64) (a multiply-high range reduction), or by a
// Zipf(1.1) law over all ids through an integer quantile table (so that the
// device and the host generator draw identical ids).  Key i is
//   word 0      = fmix32(i)                     (MurmurHash3 finaliser: a bijection,
//                                                so distinct ids give distinct keys)
//   words 2q-1, 2q (q >= 1) = the low and high 32 bits of mix((seed << 36) + (i << 4) + q)
// with mix the SplitMix64 output step (Steele, Lea, Flood 2014): one output
// per two words.  These are inputs, not part of the method: the same
// definition is implemented on the host by the seeded input generator, and a
// GPU test checks the two agree.
//
// k_gen_keys materialises keys (for the batch API); k_find_or_put_stream
// runs find-or-put on keys generated in registers, so the table is measured
// without streaming keys from HBM.
#include "coop.cuh"
#include "internal.h"
#include "table.cuh"

namespace vss {

__device__ __forceinline__ uint64_t sm_out(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t fmix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

struct StreamSpec {
  uint64_t seed;
  uint64_t seed_key;      // mix(seed)
  uint64_t n_ids;
  const uint32_t* zipf;   // 2^16 + 1 quantile entries, or null for uniform reuse
};

__device__ __forceinline__ uint64_t call_id(const StreamSpec& s, uint64_t c) {
  const uint64_t i = c >> 1;
  if (!(c & 1)) return i;
  const uint64_t r = sm_out(c ^ s.seed_key);
  if (!s.zipf) return __umul64hi(r, i + 1);
  const uint32_t cell = (uint32_t)(r >> 48);
  const uint64_t lo = s.zipf[cell], hi = s.zipf[cell + 1];
  const uint64_t width = hi > lo ? hi - lo : 1;
  uint64_t rank = lo + (r & 0xFFFFFFFFull) % width;
  rank = rank < s.n_ids ? rank : s.n_ids;
  return rank - 1;
}

template <int NV>
__device__ __forceinline__ void key_of(uint64_t seed, uint64_t id, uint32_t W, Vec<NV>& k) {
  const uint64_t base = (seed << 36) + (id << 4);
  uint32_t w[4 * NV + 1];
  w[0] = fmix32((uint32_t)id);
#pragma unroll
  for (int q = 1; 2 * q - 1 < 4 * NV; ++q) {  // words 2q-1 and 2q from one output
    const uint64_t z = sm_out(base + (uint64_t)q);
    w[2 * q - 1] = (uint32_t)z;
    w[2 * q] = (uint32_t)(z >> 32);
  }
#pragma unroll
  for (int j = 0; j < 4 * NV; ++j) w[j] = j < (int)W ? w[j] : 0u;
#pragma unroll
  for (int q = 0; q < NV; ++q) k.c[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}

template <int NV>
__global__ void __launch_bounds__(256) k_gen_keys(StreamSpec s, uint64_t c0, uint64_t n, uint32_t W,
                                                  int32_t* __restrict__ out) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (uint64_t)gridDim.x * blockDim.x) {
    Vec<NV> k;
    key_of<NV>(s.seed, call_id(s, c0 + t), W, k);
    int32_t* row = out + t * W;
#pragma unroll
    for (int j = 0; j < 4 * NV; ++j)
      if (j < (int)W) row[j] = (int32_t)vec_word(k, j);
  }
}

// Fused generator + find-or-put.  Counts new keys and sums the fingerprints
// of the keys it stored (the set digest of the fill).
template <int NV, int L, bool DEDUP, int BW>
__global__ void __launch_bounds__(256, table_min_blocks<NV>()) k_find_or_put_stream(TableView t, StreamSpec s, uint64_t c0,
                                                            uint64_t n, unsigned long long* out) {
  LocalCounters lc;
  unsigned long long n_new = 0, dig = 0;
  const unsigned lane = lane_id();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n;
       base += stride) {
    const uint64_t k = base + lane;
    const bool valid = k < n;
    Vec<NV> key;
    key_of<NV>(s.seed, valid ? call_id(s, c0 + k) : 0, t.state_words, key);
    const uint64_t h = table_hash(key, t.state_words, t.seed);
    int res = FOP_ERR;
    uint32_t idx = 0;
    bool probe = valid;
    if (DEDUP) {
      // equal keys in one warp: only the lowest lane probes; a 64-bit hash
      // match is confirmed by comparing every word
      const unsigned vmask = __ballot_sync(0xffffffffu, valid);
      const unsigned grp = __match_any_sync(0xffffffffu, h) & vmask;
      const int lead = valid && grp ? __ffs(grp) - 1 : (int)lane;
      uint32_t diff = 0;
      if (__any_sync(0xffffffffu, valid && __popc(grp) > 1)) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          diff |= __shfl_sync(0xffffffffu, key.c[j].x, lead) ^ key.c[j].x;
          diff |= __shfl_sync(0xffffffffu, key.c[j].y, lead) ^ key.c[j].y;
          diff |= __shfl_sync(0xffffffffu, key.c[j].z, lead) ^ key.c[j].z;
          diff |= __shfl_sync(0xffffffffu, key.c[j].w, lead) ^ key.c[j].w;
        }
        if (valid && lead != (int)lane && diff == 0) probe = false;
      }
    }
    if (probe) res = find_or_put<NV, L, false, BW>(t, key, h, idx, lc);
    if (res == FOP_NEW) {
      ++n_new;
      dig += fingerprint(key, t.state_words);
    }
  }
  n_new = warp_sum(n_new);
  dig = warp_sum(dig);
  const uint32_t bw = warp_sum(lc.busy_waits), rh = warp_sum(lc.rehashes);
  if (lane == 0) {
    if (n_new) {
      atomicAdd(out + 0, n_new);
      atomicAdd(&t.ctr->stored, n_new);
    }
    if (dig) atomicAdd(out + 1, dig);
    if (bw) atomicAdd(&t.ctr->busy_waits, (unsigned long long)bw);
    if (rh) atomicAdd(&t.ctr->rehashes, (unsigned long long)rh);
  }
}

// The same with G lanes per key (coop.cuh); every lane of a group generates
// the group's key.
template <int NV, int G>
__global__ void __launch_bounds__(256) k_find_or_put_stream_group(TableView t, StreamSpec s, uint64_t c0,
                                                                  uint64_t n, unsigned long long* out) {
  LocalCounters lc;
  unsigned long long n_new = 0, dig = 0;
  const unsigned lane = lane_id();
  const int gl = (int)(lane & (G - 1));
  const unsigned gmask = ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
  const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / G;
  for (uint64_t k = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; k < n; k += groups) {
    Vec<NV> key;
    key_of<NV>(s.seed, call_id(s, c0 + k), t.state_words, key);
    const uint64_t h = table_hash(key, t.state_words, t.seed);
    uint32_t idx = 0;
    const int res = find_or_put_group<NV, G>(t, key, h, idx, lc, gl, gmask);
    if (res == FOP_NEW && gl == 0) {
      ++n_new;
      dig += fingerprint(key, t.state_words);
    }
  }
  n_new = warp_sum(n_new);
  dig = warp_sum(dig);
  const uint32_t bw = warp_sum(lc.busy_waits), rh = warp_sum(lc.rehashes);
  if (lane == 0) {
    if (n_new) {
      atomicAdd(out + 0, n_new);
      atomicAdd(&t.ctr->stored, n_new);
    }
    if (dig) atomicAdd(out + 1, dig);
    if (bw) atomicAdd(&t.ctr->busy_waits, (unsigned long long)bw);
    if (rh) atomicAdd(&t.ctr->rehashes, (unsigned long long)rh);
  }
}

using StreamKernel = void (*)(TableView, StreamSpec, uint64_t, uint64_t, unsigned long long*);

template <int G>
static StreamKernel pick_stream_group(int nv) {
  switch (nv) {
    case 1: return k_find_or_put_stream_group<1, G>;
    case 2: return k_find_or_put_stream_group<2, G>;
    case 4: return k_find_or_put_stream_group<4, G>;
    case 8: return k_find_or_put_stream_group<8, G>;
    default: return nullptr;
  }
}

template <int NV, int L, int BW>
static StreamKernel pick_stream_l(bool dedup) {
  return dedup ? k_find_or_put_stream<NV, L, true, BW> : k_find_or_put_stream<NV, L, false, BW>;
}

template <int NV>
static StreamKernel pick_stream_nv(int L, int bw, bool dedup) {
  if (bw == 16) return L == 16 ? pick_stream_l<NV, 16, 16>(dedup) : pick_stream_l<NV, 32, 16>(dedup);
  switch (L) {
    case 8: return pick_stream_l<NV, 8, 32>(dedup);
    case 16: return pick_stream_l<NV, 16, 32>(dedup);
    default: return pick_stream_l<NV, 32, 32>(dedup);
  }
}

static StreamKernel pick_stream(int nv, int L, int bw, bool dedup, int group) {
  if (group == 2) return pick_stream_group<2>(nv);
  if (group == 4) return pick_stream_group<4>(nv);
  if (group == 8) return pick_stream_group<8>(nv);
  switch (nv) {
    case 1: return pick_stream_nv<1>(L, bw, dedup);
    case 2: return pick_stream_nv<2>(L, bw, dedup);
    case 4: return pick_stream_nv<4>(L, bw, dedup);
    case 8: return pick_stream_nv<8>(L, bw, dedup);
    default: return nullptr;
  }
}

static StreamSpec make_spec(uint64_t seed, uint64_t n_ids, const uint32_t* zipf) {
  StreamSpec s;
  s.seed = seed;
  // mix(seed) on the host: the same SplitMix64 output step as sm_out
  uint64_t z = seed + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  s.seed_key = z ^ (z >> 31);
  s.n_ids = n_ids;
  s.zipf = zipf;
  return s;
}

}  // namespace vss

using namespace vss;

extern "C" {

ht_status vss_gen_keys(uint64_t seed, uint64_t n_ids, uint64_t call_begin, uint64_t n_calls,
                       const uint32_t* zipf_table_dev, int state_words, int32_t* keys_dev,
                       void* stream) {
  if (n_ids == 0 || state_words < 1 || state_words > 32 || (n_calls && !keys_dev))
    return HT_ERR_INVALID;
  if (call_begin + n_calls > 2 * n_ids) return HT_ERR_INVALID;
  if (n_calls == 0) return HT_OK;
  const StreamSpec s = make_spec(seed, n_ids, zipf_table_dev);
  int dev = 0, sms = 0;
  VSS_CUDA_TRY(cudaGetDevice(&dev));
  VSS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const uint64_t want = (n_calls + 255) / 256, cap = (uint64_t)sms * 16;
  const int blocks = (int)(want < cap ? want : cap);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t W = (uint32_t)state_words;
  switch ((state_words + 3) / 4) {
    case 1: k_gen_keys<1><<<blocks, 256, 0, st>>>(s, call_begin, n_calls, W, keys_dev); break;
    case 2: k_gen_keys<2><<<blocks, 256, 0, st>>>(s, call_begin, n_calls, W, keys_dev); break;
    case 3: k_gen_keys<3><<<blocks, 256, 0, st>>>(s, call_begin, n_calls, W, keys_dev); break;
    case 4: k_gen_keys<4><<<blocks, 256, 0, st>>>(s, call_begin, n_calls, W, keys_dev); break;
    case 5: k_gen_keys<5><<<blocks, 256, 0, st>>>(s, call_begin, n_calls, W, keys_dev); break;
    case 6: k_gen_keys<6><<<blocks, 256, 0, st>>>(s, call_begin, n_calls, W, keys_dev); break;
    case 7: k_gen_keys<7><<<blocks, 256, 0, st>>>(s, call_begin, n_calls, W, keys_dev); break;
    default: k_gen_keys<8><<<blocks, 256, 0, st>>>(s, call_begin, n_calls, W, keys_dev); break;
  }
  VSS_CUDA_TRY(cudaGetLastError());
  return HT_OK;
}

ht_status ht_find_or_put_stream(ht_t* h, uint64_t seed, uint64_t n_ids, uint64_t call_begin,
                                uint64_t n_calls, const uint32_t* zipf_table_dev,
                                uint64_t* result_dev, void* stream) {
  if (!h || !result_dev || n_ids == 0 || call_begin + n_calls > 2 * n_ids) return HT_ERR_INVALID;
  StreamKernel k = pick_stream((int)h->view.nv, (int)h->params.line_buckets,
                               (int)h->view.bucket_bits, h->params.dedup != 0,
                               (int)h->params.group_lanes);
  if (!k) return HT_ERR_INVALID;
  if (n_calls == 0) return HT_OK;
  const StreamSpec s = make_spec(seed, n_ids, zipf_table_dev);
  const int threads = (int)h->params.block_threads;
  const uint64_t lanes = n_calls * h->params.group_lanes;  // G lanes per key in group mode
  // 64 blocks per SM, as for the batch API
  const uint64_t want = (lanes + threads - 1) / threads, cap = (uint64_t)h->num_sms * 64;
  const int blocks = (int)(want < cap ? want : cap);
  k<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
      h->view, s, call_begin, n_calls, reinterpret_cast<unsigned long long*>(result_dev));
  VSS_CUDA_TRY(cudaGetLastError());
  return HT_OK;
}

}  // extern "C"
