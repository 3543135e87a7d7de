// Shared device/host definitions of the GB300 visited-state store.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "reach.h"

namespace vss {

constexpr uint32_t kDone = HT_BUCKET_DONE;
constexpr uint32_t kMemoMask = HT_BUCKET_MEMO;
constexpr int kSectorBuckets = 8;  // one 32-byte L2 sector of 32-bit buckets
constexpr int kMaxNV = 8;          // up to 32 words per state (8 x 16 bytes)
constexpr uint64_t kDefaultSeed = 0x2545F4914F6CDD1DULL;

enum FopResult : int { FOP_NEW = 0, FOP_SEEN = 1, FOP_ERR = 2 };

// Device-resident counters of one table (zeroed by ht_clear).
struct __align__(16) DevCounters {
  uint32_t err;  // first latched ht_status, 0 = none
  uint32_t pad0;
  unsigned long long stored;
  unsigned long long busy_waits;
  unsigned long long rehashes;
  unsigned long long pad1[4];
};

// Everything a kernel needs to probe one table; passed by value.
struct TableView {
  uint32_t* buckets;      // [nb]
  uint4* data;            // [nb * nv] rows of nv 16-byte chunks
  DevCounters* ctr;
  uint64_t seed;
  uint32_t nb_mask;       // nb - 1
  uint32_t lines_mask;    // nb / line_buckets - 1
  uint32_t max_rehash;
  uint32_t max_spin;
  uint32_t state_words;   // W
  uint32_t nv;            // ceil(W / 4)
};

// ---------------------------------------------------------------------------
// Scoped memory operations (PTX memory model, gpu scope).  Bucket words are
// read with strong gpu-scope loads so that every probe sees the L2 copy, the
// point of coherence, never a stale L1 line.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint4 ld_relaxed_v4(const void* p) {
  uint4 v;
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
__device__ __forceinline__ uint4 ld_acquire_v4(const void* p) {
  uint4 v;
  asm volatile("ld.acquire.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void latch_error(DevCounters* c, uint32_t code) {
  atomicCAS(&c->err, 0u, code);
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// State vectors in registers: NV chunks of 4 words, padding words zero.
// ---------------------------------------------------------------------------
template <int NV>
struct Vec {
  uint4 c[NV];
};

template <int NV>
__device__ __forceinline__ uint32_t vec_word(const Vec<NV>& v, int k) {
  const uint4& q = v.c[k >> 2];
  switch (k & 3) {
    case 0: return q.x;
    case 1: return q.y;
    case 2: return q.z;
    default: return q.w;
  }
}

// Word i of v for a run-time i: a select chain (keeps v in registers).
template <int NV>
__device__ __forceinline__ uint32_t vec_get(const Vec<NV>& v, int i) {
  uint32_t r = 0;
#pragma unroll
  for (int k = 0; k < 4 * NV; ++k) r = (k == i) ? vec_word(v, k) : r;
  return r;
}

template <int NV>
__device__ __forceinline__ bool vec_eq(const Vec<NV>& a, const Vec<NV>& b) {
  uint32_t d = 0;
#pragma unroll
  for (int j = 0; j < NV; ++j)
    d |= (a.c[j].x ^ b.c[j].x) | (a.c[j].y ^ b.c[j].y) | (a.c[j].z ^ b.c[j].z) |
         (a.c[j].w ^ b.c[j].w);
  return d == 0;
}

// ---------------------------------------------------------------------------
// Table hash.  The paper leaves the hash family open (Section 3.3: h_num);
// this is a single-lane MurmurHash3-x64 style accumulation (Appleby, public
// domain MurmurHash3: per 64-bit block k *= c1, k = rotl(k,31), k *= c2,
// h ^= k, h = rotl(h,27)*5 + 0x52dce729) over the padded vector, finished with
// the MurmurHash3 fmix64 avalanche.  One hash serves every rehash round: the
// index comes from its low bits, the memo from bits 33..63, the double-hashing
// step from the memo.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdULL;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ULL;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ uint64_t murmur_block(uint64_t h, uint64_t k) {
  k *= 0x87c37b91114253d5ULL;
  k = rotl64(k, 31);
  k *= 0x4cf5ad432745937fULL;
  h ^= k;
  h = rotl64(h, 27);
  return h * 5 + 0x52dce729ULL;
}

template <int NV>
__device__ __forceinline__ uint64_t table_hash(const Vec<NV>& v, uint32_t W, uint64_t seed) {
  uint64_t h = seed;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    h = murmur_block(h, (uint64_t)v.c[j].x | ((uint64_t)v.c[j].y << 32));
    h = murmur_block(h, (uint64_t)v.c[j].z | ((uint64_t)v.c[j].w << 32));
  }
  h ^= (uint64_t)W * 4u;
  return fmix64(h);
}

__device__ __forceinline__ uint32_t memo_of(uint64_t h) {
  const uint32_t m = (uint32_t)(h >> 33);
  return m ? m : 1u;
}

// ---------------------------------------------------------------------------
// Set fingerprint of a stored state: x = W; x = sm(x ^ word) per word, with sm
// one SplitMix64 output step (Steele, Lea, Flood 2014).  Summed mod 2^64 over
// a set it gives an order-independent digest.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix_step(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

template <int NV>
__device__ __forceinline__ uint64_t fingerprint(const Vec<NV>& v, uint32_t W) {
  uint64_t x = W;
#pragma unroll
  for (int k = 0; k < 4 * NV; ++k)
    if (k < (int)W) x = splitmix_step(x ^ (uint64_t)vec_word(v, k));
  return x;
}

// Load a data row (nv chunks) with strong gpu-scope loads.
template <int NV>
__device__ __forceinline__ void load_row(const uint4* row, Vec<NV>& v) {
#pragma unroll
  for (int j = 0; j < NV; ++j) v.c[j] = ld_relaxed_v4(row + j);
}

}  // namespace vss

// Host-side helpers.
#define VSS_CUDA_TRY(expr)                              \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return HT_ERR_CUDA;          \
  } while (0)
