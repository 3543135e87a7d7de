// Shared device/host definitions of the GB300 visited-state store.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "divide.h"
#include "reach.h"

namespace vss {

constexpr uint32_t kDone = HT_BUCKET_DONE;
constexpr uint32_t kMemoMask = HT_BUCKET_MEMO;
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
  uint32_t nb_mask;       // nb - 1 (power-of-two tables)
  uint32_t lines_mask;    // lines - 1 (power-of-two tables)
  uint32_t max_rehash;
  uint32_t max_spin;
  uint32_t state_words;   // W
  uint32_t nv;            // ceil(W / 4)
  uint32_t bucket_bits;   // 32 or 16: width of a bucket word
  uint32_t lines;         // nb / line_buckets
  uint32_t rehash_linear; // 1: the next line after a full line; 0: double hashing
  DivU64 lines_div;       // division by `lines`; m == 0 marks a power-of-two table
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
// 32-byte accesses (one full L2 sector per instruction; the address must be
// 32-byte aligned).
#define VSS_V8_OUT(a, b) "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
__device__ __forceinline__ void ld_acquire_v8(const void* p, uint4& a, uint4& b) {
  asm volatile("ld.acquire.gpu.global.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : VSS_V8_OUT(a, b) : "l"(p) : "memory");
}
__device__ __forceinline__ void ld_relaxed_v8(const void* p, uint4& a, uint4& b) {
  asm volatile("ld.relaxed.gpu.global.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : VSS_V8_OUT(a, b) : "l"(p) : "memory");
}
__device__ __forceinline__ void ld_cg_v8(const void* p, uint4& a, uint4& b) {
  asm volatile("ld.global.cg.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : VSS_V8_OUT(a, b) : "l"(p) : "memory");
}
__device__ __forceinline__ void st_v8(void* p, const uint4& a, const uint4& b) {
  asm volatile("st.global.v8.u32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(a.x), "r"(a.y),
               "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
               : "memory");
}

#undef VSS_V8_OUT

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u16(const uint16_t* p) {
  unsigned short v;
  asm volatile("ld.acquire.gpu.global.u16 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u16(const uint16_t* p) {
  unsigned short v;
  asm volatile("ld.relaxed.gpu.global.u16 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u16(uint16_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u16 [%0], %1;" ::"l"(p), "h"((unsigned short)v) : "memory");
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
// Table hash.  The paper leaves the hash family open (Section 3.3: h_num).
// This one is a position-keyed additive hash finished by the MurmurHash3
// fmix64 avalanche (Appleby, public domain):
//   S(v)  = sum over words k < W of term(k, v_k)          (mod 2^64)
//   term  = z ^ (z >> 29),  z = (v_k xor c_k) * 0xBF58476D1CE4E5B9,
//           c_k = seed + (k + 1) * 0x9E3779B97F4A7C15
//   h(v)  = fmix64(S(v) + W)
// term(k, .) is injective, so vectors differing in one word never collide in
// S, and a successor that changes words p and q of its parent v gets
// S = S(v) - term(p, v_p) + term(p, x) [- term(q, v_q) + term(q, y)] in a few
// instructions.  One hash serves every rehash round: the index comes from its
// low bits, the memo from bits 33..63, the double-hashing step from the memo.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdULL;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ULL;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ uint64_t hash_term(uint64_t seed, int k, uint32_t x) {
  const uint64_t z = ((uint64_t)x ^ (seed + (uint64_t)(k + 1) * 0x9E3779B97F4A7C15ULL)) *
                     0xBF58476D1CE4E5B9ULL;
  return z ^ (z >> 29);
}

template <int NV>
__device__ __forceinline__ uint64_t hash_sum(const Vec<NV>& v, uint32_t W, uint64_t seed) {
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < 4 * NV; ++k)
    if (k < (int)W) s += hash_term(seed, k, vec_word(v, k));
  return s;
}

__device__ __forceinline__ uint64_t hash_final(uint64_t s, uint32_t W) { return fmix64(s + W); }

template <int NV>
__device__ __forceinline__ uint64_t table_hash(const Vec<NV>& v, uint32_t W, uint64_t seed) {
  return hash_final(hash_sum(v, W, seed), W);
}

__device__ __forceinline__ uint32_t memo_of(uint64_t h) {
  const uint32_t m = (uint32_t)(h >> 33);
  return m ? m : 1u;
}

// memo of a 16-bit bucket: the top 15 bits of the hash, 0 mapped to 1
__device__ __forceinline__ uint32_t memo16_of(uint64_t h) {
  const uint32_t m = (uint32_t)(h >> 49);
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

// Rows of an even number of 16-byte chunks are 32-byte aligned: move them a
// sector per instruction.
// Load a data row (nv chunks) with strong gpu-scope loads.
template <int NV>
__device__ __forceinline__ void load_row(const uint4* row, Vec<NV>& v) {
  if (NV % 2 == 0) {
#pragma unroll
    for (int j = 0; j < NV; j += 2) ld_relaxed_v8(row + j, v.c[j], v.c[(j + 1) % NV]);
  } else {
#pragma unroll
    for (int j = 0; j < NV; ++j) v.c[j] = ld_relaxed_v4(row + j);
  }
}

// Load a frontier row (written before the last grid barrier) through L2.
template <int NV>
__device__ __forceinline__ void load_row_cg(const uint4* row, Vec<NV>& v) {
  if (NV % 2 == 0) {
#pragma unroll
    for (int j = 0; j < NV; j += 2) ld_cg_v8(row + j, v.c[j], v.c[(j + 1) % NV]);
  } else {
#pragma unroll
    for (int j = 0; j < NV; ++j) v.c[j] = __ldcg(row + j);
  }
}

// Run-time row width (nv <= NV chunks; the rest of v is zero): used where one
// kernel serves tables of different widths.
template <int NV>
__device__ __forceinline__ void load_row_rt(const uint4* row, Vec<NV>& v, uint32_t nv) {
  if ((nv & 1u) == 0) {
#pragma unroll
    for (int j = 0; j < NV; j += 2) {
      if (j < (int)nv) ld_relaxed_v8(row + j, v.c[j], v.c[(j + 1) % NV]);
      else v.c[j] = v.c[(j + 1) % NV] = make_uint4(0, 0, 0, 0);
    }
  } else {
#pragma unroll
    for (int j = 0; j < NV; ++j) v.c[j] = j < (int)nv ? ld_relaxed_v4(row + j) : make_uint4(0, 0, 0, 0);
  }
}

template <int NV>
__device__ __forceinline__ void load_row_cg_rt(const uint4* row, Vec<NV>& v, uint32_t nv) {
  if ((nv & 1u) == 0) {
#pragma unroll
    for (int j = 0; j < NV; j += 2) {
      if (j < (int)nv) ld_cg_v8(row + j, v.c[j], v.c[(j + 1) % NV]);
      else v.c[j] = v.c[(j + 1) % NV] = make_uint4(0, 0, 0, 0);
    }
  } else {
#pragma unroll
    for (int j = 0; j < NV; ++j) v.c[j] = j < (int)nv ? __ldcg(row + j) : make_uint4(0, 0, 0, 0);
  }
}

template <int NV>
__device__ __forceinline__ void store_row_rt(uint4* row, const Vec<NV>& v, uint32_t nv) {
  if ((nv & 1u) == 0) {
#pragma unroll
    for (int j = 0; j < NV; j += 2)
      if (j < (int)nv) st_v8(row + j, v.c[j], v.c[(j + 1) % NV]);
  } else {
#pragma unroll
    for (int j = 0; j < NV; ++j)
      if (j < (int)nv) row[j] = v.c[j];
  }
}

template <int NV>
__device__ __forceinline__ void store_row(uint4* row, const Vec<NV>& v) {
  if (NV % 2 == 0) {
#pragma unroll
    for (int j = 0; j < NV; j += 2) st_v8(row + j, v.c[j], v.c[(j + 1) % NV]);
  } else {
#pragma unroll
    for (int j = 0; j < NV; ++j) row[j] = v.c[j];
  }
}

}  // namespace vss

// Host-side helpers.
#define VSS_CUDA_TRY(expr)                              \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return HT_ERR_CUDA;          \
  } while (0)
