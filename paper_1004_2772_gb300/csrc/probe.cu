// Random-access HBM probe: the denominator of the random-sector roofline.
//
// The store's hot path moves data in 32-byte L2 sectors at random addresses
// (one bucket sector per probe, one or two sectors per data row).  This
// kernel measures how many such random accesses per second the GPU's memory
// system sustains, with the same access shapes: every thread issues INF
// independent accesses to sectors chosen by a counter-based hash (SplitMix64
// output function of the access number) before it consumes any.  The caller
// picks INF, the blocks per SM and the threads per block, so a sweep over
// them finds the rate's plateau rather than the limit of one probe shape.
#include "internal.h"

namespace vss {

__device__ __forceinline__ uint64_t probe_mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Unit number of access a: a multiply-high range reduction of a counter-based
// hash (uniform over [0, n_units) up to a bias below 2^-32 for n_units < 2^32;
// no 64-bit division on the access path).
__device__ __forceinline__ uint64_t probe_unit(uint64_t seed, uint64_t a, uint64_t n_units) {
  return __umul64hi(probe_mix(seed ^ a), n_units);
}

// mode 0: read one 32 B sector; 1: read 64 B (two adjacent sectors, 64 B
// aligned); 2: write one 32 B sector; 3: atomicAdd on one 32-bit word;
// 4 / 5: compare-and-swap (0 -> x) on a 32- / 16-bit word; 6 / 7: relaxed
// gpu-scope store of one 32- / 16-bit word (the claim and publish steps of an
// insert, for either bucket width); 8: read 4 bytes of a random 32 B sector
// (the whole sector still comes from DRAM into L2, only 4 bytes go back to
// the SM: the memory side of mode 0 without its return traffic); 9: read 64 B
// by two lanes, 32 B each, in one load instruction; 10: read a 128 B line by
// four lanes in one instruction.  In modes 9 and 10 an access is the group's:
// n_access counts groups, and every lane of a group keeps INF of them in flight.
// INF accesses per thread are issued before any is consumed.
template <int MODE, int INF>
__global__ void __launch_bounds__(256, 1) k_probe(uint4* buf, uint64_t n_units, uint64_t n_access,
                                                uint64_t seed, unsigned long long* sink) {
  // lanes per access: one, or a pair / quad of adjacent lanes reading one unit together
  constexpr int G = MODE == 9 ? 2 : MODE == 10 ? 4 : 1;
  const uint64_t tid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x / G;
  const uint32_t part = threadIdx.x & (G - 1);  // this lane's 32 bytes of the unit
  uint32_t acc = 0;
  uint64_t base = tid * INF;
  for (; base < n_access; base += nthr * INF) {
    uint64_t u[INF];
#pragma unroll
    for (int k = 0; k < INF; ++k) u[k] = probe_unit(seed, base + k, n_units);
    if (MODE == 9 || MODE == 10) {
      if (base + INF > n_access) break;  // a partial group: the tail loop below
      uint4 v[INF][2];
#pragma unroll
      for (int k = 0; k < INF; ++k) ld_cg_v8(buf + u[k] * (2 * G) + 2 * part, v[k][0], v[k][1]);
#pragma unroll
      for (int k = 0; k < INF; ++k)
#pragma unroll
        for (int q = 0; q < 2; ++q) acc ^= v[k][q].x ^ v[k][q].y ^ v[k][q].z ^ v[k][q].w;
    } else if (MODE == 0 || MODE == 1 || MODE == 8) {
      if (base + INF > n_access) break;  // a partial group: the tail loop below
      // whole groups are unpredicated and every word read is used, so each
      // read keeps its own registers until all INF are issued
      if (MODE == 8) {
        uint32_t v[INF];
#pragma unroll
        for (int k = 0; k < INF; ++k) v[k] = __ldcg(reinterpret_cast<const unsigned int*>(buf + u[k] * 2));
#pragma unroll
        for (int k = 0; k < INF; ++k) acc ^= v[k];
      } else {
        constexpr int C = MODE == 1 ? 4 : 2;  // 16-byte chunks per unit
        uint4 v[INF][C];
#pragma unroll
        for (int k = 0; k < INF; ++k)
#pragma unroll
          for (int q = 0; q < C; q += 2) ld_cg_v8(buf + u[k] * C + q, v[k][q], v[k][q + 1]);
#pragma unroll
        for (int k = 0; k < INF; ++k)
#pragma unroll
          for (int q = 0; q < C; ++q) acc ^= v[k][q].x ^ v[k][q].y ^ v[k][q].z ^ v[k][q].w;
      }
    } else if (MODE == 2) {
#pragma unroll
      for (int k = 0; k < INF; ++k) {
        if (base + k < n_access) {
          const uint4 w = make_uint4((uint32_t)u[k], (uint32_t)k, 0u, 0u);
          st_v8(buf + u[k] * 2, w, w);
        }
      }
    } else if (MODE == 3) {
#pragma unroll
      for (int k = 0; k < INF; ++k)
        if (base + k < n_access) atomicAdd(reinterpret_cast<uint32_t*>(buf + u[k] * 2), 1u);
    } else if (MODE == 4) {
#pragma unroll
      for (int k = 0; k < INF; ++k)
        if (base + k < n_access)
          acc ^= atomicCAS(reinterpret_cast<uint32_t*>(buf + u[k] * 2), 0u, (uint32_t)u[k] | 1u);
    } else if (MODE == 5) {
#pragma unroll
      for (int k = 0; k < INF; ++k)
        if (base + k < n_access)
          acc ^= atomicCAS(reinterpret_cast<unsigned short*>(buf + u[k] * 2), (unsigned short)0,
                           (unsigned short)(u[k] | 1u));
    } else if (MODE == 6) {
#pragma unroll
      for (int k = 0; k < INF; ++k)
        if (base + k < n_access) st_relaxed(reinterpret_cast<uint32_t*>(buf + u[k] * 2), (uint32_t)k);
    } else {
#pragma unroll
      for (int k = 0; k < INF; ++k)
        if (base + k < n_access)
          st_relaxed_u16(reinterpret_cast<uint16_t*>(buf + u[k] * 2), (uint32_t)k);
    }
  }
  // reads of the last partial group (at most INF - 1 per thread), one at a time
  if (MODE == 0 || MODE == 1 || MODE == 8 || MODE == 9 || MODE == 10) {
    for (uint64_t a = base; a < n_access && a < base + INF; ++a) {
      const uint64_t u = probe_unit(seed, a, n_units);
      if (MODE == 9 || MODE == 10) {
        uint4 x, y;
        ld_cg_v8(buf + u * (2 * G) + 2 * part, x, y);
        acc ^= x.x ^ x.y ^ x.z ^ x.w ^ y.x ^ y.y ^ y.z ^ y.w;
      } else if (MODE == 8) {
        acc ^= __ldcg(reinterpret_cast<const unsigned int*>(buf + u * 2));
      } else {
        constexpr int C = MODE == 1 ? 4 : 2;
        for (int q = 0; q < C; q += 2) {
          uint4 x, y;
          ld_cg_v8(buf + u * C + q, x, y);
          acc ^= x.x ^ x.y ^ x.z ^ x.w ^ y.x ^ y.y ^ y.z ^ y.w;
        }
      }
    }
  }
  if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);  // keeps the loads alive
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (the copy engine of each SM, cp.async.bulk) of one
// 64-byte unit per access, issued by one thread:
// mode 11: global -> the thread's slot in shared memory, completion counted
//          in bytes on the thread's own mbarrier;
// mode 12: the thread's slot in shared memory -> global, completion by bulk
//          group.
// Every wait on an mbarrier is bounded: after kBulkWaitPolls polls the kernel
// records a timeout in err and waits once more, again bounded, for its copies.
// ---------------------------------------------------------------------------
constexpr uint32_t kBulkWaitPolls = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kBulkWaitPolls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src),
               "r"(bytes)
               : "memory");
}

template <int MODE, int INF>
__global__ void __launch_bounds__(256, 1) k_probe_bulk(uint4* buf, uint64_t n_units, uint64_t n_access,
                                                     uint64_t seed, unsigned long long* sink) {
  extern __shared__ __align__(128) unsigned char bulk_sm[];
  uint4* slot = reinterpret_cast<uint4*>(bulk_sm) + (size_t)threadIdx.x * INF * 4;  // INF x 64 B
  uint64_t* bars = reinterpret_cast<uint64_t*>(bulk_sm + (size_t)blockDim.x * INF * 64);
  const uint32_t bar = smem_u32(bars + threadIdx.x);
  unsigned long long* err = sink + 1;
  if (MODE == 11) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  } else {
    // the slots' contents are stored from shared memory: fill them once
    for (int k = 0; k < INF * 4; ++k) slot[k] = make_uint4(threadIdx.x, k, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
  uint32_t acc = 0, parity = 0;
  bool failed = false;
  for (uint64_t base = tid * INF; base < n_access && !failed; base += nthr * INF) {
    const int cnt = (int)(n_access - base < (uint64_t)INF ? n_access - base : (uint64_t)INF);
    uint64_t u[INF];
#pragma unroll
    for (int k = 0; k < INF; ++k) u[k] = probe_unit(seed, base + k, n_units);
    if (MODE == 11) {
      mbar_expect_tx(bar, 64u * (uint32_t)cnt);
#pragma unroll
      for (int k = 0; k < INF; ++k)
        if (k < cnt) bulk_g2s(smem_u32(slot + 4 * k), buf + u[k] * 4, 64u, bar);
      if (!mbar_wait_bounded(bar, parity)) {
        atomicExch(err, 1ull);
        failed = true;
        mbar_wait_bounded(bar, parity);  // let the copies in flight land before leaving
        break;
      }
      parity ^= 1u;
#pragma unroll
      for (int k = 0; k < INF; ++k)
        if (k < cnt)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc ^= slot[4 * k + q].x ^ slot[4 * k + q].w;
    } else {
#pragma unroll
      for (int k = 0; k < INF; ++k)
        if (k < cnt) bulk_s2g(buf + u[k] * 4, smem_u32(slot + 4 * k), 64u);
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
  }
  if (MODE == 12) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);  // keeps the copies' data alive
}

using ProbeKernel = void (*)(uint4*, uint64_t, uint64_t, uint64_t, unsigned long long*);

template <int MODE>
static ProbeKernel probe_bulk_kernel(int inf) {
  switch (inf) {
    case 1: return k_probe_bulk<MODE, 1>;
    case 2: return k_probe_bulk<MODE, 2>;
    case 4: return k_probe_bulk<MODE, 4>;
    case 8: return k_probe_bulk<MODE, 8>;
    default: return nullptr;
  }
}

// Accesses in flight per thread that each mode is compiled for: reads keep
// their data in registers until all INF have been issued (8 registers per
// 32-byte read), so 32-byte reads stop at 16 and 64-byte reads at 8 (128
// data registers), where no shape spills.  The kernels are compiled for
// blocks of at most 256 threads and may use up to 255 registers
// (__launch_bounds__(256, 1)): without that, the compiler keeps registers
// few by consuming each read before issuing the next, and the requests in
// flight are not the INF asked for.  Resident blocks per SM then follow from
// the registers a shape needs.
template <int MODE>
static ProbeKernel probe_kernel_inf(int inf) {
  constexpr int kMaxInf = MODE == 1 ? 8 : (MODE == 0 || MODE >= 9) ? 16 : 64;
  switch (inf) {
    case 1: return k_probe<MODE, 1>;
    case 2: return k_probe<MODE, 2>;
    case 4: return k_probe<MODE, 4>;
    case 8: return k_probe<MODE, 8>;
    case 16: return kMaxInf >= 16 ? k_probe<MODE, (kMaxInf >= 16 ? 16 : 1)> : nullptr;
    case 32: return kMaxInf >= 32 ? k_probe<MODE, (kMaxInf >= 32 ? 32 : 1)> : nullptr;
    case 64: return kMaxInf >= 64 ? k_probe<MODE, (kMaxInf >= 64 ? 64 : 1)> : nullptr;
    default: return nullptr;
  }
}

static ProbeKernel probe_kernel(int mode, int inf) {
  switch (mode) {
    case 0: return probe_kernel_inf<0>(inf);
    case 1: return probe_kernel_inf<1>(inf);
    case 2: return probe_kernel_inf<2>(inf);
    case 3: return probe_kernel_inf<3>(inf);
    case 4: return probe_kernel_inf<4>(inf);
    case 5: return probe_kernel_inf<5>(inf);
    case 6: return probe_kernel_inf<6>(inf);
    case 7: return probe_kernel_inf<7>(inf);
    case 8: return probe_kernel_inf<8>(inf);
    case 9: return probe_kernel_inf<9>(inf);
    case 10: return probe_kernel_inf<10>(inf);
    case 11: return probe_bulk_kernel<11>(inf);
    case 12: return probe_bulk_kernel<12>(inf);
    default: return nullptr;
  }
}

}  // namespace vss

using namespace vss;

extern "C" ht_status vss_probe_random_cfg(void* buf_dev, uint64_t bytes, uint64_t n_access, int mode,
                                          int inflight, int blocks_per_sm, int threads, void* stream,
                                          float* ms) {
  if (inflight == 0) inflight = 8;
  if (blocks_per_sm == 0) blocks_per_sm = 8;
  if (threads == 0) threads = 256;
  if (!buf_dev || !ms || mode < 0 || mode > 12 || (reinterpret_cast<uintptr_t>(buf_dev) & 255u))
    return HT_ERR_INVALID;
  if (blocks_per_sm < 1 || blocks_per_sm > 64 || threads < 32 || threads > 1024 || (threads & 31))
    return HT_ERR_INVALID;
  const ProbeKernel kern = probe_kernel(mode, inflight);
  if (!kern) return HT_ERR_INVALID;
  if (threads > 256) return HT_ERR_INVALID;  // the kernels' launch bound
  const bool bulk = mode == 11 || mode == 12;
  const uint64_t unit = mode == 1 || mode == 9 || bulk ? 64 : mode == 10 ? 128 : 32;
  const uint64_t n_units = bytes / unit;
  if (n_units < 1024 || n_access == 0) return HT_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  VSS_CUDA_TRY(cudaGetDevice(&dev));
  VSS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // the sink word lives in the first 8 bytes of the buffer's last unit (probe data is garbage)
  unsigned long long* sink =
      reinterpret_cast<unsigned long long*>(static_cast<char*>(buf_dev) + (n_units - 1) * unit);
  // bulk modes: each thread's INF 64-byte slots and its 8-byte mbarrier in shared memory
  const size_t smem = bulk ? (size_t)threads * inflight * 64 + (size_t)threads * 8 : 0;
  if (bulk) {
    VSS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // sink word and the bulk kernels' timeout word
    VSS_CUDA_TRY(cudaMemsetAsync(sink, 0, 16, s));
  }
  cudaEvent_t e0, e1;
  VSS_CUDA_TRY(cudaEventCreate(&e0));
  VSS_CUDA_TRY(cudaEventCreate(&e1));
  uint4* b = static_cast<uint4*>(buf_dev);
  const uint64_t n_use = n_units - 1;  // keep the sink unit out of the random range
  VSS_CUDA_TRY(cudaEventRecord(e0, s));
  kern<<<sms * blocks_per_sm, threads, smem, s>>>(b, n_use, n_access, 0x1234567ull, sink);
  VSS_CUDA_TRY(cudaGetLastError());
  VSS_CUDA_TRY(cudaEventRecord(e1, s));
  VSS_CUDA_TRY(cudaEventSynchronize(e1));
  VSS_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (bulk) {
    unsigned long long timed_out = 0;
    VSS_CUDA_TRY(cudaMemcpy(&timed_out, sink + 1, 8, cudaMemcpyDeviceToHost));
    if (timed_out) return HT_ERR_TIMEOUT;
  }
  return HT_OK;
}

extern "C" ht_status vss_probe_random(void* buf_dev, uint64_t bytes, uint64_t n_access, int mode,
                                      void* stream, float* ms) {
  if (mode < 0 || mode > 7) return HT_ERR_INVALID;
  return vss_probe_random_cfg(buf_dev, bytes, n_access, mode, 8, 8, 256, stream, ms);
}
