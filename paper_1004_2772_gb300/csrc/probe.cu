// Random-access HBM probe: the denominator of the random-sector roofline.
//
// The store's hot path moves data in 32-byte L2 sectors at random addresses
// (one bucket sector per probe, one or two sectors per data row).  This
// kernel measures how many such random accesses per second the GPU's memory
// system sustains, with the same access shapes: every thread issues
// kInflight independent accesses to sectors chosen by a counter-based hash
// (SplitMix64 output function of the access number) before it consumes any,
// so the number of requests in flight is limited only by residency.
#include "internal.h"

namespace vss {

constexpr int kInflight = 8;

__device__ __forceinline__ uint64_t probe_mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// mode 0: read one 32 B sector; 1: read 64 B (two adjacent sectors, 64 B
// aligned); 2: write one 32 B sector; 3: atomicAdd on one 32-bit word;
// 4 / 5: compare-and-swap (0 -> x) on a 32- / 16-bit word; 6 / 7: relaxed
// gpu-scope store of one 32- / 16-bit word (the claim and publish steps of an
// insert, for either bucket width).
template <int MODE>
__global__ void __launch_bounds__(256) k_probe(uint4* buf, uint64_t n_units, uint64_t n_access,
                                               uint64_t seed, unsigned long long* sink) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
  uint32_t acc = 0;
  for (uint64_t base = tid * kInflight; base < n_access; base += nthr * kInflight) {
    uint64_t u[kInflight];
#pragma unroll
    for (int k = 0; k < kInflight; ++k) u[k] = probe_mix(seed ^ (base + k)) % n_units;
    if (MODE == 0 || MODE == 1) {
      uint4 v[kInflight][MODE == 1 ? 4 : 2];
#pragma unroll
      for (int k = 0; k < kInflight; ++k) {
        const uint4* p = buf + u[k] * (MODE == 1 ? 4 : 2);
#pragma unroll
        for (int q = 0; q < (MODE == 1 ? 4 : 2); q += 2) ld_cg_v8(p + q, v[k][q], v[k][q + 1]);
      }
#pragma unroll
      for (int k = 0; k < kInflight; ++k)
#pragma unroll
        for (int q = 0; q < (MODE == 1 ? 4 : 2); ++q) acc ^= v[k][q].x ^ v[k][q].w;
    } else if (MODE == 2) {
#pragma unroll
      for (int k = 0; k < kInflight; ++k) {
        if (base + k < n_access) {
          const uint4 w = make_uint4((uint32_t)u[k], (uint32_t)k, 0u, 0u);
          st_v8(buf + u[k] * 2, w, w);
        }
      }
    } else if (MODE == 3) {
#pragma unroll
      for (int k = 0; k < kInflight; ++k)
        if (base + k < n_access) atomicAdd(reinterpret_cast<uint32_t*>(buf + u[k] * 2), 1u);
    } else if (MODE == 4) {
#pragma unroll
      for (int k = 0; k < kInflight; ++k)
        if (base + k < n_access)
          acc ^= atomicCAS(reinterpret_cast<uint32_t*>(buf + u[k] * 2), 0u, (uint32_t)u[k] | 1u);
    } else if (MODE == 5) {
#pragma unroll
      for (int k = 0; k < kInflight; ++k)
        if (base + k < n_access)
          acc ^= atomicCAS(reinterpret_cast<unsigned short*>(buf + u[k] * 2), (unsigned short)0,
                           (unsigned short)(u[k] | 1u));
    } else if (MODE == 6) {
#pragma unroll
      for (int k = 0; k < kInflight; ++k)
        if (base + k < n_access) st_relaxed(reinterpret_cast<uint32_t*>(buf + u[k] * 2), (uint32_t)k);
    } else {
#pragma unroll
      for (int k = 0; k < kInflight; ++k)
        if (base + k < n_access)
          st_relaxed_u16(reinterpret_cast<uint16_t*>(buf + u[k] * 2), (uint32_t)k);
    }
  }
  if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);  // keeps the loads alive
}

}  // namespace vss

using namespace vss;

extern "C" ht_status vss_probe_random(void* buf_dev, uint64_t bytes, uint64_t n_access, int mode,
                                      void* stream, float* ms) {
  if (!buf_dev || !ms || mode < 0 || mode > 7 || (reinterpret_cast<uintptr_t>(buf_dev) & 255u))
    return HT_ERR_INVALID;
  const uint64_t unit = (mode == 1) ? 64 : 32;
  const uint64_t n_units = bytes / unit;
  if (n_units < 1024 || n_access == 0) return HT_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  VSS_CUDA_TRY(cudaGetDevice(&dev));
  VSS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // the sink word lives in the first 8 bytes of the buffer's last unit (probe data is garbage)
  unsigned long long* sink =
      reinterpret_cast<unsigned long long*>(static_cast<char*>(buf_dev) + (n_units - 1) * unit);
  cudaEvent_t e0, e1;
  VSS_CUDA_TRY(cudaEventCreate(&e0));
  VSS_CUDA_TRY(cudaEventCreate(&e1));
  const int blocks = sms * 8;
  uint4* b = static_cast<uint4*>(buf_dev);
  const uint64_t n_use = n_units - 1;  // keep the sink unit out of the random range
  VSS_CUDA_TRY(cudaEventRecord(e0, s));
  switch (mode) {
    case 0: k_probe<0><<<blocks, 256, 0, s>>>(b, n_use, n_access, 0x1234567ull, sink); break;
    case 1: k_probe<1><<<blocks, 256, 0, s>>>(b, n_use, n_access, 0x1234567ull, sink); break;
    case 2: k_probe<2><<<blocks, 256, 0, s>>>(b, n_use, n_access, 0x1234567ull, sink); break;
    case 3: k_probe<3><<<blocks, 256, 0, s>>>(b, n_use, n_access, 0x1234567ull, sink); break;
    case 4: k_probe<4><<<blocks, 256, 0, s>>>(b, n_use, n_access, 0x1234567ull, sink); break;
    case 5: k_probe<5><<<blocks, 256, 0, s>>>(b, n_use, n_access, 0x1234567ull, sink); break;
    case 6: k_probe<6><<<blocks, 256, 0, s>>>(b, n_use, n_access, 0x1234567ull, sink); break;
    default: k_probe<7><<<blocks, 256, 0, s>>>(b, n_use, n_access, 0x1234567ull, sink); break;
  }
  VSS_CUDA_TRY(cudaGetLastError());
  VSS_CUDA_TRY(cudaEventRecord(e1, s));
  VSS_CUDA_TRY(cudaEventSynchronize(e1));
  VSS_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return HT_OK;
}
