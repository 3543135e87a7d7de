// Host-side internals shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

struct ht {
  vss::TableView view{};
  ht_params params{};
  uint64_t nb = 0;  // buckets: 2^log2 or lines * line_buckets
  int max_words = 0;
  int num_sms = 0;
  uint64_t bytes = 0;
  void* owned = nullptr;  // cudaMalloc'd block when created by ht_create
  unsigned long long* scan_scratch = nullptr;
};

namespace vss {
// Table sizes are bucket counts nb: a power of two, or any multiple of the
// line length whose line count fits 31 bits (constant division, Section 3.1).
constexpr uint64_t kMaxBuckets = 1ull << 31;
uint64_t table_bytes(uint64_t nb, int max_words);
ht_status resolve_params(const ht_params* in, uint64_t nb, ht_params* out);
ht_status table_init_at(ht_t* h, uint64_t nb, int max_words, const ht_params* params, void* mem,
                        uint64_t mem_bytes);
// Largest nb <= max_nb that is line_buckets times a prime (or times a power
// of two when max_nb is one); 0 if none.
uint64_t prime_line_buckets(uint64_t max_nb, uint32_t line_buckets);
ht_status table_set_words(ht_t* h, int words);
ht_status table_clear(ht_t* h, cudaStream_t s);
// A single-model run on device areas the caller carved (the server's path for
// a job that arrives at an idle GPU): table view (power of two), packed model,
// two frontiers of cap rows, run totals (solo_totals_bytes()), per-level sizes
// and start times of max_levels entries.  solo_launch clears the table and the
// totals and launches the persistent kernel on s; solo_result reads the result
// once s has finished it (synchronous copies).
struct SoloRun {
  TableView tv;
  const int* blob_dev;
  int smem_words;
  uint4* fr0;
  uint4* fr1;
  uint32_t cap;
  void* tot_dev;
  unsigned long long* level_sizes_dev;
  unsigned long long* level_ns_dev;
  uint32_t max_levels;
};
uint64_t solo_totals_bytes();
ht_status solo_launch(const SoloRun& r, int line_buckets, int threads, cudaStream_t s);
ht_status solo_result(const SoloRun& r, reach_result* out);
// Validate a model and pack it (with init) into the device blob format;
// blob header word [k]: see reach.cu.
ht_status pack_model(const reach_model* m, const int32_t* init, int max_words,
                     std::vector<int>& blob);
}  // namespace vss
