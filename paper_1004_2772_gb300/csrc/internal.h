// Host-side internals shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

struct ht {
  vss::TableView view{};
  ht_params params{};
  int log2_nb = 0;
  int max_words = 0;
  int num_sms = 0;
  uint64_t bytes = 0;
  void* owned = nullptr;  // cudaMalloc'd block when created by ht_create
  unsigned long long* scan_scratch = nullptr;
};

namespace vss {
uint64_t table_bytes(int log2_nb, int max_words);
ht_status resolve_params(const ht_params* in, int log2_nb, ht_params* out);
ht_status table_init_at(ht_t* h, int log2_nb, int max_words, const ht_params* params, void* mem,
                        uint64_t mem_bytes);
ht_status table_set_words(ht_t* h, int words);
ht_status table_clear(ht_t* h, cudaStream_t s);
// Validate a model and pack it (with init) into the device blob format;
// blob header word [k]: see reach.cu.
ht_status pack_model(const reach_model* m, const int32_t* init, int max_words,
                     std::vector<int>& blob);
}  // namespace vss
