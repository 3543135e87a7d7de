/* A plain C client of the library's C ABI (include/reach.h): no Python, no
 * torch.  It builds the tiny interleaving-style model given on the command
 * line (P processes, each a cycle 0 -> 1 -> ... -> n-1 -> 0 plus a self-loop),
 * runs reach() on a context the library allocates, and stores a key batch
 * twice through ht_find_or_put on device buffers it allocates itself, then
 * prints one line of results for the test to compare with the oracle:
 *   states transitions deadlocks levels digest seen_first seen_second
 * Usage: reach_client P n log2_buckets */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "reach.h"

#define CHECK(x)                                                              \
  do {                                                                        \
    ht_status s_ = (x);                                                       \
    if (s_ != HT_OK) {                                                        \
      fprintf(stderr, "%s -> %s\n", #x, ht_status_string(s_));                \
      return 1;                                                               \
    }                                                                         \
  } while (0)

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  const int P = atoi(argv[1]), n = atoi(argv[2]), log2 = atoi(argv[3]);
  if (P < 1 || P > 16 || n < 2 || n > 100) return 2;
  const int W = P, E = P * n * 2;
  int32_t* n_local = malloc(sizeof(int32_t) * P);
  int32_t* crit = malloc(sizeof(int32_t) * P);
  int32_t* begin = malloc(sizeof(int32_t) * (P * n + 1));
  int32_t* dst = malloc(sizeof(int32_t) * E);
  int32_t* none = malloc(sizeof(int32_t) * E);
  int32_t* zero = malloc(sizeof(int32_t) * E);
  int32_t* init = calloc(W, sizeof(int32_t));
  int e = 0;
  for (int p = 0; p < P; ++p) {
    n_local[p] = n;
    crit[p] = -1;
    for (int s = 0; s < n; ++s) {
      begin[p * n + s] = e;
      dst[e] = (s + 1) % n; none[e] = -1; zero[e] = 0; ++e;   /* the cycle */
      dst[e] = s;           none[e] = -1; zero[e] = 0; ++e;   /* a self-loop */
    }
  }
  begin[P * n] = e;
  reach_model m = {P, 0, W, E, n_local, crit, begin, dst, none, zero, none, zero};

  reach_ctx_t* ctx = NULL;
  CHECK(reach_ctx_create(log2, W, 1024, NULL, &ctx));
  uint64_t levels[1024];
  reach_result r;
  CHECK(reach(ctx, &m, init, REACH_PERSISTENT, NULL, levels, 1024, &r));
  CHECK(r.status);

  /* the table API on caller-owned device buffers: one key, stored twice */
  ht_t* h = NULL;
  CHECK(ht_create(10, W, NULL, &h));
  int32_t *keys_dev = NULL;
  uint8_t* seen_dev = NULL;
  uint32_t* idx_dev = NULL;
  if (cudaMalloc((void**)&keys_dev, sizeof(int32_t) * W) != cudaSuccess) return 1;
  if (cudaMalloc((void**)&seen_dev, 2) != cudaSuccess) return 1;
  if (cudaMalloc((void**)&idx_dev, 8) != cudaSuccess) return 1;
  if (cudaMemcpy(keys_dev, init, sizeof(int32_t) * W, cudaMemcpyHostToDevice) != cudaSuccess) return 1;
  CHECK(ht_find_or_put(h, keys_dev, 1, seen_dev, idx_dev, NULL));
  CHECK(ht_find_or_put(h, keys_dev, 1, seen_dev + 1, idx_dev + 1, NULL));
  CHECK(ht_sync(h, NULL));
  uint8_t seen[2];
  uint32_t idx[2];
  if (cudaMemcpy(seen, seen_dev, 2, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  if (cudaMemcpy(idx, idx_dev, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  if (idx[0] != idx[1]) return 1;

  printf("%llu %llu %llu %u %llu %u %u\n", (unsigned long long)r.states,
         (unsigned long long)r.transitions, (unsigned long long)r.deadlocks, r.n_levels,
         (unsigned long long)r.digest, seen[0], seen[1]);
  cudaFree(keys_dev);
  cudaFree(seen_dev);
  cudaFree(idx_dev);
  CHECK(ht_destroy(h));
  CHECK(reach_ctx_destroy(ctx));
  return 0;
}
