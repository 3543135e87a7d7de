// Batched and served reachability: shared definitions (see batch.cu).
#pragma once

#include "common.cuh"

namespace vss {

enum : uint32_t { PH_CLEAR = 0, PH_EXPAND = 1, PH_REHASH = 2, PH_DONE = 3 };

constexpr uint32_t kClearUnit = 8192;   // buckets zeroed per unit (256 per lane)
constexpr uint32_t kRehashUnit = 1024;  // old buckets re-inserted per unit (32 per lane)
constexpr uint32_t kCopyUnit = 1024;    // frontier rows copied per unit (32 per lane)
constexpr int kBatchNV = 8;             // state vectors up to 32 words
constexpr uint32_t kUnitsMax = (1u << 24) - 1;  // the claim word's unit and claimed fields
// Units of an EXPAND epoch stay at or below 2^23: warps that race past the end
// of an epoch add their claim to the claimed field anyway, and the headroom up
// to kUnitsMax keeps those additions from carrying into the units field.  A
// level of more frontier rows counts groups of rows as units (BatchModel::grp).
constexpr uint32_t kExpandUnitsMax = 1u << 23;

struct __align__(16) BatchModel {
  const int* blob;                  // packed model (global memory)
  unsigned long long* level_sizes;  // [max_levels]
  uint32_t W, nv, maxfan, spw_max;
  uint32_t max_levels;
  uint32_t log2_nb;                 // current table
  uint32_t* buckets;
  uint4* data;
  uint4* fr[2];                     // frontier rows of the current table's capacity
  uint32_t* nbuckets;               // table being built (CLEAR / REHASH), or the initial table
  uint4* ndata;
  uint4* nfr[2];
  uint32_t nlog2;
  uint32_t cur;                     // frontier holding the current level
  unsigned long long claim;         // see the file comment
  uint32_t done[2];
  uint32_t next_count[2];
  uint32_t grp[2];                  // EXPAND epochs: frontier rows per unit, by epoch parity
  uint32_t n_cur;                   // rows of fr[cur]
  uint32_t level;                   // index of the level in fr[cur]
  uint32_t n_rehash_b;              // REHASH units below this are bucket units
  uint32_t grows;
  unsigned long long states_bound;  // upper bound on the model's states (0 = unknown)
  DevCounters ctr;                  // err, stored, busy_waits, rehashes
  unsigned long long transitions, deadlocks, digest;
  uint32_t n_levels, finished;
};

struct BatchState {
  unsigned long long pool_used;
  uint32_t finished;
  uint32_t err;
  // serving
  unsigned long long seen_doorbell;  // host submissions already scanned
  uint32_t active;                   // slots holding a running job
  uint32_t scan_lock;
};

// Serving: host-mapped mailboxes.  The host writes a job's initial record into
// in[slot].rec, then bumps in[slot].seq and the doorbell; a device warp that
// has no work scans the slots whose seq changed, copies the record into the
// slot and activates it.  When the job ends, the device writes its result to
// out[slot] and then out[slot].seq = the job's seq.
struct __align__(64) ServeSlotIn {
  unsigned long long seq;
  unsigned long long pad[7];
  BatchModel rec;
};

struct __align__(64) ServeSlotOut {
  unsigned long long seq;
  unsigned long long states, transitions, deadlocks, digest, busy_waits, rehashes;
  uint32_t n_levels, status, grows, pad;
};

struct __align__(64) ServeMailbox {
  unsigned long long doorbell;  // submissions so far (host)
  uint32_t shutdown;            // host: exit once no job is active
  uint32_t pad;
};

struct BatchGlobal {
  BatchModel* models;
  BatchState* st;
  char* pool;
  unsigned long long pool_bytes;
  uint64_t seed;
  uint32_t n_models;
  uint32_t max_spin;
  uint32_t pad0;
  unsigned long long idle_ns;       // serving: leave after this long without work
  unsigned long long stuck_ns;      // no claimable work this long while jobs run: HT_ERR_TIMEOUT
  float grow_at;                    // grow when the coming level could pass this load factor
  float grow_to;                    // load factor the grown table is sized for
  // serving (null mb: a plain batch that ends when every model is done)
  ServeMailbox* mb;                 // host-mapped
  ServeSlotIn* in;                  // host-mapped [n_models]
  ServeSlotOut* out;                // host-mapped [n_models]
  unsigned long long* accepted;     // device [n_models]: seq of the job in each slot
};

// Bytes of one table generation: buckets, data rows, two frontiers.
__host__ __device__ __forceinline__ uint64_t generation_bytes(uint32_t log2, uint32_t nv) {
  const uint64_t nb = 1ull << log2;
  return ((nb * 4 + 255) & ~255ull) + 3 * ((nb * 16 * nv + 255) & ~255ull);
}

using BatchKernel = void (*)(BatchGlobal);
BatchKernel batch_kernel(int line_buckets);
size_t batch_smem_bytes(int threads);

}  // namespace vss
