/*
 * reach.h -- C ABI of the GB300 visited-state store and its reachability driver.
 *
 * The store is the lockless shared hash table of Laarman, van de Pol and Weber,
 * "Boosting Multi-Core Reachability Performance with Shared Hash Tables"
 * (Section 3): a single operation, find-or-put, over fixed-length int32 state
 * vectors (Section 3.1), an open-addressing bucket array of memoised hashes with
 * a write-busy bit (Section 3.2), states kept in a separate data array indexed
 * like the buckets, walking-the-line probing followed by double hashing
 * (Alg. "find-or-put", Alg. "Walking the (cache) line"), and CAS claiming of
 * empty buckets.  The reachability driver is a level-synchronous breadth-first
 * form of Alg. "Reachability analysis" (Section 2).
 *
 * Conventions for every call:
 *   - Pointers named *_dev are device pointers (cudaMalloc'd or from a tensor
 *     allocator); pointers named *_host are host pointers.  The library never
 *     keeps a caller pointer after the call returns, except the memory block
 *     handed to *_create_at, which the caller keeps alive until *_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Device work is enqueued on it and is asynchronous unless stated.
 *   - The return value is an ht_status.  Argument errors return at once with
 *     nothing enqueued.  Errors found on the device (table full, a write-busy
 *     wait or a barrier that ran out of its iteration limit) are latched in a
 *     device word and returned by ht_sync / the reach_* result calls.  No
 *     device loop is unbounded: every wait has an iteration limit and reports
 *     HT_ERR_TIMEOUT instead of hanging.
 *   - A handle may be used from one host thread at a time.
 */
#ifndef PAPER_1004_2772_GB300_REACH_H
#define PAPER_1004_2772_GB300_REACH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ht_status;
enum {
  HT_OK = 0,
  HT_ERR_INVALID = 1, /* bad argument; nothing was enqueued */
  HT_ERR_OOM = 2,     /* device allocation failed, or the caller's block is too small */
  HT_ERR_FULL = 3,    /* a key found no empty bucket within max_rehash lines */
  HT_ERR_TIMEOUT = 4, /* a bounded wait (write-busy bucket, level barrier) ran out */
  HT_ERR_CUDA = 5,    /* a CUDA runtime call failed */
  HT_ERR_LEVELS = 6,  /* more BFS levels than the caller's level_sizes capacity */
  HT_ERR_TOO_BIG = 7  /* the request needs more than reach_noalloc's fixed scratch array */
};

/* Bucket word layout (Section 3.2, "hash memoization" and the write bit):
 *   0            empty
 *   bit 31       0 = write (data being written), 1 = done (data complete)
 *   bits 0..30   memo = bits 33..63 of the 64-bit state hash, 0 mapped to 1.
 * The bucket index of a key is the low log2_buckets bits of the same hash
 * (Section 3.2, 2^n-sized table).  A used bucket never returns to empty and
 * never changes its memo (Fig. "State diagram of buckets"). */
#define HT_BUCKET_DONE 0x80000000u
#define HT_BUCKET_MEMO 0x7FFFFFFFu

/* Narrow bucket layout, selected by ht_params.bucket_bits = 16 (Section 1 names
 * the bucket size among the parameters left to the implementation):
 *   0            empty
 *   bit 15       write / done, as above
 *   bits 0..14   memo = bits 49..63 of the state hash, 0 mapped to 1.
 * Half the bytes per bucket, so twice as many buckets share one 32-byte sector
 * and the bucket array is half as large; a shorter memo lets more foreign keys
 * through to a data compare (about 1 in 2^15 per memo-bucket visited). */
#define HT_BUCKET16_DONE 0x8000u
#define HT_BUCKET16_MEMO 0x7FFFu

/* Tunable layout and safety limits; 0 in any field selects the default. */
typedef struct {
  uint32_t line_buckets;  /* buckets walked per line before rehashing.  32-bit buckets:
                             8, 16 or 32 (32, 64 or 128 bytes), default 32 (a
                             128-byte line, read one 32-byte sector at a time); 16-bit
                             buckets: 16 or 32 (32 or 64 bytes), default 16 */
  uint32_t max_rehash;    /* lines probed before HT_ERR_FULL; default min(lines, 4096) */
  uint32_t max_spin;      /* polls of a write-busy bucket before HT_ERR_TIMEOUT; default 2^18 */
  uint32_t block_threads; /* threads per block of the batch and expansion kernels; default 256 */
  uint32_t dedup;         /* 1 = merge equal keys inside a warp before probing (batch API) */
  uint32_t bucket_bits;   /* bucket word width: 32 (default) or 16 (the layouts above).
                             ht_scan, ht_arrays and reach_* follow it; the batch
                             and serving entry points accept only 32 */
  uint32_t group_lanes;   /* lanes per key in ht_find_or_put and ht_find_or_put_stream:
                             1 (default) = one thread walks the line a 32-byte sector
                             at a time; 2, 4 or 8 = a sub-warp group loads the whole
                             line of 4*group_lanes 32-bit buckets (32, 64 or 128
                             bytes) at once, combines the lanes' bucket masks with
                             shuffles and writes / compares the row in 16-byte chunks
                             (line_buckets must be 0 or 4*group_lanes, dedup 0).  In
                             reach_* (not with REACH_TRACE) the G lanes of a group
                             walk one successor's line together; the batch and
                             serving entry points accept only 1 */
  uint32_t rehash;        /* line sequence after the first line (Alg. "find-or-put": rehash with
                             the next hash function): 0 (default) = double hashing, the
                             line advances by an odd step taken from the memo (a step in
                             [1, lines - 1] for tables of any size); 1 = the next line
                             (linear probing over lines).  The batch and serving entry
                             points accept only 0 */
  uint64_t hash_seed;     /* seed of the table hash; default a fixed constant */
} ht_params;

/* ------------------------------------------------------------------------ */
/* The table: find-or-put over a caller's batch of keys.                      */
/* ------------------------------------------------------------------------ */

typedef struct ht ht_t;

/* Device bytes needed by a table of 2^log2_buckets buckets for state vectors of
 * state_words int32 words: 4 bytes per bucket (enough for either bucket width),
 * 16*ceil(state_words/4) bytes of data per bucket (rows padded to 16 bytes),
 * plus a small header. */
ht_status ht_bytes(int log2_buckets, int state_words, uint64_t* bytes);

/* Create an empty table (Section 3.1: no allocation during operation; the
 * whole table is claimed up front).  ht_create allocates with cudaMalloc;
 * ht_create_at carves the table out of the caller's device block `mem_dev` of
 * `mem_bytes` bytes (256-byte aligned, at least ht_bytes()).  log2_buckets in
 * [4, 31], state_words in [1, 32].  `params` may be NULL.  Synchronous. */
ht_status ht_create(int log2_buckets, int state_words, const ht_params* params, ht_t** out);
ht_status ht_create_at(int log2_buckets, int state_words, const ht_params* params, void* mem_dev,
                       uint64_t mem_bytes, ht_t** out);
ht_status ht_destroy(ht_t* h);

/* Tables of any size (Section 3.1: tables that fill the whole memory need sizes
 * that are not powers of two; division by the invariant size makes that
 * cheap).  n_buckets = lines * line_buckets, 16 <= n_buckets <= 2^31, any
 * number of lines.  The line of a key is (h / line_buckets) mod lines, computed
 * with one multiply-high by a constant prepared at creation (Granlund and
 * Montgomery 1994, unsigned case); the offset inside the line is h mod
 * line_buckets, as for power-of-two tables.  Rehash steps are 1 + a fraction
 * of (lines - 1) taken from the memo: with a prime number of lines every line
 * is reachable, with a composite one a key may see only the lines of one
 * residue class before HT_ERR_FULL.  A power-of-two n_buckets behaves exactly
 * like the log2 entry points.  Same ownership and errors as the log2 forms. */
ht_status ht_bytes_n(uint64_t n_buckets, int state_words, uint64_t* bytes);
ht_status ht_create_n_at(uint64_t n_buckets, int state_words, const ht_params* params, void* mem_dev,
                         uint64_t mem_bytes, ht_t** out);
/* The largest table whose block fits in `bytes` and whose line count is prime
 * (or a power of two), for params' line length.  HT_ERR_OOM if none fits.
 * Host only; no device call. */
ht_status ht_buckets_for_bytes(uint64_t bytes, int state_words, const ht_params* params,
                               uint64_t* n_buckets);
/* The division above, on the host, for checking: q[i] = n[i] / d, r[i] = n[i]
 * mod d for count 64-bit values, 1 <= d < 2^32.  Host only. */
ht_status vss_line_divide(uint32_t d, const uint64_t* n_host, uint64_t count, uint64_t* q_host,
                          uint32_t* r_host);

/* Empty the table and zero its counters and error word (enqueued on stream). */
ht_status ht_clear(ht_t* h, void* stream);

/* find-or-put of n keys (Alg. "find-or-put"), one thread per key.
 *   keys_dev  n rows of state_words int32, row-major, contiguous
 *   seen_dev  out, n bytes: 0 = the key was not in the table and this call
 *             stored it, 1 = the key was already stored, 2 = error (see ht_sync)
 *   idx_dev   out, n uint32: bucket index of the key; the key's vector is row
 *             idx of the data array.  May be NULL.
 * Among equal keys inside one batch exactly one gets seen = 0 when the key was
 * new; all get the same idx.  Which of them is unspecified.  Enqueued on stream. */
ht_status ht_find_or_put(ht_t* h, const int32_t* keys_dev, uint64_t n, uint8_t* seen_dev,
                         uint32_t* idx_dev, void* stream);

/* Wait for the stream and return the latched device error (HT_OK if none). */
ht_status ht_sync(ht_t* h, void* stream);

typedef struct {
  uint64_t stored;      /* keys inserted since the last clear */
  uint64_t busy_waits;  /* probes that found a memo-equal bucket still in the write state */
  uint64_t rehashes;    /* lines probed after the first, summed over keys */
  uint64_t capacity;    /* number of buckets */
  uint32_t error;       /* latched device error */
  uint32_t state_words;
} ht_stats_t;

/* Synchronises `stream`, then reads the counters. */
ht_status ht_stats(ht_t* h, void* stream, ht_stats_t* out);

/* Full scan of the bucket array: number of done buckets, number of buckets
 * still in the write state (0 after every completed call), and the sum over
 * done buckets of the fingerprint of their data row:
 *   x = state_words; for each word w: x = sm(x ^ (uint32)w); fingerprint = x,
 * sm(z) being one SplitMix64 output step (Steele, Lea, Flood 2014).
 * Synchronous (waits on stream). */
ht_status ht_scan(ht_t* h, void* stream, uint64_t* done, uint64_t* writing, uint64_t* digest);

/* Copy rows idx_dev[0..n) of the data array to out_dev (n x state_words int32). */
ht_status ht_gather(ht_t* h, const uint32_t* idx_dev, uint64_t n, int32_t* out_dev, void* stream);

/* Device pointers to the bucket array (one word of bucket_bits bits, uint32 or
 * uint16, per bucket: 2^log2_buckets or n_buckets of them) and data array
 * (rows of 4*ceil(state_words/4) int32), for inspection. */
ht_status ht_arrays(ht_t* h, uint32_t** buckets_dev, int32_t** data_dev, uint32_t* row_words);

/* ------------------------------------------------------------------------ */
/* Hash-table benchmark streams (Section 4.3 measures find-or-put throughput  */
/* on synthetic keys; these generate such keys on the device).               */
/* ------------------------------------------------------------------------ */

/* A fill with n_ids distinct keys is a stream of 2*n_ids calls: call 2i is key
 * i; call 2i+1 repeats a key drawn from r = mix(c ^ mix(seed)) -- uniformly
 * from ids [0, i] as floor(r * (i + 1) / 2^64) when zipf_table_dev is NULL,
 * else from ranks 1..n_ids of a Zipf quantile table (65537 uint32 entries: a
 * cell from the top 16 bits of r, a rank uniform inside the cell).  Key i:
 * word 0 = MurmurHash3 fmix32(i); words 2q-1 and 2q (q >= 1) = the low and
 * high 32 bits of mix((seed << 36) + (i << 4) + q), mix = one SplitMix64
 * output step.
 * vss_gen_keys writes calls [call_begin, call_begin + n_calls) as rows of
 * state_words int32 to keys_dev.  Enqueued on stream. */
ht_status vss_gen_keys(uint64_t seed, uint64_t n_ids, uint64_t call_begin, uint64_t n_calls,
                       const uint32_t* zipf_table_dev, int state_words, int32_t* keys_dev,
                       void* stream);

/* find-or-put of calls [call_begin, call_begin + n_calls) of that stream, the
 * keys generated in registers (no key traffic).  result_dev (2 uint64, the
 * caller zeroes them) accumulates the number of keys this call stored and the
 * sum of their fingerprints (the digest of ht_scan).  Needs state_words with
 * ceil(state_words/4) in {1, 2, 4, 8}.  Enqueued on stream. */
ht_status ht_find_or_put_stream(ht_t* h, uint64_t seed, uint64_t n_ids, uint64_t call_begin,
                                uint64_t n_calls, const uint32_t* zipf_table_dev,
                                uint64_t* result_dev, void* stream);

/* ------------------------------------------------------------------------ */
/* Reachability (Alg. "Reachability analysis", level-synchronous BFS).        */
/* ------------------------------------------------------------------------ */

/* A model: P processes with local automata, S shared int32 variables, state
 * vectors of W int32 words: v[0..P) local states, v[P..P+S) shared variables,
 * v[P+S..W) padding kept at 0.  All pointers are HOST pointers.
 * Edges of process p leaving local state s are edge_begin[b] .. edge_begin[b+1]
 * with b = n_local[0] + ... + n_local[p-1] + s.  Edge e is enabled in v when
 *   guard_var[e] < 0 or v[P + guard_var[e]] == guard_val[e], and
 *   not (crit[p] >= 0 and edge_dst[e] == crit[p] and another process q has
 *        crit[q] >= 0 and v[q] == crit[q]);
 * firing it sets v[p] = edge_dst[e] and, when upd_var[e] >= 0,
 * v[P + upd_var[e]] = upd_val[e].  Every enabled edge is one transition.
 * Limits (HT_ERR_INVALID otherwise): the sum over processes of the largest
 * out-degree of a local state is at most 1920 (the successors of one state
 * must fit one warp's round), and the packed model (about P + sum(n_local)
 * + 5E words) fits 128 KiB. */
typedef struct {
  int32_t n_procs;           /* P, >= 1 */
  int32_t n_shared;          /* S, >= 0 */
  int32_t state_words;       /* W, P + S <= W <= 32 */
  int32_t n_edges;           /* E */
  const int32_t* n_local;    /* [P], each in [1, 65535] */
  const int32_t* crit;       /* [P], critical local state or -1 */
  const int32_t* edge_begin; /* [sum(n_local) + 1], non-decreasing, edge_begin[0] = 0 */
  const int32_t* edge_dst;   /* [E] */
  const int32_t* guard_var;  /* [E], -1 or in [0, S) */
  const int32_t* guard_val;  /* [E] */
  const int32_t* upd_var;    /* [E], -1 or in [0, S) */
  const int32_t* upd_val;    /* [E] */
} reach_model;

typedef struct {
  uint64_t states;      /* |V| */
  uint64_t transitions; /* enabled edges summed over V = find-or-put calls */
  uint64_t deadlocks;   /* states with no enabled edge */
  uint64_t digest;      /* sum over V of the fingerprint described at ht_scan */
  uint64_t busy_waits;  /* write-busy "lock" hits (Section 4.3) */
  uint64_t rehashes;
  uint32_t n_levels;    /* BFS levels including level 0 = {init} */
  ht_status status;
} reach_result;

enum {
  REACH_PERSISTENT = 0, /* one cooperative launch runs every level (device-side level barrier) */
  REACH_PER_LEVEL = 1,  /* one launch per level; the host reads each level's size */
  REACH_GRAPH = 2,      /* CUDA graphs of 32 level launches each (captured once per loaded
                           model); the host looks at the search only between graphs */
  REACH_TRACE = 4       /* flag, with REACH_PERSISTENT and the default line length: record
                           predecessors so that reach_ctx_deadlock_trace can print a trace */
};

typedef struct reach_ctx reach_ctx_t;

/* Device bytes of a context: a table of 2^log2_buckets buckets for states of up
 * to max_state_words words, two frontier arrays of 2^log2_buckets state rows
 * (16*ceil(max_state_words/4) bytes each), a model area, counters,
 * 2*max_levels 64-bit level records and three 2^log2_buckets uint32 arrays
 * for tracing. */
ht_status reach_ctx_bytes(int log2_buckets, int max_state_words, uint32_t max_levels,
                          uint64_t* bytes);
ht_status reach_ctx_create(int log2_buckets, int max_state_words, uint32_t max_levels,
                           const ht_params* params, reach_ctx_t** out);
ht_status reach_ctx_create_at(int log2_buckets, int max_state_words, uint32_t max_levels,
                              const ht_params* params, void* mem_dev, uint64_t mem_bytes,
                              reach_ctx_t** out);
ht_status reach_ctx_destroy(reach_ctx_t* c);
/* Contexts of any table size (see ht_bytes_n): the frontiers and trace arrays
 * have n_buckets entries.  reach_ctx_buckets_for_bytes: the largest context
 * with a prime line count whose block fits in `bytes` (host only). */
ht_status reach_ctx_bytes_n(uint64_t n_buckets, int max_state_words, uint32_t max_levels,
                            uint64_t* bytes);
ht_status reach_ctx_create_n_at(uint64_t n_buckets, int max_state_words, uint32_t max_levels,
                                const ht_params* params, void* mem_dev, uint64_t mem_bytes,
                                reach_ctx_t** out);
ht_status reach_ctx_buckets_for_bytes(uint64_t bytes, int max_state_words, uint32_t max_levels,
                                      const ht_params* params, uint64_t* n_buckets);

/* Validate the model and init (host) and upload both (enqueued on stream). */
ht_status reach_ctx_load(reach_ctx_t* c, const reach_model* m, const int32_t* init_host,
                         void* stream);

/* Clear the table and explore from the loaded init.  REACH_PERSISTENT enqueues
 * everything and returns without waiting; REACH_PER_LEVEL waits on the stream
 * once per level; REACH_GRAPH waits once per 32 levels.  Results stay on the
 * device until reach_ctx_result. */
ht_status reach_ctx_run(reach_ctx_t* c, int mode, void* stream);

/* Wait for the stream and copy the result (and up to max_levels level sizes,
 * level_sizes_host may be NULL) to the host.  Returns out->status. */
ht_status reach_ctx_result(reach_ctx_t* c, void* stream, uint64_t* level_sizes_host,
                           uint32_t max_levels, reach_result* out);

/* Device time of the last reach_ctx_run, from CUDA events recorded on its
 * stream: kernel_ms spans the expansion kernel launch (persistent: the one
 * cooperative launch; per-level: from the seed launch to the end of the last
 * level launch, host gaps included), launches = kernels it launched.  Waits on
 * the events. */
ht_status reach_ctx_last_timing(reach_ctx_t* c, float* kernel_ms, uint32_t* launches);

/* The same device time for each of the most recent runs (at most 64 are
 * kept): ms_host[0..*got) = min(n, runs kept) durations, oldest first, so a
 * caller can time every launch of a loop without synchronising inside it.
 * Waits on the last run's end event. */
ht_status reach_ctx_run_times(reach_ctx_t* c, uint32_t n, float* ms_host, uint32_t* got);

/* Level start times of the last REACH_PERSISTENT run: level_ns_host[k] is the
 * device %globaltimer (ns) when level k began (k = 0: after init was
 * inserted).  Synchronises `stream`; *n_levels = entries written. */
ht_status reach_ctx_level_ns(reach_ctx_t* c, void* stream, uint64_t* level_ns_host,
                             uint32_t max_levels, uint32_t* n_levels);

/* Counterexample of the last REACH_TRACE run (Alg. "Reachability analysis":
 * a state without successors is a deadlock, "print trace"): the path from
 * init to a deadlock of the lowest BFS level that has one, as *len state rows
 * of state_words int32 (init first).  Which deadlock of that level, and which
 * of several shortest paths, is the winner of the insertion races; every
 * consecutive pair is a transition and the path has *level + 1 states.
 * *len = 0 when the model has no deadlock.  Synchronous. */
ht_status reach_ctx_deadlock_trace(reach_ctx_t* c, void* stream, int32_t* states_host,
                                   uint32_t max_len, uint32_t* len, uint32_t* level);

/* The context's table (owned by the context), for ht_scan / ht_gather. */
ht_status reach_ctx_table(reach_ctx_t* c, ht_t** table);

/* One-shot reach(model, init): load + run + result on `ctx`. */
ht_status reach(reach_ctx_t* c, const reach_model* m, const int32_t* init_host, int mode,
                void* stream, uint64_t* level_sizes_host, uint32_t max_levels, reach_result* out);

/* ------------------------------------------------------------------------ */
/* Batched reachability: many independent models in one persistent launch.   */
/* ------------------------------------------------------------------------ */

/* Each model runs its own level-synchronous BFS (Alg. "Reachability
 * analysis") on its own table, all inside one persistent kernel with no
 * grid-wide barrier: warps claim work units (frontier rows, table-clear and
 * re-insert chunks) from per-model claim words, and the warp that finishes a
 * model's level advances that model alone.  Tables start at log2_initial[i]
 * buckets (NULL or 0: an estimate -- twice the product of the local state
 * counts when the model has no shared variables, capped at 2^16) and grow at
 * a level boundary when the coming level could push them past 90% load: a new
 * table from a device pool, the old one re-inserted.  A model with a state
 * bound (the product above) grows once, to a table that holds the bound at
 * 50% load, when that table fits the pool; otherwise (no bound, or no room)
 * the new table holds the coming level's estimate at 50% load.  Unlike the
 * paper's fixed table (Section 3.1), this lets one launch serve models whose
 * sizes are only estimated.
 * Results are bit-identical to reach() on each model alone.
 *
 * pool_bytes must cover every model's initial table generation plus all
 * growth (a generation of 2^n buckets takes 4*2^n + 3*16*ceil(W/4)*2^n bytes:
 * buckets, data rows, two frontiers); a model whose growth does not fit ends
 * with HT_ERR_OOM, the others are unaffected. */
typedef struct reach_batch reach_batch_t;

ht_status reach_batch_bytes(const reach_model* models, const int32_t* const* inits_host,
                            int n_models, uint32_t max_levels, uint64_t pool_bytes,
                            uint64_t* bytes);
/* models/inits are host arrays of n_models entries; the block `mem_dev`
 * (256-byte aligned, >= reach_batch_bytes) is owned by the caller.
 * Synchronous (uploads the models). */
ht_status reach_batch_create_at(const reach_model* models, const int32_t* const* inits_host,
                                int n_models, const int32_t* log2_initial, uint32_t max_levels,
                                uint64_t pool_bytes, const ht_params* params, void* mem_dev,
                                uint64_t mem_bytes, reach_batch_t** out);
ht_status reach_batch_create(const reach_model* models, const int32_t* const* inits_host,
                             int n_models, const int32_t* log2_initial, uint32_t max_levels,
                             uint64_t pool_bytes, const ht_params* params, reach_batch_t** out);
ht_status reach_batch_destroy(reach_batch_t* b);

/* Run the whole batch (reset + one persistent launch), asynchronously on
 * `stream`.  use_graph = 1: the sequence is captured once into a CUDA graph and
 * replayed by later calls (one graph launch per run). */
ht_status reach_batch_run(reach_batch_t* b, int use_graph, void* stream);

/* Wait for `stream` and copy per-model results to outs[n_models] (status per
 * model), level sizes to level_sizes_host[n_models * max_levels] (may be
 * NULL) and growth counts to grows[n_models] (may be NULL).  Returns the first
 * error of any model, HT_OK when all succeeded. */
ht_status reach_batch_results(reach_batch_t* b, void* stream, reach_result* outs,
                              uint64_t* level_sizes_host, uint32_t* grows);

/* Device time of the last reach_batch_run (CUDA events around it). */
ht_status reach_batch_last_timing(reach_batch_t* b, float* ms);

/* ------------------------------------------------------------------------ */
/* Served reachability: a request loop with continuous batching.              */
/* ------------------------------------------------------------------------ */

/* One persistent kernel (the batched driver in serving mode) runs while jobs
 * arrive.  serve_submit queues a job; a job is admitted when one of n_slots
 * slots is free and its memory fits in the arena (the HBM budget: table
 * generation of 2^log2 buckets plus the packed model, see reach_batch); the
 * host then posts it through the slot's host-mapped mailbox and a device warp
 * with no work takes it, so it overlaps with the jobs already running.  A
 * finished job is returned by serve_poll and its memory freed, which may admit
 * queued jobs.  Each job's result equals reach() on it alone.  The kernel
 * leaves after ~2 ms without work (all device waits are bounded) and is
 * relaunched by the next submit or poll.  While fewer than 8 jobs wait and
 * the kernel is gone, jobs run one at a time on the single-model persistent
 * kernel of reach() instead, on the same stream (jobs submitted meanwhile
 * queue); 8 or more waiting jobs go to the many-job kernel together.
 * serve_status counts both kinds of launch.  One host thread at a time. */
typedef struct serve serve_t;

typedef struct {
  uint64_t job_id;
  reach_result result;   /* status HT_ERR_OOM: the job can never fit the arena */
  uint32_t grows;
  uint32_t pad;
  double submit_s;       /* host steady-clock seconds: submitted, admitted, seen done */
  double admit_s;
  double done_s;
} serve_done_t;

ht_status serve_bytes(uint64_t budget_bytes, uint32_t n_slots, uint32_t max_levels,
                      uint64_t* bytes);
/* mem_dev (256-byte aligned) of at least serve_bytes(); the arena is what
 * remains after the slot records.  Synchronous. */
ht_status serve_open_at(void* mem_dev, uint64_t mem_bytes, uint32_t n_slots, uint32_t max_levels,
                        const ht_params* params, serve_t** out);
ht_status serve_open(uint64_t budget_bytes, uint32_t n_slots, uint32_t max_levels,
                     const ht_params* params, serve_t** out);
/* Queue a job (host model and init are copied; the call returns at once).
 * log2_buckets 0: sized for 75% load of the product of the local state counts
 * (models without shared variables only). */
ht_status serve_submit(serve_t* s, const reach_model* m, const int32_t* init_host, int log2_buckets,
                       uint64_t* job_id);
/* Collect up to max_done finished jobs (and their level sizes, max_levels per
 * job, into level_sizes_host when not NULL); admits queued jobs. */
ht_status serve_poll(serve_t* s, serve_done_t* done, uint32_t max_done, uint32_t* n_done,
                     uint64_t* level_sizes_host);
ht_status serve_status(serve_t* s, uint32_t* queued, uint32_t* running, uint64_t* free_bytes,
                       uint64_t* kernel_launches);
/* Stop accepting, wait for running jobs, release everything. */
ht_status serve_close(serve_t* s);

/* ------------------------------------------------------------------------ */
/* Owner-partitioned reachability (static state-space partitioning).         */
/* ------------------------------------------------------------------------ */

/* The architecture that Sec. 4.1 describes for Spin and DiVinE 2, against
 * which the paper sets its shared table: a breadth-first exploration in which
 * a hash function assigns every successor to one worker, which checks it
 * against its own state storage.  Here n_parts owner partitions on one GPU:
 * owner(v) = the top log2(n_parts) bits of the state hash (so the memo of a
 * partition's buckets carries log2(n_parts) fewer free bits).  Partition o has
 * its own table of 2^log2_buckets_part buckets (the store of Sec. 3:
 * find-or-put, 32-bit buckets, 128-byte lines) and its own frontier.  Each BFS
 * level (Alg. "Reachability analysis") runs, over chunks of the frontier:
 *   expand   all partitions' states with the shared-table drivers' successor
 *            generator; successors and their hashes go to an outbox, counted
 *            per (source partition, owner);
 *   plan     the counts become receive offsets: owner o's inbox holds the
 *            segments (0, o), (1, o), ... (n_parts-1, o) in order -- the
 *            layout an all-to-all exchange between n_parts ranks delivers;
 *   scatter  outbox rows to their inbox segments;
 *   insert   each owner's find-or-put over its inbox, new states to its next
 *            frontier.
 * The results (states, transitions, deadlocks, level sizes, digest) equal
 * reach() on one shared table.  exchange_rows bounds the rows of one chunk
 * (outbox and inbox each hold that many; at least 960, at most 2^31).
 * n_parts is 1, 2, 4, 8 or 16; log2_buckets_part in [10, 31];
 * max_state_words in [1, 32].  Same ownership and error conventions as
 * reach_ctx_*; params may be NULL and, when given, must keep 32-bit buckets,
 * 128-byte lines and one lane per key. */
typedef struct part_reach part_reach_t;

ht_status part_reach_bytes(int n_parts, int log2_buckets_part, int max_state_words, uint64_t exchange_rows,
                           uint64_t* bytes);
/* mem_dev: 256-byte aligned, at least part_reach_bytes() bytes, kept alive by
 * the caller until part_reach_destroy.  Synchronous. */
ht_status part_reach_create_at(int n_parts, int log2_buckets_part, int max_state_words,
                               uint64_t exchange_rows, const ht_params* params, void* mem_dev,
                               uint64_t mem_bytes, part_reach_t** out);
ht_status part_reach_destroy(part_reach_t* c);

/* Explore from init (host model and init): clears every partition's table,
 * runs all levels (the host reads each level's size; enqueued on `stream` and
 * synchronous), and returns the result like reach().  part_states_host
 * (n_parts entries, may be NULL): states owned by each partition;
 * exchanged_host (may be NULL): successors sent to a partition other than the
 * one that generated them.  HT_ERR_FULL: a partition's table overflowed;
 * HT_ERR_LEVELS: more levels than max_levels. */
ht_status part_reach_run(part_reach_t* c, const reach_model* m, const int32_t* init_host, void* stream,
                         uint64_t* level_sizes_host, uint32_t max_levels, reach_result* out,
                         uint64_t* part_states_host, uint64_t* exchanged_host);

/* The exchange of the last chunk of the last run: counts_host[s * n + o]
 * successors from partition s owned by o, seg_off_host[s * n + o] the inbox
 * offset of that segment, in_begin_host[o] (n + 1 entries) the start of owner
 * o's inbox.  Synchronous. */
ht_status part_reach_last_exchange(part_reach_t* c, uint32_t* counts_host, uint32_t* seg_off_host,
                                   uint32_t* in_begin_host);

/* reach(model, init) for callers that cannot allocate device memory -- code
 * that must not call cudaMalloc (and so cannot create a context), e.g. a
 * process whose device memory is fixed at start-up.  There is no counterpart
 * in the paper; it is the persistent driver run out of one static device
 * array of 32 MiB (table, both frontiers, counters and level records) that
 * the library holds on every GPU that loads it, until the process exits.
 *   - Size limit: reach_ctx_bytes(log2_buckets, state_words, max_levels) must
 *     not exceed 32 MiB (e.g. 2^18 buckets for W <= 8, 2^17 for W <= 16);
 *     larger requests return HT_ERR_TOO_BIG and enqueue nothing.
 *   - Allocates nothing: no cudaMalloc/cudaFree, no pinned host buffers, no
 *     events.  Every call looks up the array's device address on the device
 *     current at the call (cudaGetSymbolAddress, which allocates nothing), so
 *     the address stays right after cudaDeviceReset and on a driver-API
 *     context of the caller's own.
 *   - Every call reuses the same array and clears what must start at zero.
 *     Calls that overlap on the GPU (other streams, other host threads) race
 *     on it: serialise them.
 *   - Synchronous: waits on `stream`, then returns the result like reach(). */
ht_status reach_noalloc(const reach_model* m, const int32_t* init_host, int log2_buckets,
                        const ht_params* params, void* stream, uint64_t* level_sizes_host,
                        uint32_t max_levels, reach_result* out);

/* ------------------------------------------------------------------------ */
/* Measurement.                                                              */
/* ------------------------------------------------------------------------ */

/* Random-access probe (the roofline denominator of this random-access path):
 * n_access accesses to uniformly random units of a device buffer of `bytes`
 * bytes (256-byte aligned; its contents are overwritten), unit by mode:
 *   0  read one 32-byte sector          1  read 64 bytes (two adjacent sectors)
 *   2  write one 32-byte sector         3  32-bit atomicAdd (a sector RMW in L2)
 *   4  32-bit compare-and-swap          5  16-bit compare-and-swap
 *   6  32-bit relaxed store             7  16-bit relaxed store
 * (4..7 are the claim and publish steps of an insert for either bucket width.)
 * Every thread keeps 8 accesses in flight; 8 blocks of 256 threads per SM.
 * Unit k of an access is a multiply-high range reduction of a SplitMix64 hash
 * of the access number (no division).  *ms = device time from CUDA events on
 * `stream`.  Synchronous.  Use a buffer much larger than L2 (e.g. 16 GiB). */
ht_status vss_probe_random(void* buf_dev, uint64_t bytes, uint64_t n_access, int mode, void* stream,
                           float* ms);

/* The same probe in a shape chosen by the caller, for finding where the rate
 * stops growing with the requests in flight: `inflight` accesses issued by
 * each thread before it consumes any (1, 2, 4, 8, 16, 32 or 64; reads of 32
 * bytes up to 16 and of 64 bytes up to 8, because they hold their data in
 * registers), a grid of blocks_per_sm (1..64) blocks per SM of `threads`
 * (32..256, a multiple of 32) threads; 0 in any of the three selects 8, 8
 * and 256.  Blocks beyond those resident at once (a shape's registers set
 * that number) run in waves.  One more mode:
 *   8  read 4 bytes of a random 32-byte sector (DRAM still moves the sector
 *      into L2; 4 bytes go back to the SM: the memory side of mode 0)
 *   9  read a random 64-byte unit by two lanes, 32 bytes each, in one load
 *      instruction (n_access counts units; every lane keeps `inflight`)
 *  10  read a random 128-byte line by four lanes in one instruction
 *  11  read a random 64-byte unit by one thread with one bulk asynchronous
 *      copy (cp.async.bulk) into its slot in shared memory, completion
 *      counted on the thread's own mbarrier (inflight 1, 2, 4 or 8)
 *  12  write a random 64-byte unit by one thread with one bulk asynchronous
 *      copy from its slot in shared memory (inflight 1, 2, 4 or 8)
 * Modes 11 and 12 use threads * inflight * 64 + threads * 8 bytes of shared
 * memory per block; their mbarrier waits are bounded and a wait that runs
 * out returns HT_ERR_TIMEOUT.
 * HT_ERR_INVALID for a shape or mode outside these.  Synchronous. */
ht_status vss_probe_random_cfg(void* buf_dev, uint64_t bytes, uint64_t n_access, int mode,
                               int inflight, int blocks_per_sm, int threads, void* stream,
                               float* ms);

/* Human-readable name of a status code (static storage). */
const char* ht_status_string(ht_status s);

#ifdef __cplusplus
}
#endif

#endif /* PAPER_1004_2772_GB300_REACH_H */
