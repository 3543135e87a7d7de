// Served reachability: a request loop with continuous batching.
//
// One persistent kernel (the batched driver's, in serving mode) keeps running
// while jobs arrive.  The host admits a job when a slot and memory for its
// table are free -- memory comes from one device arena whose size is the HBM
// budget, managed first-fit on the host -- writes the job's record into the
// slot's host-mapped mailbox and rings a doorbell; a device warp with nothing
// to do takes the job into its slot, so new jobs join work already on the GPU
// and their levels overlap with the running jobs' levels.  A finished job's
// result comes back through the slot's mapped out-box; the host then frees its
// memory, which may admit the next queued job.  The kernel leaves on its own
// once nothing has run for a while (every wait on the device is bounded), and
// the host relaunches it on the next submission.
//
// While the queue is short and the many-job kernel is gone, jobs run one at a
// time on the persistent single-model kernel, whose level path is shorter;
// jobs that arrive meanwhile queue, and a queue of kBatchFrom or more goes to
// the many-job kernel.  Both run on the same stream, so they never overlap.
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "batch.h"
#include "internal.h"

using namespace vss;

namespace {

uint64_t up256(uint64_t x) { return (x + 255) & ~255ull; }

// Queued jobs go to the many-job kernel once this many wait; shorter queues
// are served one job at a time on the single-model kernel.  At 20 jobs/s a
// threshold of 2 gave p99 175 ms, 4, 8 and 64 gave 122 ms (same p50).
constexpr size_t kBatchFrom = 8;

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size), 256-byte granules.
struct Arena {
  std::map<uint64_t, uint64_t> free_;  // offset -> size
  uint64_t size = 0;
  void init(uint64_t s) {
    size = s;
    free_.clear();
    if (s) free_[0] = s;
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    bytes = up256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const uint64_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = up256(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace

struct serve {
  void* owned = nullptr;
  uint32_t n_slots = 0, max_levels = 0;
  ht_params params{};
  BatchModel* slots_dev = nullptr;
  BatchState* state_dev = nullptr;
  unsigned long long* accepted_dev = nullptr;
  unsigned long long* levels_dev = nullptr;
  char* arena_dev = nullptr;
  Arena arena;
  ServeMailbox* mb = nullptr;  // host-mapped
  ServeSlotIn* in = nullptr;
  ServeSlotOut* out = nullptr;
  struct Slot {
    bool busy = false;
    bool solo = false;  // running on the single-model kernel, not in the many-job kernel
    uint64_t job = 0, seq = 0, off = 0, bytes = 0;
    double t_submit = 0, t_admit = 0;
  };
  std::vector<Slot> slots;
  struct Job {
    uint64_t id;
    std::vector<int> blob;
    uint32_t W;
    int log2;
    unsigned long long bound;
    double t_submit;
    bool no_solo = false;  // the single-model kernel cannot take it (e.g. shared memory)
  };
  std::deque<Job> pending;
  std::vector<serve_done_t> rejected;  // jobs that can never fit, reported by the next poll
  uint64_t next_job = 1, next_seq = 0, doorbell = 0;
  cudaStream_t kstream = nullptr, cstream = nullptr;
  BatchGlobal g{};
  BatchKernel kernel = nullptr;
  int blocks = 0, threads = 256;
  size_t smem = 0;
  bool launched = false;
  uint64_t launches = 0;
  // single-model path
  bool solo = false;  // a single-model run is in flight on kstream
  uint32_t solo_slot = 0;
  SoloRun solo_run{};
  void* solo_tot_dev = nullptr;
  unsigned long long* solo_ns_dev = nullptr;
  cudaEvent_t solo_ev = nullptr;
};

static uint64_t serve_fixed_bytes(uint32_t n_slots, uint32_t max_levels) {
  return up256((uint64_t)n_slots * sizeof(BatchModel)) + up256(sizeof(BatchState)) +
         up256((uint64_t)n_slots * 8) + up256((uint64_t)n_slots * max_levels * 8) +
         up256(solo_totals_bytes()) + up256((uint64_t)max_levels * 8);
}

static bool batch_busy(const serve_t* s) {
  for (auto& sl : s->slots)
    if (sl.busy && !sl.solo) return true;
  return false;
}

// Start the front job alone on the single-model kernel.  Returns false when
// it cannot (the job then goes to the many-job kernel).
static bool start_solo(serve_t* s, uint32_t slot, uint64_t off, uint64_t bytes, uint64_t blob_bytes) {
  serve_t::Job& job = s->pending.front();
  const uint32_t nv = (job.W + 3) / 4;
  const uint64_t nb = 1ull << job.log2;
  const uint32_t L = s->params.line_buckets;
  char* base = s->arena_dev + off;
  char* gp = base + blob_bytes;
  SoloRun& r = s->solo_run;
  r = SoloRun{};
  r.tv.buckets = reinterpret_cast<uint32_t*>(gp);
  r.tv.data = reinterpret_cast<uint4*>(gp + up256(nb * 4));
  r.tv.ctr = &s->slots_dev[slot].ctr;
  r.tv.seed = s->g.seed;
  r.tv.nb_mask = (uint32_t)(nb - 1);
  r.tv.lines = (uint32_t)(nb / L);
  r.tv.lines_mask = r.tv.lines - 1;
  r.tv.lines_div = DivU64{0, 0, 0};
  r.tv.max_rehash = r.tv.lines < 4096u ? r.tv.lines : 4096u;
  r.tv.max_spin = s->params.max_spin;
  r.tv.state_words = job.W;
  r.tv.nv = nv;
  r.tv.bucket_bits = 32;
  r.blob_dev = reinterpret_cast<const int*>(base);
  r.smem_words = job.blob[11];
  r.fr0 = reinterpret_cast<uint4*>(gp + up256(nb * 4) + up256(nb * 16 * nv));
  r.fr1 = reinterpret_cast<uint4*>(gp + up256(nb * 4) + 2 * up256(nb * 16 * nv));
  r.cap = (uint32_t)nb;
  r.tot_dev = s->solo_tot_dev;
  r.level_sizes_dev = s->levels_dev + (uint64_t)slot * s->max_levels;
  r.level_ns_dev = s->solo_ns_dev;
  r.max_levels = s->max_levels;
  if (solo_launch(r, (int)L, (int)s->params.block_threads, s->kstream) != HT_OK ||
      cudaEventRecord(s->solo_ev, s->kstream) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  serve_t::Slot& sl = s->slots[slot];
  sl.busy = true;
  sl.solo = true;
  sl.job = job.id;
  sl.seq = 0;
  sl.off = off;
  sl.bytes = bytes;
  sl.t_submit = job.t_submit;
  sl.t_admit = now_s();
  s->solo = true;
  s->solo_slot = slot;
  s->launches++;
  s->pending.pop_front();
  return true;
}

static ht_status ensure_running(serve_t* s) {
  if (s->launched) {
    const cudaError_t q = cudaStreamQuery(s->kstream);
    if (q == cudaErrorNotReady) return HT_OK;
    if (q != cudaSuccess) return HT_ERR_CUDA;
  }
  s->kernel<<<s->blocks, s->threads, s->smem, s->kstream>>>(s->g);
  VSS_CUDA_TRY(cudaGetLastError());
  s->launched = true;
  s->launches++;
  return HT_OK;
}

static void admit(serve_t* s) {
  if (s->solo) return;  // queued jobs wait for the single-model run
  while (!s->pending.empty()) {
    uint32_t slot = s->n_slots;
    bool any_busy = false;
    for (uint32_t i = 0; i < s->n_slots; ++i) {
      if (!s->slots[i].busy) {
        if (slot == s->n_slots) slot = i;
      } else {
        any_busy = true;
      }
    }
    if (slot == s->n_slots) return;  // every slot is running a job
    serve_t::Job& job = s->pending.front();
    const uint32_t nv = (job.W + 3) / 4;
    const uint64_t blob_bytes = up256(job.blob.size() * 4);
    const uint64_t bytes = blob_bytes + generation_bytes((uint32_t)job.log2, nv);
    uint64_t off = 0;
    if (!s->arena.alloc(bytes, &off)) {
      if (!any_busy) {  // the arena is empty and still too small: this job can never run
        serve_done_t d;
        std::memset(&d, 0, sizeof(d));
        d.job_id = job.id;
        d.result.status = HT_ERR_OOM;
        d.submit_s = d.admit_s = d.done_s = job.t_submit;
        s->rejected.push_back(d);
        s->pending.pop_front();
        continue;
      }
      return;  // wait until a running job frees memory
    }
    char* base = s->arena_dev + off;
    if (cudaMemcpyAsync(base, job.blob.data(), job.blob.size() * 4, cudaMemcpyHostToDevice,
                        s->cstream) != cudaSuccess ||
        cudaStreamSynchronize(s->cstream) != cudaSuccess) {
      cudaGetLastError();
      s->arena.release(off, bytes);
      return;
    }
    // an idle GPU and a lone job: run it on the single-model kernel
    const bool gpu_idle = !any_busy && s->pending.size() < kBatchFrom &&
                          (!s->launched || cudaStreamQuery(s->kstream) == cudaSuccess);
    if (gpu_idle && !job.no_solo) {
      if (start_solo(s, slot, off, bytes, blob_bytes)) return;
      job.no_solo = true;
    }
    const uint64_t nb = 1ull << job.log2;
    char* gp = base + blob_bytes;
    BatchModel M;
    std::memset(&M, 0, sizeof(M));
    M.blob = reinterpret_cast<const int*>(base);
    M.level_sizes = s->levels_dev + (uint64_t)slot * s->max_levels;
    M.W = job.W;
    M.nv = nv;
    M.maxfan = (uint32_t)job.blob[13];
    M.spw_max = (uint32_t)job.blob[14];
    M.max_levels = s->max_levels;
    M.log2_nb = (uint32_t)job.log2;
    M.buckets = reinterpret_cast<uint32_t*>(gp);
    M.data = reinterpret_cast<uint4*>(gp + up256(nb * 4));
    M.fr[0] = reinterpret_cast<uint4*>(gp + up256(nb * 4) + up256(nb * 16 * nv));
    M.fr[1] = reinterpret_cast<uint4*>(gp + up256(nb * 4) + 2 * up256(nb * 16 * nv));
    M.nbuckets = M.buckets;
    M.nlog2 = M.log2_nb;
    // a served job's table is sized by the host; it never grows
    M.states_bound = job.bound ? job.bound : (unsigned long long)(0.75 * (double)nb);
    const uint64_t clear_units = (nb + kClearUnit - 1) / kClearUnit;
    M.claim = ((unsigned long long)PH_CLEAR << 48) | (clear_units << 24);
    ServeSlotIn* box = s->in + slot;
    std::memcpy(&box->rec, &M, sizeof(M));
    const uint64_t seq = ++s->next_seq;
    __atomic_store_n(&box->seq, (unsigned long long)seq, __ATOMIC_RELEASE);
    __atomic_store_n(&s->mb->doorbell, (unsigned long long)++s->doorbell, __ATOMIC_RELEASE);
    serve_t::Slot& sl = s->slots[slot];
    sl.busy = true;
    sl.job = job.id;
    sl.seq = seq;
    sl.off = off;
    sl.bytes = bytes;
    sl.t_submit = job.t_submit;
    sl.t_admit = now_s();
    s->pending.pop_front();
  }
}

extern "C" {

ht_status serve_bytes(uint64_t budget_bytes, uint32_t n_slots, uint32_t max_levels,
                      uint64_t* bytes) {
  if (!bytes || n_slots < 1 || n_slots > 4096 || max_levels < 1) return HT_ERR_INVALID;
  *bytes = serve_fixed_bytes(n_slots, max_levels) + up256(budget_bytes);
  return HT_OK;
}

ht_status serve_open_at(void* mem_dev, uint64_t mem_bytes, uint32_t n_slots, uint32_t max_levels,
                        const ht_params* params, serve_t** out) {
  if (!out || !mem_dev || (reinterpret_cast<uintptr_t>(mem_dev) & 255u) || n_slots < 1 ||
      n_slots > 4096 || max_levels < 1)
    return HT_ERR_INVALID;
  *out = nullptr;
  const uint64_t fixed = serve_fixed_bytes(n_slots, max_levels);
  if (mem_bytes < fixed + (1u << 20)) return HT_ERR_OOM;
  ht_params p{};
  ht_status st = resolve_params(params, 1u << 10, &p);
  if (st != HT_OK) return st;
  // batch tables use 32-bit buckets walked by one thread per key, double hashing
  if (p.bucket_bits != 32 || p.group_lanes != 1 || p.rehash != 0) return HT_ERR_INVALID;
  serve_t* s = new (std::nothrow) serve_t();
  if (!s) return HT_ERR_OOM;
  s->n_slots = n_slots;
  s->max_levels = max_levels;
  s->params = p;
  char* q = static_cast<char*>(mem_dev);
  s->slots_dev = reinterpret_cast<BatchModel*>(q);
  q += up256((uint64_t)n_slots * sizeof(BatchModel));
  s->state_dev = reinterpret_cast<BatchState*>(q);
  q += up256(sizeof(BatchState));
  s->accepted_dev = reinterpret_cast<unsigned long long*>(q);
  q += up256((uint64_t)n_slots * 8);
  s->levels_dev = reinterpret_cast<unsigned long long*>(q);
  q += up256((uint64_t)n_slots * max_levels * 8);
  s->solo_tot_dev = q;
  q += up256(solo_totals_bytes());
  s->solo_ns_dev = reinterpret_cast<unsigned long long*>(q);
  q += up256((uint64_t)max_levels * 8);
  s->arena_dev = q;
  s->arena.init((mem_bytes - fixed) & ~255ull);
  s->slots.resize(n_slots);

  auto fail = [&](ht_status code) {
    if (s->mb) cudaFreeHost(s->mb);
    if (s->in) cudaFreeHost(s->in);
    if (s->out) cudaFreeHost(s->out);
    if (s->kstream) cudaStreamDestroy(s->kstream);
    if (s->cstream) cudaStreamDestroy(s->cstream);
    if (s->solo_ev) cudaEventDestroy(s->solo_ev);
    cudaGetLastError();
    delete s;
    return code;
  };
  if (cudaHostAlloc(reinterpret_cast<void**>(&s->mb), sizeof(ServeMailbox), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&s->in), sizeof(ServeSlotIn) * n_slots, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&s->out), sizeof(ServeSlotOut) * n_slots, cudaHostAllocMapped) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->solo_ev, cudaEventDisableTiming) != cudaSuccess)
    return fail(HT_ERR_CUDA);
  std::memset(s->mb, 0, sizeof(ServeMailbox));
  std::memset(s->in, 0, sizeof(ServeSlotIn) * n_slots);
  std::memset(s->out, 0, sizeof(ServeSlotOut) * n_slots);
  // every slot starts empty (claim word in the DONE phase)
  std::vector<BatchModel> init(n_slots);
  std::memset(init.data(), 0, sizeof(BatchModel) * n_slots);
  for (auto& M : init) M.claim = (unsigned long long)PH_DONE << 48;
  if (cudaMemcpy(s->slots_dev, init.data(), sizeof(BatchModel) * n_slots, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->state_dev, 0, sizeof(BatchState)) != cudaSuccess ||
      cudaMemset(s->accepted_dev, 0, (size_t)n_slots * 8) != cudaSuccess)
    return fail(HT_ERR_CUDA);
  ServeMailbox* mb_dev = nullptr;
  ServeSlotIn* in_dev = nullptr;
  ServeSlotOut* out_dev = nullptr;
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&mb_dev), s->mb, 0) != cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void**>(&in_dev), s->in, 0) != cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void**>(&out_dev), s->out, 0) != cudaSuccess)
    return fail(HT_ERR_CUDA);
  s->kernel = batch_kernel((int)p.line_buckets);
  s->smem = batch_smem_bytes(s->threads);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(s->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, s->kernel, s->threads, s->smem) != cudaSuccess ||
      per_sm < 1)
    return fail(HT_ERR_CUDA);
  s->blocks = per_sm * sms;
  BatchGlobal& g = s->g;
  g.models = s->slots_dev;
  g.st = s->state_dev;
  g.pool = nullptr;  // served tables never grow
  g.pool_bytes = 0;
  g.seed = p.hash_seed;
  g.n_models = n_slots;
  g.max_spin = p.max_spin;
  g.idle_ns = 2000000ull;      // 2 ms without any work: the kernel leaves (and the next
                               // job to arrive at the idle GPU runs on the single-model kernel)
  g.stuck_ns = 4000000000ull;  // 4 s with jobs in slots but nothing claimable: error
  g.grow_at = 0.9f;
  g.grow_to = 0.5f;
  g.mb = mb_dev;
  g.in = in_dev;
  g.out = out_dev;
  g.accepted = s->accepted_dev;
  *out = s;
  return HT_OK;
}

ht_status serve_open(uint64_t budget_bytes, uint32_t n_slots, uint32_t max_levels,
                     const ht_params* params, serve_t** out) {
  uint64_t bytes = 0;
  if (!out) return HT_ERR_INVALID;
  *out = nullptr;
  ht_status st = serve_bytes(budget_bytes, n_slots, max_levels, &bytes);
  if (st != HT_OK) return st;
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return HT_ERR_OOM;
  }
  st = serve_open_at(mem, bytes, n_slots, max_levels, params, out);
  if (st != HT_OK) {
    cudaFree(mem);
    return st;
  }
  (*out)->owned = mem;
  return HT_OK;
}

ht_status serve_submit(serve_t* s, const reach_model* m, const int32_t* init_host, int log2_buckets,
                       uint64_t* job_id) {
  if (!s || !m || !init_host) return HT_ERR_INVALID;
  serve_t::Job job;
  ht_status st = pack_model(m, init_host, 32, job.blob);
  if (st != HT_OK) return st;
  job.W = (uint32_t)m->state_words;
  job.bound = 0;
  if (m->n_shared == 0) {
    long double pr = 1;
    for (int k = 0; k < m->n_procs; ++k) pr *= m->n_local[k];
    job.bound = pr > 1e15 ? 0 : (unsigned long long)pr;
  }
  if (log2_buckets <= 0) {  // size for at most 75% load of the bound
    if (!job.bound) return HT_ERR_INVALID;
    log2_buckets = 10;
    while (log2_buckets < 31 && (double)(1ull << log2_buckets) * 0.75 < (double)job.bound) ++log2_buckets;
  }
  if (log2_buckets < 10 || log2_buckets > 31) return HT_ERR_INVALID;
  job.log2 = log2_buckets;
  job.id = s->next_job++;
  job.t_submit = now_s();
  if (job_id) *job_id = job.id;
  s->pending.push_back(std::move(job));
  admit(s);
  return batch_busy(s) ? ensure_running(s) : HT_OK;
}

ht_status serve_poll(serve_t* s, serve_done_t* done, uint32_t max_done, uint32_t* n_done,
                     uint64_t* level_sizes_host) {
  if (!s || !n_done || (max_done && !done)) return HT_ERR_INVALID;
  uint32_t n = 0;
  while (n < max_done && !s->rejected.empty()) {
    done[n++] = s->rejected.back();
    s->rejected.pop_back();
  }
  if (s->solo && n < max_done) {
    const cudaError_t q = cudaEventQuery(s->solo_ev);
    if (q != cudaSuccess && q != cudaErrorNotReady) return HT_ERR_CUDA;
    if (q == cudaSuccess) {
      serve_t::Slot& sl = s->slots[s->solo_slot];
      serve_done_t& d = done[n];
      std::memset(&d, 0, sizeof(d));
      d.job_id = sl.job;
      solo_result(s->solo_run, &d.result);
      d.submit_s = sl.t_submit;
      d.admit_s = sl.t_admit;
      d.done_s = now_s();
      if (level_sizes_host && d.result.n_levels) {
        const uint32_t nl = d.result.n_levels < s->max_levels ? d.result.n_levels : s->max_levels;
        VSS_CUDA_TRY(cudaMemcpy(level_sizes_host + (uint64_t)n * s->max_levels,
                                s->solo_run.level_sizes_dev, (size_t)nl * 8, cudaMemcpyDeviceToHost));
      }
      s->arena.release(sl.off, sl.bytes);
      sl.busy = false;
      sl.solo = false;
      s->solo = false;
      ++n;
    }
  }
  for (uint32_t i = 0; i < s->n_slots && n < max_done; ++i) {
    serve_t::Slot& sl = s->slots[i];
    if (!sl.busy || sl.solo) continue;
    if (__atomic_load_n(&s->out[i].seq, __ATOMIC_ACQUIRE) != sl.seq) continue;
    const ServeSlotOut& o = s->out[i];
    serve_done_t& d = done[n];
    std::memset(&d, 0, sizeof(d));
    d.job_id = sl.job;
    d.result.states = o.states;
    d.result.transitions = o.transitions;
    d.result.deadlocks = o.deadlocks;
    d.result.digest = o.digest;
    d.result.busy_waits = o.busy_waits;
    d.result.rehashes = o.rehashes;
    d.result.n_levels = o.n_levels;
    d.result.status = (ht_status)o.status;
    d.grows = o.grows;
    d.submit_s = sl.t_submit;
    d.admit_s = sl.t_admit;
    d.done_s = now_s();
    if (level_sizes_host && o.n_levels) {
      const uint32_t nl = o.n_levels < s->max_levels ? o.n_levels : s->max_levels;
      VSS_CUDA_TRY(cudaMemcpyAsync(level_sizes_host + (uint64_t)n * s->max_levels,
                                   s->levels_dev + (uint64_t)i * s->max_levels, (size_t)nl * 8,
                                   cudaMemcpyDeviceToHost, s->cstream));
      VSS_CUDA_TRY(cudaStreamSynchronize(s->cstream));
    }
    s->arena.release(sl.off, sl.bytes);
    sl.busy = false;
    ++n;
  }
  *n_done = n;
  admit(s);
  if (batch_busy(s)) {
    // a kernel that stopped with jobs still in their slots hit a device error
    if (s->launched && cudaStreamQuery(s->kstream) == cudaSuccess) {
      BatchState bst;
      VSS_CUDA_TRY(cudaMemcpy(&bst, s->state_dev, sizeof(bst), cudaMemcpyDeviceToHost));
      if (bst.err) return (ht_status)bst.err;
    }
    return ensure_running(s);
  }
  return HT_OK;
}

ht_status serve_status(serve_t* s, uint32_t* queued, uint32_t* running, uint64_t* free_bytes,
                       uint64_t* kernel_launches) {
  if (!s) return HT_ERR_INVALID;
  uint32_t r = 0;
  for (auto& sl : s->slots) r += sl.busy ? 1 : 0;
  if (queued) *queued = (uint32_t)s->pending.size();
  if (running) *running = r;
  if (free_bytes) {
    uint64_t f = 0;
    for (auto& kv : s->arena.free_) f += kv.second;
    *free_bytes = f;
  }
  if (kernel_launches) *kernel_launches = s->launches;
  return HT_OK;
}

ht_status serve_close(serve_t* s) {
  if (!s) return HT_ERR_INVALID;
  __atomic_store_n(&s->mb->shutdown, 1u, __ATOMIC_RELEASE);
  ht_status st = HT_OK;
  if (s->launched && cudaStreamSynchronize(s->kstream) != cudaSuccess) st = HT_ERR_CUDA;
  cudaStreamDestroy(s->kstream);
  cudaStreamDestroy(s->cstream);
  cudaEventDestroy(s->solo_ev);
  cudaFreeHost(s->mb);
  cudaFreeHost(s->in);
  cudaFreeHost(s->out);
  if (s->owned) cudaFree(s->owned);
  delete s;
  return st;
}

}  // extern "C"
