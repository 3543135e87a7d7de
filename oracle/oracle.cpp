// Reference oracle for the visited-state store: TEST INFRASTRUCTURE ONLY.
//
// Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
// this library.  It shares no code with the CUDA path: the set V is a plain
// std::unordered_set keyed by the whole state vector (std::hash over the bytes),
// exploration is a strict level-by-level BFS, and every number it returns has
// a plain definition:
//
//   states       |V|, the states reachable from init           (Alg. "Reachability analysis")
//   transitions  number of enabled edges summed over V, with multiplicity:
//                one find-or-put call per successor              (Section 4.3: calls = transitions)
//   deadlocks    states with no enabled edge                     (Alg. "Reachability analysis", count == 0)
//   level sizes  |{s : BFS distance(init, s) = k}|
//   digest       sum over V of g(s) mod 2^64, an order-independent fingerprint
//                of the set:  x = W;  for each word w: x = sm(x xor (uint32)w);
//                g(s) = x,   where sm(z) is one SplitMix64 output step
//                (Steele, Lea, Flood 2014): z += 0x9E3779B97F4A7C15, then
//                z = (z ^ z>>30) * 0xBF58476D1CE4E5B9,
//                z = (z ^ z>>27) * 0x94D049BB133111EB, z ^ z>>31.
//
// For a key stream (the hash-table benchmark) the answer of find-or-put is
// "was this vector inserted before" (Section 3.1, the single operation of the
// store): seen[k] = !V.insert(key_k).second, in stream order.
//
// Model semantics (edge enabling, guards, updates, the critical-state mutex)
// are those of the seeded model encoding: edge e of process p leaving local
// state s is enabled in v when v[p] == s, its guard (if any) holds on the
// shared variable, and it does not enter p's critical state while another
// process sits in its own.  Firing sets v[p] to the edge's target and applies
// the edge's update (if any).  Successors are listed for p ascending, then
// edges in CSR order.
//
// Pins: every function here is checked, without the GPU, against closed forms
// of the interleaving family, a dense brute-force fixpoint over tiny models,
// hand-enumerated models and the published SplitMix64 output values.
//
// ORACLE_PLANT: test-only build variants that each plant one plausible mistake,
// used by the tests to show that the pins catch it.  The default build (0)
// plants nothing.

#include <cstdint>
#include <cstring>
#include <string_view>
#include <unordered_set>
#include <vector>

#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

namespace {

using State = std::vector<int32_t>;

struct StateHash {
  size_t operator()(const State& s) const {
    return std::hash<std::string_view>{}(
        std::string_view(reinterpret_cast<const char*>(s.data()), s.size() * sizeof(int32_t)));
  }
};

using StateSet = std::unordered_set<State, StateHash>;

uint64_t sm_step(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t state_fingerprint(const int32_t* v, int W) {
  uint64_t x = static_cast<uint64_t>(W);
  for (int i = 0; i < W; ++i) {
#if ORACLE_PLANT == 4
    if (i == W - 1) break;  // planted: last word dropped from the fingerprint
#endif
    x = sm_step(x ^ static_cast<uint64_t>(static_cast<uint32_t>(v[i])));
  }
  return x;
}

struct Model {
  int P, S, W;
  const int32_t *n_local, *crit, *edge_begin, *edge_dst, *guard_var, *guard_val, *upd_var, *upd_val;
  std::vector<int32_t> local_base;

  void init_base() {
    local_base.assign(P, 0);
    for (int p = 1; p < P; ++p) local_base[p] = local_base[p - 1] + n_local[p - 1];
  }

  bool someone_else_critical(const State& v, int p) const {
    for (int q = 0; q < P; ++q)
      if (q != p && crit[q] >= 0 && v[q] == crit[q]) return true;
    return false;
  }

  // next-state: all successors of v, with multiplicity, in the fixed order.
  void successors(const State& v, std::vector<State>& out) const {
    out.clear();
    for (int p = 0; p < P; ++p) {
      const int s = v[p];
      const int b = local_base[p] + s;
      for (int e = edge_begin[b]; e < edge_begin[b + 1]; ++e) {
#if ORACLE_PLANT != 1
        if (guard_var[e] >= 0 && v[P + guard_var[e]] != guard_val[e]) continue;
#endif
        const int dst = edge_dst[e];
#if ORACLE_PLANT == 2
        if (crit[p] >= 0 && dst == crit[p] && someone_else_critical(v, -1)) continue;  // planted: p counted against itself
#else
        if (crit[p] >= 0 && dst == crit[p] && someone_else_critical(v, p)) continue;
#endif
        State w = v;
        w[p] = dst;
#if ORACLE_PLANT != 3
        if (upd_var[e] >= 0) w[P + upd_var[e]] = upd_val[e];
#endif
        out.push_back(std::move(w));
      }
    }
  }
};

Model make_model(int P, int S, int W, const int32_t* n_local, const int32_t* crit,
                 const int32_t* edge_begin, const int32_t* edge_dst, const int32_t* guard_var,
                 const int32_t* guard_val, const int32_t* upd_var, const int32_t* upd_val) {
  Model m{P, S, W, n_local, crit, edge_begin, edge_dst, guard_var, guard_val, upd_var, upd_val, {}};
  m.init_base();
  return m;
}

}  // namespace

extern "C" {

// One SplitMix64 output step (exported so tests can pin it to published values).
uint64_t oracle_splitmix64(uint64_t z) { return sm_step(z); }

// g(v) for one state of W words.
uint64_t oracle_state_fingerprint(const int32_t* v, int W) { return state_fingerprint(v, W); }

// Sum of g over n states (row-major n x W), mod 2^64.
uint64_t oracle_digest(const int32_t* states, uint64_t n, int W) {
  uint64_t d = 0;
  for (uint64_t i = 0; i < n; ++i) d += state_fingerprint(states + i * W, W);
  return d;
}

// Successors of one state; writes up to max_out rows of W words, returns the count
// (the full count even when larger than max_out).
int64_t oracle_successors(int P, int S, int W, const int32_t* n_local, const int32_t* crit,
                          const int32_t* edge_begin, const int32_t* edge_dst,
                          const int32_t* guard_var, const int32_t* guard_val,
                          const int32_t* upd_var, const int32_t* upd_val, const int32_t* v,
                          int32_t* out, int64_t max_out) {
  Model m = make_model(P, S, W, n_local, crit, edge_begin, edge_dst, guard_var, guard_val, upd_var,
                       upd_val);
  std::vector<State> succ;
  m.successors(State(v, v + W), succ);
  for (int64_t k = 0; k < static_cast<int64_t>(succ.size()) && k < max_out; ++k)
    std::memcpy(out + k * W, succ[k].data(), sizeof(int32_t) * W);
  return static_cast<int64_t>(succ.size());
}

// Level-synchronous BFS from init (Alg. "Reachability analysis" with T a FIFO
// processed one BFS level at a time; a successor is enqueued when find-or-put
// reports it was not seen before).
//
// Stops early (returns 1, *truncated = 1) once more than max_states states have
// been stored (|V| > max_states) or
// the level count would exceed max_levels; returns 0 on a complete run.
// When states_out is non-null, the first states_cap states are written there in
// discovery order (row-major, W words each).
int oracle_reach(int P, int S, int W, const int32_t* n_local, const int32_t* crit,
                 const int32_t* edge_begin, const int32_t* edge_dst, const int32_t* guard_var,
                 const int32_t* guard_val, const int32_t* upd_var, const int32_t* upd_val,
                 const int32_t* init, uint64_t max_states, uint32_t max_levels,
                 uint64_t* out_states, uint64_t* out_transitions, uint64_t* out_deadlocks,
                 uint64_t* out_digest, uint64_t* level_sizes, uint32_t* out_n_levels,
                 int32_t* truncated, int32_t* states_out, uint64_t states_cap) {
  Model m = make_model(P, S, W, n_local, crit, edge_begin, edge_dst, guard_var, guard_val, upd_var,
                       upd_val);
  StateSet V;
  uint64_t transitions = 0, deadlocks = 0, digest = 0, written = 0;
  uint32_t n_levels = 0;
  *truncated = 0;

  auto record = [&](const State& s) {
    digest += state_fingerprint(s.data(), W);
    if (states_out && written < states_cap)
      std::memcpy(states_out + written * W, s.data(), sizeof(int32_t) * W);
    ++written;
  };

  State s0(init, init + W);
  V.insert(s0);
  record(s0);
  std::vector<State> level{s0}, next, succ;
  if (max_levels > 0) level_sizes[n_levels] = 1;
  ++n_levels;

  while (!level.empty()) {
    next.clear();
    for (const State& s : level) {
      m.successors(s, succ);
      uint64_t count = 0;
      for (State& t : succ) {
        ++count;
        ++transitions;
#if ORACLE_PLANT == 5
        if (t == s) --transitions;  // planted: self-loops not counted as transitions
#endif
#if ORACLE_PLANT == 6
        const bool inserted = V.count(t) == 0;  // planted: membership tested, insert deferred
#else
        const bool inserted = V.insert(t).second;
#endif
        if (inserted) {  // find-or-put answered "not seen": put on the next level
          record(t);
          next.push_back(t);
          if (written > max_states) {
            *truncated = 1;
            break;
          }
        }
      }
      if (count == 0) ++deadlocks;
      if (*truncated) break;
    }
    if (*truncated) break;
#if ORACLE_PLANT == 6
    for (const State& t : next) V.insert(t);
#endif
    if (!next.empty()) {
      if (n_levels >= max_levels) {
        *truncated = 1;
        break;
      }
      level_sizes[n_levels] = next.size();
      ++n_levels;
    }
    level.swap(next);
  }

  *out_states = V.size();
  *out_transitions = transitions;
  *out_deadlocks = deadlocks;
  *out_digest = digest;
  *out_n_levels = n_levels;
  return *truncated;
}

// find-or-put over a key stream, in stream order: seen[k] = 1 when key k was
// inserted by an earlier call.  first[k] = position of the first call with the
// same key (so calls with equal keys are recognisable without trusting any hash).
// Returns the number of distinct keys; *digest = sum of g over the distinct keys.
uint64_t oracle_find_or_put_stream(const int32_t* keys, uint64_t n, int W, uint8_t* seen,
                                   uint64_t* first, uint64_t* digest) {
  struct Entry {
    State key;
    uint64_t pos;
  };
  struct EntryHash {
    size_t operator()(const Entry& e) const { return StateHash{}(e.key); }
  };
  struct EntryEq {
    bool operator()(const Entry& a, const Entry& b) const { return a.key == b.key; }
  };
  std::unordered_set<Entry, EntryHash, EntryEq> V;
  uint64_t d = 0;
  for (uint64_t k = 0; k < n; ++k) {
    Entry e{State(keys + k * W, keys + (k + 1) * W), k};
    auto [it, inserted] = V.insert(std::move(e));
    seen[k] = inserted ? 0 : 1;
    if (first) first[k] = it->pos;
    if (inserted) d += state_fingerprint(keys + k * W, W);
  }
  if (digest) *digest = d;
  return V.size();
}

}  // extern "C"
