// Runtime for streams of mixed-size requests (include/tat_service.h): plan
// cache, batching per (problem, operation), one device arena with admission
// and LRU eviction of staging slots, a stream per slot, CUDA graphs per
// (slot, batch), and the launch-shape autotuner.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "plan.hpp"
#include "tat_service.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kAlign = 256;
constexpr size_t kMaxCompositions = 4096;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

tat_status cuda_ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TAT_OK;
  fprintf(stderr, "tat service: %s: %s\n", what, cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TAT_ERR_OOM : TAT_ERR_CUDA;
}

struct Request {
  long long id;
  const float* in;
  float* out;
  Clock::time_point submitted, done;
  tat_status status = TAT_OK;
  bool completed = false;
};

struct Slot;

// First-fit allocator over the arena (offsets only; the arena is one cudaMalloc).
class Arena {
 public:
  size_t size = 0;
  char* base = nullptr;
  std::map<size_t, size_t> used;  // offset -> bytes
  size_t held = 0, peak = 0;

  bool alloc(size_t bytes, size_t* off) {
    size_t cur = 0;
    for (const auto& u : used) {
      if (u.first - cur >= bytes) break;
      cur = align_up(u.first + u.second);
    }
    if (cur + bytes > size) return false;
    used[cur] = bytes;
    held += bytes;
    peak = std::max(peak, held);
    *off = cur;
    return true;
  }
  void release(size_t off) {
    auto it = used.find(off);
    if (it == used.end()) return;
    held -= it->second;
    used.erase(it);
  }
};

struct Slot {
  std::string key;
  tat_plan_t plan = nullptr;
  tat_op op = TAT_OP_FORWARD;
  cudaStream_t stream = nullptr;
  int cap = 0;                        // images per launch (0: not resident)
  size_t off = 0, bytes = 0;          // arena region
  float* in = nullptr;
  float* out = nullptr;
  float* mid = nullptr;               // A f of a pair request (TAT_OP_PAIR only)
  void* ws = nullptr;
  size_t in_elems = 0, out_elems = 0, mid_elems = 0;
  std::map<int, cudaGraphExec_t> graphs;  // batch -> executable graph
  cudaStream_t branch = nullptr;      // captured into the single-graph flush (never runs work itself)
  cudaEvent_t staged = nullptr;       // inputs of the chunk in the single graph are on the device
  std::vector<long long> pending;
  unsigned long long last_use = 0;
  bool tuned = false;
};

struct Completion {
  tat_service_s* svc;
  std::vector<long long> ids;
};

}  // namespace

struct tat_service_s {
  tat_service_config cfg;
  int device = 0;
  Arena arena;
  std::map<std::string, tat_plan_t> plans;  // descriptor bytes -> plan
  std::map<std::string, std::unique_ptr<Slot>> slots;
  std::deque<Request> requests;
  std::mutex mu;                            // guards request completion fields
  unsigned long long tick = 0;
  tat_service_stats st{};
  // single-graph flushes: the launch stream, its completion event and the executable graphs
  // by composition (slot keys and batch sizes); dropped whenever a slot's buffers change
  // (a small pool, used in turn: consecutive flushes must not queue behind one another --
  // each slot's own stream already orders that slot's work from flush to flush)
  static constexpr int kLaunchStreams = 4;
  cudaStream_t launch_pool[kLaunchStreams] = {};
  cudaEvent_t launched_pool[kLaunchStreams] = {};
  int next_launch = 0;
  cudaStream_t launch = nullptr;  // the pool entry of the current flush
  cudaEvent_t launched = nullptr;
  std::map<std::string, cudaGraphExec_t> flush_graphs;
  // how often each composition has been flushed: a composition gets its single graph on its
  // second flush, so that a stream of ever-new compositions (random arrivals) never pays a
  // capture and instantiation per flush (bounded: cleared past kMaxCompositions entries)
  std::map<std::string, int> seen;
};

namespace {

std::string desc_key(const tat_plan_desc& d) { return std::string(reinterpret_cast<const char*>(&d), sizeof d); }

void CUDART_CB on_complete(void* p) {
  std::unique_ptr<Completion> c(static_cast<Completion*>(p));
  const Clock::time_point now = Clock::now();
  std::lock_guard<std::mutex> lock(c->svc->mu);
  for (long long id : c->ids) {
    Request& r = c->svc->requests[(size_t)id];
    r.done = now;
    r.completed = true;
  }
  c->svc->st.completed += (long long)c->ids.size();
}

void fail_now(tat_service_s* S, const std::vector<long long>& ids, tat_status why) {
  const Clock::time_point now = Clock::now();
  std::lock_guard<std::mutex> lock(S->mu);
  for (long long id : ids) {
    Request& r = S->requests[(size_t)id];
    r.status = why;
    r.done = now;
    r.completed = true;
  }
  S->st.completed += (long long)ids.size();
}

tat_status launch_op(const Slot& s, int b, cudaStream_t st) {
  const long long in_s = (long long)s.in_elems, out_s = (long long)s.out_elems;
  switch (s.op) {
    case TAT_OP_FORWARD: return tat_forward_batched(s.plan, b, s.in, in_s, s.out, out_s, s.ws, st);
    case TAT_OP_ADJOINT: return tat_adjoint_batched(s.plan, b, s.in, in_s, s.out, out_s, s.ws, st);
    case TAT_OP_INVERSE: return tat_inverse_batched(s.plan, b, s.in, in_s, s.out, out_s, s.ws, st);
    case TAT_OP_PAIR: {
      const long long mid_s = (long long)s.mid_elems;
      const tat_status e = tat_forward_batched(s.plan, b, s.in, in_s, s.mid, mid_s, s.ws, st);
      if (e != TAT_OK) return e;
      return tat_adjoint_batched(s.plan, b, s.mid, mid_s, s.out, out_s, s.ws, st);
    }
  }
  return TAT_ERR_INVALID_ARG;
}
tat_status launch_op(const Slot& s, int b) { return launch_op(s, b, s.stream); }

size_t slot_bytes(const Slot& s, int cap) {
  return align_up(s.in_elems * sizeof(float) * cap) + align_up(s.out_elems * sizeof(float) * cap) +
         align_up(s.mid_elems * sizeof(float) * cap) + align_up(tat_workspace_size(s.plan, cap));
}

void drop_graphs(Slot& s) {
  for (auto& g : s.graphs) cudaGraphExecDestroy(g.second);
  s.graphs.clear();
}

void drop_flush_graphs(tat_service_s* S) {
  for (auto& g : S->flush_graphs) cudaGraphExecDestroy(g.second);
  S->flush_graphs.clear();
}

void sync_launch_pool(tat_service_s* S) {
  for (cudaStream_t st : S->launch_pool)
    if (st) cudaStreamSynchronize(st);
}

void evict(tat_service_s* S, Slot& s) {
  cudaStreamSynchronize(s.stream);
  sync_launch_pool(S);
  drop_graphs(s);
  drop_flush_graphs(S);
  S->arena.release(s.off);
  s.cap = 0;
  s.in = s.out = s.mid = nullptr;
  s.ws = nullptr;
  ++S->st.evictions;
}

// Makes `s` resident with the largest batch cap <= max_batch that fits,
// evicting idle slots (least recently used first) when needed.
tat_status admit(tat_service_s* S, Slot& s) {
  if (s.cap > 0) return TAT_OK;
  for (int cap = S->cfg.max_batch; cap >= 1; cap /= 2) {
    const size_t need = slot_bytes(s, cap);
    size_t off = 0;
    bool ok = S->arena.alloc(need, &off);
    while (!ok) {
      Slot* victim = nullptr;
      for (auto& kv : S->slots) {
        Slot& o = *kv.second;
        if (&o == &s || o.cap == 0 || !o.pending.empty()) continue;
        if (!victim || o.last_use < victim->last_use) victim = &o;
      }
      if (!victim) break;
      evict(S, *victim);
      ok = S->arena.alloc(need, &off);
    }
    if (!ok) continue;
    drop_flush_graphs(S);  // the composition graphs hold the old buffer addresses
    s.off = off;
    s.bytes = need;
    s.cap = cap;
    char* p = S->arena.base + off;
    s.in = reinterpret_cast<float*>(p);
    p += align_up(s.in_elems * sizeof(float) * cap);
    s.out = reinterpret_cast<float*>(p);
    p += align_up(s.out_elems * sizeof(float) * cap);
    s.mid = s.mid_elems ? reinterpret_cast<float*>(p) : nullptr;
    p += align_up(s.mid_elems * sizeof(float) * cap);
    s.ws = p;
    return TAT_OK;
  }
  return TAT_ERR_OOM;
}

tat_status ensure_plan(tat_service_s* S, const tat_plan_desc& d, tat_plan_t* out) {
  const std::string k = desc_key(d);
  auto it = S->plans.find(k);
  if (it != S->plans.end()) {
    *out = it->second;
    return TAT_OK;
  }
  tat_plan_t p = nullptr;
  const tat_status s = tat_plan_create_ex(&p, &d);
  if (s != TAT_OK) return s;
  S->plans[k] = p;
  S->st.plans = (int)S->plans.size();
  *out = p;
  return TAT_OK;
}

tat_status run_chunk(tat_service_s* S, Slot& s, const std::vector<long long>& ids) {
  const int b = (int)ids.size();
  for (int i = 0; i < b; ++i) {
    const Request& r = S->requests[(size_t)ids[i]];
    tat_status e = cuda_ok(cudaMemcpyAsync(s.in + (size_t)i * s.in_elems, r.in, s.in_elems * sizeof(float),
                                           cudaMemcpyDefault, s.stream),
                           "staging copy");
    if (e != TAT_OK) return e;
  }
  auto g = s.graphs.find(b);
  if (g != s.graphs.end()) {
    tat_status e = cuda_ok(cudaGraphLaunch(g->second, s.stream), "graph launch");
    if (e != TAT_OK) return e;
    ++S->st.graph_launches;
  } else {
    tat_status e = launch_op(s, b);
    if (e != TAT_OK) return e;
    if (S->cfg.use_graphs) {
      // capture the same launch for the next chunk of this size (capture runs nothing)
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      if (cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const tat_status le = launch_op(s, b);
        const cudaError_t ce = cudaStreamEndCapture(s.stream, &graph);
        if (le == TAT_OK && ce == cudaSuccess && graph &&
            cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
          s.graphs[b] = exec;
        }
        if (graph) cudaGraphDestroy(graph);
      }
      cudaGetLastError();
    }
  }
  ++S->st.launches;
  for (int i = 0; i < b; ++i) {
    const Request& r = S->requests[(size_t)ids[i]];
    tat_status e = cuda_ok(cudaMemcpyAsync(r.out, s.out + (size_t)i * s.out_elems, s.out_elems * sizeof(float),
                                           cudaMemcpyDefault, s.stream),
                           "result copy");
    if (e != TAT_OK) return e;
  }
  Completion* c = new Completion{S, ids};
  const cudaError_t e = cudaLaunchHostFunc(s.stream, on_complete, c);
  if (e != cudaSuccess) {
    delete c;
    return cuda_ok(e, "host callback");
  }
  return TAT_OK;
}

// The first chunk of every ready slot as ONE launch: each slot's inputs are staged on its
// own stream, then one CUDA graph -- a parallel branch per slot (size), captured once per
// composition of slots and batch sizes and cached -- runs on the service's launch stream
// after all of them, and each slot copies its results out on its own stream after it.
// `launched` is set once the graph is on the launch stream: after that the chunks are
// this call's to finish or fail, never to be run again by the caller.
tat_status run_flush_graph(tat_service_s* S, const std::vector<Slot*>& ready,
                           const std::vector<std::vector<long long>>& chunk, bool* launched) {
  *launched = false;
  std::string key;
  for (size_t i = 0; i < ready.size(); ++i) {
    key += ready[i]->key;
    key += '#' + std::to_string(chunk[i].size()) + ';';
  }
  if (!S->flush_graphs.count(key)) {
    if (S->seen.size() > kMaxCompositions) S->seen.clear();
    if (++S->seen[key] < 2) return TAT_ERR_UNSUPPORTED;  // first sight: the per-slot path runs it
  }
  tat_status e = TAT_OK;
  const int li = S->next_launch;
  S->next_launch = (li + 1) % tat_service_s::kLaunchStreams;
  if (!S->launch_pool[li])
    e = cuda_ok(cudaStreamCreateWithFlags(&S->launch_pool[li], cudaStreamNonBlocking), "launch stream");
  if (e == TAT_OK && !S->launched_pool[li])
    e = cuda_ok(cudaEventCreateWithFlags(&S->launched_pool[li], cudaEventDisableTiming), "launch event");
  S->launch = S->launch_pool[li];
  S->launched = S->launched_pool[li];
  for (size_t i = 0; i < ready.size() && e == TAT_OK; ++i) {
    Slot& s = *ready[i];
    if (!s.branch) e = cuda_ok(cudaStreamCreateWithFlags(&s.branch, cudaStreamNonBlocking), "branch stream");
    if (e == TAT_OK && !s.staged)
      e = cuda_ok(cudaEventCreateWithFlags(&s.staged, cudaEventDisableTiming), "staging event");
    for (size_t k = 0; k < chunk[i].size() && e == TAT_OK; ++k) {
      const Request& r = S->requests[(size_t)chunk[i][k]];
      e = cuda_ok(cudaMemcpyAsync(s.in + k * s.in_elems, r.in, s.in_elems * sizeof(float), cudaMemcpyDefault,
                                  s.stream),
                  "staging copy");
    }
    if (e == TAT_OK) e = cuda_ok(cudaEventRecord(s.staged, s.stream), "staging event");
    if (e == TAT_OK) e = cuda_ok(cudaStreamWaitEvent(S->launch, s.staged, 0), "launch wait");
  }
  if (e != TAT_OK) return e;
  auto it = S->flush_graphs.find(key);
  if (it == S->flush_graphs.end()) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join(ready.size(), nullptr);
    bool ok = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    for (auto& j : join) ok = ok && cudaEventCreateWithFlags(&j, cudaEventDisableTiming) == cudaSuccess;
    if (ok && cudaStreamBeginCapture(S->launch, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      tat_status le = cudaEventRecord(fork, S->launch) == cudaSuccess ? TAT_OK : TAT_ERR_CUDA;
      for (size_t i = 0; i < ready.size() && le == TAT_OK; ++i) {
        Slot& s = *ready[i];
        if (cudaStreamWaitEvent(s.branch, fork, 0) != cudaSuccess) le = TAT_ERR_CUDA;
        if (le == TAT_OK) le = launch_op(s, (int)chunk[i].size(), s.branch);
        if (le == TAT_OK && cudaEventRecord(join[i], s.branch) != cudaSuccess) le = TAT_ERR_CUDA;
        if (le == TAT_OK && cudaStreamWaitEvent(S->launch, join[i], 0) != cudaSuccess) le = TAT_ERR_CUDA;
      }
      const cudaError_t ce = cudaStreamEndCapture(S->launch, &graph);
      ok = le == TAT_OK && ce == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    } else {
      ok = false;
    }
    if (graph) cudaGraphDestroy(graph);
    if (fork) cudaEventDestroy(fork);
    for (auto& j : join)
      if (j) cudaEventDestroy(j);
    cudaGetLastError();
    if (!ok) {
      if (exec) cudaGraphExecDestroy(exec);
      return TAT_ERR_CUDA;
    }
    it = S->flush_graphs.emplace(key, exec).first;
  }
  e = cuda_ok(cudaGraphLaunch(it->second, S->launch), "flush graph launch");
  if (e != TAT_OK) return e;
  *launched = true;
  ++S->st.flush_graphs;
  S->st.launches += (long long)ready.size();
  const tat_status le = cuda_ok(cudaEventRecord(S->launched, S->launch), "launch event");
  tat_status first = TAT_OK;
  for (size_t i = 0; i < ready.size(); ++i) {
    Slot& s = *ready[i];
    e = le;
    if (e == TAT_OK) e = cuda_ok(cudaStreamWaitEvent(s.stream, S->launched, 0), "result wait");
    for (size_t k = 0; k < chunk[i].size() && e == TAT_OK; ++k) {
      const Request& r = S->requests[(size_t)chunk[i][k]];
      e = cuda_ok(cudaMemcpyAsync(r.out, s.out + k * s.out_elems, s.out_elems * sizeof(float), cudaMemcpyDefault,
                                  s.stream),
                  "result copy");
    }
    if (e == TAT_OK) {
      Completion* c = new Completion{S, chunk[i]};
      const cudaError_t ce = cudaLaunchHostFunc(s.stream, on_complete, c);
      if (ce != cudaSuccess) {
        delete c;
        e = cuda_ok(ce, "host callback");
      }
    }
    if (e != TAT_OK) {  // this slot's requests fail; the other slots still complete
      cudaStreamSynchronize(s.stream);
      fail_now(S, chunk[i], e);
      if (first == TAT_OK) first = e;
    }
  }
  return first;
}

}  // namespace

extern "C" {

tat_status tat_service_config_default(tat_service_config* cfg) {
  if (!cfg) return TAT_ERR_INVALID_ARG;
  cfg->memory_budget = (size_t)8 << 30;
  cfg->max_batch = 32;
  cfg->use_graphs = 1;
  cfg->autotune = 0;
  cfg->one_graph = 1;
  return TAT_OK;
}

tat_status tat_service_create(tat_service_t* svc, const tat_service_config* cfg) {
  if (!svc) return TAT_ERR_INVALID_ARG;
  *svc = nullptr;
  if (!cfg || cfg->max_batch < 1 || cfg->memory_budget < kAlign) return TAT_ERR_INVALID_ARG;
  auto* S = new (std::nothrow) tat_service_s();
  if (!S) return TAT_ERR_OOM;
  S->cfg = *cfg;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return TAT_ERR_CUDA;
  }
  S->arena.size = cfg->memory_budget / kAlign * kAlign;
  void* p = nullptr;
  const tat_status e = cuda_ok(cudaMalloc(&p, S->arena.size), "arena allocation");
  if (e != TAT_OK) {
    delete S;
    return e;
  }
  S->arena.base = static_cast<char*>(p);
  S->st.arena_bytes = S->arena.size;
  *svc = S;
  return TAT_OK;
}

tat_status tat_service_destroy(tat_service_t S) {
  if (!S) return TAT_ERR_INVALID_ARG;
  sync_launch_pool(S);
  drop_flush_graphs(S);
  for (auto& kv : S->slots) {
    Slot& s = *kv.second;
    if (s.stream) cudaStreamSynchronize(s.stream);
    drop_graphs(s);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.branch) cudaStreamDestroy(s.branch);
    if (s.staged) cudaEventDestroy(s.staged);
  }
  for (int i = 0; i < tat_service_s::kLaunchStreams; ++i) {
    if (S->launch_pool[i]) cudaStreamDestroy(S->launch_pool[i]);
    if (S->launched_pool[i]) cudaEventDestroy(S->launched_pool[i]);
  }
  for (auto& kv : S->plans) tat_plan_destroy(kv.second);
  cudaFree(S->arena.base);
  delete S;
  return TAT_OK;
}

tat_status tat_service_submit(tat_service_t S, const tat_plan_desc* desc, tat_op op, const float* in, float* out,
                              long long* id) {
  if (!S || !desc || !in || !out || !id) return TAT_ERR_INVALID_ARG;
  if (op != TAT_OP_FORWARD && op != TAT_OP_ADJOINT && op != TAT_OP_INVERSE && op != TAT_OP_PAIR)
    return TAT_ERR_INVALID_ARG;
  tat_plan_info info;
  const tat_status q = tat_plan_query(desc, &info);
  if (q != TAT_OK) return q;
  std::string key = desc_key(*desc);
  key.push_back((char)op);
  auto& slot = S->slots[key];
  if (!slot) {
    slot.reset(new Slot());
    slot->key = key;
    slot->op = op;
    const size_t img = (size_t)desc->n * desc->n, dat = (size_t)desc->n_det * desc->n_t;
    slot->in_elems = op == TAT_OP_FORWARD || op == TAT_OP_PAIR ? img : dat;
    slot->out_elems = op == TAT_OP_FORWARD ? dat : img;
    slot->mid_elems = op == TAT_OP_PAIR ? dat : 0;
  }
  Request r;
  r.id = (long long)S->requests.size();
  r.in = in;
  r.out = out;
  r.submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->requests.push_back(r);
  }
  slot->pending.push_back(r.id);
  ++S->st.requests;
  *id = r.id;
  return TAT_OK;
}

namespace {
// Runs the pending requests of the prepared slots `ready` and clears them: with one_graph,
// the first chunk of every slot as one graph launch; the rest (and everything, without it)
// chunk by chunk on the slots' own streams.
void run_ready(tat_service_t S, std::vector<Slot*>& ready, tat_status* first_error) {
  size_t skip_first = 0;
  // (a flush of one slot is one graph launch on that slot's stream anyway)
  if (S->cfg.one_graph && S->cfg.use_graphs && ready.size() >= 2) {
    std::vector<std::vector<long long>> chunk(ready.size());
    for (size_t i = 0; i < ready.size(); ++i) {
      Slot& s = *ready[i];
      const size_t j = std::min(s.pending.size(), (size_t)s.cap);
      chunk[i].assign(s.pending.begin(), s.pending.begin() + (long)j);
    }
    bool launched = false;
    const tat_status e = run_flush_graph(S, ready, chunk, &launched);
    if (launched) skip_first = 1;
    if (e != TAT_OK && launched && *first_error == TAT_OK) *first_error = e;
  }
  for (Slot* sp : ready) {
    Slot& s = *sp;
    for (size_t i = skip_first * (size_t)s.cap; i < s.pending.size(); i += (size_t)s.cap) {
      const size_t j = std::min(s.pending.size(), i + (size_t)s.cap);
      std::vector<long long> ids(s.pending.begin() + (long)i, s.pending.begin() + (long)j);
      const tat_status e = run_chunk(S, s, ids);
      if (e != TAT_OK) {
        fail_now(S, ids, e);
        if (*first_error == TAT_OK) *first_error = e;
      }
    }
    s.pending.clear();
  }
  ready.clear();
}
}  // namespace

tat_status tat_service_flush(tat_service_t S) {
  if (!S) return TAT_ERR_INVALID_ARG;
  tat_status first_error = TAT_OK;
  std::vector<Slot*> ready;  // slots with pending requests, plan and buffers in place
  for (auto& kv : S->slots) {
    Slot& s = *kv.second;
    if (s.pending.empty()) continue;
    s.last_use = ++S->tick;
    tat_plan_desc d;
    std::memcpy(&d, s.key.data(), sizeof d);
    tat_status e = s.plan ? TAT_OK : ensure_plan(S, d, &s.plan);
    if (e == TAT_OK && !s.stream) e = cuda_ok(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking), "stream");
    if (e == TAT_OK) e = admit(S, s);
    if (e == TAT_ERR_OOM && !ready.empty()) {
      // the slots prepared so far hold the memory: run them now (they become evictable once
      // their requests are issued) and admit this one after them
      run_ready(S, ready, &first_error);
      e = admit(S, s);
    }
    if (e == TAT_OK && S->cfg.autotune && !s.tuned && s.op != TAT_OP_INVERSE) {
      // tune on zeroed slot buffers at the slot's batch size (the knobs belong to the plan)
      const tat_plan_desc& pd = d;
      const size_t img = (size_t)pd.n * pd.n, dat = (size_t)pd.n_det * pd.n_t;
      float* fbuf = s.op == TAT_OP_ADJOINT ? s.out : s.in;
      float* gbuf = s.op == TAT_OP_PAIR ? s.mid : (s.op == TAT_OP_FORWARD ? s.out : s.in);
      cudaMemsetAsync(fbuf, 0, img * sizeof(float) * s.cap, s.stream);
      cudaMemsetAsync(gbuf, 0, dat * sizeof(float) * s.cap, s.stream);
      e = tat_plan_autotune(s.plan, s.cap, fbuf, gbuf, fbuf, s.ws, s.stream, nullptr, nullptr, nullptr, nullptr,
                            nullptr);
      drop_graphs(s);
      drop_flush_graphs(S);
      s.tuned = true;
    }
    if (e != TAT_OK) {
      fail_now(S, s.pending, e);
      s.pending.clear();
      if (first_error == TAT_OK) first_error = e;
      continue;
    }
    ready.push_back(&s);
  }
  run_ready(S, ready, &first_error);
  S->st.slots = 0;
  for (auto& kv : S->slots) S->st.slots += kv.second->cap > 0 ? 1 : 0;
  S->st.peak_bytes = S->arena.peak;
  return first_error;
}

tat_status tat_service_synchronize(tat_service_t S) {
  if (!S) return TAT_ERR_INVALID_ARG;
  tat_status r = TAT_OK;
  for (cudaStream_t st : S->launch_pool)
    if (st && r == TAT_OK) r = cuda_ok(cudaStreamSynchronize(st), "synchronize");
  for (auto& kv : S->slots)
    if (kv.second->stream) {
      const tat_status e = cuda_ok(cudaStreamSynchronize(kv.second->stream), "synchronize");
      if (r == TAT_OK) r = e;
    }
  return r;
}

tat_status tat_service_latency(tat_service_t S, long long id, double* ms, tat_status* status) {
  if (!S || !ms || id < 0) return TAT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  if ((size_t)id >= S->requests.size()) return TAT_ERR_INVALID_ARG;
  const Request& r = S->requests[(size_t)id];
  if (!r.completed) return TAT_ERR_INVALID_ARG;
  *ms = std::chrono::duration<double, std::milli>(r.done - r.submitted).count();
  if (status) *status = r.status;
  return TAT_OK;
}

tat_status tat_service_get_stats(tat_service_t S, tat_service_stats* out) {
  if (!S || !out) return TAT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  *out = S->st;
  out->peak_bytes = S->arena.peak;
  return TAT_OK;
}

tat_status tat_plan_set_launch_shape(tat_plan_t plan, int strip, int row_pairs, int cols_threads, int row_threads) {
  if (!plan || strip < 1 || row_pairs < 1 || cols_threads < 32 || row_threads < 0) return TAT_ERR_INVALID_ARG;
  const tat::LaunchCfg old = plan->cfg;
  plan->cfg.strip = strip;
  plan->cfg.rows_pairs = row_pairs;
  plan->cfg.cols_threads = cols_threads;
  if (row_threads > 0) plan->cfg.nt_rows = row_threads;
  if (row_pairs * plan->cfg.nt_rows > 1024 || tat::validate_shapes(plan) != TAT_OK) {
    plan->cfg = old;
    return TAT_ERR_UNSUPPORTED;
  }
  return TAT_OK;
}

}  // extern "C"

namespace {
// Selects the pass order of the length-2M transform: its tables and thread count with it.
void apply_order_2M(tat_plan_t plan, int order) {
  plan->cfg.order_2M = order;
  plan->cfg.nt_2M = plan->nt_2M_v[order];
  plan->d.f2M = plan->f2M_v[order];
}
}  // namespace

extern "C" {

tat_status tat_plan_set_fft_order(tat_plan_t plan, int order) {
  if (!plan || (order != 0 && order != 1)) return TAT_ERR_INVALID_ARG;
  const int old = plan->cfg.order_2M;
  apply_order_2M(plan, order);
  if (tat::validate_shapes(plan) != TAT_OK) {
    apply_order_2M(plan, old);
    return TAT_ERR_UNSUPPORTED;
  }
  return TAT_OK;
}

tat_status tat_plan_get_fft_order(tat_plan_t plan, int* order) {
  if (!plan || !order) return TAT_ERR_INVALID_ARG;
  *order = plan->cfg.order_2M;
  return TAT_OK;
}

tat_status tat_plan_set_column_split(tat_plan_t plan, int mask) {
  if (!plan || mask < 0 || mask > 3) return TAT_ERR_INVALID_ARG;
  const int old = plan->cfg.cols_split;
  plan->cfg.cols_split = mask;
  if (tat::validate_shapes(plan) != TAT_OK) {
    plan->cfg.cols_split = old;
    return TAT_ERR_UNSUPPORTED;
  }
  return TAT_OK;
}

tat_status tat_plan_get_column_split(tat_plan_t plan, int* mask) {
  if (!plan || !mask) return TAT_ERR_INVALID_ARG;
  *mask = plan->cfg.cols_split;
  return TAT_OK;
}

tat_status tat_plan_autotune(tat_plan_t plan, int batch, float* f, float* g, float* f_out, void* workspace,
                             tat_stream_t stream, double* ms_best, int* strip_out, int* rp_out, int* cols_threads_out,
                             int* row_threads_out) {
  if (!plan || batch < 1 || !f || !g || !f_out || !workspace) return TAT_ERR_INVALID_ARG;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const tat::LaunchCfg base = plan->cfg;
  const long long fs = (long long)plan->d.n * plan->d.n, gs = (long long)plan->d.n_det * plan->d.n_t;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return TAT_ERR_CUDA;
  }
  tat::LaunchCfg best = base;
  float best_ms = 1e30f;
  tat_status err = TAT_OK;
  // Times plan->cfg on one pair (after one warm-up pair); keeps it when it is the fastest so far.
  auto trial = [&]() {
    if (tat::validate_shapes(plan) != TAT_OK) return;
    float ms = 0.f;
    for (int rep = 0; rep < 3 && err == TAT_OK; ++rep) {
      cudaEventRecord(e0, st);
      err = tat::launch_forward(plan, batch, f, fs, g, gs, workspace, st);
      if (err == TAT_OK) err = tat::launch_adjoint(plan, batch, g, gs, f_out, fs, workspace, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) err = TAT_ERR_CUDA;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0) ms += t;  // first repetition is the warm-up
    }
    if (err == TAT_OK && ms / 2.f < best_ms) {
      best_ms = ms / 2.f;
      best = plan->cfg;
    }
  };
  for (int strip : {2, 4, 8, 16, 32})
    for (int rp : {1, 2, 4}) {
      if (err != TAT_OK) break;
      plan->cfg = base;
      plan->cfg.strip = strip;
      plan->cfg.rows_pairs = rp;
      if (rp * plan->cfg.nt_rows <= 1024) trial();
    }
  // then smaller column CTAs for the chosen strip and row pairs (more of them per SM, where the
  // four-step column FFT keeps fewer than 256 threads busy), and strips around the chosen one;
  // not when both column stages of the pair run the split transform, whose CTA size is fixed
  // (the knob would change nothing the pair times, only A^-1's four-step column stage)
  const tat::LaunchCfg first = best;
  const int N = plan->d.N;
  const bool split_ok = (N == 512 || N == 1024 || N == 2048 || N == 4096 || N == 8192) &&
                        plan->d.n <= (N == 8192 ? 1024 : 512);
  const bool pair_split = split_ok && (first.cols_split & 3) == 3;
  for (int threads : {64, 128, 384})
    for (int strip : {first.strip / 2, first.strip, first.strip * 2}) {
      if (err != TAT_OK || pair_split || strip < 2 || strip > 32 || threads == first.cols_threads) continue;
      plan->cfg = first;
      plan->cfg.cols_threads = threads;
      plan->cfg.strip = strip;
      trial();
    }
  // then fewer threads per row pair (more pairs per CTA) for the four-step lengths up to 1024
  const tat::LaunchCfg second = best;
  if (plan->d.N <= 1024)
    for (int threads : {64, 128})
      for (int rp : {second.rows_pairs, 2 * second.rows_pairs, 4 * second.rows_pairs}) {
        if (err != TAT_OK || threads >= second.nt_rows || rp * threads > 1024) continue;
        plan->cfg = second;
        plan->cfg.nt_rows = threads;
        plan->cfg.rows_pairs = rp;
        trial();
      }
  // and the stages with and without programmatic dependent launch
  if (err == TAT_OK) {
    plan->cfg = best;
    plan->cfg.pdl = !best.pdl;
    trial();
  }
  // and the other pass order of the cosine/sine stages' length-2M FFT (radix-3 passes first
  // or last), which moves the zero band of the extension and the kept outputs between passes
  if (err == TAT_OK) {
    plan->cfg = best;
    apply_order_2M(plan, 1 - best.order_2M);
    trial();
  }
  // and the other column transforms where both exist (N = 512 .. 8192 with few enough rows),
  // with the best strip among its neighbours and, where a column stage then runs the
  // four-step transform, each of the column CTA sizes
  if (err == TAT_OK && split_ok) {
    const tat::LaunchCfg third = best;
    for (int split = 0; split < 4; ++split)
      for (int strip : {third.strip / 2, third.strip, third.strip * 2})
        for (int threads : {64, 128, 256, 384}) {
          if (err != TAT_OK || split == third.cols_split || strip < 2 || strip > 32) continue;
          if (split == 3 ? threads != third.cols_threads : threads == 384 && N <= 1024) continue;
          plan->cfg = third;
          apply_order_2M(plan, third.order_2M);
          plan->cfg.cols_split = split;
          plan->cfg.strip = strip;
          plan->cfg.cols_threads = threads;
          trial();  // skips shapes the kernels do not take
        }
  }
  plan->cfg = err == TAT_OK ? best : base;
  apply_order_2M(plan, plan->cfg.order_2M);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != TAT_OK) return err;
  if (ms_best) *ms_best = best_ms;
  if (strip_out) *strip_out = best.strip;
  if (rp_out) *rp_out = best.rows_pairs;
  if (cols_threads_out) *cols_threads_out = best.cols_threads;
  if (row_threads_out) *row_threads_out = best.nt_rows;
  return TAT_OK;
}

}  // extern "C"
