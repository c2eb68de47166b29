// batch.cu -- launch-shape autotuner and batched (mixed-model) ensembles under one CUDA graph.
//
// Uneven ensembles make lanes of a warp finish at different times (adaptive stepping, Sec.
// 6.4; mixed stiff / non-stiff / SDE work).  Within one (model, method) the persistent
// schedule refills idle lanes; across models the batch runs one persistent kernel per
// sub-problem, each with its own register budget, on forked streams captured into a single
// CUDA graph, so one graph launch solves the whole batch and a kernel's tail overlaps with
// the next kernels instead of leaving SMs idle between separate launches.  The autotuner
// times candidate block sizes and trajectories-per-thread on the caller's own inputs (the
// kernel-occupancy tuning the paper leaves to KernelAbstractions, Sec. 5.1) and remembers
// the winner per (model, method, precision, layout, size class, SM count).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ens_internal.h"

namespace ens {

namespace {

bool fixed_method(int alg) {
  return alg == ENS_TSIT5_FIXED || alg == ENS_RK4 || alg == ENS_EM || alg == ENS_SIEA;
}

typedef std::tuple<int, int, int, int, int, int, int> TuneKey;
std::map<TuneKey, LaunchCfg> g_tuned;
std::mutex g_tuned_mu;

TuneKey tune_key(int rhs_id, long long N, const ens_opts* o, int sms) {
  int nbits = 0;
  while (nbits < 62 && (1LL << (nbits + 1)) <= N) ++nbits;  // size class floor(log2 N)
  // output kind: final state, save times (cut steps or dense), every-step record -- they run
  // different kernels (the paired one only for the final state)
  const int kind = o->step_cap > 0 ? 3 : o->n_save > 0 ? (o->dense ? 2 : 1) : 0;
  return TuneKey(rhs_id, o->alg, o->dtype, o->layout, nbits, kind, sms);
}

LaunchCfg default_launch(const ens_opts* o, int sms) {
  LaunchCfg c;
  c.schedule = o->schedule;
  if (c.schedule == ENS_SCHED_AUTO)
    c.schedule = fixed_method(o->alg) ? ENS_SCHED_DIRECT : ENS_SCHED_PERSISTENT;
  c.block = o->block ? o->block : 128;
  c.tpt = o->tpt ? o->tpt : 1;
  c.num_sms = sms;
  c.bps = o->blocks_per_sm;
  return c;
}

}  // namespace

// fixed-step Tsit5 / RK4 problems the paired direct kernel serves (FP32, final state only,
// autonomous models without events)
static bool fixed_pairs(int rhs_id, const ens_opts* o) {
  return (o->alg == ENS_TSIT5_FIXED || o->alg == ENS_RK4) && o->dtype == ENS_F32 &&
         o->n_save == 0 &&
         (rhs_id == ENS_RHS_LORENZ || rhs_id == ENS_RHS_ROBERTSON || rhs_id == ENS_RHS_GBM ||
          rhs_id == ENS_RHS_OREGO);
}

LaunchCfg resolve_launch(int rhs_id, long long N, const ens_opts* o, int num_sms) {
  LaunchCfg c = default_launch(o, num_sms);
  // the paired fixed-step kernel is the default where it applies (faster at every block size
  // measured: 3.42 against 4.10 ms on 2^20 Lorenz trajectories, 1,000 steps)
  if (!o->tpt && c.schedule == ENS_SCHED_DIRECT && fixed_pairs(rhs_id, o)) c.tpt = 2;
  if (o->block == 0 && o->tpt == 0 && o->blocks_per_sm == 0) {
    std::lock_guard<std::mutex> lock(g_tuned_mu);
    auto it = g_tuned.find(tune_key(rhs_id, N, o, num_sms));
    if (it != g_tuned.end() && (o->schedule == ENS_SCHED_AUTO ||
                                o->schedule == it->second.schedule)) {
      c = it->second;
      c.num_sms = num_sms;
    }
  }
  return c;
}

bool one_per_thread(const ens_opts* o) {
  return o->alg == ENS_ROS23 || o->alg == ENS_RODAS4 || o->alg == ENS_RODAS5P ||
         (o->alg == ENS_TSIT5_ADAPTIVE && ((o->dense && o->n_save > 0) || o->step_cap > 0));
}

// Time every candidate launch shape of one solve (the solve really runs and writes its
// outputs) and record the fastest in the tuning cache.  Synchronises the stream.
int tune_problem(int rhs_id, const ens_opts* o, const SolveArgs& a, const SolveScratch& sc,
                 int sms, cudaStream_t s, LaunchCfg* best, float* best_ms) {
  const LaunchCfg base = default_launch(o, sms);
  std::vector<LaunchCfg> cand;
  const int blocks[] = {64, 128, 256, 512};
  for (int b : blocks) {
    if (o->block && b != o->block) continue;
    if (base.schedule == ENS_SCHED_DIRECT) {
      for (int t : {1, 2}) {  // two per thread: the paired fixed-step kernel, where it applies
        if (o->tpt && t != o->tpt) continue;
        if (t == 2 && !o->tpt && !fixed_pairs(rhs_id, o)) continue;
        LaunchCfg c = base;
        c.block = b;
        c.tpt = t;
        cand.push_back(c);
      }
    } else {
      for (int t : {1, 2}) {
        if (o->tpt && t != o->tpt) continue;
        // Rosenbrock23 and the dense-output / step-record Tsit5 kernels run one trajectory
        // per thread whatever is asked: tpt 2 would repeat tpt 1
        if (t == 2 && !o->tpt && one_per_thread(o)) continue;
        for (int f : {0, -3, -2}) {  // all resident blocks that fit, 3/4, 1/2 of them
          if (o->blocks_per_sm && f != 0) continue;
          LaunchCfg c = base;
          c.block = b;
          c.tpt = t;
          if (!o->blocks_per_sm) c.bps = f;
          cand.push_back(c);
        }
      }
    }
  }
  if (cand.empty()) cand.push_back(base);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return set_last_error(ENS_ECUDA, "event create");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_last_error(ENS_ECUDA, "event create");
  }
  int rc = ENS_OK;
  float bms = 1e30f;
  LaunchCfg bc = base;
  for (const LaunchCfg& c : cand) {
    float tmin = 1e30f;
    for (int rep = 0; rep < 3 && rc == ENS_OK; ++rep) {  // one warm-up, two timed runs
      bool sup = false;
      cudaEventRecord(e0, s);
      cudaError_t e = enqueue_solve(rhs_id, o, a, c, sc, s, &sup);
      cudaEventRecord(e1, s);
      if (e == cudaErrorLaunchOutOfResources || e == cudaErrorInvalidConfiguration) {
        // this block size does not fit the kernel's registers / shared memory: not a candidate
        cudaEventSynchronize(e1);
        tmin = 1e30f;
        break;
      }
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (!sup) rc = set_last_error(ENS_ENOTSUP, "algorithm not available for this model");
      else if (e != cudaSuccess) rc = set_last_error(ENS_ECUDA, cudaGetErrorString(e));
      float ms = 0.f;
      if (rc == ENS_OK && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        tmin = std::min(tmin, ms);
    }
    if (rc != ENS_OK) break;
    if (tmin < bms) {
      bms = tmin;
      bc = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != ENS_OK) return rc;
  if (bms >= 1e30f) return set_last_error(ENS_ECUDA, "no launch shape fits this kernel");
  {
    std::lock_guard<std::mutex> lock(g_tuned_mu);
    g_tuned[tune_key(rhs_id, a.N, o, sms)] = bc;
  }
  *best = bc;
  *best_ms = bms;
  return ENS_OK;
}

}  // namespace ens

using namespace ens;

// ============================================================================ batch plans
struct ens_batch {
  struct Item {
    int rhs_id;
    ens_opts o;
    SolveArgs a;
    LaunchCfg cfg;
    SolveScratch sc;
    float tuned_ms;
    cudaStream_t st;
    cudaEvent_t done;
    int slot;      // kind of the fused kernel (mixed_slot), -1: none
    LaunchCfg fcfg;  // its shape inside the fused kernel (persistent, block 128)
  };
  std::vector<Item> items;
  std::vector<int> order;  // launch order (longest measured first when tuned)
  float graph_ms[3];       // measured graph times: concurrent, serial, fused (0: not measured)
  bool fusable;            // the items fit the fused kernel
  int fblock;              // the fused kernel's block size
  int sms;
  unsigned long long* slots;  // device: per item, the lane slots its persistent loops issued
  void* scratch;
  cudaStream_t cap;
  cudaEvent_t fork;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int flags;
  int device;
};

namespace {

int batch_fail(ens_batch* b, int code, const char* msg);

cudaError_t enqueue_batch(ens_batch* b, cudaStream_t s, bool* sup) {
  *sup = true;
  cudaError_t e0 =
      cudaMemsetAsync(b->slots, 0, sizeof(unsigned long long) * b->items.size(), s);
  if (e0 != cudaSuccess) return e0;
  if (b->flags & ENS_BATCH_FUSED) {
    // every item's ordering pass and queue reset, then the one kernel over all of them
    const SolveArgs* by_slot[3] = {nullptr, nullptr, nullptr};
    int order[3], n = 0;
    for (int i : b->order) {
      ens_batch::Item& it = b->items[i];
      SolveArgs a = it.a;
      cudaError_t e = prepare_solve(it.rhs_id, &it.o, &a, it.fcfg, it.sc, s);
      if (e != cudaSuccess) return e;
      it.a.order = a.order;  // the prepared arguments (queue, order) stay with the item
      it.a.queue = a.queue;
      by_slot[it.slot] = &it.a;
      order[n++] = it.slot;
    }
    return launch_mixed(by_slot, order, n, b->fblock, b->sms, s);
  }
  if (b->flags & ENS_BATCH_SERIAL) {
    for (int i : b->order) {
      ens_batch::Item& it = b->items[i];
      cudaError_t e = enqueue_solve(it.rhs_id, &it.o, it.a, it.cfg, it.sc, s, sup);
      if (e != cudaSuccess || !*sup) return e;
    }
    return cudaSuccess;
  }
  cudaError_t e = cudaEventRecord(b->fork, s);
  for (int i : b->order) {
    if (e != cudaSuccess) return e;
    ens_batch::Item& it = b->items[i];
    e = cudaStreamWaitEvent(it.st, b->fork, 0);
    if (e == cudaSuccess) e = enqueue_solve(it.rhs_id, &it.o, it.a, it.cfg, it.sc, it.st, sup);
    if (!*sup) return e;
    if (e == cudaSuccess) e = cudaEventRecord(it.done, it.st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, it.done, 0);
  }
  return e;
}

void batch_free(ens_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto& it : b->items) {
    if (it.st) cudaStreamDestroy(it.st);
    if (it.done) cudaEventDestroy(it.done);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->scratch) cudaFree(b->scratch);
  delete b;
}

int batch_fail(ens_batch* b, int code, const char* msg) {
  batch_free(b);
  return set_last_error(code, msg);
}

// capture the plan's launches (concurrent or serial by b->flags) into an instantiated graph
int capture_graph(ens_batch* b, cudaGraph_t* g, cudaGraphExec_t* x) {
  *g = nullptr;
  *x = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));
  bool sup = true;
  cudaError_t e1 = enqueue_batch(b, b->cap, &sup);
  e = cudaStreamEndCapture(b->cap, g);
  if (!sup) return set_last_error(ENS_ENOTSUP, "algorithm not available for this model");
  if (e1 != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e1));
  if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));
  e = cudaGraphInstantiate(x, *g, 0);
  if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));
  return ENS_OK;
}

// one warm-up launch, then the median of three timed launches (ms); synchronises s
int time_graph(cudaGraphExec_t x, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return set_last_error(ENS_ECUDA, "event create");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_last_error(ENS_ECUDA, "event create");
  }
  float t[3] = {0.f, 0.f, 0.f};
  cudaError_t e = cudaGraphLaunch(x, s);
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(x, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t[r], e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));
  std::sort(t, t + 3);
  *ms = t[1];
  return ENS_OK;
}

}  // namespace

extern "C" {

int ens_batch_create(ens_batch** out, const ens_batch_item* items, int n_items, int flags,
                     void* cuda_stream) {
  if (!out) return set_last_error(ENS_EINVAL, "null output pointer");
  *out = nullptr;
  if (n_items < 1 || n_items > ENS_BATCH_MAX_ITEMS || !items)
    return set_last_error(ENS_EINVAL, "n_items must be in [1, ENS_BATCH_MAX_ITEMS]");
  if (flags & ~(ENS_BATCH_GRAPH | ENS_BATCH_AUTOTUNE | ENS_BATCH_SERIAL | ENS_BATCH_FUSED))
    return set_last_error(ENS_EINVAL, "unknown flags");
  if ((flags & ENS_BATCH_SERIAL) && (flags & ENS_BATCH_FUSED))
    return set_last_error(ENS_EINVAL, "ENS_BATCH_SERIAL and ENS_BATCH_FUSED exclude each other");
  for (int i = 0; i < n_items; ++i) {
    const ens_batch_item& it = items[i];
    int rc = validate_problem(it.rhs_id, it.N, it.params, it.u0, it.tspan, &it.opts, it.out);
    if (rc) return rc;
  }
  ens_batch* b = new ens_batch();
  b->scratch = nullptr;
  b->cap = nullptr;
  b->fork = nullptr;
  b->graph = nullptr;
  b->exec = nullptr;
  b->slots = nullptr;
  b->flags = flags;
  int sms = 0;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) return batch_fail(b, ENS_ECUDA, cudaGetErrorString(e));
  b->sms = sms;
  b->fblock = 64;  // 110 registers: 9 blocks of 64 (18 warps) per SM against 4 of 128
  // the fused kernel takes at most one item of each of its kinds, none of them empty
  {
    int seen = 0;
    b->fusable = true;
    for (int i = 0; i < n_items; ++i) {
      const int k = mixed_slot(items[i].rhs_id, &items[i].opts);
      if (k < 0 || (seen & (1 << k)) || items[i].N == 0) b->fusable = false;
      if (k >= 0) seen |= 1 << k;
    }
  }
  if ((flags & ENS_BATCH_FUSED) && !b->fusable) {
    delete b;
    return set_last_error(ENS_ENOTSUP,
                          "ENS_BATCH_FUSED takes at most one each of Lorenz FP32 adaptive "
                          "Tsit5, Robertson FP32 Rosenbrock23 and GBM FP32 Euler-Maruyama, "
                          "without save times or step records");
  }
  // one scratch block: per item a 256-byte queue slot, the bucket cursors, order, keys and
  // the starting steps the ordering pre-pass keeps (8 bytes a trajectory)
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  std::vector<size_t> off(n_items);
  size_t total = 0;
  for (int i = 0; i < n_items; ++i) {
    off[i] = total;
    const long long N = items[i].N;
    total += 256 + up(4 * (size_t)kCostHistWords) + up(4 * (size_t)N) + up(2 * (size_t)N) +
             up(8 * (size_t)N);
  }
  const size_t slots_off = total;
  total += up(sizeof(unsigned long long) * n_items);
  if (cudaMalloc(&b->scratch, total) != cudaSuccess)
    return batch_fail(b, ENS_ENOMEM, "batch scratch");
  b->slots = (unsigned long long*)((char*)b->scratch + slots_off);
  b->items.resize(n_items);
  for (int i = 0; i < n_items; ++i) {
    const ens_batch_item& src = items[i];
    ens_batch::Item& it = b->items[i];
    std::memset(&it, 0, sizeof(it));
    it.rhs_id = src.rhs_id;
    it.o = src.opts;
    fill_solve_args(&it.a, src.N, src.params, src.u0, src.tspan, &src.opts, src.out, src.status,
                    src.stats);
    it.o.saveat = nullptr;  // the save times now live in it.a (copied); the plan keeps no
                            // pointer into the caller's host memory
    it.o.kernel_start = it.o.kernel_stop = nullptr;  // no timing events inside a plan
    it.cfg = resolve_launch(src.rhs_id, src.N, &src.opts, sms);
    it.a.slots = b->slots + i;
    it.slot = mixed_slot(src.rhs_id, &src.opts);
    it.fcfg = LaunchCfg{};
    it.fcfg.schedule = ENS_SCHED_PERSISTENT;
    it.fcfg.block = 128;
    it.fcfg.tpt = 1;
    it.fcfg.num_sms = sms;
    char* base = (char*)b->scratch + off[i];
    it.sc.queue = (unsigned long long*)base;
    it.sc.hist = (unsigned int*)(base + 256);
    it.sc.order = (int*)(base + 256 + up(4 * (size_t)kCostHistWords));
    it.sc.bucket = (unsigned short*)(base + 256 + up(4 * (size_t)kCostHistWords) +
                                     up(4 * (size_t)src.N));
    it.sc.h0 = base + 256 + up(4 * (size_t)kCostHistWords) + up(4 * (size_t)src.N) +
               up(2 * (size_t)src.N);
    if (cudaStreamCreateWithFlags(&it.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&it.done, cudaEventDisableTiming) != cudaSuccess)
      return batch_fail(b, ENS_ECUDA, "stream / event creation");
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return batch_fail(b, ENS_ECUDA, "stream / event creation");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (flags & ENS_BATCH_AUTOTUNE) {
    for (int i = 0; i < n_items; ++i) {
      ens_batch::Item& it = b->items[i];
      if (it.a.N == 0) continue;
      // the trial solves need the save times in the options only for the cache key
      ens_opts o = items[i].opts;
      o.kernel_start = o.kernel_stop = nullptr;
      int rc = tune_problem(it.rhs_id, &o, it.a, it.sc, sms, s, &it.cfg, &it.tuned_ms);
      if (rc) {
        batch_free(b);
        return rc;
      }
    }
  }
  b->order.resize(n_items);
  for (int i = 0; i < n_items; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    return b->items[x].tuned_ms > b->items[y].tuned_ms;  // longest first (ties: input order)
  });
  // items with no trajectories launch nothing
  b->order.erase(std::remove_if(b->order.begin(), b->order.end(),
                                [&](int i) { return b->items[i].a.N == 0; }),
                 b->order.end());
  b->graph_ms[0] = b->graph_ms[1] = b->graph_ms[2] = 0.f;
  if (flags & ENS_BATCH_GRAPH) {
    // wait for the tuning runs (and any caller work on s) before capturing on a private stream
    if (cudaStreamSynchronize(s) != cudaSuccess) return batch_fail(b, ENS_ECUDA, "sync");
    const bool compare = (flags & ENS_BATCH_AUTOTUNE) && !(flags & ENS_BATCH_SERIAL) &&
                         !(flags & ENS_BATCH_FUSED) && b->order.size() > 1;
    if (!compare) {
      int rc = capture_graph(b, &b->graph, &b->exec);
      if (rc) return batch_fail(b, rc, ens_last_error());
    } else {
      // concurrent kernels can share the SMs well or crowd each other (a persistent grid
      // sized for the whole GPU leaves little room beside it); the fused kernel shares one
      // grid: capture each form the items allow, time them, keep the fastest
      // candidates: concurrent, serial, fused with blocks of 64 and of 128
      const int forms[4] = {0, ENS_BATCH_SERIAL, ENS_BATCH_FUSED, ENS_BATCH_FUSED};
      const int fblocks[4] = {0, 0, 64, 128};
      int best = -1, best_fblock = 64;
      float best_ms = 0.f;
      for (int f = 0; f < 4; ++f) {
        if (forms[f] == ENS_BATCH_FUSED && !b->fusable) continue;
        b->flags = (flags & ~(ENS_BATCH_SERIAL | ENS_BATCH_FUSED)) | forms[f];
        if (fblocks[f]) b->fblock = fblocks[f];
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        float ms = 0.f;
        int rc = capture_graph(b, &g, &x);
        if (!rc) rc = time_graph(x, s, &ms);
        if (rc) {
          if (x) cudaGraphExecDestroy(x);
          if (g) cudaGraphDestroy(g);
          return batch_fail(b, rc, ens_last_error());
        }
        const int slot = f < 2 ? f : 2;  // graph_ms: concurrent, serial, best fused
        if (b->graph_ms[slot] == 0.f || ms < b->graph_ms[slot]) b->graph_ms[slot] = ms;
        if (best < 0 || ms < best_ms) {
          std::swap(g, b->graph);
          std::swap(x, b->exec);
          best = f;
          best_ms = ms;
          if (fblocks[f]) best_fblock = fblocks[f];
        }
        if (x) cudaGraphExecDestroy(x);
        if (g) cudaGraphDestroy(g);
      }
      b->flags = (flags & ~(ENS_BATCH_SERIAL | ENS_BATCH_FUSED)) | forms[best];
      b->fblock = best_fblock;
    }
  }
  *out = b;
  return ENS_OK;
}

int ens_batch_run(ens_batch* b, void* cuda_stream) {
  if (!b) return set_last_error(ENS_EINVAL, "null batch");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e;
  if (b->exec) {
    e = cudaGraphLaunch(b->exec, s);
  } else {
    bool sup = true;
    e = enqueue_batch(b, s, &sup);
    if (!sup) return set_last_error(ENS_ENOTSUP, "algorithm not available for this model");
  }
  if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));
  return ENS_OK;
}

int ens_batch_info(const ens_batch* b, int item, ens_batch_item_info* info) {
  if (!b || !info) return set_last_error(ENS_EINVAL, "null argument");
  if (item < 0 || item >= (int)b->items.size()) return set_last_error(ENS_EINVAL, "bad item");
  const ens_batch::Item& it = b->items[item];
  info->schedule = it.cfg.schedule;
  info->block = it.cfg.block;
  info->tpt = it.cfg.tpt;
  info->blocks_per_sm = it.cfg.bps;
  info->tuned_ms = it.tuned_ms;
  int pos = -1;
  for (size_t k = 0; k < b->order.size(); ++k)
    if (b->order[k] == item) pos = (int)k;
  info->launch_position = pos;
  info->graph = b->exec != nullptr;
  info->serial = (b->flags & ENS_BATCH_SERIAL) != 0;
  info->fused = (b->flags & ENS_BATCH_FUSED) != 0;
  info->graph_ms_concurrent = b->graph_ms[0];
  info->graph_ms_serial = b->graph_ms[1];
  info->graph_ms_fused = b->graph_ms[2];
  info->lane_slots = 0;
  cudaError_t e = cudaMemcpy(&info->lane_slots, b->slots + item, sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_last_error(ENS_ECUDA, cudaGetErrorString(e));
  return ENS_OK;
}

int ens_batch_destroy(ens_batch* b) {
  if (!b) return ENS_OK;
  cudaDeviceSynchronize();
  batch_free(b);
  return ENS_OK;
}

}  // extern "C"
