// tqr_api.cpp -- the C ABI of libtqr (declared in include/tqr.h).
//
// Host-side orchestration only: argument checks, workspace layout, the plan
// cache, host/device pointer staging and kernel launches.  All arithmetic of
// the factorization runs in the kernels of tqr_engine.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <string>
#include <tuple>
#include <vector>

#include "tqr.h"
#include "tqr_api_internal.h"
#include "tqr_engine.h"
#include "tqr_plan.h"

namespace tqr {

// The device's bounded waits give up after this long (TQR_WAIT_LIMIT_MS in
// the environment overrides it, e.g. for runs under a profiler's replay,
// which slows launches by orders of magnitude).
static long long initial_wait_limit_ms() {
  const char* e = std::getenv("TQR_WAIT_LIMIT_MS");
  if (e != nullptr) {
    const long long v = std::atoll(e);
    if (v > 0) return v;
  }
  return 20000;
}
static long long g_wait_limit_ms = initial_wait_limit_ms();
static int g_policy = -1;
static int g_max_ctas = 0;
static std::mutex g_mu;

void set_schedule(int policy, int max_ctas) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_policy = policy;
  g_max_ctas = max_ctas;
}

// Tuning overrides of the slab width (0: automatic) and of the reduction-tree
// domain size (-1: automatic, 0: flat panel).
static std::atomic<int> g_force_cs{0};
static std::atomic<int> g_force_d{-1};

void set_shape_override(int cs, int D) {
  g_force_cs.store(cs);
  g_force_d.store(D);
}
static thread_local std::string g_last_error;

void set_last_error(const std::string& s) { g_last_error = s; }
const char* last_error() { return g_last_error.c_str(); }

int device_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  static std::map<int, int> cache;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  cache[dev] = sms;
  return sms;
}

long long wait_limit_ns() { return g_wait_limit_ms * 1000000LL; }

// Tile shape choice: the widest slab (32, 16 or 8 columns dividing nb) that
// keeps the most CTAs per SM (up to 2: 128 registers x 256 threads).
bool choose_shape(int nb, int ib, int esize, int* cs, int* ctas_per_sm, int* smem, int rows) {
  const int kSmemPerSM = 233472, kSmemPerBlock = 232448, kReserved = 1024;
  int best_cs = 0, best_occ = 0, best_smem = 0;
  // a forced width (tuning override) where it fits, else the automatic choice
  const int forced = g_force_cs.load();
  for (int pass = forced > 0 ? 0 : 1; pass < 2 && best_occ == 0; ++pass) {
    for (int c : {32, 16, 8}) {
      if (c > nb || nb % c != 0) continue;
      if (pass == 0 && c != forced) continue;
      if (ib * c > kThreads * kMaxOutPerThread) continue;
      const SmemLayout L = smem_layout(nb, ib, c, esize, rows);
      if (L.bytes > kSmemPerBlock) continue;
      int occ = kSmemPerSM / (L.bytes + kReserved);
      if (occ > 2) occ = 2;
      if (occ > best_occ) {
        best_occ = occ;
        best_cs = c;
        best_smem = L.bytes;
      }
    }
  }
  if (best_occ == 0) return false;
  *cs = best_cs;
  *ctas_per_sm = best_occ;
  *smem = best_smem;
  return true;
}

// Prefix tables of the tree variant for host-side planning, one per
// (p, kt, D); kept for the life of the process (a few KB each).
const int32_t* host_vtab(const Inst& I) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, std::vector<int32_t>> tabs;
  std::lock_guard<std::mutex> lk(mu);
  std::vector<int32_t>& v = tabs[std::make_tuple(I.p, I.kt, I.D)];
  if (v.empty()) tree_table(I, v);
  return v.data();
}

Inst make_inst(int mode, int64_t m, int64_t n, int nb, int ib, int cs, int nrhs, int trsm) {
  Inst I = {};
  I.m = static_cast<int>(m);
  I.n = static_cast<int>(n);
  I.p = static_cast<int>(std::max<int64_t>(1, (m + nb - 1) / nb));
  I.q = static_cast<int>(std::max<int64_t>(1, (n + nb - 1) / nb));
  I.kt = std::min(I.p, I.q);
  I.nrhs = nrhs;
  I.qb = nrhs > 0 ? (nrhs + nb - 1) / nb : 0;
  I.nb = nb;
  I.ib = ib;
  I.cs = cs;
  I.NS = nb / cs;
  I.mode = mode;
  I.trsm = trsm;
  return I;
}

// ---------------------------------------------------------------- memory
// Library workspaces and staging buffers come from a stream-ordered pool per
// device that keeps freed memory for reuse.  The device's default pool gives
// freed memory back to the driver at every synchronization, so a call that
// follows a synchronization (every call on host buffers) would map its
// gigabytes of workspace afresh.  tqr_release_memory() hands it back.
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

static cudaMemPool_t lib_pool(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  } else {
    cudaGetLastError();
    pool = nullptr;  // the device's default pool then
  }
  g_pools[dev] = pool;
  return pool;
}

cudaError_t lib_malloc(void** p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool = lib_pool(dev);
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

cudaError_t copy_cols(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t height,
                      cudaMemcpyKind kind, cudaStream_t st) {
  if (dpitch == width && spitch == width) return cudaMemcpyAsync(dst, src, width * height, kind, st);
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, height, kind, st);
}

int release_memory() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : g_pools) {
    if (!kv.second) continue;
    if (cudaSetDevice(kv.first) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemPoolTrimTo(kv.second, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaSetDevice(cur);
      return TQR_ERR_CUDA;
    }
  }
  cudaSetDevice(cur);
  return TQR_OK;
}

// ---------------------------------------------------------------- plan cache
// Task lists live in stream-ordered allocations made, uploaded and freed on a
// private stream per device: no cudaMalloc / cudaFree (the latter waits for
// the whole device) runs while launches on other streams are in flight.
static cudaStream_t plan_stream(int dev) {
  static std::mutex mu;
  static std::map<int, cudaStream_t> streams;
  std::lock_guard<std::mutex> lk(mu);
  auto it = streams.find(dev);
  if (it != streams.end()) return it->second;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    s = nullptr;
  }
  streams[dev] = s;
  return s;
}

struct DevPlan {
  TaskX* d_tasks = nullptr;
  int ntasks = 0;
  int grid = 0;
  PlanStats stats;
  int device = -1;
  ~DevPlan() {
    if (d_tasks) {
      int cur = -1;
      cudaGetDevice(&cur);
      if (device >= 0 && device != cur) cudaSetDevice(device);
      // no launch still reads the list (in-flight holders keep it alive)
      if (cudaFreeAsync(d_tasks, plan_stream(device)) != cudaSuccess) cudaGetLastError();
      if (device >= 0 && device != cur) cudaSetDevice(cur);
    }
  }
};

// A plan depends on the instance only through its task-list structure: the
// tile grid (p, q), the right-hand-side tile columns and the slab count of
// the last one, nb, ib, cs, the mode and its flags -- not on m, n or nrhs
// themselves (edge tiles and slab widths are read from the instance on the
// device).  Keying on the structure lets differently sized problems on the
// same grid share one plan.
typedef std::tuple<int, int, int, int, int, int, int, int, int, int, int, int, int, int> PlanKey;

static std::list<std::pair<PlanKey, std::shared_ptr<DevPlan>>> g_plans;
static const size_t kMaxPlans = 512;
static const size_t kMaxPlanBytes = size_t(256) << 20;  // device task lists held by the cache

// Launches keep their plan alive until their completion event fires: a plan
// evicted from the cache while a kernel on some stream still reads its task
// list is freed only after that kernel is done.
static std::list<std::pair<cudaEvent_t, std::shared_ptr<DevPlan>>> g_inflight;
static std::vector<cudaEvent_t> g_event_pool;

static void prune_inflight_locked() {
  for (auto it = g_inflight.begin(); it != g_inflight.end();) {
    if (cudaEventQuery(it->first) == cudaSuccess) {
      g_event_pool.push_back(it->first);
      it = g_inflight.erase(it);
    } else {
      cudaGetLastError();
      ++it;
    }
  }
}

static void hold_until_done(const std::shared_ptr<DevPlan>& plan, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  prune_inflight_locked();
  cudaEvent_t ev = nullptr;
  if (!g_event_pool.empty()) {
    ev = g_event_pool.back();
    g_event_pool.pop_back();
  } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(st);  // no event: keep the plan alive by waiting
    return;
  }
  cudaEventRecord(ev, st);
  g_inflight.emplace_back(ev, plan);
}

static PlanKey key_of(const Inst& I, int esize, int grid, int dev, int policy) {
  const int last = I.qb > 0 ? slabs_of_col(I, I.q + I.qb - 1) : 0;
  return PlanKey(I.mode + 16 * I.lu + 32 * I.pair, I.p, I.q, I.nb, I.ib, I.cs, I.qb * 256 + last, I.trsm, esize, grid,
                 dev, policy, I.D, 0);
}

std::shared_ptr<DevPlan> get_plan(const Inst& I, int esize, int ctas_per_sm, int* status, int grid_cap) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int sms = device_sms();
  std::vector<TaskX> seq;
  int policy, max_ctas;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    policy = g_policy;
    max_ctas = g_max_ctas;
  }
  // grid: at most ctas_per_sm CTAs per SM (and the debug cap)
  int max_grid = sms * ctas_per_sm;
  if (max_ctas > 0 && max_ctas < max_grid) max_grid = max_ctas;
  if (grid_cap > 0 && grid_cap < max_grid) max_grid = grid_cap;
  // the grid of a cached plan is min(max_grid, ntasks); look up by max_grid
  const PlanKey want = key_of(I, esize, max_grid, dev, policy);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_plans.begin(); it != g_plans.end(); ++it) {
      if (it->first == want) {
        auto p = it->second;
        g_plans.splice(g_plans.begin(), g_plans, it);
        return p;
      }
    }
  }
  // planning runs on the host: the tree variant's table must be host memory
  Inst Ih = I;
  if (Ih.D > 0) Ih.vtab = host_vtab(Ih);
  seq_tasks(Ih, 0, seq);
  auto plan = std::make_shared<DevPlan>();
  plan->device = dev;
  plan->ntasks = static_cast<int>(seq.size());
  plan->grid = std::max(1, std::min<int>(max_grid, plan->ntasks));
  if (!seq.empty()) {
    std::vector<TaskX> ordered;
    std::string err;
    std::vector<Inst> insts(1, Ih);
    // capped launches (concurrent server requests, many distinct shapes) take
    // the bottom-level order without the list-scheduling simulation: about a
    // third of the planning time, and a shared device is not the simulated one
    const bool ok = (grid_cap > 0 && policy < 0)
                        ? order_bottom_level(insts, seq, esize, ctas_per_sm, plan->grid, ordered, &plan->stats, &err)
                        : order_tasks(insts, seq, plan->grid, esize, ctas_per_sm, policy, ordered, &plan->stats, &err);
    if (!ok) {
      set_last_error(err);
      *status = TQR_ERR_UNSUPPORTED;
      return nullptr;
    }
    // a capped launch shares the device: take about twice the graph's average
    // parallelism (work / critical path), not CTAs that would mostly wait
    if (grid_cap > 0 && plan->stats.critical_path_s > 0) {
      const double par = plan->stats.work_s / plan->stats.critical_path_s;
      const int want = static_cast<int>(std::min<double>(plan->grid, std::max(8.0, std::ceil(2.0 * par))));
      plan->grid = std::max(1, std::min(plan->grid, want));
    }
    cudaStream_t ps = plan_stream(dev);
    if (lib_malloc(reinterpret_cast<void**>(&plan->d_tasks), sizeof(TaskX) * ordered.size(), ps) !=
        cudaSuccess) {
      cudaGetLastError();
      plan->d_tasks = nullptr;
      *status = TQR_ERR_NOMEM;
      return nullptr;
    }
    // published only once uploaded: other threads may launch it on any stream
    if (cudaMemcpyAsync(plan->d_tasks, ordered.data(), sizeof(TaskX) * ordered.size(), cudaMemcpyHostToDevice,
                        ps) != cudaSuccess ||
        cudaStreamSynchronize(ps) != cudaSuccess) {
      *status = TQR_ERR_CUDA;
      return nullptr;
    }
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_plans.emplace_front(want, plan);
  size_t bytes = 0;
  for (const auto& e : g_plans) bytes += sizeof(TaskX) * static_cast<size_t>(e.second->ntasks);
  while (g_plans.size() > 1 && (g_plans.size() > kMaxPlans || bytes > kMaxPlanBytes)) {
    bytes -= sizeof(TaskX) * static_cast<size_t>(g_plans.back().second->ntasks);
    g_plans.pop_back();
  }
  return plan;
}

// ---------------------------------------------------------------- timing
struct TimingState {
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
};
static TimingState g_timing;

static std::pair<cudaEvent_t, cudaEvent_t> timing_pair() {
  std::pair<cudaEvent_t, cudaEvent_t> p(nullptr, nullptr);
  if (!g_timing.pool.empty()) {
    p = g_timing.pool.back();
    g_timing.pool.pop_back();
    return p;
  }
  cudaEventCreate(&p.first);
  cudaEventCreate(&p.second);
  return p;
}

int timing_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_timing.on = on != 0;
  return 0;
}

int timing_read(double* ms, int64_t* launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  double total = 0;
  int64_t cnt = 0;
  int rc = 0;
  for (auto& p : g_timing.pending) {
    float t = 0;
    if (cudaEventSynchronize(p.second) != cudaSuccess || cudaEventElapsedTime(&t, p.first, p.second) != cudaSuccess)
      rc = 1;
    total += t;
    ++cnt;
    g_timing.pool.push_back(p);
  }
  g_timing.pending.clear();
  if (ms) *ms = total;
  if (launches) *launches = cnt;
  return rc;
}

void clear_plans() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_plans.clear();
  prune_inflight_locked();
}

// ---------------------------------------------------------------- tree
// Domain size of the reduction-tree variant for an m x n factorization: the
// candidate (flat Algorithm 1 or D in {64, ..., 1} tile rows) with the
// smallest max(critical path, work / CTAs) under the scheduler's cost model;
// the flat panel is kept unless a tree is at least 5% better.  Cached.
int choose_domain(int64_t m, int64_t n, int nb, int ib, int esize) {
  // the choice depends on the tile grid only
  static std::mutex mu;
  static std::map<std::tuple<int64_t, int64_t, int, int, int>, int> cache;
  const int64_t p = std::max<int64_t>(1, (m + nb - 1) / nb), q = std::max<int64_t>(1, (n + nb - 1) / nb);
  const int forced = g_force_d.load();
  if (forced >= 0) return forced < p ? forced : 0;
  const auto key = std::make_tuple(p, q, nb, ib, esize);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  int cs, occ, smem;
  if (!choose_shape(nb, ib, esize, &cs, &occ, &smem)) return 0;
  const int workers = std::max(1, device_sms()) * occ;
  auto estimate = [&](int D, double* cp, double* work) {
    Inst I = make_inst(M_FACTOR, m, n, nb, ib, cs, 0, 0);
    I.D = D;
    if (D > 0) I.vtab = host_vtab(I);
    critical_path_estimate(I, esize, occ, cp, work);
  };
  double cp0 = 0, work0 = 0;
  estimate(0, &cp0, &work0);
  const double flat = std::max(cp0, work0 / workers);
  int best_d = 0;
  double best = flat;
  // work-bound: a tree only adds work; otherwise the tree candidates are
  // estimated side by side (one host thread each: each is a pass over the
  // task list, tens of ms in all for the largest grids)
  if (cp0 > work0 / workers) {
    std::vector<int> cands;
    for (int D : {64, 32, 16, 8, 4, 2, 1})
      if (D < p) cands.push_back(D);
    std::vector<double> est(cands.size(), INFINITY);
    std::vector<std::thread> th;
    for (size_t a = 0; a < cands.size(); ++a)
      th.emplace_back([&, a]() {
        double cp = 0, work = 0;
        estimate(cands[a], &cp, &work);
        est[a] = std::max(cp, work / workers);
      });
    for (auto& t : th) t.join();
    for (size_t a = 0; a < cands.size(); ++a)
      if (est[a] < best) {
        best = est[a];
        best_d = cands[a];
      }
  }
  if (best_d != 0 && !(best < 0.95 * flat)) best_d = 0;
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = best_d;
  return best_d;
}

// Points I.vtab at the workspace copy of the tree table and uploads it.
int upload_vtab(Inst& I, char* ws, const WsLayout& W, cudaStream_t st) {
  if (I.D <= 0) {
    I.vtab = nullptr;
    return TQR_OK;
  }
  I.vtab = reinterpret_cast<const int32_t*>(ws + W.oVtab);
  const int32_t* h = host_vtab(I);
  return cudaMemcpyAsync(ws + W.oVtab, h, sizeof(int32_t) * static_cast<size_t>(I.kt + 1) * I.p,
                         cudaMemcpyHostToDevice, st) == cudaSuccess
             ? TQR_OK
             : TQR_ERR_CUDA;
}

// ---------------------------------------------------------------- workspace
static size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

WsLayout ws_layout(const Inst& I, int esize, bool with_t) {
  WsLayout W;
  const size_t nb2 = static_cast<size_t>(I.nb) * I.nb;
  size_t o = 0;
  W.oA = o;
  o += al256(nb2 * I.p * I.q * esize);
  W.oB = o;
  o += al256(nb2 * I.p * I.qb * esize);
  W.oT = o;
  if (with_t) o += al256(static_cast<size_t>(t_elems(I.p, I.q, I.nb, I.ib)) * esize * (I.D > 0 ? 2 : 1));
  W.oVtab = o;
  if (I.D > 0) o += al256(sizeof(int32_t) * static_cast<size_t>(I.kt + 1) * I.p);
  W.oVer = o;
  o += al256(sizeof(int) * static_cast<size_t>(I.p) * (I.q + I.qb) * I.NS);
  W.oInst = o;
  o += al256(sizeof(Inst));
  W.oCtl = o;
  o += al256(ctl_bytes());
  W.bytes = o;
  return W;
}

// Clears the counters and control block, uploads the instance and runs the
// plan.  `I` must already hold the device pointers.
template <typename real>
int run_plan(const Inst& I, char* ws, const WsLayout& W, int ctas_per_sm, int smem, cudaStream_t st, int grid_cap,
             double* err_out) {
  int status = TQR_OK;
  std::shared_ptr<DevPlan> plan = get_plan(I, sizeof(real), ctas_per_sm, &status, grid_cap);
  if (!plan) return status;
  if (plan->ntasks == 0) return TQR_OK;
  if (cudaMemsetAsync(ws + W.oVer, 0, W.oCtl + ctl_bytes() - W.oVer, st) != cudaSuccess) return TQR_ERR_CUDA;
  if (cudaMemcpyAsync(ws + W.oInst, &I, sizeof(Inst), cudaMemcpyHostToDevice, st) != cudaSuccess) return TQR_ERR_CUDA;
  std::pair<cudaEvent_t, cudaEvent_t> ev(nullptr, nullptr);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_timing.on) {
      ev = timing_pair();
      cudaEventRecord(ev.first, st);
    }
  }
  cudaError_t e = launch_run<real>(plan->d_tasks, plan->ntasks, reinterpret_cast<const Inst*>(ws + W.oInst),
                                   ws + W.oCtl, wait_limit_ns(), plan->grid, smem, st, I.lu ? 1 : (I.pair ? 2 : 0));
  if (e == cudaSuccess && err_out != nullptr) e = launch_fold_error(ws + W.oCtl, plan->d_tasks, plan->ntasks, err_out, st);
  if (ev.first) {
    cudaEventRecord(ev.second, st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_timing.pending.push_back(ev);
  }
  hold_until_done(plan, st);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return TQR_ERR_CUDA;
  }
  return TQR_OK;
}

template int run_plan<double>(const Inst&, char*, const WsLayout&, int, int, cudaStream_t, int, double*);
template int run_plan<float>(const Inst&, char*, const WsLayout&, int, int, cudaStream_t, int, double*);

// ---------------------------------------------------------------- several graphs, one launch
// Independent task graphs of one factorization's operands (say Q^T f and a
// triangular solve of another vector) run as one persistent launch, so
// their dependency chains overlap instead of adding up.  Cached by the
// instances' structures.
static std::list<std::pair<std::vector<PlanKey>, std::shared_ptr<DevPlan>>> g_mplans;
static const size_t kMaxMultiPlans = 64;

template <typename real>
int run_plan_multi(const Inst* insts, int count, Inst* d_insts, void* d_ctl, int ctas_per_sm, int smem,
                   cudaStream_t st, int grid_cap, double* err_out) {
  int dev = 0;
  cudaGetDevice(&dev);
  int policy, max_ctas;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    policy = g_policy;
    max_ctas = g_max_ctas;
  }
  int max_grid = device_sms() * ctas_per_sm;
  if (max_ctas > 0 && max_ctas < max_grid) max_grid = max_ctas;
  if (grid_cap > 0 && grid_cap < max_grid) max_grid = grid_cap;
  std::vector<PlanKey> want;
  for (int a = 0; a < count; ++a) want.push_back(key_of(insts[a], sizeof(real), max_grid, dev, policy));
  std::shared_ptr<DevPlan> plan;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_mplans.begin(); it != g_mplans.end(); ++it)
      if (it->first == want) {
        plan = it->second;
        g_mplans.splice(g_mplans.begin(), g_mplans, it);
        break;
      }
  }
  if (!plan) {
    std::vector<Inst> hi(insts, insts + count);
    for (Inst& I : hi)
      if (I.D > 0) I.vtab = host_vtab(I);
    std::vector<TaskX> seq, ordered;
    for (int a = 0; a < count; ++a) seq_tasks(hi[a], a, seq);
    plan = std::make_shared<DevPlan>();
    plan->device = dev;
    plan->ntasks = static_cast<int>(seq.size());
    plan->grid = std::max(1, std::min<int>(max_grid, plan->ntasks));
    if (!seq.empty()) {
      std::string err;
      const bool ok = (grid_cap > 0 && policy < 0)
                          ? order_bottom_level(hi, seq, sizeof(real), ctas_per_sm, plan->grid, ordered, &plan->stats,
                                               &err)
                          : order_tasks(hi, seq, plan->grid, sizeof(real), ctas_per_sm, policy, ordered,
                                        &plan->stats, &err);
      if (!ok) {
        set_last_error(err);
        return TQR_ERR_UNSUPPORTED;
      }
      cudaStream_t ps = plan_stream(dev);
      if (lib_malloc(reinterpret_cast<void**>(&plan->d_tasks), sizeof(TaskX) * ordered.size(), ps) !=
          cudaSuccess) {
        cudaGetLastError();
        plan->d_tasks = nullptr;
        return TQR_ERR_NOMEM;
      }
      if (cudaMemcpyAsync(plan->d_tasks, ordered.data(), sizeof(TaskX) * ordered.size(), cudaMemcpyHostToDevice,
                          ps) != cudaSuccess ||
          cudaStreamSynchronize(ps) != cudaSuccess)
        return TQR_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_mplans.emplace_front(want, plan);
    while (g_mplans.size() > kMaxMultiPlans) g_mplans.pop_back();
  }
  if (plan->ntasks == 0) return TQR_OK;
  // counters of every instance and the launch's control block start at zero
  for (int a = 0; a < count; ++a) {
    const Inst& I = insts[a];
    const size_t nctr = static_cast<size_t>(I.p) * (I.q + I.qb) * I.NS;
    if (cudaMemsetAsync(I.ver, 0, sizeof(int) * nctr, st) != cudaSuccess) return TQR_ERR_CUDA;
  }
  if (cudaMemsetAsync(d_ctl, 0, ctl_bytes(), st) != cudaSuccess ||
      cudaMemcpyAsync(d_insts, insts, sizeof(Inst) * count, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return TQR_ERR_CUDA;
  std::pair<cudaEvent_t, cudaEvent_t> ev(nullptr, nullptr);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_timing.on) {
      ev = timing_pair();
      cudaEventRecord(ev.first, st);
    }
  }
  cudaError_t e = launch_run<real>(plan->d_tasks, plan->ntasks, d_insts, d_ctl, wait_limit_ns(), plan->grid, smem,
                                   st, insts[0].lu ? 1 : (insts[0].pair ? 2 : 0));
  if (e == cudaSuccess && err_out != nullptr) e = launch_fold_error(d_ctl, plan->d_tasks, plan->ntasks, err_out, st);
  if (ev.first) {
    cudaEventRecord(ev.second, st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_timing.pending.push_back(ev);
  }
  hold_until_done(plan, st);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return TQR_ERR_CUDA;
  }
  return TQR_OK;
}

template int run_plan_multi<double>(const Inst*, int, Inst*, void*, int, int, cudaStream_t, int, double*);
template int run_plan_multi<float>(const Inst*, int, Inst*, void*, int, int, cudaStream_t, int, double*);

// ---------------------------------------------------------------- pointers
int ptr_kind(const void* p) {
  if (p == nullptr) return PTR_NULL;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PTR_HOST;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return PTR_DEVICE;
  return PTR_HOST;
}

int check_tiles(int nb, int ib, int arg_nb, int arg_ib) {
  if (nb < 8 || nb > 256 || nb % 8 != 0) return -arg_nb;
  if (ib < 1 || ib > 64 || nb % ib != 0) return -arg_ib;
  return 0;
}

}  // namespace tqr

using namespace tqr;

// ---------------------------------------------------------------- factor
template <typename real>
static int factor_device(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, int D, int pair, real* T,
                         void* work, size_t work_bytes, cudaStream_t st) {
  int cs, occ, smem;
  if (!choose_shape(nb, ib, sizeof(real), &cs, &occ, &smem, pair ? 2 * nb : 0)) return TQR_ERR_UNSUPPORTED;
  Inst I = make_inst(M_FACTOR, m, n, nb, ib, cs, 0, 0);
  I.D = D;
  I.pair = pair;
  const WsLayout W = ws_layout(I, sizeof(real), false);
  char* ws = static_cast<char*>(work);
  bool own = false;
  if (ws == nullptr) {
    if (lib_malloc(reinterpret_cast<void**>(&ws), W.bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return TQR_ERR_NOMEM;
    }
    own = true;
  } else if (work_bytes < W.bytes) {
    return -10;
  }
  I.A = ws + W.oA;
  I.B = nullptr;
  I.T = T;
  I.ver = reinterpret_cast<int*>(ws + W.oVer);
  const int sms = device_sms();
  int status = upload_vtab(I, ws, W, st);
  if (status == TQR_OK &&
      launch_pack<real>(A, lda, static_cast<int>(m), static_cast<int>(n), static_cast<real*>(I.A), I.p, I.q, nb, sms,
                        st) != cudaSuccess)
    status = TQR_ERR_CUDA;
  if (status == TQR_OK) status = run_plan<real>(I, ws, W, occ, smem, st);
  if (status == TQR_OK &&
      launch_unpack<real>(static_cast<real*>(I.A), I.p, nb, A, lda, static_cast<int>(m), static_cast<int>(n), sms, st) !=
          cudaSuccess)
    status = TQR_ERR_CUDA;
  if (own) cudaFreeAsync(ws, st);
  return status;
}

static int factor_common(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, int D, int pair, double* T,
                         void* work, size_t work_bytes, void* stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (m > (1LL << 30) || n > (1LL << 30)) return TQR_ERR_UNSUPPORTED;
  if (lda < std::max<int64_t>(1, m)) return -4;
  int c = check_tiles(nb, ib, 5, 6);
  if (c) return c;
  if (m == 0 || n == 0) return TQR_OK;
  if (A == nullptr) return -3;
  if (T == nullptr) return -7;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ka = ptr_kind(A), kt = ptr_kind(T);
  if (ka != kt) return -7;
  if (ka == PTR_DEVICE) return factor_device<double>(m, n, A, lda, nb, ib, D, pair, T, work, work_bytes, st);
  // host buffers: stage through the device, synchronously
  const size_t tbytes = tqr_t_size(m, n, nb, ib) * (D > 0 ? 2 : 1);
  double *dA = nullptr, *dT = nullptr;
  if (lib_malloc(reinterpret_cast<void**>(&dA), sizeof(double) * m * n, st) != cudaSuccess ||
      lib_malloc(reinterpret_cast<void**>(&dT), tbytes, st) != cudaSuccess) {
    cudaGetLastError();
    if (dA) cudaFreeAsync(dA, st);
    return TQR_ERR_NOMEM;
  }
  int status = TQR_OK;
  // slots the variant leaves unused (tree, pairs) come back as zeros
  if (copy_cols(dA, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m, n,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(dT, 0, tbytes, st) != cudaSuccess)
    status = TQR_ERR_CUDA;
  if (status == TQR_OK) status = factor_device<double>(m, n, dA, m, nb, ib, D, pair, dT, work, work_bytes, st);
  if (status == TQR_OK &&
      (copy_cols(A, sizeof(double) * lda, dA, sizeof(double) * m, sizeof(double) * m, n,
                         cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaMemcpyAsync(T, dT, tbytes, cudaMemcpyDeviceToHost, st) != cudaSuccess))
    status = TQR_ERR_CUDA;
  cudaFreeAsync(dA, st);
  cudaFreeAsync(dT, st);
  int dev_status = TQR_OK;
  if (read_status(&dev_status, st) != cudaSuccess) return TQR_ERR_CUDA;
  if (status == TQR_OK) status = dev_status;
  return status;
}

// ---------------------------------------------------------------- apply
// How the right-hand-side tiles are filled and returned.
//   RHS_PLAIN       B is m x nrhs (ldb), packed and unpacked as is
//   RHS_TRANSPOSED  B holds C = X^T, nrhs x m (ldb >= nrhs); the tiles hold X
//   RHS_IDENTITY    the tiles start as the leading nrhs columns of I_m; B
//                   (m x nrhs) receives the result
enum RhsForm { RHS_PLAIN = 0, RHS_TRANSPOSED = 1, RHS_IDENTITY = 2 };

template <typename real>
static int apply_device(int mode, int form, int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb,
                        int ib, int D, int pair, const real* T, double* B, int64_t ldb, cudaStream_t st) {
  int cs, occ, smem;
  if (!choose_shape(nb, ib, sizeof(real), &cs, &occ, &smem, pair ? 2 * nb : 0)) return TQR_ERR_UNSUPPORTED;
  Inst I = make_inst(mode, m, n, nb, ib, cs, static_cast<int>(nrhs), 0);
  I.D = D;
  I.pair = pair;
  const WsLayout W = ws_layout(I, sizeof(real), false);
  char* ws = nullptr;
  if (lib_malloc(reinterpret_cast<void**>(&ws), W.bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return TQR_ERR_NOMEM;
  }
  I.A = ws + W.oA;
  I.B = ws + W.oB;
  I.T = const_cast<real*>(T);
  I.ver = reinterpret_cast<int*>(ws + W.oVer);
  const int sms = device_sms();
  const int mi = static_cast<int>(m), ni = static_cast<int>(n), ri = static_cast<int>(nrhs);
  real* Bt = static_cast<real*>(I.B);
  int status = n > 0 ? upload_vtab(I, ws, W, st) : TQR_OK;
  cudaError_t e = cudaSuccess;
  if (status == TQR_OK && n > 0) e = launch_pack<real>(A, lda, mi, ni, static_cast<real*>(I.A), I.p, I.q, nb, sms, st);
  if (status == TQR_OK && e == cudaSuccess) {
    if (form == RHS_PLAIN) e = launch_pack<real>(B, ldb, mi, ri, Bt, I.p, I.qb, nb, sms, st);
    else if (form == RHS_TRANSPOSED) e = launch_pack_t<real>(B, ldb, mi, ri, Bt, I.p, I.qb, nb, sms, st);
    else e = launch_identity<real>(mi, ri, Bt, I.p, I.qb, nb, sms, st);
  }
  if (e != cudaSuccess) status = TQR_ERR_CUDA;
  if (status == TQR_OK && n > 0) status = run_plan<real>(I, ws, W, occ, smem, st);
  if (status == TQR_OK) {
    e = form == RHS_TRANSPOSED ? launch_unpack_t<real>(Bt, I.p, nb, B, ldb, mi, ri, sms, st)
                               : launch_unpack<real>(Bt, I.p, nb, B, ldb, mi, ri, sms, st);
    if (e != cudaSuccess) status = TQR_ERR_CUDA;
  }
  cudaFreeAsync(ws, st);
  return status;
}

// Device or host operands.  B is brows x bcols with leading dimension ldb
// (m x nrhs, or nrhs x m for RHS_TRANSPOSED).  Host operands are staged
// through device copies on the stream; the call then synchronizes.
static int apply_staged(int mode, int form, int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb,
                        int ib, int D, int pair, const double* T, double* B, int64_t ldb, int argA, int argT, int argB,
                        void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t brows = form == RHS_TRANSPOSED ? nrhs : m, bcols = form == RHS_TRANSPOSED ? m : nrhs;
  const int ka = n > 0 ? ptr_kind(A) : ptr_kind(B);
  if (n > 0 && ptr_kind(T) != ka) return -argT;
  if (ptr_kind(B) != ka) return -argB;
  if (ka == PTR_DEVICE) return apply_device<double>(mode, form, m, n, nrhs, A, lda, nb, ib, D, pair, T, B, ldb, st);
  const size_t tbytes = tqr_t_size(m, n, nb, ib) * (D > 0 ? 2 : 1);
  double *dA = nullptr, *dT = nullptr, *dB = nullptr;
  if (lib_malloc(reinterpret_cast<void**>(&dA), sizeof(double) * std::max<int64_t>(1, m * n), st) != cudaSuccess ||
      lib_malloc(reinterpret_cast<void**>(&dT), std::max<size_t>(8, tbytes), st) != cudaSuccess ||
      lib_malloc(reinterpret_cast<void**>(&dB), sizeof(double) * brows * bcols, st) != cudaSuccess) {
    cudaGetLastError();
    if (dA) cudaFreeAsync(dA, st);
    if (dT) cudaFreeAsync(dT, st);
    return TQR_ERR_NOMEM;
  }
  int status = TQR_OK;
  if ((n > 0 && (copy_cols(dA, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m, n,
                                   cudaMemcpyHostToDevice, st) != cudaSuccess ||
                 cudaMemcpyAsync(dT, T, tbytes, cudaMemcpyHostToDevice, st) != cudaSuccess)) ||
      (form != RHS_IDENTITY && copy_cols(dB, sizeof(double) * brows, B, sizeof(double) * ldb,
                                                 sizeof(double) * brows, bcols, cudaMemcpyHostToDevice,
                                                 st) != cudaSuccess))
    status = TQR_ERR_CUDA;
  if (status == TQR_OK)
    status = apply_device<double>(mode, form, m, n, nrhs, dA, std::max<int64_t>(1, m), nb, ib, D, pair, dT, dB,
                                  brows, st);
  if (status == TQR_OK && copy_cols(B, sizeof(double) * ldb, dB, sizeof(double) * brows,
                                            sizeof(double) * brows, bcols, cudaMemcpyDeviceToHost,
                                            st) != cudaSuccess)
    status = TQR_ERR_CUDA;
  cudaFreeAsync(dA, st);
  cudaFreeAsync(dT, st);
  cudaFreeAsync(dB, st);
  int dev_status = TQR_OK;
  if (read_status(&dev_status, st) != cudaSuccess) return TQR_ERR_CUDA;
  if (status == TQR_OK) status = dev_status;
  return status;
}

static int apply_common(char trans, int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib,
                        int D, int pair, const double* T, double* B, int64_t ldb, void* stream) {
  if (trans != 'T' && trans != 'N' && trans != 't' && trans != 'n') return -1;
  trans = (trans == 't' || trans == 'T') ? 'T' : 'N';
  if (m < 0) return -2;
  if (n < 0) return -3;
  if (nrhs < 0) return -4;
  if (m > (1LL << 30) || n > (1LL << 30) || nrhs > (1LL << 30)) return TQR_ERR_UNSUPPORTED;
  if (lda < std::max<int64_t>(1, m)) return -6;
  int c = check_tiles(nb, ib, 7, 8);
  if (c) return c;
  if (ldb < std::max<int64_t>(1, m)) return -11;
  if (m == 0 || n == 0 || nrhs == 0) return TQR_OK;
  if (A == nullptr) return -5;
  if (T == nullptr) return -9;
  if (B == nullptr) return -10;
  return apply_staged(trans == 'T' ? M_APPLY_QT : M_APPLY_Q, RHS_PLAIN, m, n, nrhs, A, lda, nb, ib, D, pair, T, B,
                      ldb, 5, 9, 10, stream);
}

extern "C" {

const char* tqr_version(void) { return "tqr 0.1 sm_103a"; }

size_t tqr_t_size(int64_t m, int64_t n, int nb, int ib) {
  if (m < 0 || n < 0 || check_tiles(nb, ib, 1, 2) != 0) return 0;
  const int p = static_cast<int>(std::max<int64_t>(1, (m + nb - 1) / nb));
  const int q = static_cast<int>(std::max<int64_t>(1, (n + nb - 1) / nb));
  return sizeof(double) * static_cast<size_t>(t_elems(p, q, nb, ib));
}

size_t tqr_work_size(int64_t m, int64_t n, int nb, int ib) {
  if (m < 0 || n < 0 || check_tiles(nb, ib, 1, 2) != 0) return 0;
  int cs, occ, smem;
  if (!choose_shape(nb, ib, sizeof(double), &cs, &occ, &smem)) return 0;
  const Inst I = make_inst(M_FACTOR, m, n, nb, ib, cs, 0, 0);
  return ws_layout(I, sizeof(double), false).bytes;
}

int tqr_factor(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* T, void* stream) {
  return factor_common(m, n, A, lda, nb, ib, 0, 0, T, nullptr, 0, stream);
}

int tqr_factor_ws(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* T, void* work,
                  size_t work_bytes, void* stream) {
  if (work == nullptr) return -8;
  if (ptr_kind(work) != PTR_DEVICE) return -8;
  if (reinterpret_cast<uintptr_t>(work) % 256 != 0) return -8;
  return factor_common(m, n, A, lda, nb, ib, 0, 0, T, work, work_bytes, stream);
}

int tqr_apply_qt(char trans, int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib,
                 const double* T, double* B, int64_t ldb, void* stream) {
  return apply_common(trans, m, n, nrhs, A, lda, nb, ib, 0, 0, T, B, ldb, stream);
}

size_t tqr_t_size_tree(int64_t m, int64_t n, int nb, int ib) { return 2 * tqr_t_size(m, n, nb, ib); }

int tqr_factor_tree(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, int* D, double* T, void* stream) {
  if (D == nullptr || *D < 0) return -7;
  if (m < 0) return -1;
  if (n < 0) return -2;
  const int c = check_tiles(nb, ib, 5, 6);
  if (c) return c;
  if (*D == 0 && m > 0 && n > 0) {
    *D = choose_domain(m, n, nb, ib, sizeof(double));
    if (*D == 0) *D = static_cast<int>((m + nb - 1) / nb);  // one domain: Algorithm 1's flat panel
  }
  const int r = factor_common(m, n, A, lda, nb, ib, *D, 0, T, nullptr, 0, stream);
  return r == -7 ? -8 : r;  // T is argument 8 here
}

int tqr_apply_qt_tree(char trans, int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib,
                      int D, const double* T, double* B, int64_t ldb, void* stream) {
  if (D < 1) return -9;
  const int r = apply_common(trans, m, n, nrhs, A, lda, nb, ib, D, 0, T, B, ldb, stream);
  return (r <= -9) ? r - 1 : r;  // arguments after ib shift by one
}

int tqr_ormqr(char side, char trans, int64_t m, int64_t n, const double* A, int64_t lda, int nb, int ib, int D,
              const double* T, int64_t mc, int64_t nc, double* C, int64_t ldc, void* stream) {
  const bool left = side == 'L' || side == 'l';
  if (!left && side != 'R' && side != 'r') return -1;
  if (trans != 'T' && trans != 'N' && trans != 't' && trans != 'n') return -2;
  const bool tr = trans == 'T' || trans == 't';
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (lda < std::max<int64_t>(1, m)) return -6;
  const int c = check_tiles(nb, ib, 7, 8);
  if (c) return c;
  if (D < 0) return -9;
  if (mc < 0 || (left && mc != m)) return -11;
  if (nc < 0 || (!left && nc != m)) return -12;
  if (ldc < std::max<int64_t>(1, mc)) return -14;
  if (m > (1LL << 30) || n > (1LL << 30) || mc > (1LL << 30) || nc > (1LL << 30)) return TQR_ERR_UNSUPPORTED;
  if (m == 0 || n == 0 || mc == 0 || nc == 0) return TQR_OK;
  if (A == nullptr) return -5;
  if (T == nullptr) return -10;
  if (C == nullptr) return -13;
  // left: op(Q) C directly; right: C op(Q) = (op(Q)^T C^T)^T on the transposed tiles
  const bool qt = left ? tr : !tr;
  return apply_staged(qt ? M_APPLY_QT : M_APPLY_Q, left ? RHS_PLAIN : RHS_TRANSPOSED, m, n, left ? nc : mc, A, lda,
                      nb, ib, D, 0, T, C, ldc, 5, 10, 13, stream);
}

int tqr_orgqr(int64_t m, int64_t n, const double* A, int64_t lda, int nb, int ib, int D, const double* T,
              int64_t ncols, double* Q, int64_t ldq, void* stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (lda < std::max<int64_t>(1, m)) return -4;
  const int c = check_tiles(nb, ib, 5, 6);
  if (c) return c;
  if (D < 0) return -7;
  if (ncols < 0 || ncols > m) return -9;
  if (ldq < std::max<int64_t>(1, m)) return -11;
  if (m > (1LL << 30) || n > (1LL << 30)) return TQR_ERR_UNSUPPORTED;
  if (m == 0 || ncols == 0) return TQR_OK;
  if (n > 0 && A == nullptr) return -3;
  if (n > 0 && T == nullptr) return -8;
  if (Q == nullptr) return -10;
  // identity columns skip the steps that cannot touch them
  return apply_staged(M_FORM_Q, RHS_IDENTITY, m, n, ncols, A, lda, nb, ib, D, 0, T, Q, ldq, 3, 8, 10, stream);
}

int tqr_factor_pairs(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* T, void* stream) {
  return factor_common(m, n, A, lda, nb, ib, 0, 1, T, nullptr, 0, stream);
}

int tqr_apply_qt_pairs(char trans, int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib,
                       const double* T, double* B, int64_t ldb, void* stream) {
  return apply_common(trans, m, n, nrhs, A, lda, nb, ib, 0, 1, T, B, ldb, stream);
}

int tqr_stream_status(void* stream) {
  int s = TQR_OK;
  if (read_status(&s, static_cast<cudaStream_t>(stream)) != cudaSuccess) return TQR_ERR_CUDA;
  return s;
}

int tqr_release_memory(void) { return release_memory(); }

int64_t tqr_set_wait_limit_ms(int64_t ms) {
  const int64_t old = g_wait_limit_ms;
  if (ms > 0) g_wait_limit_ms = ms;
  return old;
}

}  // extern "C"
