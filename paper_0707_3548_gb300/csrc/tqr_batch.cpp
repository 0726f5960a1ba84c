// tqr_batch.cpp -- many independent factorizations in one persistent launch
// (tqr_batch_submit / tqr_batch_poll / tqr_batch_wait) and the tile-size
// autotuner (tqr_autotune).
//
// A batch is one global task list over all its matrices: every matrix keeps
// its own tiles, T, version counters and (nb, ib), and its tasks are merged
// into a single priority order (decreasing longest remaining path), so the
// tiles of all instances interleave on the SMs of one persistent kernel.
// The batch's device work -- descriptor upload, counter reset, batched pack,
// the task kernel, batched unpack and the status read-back -- is captured once
// per batch shape in a CUDA graph; resubmitting a batch of the same shapes
// (any matrices) refills a pinned descriptor buffer and relaunches the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "tqr.h"
#include "tqr_api_internal.h"
#include "tqr_engine.h"
#include "tqr_plan.h"

namespace tqr {

// ---------------------------------------------------------------- autotuner
// Tile sizes for batched factorizations, from measurement: on a 4096-matrix
// batch (m log-uniform in [64, 2048], n uniform in [32, m]) one nb = 128,
// ib = 16 for every matrix beat every other uniform choice (nb 64, 96, 128 x
// ib 16, 32) and a cost-model choice that mixed nb = 32 .. 256 by half-octave
// size class (0.829 against 0.757 .. 0.821 and 0.790 TFLOP/s): the update
// kernels lose more to small tiles than padding costs.  Matrices smaller
// than 128 take the smallest power of two that holds them (at least 16).
// A class measured by tqr_autotune_run (tqr_tune.cu) answers from the
// tuner's table instead.
void autotune(int64_t m, int64_t n, int* nb_out, int* ib_out) {
  if (tune_lookup(m, n, nb_out, ib_out)) return;
  const int64_t mx = std::max(m, n);
  int nb = 16;
  while (nb < 128 && nb < mx) nb *= 2;
  *nb_out = nb;
  *ib_out = std::min(16, nb);
}

// ---------------------------------------------------------------- plans
struct BatchPlan {
  std::vector<std::tuple<int64_t, int64_t, int, int>> shape;  // (m, n, nb, ib) per item
  int count = 0;
  int device = -1;
  int pair = 0;                // 2b x b bottoms (tqr_batch_submit_pairs)
  int smem = 0, grid = 0, ntasks = 0;
  PlanStats stats;
  char* ws = nullptr;          // tiles + counters + control, device
  size_t ws_bytes = 0, ver_off = 0, ver_bytes = 0, ctl_off = 0;
  Inst* d_insts = nullptr;     // device
  PackDesc* d_pack = nullptr;  // device
  TaskX* d_tasks = nullptr;    // device
  Inst* h_insts = nullptr;     // pinned
  PackDesc* h_pack = nullptr;  // pinned
  int* h_status = nullptr;     // pinned
  int* d_bad = nullptr;        // device: per-matrix non-finite flags
  int* h_bad = nullptr;        // pinned copy of d_bad
  std::vector<size_t> tile_off, ctr_off;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  ~BatchPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (done) cudaEventDestroy(done);
    if (ws) cudaFree(ws);
    if (d_insts) cudaFree(d_insts);
    if (d_pack) cudaFree(d_pack);
    if (d_tasks) cudaFree(d_tasks);
    if (d_bad) cudaFree(d_bad);
    if (h_bad) cudaFreeHost(h_bad);
    if (h_insts) cudaFreeHost(h_insts);
    if (h_pack) cudaFreeHost(h_pack);
    if (h_status) cudaFreeHost(h_status);
  }
};

static std::mutex g_bmu;
static std::vector<std::shared_ptr<BatchPlan>> g_bplans;  // most recent first
static const size_t kMaxBatchPlans = 4;
struct Ticket {
  std::shared_ptr<BatchPlan> plan;
  int count;
  bool finished;
  int status;
  std::vector<int> item;  // per-matrix statuses, copied out when finished
};
static std::map<uint64_t, Ticket> g_tickets;
static uint64_t g_next_ticket = 1;

static size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Marks a ticket finished (its plan's launch done, or failed) and copies its
// statuses out of the plan's read-back buffers, before a later submission of
// the same plan can overwrite them.  Called with g_bmu held.
static void finish_ticket(Ticket& T, cudaError_t e) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    T.status = TQR_ERR_CUDA;
  } else {
    T.status = T.plan->h_status[1] != 0 ? TQR_ERR_TIMEOUT : TQR_OK;
  }
  // a matrix with a NaN or an infinity reports TQR_ERR_NONFINITE (the others
  // of the batch are unaffected: every matrix has its own tiles and DAG)
  T.item.assign(T.count, TQR_OK);
  for (int a = 0; a < T.count; ++a)
    T.item[a] = T.status != TQR_OK ? T.status : (T.plan->h_bad[a] != 0 ? TQR_ERR_NONFINITE : TQR_OK);
  T.finished = true;
  T.plan->busy = false;
}

static int build_batch_plan(const std::vector<std::tuple<int64_t, int64_t, int, int>>& shape, int pair,
                            std::shared_ptr<BatchPlan>* out) {
  auto P = std::make_shared<BatchPlan>();
  P->shape = shape;
  P->pair = pair;
  P->count = static_cast<int>(shape.size());
  cudaGetDevice(&P->device);
  std::vector<Inst> insts(shape.size());
  size_t off = 0;
  P->tile_off.resize(shape.size());
  P->ctr_off.resize(shape.size());
  int max_smem = 0, min_occ = 2;
  for (size_t a = 0; a < shape.size(); ++a) {
    const int64_t m = std::get<0>(shape[a]), n = std::get<1>(shape[a]);
    const int nb = std::get<2>(shape[a]), ib = std::get<3>(shape[a]);
    int cs, occ, smem;
    if (!choose_shape(nb, ib, 8, &cs, &occ, &smem, pair ? 2 * nb : 0)) return TQR_ERR_UNSUPPORTED;
    max_smem = std::max(max_smem, smem);
    min_occ = std::min(min_occ, occ);
    insts[a] = make_inst(M_FACTOR, m, n, nb, ib, cs, 0, 0);
    insts[a].pair = pair;
    P->tile_off[a] = off;
    off += al256(sizeof(double) * static_cast<size_t>(insts[a].p) * insts[a].q * nb * nb);
  }
  P->ver_off = off;
  for (size_t a = 0; a < shape.size(); ++a) {
    P->ctr_off[a] = off;
    off += al256(sizeof(int) * static_cast<size_t>(insts[a].p) * insts[a].q * insts[a].NS);
  }
  P->ctl_off = off;
  P->ver_bytes = off - P->ver_off + al256(ctl_bytes());
  off += al256(ctl_bytes());
  P->ws_bytes = off;
  // global task list
  std::vector<TaskX> seq, ordered;
  for (size_t a = 0; a < shape.size(); ++a) seq_tasks(insts[a], static_cast<int>(a), seq);
  P->ntasks = static_cast<int>(seq.size());
  const int sms = device_sms();
  P->grid = std::max(1, std::min(sms * min_occ, P->ntasks));
  P->smem = max_smem;
  std::string err;
  if (!order_bottom_level(insts, seq, 8, min_occ, P->grid, ordered, &P->stats, &err)) {
    set_last_error(err);
    return TQR_ERR_UNSUPPORTED;
  }
  if (cudaMalloc(&P->ws, P->ws_bytes) != cudaSuccess ||
      cudaMalloc(&P->d_insts, sizeof(Inst) * shape.size()) != cudaSuccess ||
      cudaMalloc(&P->d_pack, sizeof(PackDesc) * shape.size()) != cudaSuccess ||
      cudaMalloc(&P->d_tasks, sizeof(TaskX) * std::max<size_t>(1, ordered.size())) != cudaSuccess ||
      cudaMallocHost(&P->h_insts, sizeof(Inst) * shape.size()) != cudaSuccess ||
      cudaMallocHost(&P->h_pack, sizeof(PackDesc) * shape.size()) != cudaSuccess ||
      cudaMallocHost(&P->h_status, sizeof(int) * 4) != cudaSuccess ||
      cudaMalloc(&P->d_bad, sizeof(int) * shape.size()) != cudaSuccess ||
      cudaMallocHost(&P->h_bad, sizeof(int) * shape.size()) != cudaSuccess) {
    cudaGetLastError();
    return TQR_ERR_NOMEM;
  }
  if (!ordered.empty() &&
      cudaMemcpy(P->d_tasks, ordered.data(), sizeof(TaskX) * ordered.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return TQR_ERR_CUDA;
  for (size_t a = 0; a < shape.size(); ++a) {
    Inst I = insts[a];
    I.A = P->ws + P->tile_off[a];
    I.B = nullptr;
    I.T = nullptr;  // per submit
    I.ver = reinterpret_cast<int*>(P->ws + P->ctr_off[a]);
    P->h_insts[a] = I;
    PackDesc& d = P->h_pack[a];
    d.A = nullptr;
    d.lda = 0;
    d.Ab = I.A;
    d.m = I.m;
    d.n = I.n;
    d.p = I.p;
    d.q = I.q;
    d.nb = I.nb;
    d.pad = 0;
  }
  if (cudaEventCreateWithFlags(&P->done, cudaEventDisableTiming) != cudaSuccess) return TQR_ERR_CUDA;
  // capture the batch's device work once
  int occ_dummy = 0;
  if (occupancy<double>(P->smem, &occ_dummy) != cudaSuccess) return TQR_ERR_CUDA;
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return TQR_ERR_CUDA;
  cudaGraph_t graph = nullptr;
  int status = TQR_OK;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) status = TQR_ERR_CUDA;
  if (status == TQR_OK) {
    const size_t n = shape.size();
    if (cudaMemcpyAsync(P->d_insts, P->h_insts, sizeof(Inst) * n, cudaMemcpyHostToDevice, cap) != cudaSuccess ||
        cudaMemcpyAsync(P->d_pack, P->h_pack, sizeof(PackDesc) * n, cudaMemcpyHostToDevice, cap) != cudaSuccess ||
        cudaMemsetAsync(P->ws + P->ver_off, 0, P->ver_bytes, cap) != cudaSuccess ||
        cudaMemsetAsync(P->d_bad, 0, sizeof(int) * n, cap) != cudaSuccess ||
        launch_pack_batched<double>(P->d_pack, P->count, cap, P->d_bad) != cudaSuccess ||
        (P->ntasks > 0 && launch_run<double>(P->d_tasks, P->ntasks, P->d_insts, P->ws + P->ctl_off, wait_limit_ns(),
                                             P->grid, P->smem, cap, P->pair ? 2 : 0) != cudaSuccess) ||
        launch_unpack_batched<double>(P->d_pack, P->count, cap) != cudaSuccess ||
        cudaMemcpyAsync(P->h_status, P->ws + P->ctl_off, sizeof(int) * 4, cudaMemcpyDeviceToHost, cap) !=
            cudaSuccess ||
        cudaMemcpyAsync(P->h_bad, P->d_bad, sizeof(int) * n, cudaMemcpyDeviceToHost, cap) != cudaSuccess)
      status = TQR_ERR_CUDA;
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    if (e != cudaSuccess) status = TQR_ERR_CUDA;
  }
  if (status == TQR_OK && cudaGraphInstantiate(&P->exec, graph, 0) != cudaSuccess) status = TQR_ERR_CUDA;
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  cudaGetLastError();
  if (status != TQR_OK) return status;
  *out = P;
  return TQR_OK;
}

}  // namespace tqr

using namespace tqr;

extern "C" {

int tqr_autotune(int64_t m, int64_t n, int* nb, int* ib) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (nb == nullptr) return -3;
  if (ib == nullptr) return -4;
  autotune(m, n, nb, ib);
  return TQR_OK;
}

static int batch_submit(int count, const tqr_desc* d, int pair, uint64_t* ticket, void* stream) {
  if (count < 1) return -1;
  if (d == nullptr) return -2;
  if (ticket == nullptr) return -3;
  std::vector<std::tuple<int64_t, int64_t, int, int>> shape(static_cast<size_t>(count));
  for (int a = 0; a < count; ++a) {
    const tqr_desc& x = d[a];
    int nb = x.nb, ib = x.ib;
    if (nb == 0 && ib == 0) autotune(x.m, x.n, &nb, &ib);
    if (x.m < 1 || x.n < 1 || x.m > (1 << 30) || x.n > (1 << 30) || x.A == nullptr || x.T == nullptr ||
        x.lda < x.m || check_tiles(nb, ib, 1, 2) != 0)
      return -2;
    if (ptr_kind(x.A) != PTR_DEVICE || ptr_kind(x.T) != PTR_DEVICE) return -2;
    shape[a] = std::make_tuple(x.m, x.n, nb, ib);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(g_bmu);
  int dev = 0;
  cudaGetDevice(&dev);
  std::shared_ptr<BatchPlan> P;
  for (size_t a = 0; a < g_bplans.size(); ++a)
    if (g_bplans[a]->device == dev && g_bplans[a]->pair == pair && g_bplans[a]->shape == shape) {
      P = g_bplans[a];
      g_bplans.erase(g_bplans.begin() + a);
      g_bplans.insert(g_bplans.begin(), P);
      break;
    }
  if (!P) {
    const int s = build_batch_plan(shape, pair, &P);
    if (s != TQR_OK) return s;
    g_bplans.insert(g_bplans.begin(), P);
    while (g_bplans.size() > kMaxBatchPlans) g_bplans.pop_back();
  }
  if (P->busy) {
    const cudaError_t q = cudaEventQuery(P->done);
    if (q == cudaErrorNotReady) return TQR_ERR_BUSY;
    // the previous batch on this plan finished unpolled: keep its statuses
    for (auto& kv : g_tickets)
      if (kv.second.plan == P && !kv.second.finished) finish_ticket(kv.second, q);
    P->busy = false;
  }
  for (int a = 0; a < count; ++a) {
    P->h_insts[a].T = d[a].T;
    P->h_pack[a].A = d[a].A;
    P->h_pack[a].lda = d[a].lda;
  }
  if (cudaGraphLaunch(P->exec, st) != cudaSuccess || cudaEventRecord(P->done, st) != cudaSuccess) {
    cudaGetLastError();
    return TQR_ERR_CUDA;
  }
  P->busy = true;
  const uint64_t t = g_next_ticket++;
  g_tickets[t] = Ticket{P, count, false, TQR_OK, {}};
  *ticket = t;
  return TQR_OK;
}

int tqr_batch_submit(int count, const tqr_desc* d, uint64_t* ticket, void* stream) {
  return batch_submit(count, d, 0, ticket, stream);
}

int tqr_batch_submit_pairs(int count, const tqr_desc* d, uint64_t* ticket, void* stream) {
  return batch_submit(count, d, 1, ticket, stream);
}

static int poll_locked(uint64_t ticket, bool wait, int* done, int* status_per_item) {
  auto it = g_tickets.find(ticket);
  if (it == g_tickets.end()) return -1;
  Ticket& T = it->second;
  if (!T.finished) {
    cudaError_t e = wait ? cudaEventSynchronize(T.plan->done) : cudaEventQuery(T.plan->done);
    if (e == cudaErrorNotReady) {
      if (done) *done = 0;
      return TQR_OK;
    }
    finish_ticket(T, e);
  }
  if (done) *done = 1;
  int s = T.status;
  for (int a = 0; a < T.count; ++a) {
    if (status_per_item) status_per_item[a] = T.item[a];
    if (s == TQR_OK) s = T.item[a];
  }
  g_tickets.erase(it);
  return s;
}

int tqr_batch_poll(uint64_t ticket, int* done, int* status_per_item) {
  if (done == nullptr) return -2;
  std::lock_guard<std::mutex> lk(g_bmu);
  return poll_locked(ticket, false, done, status_per_item);
}

int tqr_batch_wait(uint64_t ticket, int* status_per_item) {
  std::lock_guard<std::mutex> lk(g_bmu);
  int done = 0;
  return poll_locked(ticket, true, &done, status_per_item);
}

}  // extern "C"
