// tqr_server.cpp -- least-squares request server with continuous batching
// (tqr_server_* in include/tqr.h).
//
// Requests (A, B, precision class) enter a FIFO queue.  `slots` worker
// threads, each with its own CUDA stream, admit requests as soon as a slot is
// free and the HBM budget has room; the admitted requests' task graphs run
// concurrently on the device (each persistent launch is capped to
// grid_cap CTAs so several requests share the SMs), so a request that
// arrives while others are running starts at once instead of waiting for a
// batch boundary.  Factorizations stay resident (LRU, inside the budget)
// under the caller's matrix id: a later request with the same id and
// precision class skips the factorization and runs Q^T B and the back
// substitution only (plus refinement for the FP32 class).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <cstdio>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "tqr.h"
#include "tqr_api_internal.h"
#include "tqr_engine.h"
#include "tqr_ls.h"

namespace tqr {

using Clock = std::chrono::steady_clock;

struct Entry {                 // a resident factorization
  uint64_t id = 0;
  int prec = 0;
  LsJob job;
  char* ws = nullptr;
  size_t bytes = 0;              // ws plus ws64
  bool busy = false;
  int device = 0;
  // FP32 class only: the FP64 factorization of the resident copy of A, made
  // when FP32 refinement could not finish; later requests use it directly
  LsJob job64;
  char* ws64 = nullptr;
  bool has64 = false;
};

struct Request {
  uint64_t rid = 0, matrix = 0;
  int64_t m = 0, n = 0, nrhs = 0, lda = 0, ldb = 0, ldx = 0;
  const double* A = nullptr;
  const double* B = nullptr;
  double* X = nullptr;
  int prec = 0;
  double tol = 1e-12;
  Clock::time_point t_submit, t_start, t_end;
  bool done = false;
  int status = 0, iters = 0, reused = 0;
  double berr = 0;
  tqr_ls_info info = {};
};

}  // namespace tqr

struct tqr_server {
  size_t budget = 0;
  int slots = 1, grid_cap = 0, device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<tqr::Request>> pending;
  std::map<uint64_t, std::shared_ptr<tqr::Request>> reqs;
  std::list<std::shared_ptr<tqr::Entry>> cache;  // most recently used first
  size_t in_use = 0;                              // resident + running bytes
  uint64_t next_rid = 1;
  bool stop = false;
  // request workspaces come from the server's own stream-ordered pool, which
  // keeps freed memory (up to the budget) instead of returning it to the
  // driver at every synchronization, so admitting a request does not map
  // fresh physical memory
  cudaMemPool_t pool = nullptr;
  std::vector<std::thread> workers;
  std::vector<double> lat_ms;  // completed requests
  int64_t completed = 0, reused = 0, failed = 0;
  std::string last_failure;    // description of the latest failed request
  // sized least-squares jobs per (m, n, class): sizing picks the tile grid's
  // tree domain by a critical-path estimate per candidate (tens of ms for the
  // largest grids), done outside the lock the first time a shape arrives
  std::map<std::tuple<int64_t, int64_t, int>, std::pair<bool, tqr::LsJob>> shapes;
};

namespace tqr {

static std::shared_ptr<Entry> find_entry(tqr_server* S, const Request& R) {
  for (auto it = S->cache.begin(); it != S->cache.end(); ++it)
    if ((*it)->id == R.matrix && (*it)->prec == R.prec && (*it)->job.m == R.m && (*it)->job.n == R.n) return *it;
  return nullptr;
}

// Frees idle resident factorizations (least recently used first) until
// `need` more bytes fit in the budget.  Called with the lock held.
static bool make_room(tqr_server* S, size_t need, cudaStream_t st) {
  while (S->in_use + need > S->budget) {
    auto victim = S->cache.end();
    for (auto it = S->cache.begin(); it != S->cache.end(); ++it)
      if (!(*it)->busy) victim = it;
    if (victim == S->cache.end()) return false;
    cudaFreeAsync((*victim)->ws, st);
    if ((*victim)->ws64) cudaFreeAsync((*victim)->ws64, st);
    S->in_use -= (*victim)->bytes;
    S->cache.erase(victim);
  }
  return true;
}

// FP64 factorization of an FP32 entry's resident copy of A (its fallback);
// the extra bytes are returned for the budget's accounting.
static int make_fp64(tqr_server* S, Entry& E, cudaStream_t st, size_t* extra) {
  *extra = 0;
  if (!E.job64.init(E.job.m, E.job.n, E.job.rhs_cap, E.job.nb, E.job.ib, TQR_PREC_FP64, S->grid_cap))
    return TQR_ERR_UNSUPPORTED;
  if ((S->pool ? cudaMallocFromPoolAsync(reinterpret_cast<void**>(&E.ws64), E.job64.bytes, S->pool, st)
               : cudaMallocAsync(reinterpret_cast<void**>(&E.ws64), E.job64.bytes, st)) != cudaSuccess) {
    cudaGetLastError();
    E.ws64 = nullptr;
    return TQR_ERR_NOMEM;
  }
  E.job64.bind(E.ws64, false);
  *extra = E.job64.bytes;
  const int s = E.job64.factor_solve(E.job.Acopy, E.job.m, nullptr, 0, 0, st);
  if (s == TQR_OK) E.has64 = true;
  return s;
}

static void run_request(tqr_server* S, Request& R, cudaStream_t st, std::unique_lock<std::mutex>& lk,
                        std::shared_ptr<Entry> entry, bool fresh) {
  lk.unlock();
  int status = TQR_OK;
  Entry& E = *entry;
  const int nrhs = static_cast<int>(R.nrhs);
  size_t extra = 0;
  bool fp32_tried = false;
  if (fresh) {
    status = E.job.factor_solve(R.A, R.lda, R.B, R.ldb, nrhs, st);
    if (status == kLsFp32Range) {
      // A outside FP32's range: the entry keeps an FP64 factorization
      R.info.fp32_status = TQR_ERR_UNSUPPORTED;
      status = copy_cols(E.job.Acopy, sizeof(double) * R.m, R.A, sizeof(double) * R.lda, sizeof(double) * R.m, R.n,
                         cudaMemcpyDeviceToDevice, st) == cudaSuccess
                   ? make_fp64(S, E, st, &extra)
                   : TQR_ERR_CUDA;
      if (status == TQR_OK) status = E.job64.solve(R.B, R.ldb, nrhs, st);
    } else {
      fp32_tried = true;
    }
  } else if (E.has64) {
    status = E.job64.solve(R.B, R.ldb, nrhs, st);
  } else {
    status = E.job.solve(R.B, R.ldb, nrhs, st);
    fp32_tried = true;
  }
  LsJob& J = fp32_tried ? E.job : E.job64;
  if (status == TQR_OK) status = J.finish(E.job.Acopy, R.m, R.B, R.ldb, nrhs, R.X, R.ldx, R.tol, 40, &R.info, st);
  if (fp32_tried && E.prec == TQR_PREC_FP32 && status == kLsStalled) {
    // FP32 refinement could not finish: solve from an FP64 factorization of
    // the resident copy, kept for the entry's later requests
    const int s32 = status;
    const double b32 = R.info.berr;
    const int it32 = R.info.iters, in32 = R.info.inner_iters;
    const double g32 = R.info.gmres_res;
    status = make_fp64(S, E, st, &extra);
    if (status == TQR_OK) status = E.job64.solve(R.B, R.ldb, nrhs, st);
    if (status == TQR_OK) status = E.job64.finish(E.job.Acopy, R.m, R.B, R.ldb, nrhs, R.X, R.ldx, R.tol, 0, &R.info, st);
    R.info.fp32_status = s32 == kLsStalled ? TQR_ERR_NOCONV : s32;
    R.info.berr_fp32 = b32;
    R.info.iters = it32;
    R.info.inner_iters = in32;
    R.info.gmres_res = g32;
  }
  if (E.prec == TQR_PREC_FP32 && E.has64) R.info.path = TQR_LS_PATH_FP64_FALLBACK;
  if (status == kLsStalled || status == kLsFp32Range) status = TQR_ERR_NOCONV;
  R.iters = R.info.iters;
  R.berr = R.info.berr;
  // every launch of the request reported into its job's own error record
  // (read by finish); the device-wide sticky status is not read here, since
  // it mixes the concurrent requests' launches
  if (cudaStreamSynchronize(st) != cudaSuccess && status == TQR_OK) status = TQR_ERR_CUDA;
  std::string why;
  if (status != TQR_OK) {
    char msg[256];
    const double* e = E.job.err_host[0] != 0.0 ? E.job.err_host : E.job64.err_host;
    int len = std::snprintf(msg, sizeof msg, "request %llu (matrix %llu, %lld x %lld, %lld rhs, %s): status %d",
                            static_cast<unsigned long long>(R.rid), static_cast<unsigned long long>(R.matrix),
                            static_cast<long long>(R.m), static_cast<long long>(R.n), static_cast<long long>(R.nrhs),
                            R.prec == TQR_PREC_FP32 ? "fp32r" : "fp64", status);
    if (e[0] != 0.0 && len > 0 && len < static_cast<int>(sizeof msg))
      std::snprintf(msg + len, sizeof msg - len, "; task-kernel %s wait ran out in task kind %d (k %d i %d j %d s %d l %d)",
                    e[1] == 2.0 ? "bulk-copy" : e[1] == 1.0 ? "dependency" : "other", static_cast<int>(e[2]),
                    static_cast<int>(e[3]), static_cast<int>(e[4]), static_cast<int>(e[5]), static_cast<int>(e[6]),
                    static_cast<int>(e[7]));
    why = msg;
  }
  lk.lock();
  if (!why.empty()) S->last_failure = why;
  if (extra) {
    E.bytes += extra;
    S->in_use += extra;
  }
  R.status = status;
  R.reused = fresh ? 0 : 1;
  R.t_end = Clock::now();
  R.done = true;
  E.busy = false;
  if (fresh && !(status == TQR_OK || status == TQR_ERR_NOCONV)) {
    // a failed factorization is not kept
    for (auto it = S->cache.begin(); it != S->cache.end(); ++it)
      if (it->get() == &E) {
        cudaFreeAsync(E.ws, st);
        if (E.ws64) cudaFreeAsync(E.ws64, st);
        S->in_use -= E.bytes;
        S->cache.erase(it);
        break;
      }
  }
  S->completed++;
  if (!fresh) S->reused++;
  if (status != TQR_OK) S->failed++;
  S->lat_ms.push_back(std::chrono::duration<double, std::milli>(R.t_end - R.t_submit).count());
  S->cv_done.notify_all();
  S->cv_work.notify_all();
}

static void worker(tqr_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    // the first pending request that can run now: its resident factor is
    // idle, or there is room in the budget for a new factorization
    std::shared_ptr<Request> R;
    std::shared_ptr<Entry> entry;
    bool fresh = false;
    bool rescan = false;
    for (auto it = S->pending.begin(); it != S->pending.end() && !R; ++it) {
      std::shared_ptr<Entry> e = find_entry(S, **it);
      if (e) {
        if (e->busy) continue;  // same matrix running: keep FIFO per matrix
        R = *it;
        entry = e;
        S->pending.erase(it);
        break;
      }
      // a new factorization; only the head of the queue may evict, so large
      // requests are not starved by smaller ones behind them
      const auto key = std::make_tuple((*it)->m, (*it)->n, (*it)->prec);
      auto sized = S->shapes.find(key);
      if (sized == S->shapes.end()) {
        // size this shape without holding the lock, then scan again (the
        // queue may have changed meanwhile)
        const int64_t m = (*it)->m, n = (*it)->n;
        const int prec = (*it)->prec, cap = S->grid_cap;
        lk.unlock();
        int nb = 0, ib = 0;
        autotune(m, n, &nb, &ib);
        LsJob tmpl;
        const bool ok = tmpl.init(static_cast<int>(m), static_cast<int>(n), 16, nb, ib, prec, cap);
        lk.lock();
        if (S->shapes.size() >= 4096) S->shapes.clear();
        S->shapes.emplace(key, std::make_pair(ok, tmpl));
        rescan = true;
        break;
      }
      auto job = std::make_shared<Entry>();
      auto refuse = [&](int code) {
        (*it)->status = code;
        (*it)->t_start = (*it)->t_end = Clock::now();
        (*it)->done = true;
        char msg[160];
        std::snprintf(msg, sizeof msg, "request %llu (matrix %llu, %lld x %lld): refused at admission, status %d",
                      static_cast<unsigned long long>((*it)->rid), static_cast<unsigned long long>((*it)->matrix),
                      static_cast<long long>((*it)->m), static_cast<long long>((*it)->n), code);
        S->last_failure = msg;
        S->completed++;
        S->failed++;
        S->pending.erase(it);
        S->cv_done.notify_all();
      };
      job->job = sized->second.second;
      if (!sized->second.first) {
        refuse(TQR_ERR_UNSUPPORTED);
        break;
      }
      job->bytes = job->job.bytes_with_acopy();
      if (job->bytes > S->budget) {
        // can never be admitted: refuse it instead of waiting for room
        refuse(TQR_ERR_NOMEM);
        break;
      }
      const bool head = (it == S->pending.begin());
      if (S->in_use + job->bytes > S->budget && !(head && make_room(S, job->bytes, st))) {
        if (head) break;  // wait for memory to free up
        continue;
      }
      char* ws = nullptr;
      if ((S->pool ? cudaMallocFromPoolAsync(reinterpret_cast<void**>(&ws), job->bytes, S->pool, st)
                   : cudaMallocAsync(reinterpret_cast<void**>(&ws), job->bytes, st)) != cudaSuccess) {
        cudaGetLastError();
        break;  // device memory is short of the budget: retry after a completion
      }
      job->ws = ws;
      job->id = (*it)->matrix;
      job->prec = (*it)->prec;
      job->device = S->device;
      job->job.bind(ws, true);
      S->in_use += job->bytes;
      S->cache.push_front(job);
      R = *it;
      entry = job;
      fresh = true;
      S->pending.erase(it);
      break;
    }
    if (rescan) continue;
    if (R) {
      entry->busy = true;
      // move to the front of the LRU list
      for (auto it = S->cache.begin(); it != S->cache.end(); ++it)
        if (*it == entry) {
          S->cache.splice(S->cache.begin(), S->cache, it);
          break;
        }
      R->t_start = Clock::now();
      run_request(S, *R, st, lk, entry, fresh);
      continue;
    }
    if (S->stop && S->pending.empty()) break;
    S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    if (S->stop && S->pending.empty()) break;
  }
  lk.unlock();
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
}

}  // namespace tqr

using namespace tqr;

extern "C" {

int tqr_server_create(size_t hbm_budget_bytes, int slots, int grid_cap, tqr_server** out) {
  if (hbm_budget_bytes < (1u << 20)) return -1;
  if (slots < 1 || slots > 64) return -2;
  if (grid_cap < 0) return -3;
  if (out == nullptr) return -4;
  tqr_server* S = new tqr_server();
  S->budget = hbm_budget_bytes;
  S->slots = slots;
  cudaGetDevice(&S->device);
  const int sms = device_sms();
  // default: half the device's resident CTAs (2 per SM) with 8 slots, scaling
  // as 1/slots.  Measured with 8 slots against a quarter and 3/4 and all of
  // them: a large request finishes sooner with more CTAs, and the hardware
  // interleaves the CTAs of concurrent launches, so p99 at 60 req/s fell from
  // 495 to 255 ms (FP64) and 119 to 98 ms (refined FP32), and saturation rose
  // 3 % (FP64); larger caps lost throughput at saturation.
  S->grid_cap = grid_cap > 0 ? grid_cap : std::max(8, std::min(2 * sms, (8 * sms) / slots));
  {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    if (cudaMemPoolCreate(&S->pool, &props) == cudaSuccess) {
      uint64_t keep = hbm_budget_bytes;
      cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      cudaGetLastError();
      S->pool = nullptr;  // fall back to the device's default pool
    }
  }
  for (int a = 0; a < slots; ++a) S->workers.emplace_back(worker, S);
  *out = S;
  return TQR_OK;
}

int tqr_server_destroy(tqr_server* S) {
  if (S == nullptr) return -1;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& e : S->cache) {
    cudaFreeAsync(e->ws, nullptr);
    if (e->ws64) cudaFreeAsync(e->ws64, nullptr);
  }
  cudaDeviceSynchronize();
  if (S->pool) cudaMemPoolDestroy(S->pool);
  delete S;
  return TQR_OK;
}

int tqr_server_submit(tqr_server* S, uint64_t matrix_id, int64_t m, int64_t n, int64_t nrhs, const double* A,
                      int64_t lda, const double* B, int64_t ldb, double* X, int64_t ldx, int prec, double tol,
                      uint64_t* request) {
  if (S == nullptr) return -1;
  if (m < 1 || m > (1 << 30)) return -3;
  if (n < 1 || n > m) return -4;
  if (nrhs < 1 || nrhs > 16) return -5;
  if (A == nullptr || ptr_kind(A) != PTR_DEVICE) return -6;
  if (lda < m) return -7;
  if (B == nullptr || ptr_kind(B) != PTR_DEVICE) return -8;
  if (ldb < m) return -9;
  if (X == nullptr || ptr_kind(X) != PTR_DEVICE) return -10;
  if (ldx < n) return -11;
  if (prec != TQR_PREC_FP64 && prec != TQR_PREC_FP32) return -12;
  if (!(tol >= 0)) return -13;
  if (request == nullptr) return -14;
  auto R = std::make_shared<Request>();
  R->matrix = matrix_id;
  R->m = m;
  R->n = n;
  R->nrhs = nrhs;
  R->A = A;
  R->lda = lda;
  R->B = B;
  R->ldb = ldb;
  R->X = X;
  R->ldx = ldx;
  R->prec = prec;
  R->tol = tol;
  R->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    R->rid = S->next_rid++;
    S->reqs[R->rid] = R;
    S->pending.push_back(R);
    *request = R->rid;
  }
  S->cv_work.notify_one();
  return TQR_OK;
}

static int report(tqr_server* S, uint64_t request, bool wait, int* done, int* status, int* iters, double* berr,
                  double* latency_ms, int* reused, tqr_ls_info* info = nullptr) {
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(request);
  if (it == S->reqs.end()) return -2;
  std::shared_ptr<Request> R = it->second;
  if (wait)
    while (!R->done) S->cv_done.wait(lk);
  if (done) *done = R->done ? 1 : 0;
  if (!R->done) return TQR_OK;
  if (status) *status = R->status;
  if (iters) *iters = R->iters;
  if (berr) *berr = R->berr;
  if (reused) *reused = R->reused;
  if (info) *info = R->info;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(R->t_end - R->t_submit).count();
  S->reqs.erase(it);
  return TQR_OK;
}

int tqr_server_poll(tqr_server* S, uint64_t request, int* done, int* status, int* iters, double* berr,
                    double* latency_ms, int* reused) {
  if (S == nullptr) return -1;
  if (done == nullptr) return -3;
  return report(S, request, false, done, status, iters, berr, latency_ms, reused);
}

int tqr_server_wait(tqr_server* S, uint64_t request, int* status, int* iters, double* berr, double* latency_ms,
                    int* reused) {
  if (S == nullptr) return -1;
  int done = 0;
  return report(S, request, true, &done, status, iters, berr, latency_ms, reused);
}

int tqr_server_wait_info(tqr_server* S, uint64_t request, int* status, tqr_ls_info* info, double* latency_ms,
                         int* reused) {
  if (S == nullptr) return -1;
  int done = 0;
  return report(S, request, true, &done, status, nullptr, nullptr, latency_ms, reused, info);
}

int tqr_server_stats(tqr_server* S, double* out) {
  if (S == nullptr) return -1;
  if (out == nullptr) return -2;
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> l(S->lat_ms);
  std::sort(l.begin(), l.end());
  auto pct = [&l](double q) {
    if (l.empty()) return 0.0;
    size_t k = static_cast<size_t>(q * (l.size() - 1) + 0.5);
    return l[std::min(k, l.size() - 1)];
  };
  out[0] = static_cast<double>(S->completed);
  out[1] = pct(0.50);
  out[2] = pct(0.99);
  out[3] = static_cast<double>(S->in_use);
  out[4] = static_cast<double>(S->reused);
  out[5] = static_cast<double>(S->failed);
  out[6] = static_cast<double>(S->pending.size());
  out[7] = static_cast<double>(S->cache.size());
  return TQR_OK;
}

int tqr_debug_server_last_failure(tqr_server* S, char* buf, size_t len) {
  if (S == nullptr) return -1;
  if (buf == nullptr || len == 0) return -2;
  std::lock_guard<std::mutex> lk(S->mu);
  std::snprintf(buf, len, "%s", S->last_failure.c_str());
  return TQR_OK;
}

}  // extern "C"
