// tqr_noalloc.cu -- tqr_factor_noalloc: the tiled QR factorization with all
// of its device scratch in one file-scope static array, for callers that
// cannot allocate device memory (see include/tqr.h).
//
// The scratch holds the Block Data Layout tiles, the version counters, the
// instance descriptor, the control block and the task list.  Host code must
// not use the array's name as a device address: at set-up, once per device
// and with that device current, cudaGetSymbolAddress gives the address that
// is passed to the kernels.  The task list is written into a static host
// array (Algorithm 1's sequential order, a topological order of the DAG) and
// copied to the device; nothing is allocated on the device or on the host.
#include <cuda_runtime.h>

#include <mutex>

#include "tqr.h"
#include "tqr_api_internal.h"
#include "tqr_engine.h"

namespace tqr {

constexpr size_t kNaTileBytes = static_cast<size_t>(TQR_NOALLOC_MAX_TILE_ELEMS) * sizeof(double);
constexpr size_t kNaCtrBytes = static_cast<size_t>(TQR_NOALLOC_MAX_COUNTERS) * sizeof(int);
constexpr size_t kNaTaskBytes = static_cast<size_t>(TQR_NOALLOC_MAX_TASKS) * sizeof(TaskX);
constexpr size_t kNaOffCtr = kNaTileBytes;
constexpr size_t kNaOffTask = kNaOffCtr + kNaCtrBytes;
constexpr size_t kNaOffInst = kNaOffTask + kNaTaskBytes;
constexpr size_t kNaOffCtl = kNaOffInst + 256;
static_assert(sizeof(tqr::Inst) <= 256, "the instance slot of the static scratch is 256 bytes");
constexpr size_t kNaBytes = kNaOffCtl + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
static char* g_na_addr[kNaMaxDevices];   // device address of the array, per device
static TaskX g_na_tasks[TQR_NOALLOC_MAX_TASKS];
static std::mutex g_na_mu;

// Algorithm 1's tasks in sequential order, written into `out`; returns the
// count, or -1 if it would exceed `cap`.
static long long na_tasks(const Inst& I, TaskX* out, long long cap) {
  long long n = 0;
  auto put = [&](int kind, int k, int i, int j, int s) {
    if (n < cap) {
      TaskX& t = out[n];
      t.kind = kind; t.s = s; t.inst = 0; t.k = k; t.i = i; t.j = j; t.l = 0; t.pad = 0;
    }
    ++n;
  };
  for (int k = 0; k < I.kt; ++k) {
    put(K_GEQRT, k, k, k, 0);
    for (int j = k + 1; j < I.q; ++j)
      for (int s = 0; s < I.NS; ++s) put(K_LARFB, k, k, j, s);
    for (int i = k + 1; i < I.p; ++i) {
      put(K_TSQRT, k, i, k, 0);
      for (int j = k + 1; j < I.q; ++j)
        for (int s = 0; s < I.NS; ++s) put(K_SSRFB, k, i, j, s);
    }
  }
  return n <= cap ? n : -1;
}

}  // namespace tqr

using namespace tqr;

extern "C" int tqr_factor_noalloc(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* T,
                                  void* stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (lda < (m > 1 ? m : 1)) return -4;
  const int c = check_tiles(nb, ib, 5, 6);
  if (c) return c;
  if (m == 0 || n == 0) return TQR_OK;
  if (A == nullptr) return -3;
  if (T == nullptr) return -7;
  if (ptr_kind(A) != PTR_DEVICE) return -3;
  if (ptr_kind(T) != PTR_DEVICE) return -7;
  int cs, occ, smem;
  if (!choose_shape(nb, ib, sizeof(double), &cs, &occ, &smem)) return TQR_ERR_UNSUPPORTED;
  if (m > (1LL << 30) || n > (1LL << 30)) return TQR_ERR_TOO_LARGE;
  Inst I = make_inst(M_FACTOR, m, n, nb, ib, cs, 0, 0);
  const long long tile_elems = static_cast<long long>(I.p) * I.q * nb * nb;
  const long long counters = static_cast<long long>(I.p) * I.q * I.NS;
  if (tile_elems > TQR_NOALLOC_MAX_TILE_ELEMS || counters > TQR_NOALLOC_MAX_COUNTERS) return TQR_ERR_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return TQR_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (g_na_addr[dev] == nullptr) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) return TQR_ERR_CUDA;
    g_na_addr[dev] = static_cast<char*>(ptr);
  }
  char* base = g_na_addr[dev];
  const long long ntasks = na_tasks(I, g_na_tasks, TQR_NOALLOC_MAX_TASKS);
  if (ntasks < 0) return TQR_ERR_TOO_LARGE;
  I.A = base;
  I.B = nullptr;
  I.T = T;
  I.ver = reinterpret_cast<int*>(base + kNaOffCtr);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TQR_ERR_CUDA;
  long long grid = static_cast<long long>(sms) * occ;
  if (grid > ntasks) grid = ntasks;
  if (grid < 1) grid = 1;
  TaskX* dtasks = reinterpret_cast<TaskX*>(base + kNaOffTask);
  // the counters and the control block must start at zero on every call;
  // the tiles are fully rewritten by the pack kernel (padding included)
  if (cudaMemsetAsync(base + kNaOffCtr, 0, sizeof(int) * counters, st) != cudaSuccess ||
      cudaMemsetAsync(base + kNaOffCtl, 0, 256, st) != cudaSuccess ||
      cudaMemcpyAsync(dtasks, g_na_tasks, sizeof(TaskX) * ntasks, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + kNaOffInst, &I, sizeof(Inst), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return TQR_ERR_CUDA;
  if (launch_pack<double>(A, lda, static_cast<int>(m), static_cast<int>(n), static_cast<double*>(I.A), I.p, I.q, nb,
                          sms, st) != cudaSuccess)
    return TQR_ERR_CUDA;
  if (launch_run<double>(dtasks, static_cast<int>(ntasks), reinterpret_cast<const Inst*>(base + kNaOffInst),
                         base + kNaOffCtl, wait_limit_ns(), static_cast<int>(grid), smem, st) != cudaSuccess)
    return TQR_ERR_CUDA;
  if (launch_unpack<double>(static_cast<double*>(I.A), I.p, nb, A, lda, static_cast<int>(m), static_cast<int>(n), sms,
                            st) != cudaSuccess)
    return TQR_ERR_CUDA;
  return TQR_OK;
}
