// tqr_noalloc.cu -- tqr_factor_noalloc: the tiled QR factorization with all
// of its device scratch in one file-scope static array, for callers that
// cannot allocate device memory (see include/tqr.h).
//
// The scratch holds the Block Data Layout tiles, the version counters, the
// instance descriptor, the control block and the task list.  Host code must
// not use the array's name as a device address: at set-up, once per device
// and with that device current, cudaGetSymbolAddress gives the address that
// is passed to the kernels.  The GPU work of a call reads no host memory: a
// set-up kernel receives the instance descriptor as a kernel parameter,
// writes it and Algorithm 1's task list (its sequential order, a
// topological order of the DAG) into the array and clears the counters and
// control words, so nothing the host keeps -- a stack frame, a host array
// the next call rewrites -- is referenced once the call has returned.
// Nothing is allocated on the device or on the host.
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
static std::mutex g_na_mu;

// Tasks of step k of Algorithm 1 with NS slab tasks per tile update:
// GEQRT(k), LARFB(k, j, s) for j > k, then per row i > k TSQRT(k, i) and
// SSRFB(k, i, j, s) for j > k.
__host__ __device__ inline long long na_step_tasks(int p, int q, int NS, int k) {
  const long long a = static_cast<long long>(q - k - 1) * NS;
  return 1 + a + static_cast<long long>(p - k - 1) * (1 + a);
}

static long long na_count(const Inst& I) {
  long long n = 0;
  for (int k = 0; k < I.kt; ++k) n += na_step_tasks(I.p, I.q, I.NS, k);
  return n;
}

// Writes the instance, Algorithm 1's tasks in sequential order, and zeroes
// the counters and the control block.  Task e belongs to the step k whose
// range of indices holds it; within the step its position gives its kind and
// indices (the order of na_step_tasks).
__global__ void na_setup_kernel(Inst I, Inst* __restrict__ dinst, TaskX* __restrict__ tasks, long long ntasks,
                                int* __restrict__ ctr, long long nctr, unsigned char* __restrict__ ctl) {
  const long long tid = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  if (tid == 0) *dinst = I;
  for (long long e = tid; e < 256; e += stride) ctl[e] = 0;
  for (long long e = tid; e < nctr; e += stride) ctr[e] = 0;
  for (long long e = tid; e < ntasks; e += stride) {
    int k = 0;
    long long off = 0;
    while (k < I.kt - 1 && off + na_step_tasks(I.p, I.q, I.NS, k) <= e) off += na_step_tasks(I.p, I.q, I.NS, k++);
    long long w = e - off;
    const long long a = static_cast<long long>(I.q - k - 1) * I.NS;
    TaskX t;
    t.inst = 0; t.k = k; t.l = 0; t.pad = 0;
    if (w == 0) {
      t.kind = K_GEQRT; t.i = k; t.j = k; t.s = 0;
    } else if (w <= a) {
      w -= 1;
      t.kind = K_LARFB; t.i = k; t.j = k + 1 + static_cast<int>(w / I.NS); t.s = static_cast<int>(w % I.NS);
    } else {
      w -= 1 + a;
      const long long row = w / (1 + a), pos = w % (1 + a);
      t.i = k + 1 + static_cast<int>(row);
      if (pos == 0) {
        t.kind = K_TSQRT; t.j = k; t.s = 0;
      } else {
        t.kind = K_SSRFB; t.j = k + 1 + static_cast<int>((pos - 1) / I.NS); t.s = static_cast<int>((pos - 1) % I.NS);
      }
    }
    tasks[e] = t;
  }
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
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (g_na_addr[dev] == nullptr) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || ptr == nullptr) return TQR_ERR_CUDA;
      g_na_addr[dev] = static_cast<char*>(ptr);
    }
    base = g_na_addr[dev];
  }
  const long long ntasks = na_count(I);
  if (ntasks > TQR_NOALLOC_MAX_TASKS) return TQR_ERR_TOO_LARGE;
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
  Inst* dinst = reinterpret_cast<Inst*>(base + kNaOffInst);
  // the counters and the control block must start at zero on every call
  // (the set-up kernel clears them); the tiles are fully rewritten by the
  // pack kernel, padding included
  const long long setup_items = ntasks > counters ? ntasks : counters;
  long long setup_grid = (setup_items + 255) / 256;
  if (setup_grid > 4LL * sms) setup_grid = 4LL * sms;
  if (setup_grid < 1) setup_grid = 1;
  na_setup_kernel<<<static_cast<int>(setup_grid), 256, 0, st>>>(I, dinst, dtasks, ntasks, I.ver, counters,
                                                                reinterpret_cast<unsigned char*>(base + kNaOffCtl));
  if (cudaGetLastError() != cudaSuccess) return TQR_ERR_CUDA;
  if (launch_pack<double>(A, lda, static_cast<int>(m), static_cast<int>(n), static_cast<double*>(I.A), I.p, I.q, nb,
                          sms, st) != cudaSuccess)
    return TQR_ERR_CUDA;
  if (launch_run<double>(dtasks, static_cast<int>(ntasks), dinst, base + kNaOffCtl, wait_limit_ns(),
                         static_cast<int>(grid), smem, st) != cudaSuccess)
    return TQR_ERR_CUDA;
  if (launch_unpack<double>(static_cast<double*>(I.A), I.p, nb, A, lda, static_cast<int>(m), static_cast<int>(n), sms,
                            st) != cudaSuccess)
    return TQR_ERR_CUDA;
  return TQR_OK;
}
