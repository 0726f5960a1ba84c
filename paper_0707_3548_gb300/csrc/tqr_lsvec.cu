// tqr_lsvec.cu -- kernels for the refinement of least-squares solutions with
// few right-hand sides: triangular solves with the tiled R and products with
// an explicit thin Q, for one to kMaxVecRhs right-hand sides.
//
// The refinement steps apply R^-1, R^-T, Q and Q^T to single vectors many
// times.  Run through the tile task graph, each of those is a chain of small
// tasks (about 40 us each); here they are one launch each:
//  * trsv_kernel: R x = y or R^T x = y by blocked substitution on the Block
//    Data Layout tiles of the factorization (R on and above the diagonal of
//    tile row k).  Each CTA takes the next tile row in solve order with one
//    atomic ticket, accumulates the contributions of the rows solved before
//    it as they are published (acquire loads of per-row flags), solves its
//    diagonal triangle by substitution -- so the solve keeps the backward
//    stability of triangular substitution -- and publishes its rows.
//    Tickets follow the solve order, so the earliest unsolved row never waits
//    and no co-residency of the CTAs is needed.  Waits are bounded: on expiry
//    the kernel records an error and every CTA returns.
//  * q1t_kernel / q1n_kernel: d = Q1^T f and u = f - Q1 y with the explicit
//    thin Q1 (m x n) held in tiles, FP32 products summed per tile and the
//    partial sums over tiles combined in FP64 in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "tqr.h"
#include "tqr_api_internal.h"
#include "tqr_ls.h"

namespace tqr {

constexpr int kVecThreads = 256;

__device__ __forceinline__ long long vec_globaltimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire_flag(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_flag(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Control words of one trsv launch: [0] ticket, [1] abort, [2] error, then
// one flag per tile row (all zero before the launch).
struct TrsvCtl {
  int ticket, abort, error, pad;
};

// Waits (thread 0) until flag f is set; false if the wait ran out or another
// CTA aborted.  The result is broadcast through shared memory.
__device__ bool wait_flag(const int* f, TrsvCtl* ctl, long long limit_ns, int* s_ok, double* err_out) {
  if (threadIdx.x == 0) {
    int ok = 1;
    const long long t0 = vec_globaltimer();
    while (ld_acquire_flag(f) == 0) {
      if (ld_acquire_flag(&ctl->abort) != 0) {
        ok = 0;
        break;
      }
      if (vec_globaltimer() - t0 > limit_ns) {
        atomicExch(&ctl->error, TQR_ERR_TIMEOUT);
        atomicExch(&ctl->abort, 1);
        if (err_out) *err_out = static_cast<double>(TQR_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(100);
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// One tile (nb x nb, column-major, 16-byte aligned) in 16-byte pieces: each
// thread holds up to kTileChunks of them in registers, so the loads of the
// next tile are in flight while the current one is used or a flag awaited.
constexpr int kTileChunks = 16;

template <typename real>
__device__ __forceinline__ void tile_fetch(const real* tile, int nb, uint4 (&buf)[kTileChunks]) {
  const int chunks = nb * nb * static_cast<int>(sizeof(real)) / 16;
  const uint4* src = reinterpret_cast<const uint4*>(tile);
#pragma unroll
  for (int i = 0; i < kTileChunks; ++i) {
    const int e = threadIdx.x + i * kVecThreads;
    if (e < chunks) buf[i] = __ldcg(src + e);
  }
}

// The fetched tile into shared memory with leading dimension ldt (nb + 1:
// row and column walks across lanes both fall on distinct banks).
template <typename real>
__device__ __forceinline__ void tile_store(const uint4 (&buf)[kTileChunks], int nb, real* sT, int ldt) {
  constexpr int per = 16 / static_cast<int>(sizeof(real));
  const int chunks = nb * nb * static_cast<int>(sizeof(real)) / 16;
#pragma unroll
  for (int i = 0; i < kTileChunks; ++i) {
    const int e = threadIdx.x + i * kVecThreads;
    if (e < chunks) {
      const real* v = reinterpret_cast<const real*>(&buf[i]);
      const int lin = e * per, r = lin % nb, c = lin / nb;  // nb % per == 0: one column per piece
#pragma unroll
      for (int q = 0; q < per; ++q) sT[r + q + c * ldt] = v[q];
    }
  }
}

// R X = Y (TRANS false, rows solved from the last tile row up) or
// R^T X = Y (TRANS true, from the first down).  R: the upper triangle of the
// tiles (k, j), j >= k, of an n-column factorization (tile rows 0 .. qn-1,
// qn = ceil(n / nb)), p tile rows in the BDL array.  Y, X: n x nrhs, FP64,
// column-major; X may alias Y.  Requires nb * nb * sizeof(real) <= 16
// kTileChunks kVecThreads bytes and nb <= 128 (four rows per lane in the
// substitution).  Dynamic shared memory: trsv_smem.
template <typename real, bool TRANS>
__global__ void __launch_bounds__(kVecThreads) trsv_kernel(const real* __restrict__ A, int p, int nb, int n,
                                                           int nrhs, const double* Y, long long ldy, double* X,
                                                           long long ldx, int* ctl_words, long long limit_ns,
                                                           double* err_out) {
  extern __shared__ __align__(16) unsigned char vec_smem[];
  const int ld = nb + 1;
  real* sT = reinterpret_cast<real*>(vec_smem);  // off-diagonal tiles, then the diagonal one
  real* sD = sT;
  real* sC = sT + nb * ld;                        // right-hand side, then solution (nb x nrhs)
  real* sV = sC + nb * nrhs;                      // a published block (nb x nrhs)
  real* sP = sV + nb * nrhs;                      // partial sums (kVecThreads x nrhs)
  real* sRd = sP + kVecThreads * nrhs;            // reciprocals of the diagonal
  __shared__ int s_row, s_ok;
  TrsvCtl* ctl = reinterpret_cast<TrsvCtl*>(ctl_words);
  int* flags = ctl_words + 4;
  const int qn = (n + nb - 1) / nb;
  const long long nb2 = static_cast<long long>(nb) * nb;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int parts = kVecThreads / nb;             // threads per row (column) of a tile product
  const int u = tid % nb, h = tid / nb;
  uint4 buf[kTileChunks];
  for (;;) {
    if (tid == 0) s_row = ld_acquire_flag(&ctl->abort) != 0 ? qn : atomicAdd(&ctl->ticket, 1);
    __syncthreads();
    const int t = s_row;
    __syncthreads();
    if (t >= qn) return;
    const int k = TRANS ? t : qn - 1 - t;        // tile row solved by this ticket
    const int r0 = k * nb;
    const int rows = min(nb, n - r0);
    const real* Dk = A + (static_cast<long long>(k) + static_cast<long long>(k) * p) * nb2;
    for (int e = tid; e < nb * nrhs; e += kVecThreads) {
      const int r = e % nb, c = e / nb;
      sC[e] = r < rows ? static_cast<real>(Y[r0 + r + c * ldy]) : real(0);
    }
    // contributions of the rows solved before this one, in solve order; the
    // next tile (the diagonal one after the last) is fetched while the
    // current one is used
    const int nl = TRANS ? k : qn - 1 - k;
    auto off_tile = [&](int l) {
      return TRANS ? A + (static_cast<long long>(l) + static_cast<long long>(k) * p) * nb2   // tile (l, k)
                   : A + (static_cast<long long>(k) + static_cast<long long>(l) * p) * nb2;  // tile (k, l)
    };
    tile_fetch(nl > 0 ? off_tile(TRANS ? 0 : qn - 1) : Dk, nb, buf);
    for (int a = 0; a < nl; ++a) {
      const int l = TRANS ? a : qn - 1 - a;
      if (!wait_flag(&flags[l], ctl, limit_ns, &s_ok, err_out)) return;
      tile_store(buf, nb, sT, ld);
      tile_fetch(a + 1 < nl ? off_tile(TRANS ? a + 1 : qn - 2 - a) : Dk, nb, buf);
      const int lrows = min(nb, n - l * nb);
      for (int e = tid; e < nb * nrhs; e += kVecThreads) {
        const int r = e % nb, c = e / nb;
        sV[e] = r < lrows ? static_cast<real>(__ldcg(X + l * nb + r + c * ldx)) : real(0);
      }
      __syncthreads();
      // R^T: C(u) -= sum_w T(w, u) V(w);  R: C(u) -= sum_w T(u, w) V(w);
      // thread (u, h) sums its part of w
      if (h < parts) {
        const int w0 = h * nb / parts, w1 = (h + 1) * nb / parts;
        for (int c = 0; c < nrhs; ++c) {
          real acc = real(0);
          const real* vv = sV + c * nb;
          if (TRANS) {
            for (int w = w0; w < w1; ++w) acc = fma(sT[w + u * ld], vv[w], acc);
          } else {
            for (int w = w0; w < w1; ++w) acc = fma(sT[u + w * ld], vv[w], acc);
          }
          sP[c * kVecThreads + h * nb + u] = acc;
        }
      }
      __syncthreads();
      for (int e = tid; e < nb * nrhs; e += kVecThreads) {
        const int r = e % nb, c = e / nb;
        real acc = real(0);
        for (int hh = 0; hh < parts; ++hh) acc += sP[c * kVecThreads + hh * nb + r];
        sC[e] -= acc;
      }
      __syncthreads();
    }
    __syncthreads();
    tile_store(buf, nb, sD, ld);  // the diagonal tile
    __syncthreads();
    for (int e = tid; e < rows; e += kVecThreads) sRd[e] = real(1) / sD[e + e * ld];
    __syncthreads();
    // substitution with the diagonal triangle in blocks of 32 rows: warp 0
    // solves a block with the right-hand side and the block's triangle in
    // registers (lane i owns row i of the block), then every thread folds
    // the block's solution into the rows still to be solved.
    // R^T (lower): x_s = c_s / d_s, c_i -= D(s, i) x_s for i > s;
    // R (upper):   the same from the last row up, with D(i, s), i < s.
    const int nblk = (rows + 31) / 32;
    for (int bb = 0; bb < nblk; ++bb) {
      const int b = TRANS ? bb : nblk - 1 - bb;
      const int base = 32 * b, i = base + lane;
      if (wid == 0) {
        real Lrow[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const int col = base + t;
          Lrow[t] = (i < rows && col < rows) ? (TRANS ? sD[col + i * ld] : sD[i + col * ld]) : real(0);
        }
        for (int c = 0; c < nrhs; ++c) {
          real v = i < rows ? sC[i + c * nb] : real(0);
#pragma unroll
          for (int tt = 0; tt < 32; ++tt) {
            const int t = TRANS ? tt : 31 - tt;
            if (base + t >= rows) continue;  // uniform over the warp
            const real xs = __shfl_sync(0xffffffffu, v * sRd[base + t], t);
            if (lane == t) {
              v = xs;
            } else if (TRANS ? lane > t : lane < t) {
              v = fma(-Lrow[t], xs, v);
            }
          }
          if (i < rows) sC[i + c * nb] = v;
        }
      }
      __syncthreads();
      // rows outside the block: R^T the rows after it, R the rows before it
      const int o0 = TRANS ? base + 32 : 0, o1 = TRANS ? rows : base;
      const int bw = min(32, rows - base);
      for (int e = tid; e < (o1 - o0) * nrhs; e += kVecThreads) {
        const int w = o0 + e % (o1 - o0), c = e / (o1 - o0);
        real acc = real(0);
        for (int t = 0; t < bw; ++t)
          acc = fma(TRANS ? sD[(base + t) + w * ld] : sD[w + (base + t) * ld], sC[base + t + c * nb], acc);
        sC[w + c * nb] -= acc;
      }
      __syncthreads();
    }
    for (int e = tid; e < rows * nrhs; e += kVecThreads) {
      const int r = e % rows, c = e / rows;
      X[r0 + r + c * ldx] = static_cast<double>(sC[r + c * nb]);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release_flag(&flags[k], 1);
  }
}

// d(j, c) partial sums = sum over the tile rows of split s of Q1(r, j) f(r, c):
// grid (tile columns, splits, nrhs); one warp per column of the tile column,
// lanes over rows.  part: splits x n x nrhs (FP32 sums of one split).
__global__ void __launch_bounds__(kVecThreads) q1t_partial(const float* __restrict__ Q, int p, int nb, int m,
                                                           int n, const double* __restrict__ F, long long ldf,
                                                           float fscale, int rows_per_split,
                                                           float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char vec_smem[];
  float* sf = reinterpret_cast<float*>(vec_smem);         // rows_per_split tiles of f
  const int jt = blockIdx.x, s = blockIdx.y, c = blockIdx.z;
  const int i0 = s * rows_per_split, i1 = min(p, i0 + rows_per_split);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < (i1 - i0) * nb; e += kVecThreads) {
    const int r = i0 * nb + e;
    sf[e] = r < m ? static_cast<float>(F[r + c * ldf]) * fscale : 0.0f;
  }
  __syncthreads();
  const long long nb2 = static_cast<long long>(nb) * nb;
  for (int jj = wid; jj < nb; jj += kVecThreads / 32) {
    const int j = jt * nb + jj;
    float acc = 0.0f;
    for (int i = i0; i < i1; ++i) {
      const float* col = Q + (static_cast<long long>(i) + static_cast<long long>(jt) * p) * nb2 +
                         static_cast<long long>(jj) * nb;
      for (int r = lane; r < nb; r += 32) acc = fmaf(col[r], sf[(i - i0) * nb + r], acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && j < n) part[(static_cast<long long>(s) * gridDim.z + c) * n + j] = acc;
  }
}

// U(r, c) partial sums over the tile columns of split s of Q1(r, j) Y(j, c):
// grid (tile rows, splits, nrhs), one thread per row of the tile row.
// part: splits x m x nrhs.
__global__ void __launch_bounds__(kVecThreads) q1n_partial(const float* __restrict__ Q, int p, int nb, int m,
                                                           int n, const double* __restrict__ Yv, long long ldy,
                                                           float yscale, int cols_per_split,
                                                           float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char vec_smem[];
  float* sy = reinterpret_cast<float*>(vec_smem);         // cols_per_split tiles of y
  const int it = blockIdx.x, s = blockIdx.y, c = blockIdx.z;
  const int qn = (n + nb - 1) / nb;
  const int j0 = s * cols_per_split, j1 = min(qn, j0 + cols_per_split);
  for (int e = threadIdx.x; e < (j1 - j0) * nb; e += kVecThreads) {
    const int j = j0 * nb + e;
    sy[e] = j < n ? static_cast<float>(Yv[j + c * ldy]) * yscale : 0.0f;
  }
  __syncthreads();
  const long long nb2 = static_cast<long long>(nb) * nb;
  // threads (r, h): row r of the tile row, column quarter h of each tile;
  // four independent sums keep several loads in flight per thread
  const int parts = kVecThreads / nb;
  const int r = threadIdx.x % nb, h = threadIdx.x / nb;
  float* red = sy + (j1 - j0) * nb;               // parts x nb partial sums
  float acc = 0.0f;
  if (h < parts) {
    float a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    const int c0 = h * nb / parts, c1 = (h + 1) * nb / parts;
    for (int jt = j0; jt < j1; ++jt) {
      const float* tl = Q + (static_cast<long long>(it) + static_cast<long long>(jt) * p) * nb2 + r;
      const float* yy = sy + (jt - j0) * nb;
      int jj = c0;
      for (; jj + 3 < c1; jj += 4) {
        acc = fmaf(__ldcg(tl + static_cast<long long>(jj) * nb), yy[jj], acc);
        a1 = fmaf(__ldcg(tl + static_cast<long long>(jj + 1) * nb), yy[jj + 1], a1);
        a2 = fmaf(__ldcg(tl + static_cast<long long>(jj + 2) * nb), yy[jj + 2], a2);
        a3 = fmaf(__ldcg(tl + static_cast<long long>(jj + 3) * nb), yy[jj + 3], a3);
      }
      for (; jj < c1; ++jj) acc = fmaf(__ldcg(tl + static_cast<long long>(jj) * nb), yy[jj], acc);
    }
    red[h * nb + r] = (acc + a1) + (a2 + a3);
  }
  __syncthreads();
  if (threadIdx.x < nb) {
    float sum = 0.0f;
    for (int hh = 0; hh < parts; ++hh) sum += red[hh * nb + threadIdx.x];
    const int row = it * nb + threadIdx.x;
    if (row < m) part[(static_cast<long long>(s) * gridDim.z + c) * m + row] = sum;
  }
}

// out(r, c) = alpha * Z(r, c) + beta * sum_s part(s, r, c)   (FP64, fixed order)
__global__ void vec_combine(const float* __restrict__ part, int nsplit, int rows, int nrhs,
                            const double* __restrict__ Z, long long ldz, double alpha, double beta,
                            double* __restrict__ out, long long ldo) {
  const long long total = static_cast<long long>(rows) * nrhs;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(e % rows), c = static_cast<int>(e / rows);
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += static_cast<double>(part[(static_cast<long long>(s) * nrhs + c) * rows + r]);
    double v = beta * acc;
    if (Z) v += alpha * Z[r + c * ldz];
    out[r + c * ldo] = v;
  }
}

// ---------------------------------------------------------------- host side
size_t trsv_ctl_ints(int n, int nb) { return 4 + static_cast<size_t>((n + nb - 1) / nb); }

size_t trsv_smem(int nb, int nrhs, int esize) {
  return static_cast<size_t>(esize) * (static_cast<size_t>(nb) * (nb + 1) + 2 * static_cast<size_t>(nb) * nrhs +
                                       static_cast<size_t>(kVecThreads) * nrhs + nb);
}

// The kernels' dynamic shared-memory limits are raised once per device
// (under a lock), not at every launch: the request server launches them from
// several host threads at once.
constexpr int kVecSmemMax = 200 * 1024;
static std::mutex g_vec_mu;
static bool g_vec_ready[64];

static cudaError_t vec_setup() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_vec_mu);
  if (g_vec_ready[dev]) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kVecSmemMax);
    if (r != cudaSuccess && e == cudaSuccess) e = r;
  };
  set(reinterpret_cast<const void*>(trsv_kernel<float, true>));
  set(reinterpret_cast<const void*>(trsv_kernel<float, false>));
  set(reinterpret_cast<const void*>(trsv_kernel<double, true>));
  set(reinterpret_cast<const void*>(trsv_kernel<double, false>));
  set(reinterpret_cast<const void*>(q1t_partial));
  set(reinterpret_cast<const void*>(q1n_partial));
  if (e == cudaSuccess) g_vec_ready[dev] = true;
  return e;
}

bool trsv_fits(int nb, int nrhs, int esize) {
  return nrhs <= kMaxVecRhs && nb <= 128 && static_cast<size_t>(nb) * nb * esize <= 16u * kTileChunks * kVecThreads &&
         trsv_smem(nb, nrhs, esize) <= static_cast<size_t>(kVecSmemMax);
}

template <typename real>
cudaError_t launch_trsv(bool trans, const real* tiles, int p, int nb, int n, int nrhs, const double* Y, long long ldy,
                        double* X, long long ldx, int* ctl, long long limit_ns, double* err_out, cudaStream_t st) {
  const size_t smem = trsv_smem(nb, nrhs, sizeof(real));
  const int qn = (n + nb - 1) / nb;
  // a few CTAs keep up with the wavefront of tile rows (each folds in the
  // rows solved before its own while it waits); more would only hold SMs
  // that concurrent work could use
  const int grid = std::max(1, std::min(qn, 8));
  cudaError_t e = vec_setup();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ctl, 0, sizeof(int) * trsv_ctl_ints(n, nb), st);
  if (e != cudaSuccess) return e;
  if (trans) {
    trsv_kernel<real, true><<<grid, kVecThreads, smem, st>>>(tiles, p, nb, n, nrhs, Y, ldy, X, ldx, ctl, limit_ns,
                                                             err_out);
  } else {
    trsv_kernel<real, false><<<grid, kVecThreads, smem, st>>>(tiles, p, nb, n, nrhs, Y, ldy, X, ldx, ctl, limit_ns,
                                                              err_out);
  }
  return cudaGetLastError();
}

template cudaError_t launch_trsv<float>(bool, const float*, int, int, int, int, const double*, long long, double*,
                                        long long, int*, long long, double*, cudaStream_t);
template cudaError_t launch_trsv<double>(bool, const double*, int, int, int, int, const double*, long long, double*,
                                         long long, int*, long long, double*, cudaStream_t);

int q1_splits(int tiles_along) {
  // enough blocks for the SMs: about 4 per SM over the whole grid
  const int want = std::max(1, (4 * device_sms() + tiles_along - 1) / std::max(1, tiles_along));
  return want;
}

cudaError_t launch_q1t(const float* Q, int p, int nb, int m, int n, int nrhs, const double* F, long long ldf,
                       double fscale, float* part, int splits_cap, double* D, long long ldd, cudaStream_t st) {
  const int qn = (n + nb - 1) / nb;
  int splits = std::min(std::min(q1_splits(qn), p), splits_cap);
  const int per = (p + splits - 1) / splits;
  splits = (p + per - 1) / per;
  const size_t smem = sizeof(float) * static_cast<size_t>(per) * nb;
  const cudaError_t e = vec_setup();
  if (e != cudaSuccess) return e;
  q1t_partial<<<dim3(qn, splits, nrhs), kVecThreads, smem, st>>>(Q, p, nb, m, n, F, ldf, static_cast<float>(fscale),
                                                                  per, part);
  const long long total = static_cast<long long>(n) * nrhs;
  vec_combine<<<static_cast<int>(std::min<long long>((total + 255) / 256, 8LL * device_sms())), 256, 0, st>>>(
      part, splits, n, nrhs, nullptr, 0, 0.0, 1.0 / fscale, D, ldd);
  return cudaGetLastError();
}

cudaError_t launch_q1n(const float* Q, int p, int nb, int m, int n, int nrhs, const double* Yv, long long ldy,
                       double yscale, const double* F, long long ldf, float* part, int splits_cap, double* U,
                       long long ldu, cudaStream_t st) {
  const int qn = (n + nb - 1) / nb;
  int splits = std::min(std::min(q1_splits(p), qn), splits_cap);
  const int per = (qn + splits - 1) / splits;
  splits = (qn + per - 1) / per;
  const size_t smem = sizeof(float) * (static_cast<size_t>(per) * nb + kVecThreads);
  const cudaError_t e = vec_setup();
  if (e != cudaSuccess) return e;
  q1n_partial<<<dim3(p, splits, nrhs), kVecThreads, smem, st>>>(Q, p, nb, m, n, Yv, ldy, static_cast<float>(yscale),
                                                                 per, part);
  const long long total = static_cast<long long>(m) * nrhs;
  vec_combine<<<static_cast<int>(std::min<long long>((total + 255) / 256, 8LL * device_sms())), 256, 0, st>>>(
      part, splits, m, nrhs, F, ldf, 1.0, -1.0 / yscale, U, ldu);
  return cudaGetLastError();
}

}  // namespace tqr
