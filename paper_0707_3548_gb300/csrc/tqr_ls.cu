// tqr_ls.cu -- least squares on top of the tiled QR (tqr_solve_ls).
//
// FP64: one task graph factors A, applies Q^T to the right-hand sides (they
// ride along as extra tile columns of Algorithm 1) and back-substitutes with
// R (Section 5 of the paper names applying Q as the factorization's natural
// companion).
//
// FP32 + refinement: the same graph in FP32 (column norms and tau in FP64)
// gives x0; for well-conditioned A the corrected semi-normal equations
//     dx = R^-1 R^-T A^T (b - A x)
// refine it (two triangular solves per step, FP64 residuals); otherwise, or
// once they stop halving the backward error, Bjorck's iterative refinement
// of the augmented system
//     [I A; A^T 0] [r; x] = [b; 0]
// runs with FP64 residuals  f = b - r - A x,  g = -A^T r  and corrections from
// the FP32 factors:  h = R^-T g,  d = Q^T f,  dx = R^-1 (d1 - h),
// dr = Q [h; d2],  until the normwise backward error
//     max_c ||A^T (b_c - A x_c)|| / (||A||_F (||A||_F ||x_c|| + ||b_c||))
// is at most tol.  The FP64 work (residuals, A^T products, norms) runs in the
// kernels below; they are bound by the FP64 pipe or by HBM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "tqr.h"
#include "tqr_api_internal.h"
#include "tqr_engine.h"
#include "tqr_ls.h"

namespace tqr {

constexpr int kLsThreads = 256;
constexpr int kRhsChunk = 8;

// Y(r, c) = Z(r, c) - sum_{j in split} A(r, j) X(j, c), written per split
// into P[split] (m x nrhs, ld m); a second kernel sums the splits in order.
__global__ void __launch_bounds__(kLsThreads) gemm_nn_partial(const double* __restrict__ A, long long lda, int m,
                                                              int n, const double* __restrict__ X, long long ldx,
                                                              int nrhs, int split_len,
                                                              double* __restrict__ P) {
  __shared__ double xs[64][kRhsChunk];
  const int r = blockIdx.x * kLsThreads + threadIdx.x;
  const int j0 = blockIdx.y * split_len;
  const int j1 = min(n, j0 + split_len);
  for (int c0 = 0; c0 < nrhs; c0 += kRhsChunk) {
    const int cw = min(kRhsChunk, nrhs - c0);
    double acc[kRhsChunk];
#pragma unroll
    for (int c = 0; c < kRhsChunk; ++c) acc[c] = 0.0;
    for (int jb = j0; jb < j1; jb += 64) {
      const int jw = min(64, j1 - jb);
      __syncthreads();
      for (int e = threadIdx.x; e < 64 * kRhsChunk; e += kLsThreads) {
        const int jj = e % 64, c = e / 64;
        xs[jj][c] = (jj < jw && c < cw) ? X[(jb + jj) + static_cast<long long>(c0 + c) * ldx] : 0.0;
      }
      __syncthreads();
      if (r < m) {
        for (int jj = 0; jj < jw; ++jj) {
          const double a = A[r + static_cast<long long>(jb + jj) * lda];
#pragma unroll
          for (int c = 0; c < kRhsChunk; ++c) acc[c] = fma(a, xs[jj][c], acc[c]);
        }
      }
    }
    if (r < m)
      for (int c = 0; c < cw; ++c)
        P[(static_cast<long long>(blockIdx.y) * nrhs + c0 + c) * m + r] = acc[c];
  }
}

// Y = alpha * Z + beta * W - sum_s P[s]   (all m x nrhs; Z, W may be null)
__global__ void combine_partials(const double* __restrict__ P, int nsplit, int m, int nrhs,
                                 const double* __restrict__ Z, long long ldz, double alpha,
                                 const double* __restrict__ Wm, long long ldw, double beta, double* __restrict__ Y,
                                 long long ldy) {
  const long long total = static_cast<long long>(m) * nrhs;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(e % m), c = static_cast<int>(e / m);
    double v = 0.0;
    if (Z) v = alpha * Z[r + c * ldz];
    if (Wm) v += beta * Wm[r + c * ldw];
    for (int s = 0; s < nsplit; ++s) v -= P[(static_cast<long long>(s) * nrhs + c) * m + r];
    Y[r + c * ldy] = v;
  }
}

// G(j, c) = alpha * sum_r A(r, j) R(r, c): one warp per column j.
__global__ void __launch_bounds__(kLsThreads) gemm_tn(const double* __restrict__ A, long long lda, int m, int n,
                                                      const double* __restrict__ R, long long ldr, int nrhs,
                                                      double alpha, double* __restrict__ G, long long ldg) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (kLsThreads / 32) + (threadIdx.x >> 5);
  if (j >= n) return;
  const double* a = A + static_cast<long long>(j) * lda;
  for (int c0 = 0; c0 < nrhs; c0 += kRhsChunk) {
    const int cw = min(kRhsChunk, nrhs - c0);
    double acc[kRhsChunk];
#pragma unroll
    for (int c = 0; c < kRhsChunk; ++c) acc[c] = 0.0;
    for (int r = lane; r < m; r += 32) {
      const double av = a[r];
#pragma unroll
      for (int c = 0; c < kRhsChunk; ++c)
        if (c < cw) acc[c] = fma(av, R[r + static_cast<long long>(c0 + c) * ldr], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kRhsChunk; ++c) {
      double v = acc[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && c < cw) G[j + static_cast<long long>(c0 + c) * ldg] = alpha * v;
    }
  }
}

// Per-column sums of squares of an m x ncols column-major matrix into
// out[c] (deterministic: one block per column, fixed reduction tree).
__global__ void __launch_bounds__(kLsThreads) col_sumsq(const double* __restrict__ X, long long ldx, int m,
                                                        double* __restrict__ out) {
  __shared__ double red[kLsThreads / 32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int r = threadIdx.x; r < m; r += kLsThreads) {
    const double v = X[r + static_cast<long long>(c) * ldx];
    s = fma(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kLsThreads / 32; ++w) t += red[w];
    out[c] = t;
  }
}

// out[0] = x[0] + ... + x[n-1] (one block, fixed order).
__global__ void __launch_bounds__(kLsThreads) vec_sum(const double* __restrict__ x, int n, double* __restrict__ out) {
  __shared__ double red[kLsThreads / 32];
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += kLsThreads) s += x[r];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kLsThreads / 32; ++w) t += red[w];
    out[0] = t;
  }
}

// min and max |R(i, i)| over i < n of the tiled factor (diagonal tiles).
template <typename real>
__global__ void diag_minmax(const real* __restrict__ Ab, int p, int nb, int n, double* __restrict__ out) {
  __shared__ double smin[kLsThreads], smax[kLsThreads];
  double mn = INFINITY, mx = 0.0;
  for (int i = threadIdx.x; i < n; i += kLsThreads) {
    const int t = i / nb, r = i - t * nb;
    const double v = fabs(static_cast<double>(
        Ab[(static_cast<long long>(t) + static_cast<long long>(t) * p) * nb * nb + static_cast<long long>(r) * nb + r]));
    mn = fmin(mn, v);
    mx = fmax(mx, v);
  }
  smin[threadIdx.x] = mn;
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int s = kLsThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = smin[0];
    out[1] = smax[0];
  }
}

// Y(0:rows, :) = alpha X1 + beta X2 (column-major, any of X1/X2 null = 0).
// (Y may alias X1 or X2: every element is read and written by one thread.)
__global__ void axpby(int rows, int cols, double alpha, const double* X1, long long ld1, double beta,
                      const double* X2, long long ld2, double* Y, long long ldy) {
  const long long total = static_cast<long long>(rows) * cols;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(e % rows), c = static_cast<int>(e / rows);
    double v = 0.0;
    if (X1) v = alpha * X1[r + c * ld1];
    if (X2) v += beta * X2[r + c * ld2];
    Y[r + c * ldy] = v;
  }
}

static int ew_grid(long long total) {
  const int sms = device_sms();
  long long g = (total + 255) / 256;
  return static_cast<int>(std::max<long long>(1, std::min<long long>(g, static_cast<long long>(sms) * 8)));
}

// FP64 helpers on the stream -------------------------------------------------
static LsScratch ls_scratch_shape(int m, int n, int nrhs) {
  const int sms = device_sms();
  const int row_blocks = (m + kLsThreads - 1) / kLsThreads;
  int nsplit = std::max(1, std::min(n, (4 * sms + row_blocks - 1) / row_blocks));
  nsplit = std::min(nsplit, 64);
  LsScratch s;
  s.part = nullptr;
  s.nsplit = nsplit;
  s.split_len = (n + nsplit - 1) / nsplit;
  s.nsplit = (n + s.split_len - 1) / s.split_len;
  (void)nrhs;
  return s;
}

// Y = alpha Z + beta W - A X
static cudaError_t resid(const LsScratch& sc, const double* A, long long lda, int m, int n, const double* X,
                         long long ldx, int nrhs, const double* Z, long long ldz, double alpha, const double* Wm,
                         long long ldw, double beta, double* Y, long long ldy, cudaStream_t st) {
  dim3 grid((m + kLsThreads - 1) / kLsThreads, sc.nsplit);
  gemm_nn_partial<<<grid, kLsThreads, 0, st>>>(A, lda, m, n, X, ldx, nrhs, sc.split_len, sc.part);
  combine_partials<<<ew_grid(static_cast<long long>(m) * nrhs), 256, 0, st>>>(sc.part, sc.nsplit, m, nrhs, Z, ldz,
                                                                            alpha, Wm, ldw, beta, Y, ldy);
  return cudaGetLastError();
}

static cudaError_t atr(const double* A, long long lda, int m, int n, const double* R, long long ldr, int nrhs,
                       double alpha, double* G, long long ldg, cudaStream_t st) {
  const int wpb = kLsThreads / 32;
  gemm_tn<<<(n + wpb - 1) / wpb, kLsThreads, 0, st>>>(A, lda, m, n, R, ldr, nrhs, alpha, G, ldg);
  return cudaGetLastError();
}

struct BerrBufs {
  double* G;     // n x nrhs
  double* nrm;   // 3 * nrhs
};

static size_t al(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// ---------------------------------------------------------------------------
// LsJob: device state of one least-squares problem.  The tiles of A (and T)
// double as a resident factorization: after factor_solve() a later solve()
// with new right-hand sides reuses them (Q^T B and back substitution only).
bool LsJob::init(int m_, int n_, int rhs_cap_, int nb_, int ib_, int prec_, int grid_cap_) {
  m = m_;
  n = n_;
  rhs_cap = rhs_cap_;
  nb = nb_;
  ib = ib_;
  prec = prec_;
  esize = prec == TQR_PREC_FP64 ? 8 : 4;
  grid_cap = grid_cap_;
  if (!choose_shape(nb, ib, esize, &cs, &occ, &smem)) return false;
  I = make_inst(M_FACTOR, m, n, nb, ib, cs, rhs_cap, 1);
  I.D = choose_domain(m, n, nb, ib, esize);  // reduction tree when it shortens the run
  // (2b x b bottoms measured no faster here: 527 vs 519 ms for the FP64
  // solve at 16384 x 4096, so least squares keeps b x b tiles)
  W = ws_layout(I, esize, true);
  sc = ls_scratch_shape(m, n, rhs_cap);
  const size_t mr = static_cast<size_t>(m) * rhs_cap, nr = static_cast<size_t>(n) * rhs_cap;
  size_t o = al(W.bytes);
  o_part = o;  o += al(sizeof(double) * sc.nsplit * mr);
  o_e = o;     o += al(sizeof(double) * mr);
  o_r = o;     o += al(sizeof(double) * mr);
  o_f = o;     o += al(sizeof(double) * mr);
  o_d = o;     o += al(sizeof(double) * mr);
  o_g = o;     o += al(sizeof(double) * std::max(nr, static_cast<size_t>(n)));
  o_h = o;     o += al(sizeof(double) * nr);
  o_x = o;     o += al(sizeof(double) * nr);
  o_G = o;     o += al(sizeof(double) * nr);
  o_nrm = o;   o += al(sizeof(double) * (4 * rhs_cap + 4));
  o_b2 = o;    o += al(W.oT - W.oB);                       // as large as the first tile array
  o_ver2 = o;  o += al(sizeof(int) * static_cast<size_t>(I.p) * (I.q + I.qb) * I.NS);
  o_inst2 = o; o += al(2 * sizeof(Inst));
  o_acopy = o;
  bytes = o;
  return true;
}

size_t LsJob::bytes_with_acopy() const { return bytes + al(sizeof(double) * static_cast<size_t>(m) * n); }

void LsJob::bind(char* base, bool with_acopy) {
  ws = base;
  sc.part = reinterpret_cast<double*>(ws + o_part);
  I.A = ws + W.oA;
  I.B = ws + W.oB;
  I.T = ws + W.oT;
  I.ver = reinterpret_cast<int*>(ws + W.oVer);
  Acopy = with_acopy ? reinterpret_cast<double*>(ws + o_acopy) : nullptr;
}

int LsJob::run_mode(int mode, int trsm, int nrhs_now, cudaStream_t st) {
  I.mode = mode;
  I.trsm = trsm;
  I.nrhs = nrhs_now;
  I.qb = (nrhs_now + nb - 1) / nb;
  return esize == 8 ? run_plan<double>(I, ws, W, occ, smem, st, grid_cap)
                    : run_plan<float>(I, ws, W, occ, smem, st, grid_cap);
}

int LsJob::pack_rhs(const double* src, long long lds, int rows, int nrhs, cudaStream_t st, void* tiles) {
  const int sms = device_sms();
  const int qb = (nrhs + nb - 1) / nb;
  void* B = tiles ? tiles : I.B;
  cudaError_t e = esize == 8
                      ? launch_pack<double>(src, lds, rows, nrhs, static_cast<double*>(B), I.p, qb, nb, sms, st)
                      : launch_pack<float>(src, lds, rows, nrhs, static_cast<float*>(B), I.p, qb, nb, sms, st);
  return e == cudaSuccess ? TQR_OK : TQR_ERR_CUDA;
}

int LsJob::unpack_rhs(double* dst, long long ldd, int rows, int nrhs, cudaStream_t st, const void* tiles) {
  const int sms = device_sms();
  const void* B = tiles ? tiles : I.B;
  cudaError_t e = esize == 8
                      ? launch_unpack<double>(static_cast<const double*>(B), I.p, nb, dst, ldd, rows, nrhs, sms, st)
                      : launch_unpack<float>(static_cast<const float*>(B), I.p, nb, dst, ldd, rows, nrhs, sms, st);
  return e == cudaSuccess ? TQR_OK : TQR_ERR_CUDA;
}

int LsJob::run_two(int mode_a, int mode_b, int nrhs_now, cudaStream_t st) {
  Inst two[2] = {I, I};
  for (Inst& x : two) {
    x.trsm = 0;
    x.nrhs = nrhs_now;
    x.qb = (nrhs_now + nb - 1) / nb;
  }
  two[0].mode = mode_a;
  two[1].mode = mode_b;
  two[1].B = ws + o_b2;
  two[1].ver = reinterpret_cast<int*>(ws + o_ver2);
  Inst* d_insts = reinterpret_cast<Inst*>(ws + o_inst2);
  void* d_ctl = ws + W.oCtl;
  return esize == 8 ? run_plan_multi<double>(two, 2, d_insts, d_ctl, occ, smem, st, grid_cap)
                    : run_plan_multi<float>(two, 2, d_insts, d_ctl, occ, smem, st, grid_cap);
}

// factor A (and keep the factors), x0 = the solution through those factors
int LsJob::factor_solve(const double* A, long long lda, const double* B, long long ldb, int nrhs, cudaStream_t st) {
  const int sms = device_sms();
  if (upload_vtab(I, ws, W, st) != TQR_OK) return TQR_ERR_CUDA;
  if (Acopy != nullptr &&
      copy_cols(Acopy, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m, n,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return TQR_ERR_CUDA;
  cudaError_t e = esize == 8 ? launch_pack<double>(A, lda, m, n, static_cast<double*>(I.A), I.p, I.q, nb, sms, st)
                             : launch_pack<float>(A, lda, m, n, static_cast<float*>(I.A), I.p, I.q, nb, sms, st);
  if (e != cudaSuccess) return TQR_ERR_CUDA;
  int s = pack_rhs(B, ldb, m, nrhs, st);
  if (s == TQR_OK) s = run_mode(M_FACTOR, 1, nrhs, st);
  if (s == TQR_OK) s = unpack_rhs(reinterpret_cast<double*>(ws + o_x), n, n, nrhs, st);
  if (s == TQR_OK) {
    double* dmm = reinterpret_cast<double*>(ws + o_nrm) + 4 * rhs_cap + 2;
    if (esize == 8)
      diag_minmax<double><<<1, kLsThreads, 0, st>>>(static_cast<double*>(I.A), I.p, nb, n, dmm);
    else
      diag_minmax<float><<<1, kLsThreads, 0, st>>>(static_cast<float*>(I.A), I.p, nb, n, dmm);
    double* nA2 = reinterpret_cast<double*>(ws + o_nrm) + 4 * rhs_cap;
    double* colsq = reinterpret_cast<double*>(ws + o_g);
    // ||A||_F^2: the columns' sums of squares, then their sum
    col_sumsq<<<n, kLsThreads, 0, st>>>(A, lda, m, colsq);
    vec_sum<<<1, kLsThreads, 0, st>>>(colsq, n, nA2);
    if (cudaGetLastError() != cudaSuccess) s = TQR_ERR_CUDA;
  }
  factored = (s == TQR_OK);
  return s;
}

// x0 from the resident factors: Q^T B and back substitution, one graph
int LsJob::solve(const double* B, long long ldb, int nrhs, cudaStream_t st) {
  int s = pack_rhs(B, ldb, m, nrhs, st);
  if (s == TQR_OK) s = run_mode(M_APPLY_QT, 1, nrhs, st);
  if (s == TQR_OK) s = unpack_rhs(reinterpret_cast<double*>(ws + o_x), n, n, nrhs, st);
  return s;
}

// Backward error of x, FP32 refinement, copy of x to X.  A is the FP64
// matrix (caller's or the resident copy).
int LsJob::finish(const double* A, long long lda, const double* B, long long ldb, int nrhs, double* X, long long ldx,
                  double tol, int maxit, int* iters_out, double* berr_out, cudaStream_t st) {
  const size_t mr = static_cast<size_t>(m) * nrhs, nr = static_cast<size_t>(n) * nrhs;
  double* E = reinterpret_cast<double*>(ws + o_e);
  double* Rr = reinterpret_cast<double*>(ws + o_r);
  double* F = reinterpret_cast<double*>(ws + o_f);
  double* D = reinterpret_cast<double*>(ws + o_d);
  double* Gv = reinterpret_cast<double*>(ws + o_g);
  double* H = reinterpret_cast<double*>(ws + o_h);
  double* Xw = reinterpret_cast<double*>(ws + o_x);
  BerrBufs bb;
  bb.G = reinterpret_cast<double*>(ws + o_G);
  bb.nrm = reinterpret_cast<double*>(ws + o_nrm);
  const int R = rhs_cap;  // nrm layout: [0,R) |A^T e|^2, [R,2R) |x|^2, [2R,3R) |b|^2, [4R] |A|^2, [4R+2,4R+3] diag
  double* dx2 = bb.nrm + 3 * R;
  std::vector<double> hn(4 * R + 4);
  int status = TQR_OK;
  int iters = 0;
  double berr = INFINITY;
  auto fail = [&](int s) {
    if (status == TQR_OK && s != TQR_OK) status = s;
  };
  auto read_back = [&]() {
    if (cudaMemcpyAsync(hn.data(), bb.nrm, sizeof(double) * hn.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      fail(TQR_ERR_CUDA);
  };
  auto berr_of = [&]() {
    double worst = 0.0;
    const double nA = std::sqrt(hn[4 * R]);
    for (int c = 0; c < nrhs; ++c) {
      const double num = std::sqrt(hn[c]);
      const double den = nA * (nA * std::sqrt(hn[R + c]) + std::sqrt(hn[2 * R + c]));
      const double eta = den > 0 ? num / den : (num > 0 ? INFINITY : 0.0);
      if (!(eta <= worst)) worst = eta;
    }
    return worst;
  };
  auto terms = [&]() {
    if (resid(sc, A, lda, m, n, Xw, n, nrhs, B, ldb, 1.0, nullptr, 0, 0.0, E, m, st) != cudaSuccess ||
        atr(A, lda, m, n, E, m, nrhs, 1.0, bb.G, n, st) != cudaSuccess)
      fail(TQR_ERR_CUDA);
    col_sumsq<<<nrhs, kLsThreads, 0, st>>>(bb.G, n, n, bb.nrm);
    col_sumsq<<<nrhs, kLsThreads, 0, st>>>(Xw, n, n, bb.nrm + R);
    col_sumsq<<<nrhs, kLsThreads, 0, st>>>(B, ldb, m, bb.nrm + 2 * R);
    if (cudaGetLastError() != cudaSuccess) fail(TQR_ERR_CUDA);
  };
  terms();
  read_back();
  if (status == TQR_OK) {
    // a NaN or an infinity in A or B shows in their FP64 norms
    bool finite = std::isfinite(hn[4 * R]);
    for (int c = 0; c < nrhs; ++c) finite = finite && std::isfinite(hn[2 * R + c]);
    if (!finite) status = TQR_ERR_NONFINITE;
  }
  if (status == TQR_OK) {
    // numerical rank test on R with the FP64 unit roundoff in both precisions:
    // an FP32 factor with a small pivot may still refine to an FP64 answer,
    // so refinement, not this test, judges the FP32 path
    const double eps = 1.1102230246251565e-16;
    if (!(hn[4 * R + 2] > n * eps * hn[4 * R + 3])) status = TQR_ERR_RANK;
    berr = berr_of();
  }
  if (status == TQR_OK && esize == 4) {
    // Refine until the backward error meets tol AND x has settled at FP64
    // accuracy: the last correction is below FP64 rounding (||dx|| <=
    // 2^-50 ||x||) or, with the backward error already met, no longer halves
    // (the corrections have reached the rounding noise of the FP64
    // residuals), so the answer matches an FP64 solve; stop early on
    // stagnation (neither the backward error nor the correction halves for 3
    // steps) or at maxit.
    double prev = berr, prev_dx = INFINITY, dxrel = INFINITY;
    bool settled = false;
    auto dx_rel = [&](double scale) {
      double worst = 0.0;
      for (int c = 0; c < nrhs; ++c) {
        const double xr = std::sqrt(hn[R + c]);
        const double d = std::sqrt(hn[3 * R + c]) / scale;
        const double rel = xr > 0 ? d / xr : d;
        if (!(rel <= worst)) worst = rel;
      }
      return worst;
    };
    // Corrected semi-normal equations first: dx = R^-1 R^-T A^T e with
    // e = b - A x and A^T e already on the device from the backward-error
    // terms -- two triangular-solve graphs per step and no Q application.
    // With R the factor of A + E (||E|| ~ eps ||A||) the error contracts by
    // about 2 kappa eps per step, so they run only while the spread of R's
    // diagonal (a lower bound on kappa) keeps kappa u_fp32 small, and give
    // way to the augmented-system refinement as soon as a step fails to
    // halve the backward error (a step that made it worse is undone).
    const double spread = hn[4 * R + 3] / hn[4 * R + 2];
    bool semi = spread * 0x1p-24 < 0.01;
    while (status == TQR_OK && semi && !settled && (berr > tol || dxrel > 0x1p-50) && iters < maxit) {
      // scale A^T e by a power of two near 1/max ||.|| so FP32 keeps it normal
      double gmax = 0.0;
      for (int c = 0; c < nrhs; ++c) gmax = std::max(gmax, std::sqrt(hn[c]));
      const double scale = gmax > 0 && std::isfinite(gmax) ? std::ldexp(1.0, -std::ilogb(gmax)) : 1.0;
      axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, scale, bb.G, n, 0.0, nullptr, 0, Gv, n);
      fail(pack_rhs(Gv, n, n, nrhs, st));
      if (status == TQR_OK) fail(run_mode(M_TRSMT, 0, nrhs, st));
      if (status == TQR_OK) fail(run_mode(M_TRSM, 0, nrhs, st));
      fail(unpack_rhs(Gv, n, n, nrhs, st));
      col_sumsq<<<nrhs, kLsThreads, 0, st>>>(Gv, n, n, dx2);
      axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, 1.0, Xw, n, 1.0 / scale, Gv, n, Xw, n);
      ++iters;
      terms();
      read_back();
      if (status != TQR_OK) break;
      const double b_new = berr_of();
      dxrel = dx_rel(scale);
      if (b_new <= tol && !(dxrel < 0.5 * prev_dx)) {
        settled = true;
        berr = b_new;
        break;
      }
      if (b_new > tol && !(b_new < 0.5 * prev)) {
        semi = false;
        if (!(b_new <= prev)) {
          axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, 1.0, Xw, n, -1.0 / scale, Gv, n, Xw, n);
          terms();
          read_back();
          if (status != TQR_OK) break;
          dxrel = INFINITY;
          continue;
        }
      }
      berr = b_new;
      prev = std::min(prev, berr);
      prev_dx = std::min(prev_dx, dxrel);
    }
    if (status == TQR_OK) berr = berr_of();
    if (!settled &&
        cudaMemcpyAsync(Rr, E, sizeof(double) * mr, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      fail(TQR_ERR_CUDA);
    int stall = 0;
    while (status == TQR_OK && !settled && (berr > tol || dxrel > 0x1p-50) && iters < maxit) {
      // f = b - r - A x = e - r;  g = -A^T r
      axpby<<<ew_grid(mr), 256, 0, st>>>(m, nrhs, 1.0, E, m, -1.0, Rr, m, F, m);
      if (atr(A, lda, m, n, Rr, m, nrhs, -1.0, Gv, n, st) != cudaSuccess) fail(TQR_ERR_CUDA);
      // d = Q^T f (first tiles) and h = R^-T g (second tiles): one launch
      void* B2 = ws + o_b2;
      fail(pack_rhs(F, m, m, nrhs, st));
      fail(pack_rhs(Gv, n, n, nrhs, st, B2));
      if (status == TQR_OK) fail(run_two(M_APPLY_QT, M_TRSMT, nrhs, st));
      fail(unpack_rhs(D, m, m, nrhs, st));
      fail(unpack_rhs(H, n, n, nrhs, st, B2));
      // dx = R^-1 (d1 - h) (second tiles) and dr = Q [h; d2] (first tiles): one launch
      axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, 1.0, D, m, -1.0, H, n, Gv, n);
      axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, 1.0, H, n, 0.0, nullptr, 0, D, m);
      fail(pack_rhs(D, m, m, nrhs, st));
      fail(pack_rhs(Gv, n, n, nrhs, st, B2));
      if (status == TQR_OK) fail(run_two(M_APPLY_Q, M_TRSM, nrhs, st));
      fail(unpack_rhs(D, m, m, nrhs, st));
      fail(unpack_rhs(Gv, n, n, nrhs, st, B2));
      col_sumsq<<<nrhs, kLsThreads, 0, st>>>(Gv, n, n, dx2);
      axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, 1.0, Xw, n, 1.0, Gv, n, Xw, n);
      axpby<<<ew_grid(mr), 256, 0, st>>>(m, nrhs, 1.0, Rr, m, 1.0, D, m, Rr, m);
      ++iters;
      terms();
      read_back();
      if (status != TQR_OK) break;
      berr = berr_of();
      dxrel = dx_rel(1.0);
      if (berr <= tol && !(dxrel < 0.5 * prev_dx)) break;
      if (!(berr < 0.5 * prev) && !(dxrel < 0.5 * prev_dx)) {
        if (++stall >= 3) break;
      } else {
        stall = 0;
      }
      prev = std::min(prev, berr);
      prev_dx = std::min(prev_dx, dxrel);
    }
    if (status == TQR_OK && !(berr <= tol)) status = TQR_ERR_NOCONV;
  }
  if (X != nullptr &&
      copy_cols(X, sizeof(double) * ldx, Xw, sizeof(double) * n, sizeof(double) * n, nrhs,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    fail(TQR_ERR_CUDA);
  if (iters_out) *iters_out = iters;
  if (berr_out) *berr_out = berr;
  return status;
}

static int solve_device(int64_t m64, int64_t n64, int64_t nrhs64, const double* A, int64_t lda, const double* B,
                        int64_t ldb, double* X, int64_t ldx, int prec, double tol, int maxit, int* iters_out,
                        double* berr_out, int nb, int ib, cudaStream_t st) {
  LsJob job;
  if (!job.init(static_cast<int>(m64), static_cast<int>(n64), static_cast<int>(nrhs64), nb, ib, prec, 0))
    return TQR_ERR_UNSUPPORTED;
  char* ws = nullptr;
  if (lib_malloc(reinterpret_cast<void**>(&ws), job.bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return TQR_ERR_NOMEM;
  }
  job.bind(ws, false);
  int status = job.factor_solve(A, lda, B, ldb, static_cast<int>(nrhs64), st);
  if (status == TQR_OK)
    status = job.finish(A, lda, B, ldb, static_cast<int>(nrhs64), X, ldx, tol, maxit, iters_out, berr_out, st);
  cudaFreeAsync(ws, st);
  int dev_status = TQR_OK;
  if (read_status(&dev_status, st) != cudaSuccess && status == TQR_OK) status = TQR_ERR_CUDA;
  if (dev_status != TQR_OK) status = dev_status;
  return status;
}

}  // namespace tqr

using namespace tqr;

extern "C" int tqr_solve_ls(int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* B,
                            int64_t ldb, double* X, int64_t ldx, int prec, double tol, int maxit, int* iters,
                            double* berr, int nb, int ib, void* stream) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (nrhs < 1) return -3;
  if (m > (1LL << 30) || nrhs > (1LL << 20)) return TQR_ERR_UNSUPPORTED;
  if (A == nullptr) return -4;
  if (lda < m) return -5;
  if (B == nullptr) return -6;
  if (ldb < m) return -7;
  if (X == nullptr) return -8;
  if (ldx < n) return -9;
  if (prec != TQR_PREC_FP64 && prec != TQR_PREC_FP32) return -10;
  if (!(tol >= 0)) return -11;
  if (maxit < 0) return -12;
  if (nb == 0) nb = n >= 1024 ? 128 : 64;
  if (ib == 0) ib = std::min(16, nb);  // measured: ib 16 beats 32 for FP64 and FP32 factors
  const int c = check_tiles(nb, ib, 15, 16);
  if (c) return c;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ka = ptr_kind(A);
  if (ptr_kind(B) != ka) return -6;
  if (ptr_kind(X) != ka) return -8;
  if (ka == PTR_DEVICE)
    return solve_device(m, n, nrhs, A, lda, B, ldb, X, ldx, prec, tol, maxit, iters, berr, nb, ib, st);
  double *dA = nullptr, *dB = nullptr, *dX = nullptr;
  if (lib_malloc(reinterpret_cast<void**>(&dA), sizeof(double) * m * n, st) != cudaSuccess ||
      lib_malloc(reinterpret_cast<void**>(&dB), sizeof(double) * m * nrhs, st) != cudaSuccess ||
      lib_malloc(reinterpret_cast<void**>(&dX), sizeof(double) * n * nrhs, st) != cudaSuccess) {
    cudaGetLastError();
    if (dA) cudaFreeAsync(dA, st);
    if (dB) cudaFreeAsync(dB, st);
    return TQR_ERR_NOMEM;
  }
  int status = TQR_OK;
  if (copy_cols(dA, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m, n,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
      copy_cols(dB, sizeof(double) * m, B, sizeof(double) * ldb, sizeof(double) * m, nrhs,
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
    status = TQR_ERR_CUDA;
  if (status == TQR_OK) status = solve_device(m, n, nrhs, dA, m, dB, m, dX, n, prec, tol, maxit, iters, berr, nb, ib, st);
  if ((status == TQR_OK || status == TQR_ERR_NOCONV || status == TQR_ERR_RANK) &&
      copy_cols(X, sizeof(double) * ldx, dX, sizeof(double) * n, sizeof(double) * n, nrhs,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
    status = TQR_ERR_CUDA;
  cudaFreeAsync(dA, st);
  cudaFreeAsync(dB, st);
  cudaFreeAsync(dX, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return TQR_ERR_CUDA;
  return status;
}
