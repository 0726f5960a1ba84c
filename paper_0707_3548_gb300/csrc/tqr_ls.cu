// tqr_ls.cu -- least squares on top of the tiled QR (tqr_solve_ls and the
// resident handle tqr_ls_factor / tqr_ls_solve / tqr_ls_release).
//
// FP64: one task graph factors A, applies Q^T to the right-hand sides (they
// ride along as extra tile columns of Algorithm 1) and back-substitutes with
// R (Section 5 of the paper names applying Q as the factorization's natural
// companion).
//
// FP32 + refinement: the same graph in FP32 (column norms and tau in FP64)
// gives x0, refined with FP64 residuals in up to three forms, each taking
// over when the one before cannot finish:
//  (1) the corrected semi-normal equations dx = R^-1 R^-T A^T (b - A x), for
//      well-conditioned A (two triangular solves per step);
//  (2) Bjorck's iterative refinement of the augmented system
//          [I A; A^T 0] [r; x] = [b; 0]
//      with f = b - r - A x, g = -A^T r and corrections from the FP32
//      factors:  h = R^-T g,  d = Q^T f,  dx = R^-1 (d1 - h),  dr = Q [h; d2];
//  (3) GMRES-IR (Carson, Higham and Pranesh 2020): the same correction
//      equation solved by GMRES, left-preconditioned with (2)'s correction,
//      for kappa(A) u_fp32 near or above 1, where (2) no longer contracts.
// The normwise backward error
//     max_c ||A^T (b_c - A x_c)|| / (||A||_F (||A||_F ||x_c|| + ||b_c||))
// must reach tol and x must settle; a problem that does not is solved again
// in FP64.  The FP64 work (residuals, A^T products, norms, GMRES) runs in the
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
        if (cw == 1) {  // one right-hand side: one FMA per element of A
          for (int jj = 0; jj < jw; ++jj) acc[0] = fma(A[r + static_cast<long long>(jb + jj) * lda], xs[jj][0], acc[0]);
        } else {
          for (int jj = 0; jj < jw; ++jj) {
            const double a = A[r + static_cast<long long>(jb + jj) * lda];
#pragma unroll
            for (int c = 0; c < kRhsChunk; ++c) acc[c] = fma(a, xs[jj][c], acc[c]);
          }
        }
      }
    }
    if (r < m)
      for (int c = 0; c < cw; ++c)
        P[(static_cast<long long>(blockIdx.y) * nrhs + c0 + c) * m + r] = acc[c];
  }
}

// Y = alpha * Z + beta * W + gamma * sum_s P[s]   (all m x nrhs; Z, W may be
// null; gamma = -1 gives a residual, +1 the product A X added)
__global__ void combine_partials(const double* __restrict__ P, int nsplit, int m, int nrhs,
                                 const double* __restrict__ Z, long long ldz, double alpha,
                                 const double* __restrict__ Wm, long long ldw, double beta, double gamma,
                                 double* __restrict__ Y, long long ldy) {
  const long long total = static_cast<long long>(m) * nrhs;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(e % m), c = static_cast<int>(e / m);
    double v = 0.0;
    if (Z) v = alpha * Z[r + c * ldz];
    if (Wm) v += beta * Wm[r + c * ldw];
    double ax = 0.0;
    for (int s = 0; s < nsplit; ++s) ax += P[(static_cast<long long>(s) * nrhs + c) * m + r];
    Y[r + c * ldy] = fma(gamma, ax, v);
  }
}

// Power of two near 1 / nA (1 for zero or non-finite nA): the exact scale
// that keeps products of A's entries with vectors of A's size finite.
__host__ __device__ inline double norm_scale(double nA) {
  return nA > 0.0 && nA <= 1.7976931348623157e308 ? ldexp(1.0, -ilogb(nA)) : 1.0;
}

// G(j, c) = alpha * sum_r (s A(r, j)) R(r, c): one warp per column j, with
// s = norm_scale(*nA) when nA is given (else 1) -- the backward error's
// A^T r, whose true size ||A|| ||r|| may exceed FP64's range, is formed as
// s A^T r.
__global__ void __launch_bounds__(kLsThreads) gemm_tn(const double* __restrict__ A, long long lda, int m, int n,
                                                      const double* __restrict__ R, long long ldr, int nrhs,
                                                      double alpha, double* __restrict__ G, long long ldg,
                                                      const double* __restrict__ nA) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (kLsThreads / 32) + (threadIdx.x >> 5);
  if (j >= n) return;
  const double s = nA ? norm_scale(*nA) : 1.0;
  const double* a = A + static_cast<long long>(j) * lda;
  // the scale is an exact power of two, so applying it once to a lane's sum
  // gives the value of scaling every product (rounding commutes with it) up
  // to products below FP64's normal range.  That form skips one FP64
  // multiply per element, half of this kernel's FP64 instructions; it runs
  // while s <= 2^200 (||A||_F >= 2^-200: the unscaled products are not the
  // ones that underflow), and a lane whose unscaled sum overflows (or meets a
  // NaN) takes the scaled loop instead.
  const bool post = s <= 0x1p200;
  for (int c0 = 0; c0 < nrhs; c0 += kRhsChunk) {
    const int cw = min(kRhsChunk, nrhs - c0);
    double acc[kRhsChunk];
#pragma unroll
    for (int c = 0; c < kRhsChunk; ++c) acc[c] = 0.0;
    if (cw == 1) {
      // one right-hand side: no predicated FMAs (they would still take
      // issue slots of the FP64 pipe), four independent partial sums
      const double* rr = R + static_cast<long long>(c0) * ldr;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int r = lane;
      if (post) {
        for (; r + 96 < m; r += 128) {
          a0 = fma(a[r], rr[r], a0);
          a1 = fma(a[r + 32], rr[r + 32], a1);
          a2 = fma(a[r + 64], rr[r + 64], a2);
          a3 = fma(a[r + 96], rr[r + 96], a3);
        }
        for (; r < m; r += 32) a0 = fma(a[r], rr[r], a0);
      }
      double v = (a0 + ((a1 + a2) + a3)) * s;
      if (!post || !isfinite(v)) {
        a0 = a1 = a2 = a3 = 0.0;
        r = lane;
        for (; r + 96 < m; r += 128) {
          a0 = fma(a[r] * s, rr[r], a0);
          a1 = fma(a[r + 32] * s, rr[r + 32], a1);
          a2 = fma(a[r + 64] * s, rr[r + 64], a2);
          a3 = fma(a[r + 96] * s, rr[r + 96], a3);
        }
        for (; r < m; r += 32) a0 = fma(a[r] * s, rr[r], a0);
        v = a0 + ((a1 + a2) + a3);
      }
      acc[0] = v;
    } else {
      for (int r = lane; r < m; r += 32) {
        const double av = a[r] * s;
#pragma unroll
        for (int c = 0; c < kRhsChunk; ++c)
          if (c < cw) acc[c] = fma(av, R[r + static_cast<long long>(c0 + c) * ldr], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < kRhsChunk; ++c) {
      if (c >= cw) break;  // uniform over the warp
      double v = acc[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) G[j + static_cast<long long>(c0 + c) * ldg] = alpha * v;
    }
  }
}

// Block-wide reductions over kLsThreads threads (fixed order: deterministic).
__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kLsThreads / 32; ++w) t = fmax(t, red[w]);
  return t;
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kLsThreads / 32; ++w) t += red[w];
  return t;
}

// 2-norm of each column of an m x ncols column-major matrix into out[c], one
// block per column, without overflow or underflow: the column is scaled by
// the power of two 2^-e nearest below 1/max|x| (exact in binary), its sum
// of squares taken, and the root scaled back (the scaling in the manner of
// LAPACK's dnrm2, with a power of two so the scaling itself is exact).  A
// NaN or an infinity in the column gives a non-finite norm.
__global__ void __launch_bounds__(kLsThreads) col_nrm2(const double* __restrict__ X, long long ldx, int m,
                                                       double* __restrict__ out) {
  __shared__ double red[kLsThreads / 32];
  const double* x = X + static_cast<long long>(blockIdx.x) * ldx;
  double mx = 0.0;
  bool bad = false;
  for (int r = threadIdx.x; r < m; r += kLsThreads) {
    const double a = fabs(x[r]);
    bad = bad || !(a <= 1.7976931348623157e308);  // NaN or infinity
    mx = fmax(mx, a);
  }
  mx = block_max(bad ? INFINITY : mx, red);
  if (!(mx <= 1.7976931348623157e308)) {
    if (threadIdx.x == 0) out[blockIdx.x] = NAN;
    return;
  }
  if (mx == 0.0) {
    if (threadIdx.x == 0) out[blockIdx.x] = 0.0;
    return;
  }
  const int e = ilogb(mx);  // mx in [2^e, 2^(e+1)): x * 2^-e is below 2 in magnitude
  double s = 0.0;
  for (int r = threadIdx.x; r < m; r += kLsThreads) {
    const double v = scalbn(x[r], -e);
    s = fma(v, v, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = scalbn(sqrt(s), e);
}

// GMRES (Arnoldi) helpers.  The basis vectors of all right-hand sides live
// in one array: vector i of right-hand side c is the N-vector at
// V + (i * nrhs + c) * N (N = m + n: [u; v] of the augmented system).
// out[i + c * ldo] = V_i(:, c)^T w(:, c) for i < nvec: one block per (i, c).
__global__ void __launch_bounds__(kLsThreads) gmres_dots(const double* __restrict__ V, int nvec, long long N,
                                                         int nrhs, const double* __restrict__ w,
                                                         double* __restrict__ out, int ldo) {
  __shared__ double red[kLsThreads / 32];
  const int i = blockIdx.x, c = blockIdx.y;
  if (i >= nvec) return;
  const double* v = V + (static_cast<long long>(i) * nrhs + c) * N;
  const double* x = w + static_cast<long long>(c) * N;
  double s = 0.0;
  for (long long r = threadIdx.x; r < N; r += kLsThreads) s = fma(v[r], x[r], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[i + c * ldo] = s;
}

// w(:, c) -= sum_{i < nvec} coef[i + c * ldc] V_i(:, c)
__global__ void gmres_axpy(const double* __restrict__ V, int nvec, long long N, int nrhs,
                           const double* __restrict__ coef, int ldc, double* __restrict__ w) {
  const long long total = N * nrhs;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e / N);
    const long long r = e - static_cast<long long>(c) * N;
    double acc = w[e];
    for (int i = 0; i < nvec; ++i) acc = fma(-coef[i + c * ldc], V[(static_cast<long long>(i) * nrhs + c) * N + r], acc);
    w[e] = acc;
  }
}

// w(:, c) *= 1 / nrm[c]  (a zero norm -- a breakdown -- leaves a zero vector)
__global__ void col_scale_inv(double* __restrict__ w, long long N, int nrhs, const double* __restrict__ nrm) {
  const long long total = N * nrhs;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e / N);
    const double d = nrm[c];
    w[e] = d > 0.0 ? w[e] / d : 0.0;
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

// Y = alpha Z + beta W + gamma A X
static cudaError_t resid(const LsScratch& sc, const double* A, long long lda, int m, int n, const double* X,
                         long long ldx, int nrhs, const double* Z, long long ldz, double alpha, const double* Wm,
                         long long ldw, double beta, double gamma, double* Y, long long ldy, cudaStream_t st) {
  dim3 grid((m + kLsThreads - 1) / kLsThreads, sc.nsplit);
  gemm_nn_partial<<<grid, kLsThreads, 0, st>>>(A, lda, m, n, X, ldx, nrhs, sc.split_len, sc.part);
  combine_partials<<<ew_grid(static_cast<long long>(m) * nrhs), 256, 0, st>>>(sc.part, sc.nsplit, m, nrhs, Z, ldz,
                                                                            alpha, Wm, ldw, beta, gamma, Y, ldy);
  return cudaGetLastError();
}

// G = alpha s A^T R, s = norm_scale(*nA) (nA null: s = 1)
static cudaError_t atr(const double* A, long long lda, int m, int n, const double* R, long long ldr, int nrhs,
                       double alpha, double* G, long long ldg, cudaStream_t st, const double* nA = nullptr) {
  const int wpb = kLsThreads / 32;
  gemm_tn<<<(n + wpb - 1) / wpb, kLsThreads, 0, st>>>(A, lda, m, n, R, ldr, nrhs, alpha, G, ldg, nA);
  return cudaGetLastError();
}

// ||A||_F (and the column norms on the way) into nA, overflow-free
static cudaError_t fro_norm(const double* A, long long lda, int m, int n, double* colnrm, double* nA,
                            cudaStream_t st) {
  col_nrm2<<<n, kLsThreads, 0, st>>>(A, lda, m, colnrm);
  col_nrm2<<<1, kLsThreads, 0, st>>>(colnrm, n, n, nA);
  return cudaGetLastError();
}

struct BerrBufs {
  double* G;     // n x nrhs
  double* nrm;   // 4 * nrhs + 4
};

static size_t al(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// GMRES-IR constants: Krylov steps per outer step (restart length), relative
// residual the inner solve stops at, and the limit on inner steps in total.
constexpr int kGmresRestart = 30;
constexpr double kGmresInnerTol = 1e-3;
constexpr int kGmresMaxInner = 300;
// GMRES-IR runs only while the FP32 factor's diagonal spread puts
// kappa u_fp32 below 0.03, and stops after a cycle that left the relative
// residual above 0.1: beyond that the FP32 factors, applied in FP32, no
// longer precondition the augmented system well enough for GMRES to
// converge in a few steps (their rounding acts as a perturbation of the
// operator), and an FP64 solve is the faster way to the answer.  Measured on
// U diag(sigma) V^T problems: kappa = 1e7 gives a spread times u_fp32 of
// 0.017-0.023 and converges (35-45 GMRES steps); kappa = 1e8 gives
// 0.042-0.083 and stalls (relative residual 0.76-0.93 after 30 steps).
constexpr double kGmresSpreadLimit = 0.03;
constexpr double kGmresGiveUp = 0.1;
// The FP32 factorization is used only for A with 2^-40 <= ||A||_F <= 2^40:
// every entry is then at most 2^40, so the FP32 products of the panel and
// update kernels stay below 2^80, far from FP32's overflow at 2^128; other
// problems are solved in FP64.
constexpr double kFp32NormLo = 0x1p-40, kFp32NormHi = 0x1p40;

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
  factored = false;
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
  o_nrm = o;   o += al(sizeof(double) * (4 * rhs_cap + 12));
  o_b2 = o;    o += al(W.oT - W.oB);                       // as large as the first tile array
  o_ver2 = o;  o += al(sizeof(int) * static_cast<size_t>(I.p) * (I.q + I.qb) * I.NS);
  o_inst2 = o; o += al(2 * sizeof(Inst));
  o_tctl = o;  o += al(sizeof(int) * trsv_ctl_ints(n, nb));
  o_y = o;     o += al(sizeof(double) * nr);
  o_acopy = o;
  bytes = o;
  return true;
}

size_t LsJob::bytes_with_acopy() const { return bytes + al(sizeof(double) * static_cast<size_t>(m) * n); }

double* LsJob::err_rec() const { return reinterpret_cast<double*>(ws + o_nrm) + 4 * rhs_cap + 4; }

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
  return esize == 8 ? run_plan<double>(I, ws, W, occ, smem, st, grid_cap, err_rec())
                    : run_plan<float>(I, ws, W, occ, smem, st, grid_cap, err_rec());
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
  return esize == 8 ? run_plan_multi<double>(two, 2, d_insts, d_ctl, occ, smem, st, grid_cap, err_rec())
                    : run_plan_multi<float>(two, 2, d_insts, d_ctl, occ, smem, st, grid_cap, err_rec());
}

int LsJob::fast_ok(int nrhs) const { return esize == 4 && trsv_fits(nb, nrhs, 4) ? 1 : 0; }

// R X = Y or R^T X = Y with the FP32 factor's R, one launch (fast_ok).  A
// wait that runs out is recorded in the backward-error read-back area
// (slot 4 rhs_cap + 1) and reported by finish.
int LsJob::trsv(bool trans, const double* Y, long long ldy, double* X, long long ldx, int nrhs, cudaStream_t st) {
  double* err = reinterpret_cast<double*>(ws + o_nrm) + 4 * rhs_cap + 1;
  return launch_trsv<float>(trans, static_cast<const float*>(I.A), I.p, nb, n, nrhs, Y, ldy, X, ldx,
                            reinterpret_cast<int*>(ws + o_tctl), wait_limit_ns(), err, st) == cudaSuccess
             ? TQR_OK
             : TQR_ERR_CUDA;
}

// The explicit thin Q1 (m x n, FP32 tiles): the identity's first n columns
// through the factorization's Q (the M_FORM_Q task graph), once per solve.
int LsJob::form_q1(cudaStream_t st) {
  if (vws != nullptr) return TQR_OK;
  Inst Iq = I;
  Iq.mode = M_FORM_Q;
  Iq.trsm = 0;
  Iq.nrhs = n;
  Iq.qb = I.q;
  const size_t tiles = al(sizeof(float) * static_cast<size_t>(nb) * nb * I.p * I.q);
  size_t o = tiles;
  vo_ver = o;  o += al(sizeof(int) * static_cast<size_t>(I.p) * (2 * I.q) * I.NS);
  vo_inst = o; o += al(sizeof(Inst));
  vo_ctl = o;  o += al(ctl_bytes());
  vo_part = o; o += al(sizeof(float) * kQ1SplitsCap * static_cast<size_t>(std::max(m, n)) * rhs_cap);
  vbytes = o;
  if (lib_malloc(reinterpret_cast<void**>(&vws), vbytes, st) != cudaSuccess) {
    cudaGetLastError();
    vws = nullptr;
    return TQR_ERR_NOMEM;
  }
  Iq.B = vws;
  Iq.ver = reinterpret_cast<int*>(vws + vo_ver);
  if (launch_identity<float>(m, n, static_cast<float*>(Iq.B), I.p, I.q, nb, device_sms(), st) != cudaSuccess)
    return TQR_ERR_CUDA;
  WsLayout W2 = {};
  W2.oVer = vo_ver;
  W2.oInst = vo_inst;
  W2.oCtl = vo_ctl;
  W2.bytes = vbytes;
  return run_plan<float>(Iq, vws, W2, occ, smem, st, grid_cap, err_rec());
}

void LsJob::free_q1(cudaStream_t st) {
  if (vws) cudaFreeAsync(vws, st);
  vws = nullptr;
}

// [U; V] = M^-1 [F; G] with M = [I, QR; (QR)^T, 0] from the factors in the
// tiles: d = Q^T F and h = R^-T G (one launch), then V = R^-1 (d1 - h) and
// U = Q [h; d2] (one launch) -- the correction of the augmented-system
// refinement, and the preconditioner of GMRES-IR.  F: m x nrhs (ldf), G:
// n x nrhs (ldg), U: m x nrhs (ldu), V: n x nrhs (ldv).  The inputs are
// packed into the tiles before the scratch D, H and the G buffer are
// written, so F and G may be those buffers.
int LsJob::precond(const double* F, long long ldf, const double* G, long long ldg, double* U, long long ldu,
                   double* V, long long ldv, int nrhs, cudaStream_t st) {
  if (vws != nullptr) {
    // explicit Q1: h = R^-T g, y = Q1^T f - h, V = R^-1 y, U = f - Q1 y
    // (= Q [h; d2] with d2 = Q2^T f, since Q1 Q1^T + Q2 Q2^T = I)
    double* Hh = reinterpret_cast<double*>(ws + o_h);
    double* Yy = reinterpret_cast<double*>(ws + o_y);
    float* Q1 = reinterpret_cast<float*>(vws);
    float* part = reinterpret_cast<float*>(vws + vo_part);
    const size_t nr = static_cast<size_t>(n) * nrhs;
    int s = trsv(true, G, ldg, Hh, n, nrhs, st);
    if (s == TQR_OK &&
        launch_q1t(Q1, I.p, nb, m, n, nrhs, F, ldf, 1.0, part, kQ1SplitsCap, Yy, n, st) != cudaSuccess)
      s = TQR_ERR_CUDA;
    if (s != TQR_OK) return s;
    axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, 1.0, Yy, n, -1.0, Hh, n, Yy, n);
    if (cudaGetLastError() != cudaSuccess) return TQR_ERR_CUDA;
    s = trsv(false, Yy, n, V, ldv, nrhs, st);
    if (s == TQR_OK &&
        launch_q1n(Q1, I.p, nb, m, n, nrhs, Yy, n, 1.0, F, ldf, part, kQ1SplitsCap, U, ldu, st) != cudaSuccess)
      s = TQR_ERR_CUDA;
    return s;
  }
  double* D = reinterpret_cast<double*>(ws + o_d);
  double* H = reinterpret_cast<double*>(ws + o_h);
  double* Gv = reinterpret_cast<double*>(ws + o_g);
  void* B2 = ws + o_b2;
  const size_t nr = static_cast<size_t>(n) * nrhs;
  int s = pack_rhs(F, ldf, m, nrhs, st);
  if (s == TQR_OK) s = pack_rhs(G, ldg, n, nrhs, st, B2);
  if (s == TQR_OK) s = run_two(M_APPLY_QT, M_TRSMT, nrhs, st);
  if (s == TQR_OK) s = unpack_rhs(D, m, m, nrhs, st);
  if (s == TQR_OK) s = unpack_rhs(H, n, n, nrhs, st, B2);
  if (s != TQR_OK) return s;
  axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, 1.0, D, m, -1.0, H, n, Gv, n);
  axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, 1.0, H, n, 0.0, nullptr, 0, D, m);
  if (cudaGetLastError() != cudaSuccess) return TQR_ERR_CUDA;
  s = pack_rhs(D, m, m, nrhs, st);
  if (s == TQR_OK) s = pack_rhs(Gv, n, n, nrhs, st, B2);
  if (s == TQR_OK) s = run_two(M_APPLY_Q, M_TRSM, nrhs, st);
  if (s == TQR_OK) s = unpack_rhs(U, ldu, m, nrhs, st);
  if (s == TQR_OK) s = unpack_rhs(V, ldv, n, nrhs, st, B2);
  return s;
}

// Factors A (and keeps the factors) and, with nrhs > 0, runs Q^T B and the
// back substitution in the same graph: x0 through those factors.  Also
// ||A||_F and R's extreme diagonal entries for the solve's checks.  The FP32
// class first checks that A suits FP32 (kLsFp32Range if not).
int LsJob::factor_solve(const double* A, long long lda, const double* B, long long ldb, int nrhs, cudaStream_t st) {
  const int sms = device_sms();
  factored = false;
  double* nrm = reinterpret_cast<double*>(ws + o_nrm);
  double* colnrm = reinterpret_cast<double*>(ws + o_g);
  std::fill(err_host, err_host + 8, 0.0);
  if (cudaMemsetAsync(err_rec(), 0, 8 * sizeof(double), st) != cudaSuccess) return TQR_ERR_CUDA;
  if (fro_norm(A, lda, m, n, colnrm, nrm + 4 * rhs_cap, st) != cudaSuccess) return TQR_ERR_CUDA;
  if (esize == 4) {
    double h = 0.0;
    if (cudaMemcpyAsync(&h, nrm + 4 * rhs_cap, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return TQR_ERR_CUDA;
    if (!std::isfinite(h)) return TQR_ERR_NONFINITE;
    if (!(h >= kFp32NormLo && h <= kFp32NormHi)) return kLsFp32Range;
  }
  if (upload_vtab(I, ws, W, st) != TQR_OK) return TQR_ERR_CUDA;
  if (Acopy != nullptr &&
      copy_cols(Acopy, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m, n,
                cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return TQR_ERR_CUDA;
  cudaError_t e = esize == 8 ? launch_pack<double>(A, lda, m, n, static_cast<double*>(I.A), I.p, I.q, nb, sms, st)
                             : launch_pack<float>(A, lda, m, n, static_cast<float*>(I.A), I.p, I.q, nb, sms, st);
  if (e != cudaSuccess) return TQR_ERR_CUDA;
  int s = TQR_OK;
  if (nrhs > 0) {
    s = pack_rhs(B, ldb, m, nrhs, st);
    if (s == TQR_OK) s = run_mode(M_FACTOR, 1, nrhs, st);
    if (s == TQR_OK) s = unpack_rhs(reinterpret_cast<double*>(ws + o_x), n, n, nrhs, st);
  } else {
    s = run_mode(M_FACTOR, 0, 0, st);
  }
  if (s == TQR_OK) {
    double* dmm = nrm + 4 * rhs_cap + 2;
    if (esize == 8)
      diag_minmax<double><<<1, kLsThreads, 0, st>>>(static_cast<double*>(I.A), I.p, nb, n, dmm);
    else
      diag_minmax<float><<<1, kLsThreads, 0, st>>>(static_cast<float*>(I.A), I.p, nb, n, dmm);
    if (cudaGetLastError() != cudaSuccess) s = TQR_ERR_CUDA;
  }
  factored = (s == TQR_OK);
  return s;
}

// x0 from the resident factors: Q^T B and back substitution, one graph
int LsJob::solve(const double* B, long long ldb, int nrhs, cudaStream_t st) {
  std::fill(err_host, err_host + 8, 0.0);
  if (cudaMemsetAsync(err_rec(), 0, 8 * sizeof(double), st) != cudaSuccess) return TQR_ERR_CUDA;
  int s = pack_rhs(B, ldb, m, nrhs, st);
  if (s == TQR_OK) s = run_mode(M_APPLY_QT, 1, nrhs, st);
  if (s == TQR_OK) s = unpack_rhs(reinterpret_cast<double*>(ws + o_x), n, n, nrhs, st);
  return s;
}

// Backward error of x, FP32 refinement, copy of x to X.  A is the FP64
// matrix (caller's or the resident copy).
int LsJob::finish(const double* A, long long lda, const double* B, long long ldb, int nrhs, double* X, long long ldx,
                  double tol, int maxit, tqr_ls_info* info, cudaStream_t st) {
  const size_t mr = static_cast<size_t>(m) * nrhs, nr = static_cast<size_t>(n) * nrhs;
  double* E = reinterpret_cast<double*>(ws + o_e);
  double* Rr = reinterpret_cast<double*>(ws + o_r);
  double* F = reinterpret_cast<double*>(ws + o_f);
  double* D = reinterpret_cast<double*>(ws + o_d);
  double* Gv = reinterpret_cast<double*>(ws + o_g);
  double* Xw = reinterpret_cast<double*>(ws + o_x);
  BerrBufs bb;
  bb.G = reinterpret_cast<double*>(ws + o_G);
  bb.nrm = reinterpret_cast<double*>(ws + o_nrm);
  // nrm layout (norms, not squares): [0,R) ||A^T e||, [R,2R) ||x||, [2R,3R) ||b||,
  // [3R,4R) ||dx||, [4R] ||A||_F, [4R+1] the triangular-solve kernel's
  // error, [4R+2], [4R+3] min and max |r_ii|, [4R+4, 4R+12) the task-kernel
  // launches' error record
  const int R = rhs_cap;
  double* dx2 = bb.nrm + 3 * R;
  std::vector<double> hn(4 * R + 12);
  int status = TQR_OK;
  int iters = 0, inner = 0, path = esize == 8 ? TQR_LS_PATH_FP64 : TQR_LS_PATH_FP32;
  double berr = INFINITY, gres = 0.0;
  auto fail = [&](int s) {
    if (status == TQR_OK && s != TQR_OK) status = s;
  };
  auto read_back = [&]() {
    if (cudaMemcpyAsync(hn.data(), bb.nrm, sizeof(double) * hn.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      fail(TQR_ERR_CUDA);
    if (hn[4 * R + 1] != 0.0) fail(TQR_ERR_TIMEOUT);  // a triangular-solve wait ran out
    if (hn[4 * R + 4] != 0.0) {                       // a task-kernel wait ran out
      for (int a = 0; a < 8; ++a) err_host[a] = hn[4 * R + 4 + a];
      fail(static_cast<int>(hn[4 * R + 4]));
    }
  };
  // the triangular-solve kernel's error slot starts clear
  if (cudaMemsetAsync(bb.nrm + 4 * R + 1, 0, sizeof(double), st) != cudaSuccess) fail(TQR_ERR_CUDA);
  // hn[c] holds s ||A^T e|| with s = norm_scale(||A||_F) (exact power of
  // two), so the ratio is formed as s||A^T e|| / ((s ||A||) (||A|| ||x|| + ||b||))
  // -- every factor finite for any finite data
  auto berr_of = [&]() {
    double worst = 0.0;
    const double nA = hn[4 * R];
    const double sA = norm_scale(nA);
    for (int c = 0; c < nrhs; ++c) {
      const double num = hn[c];
      const double den = (sA * nA) * (nA * hn[R + c] + hn[2 * R + c]);
      // a NaN anywhere (x included) makes the backward error NaN
      const double eta = std::isnan(num) || std::isnan(den) ? NAN
                         : den > 0                          ? num / den
                         : (num > 0 ? INFINITY : 0.0);
      if (std::isnan(eta)) return static_cast<double>(NAN);
      if (!(eta <= worst)) worst = eta;
    }
    return worst;
  };
  // e = b - A x, A^T e and the norms of the backward error
  auto terms = [&]() {
    if (resid(sc, A, lda, m, n, Xw, n, nrhs, B, ldb, 1.0, nullptr, 0, 0.0, -1.0, E, m, st) != cudaSuccess ||
        atr(A, lda, m, n, E, m, nrhs, 1.0, bb.G, n, st, bb.nrm + 4 * R) != cudaSuccess)
      fail(TQR_ERR_CUDA);
    col_nrm2<<<nrhs, kLsThreads, 0, st>>>(bb.G, n, n, bb.nrm);
    col_nrm2<<<nrhs, kLsThreads, 0, st>>>(Xw, n, n, bb.nrm + R);
    col_nrm2<<<nrhs, kLsThreads, 0, st>>>(B, ldb, m, bb.nrm + 2 * R);
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
  double prev = berr, prev_dx = INFINITY, dxrel = INFINITY;
  bool settled = false;
  auto dx_rel = [&](double scale) {
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
      const double xr = hn[R + c];
      const double d = hn[3 * R + c] / scale;
      const double rel = xr > 0 ? d / xr : d;
      if (!(rel <= worst)) worst = rel;
    }
    return worst;
  };
  // Refinement runs until the backward error meets tol AND x has settled at
  // FP64 accuracy: the last correction is below FP64 rounding (||dx|| <=
  // 2^-50 ||x||) or, with the backward error already met, no longer halves
  // (the corrections have reached the rounding noise of the FP64
  // residuals), so the answer matches an FP64 solve; a form gives way to the
  // next on stagnation (neither the backward error nor the correction halves
  // for 3 steps), and the whole refinement stops at maxit.
  auto more = [&]() { return status == TQR_OK && !settled && (berr > tol || dxrel > 0x1p-50) && iters < maxit; };
  // spread of R's diagonal: a lower bound on kappa(A) (R from A + E)
  const double spread = hn[4 * R + 3] / hn[4 * R + 2];
  if (status == TQR_OK && esize == 4) {
    // (1) Corrected semi-normal equations: dx = R^-1 R^-T A^T e with e = b -
    // A x and A^T e already on the device from the backward-error terms --
    // two triangular-solve graphs per step and no Q application.  With R the
    // factor of A + E (||E|| ~ eps ||A||) the error contracts by about
    // 2 kappa eps per step, so they run only while the spread of R's
    // diagonal keeps kappa u_fp32 small, and give way to the augmented-system
    // refinement as soon as a step fails to halve the backward error (a step
    // that made it worse is undone).
    bool semi = spread * 0x1p-24 < 0.01;
    if (semi) path = TQR_LS_PATH_FP32_SEMINORMAL;
    while (semi && more()) {
      // the device holds s A^T e (s = norm_scale(||A||_F)); scale it by a
      // power of two near 1/max ||.|| so FP32 keeps it normal: Gv = g A^T e
      // with g = gs s, and the correction is R^-1 R^-T Gv / g
      double gmax = 0.0;
      for (int c = 0; c < nrhs; ++c) gmax = std::max(gmax, hn[c]);
      const double gs = gmax > 0 && std::isfinite(gmax) ? std::ldexp(1.0, -std::ilogb(gmax)) : 1.0;
      const double scale = gs * norm_scale(hn[4 * R]);
      axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, gs, bb.G, n, 0.0, nullptr, 0, Gv, n);
      if (fast_ok(nrhs)) {
        // R^-T then R^-1 by the triangular-solve kernel, in place
        fail(trsv(true, Gv, n, Gv, n, nrhs, st));
        if (status == TQR_OK) fail(trsv(false, Gv, n, Gv, n, nrhs, st));
      } else {
        fail(pack_rhs(Gv, n, n, nrhs, st));
        if (status == TQR_OK) fail(run_mode(M_TRSMT, 0, nrhs, st));
        if (status == TQR_OK) fail(run_mode(M_TRSM, 0, nrhs, st));
        fail(unpack_rhs(Gv, n, n, nrhs, st));
      }
      col_nrm2<<<nrhs, kLsThreads, 0, st>>>(Gv, n, n, dx2);
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
    // (2) Bjorck's refinement of the augmented system [I A; A^T 0][r; x] =
    // [b; 0], corrections through the factors (precond).  It contracts by
    // about kappa u_fp32 per step, so it is skipped when R's diagonal spread
    // already puts kappa u_fp32 above 0.02, and gives way to GMRES-IR when
    // it stagnates.
    int stall = 0;
    const bool aug = spread * 0x1p-24 < 0.02;
    if (aug && more()) path = TQR_LS_PATH_FP32_AUGMENTED;
    // the refinements with Q apply it through the explicit thin Q1 when the
    // few-right-hand-side kernels take this problem
    if (more() && fast_ok(nrhs) && (aug || spread * 0x1p-24 < kGmresSpreadLimit)) fail(form_q1(st));
    while (aug && more()) {
      // f = b - r - A x = e - r;  g = -A^T r;  [dr; dx] = M^-1 [f; g]
      axpby<<<ew_grid(mr), 256, 0, st>>>(m, nrhs, 1.0, E, m, -1.0, Rr, m, F, m);
      if (atr(A, lda, m, n, Rr, m, nrhs, -1.0, Gv, n, st) != cudaSuccess) fail(TQR_ERR_CUDA);
      if (status == TQR_OK) fail(precond(F, m, Gv, n, D, m, Gv, n, nrhs, st));
      col_nrm2<<<nrhs, kLsThreads, 0, st>>>(Gv, n, n, dx2);
      axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, 1.0, Xw, n, 1.0, Gv, n, Xw, n);
      axpby<<<ew_grid(mr), 256, 0, st>>>(m, nrhs, 1.0, Rr, m, 1.0, D, m, Rr, m);
      ++iters;
      terms();
      read_back();
      if (status != TQR_OK) break;
      berr = berr_of();
      dxrel = dx_rel(1.0);
      if (berr <= tol && !(dxrel < 0.5 * prev_dx)) {
        settled = true;
        break;
      }
      if (!(berr < 0.5 * prev) && !(dxrel < 0.5 * prev_dx)) {
        if (++stall >= 3) break;
      } else {
        stall = 0;
      }
      prev = std::min(prev, berr);
      prev_dx = std::min(prev_dx, dxrel);
    }
    // (3) GMRES-IR (Carson, Higham and Pranesh 2020): each outer step solves
    // the correction equation [I A; A^T 0][dr; dx] = [f; g] by GMRES on the
    // system left-preconditioned with precond (M^-1 applied in the factors'
    // precision, the augmented operator and all GMRES arithmetic in FP64).
    if (more() && spread * 0x1p-24 < kGmresSpreadLimit) {
      path = TQR_LS_PATH_FP32_GMRES;
      const long long N = static_cast<long long>(m) + n;
      const int K = kGmresRestart;
      const size_t basis = sizeof(double) * static_cast<size_t>(K + 1) * N * nrhs;
      const size_t zbytes = sizeof(double) * static_cast<size_t>(N) * nrhs;
      const size_t hbytes = sizeof(double) * static_cast<size_t>(2 * (K + 1) + 1) * nrhs;
      char* gm = nullptr;
      if (lib_malloc(reinterpret_cast<void**>(&gm), al(basis) + al(zbytes) + al(hbytes), st) != cudaSuccess) {
        cudaGetLastError();
        gm = nullptr;
        fail(TQR_ERR_NOMEM);
      }
      double* Vb = reinterpret_cast<double*>(gm);
      double* Z = reinterpret_cast<double*>(gm + al(basis));
      double* h1 = reinterpret_cast<double*>(gm + al(basis) + al(zbytes));  // (K+1) x nrhs, then h2, then ||w||
      double* h2 = h1 + static_cast<size_t>(K + 1) * nrhs;
      double* hw = h2 + static_cast<size_t>(K + 1) * nrhs;
      // host side of GMRES per right-hand side c: Hessenberg columns after
      // the Givens rotations (upper triangle, column-major (K+1) x K), the
      // rotations, the rotated right-hand side g and the step count k_c at
      // which the column converged
      std::vector<double> Hh(static_cast<size_t>(K + 1) * K * nrhs), cs(static_cast<size_t>(K) * nrhs),
          sn(static_cast<size_t>(K) * nrhs), g(static_cast<size_t>(K + 1) * nrhs), beta(nrhs), hh(2 * (K + 1) * nrhs + nrhs),
          y(static_cast<size_t>(K + 1) * nrhs);
      std::vector<int> kc(nrhs);
      auto vec = [&](int i) { return Vb + static_cast<size_t>(i) * nrhs * N; };
      auto normalize = [&](double* w) {
        col_nrm2<<<nrhs, kLsThreads, 0, st>>>(w, N, static_cast<int>(N), hw);
        col_scale_inv<<<ew_grid(N * nrhs), 256, 0, st>>>(w, N, nrhs, hw);
        if (cudaGetLastError() != cudaSuccess) fail(TQR_ERR_CUDA);
      };
      int stall = 0;
      prev = berr;
      prev_dx = INFINITY;
      while (more() && inner < kGmresMaxInner) {
        // s = M^-1 [f; g] with f = e - r, g = -A^T r: the first basis vector
        axpby<<<ew_grid(mr), 256, 0, st>>>(m, nrhs, 1.0, E, m, -1.0, Rr, m, F, m);
        if (atr(A, lda, m, n, Rr, m, nrhs, -1.0, Gv, n, st) != cudaSuccess) fail(TQR_ERR_CUDA);
        if (status == TQR_OK) fail(precond(F, m, Gv, n, vec(0), N, vec(0) + m, N, nrhs, st));
        normalize(vec(0));
        if (status == TQR_OK && (cudaMemcpyAsync(beta.data(), hw, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st) !=
                                     cudaSuccess ||
                                 cudaStreamSynchronize(st) != cudaSuccess))
          fail(TQR_ERR_CUDA);
        if (status != TQR_OK) break;
        int open = 0;
        for (int c = 0; c < nrhs; ++c) {
          std::fill(g.begin() + static_cast<size_t>(c) * (K + 1), g.begin() + static_cast<size_t>(c + 1) * (K + 1), 0.0);
          g[static_cast<size_t>(c) * (K + 1)] = beta[c];
          kc[c] = (beta[c] > 0.0 && std::isfinite(beta[c])) ? -1 : 0;  // -1: still iterating
          open += kc[c] < 0;
        }
        int steps = 0;
        for (int j = 0; j < K && open > 0 && inner < kGmresMaxInner; ++j) {
          double* vj = vec(j);
          double* w = vec(j + 1);
          // [u_j + A v_j; A^T u_j], then M^-1 of it into w
          if (resid(sc, A, lda, m, n, vj + m, N, nrhs, vj, N, 1.0, nullptr, 0, 0.0, 1.0, F, m, st) != cudaSuccess ||
              atr(A, lda, m, n, vj, N, nrhs, 1.0, Gv, n, st) != cudaSuccess)
            fail(TQR_ERR_CUDA);
          if (status == TQR_OK) fail(precond(F, m, Gv, n, w, N, w + m, N, nrhs, st));
          // classical Gram-Schmidt, twice (as stable as modified Gram-Schmidt
          // and two reductions per step instead of j + 1)
          gmres_dots<<<dim3(j + 1, nrhs), kLsThreads, 0, st>>>(Vb, j + 1, N, nrhs, w, h1, K + 1);
          gmres_axpy<<<ew_grid(N * nrhs), 256, 0, st>>>(Vb, j + 1, N, nrhs, h1, K + 1, w);
          gmres_dots<<<dim3(j + 1, nrhs), kLsThreads, 0, st>>>(Vb, j + 1, N, nrhs, w, h2, K + 1);
          gmres_axpy<<<ew_grid(N * nrhs), 256, 0, st>>>(Vb, j + 1, N, nrhs, h2, K + 1, w);
          normalize(w);
          if (status == TQR_OK && (cudaMemcpyAsync(hh.data(), h1, hbytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                                   cudaStreamSynchronize(st) != cudaSuccess))
            fail(TQR_ERR_CUDA);
          if (status != TQR_OK) break;
          ++inner;
          steps = j + 1;
          for (int c = 0; c < nrhs; ++c) {
            if (kc[c] >= 0) continue;
            double* Hc = Hh.data() + static_cast<size_t>(c) * (K + 1) * K;
            double* col = Hc + static_cast<size_t>(j) * (K + 1);
            for (int i = 0; i <= j; ++i)
              col[i] = hh[i + static_cast<size_t>(c) * (K + 1)] + hh[(K + 1) * static_cast<size_t>(nrhs) + i + static_cast<size_t>(c) * (K + 1)];
            col[j + 1] = hh[2 * (K + 1) * static_cast<size_t>(nrhs) + c];
            // earlier rotations, then the one that zeroes col[j + 1]
            double* csc = cs.data() + static_cast<size_t>(c) * K;
            double* snc = sn.data() + static_cast<size_t>(c) * K;
            for (int i = 0; i < j; ++i) {
              const double a = col[i], b2 = col[i + 1];
              col[i] = csc[i] * a + snc[i] * b2;
              col[i + 1] = -snc[i] * a + csc[i] * b2;
            }
            const double rho = std::hypot(col[j], col[j + 1]);
            const double cj = rho > 0 ? col[j] / rho : 1.0, sj = rho > 0 ? col[j + 1] / rho : 0.0;
            csc[j] = cj;
            snc[j] = sj;
            col[j] = rho;
            col[j + 1] = 0.0;
            double* gc = g.data() + static_cast<size_t>(c) * (K + 1);
            gc[j + 1] = -sj * gc[j];
            gc[j] = cj * gc[j];
            const double res = std::fabs(gc[j + 1]) / beta[c];
            const bool breakdown = !(hh[2 * (K + 1) * static_cast<size_t>(nrhs) + c] > 0.0);
            if (res <= kGmresInnerTol || breakdown || !std::isfinite(res)) {
              kc[c] = j + 1;
              --open;
            }
          }
        }
        if (status != TQR_OK) break;
        // y_c from the rotated triangle (k_c steps), z = sum_i y_i v_i
        int kmax = 0;
        gres = 0.0;
        for (int c = 0; c < nrhs; ++c) {
          if (kc[c] < 0) kc[c] = steps;
          kmax = std::max(kmax, kc[c]);
          if (kc[c] > 0) gres = std::max(gres, std::fabs(g[static_cast<size_t>(c) * (K + 1) + kc[c]]) / beta[c]);
          const double* Hc = Hh.data() + static_cast<size_t>(c) * (K + 1) * K;
          const double* gc = g.data() + static_cast<size_t>(c) * (K + 1);
          double* yc = y.data() + static_cast<size_t>(c) * (K + 1);
          std::fill(yc, yc + K + 1, 0.0);
          for (int i = kc[c] - 1; i >= 0; --i) {
            double t = gc[i];
            for (int l = i + 1; l < kc[c]; ++l) t -= Hc[i + static_cast<size_t>(l) * (K + 1)] * yc[l];
            const double d = Hc[i + static_cast<size_t>(i) * (K + 1)];
            yc[i] = d != 0.0 ? t / d : 0.0;
          }
          for (int i = 0; i < kc[c]; ++i) yc[i] = -yc[i];  // gmres_axpy subtracts
        }
        if (cudaMemcpyAsync(h1, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(Z, 0, zbytes, st) != cudaSuccess)
          fail(TQR_ERR_CUDA);
        gmres_axpy<<<ew_grid(N * nrhs), 256, 0, st>>>(Vb, kmax, N, nrhs, h1, K + 1, Z);
        // x += dz_v, r += dz_u
        col_nrm2<<<nrhs, kLsThreads, 0, st>>>(Z + m, N, n, dx2);
        axpby<<<ew_grid(nr), 256, 0, st>>>(n, nrhs, 1.0, Xw, n, 1.0, Z + m, N, Xw, n);
        axpby<<<ew_grid(mr), 256, 0, st>>>(m, nrhs, 1.0, Rr, m, 1.0, Z, N, Rr, m);
        if (cudaGetLastError() != cudaSuccess) fail(TQR_ERR_CUDA);
        ++iters;
        terms();
        read_back();
        if (status != TQR_OK) break;
        berr = berr_of();
        dxrel = dx_rel(1.0);
        if (berr <= tol && !(dxrel < 0.5 * prev_dx)) {
          settled = true;
          break;
        }
        if (!(gres <= kGmresGiveUp)) break;
        if (!(berr < 0.5 * prev) && !(dxrel < 0.5 * prev_dx)) {
          if (++stall >= 3) break;
        } else {
          stall = 0;
        }
        prev = std::min(prev, berr);
        prev_dx = std::min(prev_dx, dxrel);
      }
      if (gm) cudaFreeAsync(gm, st);
    }
    // short of tol: maxit (the caller's limit) ends the solve with
    // TQR_ERR_NOCONV; stagnation hands the problem to an FP64 solve
    if (status == TQR_OK && !(berr <= tol)) status = iters >= maxit ? TQR_ERR_NOCONV : kLsStalled;
  }
  free_q1(st);
  if (X != nullptr &&
      copy_cols(X, sizeof(double) * ldx, Xw, sizeof(double) * n, sizeof(double) * n, nrhs,
                cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    fail(TQR_ERR_CUDA);
  if (info) {
    info->path = path;
    info->iters = iters;
    info->inner_iters = inner;
    info->berr = berr;
    info->gmres_res = gres;
    info->r_spread = hn[4 * R + 3] / hn[4 * R + 2];
  }
  return status;
}

// The FP32 class's way out: a problem FP32 refinement cannot finish (no
// convergence, or A outside FP32's comfortable range) is solved again in
// FP64 from its FP64 data.
static bool wants_fp64(int status) { return status == kLsStalled || status == kLsFp32Range; }

static thread_local tqr_ls_info t_last_info = {};

static int solve_device_prec(int64_t m64, int64_t n64, int64_t nrhs64, const double* A, int64_t lda,
                             const double* B, int64_t ldb, double* X, int64_t ldx, int prec, double tol, int maxit,
                             tqr_ls_info* info, int nb, int ib, cudaStream_t st) {
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
    status = job.finish(A, lda, B, ldb, static_cast<int>(nrhs64), X, ldx, tol, maxit, info, st);
  cudaFreeAsync(ws, st);
  int dev_status = TQR_OK;
  if (read_status(&dev_status, st) != cudaSuccess && status == TQR_OK) status = TQR_ERR_CUDA;
  if (dev_status != TQR_OK) status = dev_status;
  return status;
}

static int solve_device(int64_t m64, int64_t n64, int64_t nrhs64, const double* A, int64_t lda, const double* B,
                        int64_t ldb, double* X, int64_t ldx, int prec, double tol, int maxit, tqr_ls_info* info,
                        int nb, int ib, cudaStream_t st) {
  tqr_ls_info first = {};
  first.path = prec == TQR_PREC_FP64 ? TQR_LS_PATH_FP64 : TQR_LS_PATH_FP32;
  int status = solve_device_prec(m64, n64, nrhs64, A, lda, B, ldb, X, ldx, prec, tol, maxit, &first, nb, ib, st);
  *info = first;
  info->fp32_status = TQR_OK;
  info->berr_fp32 = prec == TQR_PREC_FP32 ? first.berr : 0.0;
  if (prec == TQR_PREC_FP32 && wants_fp64(status)) {
    tqr_ls_info second = {};
    const int s32 = status;
    status = solve_device_prec(m64, n64, nrhs64, A, lda, B, ldb, X, ldx, TQR_PREC_FP64, tol, 0, &second, nb, ib, st);
    info->fp32_status = s32 == kLsFp32Range ? TQR_ERR_UNSUPPORTED : TQR_ERR_NOCONV;
    info->path = TQR_LS_PATH_FP64_FALLBACK;
    info->berr = second.berr;
  }
  if (status == kLsStalled || status == kLsFp32Range) status = TQR_ERR_NOCONV;
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
  tqr_ls_info info = {};
  int status = TQR_OK;
  if (ka == PTR_DEVICE) {
    status = solve_device(m, n, nrhs, A, lda, B, ldb, X, ldx, prec, tol, maxit, &info, nb, ib, st);
  } else {
    double *dA = nullptr, *dB = nullptr, *dX = nullptr;
    if (lib_malloc(reinterpret_cast<void**>(&dA), sizeof(double) * m * n, st) != cudaSuccess ||
        lib_malloc(reinterpret_cast<void**>(&dB), sizeof(double) * m * nrhs, st) != cudaSuccess ||
        lib_malloc(reinterpret_cast<void**>(&dX), sizeof(double) * n * nrhs, st) != cudaSuccess) {
      cudaGetLastError();
      if (dA) cudaFreeAsync(dA, st);
      if (dB) cudaFreeAsync(dB, st);
      return TQR_ERR_NOMEM;
    }
    if (copy_cols(dA, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m, n, cudaMemcpyHostToDevice,
                  st) != cudaSuccess ||
        copy_cols(dB, sizeof(double) * m, B, sizeof(double) * ldb, sizeof(double) * m, nrhs, cudaMemcpyHostToDevice,
                  st) != cudaSuccess)
      status = TQR_ERR_CUDA;
    if (status == TQR_OK)
      status = solve_device(m, n, nrhs, dA, m, dB, m, dX, n, prec, tol, maxit, &info, nb, ib, st);
    if ((status == TQR_OK || status == TQR_ERR_NOCONV || status == TQR_ERR_RANK) &&
        copy_cols(X, sizeof(double) * ldx, dX, sizeof(double) * n, sizeof(double) * n, nrhs, cudaMemcpyDeviceToHost,
                  st) != cudaSuccess)
      status = TQR_ERR_CUDA;
    cudaFreeAsync(dA, st);
    cudaFreeAsync(dB, st);
    cudaFreeAsync(dX, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return TQR_ERR_CUDA;
  }
  if (iters) *iters = info.iters;
  if (berr) *berr = info.berr;
  t_last_info = info;
  return status;
}

extern "C" int tqr_ls_last_info(tqr_ls_info* info) {
  if (info == nullptr) return -1;
  *info = t_last_info;
  return TQR_OK;
}

// ---------------------------------------------------------------------------
// Resident factorization handle: tqr_ls_factor / tqr_ls_solve / tqr_ls_release.
struct tqr_ls {
  tqr::LsJob job;             // the requested class's factorization, with the FP64 copy of A
  char* ws = nullptr;
  tqr::LsJob job64;           // FP64 factorization made after an FP32 fallback
  char* ws64 = nullptr;
  bool has64 = false;
  int prec = 0;
  int device = 0;
};

namespace tqr {

// FP64 factorization of the handle's resident copy of A (for the FP32
// class's fallback).
static int ls_make_fp64(tqr_ls* h, cudaStream_t st) {
  if (h->has64) return TQR_OK;
  if (!h->job64.init(h->job.m, h->job.n, h->job.rhs_cap, h->job.nb, h->job.ib, TQR_PREC_FP64, 0))
    return TQR_ERR_UNSUPPORTED;
  if (lib_malloc(reinterpret_cast<void**>(&h->ws64), h->job64.bytes, st) != cudaSuccess) {
    cudaGetLastError();
    h->ws64 = nullptr;
    return TQR_ERR_NOMEM;
  }
  h->job64.bind(h->ws64, false);
  const int s = h->job64.factor_solve(h->job.Acopy, h->job.m, nullptr, 0, 0, st);
  if (s != TQR_OK) {
    cudaFreeAsync(h->ws64, st);
    h->ws64 = nullptr;
    return s;
  }
  h->has64 = true;
  return TQR_OK;
}

}  // namespace tqr

extern "C" int tqr_ls_factor(int64_t m, int64_t n, const double* A, int64_t lda, int prec, int nb, int ib,
                             int64_t rhs_cap, void* stream, tqr_ls** out) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (A == nullptr || ptr_kind(A) != PTR_DEVICE) return -3;
  if (lda < m) return -4;
  if (prec != TQR_PREC_FP64 && prec != TQR_PREC_FP32) return -5;
  if (rhs_cap < 1 || rhs_cap > (1 << 20)) return -8;
  if (out == nullptr) return -10;
  *out = nullptr;
  if (m > (1LL << 30)) return TQR_ERR_UNSUPPORTED;
  if (nb == 0) nb = n >= 1024 ? 128 : 64;
  if (ib == 0) ib = std::min(16, nb);
  const int c = check_tiles(nb, ib, 6, 7);
  if (c) return c;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tqr_ls* h = new tqr_ls();
  h->prec = prec;
  cudaGetDevice(&h->device);
  if (!h->job.init(static_cast<int>(m), static_cast<int>(n), static_cast<int>(rhs_cap), nb, ib, prec, 0)) {
    delete h;
    return TQR_ERR_UNSUPPORTED;
  }
  if (lib_malloc(reinterpret_cast<void**>(&h->ws), h->job.bytes_with_acopy(), st) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return TQR_ERR_NOMEM;
  }
  h->job.bind(h->ws, true);
  int s = h->job.factor_solve(A, lda, nullptr, 0, 0, st);
  if (s == kLsFp32Range) {
    // A outside FP32's range: keep the FP64 copy, factor it in FP64
    if (copy_cols(h->job.Acopy, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m, n,
                  cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      s = TQR_ERR_CUDA;
    else
      s = ls_make_fp64(h, st);
  }
  if (s != TQR_OK) {
    if (h->ws64) cudaFreeAsync(h->ws64, st);
    cudaFreeAsync(h->ws, st);
    delete h;
    return s;
  }
  *out = h;
  return TQR_OK;
}

extern "C" int tqr_ls_solve(tqr_ls* h, int64_t nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                            double tol, int maxit, tqr_ls_info* info, void* stream) {
  if (h == nullptr) return -1;
  if (nrhs < 1 || nrhs > h->job.rhs_cap) return -2;
  if (B == nullptr || ptr_kind(B) != PTR_DEVICE) return -3;
  if (ldb < h->job.m) return -4;
  if (X == nullptr || ptr_kind(X) != PTR_DEVICE) return -5;
  if (ldx < h->job.n) return -6;
  if (!(tol >= 0)) return -7;
  if (maxit < 0) return -8;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int k = static_cast<int>(nrhs);
  tqr_ls_info inf = {};
  int status = TQR_OK;
  const bool use32 = h->prec == TQR_PREC_FP32 && !h->has64;
  LsJob& J = use32 || !h->has64 ? h->job : h->job64;
  inf.path = J.esize == 8 ? TQR_LS_PATH_FP64 : TQR_LS_PATH_FP32;
  status = J.solve(B, ldb, k, st);
  if (status == TQR_OK) status = J.finish(h->job.Acopy, h->job.m, B, ldb, k, X, ldx, tol, maxit, &inf, st);
  inf.berr_fp32 = use32 ? inf.berr : 0.0;
  if (use32 && wants_fp64(status)) {
    // refinement cannot finish from the FP32 factors: factor in FP64 once,
    // keep it for the handle's later solves, and solve this one again
    const int s32 = status;
    tqr_ls_info second = {};
    status = ls_make_fp64(h, st);
    if (status == TQR_OK) status = h->job64.solve(B, ldb, k, st);
    if (status == TQR_OK)
      status = h->job64.finish(h->job.Acopy, h->job.m, B, ldb, k, X, ldx, tol, 0, &second, st);
    inf.fp32_status = s32 == kLsFp32Range ? TQR_ERR_UNSUPPORTED : TQR_ERR_NOCONV;
    inf.path = TQR_LS_PATH_FP64_FALLBACK;
    inf.berr = second.berr;
  } else if (h->prec == TQR_PREC_FP32 && h->has64) {
    inf.path = TQR_LS_PATH_FP64_FALLBACK;
  }
  if (status == kLsStalled || status == kLsFp32Range) status = TQR_ERR_NOCONV;
  int dev_status = TQR_OK;
  if (read_status(&dev_status, st) != cudaSuccess && status == TQR_OK) status = TQR_ERR_CUDA;
  if (dev_status != TQR_OK) status = dev_status;
  if (info) *info = inf;
  t_last_info = inf;
  return status;
}

extern "C" int tqr_ls_release(tqr_ls* h, void* stream) {
  if (h == nullptr) return -1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int status = TQR_OK;
  if (h->ws64 && cudaFreeAsync(h->ws64, st) != cudaSuccess) status = TQR_ERR_CUDA;
  if (h->ws && cudaFreeAsync(h->ws, st) != cudaSuccess) status = TQR_ERR_CUDA;
  delete h;
  return status;
}
