// tqr_lu.cpp -- C ABI of the tiled LU with pairwise pivoting: the LU analogue
// of Algorithm 1 that the paper's conclusion (Section 5) names.  The task
// lists are the QR ones with GETRF / GESSM / TSTRF / SSSSM in place of
// GEQRT / LARFB / TSQRT / SSRFB (same data flow, so the same dependency
// rules and the same persistent scheduler); the solve is the forward
// transformations on the right-hand-side tiles followed by the back
// substitution with U, as one task graph.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/tqr.h"
#include "tqr_api_internal.h"
#include "tqr_engine.h"

using namespace tqr;

namespace {

// mode M_FACTOR: A (m x n) is factored in place.  mode M_APPLY_QT: A holds
// the factors of a square n x n matrix and B (n x nrhs) is overwritten with
// A^-1 B.
int lu_device(int mode, int64_t m, int64_t n, int64_t nrhs, double* A, int64_t lda, int nb, int ib, double* L,
              int32_t* piv, double* B, int64_t ldb, int pair, cudaStream_t st) {
  int cs, occ, smem;
  if (!choose_shape(nb, ib, sizeof(double), &cs, &occ, &smem, pair ? 2 * nb : 0)) return TQR_ERR_UNSUPPORTED;
  const bool solve = mode == M_APPLY_QT;
  Inst I = make_inst(mode, m, n, nb, ib, cs, solve ? static_cast<int>(nrhs) : 0, solve ? 1 : 0);
  I.lu = 1;
  I.pair = pair;
  const WsLayout W = ws_layout(I, sizeof(double), false);
  char* ws = nullptr;
  if (lib_malloc(reinterpret_cast<void**>(&ws), W.bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return TQR_ERR_NOMEM;
  }
  I.A = ws + W.oA;
  I.B = solve ? ws + W.oB : nullptr;
  I.T = L;
  I.piv = piv;
  I.ver = reinterpret_cast<int*>(ws + W.oVer);
  const int sms = device_sms();
  const int mi = static_cast<int>(m), ni = static_cast<int>(n), ri = static_cast<int>(nrhs);
  int status = TQR_OK;
  if (launch_pack<double>(A, lda, mi, ni, static_cast<double*>(I.A), I.p, I.q, nb, sms, st) != cudaSuccess ||
      (solve && launch_pack<double>(B, ldb, mi, ri, static_cast<double*>(I.B), I.p, I.qb, nb, sms, st) != cudaSuccess))
    status = TQR_ERR_CUDA;
  if (status == TQR_OK) status = run_plan<double>(I, ws, W, occ, smem, st);
  if (status == TQR_OK) {
    const cudaError_t e =
        solve ? launch_unpack<double>(static_cast<double*>(I.B), I.p, nb, B, ldb, mi, ri, sms, st)
              : launch_unpack<double>(static_cast<double*>(I.A), I.p, nb, A, lda, mi, ni, sms, st);
    if (e != cudaSuccess) status = TQR_ERR_CUDA;
  }
  cudaFreeAsync(ws, st);
  return status;
}

// Host operands: staged through device copies; synchronizes the stream.
int lu_staged(int mode, int64_t m, int64_t n, int64_t nrhs, double* A, int64_t lda, int nb, int ib, double* L,
              int32_t* piv, double* B, int64_t ldb, int pair, cudaStream_t st) {
  const bool solve = mode == M_APPLY_QT;
  const size_t lbytes = tqr_t_size(m, n, nb, ib), pbytes = tqr_lu_piv_size(m, n, nb);
  double *dA = nullptr, *dL = nullptr, *dB = nullptr;
  int32_t* dP = nullptr;
  if (lib_malloc(reinterpret_cast<void**>(&dA), sizeof(double) * m * n, st) != cudaSuccess ||
      lib_malloc(reinterpret_cast<void**>(&dL), lbytes, st) != cudaSuccess ||
      lib_malloc(reinterpret_cast<void**>(&dP), pbytes, st) != cudaSuccess ||
      (solve && lib_malloc(reinterpret_cast<void**>(&dB), sizeof(double) * m * nrhs, st) != cudaSuccess)) {
    cudaGetLastError();
    if (dA) cudaFreeAsync(dA, st);
    if (dL) cudaFreeAsync(dL, st);
    if (dP) cudaFreeAsync(dP, st);
    return TQR_ERR_NOMEM;
  }
  int status = TQR_OK;
  if (copy_cols(dA, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m, n,
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
    status = TQR_ERR_CUDA;
  if (status == TQR_OK && solve &&
      (cudaMemcpyAsync(dL, L, lbytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
       cudaMemcpyAsync(dP, piv, pbytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
       copy_cols(dB, sizeof(double) * m, B, sizeof(double) * ldb, sizeof(double) * m, nrhs,
                         cudaMemcpyHostToDevice, st) != cudaSuccess))
    status = TQR_ERR_CUDA;
  // slots a pair factorization leaves unused come back as zeros
  if (status == TQR_OK && !solve &&
      (cudaMemsetAsync(dL, 0, lbytes, st) != cudaSuccess || cudaMemsetAsync(dP, 0, pbytes, st) != cudaSuccess))
    status = TQR_ERR_CUDA;
  if (status == TQR_OK) status = lu_device(mode, m, n, nrhs, dA, m, nb, ib, dL, dP, dB, m, pair, st);
  if (status == TQR_OK) {
    cudaError_t e = cudaSuccess;
    if (solve) {
      e = copy_cols(B, sizeof(double) * ldb, dB, sizeof(double) * m, sizeof(double) * m, nrhs,
                            cudaMemcpyDeviceToHost, st);
    } else {
      e = copy_cols(A, sizeof(double) * lda, dA, sizeof(double) * m, sizeof(double) * m, n,
                            cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(L, dL, lbytes, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(piv, dP, pbytes, cudaMemcpyDeviceToHost, st);
    }
    if (e != cudaSuccess) status = TQR_ERR_CUDA;
  }
  cudaFreeAsync(dA, st);
  cudaFreeAsync(dL, st);
  cudaFreeAsync(dP, st);
  if (dB) cudaFreeAsync(dB, st);
  int dev_status = TQR_OK;
  if (read_status(&dev_status, st) != cudaSuccess) return TQR_ERR_CUDA;
  if (status == TQR_OK) status = dev_status;
  return status;
}

}  // namespace

extern "C" {

size_t tqr_lu_piv_size(int64_t m, int64_t n, int nb) {
  if (m < 0 || n < 0 || nb < 1) return 0;
  const int p = static_cast<int>(std::max<int64_t>(1, (m + nb - 1) / nb));
  const int q = static_cast<int>(std::max<int64_t>(1, (n + nb - 1) / nb));
  const int kt = std::min(p, q);
  return sizeof(int32_t) * static_cast<size_t>(piv_offset(p, nb, kt, kt));
}

static int lu_factor_common(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* L, int32_t* piv,
                            int pair, void* stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (m > (1LL << 30) || n > (1LL << 30)) return TQR_ERR_UNSUPPORTED;
  if (lda < std::max<int64_t>(1, m)) return -4;
  const int c = check_tiles(nb, ib, 5, 6);
  if (c) return c;
  if (m == 0 || n == 0) return TQR_OK;
  if (A == nullptr) return -3;
  if (L == nullptr) return -7;
  if (piv == nullptr) return -8;
  const int ka = ptr_kind(A);
  if (ptr_kind(L) != ka) return -7;
  if (ptr_kind(piv) != ka) return -8;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (ka == PTR_DEVICE) return lu_device(M_FACTOR, m, n, 0, A, lda, nb, ib, L, piv, nullptr, 0, pair, st);
  return lu_staged(M_FACTOR, m, n, 0, A, lda, nb, ib, L, piv, nullptr, 0, pair, st);
}

static int lu_solve_common(int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib, const double* L,
                           const int32_t* piv, double* B, int64_t ldb, int pair, void* stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (n > (1LL << 30) || nrhs > (1LL << 30)) return TQR_ERR_UNSUPPORTED;
  if (lda < std::max<int64_t>(1, n)) return -4;
  const int c = check_tiles(nb, ib, 5, 6);
  if (c) return c;
  if (ldb < std::max<int64_t>(1, n)) return -10;
  if (n == 0 || nrhs == 0) return TQR_OK;
  if (A == nullptr) return -3;
  if (L == nullptr) return -7;
  if (piv == nullptr) return -8;
  if (B == nullptr) return -9;
  const int ka = ptr_kind(A);
  if (ptr_kind(L) != ka) return -7;
  if (ptr_kind(piv) != ka) return -8;
  if (ptr_kind(B) != ka) return -9;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* a = const_cast<double*>(A);
  double* l = const_cast<double*>(L);
  int32_t* pv = const_cast<int32_t*>(piv);
  if (ka == PTR_DEVICE) return lu_device(M_APPLY_QT, n, n, nrhs, a, lda, nb, ib, l, pv, B, ldb, pair, st);
  return lu_staged(M_APPLY_QT, n, n, nrhs, a, lda, nb, ib, l, pv, B, ldb, pair, st);
}

int tqr_lu_factor(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* L, int32_t* piv,
                  void* stream) {
  return lu_factor_common(m, n, A, lda, nb, ib, L, piv, 0, stream);
}

int tqr_lu_solve(int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib, const double* L,
                 const int32_t* piv, double* B, int64_t ldb, void* stream) {
  return lu_solve_common(n, nrhs, A, lda, nb, ib, L, piv, B, ldb, 0, stream);
}

int tqr_lu_factor_pairs(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* L, int32_t* piv,
                        void* stream) {
  return lu_factor_common(m, n, A, lda, nb, ib, L, piv, 1, stream);
}

int tqr_lu_solve_pairs(int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib, const double* L,
                       const int32_t* piv, double* B, int64_t ldb, void* stream) {
  return lu_solve_common(n, nrhs, A, lda, nb, ib, L, piv, B, ldb, 1, stream);
}

}  // extern "C"
