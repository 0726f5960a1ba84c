// tqr_ls.h -- one least-squares problem's device state (tqr_ls.cu), shared by
// tqr_solve_ls and the request server.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "tqr.h"
#include "tqr_api_internal.h"
#include "tqr_graph.h"

namespace tqr {

// factor_solve of the FP32 class: A lies outside the range the FP32
// factorization handles (the caller solves in FP64 instead).  Internal only.
constexpr int kLsFp32Range = 1000;
// finish of the FP32 class: every refinement form stagnated (or GMRES used
// up its steps) before maxit -- the caller solves in FP64 instead.  Internal.
constexpr int kLsStalled = 1001;

// ---- few-right-hand-side kernels of the refinement (tqr_lsvec.cu)
constexpr int kMaxVecRhs = 16;
size_t trsv_ctl_ints(int n, int nb);
size_t trsv_smem(int nb, int nrhs, int esize);
bool trsv_fits(int nb, int nrhs, int esize);
// R X = Y (trans false) or R^T X = Y (trans true) with the R of the tiles;
// ctl: trsv_ctl_ints(n, nb) ints of device memory (cleared here); a wait
// that runs out writes TQR_ERR_TIMEOUT to *err_out (may be null).
template <typename real>
cudaError_t launch_trsv(bool trans, const real* tiles, int p, int nb, int n, int nrhs, const double* Y,
                        long long ldy, double* X, long long ldx, int* ctl, long long limit_ns, double* err_out,
                        cudaStream_t st);
// D = Q1^T F (n x nrhs) and U = F - Q1 Y (m x nrhs) with the explicit thin
// Q1 in FP32 tiles; inputs are multiplied by the scale (a power of two)
// before rounding to FP32 and the results divided by it.  part: scratch of
// at most splits_cap * max(m, n) * nrhs floats.
cudaError_t launch_q1t(const float* Q, int p, int nb, int m, int n, int nrhs, const double* F, long long ldf,
                       double fscale, float* part, int splits_cap, double* D, long long ldd, cudaStream_t st);
cudaError_t launch_q1n(const float* Q, int p, int nb, int m, int n, int nrhs, const double* Yv, long long ldy,
                       double yscale, const double* F, long long ldf, float* part, int splits_cap, double* U,
                       long long ldu, cudaStream_t st);
constexpr int kQ1SplitsCap = 64;

struct LsScratch {
  double* part;  // nsplit * m * nrhs partial products
  int nsplit;
  int split_len;
};

struct LsJob {
  int m = 0, n = 0, rhs_cap = 0, nb = 0, ib = 0, prec = 0, esize = 8;
  int cs = 0, occ = 0, smem = 0, grid_cap = 0;
  Inst I = {};
  WsLayout W = {};
  LsScratch sc = {};
  size_t o_part = 0, o_e = 0, o_r = 0, o_f = 0, o_d = 0, o_g = 0, o_h = 0, o_x = 0, o_G = 0, o_nrm = 0, o_acopy = 0;
  // a second right-hand-side tile array, its counters, and room for two
  // instances: two independent graphs of the refinement step in one launch
  size_t o_b2 = 0, o_ver2 = 0, o_inst2 = 0;
  size_t o_tctl = 0;  // control words of the triangular-solve kernel
  size_t o_y = 0;     // n x rhs_cap scratch of the fast preconditioner
  size_t bytes = 0;  // workspace without the FP64 copy of A
  // FP32 class, refinement with Q (augmented / GMRES-IR): the explicit thin
  // Q1 in FP32 tiles, formed once from the factors, with its launch state
  // and the GEMV scratch (allocated on first use, freed by finish)
  char* vws = nullptr;
  size_t vo_ver = 0, vo_inst = 0, vo_ctl = 0, vo_part = 0, vbytes = 0;
  int fast_ok(int nrhs) const;  // the few-right-hand-side kernels apply
  int form_q1(cudaStream_t st);
  void free_q1(cudaStream_t st);
  int trsv(bool trans, const double* Y, long long ldy, double* X, long long ldx, int nrhs, cudaStream_t st);
  char* ws = nullptr;
  double* Acopy = nullptr;
  bool factored = false;
  // the error record of this job's own task-kernel launches (device, 8
  // doubles after the norms: code, where, task kind, k, i, j, s, l), cleared
  // by factor_solve and solve and read by finish; err_host is finish's copy
  double* err_rec() const;
  double err_host[8] = {};

  // sizes for m x n with up to rhs_cap right-hand sides; false if the tile
  // shape is unsupported
  bool init(int m, int n, int rhs_cap, int nb, int ib, int prec, int grid_cap);
  size_t bytes_with_acopy() const;
  void bind(char* base, bool with_acopy);
  // factor A (nrhs = 0: factor only) and with nrhs > 0 solve through it
  int factor_solve(const double* A, long long lda, const double* B, long long ldb, int nrhs, cudaStream_t st);
  int solve(const double* B, long long ldb, int nrhs, cudaStream_t st);
  // backward error, refinement (FP32 class) and the copy of x to X; info
  // (may be null) receives the path, steps and backward error
  int finish(const double* A, long long lda, const double* B, long long ldb, int nrhs, double* X, long long ldx,
             double tol, int maxit, tqr_ls_info* info, cudaStream_t st);
  // [U; V] = M^-1 [F; G] through the factors (augmented-system correction)
  int precond(const double* F, long long ldf, const double* G, long long ldg, double* U, long long ldu, double* V,
              long long ldv, int nrhs, cudaStream_t st);
  int run_mode(int mode, int trsm, int nrhs, cudaStream_t st);
  int pack_rhs(const double* src, long long lds, int rows, int nrhs, cudaStream_t st, void* tiles = nullptr);
  int unpack_rhs(double* dst, long long ldd, int rows, int nrhs, cudaStream_t st, const void* tiles = nullptr);
  // mode_a on the first right-hand-side tiles and mode_b on the second, as
  // one launch (neither appends a triangular solve)
  int run_two(int mode_a, int mode_b, int nrhs, cudaStream_t st);
};

}  // namespace tqr
