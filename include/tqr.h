/*
 * tqr.h -- C ABI of libtqr, a GB300 (sm_103a) tiled Householder QR and
 * least-squares library.
 *
 * Method: the tiled QR factorization of Buttari, Langou, Kurzak and Dongarra,
 * "Parallel Tiled QR Factorization for Multicore Architectures": the matrix is
 * cut into nb x nb tiles held in Block Data Layout (Section 3.4) and factored
 * by the four tile kernels GEQRT, LARFB, TSQRT and SSRFB (Section 3.1) in the
 * order of Algorithm 1, executed out of order over the task dependency DAG
 * (Section 3.3).  The kernels use inner blocking ib: each tile's nb columns
 * are handled as nb/ib blocks with one ib x ib compact-WY factor T_l each.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are column-major with a leading dimension (LAPACK style).
 * - Pointers may be DEVICE pointers (cudaMalloc / PyTorch CUDA tensors) or
 *   HOST pointers (pageable or pinned).  The library asks CUDA which one it
 *   is given.  Device pointers: the call is asynchronous on `stream` and
 *   returns once the work is enqueued.  Host pointers: the library copies
 *   the data to the device, runs, copies results back and synchronizes the
 *   stream before returning.  All pointers of one call must be of one kind.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 * - The caller owns every buffer it passes.  Scratch memory the library needs
 *   is allocated stream-ordered (cudaMallocAsync) and released on the same
 *   stream, unless the *_ws variant is used with a caller-provided workspace.
 * - Return value: 0 on success; -i if argument i (1-based) is invalid, in
 *   which case nothing is enqueued; a positive TQR_ERR_* code otherwise.
 *   Errors never abort the process and never trap the GPU.  A device-side
 *   failure of an asynchronous call (TQR_ERR_TIMEOUT) is reported by
 *   tqr_stream_status().
 * - Supported tile sizes: 8 <= nb <= 256, nb % 8 == 0; ib divides nb and
 *   ib <= 64.
 */
#ifndef TQR_H
#define TQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TQR_OK = 0,
  TQR_ERR_CUDA = 1,        /* a CUDA runtime call failed */
  TQR_ERR_NOMEM = 2,       /* device or pinned memory could not be allocated */
  TQR_ERR_TIMEOUT = 3,     /* a dependency wait in the device scheduler ran out */
  TQR_ERR_RANK = 4,        /* least squares: |r_ii| <= n * eps * max|r_jj| */
  TQR_ERR_NOCONV = 5,      /* least squares: refinement did not reach tol */
  TQR_ERR_BUSY = 6,        /* batch / server: no free slot right now */
  TQR_ERR_UNSUPPORTED = 7, /* valid arguments outside what this build supports */
  TQR_ERR_TOO_LARGE = 8,   /* tqr_factor_noalloc: problem exceeds its static scratch */
  TQR_ERR_NONFINITE = 9    /* an input matrix holds a NaN or an infinity */
};

enum { TQR_PREC_FP64 = 0, TQR_PREC_FP32 = 1 };

/*
 * Version string of the library ("tqr <major>.<minor> sm_103a").
 */
const char* tqr_version(void);

/*
 * Bytes needed for the T array of an m x n factorization with tile nb and
 * inner block ib.  Section 3.1: every GEQRT(k) and every TSQRT(k, i) produces
 * a T_ik; here each is an ib x nb array (block l's ib x ib upper triangular
 * T_l in columns l*ib .. l*ib+ib-1, column-major, leading dimension ib).
 * With p = ceil(m/nb), q = ceil(n/nb), kt = min(p, q), the blocks are stored
 * for k = 0..kt-1 and i = k..p-1 in that order:
 *     offset(i, k) = (k*p - k*(k-1)/2 + (i - k)) * ib * nb  elements.
 * Returns 0 for invalid sizes.
 */
size_t tqr_t_size(int64_t m, int64_t n, int nb, int ib);

/*
 * Bytes of device scratch tqr_factor_ws needs for these sizes (the tile
 * buffer in Block Data Layout, dependency counters and the task list).
 */
size_t tqr_work_size(int64_t m, int64_t n, int nb, int ib);

/*
 * Tiled QR factorization, Algorithm 1 of the paper (Sections 3.1-3.4).
 *   m, n   (args 1, 2)  matrix size, m >= 0, n >= 0
 *   A      (arg 3)      m x n, column-major; on exit R is on and above the
 *                       diagonal, V_kk strictly below the diagonal of each
 *                       diagonal tile and V_ik in every tile below it
 *   lda    (arg 4)      >= max(1, m)
 *   nb, ib (args 5, 6)  tile size and inner block size
 *   T      (arg 7)      tqr_t_size(m, n, nb, ib) bytes of doubles, written
 *   stream (arg 8)
 * The result can only be used with the same nb, ib and T.  Rank-deficient
 * input is factored (zero columns give tau = 0).  The factorization is
 * deterministic: the task order on the GPU does not change a single bit.
 * A NaN or an infinity in A is reported as TQR_ERR_NONFINITE -- by the call
 * itself for host buffers, by tqr_stream_status for device buffers -- and
 * the output is then undefined; the same holds for every factorization
 * entry point below (tree, 2b x b, LU, allocation-free).
 */
int tqr_factor(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib,
               double* T, void* stream);

/*
 * As tqr_factor, with caller-provided device scratch `work` of at least
 * tqr_work_size(m, n, nb, ib) bytes (256-byte aligned) at args 8-9.
 */
int tqr_factor_ws(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib,
                  double* T, void* work, size_t work_bytes, void* stream);

/*
 * Apply Q or Q^T from a tqr_factor result to B (m x nrhs), in place
 * (the DORMQR analogue named in Section 5 of the paper).
 *   trans  (arg 1)  'T': B <- Q^T B (Algorithm 1's order: LARFB on row block
 *                   k, then SSRFB on the pairs (k, i));  'N': B <- Q B
 *                   (the same steps transposed, in reverse order)
 *   m, n   (args 2, 3), nrhs (arg 4) >= 0
 *   A, lda (args 5, 6)  factored matrix from tqr_factor
 *   nb, ib (args 7, 8), T (arg 9) as passed to tqr_factor
 *   B, ldb (args 10, 11) m x nrhs, ldb >= max(1, m)
 * Forming Q explicitly is trans = 'N' applied to the identity.
 */
int tqr_apply_qt(char trans, int64_t m, int64_t n, int64_t nrhs,
                 const double* A, int64_t lda, int nb, int ib, const double* T,
                 double* B, int64_t ldb, void* stream);

/*
 * Reduction-tree variant of the factorization (an extension; the paper's
 * panel is Algorithm 1's flat chain TSQRT(k, k+1), TSQRT(k, k+2), ...).  In
 * step k the rows k..p-1 are cut into domains of D tile rows; each domain is
 * factored flat with its first row as head (GEQRT of the head tile, TSQRT of
 * the head's triangle with every later row of the domain), then the heads'
 * triangles merge by a binary tree of TTQRT kernels (QR of two stacked upper
 * triangles; their reflectors are upper triangular and overwrite the
 * eliminated head's triangle, its lower part keeping that head's GEQRT
 * reflectors).  The panel's critical path drops from p - k tasks to about
 * D + log2((p - k) / D), which is what tall-skinny matrices need.
 *   tqr_t_size_tree: bytes of T for this variant (twice tqr_t_size: the
 *     GEQRT/TSQRT factors in tqr_t_size's layout, then the TTQRT factors of
 *     the eliminated heads in the same layout).
 *   tqr_factor_tree(m, n, A, lda, nb, ib, D, T, stream): as tqr_factor; *D
 *     (arg 7) is the domain size in tile rows, or 0 to let the library choose
 *     it (from a model of the task graph's critical path and work; the flat
 *     panel when no tree is clearly better) -- the chosen value is written
 *     back.  T (arg 8) has tqr_t_size_tree bytes.
 *   tqr_apply_qt_tree(trans, m, n, nrhs, A, lda, nb, ib, D, T, B, ldb,
 *     stream): tqr_apply_qt for factors of tqr_factor_tree with domain size D
 *     (arg 9).
 */
size_t tqr_t_size_tree(int64_t m, int64_t n, int nb, int ib);
int tqr_factor_tree(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, int* D,
                    double* T, void* stream);
int tqr_apply_qt_tree(char trans, int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                      int nb, int ib, int D, const double* T, double* B, int64_t ldb, void* stream);

/*
 * 2b x b bottoms -- Section 3.2 remarks that non-square 2b x b blocks cut the
 * tiled algorithm's extra work from 25 % to 12.5 % (Section 5 repeats it).
 * Algorithm 1 with the tile rows below each diagonal tile taken in pairs
 * (k+1, k+2), (k+3, k+4), ... (the last alone if their count is odd): every
 * TSQRT factors R_kk stacked on a 2b x b block and every SSRFB updates the
 * top tile with a 2b-row bottom, so the T factors' extra work is spread over
 * twice the rows.  Tiles stay b x b in memory (a pair is two storage tiles).
 *   tqr_factor_pairs(m, n, A, lda, nb, ib, T, stream): arguments and errors
 *     as tqr_factor; T has tqr_t_size bytes (the slot of each pair's second
 *     row is unused).  R is that of tqr_factor up to rounding; the
 *     reflectors differ and belong to this variant only.
 *   tqr_apply_qt_pairs(trans, m, n, nrhs, A, lda, nb, ib, T, B, ldb, stream):
 *     tqr_apply_qt for factors of tqr_factor_pairs.
 */
int tqr_factor_pairs(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* T,
                     void* stream);
int tqr_apply_qt_pairs(char trans, int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                       int nb, int ib, const double* T, double* B, int64_t ldb, void* stream);

/*
 * Applying and forming Q -- the DORMQR / DORGQR pair that the paper's
 * conclusion (Section 5) names as direct derivations of the tiled
 * factorization.  Q is the m x m orthogonal factor of a factorization made by
 * tqr_factor (D = 0) or tqr_factor_tree (D = its domain size), given by the
 * factored A (m x n, lda), nb, ib and T exactly as that call left them.
 *
 * tqr_ormqr(side, trans, m, n, A, lda, nb, ib, D, T, mc, nc, C, ldc, stream)
 *   side   (arg 1)   'L': C <- op(Q) C, C is m x nc (mc must equal m)
 *                    'R': C <- C op(Q), C is mc x m (nc must equal m)
 *   trans  (arg 2)   'N': op(Q) = Q, 'T': op(Q) = Q^T
 *   m, n   (args 3, 4), A, lda (5, 6), nb, ib (7, 8): the factorization
 *   D      (arg 9)   0 for tqr_factor, the domain size for tqr_factor_tree
 *   T      (arg 10)  tqr_t_size (D = 0) or tqr_t_size_tree bytes
 *   mc, nc (args 11, 12), C, ldc (13, 14): column-major, ldc >= max(1, mc),
 *                    overwritten with the product
 *   The right side runs as the left-side task graph on C^T: the library packs
 *   C transposed into its tiles and unpacks it back, since
 *   C Q = (Q^T C^T)^T and C Q^T = (Q C^T)^T.
 *
 * tqr_orgqr(m, n, A, lda, nb, ib, D, T, ncols, Q, ldq, stream)
 *   Writes the first ncols (0 <= ncols <= m, arg 9) columns of Q to Q (arg 10,
 *   m x ncols, ldq >= max(1, m), arg 11); ncols = n gives the thin Q of
 *   A = Q R.  Other arguments as for tqr_ormqr (A is arg 3, T arg 8).  Step
 *   k of the reverse accumulation skips the identity's tile columns < k,
 *   which its reflectors (flat or tree) cannot reach -- they touch rows
 *   >= k*nb only -- so the work is that of the factorization's updates, not
 *   of a full m x ncols product.
 *
 * Both calls: A, T, C / Q all on the device (asynchronous on stream) or all
 * on the host (staged through device copies; the call synchronizes).  They
 * return 0, -i for an invalid argument i, TQR_ERR_NOMEM, TQR_ERR_CUDA or a
 * device status (TQR_ERR_TIMEOUT).  m, n, mc, nc above 2^30 give
 * TQR_ERR_UNSUPPORTED; empty operands return 0 at once (n = 0 means Q = I).
 */
int tqr_ormqr(char side, char trans, int64_t m, int64_t n, const double* A, int64_t lda, int nb,
              int ib, int D, const double* T, int64_t mc, int64_t nc, double* C, int64_t ldc,
              void* stream);
int tqr_orgqr(int64_t m, int64_t n, const double* A, int64_t lda, int nb, int ib, int D,
              const double* T, int64_t ncols, double* Q, int64_t ldq, void* stream);

/*
 * Tiled LU with pairwise pivoting -- the LU analogue of Algorithm 1 that the
 * paper's conclusion (Section 5) names.  Algorithm 1's loop nest with
 *   GETRF(k)       partially pivoted LU of tile (k,k)
 *   GESSM(k,j)     tile (k,j) <- L_kk^-1 P_kk tile (k,j)
 *   TSTRF(k,i)     LU of [U_kk; tile (i,k)], pivoting row c of U_kk against
 *                  the rows of tile (i,k) for each column c (pairwise)
 *   SSSSM(k,i,j)   [tile (k,j); tile (i,j)] <- TSTRF(k,i)'s transformations
 * in ib-column blocks (within a block interchanges move whole block rows;
 * blocks apply in sequence).  The result is not P A = L U with one
 * permutation: it is U (upper triangle of A) plus the sequence of
 * transformations, which tqr_lu_solve replays.
 *
 * tqr_lu_piv_size(m, n, nb): bytes of the pivot array (int32, nb per tile
 *   pair (i, k), i >= k).  The L array has tqr_t_size(m, n, nb, ib) bytes.
 * tqr_lu_factor(m, n, A, lda, nb, ib, L, piv, stream)
 *   A (arg 3, m x n, lda >= max(1, m)) is overwritten with U on and above its
 *   diagonal and the multipliers below; L (arg 7) receives, per tile pair and
 *   ib block, the inverse of the block's unit lower triangle (ib x ib,
 *   stored transposed); piv (arg 8) the interchanges: for GETRF tiles the
 *   tile row exchanged with row c, for TSTRF pairs -1 (no exchange) or the
 *   bottom tile's row exchanged with row c of U_kk.  nb, ib (args 5, 6) as
 *   for tqr_factor.  An exact zero pivot leaves its column unscaled; a zero
 *   then remains on U's diagonal (tqr_lu_solve divides by it).
 * tqr_lu_solve(n, nrhs, A, lda, nb, ib, L, piv, B, ldb, stream)
 *   A, L, piv (args 3, 7, 8): the factors of a square n x n matrix from
 *   tqr_lu_factor with the same nb, ib; B (arg 9, n x nrhs, ldb >= max(1, n),
 *   arg 10) is overwritten with A^-1 B: the transformations and the back
 *   substitution with U run as one task graph.
 * All device pointers (asynchronous on stream) or all host pointers (staged,
 * the call synchronizes).  Returns 0, -i for an invalid argument i,
 * TQR_ERR_NOMEM, TQR_ERR_CUDA, TQR_ERR_UNSUPPORTED (sizes above 2^30) or a
 * device status (TQR_ERR_TIMEOUT).
 */
size_t tqr_lu_piv_size(int64_t m, int64_t n, int nb);
/*
 * tqr_lu_factor_pairs / tqr_lu_solve_pairs: the same with 2b x b bottoms (as
 * tqr_factor_pairs): the rows below each diagonal tile are taken in pairs, so
 * each TSTRF pivots row c of U_kk against 2b rows (a pair's interchanges
 * index its 2b rows, 0 .. 2b-1) and each SSSSM updates the top tile with a
 * 2b-row bottom.  Arguments, sizes and errors as tqr_lu_factor /
 * tqr_lu_solve; the factors of one variant are solved by the same variant.
 */
int tqr_lu_factor(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* L,
                  int32_t* piv, void* stream);
int tqr_lu_solve(int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib,
                 const double* L, const int32_t* piv, double* B, int64_t ldb, void* stream);
int tqr_lu_factor_pairs(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* L,
                        int32_t* piv, void* stream);
int tqr_lu_solve_pairs(int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib,
                       const double* L, const int32_t* piv, double* B, int64_t ldb, void* stream);

/*
 * Least squares  min ||A x - b||_2  for full-rank A, m >= n, through the
 * tiled QR: x = R[0:n,0:n]^{-1} (Q^T b)[0:n].  The factorization, Q^T B and
 * the back substitution run as one task graph on the device.
 *   m, n, nrhs (args 1-3)   m >= n >= 1, nrhs >= 1
 *   A, lda     (args 4, 5)  m x n, NOT modified (the library factors a copy)
 *   B, ldb     (args 6, 7)  m x nrhs right-hand sides
 *   X, ldx     (args 8, 9)  n x nrhs solutions, ldx >= n
 *   prec       (arg 10)     TQR_PREC_FP64: plain FP64.  TQR_PREC_FP32: the
 *                           factorization in FP32 (norms and tau in FP64),
 *                           then refinement with FP64 residuals until the
 *                           backward error is <= tol and x has settled (the
 *                           last correction is at most 2^-50 ||x|| or no
 *                           longer halves): first the corrected semi-normal
 *                           equations x += R^-1 R^-T A^T (b - A x) while the
 *                           spread of R's diagonal puts kappa u_fp32 below
 *                           0.01 and each step halves the backward error;
 *                           then Bjorck's refinement of the augmented system
 *                           [I A; A^T 0][r; x] = [b; 0] (while kappa u_fp32
 *                           seems below 0.02 and it keeps converging); then
 *                           GMRES-IR on the same system, left-preconditioned
 *                           by the FP32 factors (Carson, Higham and Pranesh
 *                           2020), while kappa u_fp32 seems below 0.03 and
 *                           each GMRES cycle gets its residual below 0.1.
 *                           A problem none of them finishes -- or
 *                           whose ||A||_F lies outside [2^-40, 2^40] -- is
 *                           solved again in plain FP64 (tqr_ls_last_info
 *                           tells which path gave the result)
 *   tol        (arg 11)     backward-error target for refinement (e.g. 1e-12)
 *   maxit      (arg 12)     refinement iteration limit
 *   iters      (arg 13)     out (may be NULL): refinement steps taken (outer
 *                           steps of every form, FP32 attempt)
 *   berr       (arg 14)     out (may be NULL): final normwise backward error
 *                           max_c ||A^T r_c|| / (||A||_F (||A||_F ||x_c|| + ||b_c||))
 *   nb, ib     (args 15-16) tile and inner block size (0, 0 = library choice)
 *   stream     (arg 17)
 * Tall problems use the reduction-tree variant when the library's model of
 * the task graph predicts a shorter run (see tqr_factor_tree).
 * Synchronizes the stream (the refinement loop needs the backward error on
 * the host).  Norms are taken with power-of-two scaling, so finite entries
 * of any magnitude give finite norms.  Returns TQR_ERR_NONFINITE when A or
 * B holds a NaN or an infinity (they propagate into X), TQR_ERR_RANK for a
 * numerically rank-deficient R and TQR_ERR_NOCONV when the FP32 class
 * reaches maxit with the backward error above tol (X then holds the last
 * iterate; maxit = 0 returns the unrefined FP32 solution this way).
 * Refinement that stagnates before maxit is not an error: the problem is
 * solved again in FP64.  The FP64 class is not refined and never returns
 * TQR_ERR_NOCONV.
 */
int tqr_solve_ls(int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                 const double* B, int64_t ldb, double* X, int64_t ldx, int prec,
                 double tol, int maxit, int* iters, double* berr, int nb, int ib,
                 void* stream);

/*
 * How a least-squares result was reached.  path: the last form that ran --
 *   TQR_LS_PATH_FP64            plain FP64 factorization and solve
 *   TQR_LS_PATH_FP32            FP32 factorization, no refinement step ran
 *   TQR_LS_PATH_FP32_SEMINORMAL corrected semi-normal refinement
 *   TQR_LS_PATH_FP32_AUGMENTED  augmented-system refinement
 *   TQR_LS_PATH_FP32_GMRES      GMRES-IR
 *   TQR_LS_PATH_FP64_FALLBACK   the FP32 class gave up and FP64 solved it
 *                               (fp32_status: TQR_ERR_NOCONV, or
 *                               TQR_ERR_UNSUPPORTED for ||A||_F outside
 *                               FP32's range)
 * iters: outer refinement steps; inner_iters: GMRES steps; berr: the final
 * backward error; berr_fp32: the one the FP32 refinement reached;
 * gmres_res: the relative residual the last GMRES cycle reached (max over
 * right-hand sides; 0 if GMRES did not run); r_spread: max |r_ii| / min |r_ii|
 * of the factor the refinement used (a lower bound on kappa(A) that selects
 * the refinement form).
 * tqr_ls_last_info(&info) returns this for the calling thread's last
 * tqr_solve_ls or tqr_ls_solve (0, or -1 for a NULL pointer).
 */
enum {
  TQR_LS_PATH_FP64 = 0,
  TQR_LS_PATH_FP32 = 1,
  TQR_LS_PATH_FP32_SEMINORMAL = 2,
  TQR_LS_PATH_FP32_AUGMENTED = 3,
  TQR_LS_PATH_FP32_GMRES = 4,
  TQR_LS_PATH_FP64_FALLBACK = 5
};
typedef struct tqr_ls_info {
  int32_t path, iters, inner_iters, fp32_status;
  double berr, berr_fp32, gmres_res, r_spread;
} tqr_ls_info;
int tqr_ls_last_info(tqr_ls_info* info);

/*
 * A least-squares factorization kept resident for repeated right-hand sides
 * (solves with new B skip the factorization: Q^T B and the back
 * substitution, plus refinement for the FP32 class).
 *
 * tqr_ls_factor(m, n, A, lda, prec, nb, ib, rhs_cap, stream, &h)
 *   m >= n >= 1 (args 1, 2); A (arg 3, device, m x n, lda >= m, arg 4) is
 *   copied: the handle keeps an FP64 copy for the refinement residuals and
 *   the backward error, so A may change afterwards; prec (arg 5) as for
 *   tqr_solve_ls; nb, ib (args 6, 7; 0, 0 = library choice); rhs_cap (arg 8)
 *   the most right-hand sides one solve may take.  Device memory: the tiles,
 *   the copy of A and work arrays for rhs_cap columns.  Asynchronous on
 *   stream, except that the FP32 class synchronizes once to check ||A||_F
 *   (outside [2^-40, 2^40] the handle factors in FP64 instead).  Returns
 *   0 and *h, -i, TQR_ERR_NOMEM, TQR_ERR_UNSUPPORTED or TQR_ERR_CUDA.
 * tqr_ls_solve(h, nrhs, B, ldb, X, ldx, tol, maxit, info, stream)
 *   B (device, m x nrhs, 1 <= nrhs <= rhs_cap), X (device, n x nrhs);
 *   tol, maxit and the result codes as tqr_solve_ls; info (may be NULL) as
 *   tqr_ls_info.  An FP32 handle whose refinement cannot finish factors its
 *   copy of A in FP64 once and answers this and every later solve from that
 *   (path TQR_LS_PATH_FP64_FALLBACK).  Synchronizes the stream.
 * tqr_ls_release(h, stream)
 *   frees the handle's device memory stream-ordered on `stream` (give the
 *   stream of its last solve, or a later point); 0 or TQR_ERR_CUDA.
 * One handle serves one thread at a time, on the device that was current
 * when it was made.
 */
typedef struct tqr_ls tqr_ls;
int tqr_ls_factor(int64_t m, int64_t n, const double* A, int64_t lda, int prec, int nb, int ib,
                  int64_t rhs_cap, void* stream, tqr_ls** h);
int tqr_ls_solve(tqr_ls* h, int64_t nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                 double tol, int maxit, tqr_ls_info* info, void* stream);
int tqr_ls_release(tqr_ls* h, void* stream);

/*
 * One matrix of a batch (tqr_batch_submit).
 *   m, n    size (>= 1 each)
 *   A, lda  device pointer, column-major, overwritten as by tqr_factor
 *   T       device pointer, tqr_t_size(m, n, nb, ib) bytes, written
 *   nb, ib  tile sizes; nb = ib = 0 takes tqr_autotune's choice (size T
 *           with tqr_autotune's nb and ib first)
 */
typedef struct tqr_desc {
  int64_t m, n;
  double* A;
  int64_t lda;
  double* T;
  int32_t nb, ib;
} tqr_desc;

/*
 * Tile sizes for one m x n factorization inside a batch (and for the
 * server's requests).  Size classes are ceil(log2 m) x ceil(log2 n).  A class
 * measured by tqr_autotune_run answers with its measured winner; any other
 * class takes the fixed rule nb = 128, ib = 16, except that a matrix smaller
 * than 128 takes the smallest power of two (>= 16) that holds it.  Writes
 * *nb, *ib.  Returns 0 or -i.
 */
int tqr_autotune(int64_t m, int64_t n, int* nb, int* ib);

/*
 * The measured autotuner (the paper's b and inner blocking, Sections 3.1-3.2,
 * chosen per size class by timing them on this GPU).
 *   tqr_autotune_run(m, n, stream): unless the class of m x n is already in
 *     the table, factors batches of copies of one representative matrix of
 *     the class (its geometric middle; enough copies for ~1e11 flops, 8 to
 *     1024, so that the batch runs in the throughput regime of a large
 *     mixed batch) in one persistent launch each, for every candidate nb in
 *     {16, 32, 64, 96, 128, 192, 256} (up to the smallest that holds the
 *     matrix) and ib in {8, 16, 32} dividing nb; keeps the (nb, ib) with the
 *     least device time per matrix (one timed run after one that builds the
 *     plan).  Allocates its matrices from the library's pool and
 *     synchronizes the stream.  Returns 0, -i, TQR_ERR_NOMEM or a batch
 *     status.
 *   tqr_autotune_save(path) / tqr_autotune_load(path): the table as text,
 *     one class per line ("mb nbin nb ib us_per_matrix", '#' comments); load
 *     merges, and rejects a malformed file as a whole (TQR_ERR_UNSUPPORTED,
 *     as for a file that cannot be opened).
 *   tqr_autotune_clear(): empties the table (every class back to the rule).
 *   tqr_autotune_batch(count, ms, ns, stream): tunes for one batch of
 *     shapes (ms[a] x ns[a], a < count): measures every class present with
 *     tqr_autotune_run, then factors synthetic matrices of exactly these
 *     shapes as one batch under five tile policies -- the fixed rule, the
 *     rule with ib 8, the measured per-class table, that table with ib 16,
 *     and the table for matrices up to 512 with the rule above -- and writes
 *     the fastest policy's choice for each of the batch's classes into the
 *     table (the rule is a candidate, so the batch never runs slower than
 *     under the rule, up to timing noise).  Allocates the batch's matrices
 *     from the library's pool; synchronizes.  Returns 0, -i, TQR_ERR_NOMEM
 *     or a batch status.
 */
int tqr_autotune_run(int64_t m, int64_t n, void* stream);
int tqr_autotune_save(const char* path);
int tqr_autotune_load(const char* path);
int tqr_autotune_clear(void);
int tqr_autotune_batch(int count, const int64_t* ms, const int64_t* ns, void* stream);

/*
 * Factor `count` independent matrices in ONE persistent launch whose global
 * task DAG interleaves the tiles of all of them (Algorithm 1 per matrix;
 * tasks ordered by decreasing longest remaining path).  Every descriptor's A
 * and T must be device memory.  The batch's device work is captured in a
 * CUDA graph the first time a batch of these exact shapes is submitted and
 * replayed afterwards.  Asynchronous on `stream`; *ticket identifies the
 * batch for tqr_batch_poll / tqr_batch_wait.  Returns 0, -i for invalid
 * argument i (-2: some descriptor is invalid), TQR_ERR_BUSY if a batch of
 * the same shapes is still running (poll it first), or another TQR_ERR_*.
 * Results are identical to factoring each matrix alone with the same nb, ib.
 */
int tqr_batch_submit(int count, const tqr_desc* descs, uint64_t* ticket, void* stream);

/*
 * tqr_batch_submit with 2b x b bottoms (the paper's non-square blocks, as
 * tqr_factor_pairs): every matrix is factored with its tile rows below the
 * diagonal taken in pairs.  Arguments, asynchrony, tickets and errors as
 * tqr_batch_submit; results (A and the T layout) are identical to
 * tqr_factor_pairs of each matrix alone with the same nb, ib, so Q is
 * applied with tqr_apply_qt_pairs.
 */
int tqr_batch_submit_pairs(int count, const tqr_desc* descs, uint64_t* ticket, void* stream);

/*
 * Non-blocking completion check.  *done = 1 when the batch has finished;
 * then status_per_item (may be NULL, else `count` ints) receives each
 * matrix's status (TQR_ERR_NONFINITE for a matrix holding a NaN or an
 * infinity, the others of the batch unaffected) and the ticket is consumed.
 * Returns the batch status (0, TQR_ERR_TIMEOUT, TQR_ERR_CUDA, or
 * TQR_ERR_NONFINITE if some matrix held one) once done, 0 while running, -1
 * for an unknown ticket.  A finished batch keeps its statuses for its ticket
 * even when a later submission of the same shapes reuses its plan.
 */
int tqr_batch_poll(uint64_t ticket, int* done, int* status_per_item);

/* Blocking form of tqr_batch_poll. */
int tqr_batch_wait(uint64_t ticket, int* status_per_item);

/*
 * Least-squares request server with continuous batching.
 *
 * Requests enter a FIFO queue; `slots` worker threads, each with its own
 * CUDA stream, admit a request as soon as a slot is free and the HBM budget
 * has room, so requests that arrive while others run start at once and their
 * task graphs overlap on the device (every persistent launch of a request is
 * capped at grid_cap CTAs; 0 = min(2 * SMs, 8 * SMs / slots)).  Factorizations stay
 * resident under the caller's matrix id (least recently used first out when
 * the budget is needed): a later request with the same id, size and
 * precision class skips the factorization (Q^T B and the back substitution
 * only, plus refinement for the FP32 class).
 *
 *   tqr_server_create(budget_bytes, slots, grid_cap, &server)
 *   tqr_server_submit(server, matrix_id, m, n, nrhs, A, lda, B, ldb, X, ldx,
 *                     prec, tol, &request)
 *       A (m x n), B (m x nrhs, 1 <= nrhs <= 16) and X (n x nrhs) are device
 *       pointers owned by the caller; A and B must stay unchanged and X
 *       untouched until the request completes.  prec: TQR_PREC_FP64 (plain
 *       FP64) or TQR_PREC_FP32 (FP32 factorization, FP64-residual refinement
 *       to backward error <= tol).  Returns at once.
 *   tqr_server_poll(server, request, &done, &status, &iters, &berr,
 *                   &latency_ms, &reused)   non-blocking; once done the
 *       request is forgotten.  latency_ms counts from submit to completion.
 *       status: that of tqr_solve_ls, or TQR_ERR_NOMEM for a request whose
 *       workspace exceeds the whole budget (refused at admission, not
 *       queued forever), TQR_ERR_UNSUPPORTED for a shape the kernels cannot
 *       take.
 *   tqr_server_wait(...)                     blocking form
 *   tqr_server_wait_info(server, request, &status, &info, &latency_ms,
 *                        &reused)            blocking, with the tqr_ls_info
 *       of the solve.  An FP32-class request whose refinement cannot finish
 *       is answered from an FP64 factorization of the resident copy of A,
 *       which the entry keeps for its later requests (path
 *       TQR_LS_PATH_FP64_FALLBACK; its bytes join the budget's accounting
 *       when it is made, even if that overshoots the budget)
 *   tqr_server_stats(server, out[8])         completed, p50 and p99 latency
 *       (ms) over completed requests, resident+running bytes, requests that
 *       reused a resident factorization, failed, queued, resident entries
 *   tqr_server_destroy(server)               finishes queued requests, frees
 * Every call returns 0 or -i for invalid argument i.
 */
typedef struct tqr_server tqr_server;
int tqr_server_create(size_t hbm_budget_bytes, int slots, int grid_cap, tqr_server** out);
int tqr_server_submit(tqr_server* server, uint64_t matrix_id, int64_t m, int64_t n, int64_t nrhs,
                      const double* A, int64_t lda, const double* B, int64_t ldb, double* X,
                      int64_t ldx, int prec, double tol, uint64_t* request);
int tqr_server_poll(tqr_server* server, uint64_t request, int* done, int* status, int* iters,
                    double* berr, double* latency_ms, int* reused);
int tqr_server_wait(tqr_server* server, uint64_t request, int* status, int* iters, double* berr,
                    double* latency_ms, int* reused);
int tqr_server_wait_info(tqr_server* server, uint64_t request, int* status, tqr_ls_info* info,
                         double* latency_ms, int* reused);
int tqr_server_stats(tqr_server* server, double* out);
int tqr_server_destroy(tqr_server* server);

/*
 * tqr_factor without any memory allocation.  (The paper has no counterpart:
 * this is a deployment variant of Algorithm 1.)
 *
 * Some callers cannot allocate device memory at the point where they need a
 * factorization: a process whose device memory has all been handed to another
 * allocator up front (a framework's caching allocator or a serving process
 * that reserves HBM at start-up), or latency-critical code that may not risk
 * an allocation's delay or failure.  This entry point allocates nothing: no
 * cudaMalloc, cudaMallocAsync, cudaFree or other allocating routine, on the
 * device or on the host.  Its scratch -- the Block Data Layout tiles, the
 * dependency counters, the task list and the control words -- lives in one
 * file-scope static device array of about 31 MiB that every GPU which loads
 * libtqr holds until the process exits.
 *
 * Arguments, result and T layout are those of tqr_factor; A and T must be
 * device pointers (host buffers would need staging memory; -3 / -7).
 * Limits: the zero-padded matrix may hold at most TQR_NOALLOC_MAX_TILE_ELEMS
 * doubles (ceil(m/nb) * ceil(n/nb) * nb^2, e.g. 1536 x 2048 with nb = 128),
 * at most TQR_NOALLOC_MAX_COUNTERS slab counters and TQR_NOALLOC_MAX_TASKS
 * tasks; larger problems return TQR_ERR_TOO_LARGE and enqueue nothing.
 * Tasks run in Algorithm 1's sequential order (no schedule simulation); the
 * result is bit-identical to tqr_factor's.  The GPU work of a call reads no
 * host memory: the instance descriptor travels as a kernel parameter and a
 * set-up kernel writes the task list into the array.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call, on every stream, shares the one
 * array per device and it keeps the previous call's contents: the call
 * clears the counters and control words it needs zeroed and overwrites the
 * tiles.  Calls whose GPU work overlaps (on different streams, or from
 * different host threads) race on the array and give undefined results;
 * serialize them, e.g. on one stream.  Asynchronous on `stream`; device-side
 * wait timeouts are reported by tqr_stream_status().
 */
#define TQR_NOALLOC_MAX_TILE_ELEMS (3 * 1024 * 1024)
#define TQR_NOALLOC_MAX_COUNTERS (1024 * 1024)
#define TQR_NOALLOC_MAX_TASKS 65536
int tqr_factor_noalloc(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib,
                       double* T, void* stream);

/*
 * Device status of the asynchronous calls made on `stream`: synchronizes the
 * stream and returns TQR_OK, TQR_ERR_NONFINITE (an input matrix held a NaN
 * or an infinity), TQR_ERR_TIMEOUT (a scheduler wait ran out; the
 * affected output is undefined), TQR_ERR_UNSUPPORTED (a launch met a task
 * kind its kernel does not implement; output undefined) or TQR_ERR_CUDA.
 * Clears the recorded status.
 */
int tqr_stream_status(void* stream);

/*
 * Workspaces and staging buffers of the calls come from a stream-ordered pool
 * per device that keeps freed memory for the next call (so calls do not map
 * fresh device memory each time).  tqr_release_memory() synchronizes the
 * devices the library used and returns that cached memory to the driver.
 * Returns 0 or TQR_ERR_CUDA.
 */
int tqr_release_memory(void);

/*
 * Dependency-wait limit of the device scheduler in milliseconds (default
 * 20000, or TQR_WAIT_LIMIT_MS from the environment when the library loads).
 * A wait that exceeds it makes every CTA of that launch stop and the call
 * report TQR_ERR_TIMEOUT.  Returns the previous value.
 */
int64_t tqr_set_wait_limit_ms(int64_t ms);

#ifdef __cplusplus
}
#endif

#endif /* TQR_H */
