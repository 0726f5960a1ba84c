/*
 * tqr_debug.h -- host-only introspection of libtqr's task plans.
 *
 * These calls need no GPU: they build the task list of one launch on the
 * host (the same code path the device launches use) so that tests can check
 * the scheduling rules without running kernels.
 */
#ifndef TQR_DEBUG_H
#define TQR_DEBUG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Builds the ordered task list of one launch.
 *   mode     (arg 1)  0 factor, 1 apply Q^T, 2 apply Q, 3 back substitution,
 *                     4 forward substitution with R^T, 5 apply Q to the
 *                     leading columns of the identity (explicit Q; step k
 *                     skips right-hand-side tile columns < k; flat panel
 *                     or tree); add 16 to modes 0, 1 and 3 for
 *                     the tiled LU's task lists (GETRF / GESSM / TSTRF /
 *                     SSSSM kinds 13-16, D must be 0); add 32 to modes 0-4
 *                     for 2b x b bottoms (pairs of tile rows below the
 *                     diagonal: TSQRT2 / SSRFB2 / SSRFB2_N kinds 17-19 with
 *                     l = the group's row count, D must be 0; with 16 as
 *                     well: the LU's TSTRF2 / SSSSM2, kinds 20-21)
 *   m, n     (args 2, 3), nb, ib (args 4, 5) as for tqr_factor
 *   cs       (arg 6)  slab width (columns) of the column-slab tasks; must
 *                     divide nb
 *   nrhs     (arg 7)  right-hand-side columns (0: none)
 *   trsm     (arg 8)  factor / apply-Q^T mode: append the back substitution
 *   D        (arg 9)  0: Algorithm 1's flat panel; > 0: reduction-tree
 *                     variant with domains of D tile rows
 *   workers  (arg 10) CTAs assumed by the list-scheduling simulation
 *   policy   (arg 11) -1 best of both, 0 paper priorities, 1 bottom level,
 *                     2 bottom-level sort without simulation
 *   out      (arg 12) int32[8 * cap]: per task kind, s, inst, k, i, j, l, 0
 *                     (may be NULL to query the count)
 *   cap      (arg 13) capacity of `out` in tasks
 *   stats    (arg 14) double[6] or NULL: chosen makespan, other makespan,
 *                     policy, edges, critical path, total work (seconds of
 *                     the cost model)
 * Returns the number of tasks (>= 0), or -i for invalid argument i, or
 * -100 if the rules contradict the sequential order (message via
 * tqr_debug_last_error).
 */
int64_t tqr_debug_plan(int mode, int64_t m, int64_t n, int nb, int ib, int cs, int nrhs, int trsm, int D,
                       int workers, int policy, int32_t* out, int64_t cap, double* stats);

/*
 * The version waits and signals the device scheduler derives for one task
 * (kind, k, i, j, s, l as in tqr_debug_plan) of a launch described by
 * (mode, m, n, nb, ib, cs, nrhs, D).  waits: int32[4*3] (counter, count,
 * version), signals: int32[3*2] (counter, count).  Returns
 * nwaits + 16 * nsignals.
 */
/*
 * Critical path and total work (seconds of the scheduler's cost model, FP64,
 * or FP32 with the mode flag 64; 2 CTAs per SM) of the launch described as
 * for tqr_debug_plan, computed in
 * one pass over the sequential task order (the estimate the library uses to
 * choose the tree variant's domain size).  out: double[2].  Returns 0, or -1
 * / -2 for invalid arguments.
 */
int tqr_debug_critical_path(int mode, int64_t m, int64_t n, int nb, int ib, int cs, int nrhs, int trsm, int D,
                            double* out);

int tqr_debug_rules(int mode, int64_t m, int64_t n, int nb, int ib, int cs, int nrhs, int D, const int32_t* task,
                    int32_t* waits, int32_t* signals);

/*
 * Overrides the scheduling of later launches (for tests): policy -1 (best of
 * both, default), 0 (paper priorities) or 1 (bottom level); max_ctas > 0
 * caps the persistent grid (0: no cap).  The result of a factorization does
 * not depend on either.  Returns 0, or -1 / -2 for an invalid argument.
 */
int tqr_debug_set_schedule(int policy, int max_ctas);

/*
 * Tuning overrides for later launches: cs (0: automatic, else 8, 16 or 32)
 * forces the slab width where the shared-memory layout allows it; D (-1:
 * automatic, 0: flat panel, else the domain size in tile rows) replaces the
 * library's choice of reduction tree wherever it makes one (tqr_factor_tree
 * with D = 0, tqr_solve_ls, the server).  Returns 0, or -1 / -2 for an
 * invalid argument.
 */
int tqr_debug_set_shape(int cs, int D);

/*
 * Launches the device scheduler on a task whose input is never produced
 * (a TSQRT whose GEQRT is missing), with the given wait limit in
 * milliseconds, and returns the status the launch reports: TQR_ERR_TIMEOUT
 * when the bounded wait gives up as designed.  Uses the current device.
 */
int tqr_debug_stalled_launch(int64_t limit_ms, void* stream);

/*
 * Kernel timing for benchmarks.  While enabled (enable = 1), every launch of
 * the persistent task kernel is bracketed by CUDA events on its stream.
 * tqr_debug_timing_read synchronizes those events and returns the summed
 * milliseconds and the number of launches since the last read (or since
 * enabling), then clears them.  Returns 0 or TQR_ERR_CUDA.
 */
int tqr_debug_timing(int enable);
int tqr_debug_timing_read(double* ms, int64_t* launches);

/*
 * Measures this GPU's FP64 FMA throughput with a register-resident DFMA loop
 * (every SM, 8 independent chains per thread).  Writes TFLOP/s to *tflops.
 * Returns 0 or TQR_ERR_CUDA.
 */
int tqr_debug_fp64_peak(double* tflops, void* stream);

/*
 * Task trace of later task-kernel launches on the current device: for every
 * ticket t < capacity, thread 0 of the CTA that ran it writes eight uint64
 * words at buffer + 8 t -- global-timer ns when the ticket was taken, when
 * its dependencies were met and when it finished; smid | kind << 16 |
 * inst << 32; k; i; j; s | l << 32.  Tickets are positions in the launch's
 * ordered task list, so concurrent launches overwrite each other's records.
 * buffer: device memory of 64 * capacity bytes owned by the caller, or NULL
 * to stop tracing (capacity is then ignored).  Synchronous.  Returns 0, -1
 * when buffer is not 8-byte aligned device memory, -2 for a negative
 * capacity, or TQR_ERR_CUDA.
 */
int tqr_debug_trace(void* buffer, int64_t capacity);

/*
 * Autotuner table without a GPU (tests of the class map, the lookup and the
 * file format): tqr_debug_autotune_class writes the size class of m x n
 * (ceil(log2 m), ceil(log2 n)); tqr_debug_autotune_put stores (nb, ib, us)
 * for the class of m x n as if tqr_autotune_run had measured it.  Return 0
 * or -3 (invalid output pointer, or nb / ib outside what the kernels take).
 */
int tqr_debug_autotune_class(int64_t m, int64_t n, int* mb, int* nbin);
int tqr_debug_autotune_put(int64_t m, int64_t n, int nb, int ib, double us);

/* Last error message of this thread ("" if none). */
const char* tqr_debug_last_error(void);

/*
 * Description of the server's latest failed request ("" if none): its id,
 * matrix id, shape, class and status, and for a device wait that ran out
 * in a task kernel, whether it was a dependency or a bulk-copy wait and the
 * task (kind, k, i, j, s, l as in tqr_debug_plan) it was running.  Written
 * into buf (len bytes, NUL-terminated, truncated to fit).  Returns 0, -1
 * for a null server or -2 for a null or empty buffer.
 */
struct tqr_server;
int tqr_debug_server_last_failure(struct tqr_server* server, char* buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* TQR_DEBUG_H */
