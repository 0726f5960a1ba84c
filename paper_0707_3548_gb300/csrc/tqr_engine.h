// tqr_engine.h -- host-side entry points of the device engine (tqr_engine.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "tqr_graph.h"

namespace tqr {

template <typename real>
cudaError_t launch_pack(const double* A, long long lda, int m, int n, real* Ab, int p, int q, int nb, int sms,
                        cudaStream_t st);
template <typename real>
cudaError_t launch_unpack(const real* Ab, int p, int nb, double* A, long long lda, int m, int n, int sms,
                          cudaStream_t st);
// Transposed pack/unpack: X = C^T (mt x nt, X(a, b) = C[b + a*ldc]) to and
// from BDL tiles; identity: the leading ncols columns of I_m in BDL.
template <typename real>
cudaError_t launch_pack_t(const double* C, long long ldc, int mt, int nt, real* Ab, int p, int q, int nb, int sms,
                          cudaStream_t st);
template <typename real>
cudaError_t launch_unpack_t(const real* Ab, int p, int nb, double* C, long long ldc, int mt, int nt, int sms,
                            cudaStream_t st);
template <typename real>
cudaError_t launch_identity(int m, int ncols, real* Ab, int p, int q, int nb, int sms, cudaStream_t st);
// variant: 0 the QR task kernel, 1 the tiled LU's (FP64 only), 2 the one
// with the 2b x b bottom kernels (Inst.pair).
template <typename real>
cudaError_t launch_run(const TaskX* tasks, int ntasks, const Inst* insts, void* ctl, long long limit_ns, int grid,
                       int smem_bytes, cudaStream_t st, int variant = 0);
template <typename real>
cudaError_t occupancy(int smem_bytes, int* blocks_per_sm);

// One matrix of a batch for the batched pack/unpack kernels.
struct PackDesc {
  double* A;      // caller's column-major matrix
  long long lda;
  void* Ab;       // its tiles in Block Data Layout
  int m, n, p, q, nb, pad;
};
// bad (device, count ints, zeroed by the caller; may be null): entry b is
// set to TQR_ERR_NONFINITE when matrix b holds a NaN or an infinity.
template <typename real>
cudaError_t launch_pack_batched(const PackDesc* d, int count, cudaStream_t st, int* bad = nullptr);
template <typename real>
cudaError_t launch_unpack_batched(const PackDesc* d, int count, cudaStream_t st);

// Copies the sticky device status to *status (synchronizing st) and clears it.
cudaError_t read_status(int* status, cudaStream_t st);
// After a task-kernel launch on st: its error record (control block `ctl`)
// into out[0..7] = code, where (1 dependency wait, 2 bulk-copy wait, 3 task
// kind), failing task's kind, k, i, j, s, l -- unless out[0] is already
// nonzero.  out must start zeroed.
cudaError_t launch_fold_error(const void* ctl, const TaskX* tasks, int ntasks, double* out, cudaStream_t st);
size_t ctl_bytes();
// FP64 FMA throughput probe (TFLOP/s).
cudaError_t fp64_peak(double* tflops, cudaStream_t st);
// Points the task kernels' trace at buffer (8 words per task, device memory
// of the current device; nullptr turns the trace off).  Synchronous.
cudaError_t set_trace(void* buffer, long long capacity);

}  // namespace tqr
