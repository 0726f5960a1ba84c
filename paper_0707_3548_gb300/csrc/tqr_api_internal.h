// tqr_api_internal.h -- helpers shared by the C ABI translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <memory>
#include <string>

#include "tqr_graph.h"

namespace tqr {

enum { PTR_NULL = 0, PTR_HOST = 1, PTR_DEVICE = 2 };

struct WsLayout {
  size_t oA, oB, oT, oVtab, oVer, oInst, oCtl, bytes;
};

void set_last_error(const std::string& s);
const char* last_error();
int device_sms();
long long wait_limit_ns();
// rows: the tallest operand of the launch (0: nb; 2 nb for 2b x b bottoms).
bool choose_shape(int nb, int ib, int esize, int* cs, int* ctas_per_sm, int* smem, int rows = 0);
Inst make_inst(int mode, int64_t m, int64_t n, int nb, int ib, int cs, int nrhs, int trsm);
WsLayout ws_layout(const Inst& I, int esize, bool with_t);
// grid_cap > 0 limits the persistent grid (concurrent launches share SMs).
// err_out (device, 8 doubles, zeroed by the caller) receives the launch's
// own error record (launch_fold_error), independent of other launches.
template <typename real>
int run_plan(const Inst& I, char* ws, const WsLayout& W, int ctas_per_sm, int smem, cudaStream_t st,
             int grid_cap = 0, double* err_out = nullptr);
// Several instances' task graphs in one persistent launch.  insts[a].ver
// must be disjoint counter regions (zeroed here), d_insts device room for
// `count` instances, d_ctl the launch's control block (ctl_bytes()).  The
// host array's Inst.vtab may be a device pointer (the host copy is rebuilt).
template <typename real>
int run_plan_multi(const Inst* insts, int count, Inst* d_insts, void* d_ctl, int ctas_per_sm, int smem,
                   cudaStream_t st, int grid_cap = 0, double* err_out = nullptr);
// Stream-ordered allocation from the library's pool (keeps freed memory).
cudaError_t lib_malloc(void** p, size_t bytes, cudaStream_t st);
int release_memory();
// Column-major matrix copy (cudaMemcpy2DAsync arguments): one flat copy when
// both sides are contiguous -- a 2-D copy of many columns is much slower.
cudaError_t copy_cols(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t height,
                      cudaMemcpyKind kind, cudaStream_t st);
int ptr_kind(const void* p);
int check_tiles(int nb, int ib, int arg_nb, int arg_ib);
void clear_plans();
void autotune(int64_t m, int64_t n, int* nb, int* ib);
// The measured autotuner's table (tqr_tune.cu): true and (nb, ib) if the
// size class of m x n has been tuned.
bool tune_lookup(int64_t m, int64_t n, int* nb, int* ib);
// Host copy of the tree variant's prefix table for planning (Inst.D > 0).
const int32_t* host_vtab(const Inst& I);
// Tree variant: chosen domain size (0 = flat) and the device table upload.
int choose_domain(int64_t m, int64_t n, int nb, int ib, int esize);
int upload_vtab(Inst& I, char* ws, const WsLayout& W, cudaStream_t st);
void set_schedule(int policy, int max_ctas);
void set_shape_override(int cs, int D);
int timing_enable(int on);
int timing_read(double* ms, int64_t* launches);

}  // namespace tqr
