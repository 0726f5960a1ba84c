// tqr_debug.cpp -- host-only plan introspection (include/tqr_debug.h).
#include "tqr_debug.h"

#include <string>
#include <vector>

#include "tqr.h"
#include "tqr_api_internal.h"
#include "tqr_engine.h"
#include "tqr_plan.h"

using namespace tqr;

extern "C" {

int64_t tqr_debug_plan(int mode, int64_t m, int64_t n, int nb, int ib, int cs, int nrhs, int trsm, int D,
                       int workers, int policy, int32_t* out, int64_t cap, double* stats) {
  const int lu = (mode & 16) ? 1 : 0;
  const int pair = (mode & 32) ? 1 : 0;
  mode &= ~48;
  if (mode < 0 || mode > M_FORM_Q) return -1;
  if (lu && mode != M_FACTOR && mode != M_APPLY_QT && mode != M_TRSM) return -1;
  if (pair && mode == M_FORM_Q) return -1;
  if ((lu || pair) && D > 0) return -9;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (check_tiles(nb, ib, 4, 5) != 0) return check_tiles(nb, ib, 4, 5);
  if (cs < 1 || nb % cs != 0) return -6;
  if (nrhs < 0) return -7;
  if (mode != 0 && nrhs == 0) return -7;
  if (trsm && (nrhs == 0 || m < n || (mode != 0 && mode != 1))) return -8;
  if (D < 0) return -9;
  if (workers < 1) return -10;
  if (policy < -1 || policy > 2) return -11;
  Inst I = make_inst(mode, m, n, nb, ib, cs, nrhs, trsm);
  I.D = D;
  I.lu = lu;
  I.pair = pair;
  if (D > 0) I.vtab = host_vtab(I);
  std::vector<TaskX> seq, ordered;
  seq_tasks(I, 0, seq);
  PlanStats st;
  std::string err;
  std::vector<Inst> insts(1, I);
  const bool ok = seq.empty() || (policy == 2 ? order_bottom_level(insts, seq, 8, 2, workers, ordered, &st, &err)
                                               : order_tasks(insts, seq, workers, 8, 2, policy, ordered, &st, &err));
  if (!ok) {
    set_last_error(err);
    return -100;
  }
  if (out != nullptr) {
    const int64_t cnt = static_cast<int64_t>(ordered.size()) < cap ? static_cast<int64_t>(ordered.size()) : cap;
    for (int64_t a = 0; a < cnt; ++a) {
      const TaskX& t = ordered[a];
      int32_t* o = out + 8 * a;
      o[0] = t.kind; o[1] = t.s; o[2] = t.inst; o[3] = t.k; o[4] = t.i; o[5] = t.j; o[6] = t.l; o[7] = 0;
    }
  }
  if (stats != nullptr) {
    stats[0] = st.makespan_s;
    stats[1] = st.makespan_other;
    stats[2] = st.policy;
    stats[3] = static_cast<double>(st.edges);
    stats[4] = st.critical_path_s;
    stats[5] = st.work_s;
  }
  return static_cast<int64_t>(seq.size());
}

int tqr_debug_critical_path(int mode, int64_t m, int64_t n, int nb, int ib, int cs, int nrhs, int trsm, int D,
                            double* out) {
  const int lu = (mode & 16) ? 1 : 0;
  const int pair = (mode & 32) ? 1 : 0;
  const int esize = (mode & 64) ? 4 : 8;
  mode &= ~112;
  if (mode < 0 || mode > M_FORM_Q || out == nullptr) return -1;
  if (m < 1 || n < 1 || check_tiles(nb, ib, 4, 5) != 0 || cs < 1 || nb % cs != 0) return -2;
  Inst I = make_inst(mode, m, n, nb, ib, cs, nrhs, trsm);
  I.D = D;
  I.lu = lu;
  I.pair = pair;
  if (D > 0) I.vtab = host_vtab(I);
  critical_path_estimate(I, esize, 2, &out[0], &out[1]);
  return 0;
}

int tqr_debug_rules(int mode, int64_t m, int64_t n, int nb, int ib, int cs, int nrhs, int D, const int32_t* task,
                    int32_t* waits, int32_t* signals) {
  const int lu = (mode & 16) ? 1 : 0;
  const int pair = (mode & 32) ? 1 : 0;
  Inst I = make_inst(mode & ~48, m, n, nb, ib, cs, nrhs, 1);
  I.D = D;
  I.lu = lu;
  I.pair = pair;
  if (D > 0) I.vtab = host_vtab(I);
  TaskX t;
  t.kind = task[0]; t.s = task[1]; t.inst = task[2]; t.k = task[3]; t.i = task[4]; t.j = task[5]; t.l = task[6];
  t.pad = 0;
  Wait w[kMaxWaits];
  Signal sg[kMaxSignals];
  int nsig = 0;
  const int nw = task_rules(I, t, w, sg, &nsig);
  for (int a = 0; a < nw; ++a) {
    waits[3 * a] = w[a].ctr; waits[3 * a + 1] = w[a].cnt; waits[3 * a + 2] = w[a].ver;
  }
  for (int a = 0; a < nsig; ++a) {
    signals[2 * a] = sg[a].ctr; signals[2 * a + 1] = sg[a].cnt;
  }
  return nw + 16 * nsig;
}

int tqr_debug_set_schedule(int policy, int max_ctas) {
  if (policy < -1 || policy > 1) return -1;
  if (max_ctas < 0) return -2;
  set_schedule(policy, max_ctas);
  clear_plans();
  return 0;
}

int tqr_debug_set_shape(int cs, int D) {
  if (cs != 0 && cs != 8 && cs != 16 && cs != 32) return -1;
  if (D < -1) return -2;
  set_shape_override(cs, D);
  clear_plans();
  return 0;
}

int tqr_debug_stalled_launch(int64_t limit_ms, void* stream) {
  if (limit_ms < 1) return -1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // a 2 x 1 tile grid whose only task is TSQRT(0, 1): it waits for GEQRT(0),
  // which is not in the list, so its dependency wait must run out
  int cs, occ, smem;
  if (!choose_shape(16, 8, 8, &cs, &occ, &smem)) return TQR_ERR_UNSUPPORTED;
  Inst I = make_inst(M_FACTOR, 32, 16, 16, 8, cs, 0, 0);
  const WsLayout W = ws_layout(I, 8, true);
  char* ws = nullptr;
  if (lib_malloc(reinterpret_cast<void**>(&ws), W.bytes + 256, st) != cudaSuccess) {
    cudaGetLastError();
    return TQR_ERR_NOMEM;
  }
  I.A = ws + W.oA;
  I.B = nullptr;
  I.T = ws + W.oT;
  I.ver = reinterpret_cast<int*>(ws + W.oVer);
  TaskX t;
  t.kind = K_TSQRT; t.s = 0; t.inst = 0; t.k = 0; t.i = 1; t.j = 0; t.l = 0; t.pad = 0;
  TaskX* dt = reinterpret_cast<TaskX*>(ws + W.bytes);
  int status = TQR_OK;
  if (cudaMemsetAsync(ws, 0, W.bytes, st) != cudaSuccess ||
      cudaMemcpyAsync(dt, &t, sizeof(TaskX), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(ws + W.oInst, &I, sizeof(Inst), cudaMemcpyHostToDevice, st) != cudaSuccess)
    status = TQR_ERR_CUDA;
  if (status == TQR_OK &&
      launch_run<double>(dt, 1, reinterpret_cast<const Inst*>(ws + W.oInst), ws + W.oCtl, limit_ms * 1000000LL, 1,
                         smem, st) != cudaSuccess)
    status = TQR_ERR_CUDA;
  cudaFreeAsync(ws, st);
  int dev_status = TQR_OK;
  if (read_status(&dev_status, st) != cudaSuccess) return TQR_ERR_CUDA;
  return status != TQR_OK ? status : dev_status;
}

int tqr_debug_timing(int enable) { return timing_enable(enable); }

int tqr_debug_timing_read(double* ms, int64_t* launches) { return timing_read(ms, launches) ? TQR_ERR_CUDA : 0; }

int tqr_debug_fp64_peak(double* tflops, void* stream) {
  if (tflops == nullptr) return -1;
  return fp64_peak(tflops, static_cast<cudaStream_t>(stream)) == cudaSuccess ? 0 : TQR_ERR_CUDA;
}

int tqr_debug_trace(void* buffer, int64_t capacity) {
  if (buffer != nullptr && capacity < 0) return -2;
  // the kernels write the records: only device memory, 8-byte aligned
  if (buffer != nullptr &&
      (ptr_kind(buffer) != PTR_DEVICE || (reinterpret_cast<uintptr_t>(buffer) & 7) != 0))
    return -1;
  return set_trace(buffer, buffer != nullptr ? capacity : 0) == cudaSuccess ? 0 : TQR_ERR_CUDA;
}

const char* tqr_debug_last_error(void) { return last_error(); }

}  // extern "C"
