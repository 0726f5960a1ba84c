// tqr_engine.cu -- device side of libtqr: the tile kernels of the tiled QR
// (Section 3.1 of Buttari, Langou, Kurzak, Dongarra), the persistent task
// scheduler that runs them over the tile DAG (Section 3.3), and the Block
// Data Layout pack/unpack kernels (Section 3.4).
//
// One CTA executes one task at a time.  Tasks come from a list ordered by
// priority; a CTA takes the next task with one atomic ticket, waits (bounded)
// until the version counters of the task's operands say its inputs are final,
// runs the tile kernel in shared memory and then bumps the counters of what it
// wrote.  Since tickets are handed out in list order and the list is a
// topological order of the DAG, the oldest unfinished task always has its
// inputs ready, so the scheme cannot deadlock and needs no co-residency.
//
// Arithmetic: FP64 tiles use DFMA (the FP64 tensor path measured slower on
// this part); FP32 tiles compute in FP32 while column norms, beta and tau are
// computed in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tqr_graph.h"
#include "tqr_engine.h"

namespace tqr {

// ---------------------------------------------------------------- primitives
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// 1-D bulk copy (TMA engine) global -> shared, completing on an mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <typename real>
__device__ __forceinline__ real ldg_cg(const real* p) {
  return __ldcg(p);
}

template <typename real>
__device__ __forceinline__ real warp_sum(real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

template <typename real>
__device__ __forceinline__ unsigned long long abs_bits(real x);
template <>
__device__ __forceinline__ unsigned long long abs_bits<double>(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}
template <>
__device__ __forceinline__ unsigned long long abs_bits<float>(float x) {
  return static_cast<unsigned long long>(__double_as_longlong(static_cast<double>(x))) &
         0x7fffffffffffffffull;
}

// max |x| over x[0..len) across the warp, exact (the ordering of IEEE
// magnitudes is the ordering of their bit patterns, NaN above infinity).
__device__ __forceinline__ double warp_amax(const double* x, int len, int lane) {
  unsigned long long mx = 0;
  for (int r = lane; r < len; r += 32) {
    const unsigned long long b = abs_bits(x[r]);
    mx = b > mx ? b : mx;
  }
  mx = warp_max_u64(mx);
  return __longlong_as_double(static_cast<long long>(mx));
}

// ---------------------------------------------------------------- context
struct Ctl {
  int next;       // next ticket
  int error;      // 0, or TQR_ERR_TIMEOUT
  int err_task;   // task index whose wait ran out
  int err_where;  // 1: dependency wait, 2: bulk-copy wait, 3: task kind not in this kernel
};

__device__ int g_status;  // sticky device status of asynchronous launches

// Task trace (a debugging aid, off unless a buffer is set): thread 0 of each
// CTA writes, for every ticket t < g_trace_cap, eight words at
// g_trace + 8 t: the global-timer ns when the ticket was taken, when its
// dependencies were met and when the task finished; smid | kind << 16 |
// inst << 32; k; i; j; s | l << 32.
__device__ unsigned long long* g_trace;
__device__ long long g_trace_cap;

__device__ __forceinline__ void trace_begin(int t, unsigned long long t_ticket, const TaskX& x) {
  unsigned long long* tr = g_trace;
  if (tr == nullptr || t >= g_trace_cap) return;
  unsigned smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  unsigned long long* r = tr + 8LL * t;
  r[0] = t_ticket;
  r[1] = gtimer();
  r[3] = static_cast<unsigned long long>(smid) | (static_cast<unsigned long long>(x.kind & 0xffff) << 16) |
         (static_cast<unsigned long long>(static_cast<unsigned>(x.inst)) << 32);
  r[4] = static_cast<unsigned long long>(x.k);
  r[5] = static_cast<unsigned long long>(x.i);
  r[6] = static_cast<unsigned long long>(x.j);
  r[7] = static_cast<unsigned long long>(static_cast<unsigned>(x.s)) |
         (static_cast<unsigned long long>(static_cast<unsigned>(x.l)) << 32);
}

__device__ __forceinline__ void trace_end(int t) {
  unsigned long long* tr = g_trace;
  if (tr == nullptr || t >= g_trace_cap) return;
  tr[8LL * t + 2] = gtimer();
}

template <typename real>
struct Ctx {
  real *P, *P2, *T, *S, *Top, *W, *Rb, *Part;  // P2: nullptr when the layout has none
  real *TopS, *Tst;                              // FP32 update staging, or nullptr
  double* red;       // reduction scratch (>= 2*kThreads + 160 doubles)
  uint32_t bar;
  uint32_t phase;
  int nb, ib, cs;
  int ldP, ldT, ldS;
  Ctl* ctl;
  long long limit_ns;
  int task;
};

template <typename real>
__device__ void set_error(Ctx<real>& cx, int where) {
  if (atomicCAS(&cx.ctl->error, 0, 3 /* TQR_ERR_TIMEOUT */) == 0) {
    cx.ctl->err_task = cx.task;
    cx.ctl->err_where = where;
  }
  atomicCAS(&g_status, 0, 3);
}

// A task kind this kernel does not implement (a plan built for another
// kernel variant): stop every CTA and report TQR_ERR_UNSUPPORTED.
template <typename real>
__device__ void fail_kind(Ctx<real>& cx) {
  if (threadIdx.x == 0) {
    if (atomicCAS(&cx.ctl->error, 0, 7 /* TQR_ERR_UNSUPPORTED */) == 0) {
      cx.ctl->err_task = cx.task;
      cx.ctl->err_where = 3;
    }
    atomicCAS(&g_status, 0, 7);
  }
}

// Wait for the current bulk-copy phase; bounded by the wait limit.
template <typename real>
__device__ void bulk_wait(Ctx<real>& cx) {
  if (!mbar_try_wait(cx.bar, cx.phase)) {
    const unsigned long long t0 = gtimer();
    int it = 0;
    while (!mbar_try_wait(cx.bar, cx.phase)) {
      if ((++it & 63) == 0) {
        if (ld_relaxed(&cx.ctl->error) != 0) break;
        if ((long long)(gtimer() - t0) > cx.limit_ns) {
          set_error(cx, 2);
          break;
        }
      }
    }
  }
  cx.phase ^= 1u;
}

// Copy ncols full columns (rows elements each, contiguous in global memory
// with stride gld) into shared memory (stride sld) with the bulk-copy engine.
// rows * sizeof(real) and every address must be 16-byte multiples.
template <typename real>
__device__ void bulk_cols(Ctx<real>& cx, real* dst, int sld, const real* src, long long gld, int rows,
                          int ncols) {
  const uint32_t bytes = static_cast<uint32_t>(rows) * sizeof(real);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    if (lane == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(cx.bar, bytes * ncols);
    }
    __syncwarp();
    for (int c = lane; c < ncols; c += 32)
      bulk_g2s(smem_u32(dst + c * sld), src + c * gld, bytes, cx.bar);
  }
  bulk_wait(cx);
}

// Pieces of one bulk phase, issued by warp 0: bulk_expect (lane 0 announces
// the phase's total bytes), __syncwarp, then bulk_issue_cols per column set.
template <typename real>
__device__ __forceinline__ void bulk_expect(Ctx<real>& cx, uint32_t bytes) {
  if (threadIdx.x == 0) {
    fence_proxy_async();
    mbar_arrive_expect_tx(cx.bar, bytes);
  }
}

template <typename real>
__device__ __forceinline__ void bulk_issue_cols(Ctx<real>& cx, real* dst, int sld, const real* src, long long gld,
                                                int rows, int ncols) {
  const uint32_t b = static_cast<uint32_t>(rows) * sizeof(real);
  for (int c = threadIdx.x; c < ncols; c += 32) bulk_g2s(smem_u32(dst + c * sld), src + c * gld, b, cx.bar);
}

// Asynchronous form for warp 0 only: one bulk phase that fills two column
// sets (n1 columns of r1 rows, then n2 of r2; n2 may be 0).  Completes at the
// next bulk_wait of every thread; nothing else may use the barrier before.
template <typename real>
__device__ void bulk_cols2_issue(Ctx<real>& cx, real* d1, int sld1, const real* s1, long long gld1, int r1, int n1,
                                 real* d2, int sld2, const real* s2, long long gld2, int r2, int n2) {
  const int lane = threadIdx.x;
  const uint32_t b1 = static_cast<uint32_t>(r1) * sizeof(real), b2 = static_cast<uint32_t>(r2) * sizeof(real);
  if (lane == 0) {
    fence_proxy_async();
    mbar_arrive_expect_tx(cx.bar, b1 * n1 + b2 * n2);
  }
  __syncwarp();
  for (int c = lane; c < n1; c += 32) bulk_g2s(smem_u32(d1 + c * sld1), s1 + c * gld1, b1, cx.bar);
  for (int c = lane; c < n2; c += 32) bulk_g2s(smem_u32(d2 + c * sld2), s2 + c * gld2, b2, cx.bar);
}

// Plain strided copies (L2 only; data may come from other SMs).
template <typename real>
__device__ void load_block(real* dst, int sld, const real* src, long long gld, int rows, int ncols) {
  for (int e = threadIdx.x; e < rows * ncols; e += kThreads) {
    int r = e % rows, c = e / rows;
    dst[r + c * sld] = ldg_cg(src + r + c * gld);
  }
}

template <typename real>
__device__ void store_block(real* dst, long long gld, const real* src, int sld, int rows, int ncols) {
  for (int e = threadIdx.x; e < rows * ncols; e += kThreads) {
    int r = e % rows, c = e / rows;
    dst[r + c * gld] = src[r + c * sld];
  }
}

// ---------------------------------------------------------------- tile ops
// One block reflector applied to a column slab (Section 3.1, DLARFB/DSSRFB
// with compact WY):
//   W    = L^T Top + V^T S          (L = identity when L == nullptr)
//   W    = T^T W (trans) or T W
//   Top -= L W,   S -= V W
// V is nv x ib (ldv), L the unit lower ib x ib block (read below its
// diagonal only), Top ib x w (ldt), S nv x w (lds), T ib x ib (ldT).
template <typename real>
__device__ void apply_block(const real* __restrict__ V, int ldv, int nv, const real* __restrict__ L, int ldl,
                            real* Top, int ldt, real* S, int lds, const real* __restrict__ Tm, int ldT,
                            int ib, int w, real* W, bool trans) {
  const int tid = threadIdx.x;
  const int nout = ib * w;
  // Phase 1: W(r,c) = Top(r,c) + sum_{t>r} L(t,r) Top(t,c) + sum_t V(t,r) S(t,c).
  // Each output is one FMA chain seeded with Top(r,c); a thread carries two
  // outputs (o and o + kThreads) for instruction-level parallelism, so no
  // FP64 instruction is spent beyond the multiply-adds themselves.
  for (int o = tid; o < nout; o += 2 * kThreads) {
    const int o2 = o + kThreads;
    const bool two = o2 < nout;
    const int r1 = o % ib, c1 = o / ib;
    const int r2 = two ? o2 % ib : r1, c2 = two ? o2 / ib : c1;
    const real* v1 = V + r1 * ldv;
    const real* v2 = V + r2 * ldv;
    const real* s1 = S + c1 * lds;
    const real* s2 = S + c2 * lds;
    real a1 = Top[r1 + c1 * ldt], a2 = Top[r2 + c2 * ldt];
    if (L != nullptr) {
      for (int t = r1 + 1; t < ib; ++t) a1 = fma(L[t + r1 * ldl], Top[t + c1 * ldt], a1);
      for (int t = r2 + 1; t < ib; ++t) a2 = fma(L[t + r2 * ldl], Top[t + c2 * ldt], a2);
    }
    if (two) {
#pragma unroll 4
      for (int t = 0; t < nv; ++t) {
        a1 = fma(v1[t], s1[t], a1);
        a2 = fma(v2[t], s2[t], a2);
      }
      W[o2] = a2;
    } else {
#pragma unroll 4
      for (int t = 0; t < nv; ++t) a1 = fma(v1[t], s1[t], a1);
    }
    W[o] = a1;
  }
  __syncthreads();
  // Phase 2: W = T^T W (trans) or T W, T upper triangular.
  real tmp[kMaxOutPerThread];
  {
    int cnt = 0;
    for (int o = tid; o < nout; o += kThreads, ++cnt) {
      const int r = o % ib, c = o / ib;
      const real* wc = W + c * ib;
      real a;
      if (trans) {
        a = Tm[r * ldT] * wc[0];
        for (int s = 1; s <= r; ++s) a = fma(Tm[s + r * ldT], wc[s], a);
      } else {
        a = Tm[r + r * ldT] * wc[r];
        for (int s = r + 1; s < ib; ++s) a = fma(Tm[r + s * ldT], wc[s], a);
      }
      tmp[cnt] = a;
    }
  }
  __syncthreads();
  {
    int cnt = 0;
    for (int o = tid; o < nout; o += kThreads, ++cnt) W[o] = tmp[cnt];
  }
  __syncthreads();
  // Phase 3: Top -= L W (unit lower), S -= V W; single FMA chains seeded with
  // the old value, two outputs per thread.
  for (int o = tid; o < nout; o += kThreads) {
    const int r = o % ib, c = o / ib;
    const real* wc = W + c * ib;
    real a = Top[r + c * ldt] - wc[r];
    if (L != nullptr)
      for (int t = 0; t < r; ++t) a = fma(-L[r + t * ldl], wc[t], a);
    Top[r + c * ldt] = a;
  }
  const int nS = nv * w;
  for (int o = tid; o < nS; o += 2 * kThreads) {
    const int o2 = o + kThreads;
    const bool two = o2 < nS;
    const int t1 = o % nv, c1 = o / nv;
    const int t2 = two ? o2 % nv : t1, c2 = two ? o2 / nv : c1;
    const real* w1 = W + c1 * ib;
    const real* w2 = W + c2 * ib;
    real a1 = S[t1 + c1 * lds], a2 = S[t2 + c2 * lds];
    if (two) {
#pragma unroll 4
      for (int r = 0; r < ib; ++r) {
        a1 = fma(-V[t1 + r * ldv], w1[r], a1);
        a2 = fma(-V[t2 + r * ldv], w2[r], a2);
      }
      S[t2 + c2 * lds] = a2;
    } else {
#pragma unroll 4
      for (int r = 0; r < ib; ++r) a1 = fma(-V[t1 + r * ldv], w1[r], a1);
    }
    S[t1 + c1 * lds] = a1;
  }
  __syncthreads();
}

// FP32 form of apply_block with 4 x 4 register micro-tiles (the FP32 pipe is
// ~58x the FP64 one, so here shared-memory traffic, not arithmetic, is the
// limit).  Requires ib, w, nv multiples of 4, leading dimensions multiples of
// 4, 16-byte aligned V, S and ib (w + 4) <= 17 kThreads (checked by the
// caller).
//   Phase 1: W = Top + L^T Top + V^T S.  The (ib/4) x (w/4) micro-tiles are
//            split over the rows of V and S (split-K); each thread writes its
//            16 partial sums to Part, then every output sums its partials in
//            a fixed order (deterministic).
//   Phase 3: S -= V W with one 4 x 4 micro-tile per thread per pass.
// Partial sums sit at stride 17 (one bank per lane when a warp stores them),
// and T W goes row-major (ld w + 4) into the partial-sum area, so phase 3
// reads four of its columns with one 16-byte load.
__device__ void apply_block_f32(const float* __restrict__ V, int ldv, int nv, const float* __restrict__ L, int ldl,
                                float* Top, int ldt, float* S, int lds, const float* __restrict__ Tm, int ldT,
                                int ib, int w, float* W, float* Part, bool trans) {
  const int tid = threadIdx.x;
  const int nout = ib * w;
  const int rt = ib / 4, MT = rt * (w / 4);
  const int KS = kThreads / MT;
  const int chunk = ((nv + 4 * KS - 1) / (4 * KS)) * 4;
  {
    const int tile = tid % MT, ks = tid / MT;
    if (ks < KS) {
      const int r0 = 4 * (tile % rt), c0 = 4 * (tile / rt);
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
      const int t1 = min(nv, (ks + 1) * chunk);
      for (int t = ks * chunk; t < t1; t += 4) {
        float4 vq[4], sq[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) vq[i] = *reinterpret_cast<const float4*>(V + t + (r0 + i) * ldv);
#pragma unroll
        for (int j = 0; j < 4; ++j) sq[j] = *reinterpret_cast<const float4*>(S + t + (c0 + j) * lds);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j] = fmaf(vq[i].x, sq[j].x, acc[i][j]);
            acc[i][j] = fmaf(vq[i].y, sq[j].y, acc[i][j]);
            acc[i][j] = fmaf(vq[i].z, sq[j].z, acc[i][j]);
            acc[i][j] = fmaf(vq[i].w, sq[j].w, acc[i][j]);
          }
      }
      float* pp = Part + (ks * MT + tile) * 17;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) pp[i * 4 + j] = acc[i][j];
    }
  }
  __syncthreads();
  for (int o = tid; o < nout; o += kThreads) {
    const int r = o % ib, c = o / ib;
    const int tile = (r / 4) + (c / 4) * rt;
    float a = Top[r + c * ldt];
    if (L != nullptr)
      for (int t = r + 1; t < ib; ++t) a = fmaf(L[t + r * ldl], Top[t + c * ldt], a);
    for (int ks = 0; ks < KS; ++ks) a += Part[(ks * MT + tile) * 17 + (r % 4) * 4 + (c % 4)];
    W[o] = a;
  }
  __syncthreads();
  // T W (or T^T W), row-major with ld w + 4, into the partial-sum area (free
  // once W is summed): no in-place rewrite, one barrier less
  const int ldw = w + 4;
  float* W2 = Part;
  for (int o = tid; o < nout; o += kThreads) {
    const int r = o % ib, c = o / ib;
    const float* wc = W + c * ib;
    float a;
    if (trans) {
      a = Tm[r * ldT] * wc[0];
      for (int q = 1; q <= r; ++q) a = fmaf(Tm[q + r * ldT], wc[q], a);
    } else {
      a = Tm[r + r * ldT] * wc[r];
      for (int q = r + 1; q < ib; ++q) a = fmaf(Tm[r + q * ldT], wc[q], a);
    }
    W2[c + r * ldw] = a;
  }
  __syncthreads();
  for (int o = tid; o < nout; o += kThreads) {
    const int r = o % ib, c = o / ib;
    float a = Top[r + c * ldt] - W2[c + r * ldw];
    if (L != nullptr)
      for (int t = 0; t < r; ++t) a = fmaf(-L[r + t * ldl], W2[c + t * ldw], a);
    Top[r + c * ldt] = a;
  }
  const int ntile = (nv / 4) * (w / 4);
  for (int tile = tid; tile < ntile; tile += kThreads) {
    const int t0 = 4 * (tile % (nv / 4)), c0 = 4 * (tile / (nv / 4));
    float4 acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = *reinterpret_cast<const float4*>(S + t0 + (c0 + j) * lds);
    for (int r = 0; r < ib; ++r) {
      const float4 vq = *reinterpret_cast<const float4*>(V + t0 + r * ldv);
      const float4 wq = *reinterpret_cast<const float4*>(W2 + c0 + r * ldw);
      const float wv[4] = {wq.x, wq.y, wq.z, wq.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[j].x = fmaf(-vq.x, wv[j], acc[j].x);
        acc[j].y = fmaf(-vq.y, wv[j], acc[j].y);
        acc[j].z = fmaf(-vq.z, wv[j], acc[j].z);
        acc[j].w = fmaf(-vq.w, wv[j], acc[j].w);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) *reinterpret_cast<float4*>(S + t0 + (c0 + j) * lds) = acc[j];
  }
  __syncthreads();
}

// Dispatch: the register-blocked FP32 form when the shapes allow it.
template <typename real>
__device__ __forceinline__ void apply_any(const real* V, int ldv, int nv, const real* L, int ldl, real* Top, int ldt,
                                          real* S, int lds, const real* Tm, int ldT, int ib, int w, real* W,
                                          real* Part, bool trans) {
  if constexpr (sizeof(real) == 4) {
    const bool ok = (ib % 4 == 0) && (w % 4 == 0) && (nv % 4 == 0) && (ldv % 4 == 0) && (lds % 4 == 0) &&
                    ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(S)) & 15) == 0 &&
                    (ib / 4) * (w / 4) <= kThreads && ib * (w + 4) <= kThreads * 17;
    if (ok) {
      apply_block_f32(V, ldv, nv, L, ldl, Top, ldt, S, lds, Tm, ldT, ib, w, W, Part, trans);
      return;
    }
  }
  apply_block<real>(V, ldv, nv, L, ldl, Top, ldt, S, lds, Tm, ldT, ib, w, W, trans);
}

// Column measure for the reflector, by one warp (every lane returns the same
// bits: xor-butterfly reductions).  Sets *squared and returns
//   ||x||^2 (*squared = true) for FP32 columns (each square is exact in FP64
//   and lies in [2^-298, 2^256]) and for FP64 columns of a normal-range
//   panel whose sum of squares lies in [2^-900, 2^900] (no square that
//   matters can have been lost to underflow, none can overflow); the square
//   root is then left to make_refl -- one FP64 square root per column
//   instead of two (on this GPU each FP64 instruction of a lone warp costs
//   tens of cycles, and the panel's column chain is serial);
//   ||x|| (*squared = false) otherwise, taken on x scaled by an exact power
//   of two when max|x| is outside [2^-500, 2^500].
template <typename real>
__device__ double warp_norm(const real* x, int len, bool extreme, bool* squared) {
  const int lane = threadIdx.x & 31;
  double ssq = 0.0;
  for (int r = lane; r < len; r += 32) {
    const double v = static_cast<double>(x[r]);
    ssq = fma(v, v, ssq);
  }
  ssq = warp_sum(ssq);
  *squared = true;
  if constexpr (sizeof(real) == 4) {
    return ssq;
  } else {
    if (!extreme && ssq >= 0x1p-900 && ssq <= 0x1p900) return ssq;
    *squared = false;
    const double amax = warp_amax(x, len, lane);
    if (amax != 0.0 && isfinite(amax) && (amax < 0x1p-500 || amax > 0x1p500)) {
      const int e = ilogb(amax);
      const double sc = scalbn(1.0, -e);
      double s2 = 0.0;
      for (int r = lane; r < len; r += 32) {
        const double v = static_cast<double>(x[r]) * sc;
        s2 = fma(v, v, s2);
      }
      s2 = warp_sum(s2);
      return scalbn(sqrt(s2), e);
    }
    return sqrt(ssq);
  }
}

// Householder reflector (LAPACK convention, FP64) from alpha and the
// column measure of x2 (warp_norm):
//   beta = -sign(alpha) ||[alpha; x2]||, tau = (beta - alpha)/beta and the
//   scale 1/(alpha - beta) of v.  Pure function of its inputs, so threads
//   that call it on the same values agree bit for bit.
struct Refl {
  double tau, beta, scal;
};

// xm = ||x2||^2 (squared): ||[alpha; x2]|| = sqrt(alpha^2 + ||x2||^2) needs
// no overflow guard (|alpha| stays below 2^490 in a normal-range panel, and
// FP32 data is far inside FP64's range), and tau and the scale share one
// FP64 reciprocal: with d = alpha - beta, 1/d = beta/(d beta) and
// tau = -d/beta = -d^2/(d beta) (a few ulps from the two divisions).
// xm = ||x2||: hypot and two divisions, safe for any finite entries.
template <typename real>
__device__ __forceinline__ Refl make_refl(double alpha, double xm, bool squared) {
  Refl f;
  if (xm == 0.0) {
    f.tau = 0.0;
    f.beta = alpha;
    f.scal = 0.0;
  } else if (squared && sizeof(real) == 4 && xm >= 0x1p-20 * (alpha * alpha)) {
    // FP32 panels: with a = |alpha|, s = a^2 + xm and h = sqrt(s),
    //   beta = -sign(alpha) h,  tau = 1 + a / h,  1/d = sign(alpha) (h - a) / xm,
    // so the two long FP64 operations, 1/sqrt(s) and 1/xm, run side by side
    // instead of a square root followed by a division (each costs hundreds of
    // cycles on the panel's serial column chain).  h - a loses at most
    // log2(4 a^2 / xm) <= 22 bits to cancellation, leaving 1/d far more
    // accurate than the FP32 value it is rounded to; smaller xm takes the
    // general formula below.
    const double a = fabs(alpha);
    const double sv = fma(a, a, xm);
    const double r = rsqrt(sv);
    const double q = 1.0 / xm;
    const double h = sv * r;
    f.beta = (alpha >= 0.0) ? -h : h;  // sign(0) = +1, also for -0.0
    f.tau = fma(a, r, 1.0);
    const double sc = (h - a) * q;
    f.scal = (alpha >= 0.0) ? sc : -sc;
  } else if (squared) {
    const double h = sqrt(fma(alpha, alpha, xm));
    f.beta = (alpha >= 0.0) ? -h : h;  // sign(0) = +1, also for -0.0
    const double d = alpha - f.beta;
    const double rc = 1.0 / (d * f.beta);
    f.scal = f.beta * rc;
    f.tau = -(d * d) * rc;
  } else {
    const double h = hypot(alpha, xm);
    f.beta = (alpha >= 0.0) ? -h : h;  // sign(0) = +1, also for -0.0
    f.tau = (f.beta - alpha) / f.beta;
    f.scal = 1.0 / (alpha - f.beta);
  }
  return f;
}

template <typename real, bool TS>
__device__ __forceinline__ void publish_refl(double* red, int c, double alpha, double xn, bool squared) {
  const Refl f = make_refl<real>(alpha, xn, squared);
  double* d = red + 4 * (c % 3);
  d[0] = f.tau;
  d[1] = f.beta;
  d[2] = f.scal;
  real* r = reinterpret_cast<real*>(red + 12) + 2 * (c % 3);
  r[0] = static_cast<real>(f.tau);
  r[1] = static_cast<real>(f.scal);
}

//
// The dot products x^T p_d use the unscaled x, which is exact in range while
// the panel's entries stay within [2^-480, 2^480]: products then neither
// overflow nor underflow to nothing.  A FP64 panel with a larger or a
// nonzero smaller max |entry| takes the dot products on v = s x instead
// (one more multiply per element), so entries up to the FP64 limits
// factor without overflow (decided once per panel, uniformly per block).
template <typename real, bool TS>
__device__ void panel_qr(real* P, int ldP, int nr, int ib, real* R, int ldr, double* red, double* taus) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int nwarps = kThreads / 32;
  bool extreme = false;
  if constexpr (sizeof(real) == 8) {
    __shared__ unsigned long long s_amax;
    if (tid == 0) s_amax = 0;
    __syncthreads();
    unsigned long long mx = 0;
    for (int e = tid; e < nr * ib; e += kThreads) {
      const unsigned long long b = abs_bits(P[(e % nr) + (e / nr) * ldP]);
      mx = b > mx ? b : mx;
    }
    if (TS)  // the top triangle's entries enter alpha and the updates too
      for (int e = tid; e < ib * ib; e += kThreads) {
        const int i = e % ib, j = e / ib;
        if (i <= j) {
          const unsigned long long b = abs_bits(R[i + j * ldr]);
          mx = b > mx ? b : mx;
        }
      }
    mx = warp_max_u64(mx);
    if (lane == 0 && mx != 0) atomicMax(&s_amax, mx);
    __syncthreads();
    const double amax = __longlong_as_double(static_cast<long long>(s_amax));
    extreme = amax > 0x1p480 || (amax != 0.0 && amax < 0x1p-480);
  }
  // FP32 panels keep each column's FP64 sum of squares of the rows the next
  // reflectors see (TS: all rows of the bottom block; else the rows from the
  // current step down) and downdate it as reflectors are applied: an
  // orthogonal reflector keeps top^2 + ||x||^2, so the next column's
  // measure costs two FMAs on the chain instead of a warp reduction.  Where
  // more than 16 bits of a sum have cancelled since it was last formed
  // directly, it is formed directly again (its error then stays far below
  // FP32's unit roundoff, which bounds the reflectors' stored precision).
  double* s2 = red + 32;       // running sums, ib <= 64
  double* s2ref = red + 96;    // the sums when last formed directly
  if constexpr (sizeof(real) == 4) {
    for (int d = wid; d < ib; d += nwarps) {
      bool sq;
      const double v = warp_norm<real>(P + d * ldP, nr, false, &sq);
      if (lane == 0) {
        s2[d] = v;
        s2ref[d] = v;
      }
    }
  }
  // reflector of column 0
  if (wid == 0) {
    bool sq;
    const double xn = TS ? warp_norm<real>(P, nr, extreme, &sq) : warp_norm<real>(P + 1, nr - 1, extreme, &sq);
    if (lane == 0) publish_refl<real, TS>(red, 0, static_cast<double>(TS ? R[0] : P[0]), xn, sq);
  }
  __syncthreads();
  for (int c = 0; c <= ib; ++c) {
    // deferred writes of column c-1 (by the last warp: warp 0 carries the
    // column chain)
    if (wid == nwarps - 1 && c > 0) {
      const double* pf = red + 4 * ((c - 1) % 3);
      real* pp = P + (c - 1) * ldP;
      const int r0p = TS ? 0 : c;
      const real sp = static_cast<real>(pf[2]);
      for (int r = r0p + lane; r < nr; r += 32) pp[r] *= sp;
      if (lane == 0) {
        if constexpr (TS)
          R[(c - 1) + (c - 1) * ldr] = static_cast<real>(pf[1]);
        else
          pp[c - 1] = static_cast<real>(pf[1]);
        taus[c - 1] = pf[0];
      }
    }
    if (c == ib) break;
    real* pc = P + c * ldP;
    const int r0 = TS ? 0 : c + 1;
    const real* rf = reinterpret_cast<const real*>(red + 12) + 2 * (c % 3);
    const real tau = rf[0];
    const real scal = rf[1];
    // warp 0 updates column c + 1 and derives its reflector (the serial
    // chain); warps 1 .. nwarps-1 update columns c + 2 .. ib-1 meanwhile
    for (int d = wid == 0 ? c + 1 : c + 1 + wid; d < ib && (wid != 0 || d == c + 1);
         d += (wid == 0 ? 1 : nwarps - 1)) {
      real* pd = P + d * ldP;
      real top_old = real(0), top_new = real(0);
      if (tau != real(0)) {
        real acc = real(0);
        if (!extreme) {
          for (int r = r0 + lane; r < nr; r += 32) acc = fma(pc[r], pd[r], acc);
        } else {
          for (int r = r0 + lane; r < nr; r += 32) acc = fma(pc[r] * scal, pd[r], acc);
        }
        acc = warp_sum(acc);
        real top;
        if constexpr (TS)
          top = R[c + d * ldr];
        else
          top = pd[c];
        const real wv = extreme ? tau * (acc + top) : tau * fma(scal, acc, top);
        const real coef = -(wv * scal);
        for (int r = r0 + lane; r < nr; r += 32) pd[r] = fma(coef, pc[r], pd[r]);
        top_old = top;
        top_new = top - wv;
        if (lane == 0) {
          if constexpr (TS)
            R[c + d * ldr] = top_new;
          else
            pd[c] = top_new;
        }
      } else if (!TS) {
        top_new = pd[c];
      }
      if constexpr (sizeof(real) == 4) {
        // TS: ||x||^2 += top_old^2 - top_new^2; else the sum drops row c
        if (lane == 0) {
          const double to = top_old, tn = top_new;
          s2[d] = TS ? fma(-tn, tn, fma(to, to, s2[d])) : fma(-tn, tn, s2[d]);
        }
      }
      if (d == c + 1) {
        // this warp owns the next column: its reflector, for step c + 1
        __syncwarp();
        bool sq = true;
        double xn = 0.0;
        bool direct = true;
        if constexpr (sizeof(real) == 4) {
          double xm = 0.0;
          if (lane == 0) {
            const double al = static_cast<double>(TS ? R[(c + 1) + (c + 1) * ldr] : pd[c + 1]);
            xm = TS ? s2[d] : fma(-al, al, s2[d]);
          }
          xm = __shfl_sync(0xffffffffu, xm, 0);
          direct = !(xm >= 0x1p-16 * s2ref[d]);
          xn = xm;
        }
        if (direct) {
          xn = TS ? warp_norm<real>(pd, nr, extreme, &sq) : warp_norm<real>(pd + c + 2, nr - c - 2, extreme, &sq);
          if constexpr (sizeof(real) == 4) {
            // the sums restart from the direct value
            if (lane == 0) {
              const double al = static_cast<double>(TS ? R[(c + 1) + (c + 1) * ldr] : pd[c + 1]);
              s2[d] = TS ? xn : fma(al, al, xn);
              s2ref[d] = s2[d];
            }
          }
        }
        if (lane == 0) {
          const double alpha = static_cast<double>(TS ? R[(c + 1) + (c + 1) * ldr] : pd[c + 1]);
          publish_refl<real, TS>(red, c + 1, alpha, xn, sq);
        }
      }
    }
    __syncthreads();
  }
  __syncthreads();
}

// Compact-WY T of the panel's reflectors (DLARFT, forward, columnwise):
//   T(c,c) = tau_c,  T(0:c, c) = -tau_c T(0:c, 0:c) (V(:,0:c)^T v_c).
// The Gram products Y(a,b) = v_a^T v_b (a < b) go to Y (ib x ib, ld ib).
template <typename real, bool TS>
__device__ void form_t(const real* P, int ldP, int nr, int ib, const double* taus, real* Y, real* Tm,
                       int ldT) {
  const int tid = threadIdx.x;
  const int npairs = ib * ib;
  for (int e = tid; e < npairs; e += kThreads) {
    const int a = e % ib, b = e / ib;
    if (a >= b) continue;
    const real* pa = P + a * ldP;
    const real* pb = P + b * ldP;
    real acc = real(0);
    if (!TS) {
      // v_a = [0..0, 1 at a, P(a+1:, a)], v_b = [0..0, 1 at b, P(b+1:, b)]
      acc = pa[b];
      for (int r = b + 1; r < nr; ++r) acc += pa[r] * pb[r];
    } else {
      for (int r = 0; r < nr; ++r) acc += pa[r] * pb[r];
    }
    Y[a + b * ib] = acc;
  }
  // T by doubling diagonal blocks: with Q1 = I - V1 T11 V1^T and
  // Q2 = I - V2 T22 V2^T, Q1 Q2 = I - V T V^T with T12 = -T11 (V1^T V2) T22.
  // Blocks of size bs already hold their T; each level merges neighbours
  // (block 2 may be short when ib is not a power of two), so the dependent
  // chain is 2 (1 + 2 + 4 + ...) multiply-adds and one barrier pair per level
  // instead of the column recurrence's ib (ib - 1) / 2 on one warp.
  // W = Y12 T22 is kept in Y's unused lower triangle (W(a, b) at Y[b + a ib]).
  for (int e = tid; e < ib * ib; e += kThreads) {
    const int r = e % ib, c = e / ib;
    Tm[r + c * ldT] = r == c ? static_cast<real>(taus[c]) : real(0);
  }
  __syncthreads();
  for (int bs = 1; bs < ib; bs *= 2) {
    const int span = (ib + 2 * bs - 1) / (2 * bs) * bs * bs;
    for (int e = tid; e < span; e += kThreads) {
      const int g0 = 2 * bs * (e / (bs * bs)), rem = e % (bs * bs);
      const int a = g0 + rem % bs, b = g0 + bs + rem / bs;
      if (b >= ib) continue;
      real acc = real(0);
      for (int t = g0 + bs; t <= b; ++t) acc = fma(Y[a + t * ib], Tm[t + b * ldT], acc);
      Y[b + a * ib] = acc;
    }
    __syncthreads();
    for (int e = tid; e < span; e += kThreads) {
      const int g0 = 2 * bs * (e / (bs * bs)), rem = e % (bs * bs);
      const int a = g0 + rem % bs, b = g0 + bs + rem / bs;
      if (b >= ib) continue;
      real acc = real(0);
      for (int t = a; t < g0 + bs; ++t) acc = fma(Tm[a + t * ldT], Y[b + t * ib], acc);
      Tm[a + b * ldT] = -acc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- tasks
template <typename real>
__device__ __forceinline__ real* tile_ptr(const Inst& I, int i, int j) {
  const long long nb2 = static_cast<long long>(I.nb) * I.nb;
  if (j < I.q) return static_cast<real*>(I.A) + (static_cast<long long>(i) + static_cast<long long>(j) * I.p) * nb2;
  return static_cast<real*>(I.B) + (static_cast<long long>(i) + static_cast<long long>(j - I.q) * I.p) * nb2;
}

template <typename real>
__device__ __forceinline__ real* t_ptr(const Inst& I, int i, int k) {
  return static_cast<real*>(I.T) + t_offset(I.p, I.nb, I.ib, i, k);
}

// T factors of the tree variant's TTQRT of eliminated head (i, k).
template <typename real>
__device__ __forceinline__ real* t2_ptr(const Inst& I, int i, int k) {
  return static_cast<real*>(I.T) + t2_offset(I.p, I.q, I.nb, I.ib, i, k);
}

// Rows of tile row i that lie inside the matrix (below them the tiles hold
// zero padding, in A, in the right-hand sides and in the reflectors), rounded
// up to a multiple of 4 (the FP32 micro-tiles' granularity).  The TS / SS
// kernels take only these rows: the padding would add exact zeros to every
// sum and leave itself unchanged.
__device__ __forceinline__ int live_rows(const Inst& I, int i) {
  const int v = I.m - i * I.nb;
  if (v >= I.nb) return I.nb;
  const int r = (v + 3) & ~3;
  return r < I.nb ? r : I.nb;
}

// Width of slab s of tile column j.
__device__ __forceinline__ int slab_width(const Inst& I, int j, int s) {
  int w = I.cs;
  if (j >= I.q) {
    const int c0 = (j - I.q) * I.nb + s * I.cs;
    int rem = I.nrhs - c0;
    if (rem < w) w = rem;
  }
  return w;
}

// GEQRT(k) on tile (row, k): Section 3.1 DGEQT2 with inner blocking (row = k
// in Algorithm 1; a domain head in the tree variant).
template <typename real>
__device__ void exec_geqrt(Ctx<real>& cx, const Inst& I, int k, int row) {
  const int nb = I.nb, ib = I.ib, cs = I.cs;
  real* A = tile_ptr<real>(I, row, k);
  real* Tg = t_ptr<real>(I, row, k);
  double* taus = cx.red + 2 * kThreads;
  for (int l0 = 0; l0 < nb; l0 += ib) {
    const int nr = nb - l0;
    load_block(cx.P, cx.ldP, A + l0 + static_cast<long long>(l0) * nb, nb, nr, ib);
    __syncthreads();
    panel_qr<real, false>(cx.P, cx.ldP, nr, ib, nullptr, 0, cx.red, taus);
    store_block(A + l0 + static_cast<long long>(l0) * nb, nb, cx.P, cx.ldP, nr, ib);
    form_t<real, false>(cx.P, cx.ldP, nr, ib, taus, cx.Rb, cx.T, cx.ldT);
    store_block(Tg + static_cast<long long>(l0) * ib, ib, cx.T, cx.ldT, ib, ib);
    for (int c0 = l0 + ib; c0 < nb; c0 += cs) {
      const int w = nb - c0 < cs ? nb - c0 : cs;
      load_block(cx.S, cx.ldS, A + l0 + static_cast<long long>(c0) * nb, nb, nr, w);
      __syncthreads();
      apply_any<real>(cx.P + ib, cx.ldP, nr - ib, cx.P, cx.ldP, cx.S, cx.ldS, cx.S + ib, cx.ldS, cx.T, cx.ldT,
                        ib, w, cx.W, cx.Part, true);
      store_block(A + l0 + static_cast<long long>(c0) * nb, nb, cx.S, cx.ldS, nr, w);
      __syncthreads();
    }
    __syncthreads();
  }
}

// TSQRT(k, i) with top tile (head, k): Section 3.1 DTSQT2 with inner
// blocking (head = k in Algorithm 1).  tt: the tree variant's TTQRT -- the
// bottom is the upper triangle of (i, k) (its strictly lower part holds that
// head's GEQRT reflectors and is neither read nor written); block l's
// reflectors then live in its first l0 + ib rows only.
template <typename real>
__device__ void exec_tsqrt(Ctx<real>& cx, const Inst& I, int k, int head, int i, bool tt) {
  const int nb = I.nb, ib = I.ib, cs = I.cs;
  real* Rt = tile_ptr<real>(I, head, k);
  real* Ai = tile_ptr<real>(I, i, k);
  real* Tg = tt ? t2_ptr<real>(I, i, k) : t_ptr<real>(I, i, k);
  double* taus = cx.red + 2 * kThreads;
  real* Rb = cx.Rb;  // ib x ib triangle, ld ib
  for (int l0 = 0; l0 < nb; l0 += ib) {
    // the triangle's block (upper part only; its lower part holds V_kk)
    for (int e = threadIdx.x; e < ib * ib; e += kThreads) {
      const int r = e % ib, c = e / ib;
      Rb[r + c * ib] = (r <= c) ? ldg_cg(Rt + (l0 + r) + static_cast<long long>(l0 + c) * nb) : real(0);
    }
    bulk_cols(cx, cx.P, cx.ldP, Ai + static_cast<long long>(l0) * nb, nb, nb, ib);
    const int nv = tt ? l0 + ib : live_rows(I, i);  // rows that can hold reflector entries
    if (tt)
      for (int e = threadIdx.x; e < nv * ib; e += kThreads) {
        const int r = e % nv, c = e / nv;
        if (r > l0 + c) cx.P[r + c * cx.ldP] = real(0);
      }
    __syncthreads();
    panel_qr<real, true>(cx.P, cx.ldP, nv, ib, Rb, ib, cx.red, taus);
    for (int e = threadIdx.x; e < ib * ib; e += kThreads) {
      const int r = e % ib, c = e / ib;
      if (r <= c) Rt[(l0 + r) + static_cast<long long>(l0 + c) * nb] = Rb[r + c * ib];
    }
    if (tt) {
      for (int e = threadIdx.x; e < nv * ib; e += kThreads) {
        const int r = e % nv, c = e / nv;
        if (r <= l0 + c) Ai[r + static_cast<long long>(l0 + c) * nb] = cx.P[r + c * cx.ldP];
      }
    } else {
      store_block(Ai + static_cast<long long>(l0) * nb, nb, cx.P, cx.ldP, nb, ib);
    }
    __syncthreads();
    form_t<real, true>(cx.P, cx.ldP, nv, ib, taus, cx.Rb, cx.T, cx.ldT);
    store_block(Tg + static_cast<long long>(l0) * ib, ib, cx.T, cx.ldT, ib, ib);
    for (int c0 = l0 + ib; c0 < nb; c0 += cs) {
      const int w = nb - c0 < cs ? nb - c0 : cs;
      load_block(cx.Top, ib, Rt + l0 + static_cast<long long>(c0) * nb, nb, ib, w);
      bulk_cols(cx, cx.S, cx.ldS, Ai + static_cast<long long>(c0) * nb, nb, nb, w);
      __syncthreads();
      apply_any<real>(cx.P, cx.ldP, nv, nullptr, 0, cx.Top, ib, cx.S, cx.ldS, cx.T, cx.ldT, ib, w, cx.W, cx.Part, true);
      store_block(Rt + l0 + static_cast<long long>(c0) * nb, nb, cx.Top, ib, ib, w);
      store_block(Ai + static_cast<long long>(c0) * nb, nb, cx.S, cx.ldS, nv, w);
      __syncthreads();
    }
    __syncthreads();
  }
}

// LARFB(k, j, s) on row `row`: slab s of tile (row, j) <- Q^T (or Q) of the
// GEQRT'ed tile (row, k) times it (row = k in Algorithm 1).
template <typename real>
__device__ void exec_larfb(Ctx<real>& cx, const Inst& I, int k, int row, int j, int s, bool trans) {
  const int nb = I.nb, ib = I.ib;
  const real* Vt = tile_ptr<real>(I, row, k);
  const real* Tg = t_ptr<real>(I, row, k);
  real* C = tile_ptr<real>(I, row, j) + static_cast<long long>(s) * I.cs * nb;
  const int w = slab_width(I, j, s);
  bulk_cols(cx, cx.S, cx.ldS, C, nb, nb, w);
  const int nblk = nb / ib;
  for (int bb = 0; bb < nblk; ++bb) {
    const int l = trans ? bb : nblk - 1 - bb;
    const int l0 = l * ib, nr = nb - l0;
    // V_l: unit lower block; read only below the diagonal (the triangle above
    // may be rewritten concurrently by TSQRT of the same step)
    for (int e = threadIdx.x; e < nr * ib; e += kThreads) {
      const int r = e % nr, c = e / nr;
      if (r > c) cx.P[r + c * cx.ldP] = ldg_cg(Vt + (l0 + r) + static_cast<long long>(l0 + c) * nb);
    }
    load_block(cx.T, cx.ldT, Tg + static_cast<long long>(l0) * ib, ib, ib, ib);
    __syncthreads();
    apply_any<real>(cx.P + ib, cx.ldP, nr - ib, cx.P, cx.ldP, cx.S + l0, cx.ldS, cx.S + l0 + ib, cx.ldS, cx.T,
                      cx.ldT, ib, w, cx.W, cx.Part, trans);
  }
  store_block(C, nb, cx.S, cx.ldS, nb, w);
  __syncthreads();
}

// SSRFB(k, i, j, s): slab s of [(head, j); (i, j)] <- Q_ik^T (or Q_ik) times
// it (head = k in Algorithm 1).  tt: the tree variant's TTMQR, whose
// reflectors are the upper triangle of (i, k) (block l: first l0 + ib rows).
template <typename real>
__device__ void exec_ssrfb(Ctx<real>& cx, const Inst& I, int k, int head, int i, int j, int s, bool trans, bool tt) {
  const int nb = I.nb, ib = I.ib;
  const real* Vt = tile_ptr<real>(I, i, k);
  const real* Tg = tt ? t2_ptr<real>(I, i, k) : t_ptr<real>(I, i, k);
  const long long soff = static_cast<long long>(s) * I.cs * nb;
  real* Ct = tile_ptr<real>(I, head, j) + soff;
  real* Cb = tile_ptr<real>(I, i, j) + soff;
  const int w = slab_width(I, j, s);
  const int nblk = nb / ib;
  if (cx.TopS != nullptr) {
    // FP32: the bottom slab, the whole top slab, all T blocks and the first
    // V block arrive in one bulk phase; block l+1's V is copied into the
    // other buffer while block l is applied; both slabs go back at the end
    // (same arithmetic, same order as below).
    const int lf = trans ? 0 : nblk - 1;
    if (threadIdx.x < 32) {
      const uint32_t cb = static_cast<uint32_t>(nb) * sizeof(real);
      bulk_expect(cx, cb * (2 * w + ib) + static_cast<uint32_t>(ib) * nb * sizeof(real));
      __syncwarp();
      bulk_issue_cols(cx, cx.S, cx.ldS, Cb, nb, nb, w);
      bulk_issue_cols(cx, cx.TopS, cx.ldS, Ct, nb, nb, w);
      bulk_issue_cols(cx, cx.Tst, 0, Tg, 0, ib * nb, 1);
      bulk_issue_cols(cx, cx.P, cx.ldP, Vt + static_cast<long long>(lf) * ib * nb, nb, nb, ib);
    }
    bulk_wait(cx);
    for (int bb = 0; bb < nblk; ++bb) {
      const int l = trans ? bb : nblk - 1 - bb;
      const int l0 = l * ib;
      real* Pc = (bb & 1) ? cx.P2 : cx.P;
      if (bb + 1 < nblk && threadIdx.x < 32) {
        const int ln = trans ? bb + 1 : nblk - 2 - bb;
        bulk_expect(cx, static_cast<uint32_t>(nb) * ib * sizeof(real));
        __syncwarp();
        bulk_issue_cols(cx, (bb & 1) ? cx.P : cx.P2, cx.ldP, Vt + static_cast<long long>(ln) * ib * nb, nb, nb, ib);
      }
      for (int e = threadIdx.x; e < ib * ib; e += kThreads) {
        const int r = e % ib, c = e / ib;
        cx.T[r + c * cx.ldT] = cx.Tst[l0 * ib + r + c * ib];
      }
      const int nv = tt ? l0 + ib : live_rows(I, i);
      if (tt)
        for (int e = threadIdx.x; e < nv * ib; e += kThreads) {
          const int r = e % nv, c = e / nv;
          if (r > l0 + c) Pc[r + c * cx.ldP] = real(0);
        }
      __syncthreads();
      apply_any<real>(Pc, cx.ldP, nv, nullptr, 0, cx.TopS + l0, cx.ldS, cx.S, cx.ldS, cx.T, cx.ldT, ib, w, cx.W,
                      cx.Part, trans);
      if (bb + 1 < nblk) bulk_wait(cx);
    }
    store_block(Cb, nb, cx.S, cx.ldS, nb, w);
    store_block(Ct, nb, cx.TopS, cx.ldS, nb, w);
    __syncthreads();
    return;
  }
  if (cx.P2 != nullptr) {
    // Pipelined: block l+1's V is copied into the other buffer while block l
    // is applied (same arithmetic, same order as below).
    const int lf = trans ? 0 : nblk - 1;
    if (threadIdx.x < 32)
      bulk_cols2_issue(cx, cx.S, cx.ldS, Cb, nb, nb, w, cx.P, cx.ldP, Vt + static_cast<long long>(lf) * ib * nb, nb,
                       nb, ib);
    bulk_wait(cx);
    for (int bb = 0; bb < nblk; ++bb) {
      const int l = trans ? bb : nblk - 1 - bb;
      const int l0 = l * ib;
      real* Pc = (bb & 1) ? cx.P2 : cx.P;
      if (bb + 1 < nblk && threadIdx.x < 32) {
        const int ln = trans ? bb + 1 : nblk - 2 - bb;
        bulk_cols2_issue(cx, (bb & 1) ? cx.P : cx.P2, cx.ldP, Vt + static_cast<long long>(ln) * ib * nb, nb, nb, ib,
                         static_cast<real*>(nullptr), 0, static_cast<const real*>(nullptr), 0, 0, 0);
      }
      load_block(cx.T, cx.ldT, Tg + static_cast<long long>(l0) * ib, ib, ib, ib);
      load_block(cx.Top, ib, Ct + l0, nb, ib, w);
      const int nv = tt ? l0 + ib : live_rows(I, i);
      if (tt)
        for (int e = threadIdx.x; e < nv * ib; e += kThreads) {
          const int r = e % nv, c = e / nv;
          if (r > l0 + c) Pc[r + c * cx.ldP] = real(0);
        }
      __syncthreads();
      apply_any<real>(Pc, cx.ldP, nv, nullptr, 0, cx.Top, ib, cx.S, cx.ldS, cx.T, cx.ldT, ib, w, cx.W, cx.Part, trans);
      store_block(Ct + l0, nb, cx.Top, ib, ib, w);
      __syncthreads();
      if (bb + 1 < nblk) bulk_wait(cx);
    }
    store_block(Cb, nb, cx.S, cx.ldS, nb, w);
    __syncthreads();
    return;
  }
  bulk_cols(cx, cx.S, cx.ldS, Cb, nb, nb, w);
  for (int bb = 0; bb < nblk; ++bb) {
    const int l = trans ? bb : nblk - 1 - bb;
    const int l0 = l * ib;
    load_block(cx.T, cx.ldT, Tg + static_cast<long long>(l0) * ib, ib, ib, ib);
    load_block(cx.Top, ib, Ct + l0, nb, ib, w);
    bulk_cols(cx, cx.P, cx.ldP, Vt + static_cast<long long>(l0) * nb, nb, nb, ib);
    const int nv = tt ? l0 + ib : live_rows(I, i);
    if (tt)
      for (int e = threadIdx.x; e < nv * ib; e += kThreads) {
        const int r = e % nv, c = e / nv;
        if (r > l0 + c) cx.P[r + c * cx.ldP] = real(0);
      }
    __syncthreads();
    apply_any<real>(cx.P, cx.ldP, nv, nullptr, 0, cx.Top, ib, cx.S, cx.ldS, cx.T, cx.ldT, ib, w, cx.W, cx.Part, trans);
    store_block(Ct + l0, nb, cx.Top, ib, ib, w);
    __syncthreads();
  }
  store_block(Cb, nb, cx.S, cx.ldS, nb, w);
  __syncthreads();
}

// S(0:nv, 0:w) -= V(0:nv, 0:kk) X(0:kk, 0:w)   (V ld ldv, X ld ldx)
template <typename real>
__device__ void gemm_sub(real* S, int lds, int nv, int w, const real* V, int ldv, const real* X, int ldx, int kk) {
  for (int o = threadIdx.x; o < nv * w; o += kThreads) {
    const int t = o % nv, c = o / nv;
    const real* xc = X + c * ldx;
    real a0 = real(0), a1 = real(0);
    int r = 0;
    for (; r + 1 < kk; r += 2) {
      a0 += V[t + r * ldv] * xc[r];
      a1 += V[t + (r + 1) * ldv] * xc[r + 1];
    }
    if (r < kk) a0 += V[t + r * ldv] * xc[r];
    S[t + c * lds] -= a0 + a1;
  }
}

// Triangular solves of one ib x ib diagonal block for w right-hand-side
// columns in shared memory (x = S + c ldS + b0), one warp per column, in
// column (axpy) order: once x_r is final it is broadcast and every lane
// removes its multiple from the rows still open.  Reciprocals of the
// diagonal are taken once per block, all lanes at once (an FP64 division
// costs hundreds of cycles on this GPU), into rinv (ib entries).  Rows at or
// past nvalid (zero padding) get x = 0.
//   upper = true:  T x = c (T upper, ld ldT), r = ib-1 .. 0
//   upper = false: T^T x = c,                  r = 0 .. ib-1
template <typename real, bool upper>
__device__ void tri_block_solve(real* S, int ldS, int b0, int w, const real* T, int ldT, int ib, int nvalid,
                                real* rinv) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < ib; t += kThreads)
    rinv[t] = (b0 + t < nvalid) ? real(1) / T[t + t * ldT] : real(0);
  __syncthreads();
  for (int c = wid; c < w; c += kThreads / 32) {
    real* x = S + c * ldS + b0;
    for (int q = 0; q < ib; ++q) {
      const int r = upper ? ib - 1 - q : q;
      const real xr = x[r] * rinv[r];
      __syncwarp();
      if (lane == 0) x[r] = xr;
      if constexpr (upper) {
        for (int t = lane; t < r; t += 32) x[t] = fma(-T[t + r * ldT], xr, x[t]);
      } else {
        for (int t = r + 1 + lane; t < ib; t += 32) x[t] = fma(-T[r + t * ldT], xr, x[t]);
      }
      __syncwarp();
    }
  }
}

// TRSM_UPD(k, l, j, s): C_k -= R_kl X_l on slab s of right-hand-side column j.
template <typename real>
__device__ void exec_trsm_upd(Ctx<real>& cx, const Inst& I, int k, int l, int j, int s) {
  const int nb = I.nb, ib = I.ib;
  const long long soff = static_cast<long long>(s) * I.cs * nb;
  real* C = tile_ptr<real>(I, k, j) + soff;
  const real* X = tile_ptr<real>(I, l, j) + soff;
  const real* R = tile_ptr<real>(I, k, l);
  const int w = slab_width(I, j, s);
  bulk_cols(cx, cx.S, cx.ldS, C, nb, nb, w);
  for (int c0 = 0; c0 < nb; c0 += ib) {
    bulk_cols(cx, cx.P, cx.ldP, R + static_cast<long long>(c0) * nb, nb, nb, ib);
    load_block(cx.W, ib, X + c0, nb, ib, w);
    __syncthreads();
    gemm_sub(cx.S, cx.ldS, nb, w, cx.P, cx.ldP, cx.W, ib, ib);
    __syncthreads();
  }
  store_block(C, nb, cx.S, cx.ldS, nb, w);
  __syncthreads();
}

// TRSM_SOLVE(k, j, s): X_k = R_kk^{-1} C_k (upper triangular, blocked by ib
// from the bottom).  Rows past n (zero padding) get x = 0.
template <typename real>
__device__ void exec_trsm_solve(Ctx<real>& cx, const Inst& I, int k, int j, int s) {
  const int nb = I.nb, ib = I.ib;
  const long long soff = static_cast<long long>(s) * I.cs * nb;
  real* C = tile_ptr<real>(I, k, j) + soff;
  const real* R = tile_ptr<real>(I, k, k);
  const int w = slab_width(I, j, s);
  const int nvalid = I.n - k * nb;  // rows of this tile inside the matrix
  bulk_cols(cx, cx.S, cx.ldS, C, nb, nb, w);
  for (int b0 = nb - ib; b0 >= 0; b0 -= ib) {
    for (int e = threadIdx.x; e < ib * ib; e += kThreads) {
      const int r = e % ib, c = e / ib;
      cx.T[r + c * cx.ldT] = (r <= c) ? ldg_cg(R + (b0 + r) + static_cast<long long>(b0 + c) * nb) : real(0);
    }
    __syncthreads();
    tri_block_solve<real, true>(cx.S, cx.ldS, b0, w, cx.T, cx.ldT, ib, nvalid, cx.W);
    __syncthreads();
    if (b0 > 0) {
      load_block(cx.P, cx.ldP, R + static_cast<long long>(b0) * nb, nb, b0, ib);
      __syncthreads();
      gemm_sub(cx.S, cx.ldS, b0, w, cx.P, cx.ldP, cx.S + b0, cx.ldS, ib);
      __syncthreads();
    }
  }
  store_block(C, nb, cx.S, cx.ldS, nb, w);
  __syncthreads();
}

// TRSMT_UPD(k, l, j, s): C_k -= R_lk^T X_l  (l < k).
template <typename real>
__device__ void exec_trsmt_upd(Ctx<real>& cx, const Inst& I, int k, int l, int j, int s) {
  const int nb = I.nb, ib = I.ib;
  const long long soff = static_cast<long long>(s) * I.cs * nb;
  real* C = tile_ptr<real>(I, k, j) + soff;
  const real* X = tile_ptr<real>(I, l, j) + soff;
  const real* R = tile_ptr<real>(I, l, k);
  const int w = slab_width(I, j, s);
  bulk_cols(cx, cx.S, cx.ldS, X, nb, nb, w);
  for (int r0 = 0; r0 < nb; r0 += ib) {
    bulk_cols(cx, cx.P, cx.ldP, R + static_cast<long long>(r0) * nb, nb, nb, ib);
    load_block(cx.Top, ib, C + r0, nb, ib, w);
    __syncthreads();
    for (int o = threadIdx.x; o < ib * w; o += kThreads) {
      const int r = o % ib, c = o / ib;
      const real* pr = cx.P + r * cx.ldP;
      const real* xc = cx.S + c * cx.ldS;
      real a0 = real(0), a1 = real(0);
      int t = 0;
      for (; t + 1 < nb; t += 2) {
        a0 += pr[t] * xc[t];
        a1 += pr[t + 1] * xc[t + 1];
      }
      if (t < nb) a0 += pr[t] * xc[t];
      cx.Top[r + c * ib] -= a0 + a1;
    }
    __syncthreads();
    store_block(C + r0, nb, cx.Top, ib, ib, w);
    __syncthreads();
  }
}

// TRSMT_SOLVE(k, j, s): X_k = R_kk^{-T} C_k (forward substitution by ib blocks).
template <typename real>
__device__ void exec_trsmt_solve(Ctx<real>& cx, const Inst& I, int k, int j, int s) {
  const int nb = I.nb, ib = I.ib;
  const long long soff = static_cast<long long>(s) * I.cs * nb;
  real* C = tile_ptr<real>(I, k, j) + soff;
  const real* R = tile_ptr<real>(I, k, k);
  const int w = slab_width(I, j, s);
  const int nvalid = I.n - k * nb;
  bulk_cols(cx, cx.S, cx.ldS, C, nb, nb, w);
  for (int b0 = 0; b0 < nb; b0 += ib) {
    for (int e = threadIdx.x; e < ib * ib; e += kThreads) {
      const int r = e % ib, c = e / ib;
      cx.T[r + c * cx.ldT] = (r <= c) ? ldg_cg(R + (b0 + r) + static_cast<long long>(b0 + c) * nb) : real(0);
    }
    __syncthreads();
    tri_block_solve<real, false>(cx.S, cx.ldS, b0, w, cx.T, cx.ldT, ib, nvalid, cx.W);
    __syncthreads();
    const int nbelow = nb - b0 - ib;
    if (nbelow > 0) {
      // P(r', t) = R(b0 + t, b0 + ib + r'): the block row to the right, transposed
      for (int e = threadIdx.x; e < nbelow * ib; e += kThreads) {
        const int rr = e % nbelow, t = e / nbelow;
        cx.P[rr + t * cx.ldP] = ldg_cg(R + (b0 + t) + static_cast<long long>(b0 + ib + rr) * nb);
      }
      __syncthreads();
      gemm_sub(cx.S + b0 + ib, cx.ldS, nbelow, w, cx.P, cx.ldP, cx.S + b0, cx.ldS, ib);
      __syncthreads();
    }
  }
  store_block(C, nb, cx.S, cx.ldS, nb, w);
  __syncthreads();
}

// ---------------------------------------------------------------- 2b x b bottoms
// TSQRT2(k, h, rows): TSQRT with the bottom made of `rows` stacked tiles
// (h .. h+rows-1, k): the 2b x b blocks of Section 3.2's remark, held as b x b
// storage tiles.  The panel and slabs are staged with rows*nb rows.
template <typename real>
__device__ void exec_tsqrt2(Ctx<real>& cx, const Inst& I, int k, int h, int rows) {
  const int nb = I.nb, ib = I.ib, cs = I.cs, nv = (rows - 1) * nb + live_rows(I, h + rows - 1);
  real* Rt = tile_ptr<real>(I, k, k);
  real* Tg = t_ptr<real>(I, h, k);
  double* taus = cx.red + 2 * kThreads;
  real* Rb = cx.Rb;  // ib x ib triangle, ld ib
  for (int l0 = 0; l0 < nb; l0 += ib) {
    for (int e = threadIdx.x; e < ib * ib; e += kThreads) {
      const int r = e % ib, c = e / ib;
      Rb[r + c * ib] = (r <= c) ? ldg_cg(Rt + (l0 + r) + static_cast<long long>(l0 + c) * nb) : real(0);
    }
    for (int a = 0; a < rows; ++a)
      bulk_cols(cx, cx.P + a * nb, cx.ldP, tile_ptr<real>(I, h + a, k) + static_cast<long long>(l0) * nb, nb, nb, ib);
    __syncthreads();
    panel_qr<real, true>(cx.P, cx.ldP, nv, ib, Rb, ib, cx.red, taus);
    for (int e = threadIdx.x; e < ib * ib; e += kThreads) {
      const int r = e % ib, c = e / ib;
      if (r <= c) Rt[(l0 + r) + static_cast<long long>(l0 + c) * nb] = Rb[r + c * ib];
    }
    for (int a = 0; a < rows; ++a)
      store_block(tile_ptr<real>(I, h + a, k) + static_cast<long long>(l0) * nb, nb, cx.P + a * nb, cx.ldP, nb, ib);
    __syncthreads();
    form_t<real, true>(cx.P, cx.ldP, nv, ib, taus, cx.Rb, cx.T, cx.ldT);
    store_block(Tg + static_cast<long long>(l0) * ib, ib, cx.T, cx.ldT, ib, ib);
    for (int c0 = l0 + ib; c0 < nb; c0 += cs) {
      const int w = nb - c0 < cs ? nb - c0 : cs;
      load_block(cx.Top, ib, Rt + l0 + static_cast<long long>(c0) * nb, nb, ib, w);
      for (int a = 0; a < rows; ++a)
        bulk_cols(cx, cx.S + a * nb, cx.ldS, tile_ptr<real>(I, h + a, k) + static_cast<long long>(c0) * nb, nb, nb, w);
      __syncthreads();
      apply_any<real>(cx.P, cx.ldP, nv, nullptr, 0, cx.Top, ib, cx.S, cx.ldS, cx.T, cx.ldT, ib, w, cx.W, cx.Part, true);
      store_block(Rt + l0 + static_cast<long long>(c0) * nb, nb, cx.Top, ib, ib, w);
      for (int a = 0; a < rows; ++a)
        store_block(tile_ptr<real>(I, h + a, k) + static_cast<long long>(c0) * nb, nb, cx.S + a * nb, cx.ldS, nb, w);
      __syncthreads();
    }
    __syncthreads();
  }
}

// SSRFB2(k, h, rows, j, s): slab s of [(k, j); (h .. h+rows-1, j)] <- the
// transformations of TSQRT2(k, h, rows) (Q^T if trans, else Q).
template <typename real>
__device__ void exec_ssrfb2(Ctx<real>& cx, const Inst& I, int k, int h, int rows, int j, int s, bool trans) {
  const int nb = I.nb, ib = I.ib, nv = (rows - 1) * nb + live_rows(I, h + rows - 1);
  const real* Tg = t_ptr<real>(I, h, k);
  const long long soff = static_cast<long long>(s) * I.cs * nb;
  real* Ct = tile_ptr<real>(I, k, j) + soff;
  const int w = slab_width(I, j, s);
  const int nblk = nb / ib;
  const uint32_t cb = static_cast<uint32_t>(nb) * sizeof(real);
  // each block's V pieces go out as one bulk phase before its T and Top
  // loads, so the copy and the loads overlap (the first phase also carries
  // the bottom slabs)
  for (int bb = 0; bb < nblk; ++bb) {
    const int blk = trans ? bb : nblk - 1 - bb;
    const int l0 = blk * ib;
    if (threadIdx.x < 32) {
      bulk_expect(cx, cb * rows * (ib + (bb == 0 ? w : 0)));
      __syncwarp();
      if (bb == 0)
        for (int a = 0; a < rows; ++a)
          bulk_issue_cols(cx, cx.S + a * nb, cx.ldS, tile_ptr<real>(I, h + a, j) + soff, nb, nb, w);
      for (int a = 0; a < rows; ++a)
        bulk_issue_cols(cx, cx.P + a * nb, cx.ldP, tile_ptr<real>(I, h + a, k) + static_cast<long long>(l0) * nb,
                        nb, nb, ib);
    }
    load_block(cx.T, cx.ldT, Tg + static_cast<long long>(l0) * ib, ib, ib, ib);
    load_block(cx.Top, ib, Ct + l0, nb, ib, w);
    bulk_wait(cx);
    __syncthreads();
    apply_any<real>(cx.P, cx.ldP, nv, nullptr, 0, cx.Top, ib, cx.S, cx.ldS, cx.T, cx.ldT, ib, w, cx.W, cx.Part, trans);
    store_block(Ct + l0, nb, cx.Top, ib, ib, w);
    __syncthreads();
  }
  for (int a = 0; a < rows; ++a) store_block(tile_ptr<real>(I, h + a, j) + soff, nb, cx.S + a * nb, cx.ldS, nb, w);
  __syncthreads();
}

// ---------------------------------------------------------------- tiled LU
// Pairwise-pivoting LU kernels (the LU analogue of Algorithm 1, Section 5).
// Each works in blocks of ib columns: within a block the interchanges act on
// whole block rows; applying a block to other columns is its interchanges in
// order, then W = L11^-1 Top, Top = W, S -= L21 W.  L11^-1 (unit lower) is
// formed once by the factoring kernel and stored transposed in the ib x ib
// slot that QR uses for T_l, so that X(r, s) = Tm[s + r * ldT] (s <= r).

// Row of largest magnitude in x[r0..n), ties to the smallest index; one warp,
// every lane returns the same index (n if the range is empty).
template <typename real>
__device__ int warp_iamax(const real* x, int r0, int n, unsigned long long* best_out) {
  const int lane = threadIdx.x & 31;
  unsigned long long best = 0;
  int bi = n;
  for (int r = r0 + lane; r < n; r += 32) {
    const unsigned long long b = abs_bits(x[r]);
    if (bi == n || b > best) {
      best = b;
      bi = r;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oi != n && (bi == n || ob > best || (ob == best && oi < bi))) {
      best = ob;
      bi = oi;
    }
  }
  if (best_out) *best_out = best;
  return bi;
}

// X = L^-1 for the unit lower ib x ib triangle below the diagonal of L (ld
// ldl), written as Tm[s + r * ldT] = X(r, s) (zeros for s > r).  One thread
// per column s of X (forward substitution down the column).
template <typename real>
__device__ void unit_lower_inverse_t(const real* L, int ldl, int ib, real* Tm, int ldT) {
  for (int s = threadIdx.x; s < ib; s += kThreads) {
    for (int r = 0; r < s; ++r) Tm[s + r * ldT] = real(0);
    Tm[s + s * ldT] = real(1);
    for (int r = s + 1; r < ib; ++r) {
      real a = -L[r + s * ldl];
      for (int t = s + 1; t < r; ++t) a = fma(-L[r + t * ldl], Tm[s + t * ldT], a);
      Tm[s + r * ldT] = a;
    }
  }
}

// One LU block applied to a column slab after its interchanges:
//   W = X Top (X = L11^-1 from Tm), Top = W, S -= V W.
// V is nv x ib (ldv), Top ib x w (ldt), S nv x w (lds).
template <typename real>
__device__ void apply_block_lu(const real* __restrict__ V, int ldv, int nv, real* Top, int ldt, real* S, int lds,
                               const real* __restrict__ Tm, int ldT, int ib, int w, real* W) {
  const int tid = threadIdx.x;
  const int nout = ib * w;
  for (int o = tid; o < nout; o += kThreads) {
    const int r = o % ib, c = o / ib;
    const real* tc = Top + c * ldt;
    real a = tc[r];
    for (int s = 0; s < r; ++s) a = fma(Tm[s + r * ldT], tc[s], a);
    W[o] = a;
  }
  __syncthreads();
  for (int o = tid; o < nout; o += kThreads) Top[(o % ib) + (o / ib) * ldt] = W[o];
  const int nS = nv * w;
  for (int o = tid; o < nS; o += 2 * kThreads) {
    const int o2 = o + kThreads;
    const bool two = o2 < nS;
    const int t1 = o % nv, c1 = o / nv;
    const int t2 = two ? o2 % nv : t1, c2 = two ? o2 / nv : c1;
    const real* w1 = W + c1 * ib;
    const real* w2 = W + c2 * ib;
    real a1 = S[t1 + c1 * lds], a2 = S[t2 + c2 * lds];
    if (two) {
#pragma unroll 4
      for (int r = 0; r < ib; ++r) {
        a1 = fma(-V[t1 + r * ldv], w1[r], a1);
        a2 = fma(-V[t2 + r * ldv], w2[r], a2);
      }
      S[t2 + c2 * lds] = a2;
    } else {
#pragma unroll 4
      for (int r = 0; r < ib; ++r) a1 = fma(-V[t1 + r * ldv], w1[r], a1);
    }
    S[t1 + c1 * lds] = a1;
  }
  __syncthreads();
}

// Interchanges of one GETRF block on a slab whose row 0 is the block's first
// row: rows q <-> pv[q] (pv[q] >= q, < rows), in order; one thread per column.
template <typename real>
__device__ void swap_rows_local(real* S, int lds, int rows, int w, const int* pv, int ib) {
  for (int c = threadIdx.x; c < w; c += kThreads) {
    real* col = S + c * lds;
    for (int q = 0; q < ib; ++q) {
      const int r = pv[q];
      if (r > q && r < rows) {
        const real t = col[q];
        col[q] = col[r];
        col[r] = t;
      }
    }
  }
}

// Interchanges of one TSTRF block: top row q <-> bottom row pv[q] (>= 0).
template <typename real>
__device__ void swap_rows_pair(real* Top, int ldt, real* S, int lds, int rows, int w, const int* pv, int ib) {
  for (int c = threadIdx.x; c < w; c += kThreads) {
    real* tc = Top + c * ldt;
    real* sc = S + c * lds;
    for (int q = 0; q < ib; ++q) {
      const int r = pv[q];
      if (r >= 0 && r < rows) {
        const real t = tc[q];
        tc[q] = sc[r];
        sc[r] = t;
      }
    }
  }
}

// Partially pivoted LU of the nr x ib panel P (GETRF's block): pivot rows
// from c .. nr-1 for column c; pv[c] receives the chosen row.
template <typename real>
__device__ void panel_lu(real* P, int ldP, int nr, int ib, int* pv) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int c = 0; c < ib; ++c) {
    real* pc = P + c * ldP;
    if (wid == 0) {
      int r = warp_iamax<real>(pc, c, nr, nullptr);
      if (r >= nr) r = c;
      if (lane == 0) pv[c] = r;
    }
    __syncthreads();
    const int r = pv[c];
    if (r != c)
      for (int d = tid; d < ib; d += kThreads) {
        const real t = P[c + d * ldP];
        P[c + d * ldP] = P[r + d * ldP];
        P[r + d * ldP] = t;
      }
    __syncthreads();
    const real piv = pc[c];
    if (piv != real(0))
      for (int rr = c + 1 + tid; rr < nr; rr += kThreads) pc[rr] = pc[rr] / piv;
    __syncthreads();
    const int ncol = ib - c - 1, nrow = nr - c - 1;
    for (int e = tid; e < ncol * nrow; e += kThreads) {
      const int rr = c + 1 + e % nrow, d = c + 1 + e / nrow;
      P[rr + d * ldP] = fma(-pc[rr], P[c + d * ldP], P[rr + d * ldP]);
    }
    __syncthreads();
  }
}

// Pairwise-pivoted LU of [Rb; P] (Rb: the ib x ib top block, ld ib, upper
// triangular on entry; P: nv x ib bottom rows): for column c the pivot is row
// c of Rb (ties) or the largest bottom row; pv[c] = -1 or that row.  Block
// rows are exchanged whole; only bottom rows are eliminated.
template <typename real>
__device__ void panel_tslu(real* Rb, real* P, int ldP, int nv, int ib, int* pv) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int c = 0; c < ib; ++c) {
    real* pc = P + c * ldP;
    if (wid == 0) {
      unsigned long long best = 0;
      const int r = warp_iamax<real>(pc, 0, nv, &best);
      const bool top = r >= nv || abs_bits(Rb[c + c * ib]) >= best;
      if (lane == 0) pv[c] = top ? -1 : r;
    }
    __syncthreads();
    const int r = pv[c];
    if (r >= 0)
      for (int d = tid; d < ib; d += kThreads) {
        const real t = Rb[c + d * ib];
        Rb[c + d * ib] = P[r + d * ldP];
        P[r + d * ldP] = t;
      }
    __syncthreads();
    const real piv = Rb[c + c * ib];
    if (piv != real(0))
      for (int rr = tid; rr < nv; rr += kThreads) pc[rr] = pc[rr] / piv;
    __syncthreads();
    const int ncol = ib - c - 1;
    for (int e = tid; e < ncol * nv; e += kThreads) {
      const int rr = e % nv, d = c + 1 + e / nv;
      P[rr + d * ldP] = fma(-pc[rr], Rb[c + d * ib], P[rr + d * ldP]);
    }
    __syncthreads();
  }
}

template <typename real>
__device__ __forceinline__ int32_t* piv_ptr(const Inst& I, int i, int k) {
  return I.piv + piv_offset(I.p, I.nb, i, k);
}

// GETRF(k): partially pivoted LU of tile (k, k) in ib blocks.
template <typename real>
__device__ void exec_getrf(Ctx<real>& cx, const Inst& I, int k) {
  const int nb = I.nb, ib = I.ib, cs = I.cs;
  real* A = tile_ptr<real>(I, k, k);
  real* Lg = t_ptr<real>(I, k, k);
  int32_t* pg = piv_ptr<real>(I, k, k);
  int* pv = reinterpret_cast<int*>(cx.red + 2 * kThreads);
  for (int l0 = 0; l0 < nb; l0 += ib) {
    const int nr = nb - l0;
    load_block(cx.P, cx.ldP, A + l0 + static_cast<long long>(l0) * nb, nb, nr, ib);
    __syncthreads();
    panel_lu<real>(cx.P, cx.ldP, nr, ib, pv);
    store_block(A + l0 + static_cast<long long>(l0) * nb, nb, cx.P, cx.ldP, nr, ib);
    if (threadIdx.x < ib) pg[l0 + threadIdx.x] = l0 + pv[threadIdx.x];
    unit_lower_inverse_t<real>(cx.P, cx.ldP, ib, cx.T, cx.ldT);
    __syncthreads();
    store_block(Lg + static_cast<long long>(l0) * ib, ib, cx.T, cx.ldT, ib, ib);
    for (int c0 = l0 + ib; c0 < nb; c0 += cs) {
      const int w = nb - c0 < cs ? nb - c0 : cs;
      load_block(cx.S, cx.ldS, A + l0 + static_cast<long long>(c0) * nb, nb, nr, w);
      __syncthreads();
      swap_rows_local<real>(cx.S, cx.ldS, nr, w, pv, ib);
      __syncthreads();
      apply_block_lu<real>(cx.P + ib, cx.ldP, nr - ib, cx.S, cx.ldS, cx.S + ib, cx.ldS, cx.T, cx.ldT, ib, w, cx.W);
      store_block(A + l0 + static_cast<long long>(c0) * nb, nb, cx.S, cx.ldS, nr, w);
      __syncthreads();
    }
    __syncthreads();
  }
}

// GESSM(k, j, s): slab s of tile (k, j) <- L_kk^-1 P_kk times it.
template <typename real>
__device__ void exec_gessm(Ctx<real>& cx, const Inst& I, int k, int j, int s) {
  const int nb = I.nb, ib = I.ib;
  const real* Lt = tile_ptr<real>(I, k, k);
  const real* Lg = t_ptr<real>(I, k, k);
  const int32_t* pg = piv_ptr<real>(I, k, k);
  int* pv = reinterpret_cast<int*>(cx.red + 2 * kThreads);
  real* C = tile_ptr<real>(I, k, j) + static_cast<long long>(s) * I.cs * nb;
  const int w = slab_width(I, j, s);
  bulk_cols(cx, cx.S, cx.ldS, C, nb, nb, w);
  for (int l0 = 0; l0 < nb; l0 += ib) {
    const int nr = nb - l0, nv = nr - ib;
    // L21 of block l: strictly below the diagonal (TSQRT-like kernels of the
    // same step may rewrite the tile's upper triangle meanwhile)
    for (int e = threadIdx.x; e < nv * ib; e += kThreads) {
      const int r = e % nv, c = e / nv;
      cx.P[r + c * cx.ldP] = ldg_cg(Lt + (l0 + ib + r) + static_cast<long long>(l0 + c) * nb);
    }
    load_block(cx.T, cx.ldT, Lg + static_cast<long long>(l0) * ib, ib, ib, ib);
    if (threadIdx.x < ib) pv[threadIdx.x] = ldg_cg(pg + l0 + threadIdx.x) - l0;
    __syncthreads();
    swap_rows_local<real>(cx.S + l0, cx.ldS, nr, w, pv, ib);
    __syncthreads();
    apply_block_lu<real>(cx.P, cx.ldP, nv, cx.S + l0, cx.ldS, cx.S + l0 + ib, cx.ldS, cx.T, cx.ldT, ib, w, cx.W);
  }
  store_block(C, nb, cx.S, cx.ldS, nb, w);
  __syncthreads();
}

// TSTRF(k, i): pairwise-pivoted LU of [U_kk; A_ik] in ib blocks; with
// rows = 2 the bottom is the 2b x b block of tiles (i, k), (i+1, k) and the
// interchanges index its 2b rows.  Writes U_kk's upper triangle, the
// multipliers in the bottom tiles, the pivots and L11^-1 under row i.
template <typename real>
__device__ void exec_tstrf(Ctx<real>& cx, const Inst& I, int k, int i, int rows = 1) {
  const int nb = I.nb, ib = I.ib, cs = I.cs, nv = rows * nb;
  real* Ut = tile_ptr<real>(I, k, k);
  real* Lg = t_ptr<real>(I, i, k);
  int32_t* pg = piv_ptr<real>(I, i, k);
  int* pv = reinterpret_cast<int*>(cx.red + 2 * kThreads);
  real* Rb = cx.Rb;  // ib x ib, ld ib
  for (int l0 = 0; l0 < nb; l0 += ib) {
    for (int e = threadIdx.x; e < ib * ib; e += kThreads) {
      const int r = e % ib, c = e / ib;
      Rb[r + c * ib] = (r <= c) ? ldg_cg(Ut + (l0 + r) + static_cast<long long>(l0 + c) * nb) : real(0);
    }
    for (int a = 0; a < rows; ++a)
      bulk_cols(cx, cx.P + a * nb, cx.ldP, tile_ptr<real>(I, i + a, k) + static_cast<long long>(l0) * nb, nb, nb, ib);
    __syncthreads();
    panel_tslu<real>(Rb, cx.P, cx.ldP, nv, ib, pv);
    for (int e = threadIdx.x; e < ib * ib; e += kThreads) {
      const int r = e % ib, c = e / ib;
      if (r <= c) Ut[(l0 + r) + static_cast<long long>(l0 + c) * nb] = Rb[r + c * ib];
    }
    for (int a = 0; a < rows; ++a)
      store_block(tile_ptr<real>(I, i + a, k) + static_cast<long long>(l0) * nb, nb, cx.P + a * nb, cx.ldP, nb, ib);
    if (threadIdx.x < ib) pg[l0 + threadIdx.x] = pv[threadIdx.x];
    unit_lower_inverse_t<real>(Rb, ib, ib, cx.T, cx.ldT);
    __syncthreads();
    store_block(Lg + static_cast<long long>(l0) * ib, ib, cx.T, cx.ldT, ib, ib);
    for (int c0 = l0 + ib; c0 < nb; c0 += cs) {
      const int w = nb - c0 < cs ? nb - c0 : cs;
      load_block(cx.Top, ib, Ut + l0 + static_cast<long long>(c0) * nb, nb, ib, w);
      for (int a = 0; a < rows; ++a)
        bulk_cols(cx, cx.S + a * nb, cx.ldS, tile_ptr<real>(I, i + a, k) + static_cast<long long>(c0) * nb, nb, nb, w);
      __syncthreads();
      swap_rows_pair<real>(cx.Top, ib, cx.S, cx.ldS, nv, w, pv, ib);
      __syncthreads();
      apply_block_lu<real>(cx.P, cx.ldP, nv, cx.Top, ib, cx.S, cx.ldS, cx.T, cx.ldT, ib, w, cx.W);
      store_block(Ut + l0 + static_cast<long long>(c0) * nb, nb, cx.Top, ib, ib, w);
      for (int a = 0; a < rows; ++a)
        store_block(tile_ptr<real>(I, i + a, k) + static_cast<long long>(c0) * nb, nb, cx.S + a * nb, cx.ldS, nb, w);
      __syncthreads();
    }
    __syncthreads();
  }
}

// SSSSM(k, i, j, s): slab s of [(k, j); (i .. i+rows-1, j)] <- TSTRF(k, i)'s
// transformations applied to it.
template <typename real>
__device__ void exec_ssssm(Ctx<real>& cx, const Inst& I, int k, int i, int j, int s, int rows = 1) {
  const int nb = I.nb, ib = I.ib, nv = rows * nb;
  const real* Lg = t_ptr<real>(I, i, k);
  const int32_t* pg = piv_ptr<real>(I, i, k);
  int* pv = reinterpret_cast<int*>(cx.red + 2 * kThreads);
  const long long soff = static_cast<long long>(s) * I.cs * nb;
  real* Ct = tile_ptr<real>(I, k, j) + soff;
  const int w = slab_width(I, j, s);
  const uint32_t cb = static_cast<uint32_t>(nb) * sizeof(real);
  // each block's L pieces go out as one bulk phase before its other loads,
  // so the copy and the loads overlap (the first phase also carries the
  // bottom slabs)
  for (int l0 = 0; l0 < nb; l0 += ib) {
    if (threadIdx.x < 32) {
      bulk_expect(cx, cb * rows * (ib + (l0 == 0 ? w : 0)));
      __syncwarp();
      if (l0 == 0)
        for (int a = 0; a < rows; ++a)
          bulk_issue_cols(cx, cx.S + a * nb, cx.ldS, tile_ptr<real>(I, i + a, j) + soff, nb, nb, w);
      for (int a = 0; a < rows; ++a)
        bulk_issue_cols(cx, cx.P + a * nb, cx.ldP, tile_ptr<real>(I, i + a, k) + static_cast<long long>(l0) * nb,
                        nb, nb, ib);
    }
    load_block(cx.T, cx.ldT, Lg + static_cast<long long>(l0) * ib, ib, ib, ib);
    load_block(cx.Top, ib, Ct + l0, nb, ib, w);
    if (threadIdx.x < ib) pv[threadIdx.x] = ldg_cg(pg + l0 + threadIdx.x);
    bulk_wait(cx);
    __syncthreads();
    swap_rows_pair<real>(cx.Top, ib, cx.S, cx.ldS, nv, w, pv, ib);
    __syncthreads();
    apply_block_lu<real>(cx.P, cx.ldP, nv, cx.Top, ib, cx.S, cx.ldS, cx.T, cx.ldT, ib, w, cx.W);
    store_block(Ct + l0, nb, cx.Top, ib, ib, w);
    __syncthreads();
  }
  for (int a = 0; a < rows; ++a) store_block(tile_ptr<real>(I, i + a, j) + soff, nb, cx.S + a * nb, cx.ldS, nb, w);
  __syncthreads();
}

// ---------------------------------------------------------------- scheduler
// Thread 0 waits until every counter of every wait has reached its version.
template <bool PAIR>
__device__ __forceinline__ int device_rules(const Inst& I, const TaskX& t, Wait* w, Signal* sg, int* nsig) {
  if constexpr (PAIR)
    return task_rules(I, t, w, sg, nsig);
  else
    return task_rules_base(I, t, w, sg, nsig);
}

template <typename real, bool PAIR>
__device__ bool wait_deps(Ctx<real>& cx, const Inst& I, const TaskX& t) {
  Wait w[kMaxWaits];
  Signal sg[kMaxSignals];
  int nsig;
  const int nw = device_rules<PAIR>(I, t, w, sg, &nsig);
  unsigned long long t0 = 0;
  for (int a = 0; a < nw; ++a) {
    for (int c = 0; c < w[a].cnt; ++c) {
      const int* ctr = I.ver + w[a].ctr + c;
      if (ld_acquire(ctr) >= w[a].ver) continue;
      if (t0 == 0) t0 = gtimer();
      unsigned ns = 32;
      while (ld_acquire(ctr) < w[a].ver) {
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
        if (ld_relaxed(&cx.ctl->error) != 0) return false;
        if ((long long)(gtimer() - t0) > cx.limit_ns) {
          set_error(cx, 1);
          return false;
        }
      }
    }
  }
  return true;
}

template <bool PAIR>
__device__ void signal_done(const Inst& I, const TaskX& t) {
  Wait w[kMaxWaits];
  Signal sg[kMaxSignals];
  int nsig;
  device_rules<PAIR>(I, t, w, sg, &nsig);
  __threadfence();
  for (int a = 0; a < nsig; ++a)
    for (int c = 0; c < sg[a].cnt; ++c) atomicAdd(I.ver + sg[a].ctr + c, 1);
}

// The persistent task loop.  LU: the tiled LU's kernel (its own kernel, so
// the LU tile kernels do not enter the QR kernel's register allocation).
enum KernelVariant { KV_QR = 0, KV_LU = 1, KV_PAIR = 2 };

template <typename real, int V>
__device__ __forceinline__ void task_loop(const TaskX* __restrict__ tasks, int ntasks, const Inst* __restrict__ insts,
                                          Ctl* ctl, long long limit_ns) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ TaskX s_task;
  __shared__ Inst s_inst;
  __shared__ int s_go;

  Ctx<real> cx;
  cx.task = 0;
  cx.ctl = ctl;
  cx.limit_ns = limit_ns;
  cx.phase = 0;
  int cur_nb = -1, cur_ib = -1, cur_cs = -1, cur_pair = -1;
  int cur_inst = -1;  // thread 0: index of the descriptor held in s_inst (fixed during a launch)
  if (threadIdx.x == 0) {
    // the barrier sits at the end of the largest layout; its offset is passed
    // through the kernel's dynamic size
    uint32_t dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    mbar_init(smem_u32(smem + dyn - 16), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    uint32_t dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    cx.bar = smem_u32(smem + dyn - 16);
  }
  __syncthreads();

  while (true) {
    if (threadIdx.x == 0) {
      int go = 0;
      if (ld_relaxed(&ctl->error) == 0) {
        const int t = atomicAdd(&ctl->next, 1);
        if (t < ntasks) {
          const unsigned long long t_ticket = g_trace != nullptr ? gtimer() : 0ull;
          s_task = tasks[t];
          if (s_task.inst != cur_inst) {
            s_inst = insts[s_task.inst];
            cur_inst = s_task.inst;
          }
          cx.task = t;
          go = wait_deps<real, V != KV_QR>(cx, s_inst, s_task) ? 1 : 0;
          if (go) trace_begin(t, t_ticket, s_task);
        }
      }
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const TaskX t = s_task;
    const Inst& I = s_inst;
    if (I.nb != cur_nb || I.ib != cur_ib || I.cs != cur_cs || I.pair != cur_pair) {
      const SmemLayout L = smem_layout(I.nb, I.ib, I.cs, sizeof(real), I.pair ? 2 * I.nb : 0);
      cx.P = reinterpret_cast<real*>(smem + L.oP);
      cx.P2 = L.oP2 >= 0 ? reinterpret_cast<real*>(smem + L.oP2) : nullptr;
      cx.TopS = L.oTopS >= 0 ? reinterpret_cast<real*>(smem + L.oTopS) : nullptr;
      cx.Tst = L.oTst >= 0 ? reinterpret_cast<real*>(smem + L.oTst) : nullptr;
      cx.T = reinterpret_cast<real*>(smem + L.oT);
      cx.S = reinterpret_cast<real*>(smem + L.oS);
      cx.Top = reinterpret_cast<real*>(smem + L.oTop);
      cx.W = reinterpret_cast<real*>(smem + L.oW);
      cx.red = reinterpret_cast<double*>(smem + L.oRed);
      cx.Part = reinterpret_cast<real*>(smem + L.oPart);
      cx.Rb = L.r_in_s ? cx.S : cx.Top;
      cx.nb = I.nb;
      cx.ib = I.ib;
      cx.cs = I.cs;
      cx.ldP = ld_pad(I.pair ? 2 * I.nb : I.nb, sizeof(real));
      cx.ldS = cx.ldP;
      cx.ldT = I.ib + 1;
      cur_nb = I.nb;
      cur_ib = I.ib;
      cur_cs = I.cs;
      cur_pair = I.pair;
    }
    if constexpr (V == KV_PAIR) {
      switch (t.kind) {
        case K_GEQRT: exec_geqrt(cx, I, t.k, t.i); break;
        case K_LARFB: exec_larfb(cx, I, t.k, t.i, t.j, t.s, true); break;
        case K_LARFB_N: exec_larfb(cx, I, t.k, t.i, t.j, t.s, false); break;
        case K_TSQRT2: exec_tsqrt2(cx, I, t.k, t.i, t.l); break;
        case K_SSRFB2: exec_ssrfb2(cx, I, t.k, t.i, t.l, t.j, t.s, true); break;
        case K_SSRFB2_N: exec_ssrfb2(cx, I, t.k, t.i, t.l, t.j, t.s, false); break;
        case K_TRSM_UPD: exec_trsm_upd(cx, I, t.k, t.l, t.j, t.s); break;
        case K_TRSM_SOLVE: exec_trsm_solve(cx, I, t.k, t.j, t.s); break;
        case K_TRSMT_UPD: exec_trsmt_upd(cx, I, t.k, t.l, t.j, t.s); break;
        case K_TRSMT_SOLVE: exec_trsmt_solve(cx, I, t.k, t.j, t.s); break;
        default: fail_kind(cx); break;
      }
    } else if constexpr (V == KV_LU) {
      switch (t.kind) {
        case K_GETRF: exec_getrf(cx, I, t.k); break;
        case K_GESSM: exec_gessm(cx, I, t.k, t.j, t.s); break;
        case K_TSTRF: exec_tstrf(cx, I, t.k, t.i); break;
        case K_SSSSM: exec_ssssm(cx, I, t.k, t.i, t.j, t.s); break;
        case K_TSTRF2: exec_tstrf(cx, I, t.k, t.i, t.l); break;
        case K_SSSSM2: exec_ssssm(cx, I, t.k, t.i, t.j, t.s, t.l); break;
        case K_TRSM_UPD: exec_trsm_upd(cx, I, t.k, t.l, t.j, t.s); break;
        case K_TRSM_SOLVE: exec_trsm_solve(cx, I, t.k, t.j, t.s); break;
        default: fail_kind(cx); break;
      }
    } else switch (t.kind) {
      case K_GEQRT: exec_geqrt(cx, I, t.k, t.i); break;
      case K_TSQRT: exec_tsqrt(cx, I, t.k, I.D > 0 ? t.l : t.k, t.i, false); break;
      case K_LARFB: exec_larfb(cx, I, t.k, t.i, t.j, t.s, true); break;
      case K_LARFB_N: exec_larfb(cx, I, t.k, t.i, t.j, t.s, false); break;
      case K_SSRFB: exec_ssrfb(cx, I, t.k, I.D > 0 ? t.l : t.k, t.i, t.j, t.s, true, false); break;
      case K_SSRFB_N: exec_ssrfb(cx, I, t.k, I.D > 0 ? t.l : t.k, t.i, t.j, t.s, false, false); break;
      case K_TTQRT: exec_tsqrt(cx, I, t.k, t.l, t.i, true); break;
      case K_TTMQR: exec_ssrfb(cx, I, t.k, t.l, t.i, t.j, t.s, true, true); break;
      case K_TTMQR_N: exec_ssrfb(cx, I, t.k, t.l, t.i, t.j, t.s, false, true); break;
      case K_TRSM_UPD: exec_trsm_upd(cx, I, t.k, t.l, t.j, t.s); break;
      case K_TRSM_SOLVE: exec_trsm_solve(cx, I, t.k, t.j, t.s); break;
      case K_TRSMT_UPD: exec_trsmt_upd(cx, I, t.k, t.l, t.j, t.s); break;
      case K_TRSMT_SOLVE: exec_trsmt_solve(cx, I, t.k, t.j, t.s); break;
      default: fail_kind(cx); break;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      trace_end(cx.task);
      signal_done<V != KV_QR>(I, t);
    }
  }
}

template <typename real>
__global__ void __launch_bounds__(kThreads, 2) run_tasks_kernel(const TaskX* __restrict__ tasks, int ntasks,
                                                             const Inst* __restrict__ insts, Ctl* ctl,
                                                             long long limit_ns) {
  task_loop<real, KV_QR>(tasks, ntasks, insts, ctl, limit_ns);
}

template <typename real>
__global__ void __launch_bounds__(kThreads, 2) run_lu_tasks_kernel(const TaskX* __restrict__ tasks, int ntasks,
                                                                   const Inst* __restrict__ insts, Ctl* ctl,
                                                                   long long limit_ns) {
  task_loop<real, KV_LU>(tasks, ntasks, insts, ctl, limit_ns);
}

// 2b x b bottoms: GEQRT / LARFB with the paired TS kernels.
template <typename real>
__global__ void __launch_bounds__(kThreads) run_pair_tasks_kernel(const TaskX* __restrict__ tasks, int ntasks,
                                                                  const Inst* __restrict__ insts, Ctl* ctl,
                                                                  long long limit_ns) {
  task_loop<real, KV_PAIR>(tasks, ntasks, insts, ctl, limit_ns);
}

// ---------------------------------------------------------------- BDL
// Column-major (ld) -> Block Data Layout tiles (Section 3.4), zero padded.
// One warp per tile column: the column's rows are contiguous both in the
// caller's matrix and in the tile, so lanes walk consecutive addresses on
// both sides, and the tile coordinates cost one division per column rather
// than per element.
template <typename S, typename D>
__global__ void pack_kernel(const S* __restrict__ A, long long lda, int m, int n, D* __restrict__ Ab, int p,
                            int q, int nb) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  const long long units = static_cast<long long>(p) * q * nb;  // tile columns
  for (long long u = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5; u < units;
       u += nwarps) {
    const long long t = u / nb;
    const int c = static_cast<int>(u - t * nb);
    const int ti = static_cast<int>(t % p), tj = static_cast<int>(t / p);
    const long long gj = static_cast<long long>(tj) * nb + c, gi0 = static_cast<long long>(ti) * nb;
    int valid = 0;
    if (gj < n) {
      const long long v = m - gi0;
      valid = v <= 0 ? 0 : (v >= nb ? nb : static_cast<int>(v));
    }
    const S* src = A + gi0 + gj * lda;
    D* dst = Ab + t * nb * static_cast<long long>(nb) + static_cast<long long>(c) * nb;
    bool bad = false;
#pragma unroll 4
    for (int r = lane; r < nb; r += 32) {
      const S v = r < valid ? src[r] : S(0);
      bad = bad || !isfinite(v);
      dst[r] = static_cast<D>(v);
    }
    // a NaN or an infinity in the input: the sticky device status reports
    // TQR_ERR_NONFINITE (9) to the call (host buffers) or tqr_stream_status
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicCAS(&g_status, 0, 9);
  }
}

template <typename S, typename D>
__global__ void unpack_kernel(const S* __restrict__ Ab, int p, int nb, D* __restrict__ A, long long lda, int m,
                              int n) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  const int q = (n + nb - 1) / nb;
  const long long units = static_cast<long long>(p) * q * nb;  // tile columns
  for (long long u = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5; u < units;
       u += nwarps) {
    const long long t = u / nb;
    const int c = static_cast<int>(u - t * nb);
    const int ti = static_cast<int>(t % p), tj = static_cast<int>(t / p);
    const long long gj = static_cast<long long>(tj) * nb + c, gi0 = static_cast<long long>(ti) * nb;
    if (gj >= n || gi0 >= m) continue;
    const long long v = m - gi0;
    const int valid = v >= nb ? nb : static_cast<int>(v);
    const S* src = Ab + t * nb * static_cast<long long>(nb) + static_cast<long long>(c) * nb;
    D* dst = A + gi0 + gj * lda;
#pragma unroll 4
    for (int r = lane; r < valid; r += 32) dst[r] = static_cast<D>(src[r]);
  }
}

// Batched pack/unpack: blockIdx.y (strided) picks the matrix, blockIdx.x
// and the threads stride over its elements.
template <typename D>
__global__ void pack_batched_kernel(const PackDesc* __restrict__ descs, int count, int* __restrict__ bad) {
  for (int b = blockIdx.y; b < count; b += gridDim.y) {
    const PackDesc d = descs[b];
    const long long nb2 = static_cast<long long>(d.nb) * d.nb;
    const long long total = nb2 * d.p * d.q;
    D* Ab = static_cast<D*>(d.Ab);
    bool nonfinite = false;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
      const long long tile = e / nb2;
      const int rem = static_cast<int>(e - tile * nb2);
      const int r = rem % d.nb, c = rem / d.nb;
      const int ti = static_cast<int>(tile % d.p), tj = static_cast<int>(tile / d.p);
      const long long gi = static_cast<long long>(ti) * d.nb + r, gj = static_cast<long long>(tj) * d.nb + c;
      const double v = (gi < d.m && gj < d.n) ? d.A[gi + gj * d.lda] : 0.0;
      nonfinite = nonfinite || !isfinite(v);
      Ab[e] = static_cast<D>(v);
    }
    // a NaN or an infinity in matrix b: its status (the same value from
    // every thread that saw one)
    if (nonfinite && bad != nullptr) bad[b] = 9;  // TQR_ERR_NONFINITE
  }
}

template <typename S>
__global__ void unpack_batched_kernel(const PackDesc* __restrict__ descs, int count) {
  for (int b = blockIdx.y; b < count; b += gridDim.y) {
    const PackDesc d = descs[b];
    const long long total = static_cast<long long>(d.m) * d.n;
    const S* Ab = static_cast<const S*>(d.Ab);
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
      const int gi = static_cast<int>(e % d.m), gj = static_cast<int>(e / d.m);
      const int ti = gi / d.nb, r = gi - ti * d.nb;
      const int tj = gj / d.nb, c = gj - tj * d.nb;
      d.A[gi + static_cast<long long>(gj) * d.lda] = static_cast<double>(
          Ab[(static_cast<long long>(ti) + static_cast<long long>(tj) * d.p) * d.nb * d.nb +
             static_cast<long long>(c) * d.nb + r]);
    }
  }
}

// Transposed operands (right-hand application C op(Q) = (op(Q)^T C^T)^T):
// X = C^T, mt x nt with X(a, b) = C[b + a*ldc], goes into BDL tiles (p x q,
// zero padded) and comes back the same way.  32 x 32 blocks pass through
// shared memory so that both C (along b) and the tiles (along a) are
// accessed with consecutive lanes on consecutive addresses.  256 threads:
// lane tx = threadIdx.x % 32, row group ty = threadIdx.x / 32 (8 groups).
template <typename D>
__global__ void pack_t_kernel(const double* __restrict__ C, long long ldc, int mt, int nt, D* __restrict__ Ab,
                              int p, int q, int nb) {
  __shared__ double tile[32][33];
  const long long rows = static_cast<long long>(p) * nb, cols = static_cast<long long>(q) * nb;
  const long long ba = (rows + 31) / 32, bb = (cols + 31) / 32;
  const long long nb2 = static_cast<long long>(nb) * nb;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (long long blk = blockIdx.x; blk < ba * bb; blk += gridDim.x) {
    const long long a0 = (blk % ba) * 32, b0 = (blk / ba) * 32;
    for (int r = ty; r < 32; r += 8) {
      const long long a = a0 + r, b = b0 + tx;
      tile[r][tx] = (a < mt && b < nt) ? C[b + a * ldc] : 0.0;   // X(a0 + r, b0 + tx)
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const long long a = a0 + tx, b = b0 + r;
      if (a < rows && b < cols) {
        const long long ti = a / nb, tj = b / nb;
        Ab[(ti + tj * p) * nb2 + (b - tj * nb) * nb + (a - ti * nb)] = static_cast<D>(tile[tx][r]);
      }
    }
    __syncthreads();
  }
}

template <typename S>
__global__ void unpack_t_kernel(const S* __restrict__ Ab, int p, int nb, double* __restrict__ C, long long ldc,
                                int mt, int nt) {
  __shared__ double tile[32][33];
  const long long ba = (static_cast<long long>(mt) + 31) / 32, bb = (static_cast<long long>(nt) + 31) / 32;
  const long long nb2 = static_cast<long long>(nb) * nb;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (long long blk = blockIdx.x; blk < ba * bb; blk += gridDim.x) {
    const long long a0 = (blk % ba) * 32, b0 = (blk / ba) * 32;
    for (int r = ty; r < 32; r += 8) {
      const long long a = a0 + tx, b = b0 + r;
      double v = 0.0;
      if (a < mt && b < nt) {
        const long long ti = a / nb, tj = b / nb;
        v = static_cast<double>(Ab[(ti + tj * p) * nb2 + (b - tj * nb) * nb + (a - ti * nb)]);
      }
      tile[r][tx] = v;                                            // X(a0 + tx, b0 + r)
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const long long a = a0 + r, b = b0 + tx;
      if (a < mt && b < nt) C[b + a * ldc] = tile[tx][r];
    }
    __syncthreads();
  }
}

// The leading ncols columns of the m x m identity in BDL (p x q tiles).
template <typename D>
__global__ void identity_kernel(int m, int ncols, D* __restrict__ Ab, int p, int q, int nb) {
  const long long nb2 = static_cast<long long>(nb) * nb;
  const long long total = nb2 * p * q;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long tile = e / nb2;
    const int rem = static_cast<int>(e - tile * nb2);
    const int r = rem % nb, c = rem / nb;
    const long long gi = (tile % p) * nb + r, gj = (tile / p) * nb + c;
    Ab[e] = (gi == gj && gi < m && gj < ncols) ? D(1) : D(0);
  }
}

__global__ void status_reset_kernel() { g_status = 0; }

// A launch's error record into out[0..7] (code, where, and the failing
// task's kind, k, i, j, s, l) unless out[0] already holds one.  Runs after
// the launch on its stream, so the record belongs to that launch alone
// (g_status is shared by every launch on the device).
__global__ void fold_error_kernel(const Ctl* ctl, const TaskX* tasks, int ntasks, double* out) {
  const int e = ctl->error;
  if (e == 0 || out[0] != 0.0) return;
  out[0] = e;
  out[1] = ctl->err_where;
  const int t = ctl->err_task;
  if (t >= 0 && t < ntasks) {
    const TaskX x = tasks[t];
    out[2] = x.kind;
    out[3] = x.k;
    out[4] = x.i;
    out[5] = x.j;
    out[6] = x.s;
    out[7] = x.l;
  }
}

cudaError_t launch_fold_error(const void* ctl, const TaskX* tasks, int ntasks, double* out, cudaStream_t st) {
  fold_error_kernel<<<1, 1, 0, st>>>(static_cast<const Ctl*>(ctl), tasks, ntasks, out);
  return cudaGetLastError();
}

cudaError_t set_trace(void* buffer, long long capacity) {
  unsigned long long* b = static_cast<unsigned long long*>(buffer);
  const long long cap = buffer != nullptr ? capacity : 0;
  cudaError_t e = cudaMemcpyToSymbol(g_trace, &b, sizeof(b));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_trace_cap, &cap, sizeof(cap));
  return e;
}

// ---------------------------------------------------------------- host launchers
static int grid_for(long long work, int sms) {
  long long g = (work + 255) / 256;
  long long cap = static_cast<long long>(sms) * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

// Warp-per-tile-column copies: 8 warps per block, up to 16 blocks per SM.
static int grid_for_columns(long long columns, int sms) {
  long long g = (columns + 7) / 8;
  const long long cap = static_cast<long long>(sms) * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

template <typename real>
cudaError_t launch_pack(const double* A, long long lda, int m, int n, real* Ab, int p, int q, int nb, int sms,
                        cudaStream_t st) {
  const long long columns = static_cast<long long>(p) * q * nb;
  pack_kernel<double, real><<<grid_for_columns(columns, sms), 256, 0, st>>>(A, lda, m, n, Ab, p, q, nb);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_unpack(const real* Ab, int p, int nb, double* A, long long lda, int m, int n, int sms,
                          cudaStream_t st) {
  if (static_cast<long long>(m) * n == 0) return cudaSuccess;
  const long long columns = static_cast<long long>(p) * ((n + nb - 1) / nb) * nb;
  unpack_kernel<real, double><<<grid_for_columns(columns, sms), 256, 0, st>>>(Ab, p, nb, A, lda, m, n);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_pack_t(const double* C, long long ldc, int mt, int nt, real* Ab, int p, int q, int nb, int sms,
                          cudaStream_t st) {
  const long long blocks = ((static_cast<long long>(p) * nb + 31) / 32) * ((static_cast<long long>(q) * nb + 31) / 32);
  const long long cap = static_cast<long long>(sms) * 8;
  pack_t_kernel<real><<<static_cast<int>(blocks < cap ? blocks : cap), 256, 0, st>>>(C, ldc, mt, nt, Ab, p, q, nb);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_unpack_t(const real* Ab, int p, int nb, double* C, long long ldc, int mt, int nt, int sms,
                            cudaStream_t st) {
  if (static_cast<long long>(mt) * nt == 0) return cudaSuccess;
  const long long blocks = ((static_cast<long long>(mt) + 31) / 32) * ((static_cast<long long>(nt) + 31) / 32);
  const long long cap = static_cast<long long>(sms) * 8;
  unpack_t_kernel<real><<<static_cast<int>(blocks < cap ? blocks : cap), 256, 0, st>>>(Ab, p, nb, C, ldc, mt, nt);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_identity(int m, int ncols, real* Ab, int p, int q, int nb, int sms, cudaStream_t st) {
  const long long total = static_cast<long long>(nb) * nb * p * q;
  identity_kernel<real><<<grid_for(total, sms), 256, 0, st>>>(m, ncols, Ab, p, q, nb);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_pack_batched(const PackDesc* d, int count, cudaStream_t st, int* bad) {
  if (count <= 0) return cudaSuccess;
  dim3 grid(8, count < 65535 ? count : 65535);
  pack_batched_kernel<real><<<grid, 256, 0, st>>>(d, count, bad);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_unpack_batched(const PackDesc* d, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  dim3 grid(8, count < 65535 ? count : 65535);
  unpack_batched_kernel<real><<<grid, 256, 0, st>>>(d, count);
  return cudaGetLastError();
}

// The kernel's dynamic shared-memory limit is set to the largest value the
// device allows (its opt-in per-block maximum minus the kernel's static
// shared memory), the same value on every call: launches from several host
// threads with different tile shapes must not lower it under one another.
// Occupancy follows each launch's own size, not this limit.
template <typename real>
static const void* task_kernel(int variant) {
  if (variant == KV_LU) return reinterpret_cast<const void*>(run_lu_tasks_kernel<real>);
  if (variant == KV_PAIR) return reinterpret_cast<const void*>(run_pair_tasks_kernel<real>);
  return reinterpret_cast<const void*>(run_tasks_kernel<real>);
}

template <typename real>
cudaError_t max_dyn_smem(int* out, int lu) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, task_kernel<real>(lu));
  if (e != cudaSuccess) return e;
  *out = optin - static_cast<int>(fa.sharedSizeBytes);
  return cudaSuccess;
}

template <typename real>
cudaError_t set_max_dyn_smem(int smem_bytes, int lu) {
  int mx = 0;
  cudaError_t e = max_dyn_smem<real>(&mx, lu);
  if (e != cudaSuccess) return e;
  if (smem_bytes > mx) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(task_kernel<real>(lu), cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

template <typename real>
cudaError_t launch_run(const TaskX* tasks, int ntasks, const Inst* insts, void* ctl, long long limit_ns, int grid,
                       int smem_bytes, cudaStream_t st, int variant) {
  cudaError_t e = set_max_dyn_smem<real>(smem_bytes, variant);
  if (e != cudaSuccess) return e;
  if (variant == KV_LU)
    run_lu_tasks_kernel<real><<<grid, kThreads, smem_bytes, st>>>(tasks, ntasks, insts, static_cast<Ctl*>(ctl),
                                                                  limit_ns);
  else if (variant == KV_PAIR)
    run_pair_tasks_kernel<real><<<grid, kThreads, smem_bytes, st>>>(tasks, ntasks, insts, static_cast<Ctl*>(ctl),
                                                                    limit_ns);
  else
    run_tasks_kernel<real><<<grid, kThreads, smem_bytes, st>>>(tasks, ntasks, insts, static_cast<Ctl*>(ctl), limit_ns);
  return cudaGetLastError();
}

template <typename real>
cudaError_t occupancy(int smem_bytes, int* blocks_per_sm) {
  cudaError_t e = set_max_dyn_smem<real>(smem_bytes, KV_QR);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, run_tasks_kernel<real>, kThreads, smem_bytes);
  if (e != cudaSuccess || sizeof(real) != 8) return e;
  // the LU instantiation (FP64 only) must fit the same number of CTAs
  int lu_blocks = 0;
  e = set_max_dyn_smem<real>(smem_bytes, KV_LU);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lu_blocks, run_lu_tasks_kernel<real>, kThreads, smem_bytes);
  if (e == cudaSuccess && lu_blocks < *blocks_per_sm) *blocks_per_sm = lu_blocks;
  return e;
}

cudaError_t read_status(int* status, cudaStream_t st) {
  cudaError_t e = cudaMemcpyFromSymbolAsync(status, g_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  status_reset_kernel<<<1, 1, 0, st>>>();
  return cudaGetLastError();
}

size_t ctl_bytes() { return sizeof(Ctl); }

// Register-resident DFMA chains: 8 independent FMAs per iteration per thread.
__global__ void dfma_probe_kernel(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

cudaError_t fp64_peak(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 4, iters = 4000;
  double* out = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&out), sizeof(double) * threads * blocks, st);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dfma_probe_kernel<<<blocks, threads, 0, st>>>(out, 100, 0.999, 1e-3);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    dfma_probe_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.999, 1e-3);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  cudaStreamSynchronize(st);
  *tflops = 2.0 * 8.0 * iters * static_cast<double>(blocks) * threads / (best * 1e-3) / 1e12;
  return e;
}

template cudaError_t launch_pack<double>(const double*, long long, int, int, double*, int, int, int, int,
                                         cudaStream_t);
template cudaError_t launch_pack<float>(const double*, long long, int, int, float*, int, int, int, int,
                                        cudaStream_t);
template cudaError_t launch_unpack<double>(const double*, int, int, double*, long long, int, int, int,
                                           cudaStream_t);
template cudaError_t launch_unpack<float>(const float*, int, int, double*, long long, int, int, int, cudaStream_t);
template cudaError_t launch_run<double>(const TaskX*, int, const Inst*, void*, long long, int, int, cudaStream_t,
                                        int);
template cudaError_t launch_run<float>(const TaskX*, int, const Inst*, void*, long long, int, int, cudaStream_t,
                                       int);
template cudaError_t occupancy<double>(int, int*);
template cudaError_t launch_pack_t<double>(const double*, long long, int, int, double*, int, int, int, int,
                                           cudaStream_t);
template cudaError_t launch_unpack_t<double>(const double*, int, int, double*, long long, int, int, int,
                                             cudaStream_t);
template cudaError_t launch_identity<double>(int, int, double*, int, int, int, int, cudaStream_t);
template cudaError_t launch_identity<float>(int, int, float*, int, int, int, int, cudaStream_t);
template cudaError_t launch_pack_batched<double>(const PackDesc*, int, cudaStream_t, int*);
template cudaError_t launch_unpack_batched<double>(const PackDesc*, int, cudaStream_t);
template cudaError_t occupancy<float>(int, int*);

}  // namespace tqr
