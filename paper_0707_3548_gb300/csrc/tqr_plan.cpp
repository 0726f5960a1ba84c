// tqr_plan.cpp -- host-side task lists, DAG derivation and list-scheduling
// order (see tqr_plan.h).
#include "tqr_plan.h"

#include <algorithm>
#include <queue>
#include <utility>

namespace tqr {

static TaskX mk(int kind, int inst, int k, int i, int j, int s, int l = 0) {
  TaskX t;
  t.kind = kind;
  t.s = s;
  t.inst = inst;
  t.k = k;
  t.i = i;
  t.j = j;
  t.l = l;
  t.pad = 0;
  return t;
}

// Reduction-tree variant: Algorithm 1's step k with the rows cut into
// domains (GEQRT on each head, TSQRT/SSRFB of the head with each later row of
// its domain) followed by the binary tree of TT merges of the heads.  `cols`
// selects the updated tile columns: all j > k (factor) or only the
// right-hand-side columns (apply).
static void tree_step(const Inst& I, int x, int k, bool factor, std::vector<TaskX>& out) {
  const int p = I.p, D = I.D, qt = I.q + I.qb;
  const int j0 = factor ? k + 1 : I.q;
  std::vector<int> heads;
  for (int h = k; h < p; h += D) heads.push_back(h);
  for (int h : heads) {
    if (factor) out.push_back(mk(K_GEQRT, x, k, h, k, 0));
    for (int j = j0; j < qt; ++j)
      for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_LARFB, x, k, h, j, s));
    for (int i = h + 1; i < h + D && i < p; ++i) {
      if (factor) out.push_back(mk(K_TSQRT, x, k, i, k, 0, h));
      for (int j = j0; j < qt; ++j)
        for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_SSRFB, x, k, i, j, s, h));
    }
  }
  const int H = static_cast<int>(heads.size());
  for (int L = 0; (1 << L) < H; ++L)
    for (int d = 0; d + (1 << L) < H; d += (2 << L)) {
      const int a = heads[d], b = heads[d + (1 << L)];
      if (factor) out.push_back(mk(K_TTQRT, x, k, b, k, 0, a));
      for (int j = j0; j < qt; ++j)
        for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_TTMQR, x, k, b, j, s, a));
    }
}

static void trsm_tasks(const Inst& I, int x, std::vector<TaskX>& out) {
  const int q = I.q, kt = I.kt, qt = I.q + I.qb;
  for (int j = q; j < qt; ++j)
    for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s)
      for (int k = kt - 1; k >= 0; --k) {
        for (int l = kt - 1; l > k; --l) out.push_back(mk(K_TRSM_UPD, x, k, k, j, s, l));
        out.push_back(mk(K_TRSM_SOLVE, x, k, k, j, s));
      }
}

static bool tree_seq(const Inst& I, int x, std::vector<TaskX>& out) {
  if (I.D <= 0) return false;
  switch (I.mode) {
    case M_FACTOR:
      for (int k = 0; k < I.kt; ++k) tree_step(I, x, k, true, out);
      if (I.trsm) trsm_tasks(I, x, out);
      return true;
    case M_APPLY_QT:
      for (int k = 0; k < I.kt; ++k) tree_step(I, x, k, false, out);
      if (I.trsm) trsm_tasks(I, x, out);
      return true;
    case M_APPLY_Q:
    case M_FORM_Q: {
      // the transposed updates in exactly the reverse order; explicit Q
      // columns skip the steps after their own tile column
      std::vector<TaskX> fw;
      for (int k = 0; k < I.kt; ++k) tree_step(I, x, k, false, fw);
      for (size_t a = fw.size(); a-- > 0;) {
        TaskX t = fw[a];
        if (I.mode == M_FORM_Q && t.j - I.q < t.k) continue;
        t.kind = t.kind == K_LARFB ? K_LARFB_N : t.kind == K_SSRFB ? K_SSRFB_N : K_TTMQR_N;
        out.push_back(t);
      }
      return true;
    }
    default:
      return false;  // triangular solves do not depend on the tree
  }
}

void tree_table(const Inst& I, std::vector<int32_t>& vt) {
  vt.assign(static_cast<size_t>(I.kt + 1) * I.p, 0);
  for (int k = 0; k < I.kt; ++k)
    for (int r = 0; r < I.p; ++r)
      vt[static_cast<size_t>(k + 1) * I.p + r] =
          vt[static_cast<size_t>(k) * I.p + r] + (r >= k ? tree_writes(I, k, r) : 0);
}

static void seq_tasks_qr(const Inst& I, int x, std::vector<TaskX>& out);

// LU task lists are the QR ones (flat panel) with the LU kinds substituted.
void seq_tasks(const Inst& I, int x, std::vector<TaskX>& out) {
  const size_t first = out.size();
  seq_tasks_qr(I, x, out);
  if (I.lu)
    for (size_t a = first; a < out.size(); ++a) out[a].kind = lu_kind(out[a].kind);
}

// 2b x b bottoms: Algorithm 1 with the rows below the diagonal tile taken in
// groups of two (the last may be one).  Task field l holds the group size.
static void pair_step(const Inst& I, int x, int k, bool factor, std::vector<TaskX>& out) {
  const int p = I.p, qt = I.q + I.qb;
  const int j0 = factor ? k + 1 : I.q;
  if (factor) out.push_back(mk(K_GEQRT, x, k, k, k, 0));
  for (int j = j0; j < qt; ++j)
    for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_LARFB, x, k, k, j, s));
  for (int h = k + 1; h < p; h += 2) {
    const int l = h + 1 < p ? 2 : 1;
    if (factor) out.push_back(mk(K_TSQRT2, x, k, h, k, 0, l));
    for (int j = j0; j < qt; ++j)
      for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_SSRFB2, x, k, h, j, s, l));
  }
}

static bool pair_seq(const Inst& I, int x, std::vector<TaskX>& out) {
  if (!I.pair) return false;
  switch (I.mode) {
    case M_FACTOR:
    case M_APPLY_QT:
      for (int k = 0; k < I.kt; ++k) pair_step(I, x, k, I.mode == M_FACTOR, out);
      if (I.trsm) trsm_tasks(I, x, out);
      return true;
    case M_APPLY_Q: {
      std::vector<TaskX> fw;
      for (int k = 0; k < I.kt; ++k) pair_step(I, x, k, false, fw);
      for (size_t a = fw.size(); a-- > 0;) {
        TaskX t = fw[a];
        t.kind = t.kind == K_LARFB ? K_LARFB_N : K_SSRFB2_N;
        out.push_back(t);
      }
      return true;
    }
    default:
      return false;  // triangular solves do not depend on the pairing
  }
}

static void seq_tasks_qr(const Inst& I, int x, std::vector<TaskX>& out) {
  if (tree_seq(I, x, out)) return;
  if (pair_seq(I, x, out)) return;
  const int p = I.p, q = I.q, kt = I.kt, qt = I.q + I.qb;
  switch (I.mode) {
    case M_FACTOR:
      // Algorithm 1 (Section 3.1): for k { GEQRT; LARFB over j; for i { TSQRT; SSRFB over j } }
      for (int k = 0; k < kt; ++k) {
        out.push_back(mk(K_GEQRT, x, k, k, k, 0));
        for (int j = k + 1; j < qt; ++j)
          for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_LARFB, x, k, k, j, s));
        for (int i = k + 1; i < p; ++i) {
          out.push_back(mk(K_TSQRT, x, k, i, k, 0));
          for (int j = k + 1; j < qt; ++j)
            for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_SSRFB, x, k, i, j, s));
        }
      }
      if (I.trsm) {
        for (int j = q; j < qt; ++j)
          for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s)
            for (int k = kt - 1; k >= 0; --k) {
              for (int l = kt - 1; l > k; --l) out.push_back(mk(K_TRSM_UPD, x, k, k, j, s, l));
              out.push_back(mk(K_TRSM_SOLVE, x, k, k, j, s));
            }
      }
      break;
    case M_APPLY_QT:
      for (int k = 0; k < kt; ++k) {
        for (int j = q; j < qt; ++j)
          for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_LARFB, x, k, k, j, s));
        for (int i = k + 1; i < p; ++i)
          for (int j = q; j < qt; ++j)
            for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_SSRFB, x, k, i, j, s));
      }
      if (I.trsm) {
        for (int j = q; j < qt; ++j)
          for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s)
            for (int k = kt - 1; k >= 0; --k) {
              for (int l = kt - 1; l > k; --l) out.push_back(mk(K_TRSM_UPD, x, k, k, j, s, l));
              out.push_back(mk(K_TRSM_SOLVE, x, k, k, j, s));
            }
      }
      break;
    case M_APPLY_Q:
      for (int k = kt - 1; k >= 0; --k) {
        for (int i = p - 1; i > k; --i)
          for (int j = q; j < qt; ++j)
            for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_SSRFB_N, x, k, i, j, s));
        for (int j = q; j < qt; ++j)
          for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_LARFB_N, x, k, k, j, s));
      }
      break;
    case M_FORM_Q:
      for (int k = kt - 1; k >= 0; --k) {
        const int j0 = q + k < qt ? q + k : qt;
        for (int i = p - 1; i > k; --i)
          for (int j = j0; j < qt; ++j)
            for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_SSRFB_N, x, k, i, j, s));
        for (int j = j0; j < qt; ++j)
          for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s) out.push_back(mk(K_LARFB_N, x, k, k, j, s));
      }
      break;
    case M_TRSM:
      for (int j = q; j < qt; ++j)
        for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s)
          for (int k = kt - 1; k >= 0; --k) {
            for (int l = kt - 1; l > k; --l) out.push_back(mk(K_TRSM_UPD, x, k, k, j, s, l));
            out.push_back(mk(K_TRSM_SOLVE, x, k, k, j, s));
          }
      break;
    case M_TRSMT:
      for (int j = q; j < qt; ++j)
        for (int s = 0, ns = slabs_of_col(I, j); s < ns; ++s)
          for (int k = 0; k < kt; ++k) {
            for (int l = 0; l < k; ++l) out.push_back(mk(K_TRSMT_UPD, x, k, k, j, s, l));
            out.push_back(mk(K_TRSMT_SOLVE, x, k, k, j, s));
          }
      break;
    default:
      break;
  }
}

// Global counter id: instances get disjoint ranges.
static std::vector<int64_t> counter_bases(const std::vector<Inst>& insts) {
  std::vector<int64_t> base(insts.size() + 1, 0);
  for (size_t a = 0; a < insts.size(); ++a) {
    const Inst& I = insts[a];
    base[a + 1] = base[a] + static_cast<int64_t>(I.p) * (I.q + I.qb) * I.NS;
  }
  return base;
}

bool build_dag(const std::vector<Inst>& insts, const std::vector<TaskX>& seq, std::vector<int>& indeg,
               std::vector<int64_t>& succ_ptr, std::vector<int>& succ, std::string* err) {
  const std::vector<int64_t> base = counter_bases(insts);
  const int64_t nctr = base.back();
  const int64_t n = static_cast<int64_t>(seq.size());
  // writers of every counter, in sequential order (CSR, two passes)
  std::vector<int64_t> wptr(nctr + 1, 0);
  Wait w[kMaxWaits];
  Signal sg[kMaxSignals];
  int nsig;
  for (int64_t t = 0; t < n; ++t) {
    const Inst& I = insts[seq[t].inst];
    task_rules(I, seq[t], w, sg, &nsig);
    for (int a = 0; a < nsig; ++a)
      for (int c = 0; c < sg[a].cnt; ++c) wptr[base[seq[t].inst] + sg[a].ctr + c + 1]++;
  }
  for (int64_t c = 0; c < nctr; ++c) wptr[c + 1] += wptr[c];
  std::vector<int> writers(static_cast<size_t>(wptr[nctr]));
  std::vector<int64_t> fill(wptr.begin(), wptr.end() - 1);
  for (int64_t t = 0; t < n; ++t) {
    const Inst& I = insts[seq[t].inst];
    const int nw = task_rules(I, seq[t], w, sg, &nsig);
    for (int a = 0; a < nsig; ++a)
      for (int c = 0; c < sg[a].cnt; ++c) {
        const int ctr = sg[a].ctr + c;
        const int64_t g = base[seq[t].inst] + ctr;
        const int64_t pos = fill[g] - wptr[g];
        // the writer must wait for exactly `pos` earlier writers of this counter
        int need = -1;
        for (int b = 0; b < nw; ++b)
          if (ctr >= w[b].ctr && ctr < w[b].ctr + w[b].cnt) need = w[b].ver;
        if (need != pos) {
          if (err)
            *err = "rule mismatch: task " + std::to_string(t) + " kind " + std::to_string(seq[t].kind) +
                   " writes counter " + std::to_string(ctr) + " as writer #" + std::to_string(pos) +
                   " but waits for version " + std::to_string(need);
          return false;
        }
        writers[fill[g]++] = static_cast<int>(t);
      }
  }
  // predecessors: the v-th writer of every waited counter
  std::vector<std::vector<int>> preds(static_cast<size_t>(n));
  for (int64_t t = 0; t < n; ++t) {
    const Inst& I = insts[seq[t].inst];
    const int nw = task_rules(I, seq[t], w, sg, &nsig);
    std::vector<int>& pr = preds[t];
    for (int b = 0; b < nw; ++b) {
      if (w[b].ver <= 0) continue;
      for (int c = 0; c < w[b].cnt; ++c) {
        const int64_t g = base[seq[t].inst] + w[b].ctr + c;
        if (wptr[g + 1] - wptr[g] < w[b].ver) {
          if (err)
            *err = "rule error: task " + std::to_string(t) + " waits for version " + std::to_string(w[b].ver) +
                   " of a counter with only " + std::to_string(wptr[g + 1] - wptr[g]) + " writers";
          return false;
        }
        const int pw = writers[wptr[g] + w[b].ver - 1];
        if (pw >= t) {
          if (err) *err = "rule error: task " + std::to_string(t) + " depends on a later task";
          return false;
        }
        pr.push_back(pw);
      }
    }
    std::sort(pr.begin(), pr.end());
    pr.erase(std::unique(pr.begin(), pr.end()), pr.end());
  }
  indeg.assign(static_cast<size_t>(n), 0);
  succ_ptr.assign(static_cast<size_t>(n + 1), 0);
  for (int64_t t = 0; t < n; ++t) {
    indeg[t] = static_cast<int>(preds[t].size());
    for (int pw : preds[t]) succ_ptr[pw + 1]++;
  }
  for (int64_t t = 0; t < n; ++t) succ_ptr[t + 1] += succ_ptr[t];
  succ.assign(static_cast<size_t>(succ_ptr[n]), 0);
  std::vector<int64_t> sf(succ_ptr.begin(), succ_ptr.end() - 1);
  for (int64_t t = 0; t < n; ++t)
    for (int pw : preds[t]) succ[sf[pw]++] = static_cast<int>(t);
  return true;
}

// Seconds for one task on one CTA.  FP64: 1.19e12 flop/s over 152 SMs shared
// by ctas_per_sm CTAs (measured DFMA rate).  FP32, from the device task
// trace at nb = 128, ib = 16: update tasks run at ~60 GFLOP/s per CTA (two
// per SM) after ~10 us of fixed cost (staging, descriptor, dependency
// handshake), panels ~3.5 us per column.  Panels pay a per-column latency
// (reductions and barriers): FP64 6.5 us, the device trace's TSQRT time per
// column at nb = 128 (its FP64 chain shares the pipe with the co-resident
// CTA's updates); against the earlier 2 us it orders panels earlier, which
// measured +7 % at 4096^2, +2 % at 8192^2 and -1.7 % time for the FP64 least
// squares at 16384 x 4096 (-1.5 % at 2048^2 with nb = 32, the rest unchanged).
double task_cost(const Inst& I, const TaskX& t, int esize, int ctas_per_sm) {
  const double sm_rate = esize == 8 ? 1.19e12 / 152.0 : 2 * 60.0e9;
  const double rate = sm_rate / (ctas_per_sm > 0 ? ctas_per_sm : 1);
  const double nb = I.nb, ib = I.ib;
  const double col_lat = esize == 8 ? 6.5e-6 : 3.5e-6, blk_lat = 1.0e-6;
  // LU panel columns (argmax, interchange, scale: no norm or reflector)
  // keep the earlier 2 us calibration
  const double lu_col = esize == 8 ? 2.0e-6 : 3.5e-6;
  const double fixed = esize == 8 ? 0.0 : 10.0e-6;
  double w = I.cs;
  if (t.j >= I.q) {
    const double c0 = static_cast<double>(t.j - I.q) * I.nb + static_cast<double>(t.s) * I.cs;
    w = std::min<double>(I.cs, I.nrhs - c0);
  }
  double f = 0, lat = 0;
  switch (t.kind) {
    case K_TSQRT2:
      for (double l0 = 0; l0 < nb; l0 += ib) f += 3.0 * t.l * nb * ib * ib + 4.0 * t.l * nb * ib * (nb - l0 - ib);
      lat = nb * col_lat;
      break;
    case K_SSRFB2:
    case K_SSRFB2_N:
      f = (nb / ib) * (4.0 * t.l * nb * ib * w + ib * ib * w);
      lat = (nb / ib) * blk_lat;
      break;
    case K_TSTRF2:
      f = t.l * nb * nb * nb;
      lat = 2.0 * nb * lu_col;
      break;
    case K_SSSSM2:
      f = (nb / ib) * (2.0 * t.l * nb * ib * w + ib * ib * w);
      lat = (nb / ib) * blk_lat;
      break;
    case K_GETRF:
      f = 2.0 * nb * nb * nb / 3.0;
      lat = 2.0 * nb * lu_col;
      break;
    case K_TSTRF:
      f = nb * nb * nb;
      lat = 2.0 * nb * lu_col;
      break;
    case K_GESSM:
      f = nb * nb * w;
      lat = (nb / ib) * blk_lat;
      break;
    case K_SSSSM:
      f = (nb / ib) * (2.0 * nb * ib * w + ib * ib * w);
      lat = (nb / ib) * blk_lat;
      break;
    case K_GEQRT:
      for (double l0 = 0; l0 < nb; l0 += ib) {
        const double nr = nb - l0;
        f += 3.0 * nr * ib * ib + 4.0 * nr * ib * (nb - l0 - ib);
      }
      lat = nb * col_lat;
      break;
    case K_TSQRT:
      for (double l0 = 0; l0 < nb; l0 += ib) f += 3.0 * nb * ib * ib + 4.0 * nb * ib * (nb - l0 - ib);
      lat = nb * col_lat;
      break;
    case K_LARFB:
    case K_LARFB_N:
      for (double l0 = 0; l0 < nb; l0 += ib) f += 4.0 * (nb - l0) * ib * w + ib * ib * w;
      lat = (nb / ib) * blk_lat;
      break;
    case K_SSRFB:
    case K_SSRFB_N:
      f = (nb / ib) * (4.0 * nb * ib * w + ib * ib * w);
      lat = (nb / ib) * blk_lat;
      break;
    case K_TTQRT:
      for (double l0 = 0; l0 < nb; l0 += ib)
        f += 1.5 * (l0 + ib) * ib * ib + 2.0 * (l0 + ib) * ib * (nb - l0 - ib);
      lat = nb * col_lat;
      break;
    case K_TTMQR:
    case K_TTMQR_N:
      for (double l0 = 0; l0 < nb; l0 += ib) f += 4.0 * (l0 + ib) * ib * w + ib * ib * w;
      lat = (nb / ib) * blk_lat;
      break;
    case K_TRSM_UPD:
    case K_TRSMT_UPD:
      f = 2.0 * nb * nb * w;
      lat = blk_lat;
      break;
    case K_TRSM_SOLVE:
    case K_TRSMT_SOLVE:
      f = nb * nb * w;
      lat = nb * 0.25e-6;
      break;
    default:
      break;
  }
  return f / rate + lat + fixed;
}

static int kind_rank(int kind) {
  switch (qr_kind(kind)) {
    case K_GEQRT: return 0;
    case K_TSQRT:
    case K_TTQRT: return 1;
    case K_LARFB:
    case K_LARFB_N: return 2;
    case K_SSRFB:
    case K_SSRFB_N:
    case K_TTMQR:
    case K_TTMQR_N: return 3;
    case K_TRSM_SOLVE:
    case K_TRSMT_SOLVE: return 4;
    default: return 5;
  }
}

struct Key {
  double a;
  int64_t b;
};

static double simulate(const std::vector<int>& indeg0, const std::vector<int64_t>& succ_ptr,
                       const std::vector<int>& succ, const std::vector<double>& cost, const std::vector<Key>& key,
                       int workers, std::vector<int>* order) {
  const int64_t n = static_cast<int64_t>(cost.size());
  std::vector<int> indeg(indeg0);
  // ready: smaller key first
  auto cmp = [&key](int x, int y) {
    if (key[x].a != key[y].a) return key[x].a > key[y].a;
    return key[x].b > key[y].b;
  };
  std::priority_queue<int, std::vector<int>, decltype(cmp)> ready(cmp);
  typedef std::pair<double, int> Ev;
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> running;
  for (int64_t t = 0; t < n; ++t)
    if (indeg[t] == 0) ready.push(static_cast<int>(t));
  double now = 0;
  int idle = workers;
  int64_t done = 0;
  if (order) order->clear();
  while (done < n) {
    while (idle > 0 && !ready.empty()) {
      const int t = ready.top();
      ready.pop();
      if (order) order->push_back(t);
      running.push(Ev(now + cost[t], t));
      --idle;
    }
    if (running.empty()) break;  // cannot happen for a valid DAG
    const Ev ev = running.top();
    running.pop();
    now = ev.first;
    ++idle;
    ++done;
    for (int64_t e = succ_ptr[ev.second]; e < succ_ptr[ev.second + 1]; ++e)
      if (--indeg[succ[e]] == 0) ready.push(succ[e]);
  }
  return now;
}

bool order_tasks(const std::vector<Inst>& insts, const std::vector<TaskX>& seq, int workers, int esize,
                 int ctas_per_sm, int policy, std::vector<TaskX>& ordered, PlanStats* stats, std::string* err) {
  std::vector<int> indeg;
  std::vector<int64_t> succ_ptr;
  std::vector<int> succ;
  if (!build_dag(insts, seq, indeg, succ_ptr, succ, err)) return false;
  const int64_t n = static_cast<int64_t>(seq.size());
  std::vector<double> cost(static_cast<size_t>(n));
  double work = 0;
  for (int64_t t = 0; t < n; ++t) {
    cost[t] = task_cost(insts[seq[t].inst], seq[t], esize, ctas_per_sm);
    work += cost[t];
  }
  // bottom level (longest path to an exit), sequential order is topological
  std::vector<double> bl(static_cast<size_t>(n), 0.0);
  double cp = 0;
  for (int64_t t = n - 1; t >= 0; --t) {
    double mx = 0;
    for (int64_t e = succ_ptr[t]; e < succ_ptr[t + 1]; ++e) mx = std::max(mx, bl[succ[e]]);
    bl[t] = cost[t] + mx;
    cp = std::max(cp, bl[t]);
  }
  std::vector<Key> k0(static_cast<size_t>(n)), k1(static_cast<size_t>(n));
  for (int64_t t = 0; t < n; ++t) {
    const TaskX& x = seq[t];
    // paper: kind priority, then smaller k (TRSM: later k first), then sequence
    const int kk = (x.kind == K_TRSM_UPD || x.kind == K_TRSM_SOLVE) ? -x.k : x.k;
    k0[t].a = kind_rank(x.kind) * 1e9 + kk;
    k0[t].b = t;
    k1[t].a = -bl[t];
    k1[t].b = t;
  }
  std::vector<int> o0, o1;
  double m0 = 0, m1 = 0;
  if (policy != 1) m0 = simulate(indeg, succ_ptr, succ, cost, k0, workers, &o0);
  if (policy != 0) m1 = simulate(indeg, succ_ptr, succ, cost, k1, workers, &o1);
  int chosen = policy;
  if (policy < 0) chosen = (m1 < m0) ? 1 : 0;
  const std::vector<int>& o = chosen == 1 ? o1 : o0;
  if (static_cast<int64_t>(o.size()) != n) {
    if (err) *err = "simulation did not schedule every task";
    return false;
  }
  ordered.resize(static_cast<size_t>(n));
  for (int64_t a = 0; a < n; ++a) ordered[a] = seq[o[a]];
  if (stats) {
    stats->policy = chosen;
    stats->makespan_s = chosen == 1 ? m1 : m0;
    stats->makespan_other = chosen == 1 ? m0 : m1;
    stats->edges = static_cast<int64_t>(succ.size());
    stats->critical_path_s = cp;
    stats->work_s = work;
  }
  return true;
}

void critical_path_estimate(const Inst& I, int esize, int ctas_per_sm, double* critical_path_s, double* work_s) {
  std::vector<TaskX> seq;
  seq_tasks(I, 0, seq);
  const int64_t nctr = static_cast<int64_t>(I.p) * (I.q + I.qb) * I.NS;
  std::vector<double> ready(static_cast<size_t>(nctr), 0.0);
  Wait w[kMaxWaits];
  Signal sg[kMaxSignals];
  int nsig;
  double cp = 0, work = 0;
  for (const TaskX& t : seq) {
    const int nw = task_rules(I, t, w, sg, &nsig);
    double start = 0;
    for (int a = 0; a < nw; ++a)
      for (int c = 0; c < w[a].cnt; ++c) start = std::max(start, ready[w[a].ctr + c]);
    const double cost = task_cost(I, t, esize, ctas_per_sm);
    const double fin = start + cost;
    work += cost;
    for (int a = 0; a < nsig; ++a)
      for (int c = 0; c < sg[a].cnt; ++c) ready[sg[a].ctr + c] = fin;
    cp = std::max(cp, fin);
  }
  *critical_path_s = cp;
  *work_s = work;
}

bool order_bottom_level(const std::vector<Inst>& insts, const std::vector<TaskX>& seq, int esize, int ctas_per_sm,
                        int workers, std::vector<TaskX>& ordered, PlanStats* stats, std::string* err) {
  const std::vector<int64_t> base = counter_bases(insts);
  const int64_t nctr = base.back();
  const int64_t n = static_cast<int64_t>(seq.size());
  // every task's rules once (the three passes below reuse them)
  struct Rules {
    Wait w[kMaxWaits];
    Signal sg[kMaxSignals];
    int8_t nw, nsig;
  };
  std::vector<Rules> rules(static_cast<size_t>(n));
  std::vector<int64_t> wptr(nctr + 1, 0);
  for (int64_t t = 0; t < n; ++t) {
    Rules& R = rules[t];
    int nsig = 0;
    R.nw = static_cast<int8_t>(task_rules(insts[seq[t].inst], seq[t], R.w, R.sg, &nsig));
    R.nsig = static_cast<int8_t>(nsig);
    for (int a = 0; a < nsig; ++a)
      for (int c = 0; c < R.sg[a].cnt; ++c) wptr[base[seq[t].inst] + R.sg[a].ctr + c + 1]++;
  }
  for (int64_t c = 0; c < nctr; ++c) wptr[c + 1] += wptr[c];
  std::vector<int> writers(static_cast<size_t>(wptr[nctr]));
  {
    std::vector<int64_t> fill(wptr.begin(), wptr.end() - 1);
    for (int64_t t = 0; t < n; ++t) {
      const Rules& R = rules[t];
      for (int a = 0; a < R.nsig; ++a)
        for (int c = 0; c < R.sg[a].cnt; ++c) {
          const int ctr = R.sg[a].ctr + c;
          const int64_t g = base[seq[t].inst] + ctr;
          int need = -1;
          for (int b = 0; b < R.nw; ++b)
            if (ctr >= R.w[b].ctr && ctr < R.w[b].ctr + R.w[b].cnt) need = R.w[b].ver;
          if (need != fill[g] - wptr[g]) {
            if (err) *err = "rule mismatch in task " + std::to_string(t);
            return false;
          }
          writers[fill[g]++] = static_cast<int>(t);
        }
    }
  }
  std::vector<double> bl(static_cast<size_t>(n)), maxsucc(static_cast<size_t>(n), 0.0);
  double work = 0, cp = 0;
  for (int64_t t = n - 1; t >= 0; --t) {
    const Inst& I = insts[seq[t].inst];
    const double c = task_cost(I, seq[t], esize, ctas_per_sm);
    work += c;
    bl[t] = c + maxsucc[t];
    cp = std::max(cp, bl[t]);
    const Rules& R = rules[t];
    for (int b = 0; b < R.nw; ++b) {
      if (R.w[b].ver <= 0) continue;
      for (int cc = 0; cc < R.w[b].cnt; ++cc) {
        const int64_t g = base[seq[t].inst] + R.w[b].ctr + cc;
        if (wptr[g + 1] - wptr[g] < R.w[b].ver) {
          if (err) *err = "rule error: missing writer for task " + std::to_string(t);
          return false;
        }
        const int pw = writers[wptr[g] + R.w[b].ver - 1];
        if (pw >= t) {
          if (err) *err = "rule error: task depends on a later task";
          return false;
        }
        if (bl[t] > maxsucc[pw]) maxsucc[pw] = bl[t];
      }
    }
  }
  // decreasing bottom level, ties by sequential index (keys sorted in place:
  // no indirection in the comparisons)
  std::vector<std::pair<double, int>> key(static_cast<size_t>(n));
  for (int64_t t = 0; t < n; ++t) key[t] = std::make_pair(-bl[t], static_cast<int>(t));
  std::sort(key.begin(), key.end());
  ordered.resize(static_cast<size_t>(n));
  for (int64_t a = 0; a < n; ++a) ordered[a] = seq[key[a].second];
  if (stats) {
    stats->policy = 2;
    stats->critical_path_s = cp;
    stats->work_s = work;
    stats->makespan_s = std::max(cp, work / std::max(1, workers));
    stats->makespan_other = 0;
    stats->edges = 0;
  }
  return true;
}

}  // namespace tqr
