// tqr_graph.h -- task descriptors and the data-flow rules of the tile DAG.
//
// Shared by the host plan builder and the device scheduler (both compile it).
//
// The paper (Section 3.3) runs Algorithm 1 as a DAG of tile tasks whose edges
// are the data dependencies between them.  Here the DAG is never stored: each
// tile column slab (i, j, s) owns a version counter that counts the tasks that
// have written it, and every task knows, from its indices alone, which version
// of each operand it needs.  A task may start once every counter it waits on
// has reached the required version; when it ends it increments the counters of
// what it wrote.  Because every writer of a slab also waits for that slab's
// previous version, the writers of each slab run in exactly the order of the
// sequential algorithm, so the result does not depend on the schedule.
//
// Operand versions below are counts of earlier writers of the slab in the
// sequential order of the mode:
//   FACTOR  (Algorithm 1; optional right-hand-side tile columns j >= q are
//            updated like trailing columns, i.e. Q^T B; optional back
//            substitution X = R^-1 (Q^T B)[0:n] appended)
//   APPLY_QT (factors final: LARFB/SSRFB on B only, Algorithm 1's order;
//            optional back substitution appended, as in FACTOR)
//   APPLY_Q  (factors final: the transposed steps in reverse order)
//   TRSM     (factors final: back substitution on B only)
//   TRSMT    (factors final: forward substitution R^T X = B)
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define TQR_HD __host__ __device__ __forceinline__
#else
#define TQR_HD inline
#endif

namespace tqr {

enum Kind : int {
  K_GEQRT = 0,       // Section 3.1 DGEQT2 on tile (k,k)
  K_TSQRT = 1,       // Section 3.1 DTSQT2 on (k,k) upper triangle + (i,k)
  K_LARFB = 2,       // Section 3.1 DLARFB: slab s of (k,j) <- Q_kk^T (k,j)
  K_SSRFB = 3,       // Section 3.1 DSSRFB: slab s of [(k,j); (i,j)] <- Q_ik^T [.]
  K_LARFB_N = 4,     // (k,j) slab <- Q_kk (k,j)            (apply Q)
  K_SSRFB_N = 5,     // [(k,j); (i,j)] slab <- Q_ik [.]     (apply Q)
  K_TRSM_UPD = 6,    // C_k <- C_k - R_kl X_l   (l > k), slab s of column j
  K_TRSM_SOLVE = 7,  // X_k <- R_kk^-1 C_k
  K_TRSMT_UPD = 8,   // C_k <- C_k - R_lk^T X_l (l < k)
  K_TRSMT_SOLVE = 9, // X_k <- R_kk^-T C_k
  // reduction-tree variant (Inst.D > 0): TSQRT/SSRFB carry the domain head
  // in l; GEQRT/LARFB act on head row i; TT kernels merge head l (kept) and
  // head i (eliminated), whose tile keeps the TT reflectors in its upper
  // triangle
  K_TTQRT = 10,      // QR of the triangles of (l,k) and (i,k)
  K_TTMQR = 11,      // slab s of [(l,j); (i,j)] <- Q_tt^T [.]
  K_TTMQR_N = 12,    // slab s of [(l,j); (i,j)] <- Q_tt [.]
  // tiled LU with pairwise pivoting (Inst.lu = 1, flat panel only): the same
  // loop nest and data flow as GEQRT / LARFB / TSQRT / SSRFB, so the same
  // dependency rules (qr_kind maps them)
  K_GETRF = 13,      // (k,k) -> L_kk, U_kk, row interchanges within the tile
  K_GESSM = 14,      // slab s of (k,j) <- L_kk^-1 P_kk (k,j)
  K_TSTRF = 15,      // [U_kk; (i,k)] -> U_kk, L_ik, pairwise interchanges
  K_SSSSM = 16,      // slab s of [(k,j); (i,j)] <- TSTRF(k,i)'s transformations [.]
  // 2b x b bottoms (Inst.pair = 1, flat panel only): the rows below the
  // diagonal tile are taken in groups of l = 2 tile rows (the last may be 1)
  // starting at row i; TSQRT2 factors [R_kk; (i..i+l-1, k)], SSRFB2 updates
  // slab s of [(k,j); (i..i+l-1, j)]
  K_TSQRT2 = 17,
  K_SSRFB2 = 18,
  K_SSRFB2_N = 19,   // (apply Q)
  K_TSTRF2 = 20,     // the tiled LU's TSTRF / SSSSM on 2b x b bottoms
  K_SSSSM2 = 21,
  K_NKINDS = 22
};

// Most waits / signals a task has (SSRFB2: 4 waits, 3 signals).
constexpr int kMaxWaits = 4;
constexpr int kMaxSignals = 3;

// The QR kind whose data flow an LU kind shares.
TQR_HD int qr_kind(int kind) {
  switch (kind) {
    case K_TSQRT2: return K_TSQRT;
    case K_SSRFB2: return K_SSRFB;
    case K_SSRFB2_N: return K_SSRFB_N;
    case K_TSTRF2: return K_TSQRT;
    case K_SSSSM2: return K_SSRFB;
    case K_GETRF: return K_GEQRT;
    case K_GESSM: return K_LARFB;
    case K_TSTRF: return K_TSQRT;
    case K_SSSSM: return K_SSRFB;
    default: return kind;
  }
}

// The LU kind replacing a QR kind in an LU task list.
TQR_HD int lu_kind(int kind) {
  switch (kind) {
    case K_GEQRT: return K_GETRF;
    case K_LARFB: return K_GESSM;
    case K_TSQRT: return K_TSTRF;
    case K_SSRFB: return K_SSSSM;
    case K_TSQRT2: return K_TSTRF2;
    case K_SSRFB2: return K_SSSSM2;
    default: return kind;
  }
}

// M_FORM_Q: M_APPLY_Q on right-hand sides that start as the leading columns
// of the identity (flat panel only).  Column c of the identity has no entry in
// the rows that step k's reflectors touch (rows >= k*nb) when c < k*nb, so
// step k skips right-hand-side tile columns jb < k: those stay exact.
enum Mode : int { M_FACTOR = 0, M_APPLY_QT = 1, M_APPLY_Q = 2, M_TRSM = 3, M_TRSMT = 4, M_FORM_Q = 5 };

// One task (32 bytes, two vector loads on the device).  k: elimination step;
// i: row tile; j: column tile (A columns < q, right-hand-side columns >= q);
// s: column slab of tile column j; l: the second tile index of TRSM updates.
struct TaskX {
  int32_t kind, s, inst, k, i, j, l, pad;
};

// Per-problem description (device copy lives in global memory).
struct Inst {
  void* A;          // BDL tiles of A: tile (i,j) at ((i + j*p) * nb * nb) elements
  void* B;          // BDL tiles of the right-hand sides: tile (i, q+jb) at
                    // ((i + jb*p) * nb * nb) elements
  void* T;          // T blocks (element type of A), see t_offset
  int32_t* ver;     // version counters, (j*p + i)*NS + s for j in [0, q+qb)
  int32_t m, n, p, q, kt, qb, nrhs;
  int32_t nb, ib, cs, NS;   // NS = nb/cs slabs per full tile column
  int32_t mode;
  int32_t trsm;             // FACTOR mode: back substitution appended (1) or not (0)
  int32_t D;                // 0: Algorithm 1's flat panel; >0: domains of D tile rows + binary tree
  int32_t lu;               // 1: LU kernels (GETRF/GESSM/TSTRF/SSSSM) in place of the QR ones
  const int32_t* vtab;      // tree variant: writes per trailing tile of row r before step k,
                            // vtab[k * p + r] for k = 0..kt (see tree_writes)
  int32_t* piv;             // LU: row interchanges, nb per (i,k) slot at piv_offset
  int32_t pair;             // 1: 2b x b bottoms (K_TSQRT2 / K_SSRFB2 kinds)
  int32_t pad1;
};

// Number of slabs of tile column j (A columns: NS; right-hand-side columns:
// enough slabs to cover the real columns of that tile column).
TQR_HD int slabs_of_col(const Inst& I, int j) {
  if (j < I.q) return I.NS;
  int c0 = (j - I.q) * I.nb;
  int w = I.nrhs - c0;
  if (w > I.nb) w = I.nb;
  if (w <= 0) return 0;
  return (w + I.cs - 1) / I.cs;
}

TQR_HD int ctr_index(const Inst& I, int i, int j, int s) { return (j * I.p + i) * I.NS + s; }

// A wait: counters ctr .. ctr+cnt-1 must all be >= ver.
struct Wait { int ctr, cnt, ver; };
// A signal: counters ctr .. ctr+cnt-1 are incremented.
struct Signal { int ctr, cnt; };

// ---- reduction-tree variant --------------------------------------------
// Step k cuts rows k..p-1 into domains of D rows; domain d has head row
// k + d*D.  Within a domain the head is GEQRT'ed and TSQRT'ed with each later
// row (positions 1, 2, ... of the head's writers in the step); then the
// heads merge in a binary tree: at level L head index d (multiple of 2^(L+1))
// absorbs head d + 2^L, if present.
struct TreePos {
  int d, mi, h, dsz, H;  // domain, index in the domain (0 = head), head row, domain size, #domains
};

TQR_HD TreePos tree_pos(const Inst& I, int k, int r) {
  TreePos t;
  const int o = r - k;
  t.d = o / I.D;
  t.mi = o - t.d * I.D;
  t.h = k + t.d * I.D;
  t.dsz = (I.p - t.h) < I.D ? (I.p - t.h) : I.D;
  t.H = (I.p - k + I.D - 1) / I.D;
  return t;
}

// Merges head d takes part in as the surviving head at levels below lvl.
TQR_HD int tree_cnt_a(int d, int lvl, int H) {
  int c = 0;
  for (int L = 0; L < lvl && (1 << L) < H; ++L)
    if (d % (2 << L) == 0 && d + (1 << L) < H) ++c;
  return c;
}

// Level at which head d (> 0) is eliminated: its lowest set bit.
TQR_HD int tree_level(int d) {
  int L = 0;
  while (!(d & (1 << L))) ++L;
  return L;
}

// Writes a trailing tile (or the panel tile) of row r >= k receives in step k.
TQR_HD int tree_writes(const Inst& I, int k, int r) {
  const TreePos t = tree_pos(I, k, r);
  if (t.mi > 0) return 1;
  return t.dsz + tree_cnt_a(t.d, 31, t.H) + (t.d > 0 ? 1 : 0);
}

TQR_HD int tree_base(const Inst& I, int k, int r) { return I.vtab[k * I.p + r]; }
TQR_HD int tree_fin(const Inst& I, int r) { return I.vtab[I.kt * I.p + r]; }

// Rules of the tree variant (all modes).  Forward modes (FACTOR, APPLY_QT)
// need version base + pos for the writer at position pos of step k; APPLY_Q
// replays the same writers in reverse, so it needs fin - 1 - (base + pos).
TQR_HD int tree_rules(const Inst& I, const TaskX& t, Wait* w, Signal* sg, int* nsig) {
  const int kt = I.kt, NS = I.NS;
  const int k = t.k, i = t.i, j = t.j, s = t.s, l = t.l;
  const bool a_final = I.mode != M_FACTOR;
  const bool rev = I.mode == M_APPLY_Q || I.mode == M_FORM_Q;
  int nw = 0;
  *nsig = 0;
  // reverse modes replay the writers backwards: the version is the number of
  // writes after this one in forward order.  M_FORM_Q only runs steps <= jb
  // on right-hand-side tile column jb = j - q, so a tile's forward writes end
  // with step min(jb + 1, kt).
  auto ver = [&](int r, int pos) {
    const int f = tree_base(I, k, r) + pos;
    if (!rev) return f;
    int fin = tree_fin(I, r);
    if (I.mode == M_FORM_Q) {
      const int last = j - I.q + 1 < kt ? j - I.q + 1 : kt;
      fin = I.vtab[last * I.p + r];
    }
    return fin - 1 - f;
  };
  switch (t.kind) {
    case K_GEQRT:
      w[nw++] = {ctr_index(I, i, k, 0), NS, tree_base(I, k, i)};
      sg[(*nsig)++] = {ctr_index(I, i, k, 0), NS};
      break;
    case K_LARFB:
    case K_LARFB_N:
      if (!a_final) w[nw++] = {ctr_index(I, i, k, 0), NS, tree_base(I, k, i) + 1};
      w[nw++] = {ctr_index(I, i, j, s), 1, ver(i, 0)};
      sg[(*nsig)++] = {ctr_index(I, i, j, s), 1};
      break;
    case K_TSQRT: {
      const TreePos ti = tree_pos(I, k, i);
      w[nw++] = {ctr_index(I, l, k, 0), NS, tree_base(I, k, l) + ti.mi};
      w[nw++] = {ctr_index(I, i, k, 0), NS, tree_base(I, k, i)};
      sg[(*nsig)++] = {ctr_index(I, l, k, 0), NS};
      sg[(*nsig)++] = {ctr_index(I, i, k, 0), NS};
      break;
    }
    case K_SSRFB:
    case K_SSRFB_N: {
      const TreePos ti = tree_pos(I, k, i);
      if (!a_final) w[nw++] = {ctr_index(I, i, k, 0), NS, tree_base(I, k, i) + 1};
      w[nw++] = {ctr_index(I, l, j, s), 1, ver(l, ti.mi)};
      w[nw++] = {ctr_index(I, i, j, s), 1, ver(i, 0)};
      sg[(*nsig)++] = {ctr_index(I, l, j, s), 1};
      sg[(*nsig)++] = {ctr_index(I, i, j, s), 1};
      break;
    }
    case K_TTQRT:
    case K_TTMQR:
    case K_TTMQR_N: {
      const TreePos ta = tree_pos(I, k, l), tb = tree_pos(I, k, i);
      const int L = tree_level(tb.d);
      const int pa = ta.dsz + tree_cnt_a(ta.d, L, ta.H);
      const int pb = tb.dsz + tree_cnt_a(tb.d, L, tb.H);
      if (t.kind == K_TTQRT) {
        w[nw++] = {ctr_index(I, l, k, 0), NS, tree_base(I, k, l) + pa};
        w[nw++] = {ctr_index(I, i, k, 0), NS, tree_base(I, k, i) + pb};
        sg[(*nsig)++] = {ctr_index(I, l, k, 0), NS};
        sg[(*nsig)++] = {ctr_index(I, i, k, 0), NS};
      } else {
        if (!a_final) w[nw++] = {ctr_index(I, i, k, 0), NS, tree_base(I, k, i) + pb + 1};
        w[nw++] = {ctr_index(I, l, j, s), 1, ver(l, pa)};
        w[nw++] = {ctr_index(I, i, j, s), 1, ver(i, pb)};
        sg[(*nsig)++] = {ctr_index(I, l, j, s), 1};
        sg[(*nsig)++] = {ctr_index(I, i, j, s), 1};
      }
      break;
    }
    case K_TRSM_UPD: {
      // after the factorization (or Q^T B) every tile of row r has fin(r) writes
      const bool fw = (I.mode == M_FACTOR || I.mode == M_APPLY_QT);
      if (!a_final) w[nw++] = {ctr_index(I, k, l, 0), NS, tree_fin(I, k)};
      w[nw++] = {ctr_index(I, l, j, s), 1, (fw ? tree_fin(I, l) : 0) + (kt - l)};
      w[nw++] = {ctr_index(I, k, j, s), 1, (fw ? tree_fin(I, k) : 0) + (kt - 1 - l)};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      break;
    }
    case K_TRSM_SOLVE: {
      const bool fw = (I.mode == M_FACTOR || I.mode == M_APPLY_QT);
      if (!a_final) w[nw++] = {ctr_index(I, k, k, 0), NS, tree_fin(I, k)};
      w[nw++] = {ctr_index(I, k, j, s), 1, (fw ? tree_fin(I, k) : 0) + (kt - 1 - k)};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      break;
    }
    default:
      break;
  }
  return nw;
}

// ---- 2b x b bottoms ----------------------------------------------------
// Groups of step k: rows k+1, k+2 | k+3, k+4 | ...; the last may hold one row.
TQR_HD int pair_groups(const Inst& I, int k) { return (I.p - k - 1 + 1) / 2; }
TQR_HD int pair_index(int k, int h) { return (h - k - 1) / 2; }

// Writes every tile of row r < kt has received at the end of the
// factorization (or of Q^T B on a right-hand side): one per earlier step,
// plus GEQRT/LARFB and one per bottom group (or bottom row) of its own step.
TQR_HD int fin_row(const Inst& I, int r) {
  if (!I.pair) return I.p;
  return r + 1 + pair_groups(I, r);
}

// Rules of the pair kinds (and LARFB_N, whose count depends on the groups).
TQR_HD int pair_rules(const Inst& I, const TaskX& t, Wait* w, Signal* sg, int* nsig) {
  const int kt = I.kt, NS = I.NS;
  const int k = t.k, h = t.i, j = t.j, s = t.s, l = t.l;
  const bool a_final = I.mode != M_FACTOR;
  const int g = pair_index(k, h);
  int nw = 0;
  *nsig = 0;
  // reverse-order writes a right-hand-side tile of row r got before step k
  auto bot = [&](int r) {
    const int mr = r < kt ? r : kt;
    return (r < kt ? pair_groups(I, r) + 1 : 0) + (mr - 1 - k);
  };
  switch (t.kind) {
    case K_TSQRT2:
      w[nw++] = {ctr_index(I, k, k, 0), NS, k + 1 + g};
      for (int a = 0; a < l; ++a) w[nw++] = {ctr_index(I, h + a, k, 0), NS, k};
      sg[(*nsig)++] = {ctr_index(I, k, k, 0), NS};
      for (int a = 0; a < l; ++a) sg[(*nsig)++] = {ctr_index(I, h + a, k, 0), NS};
      break;
    case K_SSRFB2:
      if (!a_final) w[nw++] = {ctr_index(I, h, k, 0), NS, k + 1};
      w[nw++] = {ctr_index(I, k, j, s), 1, k + 1 + g};
      for (int a = 0; a < l; ++a) w[nw++] = {ctr_index(I, h + a, j, s), 1, k};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      for (int a = 0; a < l; ++a) sg[(*nsig)++] = {ctr_index(I, h + a, j, s), 1};
      break;
    case K_SSRFB2_N:
      // sequential order: for k = kt-1..0 { groups in reverse: SSRFB2_N; LARFB_N(k) }
      w[nw++] = {ctr_index(I, k, j, s), 1, pair_groups(I, k) - 1 - g};
      for (int a = 0; a < l; ++a) w[nw++] = {ctr_index(I, h + a, j, s), 1, bot(h + a)};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      for (int a = 0; a < l; ++a) sg[(*nsig)++] = {ctr_index(I, h + a, j, s), 1};
      break;
    case K_LARFB_N:
      w[nw++] = {ctr_index(I, k, j, s), 1, pair_groups(I, k)};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      break;
    default:
      break;
  }
  return nw;
}

// Fills up to kMaxWaits waits and kMaxSignals signals; returns the number of waits, writes the
// number of signals to *nsig.  `a_final` (APPLY/TRSM modes): A's tiles were
// factored by an earlier launch, so waits on them are dropped.
// task_rules_base: every rule but the 2b x b bottoms' (the QR and LU task
// kernels evaluate only this one: the pair branch would weigh on their
// register allocation, and they never run pair tasks).
TQR_HD int task_rules_base(const Inst& I, const TaskX& t0, Wait* w, Signal* sg, int* nsig) {
  TaskX t = t0;
  t.kind = qr_kind(t0.kind);
  if (I.D > 0 && t.kind != K_TRSMT_UPD && t.kind != K_TRSMT_SOLVE &&
      !((t.kind == K_TRSM_UPD || t.kind == K_TRSM_SOLVE) && I.mode == M_TRSM))
    return tree_rules(I, t, w, sg, nsig);
  const int p = I.p, kt = I.kt, NS = I.NS;
  const int k = t.k, i = t.i, j = t.j, s = t.s, l = t.l;
  const bool a_final = I.mode != M_FACTOR;
  int nw = 0;
  *nsig = 0;
  switch (t.kind) {
    case K_GEQRT:
      w[nw++] = {ctr_index(I, k, k, 0), NS, k};
      sg[(*nsig)++] = {ctr_index(I, k, k, 0), NS};
      break;
    case K_TSQRT:
      w[nw++] = {ctr_index(I, k, k, 0), NS, i};
      w[nw++] = {ctr_index(I, i, k, 0), NS, k};
      sg[(*nsig)++] = {ctr_index(I, k, k, 0), NS};
      sg[(*nsig)++] = {ctr_index(I, i, k, 0), NS};
      break;
    case K_LARFB:
      if (!a_final) w[nw++] = {ctr_index(I, k, k, 0), NS, k + 1};
      w[nw++] = {ctr_index(I, k, j, s), 1, k};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      break;
    case K_SSRFB:
      if (!a_final) w[nw++] = {ctr_index(I, i, k, 0), NS, k + 1};
      w[nw++] = {ctr_index(I, k, j, s), 1, i};
      w[nw++] = {ctr_index(I, i, j, s), 1, k};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      sg[(*nsig)++] = {ctr_index(I, i, j, s), 1};
      break;
    case K_SSRFB_N: {
      // sequential order: for k = kt-1..0 { for i = p-1..k+1 SSRFB_N(k,i); LARFB_N(k) }.
      // Tile (i,j) receives one write from each step k' in (k, min(i,kt)) and
      // p - i writes from step i (if i < kt); M_FORM_Q keeps only steps
      // k' <= jb = j - q.
      int mi = i < kt ? i : kt;
      bool own = i < kt;
      if (I.mode == M_FORM_Q) {
        const int jb1 = j - I.q + 1;
        if (jb1 < mi) mi = jb1;
        own = own && i < jb1;
      }
      int bot = (own ? (p - i) : 0) + (mi - 1 - k);
      w[nw++] = {ctr_index(I, k, j, s), 1, p - 1 - i};
      w[nw++] = {ctr_index(I, i, j, s), 1, bot};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      sg[(*nsig)++] = {ctr_index(I, i, j, s), 1};
      break;
    }
    case K_LARFB_N:
      w[nw++] = {ctr_index(I, k, j, s), 1, p - 1 - k};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      break;
    case K_TRSM_UPD: {
      // C_k -= R_kl X_l, l = kt-1 .. k+1, then SOLVE(k).  In FACTOR and
      // APPLY_QT modes the right-hand sides first received p writes (rows
      // < kt) from Algorithm 1's updates, and in FACTOR mode R's tiles (k, l),
      // k <= l < q, end at version p.
      const bool fw = (I.mode == M_FACTOR || I.mode == M_APPLY_QT);
      if (!a_final) w[nw++] = {ctr_index(I, k, l, 0), NS, fin_row(I, k)};
      w[nw++] = {ctr_index(I, l, j, s), 1, (fw ? fin_row(I, l) : 0) + (kt - l)};
      w[nw++] = {ctr_index(I, k, j, s), 1, (fw ? fin_row(I, k) : 0) + (kt - 1 - l)};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      break;
    }
    case K_TRSM_SOLVE: {
      const int base = (I.mode == M_FACTOR || I.mode == M_APPLY_QT) ? fin_row(I, k) : 0;
      if (!a_final) w[nw++] = {ctr_index(I, k, k, 0), NS, fin_row(I, k)};
      w[nw++] = {ctr_index(I, k, j, s), 1, base + (kt - 1 - k)};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      break;
    }
    case K_TRSMT_UPD:
      // forward substitution: C_k -= R_lk^T X_l for l = 0 .. k-1, then SOLVE
      w[nw++] = {ctr_index(I, l, j, s), 1, l + 1};
      w[nw++] = {ctr_index(I, k, j, s), 1, l};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      break;
    case K_TRSMT_SOLVE:
      w[nw++] = {ctr_index(I, k, j, s), 1, k};
      sg[(*nsig)++] = {ctr_index(I, k, j, s), 1};
      break;
    default:
      break;
  }
  return nw;
}

TQR_HD int task_rules(const Inst& I, const TaskX& t0, Wait* w, Signal* sg, int* nsig) {
  if (I.pair) {
    // the LU pair kinds share the QR pair kinds' data flow
    const int k2 = t0.kind == K_TSTRF2 ? K_TSQRT2 : (t0.kind == K_SSSSM2 ? K_SSRFB2 : t0.kind);
    if (k2 == K_TSQRT2 || k2 == K_SSRFB2 || k2 == K_SSRFB2_N || k2 == K_LARFB_N) {
      TaskX t = t0;
      t.kind = k2;
      return pair_rules(I, t, w, sg, nsig);
    }
  }
  return task_rules_base(I, t0, w, sg, nsig);
}

// Offset (in elements) of T block (i, k), i >= k, each ib x nb.
TQR_HD int64_t t_offset(int p, int nb, int ib, int i, int k) {
  int64_t idx = (int64_t)k * p - (int64_t)k * (k - 1) / 2 + (i - k);
  return idx * (int64_t)ib * nb;
}

// LU pivots of slot (i, k): nb int32 at this offset (the slots of t_offset).
TQR_HD int64_t piv_offset(int p, int nb, int i, int k) {
  int64_t idx = (int64_t)k * p - (int64_t)k * (k - 1) / 2 + (i - k);
  return idx * (int64_t)nb;
}

TQR_HD int64_t t_elems(int p, int q, int nb, int ib) {
  int kt = p < q ? p : q;
  return t_offset(p, nb, ib, kt, kt);  // first index past the last block
}

// Tree variant: the TTQRT factors of eliminated head (b, k) follow the
// GEQRT/TSQRT ones with the same indexing.
TQR_HD int64_t t2_offset(int p, int q, int nb, int ib, int b, int k) {
  return t_elems(p, q, nb, ib) + t_offset(p, nb, ib, b, k);
}

}  // namespace tqr

namespace tqr {

// Threads per CTA of the persistent task kernel.
constexpr int kThreads = 256;
// Largest ib * cs (outputs of one W block) handled per thread batch.
constexpr int kMaxOutPerThread = 8;

// Shared-memory layout of the task kernel (byte offsets, 16-byte aligned):
//   P   nb x ib    panel being factored / reflector block V_l
//   T   ib x ib    T_l
//   S   nb x cs    column slab being updated (bottom tile or whole slab);
//                  also holds TSQRT's ib x ib triangle when it fits
//   Top ib x cs    top rows of a TSQRT/SSRFB update (ib x ib if it must hold
//                  TSQRT's triangle)
//   W   ib x cs    W = V^T S products
//   Red doubles    reduction scratch and per-column scalars
//   Part           FP32 only: split-K partials of the blocked W = V^T S
//   Bar 8 bytes    mbarrier for the bulk (TMA) copies
struct SmemLayout {
  int oP, oP2, oT, oS, oTop, oW, oRed, oPart, oBar, bytes;  // oP2 < 0: no second panel buffer
  int oTopS, oTst;  // FP32 update staging (top slab, all T blocks); < 0: absent
  bool r_in_s;
};

TQR_HD int align16(int x) { return (x + 15) & ~15; }

// Leading dimension of the nb-row panels and slabs in shared memory: padded
// by 16 bytes so columns stay 16-byte aligned for the bulk copies while
// lanes that walk along a row do not all hit one bank.
TQR_HD int ld_pad(int nb, int esize) { return nb + 16 / esize; }

// rows: the tallest operand (nb, or 2 nb for 2b x b bottoms).
TQR_HD SmemLayout smem_layout(int nb, int ib, int cs, int esize, int rows = 0) {
  SmemLayout L;
  const int ld = ld_pad(rows > nb ? rows : nb, esize);
  L.r_in_s = (ld * cs >= ib * ib);
  int top_elems = ib * cs;
  if (!L.r_in_s && ib * ib > top_elems) top_elems = ib * ib;
  int o = 0;
  L.oP = o;   o += align16(ld * ib * esize);
  // second reflector-block buffer (b x b layouts, blocks up to 32 KB): the
  // update tasks load block l+1's V while applying block l
  L.oP2 = -1;
  if (rows <= nb && ld * ib * esize <= 32768) {
    L.oP2 = o;
    o += align16(ld * ib * esize);
  }
  // FP32 with the second buffer: the update tasks also stage the whole top
  // slab and all ib x ib T blocks of the tile once per task
  L.oTopS = -1;
  L.oTst = -1;
  if (esize == 4 && L.oP2 >= 0) {
    L.oTopS = o;
    o += align16(ld * cs * esize);
    L.oTst = o;
    o += align16(ib * nb * esize);
  }
  L.oT = o;   o += align16(ib * (ib + 1) * esize);
  L.oS = o;   o += align16(ld * cs * esize);
  L.oTop = o; o += align16(top_elems * esize);
  L.oW = o;   o += align16(ib * cs * esize);
  L.oRed = o; o += align16((2 * kThreads + 2 * 64 + 32) * 8);
  // FP32 only: split-K partial sums of the register-blocked update (16 per
  // thread, stride 17 so a warp's stores fall in distinct banks)
  L.oPart = o; if (esize == 4) o += align16(kThreads * 17 * esize);
  L.oBar = o; o += 16;
  L.bytes = o;
  return L;
}

}  // namespace tqr
