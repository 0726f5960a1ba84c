"""Tile kernels and Algorithm 1 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper, Section 3.1: four elementary operations on b x b tiles
  GEQRT  (DGEQT2)  A_kk -> V_kk, R_kk and T_kk
  LARFB  (DLARFB)  A_kj <- (I - V_kk T_kk V_kk^T)^T A_kj
  TSQRT  (DTSQT2)  [R_kk; A_ik] -> [I; V_ik], R~_kk and T_ik
  SSRFB  (DSSRFB)  [A_kj; A_ij] <- (I - [I; V_ik] T_ik [I; V_ik]^T)^T [A_kj; A_ij]
and Algorithm 1, the loop nest k / j / i / j that drives them.

Readings of the paper used here (each listed with the design notes):
* The update formulas print (I - V T V^T); with T from the forward recurrence
  that is H_0...H_{b-1} = Q, so the factorization must apply its transpose
  (I - V T^T V^T).  A wrong orientation fails A = QR.
* Inner blocking: the paper's kernels are unblocked (ib = b).  With ib < b the
  b columns of a tile are handled in b/ib blocks; block l has its own ib x ib
  T_l, stored side by side as an ib x b array per tile.  Within a block the
  columns are factored one by one (as DGEQR2); the block's reflectors are then
  applied to the tile's trailing columns at once.  Block l of a TSQRT touches
  rows l*ib .. (l+1)*ib-1 of the top triangle and every row of the bottom tile.
  LARFB / SSRFB apply blocks l = 0, 1, ... (Q^T) or in reverse (Q).
  ib = b reproduces the paper's unblocked kernels exactly.
* Edge tiles: A is zero-padded to p*b x q*b.  Zero rows stay zero under the
  reflectors and zero columns get tau = 0, so R[:m, :n] is unchanged.
* The second loop of Algorithm 1 prints "i = k+1, k+1, ..."; read k+1, k+2, ...

The end of the file adds the reduction-tree variant (tree_qr), an extension
beyond the paper's flat panel.
"""

import math

import numpy as np

from .householder import householder, geqr2, unit_lower, larft


def _stacked_v(V2, l0, ib, nb):
    """Explicit [I; V2] for block l of a TSQRT: (b + rows of V2) x ib, with
    the identity's ones in rows l0 .. l0+ib-1 of the top tile (Section 3.1,
    DTSQT2)."""
    Vfull = np.zeros((nb + V2.shape[0], ib))
    for c in range(ib):
        Vfull[l0 + c, c] = 1.0
    Vfull[nb:, :] = V2
    return Vfull


def geqrt(Akk, ib):
    """DGEQT2 with inner blocking ib.  Section 3.1.

    Returns (F, T): F holds R_kk on/above the diagonal and V_kk below it;
    T is ib x b, block l in columns l*ib .. (l+1)*ib-1.
    """
    F = np.array(Akk, dtype=np.float64, copy=True)
    nb = F.shape[0]
    assert F.shape == (nb, nb) and nb % ib == 0
    T = np.zeros((ib, nb))
    for l0 in range(0, nb, ib):
        l1 = l0 + ib
        panel, tau = geqr2(F[l0:, l0:l1])         # DGEQR2 on the ib-wide panel
        F[l0:, l0:l1] = panel
        V = unit_lower(panel, ib)
        Tl = larft(V, tau)
        T[:, l0:l1] = Tl
        C = F[l0:, l1:]
        F[l0:, l1:] = C - V @ (Tl.T @ (V.T @ C))  # (I - V T_l^T V^T) on the rest
    return F, T


def larfb(C, Fkk, Tkk, ib, trans=True):
    """DLARFB: apply the reflectors of a GEQRT'ed diagonal tile to C (b x w).

    trans=True applies Q_kk^T = product over blocks l = 0, 1, ... of
    (I - V_l T_l^T V_l^T); trans=False applies Q_kk (blocks in reverse, T_l).
    """
    C = np.array(C, dtype=np.float64, copy=True)
    nb = Fkk.shape[0]
    blocks = list(range(0, nb, ib))
    if not trans:
        blocks.reverse()
    for l0 in blocks:
        l1 = l0 + ib
        V = unit_lower(Fkk[l0:, l0:l1], ib)
        Tl = Tkk[:, l0:l1]
        op = Tl.T if trans else Tl
        C[l0:, :] -= V @ (op @ (V.T @ C[l0:, :]))
    return C


def tsqrt(Rkk, Aik, ib):
    """DTSQT2 with inner blocking ib: QR of the triangle R_kk stacked on A_ik.

    Returns (R, V, T): R is Rkk with its upper triangle replaced by R~_kk (its
    strictly lower part, which holds V_kk, is left as it was); V overwrites
    A_ik; T is ib x b.  Section 3.1.
    """
    R = np.array(Rkk, dtype=np.float64, copy=True)
    A = np.array(Aik, dtype=np.float64, copy=True)
    nb = R.shape[0]
    # the bottom may be taller than b (the 2b x b tiles of Section 3.2's remark)
    assert R.shape == (nb, nb) and A.shape[1] == nb and nb % ib == 0
    T = np.zeros((ib, nb))
    for l0 in range(0, nb, ib):
        l1 = l0 + ib
        tau = np.zeros(ib)
        for c in range(l0, l1):
            # the reflector's top part is e_c: rows above c were annihilated
            # earlier and rows below c of the triangle are zero
            t, v2, beta = householder(R[c, c], A[:, c])
            R[c, c] = beta
            A[:, c] = v2
            tau[c - l0] = t
            if t != 0.0 and c + 1 < l1:
                w = R[c, c + 1:l1] + v2 @ A[:, c + 1:l1]
                R[c, c + 1:l1] -= t * w
                A[:, c + 1:l1] -= t * np.outer(v2, w)
        Vfull = _stacked_v(A[:, l0:l1], l0, ib, nb)
        Tl = larft(Vfull, tau)
        T[:, l0:l1] = Tl
        if l1 < nb:
            C = np.vstack([R[:, l1:], A[:, l1:]])
            C -= Vfull @ (Tl.T @ (Vfull.T @ C))
            R[l0:l1, l1:] = C[l0:l1, :]        # only the block's rows change
            A[:, l1:] = C[nb:, :]
    return R, A, T


def ssrfb(Akj, Aij, Vik, Tik, ib, trans=True):
    """DSSRFB: apply the reflectors [I; V_ik], T_ik of a TSQRT to the stacked
    pair [A_kj; A_ij] (each b x w).  Section 3.1.

    trans=True applies Q^T (blocks l = 0, 1, ..., T_l^T); trans=False Q.
    """
    nb = Vik.shape[1]                       # the top is b rows; the bottom may be taller
    C = np.vstack([np.asarray(Akj, dtype=np.float64),
                   np.asarray(Aij, dtype=np.float64)])
    blocks = list(range(0, nb, ib))
    if not trans:
        blocks.reverse()
    for l0 in blocks:
        l1 = l0 + ib
        Vfull = _stacked_v(Vik[:, l0:l1], l0, ib, nb)
        Tl = Tik[:, l0:l1]
        op = Tl.T if trans else Tl
        C -= Vfull @ (op @ (Vfull.T @ C))
    return C[:nb, :].copy(), C[nb:, :].copy()


class TiledFactors:
    """Result of Algorithm 1: the padded p*b x q*b array holding R and the
    tiled V, and the T blocks keyed by (i, k)."""

    def __init__(self, m, n, nb, ib, Ap, T):
        self.m, self.n, self.nb, self.ib = m, n, nb, ib
        self.p = Ap.shape[0] // nb
        self.q = Ap.shape[1] // nb
        self.Ap = Ap
        self.T = T

    def tile(self, i, j):
        nb = self.nb
        return self.Ap[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb]

    @property
    def F(self):
        """m x n array with R on/above the diagonal and the tiled V below."""
        return self.Ap[:self.m, :self.n].copy()

    @property
    def R(self):
        return np.triu(self.Ap[:self.m, :self.n])


def grid(m, n, nb):
    """Tile counts p = ceil(m/b), q = ceil(n/b)."""
    return max(1, math.ceil(m / nb)), max(1, math.ceil(n / nb))


def tiled_qr(A, nb, ib):
    """Algorithm 1 of the paper on the zero-padded tile grid."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    p, q = grid(m, n, nb)
    Ap = np.zeros((p * nb, q * nb))
    Ap[:m, :n] = A
    f = TiledFactors(m, n, nb, ib, Ap, {})
    tile = f.tile
    for k in range(min(p, q)):
        Fkk, Tkk = geqrt(tile(k, k), ib)
        tile(k, k)[:] = Fkk
        f.T[(k, k)] = Tkk
        for j in range(k + 1, q):
            tile(k, j)[:] = larfb(tile(k, j), tile(k, k), Tkk, ib, trans=True)
        for i in range(k + 1, p):
            R, V, Tik = tsqrt(tile(k, k), tile(i, k), ib)
            tile(k, k)[:] = R
            tile(i, k)[:] = V
            f.T[(i, k)] = Tik
            for j in range(k + 1, q):
                top, bot = ssrfb(tile(k, j), tile(i, j), V, Tik, ib, trans=True)
                tile(k, j)[:] = top
                tile(i, j)[:] = bot
    return f


def _padded_rows(f, B):
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    assert B.shape[0] == f.m
    Bp = np.zeros((f.p * f.nb, B.shape[1]))
    Bp[:f.m] = B
    return Bp


def apply_qt(f, B):
    """Q^T B from the tiled factors, replaying Algorithm 1's order: LARFB on
    row block k, then SSRFB on the pairs (k, i)."""
    Bp = _padded_rows(f, B)
    nb = f.nb
    rows = lambda i: slice(i * nb, (i + 1) * nb)
    for k in range(min(f.p, f.q)):
        Bp[rows(k)] = larfb(Bp[rows(k)], f.tile(k, k), f.T[(k, k)], f.ib, trans=True)
        for i in range(k + 1, f.p):
            top, bot = ssrfb(Bp[rows(k)], Bp[rows(i)], f.tile(i, k), f.T[(i, k)],
                             f.ib, trans=True)
            Bp[rows(k)], Bp[rows(i)] = top, bot
    return Bp[:f.m]


def apply_q(f, B):
    """Q B: the transposes of apply_qt's steps in reverse order."""
    Bp = _padded_rows(f, B)
    nb = f.nb
    rows = lambda i: slice(i * nb, (i + 1) * nb)
    for k in reversed(range(min(f.p, f.q))):
        for i in reversed(range(k + 1, f.p)):
            top, bot = ssrfb(Bp[rows(k)], Bp[rows(i)], f.tile(i, k), f.T[(i, k)],
                             f.ib, trans=False)
            Bp[rows(k)], Bp[rows(i)] = top, bot
        Bp[rows(k)] = larfb(Bp[rows(k)], f.tile(k, k), f.T[(k, k)], f.ib, trans=False)
    return Bp[:f.m]


def form_q(f, ncols=None):
    """Explicit Q (m x ncols, default m x m) = Q applied to the identity."""
    if ncols is None:
        ncols = f.m
    return apply_q(f, np.eye(f.m, ncols))


# ---------------------------------------------------------------------------
# Reduction-tree variant (an extension: the paper's panel is the flat chain of
# Algorithm 1).  For step k the rows k..p-1 are cut into domains of D tile
# rows.  Each domain is factored as in Algorithm 1 with its first row as the
# head (GEQRT on the head tile, TSQRT of the head's triangle with each later
# row of the domain); then the heads' triangles are merged by a binary tree of
# TTQRT (QR of two stacked upper triangles).  D >= p - k gives one domain:
# exactly Algorithm 1.  TTQRT's reflectors are upper triangular and are
# stored in the upper triangle of the eliminated head's tile (whose strictly
# lower part keeps its GEQRT reflectors); their T factors are kept apart.

def ttqrt(R1, R2, ib):
    """TTQRT: QR of the upper triangle R1 stacked on the upper triangle R2.
    This is TSQRT applied to [R1; triu(R2)]: the zeros below R2's diagonal
    stay exactly zero, so V comes out upper triangular.  Returns (R, V, T)."""
    return tsqrt(R1, np.triu(R2), ib)


def tree_heads(k, p, D):
    """Domain heads of step k: rows k, k+D, k+2D, ... below p."""
    return list(range(k, p, D))


def tree_merges(heads):
    """Binary-tree merges of the heads, level by level: at level l the head
    with index d (a multiple of 2^(l+1)) absorbs the head with index
    d + 2^l.  Returns [(level, a_row, b_row)] in execution order."""
    out = []
    H = len(heads)
    lvl = 0
    while (1 << lvl) < H:
        step = 1 << (lvl + 1)
        for d in range(0, H, step):
            if d + (1 << lvl) < H:
                out.append((lvl, heads[d], heads[d + (1 << lvl)]))
        lvl += 1
    return out


class TreeFactors(TiledFactors):
    """Tiled factors of the tree variant: T for GEQRT/TSQRT keyed (i, k), T2
    for TTQRT keyed (b, k) (b = the eliminated head)."""

    def __init__(self, m, n, nb, ib, D, Ap, T, T2):
        super().__init__(m, n, nb, ib, Ap, T)
        self.D = D
        self.T2 = T2


def _tt_v(tile):
    """The TTQRT reflectors stored in the upper triangle of a head tile."""
    return np.triu(tile)


def tree_qr(A, nb, ib, D):
    """Tiled QR with a per-panel reduction tree (domains of D tile rows)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    p, q = grid(m, n, nb)
    Ap = np.zeros((p * nb, q * nb))
    Ap[:m, :n] = A
    f = TreeFactors(m, n, nb, ib, D, Ap, {}, {})
    tile = f.tile
    for k in range(min(p, q)):
        heads = tree_heads(k, p, D)
        for h in heads:
            F, T = geqrt(tile(h, k), ib)
            tile(h, k)[:] = F
            f.T[(h, k)] = T
            for j in range(k + 1, q):
                tile(h, j)[:] = larfb(tile(h, j), tile(h, k), T, ib, trans=True)
            for i in range(h + 1, min(h + D, p)):
                R, V, T = tsqrt(tile(h, k), tile(i, k), ib)
                tile(h, k)[:] = R
                tile(i, k)[:] = V
                f.T[(i, k)] = T
                for j in range(k + 1, q):
                    top, bot = ssrfb(tile(h, j), tile(i, j), V, T, ib, trans=True)
                    tile(h, j)[:] = top
                    tile(i, j)[:] = bot
        for _, a, b in tree_merges(heads):
            R, V, T = ttqrt(tile(a, k), tile(b, k), ib)
            tile(a, k)[:] = R                                   # upper: merged R
            tile(b, k)[:] = np.tril(tile(b, k), -1) + np.triu(V)  # upper: V_tt
            f.T2[(b, k)] = T
            for j in range(k + 1, q):
                top, bot = ssrfb(tile(a, j), tile(b, j), _tt_v(tile(b, k)), T, ib, trans=True)
                tile(a, j)[:] = top
                tile(b, j)[:] = bot
    return f


def _tree_steps(f, B_rows_tile, trans):
    """Q^T (trans) or Q applied to the row tiles of a right-hand side."""
    nb, ib, D = f.nb, f.ib, f.D
    kt = min(f.p, f.q)

    def ops(k):
        out = []
        heads = tree_heads(k, f.p, D)
        for h in heads:
            out.append(("G", h, None))
            for i in range(h + 1, min(h + D, f.p)):
                out.append(("S", h, i))
        for _, a, b in tree_merges(heads):
            out.append(("T", a, b))
        return out

    steps = [(k, o) for k in range(kt) for o in ops(k)]
    if not trans:
        steps.reverse()
    Bt = B_rows_tile
    for k, (kind, a, b) in steps:
        if kind == "G":
            Bt(a)[:] = larfb(Bt(a), f.tile(a, k), f.T[(a, k)], ib, trans=trans)
        elif kind == "S":
            top, bot = ssrfb(Bt(a), Bt(b), f.tile(b, k), f.T[(b, k)], ib, trans=trans)
            Bt(a)[:], Bt(b)[:] = top, bot
        else:
            top, bot = ssrfb(Bt(a), Bt(b), _tt_v(f.tile(b, k)), f.T2[(b, k)], ib, trans=trans)
            Bt(a)[:], Bt(b)[:] = top, bot


def tree_apply_qt(f, B):
    Bp = _padded_rows(f, B)
    nb = f.nb
    _tree_steps(f, lambda i: Bp[i * nb:(i + 1) * nb], trans=True)
    return Bp[:f.m]


def tree_apply_q(f, B):
    Bp = _padded_rows(f, B)
    nb = f.nb
    _tree_steps(f, lambda i: Bp[i * nb:(i + 1) * nb], trans=False)
    return Bp[:f.m]


# ---------------------------------------------------------------------------
# Applying and forming Q (the LAPACK DORMQR / DORGQR pair that the paper's
# conclusion names as direct derivations of the tiled factorization).  These
# are the plain definitions on top of apply_q / apply_qt: the right-hand side
# forms follow from (C Q)^T = Q^T C^T and (C Q^T)^T = Q C^T, and the explicit
# Q columns are Q applied to the leading columns of the identity.

def _left(f, trans, C):
    tree = isinstance(f, TreeFactors)
    if trans:
        return tree_apply_qt(f, C) if tree else apply_qt(f, C)
    return tree_apply_q(f, C) if tree else apply_q(f, C)


def ormqr(f, side, trans, C):
    """op(Q) C (side 'L') or C op(Q) (side 'R'), op(Q) = Q^T when trans is
    'T' and Q when 'N'.  Q is m x m (m = f.m); C is m x c ('L') or c x m ('R')."""
    C = np.asarray(C, dtype=np.float64)
    t = trans in ("T", "t")
    if side in ("L", "l"):
        assert C.shape[0] == f.m
        return _left(f, t, C)
    assert C.shape[1] == f.m
    return _left(f, not t, C.T).T


def orgqr(f, ncols):
    """The first ncols columns of Q (m x ncols, 0 <= ncols <= m)."""
    assert 0 <= ncols <= f.m
    return _left(f, False, np.eye(f.m, ncols))



# ---------------------------------------------------------------------------
# 2b x b tiles below the diagonal (Section 3.2 remarks that 2b x b blocks cut
# the tiled algorithm's extra work from 25 % to 12.5 %; Section 5 repeats it).
# Reading: the diagonal tile stays b x b (GEQRT, LARFB); below it, step k
# takes the rows k+1, k+2, ... in pairs, so each TSQRT factors R_kk stacked
# on a 2b x b block (two b x b storage tiles) and each SSRFB updates the top
# tile with a 2b-row bottom.  An odd last row is a single b x b bottom.  The
# reflectors of a pair are stored in its two tiles and its T under the pair's
# first row.

def pair_groups(k, p):
    """Bottom groups of step k: [(h, rows)], rows = (h,) or (h, h + 1)."""
    out = []
    h = k + 1
    while h < p:
        rows = (h, h + 1) if h + 1 < p else (h,)
        out.append((h, rows))
        h += len(rows)
    return out


class PairFactors(TiledFactors):
    pass


def _stack(f, rows, j):
    return np.vstack([f.tile(r, j) for r in rows])


def _unstack(f, rows, j, X):
    nb = f.nb
    for a, r in enumerate(rows):
        f.tile(r, j)[:] = X[a * nb:(a + 1) * nb]


def tiled_qr_pairs(A, nb, ib):
    """Algorithm 1 with 2b x b bottoms (pair_groups) on the zero-padded grid."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    p, q = grid(m, n, nb)
    Ap = np.zeros((p * nb, q * nb))
    Ap[:m, :n] = A
    f = PairFactors(m, n, nb, ib, Ap, {})
    tile = f.tile
    for k in range(min(p, q)):
        Fkk, Tkk = geqrt(tile(k, k), ib)
        tile(k, k)[:] = Fkk
        f.T[(k, k)] = Tkk
        for j in range(k + 1, q):
            tile(k, j)[:] = larfb(tile(k, j), tile(k, k), Tkk, ib, trans=True)
        for h, rows in pair_groups(k, p):
            R, V, Th = tsqrt(tile(k, k), _stack(f, rows, k), ib)
            tile(k, k)[:] = R
            _unstack(f, rows, k, V)
            f.T[(h, k)] = Th
            for j in range(k + 1, q):
                top, bot = ssrfb(tile(k, j), _stack(f, rows, j), V, Th, ib, trans=True)
                tile(k, j)[:] = top
                _unstack(f, rows, j, bot)
    return f


def _pair_steps(f, Bp, trans):
    nb = f.nb
    rows_of = lambda i: Bp[i * nb:(i + 1) * nb]
    steps = list(range(min(f.p, f.q)))
    if not trans:
        steps.reverse()
    for k in steps:
        groups = pair_groups(k, f.p)
        if trans:
            rows_of(k)[:] = larfb(rows_of(k), f.tile(k, k), f.T[(k, k)], f.ib, trans=True)
        else:
            groups.reverse()
        for h, rows in groups:
            V = _stack(f, rows, k)
            bot = np.vstack([rows_of(r) for r in rows])
            top, bot = ssrfb(rows_of(k), bot, V, f.T[(h, k)], f.ib, trans=trans)
            rows_of(k)[:] = top
            for a, r in enumerate(rows):
                rows_of(r)[:] = bot[a * nb:(a + 1) * nb]
        if not trans:
            rows_of(k)[:] = larfb(rows_of(k), f.tile(k, k), f.T[(k, k)], f.ib, trans=False)


def pairs_apply_qt(f, B):
    Bp = _padded_rows(f, B)
    _pair_steps(f, Bp, trans=True)
    return Bp[:f.m]


def pairs_apply_q(f, B):
    Bp = _padded_rows(f, B)
    _pair_steps(f, Bp, trans=False)
    return Bp[:f.m]
