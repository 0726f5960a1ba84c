"""Tiled LU with pairwise pivoting (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's conclusion (Section 5) states that the LU factorization runs with
an algorithm analogous to the tiled QR of Section 3, citing the out-of-core
LU works, at a higher flop overhead.  Reading used here (the paper gives no
kernel detail): Algorithm 1's loop nest with four LU kernels in place of the
QR ones --

  GETRF(k)      A_kk -> L_kk, U_kk and row interchanges (partial pivoting
                within the tile)
  GESSM(k, j)   A_kj <- L_kk^-1 P_kk A_kj
  TSTRF(k, i)   [U_kk; A_ik] -> U~_kk and L_ik, pivoting between row c of
                U_kk and the rows of A_ik for each column c (pairwise, or
                "incremental", pivoting)
  SSSSM(k,i,j)  [A_kj; A_ij] <- the TSTRF transformations applied to them

Each kernel works in blocks of ib columns.  Within a block the interchanges
act on whole block rows (the block is an ordinary partially pivoted LU,
P A = L U); across blocks the transformations are applied in sequence, so an
interchange of block l leaves the multipliers of earlier blocks in place.
Applying block l to other columns: its interchanges in order, then the top
rows of the block are solved with the block's unit lower triangle L11, then
the rows below subtract L21 times them.  ib = b gives the unblocked kernels.

TSTRF's candidates for column c are row c of the (upper triangular) top and
every row of the bottom tile; the other top rows hold zeros in column c.  The
multipliers of rows that move into the top go to a separate ib x ib triangle
per block (the top tile's strictly lower part already holds L_kk).

Ties in the pivot search pick the first row in the order [top row c, bottom
rows 0..b-1] (GETRF: rows c..b-1), as LAPACK's IDAMAX does.  An exact zero
pivot leaves its column unscaled (the next TSTRF may still find a nonzero
pivot below); the solve then reports a zero on U's diagonal.
"""
import numpy as np


def _block_solve(L11, X):
    """L11^-1 X for unit lower triangular L11 (forward substitution)."""
    X = np.array(X, dtype=np.float64, copy=True)
    for r in range(1, L11.shape[0]):
        X[r] -= L11[r, :r] @ X[:r]
    return X


def getrf(A, ib):
    """GETRF on one tile (b x b).  Returns (F, piv): F holds U on and above
    the diagonal and the multipliers below; piv[c] is the tile row swapped
    with row c in column c's step (piv[c] == c: none)."""
    F = np.array(A, dtype=np.float64, copy=True)
    b = F.shape[0]
    piv = np.arange(b)
    for l0 in range(0, b, ib):
        cols = slice(l0, l0 + ib)
        for c in range(l0, l0 + ib):
            r = c + int(np.argmax(np.abs(F[c:, c])))
            piv[c] = r
            if r != c:
                F[[c, r], cols] = F[[r, c], cols]
            if F[c, c] != 0.0:
                F[c + 1:, c] = F[c + 1:, c] / F[c, c]
            F[c + 1:, c + 1:l0 + ib] -= np.outer(F[c + 1:, c], F[c, c + 1:l0 + ib])
        # the block applied to the tile's trailing columns
        rest = slice(l0 + ib, b)
        for c in range(l0, l0 + ib):
            if piv[c] != c:
                F[[c, piv[c]], rest] = F[[piv[c], c], rest]
        L11 = np.tril(F[l0:l0 + ib, l0:l0 + ib], -1) + np.eye(ib)
        F[l0:l0 + ib, rest] = _block_solve(L11, F[l0:l0 + ib, rest])
        F[l0 + ib:, rest] -= F[l0 + ib:, l0:l0 + ib] @ F[l0:l0 + ib, rest]
    return F, piv


def gessm(C, F, piv, ib):
    """L_kk^-1 P_kk C with GETRF's factors F, piv (block sequence)."""
    C = np.array(C, dtype=np.float64, copy=True)
    b = F.shape[0]
    for l0 in range(0, b, ib):
        for c in range(l0, l0 + ib):
            if piv[c] != c:
                C[[c, piv[c]]] = C[[piv[c], c]]
        L11 = np.tril(F[l0:l0 + ib, l0:l0 + ib], -1) + np.eye(ib)
        C[l0:l0 + ib] = _block_solve(L11, C[l0:l0 + ib])
        C[l0 + ib:] -= F[l0 + ib:, l0:l0 + ib] @ C[l0:l0 + ib]
    return C


def tstrf(U, A, ib):
    """TSTRF on [U; A] (U: the upper triangle of the top tile, A: the bottom
    tile).  Returns (U~, Lb, L1, piv): U~ the new upper triangle, Lb the
    bottom tile's multipliers (b x b), L1 the ib x b array of the blocks'
    unit lower triangles (block l in columns l*ib .. (l+1)*ib - 1, strictly
    lower part significant), piv[c] = -1 (top row c kept) or the bottom row
    swapped with top row c."""
    b = U.shape[0]            # columns; the bottom may be taller (2b x b blocks)
    Ut = np.triu(np.array(U, dtype=np.float64, copy=True))
    Lb = np.array(A, dtype=np.float64, copy=True)
    assert Lb.shape[1] == b
    L1 = np.zeros((ib, b))
    piv = np.full(b, -1)
    for l0 in range(0, b, ib):
        cols = slice(l0, l0 + ib)
        # the top rows of the block: U~ above the diagonal, multipliers below
        Tp = np.array(Ut[l0:l0 + ib, cols], copy=True)
        for cc in range(ib):
            c = l0 + cc
            cand = np.concatenate(([Tp[cc, cc]], Lb[:, c]))
            a = int(np.argmax(np.abs(cand)))
            if a > 0:
                r = a - 1
                piv[c] = r
                tmp = np.array(Tp[cc, :], copy=True)
                Tp[cc, :] = Lb[r, cols]
                Lb[r, cols] = tmp
            if Tp[cc, cc] != 0.0:
                Lb[:, c] = Lb[:, c] / Tp[cc, cc]
            Lb[:, c + 1:l0 + ib] -= np.outer(Lb[:, c], Tp[cc, cc + 1:])
        Ut[l0:l0 + ib, cols] = np.triu(Tp)
        L1[:, cols] = np.tril(Tp, -1)
        # the block applied to the trailing columns of [U; A]
        rest = slice(l0 + ib, b)
        top = np.array(Ut[l0:l0 + ib, rest], copy=True)
        for cc in range(ib):
            c = l0 + cc
            if piv[c] >= 0:
                r = piv[c]
                tmp = np.array(top[cc], copy=True)
                top[cc] = Lb[r, rest]
                Lb[r, rest] = tmp
        top = _block_solve(np.tril(Tp, -1) + np.eye(ib), top)
        Ut[l0:l0 + ib, rest] = top
        Lb[:, rest] -= Lb[:, cols] @ top
    return Ut, Lb, L1, piv


def ssssm(Ct, Cb, Lb, L1, piv, ib):
    """[Ct; Cb] <- TSTRF's transformations (Lb, L1, piv) applied to them."""
    Ct = np.array(Ct, dtype=np.float64, copy=True)
    Cb = np.array(Cb, dtype=np.float64, copy=True)
    b = Lb.shape[1]            # columns of the factored panel (rows of the top)
    for l0 in range(0, b, ib):
        for cc in range(ib):
            c = l0 + cc
            if piv[c] >= 0:
                r = piv[c]
                Ct[[c]], Cb[[r]] = Cb[[r]].copy(), Ct[[c]].copy()
        L11 = np.tril(L1[:, l0:l0 + ib], -1) + np.eye(ib)
        Ct[l0:l0 + ib] = _block_solve(L11, Ct[l0:l0 + ib])
        Cb -= Lb[:, l0:l0 + ib] @ Ct[l0:l0 + ib]
    return Ct, Cb


class TiledLU:
    """Tiles of the factored, zero-padded A (U above the diagonal tiles' and
    in the tiles right of them, multipliers elsewhere), GETRF/TSTRF pivots
    and the TSTRF triangles L1[(i, k)]."""

    def __init__(self, m, n, nb, ib, Ap, piv, L1):
        self.m, self.n, self.nb, self.ib = m, n, nb, ib
        self.p, self.q = -(-m // nb), -(-n // nb)
        self.Ap, self.piv, self.L1 = Ap, piv, L1

    def tile(self, i, j):
        nb = self.nb
        return self.Ap[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb]

    @property
    def U(self):
        """The upper triangular factor (m x n, from the padded tiles)."""
        return np.triu(self.Ap)[:self.m, :self.n]


def tiled_lu(A, nb, ib):
    """Algorithm 1's loop nest with the LU kernels on the zero-padded A.
    Zero padding: a zero row never becomes a pivot over a nonzero candidate
    and a padded column of zeros gets no multipliers, so the factors of
    A[:m, :n] are unchanged.  Requires ib | nb."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    assert nb % ib == 0
    p, q = -(-m // nb), -(-n // nb)
    Ap = np.zeros((p * nb, q * nb))
    Ap[:m, :n] = A
    f = TiledLU(m, n, nb, ib, Ap, {}, {})
    t = f.tile
    for k in range(min(p, q)):
        F, pv = getrf(t(k, k), ib)
        t(k, k)[:] = F
        f.piv[(k, k)] = pv
        for j in range(k + 1, q):
            t(k, j)[:] = gessm(t(k, j), F, pv, ib)
        for i in range(k + 1, p):
            Ut, Lb, L1, pv2 = tstrf(t(k, k), t(i, k), ib)
            t(k, k)[:] = np.tril(t(k, k), -1) + Ut
            t(i, k)[:] = Lb
            f.piv[(i, k)] = pv2
            f.L1[(i, k)] = L1
            for j in range(k + 1, q):
                top, bot = ssssm(t(k, j), t(i, j), Lb, L1, pv2, ib)
                t(k, j)[:] = top
                t(i, j)[:] = bot
    return f


def apply_linv(f, B):
    """The factorization's transformations (everything but U) applied to B
    in Algorithm 1's order: B <- ... SSSSM(k, i) ... GESSM(k) ... B."""
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    nb = f.nb
    Bp = np.zeros((f.p * nb, B.shape[1]))
    Bp[:f.m] = B
    rows = lambda i: slice(i * nb, (i + 1) * nb)
    for k in range(min(f.p, f.q)):
        Bp[rows(k)] = gessm(Bp[rows(k)], f.tile(k, k), f.piv[(k, k)], f.ib)
        for i in range(k + 1, f.p):
            top, bot = ssssm(Bp[rows(k)], Bp[rows(i)], f.tile(i, k), f.L1[(i, k)], f.piv[(i, k)], f.ib)
            Bp[rows(k)], Bp[rows(i)] = top, bot
    return Bp[:f.m]


def lu_solve(f, B):
    """X = A^-1 B for square A: the transformations, then back substitution
    with U."""
    assert f.m == f.n
    Y = apply_linv(f, B)
    U = f.U
    X = np.array(Y, dtype=np.float64, copy=True)
    n = f.n
    for r in range(n - 1, -1, -1):
        X[r] = (X[r] - U[r, r + 1:] @ X[r + 1:]) / U[r, r]
    return X



# ---------------------------------------------------------------------------
# 2b x b bottoms (the non-square blocks of Section 3.2's remark, applied to
# the LU analogue): the rows below each diagonal tile are taken in pairs, so
# each TSTRF pivots row c of U_kk against 2b rows and each SSSSM updates the
# top tile with a 2b-row bottom.  The interchanges of a pair index its 2b
# rows (0 .. 2b-1); its multipliers are stored in its two tiles and its L1
# triangles under its first row.

def _pair_groups(k, p):
    out, h = [], k + 1
    while h < p:
        rows = (h, h + 1) if h + 1 < p else (h,)
        out.append((h, rows))
        h += len(rows)
    return out


def tiled_lu_pairs(A, nb, ib):
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    assert nb % ib == 0
    p, q = -(-m // nb), -(-n // nb)
    Ap = np.zeros((p * nb, q * nb))
    Ap[:m, :n] = A
    f = TiledLU(m, n, nb, ib, Ap, {}, {})
    t = f.tile
    stack = lambda rows, j: np.vstack([t(r, j) for r in rows])

    def unstack(rows, j, X):
        for a, r in enumerate(rows):
            t(r, j)[:] = X[a * nb:(a + 1) * nb]

    for k in range(min(p, q)):
        F, pv = getrf(t(k, k), ib)
        t(k, k)[:] = F
        f.piv[(k, k)] = pv
        for j in range(k + 1, q):
            t(k, j)[:] = gessm(t(k, j), F, pv, ib)
        for h, rows in _pair_groups(k, p):
            Ut, Lb, L1, pv2 = tstrf(t(k, k), stack(rows, k), ib)
            t(k, k)[:] = np.tril(t(k, k), -1) + Ut
            unstack(rows, k, Lb)
            f.piv[(h, k)] = pv2
            f.L1[(h, k)] = L1
            for j in range(k + 1, q):
                top, bot = ssssm(t(k, j), stack(rows, j), Lb, L1, pv2, ib)
                t(k, j)[:] = top
                unstack(rows, j, bot)
    f.pairs = True
    return f


def pairs_apply_linv(f, B):
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    nb = f.nb
    Bp = np.zeros((f.p * nb, B.shape[1]))
    Bp[:f.m] = B
    rows_of = lambda i: slice(i * nb, (i + 1) * nb)
    for k in range(min(f.p, f.q)):
        Bp[rows_of(k)] = gessm(Bp[rows_of(k)], f.tile(k, k), f.piv[(k, k)], f.ib)
        for h, rows in _pair_groups(k, f.p):
            Lb = np.vstack([f.tile(r, k) for r in rows])
            bot = np.vstack([Bp[rows_of(r)] for r in rows])
            top, bot = ssssm(Bp[rows_of(k)], bot, Lb, f.L1[(h, k)], f.piv[(h, k)], f.ib)
            Bp[rows_of(k)] = top
            for a, r in enumerate(rows):
                Bp[rows_of(r)] = bot[a * nb:(a + 1) * nb]
    return Bp[:f.m]


def pairs_lu_solve(f, B):
    assert f.m == f.n
    X = pairs_apply_linv(f, B)
    U = f.U
    for r in range(f.n - 1, -1, -1):
        X[r] = (X[r] - U[r, r + 1:] @ X[r + 1:]) / U[r, r]
    return X
