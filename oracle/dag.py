"""Task set, dependency DAG and operation count of Algorithm 1 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section 3.3: Algorithm 1 is a DAG whose nodes are the tile tasks and whose
edges are the data dependencies between them (read-after-write and
write-after-write on tiles).  The edges are derived here from first
principles, by replaying Algorithm 1 and recording for each tile its last
writer and its readers (a plain data-flow analysis), not from a formula.

Section 3.3 also fixes the scheduling priorities: GEQRT highest, then TSQRT,
LARFB and SSRFB.  Section 3.2 gives the per-kernel operation counts
(GEQRT 2b^3, LARFB 3b^3, TSQRT 10/3 b^3, SSRFB 5b^3) and their sum (Eq.
opcount).

Tasks are tuples (kind, k, i, j) with kind in GEQRT / LARFB / TSQRT / SSRFB;
unused indices are -1.
"""

GEQRT, LARFB, TSQRT, SSRFB = "GEQRT", "LARFB", "TSQRT", "SSRFB"

#: Section 3.3 priority order, highest first.
PRIORITY = {GEQRT: 0, TSQRT: 1, LARFB: 2, SSRFB: 3}

#: Section 3.2 per-task operation counts in units of b^3 (ib = b).
KERNEL_FLOPS_B3 = {GEQRT: 2.0, LARFB: 3.0, TSQRT: 10.0 / 3.0, SSRFB: 5.0}


def tasks(p, q):
    """Algorithm 1's tasks in its own sequential order."""
    out = []
    for k in range(min(p, q)):
        out.append((GEQRT, k, k, k))
        for j in range(k + 1, q):
            out.append((LARFB, k, k, j))
        for i in range(k + 1, p):
            out.append((TSQRT, k, i, k))
            for j in range(k + 1, q):
                out.append((SSRFB, k, i, j))
    return out


def _accesses(task):
    """(reads, writes) of a task as sets of (tile, part) where part is 'U'
    (upper triangle incl. diagonal), 'L' (strictly lower) or 'F' (full).
    Section 3.1: GEQRT writes all of A_kk; LARFB reads V_kk (lower) and T_kk,
    writes A_kj; TSQRT reads/writes R_kk (upper) and A_ik, writes T_ik; SSRFB
    reads V_ik (A_ik) and T_ik, reads/writes A_kj and A_ij."""
    kind, k, i, j = task
    if kind == GEQRT:
        return ({((k, k), "F")}, {((k, k), "F"), (("T", k, k), "F")})
    if kind == LARFB:
        return ({((k, k), "L"), (("T", k, k), "F"), ((k, j), "F")},
                {((k, j), "F")})
    if kind == TSQRT:
        return ({((k, k), "U"), ((i, k), "F")},
                {((k, k), "U"), ((i, k), "F"), (("T", i, k), "F")})
    if kind == SSRFB:
        return ({((i, k), "F"), (("T", i, k), "F"), ((k, j), "F"), ((i, j), "F")},
                {((k, j), "F"), ((i, j), "F")})
    raise ValueError(kind)


def _overlap(a, b):
    """Do two parts of the same tile share an element?"""
    return a == "F" or b == "F" or a == b


def edges(p, q):
    """Dependency edges (pred, succ) from replaying Algorithm 1 sequentially:
    RAW, WAR and WAW on overlapping tile parts.  Transitively redundant edges
    are kept; use ``reduced_edges`` for the minimal set."""
    order = tasks(p, q)
    last_writer = {}    # (tile, part) -> task
    readers = {}        # (tile, part) -> list of tasks since last write
    out = set()
    for t in order:
        reads, writes = _accesses(t)
        for tile, part in reads:
            for (tile2, part2), w in last_writer.items():
                if tile2 == tile and _overlap(part, part2):
                    out.add((w, t))
        for tile, part in writes:
            for (tile2, part2), w in last_writer.items():
                if tile2 == tile and _overlap(part, part2):
                    out.add((w, t))
            for (tile2, part2), rs in readers.items():
                if tile2 == tile and _overlap(part, part2):
                    for r in rs:
                        if r != t:
                            out.add((r, t))
        for tile, part in reads:
            readers.setdefault((tile, part), []).append(t)
        for tile, part in writes:
            # a write of a part supersedes earlier writes/reads of the parts it covers
            for key in list(last_writer):
                if key[0] == tile and (part == "F" or key[1] == part):
                    del last_writer[key]
            for key in list(readers):
                if key[0] == tile and (part == "F" or key[1] == part):
                    del readers[key]
            last_writer[(tile, part)] = t
    return out


def reduced_edges(p, q):
    """Transitive reduction of ``edges`` (the DAG's Hasse diagram)."""
    e = edges(p, q)
    succ = {}
    for a, b in e:
        succ.setdefault(a, set()).add(b)
    order = tasks(p, q)
    pos = {t: n for n, t in enumerate(order)}
    # reachability by DFS in topological order (small graphs only)
    reach = {}
    for t in reversed(order):
        r = set()
        for s in succ.get(t, ()):
            r.add(s)
            r |= reach[s]
        reach[t] = r
    keep = set()
    for a, b in e:
        # drop (a, b) if some other successor c of a reaches b
        if not any(b in reach[c] for c in succ[a] if c != b and pos[c] < pos[b]):
            keep.add((a, b))
    return keep


def counts_per_step(p, q):
    """Number of tasks of each kind per outer step k, counted from the
    enumeration (Section 3.2 states 1, q-k, p-k and (p-k)(q-k) with k
    counted from 1; here k counts from 0)."""
    out = []
    for k in range(min(p, q)):
        c = {GEQRT: 0, LARFB: 0, TSQRT: 0, SSRFB: 0}
        for t in tasks(p, q):
            if t[1] == k:
                c[t[0]] += 1
        out.append(c)
    return out


def opcount_tiles(p, q):
    """Sum of the per-task counts of Section 3.2 over Algorithm 1, in b^3."""
    return sum(KERNEL_FLOPS_B3[t[0]] for t in tasks(p, q))


def lapack_flops(m, n):
    """2 n^2 (m - n/3), the Householder QR count of Section 2 (m >= n)."""
    return 2.0 * n * n * (m - n / 3.0)


def critical_path(p, q, weights=None):
    """Longest weighted path through the DAG (weights in b^3 by kind)."""
    w = weights or KERNEL_FLOPS_B3
    e = edges(p, q)
    preds = {}
    for a, b in e:
        preds.setdefault(b, []).append(a)
    best = {}
    for t in tasks(p, q):
        best[t] = w[t[0]] + max((best[a] for a in preds.get(t, ())), default=0.0)
    return max(best.values())


# ---------------------------------------------------------------------------
# 2b x b bottoms (Section 3.2's remark: 2b x b blocks cut the extra work from
# 25 % to 12.5 %).  The per-task counts follow the same accounting as the
# b x b ones: a TSQRT whose bottom has h*b rows does the Householder updates
# (2 h b^3) and the T formation (h b^3 + b^3/3); an SSRFB forms W = top +
# V^T bottom (2 h b^3), T^T W (b^3) and bottom -= V W (2 h b^3).  h = 1 gives
# Section 3.2's 10/3 and 5.

def tall_kernel_flops_b3(kind, h):
    """Per-task count in b^3 of a TS kernel with an h*b-row bottom."""
    if kind == TSQRT:
        return 3.0 * h + 1.0 / 3.0
    if kind == SSRFB:
        return 4.0 * h + 1.0
    return KERNEL_FLOPS_B3[kind]


def opcount_pairs(p, q):
    """Operation count in b^3 of Algorithm 1 with the rows below each
    diagonal tile taken in pairs (2b x b bottoms; an odd last row alone)."""
    total = 0.0
    for k in range(min(p, q)):
        total += KERNEL_FLOPS_B3[GEQRT] + (q - k - 1) * KERNEL_FLOPS_B3[LARFB]
        i = k + 1
        while i < p:
            h = 2 if i + 1 < p else 1
            total += tall_kernel_flops_b3(TSQRT, h) + (q - k - 1) * tall_kernel_flops_b3(SSRFB, h)
            i += h
    return total
