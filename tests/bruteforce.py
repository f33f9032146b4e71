"""Brute-force enumeration helpers for the pins (small rows and tiny ILPs only).

Everything here follows the definitions directly: the feasible set of a row by enumerating
{0,1}^k, min-marginals as constrained minima over that set (Sec. 3.2, eq. min-marginals),
the ILP optimum by enumerating all points, and BDD walks along lo/hi arcs.
"""
from __future__ import annotations

import numpy as np

TOP, BOT = -1, -2


def assignments(k: int) -> np.ndarray:
    """All points of {0,1}^k as rows; bit t of the row index is x_t."""
    idx = np.arange(2 ** k, dtype=np.int64)
    return ((idx[:, None] >> np.arange(k)) & 1).astype(np.int64)


def row_feasible(vals, b, sense) -> np.ndarray:
    X = assignments(len(vals))
    s = X @ np.asarray(vals, np.int64)
    if sense < 0:
        return s <= b
    if sense > 0:
        return s >= b
    return s == b


def canonical_rows(inst):
    """Rows with zero coefficients dropped and columns sorted ascending."""
    out = []
    for cols, vals, b, sense in inst.rows():
        keep = vals != 0
        cols, vals = cols[keep], vals[keep]
        o = np.argsort(cols, kind="stable")
        out.append((cols[o].astype(np.int64), vals[o].astype(np.int64), b, sense))
    return out


def split_bdds(canon):
    """Split a canonical export into per-BDD lists of layers (lo, hi, minsum, var)."""
    bdds = []
    o = 0
    v = 0
    for depth in canon["bdd_depth"]:
        layers = []
        for _ in range(int(depth)):
            w = int(canon["occ_width"][o])
            layers.append(dict(var=int(canon["occ_var"][o]), csr=int(canon["occ_csr"][o]),
                               lo=canon["lo"][v:v + w].astype(np.int64),
                               hi=canon["hi"][v:v + w].astype(np.int64),
                               minsum=canon["minsum"][v:v + w].astype(np.int64)
                               if "minsum" in canon else None))
            o += 1
            v += w
        bdds.append(layers)
    return bdds


def walk(layers, x) -> tuple[bool, list[int]]:
    """Follow arcs for assignment x (one bit per layer); returns (accepted, visited node ids)."""
    node = 0
    path = []
    for l, lay in enumerate(layers):
        path.append(node)
        nxt = lay["hi"][node] if x[l] else lay["lo"][node]
        if nxt == BOT:
            return False, path
        if nxt == TOP:
            assert l == len(layers) - 1, "top reached before the last layer"
            return True, path
        node = int(nxt)
    raise AssertionError("path ran past the last layer")


def layer_subfunction_count(feas: np.ndarray, k: int, l: int) -> int:
    """Number of distinct not-identically-false subfunctions after fixing x_0..x_{l-1}."""
    T = feas.reshape(2 ** (k - l), 2 ** l).T  # rows: prefixes (low bits), cols: suffixes
    T = T[T.any(axis=1)]
    if T.shape[0] == 0:
        return 0
    return int(np.unique(np.packbits(T, axis=1), axis=0).shape[0])


def min_marginals_enum(vals, b, sense, lam):
    """m^beta_t = min over feasible x with x_t = beta of x.lam (eq. min-marginals)."""
    k = len(vals)
    X = assignments(k)
    feas = row_feasible(vals, b, sense)
    cost = X @ np.asarray(lam, np.float64)
    m0 = np.full(k, np.inf)
    m1 = np.full(k, np.inf)
    for t in range(k):
        s0 = feas & (X[:, t] == 0)
        s1 = feas & (X[:, t] == 1)
        if s0.any():
            m0[t] = cost[s0].min()
        if s1.any():
            m1[t] = cost[s1].min()
    E = cost[feas].min()
    return m0, m1, E, int(feas.sum())


def ilp_optimum(inst) -> float:
    """min c.x over all feasible x in {0,1}^n (n <= 22)."""
    n = inst.n
    assert n <= 22
    X = assignments(n)
    ok = np.ones(X.shape[0], dtype=bool)
    for cols, vals, b, sense in inst.rows():
        s = X[:, cols] @ vals.astype(np.int64)
        ok &= (s <= b) if sense < 0 else ((s >= b) if sense > 0 else (s == b))
    cost = X @ inst.c.astype(np.float64)
    return float(cost[ok].min())


def potts_map(H, W, L, c) -> float:
    """Minimum Potts energy over all labelings of an HxW grid (local-polytope costs c)."""
    import itertools
    npx = H * W
    edges = []
    for r in range(H):
        for q in range(W):
            i = r * W + q
            if q < W - 1:
                edges.append((i, i + 1))
            if r < H - 1:
                edges.append((i, i + W))
    nx = npx * L
    best = np.inf
    for lab in itertools.product(range(L), repeat=npx):
        e = sum(float(c[i * L + lab[i]]) for i in range(npx))
        for t, (i, j) in enumerate(edges):
            e += float(c[nx + t * L * L + lab[i] * L + lab[j]])
        best = min(best, e)
    return best


# ------------------------------------------------------------------------------------------
# Alg. 1 and the deferred-averaging schedule by enumeration, with a variable order
# (Appendix A.3) and the SRMP averaging sets (Appendix A.4)
# ------------------------------------------------------------------------------------------

class EnumDual:
    """Dual state lambda^j_i per row j and position t (variables of the row in the order given
    by rank), with min-marginals and energies taken by enumeration of X_j."""

    def __init__(self, inst, rank=None):
        rank = np.arange(inst.n) if rank is None else np.asarray(rank)
        self.n = inst.n
        self.c = inst.c.astype(np.float64)
        self.rows = []
        for cols, vals, b, sense in canonical_rows(inst):
            o = np.argsort(rank[cols], kind="stable")
            self.rows.append((cols[o], vals[o], b, sense))
        self.occ = [[] for _ in range(inst.n)]  # per variable: (row, position), rows ascending
        for j, (cols, _, _, _) in enumerate(self.rows):
            for t, i in enumerate(cols):
                self.occ[int(i)].append((j, t))
        self.order = np.argsort(rank, kind="stable")
        self.lam = [np.array([self.c[i] / len(self.occ[i]) for i in cols]) for cols, *_ in self.rows]
        self.P = np.zeros(inst.n)

    def mm(self, j):
        cols, vals, b, sense = self.rows[j]
        return min_marginals_enum(vals, b, sense, self.lam[j])

    def bound(self):
        tot = sum(self.mm(j)[2] for j in range(len(self.rows)))
        s = np.zeros(self.n)
        for j, (cols, *_) in enumerate(self.rows):
            s[cols] += self.lam[j]
        return tot + np.minimum(0.0, self.c - s).sum()

    def takes(self, j, t, forward):
        """(j, position t) is in J_i^> (forward) / J_i^< (backward)."""
        return t < len(self.rows[j][0]) - 1 if forward else t > 0

    def weights(self, i, forward, srmp):
        """Share of the summed difference that each subproblem of variable i receives."""
        occ = self.occ[i]
        if not occ:
            return []
        if srmp:
            mask = [self.takes(j, t, forward) for j, t in occ]
            if any(mask):
                return [1.0 / sum(mask) if m else 0.0 for m in mask]
        return [1.0 / len(occ)] * len(occ)


def _diff(m0, m1):
    return 0.0 if np.isinf(m0) or np.isinf(m1) else m1 - m0


def sequential_enum(inst, iters, rank=None, srmp=False):
    """Alg. 1: forward then backward over the variable order; eq. mma-update, or
    eq. srmp-update with J_i^> forward and J_i^< backward.  Returns the bound per iteration."""
    D = EnumDual(inst, rank)
    trace = []
    for _ in range(iters):
        for forward, seq in ((True, D.order), (False, D.order[::-1])):
            for i in seq:
                occ = D.occ[int(i)]
                if not occ:
                    continue
                d = []
                for j, t in occ:
                    m0, m1, _, _ = D.mm(j)
                    d.append(_diff(m0[t], m1[t]))
                S = sum(d)
                for (j, t), dj, w in zip(occ, d, D.weights(int(i), forward, srmp)):
                    D.lam[j][t] += -dj + w * S
        trace.append(D.bound())
    return np.array(trace)


def parallel_enum(inst, iters, omega=0.5, rank=None, srmp=False):
    """Deferred averaging: every BDD runs its layers in order; the share of the previous sweep's
    sum P_i is added at the visit, lambda moves by -omega (m1 - m0), P_i = the sum of those
    moves after the sweep.  Returns the bound after each backward sweep."""
    D = EnumDual(inst, rank)
    trace = []
    for _ in range(iters):
        for forward in (True, False):
            share = [np.zeros(len(cols)) for cols, *_ in D.rows]
            for i in range(D.n):
                for (j, t), w in zip(D.occ[i], D.weights(i, forward, srmp)):
                    share[j][t] = w * D.P[i]
            Pn = np.zeros(D.n)
            for j, (cols, *_) in enumerate(D.rows):
                k = len(cols)
                for t in (range(k) if forward else range(k - 1, -1, -1)):
                    D.lam[j][t] += share[j][t]
                    m0, m1, _, _ = D.mm(j)
                    dlt = omega * _diff(m0[t], m1[t])
                    D.lam[j][t] -= dlt
                    Pn[cols[t]] += dlt
            D.P = Pn
        trace.append(D.bound())
    return np.array(trace)
