"""Seeded generators for the synthetic workloads.

Every generator returns an :class:`Instance`: a 0-1 ILP ``min c.x  s.t.  a_j.x (sense_j) b_j``
given as an integer CSR matrix.  The shapes follow the ILP formulations of the paper's
experiment appendix (Appendix E: MRF local polytope, graph matching, cell tracking, discrete
tomography); the sizes are the synthetic stand-ins for its datasets, which are not used.

Variable numbering convention: unary/assignment variables first, then pairwise/auxiliary
ones, so that a constraint row lists its variables in ascending index order.

Only ``numpy.random.default_rng(seed)`` is used, so the same seed gives the same instance on
every machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SENSE_LE = -1  # a.x <= b
SENSE_EQ = 0   # a.x == b
SENSE_GE = 1   # a.x >= b


@dataclass
class Instance:
    """A 0-1 ILP in CSR form.

    row_ptr: int64[m+1]; col: int32[nnz]; val: int32[nnz]; b: int32[m]; sense: int8[m];
    c: float32[n].  ``parts`` optionally lists (var_offset, row_offset) of independent
    sub-instances packed block-diagonally into this one.
    """

    name: str
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    b: np.ndarray
    sense: np.ndarray
    c: np.ndarray
    meta: dict = field(default_factory=dict)
    var_parts: np.ndarray | None = None  # int64[P+1] variable offsets of packed instances
    row_parts: np.ndarray | None = None  # int64[P+1] row offsets of packed instances

    @property
    def m(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def rows(self):
        for j in range(self.m):
            s, e = int(self.row_ptr[j]), int(self.row_ptr[j + 1])
            yield self.col[s:e], self.val[s:e], int(self.b[j]), int(self.sense[j])

    def dense(self) -> np.ndarray:
        A = np.zeros((self.m, self.n), dtype=np.int64)
        for j in range(self.m):
            s, e = int(self.row_ptr[j]), int(self.row_ptr[j + 1])
            A[j, self.col[s:e]] += self.val[s:e]
        return A


def _from_rows(name, n, rows, c, meta=None) -> Instance:
    """rows: list of (cols, vals, b, sense)."""
    m = len(rows)
    lens = np.fromiter((len(r[0]) for r in rows), dtype=np.int64, count=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    col = np.concatenate([np.asarray(r[0], dtype=np.int32) for r in rows]) if m else np.zeros(0, np.int32)
    val = np.concatenate([np.asarray(r[1], dtype=np.int32) for r in rows]) if m else np.zeros(0, np.int32)
    b = np.array([r[2] for r in rows], dtype=np.int32)
    sense = np.array([r[3] for r in rows], dtype=np.int8)
    return Instance(name, int(n), row_ptr, col, val, b, sense, np.asarray(c, dtype=np.float32), meta or {})


# ----------------------------------------------------------------------------------------
# Markov random field in local-polytope ILP form (Appendix E.1)
# ----------------------------------------------------------------------------------------

def _grid_edges(H: int, W: int):
    """4-connected grid edges, ordered by source pixel (row-major), right edge then down edge."""
    idx = np.arange(H * W, dtype=np.int64).reshape(H, W)
    right = np.zeros((H, W), dtype=bool)
    right[:, : W - 1] = True
    down = np.zeros((H, W), dtype=bool)
    down[: H - 1, :] = True
    src = np.stack([idx, idx], axis=-1)
    dst = np.stack([idx + 1, idx + W], axis=-1)
    ok = np.stack([right, down], axis=-1)
    return src[ok].astype(np.int64), dst[ok].astype(np.int64)


def _potts_arrays(H: int, W: int, L: int, unary: np.ndarray, pair_weight: float):
    """Vectorised CSR pieces of the Potts local-polytope ILP.

    Variables: x[i, l] = i*L + l (i pixel), then y[e, l, l'] = nx + e*L*L + l*L + l'.
    Rows: one-hot sum_l x[i,l] = 1 per pixel; then per edge e=(i,j) the L rows
    sum_l' y[e,l,l'] - x[i,l] = 0 and the L rows sum_l y[e,l,l'] - x[j,l'] = 0.
    The per-edge row sum y = 1 is implied by these and is left out.
    """
    npx = H * W
    src, dst = _grid_edges(H, W)
    E = src.shape[0]
    nx = npx * L
    n = nx + E * L * L
    # one-hot rows
    oh_cols = np.arange(nx, dtype=np.int64).reshape(npx, L)
    oh_vals = np.ones((npx, L), dtype=np.int32)
    # marginalisation rows: [E, 2L, L+1]
    ll = np.arange(L, dtype=np.int64)
    ybase = nx + np.arange(E, dtype=np.int64) * L * L  # [E]
    left_x = src[:, None] * L + ll[None, :]  # [E, L]  x[i,l]
    left_y = ybase[:, None, None] + ll[None, :, None] * L + ll[None, None, :]  # [E, l, l']
    right_x = dst[:, None] * L + ll[None, :]  # x[j,l']
    right_y = ybase[:, None, None] + ll[None, None, :] * L + ll[None, :, None]  # [E, l', l]
    mcols = np.empty((E, 2 * L, L + 1), dtype=np.int64)
    mcols[:, :L, 0] = left_x
    mcols[:, :L, 1:] = left_y
    mcols[:, L:, 0] = right_x
    mcols[:, L:, 1:] = right_y
    mvals = np.ones((E, 2 * L, L + 1), dtype=np.int32)
    mvals[:, :, 0] = -1
    m = npx + E * 2 * L
    row_len = np.concatenate([np.full(npx, L, np.int64), np.full(E * 2 * L, L + 1, np.int64)])
    col = np.concatenate([oh_cols.ravel(), mcols.ravel()]).astype(np.int32)
    val = np.concatenate([oh_vals.ravel(), mvals.ravel()])
    b = np.concatenate([np.ones(npx, np.int32), np.zeros(E * 2 * L, np.int32)])
    sense = np.zeros(m, dtype=np.int8)
    pair = (pair_weight * (ll[:, None] != ll[None, :])).astype(np.float32)  # [L, L]
    c = np.concatenate([np.asarray(unary, np.float32).ravel(), np.tile(pair.ravel(), E)])
    return n, row_len, col, val, b, sense, c, E


def _assemble(name, n, row_len, col, val, b, sense, c, meta) -> Instance:
    row_ptr = np.zeros(row_len.shape[0] + 1, dtype=np.int64)
    np.cumsum(row_len, out=row_ptr[1:])
    return Instance(name, int(n), row_ptr, col, val, b, sense, c.astype(np.float32), meta)


def potts_mrf(H: int = 20, W: int = 20, L: int = 3, seed: int = 0, pair_weight: float = 0.5,
              rng: np.random.Generator | None = None) -> Instance:
    """Potts MRF on an HxW 4-connected grid with L labels; unary costs N(0,1),
    pairwise cost pair_weight*[l != l'] (the 20x20x3 MRF workload at the defaults)."""
    rng = np.random.default_rng(seed) if rng is None else rng
    unary = rng.standard_normal(H * W * L).astype(np.float32)
    n, row_len, col, val, b, sense, c, E = _potts_arrays(H, W, L, unary, pair_weight)
    return _assemble(f"potts_{H}x{W}x{L}", n, row_len, col, val, b, sense, c,
                     {"H": H, "W": W, "L": L, "edges": E, "seed": seed})


def potts_grid_2label(H: int, W: int, seed: int) -> Instance:
    """Tiny 2-label Potts instance for brute-force pins."""
    return potts_mrf(H, W, 2, seed=seed)


def potts_batch_shape(s: int, side_range=(16, 128), label_range=(2, 8)):
    """(side, labels) that instance s of the Potts batch draws (the first two draws of
    ``default_rng(s)``), without generating its costs."""
    rng = np.random.default_rng(s)
    side = int(rng.integers(side_range[0], side_range[1] + 1))
    L = int(rng.integers(label_range[0], label_range[1] + 1))
    return side, L


def potts_batch_member(s: int, side_range=(16, 128), label_range=(2, 8)) -> Instance:
    """Instance s of the Potts batch on its own (same draws as inside :func:`potts_batch`)."""
    rng = np.random.default_rng(s)
    side = int(rng.integers(side_range[0], side_range[1] + 1))
    L = int(rng.integers(label_range[0], label_range[1] + 1))
    unary = rng.standard_normal(side * side * L).astype(np.float32)
    n, row_len, col, val, b, sense, c, E = _potts_arrays(side, side, L, unary, 0.5)
    return _assemble(f"potts_batch_member_{s}", n, row_len, col, val, b, sense, c,
                     {"seed": s, "side": side, "L": L, "edges": E})


def potts_batch(count: int = 256, side_range=(16, 128), label_range=(2, 8), first_seed: int = 0,
                stride: int = 1, seeds=None) -> Instance:
    """Block-diagonal packing of independent Potts instances of uneven size.

    Instance s (s = first_seed + k*stride, or the listed `seeds`) draws side ~ U{side_range},
    labels ~ U{label_range} and its costs as in :func:`potts_mrf`, all from ``default_rng(s)``.
    """
    cols, vals, bs, senses, cs, lens = [], [], [], [], [], []
    var_parts, row_parts = [0], [0]
    voff = 0
    sizes = []
    seed_list = list(seeds) if seeds is not None else [first_seed + k * stride for k in range(count)]
    count = len(seed_list)
    for k in range(count):
        s = seed_list[k]
        rng = np.random.default_rng(s)
        side = int(rng.integers(side_range[0], side_range[1] + 1))
        L = int(rng.integers(label_range[0], label_range[1] + 1))
        unary = rng.standard_normal(side * side * L).astype(np.float32)
        n, row_len, col, val, b, sense, c, E = _potts_arrays(side, side, L, unary, 0.5)
        cols.append(col.astype(np.int64) + voff)
        vals.append(val)
        bs.append(b)
        senses.append(sense)
        cs.append(c)
        lens.append(row_len)
        voff += n
        var_parts.append(voff)
        row_parts.append(row_parts[-1] + row_len.shape[0])
        sizes.append((s, side, L))
    col = np.concatenate(cols)
    if voff >= 2**31:
        raise ValueError("packed batch exceeds int32 variable indices")
    inst = _assemble(f"potts_batch_{count}", voff, np.concatenate(lens), col.astype(np.int32),
                     np.concatenate(vals), np.concatenate(bs), np.concatenate(senses),
                     np.concatenate(cs), {"instances": sizes})
    inst.var_parts = np.asarray(var_parts, dtype=np.int64)
    inst.row_parts = np.asarray(row_parts, dtype=np.int64)
    return inst


# ----------------------------------------------------------------------------------------
# Sparse graph matching with linearised quadratic terms (Appendix E.2 shape)
# ----------------------------------------------------------------------------------------

def sparse_matching(n_left: int = 300, n_right: int = 300, k: int = 10, n_pairs: int = 20000,
                    seed: int = 0, pair_sigma: float = 0.3) -> Instance:
    """Each left point has k distinct random right candidates (assignment variables x,
    costs U(-1,0)); rows: sum = 1 per left point, sum <= 1 per right point with a candidate.
    n_pairs distinct quadratic pairs (x_a, x_b) with different left and different right points
    are linearised by z <= x_a, z <= x_b, cost of z ~ N(0, pair_sigma)."""
    rng = np.random.default_rng(seed)
    cand = np.stack([np.sort(rng.choice(n_right, size=k, replace=False)) for _ in range(n_left)])
    nx = n_left * k
    x_left = np.repeat(np.arange(n_left), k)
    x_right = cand.ravel()
    rows = []
    for l in range(n_left):
        rows.append((np.arange(l * k, (l + 1) * k), np.ones(k), 1, SENSE_EQ))
    for r in range(n_right):
        xs = np.nonzero(x_right == r)[0]
        if xs.size:
            rows.append((xs, np.ones(xs.size), 1, SENSE_LE))
    # distinct pairs a < b with different left and different right points
    chosen = []
    seen = set()
    while len(chosen) < n_pairs:
        a = rng.integers(0, nx, size=4 * n_pairs)
        b = rng.integers(0, nx, size=4 * n_pairs)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        ok = (x_left[lo] != x_left[hi]) & (x_right[lo] != x_right[hi])
        for p, q in zip(lo[ok].tolist(), hi[ok].tolist()):
            key = p * nx + q
            if key not in seen:
                seen.add(key)
                chosen.append((p, q))
                if len(chosen) == n_pairs:
                    break
    pairs = np.asarray(chosen, dtype=np.int64)
    for t, (p, q) in enumerate(pairs.tolist()):
        z = nx + t
        rows.append((np.array([p, z]), np.array([-1, 1]), 0, SENSE_LE))
        rows.append((np.array([q, z]), np.array([-1, 1]), 0, SENSE_LE))
    cx = rng.uniform(-1.0, 0.0, size=nx)
    cz = rng.normal(0.0, pair_sigma, size=n_pairs)
    c = np.concatenate([cx, cz]).astype(np.float32)
    return _from_rows(f"matching_{n_left}x{n_right}", nx + n_pairs, rows, c,
                      {"n_left": n_left, "n_right": n_right, "k": k, "pairs": n_pairs, "seed": seed})


# ----------------------------------------------------------------------------------------
# Discrete tomography: Potts MRF plus integer projection equalities (Appendix E.4 shape)
# ----------------------------------------------------------------------------------------

def tomography_ground_truth(side: int, levels: int, n_seeds: int, rng) -> np.ndarray:
    """Piecewise-constant image: nearest-seed (Voronoi) regions with random levels."""
    pts = rng.uniform(0, side, size=(n_seeds, 2))
    lev = rng.integers(0, levels, size=n_seeds)
    rr, cc = np.meshgrid(np.arange(side) + 0.5, np.arange(side) + 0.5, indexing="ij")
    d2 = (rr[..., None] - pts[:, 0]) ** 2 + (cc[..., None] - pts[:, 1]) ** 2
    return lev[np.argmin(d2, axis=-1)].astype(np.int64)


def tomography_lines(side: int):
    """Projection lines as lists of pixel ids: rows, columns, diagonals (r-c const) and
    anti-diagonals (r+c const), each listed in ascending pixel order."""
    idx = np.arange(side * side).reshape(side, side)
    lines = [idx[r, :] for r in range(side)]
    lines += [idx[:, c] for c in range(side)]
    lines += [np.sort(np.diagonal(idx, offset=o)) for o in range(-(side - 1), side)]
    flip = idx[:, ::-1]
    lines += [np.sort(np.diagonal(flip, offset=o)) for o in range(-(side - 1), side)]
    return lines


def tomography(side: int = 64, levels: int = 3, smooth: float = 0.2, n_seeds: int = 16,
               seed: int = 0, unary_sigma: float = 0.0) -> Instance:
    """Discrete tomography: one-hot x over `levels` intensities per pixel, Potts smoothness
    `smooth` between 4-neighbours (local polytope rows), zero unary costs, and projection
    equalities sum_{pixel in line} sum_l l*x[pixel,l] = p_line for rows, columns and both
    diagonal directions, p taken from a random piecewise-constant ground truth.
    ``unary_sigma > 0`` adds N(0, unary_sigma) unary tie-break costs (drawn after the ground
    truth), which moves the non-smooth method off its all-zero fixed point."""
    rng = np.random.default_rng(seed)
    gt = tomography_ground_truth(side, levels, n_seeds, rng)
    unary = np.zeros(side * side * levels, dtype=np.float32)
    if unary_sigma > 0:
        unary = rng.normal(0.0, unary_sigma, size=unary.shape).astype(np.float32)
    n, row_len, col, val, b, sense, c, E = _potts_arrays(side, side, levels, unary, smooth)
    pcols, pvals, plen, pb = [], [], [], []
    flat = gt.ravel()
    for line in tomography_lines(side):
        cols = (line[:, None] * levels + np.arange(1, levels)[None, :]).ravel()
        vals = np.tile(np.arange(1, levels), line.size)
        pcols.append(cols)
        pvals.append(vals)
        plen.append(cols.size)
        pb.append(int(flat[line].sum()))
    row_len = np.concatenate([row_len, np.asarray(plen, np.int64)])
    col = np.concatenate([col, np.concatenate(pcols).astype(np.int32)])
    val = np.concatenate([val, np.concatenate(pvals).astype(np.int32)])
    b = np.concatenate([b, np.asarray(pb, np.int32)])
    sense = np.concatenate([sense, np.zeros(len(pb), np.int8)])
    return _assemble(f"tomography_{side}x{side}x{levels}", n, row_len, col, val, b, sense, c,
                     {"side": side, "levels": levels, "projections": len(pb), "seed": seed,
                      "unary_sigma": unary_sigma, "ground_truth": gt})


# ----------------------------------------------------------------------------------------
# Cell-tracking-shaped flow ILP (Appendix E.3 shape)
# ----------------------------------------------------------------------------------------

def tracking(frames: int = 50, dets: int = 200, knn: int = 5, seed: int = 0) -> Instance:
    """Detections at uniform positions per frame.  Per detection d: x_d, appear_d, disappear_d
    (ids 3d, 3d+1, 3d+2).  Transitions from d to its knn nearest detections of the next frame,
    then divisions for each pair of those neighbours.  Rows: in-flow
    appear + transitions in + divisions in - x = 0; out-flow disappear + transitions out +
    divisions out - x = 0; children transitions out + 2*divisions out <= 2.  Costs N(0,1)."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, 1, size=(frames, dets, 2))
    D = frames * dets
    pairs = [(a, b) for a in range(knn) for b in range(a + 1, knn)]
    npair = len(pairs)
    nsrc = (frames - 1) * dets
    t_base = 3 * D
    d_base = t_base + nsrc * knn
    n = d_base + nsrc * npair
    nbr = np.zeros((nsrc, knn), dtype=np.int64)
    for f in range(frames - 1):
        d2 = ((pos[f][:, None, :] - pos[f + 1][None, :, :]) ** 2).sum(-1)
        nn = np.argsort(d2, axis=1, kind="stable")[:, :knn]
        nbr[f * dets:(f + 1) * dets] = (f + 1) * dets + np.sort(nn, axis=1)
    in_vars = [[] for _ in range(D)]
    in_vals = [[] for _ in range(D)]
    for s in range(nsrc):
        for t in range(knn):
            in_vars[nbr[s, t]].append(t_base + s * knn + t)
            in_vals[nbr[s, t]].append(1)
        for p, (a, b) in enumerate(pairs):
            for child in (nbr[s, a], nbr[s, b]):
                in_vars[child].append(d_base + s * npair + p)
                in_vals[child].append(1)
    rows = []
    for d in range(D):
        cols = [3 * d, 3 * d + 1] + in_vars[d]
        vals = [-1, 1] + in_vals[d]
        o = np.argsort(cols, kind="stable")
        rows.append((np.asarray(cols)[o], np.asarray(vals)[o], 0, SENSE_EQ))
    for d in range(D):
        cols = [3 * d, 3 * d + 2]
        vals = [-1, 1]
        if d < nsrc:
            cols += list(range(t_base + d * knn, t_base + (d + 1) * knn))
            vals += [1] * knn
            cols += list(range(d_base + d * npair, d_base + (d + 1) * npair))
            vals += [1] * npair
        rows.append((np.asarray(cols), np.asarray(vals), 0, SENSE_EQ))
    for d in range(nsrc):
        cols = list(range(t_base + d * knn, t_base + (d + 1) * knn)) + \
            list(range(d_base + d * npair, d_base + (d + 1) * npair))
        vals = [1] * knn + [2] * npair
        rows.append((np.asarray(cols), np.asarray(vals), 2, SENSE_LE))
    c = rng.standard_normal(n).astype(np.float32)
    return _from_rows(f"tracking_{frames}x{dets}", n, rows, c,
                      {"frames": frames, "dets": dets, "knn": knn, "seed": seed})


# ----------------------------------------------------------------------------------------
# Random small ILPs for brute-force pins
# ----------------------------------------------------------------------------------------

def random_ilp(n: int, m: int, max_row_vars: int, seed: int, coef: int = 3,
               senses=(SENSE_LE, SENSE_EQ, SENSE_GE)) -> Instance:
    """Random rows over <= max_row_vars distinct variables with nonzero integer coefficients in
    [-coef, coef]; right-hand sides chosen so a random 0-1 point is feasible for every row."""
    rng = np.random.default_rng(seed)
    x0 = rng.integers(0, 2, size=n)
    rows = []
    for _ in range(m):
        k = int(rng.integers(1, min(max_row_vars, n) + 1))
        cols = np.sort(rng.choice(n, size=k, replace=False))
        vals = rng.integers(1, coef + 1, size=k) * rng.choice([-1, 1], size=k)
        s = int(rng.choice(list(senses)))
        lhs = int(vals @ x0[cols])
        if s == SENSE_EQ:
            b = lhs
        elif s == SENSE_LE:
            b = lhs + int(rng.integers(0, 3))
        else:
            b = lhs - int(rng.integers(0, 3))
        rows.append((cols, vals, b, s))
    c = rng.standard_normal(n).astype(np.float32)
    return _from_rows(f"random_ilp_n{n}_m{m}_s{seed}", n, rows, c, {"x0": x0, "seed": seed})


# ----------------------------------------------------------------------------------------
# The five workload configurations
# ----------------------------------------------------------------------------------------

CONFIG_NAMES = [
    "potts_20x20x3",
    "matching_300x300_k10_p20000",
    "tomography_64x64x3",
    "tracking_50x200_k5",
    "potts_batch_256",
]
CONFIG_ITERS = [100, 500, 1000, 50, 200]


def config(k: int) -> Instance:
    """Workload k: 0 Potts 20x20x3; 1 sparse matching 300x300; 2 tomography 64x64x3;
    3 tracking 50x200; 4 batch of 256 uneven Potts instances."""
    if k == 0:
        return potts_mrf(20, 20, 3, seed=0)
    if k == 1:
        return sparse_matching(seed=0)
    if k == 2:
        return tomography(seed=0)
    if k == 3:
        return tracking(seed=0)
    if k == 4:
        return potts_batch(256)
    raise ValueError(k)
