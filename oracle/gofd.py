"""Plain FP64 CPU oracle of the grid-overlay FD method (GoFD) for the
fractional Laplacian (Huang & Shen, "A grid-overlay finite difference method
for the fractional Laplacian on arbitrary bounded domains", arXiv 2307.14437).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The CUDA
library never calls it, and it imports nothing from the CUDA package: the two
share no code.  Inputs come from ``meshgen`` (seeded generators only).

Every function states the passage of the paper it follows.  It is written to
be checked against the paper by eye: plain loops or whole-array NumPy/SciPy
primitives (FFT, DCT, sparse products), no blocking or fusion.  Where the
paper is silent the reading taken is stated in the docstring (readings R1..R12
of the design notes).

Parity status of each function (what pins it is in ``tests/test_oracle_*.py``):
  grid / locate / weights / transfer   pinned (exact rationals, grid-aligned mesh,
                                        Lemma 3.1 invariants, linear precision)
  coefficients (Filon + Richardson)    pinned (1D Gamma formula (T-1D-0), s=1 5-point,
                                        Gauss-Legendre quadrature of (T-1) in 2D and 3D,
                                        tail law); coefficients_at equals it entry by entry
  symbol, A_FD apply                   pinned (direct DFT, direct Toeplitz sum,
                                        s=1 Laplacian, symmetry, positivity)
  stiffness apply, rhs, cg             pinned (grid-aligned special case = (FD-1),
                                        unit-ball closed form (exam-2), f=1 identity)
  ic1 factor / pcg                     pinned (complete pattern = exact Cholesky,
                                        L L^T = A on the kept pattern)
  jacobi_diagonal                      pinned (the diagonal of S assembled column by
                                        column from the stiffness product)
  circulant_inverse_apply / _precond   pinned (dense circulant solve on a small P,
                                        C applied to C^{-1} v by the direct Toeplitz
                                        wrap, symmetry, positivity, grid-aligned mesh
                                        where I is a selection and D_h = 1)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction
from itertools import combinations

import numpy as np
import scipy.fft
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import gamma as Gamma


class OracleError(RuntimeError):
    """Raised for inputs the method rejects (degenerate simplex, bad grid...)."""


# ============================================================================
# 1. Overlay grid  (Section 3.1: a uniform grid over a cube covering Omega)
# ============================================================================

def grid_shape(box_lo, box_hi, h):
    """Nodes per axis n_i = (hi_i - lo_i)/h + 1, which must be an integer.

    Reading R2: the paper's grid has 2N+1 nodes on (-R,R)^d with spacing R/N
    (Section 3.1); any n_i >= 2 on any box is accepted here.
    """
    lo = np.asarray(box_lo, dtype=np.float64)
    hi = np.asarray(box_hi, dtype=np.float64)
    q = (hi - lo) / h
    n = np.rint(q).astype(np.int64)
    if np.any(np.abs(q - n) > 1e-9 * np.maximum(1.0, np.abs(q))) or np.any(n < 1):
        raise OracleError("(hi-lo)/h must be a positive integer on every axis")
    return tuple(int(v) + 1 for v in n)


def grid_axis_coords(lo: float, h: float, n: int) -> np.ndarray:
    """x_k = lo + k*h: one rounded product, then one rounded sum (no FMA)."""
    k = np.arange(n, dtype=np.float64)
    prod = k * h
    return lo + prod


def grid_node_coords(box_lo, h, n, nodes) -> np.ndarray:
    """Coordinates of linear grid indices (axis 0 fastest)."""
    d = len(n)
    nodes = np.asarray(nodes, dtype=np.int64)
    out = np.empty((len(nodes), d))
    rem = nodes.copy()
    for ax in range(d):
        k = rem % n[ax]
        rem //= n[ax]
        out[:, ax] = grid_axis_coords(box_lo[ax], h, n[ax])[k]
    return out


# ============================================================================
# 2. Point location and P1 interpolation weights  (Section 3.1, (IhFD-1))
# ============================================================================

def _det_fraction(rows):
    """Exact determinant of a small square matrix of Fractions (Laplace expansion)."""
    m = len(rows)
    if m == 1:
        return rows[0][0]
    if m == 2:
        return rows[0][0] * rows[1][1] - rows[0][1] * rows[1][0]
    tot = Fraction(0)
    for c in range(m):
        minor = [r[:c] + r[c + 1:] for r in rows[1:]]
        term = rows[0][c] * _det_fraction(minor)
        tot += term if c % 2 == 0 else -term
    return tot


def orient_exact(points) -> Fraction:
    """Exact orientation determinant det[p_1-p_0, ..., p_d-p_0] of d+1 points.

    The double inputs are converted to exact rationals, so the sign is exact.
    """
    P = [[Fraction(float(c)) for c in p] for p in points]
    rows = [[P[j][a] - P[0][a] for a in range(len(P[0]))] for j in range(1, len(P))]
    return _det_fraction(rows)


def _orient_float_with_bound(pts):
    """Float orientation determinants of stacked point sets and a generous bound.

    pts: (..., d+1, d).  Returns (det, bound) with |det - exact| < bound: the
    bound is 1e-12 times the permanent of the difference matrix, far above the
    few-ulp error of the evaluation, so every sign with |det| > bound is exact.
    """
    e = pts[..., 1:, :] - pts[..., :1, :]
    d = e.shape[-1]
    if d == 1:
        return e[..., 0, 0], 1e-12 * np.abs(e[..., 0, 0]) + 1e-300
    if d == 2:
        t1 = e[..., 0, 0] * e[..., 1, 1]
        t2 = e[..., 0, 1] * e[..., 1, 0]
        return t1 - t2, 1e-12 * (np.abs(t1) + np.abs(t2)) + 1e-300
    det = np.zeros(e.shape[:-2])
    perm = np.zeros(e.shape[:-2])
    for (i, j, k), sgn in (((0, 1, 2), 1), ((1, 2, 0), 1), ((2, 0, 1), 1),
                           ((0, 2, 1), -1), ((2, 1, 0), -1), ((1, 0, 2), -1)):
        t = e[..., 0, i] * e[..., 1, j] * e[..., 2, k]
        det = det + sgn * t
        perm = perm + np.abs(t)
    return det, 1e-12 * perm + 1e-300


def element_orientations(verts, simp) -> np.ndarray:
    """Exact sign (+1/-1) of every simplex; a zero volume is rejected."""
    det, bnd = _orient_float_with_bound(verts[simp])
    sign = np.sign(det).astype(np.int64)
    for e in np.nonzero(np.abs(det) <= bnd)[0]:
        ex = orient_exact(verts[simp[e]])
        sign[e] = (ex > 0) - (ex < 0)
    if np.any(sign == 0):
        raise OracleError("degenerate simplex (zero volume)")
    return sign


def locate(verts, simp, box_lo, h, n, nodes=None, chunk=256):
    """Owner simplex of each overlay node, or -1 (Section 3.1, (IhFD-1)).

    A node x is in the closed simplex K=(v_0..v_d) iff no determinant
    D_i = orient(v_0..x (in slot i)..v_d) has the sign opposite to orient(K).
    Every (node, simplex) pair is tested; the owner is the smallest simplex
    index whose closed simplex contains the node (reading R9: ties on shared
    facets go to the lowest element index).  Signs are exact: float
    determinants decide when far from zero, exact rationals otherwise.
    """
    verts = np.asarray(verts, dtype=np.float64)
    simp = np.asarray(simp, dtype=np.int64)
    d = verts.shape[1]
    N = int(np.prod(n))
    if nodes is None:
        nodes = np.arange(N, dtype=np.int64)
    nodes = np.asarray(nodes, dtype=np.int64)
    osign = element_orientations(verts, simp)
    X = grid_node_coords(box_lo, h, n, nodes)
    V = verts[simp]                                   # (E, d+1, d)
    owner = np.full(len(nodes), -1, dtype=np.int64)
    for c0 in range(0, len(nodes), chunk):
        xs = X[c0:c0 + chunk]                         # (C, d)
        inside = np.ones((len(xs), len(simp)), dtype=bool)
        unsure = np.zeros((len(xs), len(simp)), dtype=bool)
        for i in range(d + 1):
            pts = np.broadcast_to(V[None], (len(xs),) + V.shape).copy()
            pts[:, :, i, :] = xs[:, None, :]
            det, bnd = _orient_float_with_bound(pts)
            s = det * osign[None, :]
            sure = np.abs(det) > bnd
            inside &= ~(sure & (s < 0))
            unsure |= ~sure
        for (a, e) in zip(*np.nonzero(inside & unsure)):
            ok = True
            for i in range(d + 1):
                pts = V[e].copy()
                pts[i] = xs[a]
                ex = orient_exact(pts)
                if ex * osign[e] < 0:
                    ok = False
                    break
            inside[a, e] = ok
        has = inside.any(axis=1)
        first = np.argmax(inside, axis=1)
        owner[c0:c0 + chunk] = np.where(has, first, -1)
    return owner


def locate_pruned(verts, simp, box_lo, h, n):
    """locate() for all nodes, testing each node only against the simplices
    whose bounding box contains it (a node outside a simplex's bounding box is
    outside the simplex, so the owner is unchanged).  Same exact predicate and
    lowest-index tie rule as locate(); for full-size meshes.
    """
    verts = np.asarray(verts, dtype=np.float64)
    simp = np.asarray(simp, dtype=np.int64)
    d = verts.shape[1]
    osign = element_orientations(verts, simp)
    V = verts[simp]
    bmin = V.min(axis=1)
    bmax = V.max(axis=1)
    axes = [grid_axis_coords(box_lo[a], h, n[a]) for a in range(d)]
    # candidate index ranges per axis (exact coordinate comparison)
    lo_k = [np.searchsorted(axes[a], bmin[:, a], side="left") for a in range(d)]
    hi_k = [np.searchsorted(axes[a], bmax[:, a], side="right") for a in range(d)]
    counts = np.ones(len(simp), dtype=np.int64)
    for a in range(d):
        counts *= np.maximum(0, hi_k[a] - lo_k[a])
    elem = np.repeat(np.arange(len(simp)), counts)
    off = np.arange(counts.sum()) - np.repeat(np.cumsum(counts) - counts, counts)
    node = np.zeros(len(elem), dtype=np.int64)
    stride = 1
    rem = off.copy()
    for a in range(d):
        ext = np.maximum(0, hi_k[a] - lo_k[a])[elem]
        k = lo_k[a][elem] + rem % ext
        rem //= ext
        node += k * stride
        stride *= n[a]
    owner = np.full(int(np.prod(n)), -1, dtype=np.int64)
    chunk = 1 << 20
    for c0 in range(0, len(elem), chunk):
        e = elem[c0:c0 + chunk]
        k = node[c0:c0 + chunk]
        X = grid_node_coords(box_lo, h, n, k)
        inside = np.ones(len(e), dtype=bool)
        unsure = np.zeros(len(e), dtype=bool)
        for i in range(d + 1):
            pts = V[e].copy()
            pts[:, i, :] = X
            det, bnd = _orient_float_with_bound(pts)
            sure = np.abs(det) > bnd
            inside &= ~(sure & (det * osign[e] < 0))
            unsure |= ~sure
        for j in np.nonzero(inside & unsure)[0]:
            for i in range(d + 1):
                pts = V[e[j]].copy()
                pts[i] = X[j]
                if orient_exact(pts) * osign[e[j]] < 0:
                    inside[j] = False
                    break
        ki = k[inside]
        ei = e[inside]
        order = np.lexsort((ei, ki))
        ki, ei = ki[order], ei[order]
        first = np.ones(len(ki), dtype=bool)
        first[1:] = ki[1:] != ki[:-1]
        cur = owner[ki[first]]
        cand = ei[first]
        owner[ki[first]] = np.where((cur < 0) | (cand < cur), cand, cur)
    return owner


def barycentric_exact(verts, simp_e, x):
    """phi_i(x) = D_i / orient(K), computed exactly then rounded to double.

    Lemma 3.4: the i-th barycentric coordinate is the signed volume of the
    simplex with vertex i replaced by x over the volume of K.
    """
    V = np.asarray(verts[np.asarray(simp_e)], dtype=np.float64)
    full = orient_exact(V)
    out = []
    for i in range(len(V)):
        pts = V.copy()
        pts[i] = x
        out.append(float(orient_exact(pts) / full))
    return np.array(out)


def barycentric_float(verts, simp, owner_elems, X):
    """Float barycentric coordinates (for large cases), clamped to [0,1].

    A coordinate is exactly 0 when the node lies on the facet opposite that
    vertex (exact orientation test), as the exactly rounded value is.
    """
    V = verts[simp[owner_elems]]
    full, _ = _orient_float_with_bound(V)
    d = verts.shape[1]
    out = np.empty((d + 1, len(X)))
    for i in range(d + 1):
        pts = V.copy()
        pts[:, i, :] = X
        di, bnd = _orient_float_with_bound(pts)
        wi = np.clip(di / full, 0.0, 1.0)
        for r in np.nonzero(np.abs(di) <= bnd)[0]:
            if orient_exact(pts[r]) == 0:
                wi[r] = 0.0
        out[i] = wi
    return out


def ell_layout(verts, simp, box_lo, h, n, owner, exact=True):
    """Canonical ELL form of I_h^FD over the located nodes.

    Rows are the located nodes in increasing linear grid index; slot a of row
    k holds (simp[owner_k][a], phi of that vertex at x_k): entry (k, j) of
    I_h^FD is phi_j(x_k) (IhFD-1).  Returns (nodes, idx[d+1, n_loc] int64,
    w[d+1, n_loc] float64).
    """
    nodes = np.nonzero(owner >= 0)[0]
    own = owner[nodes]
    idx = np.asarray(simp, dtype=np.int64)[own].T.copy()
    X = grid_node_coords(box_lo, h, n, nodes)
    if exact:
        w = np.empty(idx.shape)
        for r, (e, x) in enumerate(zip(own, X)):
            w[:, r] = barycentric_exact(verts, simp[e], x)
    else:
        w = barycentric_float(verts, np.asarray(simp, dtype=np.int64), own, X)
    return nodes, idx, w


def transfer_matrix(nodes, idx, w, n_grid, n_v):
    """I_h^FD as a sparse (n^d x N_v) matrix (IhFD-1)."""
    rows = np.repeat(nodes[None, :], idx.shape[0], axis=0).ravel()
    return sp.csr_matrix((w.ravel(), (rows, idx.ravel())), shape=(n_grid, n_v))


# ============================================================================
# 3. Mesh quantities  (Section 3.1: D_h, heights, boundary vertices)
# ============================================================================

def boundary_vertices(simp, n_v) -> np.ndarray:
    """Vertices on facets that belong to exactly one simplex (reading R7)."""
    count = {}
    d1 = simp.shape[1]
    for s in np.asarray(simp, dtype=np.int64):
        for f in combinations(sorted(int(v) for v in s), d1 - 1):
            count[f] = count.get(f, 0) + 1
    bnd = np.zeros(n_v, dtype=bool)
    for f, c in count.items():
        if c == 1:
            bnd[list(f)] = True
    return bnd


def column_sums(I) -> np.ndarray:
    """D_{h,j} = sum_k (I_h^FD)_{k,j}  (Lemma 3.1 (iv))."""
    return np.asarray(I.sum(axis=0)).ravel()


def element_heights(verts, simp) -> np.ndarray:
    """a_K = min_j a_j, a_j = distance from vertex j to its opposite facet.

    a_j = d |K| / |S_j| with |S_j| the (d-1)-volume of the facet (Section 3.1,
    before Lemma 3.3).
    """
    V = verts[np.asarray(simp, dtype=np.int64)]
    E, d1, d = V.shape
    d = d1 - 1
    volK = np.abs(np.linalg.det(V[:, 1:] - V[:, :1])) / math.factorial(d)
    aK = np.full(E, np.inf)
    for j in range(d1):
        F = np.delete(V, j, axis=1)                     # (E, d, d)
        if d == 1:
            area = np.ones(E)
        else:
            G = F[:, 1:] - F[:, :1]                     # (E, d-1, d)
            gram = np.einsum("eik,ejk->eij", G, G)
            area = np.sqrt(np.abs(np.linalg.det(gram))) / math.factorial(d - 1)
        aK = np.minimum(aK, d * volK / area)
    return aK


# ============================================================================
# 4. FD coefficients T  (Section 2.3: (T-0), (psi-2), (T-3), (Tp-1D-2))
# ============================================================================

PAPER_FILON_M = {1: 2 ** 14, 2: 2 ** 14, 3: 2 ** 11}


def richardson_exponents(d: int, s: float, levels: int):
    """Leading error exponents of the Filon sums, ascending (reading R5).

    The Filon factor sinc^2(p/M) contributes M^-2, M^-4, ...; the |xi|^{2s}
    singularity of psi contributes M^-(d+2s), M^-(d+2s+2), ...  The first
    levels-1 distinct values are eliminated.
    """
    cand = set()
    for m in range(1, levels + 1):
        cand.add(round(2.0 * m, 12))
        cand.add(round(d + 2.0 * s + 2.0 * (m - 1), 12))
    cand = sorted(c for c in cand)
    return cand[: levels - 1]


def default_filon_M(d: int, n: int, levels: int = 4) -> int:
    """Paper's finest M (2^14 in 2D, 2^11 in 3D), raised so that M/2^(L-1) >= n."""
    M = PAPER_FILON_M[d]
    while M // (2 ** (levels - 1)) < n:
        M *= 2
    return M


def psi_tilde_samples(d: int, s: float, M: int) -> np.ndarray:
    """psi~(xi) = (sum_i 4 cos^2(pi xi_i))^s at xi_i = j_i/M, j_i in [0, M/2]  (psi-2).

    psi~ is even about xi_i = 1/2 and 1-periodic, so the half range holds all
    distinct samples.
    """
    j = np.arange(M // 2 + 1, dtype=np.float64)
    c = 4.0 * np.cos(np.pi * j / M) ** 2
    tot = np.zeros((M // 2 + 1,) * d)
    for ax in range(d):
        shape = [1] * d
        shape[ax] = M // 2 + 1
        tot = tot + c.reshape(shape)
    return tot ** s


def filon_coefficients(d: int, s: float, n: int, M: int) -> np.ndarray:
    """Filon-linear approximation of T_p, 0 <= p_i < n, with M panels per axis.

    (Tp-1D-2) equals T_p = (-1)^p sinc^2(p/M) (1/M) sum_j psi~_j e^{i 2 pi p j/M}
    (shift the second difference onto the exponential); in d dimensions the
    piecewise-multilinear interpolant of psi~ is integrated exactly, which is
    the tensor product of the 1D factors (reading R4).  The trapezoid sum
    (T-3) over j in [0,M)^d of the even samples is a DCT-I of the half range.
    """
    f = psi_tilde_samples(d, s, M)
    # the trapezoid sum is M-periodic and even in each p_i: for M/2 < p < M it
    # equals the value at M - p (needed when n > M/2 + 1 on a coarse level)
    p_idx = np.arange(n) % M
    p_idx = np.minimum(p_idx, M - p_idx)
    for ax in range(d):
        f = scipy.fft.dct(f, type=1, axis=ax)
        f = np.take(f, p_idx, axis=ax)
    f = f / float(M) ** d
    p = np.arange(n, dtype=np.float64)
    fac = (-1.0) ** p * np.sinc(p / M) ** 2
    for ax in range(d):
        shape = [1] * d
        shape[ax] = n
        f = f * fac.reshape(shape)
    return f


def coefficients(d: int, s: float, n: int, M: int | None = None, levels: int = 4) -> np.ndarray:
    """T_p for 0 <= p_i < n by Filon quadrature plus Richardson extrapolation.

    Section 2.3: Filon sums at M, M/2, ..., M/2^(levels-1) combined by a
    Richardson tableau that removes the exponents of richardson_exponents().
    Returns T with shape (n,)*d, axis order (p_{d-1}, ..., p_0) (T is symmetric
    in its axes, (T-2)).
    """
    if M is None:
        M = default_filon_M(d, n, levels)
    if M // (2 ** (levels - 1)) < n:
        raise OracleError("coarsest Filon level must have M_l >= n")
    if levels == 1:
        return filon_coefficients(d, s, n, M)
    exps = richardson_exponents(d, s, levels)
    R = [filon_coefficients(d, s, n, M // 2 ** l) for l in range(levels)]
    for e in exps:
        r = 2.0 ** e
        R = [(r * R[l] - R[l + 1]) / (r - 1.0) for l in range(len(R) - 1)]
    return R[0]


def filon_coefficients_at(d: int, s: float, ps: np.ndarray, M: int) -> np.ndarray:
    """filon_coefficients() at a list of multi-indices ps (K x d), for grids
    whose full coefficient array is too large to form.

    The same formula written out as a sum instead of a DCT-I: with weight 1 at
    j_i in {0, M/2} and 2 inside, the trapezoid sum (T-3) over one period is
    sum_{j in [0,M/2]^d} wt_j psi~_j prod_i cos(2 pi p_i j_i / M), taken one
    axis at a time (3D: one j_2 plane at a time); then the Filon factor
    prod_i (-1)^{p_i} sinc^2(p_i/M) / M (reading R4).
    """
    ps = np.atleast_2d(np.asarray(ps, dtype=np.int64))
    if ps.shape[1] != d:
        raise OracleError("ps must have d columns")
    H = M // 2 + 1
    j = np.arange(H, dtype=np.int64)
    c = 4.0 * np.cos(np.pi * j.astype(np.float64) / M) ** 2
    wt = np.where((j == 0) | (j == M // 2), 1.0, 2.0)
    # cos(2 pi p j / M) from the exact residue (p j) mod M
    A = [wt[:, None] * np.cos(2.0 * np.pi * ((j[:, None] * ps[None, :, ax]) % M) / M) for ax in range(d)]
    if d == 1:
        S = (c ** s) @ A[0]
    elif d == 2:
        F = (c[:, None] + c[None, :]) ** s                   # F[j0, j1]
        S = np.sum((F.T @ A[0]) * A[1], axis=0)
    else:
        S = np.zeros(len(ps))
        base = c[:, None] + c[None, :]
        for j2 in range(H):
            F = (base + c[j2]) ** s
            S += np.sum((F.T @ A[0]) * A[1], axis=0) * A[2][j2]
    fac = np.prod((-1.0) ** ps * np.sinc(ps / M) ** 2, axis=1)
    return fac * S / float(M) ** d


def coefficients_at(d: int, s: float, ps, M: int, levels: int = 4) -> np.ndarray:
    """coefficients() at a list of multi-indices ps (K x d): the Filon sums of
    filon_coefficients_at() at M, M/2, ..., combined by the same Richardson
    tableau (Section 2.3, reading R5)."""
    ps = np.atleast_2d(np.asarray(ps, dtype=np.int64))
    if M // (2 ** (levels - 1)) <= int(ps.max(initial=0)):
        raise OracleError("coarsest Filon level must have M_l > max p")
    R = [filon_coefficients_at(d, s, ps, M // 2 ** l) for l in range(levels)]
    if levels == 1:
        return R[0]
    for e in richardson_exponents(d, s, levels):
        r = 2.0 ** e
        R = [(r * R[l] - R[l + 1]) / (r - 1.0) for l in range(len(R) - 1)]
    return R[0]


def coefficients_1d_gamma(s: float, n: int) -> np.ndarray:
    """(T-1D-0): T_p = (-1)^p Gamma(2s+1) / (Gamma(p+s+1) Gamma(s-p+1))."""
    p = np.arange(n, dtype=np.float64)
    return (-1.0) ** p * Gamma(2 * s + 1) / (Gamma(p + s + 1) * Gamma(s - p + 1))


# ============================================================================
# 5. A_FD and its circulant symbol  (Section 2.2, (A-1), (AFD-1), (AU-1))
# ============================================================================

def circulant_size(n: int) -> int:
    """P = smallest power of two >= 2n-2 (reading R3).

    Offsets |m| <= n-1 need 2n-1 slots, but +-(n-1) may share one slot since
    T_{n-1} = T_{-(n-1)} (T-2): the paper's 4N = 2(2N+1)-2 (Section 2.2).
    P = 2n when n is a power of two.
    """
    P = 1
    while P < 2 * n - 2:
        P *= 2
    return max(P, 2)


def circulant_first_column(T: np.ndarray, P: int) -> np.ndarray:
    """Even circulant embedding c of T: c[m mod P] = T_{|m|} for |m_i| < n, 0 elsewhere."""
    d = T.ndim
    n = T.shape[0]
    c = np.zeros((P,) * d)
    idx1 = np.concatenate([np.arange(n), P - np.arange(1, n)])
    src1 = np.concatenate([np.arange(n), np.arange(1, n)])
    c[np.ix_(*([idx1] * d))] = T[np.ix_(*([src1] * d))]
    return c


def symbol(T: np.ndarray, P: int) -> np.ndarray:
    """Real, even circulant symbol lambda = DFT_P(c), kept on [0, P/2]^d.

    Section 2.2: the DFT of the embedded T ("T-check").  The full complex FFT
    is taken; its imaginary part vanishes by evenness.
    """
    d = T.ndim
    lam = np.fft.fftn(circulant_first_column(T, P))
    if np.max(np.abs(lam.imag)) > 1e-9 * max(1.0, np.max(np.abs(lam.real))):
        raise OracleError("symbol is not real")
    return np.ascontiguousarray(lam.real[(slice(0, P // 2 + 1),) * d])


def afd_apply_direct(T: np.ndarray, v: np.ndarray) -> np.ndarray:
    """w_k = sum_m T_{|k-m|} v_m over the finite grid  ((A-1), (AFD-1)).

    Direct Toeplitz sum, O(N^2): for tiny grids.  v has shape (n,)*d with
    axis order (k_{d-1}, ..., k_0).
    """
    d = T.ndim
    n = v.shape[0]
    w = np.zeros_like(v, dtype=np.float64)
    grids = np.meshgrid(*([np.arange(n)] * d), indexing="ij")
    flat_pos = np.stack([g.ravel() for g in grids], axis=1)
    vf = v.ravel()
    for a, k in enumerate(flat_pos):
        off = np.abs(flat_pos - k[None, :])
        w.flat[a] = np.sum(T[tuple(off.T)] * vf)
    return w


def _full_symbol(lam_half: np.ndarray, P: int) -> np.ndarray:
    """Unfold the even half-symbol to (P,)*d."""
    d = lam_half.ndim
    idx = np.concatenate([np.arange(P // 2 + 1), np.arange(P // 2 - 1, 0, -1)])
    return lam_half[np.ix_(*([idx] * d))]


def afd_apply_fft(lam_half: np.ndarray, v: np.ndarray, P: int, workers: int | None = None) -> np.ndarray:
    """A_FD v by zero-padded circulant convolution  (Section 2.2, (AU-1)).

    Zero-pad v to P^d, FFT, multiply by the symbol, inverse FFT, keep the
    corner [0,n)^d.  (The paper's (-1)^{p+2N} factors come from its centred
    index range; with the un-shifted embedding they do not appear.)
    """
    d = v.ndim
    n = v.shape[0]
    vp = np.zeros((P,) * d)
    vp[(slice(0, n),) * d] = v
    lam = _full_symbol(lam_half, P)
    V = scipy.fft.fftn(vp, workers=workers)
    w = scipy.fft.ifftn(V * lam, workers=workers).real
    return np.ascontiguousarray(w[(slice(0, n),) * d])


# ============================================================================
# 6. The GoFD system  (Section 3.2: (GoFD-1), (GoFD-2), (GoFD-3))
# ============================================================================

@dataclass
class Problem:
    """Everything the oracle derives from (mesh, alpha, h, box)."""
    d: int
    verts: np.ndarray
    simp: np.ndarray
    alpha: float
    s: float
    h: float
    box_lo: np.ndarray
    box_hi: np.ndarray
    n: tuple
    owner: np.ndarray
    nodes: np.ndarray
    ell_idx: np.ndarray
    ell_w: np.ndarray
    I: sp.csr_matrix
    boundary: np.ndarray
    interior: np.ndarray
    Dh: np.ndarray
    a_h: float
    M: int
    levels: int
    T: np.ndarray
    P: int
    lam: np.ndarray
    extra: dict = field(default_factory=dict)

    @property
    def n_grid(self) -> int:
        return int(np.prod(self.n))

    def grid_vector(self, flat: np.ndarray) -> np.ndarray:
        """Flat (axis 0 fastest) -> array with axes (k_{d-1}, ..., k_0)."""
        return flat.reshape(tuple(reversed(self.n)))


def build(d, verts, simp, alpha, h, box_lo, box_hi, M=None, levels=4, exact_weights=True,
          coeff_T=None, pruned=False) -> Problem:
    """Set up the oracle's GoFD problem: grid, I_h^FD, D_h, a_h, T, symbol.

    pruned=True locates with locate_pruned() (same owners, for large meshes).
    """
    verts = np.asarray(verts, dtype=np.float64)
    simp = np.asarray(simp, dtype=np.int64)
    if not (0.0 < alpha <= 2.0):
        raise OracleError("alpha must be in (0, 2]")
    s = alpha / 2.0
    box_lo = np.asarray(box_lo, dtype=np.float64)
    box_hi = np.asarray(box_hi, dtype=np.float64)
    n = grid_shape(box_lo, box_hi, h)
    if len(set(n)) != 1:
        raise OracleError("the oracle supports cubic grids only")
    if np.any(verts < box_lo) or np.any(verts > box_hi):
        raise OracleError("mesh vertex outside the box")
    owner = locate_pruned(verts, simp, box_lo, h, n) if pruned else locate(verts, simp, box_lo, h, n)
    nodes, idx, w = ell_layout(verts, simp, box_lo, h, n, owner, exact=exact_weights)
    I = transfer_matrix(nodes, idx, w, int(np.prod(n)), len(verts))
    bnd = boundary_vertices(simp, len(verts))
    interior = np.nonzero(~bnd)[0]
    Dh = column_sums(I)
    a_h = float(element_heights(verts, simp).min())
    nn = n[0]
    if coeff_T is None:
        if M is None:
            M = default_filon_M(d, nn, levels)
        T = coefficients(d, s, nn, M, levels) if d > 1 else coefficients(1, s, nn, M, levels)
    else:
        T = coeff_T
    P = circulant_size(nn)
    lam = symbol(T, P)
    return Problem(d=d, verts=verts, simp=simp, alpha=alpha, s=s, h=h, box_lo=box_lo,
                   box_hi=box_hi, n=n, owner=owner, nodes=nodes, ell_idx=idx, ell_w=w, I=I,
                   boundary=bnd, interior=interior, Dh=Dh, a_h=a_h, M=M or 0, levels=levels,
                   T=T, P=P, lam=lam)


def afd_apply(prob: Problem, v_flat: np.ndarray, method: str = "fft") -> np.ndarray:
    v = prob.grid_vector(v_flat)
    if method == "direct":
        w = afd_apply_direct(prob.T, v)
    else:
        w = afd_apply_fft(prob.lam, v, prob.P)
    return w.ravel()


def stiffness_apply(prob: Problem, u: np.ndarray, method: str = "fft") -> np.ndarray:
    """y = (I_h^FD)^T A_FD I_h^FD u on the interior block  ((GoFD-2), Remark 3.3).

    Vectors are vertex-indexed (N_v); boundary entries of u are taken as 0
    (homogeneous Dirichlet condition) and boundary entries of y are set to 0.
    """
    uu = np.zeros(len(prob.verts))
    uu[prob.interior] = u[prob.interior]
    v = prob.I @ uu
    w = afd_apply(prob, v, method)
    y = prob.I.T @ w
    out = np.zeros(len(prob.verts))
    out[prob.interior] = y[prob.interior]
    return out


def fraclap_apply(prob: Problem, u: np.ndarray, method: str = "fft") -> np.ndarray:
    """h^{-2s} A_h u with A_h = D_h^{-1} I^T A_FD I  ((Ah-1)), interior entries."""
    y = stiffness_apply(prob, u, method)
    out = np.zeros_like(y)
    ii = prob.interior
    out[ii] = y[ii] / prob.Dh[ii] / prob.h ** (2 * prob.s)
    return out


def located_mask(prob: Problem) -> np.ndarray:
    """Reading R8: a grid node is in Omega iff it is located in the mesh."""
    m = np.zeros(prob.n_grid)
    m[prob.nodes] = 1.0
    return m


def rhs_grid(prob: Problem, f_fd: np.ndarray) -> np.ndarray:
    """b = h^{2s} (I_h^FD)^T f_FD with f_FD = 0 off the mesh  ((GoFD-2))."""
    b = prob.h ** (2 * prob.s) * (prob.I.T @ (located_mask(prob) * f_fd))
    out = np.zeros(len(prob.verts))
    out[prob.interior] = b[prob.interior]
    return out


def rhs_vertex(prob: Problem, f_h: np.ndarray) -> np.ndarray:
    """b = h^{2s} D_h f_h  ((GoFD-3) multiplied through by h^{2s} D_h)."""
    out = np.zeros(len(prob.verts))
    ii = prob.interior
    out[ii] = prob.h ** (2 * prob.s) * prob.Dh[ii] * f_h[ii]
    return out


def cg(apply, b: np.ndarray, interior: np.ndarray, tol: float, maxit: int = 100000,
       precond=None, x0=None):
    """Conjugate gradients on the interior block (Section 3.2, reading R12).

    x0 = 0 unless given; stops when the recursively updated residual satisfies
    ||r|| <= tol ||b||, then reports the true residual ||b - S x|| / ||b||.
    ``precond`` (optional) maps a residual to M^{-1} r.  Returns (x, info).
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    mask = np.zeros_like(b)
    mask[interior] = 1.0
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, {"iters": 0, "rel_res": 0.0}
    r = mask * (b - apply(x))
    z = precond(r) if precond else r
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit and np.linalg.norm(r) > tol * bn:
        q = apply(p)
        a = rz / (p @ q)
        x = x + a * p
        r = r - a * q
        z = precond(r) if precond else r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    true = np.linalg.norm(mask * (b - apply(x))) / bn
    return x, {"iters": it, "rel_res": float(true)}


def solve(prob: Problem, b: np.ndarray, tol: float = 1e-10, method: str = "fft", maxit=100000,
          precond=None):
    return cg(lambda u: stiffness_apply(prob, u, method), b, prob.interior, tol, maxit, precond)


# ============================================================================
# 7. Sparse preconditioner  (Section 3.3, (Ah-4))
# ============================================================================

def stencil_offsets(d: int, pattern: int):
    """Offsets of the 5/7-point (|delta|_1 <= 1) or 9/27-point ({-1,0,1}^d) pattern."""
    import itertools
    offs = list(itertools.product((-1, 0, 1), repeat=d))
    if pattern in (5, 7, 3):
        offs = [o for o in offs if sum(abs(c) for c in o) <= 1]
    return offs


def stencil_matrix(prob: Problem, pattern: int) -> sp.csr_matrix:
    """A_FD^{(k)}: the entries of A_FD at the stencil positions (reading R14)."""
    n = prob.n
    d = prob.d
    N = prob.n_grid
    rows, cols, vals = [], [], []
    ks = np.arange(N)
    coords = []
    rem = ks.copy()
    for ax in range(d):
        coords.append(rem % n[ax])
        rem //= n[ax]
    strides = [int(np.prod(n[:ax])) for ax in range(d)]
    for off in stencil_offsets(d, pattern):
        ok = np.ones(N, dtype=bool)
        tgt = ks.copy()
        for ax in range(d):
            c = coords[ax] + off[ax]
            ok &= (c >= 0) & (c < n[ax])
            tgt += off[ax] * strides[ax]
        tval = prob.T[tuple(abs(o) for o in reversed(off))]
        rows.append(ks[ok])
        cols.append(tgt[ok])
        vals.append(np.full(ok.sum(), tval))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


def preconditioner_matrix(prob: Problem, pattern: int) -> sp.csr_matrix:
    """A_h^{(k)} = I^T A_FD^{(k)} I restricted to the interior block  ((Ah-4)).

    Reading R13: the pattern is structural -- (i, j) is stored iff some grid
    node k and stencil offset delta give a product phi_i(x_k) T_delta
    phi_j(x_{k+delta}) of nonzero factors; an entry whose contributions cancel
    stays in the pattern with its (possibly zero) value.  Zero factors (a grid
    node on a facet has a zero barycentric weight) contribute nothing.
    """
    Ii = prob.I[:, prob.interior].tocsr()
    S = stencil_matrix(prob, pattern).tocsr()
    Ib = Ii.copy()
    Ib.data = (Ib.data != 0).astype(np.float64)
    Ib.eliminate_zeros()
    Sb = S.copy()
    Sb.data = (Sb.data != 0).astype(np.float64)
    Sb.eliminate_zeros()
    struct = (Ib.T @ Sb @ Ib).tocsr()
    struct.sort_indices()
    num = (Ii.T @ S @ Ii).tocsr()
    rows = np.repeat(np.arange(struct.shape[0]), np.diff(struct.indptr))
    vals = np.asarray(num[rows, struct.indices]).ravel() if struct.nnz else np.zeros(0)
    return sp.csr_matrix((vals, struct.indices.copy(), struct.indptr.copy()), shape=struct.shape)


def ic_symbolic(A: sp.csr_matrix, level: int = 1):
    """Level-of-fill pattern of the lower factor (reading R13).

    lev(i,j) = 0 where A_ij != 0; a fill entry created through pivot k gets
    lev(i,k) + lev(k,j) + 1; entries with lev <= level are kept.  Returns one
    sorted column list (j <= i) per row.
    """
    N = A.shape[0]
    A = A.tocsr()
    lev_rows = []
    upper = []          # upper[k] = {j: lev(k,j)} for j > k (the factor's row k of U)
    for i in range(N):
        row = {int(j): 0 for j in A.indices[A.indptr[i]:A.indptr[i + 1]]}
        row[i] = 0
        # eliminate with pivots k < i in increasing order
        ks = sorted(k for k in row if k < i)
        done = set()
        while ks:
            k = ks.pop(0)
            if k in done:
                continue
            done.add(k)
            lik = row[k]
            for j, lkj in upper[k].items():
                lv = lik + lkj + 1
                if lv <= level and lv < row.get(j, 10 ** 9):
                    if j not in row and j < i:
                        ks.append(j)
                        ks.sort()
                    row[j] = lv
        lev_rows.append(row)
        upper.append({j: l for j, l in row.items() if j > i})
    # symmetric pattern: lower triangle of row i = {j <= i}
    return [sorted(j for j in r if j <= i) for i, r in enumerate(lev_rows)]


def ic_numeric(A: sp.csr_matrix, pattern, shift: float = 0.0) -> sp.csr_matrix:
    """Incomplete Cholesky L (L L^T ~ A) on a given lower pattern.

    Row by row: L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj for j in pattern(i),
    L_ii = sqrt(A_ii (1+shift) - sum_{k<i} L_ik^2); updates outside the pattern
    are dropped.  Raises OracleError on a non-positive pivot.
    """
    N = A.shape[0]
    A = A.tocsr()
    Lrows = []
    for i in range(N):
        arow = dict(zip(A.indices[A.indptr[i]:A.indptr[i + 1]].tolist(),
                        A.data[A.indptr[i]:A.indptr[i + 1]].tolist()))
        li = {}
        for j in pattern[i]:
            if j == i:
                continue
            acc = arow.get(j, 0.0)
            lj = Lrows[j]
            for k, v in li.items():
                if k in lj:
                    acc -= v * lj[k]
            li[j] = acc / lj[j]
        diag = arow.get(i, 0.0) * (1.0 + shift) - sum(v * v for v in li.values())
        if not diag > 0.0:
            raise OracleError(f"non-positive pivot at row {i}")
        li[i] = math.sqrt(diag)
        Lrows.append(li)
    rows, cols, vals = [], [], []
    for i, li in enumerate(Lrows):
        for j, v in li.items():
            rows.append(i)
            cols.append(j)
            vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def ic_factor(A: sp.csr_matrix, level: int = 1, max_tries: int = 20):
    """IC(level) with a diagonal shift on breakdown: 0, 1e-3, 2e-3, 4e-3, ..."""
    pat = ic_symbolic(A, level)
    shift = 0.0
    for t in range(max_tries):
        try:
            return ic_numeric(A, pat, shift), shift
        except OracleError:
            shift = 1e-3 * 2 ** t
    raise OracleError("IC breakdown")


def ic_apply(L: sp.csr_matrix, r: np.ndarray) -> np.ndarray:
    """z = L^{-T} L^{-1} r."""
    y = spla.spsolve_triangular(L, r, lower=True)
    return spla.spsolve_triangular(L.T.tocsr(), y, lower=False)


def pcg_ic(prob: Problem, b: np.ndarray, pattern: int = 9, tol: float = 1e-10, maxit=100000,
           perm=None):
    """PCG on (GoFD-2) preconditioned by IC(1) of A_h^{(k)} (Section 3.3)."""
    A = preconditioner_matrix(prob, pattern)
    ii = prob.interior
    if perm is None:
        perm = np.arange(len(ii))
    Ap = A[perm][:, perm].tocsr()
    L, shift = ic_factor(Ap, 1)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))

    def precond(r):
        rp = r[ii][perm]
        z = ic_apply(L, rp)
        out = np.zeros_like(r)
        out[ii] = z[inv]
        return out

    x, info = solve(prob, b, tol, maxit=maxit, precond=precond)
    info["ic_shift"] = shift
    return x, info


def circulant_inverse_apply(prob: Problem, v_flat: np.ndarray) -> np.ndarray:
    """R C^{-1} R^T v: the inverse of the P^d circulant C whose first column is
    the even embedding of T (Section 2.2; C restricted to the grid is A_FD),
    applied to the grid vector v zero-padded to P^d, kept on the n^d corner.
    C^{-1} has the symbol 1/lambda (lambda > 0: T_0 > 0 and T_m < 0 for m != 0,
    so every lambda_k >= lambda_0 = the sum of the embedded T > 0)."""
    d = prob.d
    n = prob.n[0]
    P = prob.P
    vp = np.zeros((P,) * d)
    vp[(slice(0, n),) * d] = prob.grid_vector(v_flat)
    lam = _full_symbol(prob.lam, P)
    w = scipy.fft.ifftn(scipy.fft.fftn(vp) / lam).real
    return np.ascontiguousarray(w[(slice(0, n),) * d]).ravel()


def circulant_precond(prob: Problem, r: np.ndarray) -> np.ndarray:
    """z = M^{-1} r for the circulant alternative of Section 3.3 (reading R24):
    M = I^T C I with C the circulant of A_FD; its inverse is taken as
    M^{-1} = D_h^{-1} I^T C^{-1} I D_h^{-1}, i.e. (I^T C I)^{-1} with I replaced
    by its lumped pseudo-inverse D_h^{-1} I^T (the barycentric weights of a
    grid node sum to 1, so I^T I 1 = D_h).  Interior entries only."""
    ii = prob.interior
    dinv = np.zeros(len(prob.verts))
    dinv[ii] = 1.0 / prob.Dh[ii]
    v = prob.I @ (dinv * r)
    w = circulant_inverse_apply(prob, v)
    y = prob.I.T @ w
    out = np.zeros_like(r)
    out[ii] = dinv[ii] * y[ii]
    return out


def pcg_circulant(prob: Problem, b: np.ndarray, tol: float = 1e-10, maxit=100000):
    """PCG on (GoFD-2) with the circulant preconditioner (circulant_precond)."""
    return solve(prob, b, tol, maxit=maxit, precond=lambda r: circulant_precond(prob, r))


def jacobi_diagonal(prob: Problem) -> np.ndarray:
    """Diagonal of S over the interior vertices (not in the paper; the scaling
    behind the library's diagonal preconditioner):
    S_jj = sum_{k,m} phi_j(x_k) T(|k-m|) phi_j(x_m) over the grid nodes of the
    support of phi_j, T taken at the per-axis distances, written out row by row."""
    I = prob.I.tocsc()
    n = prob.n
    d = prob.d
    out = np.empty(len(prob.interior))
    for r, j in enumerate(prob.interior):
        nodes = I.indices[I.indptr[j]:I.indptr[j + 1]]
        w = I.data[I.indptr[j]:I.indptr[j + 1]]
        coords = []
        rem = nodes.copy()
        for ax in range(d):
            coords.append(rem % n[ax])
            rem = rem // n[ax]
        # T is indexed (k_{d-1}, ..., k_0)
        idx = tuple(np.abs(coords[ax][:, None] - coords[ax][None, :]) for ax in reversed(range(d)))
        out[r] = w @ prob.T[idx] @ w
    return out


def pcg_jacobi(prob: Problem, b: np.ndarray, tol: float = 1e-10, maxit=100000):
    """PCG on (GoFD-2) scaled by the diagonal of S (jacobi_diagonal)."""
    ii = prob.interior
    dinv = 1.0 / jacobi_diagonal(prob)

    def precond(r):
        out = np.zeros_like(r)
        out[ii] = r[ii] * dinv
        return out

    return solve(prob, b, tol, maxit=maxit, precond=precond)


# ============================================================================
# 7b. Adjoint of the vertex-data solve (differentiating (GoFD-3))
# ============================================================================

def barycentric_gradients(verts, simp_rows):
    """grad phi_a (constant on each simplex): (m, d+1, d)."""
    V = verts[simp_rows]
    d = V.shape[2]
    J = np.transpose(V[:, 1:, :] - V[:, :1, :], (0, 2, 1))      # J[:, r, c] = X_{c+1,r} - X_{0,r}
    Ji = np.linalg.inv(J)
    G = np.empty((len(V), d + 1, d))
    G[:, 1:, :] = Ji
    G[:, 0, :] = -Ji.sum(axis=1)
    return G


def adjoint_vertex(prob: Problem, f_h: np.ndarray, u: np.ndarray, g: np.ndarray, tol: float = 1e-13):
    """dL/df and dL/dX for u = S(X)^{-1} h^{2s} D_h(X) f  ((GoFD-3)), given g = dL/du.

    With S lambda = g: dL = lambda^T (db - dS u).  b = h^{2s} D_h f gives
    dL/df = h^{2s} D_h lambda.  For X: phi_a(x_k) depends on the vertices of the
    owner simplex K (held fixed) with d phi_a/d X_{j,c} = -phi_j d phi_a/d x_c, so
    dL/dX_{j,c} = sum_k phi_j(x_k) [d_c(I_h lambda) (A_FD I u)_k
                                   + d_c(I_h u) (A_FD I lambda)_k
                                   - h^{2s} d_c(I_h(lambda f))]   on K.
    Returns (grad_f[N_v], grad_X[N_v, d]).
    """
    ii = prob.interior
    nv = len(prob.verts)
    gg = np.zeros(nv)
    gg[ii] = g[ii]
    lam, _ = cg(lambda x: stiffness_apply(prob, x), gg, ii, tol)
    h2s = prob.h ** (2 * prob.s)
    grad_f = np.zeros(nv)
    grad_f[ii] = h2s * prob.Dh[ii] * lam[ii]
    uu = np.zeros(nv)
    uu[ii] = u[ii]
    w_u = afd_apply(prob, prob.I @ uu)
    w_l = afd_apply(prob, prob.I @ lam)
    K = prob.owner[prob.nodes]
    verts_K = np.asarray(prob.simp)[K]                         # (n_loc, d+1) == ell_idx.T
    G = barycentric_gradients(prob.verts, verts_K)
    gl = np.einsum("na,nac->nc", lam[verts_K], G)
    gu = np.einsum("na,nac->nc", uu[verts_K], G)
    glf = np.einsum("na,nac->nc", (lam * f_h)[verts_K], G)
    c = gl * w_u[prob.nodes][:, None] + gu * w_l[prob.nodes][:, None] - h2s * glf
    grad_X = np.zeros((nv, prob.d))
    for a in range(prob.d + 1):
        np.add.at(grad_X, prob.ell_idx[a], prob.ell_w[a][:, None] * c)
    return grad_f, grad_X


# ============================================================================
# 8. Closed form on the unit ball  ((exam-0), (exam-2) with k = 0)
# ============================================================================

def ball_constant(d: int, s: float) -> float:
    """u = C (1-|x|^2)_+^s solves (-Delta)^s u = 1 on B(0,1):
    C = Gamma(d/2) / (2^{2s} Gamma(1+s) Gamma(d/2+s))  ((exam-0) with k=0)."""
    return Gamma(d / 2.0) / (2.0 ** (2 * s) * Gamma(1 + s) * Gamma(d / 2.0 + s))


def ball_exact(points: np.ndarray, s: float) -> np.ndarray:
    d = points.shape[1]
    r2 = np.sum(points * points, axis=1)
    return ball_constant(d, s) * np.maximum(0.0, 1.0 - r2) ** s


def lumped_l2(verts, simp, e: np.ndarray) -> float:
    """(sum_j m_j e_j^2)^{1/2}, m_j = sum_{K ni j} |K|/(d+1)  (reading R16)."""
    d = verts.shape[1]
    V = verts[simp]
    vol = np.abs(np.linalg.det(V[:, 1:] - V[:, :1])) / math.factorial(d)
    m = np.zeros(len(verts))
    for a in range(d + 1):
        np.add.at(m, simp[:, a], vol / (d + 1))
    return float(np.sqrt(np.sum(m * e * e)))
