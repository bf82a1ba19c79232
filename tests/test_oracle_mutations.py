"""Planted mistakes in the oracle (on the CPU) must each fail one of its pins.

Each test patches one plausible error into a copy of an oracle function --
a dropped term, a wrong sign, a wrong index or tie rule, a missing boundary
condition -- and checks that the corresponding pin detects it.
"""
import json
import os

import numpy as np
from scipy.special import gamma as G

import meshgen as mg
from oracle import gofd as o

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gamma_pin_error(mod, s=0.75, n=32):
    T = mod.coefficients(1, s, n, M=2 ** 12)
    p = np.arange(n)
    exact = (-1.0) ** p * G(2 * s + 1) / (G(p + s + 1) * G(s - p + 1))
    return np.abs(T - exact).max()


def test_dropped_singular_exponent_is_caught(monkeypatch):
    # Richardson that ignores the |xi|^{2s} singularity (even powers only)
    assert _gamma_pin_error(o) < 1e-13
    monkeypatch.setattr(o, "richardson_exponents", lambda d, s, levels: [2.0, 4.0, 6.0][: levels - 1])
    assert _gamma_pin_error(o) > 1e-10


def test_wrong_sign_factor_is_caught(monkeypatch):
    real = o.filon_coefficients

    def wrong_sign(d, s, n, M):
        f = real(d, s, n, M)
        fac = (-1.0) ** np.arange(n)
        for ax in range(d):
            shape = [1] * d
            shape[ax] = n
            f = f * fac.reshape(shape)                 # undoes (-1)^p of (T-0)
        return f

    monkeypatch.setattr(o, "filon_coefficients", wrong_sign)
    T = o.coefficients(2, 1.0, 4, M=2 ** 10)
    assert abs(T[0, 1] - (-1.0)) > 0.5                 # the 5-point pin fails


def test_wrong_tie_rule_is_caught(monkeypatch):
    g = json.load(open(os.path.join(GOLD, "two_triangles.json")))
    v = np.array(g["vertices"])
    s = np.array(g["simplices"])
    lo = np.array(g["box_lo"])
    n = o.grid_shape(lo, g["box_hi"], g["h"])
    # reverse the element order and map back: equivalent to "highest index wins"
    own = o.locate(v, s[::-1], lo, g["h"], n)
    own = np.where(own >= 0, len(s) - 1 - own, -1)
    assert own.tolist() != g["owner"]


def test_missing_dirichlet_mask_is_caught(monkeypatch):
    d, nn = 2, 11
    lo, hi, h = mg.grid_box(d, nn)
    verts, simp = mg.grid_aligned_mesh(d, -1.0, h, 6, origin_cells=2)
    P = o.build(d, verts, simp, 1.2, h, lo, hi, M=2 ** 10)
    u = mg.random_vector(len(verts), 9)

    def leaky(prob, uu, method="fft"):          # boundary values not zeroed
        v = prob.I @ uu
        w = o.afd_apply(prob, v, method)
        y = prob.I.T @ w
        out = np.zeros(len(prob.verts))
        out[prob.interior] = y[prob.interior]
        return out

    k = np.rint((verts - lo) / h).astype(np.int64)
    lin = k[:, 0] + nn * k[:, 1]
    v = np.zeros(P.n_grid)
    uz = np.where(P.boundary, 0.0, u)
    v[lin] = uz
    ref = np.where(P.boundary, 0.0, o.afd_apply_direct(P.T, v.reshape(nn, nn)).ravel()[lin])
    assert np.abs(o.stiffness_apply(P, u) - ref).max() < 1e-13
    assert np.abs(leaky(P, u) - ref).max() > 1e-3


def test_short_circulant_is_caught():
    # P >= 2n-2 is exact; one slot less wraps distinct offsets onto each other
    n = 9
    T = o.coefficients(2, 0.75, n, M=2 ** 10)
    v = np.random.default_rng(3).uniform(-1, 1, size=(n, n))
    ref = o.afd_apply_direct(T, v)
    assert np.abs(o.afd_apply_fft(o.symbol(T, 16), v, 16) - ref).max() < 1e-13
    c = o.circulant_first_column(T, 15)
    lam = np.fft.fftn(c).real[:8, :8]
    vp = np.zeros((15, 15))
    vp[:n, :n] = v
    full = np.fft.fftn(c).real
    bad = np.fft.ifftn(np.fft.fftn(vp) * full).real[:n, :n]
    assert np.abs(bad - ref).max() > 1e-4


def _mutant(fn, old, new):
    """A copy of oracle function `fn` with the source text `old` replaced."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(fn))
    assert old in src, old
    ns = dict(fn.__globals__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    return ns[fn.__name__]


def _four_cycle():
    import scipy.sparse as sp
    return sp.csr_matrix(np.array([[4, -1, 0, -1], [-1, 4, -1, 0], [0, -1, 4, -1], [-1, 0, -1, 4.0]]))


def test_fill_level_off_by_one_is_caught(monkeypatch):
    # a fill entry through pivot k at level lev(i,k) + lev(k,j) (no + 1): IC(0)
    # then keeps fill, and the hand-worked level-0 pattern of the 4-cycle fails
    A = _four_cycle()
    assert o.ic_symbolic(A, 0) == [[0], [0, 1], [1, 2], [0, 2, 3]]
    monkeypatch.setattr(o, "ic_symbolic", _mutant(o.ic_symbolic, "lik + lkj + 1", "lik + lkj"))
    assert o.ic_symbolic(A, 0) != [[0], [0, 1], [1, 2], [0, 2, 3]]


def test_dropped_cross_terms_in_the_factor_are_caught(monkeypatch):
    # L_ij without the sum over earlier columns: at full fill the factor is
    # no longer the exact Cholesky factor
    import scipy.sparse as sp
    rng = np.random.default_rng(1)
    A = sp.random(30, 30, density=0.15, random_state=rng)
    A = A + A.T
    A = (A + sp.diags(np.abs(A).sum(axis=1).A.ravel() + 1.0)).tocsr()
    ref = np.linalg.cholesky(A.toarray())
    L, _ = o.ic_factor(A, level=100)
    assert np.abs(L.toarray() - ref).max() < 1e-12
    monkeypatch.setattr(o, "ic_numeric", _mutant(o.ic_numeric, "acc -= v * lj[k]", "acc -= 0.0 * v * lj[k]"))
    L, _ = o.ic_factor(A, level=100)
    assert np.abs(L.toarray() - ref).max() > 1e-3


def test_one_sided_diagonal_scaling_is_caught(monkeypatch):
    # M^{-1} = D_h^{-1} I^T C^{-1} I D_h^{-1}: dropping the right-hand scaling
    # breaks the symmetry pin (the grid-aligned pin has D_h = 1 and cannot see it)
    v, s = mg.disk_ring_mesh(rings=8, seed=3)
    lo, hi, h = mg.grid_box(2, 25)
    P = o.build(2, v, s, 1.5, h, lo, hi, M=2 ** 10, exact_weights=False)
    a = mg.random_vector(len(P.verts), 12)
    b = mg.random_vector(len(P.verts), 13)
    a[P.boundary] = 0.0
    b[P.boundary] = 0.0

    def asym():
        Ma, Mb = o.circulant_precond(P, a), o.circulant_precond(P, b)
        return abs(a @ Mb - b @ Ma) / abs(a @ Mb)

    assert asym() <= 1e-12
    monkeypatch.setattr(o, "circulant_precond", _mutant(o.circulant_precond, "prob.I @ (dinv * r)", "prob.I @ r"))
    assert asym() > 1e-6


def test_symbol_instead_of_its_inverse_is_caught(monkeypatch):
    # C^{-1} applied as a product with lambda instead of a division: the dense
    # circulant solve pin fails
    d, n = 2, 5
    T = o.coefficients(d, 0.6, n, 2 ** 10)
    P = o.circulant_size(n)
    c = o.circulant_first_column(T, P)
    idx = np.stack(np.meshgrid(*[np.arange(P)] * d, indexing="ij"), -1).reshape(-1, d)
    diff = (idx[:, None, :] - idx[None, :, :]) % P
    C = c[tuple(diff[..., a] for a in range(d))]
    vg = np.random.default_rng(7).standard_normal((n,) * d)
    vp = np.zeros((P,) * d)
    vp[(slice(0, n),) * d] = vg
    want = np.linalg.solve(C, vp.ravel()).reshape((P,) * d)[(slice(0, n),) * d].ravel()

    class _G:
        pass
    g = _G()
    g.d, g.n, g.P, g.lam = d, (n,) * d, P, o.symbol(T, P)
    g.grid_vector = lambda f: f.reshape((n,) * d)
    assert np.abs(o.circulant_inverse_apply(g, vg.ravel()) - want).max() <= 1e-12 * np.abs(want).max()
    bad = _mutant(o.circulant_inverse_apply, "scipy.fft.fftn(vp) / lam", "scipy.fft.fftn(vp) * lam")
    assert np.abs(bad(g, vg.ravel()) - want).max() > 1e-3 * np.abs(want).max()


def test_diagonal_without_cross_pairs_is_caught(monkeypatch):
    # S_jj keeps only the pairs k = m (sum_k w_k^2 T_0): the column-by-column
    # diagonal of S assembled from the stiffness product disagrees
    v, s = mg.disk_ring_mesh(rings=4, seed=mg.seed_for(1, 9))
    lo, hi, h = mg.grid_box(2, 13)
    ref = o.build(2, v, s, 1.3, h, lo, hi, M=2 ** 9)
    want = np.empty(len(ref.interior))
    for r, j in enumerate(ref.interior):
        e = np.zeros(len(v))
        e[j] = 1.0
        want[r] = o.stiffness_apply(ref, e)[j]
    assert np.abs(o.jacobi_diagonal(ref) - want).max() <= 1e-12 * np.abs(want).max()
    bad = _mutant(o.jacobi_diagonal, "out[r] = w @ prob.T[idx] @ w", "out[r] = (w * w) @ np.diagonal(prob.T[idx])")
    assert np.abs(bad(ref) - want).max() > 1e-3 * np.abs(want).max()


def test_dropped_scale_of_the_grid_rhs_is_caught(monkeypatch):
    # (GoFD-2) without its h^{2s}: the grid right-hand side no longer equals
    # (GoFD-3) for f = 1
    v, s = mg.disk_ring_mesh(rings=6, seed=mg.seed_for(1, 3))
    lo, hi, h = mg.grid_box(2, 21)
    P = o.build(2, v, s, 1.2, h, lo, hi, M=2 ** 9)
    b = o.rhs_vertex(P, np.ones(len(P.verts)))
    assert np.abs(o.rhs_grid(P, np.ones(P.n_grid)) - b).max() < 1e-15
    bad = _mutant(o.rhs_grid, "prob.h ** (2 * prob.s) * ", "")
    assert np.abs(bad(P, np.ones(P.n_grid)) - b).max() > 1e-3 * np.abs(b).max()
