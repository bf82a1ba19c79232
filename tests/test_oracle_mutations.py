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
