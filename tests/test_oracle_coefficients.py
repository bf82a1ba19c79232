"""Pins of the oracle's FD coefficients T and circulant symbol.

Section 2.1 ((FL-6), (T-1), (T-2)), Section 2.3 ((T-0)..(T-1D-0)) and the
circulant embedding of Section 2.2.
"""
import math

import numpy as np
import pytest
from scipy.special import gamma as G

from oracle import gofd as o


@pytest.mark.parametrize("s,tol", [(0.25, 2e-10), (0.5, 1e-14), (0.75, 1e-13), (0.95, 1e-13)])
def test_1d_filon_richardson_matches_gamma_formula(s, tol):
    # (T-1D-0) is the exact value of (T-1) in 1D
    n = 64
    T = o.coefficients(1, s, n, M=2 ** 13)
    p = np.arange(n)
    exact = (-1.0) ** p * G(2 * s + 1) / (G(p + s + 1) * G(s - p + 1))
    assert np.abs(T - exact).max() < tol


def test_1d_half_order_closed_form():
    # s = 1/2 in 1D: psi = 2|sin(xi/2)|, whose Fourier coefficients are
    # T_p = -4 / (pi (4p^2 - 1))  (elementary integral of (T-1))
    n = 40
    T = o.coefficients(1, 0.5, n, M=2 ** 12)
    p = np.arange(n)
    assert np.abs(T + 4.0 / (np.pi * (4.0 * p * p - 1.0))).max() < 1e-14


@pytest.mark.parametrize("d", [1, 2, 3])
def test_s1_gives_standard_laplacian(d):
    # s = 1: psi = sum 4 sin^2(xi_i/2) is the symbol of the (2d+1)-point
    # Laplacian (5-point) of Section 2.1, so T_0 = 2d, T_{e_i} = -1, else 0
    n = 6
    M = 2 ** 9 if d == 3 else 2 ** 10
    T = o.coefficients(d, 1.0, n, M=M)
    ref = np.zeros((n,) * d)
    ref[(0,) * d] = 2.0 * d
    for ax in range(d):
        idx = [0] * d
        idx[ax] = 1
        ref[tuple(idx)] = -1.0
    assert np.abs(T - ref).max() < 1e-13


def test_axis_symmetry_2d():
    T = o.coefficients(2, 0.6, 32, M=2 ** 11)
    assert np.abs(T - T.T).max() < 1e-15


def _gl_coefficient_2d(s, p, q, levels=45, order=24):
    """Independent route: tensor Gauss-Legendre quadrature of (T-1).

    T_{p,q} = pi^{-2} int_0^pi int_0^pi psi cos(p xi) cos(q eta) by evenness;
    the square is split into layers graded geometrically toward the singular
    corner (0,0), outer layers further subdivided for the oscillation.
    """
    x, w = np.polynomial.legendre.leggauss(order)

    def square(a0, a1, b0, b1):
        xs = 0.5 * (a1 - a0) * x + 0.5 * (a1 + a0)
        ys = 0.5 * (b1 - b0) * x + 0.5 * (b1 + b0)
        X, Y = np.meshgrid(xs, ys, indexing="ij")
        f = (4 * np.sin(X / 2) ** 2 + 4 * np.sin(Y / 2) ** 2) ** s * np.cos(p * X) * np.cos(q * Y)
        return 0.25 * (a1 - a0) * (b1 - b0) * (w[:, None] * w[None, :] * f).sum()

    tot = 0.0
    for l in range(levels):
        big = np.pi * 2.0 ** (-l)
        mid = big / 2
        sub = 8 if l == 0 else (4 if l < 3 else 1)
        for (a0, a1, b0, b1) in ((mid, big, 0, mid), (0, mid, mid, big), (mid, big, mid, big)):
            ea = np.linspace(a0, a1, sub + 1)
            eb = np.linspace(b0, b1, sub + 1)
            for i in range(sub):
                for j in range(sub):
                    tot += square(ea[i], ea[i + 1], eb[j], eb[j + 1])
    return tot / np.pi ** 2


@pytest.mark.parametrize("s", [0.25, 0.5, 0.75])
def test_2d_matches_gauss_legendre_quadrature_of_definition(s):
    T = o.coefficients(2, s, 8, M=2 ** 12)
    for (p, q) in [(0, 0), (1, 0), (1, 1), (3, 2), (7, 5)]:
        ref = _gl_coefficient_2d(s, p, q)
        assert abs(T[q, p] - ref) < 1e-10, (p, q, T[q, p], ref)


def _gl_coefficient_3d(s, p, levels=40, order=16):
    """Independent route in 3D: tensor Gauss-Legendre quadrature of (T-1),
    T_p = pi^{-3} int_{[0,pi]^3} psi prod_i cos(p_i xi_i), on cubic shells
    [0, pi 2^-l]^3 minus [0, pi 2^-l-1]^3 (seven boxes each) graded toward the
    singular corner, the outer shells further subdivided."""
    x, w = np.polynomial.legendre.leggauss(order)
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]

    def box(lo, hi):
        pts = [0.5 * (hi[a] - lo[a]) * x + 0.5 * (hi[a] + lo[a]) for a in range(3)]
        X, Y, Z = np.meshgrid(*pts, indexing="ij")
        f = ((4 * np.sin(X / 2) ** 2 + 4 * np.sin(Y / 2) ** 2 + 4 * np.sin(Z / 2) ** 2) ** s
             * np.cos(p[0] * X) * np.cos(p[1] * Y) * np.cos(p[2] * Z))
        return np.prod([(hi[a] - lo[a]) / 2 for a in range(3)]) * (W * f).sum()

    tot = 0.0
    for l in range(levels):
        big = np.pi * 2.0 ** (-l)
        mid = big / 2
        sub = 4 if l == 0 else (2 if l < 3 else 1)
        for corner in range(1, 8):
            lo = [mid if (corner >> a) & 1 else 0.0 for a in range(3)]
            hi = [big if (corner >> a) & 1 else mid for a in range(3)]
            e = [np.linspace(lo[a], hi[a], sub + 1) for a in range(3)]
            for i in range(sub):
                for j in range(sub):
                    for k in range(sub):
                        tot += box([e[0][i], e[1][j], e[2][k]], [e[0][i + 1], e[1][j + 1], e[2][k + 1]])
    return tot / np.pi ** 3


@pytest.mark.parametrize("s", [0.25, 0.75])
def test_3d_matches_gauss_legendre_quadrature_of_definition(s):
    T = o.coefficients(3, s, 4, M=2 ** 9)
    for p in [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1), (2, 1, 0), (3, 2, 1)]:
        ref = _gl_coefficient_3d(s, p)
        assert abs(T[p[2], p[1], p[0]] - ref) < 1e-10, (p, T[p[2], p[1], p[0]], ref)


@pytest.mark.parametrize("d,n,M,s", [(1, 40, 2 ** 10, 0.3), (2, 20, 2 ** 9, 0.6), (3, 9, 2 ** 8, 0.75),
                                     (3, 5, 2 ** 6, 0.25)])
def test_coefficients_at_equals_full_array(d, n, M, s):
    # the sampled evaluation (a direct trapezoid sum) equals the DCT-I route
    # entry by entry, including the last index n-1 on the coarsest level
    T = o.coefficients(d, s, n, M=M)
    rng = np.random.default_rng(d)
    ps = np.vstack([np.zeros((1, d), dtype=np.int64), np.full((1, d), n - 1), rng.integers(0, n, size=(20, d))])
    got = o.coefficients_at(d, s, ps, M)
    want = np.array([T[tuple(p[::-1])] for p in ps])
    assert np.abs(got - want).max() < 1e-14 * max(1.0, np.abs(want).max())
    with pytest.raises(o.OracleError):
        o.coefficients_at(d, s, np.full((1, d), M // 8), M)


@pytest.mark.parametrize("d,s", [(2, 0.5), (2, 0.75), (3, 0.75)])
def test_tail_follows_hypersingular_kernel(d, s):
    # T_p ~ -C_{d,s} |p|^{-(d+2s)} with C_{d,s} = 2^{2s} s Gamma(s+d/2) /
    # (pi^{d/2} Gamma(1-s)), the kernel constant of the integral fractional
    # Laplacian: the coefficients sample the kernel at lattice distances
    n = 48 if d == 2 else 24
    M = 2 ** 12 if d == 2 else 2 ** 9
    T = o.coefficients(d, s, n, M=M)
    C = 2 ** (2 * s) * s * G(s + d / 2) / (np.pi ** (d / 2) * G(1 - s))
    p = np.array([n - 8, n - 14] + [0] * (d - 2))
    val = T[tuple(reversed(p))]
    ratio = val / (-C * np.linalg.norm(p) ** (-(d + 2 * s)))
    assert abs(ratio - 1) < 2e-2


def test_coefficient_sum_rules():
    # sum_p T_p = psi(0) = 0 and sum_p (-1)^{|p|} T_p = psi(pi,...,pi) = (4d)^s:
    # evaluations of the Fourier series (T-1) at xi = 0 and xi = pi.
    d, s, n = 2, 0.75, 256
    T = o.coefficients(d, s, n, M=2 ** 12)
    w1 = np.where(np.arange(n) == 0, 1.0, 2.0)
    W = np.outer(w1, w1)
    alt = np.outer((-1.0) ** np.arange(n), (-1.0) ** np.arange(n))
    assert abs((W * alt * T).sum() - (4 * d) ** s) < 1e-6
    # the plain sum converges like n^{-2s}
    assert abs((W * T).sum()) < 5.0 * n ** (-2 * s)


def test_symbol_against_direct_dft():
    d, n = 2, 5
    T = o.coefficients(d, 0.6, n, M=2 ** 10)
    P = o.circulant_size(n)
    assert P == 2 * n - 2
    lam = o.symbol(T, P)
    # direct DFT over the P circulant slots: slot m in (-P/2, P/2] holds
    # T_{|m|} when |m| < n, else 0 (Section 2.2)
    ref = np.zeros((P // 2 + 1,) * d)
    offs = range(-P // 2 + 1, P // 2 + 1)
    for k1 in range(P // 2 + 1):
        for k0 in range(P // 2 + 1):
            acc = 0.0
            for m1 in offs:
                for m0 in offs:
                    if abs(m1) < n and abs(m0) < n:
                        acc += T[abs(m1), abs(m0)] * math.cos(2 * math.pi * (k0 * m0 + k1 * m1) / P)
            ref[k1, k0] = acc
    assert np.abs(lam - ref).max() < 1e-13


def test_symbol_approximates_fd_symbol():
    # lambda_k ~ psi(2 pi k / P): the embedded coefficients are a truncated
    # Fourier series of psi (FL-6)
    d, s, n = 2, 0.75, 128
    T = o.coefficients(d, s, n, M=2 ** 12)
    P = o.circulant_size(n)
    lam = o.symbol(T, P)
    k = np.arange(P // 2 + 1)
    xi = 2 * np.pi * k / P
    psi = (4 * np.sin(xi[:, None] / 2) ** 2 + 4 * np.sin(xi[None, :] / 2) ** 2) ** s
    assert np.abs(lam - psi).max() < 3.0 * n ** (-2 * s)


def test_circulant_size_rule():
    assert o.circulant_size(1024) == 2048
    assert o.circulant_size(128) == 256
    assert o.circulant_size(100) == 256
    assert o.circulant_size(129) == 256
    assert o.circulant_size(2) == 2


def test_richardson_exponent_reading():
    assert o.richardson_exponents(2, 0.5, 4) == [2.0, 3.0, 4.0]
    assert o.richardson_exponents(2, 1.0, 4) == [2.0, 4.0, 6.0]
    assert o.richardson_exponents(3, 0.75, 4) == [2.0, 4.0, 4.5]
    assert o.richardson_exponents(1, 0.25, 4) == [1.5, 2.0, 3.5]
