"""The adjoint (gofd_adjoint and the torch.autograd path) against the oracle's
FP64 adjoint and against central finite differences of GPU solves.

Loss L(u) = 1/2 ||u - u_target||^2 with u = S(X)^{-1} h^{2s} D_h(X) f (GoFD-3).
Finite differences in X use directions that leave every grid node's owner
simplex unchanged (the owner map is piecewise constant in X).
"""
import numpy as np
import pytest

import meshgen as mg
from oracle import gofd as o

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2307_14437_gb300 import build_native
    build_native.build()


def _gpu_loss(v, s, alpha, h, lo, hi, f, ut, tol=1e-12, mode="fp64", keep=False):
    from paper_2307_14437_gb300 import Problem
    P = Problem(v, s, alpha, h, lo, hi)
    fd = torch.tensor(f, device="cuda")
    u, _ = P.solve(fd, rhs="vertex", mode=mode, tol=tol)
    L = 0.5 * float(torch.sum((u - torch.tensor(ut, device="cuda")) ** 2))
    if keep:
        return L, P, u
    owner = P.export_transfer()[0]
    P.close()
    return L, owner


def _grads(P, f, u, ut, tol=1e-12, mode="fp64"):
    g = u - torch.tensor(ut, device="cuda")
    gf, gx, _ = P.adjoint(torch.tensor(f, device="cuda"), u, g, mode=mode, tol=tol)
    return gf.cpu().numpy(), gx.cpu().numpy()


def _small():
    v, s = mg.disk_ring_mesh(rings=5, seed=3)
    lo, hi, h = mg.grid_box(2, 23, -1.1037, 1.0963)
    return v, s, 1.2, h, lo, hi


def _graded(n):
    lo, hi, h = mg.grid_box(2, n)
    v, s = mg.graded_disk_mesh(h, seed=mg.seed_for(4, n))
    return v, s, 1.2, h, lo, hi


def test_adjoint_matches_oracle_small():
    v, s, alpha, h, lo, hi = _small()
    rng = np.random.default_rng(1)
    f = mg.target_bump(v) + 0.3
    ut = 0.05 * rng.standard_normal(len(v))
    _, P, u = _gpu_loss(v, s, alpha, h, lo, hi, f, ut, keep=True)
    gf, gx = _grads(P, f, u, ut)
    ref = o.build(2, v, s, alpha, h, lo, hi, M=P.info()["filon_M"], exact_weights=False)
    ur, _ = o.solve(ref, o.rhs_vertex(ref, f), tol=1e-14)
    rf, rx = o.adjoint_vertex(ref, f, ur, ur - ut)
    assert np.linalg.norm(gf - rf) <= 1e-8 * np.linalg.norm(rf)
    assert np.linalg.norm(gx - rx) <= 1e-8 * np.linalg.norm(rx)
    P.close()


def test_adjoint_matches_oracle_graded_24k():
    # "the FP64 oracle adjoint at 20k vertices": graded disk, 385^2 grid
    v, s, alpha, h, lo, hi = _graded(385)
    assert 15000 < len(v) < 40000
    f = mg.target_bump(v)
    ut = 0.5 * f
    _, P, u = _gpu_loss(v, s, alpha, h, lo, hi, f, ut, keep=True)
    gf, gx = _grads(P, f, u, ut)
    ref = o.build(2, v, s, alpha, h, lo, hi, M=P.info()["filon_M"], exact_weights=False, pruned=True)
    ur, _ = o.solve(ref, o.rhs_vertex(ref, f), tol=1e-13)
    rf, rx = o.adjoint_vertex(ref, f, ur, ur - ut, tol=1e-13)
    assert np.linalg.norm(gf - rf) <= 1e-8 * np.linalg.norm(rf)
    assert np.linalg.norm(gx - rx) <= 1e-8 * np.linalg.norm(rx)
    P.close()


def test_vertex_gradient_finite_differences_64_directions():
    v, s, alpha, h, lo, hi = _graded(385)
    f = mg.target_bump(v)
    ut = 0.5 * f
    L0, P, u = _gpu_loss(v, s, alpha, h, lo, hi, f, ut, keep=True)
    owner0 = P.export_transfer()[0]
    _, gx = _grads(P, f, u, ut)
    P.close()
    rng = np.random.default_rng(mg.seed_for(4, 64))
    good = 0
    eps = 1e-7
    for k in range(64):
        d = np.zeros_like(v)
        sel = rng.choice(len(v), 64, replace=False)
        d[sel] = rng.standard_normal((64, 2))
        Lp, op = _gpu_loss(v + eps * d, s, alpha, h, lo, hi, f, ut)
        Lm, om = _gpu_loss(v - eps * d, s, alpha, h, lo, hi, f, ut)
        if not (np.array_equal(op, owner0) and np.array_equal(om, owner0)):
            continue
        fd = (Lp - Lm) / (2 * eps)
        an = float(np.sum(gx * d))
        assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-3 * np.abs(gx).max()), (k, fd, an)
        good += 1
    assert good >= 32, good


def test_data_gradient_finite_differences_full_graded_2048():
    # the graded-disk differentiation workload at full size: 64 directions in f
    v, s, alpha, h, lo, hi = _graded(2048)
    f = np.ones(len(v))
    ut = np.asarray(0.0 * f)
    from paper_2307_14437_gb300 import Problem
    P = Problem(v, s, alpha, h, lo, hi)
    ft = torch.tensor(mg.target_bump(v), device="cuda")
    u_t, _ = P.solve(ft, rhs="vertex", mode="mixed", tol=1e-10)
    ut = u_t.cpu().numpy()
    fd0 = torch.tensor(f, device="cuda")
    u, _ = P.solve(fd0, rhs="vertex", mode="mixed", tol=1e-11)
    gf, gx = _grads(P, f, u, ut, tol=1e-11, mode="mixed")
    rng = np.random.default_rng(mg.seed_for(4, 2048))
    eps = 1e-3
    for k in range(64):
        d = rng.standard_normal(len(v))
        up, _ = P.solve(torch.tensor(f + eps * d, device="cuda"), rhs="vertex", mode="mixed", tol=1e-11)
        um, _ = P.solve(torch.tensor(f - eps * d, device="cuda"), rhs="vertex", mode="mixed", tol=1e-11)
        Lp = 0.5 * float(torch.sum((up - u_t) ** 2))
        Lm = 0.5 * float(torch.sum((um - u_t) ** 2))
        fd = (Lp - Lm) / (2 * eps)
        an = float(gf @ d)
        assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-12), (k, fd, an)
    assert np.isfinite(gx).all()
    P.close()


def test_vertex_gradient_finite_differences_full_graded_2048():
    # the graded-disk differentiation workload at full size (~2e5 vertices,
    # 2048^2 grid): dL/dX against central differences of GPU solves on 64
    # seeded directions, each moving 64 random vertices; a direction counts
    # only if neither perturbed mesh changes any grid node's owner simplex.
    # The solves go to 1e-13 (diagonal preconditioner, for speed) and
    # L(X+) - L(X-) is formed as 1/2 (u+ - u-).(u+ + u- - 2 u_t), so that the
    # O(eps) difference is not lost to the rounding of two O(1) losses.
    from paper_2307_14437_gb300 import Problem
    v, s, alpha, h, lo, hi = _graded(2048)
    assert len(v) > 150000
    f = mg.target_bump(v)
    ft = torch.tensor(f, device="cuda")
    P = Problem(v, s, alpha, h, lo, hi, precond=1)
    ut = 0.5 * P.solve(ft, rhs="vertex", mode="mixed", tol=1e-13)[0]
    u, _ = P.solve(ft, rhs="vertex", mode="mixed", tol=1e-13)
    owner0 = P.export_transfer()[0]
    gf, gx, _ = P.adjoint(ft, u, u - ut, mode="mixed", tol=1e-13)
    gx = gx.cpu().numpy()
    P.close()
    scale = np.abs(gx).max()
    assert np.isfinite(gx).all() and scale > 0

    def solve_at(X):
        Q = Problem(X, s, alpha, h, lo, hi, precond=1)
        uq, _ = Q.solve(ft, rhs="vertex", mode="mixed", tol=1e-13)
        same = np.array_equal(Q.export_transfer()[0], owner0)
        Q.close()
        return uq, same

    rng = np.random.default_rng(mg.seed_for(4, 2048 + 64))
    eps = 1e-7
    good = 0
    for k in range(64):
        d = np.zeros_like(v)
        sel = rng.choice(len(v), 64, replace=False)
        d[sel] = rng.standard_normal((64, 2))
        up, sp = solve_at(v + eps * d)
        um, sm = solve_at(v - eps * d)
        if not (sp and sm):
            continue
        dL = 0.5 * float(torch.dot(up - um, up + um - 2 * ut))
        fd = dL / (2 * eps)
        an = float(np.sum(gx * d))
        assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-3 * scale), (k, fd, an)
        good += 1
    assert good >= 48, good


def test_autograd_function_matches_adjoint():
    from paper_2307_14437_gb300 import gofd as G
    v, s, alpha, h, lo, hi = _small()
    rng = np.random.default_rng(1)
    f0 = mg.target_bump(v) + 0.3
    ut = torch.tensor(0.05 * rng.standard_normal(len(v)), device="cuda")
    f = torch.tensor(f0, device="cuda", requires_grad=True)
    X = torch.tensor(v, device="cuda", requires_grad=True)
    u = G.solve(f, X, s, alpha, h, lo, hi, tol=1e-12, mode="fp64")
    loss = 0.5 * torch.sum((u - ut) ** 2)
    loss.backward()
    _, P, uu = _gpu_loss(v, s, alpha, h, lo, hi, f0, ut.cpu().numpy(), keep=True)
    gf, gx = _grads(P, f0, uu, ut.cpu().numpy())
    assert np.allclose(f.grad.cpu().numpy(), gf, rtol=1e-10, atol=1e-14)
    assert np.allclose(X.grad.cpu().numpy(), gx, rtol=1e-10, atol=1e-14)
    P.close()
