"""Groups: several 2D problems on one overlay grid solved together.

Every column of every instance of a group (different meshes, different
alpha: columns converge at different iterations, and the product kernels
skip the converged ones) must reach the FP64 tolerance with the oracle's operator of its own
instance (Section 3.2, (GoFD-2)) and agree with the same instance solved
alone in FP64.  Groups of different grids go through solve_many; one group
runs on the one-warp-per-FFT kernels (circulant 2048).
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


NB = 3


def _instances(n):
    # (mesh, alpha): two disks and an L-shape; the L-shape and the second
    # disk share alpha, so they share one symbol
    d1 = mg.disk_ring_mesh(rings=8, seed=mg.seed_for(5, 1))
    d2 = mg.disk_ring_mesh(rings=11, seed=mg.seed_for(5, 2))
    ls = mg.lshape_mesh(spacing=0.09, seed=mg.seed_for(5, 3))
    return [(d1, 0.5), (d2, 1.5), (ls, 1.5)] if n < 300 else [(d1, 1.0), (ls, 0.7)]


def _build(n):
    from paper_2307_14437_gb300 import Problem
    lo, hi, h = mg.grid_box(2, n)
    probs, refs, Fs = [], [], []
    for k, ((v, s), alpha) in enumerate(_instances(n)):
        probs.append(Problem(v, s, alpha, h, lo, hi, filon_M=2 ** 12 if n <= 512 else 0))
        M = probs[-1].info()["filon_M"]
        refs.append(o.build(2, v, s, alpha, h, lo, hi, exact_weights=False, pruned=True, M=M))
        inside = mg.in_lshape if k == 2 or (n >= 300 and k == 1) else mg.in_disk
        F = mg.rhs_family(mg.grid_points(lo, h, n), NB, seed=mg.seed_for(5, 10 + k), inside=inside)
        Fs.append(torch.tensor(F, device="cuda"))
    return probs, refs, Fs


def _check(probs, refs, Fs, res, tol, single=True):
    for q, ref, F, (U, infos) in zip(probs, refs, Fs, res):
        for c in range(NB):
            f = F[c].cpu().numpy()
            b = o.rhs_grid(ref, f)
            u = U[c].cpu().numpy()
            r = np.linalg.norm(b - o.stiffness_apply(ref, u)) / np.linalg.norm(b)
            assert r <= 1.05 * tol, (c, r, infos[c])
            assert infos[c]["rel_res_fp64"] <= tol
            assert np.all(u[ref.boundary] == 0.0)
            if single and c == 0:
                u1, _ = q.solve(F[c].contiguous(), rhs="grid", mode="fp64", tol=tol)
                assert np.linalg.norm(u - u1.cpu().numpy()) <= 1e-6 * np.linalg.norm(u)


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_group_matches_oracle_and_single_solves(mode):
    from paper_2307_14437_gb300 import Group
    probs, refs, Fs = _build(129)
    g = Group(probs, NB)
    res = g.solve(Fs, mode=mode, tol=1e-8)
    _check(probs, refs, Fs, res, 1e-8)
    # tuned launch shapes: the same solutions to the same tolerance
    g.autotune()
    res2 = g.solve(Fs, mode=mode, tol=1e-8)
    _check(probs, refs, Fs, res2, 1e-8, single=False)
    g.close()
    for q in probs:
        q.close()


def test_groups_of_two_grids_through_solve_many():
    from paper_2307_14437_gb300 import grid_key, group_key, solve_many
    pa, ra, fa = _build(129)
    pb, rb, fb = _build(600)          # circulant 2048: the one-warp-per-FFT kernels
    assert all(q.info()["warp_fft_path"] == 1 for q in pb)
    probs, refs, Fs = pa + pb, ra + rb, fa + fb
    assert len({grid_key(q) for q in probs}) == 2
    # solve_many's groups: (129, 0.5), (129, 1.5) of two instances, (600, 1.0), (600, 0.7)
    assert len({group_key(q) for q in probs}) == 4
    res = solve_many(probs, Fs, mode="mixed", tol=1e-8)
    _check(probs, refs, Fs, res, 1e-8, single=False)
    for q in probs:
        q.close()


def test_group_rejects_problems_on_different_grids():
    from paper_2307_14437_gb300 import GofdError, Group, Problem
    v, s = mg.disk_ring_mesh(rings=6, seed=mg.seed_for(5, 4))
    lo, hi, h = mg.grid_box(2, 33)
    p1 = Problem(v, s, 1.0, h, lo, hi, filon_M=2 ** 10)
    lo, hi, h = mg.grid_box(2, 65)
    p2 = Problem(v, s, 1.0, h, lo, hi, filon_M=2 ** 10)
    with pytest.raises(GofdError) as e:
        Group([p1, p2], 2)
    assert e.value.code == "GOFD_E_ARG"
    p1.close()
    p2.close()
