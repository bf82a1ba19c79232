"""Manufactured solutions with k > 0 on the unit disk (Section 5, (exam-0) and
(exam-2)): for

    f = 2^{2s} Gamma(1+s+k) Gamma(d/2+s+k) / (k! Gamma(d/2+k)) P_k^{(s, d/2-1)}(2|x|^2 - 1)

the exact solution of (FL-1) on the unit ball is
u = (1 - |x|^2)_+^s P_k^{(s, d/2-1)}(2|x|^2 - 1).  The GPU solves (GoFD-3) with
vertex data on a ladder of ring meshes (overlay box 1.1 times the domain and
h_FD about a_h, as the paper takes them) and the mass-lumped L2 error must
fall at least at the rate the paper reports for fixed meshes,
O(h^{min(1, s+1/2)}) (Example 5.1, Remark 3.6).  On these meshes the observed
vertex-error order for smooth data can exceed it (the FP64 oracle gives 1.26
at s = 1/2 and 0.84 at s = 1/4 on the same ladder), so the paper's order is a
lower bound here (minus 0.15 for the finite ladder).
"""
import math

import numpy as np
import pytest

import manufactured
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


_rhs = manufactured.rhs
_exact = manufactured.exact


def _error(rings, alpha, k):
    from paper_2307_14437_gb300 import Problem
    v, s = mg.disk_ring_mesh(rings=rings, seed=mg.seed_for(6, rings))
    n = int(round(5.3 * rings)) + 1                   # h_FD about a_h
    lo, hi, h = mg.grid_box(2, n, -1.1, 1.1)
    gp = Problem(v, s, alpha, h, lo, hi)
    sv = alpha / 2
    f = torch.tensor(_rhs(k, sv, 2, v), device="cuda")
    u, info = gp.solve(f, rhs="vertex", mode="mixed", tol=1e-10)
    assert info["rel_res_fp64"] <= 1e-10
    gp.close()
    ue = _exact(k, sv, 2, v)
    return o.lumped_l2(v, s, u.cpu().numpy() - ue) / o.lumped_l2(v, s, ue)


@pytest.mark.parametrize("alpha,k", [(1.0, 3), (0.5, 2)])
def test_manufactured_solution_converges_at_the_paper_rate(alpha, k):
    ladder = [24, 48, 96]
    errs = [_error(r, alpha, k) for r in ladder]
    rate = math.log(errs[1] / errs[2]) / math.log(ladder[2] / ladder[1])
    expect = min(1.0, alpha / 2 + 0.5)
    assert errs[2] < errs[1] < errs[0], errs
    assert rate >= expect - 0.15, (rate, expect, errs)
    assert errs[2] < 0.04, errs


@pytest.mark.parametrize("alpha", [0.5, 1.5])
def test_1d_rates_of_example_5_1(alpha):
    # Example 5.1: the 1D problem with k = 0 on uniform meshes, h_FD = a_h (grid
    # nodes on the mesh vertices), box 1.1 times the domain; the paper reports
    # O(h^s) in the maximum norm and O(h^{min(1, s+1/2)}) in L2 (the FP64 oracle
    # reproduces 0.25 / 0.75 at s = 1/4 and 0.75 / 0.98 at s = 3/4)
    from paper_2307_14437_gb300 import Problem
    sv = alpha / 2
    e2, ei = [], []
    ladder = [80, 160, 320, 640]
    for cells in ladder:
        v, s = mg.interval_mesh(cells, jitter=0.0)
        gp = Problem(v, s, alpha, 2.0 / cells, [-1.1], [1.1])
        f = torch.tensor(_rhs(0, sv, 1, v), device="cuda")
        u, info = gp.solve(f, rhs="vertex", mode="fp64", tol=1e-12)
        gp.close()
        err = u.cpu().numpy() - _exact(0, sv, 1, v)
        e2.append(o.lumped_l2(v, s, err))
        ei.append(np.abs(err).max())
    r2 = math.log(e2[-2] / e2[-1]) / math.log(2)
    ri = math.log(ei[-2] / ei[-1]) / math.log(2)
    assert abs(r2 - min(1.0, sv + 0.5)) <= 0.1, (r2, e2)
    assert abs(ri - sv) <= 0.1, (ri, ei)


def _ball_error(shells, alpha, k):
    from paper_2307_14437_gb300 import Problem
    v, s = mg.ball_shell_mesh(shells=shells, seed=mg.seed_for(7, shells))
    n = int(round(5.3 * shells)) + 1                  # h_FD about 0.4 times the shell spacing
    lo, hi, h = mg.grid_box(3, n, -1.1, 1.1)
    gp = Problem(v, s, alpha, h, lo, hi)
    sv = alpha / 2
    f = torch.tensor(_rhs(k, sv, 3, v), device="cuda")
    u, info = gp.solve(f, rhs="vertex", mode="mixed", tol=1e-10)
    assert info["rel_res_fp64"] <= 1e-10
    gp.close()
    ue = _exact(k, sv, 3, v)
    return o.lumped_l2(v, s, u.cpu().numpy() - ue) / o.lumped_l2(v, s, ue)


@pytest.mark.parametrize("alpha,k", [(1.0, 0), (1.5, 2)])
def test_ball_ladder_converges(alpha, k):
    # (exam-0)/(exam-2) on the unit ball (Example 5.3 takes k = 0, s = 1/2):
    # shell meshes with 8, 16 and 32 shells (2.6e3 to 1.4e5 vertices); the
    # paper reports 3D rates slightly below O(h^{min(1, s+1/2)}) on fixed
    # meshes, so the observed order must be within 0.25 of it
    ladder = [8, 16, 32]
    errs = [_ball_error(sh, alpha, k) for sh in ladder]
    rate = math.log(errs[1] / errs[2]) / math.log(ladder[2] / ladder[1])
    expect = min(1.0, alpha / 2 + 0.5)
    print(f"ball ladder alpha={alpha} k={k}: errors {errs}, order {rate:.3f}")
    assert errs[2] < errs[1] < errs[0], errs
    assert rate >= expect - 0.25, (rate, expect, errs)
