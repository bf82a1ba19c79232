"""The manufactured solutions of Section 5 ((exam-0), (exam-2)) checked on the
CPU through the FP64 oracle, independently of the CUDA path.

k = 0 reduces to the ball constant (a separate closed form in the oracle);
for k > 0 the oracle's 1D solves (Example 5.1 setting: uniform meshes, h_FD =
a_h, box 1.1 times the domain) converge to the exact solution at the orders
the paper reports: O(h^{min(1, s+1/2)}) in L2 and O(h^s) in the maximum norm.
"""
import math

import numpy as np
import pytest

import manufactured as mf
import meshgen as mg
from oracle import gofd as o


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("s", [0.25, 0.5, 0.75])
def test_k0_is_the_ball_constant(d, s):
    x = np.zeros((3, d))
    assert np.allclose(mf.rhs(0, s, d, x), 1.0 / o.ball_constant(d, s), rtol=1e-14, atol=0)
    assert np.allclose(mf.exact(0, s, d, x), 1.0, rtol=0, atol=0)


@pytest.mark.parametrize("s,k", [(0.25, 2), (0.5, 3), (0.75, 1)])
def test_oracle_1d_converges_to_manufactured_solution(s, k):
    e2, ei = [], []
    for cells in (80, 160, 320):
        v, simp = mg.interval_mesh(cells, jitter=0.0)
        P = o.build(1, v, simp, 2 * s, 2.0 / cells, [-1.1], [1.1], M=2 ** 13)
        b = o.rhs_vertex(P, mf.rhs(k, s, 1, v))
        x, info = o.solve(P, b, 1e-12)
        assert info["rel_res"] < 1e-12
        ue = mf.exact(k, s, 1, v)
        e2.append(o.lumped_l2(v, simp, x - ue) / o.lumped_l2(v, simp, ue))
        ei.append(np.abs(x - ue).max())
    r2 = math.log(e2[1] / e2[2]) / math.log(2)
    ri = math.log(ei[1] / ei[2]) / math.log(2)
    assert abs(r2 - min(1.0, s + 0.5)) <= 0.1, (r2, e2)
    assert abs(ri - s) <= 0.1, (ri, ei)
    assert e2[2] < 0.05
