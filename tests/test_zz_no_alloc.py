"""The allocation-free A_FD entry point against the handle-based one.

gofd_afd_apply_noalloc serves callers that cannot allocate device memory when
they need the product (graph capture, framework-owned allocators, real-time
loops); its scratch is a fixed device array inside the library.  Two calls in
a row must each match gofd_afd_apply within the FP32 tolerance of the parity
tests.  This file runs last so that a failure here leaves every other test
already run.
"""
import numpy as np
import pytest

import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2307_14437_gb300 import build_native
    build_native.build()


def _problem(case):
    from paper_2307_14437_gb300 import Problem
    if case == "disk65":
        v, s = mg.disk_ring_mesh(rings=12, seed=mg.seed_for(1, 3))
        d, n, alpha, M = 2, 65, 1.2, 2 ** 10
    else:
        v, s = mg.ball_shell_mesh(shells=3, seed=mg.seed_for(3, 2))
        d, n, alpha, M = 3, 9, 1.5, 2 ** 8
    lo, hi, h = mg.grid_box(d, n)
    return Problem(v, s, alpha, h, lo, hi, filon_M=M), d, n


@pytest.mark.parametrize("case", ["disk65", "ball9"])
def test_noalloc_matches_handle_path_twice(case):
    from paper_2307_14437_gb300.gofd import afd_apply_noalloc
    prob, d, n = _problem(case)
    lam = torch.tensor(prob.symbol() / float(prob.P) ** d, dtype=torch.float32, device="cuda")
    v = torch.tensor(mg.random_vector(prob.n_grid, 31), dtype=torch.float32, device="cuda")
    ref = prob.afd_apply(v).double().cpu().numpy()
    for _ in range(2):
        w = afd_apply_noalloc(d, n, lam, v)
        got = w.double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < FP32_TOL
    prob.close()


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    from paper_2307_14437_gb300 import GofdError
    from paper_2307_14437_gb300.gofd import afd_apply_noalloc
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(GofdError) as e:
        afd_apply_noalloc(2, 1025, x, x, torch.zeros(4, dtype=torch.float32, device="cuda"))
    assert e.value.code == "GOFD_E_ARG"
