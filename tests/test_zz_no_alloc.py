"""The allocation-free A_FD entry point, gofd_afd_apply_noalloc.

Some callers cannot allocate device memory at the moment they need the
product: plug-ins inside a framework that owns all device memory through its
own allocator, and real-time loops that must not risk an allocation failure or
its latency.  This entry point keeps its scratch in a fixed device array
inside the library instead.  Two calls in a row must each match
  * the FP64 oracle's zero-padded circulant convolution (Section 2.2, (AU-1)),
    with the symbol built by the oracle from the oracle's coefficients, and
  * the existing handle-based entry point gofd_afd_apply on the same symbol,
within the FP32 tolerance of the parity tests, in 1D, in 2D (up to n = 1024,
the largest grid the scratch holds) and in 3D (up to n = 65, the largest
there).  This file runs
last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import meshgen as mg
from oracle import gofd as o

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP32_TOL = 1e-5

# (d, n, alpha, Filon M, mesh for the handle-based comparison)
CASES = {
    "interval33": (1, 33, 0.8, 2 ** 12),
    "disk65": (2, 65, 1.2, 2 ** 10),
    "disk1024": (2, 1024, 1.0, 2 ** 13),
    "ball9": (3, 9, 1.5, 2 ** 8),
    "ball65": (3, 65, 1.5, 2 ** 10),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2307_14437_gb300 import build_native
    build_native.build()


def _mesh(d):
    if d == 1:
        return mg.interval_mesh(16, seed=mg.seed_for(0, 3))
    if d == 2:
        return mg.disk_ring_mesh(rings=12, seed=mg.seed_for(1, 3))
    return mg.ball_shell_mesh(shells=3, seed=mg.seed_for(3, 2))


def _circulant(n):
    # the entry point's rule: the oracle's smallest power of two >= 2n-2,
    # raised to at least 32
    return max(32, o.circulant_size(n))


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_matches_oracle_and_handle_path_twice(case):
    from paper_2307_14437_gb300 import Problem
    from paper_2307_14437_gb300.gofd import afd_apply_noalloc
    d, n, alpha, M = CASES[case]
    P = _circulant(n)
    v = mg.random_vector(n ** d, 31)
    vd = torch.tensor(v, dtype=torch.float32, device="cuda")
    # 1. against the FP64 oracle: symbol from the oracle's own T
    T = o.coefficients(d, alpha / 2, n, M=M)
    lam_o = o.symbol(T, P)
    want = o.afd_apply_fft(lam_o, v.reshape((n,) * d), P).ravel()
    lam_od = torch.tensor(lam_o.ravel() / float(P) ** d, dtype=torch.float32, device="cuda")
    for _ in range(2):
        got = afd_apply_noalloc(d, n, lam_od, vd).double().cpu().numpy()
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < FP32_TOL
    # 2. against gofd_afd_apply on a handle with the same grid and symbol
    verts, simp = _mesh(d)
    lo, hi, h = mg.grid_box(d, n)
    prob = Problem(verts, simp, alpha, h, lo, hi, filon_M=M)
    assert prob.P == P
    ref = prob.afd_apply(vd).double().cpu().numpy()
    lam = torch.tensor(prob.symbol().ravel() / float(P) ** d, dtype=torch.float32, device="cuda")
    for _ in range(2):
        got = afd_apply_noalloc(d, n, lam, vd).double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < FP32_TOL
    prob.close()


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    from paper_2307_14437_gb300 import GofdError
    from paper_2307_14437_gb300.gofd import afd_apply_noalloc
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    # 2D n = 1025 and 3D n = 66 need more spectrum than the scratch holds;
    # 1D n = 1026 needs a circulant longer than 2048
    for d, n in ((2, 1025), (3, 66), (1, 1026)):
        with pytest.raises(GofdError) as e:
            afd_apply_noalloc(d, n, x, x, torch.zeros(4, dtype=torch.float32, device="cuda"))
        assert e.value.code == "GOFD_E_ARG"
