"""The allocation-free force entry point against the allocating one.

ljsel_compute_forces_noalloc exists for callers that cannot allocate device
memory: code running while a stream is captured into a CUDA graph (an
allocation cannot be captured), code inside a framework whose allocator owns
all device memory, or latency-critical loops that must not enter the
allocator.  It keeps its intermediate arrays in one static device array of
the library.  This test calls it through the C ABI twice in a row, on two
different systems (the second smaller than the first and with two particle
types, so stale contents of the shared array from the first call would
show), and compares each result with ljsel_create + ljsel_compute on the
same input, within the FP32 force tolerance used by the other GPU tests.
"""
import numpy as np
import pytest

from paper_2505_03438_gb300 import scenarios

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5
SUM_TOL = 2e-6


def test_noalloc_matches_allocating_path():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_03438_gb300 as lj

    cases = [scenarios.fcc_liquid(8, seed=81, jitter=0.15), scenarios.binary_mixture(seed=82, nside=10)]
    for sc in cases:
        n = len(sc["x"])
        p = lj.make_params(sc["box"], sc["eps"], sc["sigma"], sc["rcut"], sc["mass"], sc["skin"], sc["dt"])
        x = torch.tensor(sc["x"], device="cuda")
        t = torch.tensor(sc["types"], dtype=torch.int32, device="cuda")
        F = torch.full_like(x, float("nan"))
        e, w = lj.ljsel_compute_forces_noalloc(p, n, x, F, t)
        torch.cuda.synchronize()
        Fn = F.cpu().numpy()
        assert np.isfinite(Fn).all()
        ref = lj.System(sc)
        ref.set_config(method="LC", newton3=False, csf=1.0)
        Fr, er, wr = ref.compute()
        ref.close()
        rel = np.linalg.norm(Fn - Fr) / np.linalg.norm(Fr)
        assert rel <= FORCE_TOL, rel
        assert abs(e - er) <= SUM_TOL * abs(er), (e, er)
        assert abs(w - wr) <= SUM_TOL * abs(wr), (w, wr)
