"""The parity suites on the bounds-checked build (libljsel_checked.so,
compiled with -DLJSEL_CHECK).

In that build every kernel that reads a list, cell or window index checks
it against the array it indexes; an index outside records the site and is
replaced by a safe one, and the next synchronizing call returns
LJSEL_ERR_STATE.  Running the FP32/FP64 parity cases of every method, the
smallest boxes, the rows built to their exact capacity, the batched
replicas, the walls and the forces of the stepping kernels on it proves
that no check fires on those inputs (a firing check fails the child run
with LJSEL_ERR_STATE) and that the checked kernels still match the oracle.  The child process loads only the checked library
(LJSEL_LIBRARY=checked).
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suites_on_the_checked_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    env = dict(os.environ, LJSEL_LIBRARY="checked")
    sel = ("test_pairs_forces_fp32 or test_pairs_forces_fp64 or smallest_boxes or rows_ending or "
           "test_batch_pairs_forces_step0 or test_batch_edge_replicas or test_pairs_and_forces_with_walls or "
           "test_stepping_forces_fp32")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", "-k", sel,
           os.path.join(ROOT, "tests", "test_gpu_parity.py"), os.path.join(ROOT, "tests", "test_gpu_batch.py"),
           os.path.join(ROOT, "tests", "test_gpu_walls.py"), os.path.join(ROOT, "tests", "test_gpu_step_forces.py"),
           os.path.join(ROOT, "tests", "test_gpu_checked_probe.py")]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout.splitlines()[-1]
