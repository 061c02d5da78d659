"""The largest system the list format allows: 131,072,000 particles (fcc
320^3 x 4; list entries name a particle with 27 bits, so n < 2^27).

Checked against the oracle on a sample: 256 seeded particles away from the
box faces, each with every particle within 4 sigma (brute force on that
subset, no periodic images needed), then 10 steps of the fused force and
update with the energy conserved.  About 60 GB of device memory.
"""
import numpy as np
import pytest

import oracle
import paper_2505_03438_gb300 as lj
from paper_2505_03438_gb300 import scenarios

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_largest_system_sampled_against_the_oracle():
    ncell, rho = 320, 0.8442
    x, box = scenarios.fcc_lattice(ncell, rho)
    n = len(x)
    assert n == 131_072_000 and n < (1 << 27)
    rng = np.random.default_rng(71)
    x += rng.uniform(-0.05, 0.05, x.shape)
    x = np.mod(x, box[0])
    v = rng.normal(0.0, 0.85, x.shape)
    v -= v.mean(0)
    s = lj.System(x=x, v=v, types=None, box=box, skin=0.3)
    F, e, w = s.compute()
    # sample: interior particles; the generator lays particle (cell ix, iy, iz,
    # basis b) at index ((ix n + iy) n + iz) 4 + b, so a particle's
    # neighbourhood is the particles of the lattice cells within 3 cells
    L = box[0]
    idx = rng.choice(n, 4096, replace=False)
    idx = idx[np.all((x[idx] > 8.0) & (x[idx] < L - 8.0), axis=1)][:256]
    p = oracle.make_params(np.full(3, 1e6), 1.0, 1.0, 2.5, True)
    off = np.arange(-3, 4)
    worst = 0.0
    for i in idx:
        ix, iy, iz = np.unravel_index(i // 4, (ncell, ncell, ncell))
        cells = ((ix + off)[:, None, None] * ncell + (iy + off)[None, :, None]) * ncell + (iz + off)[None, None, :]
        cand = (cells.reshape(-1, 1) * 4 + np.arange(4)).reshape(-1)
        near = cand[np.all(np.abs(x[cand] - x[i]) < 4.0, axis=1)]
        sub = np.asarray(x[near], np.float32).astype(np.float64) + 1000.0  # the working positions, no images
        ref = oracle.forces_brute(sub, None, p)["F"]
        k = int(np.nonzero(near == i)[0][0])
        worst = max(worst, np.linalg.norm(F[i] - ref[k]) / max(np.linalg.norm(ref[k]), 1.0))
    assert len(idx) >= 200 and worst < 1e-4, worst
    e0 = sum(s.energy()[:2])
    s.step(10)
    e1 = sum(s.energy()[:2])
    assert abs(e1 - e0) < 1e-4 * abs(e0), (e0, e1)
    c = s.counters()
    assert c["steps"] == 10
