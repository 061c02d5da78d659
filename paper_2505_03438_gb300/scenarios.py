"""Seeded synthetic inputs shared by the GPU library's callers and the oracle.

This module holds no arithmetic of the method (no forces, no cells, no
integration): it only places particles and draws velocities, with numpy's
PCG64 generator from a stated seed, so that the GPU path and the CPU oracle
are fed the very same arrays.  The workloads stand in for the paper's
md-flexible inputs, which are not available (Sec. 6, Appendix B); their
shapes follow the homogeneous liquid, the inhomogeneous sphere-in-vapour,
the batched-replica and the binary-mixture cases of the hot path.

Every scenario is a plain dict:
  x (N,3) f64, v (N,3) f64, types (N,) i32, box (3,) f64,
  eps/sigma/rcut (nt,nt) f64, mass (nt,) f64, dt, skin, rebuild, shift, name.
"""
from __future__ import annotations

import math
import os

import numpy as np

FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


def fcc_lattice(ncell: int, density: float):
    """4*ncell^3 sites of a face-centred cubic lattice at the given number density."""
    a = (4.0 / density) ** (1.0 / 3.0)
    g = np.stack(np.meshgrid(np.arange(ncell), np.arange(ncell), np.arange(ncell), indexing="ij"), -1)
    g = g.reshape(-1, 1, 3).astype(np.float64)
    x = ((g + FCC_BASIS[None]) * a).reshape(-1, 3)
    box = np.full(3, ncell * a)
    return x, box


def maxwell_boltzmann(n: int, temperature: float, mass, rng) -> np.ndarray:
    """Gaussian velocities, zero total momentum, rescaled so that
    sum(m v^2) / (3N - 3) equals the temperature exactly (reduced units)."""
    mass = np.broadcast_to(np.asarray(mass, np.float64), (n,))
    v = rng.normal(0.0, 1.0, (n, 3)) * np.sqrt(temperature / mass)[:, None]
    p = (mass[:, None] * v).sum(0) / mass.sum()
    v -= p[None, :]
    if n > 1 and temperature > 0:
        t_now = float((mass[:, None] * v * v).sum()) / (3 * n - 3)
        v *= math.sqrt(temperature / t_now)
    return v


def _single_type(box, rc, shift=True):
    return dict(box=np.asarray(box, np.float64), eps=np.ones((1, 1)), sigma=np.ones((1, 1)),
                rcut=np.full((1, 1), rc), mass=np.ones(1), shift=shift)


def fcc_liquid(ncell: int, density=0.8442, temperature=0.72, seed=1, rc=2.5, skin=0.3,
               dt=0.005, rebuild=10, jitter=0.0, name="fcc"):
    """Single-species LJ on an fcc lattice with Maxwell-Boltzmann velocities."""
    rng = np.random.default_rng(seed)
    x, box = fcc_lattice(ncell, density)
    n = x.shape[0]
    if jitter > 0:
        x = x + rng.uniform(-jitter, jitter, x.shape)
        x = np.mod(x, box[None, :])
    v = maxwell_boltzmann(n, temperature, 1.0, rng)
    sc = dict(name=name, x=x, v=v, types=np.zeros(n, np.int32), dt=dt, skin=skin, rebuild=rebuild,
              temperature=temperature, density=density, seed=seed)
    sc.update(_single_type(box, rc))
    return sc


def small_fcc(seed=1):
    """Plain-method FP64 case: N = 4000 (10^3 fcc cells x 4), rho 0.8442, T 0.72,
    r_c 2.5 shifted, cells of side >= r_c (no skin), dt 0.005, 100 NVE steps."""
    sc = fcc_liquid(10, seed=seed, skin=0.0, rebuild=1, name="fcc_4000_fp64")
    sc["nsteps"] = 100
    return sc


def liquid_1m(seed=2):
    """Homogeneous liquid: N = 1,048,576 (64^3 fcc cells x 4), rho 0.8442,
    T 0.72, r_c 2.5, skin 0.3, rebuild every 10 steps, 1000 steps."""
    sc = fcc_liquid(64, seed=seed, name="lj_liquid_1m")
    sc["nsteps"] = 1000
    return sc


def jittered_cubic(n: int, density: float, temperature: float, rng, jitter=0.05):
    """First n sites (lexicographic) of a simple-cubic lattice with
    ceil(n^(1/3)) sites per side, each moved by U(-jitter, jitter)."""
    box_len = (n / density) ** (1.0 / 3.0)
    side = int(math.ceil(n ** (1.0 / 3.0) - 1e-12))
    h = box_len / side
    g = np.stack(np.meshgrid(np.arange(side), np.arange(side), np.arange(side), indexing="ij"), -1).reshape(-1, 3)
    x = (g[:n].astype(np.float64) + 0.5) * h
    x = np.mod(x + rng.uniform(-jitter, jitter, x.shape), box_len)
    v = maxwell_boltzmann(n, temperature, 1.0, rng)
    return x, v, np.full(3, box_len)


def replica_batch(nrep=512, seed=4, nmin=256, nmax=8192, rc=2.5, skin=0.3, dt=0.005, rebuild=10):
    """Batched replicas: N log-uniform in [nmin, nmax], density U[0.3, 0.9],
    T U[0.7, 2.0], each a jittered cubic lattice (jitter 0.05)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(nrep):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        rho = float(rng.uniform(0.3, 0.9))
        temp = float(rng.uniform(0.7, 2.0))
        x, v, box = jittered_cubic(n, rho, temp, rng)
        sc = dict(name="replica_%d" % r, x=x, v=v, types=np.zeros(n, np.int32), dt=dt, skin=skin,
                  rebuild=rebuild, temperature=temp, density=rho)
        sc.update(_single_type(box, rc))
        out.append(sc)
    return out


def binary_mixture(seed=5, nside=32, density=1.2, temperature=1.0, frac_a=0.8, skin=0.3, dt=0.005,
                   rebuild=10):
    """Binary LJ mixture: N = nside^3 on a simple-cubic lattice at density 1.2,
    A:B = 80:20 (N_A = round(0.8 N), types by seeded permutation),
    eps_AA 1, sig_AA 1, eps_AB 1.5, sig_AB 0.8, eps_BB 0.5, sig_BB 0.88,
    cutoff 2.5 sigma_ab per type pair, unit masses."""
    rng = np.random.default_rng(seed)
    n = nside ** 3
    box_len = (n / density) ** (1.0 / 3.0)
    h = box_len / nside
    g = np.stack(np.meshgrid(np.arange(nside), np.arange(nside), np.arange(nside), indexing="ij"), -1)
    x = (g.reshape(-1, 3).astype(np.float64) + 0.5) * h
    na = int(round(frac_a * n))
    types = np.ones(n, np.int32)
    types[rng.permutation(n)[:na]] = 0
    v = maxwell_boltzmann(n, temperature, 1.0, rng)
    eps = np.array([[1.0, 1.5], [1.5, 0.5]])
    sigma = np.array([[1.0, 0.8], [0.8, 0.88]])
    return dict(name="binary_32768", x=x, v=v, types=types, box=np.full(3, box_len), eps=eps, sigma=sigma,
                rcut=2.5 * sigma, mass=np.ones(2), shift=True, dt=dt, skin=skin, rebuild=rebuild,
                temperature=temperature, density=density, seed=seed)


def random_gas(n: int, box_len: float, seed: int, min_dist=0.0, rc=2.5, skin=0.3, temperature=1.0):
    """n uniform random particles in a cubic box (tiny parity cases); with
    min_dist > 0, candidates closer than min_dist to an accepted one are
    redrawn (plain O(n^2) rejection, small n only)."""
    rng = np.random.default_rng(seed)
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 1000 * n + 1000:
            raise RuntimeError("random_gas: too dense for rejection placement")
        c = rng.uniform(0.0, box_len, 3)
        if min_dist > 0 and pts:
            d = np.abs(np.asarray(pts) - c)
            d = np.minimum(d, box_len - d)
            if (d * d).sum(1).min() < min_dist * min_dist:
                continue
        pts.append(c)
    x = np.asarray(pts, np.float64).reshape(-1, 3)
    v = maxwell_boltzmann(n, temperature, 1.0, rng)
    sc = dict(name="gas_%d" % n, x=x, v=v, types=np.zeros(n, np.int32), dt=0.005, skin=skin, rebuild=10,
              temperature=temperature)
    sc.update(_single_type(np.full(3, box_len), rc))
    return sc


def perturbed_pair_params(eps, sigma, seed=5, frac=0.05):
    """Target parameters of the force-matching workload: every independent
    eps_ab, sigma_ab (a <= b) times (1 + u), u ~ U(-frac, frac) from a seeded
    PCG64 stream, kept symmetric.  The target cutoffs are 2.5 sigma*_ab."""
    rng = np.random.default_rng(seed + 1000)
    eps = np.array(eps, np.float64, copy=True)
    sigma = np.array(sigma, np.float64, copy=True)
    nt = eps.shape[0]
    for a in range(nt):
        for b in range(a, nt):
            ue, us = rng.uniform(-frac, frac, 2)
            eps[a, b] = eps[b, a] = eps[a, b] * (1.0 + ue)
            sigma[a, b] = sigma[b, a] = sigma[a, b] * (1.0 + us)
    return eps, sigma, 2.5 * sigma


def jittered_mixture(nside=7, seed=5, jitter=0.1):
    """The binary mixture on a small lattice with uniform +-jitter per
    coordinate, so that no force vanishes by symmetry (gradient checks)."""
    sc = binary_mixture(seed=seed, nside=nside)
    rng = np.random.default_rng(seed + 2000)
    sc["x"] = sc["x"] + rng.uniform(-jitter, jitter, sc["x"].shape)
    sc["name"] = "binary_%d_jittered" % len(sc["x"])
    return sc


def _rsa(center, radius, box_len, target, dmin, rng, existing=None, inside=True, min_batch=40000):
    """Random sequential addition in batches: uniform candidates, accepted
    when no accepted point lies closer than dmin (minimum image); of two
    candidates of one batch closer than dmin the later one is dropped.
    inside=True draws in the ball (center, radius); inside=False draws in the
    periodic box outside it.  Batches hold at least min_batch candidates."""
    from scipy.spatial import cKDTree
    acc = np.zeros((0, 3)) if existing is None else np.asarray(existing, np.float64)
    n0 = len(acc)
    # accepted points live in a large tree rebuilt now and then plus a small
    # tree of the points accepted since
    big = cKDTree(acc, boxsize=box_len) if len(acc) else None
    nbig = len(acc)
    tries = 0
    rate = 1.0  # accepted fraction of the last batch
    while len(acc) - n0 < target:
        tries += 1
        if tries > 100000:
            raise RuntimeError("RSA placement stalled")
        left = target - (len(acc) - n0)
        batch = int(min(max(min_batch, 1.5 * left / max(rate, 1e-3)), 400000))
        if inside:
            u = rng.normal(size=(batch, 3))
            u /= np.linalg.norm(u, axis=1, keepdims=True)
            c = center + u * (radius * rng.uniform(0.0, 1.0, (batch, 1)) ** (1.0 / 3.0))
        else:
            c = rng.uniform(0.0, box_len, (batch, 3))
            c = c[np.linalg.norm(c - center, axis=1) >= radius]
        c = np.mod(c, box_len)
        if big is not None:
            d, _ = big.query(c, k=1, distance_upper_bound=dmin)
            c = c[d >= dmin]
        if len(acc) > nbig and len(c):
            d, _ = cKDTree(acc[nbig:], boxsize=box_len).query(c, k=1, distance_upper_bound=dmin)
            c = c[d >= dmin]
        if len(c) == 0:
            continue
        # conflicts among the candidates: keep each unless an earlier kept one is too close
        pairs = cKDTree(c, boxsize=box_len).query_pairs(dmin, output_type="ndarray")
        keep = np.ones(len(c), bool)
        if len(pairs):
            keep[pairs.max(axis=1)] = False
        c = c[keep][: target - (len(acc) - n0)]
        rate = max(len(c), 1) / batch
        acc = np.concatenate([acc, c])
        if len(acc) - nbig > 0.25 * nbig + 5000:
            big = cKDTree(acc, boxsize=box_len)
            nbig = len(acc)
    return acc


def heated_sphere(seed=3, box_len=200.0, radius=40.0, rho_liquid=0.8, t_liquid=3.0, rho_vapour=0.01,
                  t_vapour=1.2, dmin=0.9, rc=2.5, skin=0.3, dt=0.005, rebuild=10):
    """Inhomogeneous workload (periodic analogue of a heating sphere): a
    liquid ball of the given radius and density at the box centre, drawn at
    the heated temperature, in a vapour filling the rest of the periodic box;
    non-overlapping random placement (RSA, minimum spacing dmin), the ball
    first.  Velocities Maxwell-Boltzmann per phase, zero momentum per phase,
    each rescaled to its temperature exactly."""
    key = "sphere_%d_%g_%g_%g_%g_%g_%g_%g" % (seed, box_len, radius, rho_liquid, t_liquid, rho_vapour, t_vapour, dmin)
    cache = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "scenarios", key + ".npz")
    if os.path.exists(cache):
        z = np.load(cache)
        x, v, n_l = z["x"], z["v"], int(z["n_l"])
    else:
        x, v, n_l = _heated_sphere_draw(seed, box_len, radius, rho_liquid, t_liquid, rho_vapour, t_vapour, dmin)
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + ".tmp.%d.npz" % os.getpid()
        np.savez(tmp, x=x, v=v, n_l=n_l)
        os.replace(tmp, cache)
    sc = dict(name="heated_sphere_%d" % len(x), x=x, v=v, types=np.zeros(len(x), np.int32), dt=dt, skin=skin,
              rebuild=rebuild, n_liquid=n_l, temperature=t_liquid, seed=seed)
    sc.update(_single_type(np.full(3, box_len), rc))
    return sc


def _heated_sphere_draw(seed, box_len, radius, rho_liquid, t_liquid, rho_vapour, t_vapour, dmin):
    rng = np.random.default_rng(seed)
    center = np.full(3, 0.5 * box_len)
    vol_ball = 4.0 / 3.0 * math.pi * radius ** 3
    n_l = int(round(rho_liquid * vol_ball))
    n_v = int(round(rho_vapour * (box_len ** 3 - vol_ball)))
    xl = _rsa(center, radius, box_len, n_l, dmin, rng, inside=True)
    xa = _rsa(center, radius, box_len, n_v, dmin, rng, existing=xl, inside=False)
    vl = maxwell_boltzmann(n_l, t_liquid, 1.0, rng)
    vv = maxwell_boltzmann(n_v, t_vapour, 1.0, rng)
    return xa, np.concatenate([vl, vv]), n_l


def _with_vapour(xd, box_len, rho_vapour, dmin, rng):
    """Dense points xd plus a vapour of the given density placed around them
    by random sequential addition (no vapour point closer than dmin to any)."""
    n_v = int(round(rho_vapour * box_len ** 3))
    if n_v == 0:
        return np.asarray(xd, np.float64)
    return _rsa(np.full(3, 0.5 * box_len), 0.0, box_len, n_v, dmin, rng, existing=xd, inside=False)


def walled_heating_sphere(n=5497, box_len=200.0, density=0.8442, temperature=0.1, seed=6, rc=3.0, skin=0.5,
                          dt=1e-4, rebuild=10):
    """The heating sphere of Sec. 6 as a synthetic input: a ball of n LJ
    particles, the n sites of an fcc lattice at the given density nearest
    the centre of a cubic box with reflective walls (ties in distance broken
    by lattice order), Maxwell-Boltzmann velocities at the starting
    temperature (zero total momentum, rescaled to it exactly).  The paper's
    run: 5497 molecules, a 200^3 box with reflective boundaries, cutoff 3,
    skin 0.5, rebuild interval 10, dt 1e-4, starting at T 0.1 and heated by
    velocity scaling every 100 iterations by at most 0.1 towards T 100."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil((2.0 * n / 4.0) ** (1.0 / 3.0))) + 2
    lat, lbox = fcc_lattice(m, density)
    c = lat - 0.5 * lbox
    order = np.argsort((c * c).sum(1), kind="stable")[:n]
    x = c[order] + 0.5 * box_len
    v = maxwell_boltzmann(n, temperature, 1.0, rng)
    sc = dict(name="walled_sphere_%d" % n, x=x, v=v, types=np.zeros(n, np.int32), dt=dt, skin=skin,
              rebuild=rebuild, temperature=temperature, seed=seed, walls=(1, 1, 1))
    sc.update(_single_type(np.full(3, box_len), rc))
    return sc


def training_scenarios(seed=7, dmin=0.9, rc=2.5, dt=0.005, rebuild=10):
    """Synthetic scenarios for the data behind the Random Forest strategy, of
    the paper's kinds (Sec. 5.3: uniform gases, clustered particles, a dense
    cuboid in a gas, spheres in a large box, an almost empty box), scaled to
    r_c = 2.5 and to sizes of 10^3 to 4.4 x 10^5 particles, and spheres in
    large boxes with reflective walls at the paper's heating-run settings.  Placement keeps
    a minimum spacing dmin so that trial steps stay physical; skins cycle
    through 0.1 ... 0.5 as in the paper's data.  Yields scenario dicts."""
    rng = np.random.default_rng(seed)
    skins = [0.1, 0.2, 0.3, 0.4, 0.5]
    k = [0]

    def make(name, x, box_len, temperature):
        x = np.mod(np.asarray(x, np.float64), box_len)
        n = len(x)
        v = maxwell_boltzmann(n, temperature, 1.0, rng)
        skin = skins[k[0] % len(skins)]
        k[0] += 1
        sc = dict(name=name, x=x, v=v, types=np.zeros(n, np.int32), dt=dt, skin=skin, rebuild=rebuild,
                  temperature=temperature)
        sc.update(_single_type(np.full(3, box_len), rc))
        return sc

    # uniform gases (random sequential addition)
    for box_len in (30.0, 60.0):
        for rho in (0.005, 0.02, 0.05, 0.1, 0.2, 0.35):
            n = int(round(rho * box_len ** 3))
            x = _rsa(np.full(3, 0.5 * box_len), 0.0, box_len, n, dmin, rng, inside=False)
            yield make("gas_L%g_rho%g" % (box_len, rho), x, box_len, 1.2)
    # liquids and dense solids (jittered fcc)
    for nside in (10, 20, 32, 48):
        for rho in (0.6, 0.75, 0.9, 1.0):
            x, box = fcc_lattice(nside, rho)
            x = x + rng.uniform(-0.05, 0.05, x.shape)
            yield make("fcc_n%d_rho%g" % (nside, rho), x, box[0], 0.8)
    # clustered: small dense balls (radius 4, density 0.6) centred on a
    # random subset of the sites of a cubic lattice of spacing 9 (balls one
    # unit apart, more than dmin: each is placed on its own)
    for nblob in (10, 20, 40, 80, 160):
        m = int(math.ceil(nblob ** (1.0 / 3.0))) + 1
        box_len = 9.0 * m
        sites = np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), -1).reshape(-1, 3)
        centres = (sites[rng.permutation(len(sites))[:nblob]] + 0.5) * 9.0
        target = int(round(0.6 * 4.0 / 3.0 * math.pi * 4.0 ** 3))
        pts = np.concatenate([_rsa(c, 4.0, box_len, target, dmin, rng, inside=True, min_batch=2000) for c in centres])
        yield make("blobs_%d" % nblob, _with_vapour(pts, box_len, 0.005, dmin, rng), box_len, 1.0)
    # a dense fcc slab of width w (density 0.8) in a gas of density 0.02
    for w in (5.0, 10.0, 20.0):
        x, box = fcc_lattice(24, 0.8)
        box_len = box[0]
        x = x[np.abs(x[:, 0] - 0.5 * box_len) < 0.5 * w]
        yield make("slab_w%g" % w, _with_vapour(x, box_len, 0.02, dmin, rng), box_len, 1.0)
    # fcc balls (density 0.8) in a dilute vapour
    for box_len, radius in ((60.0, 8.0), (60.0, 15.0), (100.0, 15.0), (100.0, 25.0), (150.0, 30.0)):
        ncell = int(math.ceil(2 * radius / (4.0 / 0.8) ** (1.0 / 3.0))) + 1
        x, box = fcc_lattice(ncell, 0.8)
        x = x - 0.5 * box[0] + 0.5 * box_len
        x = x[np.linalg.norm(x - 0.5 * box_len, axis=1) < radius]
        yield make("ball_L%g_r%g" % (box_len, radius), _with_vapour(x, box_len, 0.005, dmin, rng), box_len, 3.0)
    # an almost empty box
    x = _rsa(np.full(3, 20.0), 0.0, 40.0, 50, dmin, rng, inside=False)
    yield make("empty_L40", x, 40.0, 1.0)
    # spheres in a large box closed by reflective walls, as in the paper's
    # heating run (Sec. 6.1: cutoff 3, skin 0.5, dt 1e-4): condensed fcc balls
    # (density 0.8442) of 2,000 to 16,000 particles, and clouds of 5,000
    # particles spread over a larger radius (the later, evaporated stages)
    def walled(name, x, box_len, temperature):
        sc = make(name, x, box_len, temperature)
        sc.update(_single_type(np.full(3, box_len), 3.0))
        sc.update(dt=1e-4, skin=0.5, walls=(1, 1, 1))
        return sc

    for n_ball, box_len, temperature in ((2000, 100.0, 0.1), (4000, 200.0, 1.0), (8000, 150.0, 0.5),
                                         (16000, 250.0, 2.0)):
        m = int(math.ceil((2.0 * n_ball / 4.0) ** (1.0 / 3.0))) + 2
        lat, lbox = fcc_lattice(m, 0.8442)
        c = lat - 0.5 * lbox
        x = c[np.argsort((c * c).sum(1), kind="stable")[:n_ball]] + 0.5 * box_len
        yield walled("wball_N%d_L%g" % (n_ball, box_len), x, box_len, temperature)
    for radius, temperature in ((20.0, 20.0), (40.0, 40.0), (60.0, 60.0)):
        x = _rsa(np.full(3, 100.0), radius, 200.0, 5000, dmin, rng, inside=True, min_batch=2000)
        yield walled("wcloud_R%g" % radius, x, 200.0, temperature)
