"""Seeded synthetic inputs for the mechanical-interaction iteration.

This module only draws initial agent populations and names each workload's
parameters; it holds none of the method's arithmetic (no grid, force,
displacement or division).  Both the CUDA path (tests, bench) and the oracle
(tests) take their inputs from here.  The paper's own benchmark simulations
(Table 1) are not available, so these shapes stand in for them:

  uniform  -- 8,192 agents uniform in [0,200]^3 um, diameters U[8,12] um
  lattice  -- cell proliferation: 47^3 cubic lattice, spacing 20 um, d = 10 um
  blobs    -- 10M agents in 8 Gaussian blobs (sigma 150 um) in [0,4000]^3 um
  ensemble -- 512 independent simulations, 10^U[3,5] agents each, 0.25 volume
              fraction cubes, d = 10 um, per-simulation dt U[0.005, 0.02]
  core_shell -- 150M agents: 90% on a static FCC core (0.6 volume fraction),
              10% random walkers in a surrounding shell, d = 10 um
  cell_sorting -- two cell types mixed at random in a ball at 0.5 volume
              fraction, diameters U[9,11] um; same-type pairs adhere more
              strongly than mixed pairs (the differential-adhesion model class
              of the paper's cell-sorting comparison, whose own parameters are
              not published with it)
"""
import math
from dataclasses import dataclass, field

import numpy as np

GROW = 1
WALK = 2
DIE = 4
TYPE_SHIFT = 4


@dataclass
class Workload:
    name: str
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    diam: np.ndarray
    params: dict
    steps: int
    beh: np.ndarray = None
    sim_off: np.ndarray = None
    dt_sim: np.ndarray = None
    notes: dict = field(default_factory=dict)

    @property
    def n(self):
        return len(self.x)

    @property
    def n_sims(self):
        return 1 if self.sim_off is None else len(self.sim_off) - 1


def _f32_exact(a):
    """Round to float32 and widen again: FP32-attribute workloads store the
    diameter in float32, so both sides see the same representable value."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def uniform(n=8192, seed=1, edge=200.0, dmin=8.0, dmax_=12.0):
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.0, edge, size=(3, n))
    d = rng.uniform(dmin, dmax_, size=n)
    params = dict(R=dmax_, L=dmax_, dt=0.01, dmax=3.0, k=2.0, gamma=1.0, adherence=0.0,
                  precision="fp64", seed=seed)
    return Workload("uniform-%d" % n, p[0].copy(), p[1].copy(), p[2].copy(), d, params, steps=10)


def lattice(m=47, spacing=20.0, diam=10.0, seed=2, growth=300.0, divide_diam=20.0, steps=20):
    ax = np.arange(m, dtype=np.float64) * spacing
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    n = m ** 3
    d = np.full(n, diam)
    params = dict(R=divide_diam, L=divide_diam, dt=0.01, dmax=3.0, k=2.0, gamma=1.0, adherence=0.0,
                  precision="fp64", growth=growth,
                  divide_volume=(math.pi / 6.0) * divide_diam ** 3,
                  ratio_lo=0.9, ratio_hi=1.1, seed=seed)
    beh = np.full(n, GROW, np.uint8)
    return Workload("lattice-%d^3" % m, x.ravel().copy(), y.ravel().copy(), z.ravel().copy(), d,
                    params, steps=steps, beh=beh)


def blobs(n=10_000_000, seed=3, n_blobs=8, sigma=150.0, domain=4000.0, centre_lo=600.0,
          centre_hi=3400.0, dmin=9.0, dmax_=11.0, precision="fp32", sort_every=10, steps=100):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(centre_lo, centre_hi, size=(n_blobs, 3))
    counts = np.full(n_blobs, n // n_blobs)
    counts[: n % n_blobs] += 1
    p = np.empty((3, n))
    o = 0
    for b in range(n_blobs):
        c = counts[b]
        p[:, o:o + c] = rng.normal(0.0, sigma, size=(3, c)) + centres[b][:, None]
        o += c
    np.clip(p, 0.0, domain, out=p)
    d = rng.uniform(dmin, dmax_, size=n)
    if precision == "fp32":
        d = _f32_exact(d)
    params = dict(R=dmax_, L=dmax_, dt=0.01, dmax=3.0, k=2.0, gamma=1.0, adherence=0.0,
                  precision=precision, sort_every=sort_every, seed=seed)
    w = Workload("blobs-%d" % n, p[0].copy(), p[1].copy(), p[2].copy(), d, params, steps=steps)
    w.notes["centres"] = centres
    return w


def ensemble(n_sims=512, seed=4, log_lo=3.0, log_hi=5.0, volume_fraction=0.25, diam=10.0,
             dt_lo=0.005, dt_hi=0.02, steps=50, precision="fp32", max_agents=None):
    rng = np.random.default_rng(seed)
    ns = np.rint(10.0 ** rng.uniform(log_lo, log_hi, size=n_sims)).astype(np.int64)
    if max_agents is not None:
        ns = np.minimum(ns, max_agents)
    dts = rng.uniform(dt_lo, dt_hi, size=n_sims)
    off = np.zeros(n_sims + 1, np.int64)
    off[1:] = np.cumsum(ns)
    n = int(off[-1])
    p = np.empty((3, n))
    agent_volume = (math.pi / 6.0) * diam ** 3
    edges = np.empty(n_sims)
    for s in range(n_sims):
        edge = (ns[s] * agent_volume / volume_fraction) ** (1.0 / 3.0)
        edges[s] = edge
        p[:, off[s]:off[s + 1]] = rng.uniform(0.0, edge, size=(3, ns[s]))
    d = np.full(n, diam)
    params = dict(R=diam, L=diam, dt=0.01, dmax=3.0, k=2.0, gamma=1.0, adherence=0.0,
                  precision=precision, seed=seed)
    w = Workload("ensemble-%d" % n_sims, p[0].copy(), p[1].copy(), p[2].copy(), d, params,
                 steps=steps, sim_off=off, dt_sim=dts)
    w.notes["edges"] = edges
    return w


def _fcc_ball(radius, a, centre):
    """FCC lattice points (lattice constant a) inside a ball, generated per slab."""
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]]) * a
    K = int(math.ceil(radius / a)) + 1
    idx = np.arange(-K, K + 1, dtype=np.float64) * a
    out = []
    gy, gz = np.meshgrid(idx, idx, indexing="ij")
    gy = gy.ravel()
    gz = gz.ravel()
    r2 = radius * radius
    for xi in idx:
        for b in basis:
            px = xi + b[0]
            py = gy + b[1]
            pz = gz + b[2]
            keep = (px * px + py * py + pz * pz) < r2
            if keep.any():
                m = int(keep.sum())
                blk = np.empty((3, m))
                blk[0] = px + centre[0]
                blk[1] = py[keep] + centre[1]
                blk[2] = pz[keep] + centre[2]
                out.append(blk)
    return np.concatenate(out, axis=1)


def core_shell(n=150_000_000, seed=5, core_frac=0.9, lattice_const=15.17, diam=10.0,
               shell_volume_fraction=0.3, walk=0.5, steps=20, precision="fp32"):
    rng = np.random.default_rng(seed)
    n_core_target = core_frac * n
    density = 4.0 / lattice_const ** 3
    r_core = (3.0 * n_core_target / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    r_out_guess = r_core * 1.2 + 4 * lattice_const
    centre = np.array([r_out_guess, r_out_guess, r_out_guess])
    core = _fcc_ball(r_core, lattice_const, centre)
    n_core = core.shape[1]
    n_shell = max(n - n_core, 0)
    agent_volume = (math.pi / 6.0) * diam ** 3
    r_in = r_core + lattice_const
    shell_vol = n_shell * agent_volume / shell_volume_fraction
    r_out = (r_in ** 3 + 3.0 * shell_vol / (4.0 * math.pi)) ** (1.0 / 3.0)
    u = rng.uniform(0.0, 1.0, size=n_shell)
    rad = (r_in ** 3 + u * (r_out ** 3 - r_in ** 3)) ** (1.0 / 3.0)
    v = rng.normal(size=(3, n_shell))
    v /= np.linalg.norm(v, axis=0)
    shell = v * rad + centre[:, None]
    p = np.concatenate([core, shell], axis=1)
    beh = np.zeros(p.shape[1], np.uint8)
    beh[n_core:] = WALK
    d = np.full(p.shape[1], diam)
    params = dict(R=diam, L=diam, dt=0.01, dmax=3.0, k=2.0, gamma=1.0, adherence=0.0,
                  precision=precision, detect_static=1, walk_step=walk, seed=seed)
    w = Workload("core_shell-%d" % p.shape[1], p[0].copy(), p[1].copy(), p[2].copy(), d, params,
                 steps=steps, beh=beh)
    w.notes.update(n_core=n_core, n_shell=n_shell, r_core=r_core, r_out=r_out)
    return w


# force constants of the two-type cell-sorting workload: k equal for all
# pairs, the adhesion term gamma three times stronger between equal types
SORTING_K = [[2.0, 2.0], [2.0, 2.0]]
SORTING_GAMMA = [[1.5, 0.5], [0.5, 1.5]]


def cell_sorting(n=10_000_000, seed=6, volume_fraction=0.5, dmin=9.0, dmax_=11.0, steps=20, precision="fp32"):
    rng = np.random.default_rng(seed)
    mean_vol = (math.pi / 6.0) * ((dmin + dmax_) / 2.0) ** 3
    radius = (3.0 * n * mean_vol / volume_fraction / (4.0 * math.pi)) ** (1.0 / 3.0)
    v = rng.normal(size=(3, n))
    v /= np.linalg.norm(v, axis=0)
    p = v * (radius * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)) + (radius + 20.0)
    d = _f32_exact(rng.uniform(dmin, dmax_, n))
    types = rng.integers(0, 2, n).astype(np.uint8)
    beh = (types << TYPE_SHIFT).astype(np.uint8)
    R = float(dmax_)
    params = dict(R=R, L=R, dt=0.01, dmax=3.0, k=2.0, gamma=1.0, adherence=0.0, precision=precision,
                  type_k=SORTING_K, type_gamma=SORTING_GAMMA, seed=seed)
    return Workload("cell_sorting-%d" % n, p[0].copy(), p[1].copy(), p[2].copy(), d, params, steps=steps, beh=beh)
