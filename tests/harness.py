"""Shared helpers of the parity tests: run the oracle and the CUDA library on
the same seeded inputs and compare them."""
import math

import numpy as np

from oracle import oracle as O
from paper_2301_06984_gb300 import bdm
from paper_2301_06984_gb300 import workloads as W

ORACLE_KEYS = ("R", "L", "dt", "dmax", "k", "gamma", "adherence", "detect_static", "sort_every", "growth",
               "divide_volume", "ratio_lo", "ratio_hi", "walk_step", "seed")


def oracle_params(w, **over):
    p = {k: v for k, v in w.params.items() if k in ORACLE_KEYS}
    p.update({k: v for k, v in over.items() if k in ORACLE_KEYS})
    return O.make_params(**p)


def f32_diam(w):
    """Round a workload's diameters to float32 (what the FP32-force form stores)."""
    w.diam = np.asarray(w.diam, dtype=np.float32).astype(np.float64)
    return w


def oracle_state(w, cap=None, vol=None):
    return O.State(w.x, w.y, w.z, w.diam, vol=vol, beh=w.beh, sim_off=w.sim_off, dt_sim=w.dt_sim, cap=cap)


def gpu_sim(w, capacity=None, set_state=True, vol=None, **over):
    s = bdm.Simulation.from_workload(w, capacity=capacity, **over)
    if set_state:
        s.set_agents(w.x, w.y, w.z, w.diam, vol=vol, beh=w.beh, sim_off=w.sim_off)
    return s


def gpu_positions(s):
    a = s.get_agents()
    return np.stack([a["x"], a["y"], a["z"]]), a


def force_scale(pos, diam, off, nbr, k=2.0, gamma=1.0):
    """Per-agent sum over contacts of k*delta + gamma*sqrt(rbar*delta): the
    magnitude scale of the summed force (no cancellation), used to express the
    FP32 tolerance relative to the work that forms it."""
    n = pos.shape[1]
    cnt = np.diff(off)
    i = np.repeat(np.arange(n), cnt)
    j = nbr
    if len(j) == 0:
        return np.zeros(n)
    d = np.sqrt(((pos[:, i] - pos[:, j]) ** 2).sum(axis=0))
    ri, rj = diam[i] * 0.5, diam[j] * 0.5
    delta = np.maximum(ri + rj - d, 0.0)
    rbar = ri * rj / (ri + rj)
    term = k * delta + gamma * np.sqrt(rbar * delta)
    return np.bincount(i, weights=term, minlength=n)


def assert_fp32_forces(f_gpu, f_ref, scale, rel=2e-5, floor=1e-6, what="force"):
    err = np.sqrt(((f_gpu - f_ref) ** 2).sum(axis=0))
    bound = rel * scale + floor
    bad = np.nonzero(err > bound)[0]
    worst = float(np.max(err / bound)) if len(err) else 0.0
    assert len(bad) == 0, "%s: %d agents outside %g*scale+%g (worst ratio %.3g, first %s: err %g scale %g)" % (
        what, len(bad), rel, floor, worst, bad[:5], err[bad[0]], scale[bad[0]])
    return worst


def csr_equal(off_a, nb_a, off_b, nb_b):
    assert np.array_equal(np.asarray(off_a), np.asarray(off_b)), "CSR offsets differ"
    assert np.array_equal(np.asarray(nb_a), np.asarray(nb_b)), "CSR neighbour lists differ"


def brick_ranks_from_oracle(bxyz, nb):
    """Morton rank of each agent's 4x4x4 brick among the in-domain bricks of
    the grid, through the oracle's gap/offset DFS (Sec. 4.2)."""
    nr = [(int(v) + 3) // 4 for v in nb]
    offs = O.morton_offsets(nr)
    counters = np.array([c for c, _ in offs], dtype=np.int64)
    offsets = np.array([o for _, o in offs], dtype=np.int64)
    starts = counters + offsets  # first code of each run
    out = np.empty(len(bxyz), np.int64)
    cache = {}
    for a in range(len(bxyz)):
        key = (int(bxyz[a, 0]) >> 2, int(bxyz[a, 1]) >> 2, int(bxyz[a, 2]) >> 2)
        r = cache.get(key)
        if r is None:
            code = O.morton3(*key)
            e = int(np.searchsorted(starts, code, side="right")) - 1
            r = code - int(offsets[e])
            cache[key] = r
        out[a] = r
    return out


def small_blobs(n=200_000, seed=3):
    """Blob workload at the 10M-agent density: sigma scaled by (n / 1e7)^(1/3)."""
    scale = (n / 1.0e7) ** (1.0 / 3.0)
    return W.blobs(n=n, seed=seed, sigma=150.0 * scale, domain=4000.0 * scale, centre_lo=600.0 * scale,
                   centre_hi=3400.0 * scale)
