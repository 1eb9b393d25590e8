"""Shared helpers of the parity tests: run the oracle and the CUDA library on
the same seeded inputs and compare them."""
import math

import numpy as np

from oracle import oracle as O
from paper_2301_06984_gb300 import bdm
from paper_2301_06984_gb300 import workloads as W

ORACLE_KEYS = ("R", "L", "dt", "dmax", "k", "gamma", "adherence", "detect_static", "sort_every", "growth",
               "divide_volume", "ratio_lo", "ratio_hi", "walk_step", "seed", "death_prob", "type_k", "type_gamma", "curve")


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


# measured FP32-form errors of this run, printed in the terminal summary
# (tests/conftest.py): one entry per checked result
RECORD = []


def assert_fp32_forces(f_gpu, f_ref, scale_pair, scale_terms=None, rel=2e-5, floor=1e-6, what="force"):
    """Per-agent FP32-form force check: |F_gpu - F_oracle| <= rel * S + floor
    with S the oracle's sum over the agent's contacts of the pair-force
    magnitudes |k delta - gamma sqrt(rbar delta)|.  The worst error/bound
    ratio is also taken against the looser sum of the force terms'
    magnitudes (k delta + gamma sqrt(rbar delta)) when given, and both go to
    RECORD with the largest error."""
    err = np.sqrt(((f_gpu - f_ref) ** 2).sum(axis=0))
    bound = rel * scale_pair + floor
    bad = np.nonzero(err > bound)[0]
    worst = float(np.max(err / bound)) if len(err) else 0.0
    worst_t = None
    if scale_terms is not None and len(err):
        worst_t = float(np.max(err / (rel * scale_terms + floor)))
    RECORD.append(dict(what=what, kind="force", n=int(len(err)), worst_ratio=worst, worst_ratio_terms_base=worst_t,
                       max_err=float(err.max()) if len(err) else 0.0))
    assert len(bad) == 0, "%s: %d agents outside %g*S+%g (worst ratio %.3g, first %s: err %g S %g)" % (
        what, len(bad), rel, floor, worst, bad[:5], err[bad[0]], scale_pair[bad[0]])
    return worst


def assert_positions(pos_gpu, pos_ref, tol=1e-4, what="positions"):
    """Positions of the FP32 form against the FP64 oracle within tol (um);
    the largest deviation goes to RECORD."""
    err = float(np.abs(pos_gpu - pos_ref).max()) if pos_gpu.size else 0.0
    RECORD.append(dict(what=what, kind="position", n=int(pos_gpu.shape[-1]), max_err=err))
    assert err <= tol, "%s: max deviation %g um > %g" % (what, err, tol)
    return err


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


def production_step_vs_oracle(s, P, q=None, what="production forces"):
    """One iteration of the production path of simulation s (created with
    keep_forces) against the oracle on the state that iteration starts from.
    The forces and contact counts the iteration's own force kernel formed
    (with the static skip and the epilogue that runs in timed iterations)
    are compared with the oracle's forces on that state, for the agents q of
    the pre-iteration storage order (all when None): contacts exact, forces
    within the FP32 tolerance.  A sort step may reorder storage, so agents
    are matched by uid.  Returns the oracle state of the pre-iteration
    positions and the selected pre-iteration indices."""
    a0 = s.get_agents()
    o = O.State(a0["x"], a0["y"], a0["z"], a0["diam"], uid=a0["uid"], beh=a0["beh"])
    q = np.arange(a0["n"]) if q is None else np.asarray(q)
    s.step(1)
    f_all = s.last_forces()
    nz_all = s.last_nz()
    uid1 = s.get_agents()["uid"]
    order = np.argsort(uid1, kind="stable")
    idx = order[np.searchsorted(uid1[order], a0["uid"][q])]
    assert np.array_equal(uid1[idx], a0["uid"][q])
    f_o, nz_o, _, sc, sa = o.forces_of(P, q=q, with_scale=True, with_scale_abs=True)
    assert np.array_equal(nz_all[idx], nz_o), "%s: contact counts differ" % what
    assert_fp32_forces(f_all[:, idx], f_o, sa, sc, what=what)
    return o, q
