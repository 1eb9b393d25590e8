"""Parity at the full sizes of the five workloads.  Where the oracle cannot
follow the whole run, outputs are sampled: the oracle computes the forces of
chosen agents one by one from the GPU's own state, or independent members of
an ensemble, or the agents of a sub-box (whose neighbours all lie within the
sub-box grown by R)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_06984_gb300 import bdm
from paper_2301_06984_gb300 import workloads as W
from tests import harness as H

pytestmark = pytest.mark.gpu


def _state_of(s):
    a = s.get_agents()
    return a, O.State(a["x"], a["y"], a["z"], a["diam"], uid=a["uid"], beh=a["beh"])


def _sample(rng, n, k):
    return np.sort(rng.choice(n, size=min(k, n), replace=False))


def test_lattice_47_cubed_20_iterations_bit_exact():
    w = W.lattice()
    vol = (math.pi / 6.0) * w.diam ** 3
    cap = 4 * w.n + 16
    s = H.gpu_sim(w, capacity=cap, vol=vol)
    o = H.oracle_state(w, cap=cap, vol=vol)
    P = H.oracle_params(w)
    for t in range(w.steps):
        s.step(1)
        o.step(P)
        assert s.counters()["n_agents"] == o.n, "agent count differs after iteration %d" % (t + 1)
    pos, a = H.gpu_positions(s)
    assert a["n"] == 4 * w.n
    assert np.array_equal(a["uid"], o.uid[: o.n])
    assert np.array_equal(a["vol"], o.vol[: o.n])
    assert np.array_equal(a["diam"], o.diam[: o.n])
    assert np.array_equal(pos, o.positions())


def test_blobs_10M_sampled_forces_fp32():
    # iterations 1, 10 and 100 of the 10M-agent run: the forces the timed
    # production kernel itself formed in that iteration (kept with
    # keep_forces), for 3000 sampled agents, against the oracle's forces on the
    # state the iteration started from; plus the force-only kernel on the
    # state after iteration 100
    w = W.blobs()
    s = H.gpu_sim(w, precision="fp32", keep_forces=True)
    P = H.oracle_params(w)
    rng = np.random.default_rng(0)
    done = 0
    for it in (1, 10, 100):
        s.step(it - 1 - done)
        q = _sample(rng, s.counters()["n_agents"], 3000)
        H.production_step_vs_oracle(s, P, q=q, what="blobs 10M iteration %d, production kernel (3000 sampled)" % it)
        done = it
    f_g, nz_g, nnb_g = s.forces_now()
    a, o = _state_of(s)
    q = _sample(rng, a["n"], 3000)
    f_o, nz_o, nnb_o, sc, sa = o.forces_of(P, q=q, with_scale=True, with_scale_abs=True)
    assert np.array_equal(nnb_g[q], nnb_o) and np.array_equal(nz_g[q], nz_o)
    H.assert_fp32_forces(f_g[:, q], f_o, sa, sc, what="blobs 10M after iteration 100, force-only kernel (3000)")


def test_blobs_100k_positions_after_10_iterations_fp32():
    # a standalone 100k-agent run at the 10M workload's density: FP32 form
    # against the FP64 oracle, positions after 10 iterations (re-sort at 0)
    w = H.small_blobs(n=100_000, seed=3)
    s = H.gpu_sim(w, precision="fp32")
    o = H.oracle_state(w)
    s.step(10)
    o.step(H.oracle_params(w), 10)
    pos, a = H.gpu_positions(s)
    assert np.array_equal(a["uid"], o.uid[: o.n])
    H.assert_positions(pos, o.positions(), what="positions fp32 blobs 100k, 10 iterations")


def test_ensemble_512_members_match_independent_runs_fp32():
    w = W.ensemble()
    s = H.gpu_sim(w)
    s.step(3)
    pos, a = H.gpu_positions(s)
    assert np.array_equal(a["sim_off"], w.sim_off)
    rng = np.random.default_rng(1)
    for m in rng.choice(w.n_sims, size=6, replace=False):
        lo, hi = w.sim_off[m], w.sim_off[m + 1]
        o = O.State(w.x[lo:hi], w.y[lo:hi], w.z[lo:hi], w.diam[lo:hi])
        o.step(O.make_params(R=10.0, dt=float(w.dt_sim[m])), 3)
        H.assert_positions(pos[:, lo:hi], o.positions(), what="positions fp32 ensemble-512 member %d, 3 it." % m)


def test_core_shell_150M_static_fraction_and_subbox_forces():
    w = W.core_shell()
    s = H.gpu_sim(w, precision="fp32")
    s.step(3)
    c = s.counters()
    assert c["n_static"] >= 0.8 * w.n, c
    f_g, nz_g, nnb_g = s.forces_now()
    a = s.get_agents()
    pos = np.stack([a["x"], a["y"], a["z"]])
    # a 120 um cube straddling the core surface: static core agents, the
    # core/shell interface and walkers
    r = w.notes["r_core"]
    c0 = np.array([np.median(w.x), np.median(w.y), np.median(w.z)]) + np.array([r, 0.0, 0.0])
    half, R = 60.0, 10.0
    inner = np.all(np.abs(pos - c0[:, None]) < half, axis=0)
    outer = np.all(np.abs(pos - c0[:, None]) < half + R, axis=0)
    sel = np.nonzero(outer)[0]
    assert inner.sum() > 1000
    o = O.State(pos[0, sel], pos[1, sel], pos[2, sel], a["diam"][sel])
    qi = np.nonzero(inner[sel])[0]
    f_o, nz_o, nnb_o, sc, sa = o.forces_of(H.oracle_params(w), q=qi, with_scale=True, with_scale_abs=True)
    g = sel[qi]
    assert np.array_equal(nnb_g[g], nnb_o) and np.array_equal(nz_g[g], nz_o)
    H.assert_fp32_forces(f_g[:, g], f_o, sa, sc, what="core+shell 150M sub-box, force-only kernel")
