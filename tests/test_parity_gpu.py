"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the
same seeded inputs.  Bit-exact: grid contents and order, Morton ranks,
neighbour sets, static flags, division order and uids, and every FP64-form
result.  FP32-force form: per-agent |dF| <= 2e-5 * (sum over contacts of
k delta + gamma sqrt(rbar delta)) + 1e-6, positions after 10 iterations within
1e-4 um, integer results (neighbours, contacts) exact."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_06984_gb300 import bdm
from paper_2301_06984_gb300 import workloads as W
from tests import harness as H

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def clustered(n=6000, seed=21):
    rng = np.random.default_rng(seed)
    p = rng.normal(100.0, 18.0, (3, n))
    d = rng.uniform(8.0, 12.0, n)
    return W.Workload("clustered", p[0].copy(), p[1].copy(), p[2].copy(), d,
                      dict(R=12.0, L=12.0, dt=0.01, dmax=3.0, precision="fp64", seed=seed), steps=5)


# ------------------------------------------------------------------ grid
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_grid_matches_oracle(prec, kind):
    w = W.uniform(n=8192, seed=1) if kind == "uniform" else clustered()
    if prec == "fp32":
        H.f32_diam(w)
    s = H.gpu_sim(w, precision=prec)
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    bxyz, mort, lo, nb = o.grid(P)
    glo, gnb = s.grid_geometry()
    assert np.array_equal(glo[0], lo[0]) and np.array_equal(gnb[0], nb[0])
    assert np.array_equal(s.grid_boxes().T, bxyz)
    assert np.array_equal(s.grid_order(), o.morton_order(P))
    assert np.array_equal(s.brick_ranks(), H.brick_ranks_from_oracle(bxyz, nb[0]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_neighbor_lists_match_oracle(prec):
    w = clustered(n=5000, seed=4)
    if prec == "fp32":
        H.f32_diam(w)
    s = H.gpu_sim(w, precision=prec)
    o = H.oracle_state(w)
    off_o, nb_o = o.neighbors(H.oracle_params(w))
    off_g, nb_g = s.neighbors()
    H.csr_equal(off_g, nb_g, off_o, nb_o)


# ------------------------------------------------------------------ forces
def test_forces_fp64_bit_exact():
    w = W.uniform(n=8192, seed=1)
    s = H.gpu_sim(w, precision="fp64")
    o = H.oracle_state(w)
    f_o, nz_o, nnb_o = o.forces_of(H.oracle_params(w))
    f_g, nz_g, nnb_g = s.forces_now()
    assert np.array_equal(nnb_g, nnb_o) and np.array_equal(nz_g, nz_o)
    assert np.array_equal(f_g, f_o)


@pytest.mark.parametrize("kind", ["uniform", "clustered", "blobs"])
def test_forces_fp32_within_tolerance(kind):
    if kind == "uniform":
        w = H.f32_diam(W.uniform(n=8192, seed=1))
    elif kind == "clustered":
        w = H.f32_diam(clustered(n=6000, seed=5))
    else:
        w = H.small_blobs(n=100_000, seed=3)
    s = H.gpu_sim(w, precision="fp32")
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    f_o, nz_o, nnb_o, sc, sa = o.forces_of(P, with_scale=True, with_scale_abs=True)
    f_g, nz_g, nnb_g = s.forces_now()
    assert np.array_equal(nnb_g, nnb_o), "neighbour counts differ"
    assert np.array_equal(nz_g, nz_o), "contact counts differ"
    H.assert_fp32_forces(f_g, f_o, sa, sc, what="forces fp32 %s (force-only kernel)" % kind)


# ------------------------------------------------------------------ trajectories
def test_trajectory_fp64_bit_exact_10_steps():
    w = W.uniform(n=8192, seed=1)
    s = H.gpu_sim(w, precision="fp64", keep_forces=True)
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    for t in range(10):
        s.step(1)
        o.step(P)
        pos, a = H.gpu_positions(s)
        assert np.array_equal(pos, o.positions()), "positions differ after step %d" % (t + 1)
        assert np.array_equal(s.last_forces(), o.forces()), "forces differ at step %d" % (t + 1)
        assert np.array_equal(s.last_nz(), o.nz[: o.n])
    assert a["step"] == 10


def test_trajectory_fp32_positions_within_1e4_after_10_steps():
    w = H.f32_diam(W.uniform(n=8192, seed=1))
    s = H.gpu_sim(w, precision="fp32")
    o = H.oracle_state(w)
    s.step(10)
    o.step(H.oracle_params(w), 10)
    pos, _ = H.gpu_positions(s)
    H.assert_positions(pos, o.positions(), what="positions fp32 uniform 8192, 10 iterations")


def test_sort_step_bit_exact_fp64():
    w = W.uniform(n=8192, seed=7)
    w.params["sort_every"] = 3
    s = H.gpu_sim(w, precision="fp64", sort_every=3)
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    for t in range(7):
        s.step(1)
        o.step(P)
        pos, a = H.gpu_positions(s)
        assert np.array_equal(a["uid"], o.uid[: o.n]), "storage order differs after step %d" % (t + 1)
        assert np.array_equal(pos, o.positions())


def test_explicit_sort_matches_oracle_order():
    w = clustered(n=4000, seed=9)
    s = H.gpu_sim(w, precision="fp64")
    o = H.oracle_state(w)
    perm = o.morton_order(H.oracle_params(w))
    s.sort()
    a = s.get_agents()
    assert np.array_equal(a["uid"], perm.astype(np.uint64))
    assert np.array_equal(a["x"], w.x[perm])


# ------------------------------------------------------------------ static skip
def test_static_skip_fp64_matches_oracle_flags_and_positions():
    w = W.core_shell(n=20000, seed=5, precision="fp64")
    s = H.gpu_sim(w, precision="fp64")
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    total_static = 0
    for t in range(6):
        s.step(1)
        o.step(P)
        pos, _ = H.gpu_positions(s)
        assert np.array_equal(pos, o.positions()), "positions differ after step %d" % (t + 1)
        assert np.array_equal(s.last_static(), o.is_static[: o.n]), "static flags differ at step %d" % (t + 1)
        assert np.array_equal(s.last_nz(), o.nz[: o.n])
        total_static += int(s.last_static().sum())
    assert total_static > 0.5 * 5 * w.n


def test_static_skip_fp32_equals_no_skip():
    w = W.core_shell(n=20000, seed=5)
    a = H.gpu_sim(w, precision="fp32", detect_static=1)
    b = H.gpu_sim(w, precision="fp32", detect_static=0)
    for _ in range(5):
        a.step(1)
        b.step(1)
        pa, _ = H.gpu_positions(a)
        pb, _ = H.gpu_positions(b)
        assert np.array_equal(pa, pb)
    assert a.counters()["n_static"] > 0.5 * w.n
    o = H.oracle_state(w)
    o.step(H.oracle_params(w), 5)
    H.assert_positions(pa, o.positions(), what="positions fp32 core+shell 20k static skip, 5 iterations")


# ------------------------------------------------------------------ division
def test_division_lattice_fp64_bit_exact():
    w = W.lattice(m=10, steps=20)
    vol = (math.pi / 6.0) * w.diam ** 3
    s = H.gpu_sim(w, capacity=4 * w.n, vol=vol)
    o = H.oracle_state(w, cap=4 * w.n, vol=vol)
    P = H.oracle_params(w)
    for t in range(20):
        s.step(1)
        o.step(P)
        pos, a = H.gpu_positions(s)
        assert a["n"] == o.n, "agent count differs after step %d" % (t + 1)
        assert np.array_equal(a["uid"], o.uid[: o.n])
        assert np.array_equal(a["vol"], o.vol[: o.n])
        assert np.array_equal(a["diam"], o.diam[: o.n])
        assert np.array_equal(pos, o.positions()), "positions differ after step %d" % (t + 1)
    assert o.n == 4 * w.n


def test_division_capacity_error_keeps_state():
    w = W.lattice(m=6, steps=20)
    vol = (math.pi / 6.0) * w.diam ** 3
    s = H.gpu_sim(w, capacity=w.n + 10, vol=vol)
    with pytest.raises(bdm.BdmError) as e:
        s.step(20)
    assert e.value.code == bdm.BDM_ECAPACITY
    a = s.get_agents()
    assert a["n"] == w.n and a["step"] == 12  # divisions start in iteration 13
    o = H.oracle_state(w, vol=vol)
    o.step(H.oracle_params(w), 12)
    assert np.array_equal(np.stack([a["x"], a["y"], a["z"]]), o.positions())


# ------------------------------------------------------------------ ensemble
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ensemble_matches_independent_oracle_runs(prec):
    w = W.ensemble(n_sims=16, seed=4, log_lo=2.0, log_hi=3.3, precision=prec)
    s = H.gpu_sim(w)
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    s.step(5)
    o.step(P, 5)
    pos, a = H.gpu_positions(s)
    assert np.array_equal(a["sim_off"], w.sim_off)
    if prec == "fp64":
        assert np.array_equal(pos, o.positions())
    else:
        H.assert_positions(pos, o.positions(), what="positions fp32 ensemble 16 members, 5 iterations")


# ------------------------------------------------------------------ resume, determinism
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_resume_is_bit_exact(prec):
    w = H.f32_diam(W.uniform(n=8192, seed=2))
    a = H.gpu_sim(w, precision=prec)
    a.step(10)
    b = H.gpu_sim(w, precision=prec)
    b.step(5)
    st = b.get_agents()
    c = H.gpu_sim(w, precision=prec, set_state=False)
    c.set_agents(st["x"], st["y"], st["z"], st["diam"], uid=st["uid"], beh=st["beh"], step=st["step"],
                 next_uid=st["next_uid"])
    c.step(5)
    pa, _ = H.gpu_positions(a)
    pc, sc = H.gpu_positions(c)
    assert sc["step"] == 10
    assert np.array_equal(pa, pc)


def test_fp32_runs_are_deterministic():
    w = H.small_blobs(n=50_000, seed=8)
    w.params["sort_every"] = 2
    a = H.gpu_sim(w)
    b = H.gpu_sim(w)
    a.step(4)
    b.step(4)
    pa, aa = H.gpu_positions(a)
    pb, ab = H.gpu_positions(b)
    assert np.array_equal(pa, pb) and np.array_equal(aa["uid"], ab["uid"])


def test_device_pointers_round_trip():
    import torch
    w = H.f32_diam(W.uniform(n=4096, seed=3))
    s = bdm.Simulation.from_workload(w, precision="fp32")
    t = lambda a: torch.as_tensor(a, device="cuda")
    s.set_agents(t(w.x), t(w.y), t(w.z), t(w.diam))
    s.step(2)
    d = s.get_agents(device=True)
    h = H.gpu_sim(w, precision="fp32")
    h.step(2)
    ph, _ = H.gpu_positions(h)
    assert np.array_equal(torch.stack([d["x"], d["y"], d["z"]]).cpu().numpy(), ph)


# ------------------------------------------------------------------ edge cases
def test_empty_and_single_agent():
    w = W.uniform(n=1, seed=1)
    s = H.gpu_sim(w)
    s.step(3)
    a = s.get_agents()
    assert a["n"] == 1 and a["x"][0] == w.x[0]
    e = bdm.Simulation(R=10.0, capacity=16)
    e.set_agents(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    e.step(2)
    assert e.get_agents()["n"] == 0


def test_state_and_input_errors():
    s = bdm.Simulation(R=10.0, capacity=16)
    with pytest.raises(bdm.BdmError) as e:
        s.step(1)
    assert e.value.code == bdm.BDM_ESTATE
    x = np.array([0.0, np.nan])
    with pytest.raises(bdm.BdmError) as e:
        s.set_agents(x, np.zeros(2), np.zeros(2), np.full(2, 5.0))
    assert e.value.code == bdm.BDM_EINVAL
    with pytest.raises(bdm.BdmError) as e:
        s.set_agents(np.zeros(20), np.zeros(20), np.zeros(20), np.full(20, 5.0))
    assert e.value.code == bdm.BDM_ECAPACITY


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_crowded_box_and_coincident_agents(prec):
    # 6000 agents inside one 12 um box (the brick sort's off-chip path) plus
    # exactly coincident pairs (zero distance: neighbours without force)
    rng = np.random.default_rng(17)
    n = 6000
    p = rng.uniform(100.0, 111.0, (3, n))
    p[:, 1::500] = p[:, 0::500]
    d = np.asarray(rng.uniform(8.0, 12.0, n), np.float32).astype(np.float64)
    w = W.Workload("crowd", p[0].copy(), p[1].copy(), p[2].copy(), d, dict(R=12.0, L=12.0, precision=prec), 1)
    s = H.gpu_sim(w, precision=prec)
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    assert np.array_equal(s.grid_order(), o.morton_order(P))
    f_o, nz_o, nnb_o, sc, sa = o.forces_of(P, with_scale=True, with_scale_abs=True)
    f_g, nz_g, nnb_g = s.forces_now()
    assert np.array_equal(nnb_g, nnb_o) and np.array_equal(nz_g, nz_o)
    if prec == "fp64":
        assert np.array_equal(f_g, f_o)
    else:
        H.assert_fp32_forces(f_g, f_o, sa, sc, what="forces fp32 crowded box + coincident")


def test_grid_capacity_grows_transparently():
    # a sparse cloud over a huge box: many more bricks than the initial guess
    rng = np.random.default_rng(2)
    n = 3000
    p = rng.uniform(0.0, 6000.0, (3, n))
    w = W.Workload("sparse", p[0].copy(), p[1].copy(), p[2].copy(), np.full(n, 10.0),
                   dict(R=10.0, L=10.0, precision="fp64"), 1)
    s = H.gpu_sim(w)
    o = H.oracle_state(w)
    s.step(2)
    o.step(H.oracle_params(w), 2)
    pos, _ = H.gpu_positions(s)
    assert np.array_equal(pos, o.positions())
    assert s.counters()["n_bricks"] > (1 << 16)


# ------------------------------------------------------------------ autotuner
def test_autotune_fp64_keeps_state_and_stays_bit_exact():
    w = W.uniform(n=8192, seed=11)
    s = H.gpu_sim(w, precision="fp64")
    s.step(2)
    before, a0 = H.gpu_positions(s)
    t = s.autotune(trial_steps=2, what=bdm.TUNE_BOX_EDGE | bdm.TUNE_SORT)
    after, a1 = H.gpu_positions(s)
    assert np.array_equal(before, after) and a1["step"] == a0["step"] == 2
    assert t["box_edge"] in (12.0, 13.5, 15.0, 18.0) and t["sort_every"] in (0, 5, 10, 20)
    assert t["n_trials"] >= 9
    o = O.State(a1["x"], a1["y"], a1["z"], a1["diam"], uid=a1["uid"], step=2)
    s.step(4)
    o.step(H.oracle_params(w, L=t["box_edge"], sort_every=t["sort_every"]), 4)
    pos, a = H.gpu_positions(s)
    assert np.array_equal(a["uid"], o.uid[: o.n])
    assert np.array_equal(pos, o.positions())


@pytest.mark.parametrize("lanes", [0, -3, -4, -1, 1, 2, 4, 8, 32])
def test_fp32_force_kernels_agree_with_oracle(lanes):
    # every lanes-per-agent choice of the force kernel: same exact
    # neighbour and contact decisions, forces within the FP32 tolerance, on a
    # workload with crowded boxes (more than 32 agents) and several chunks
    w = H.small_blobs(n=60_000, seed=17)
    s = H.gpu_sim(w)
    s.set_force_kernel(lanes)
    s.step(2)
    f_g, nz_g, nnb_g = s.forces_now()
    a = s.get_agents()
    o = O.State(a["x"], a["y"], a["z"], a["diam"])
    f_o, nz_o, nnb_o, sc, sa = o.forces_of(H.oracle_params(w), with_scale=True, with_scale_abs=True)
    assert np.array_equal(nnb_g, nnb_o) and np.array_equal(nz_g, nz_o)
    H.assert_fp32_forces(f_g, f_o, sa, sc, what="forces fp32 blobs 60k, kernel lanes=%d" % lanes)
    # the workload exercises boxes of more than one 32-agent group
    bx = s.grid_boxes()
    _, occ = np.unique(bx, axis=1, return_counts=True)
    assert occ.max() > 32


@pytest.mark.parametrize("walk", [0.0, 0.5])
@pytest.mark.parametrize("lanes", [0, -3, -4, -1, 1, 2, 4, 8, 32])
def test_fp32_step_positions_every_force_kernel(lanes, walk):
    # positions after 3 FP32 iterations against the FP64 oracle for every FP32
    # force kernel.  Without random walk or growth the step runs the per-axis
    # epilogue instantiation (lanes 0-2 of an agent finish one axis each; with
    # the cost model, boxes of fewer than 4 lanes per agent keep the one-lane
    # epilogue); with the walk it runs the shared instantiation.
    w = H.small_blobs(n=20_000, seed=23)
    if walk:
        w.params["walk_step"] = walk
        w.beh = np.where(np.arange(w.n) % 2 == 0, W.WALK, 0).astype(np.uint8)
    s = H.gpu_sim(w, precision="fp32")
    s.set_force_kernel(lanes)
    o = H.oracle_state(w)
    s.step(3)
    o.step(H.oracle_params(w), 3)
    pos, a = H.gpu_positions(s)
    assert np.array_equal(a["uid"], o.uid[: o.n])
    H.assert_positions(pos, o.positions(), what="positions fp32 blobs 20k, 3 it., lanes=%d walk=%g" % (lanes, walk))
    moved = np.abs(pos - np.stack([w.x, w.y, w.z])).max()
    assert moved > 1e-3  # the agents did move


def test_autotune_fp32_lanes_keep_tolerance():
    w = H.small_blobs(n=40_000, seed=13)
    s = H.gpu_sim(w)
    t = s.autotune(trial_steps=2)
    assert t["lanes"] in (-4, 4, -3, 0)
    f_g, nz_g, nnb_g = s.forces_now()
    a = s.get_agents()
    o = O.State(a["x"], a["y"], a["z"], a["diam"])
    f_o, nz_o, nnb_o, sc, sa = o.forces_of(H.oracle_params(w, L=t["box_edge"]), with_scale=True,
                                           with_scale_abs=True)
    assert np.array_equal(nnb_g, nnb_o) and np.array_equal(nz_g, nz_o)
    H.assert_fp32_forces(f_g, f_o, sa, sc, what="forces fp32 blobs 40k after autotune")
