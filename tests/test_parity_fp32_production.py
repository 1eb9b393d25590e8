"""FP32-force form: the forces that the production force kernels form in the
iterations the benchmark times, compared element by element with the FP64
oracle on the state each iteration starts from, and the FP32 edge cases that
the kernels' fast paths depend on (pairs exactly at the cutoff, exactly
touching pairs, coincident pairs, a population far from the origin).

Tolerance, per agent: |F_gpu - F_oracle| <= 2e-5 * S + 1e-6 with S the sum
over the agent's contacts of the pair-force magnitudes
|k delta - gamma sqrt(rbar delta)|; contact counts exact.  The worst ratio of
every check is printed in the terminal summary."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_06984_gb300 import workloads as W
from tests import harness as H

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


@pytest.mark.parametrize("lanes", [4, 0, -3, -4])
def test_production_kernel_forces_blobs_100k_iterations_1_to_10(lanes):
    # no walk, no growth: the step instantiation that the 10M benchmark runs
    # (the lane-per-agent kernel's per-axis epilogue, 4 lanes per agent, the
    # default), the tiled kernel (lanes 0) and the sparse kernel (lanes -3);
    # iteration 1 is a sort step
    w = H.small_blobs(n=100_000, seed=3)
    s = H.gpu_sim(w, precision="fp32", keep_forces=True)
    s.set_force_kernel(lanes)
    P = H.oracle_params(w)
    for it in range(1, 11):
        H.production_step_vs_oracle(s, P, what="blobs 100k iteration %d, kernel lanes=%d" % (it, lanes))


@pytest.mark.parametrize("lanes", [4, 0, -3, -4])
def test_production_kernel_forces_core_shell_with_walk(lanes):
    # random walk on the shell and the static skip: the shared step
    # instantiation with the one-lane epilogue, after the static pass, for
    # the lane-per-agent, tiled and sparse kernels
    w = W.core_shell(n=20000, seed=5)
    s = H.gpu_sim(w, precision="fp32", keep_forces=True)
    s.set_force_kernel(lanes)
    P = H.oracle_params(w)
    n_static = 0
    for it in range(1, 7):
        H.production_step_vs_oracle(s, P, what="core+shell 20k iteration %d, kernel lanes=%d" % (it, lanes))
        n_static += int(s.last_static().sum())
    assert n_static > 0.5 * 5 * w.n


# ------------------------------------------------------------------ edge cases
def _lattice(m, spacing, origin=0.0):
    g = origin + np.arange(m, dtype=np.float64) * spacing
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()])


def _edge_workload(kind):
    rng = np.random.default_rng(41)
    if kind == "ties_at_cutoff":
        # lattice spacing == R: every axis neighbour sits exactly at d = R
        # (not a neighbour although the spheres overlap by 0.5 um); a tenth
        # of the agents is nudged inside the cutoff
        p = _lattice(14, 12.0, 100.0)
        d = np.full(p.shape[1], 12.5)
        sel = rng.random(p.shape[1]) < 0.1
        p[:, sel] += rng.uniform(-0.6, 0.6, (3, int(sel.sum())))
        R = 12.0
    elif kind == "touching":
        # spacing == diameter < R: axis neighbours are neighbours with
        # delta == 0 exactly (no contact); a tenth is nudged into contact
        p = _lattice(14, 10.0, 100.0)
        d = np.full(p.shape[1], 10.0)
        sel = rng.random(p.shape[1]) < 0.1
        p[:, sel] += rng.uniform(-0.4, 0.4, (3, int(sel.sum())))
        R = 12.0
    elif kind == "coincident":
        # a dense cluster in which every twentieth agent duplicates another's
        # position exactly (distance 0: a neighbour without force)
        n = 6000
        p = rng.normal(120.0, 14.0, (3, n))
        p[:, 1::20] = p[:, 0::20]
        d = rng.uniform(8.0, 12.0, n)
        R = 12.0
    else:
        # a dense cluster moved 2^17 box edges away from the origin on every
        # axis: coordinates near 1.6e6 um, where the FP32 box estimate cannot
        # decide most boxes and the FP64 path and the fixed-point frame do
        n = 6000
        p = rng.normal(120.0, 14.0, (3, n)) + float(2 ** 17) * 12.0
        d = rng.uniform(8.0, 12.0, n)
        R = 12.0
    d = np.asarray(d, np.float32).astype(np.float64)
    return W.Workload(kind, p[0].copy(), p[1].copy(), p[2].copy(), d,
                      dict(R=R, L=R, dt=0.01, dmax=3.0, precision="fp32", seed=41), steps=3)


@pytest.mark.parametrize("kind", ["ties_at_cutoff", "touching", "coincident", "far_from_origin"])
def test_fp32_edge_cases(kind):
    w = _edge_workload(kind)
    P = H.oracle_params(w)
    o = H.oracle_state(w)
    f_o, nz_o, nnb_o, sc, sa = o.forces_of(P, with_scale=True, with_scale_abs=True)
    if kind == "ties_at_cutoff":
        assert (nnb_o == 0).sum() > 0.5 * w.n  # the unmoved lattice agents have no neighbour
    if kind == "touching":
        assert ((nnb_o > 0) & (nz_o == 0)).sum() > 0.5 * w.n  # neighbours without contact
    # the force-only kernel: neighbour and contact counts exact, forces within tolerance
    s = H.gpu_sim(w, precision="fp32", keep_forces=True)
    f_g, nz_g, nnb_g = s.forces_now()
    assert np.array_equal(nnb_g, nnb_o), "neighbour counts differ"
    assert np.array_equal(nz_g, nz_o), "contact counts differ"
    H.assert_fp32_forces(f_g, f_o, sa, sc, what="edge %s, force-only kernel" % kind)
    # the production kernel over three iterations, then the positions
    o_run = H.oracle_state(w)
    for it in range(3):
        H.production_step_vs_oracle(s, P, what="edge %s iteration %d, production kernel" % (kind, it + 1))
    o_run.step(P, 3)
    pos, a = H.gpu_positions(s)
    assert np.array_equal(a["uid"], o_run.uid[: o_run.n])
    H.assert_positions(pos, o_run.positions(), what="positions edge %s, 3 iterations" % kind)


# ------------------------------------------------------- lanes per pass
def _box_count_workload(seed=44, L=12.0):
    # boxes of edge L = R on an 8 x 5 plane, box b holding exactly b + 1
    # agents (1..40), plus one box of 48: every pass shape of the
    # lane-per-agent kernel (1, 2, 3-4 agents on 32, 16, 8 lanes; 5-8 on 4;
    # 9-10 as 8 + 1-2; 11-16 on 2 lanes; 17 or more as 16 + the rest).  The
    # grid's box boundaries are the multiples of L, so an agent strictly
    # inside a cell is in that box.
    rng = np.random.default_rng(seed)
    cells = [(10 + b % 8, 10 + b // 8, 10, b + 1) for b in range(40)] + [(20, 10, 10, 48)]
    p, d = [], []
    for cx, cy, cz, c in cells:
        p.append(np.stack([rng.uniform(k * L + 0.05, (k + 1) * L - 0.05, c) for k in (cx, cy, cz)]))
        d.append(rng.uniform(8.0, 12.0, c))
    p = np.concatenate(p, axis=1)
    d = np.asarray(np.concatenate(d), np.float32).astype(np.float64)
    return W.Workload("box-counts", p[0].copy(), p[1].copy(), p[2].copy(), d,
                      dict(R=L, L=L, dt=0.01, dmax=3.0, precision="fp32", seed=seed), steps=3)


@pytest.mark.parametrize("lanes", [4, -4])
def test_lane_schedule_every_pass_shape(lanes):
    w = _box_count_workload()
    P = H.oracle_params(w)
    o = H.oracle_state(w)
    f_o, nz_o, nnb_o, sc, sa = o.forces_of(P, with_scale=True, with_scale_abs=True)
    s = H.gpu_sim(w, precision="fp32", keep_forces=True)
    s.set_force_kernel(lanes)
    f_g, nz_g, nnb_g = s.forces_now()
    assert np.array_equal(nnb_g, nnb_o), "neighbour counts differ"
    assert np.array_equal(nz_g, nz_o), "contact counts differ"
    H.assert_fp32_forces(f_g, f_o, sa, sc, what="box counts 1-40 and 48, force-only kernel, lanes=%d" % lanes)
    for it in range(1, 4):
        H.production_step_vs_oracle(s, P, what="box counts iteration %d, production kernel, lanes=%d" % (it, lanes))
