"""Small parity cases run on the -DBDM_CHECK build of the library (selected
with BDM_LIBRARY in a process of its own): every kernel path is exercised with
all device bounds checks on, the device error word must stay 0, and the
results must still match the FP64 oracle.  Run by
tests/test_check_build_gpu.py as `python -m tests.check_build_cases`."""
import math
import sys

import numpy as np

from oracle import oracle as O
from paper_2301_06984_gb300 import bdm
from paper_2301_06984_gb300 import workloads as W
from tests import harness as H


def _no_error(s, what):
    c = s.counters()
    assert c["error"] == 0, "%s: device error word %d" % (what, c["error"])


def case_uniform_fp64_sorted():
    w = W.uniform(n=8192, seed=1)
    w.params["sort_every"] = 2
    s = H.gpu_sim(w, precision="fp64", sort_every=2)
    o = H.oracle_state(w)
    s.step(4)
    o.step(H.oracle_params(w), 4)
    pos, a = H.gpu_positions(s)
    assert np.array_equal(a["uid"], o.uid[: o.n]) and np.array_equal(pos, o.positions())
    _no_error(s, "uniform fp64")


def case_blobs_fp32_production():
    w = H.small_blobs(n=30_000, seed=5)
    s = H.gpu_sim(w, precision="fp32", keep_forces=True)
    P = H.oracle_params(w)
    for it in range(3):
        H.production_step_vs_oracle(s, P, what="check build blobs iteration %d" % (it + 1))
    _no_error(s, "blobs fp32")


def case_blobs_fp32_every_kernel():
    # the tiled, sparse and lane-per-agent kernels on their own (the default
    # hybrid launch runs the last two together)
    w = H.small_blobs(n=20_000, seed=7)
    P = H.oracle_params(w)
    for lanes in (0, -3, 4):
        s = H.gpu_sim(w, precision="fp32", keep_forces=True)
        s.set_force_kernel(lanes)
        for it in range(2):
            H.production_step_vs_oracle(s, P, what="check build blobs lanes=%d iteration %d" % (lanes, it + 1))
        _no_error(s, "blobs fp32 lanes=%d" % lanes)


def case_lattice_division_removal():
    w = W.lattice(m=8, steps=16)
    w.params["death_prob"] = 0.03
    w.beh = np.full(w.n, bdm.BEH_GROW | bdm.BEH_DIE, np.uint8)
    vol = (math.pi / 6.0) * w.diam ** 3
    s = H.gpu_sim(w, capacity=4 * w.n, vol=vol)
    o = H.oracle_state(w, cap=4 * w.n, vol=vol)
    s.step(16)
    o.step(H.oracle_params(w), 16)
    pos, a = H.gpu_positions(s)
    assert a["n"] == o.n and np.array_equal(a["uid"], o.uid[: o.n]) and np.array_equal(pos, o.positions())
    _no_error(s, "lattice")


def case_core_shell_static_walk():
    w = W.core_shell(n=20000, seed=5)
    s = H.gpu_sim(w, precision="fp32")
    o = H.oracle_state(w)
    s.step(4)
    o.step(H.oracle_params(w), 4)
    pos, _ = H.gpu_positions(s)
    assert np.abs(pos - o.positions()).max() <= 1e-4 and s.counters()["n_static"] > 0
    _no_error(s, "core+shell")


def case_ensemble():
    w = W.ensemble(n_sims=8, seed=4, log_lo=2.0, log_hi=3.3, precision="fp64")
    s = H.gpu_sim(w)
    o = H.oracle_state(w)
    s.step(3)
    o.step(H.oracle_params(w), 3)
    pos, _ = H.gpu_positions(s)
    assert np.array_equal(pos, o.positions())
    _no_error(s, "ensemble")


def case_crowded_box_and_types():
    rng = np.random.default_rng(17)
    n = 6000
    p = rng.uniform(100.0, 111.0, (3, n))
    d = np.asarray(rng.uniform(8.0, 12.0, n), np.float32).astype(np.float64)
    beh = (rng.integers(0, 2, n) << bdm.TYPE_SHIFT).astype(np.uint8)
    w = W.Workload("crowd", p[0].copy(), p[1].copy(), p[2].copy(), d,
                   dict(R=12.0, L=12.0, precision="fp64", type_k=W.SORTING_K, type_gamma=W.SORTING_GAMMA), 1,
                   beh=beh)
    s = H.gpu_sim(w)
    o = H.oracle_state(w)
    f_o, nz_o, nnb_o = o.forces_of(H.oracle_params(w))
    f_g, nz_g, nnb_g = s.forces_now()
    assert np.array_equal(nnb_g, nnb_o) and np.array_equal(f_g, f_o)
    _no_error(s, "crowded box")


def case_grid_regrowth():
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
    _no_error(s, "grid regrowth")


CASES = [case_uniform_fp64_sorted, case_blobs_fp32_production, case_blobs_fp32_every_kernel,
         case_lattice_division_removal,
         case_core_shell_static_walk, case_ensemble, case_crowded_box_and_types, case_grid_regrowth]

if __name__ == "__main__":
    import torch
    assert torch.cuda.is_available()
    for case in CASES:
        case()
        print("ok", case.__name__, flush=True)
    print("library", bdm.lib()._name)
    sys.exit(0)
