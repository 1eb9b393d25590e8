"""Heterotypic adhesion (the cell-sorting model class of Sec. 6.5) on the GPU
against the FP64 oracle: agents of two types, each type pair with its own
force constants k and gamma.  FP64 form bit-exact (forces, contacts,
trajectory, division with inherited types); FP32 form: forces of the
production kernel within 2e-5 * (sum of pair-force magnitudes) + 1e-6,
contacts exact, positions within 1e-4 um."""
import math

import numpy as np
import pytest

from paper_2301_06984_gb300 import bdm
from paper_2301_06984_gb300 import workloads as W
from tests import harness as H

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield


def test_two_type_sorting_fp64_forces_and_trajectory_bit_exact():
    w = W.cell_sorting(n=8000, seed=6, precision="fp64")
    s = H.gpu_sim(w, keep_forces=True)
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    f_o, nz_o, nnb_o = o.forces_of(P)
    f_g, nz_g, nnb_g = s.forces_now()
    assert np.array_equal(nnb_g, nnb_o) and np.array_equal(nz_g, nz_o) and nz_o.sum() > 0
    assert np.array_equal(f_g, f_o)
    for t in range(10):
        s.step(1)
        o.step(P)
        pos, a = H.gpu_positions(s)
        assert np.array_equal(pos, o.positions()), "positions differ after iteration %d" % (t + 1)
        assert np.array_equal(s.last_forces(), o.forces())
    assert np.array_equal(a["beh"], o.beh[: o.n])


def test_two_type_sorting_fp32_production_forces_and_positions():
    w = W.cell_sorting(n=60000, seed=7, precision="fp32")
    s = H.gpu_sim(w, keep_forces=True)
    P = H.oracle_params(w)
    o = H.oracle_state(w)
    for it in range(1, 6):
        H.production_step_vs_oracle(s, P, what="cell sorting 60k iteration %d, production kernel" % it)
    o.step(P, 5)
    pos, a = H.gpu_positions(s)
    assert np.array_equal(a["uid"], o.uid[: o.n])
    H.assert_positions(pos, o.positions(), what="positions fp32 cell sorting 60k, 5 iterations")
    f_g, nz_g, nnb_g = s.forces_now()
    from oracle import oracle as O
    a = s.get_agents()
    st = O.State(a["x"], a["y"], a["z"], a["diam"], beh=a["beh"])
    f_o, nz_o, nnb_o, sc, sa = st.forces_of(P, with_scale=True, with_scale_abs=True)
    assert np.array_equal(nnb_g, nnb_o) and np.array_equal(nz_g, nz_o)
    H.assert_fp32_forces(f_g, f_o, sa, sc, what="cell sorting 60k after 5 iterations, force-only kernel")


def test_types_are_inherited_by_daughters_fp64():
    # the proliferation lattice with two types: daughters carry the mother's
    # type (behaviour byte), and the type-pair forces stay bit-exact
    w = W.lattice(m=8, steps=20)
    t = (np.arange(w.n) % 2).astype(np.uint8)
    w.beh = (bdm.BEH_GROW | (t << bdm.TYPE_SHIFT)).astype(np.uint8)
    w.params["type_k"] = [[2.0, 1.0], [1.0, 2.0]]
    w.params["type_gamma"] = [[1.2, 0.4], [0.4, 1.2]]
    vol = (math.pi / 6.0) * w.diam ** 3
    cap = 4 * w.n
    s = H.gpu_sim(w, capacity=cap, vol=vol)
    o = H.oracle_state(w, cap=cap, vol=vol)
    P = H.oracle_params(w)
    for it in range(16):
        s.step(1)
        o.step(P)
    pos, a = H.gpu_positions(s)
    assert a["n"] == o.n > w.n
    assert np.array_equal(a["beh"], o.beh[: o.n])
    assert np.array_equal(pos, o.positions())


def test_bad_type_tables_are_rejected():
    with pytest.raises(bdm.BdmError) as e:
        bdm.Simulation(R=10.0, capacity=10, type_k=[[2.0, 1.0], [0.5, 2.0]], type_gamma=[[1.0, 1.0], [1.0, 1.0]])
    assert e.value.code == bdm.BDM_EINVAL
    with pytest.raises(bdm.BdmError):
        bdm.Simulation(R=10.0, capacity=10, type_k=[[2.0, -1.0], [-1.0, 2.0]], type_gamma=np.ones((2, 2)))
