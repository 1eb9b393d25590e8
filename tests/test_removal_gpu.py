"""Parallel removal (Sec. 3.2) on the GPU against the FP64 oracle: agents with
the death behaviour are removed with a per-iteration probability, the removed
slots below the new size are filled by the survivors above it (ascending
order on both sides), daughters are appended before the removals.  FP64 form
bit-exact (storage order, uids, volumes, diameters, positions, static flags,
contacts); FP32 form: storage order and uids exact, positions within 1e-4 um."""
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


def _dying_lattice(m=10, death=0.03):
    # the proliferation lattice with every agent growing and able to die
    w = W.lattice(m=m, steps=20)
    w.params["death_prob"] = death
    w.beh = np.full(w.n, bdm.BEH_GROW | bdm.BEH_DIE, np.uint8)
    return w


def test_growth_division_and_removal_fp64_bit_exact_20_iterations():
    w = _dying_lattice()
    vol = (math.pi / 6.0) * w.diam ** 3
    cap = 4 * w.n
    s = H.gpu_sim(w, capacity=cap, vol=vol)
    o = H.oracle_state(w, cap=cap, vol=vol)
    P = H.oracle_params(w)
    removed = divided = 0
    for t in range(20):
        s.step(1)
        o.step(P)
        pos, a = H.gpu_positions(s)
        c = s.counters()
        assert a["n"] == o.n, "agent count differs after iteration %d" % (t + 1)
        assert c["n_removed"] == o.counters["n_removed"] and c["n_divided"] == o.counters["n_divided"]
        assert np.array_equal(a["uid"], o.uid[: o.n]), "storage order differs after iteration %d" % (t + 1)
        assert np.array_equal(a["vol"], o.vol[: o.n])
        assert np.array_equal(a["diam"], o.diam[: o.n])
        assert np.array_equal(pos, o.positions()), "positions differ after iteration %d" % (t + 1)
        removed += c["n_removed"]
        divided += c["n_divided"]
    assert removed > 100 and divided > 100  # both happened, in the same iterations too
    assert a["next_uid"] == o.next_uid


def test_removal_with_static_skip_fp64_bit_exact():
    # a static core with dying agents in it and walkers around: the boxes of
    # removed agents are dirty next iteration (flags and contacts exact)
    w = W.core_shell(n=20000, seed=5, precision="fp64")
    w.params["death_prob"] = 0.05
    w.beh = (w.beh | np.where(np.arange(w.n) % 3 == 0, bdm.BEH_DIE, 0)).astype(np.uint8)
    s = H.gpu_sim(w, precision="fp64")
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    static = 0
    for t in range(8):
        s.step(1)
        o.step(P)
        pos, a = H.gpu_positions(s)
        assert np.array_equal(a["uid"], o.uid[: o.n]), "storage order differs after iteration %d" % (t + 1)
        assert np.array_equal(pos, o.positions())
        assert np.array_equal(s.last_static(), o.is_static[: o.n]), "static flags differ at iteration %d" % (t + 1)
        assert np.array_equal(s.last_nz(), o.nz[: o.n])
        static += int(s.last_static().sum())
    assert static > 0 and o.n < 0.95 * w.n


@pytest.mark.parametrize("static", [0, 1])
def test_removal_fp32_storage_order_exact_positions_within_tolerance(static):
    w = H.small_blobs(n=50_000, seed=19)
    w.params["death_prob"] = 0.04
    w.params["detect_static"] = static
    w.params["sort_every"] = 3
    w.beh = np.where(np.arange(w.n) % 2 == 0, bdm.BEH_DIE, 0).astype(np.uint8)
    s = H.gpu_sim(w, precision="fp32", keep_forces=True)
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    for t in range(6):
        s.step(1)
        o.step(P)
        a = s.get_agents()
        assert np.array_equal(a["uid"], o.uid[: o.n]), "storage order differs after iteration %d" % (t + 1)
    pos, a = H.gpu_positions(s)
    H.assert_positions(pos, o.positions(), what="positions fp32 blobs 50k with removal, 6 it., static=%d" % static)
    assert o.n < 0.93 * w.n


def test_removal_of_every_agent_and_of_none():
    # death probability 1 on every agent: the population is empty after one
    # iteration; a probability that removes nobody leaves the order alone
    w = H.f32_diam(W.uniform(n=4096, seed=3))
    w.beh = np.full(w.n, bdm.BEH_DIE, np.uint8)
    w.params["death_prob"] = 1.0
    s = H.gpu_sim(w, precision="fp32")
    s.step(1)
    assert s.counters()["n_agents"] == 0 and s.counters()["n_removed"] == w.n
    s.step(2)
    assert s.get_agents()["n"] == 0
    w.params["death_prob"] = 1e-300
    s = H.gpu_sim(w, precision="fp64")
    o = H.oracle_state(w)
    s.step(3)
    o.step(H.oracle_params(w), 3)
    pos, a = H.gpu_positions(s)
    assert a["n"] == w.n and np.array_equal(a["uid"], np.arange(w.n, dtype=np.uint64))
    assert np.array_equal(pos, o.positions())


def test_capacity_error_with_removal_keeps_state():
    # divisions that would overflow the capacity are refused before any state
    # changes, also when some of the dividing agents die in that iteration
    w = _dying_lattice(m=6, death=0.02)
    vol = (math.pi / 6.0) * w.diam ** 3
    s = H.gpu_sim(w, capacity=w.n + 10, vol=vol)
    o = H.oracle_state(w, cap=w.n + 10, vol=vol)
    P = H.oracle_params(w)
    steps = 0
    for _ in range(20):
        try:
            o.step(P)
        except RuntimeError:
            break
        steps += 1
    assert steps < 20  # the oracle refuses the overflowing iteration
    with pytest.raises(bdm.BdmError) as e:
        s.step(20)
    assert e.value.code == bdm.BDM_ECAPACITY
    pos, a = H.gpu_positions(s)
    assert a["step"] == steps and a["n"] == o.n
    assert np.array_equal(a["uid"], o.uid[: o.n])
    assert np.array_equal(pos, o.positions())
