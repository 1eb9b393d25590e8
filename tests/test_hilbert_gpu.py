"""The Hilbert storage order (the alternative to Morton order that Sec. 4.2
compares): the grid's 4x4x4-box bricks along a 3D Hilbert curve, the boxes of
a brick in Morton order.  On the GPU each brick's rank among the in-domain
bricks is counted octant by octant down the curve's levels; the oracle sorts
by Skilling's Hilbert index.  Bit-exact: brick ranks, grid order, sort-step
storage order and the FP64 trajectory; FP32 positions within 1e-4 um."""
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


def _hilbert_brick_ranks(bxyz, nb):
    # rank of each agent's brick among all bricks of the grid, along the
    # oracle's Hilbert index (brute force over the brick grid)
    nr = [(int(v) + 3) // 4 for v in nb]
    bits = 0
    while (1 << bits) < max(nr):
        bits += 1
    keys = sorted(O.hilbert3(x, y, z, bits) for x in range(nr[0]) for y in range(nr[1]) for z in range(nr[2]))
    pos = {h: r for r, h in enumerate(keys)}
    return np.array([pos[O.hilbert3(int(b[0]) >> 2, int(b[1]) >> 2, int(b[2]) >> 2, bits)] for b in bxyz])


def _clustered(n, seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(150.0, 40.0, (3, n))
    d = np.asarray(rng.uniform(8.0, 12.0, n), np.float32).astype(np.float64)
    return W.Workload("clustered", p[0].copy(), p[1].copy(), p[2].copy(), d,
                      dict(R=12.0, L=12.0, dt=0.01, dmax=3.0, curve=1, seed=seed), steps=5)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_hilbert_grid_order_and_brick_ranks_match_oracle(prec, kind):
    if kind == "uniform":
        w = H.f32_diam(W.uniform(n=8192, seed=1, edge=500.0))
        w.params["curve"] = 1
    else:
        w = _clustered(6000, 3)
    s = H.gpu_sim(w, precision=prec)
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    bxyz, _, lo, nb = o.grid(P)
    assert np.array_equal(s.grid_boxes().T, bxyz)
    assert np.array_equal(s.brick_ranks(), _hilbert_brick_ranks(bxyz, nb[0]))
    assert np.array_equal(s.grid_order(), o.curve_order(P))
    # the Hilbert order differs from the Morton one on these grids
    assert not np.array_equal(o.curve_order(P), o.morton_order(P))


def test_hilbert_sort_steps_fp64_bit_exact():
    w = W.uniform(n=8192, seed=7, edge=300.0)
    w.params.update(curve=1, sort_every=3)
    s = H.gpu_sim(w, precision="fp64")
    o = H.oracle_state(w)
    P = H.oracle_params(w)
    for t in range(7):
        s.step(1)
        o.step(P)
        pos, a = H.gpu_positions(s)
        assert np.array_equal(a["uid"], o.uid[: o.n]), "storage order differs after step %d" % (t + 1)
        assert np.array_equal(pos, o.positions())


def test_hilbert_fp32_blobs_positions():
    w = H.small_blobs(n=100_000, seed=3)
    w.params["curve"] = 1
    s = H.gpu_sim(w, precision="fp32")
    o = H.oracle_state(w)
    s.step(10)
    o.step(H.oracle_params(w), 10)
    pos, a = H.gpu_positions(s)
    assert np.array_equal(a["uid"], o.uid[: o.n])
    H.assert_positions(pos, o.positions(), what="positions fp32 blobs 100k Hilbert order, 10 iterations")


def test_hilbert_ensemble_fp64_bit_exact():
    # each member has its own brick grid and its own curve
    w = W.ensemble(n_sims=12, seed=4, log_lo=2.0, log_hi=3.4, precision="fp64")
    w.params.update(curve=1, sort_every=2)
    s = H.gpu_sim(w)
    o = H.oracle_state(w)
    s.step(5)
    o.step(H.oracle_params(w), 5)
    pos, a = H.gpu_positions(s)
    assert np.array_equal(a["uid"], o.uid[: o.n])
    assert np.array_equal(pos, o.positions())


def test_hilbert_neighbor_lists_unchanged():
    # the curve changes the order of boxes, not which agents are neighbours
    w = _clustered(5000, 4)
    a = H.gpu_sim(w, precision="fp64")
    w.params["curve"] = 0
    b = H.gpu_sim(w, precision="fp64")
    oa, na = a.neighbors()
    ob, nb_ = b.neighbors()
    H.csr_equal(oa, na, ob, nb_)
