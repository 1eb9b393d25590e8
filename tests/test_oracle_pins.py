"""Pins of the FP64 CPU oracle against facts that do not come from the oracle:
the paper's worked Morton example (Sec. 4.2), hand-worked closed forms of the
pair force, brute-force enumeration, exact invariants (antisymmetry,
translation invariance, static skip == no skip), numpy's Philox bit generator
and numpy's cube root.  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_06984_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _state(p, d, **kw):
    return O.State(p[0], p[1], p[2], d, **kw)


# --------------------------------------------------------------------------- Philox / cbrt
@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((5, 7), (0, 0, 0, 0)),
                                     ((2**64 - 1, 123), (2**64 - 1, 3, 9, 1)),
                                     ((0xDEADBEEF, 1), (41, 2**63, 7, 2**64 - 2))])
def test_philox_matches_numpy_bit_generator(key, ctr):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    ref = bg.random_raw(8)
    # numpy increments the 256-bit counter (with carry) before each block
    c = list(ctr)
    for blk in range(2):
        i = 0
        c[i] = (c[i] + 1) % 2**64
        while c[i] == 0 and i < 3:
            i += 1
            c[i] = (c[i] + 1) % 2**64
        out = O.philox4x64_10(c, key)
        assert list(out) == list(ref[4 * blk:4 * blk + 4])


def test_cbrt_within_one_ulp_of_numpy():
    rng = np.random.default_rng(11)
    xs = np.concatenate([rng.uniform(1.0, 1e5, 20000), 10.0 ** rng.uniform(-200, 200, 5000),
                         [523.5987755982989, 4188.790204786391, 1e-300, 1e300]])
    worst = 0.0
    for x in xs:
        c, r = O.cbrt(x), float(np.cbrt(x))
        worst = max(worst, abs(c - r) / np.spacing(r))
    assert worst <= 1.0
    for k in (1, 2, 3, 10, 20, 100):
        assert O.cbrt(float(k) ** 3) == float(k)
    assert O.cbrt(-27.0) == -3.0 and O.cbrt(0.0) == 0.0


def test_unit_vector_is_unit_and_isotropic():
    v = np.array([O.unit_vector(9, uid, 3, 1) for uid in range(20000)])
    norms = np.linalg.norm(v, axis=1)
    assert np.max(np.abs(norms - 1.0)) < 4e-16
    # isotropy: E[u] = 0 and E[u u^T] = I/3 (sampling error ~ 1/sqrt(20000))
    assert np.all(np.abs(v.mean(axis=0)) < 0.02)
    assert np.allclose(v.T @ v / len(v), np.eye(3) / 3.0, atol=0.02)
    # streams differ by purpose and by step
    assert not np.allclose(O.unit_vector(9, 5, 3, 1), O.unit_vector(9, 5, 3, 2))
    assert not np.allclose(O.unit_vector(9, 5, 3, 1), O.unit_vector(9, 5, 4, 1))


def test_uniform_ratio_draw_range():
    u = np.array([O.uniform(3, uid, 0, 0) for uid in range(5000)])
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.02


# --------------------------------------------------------------------------- Morton / gaps
def _gold_lines(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            out[k] = v
    return out


def test_morton_worked_example_sec4_2():
    g = _gold_lines("morton_gap_3x3_in_4x4.txt")
    nx, ny = map(int, g["dims"])
    codes = sorted(O.morton2(x, y) for x in range(nx) for y in range(ny))
    assert codes == [int(c) for c in g["in_domain_codes"]]
    gaps = [(a, b) for a, b in zip(codes, codes[1:]) if b - a > 1]
    assert gaps == [tuple(map(int, s.split("-"))) for s in g["gaps"]]
    # the offsets array of the DFS reproduces the same ordering
    offs = O.morton_offsets([nx, ny])
    assert offs == [(0, 0), (5, 1), (6, 2), (8, 4)]
    ranked = []
    for r in range(nx * ny):
        e = max(i for i, (bc, _) in enumerate(offs) if bc <= r)
        ranked.append(r + offs[e][1])
    assert ranked == codes


def test_morton3_axis_bits():
    assert O.morton3(1, 0, 0) == 1 and O.morton3(0, 1, 0) == 2 and O.morton3(0, 0, 1) == 4
    assert O.morton3(2, 0, 0) == 8 and O.morton3(3, 3, 3) == 63
    assert O.morton3(2**20, 0, 0) == 1 << 60


@pytest.mark.parametrize("dims", [(1, 1, 1), (3, 3, 3), (5, 2, 7), (8, 8, 8), (9, 1, 4), (13, 6, 11),
                                  (2, 17, 3), (3, 5), (7, 7), (16, 3)])
def test_morton_offsets_against_brute_force(dims):
    if len(dims) == 3:
        codes = sorted(O.morton3(x, y, z) for x in range(dims[0]) for y in range(dims[1])
                       for z in range(dims[2]))
    else:
        codes = sorted(O.morton2(x, y) for x in range(dims[0]) for y in range(dims[1]))
    offs = O.morton_offsets(list(dims))
    counters = [bc for bc, _ in offs]
    assert counters == sorted(counters)
    for r, c in enumerate(codes):
        e = max(i for i, (bc, _) in enumerate(offs) if bc <= r)
        assert r + offs[e][1] == c
        # inverse mapping: rank = code - offset of the last entry at or below it
        e2 = max(i for i, (bc, of) in enumerate(offs) if bc + of <= c)
        assert c - offs[e2][1] == r


# --------------------------------------------------------------------------- pair force
def _pair_lines():
    rows = []
    with open(os.path.join(GOLD, "pair_forces.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(float(v) for v in line.split()))
    return rows


@pytest.mark.parametrize("r1,r2,d,F", _pair_lines())
def test_two_sphere_hand_worked(r1, r2, d, F):
    P = O.make_params(R=12.0)
    # along a skew axis, so every component is exercised; the touching and
    # apart cases use the x axis so that the distance is exact
    u = np.array([2.0, -1.0, 2.0]) / 3.0 if F != 0.0 else np.array([1.0, 0.0, 0.0])
    p = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0] + d * u]).T
    s = _state(p, np.array([2 * r1, 2 * r2]))
    f, nz, nnb = s.forces_of(P)
    assert nnb.tolist() == [1, 1]
    assert nz.tolist() == ([1, 1] if F != 0.0 else [0, 0])
    # force on agent 0 points from 1 to 0 (repulsive for F > 0)
    exp0 = -F * u
    assert np.allclose(f[:, 0], exp0, rtol=0, atol=1e-14)
    assert np.allclose(f[:, 1], -exp0, rtol=0, atol=1e-14)
    if F != 0.0:
        assert abs(np.linalg.norm(f[:, 0]) - abs(F)) <= 4e-16 * max(1.0, abs(F)) * 4


def test_three_collinear_equal_spheres_middle_is_zero():
    P = O.make_params(R=12.0)
    p = np.array([[0.0, 9.0, 18.0], [5.0, 5.0, 5.0], [5.0, 5.0, 5.0]])
    s = _state(p, np.full(3, 10.0))
    f, nz, _ = s.forces_of(P)
    assert f[:, 1].tolist() == [0.0, 0.0, 0.0]
    assert nz.tolist() == [1, 2, 1]
    assert f[0, 0] == -(2.0 - math.sqrt(2.5)) and f[0, 2] == (2.0 - math.sqrt(2.5))


def test_zero_force_without_overlap():
    rng = np.random.default_rng(3)
    # d in [8, 9] and lattice spacing 9.5 > max diameter: neighbours within R
    # but none overlap
    g = np.arange(6) * 9.5
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    p = np.stack([x.ravel(), y.ravel(), z.ravel()]) + rng.uniform(-0.2, 0.2, (3, 216))
    d = rng.uniform(8.0, 9.0, 216)
    s = _state(p, d)
    f, nz, nnb = s.forces_of(O.make_params(R=12.0))
    assert np.all(f == 0.0) and np.all(nz == 0) and nnb.sum() > 0


@pytest.mark.parametrize("kind", ["uniform", "lattice_ties", "clustered"])
def test_grid_neighbors_equal_brute_force(kind):
    rng = np.random.default_rng(7)
    if kind == "uniform":
        n = 2000
        p = rng.uniform(0, 80, (3, n))
        R = 10.0
    elif kind == "lattice_ties":
        g = np.arange(10) * 20.0  # spacing == R: lattice neighbours at exactly R are excluded
        z, y, x = np.meshgrid(g, g, g, indexing="ij")
        p = np.stack([x.ravel(), y.ravel(), z.ravel()])
        n = p.shape[1]
        R = 20.0
    else:
        n = 1500
        p = rng.normal(50, 6, (3, n))
        R = 7.0
    s = _state(p, np.full(n, R * 0.9))
    P = O.make_params(R=R)
    off_g, nb_g = s.neighbors(P)
    off_b, nb_b = s.neighbors_brute(P)
    assert off_g.tolist() == off_b.tolist()
    for i in range(n):
        assert sorted(nb_g[off_g[i]:off_g[i + 1]].tolist()) == nb_b[off_b[i]:off_b[i + 1]].tolist()
    if kind == "lattice_ties":
        assert len(nb_b) == 0
    else:
        assert len(nb_b) > n


def test_larger_box_edge_keeps_neighbor_sets():
    rng = np.random.default_rng(8)
    p = rng.uniform(0, 100, (3, 1200))
    s = _state(p, np.full(1200, 9.0))
    a = s.neighbors(O.make_params(R=10.0))
    b = s.neighbors(O.make_params(R=10.0, L=17.5))
    assert a[0].tolist() == b[0].tolist()
    for i in range(1200):
        assert sorted(a[1][a[0][i]:a[0][i + 1]].tolist()) == sorted(b[1][b[0][i]:b[0][i + 1]].tolist())


def test_antisymmetry_net_internal_force_vanishes():
    w = W.uniform(n=3000, seed=5)
    s = O.State(w.x, w.y, w.z, w.diam)
    f, nz, _ = s.forces_of(O.make_params(R=12.0))
    scale = np.abs(f).sum()
    assert scale > 0 and nz.sum() > 100
    assert np.all(np.abs(f.sum(axis=1)) <= 1e-12 * scale)


def test_translation_invariance_is_bit_exact():
    rng = np.random.default_rng(9)
    # dyadic positions and a power-of-two box edge: the shift is exact
    p = np.round(rng.uniform(0, 128, (3, 1500)) * 2**20) / 2**20
    d = np.round(rng.uniform(12, 16, 1500) * 2**10) / 2**10
    P = O.make_params(R=16.0)
    f0, nz0, _ = _state(p, d).forces_of(P)
    f1, nz1, _ = _state(p + np.array([[1024.0], [-512.0], [4096.0]]), d).forces_of(P)
    assert np.array_equal(f0, f1) and np.array_equal(nz0, nz1)


def test_displacement_clamp_closed_form():
    # deep overlap and a large dt: |dt F| > dmax, so the step is exactly dmax
    p = np.array([[0.0, 2.0], [0.0, 0.0], [0.0, 0.0]])
    s = _state(p, np.array([10.0, 10.0]))
    P = O.make_params(R=12.0, dt=1.0, dmax=3.0)
    s.step(P)
    pos = s.positions()
    # |step| = dmax up to the two roundings of delta * (dmax / |delta|)
    assert abs(pos[0, 0] + 3.0) <= 2e-15 and abs(pos[0, 1] - 5.0) <= 2e-15
    assert np.all(pos[1:] == 0.0)
    # small dt: displacement = dt F exactly along the axis
    s = _state(p, np.array([10.0, 10.0]))
    s.step(O.make_params(R=12.0, dt=0.01, dmax=3.0))
    F = 2 * 8.0 - math.sqrt(2.5 * 8.0)
    assert abs(s.x[0] - (-0.01 * F)) < 1e-15 and abs(s.x[1] - (2.0 + 0.01 * F)) < 1e-15


def test_adherence_threshold_blocks_small_forces():
    p = np.array([[0.0, 9.0], [0.0, 0.0], [0.0, 0.0]])
    s = _state(p, np.array([10.0, 10.0]))
    s.step(O.make_params(R=12.0, adherence=0.5))  # |F| = 0.4189 <= 0.5
    assert s.x[:2].tolist() == [0.0, 9.0]
    s.step(O.make_params(R=12.0, adherence=0.4))
    assert s.x[0] < 0.0 and s.x[1] > 9.0


# --------------------------------------------------------------------------- grid / sort
def test_grid_geometry_margin_and_boxes():
    w = W.uniform(n=2000, seed=4)
    s = O.State(w.x, w.y, w.z, w.diam)
    P = O.make_params(R=12.0)
    bxyz, mort, lo, nb = s.grid(P)
    for d, a in enumerate((w.x, w.y, w.z)):
        assert lo[0, d] <= a.min() - 12.0 + 1e-9 and lo[0, d] % 12.0 == 0.0
        assert bxyz[:, d].min() >= 1 and bxyz[:, d].max() <= nb[0, d] - 2
        exp = np.floor((a - lo[0, d]) / 12.0).astype(np.int64)
        assert np.array_equal(bxyz[:, d], exp)


def test_sort_step_gives_morton_storage_order():
    w = W.uniform(n=3000, seed=6)
    s = O.State(w.x, w.y, w.z, w.diam)
    P = O.make_params(R=12.0, sort_every=1)
    perm = s.morton_order(P)
    uid_sorted = s.uid[perm].copy()
    codes = s.grid(P)[1][perm]
    assert np.all(np.diff(codes.astype(np.float64)) >= 0)
    # stable: equal codes keep ascending storage index
    same = codes[1:] == codes[:-1]
    assert np.all(np.diff(perm)[same] > 0)
    s.step(P)
    assert np.array_equal(s.uid[:3000], uid_sorted)


def test_ensemble_members_are_independent():
    w = W.ensemble(n_sims=4, seed=12, log_lo=2.0, log_hi=2.7, precision="fp64")
    P = O.make_params(R=10.0, dt=0.01)
    s = O.State(w.x, w.y, w.z, w.diam, sim_off=w.sim_off, dt_sim=w.dt_sim)
    s.step(P, 3)
    for k in range(4):
        a, b = w.sim_off[k], w.sim_off[k + 1]
        t = O.State(w.x[a:b], w.y[a:b], w.z[a:b], w.diam[a:b], uid=np.arange(a, b, dtype=np.uint64))
        t.step(O.make_params(R=10.0, dt=float(w.dt_sim[k])), 3)
        assert np.array_equal(t.positions(), s.positions()[:, a:b])


# --------------------------------------------------------------------------- static skip
def test_static_skip_trajectory_is_bit_exact():
    w = W.core_shell(n=6000, seed=5, precision="fp64")
    P_on = O.make_params(R=10.0, detect_static=1, walk_step=0.5, seed=5)
    P_off = O.make_params(R=10.0, detect_static=0, walk_step=0.5, seed=5)
    a = O.State(w.x, w.y, w.z, w.diam, beh=w.beh)
    b = O.State(w.x, w.y, w.z, w.diam, beh=w.beh)
    n_static = 0
    for _ in range(6):
        a.step(P_on)
        b.step(P_off)
        n_static += a.counters["n_static"]
        assert np.array_equal(a.positions(), b.positions())
        assert np.array_equal(a.nz[:a.n], b.nz[:b.n])
    assert n_static > 0.3 * 5 * w.n  # the core is skipped after the first step


def test_static_requires_history_and_clean_neighbourhood():
    # two isolated agents: one still, one walker far away; after one step the
    # still agent is static; a walker that comes close makes it non-static
    p = np.array([[0.0, 100.0], [0.0, 0.0], [0.0, 0.0]])
    beh = np.array([0, W.WALK], np.uint8)
    s = _state(p, np.array([10.0, 10.0]), beh=beh)
    P = O.make_params(R=10.0, detect_static=1, walk_step=0.5, seed=1)
    s.step(P)
    assert s.is_static[:2].tolist() == [0, 0]  # no history yet
    s.step(P)
    assert s.is_static[:2].tolist() == [1, 0]
    s.x[1] = 12.0
    s.step(P)  # history says agent 1 changed; its old box was far, its new box is adjacent
    assert s.is_static[0] == 0


# --------------------------------------------------------------------------- division
def test_division_invariants_and_order():
    w = W.lattice(m=4, steps=20)
    P = O.make_params(**{k: v for k, v in w.params.items() if k != "precision"})
    s = O.State(w.x, w.y, w.z, w.diam, beh=w.beh, cap=8 * w.n)
    pi = 3.141592653589793
    n_hist = []
    for t in range(20):
        n0 = s.n
        vol_before = s.vol[:n0].copy() + P.growth
        pos_before = None
        uid_before = s.uid[:n0].copy()
        s.step(P)
        n1 = s.n
        n_hist.append(n1)
        nd = n1 - n0
        assert s.counters["n_divided"] == nd
        if nd == 0:
            continue
        # daughters: uids next_uid - nd .. in parent storage order, appended
        mothers = np.nonzero(vol_before >= P.divide_volume)[0]
        assert len(mothers) == nd
        assert s.uid[n0:n1].tolist() == list(range(int(s.next_uid) - nd, int(s.next_uid)))
        assert np.array_equal(s.uid[:n0], uid_before)
        v1, v2 = s.vol[mothers], s.vol[n0:n1]
        assert np.allclose(v1 + v2, vol_before[mothers], rtol=4e-16, atol=0)
        ratio = v1 / v2
        assert np.all(ratio >= 0.9 - 1e-12) and np.all(ratio <= 1.1 + 1e-12)
        # diameters follow the volumes
        assert np.allclose(s.diam[n0:n1], np.cbrt(6 * v2 / pi), rtol=3e-16, atol=0)
    assert n_hist[-1] == 4 * w.n  # two rounds of division in 20 iterations
    assert n_hist[11] == w.n and n_hist[12] == 2 * w.n


def test_division_preserves_volume_weighted_centre():
    # a single dividing agent far from everything: no forces, so the
    # volume-weighted centre of mother + daughter equals the mother's centre
    p = np.array([[50.0], [60.0], [70.0]])
    v_div = (math.pi / 6) * 8000.0
    s = O.State(p[0], p[1], p[2], np.array([19.9]), vol=np.array([v_div - 100.0]),
                beh=np.array([W.GROW], np.uint8), cap=4)
    P = O.make_params(R=20.0, growth=300.0, divide_volume=v_div, seed=77)
    s.step(P)
    assert s.n == 2
    v = s.vol[:2]
    c = (v[0] * s.positions()[:, 0] + v[1] * s.positions()[:, 1]) / v.sum()
    assert np.allclose(c, p[:, 0], atol=1e-12)
    sep = np.linalg.norm(s.positions()[:, 0] - s.positions()[:, 1])
    assert abs(sep - O.cbrt(6 * (v_div + 200.0) / math.pi) / 2) < 1e-12


def test_static_condition_iv_at_most_one_contact():
    # Sec. 5 condition (iv): an agent with two non-zero contact forces is never
    # static, even when they cancel and nothing around it changes.  The
    # adherence threshold keeps all three collinear spheres still.
    p = np.array([[0.0, 9.0, 18.0], [5.0, 5.0, 5.0], [5.0, 5.0, 5.0]])
    s = _state(p, np.full(3, 10.0))
    P = O.make_params(R=12.0, detect_static=1, adherence=0.5)
    s.step(P)
    s.step(P)
    assert s.nz[:3].tolist() == [1, 2, 1]
    assert s.is_static[:3].tolist() == [1, 0, 1]
    assert s.x[:3].tolist() == [0.0, 9.0, 18.0]


def test_static_old_position_of_a_mover_is_dirty():
    # a walker that leaves the neighbourhood still makes its old box dirty
    p = np.array([[0.0, 100.0], [0.0, 0.0], [0.0, 0.0]])
    beh = np.array([0, W.WALK], np.uint8)
    s = _state(p, np.array([4.0, 4.0]), beh=beh)
    P = O.make_params(R=10.0, detect_static=1, walk_step=0.5, seed=3)
    s.step(P)
    s.step(P)
    assert s.is_static[0] == 1  # the walker is far away
    s.x[1] = 12.0
    s.step(P)
    assert s.is_static[0] == 0  # its new box is next door
    s.step(P)
    assert s.is_static[0] == 0  # it keeps walking next door
    s.x[1] = 100.0
    s.step(P)
    assert s.is_static[0] == 0  # it left, but its position before the last step was next door
    s.step(P)
    assert s.is_static[0] == 1


# --------------------------------------------------------------------------- tolerance bases
def _scale_lines():
    rows = []
    with open(os.path.join(GOLD, "pair_force_scales.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(float(v) for v in line.split()))
    return rows


@pytest.mark.parametrize("r1,r2,d,s_terms,s_pair", _scale_lines())
def test_tolerance_bases_two_spheres_hand_worked(r1, r2, d, s_terms, s_pair):
    # the two per-agent tolerance bases the oracle reports, against the
    # hand-worked single-contact values (both agents see the same contact)
    P = O.make_params(R=12.0)
    p = np.array([[10.0, 10.0 + d], [10.0, 10.0], [10.0, 10.0]])
    s = _state(p, np.array([2 * r1, 2 * r2]))
    _, nz, _, sc, sa = s.forces_of(P, with_scale=True, with_scale_abs=True)
    for a in range(2):
        assert sc[a] == pytest.approx(s_terms, rel=1e-15, abs=0.0)
        assert sa[a] == pytest.approx(s_pair, rel=1e-15, abs=0.0)


def test_tolerance_base_sums_magnitudes_not_the_vector():
    # middle of three collinear equal spheres: the forces cancel exactly, but
    # the pair-force magnitudes add
    P = O.make_params(R=12.0)
    p = np.array([[0.0, 9.0, 18.0], [5.0, 5.0, 5.0], [5.0, 5.0, 5.0]])
    s = _state(p, np.full(3, 10.0))
    f, _, _, sc, sa = s.forces_of(P, with_scale=True, with_scale_abs=True)
    assert f[:, 1].tolist() == [0.0, 0.0, 0.0]
    assert sa[1] == 2.0 * (2.0 - math.sqrt(2.5))
    assert sc[1] == 2.0 * (2.0 + math.sqrt(2.5))
    assert sa[0] == 2.0 - math.sqrt(2.5) and sa[2] == sa[0]


def test_tolerance_bases_equal_brute_force_sums():
    # every ordered pair enumerated in numpy (no grid), both bases summed over
    # the contacts of each agent, including adhesive pairs (F < 0)
    rng = np.random.default_rng(31)
    n = 400
    p = rng.uniform(0.0, 45.0, (3, n))
    d = rng.uniform(8.0, 12.0, n)
    P = O.make_params(R=12.0)
    _, nz, _, sc, sa = _state(p, d).forces_of(P, with_scale=True, with_scale_abs=True)
    diff = p[:, :, None] - p[:, None, :]
    dist = np.sqrt((diff ** 2).sum(axis=0))
    r = d * 0.5
    delta = r[:, None] + r[None, :] - dist
    mask = (dist < 12.0) & (delta > 0.0)
    np.fill_diagonal(mask, False)
    rbar = np.outer(r, r) / (r[:, None] + r[None, :])
    kd = 2.0 * np.where(mask, delta, 0.0)
    gs = np.sqrt(rbar * np.where(mask, delta, 0.0))
    assert np.array_equal(nz, mask.sum(axis=1))
    assert np.any(mask & (kd - gs < 0.0)) and np.any(mask & (kd - gs > 0.0))
    np.testing.assert_allclose(sc, np.where(mask, kd + gs, 0.0).sum(axis=1), rtol=1e-13, atol=0.0)
    np.testing.assert_allclose(sa, np.where(mask, np.abs(kd - gs), 0.0).sum(axis=1), rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------- parallel removal
def _removal_lines():
    rows = []
    with open(os.path.join(GOLD, "parallel_removal.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                a, b, c = (part.split() for part in line.split("|"))
                rows.append((int(a[0]), [int(v) for v in b], [int(v) for v in c]))
    return rows


@pytest.mark.parametrize("n,removed,ids", _removal_lines())
def test_parallel_removal_hand_worked(n, removed, ids):
    # ids as uids, and every other attribute tied to the id, so that a moved
    # agent is seen to move whole
    uid = np.arange(1, n + 1, dtype=np.uint64)
    p = np.stack([uid * 1.5, uid * 2.5, uid * 3.5]).astype(np.float64)
    s = _state(p, uid * 0.25 + 8.0, uid=uid, beh=(uid % 4).astype(np.uint8))
    rm = np.zeros(n, np.uint8)
    rm[removed] = 1
    moves = s.remove(rm)
    assert s.n == len(ids)
    assert s.uid[: s.n].tolist() == ids
    u = s.uid[: s.n].astype(np.float64)
    assert np.array_equal(s.positions(), np.stack([u * 1.5, u * 2.5, u * 3.5]))
    assert np.array_equal(s.diam[: s.n], u * 0.25 + 8.0)
    assert np.array_equal(s.beh[: s.n], (s.uid[: s.n] % 4).astype(np.uint8))
    assert moves == sum(1 for i in removed if i < len(ids))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_parallel_removal_invariants(seed):
    # random removal sets: the survivors are exactly the agents not removed,
    # every survivor left of the new size keeps its slot, the holes are filled
    # by survivors from the right in ascending order, and the number of moves
    # equals the number of holes (at most the number removed)
    rng = np.random.default_rng(seed)
    n = int(rng.integers(50, 400))
    uid = rng.permutation(n).astype(np.uint64) + 1000
    p = rng.uniform(0.0, 100.0, (3, n))
    s = _state(p, np.full(n, 10.0), uid=uid)
    rm = (rng.random(n) < rng.uniform(0.05, 0.6)).astype(np.uint8)
    moves = s.remove(rm)
    m = n - int(rm.sum())
    assert s.n == m
    assert sorted(s.uid[:m].tolist()) == sorted(uid[rm == 0].tolist())
    holes = [i for i in range(m) if rm[i]]
    tail = [i for i in range(m, n) if not rm[i]]
    assert moves == len(holes) == len(tail) <= int(rm.sum())
    for i in range(m):
        src = i if not rm[i] else tail[holes.index(i)]
        assert s.uid[i] == uid[src]
        assert np.array_equal(s.positions()[:, i], p[:, src])


def test_death_draw_rate_and_behaviour_bit():
    # only DIE agents are removed, at the requested rate (binomial bound),
    # and a removed agent's Philox draw is below the probability
    n = 20000
    rng = np.random.default_rng(9)
    p = rng.uniform(0.0, 4000.0, (3, n))  # sparse: no contacts
    beh = np.where(np.arange(n) % 2 == 0, 4, 0).astype(np.uint8)
    s = _state(p, np.full(n, 10.0), beh=beh)
    P = O.make_params(R=12.0, death_prob=0.1, seed=77)
    s.step(P)
    removed = set(range(n)) - set(s.uid[: s.n].tolist())
    assert all(i % 2 == 0 for i in removed)
    k = len(removed)
    mean, sd = 0.1 * n / 2, math.sqrt(n / 2 * 0.1 * 0.9)
    assert abs(k - mean) < 5 * sd
    assert s.counters["n_removed"] == k
    for i in list(removed)[:50]:
        assert O.uniform(77, i, 0, 3) < 0.1
    for i in [j for j in range(0, n, 2) if j not in removed][:50]:
        assert O.uniform(77, i, 0, 3) >= 0.1


def test_removal_with_static_skip_is_bit_exact_and_dirties_the_removed_box():
    # pairs of slightly overlapping agents whose force is below the
    # adherence: static with one contact.  When one of a pair dies, its box is
    # dirty next iteration, so its partner is recomputed (contacts 0) instead
    # of carrying its old contact count; skip == no-skip for positions and
    # contacts
    rng = np.random.default_rng(4)
    g = np.arange(8) * 40.0
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    c = np.stack([x.ravel(), y.ravel(), z.ravel()]) + 100.0
    m = c.shape[1]
    off = np.array([[9.99], [0.0], [0.0]])
    p = np.concatenate([c, c + off], axis=1)
    n = p.shape[1]
    beh = np.concatenate([np.full(m, 4, np.uint8), np.zeros(m, np.uint8)])
    P_skip = O.make_params(R=12.0, adherence=1.0, detect_static=1, death_prob=0.2, seed=5)
    P_full = O.make_params(R=12.0, adherence=1.0, detect_static=0, death_prob=0.2, seed=5)
    a = _state(p, np.full(n, 10.0), beh=beh)
    b = _state(p, np.full(n, 10.0), beh=beh)
    partner_freed = 0
    for t in range(6):
        a.step(P_skip)
        b.step(P_full)
        assert np.array_equal(a.uid[: a.n], b.uid[: b.n])
        assert np.array_equal(a.positions(), b.positions())
        assert np.array_equal(a.nz[: a.n], b.nz[: b.n]), "contacts differ after step %d" % (t + 1)
        partner_freed += int(((b.nz[: b.n] == 0) & (b.uid[: b.n] >= m)).sum())
    assert a.counters["n_static"] > 0 and partner_freed > 0


# --------------------------------------------------------------------------- heterotypic adhesion
TYPE_K = [[2.0, 1.5], [1.5, 3.0]]
TYPE_GAMMA = [[1.0, 0.5], [0.5, 2.0]]


def _hetero_lines():
    rows = []
    with open(os.path.join(GOLD, "heterotypic_pair_forces.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                v = line.split()
                rows.append((int(v[0]), int(v[1])) + tuple(float(x) for x in v[2:]))
    return rows


@pytest.mark.parametrize("t1,t2,r1,r2,d,F", _hetero_lines())
def test_heterotypic_two_spheres_hand_worked(t1, t2, r1, r2, d, F):
    P = O.make_params(R=12.0, type_k=TYPE_K, type_gamma=TYPE_GAMMA)
    u = np.array([2.0, -1.0, 2.0]) / 3.0
    p = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0] + d * u]).T
    beh = np.array([t1 << 4, t2 << 4], np.uint8)
    f, nz, _ = _state(p, np.array([2 * r1, 2 * r2]), beh=beh).forces_of(P)
    assert nz.tolist() == [1, 1]
    assert np.allclose(f[:, 0], -F * u, rtol=0, atol=1e-14)
    assert np.allclose(f[:, 1], F * u, rtol=0, atol=1e-14)


def test_uniform_type_table_equals_one_type_bit_exact():
    # every type pair given the one-type constants: the same forces, bit for bit
    rng = np.random.default_rng(12)
    n = 1500
    p = rng.normal(60.0, 10.0, (3, n))
    d = rng.uniform(8.0, 12.0, n)
    beh = (rng.integers(0, 4, n) << 4).astype(np.uint8)
    s = _state(p, d, beh=beh)
    f1, nz1, _ = s.forces_of(O.make_params(R=12.0))
    f4, nz4, _ = s.forces_of(O.make_params(R=12.0, type_k=np.full((4, 4), 2.0), type_gamma=np.full((4, 4), 1.0)))
    assert np.array_equal(f1, f4) and np.array_equal(nz1, nz4) and nz1.sum() > 0


def test_heterotypic_antisymmetry_and_type_dependence():
    # a symmetric table keeps the pair forces antisymmetric (net internal force
    # vanishes); swapping which agents carry which type changes the forces
    rng = np.random.default_rng(13)
    n = 800
    p = rng.normal(50.0, 8.0, (3, n))
    d = rng.uniform(8.0, 12.0, n)
    beh = (rng.integers(0, 2, n) << 4).astype(np.uint8)
    P = O.make_params(R=12.0, type_k=TYPE_K, type_gamma=TYPE_GAMMA)
    f, nz, _ = _state(p, d, beh=beh).forces_of(P)
    scale = np.abs(f).sum()
    assert np.abs(f.sum(axis=1)).max() <= 1e-12 * scale
    f_sw, _, _ = _state(p, d, beh=(beh ^ 0x10).astype(np.uint8)).forces_of(P)
    assert not np.array_equal(f, f_sw) and nz.sum() > 0


# --------------------------------------------------------------------------- timing build
def test_openmp_timing_build_gives_the_same_bits():
    # the CPU baseline's parallel build of the oracle: each agent's sum stays
    # serial, so a trajectory with static skip, removal and a sort step is
    # bit-identical to the serial build's
    from oracle import build_oracle
    lib = build_oracle.build_omp()
    if lib is None:
        pytest.skip("no OpenMP in this compiler")
    w = W.core_shell(n=6000, seed=5, precision="fp64")
    w.beh = (w.beh | np.where(np.arange(w.n) % 5 == 0, 4, 0)).astype(np.uint8)
    P = O.make_params(R=10.0, detect_static=1, walk_step=0.5, sort_every=3, death_prob=0.05, seed=5)
    a = _state(np.stack([w.x, w.y, w.z]), w.diam, beh=w.beh)
    a.step(P, 5)
    with O.use_library(lib) as L:
        assert L.orc_threads() >= 1
        b = _state(np.stack([w.x, w.y, w.z]), w.diam, beh=w.beh)
        b.step(P, 5)
    assert np.array_equal(a.uid[: a.n], b.uid[: b.n])
    assert np.array_equal(a.positions(), b.positions())
    assert np.array_equal(a.nz[: a.n], b.nz[: b.n])


# --------------------------------------------------------------------------- Hilbert order (Sec. 4.2)
def _hilbert_order1():
    rows = []
    with open(os.path.join(GOLD, "hilbert_order1.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


def test_hilbert_first_order_hand_worked():
    for h, x, y, z in _hilbert_order1():
        assert O.hilbert3(x, y, z, 1) == h


@pytest.mark.parametrize("bits", [2, 3, 4])
def test_hilbert_is_a_face_adjacent_bijection(bits):
    # the defining properties of a Hilbert curve on a 2^bits cube: every
    # cell gets a distinct index in [0, 8^bits), the curve starts at the
    # origin, consecutive cells share a face, and every aligned 2^j sub-cube
    # is a contiguous run of indices
    n = 1 << bits
    idx = {}
    for x in range(n):
        for y in range(n):
            for z in range(n):
                idx[O.hilbert3(x, y, z, bits)] = (x, y, z)
    assert sorted(idx) == list(range(n ** 3))
    assert idx[0] == (0, 0, 0)
    for h in range(n ** 3 - 1):
        a, b = idx[h], idx[h + 1]
        assert sum(abs(a[d] - b[d]) for d in range(3)) == 1, (h, a, b)
    for j in range(1, bits):
        s = 1 << j
        for h0 in range(0, n ** 3, s ** 3):
            corners = {tuple(c // s for c in idx[h]) for h in range(h0, h0 + s ** 3)}
            assert len(corners) == 1


def test_hilbert_sort_step_order():
    # the sort step in Hilbert mode: agents grouped by brick (4x4x4 boxes) in
    # the bricks' Hilbert order, by box Morton code inside a brick, stable;
    # checked against a direct restatement over the oracle's own boxes
    w = W.uniform(n=3000, seed=9, edge=400.0)
    s = O.State(w.x, w.y, w.z, w.diam)
    P = O.make_params(R=12.0, curve=1)
    bxyz, _, lo, nb = s.grid(P)
    nr = [(int(v) + 3) // 4 for v in nb[0]]
    bits = max(int(np.ceil(np.log2(max(nr)))), 0)
    keys = [(O.hilbert3(int(b[0]) >> 2, int(b[1]) >> 2, int(b[2]) >> 2, bits) << 6 |
             O.morton3(int(b[0]) & 3, int(b[1]) & 3, int(b[2]) & 3), i) for i, b in enumerate(bxyz)]
    expect = [i for _, i in sorted(keys)]
    assert s.curve_order(P).tolist() == expect
    assert s.curve_order(O.make_params(R=12.0)).tolist() == s.morton_order(O.make_params(R=12.0)).tolist()
    # a sort step stores the agents in that order
    s.step(O.make_params(R=12.0, curve=1, sort_every=1, dt=0.0))
    assert s.uid[: s.n].tolist() == expect
