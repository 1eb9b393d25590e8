"""ctypes wrapper of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import this module; the product library
never does.  It holds no CUDA code and imports nothing from the package's
CUDA binding.
"""
import ctypes as C
import os

import numpy as np

from . import build_oracle

_lib = None


class use_library:
    """Temporarily route every oracle call to another build of oracle.c
    (used by the tests that plant a mistake in a copy of the oracle)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = _lib
        _lib = C.CDLL(self.path)
        _declare(_lib)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


class Params(C.Structure):
    _fields_ = [
        ("R", C.c_double), ("L", C.c_double), ("dt", C.c_double), ("dmax", C.c_double),
        ("k", C.c_double), ("gamma", C.c_double), ("adherence", C.c_double),
        ("detect_static", C.c_int32), ("sort_every", C.c_int32),
        ("growth", C.c_double), ("divide_volume", C.c_double),
        ("ratio_lo", C.c_double), ("ratio_hi", C.c_double), ("walk_step", C.c_double),
        ("seed", C.c_uint64), ("death_prob", C.c_double), ("n_types", C.c_int32), ("curve", C.c_int32),
        ("type_k", C.c_double * 16), ("type_gamma", C.c_double * 16),
    ]


_P = C.POINTER


class _State(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("cap", C.c_int64), ("n_sims", C.c_int32), ("history_valid", C.c_int32),
        ("x", _P(C.c_double)), ("y", _P(C.c_double)), ("z", _P(C.c_double)),
        ("diam", _P(C.c_double)), ("vol", _P(C.c_double)),
        ("uid", _P(C.c_uint64)), ("beh", _P(C.c_uint8)), ("sim_off", _P(C.c_int64)),
        ("dt_sim", _P(C.c_double)),
        ("changed", _P(C.c_uint8)), ("nz", _P(C.c_int32)),
        ("px", _P(C.c_double)), ("py", _P(C.c_double)), ("pz", _P(C.c_double)),
        ("step", C.c_int64), ("next_uid", C.c_uint64),
        ("fx", _P(C.c_double)), ("fy", _P(C.c_double)), ("fz", _P(C.c_double)),
        ("is_static", _P(C.c_uint8)),
        ("n_divided", C.c_int64), ("n_static", C.c_int64), ("n_coincident", C.c_int64),
        ("gx", _P(C.c_double)), ("gy", _P(C.c_double)), ("gz", _P(C.c_double)),
        ("n_ghost", C.c_int64), ("n_removed", C.c_int64),
    ]


def _declare(L):
    SP = C.POINTER(_State)
    PP = C.POINTER(Params)
    vp = C.c_void_p
    L.orc_step.argtypes = [SP, PP]
    L.orc_step.restype = C.c_int
    L.orc_grid.argtypes = [SP, PP, vp, vp, vp, vp]
    L.orc_grid.restype = C.c_int
    L.orc_morton_order.argtypes = [SP, PP, vp]
    L.orc_morton_order.restype = C.c_int
    L.orc_neighbors.argtypes = [SP, PP, vp, vp, C.c_int64]
    L.orc_neighbors.restype = C.c_int64
    L.orc_neighbors_brute.argtypes = [SP, PP, vp, vp, C.c_int64]
    L.orc_neighbors_brute.restype = C.c_int64
    L.orc_forces.argtypes = [SP, PP, C.c_int64, vp, vp, vp, vp, vp, vp]
    L.orc_forces.restype = C.c_int
    L.orc_philox4x64_10.argtypes = [vp, vp, vp]
    L.orc_philox4x64_10.restype = None
    L.orc_cbrt.argtypes = [C.c_double]
    L.orc_cbrt.restype = C.c_double
    L.orc_unit_vector.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, vp]
    L.orc_unit_vector.restype = None
    L.orc_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64]
    L.orc_uniform.restype = C.c_double
    L.orc_morton3.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
    L.orc_morton3.restype = C.c_uint64
    L.orc_morton2.argtypes = [C.c_uint64, C.c_uint64]
    L.orc_morton2.restype = C.c_uint64
    L.orc_threads.argtypes = []
    L.orc_threads.restype = C.c_int
    L.orc_curve_order.argtypes = [SP, PP, vp]
    L.orc_curve_order.restype = C.c_int
    L.orc_hilbert3.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_int]
    L.orc_hilbert3.restype = C.c_uint64
    L.orc_remove.argtypes = [SP, vp]
    L.orc_remove.restype = C.c_int64
    L.orc_morton_offsets.argtypes = [C.c_int32, vp, vp, vp, C.c_int64]
    L.orc_morton_offsets.restype = C.c_int64


DEFAULTS = dict(R=12.0, L=0.0, dt=0.01, dmax=3.0, k=2.0, gamma=1.0, adherence=0.0,
                detect_static=0, sort_every=0, growth=0.0, divide_volume=0.0,
                ratio_lo=0.9, ratio_hi=1.1, walk_step=0.0, seed=0, death_prob=0.0, curve=0)


def make_params(**kw) -> Params:
    """Oracle parameters; type_k / type_gamma (n_types x n_types nested
    lists or arrays) set the per-type-pair force constants."""
    d = dict(DEFAULTS)
    for k, v in kw.items():
        if k in d:
            d[k] = v
    if not d["L"]:
        d["L"] = d["R"]
    p = Params()
    for k, v in d.items():
        setattr(p, k, v)
    if kw.get("type_k") is not None:
        tk, tg = np.asarray(kw["type_k"], np.float64), np.asarray(kw["type_gamma"], np.float64)
        p.n_types = tk.shape[0]
        for a in range(tk.shape[0]):
            for b in range(tk.shape[1]):
                p.type_k[4 * a + b] = tk[a, b]
                p.type_gamma[4 * a + b] = tg[a, b]
    return p


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class State:
    """Agent state in numpy arrays (storage order) plus the oracle's history."""

    def __init__(self, x, y, z, diam, vol=None, uid=None, beh=None, sim_off=None, dt_sim=None,
                 step=0, next_uid=None, cap=None):
        n = len(x)
        cap = max(n, cap or n, 1)
        self.cap = cap

        def arr(v, dtype, fill=0):
            a = np.full(cap, fill, dtype=dtype)
            if v is not None:
                a[:n] = np.asarray(v, dtype=dtype)
            return a

        self.x, self.y, self.z = arr(x, np.float64), arr(y, np.float64), arr(z, np.float64)
        self.diam = arr(diam, np.float64)
        if vol is None:
            d = np.asarray(diam, dtype=np.float64)
            vol = (np.pi / 6.0) * d * d * d
        self.vol = arr(vol, np.float64)
        self.uid = arr(np.arange(n, dtype=np.uint64) if uid is None else uid, np.uint64)
        self.beh = arr(beh, np.uint8)
        self.sim_off = np.array([0, n] if sim_off is None else sim_off, dtype=np.int64)
        self.dt_sim = None if dt_sim is None else np.ascontiguousarray(dt_sim, dtype=np.float64)
        self.changed = np.zeros(cap, np.uint8)
        self.nz = np.zeros(cap, np.int32)
        self.px, self.py, self.pz = self.x.copy(), self.y.copy(), self.z.copy()
        self.fx, self.fy, self.fz = np.zeros(cap), np.zeros(cap), np.zeros(cap)
        self.is_static = np.zeros(cap, np.uint8)
        self.gx, self.gy, self.gz = np.zeros(cap), np.zeros(cap), np.zeros(cap)
        self._s = _State()
        s = self._s
        s.n, s.cap, s.n_sims, s.history_valid = n, cap, len(self.sim_off) - 1, 0
        s.step = step
        s.next_uid = n if next_uid is None else next_uid
        for name in ("x", "y", "z", "diam", "vol", "px", "py", "pz", "fx", "fy", "fz", "gx", "gy", "gz"):
            setattr(s, name, getattr(self, name).ctypes.data_as(C.POINTER(C.c_double)))
        s.uid = self.uid.ctypes.data_as(C.POINTER(C.c_uint64))
        s.beh = self.beh.ctypes.data_as(C.POINTER(C.c_uint8))
        s.sim_off = self.sim_off.ctypes.data_as(C.POINTER(C.c_int64))
        s.dt_sim = (self.dt_sim.ctypes.data_as(C.POINTER(C.c_double)) if self.dt_sim is not None
                    else C.POINTER(C.c_double)())
        s.changed = self.changed.ctypes.data_as(C.POINTER(C.c_uint8))
        s.nz = self.nz.ctypes.data_as(C.POINTER(C.c_int32))
        s.is_static = self.is_static.ctypes.data_as(C.POINTER(C.c_uint8))

    # -- views ---------------------------------------------------------------
    @property
    def n(self):
        return self._s.n

    @property
    def step_count(self):
        return self._s.step

    @property
    def next_uid(self):
        return self._s.next_uid

    @property
    def counters(self):
        s = self._s
        return dict(n_divided=s.n_divided, n_static=s.n_static, n_coincident=s.n_coincident,
                    n_removed=s.n_removed)

    def positions(self):
        n = self.n
        return np.stack([self.x[:n], self.y[:n], self.z[:n]])

    def forces(self):
        n = self.n
        return np.stack([self.fx[:n], self.fy[:n], self.fz[:n]])

    # -- calls -----------------------------------------------------------------
    def step(self, params: Params, n_steps: int = 1):
        L = lib()
        for _ in range(n_steps):
            rc = L.orc_step(C.byref(self._s), C.byref(params))
            if rc != 0:
                raise RuntimeError("orc_step failed: %d" % rc)

    def remove(self, rm):
        """Remove the agents flagged in rm (length n) by the parallel-removal
        steps of Sec. 3.2; returns the number of agents moved."""
        r = np.zeros(max(self.n, 1), np.uint8)
        r[: self.n] = np.asarray(rm, dtype=np.uint8)[: self.n]
        m = lib().orc_remove(C.byref(self._s), _ptr(r))
        if m < 0:
            raise RuntimeError("orc_remove failed: %d" % m)
        self.sim_off[-1] = self.n
        return int(m)

    def grid(self, params: Params):
        n = self.n
        ns = self._s.n_sims
        bxyz = np.zeros((max(n, 1), 3), np.int64)
        mort = np.zeros(max(n, 1), np.uint64)
        lo = np.zeros((ns, 3))
        nb = np.zeros((ns, 3), np.int64)
        rc = lib().orc_grid(C.byref(self._s), C.byref(params), _ptr(bxyz), _ptr(mort), _ptr(lo), _ptr(nb))
        if rc != 0:
            raise RuntimeError("orc_grid failed: %d" % rc)
        return bxyz[:n], mort[:n], lo, nb

    def morton_order(self, params: Params):
        perm = np.zeros(max(self.n, 1), np.int64)
        rc = lib().orc_morton_order(C.byref(self._s), C.byref(params), _ptr(perm))
        if rc != 0:
            raise RuntimeError("orc_morton_order failed: %d" % rc)
        return perm[: self.n]

    def curve_order(self, params: Params):
        """Storage order of a sort step for params.curve (0 Morton, 1 Hilbert
        over the 4x4x4-box bricks, Morton inside a brick)."""
        perm = np.zeros(max(self.n, 1), np.int64)
        rc = lib().orc_curve_order(C.byref(self._s), C.byref(params), _ptr(perm))
        if rc != 0:
            raise RuntimeError("orc_curve_order failed: %d" % rc)
        return perm[: self.n]

    def _csr(self, fn, params):
        n = self.n
        off = np.zeros(n + 1, np.int64)
        cap = 1 << 16
        while True:
            nbr = np.zeros(cap, np.int64)
            total = fn(C.byref(self._s), C.byref(params), _ptr(off), _ptr(nbr), cap)
            if total < 0:
                raise RuntimeError("neighbour enumeration failed: %d" % total)
            if total <= cap:
                return off, nbr[:total]
            cap = int(total)

    def neighbors(self, params: Params):
        return self._csr(lib().orc_neighbors, params)

    def neighbors_brute(self, params: Params):
        return self._csr(lib().orc_neighbors_brute, params)

    def forces_of(self, params: Params, q=None, with_scale=False, with_scale_abs=False):
        """Forces (3 x nq), contacts and neighbours of the agents q (all when
        None); with_scale adds the sum of the force terms' magnitudes, and
        with_scale_abs the sum of the pair-force magnitudes, per agent."""
        nq = self.n if q is None else len(q)
        qa = None if q is None else np.ascontiguousarray(q, dtype=np.int64)
        f = np.zeros((3, max(nq, 1)))
        nz = np.zeros(max(nq, 1), np.int32)
        nnb = np.zeros(max(nq, 1), np.int32)
        sc = np.zeros(max(nq, 1))
        sa = np.zeros(max(nq, 1))
        rc = lib().orc_forces(C.byref(self._s), C.byref(params), nq, _ptr(qa), _ptr(f), _ptr(nz), _ptr(nnb),
                              _ptr(sc), _ptr(sa))
        if rc != 0:
            raise RuntimeError("orc_forces failed: %d" % rc)
        out = [f[:, :nq], nz[:nq], nnb[:nq]]
        if with_scale:
            out.append(sc[:nq])
        if with_scale_abs:
            out.append(sa[:nq])
        return tuple(out)


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def cbrt(x: float) -> float:
    return lib().orc_cbrt(float(x))


def unit_vector(seed, uid, step, purpose):
    out = np.zeros(3)
    lib().orc_unit_vector(seed, uid, step, purpose, _ptr(out))
    return out


def uniform(seed, uid, step, purpose):
    return lib().orc_uniform(seed, uid, step, purpose)


def morton3(x, y, z):
    return int(lib().orc_morton3(x, y, z))


def hilbert3(x, y, z, bits):
    return int(lib().orc_hilbert3(x, y, z, bits))


def morton2(x, y):
    return int(lib().orc_morton2(x, y))


def morton_offsets(dims):
    D = len(dims)
    n = np.ascontiguousarray(dims, dtype=np.int64)
    cap = 1 << 12
    while True:
        bc = np.zeros(cap, np.int64)
        of = np.zeros(cap, np.int64)
        m = lib().orc_morton_offsets(D, _ptr(n), _ptr(bc), _ptr(of), cap)
        if m < 0:
            raise RuntimeError("orc_morton_offsets failed")
        if m <= cap:
            return list(zip(bc[:m].tolist(), of[:m].tolist()))
        cap = int(m)
