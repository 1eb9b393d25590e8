"""Python binding of the C ABI in include/bdm.h (argument marshalling only).

Every step of the mechanical-interaction iteration runs in the CUDA library
libbdm_gb300.so; this module only converts numpy arrays (host memory) or torch
CUDA tensors (device memory) into pointers and sizes.  There is no fallback:
if the library cannot be built or loaded, the first call raises.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

BDM_OK, BDM_EINVAL, BDM_ENOMEM, BDM_ECUDA, BDM_ECAPACITY, BDM_ETIMEOUT, BDM_ESTATE = 0, -1, -2, -3, -4, -5, -6
BDM_FP64, BDM_FP32_FORCE = 0, 1
BDM_HOST, BDM_DEVICE = 0, 1
CURVE_MORTON, CURVE_HILBERT = 0, 1
BEH_GROW, BEH_WALK, BEH_DIE = 1, 2, 4
TYPE_SHIFT = 4  # bits 4-5 of the behaviour byte: the agent's type
DBG_FORCES, DBG_NZ, DBG_STATIC, DBG_GRID_BOX, DBG_GRID_ORDER = 1, 2, 3, 4, 5
DBG_GRID_GEOMETRY, DBG_BRICK_RANK, DBG_NEIGHBORS, DBG_FORCES_NOW = 6, 7, 8, 9

_ERRNAMES = {-1: "BDM_EINVAL", -2: "BDM_ENOMEM", -3: "BDM_ECUDA", -4: "BDM_ECAPACITY", -5: "BDM_ETIMEOUT",
             -6: "BDM_ESTATE"}


class BdmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_ERRNAMES.get(code, code), msg))
        self.code = code


class Params(C.Structure):
    _fields_ = [
        ("interaction_radius", C.c_double), ("box_edge", C.c_double), ("dt", C.c_double),
        ("max_displacement", C.c_double), ("k", C.c_double), ("gamma", C.c_double), ("adherence", C.c_double),
        ("precision", C.c_int32), ("detect_static", C.c_int32), ("sort_every", C.c_int32), ("n_sims", C.c_int32),
        ("dt_per_sim", C.POINTER(C.c_double)), ("seed", C.c_uint64),
        ("growth_per_step", C.c_double), ("divide_volume", C.c_double), ("ratio_lo", C.c_double),
        ("ratio_hi", C.c_double), ("walk_step", C.c_double), ("capacity", C.c_int64),
        ("keep_forces", C.c_int32), ("reserved", C.c_int32), ("death_prob", C.c_double),
        ("n_types", C.c_int32), ("curve", C.c_int32), ("type_k", C.c_double * 16),
        ("type_gamma", C.c_double * 16),
    ]


class Tuning(C.Structure):
    _fields_ = [("box_edge", C.c_double), ("ms_per_step", C.c_double), ("lanes", C.c_int32),
                ("sort_every", C.c_int32), ("n_trials", C.c_int32), ("reserved", C.c_int32)]


TUNE_BOX_EDGE, TUNE_LANES, TUNE_SORT = 1, 2, 4


class Counters(C.Structure):
    _fields_ = [
        ("n_agents", C.c_int64), ("step", C.c_int64), ("next_uid", C.c_uint64), ("n_static", C.c_int64),
        ("n_moved", C.c_int64), ("n_divided", C.c_int64), ("n_candidates", C.c_int64),
        ("n_neighbors", C.c_int64), ("n_contacts", C.c_int64), ("n_exact_fallback", C.c_int64),
        ("n_boxes", C.c_int64), ("n_bricks", C.c_int64), ("n_occupied_bricks", C.c_int64),
        ("max_brick_agents", C.c_int64), ("kernels_launched", C.c_int64), ("history_valid", C.c_int32),
        ("error", C.c_int32), ("n_removed", C.c_int64), ("n_fp64_fixup", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None

# exported symbols and their signatures (the set include/bdm.h declares)
SIGNATURES = {
    "bdm_create": (C.c_int, [C.POINTER(Params), C.c_void_p, C.POINTER(C.c_void_p)]),
    "bdm_set_agents": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64, C.c_int]),
    "bdm_step": (C.c_int, [C.c_void_p, C.c_int]),
    "bdm_sort": (C.c_int, [C.c_void_p]),
    "bdm_get_agents": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "bdm_get_counters": (C.c_int, [C.c_void_p, C.POINTER(Counters)]),
    "bdm_get_debug": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "bdm_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bdm_destroy": (None, [C.c_void_p]),
    "bdm_last_error": (C.c_char_p, [C.c_void_p]),
    "bdm_version": (C.c_int, []),
    "bdm_profile_begin": (C.c_int, [C.c_void_p]),
    "bdm_profile_end": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "bdm_phase_name": (C.c_char_p, [C.c_int]),
    "bdm_forces_noalloc": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bdm_noalloc_last_error": (C.c_char_p, []),
    "bdm_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(Tuning)]),
    "bdm_set_force_kernel": (C.c_int, [C.c_void_p, C.c_int]),
}


def library_path():
    return _build.LIB


def lib():
    """Load (building first if needed) the CUDA library; raises if impossible."""
    global _LIB
    if _LIB is None:
        # BDM_LIBRARY selects an already built library (for example a build
        # variant); otherwise the in-tree library is built if stale
        path = os.environ.get("BDM_LIBRARY") or _build.build()
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is missing" % path)
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _current_stream_handle():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Simulation:
    """One simulation (or one batched ensemble) living on the current GPU.

    Parameters follow bdm_params; `precision` is "fp64" or "fp32"."""

    def __init__(self, R, capacity, box_edge=0.0, dt=0.01, dmax=3.0, k=2.0, gamma=1.0, adherence=0.0,
                 precision="fp64", detect_static=False, sort_every=0, n_sims=1, dt_per_sim=None, seed=0,
                 growth=0.0, divide_volume=0.0, ratio_lo=0.9, ratio_hi=1.1, walk_step=0.0, keep_forces=False,
                 death_prob=0.0, type_k=None, type_gamma=None, curve=0, stream=None):
        L = lib()
        p = Params()
        p.interaction_radius = R
        p.box_edge = box_edge
        p.dt = dt
        p.max_displacement = dmax
        p.k = k
        p.gamma = gamma
        p.adherence = adherence
        p.precision = BDM_FP64 if precision in ("fp64", BDM_FP64) else BDM_FP32_FORCE
        p.detect_static = int(bool(detect_static))
        p.sort_every = int(sort_every)
        p.n_sims = int(n_sims)
        self._dt = None
        if dt_per_sim is not None:
            self._dt = np.ascontiguousarray(dt_per_sim, dtype=np.float64)
            p.dt_per_sim = self._dt.ctypes.data_as(C.POINTER(C.c_double))
        p.seed = seed
        p.growth_per_step = growth
        p.divide_volume = divide_volume
        p.ratio_lo = ratio_lo
        p.ratio_hi = ratio_hi
        p.walk_step = walk_step
        p.capacity = int(capacity)
        p.keep_forces = int(bool(keep_forces))
        p.death_prob = death_prob
        p.curve = int(curve)
        if type_k is not None:
            tk, tg = np.asarray(type_k, np.float64), np.asarray(type_gamma, np.float64)
            p.n_types = tk.shape[0]
            for a in range(tk.shape[0]):
                for b in range(tk.shape[1]):
                    p.type_k[4 * a + b] = tk[a, b]
                    p.type_gamma[4 * a + b] = tg[a, b]
        self.params = p
        self.n_sims = int(n_sims)
        self.precision = p.precision
        h = C.c_void_p()
        st = stream if stream is not None else self._default_stream()
        rc = L.bdm_create(C.byref(p), st, C.byref(h))
        if rc != 0:
            raise BdmError(rc, L.bdm_last_error(None).decode())
        self._h = h

    @staticmethod
    def _default_stream():
        try:
            import torch
            if torch.cuda.is_available():
                return _current_stream_handle()
        except ImportError:
            pass
        return C.c_void_p(0)

    @classmethod
    def from_workload(cls, w, capacity=None, **over):
        p = dict(w.params)
        kw = dict(R=p["R"], box_edge=p.get("L", 0.0), dt=p.get("dt", 0.01), dmax=p.get("dmax", 3.0),
                  k=p.get("k", 2.0), gamma=p.get("gamma", 1.0), adherence=p.get("adherence", 0.0),
                  precision=p.get("precision", "fp64"), detect_static=p.get("detect_static", 0),
                  sort_every=p.get("sort_every", 0), n_sims=w.n_sims, dt_per_sim=w.dt_sim,
                  seed=p.get("seed", 0), growth=p.get("growth", 0.0), divide_volume=p.get("divide_volume", 0.0),
                  ratio_lo=p.get("ratio_lo", 0.9), ratio_hi=p.get("ratio_hi", 1.1),
                  walk_step=p.get("walk_step", 0.0), death_prob=p.get("death_prob", 0.0),
                  type_k=p.get("type_k"), type_gamma=p.get("type_gamma"), curve=p.get("curve", 0))
        kw.update(over)
        return cls(capacity=capacity or w.n, **kw)

    def _check(self, rc):
        if rc != 0:
            raise BdmError(rc, lib().bdm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().bdm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._check(lib().bdm_set_stream(self._h, stream))

    # ------------------------------------------------------------------ state
    def set_agents(self, x, y, z, diam, vol=None, uid=None, beh=None, sim_off=None, step=0, next_uid=None):
        n = len(x)
        if next_uid is None:
            next_uid = n
        if _is_torch(x):
            import torch
            xyz = torch.stack([x, y, z]).to(torch.float64).contiguous()
            d = diam.to(torch.float64).contiguous()
            v = vol.to(torch.float64).contiguous() if vol is not None else None
            u = uid.contiguous() if uid is not None else None
            b = beh.to(torch.uint8).contiguous() if beh is not None else None
            so = (torch.as_tensor(sim_off, dtype=torch.int64, device=x.device).contiguous()
                  if sim_off is not None else None)
            self._keep = (xyz, d, v, u, b, so)
            ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
            self.set_stream(_current_stream_handle())
            rc = lib().bdm_set_agents(self._h, n, ptr(xyz), ptr(d), ptr(v), ptr(u), ptr(b), ptr(so), step, next_uid,
                                      BDM_DEVICE)
        else:
            xyz = np.ascontiguousarray(np.stack([np.asarray(x), np.asarray(y), np.asarray(z)]), dtype=np.float64)
            d = np.ascontiguousarray(diam, dtype=np.float64)
            v = None if vol is None else np.ascontiguousarray(vol, dtype=np.float64)
            u = None if uid is None else np.ascontiguousarray(uid, dtype=np.uint64)
            b = None if beh is None else np.ascontiguousarray(beh, dtype=np.uint8)
            so = None if sim_off is None else np.ascontiguousarray(sim_off, dtype=np.int64)
            ptr = lambda a: a.ctypes.data_as(C.c_void_p) if a is not None else None
            rc = lib().bdm_set_agents(self._h, n, ptr(xyz), ptr(d), ptr(v), ptr(u), ptr(b), ptr(so), step, next_uid,
                                      BDM_HOST)
        self._check(rc)

    def set_workload(self, w):
        self.set_agents(w.x, w.y, w.z, w.diam, beh=w.beh, sim_off=w.sim_off)

    def step(self, n=1):
        self._check(lib().bdm_step(self._h, int(n)))

    def sort(self):
        self._check(lib().bdm_sort(self._h))

    def counters(self):
        c = Counters()
        self._check(lib().bdm_get_counters(self._h, C.byref(c)))
        return c.as_dict()

    @property
    def n(self):
        return self.counters()["n_agents"]

    def get_agents(self, device=False):
        """State in storage order: numpy arrays (host) or torch tensors (device)."""
        n = self.n
        if device:
            import torch
            dev = torch.device("cuda")
            xyz = torch.empty((3, max(n, 1)), dtype=torch.float64, device=dev)
            d = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
            u = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
            b = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
            so = torch.empty(self.n_sims + 1, dtype=torch.int64, device=dev)
            nout, st, nu = C.c_int64(), C.c_int64(), C.c_uint64()
            self.set_stream(_current_stream_handle())
            ptr = lambda t: C.c_void_p(t.data_ptr())
            rc = lib().bdm_get_agents(self._h, max(n, 1), ptr(xyz), ptr(d), None, ptr(u), ptr(b), ptr(so),
                                      C.byref(nout), C.byref(st), C.byref(nu), BDM_DEVICE)
            self._check(rc)
            return dict(x=xyz[0, :n], y=xyz[1, :n], z=xyz[2, :n], diam=d[:n], uid=u[:n], beh=b[:n], sim_off=so,
                        n=nout.value, step=st.value, next_uid=nu.value)
        cap = max(n, 1)
        xyz = np.zeros((3, cap))
        d = np.zeros(cap)
        v = np.zeros(cap)
        u = np.zeros(cap, np.uint64)
        b = np.zeros(cap, np.uint8)
        so = np.zeros(self.n_sims + 1, np.int64)
        nout, st, nu = C.c_int64(), C.c_int64(), C.c_uint64()
        ptr = lambda a: a.ctypes.data_as(C.c_void_p)
        rc = lib().bdm_get_agents(self._h, cap, ptr(xyz), ptr(d), ptr(v), ptr(u), ptr(b), ptr(so), C.byref(nout),
                                  C.byref(st), C.byref(nu), BDM_HOST)
        self._check(rc)
        return dict(x=xyz[0, :n], y=xyz[1, :n], z=xyz[2, :n], diam=d[:n], vol=v[:n], uid=u[:n], beh=b[:n],
                    sim_off=so, n=nout.value, step=st.value, next_uid=nu.value)

    def autotune(self, trial_steps=3, what=TUNE_BOX_EDGE | TUNE_LANES | TUNE_SORT):
        t = Tuning()
        self._check(lib().bdm_autotune(self._h, int(trial_steps), int(what), C.byref(t)))
        return {k: getattr(t, k) for k, _ in t._fields_ if k != "reserved"}

    def set_force_kernel(self, lanes=-4):
        """FP32 form: -4 = the hybrid launch (the default: the sparse kernel for
        bricks of fewer than 192 agents, 4 lanes per agent for the others);
        1, 2, 4, 8, 16, 32 = the lane-per-agent kernel with that many lanes per
        agent; -1 = the same with the lanes chosen per box by its cost model;
        0 = the tiled kernel; -3 = the sparse kernel (the last two evaluate the
        contacts the FP32 error analysis does not cover in double-float in
        place, with no fix-up pass)."""
        self._check(lib().bdm_set_force_kernel(self._h, int(lanes)))

    # ------------------------------------------------------------------ profiling
    def profile_begin(self):
        self._check(lib().bdm_profile_begin(self._h))

    def profile_end(self):
        ms = np.zeros(16)
        launches = np.zeros(16, np.int64)
        nph = C.c_int()
        self._check(lib().bdm_profile_end(self._h, ms.ctypes.data_as(C.c_void_p),
                                          launches.ctypes.data_as(C.c_void_p), 16, C.byref(nph)))
        return {lib().bdm_phase_name(p).decode(): (float(ms[p]), int(launches[p])) for p in range(nph.value)}

    # ------------------------------------------------------------------ debug
    def _debug(self, what, dtype, count):
        out = np.zeros(max(count, 1), dtype=dtype)
        need = C.c_int64()
        rc = lib().bdm_get_debug(self._h, what, out.ctypes.data_as(C.c_void_p), count, C.byref(need))
        if rc == BDM_ECAPACITY and need.value > count:
            return self._debug(what, dtype, int(need.value))
        self._check(rc)
        return out[: need.value]

    def last_forces(self):
        n = self.n
        return self._debug(DBG_FORCES, np.float64, 3 * n).reshape(3, n)

    def last_nz(self):
        return self._debug(DBG_NZ, np.int32, self.n)

    def last_static(self):
        return self._debug(DBG_STATIC, np.uint8, self.n)

    def grid_boxes(self):
        n = self.n
        return self._debug(DBG_GRID_BOX, np.int32, 3 * n).reshape(3, n)

    def grid_order(self):
        return self._debug(DBG_GRID_ORDER, np.int64, self.n)

    def grid_geometry(self):
        g = self._debug(DBG_GRID_GEOMETRY, np.float64, 6 * self.n_sims).reshape(self.n_sims, 6)
        return g[:, :3], g[:, 3:].astype(np.int64)

    def brick_ranks(self):
        return self._debug(DBG_BRICK_RANK, np.int64, self.n)

    def neighbors(self):
        n = self.n
        raw = self._debug(DBG_NEIGHBORS, np.int64, n + 1)
        return raw[: n + 1], raw[n + 1:]

    def forces_now(self):
        n = self.n
        raw = self._debug(DBG_FORCES_NOW, np.float64, 4 * n)
        f = raw[: 3 * n].reshape(3, n).copy()
        ints = raw[3 * n: 4 * n].view(np.int32)
        return f, ints[:n].copy(), ints[n: 2 * n].copy()
