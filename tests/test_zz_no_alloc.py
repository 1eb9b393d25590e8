"""The allocation-free entry point bdm_forces_noalloc, for callers that cannot
call cudaMalloc (host applications whose own allocator owns all device memory,
plug-ins or embedded solvers that their host forbids to allocate).  It must give
the same forces and counts as the allocating path (bdm_get_debug's
BDM_DBG_FORCES_NOW in the FP64 form, compared bit for bit as the FP64 tests
do) on two calls in a row that share its fixed scratch array.  Collected last
on purpose: the rest of the suite has run before it when -x stops here."""
import ctypes as C

import numpy as np
import pytest

from paper_2301_06984_gb300 import bdm
from paper_2301_06984_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(x, y, z, d, R):
    import torch
    n = len(x)
    dev = torch.device("cuda")
    xyz = torch.as_tensor(np.concatenate([x, y, z]), dtype=torch.float64, device=dev)
    dd = torch.as_tensor(d, dtype=torch.float64, device=dev)
    f = torch.full((3 * n,), np.nan, dtype=torch.float64, device=dev)
    cnt = torch.full((2 * n,), -1, dtype=torch.int32, device=dev)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = bdm.lib()
    rc = L.bdm_forces_noalloc(n, C.c_void_p(xyz.data_ptr()), C.c_void_p(dd.data_ptr()), R, 0.0, 2.0, 1.0,
                              C.c_void_p(f.data_ptr()), C.c_void_p(cnt.data_ptr()), st)
    assert rc == 0, L.bdm_noalloc_last_error().decode()
    torch.cuda.synchronize()
    return f.cpu().numpy().reshape(3, n), cnt.cpu().numpy().reshape(2, n)


def _allocating(x, y, z, d, R):
    s = bdm.Simulation(R=R, capacity=len(x), precision="fp64")
    s.set_agents(x, y, z, d)
    f, nz, nnb = s.forces_now()
    s.close()
    return f, np.stack([nz, nnb])


def _clustered(n, seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(60.0, 12.0, (3, n))
    return p[0].copy(), p[1].copy(), p[2].copy(), rng.uniform(8.0, 12.0, n)


def test_noalloc_forces_match_the_allocating_path_on_two_calls():
    import torch
    assert torch.cuda.is_available()
    w = W.uniform(n=8192, seed=1)
    first = (w.x, w.y, w.z, w.diam)
    second = _clustered(20000, 7)
    for args in (first, second):  # the second call reuses the scratch the first left behind
        f_na, c_na = _noalloc(*args, 12.0)
        f_al, c_al = _allocating(*args, 12.0)
        assert np.array_equal(c_na, c_al)
        assert np.array_equal(f_na, f_al)
        assert c_na[1].sum() > 0


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    n = 131073
    L = bdm.lib()
    z = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    rc = L.bdm_forces_noalloc(n, C.c_void_p(z.data_ptr()), C.c_void_p(z.data_ptr()), 10.0, 0.0, 2.0, 1.0,
                              C.c_void_p(z.data_ptr()), C.c_void_p(z.data_ptr()),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == bdm.BDM_ECAPACITY
    assert b"131072" in L.bdm_noalloc_last_error()
