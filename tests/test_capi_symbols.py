"""The C-ABI library builds for sm_103a, loads, and exports every function
include/bdm.h declares; argument checks that need no GPU.  CPU only."""
import ctypes as C
import os
import re

import pytest

from paper_2301_06984_gb300 import bdm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bdm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bdm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("bdm_create", "bdm_set_agents", "bdm_step", "bdm_sort", "bdm_get_agents", "bdm_destroy",
                 "bdm_last_error", "bdm_get_debug", "bdm_get_counters"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = bdm.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) <= set(bdm.SIGNATURES)
    assert L.bdm_version() == 200


def test_struct_layouts_match_header_sizes():
    # bdm_params: 7 doubles, 4 int32, pointer, u64, 5 doubles, i64, 2 int32,
    # death_prob, 2 int32, two tables of 16 doubles
    assert C.sizeof(bdm.Params) == 7 * 8 + 4 * 4 + 8 + 8 + 5 * 8 + 8 + 2 * 4 + 8 + 2 * 4 + 32 * 8
    assert C.sizeof(bdm.Counters) == 15 * 8 + 2 * 4 + 2 * 8


@pytest.mark.parametrize("field,value", [("interaction_radius", 0.0), ("interaction_radius", -1.0),
                                         ("box_edge", 5.0), ("n_sims", 0), ("capacity", 0), ("precision", 7),
                                         ("dt", -1.0), ("sort_every", -2), ("death_prob", -0.1),
                                         ("death_prob", 1.5)])
def test_create_rejects_bad_parameters_without_touching_the_gpu(field, value):
    L = bdm.lib()
    p = bdm.Params()
    p.interaction_radius, p.box_edge, p.dt, p.max_displacement, p.k, p.gamma = 10.0, 0.0, 0.01, 3.0, 2.0, 1.0
    p.n_sims, p.capacity, p.precision, p.ratio_lo, p.ratio_hi = 1, 100, 0, 0.9, 1.1
    setattr(p, field, value)
    h = C.c_void_p()
    rc = L.bdm_create(C.byref(p), None, C.byref(h))
    assert rc == bdm.BDM_EINVAL
    assert h.value is None
    assert len(L.bdm_last_error(None)) > 0


def test_growth_requires_fp64_single_simulation():
    L = bdm.lib()
    p = bdm.Params()
    p.interaction_radius, p.dt, p.max_displacement, p.k, p.gamma = 10.0, 0.01, 3.0, 2.0, 1.0
    p.n_sims, p.capacity, p.precision = 1, 100, bdm.BDM_FP32_FORCE
    p.growth_per_step, p.divide_volume, p.ratio_lo, p.ratio_hi = 300.0, 4000.0, 0.9, 1.1
    h = C.c_void_p()
    assert L.bdm_create(C.byref(p), None, C.byref(h)) == bdm.BDM_EINVAL


def test_null_handles_are_rejected():
    L = bdm.lib()
    assert L.bdm_step(None, 1) == bdm.BDM_EINVAL
    assert L.bdm_sort(None) == bdm.BDM_EINVAL
    L.bdm_destroy(None)


def test_removal_requires_single_simulation():
    L = bdm.lib()
    p = bdm.Params()
    p.interaction_radius, p.dt, p.max_displacement, p.k, p.gamma = 10.0, 0.01, 3.0, 2.0, 1.0
    p.n_sims, p.capacity, p.precision, p.death_prob = 4, 100, bdm.BDM_FP32_FORCE, 0.1
    h = C.c_void_p()
    assert L.bdm_create(C.byref(p), None, C.byref(h)) == bdm.BDM_EINVAL
