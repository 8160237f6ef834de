"""C-ABI checks that need no GPU: every declared symbol is exported and the
host-side validation rejects bad configurations before touching the device."""
import re
import os

import pytest

from paper_0812_2801_gb300 import emd, inputs

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "emd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(emd_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(emd.LIB_PATH):
        from paper_0812_2801_gb300 import _build
        _build.build()
    return emd.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("emd_init_system", "emd_set_ions", "emd_set_orbitals",
                     "emd_propagate", "emd_get_forces", "emd_get_energy",
                     "emd_destroy", "emd_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


@pytest.mark.parametrize("field,value", [("fd_order", 5), ("n", 4), ("h", -1.0),
                                          ("n_orb", 0), ("precision", 7),
                                          ("n", 17 * 4), ("block_orbitals", 3)])
def test_invalid_config_rejected_before_device_use(lib, field, value):
    s = inputs.small_system(n=16, h=0.35, n_atoms=2, seed=1)
    cfg = emd.config_for(s)
    setattr(cfg, field, value)
    with pytest.raises(emd.EmdError) as ei:
        emd.emd_init_system(cfg)
    assert ei.value.code == emd.EMD_EINVAL


def test_support_radius_larger_than_box_rejected(lib):
    s = inputs.small_system(n=16, h=0.25, n_atoms=2, seed=1)   # L = 4 < 5
    with pytest.raises(emd.EmdError) as ei:
        emd.emd_init_system(emd.config_for(s))
    assert ei.value.code == emd.EMD_EINVAL


def test_ground_state_rejects_null_system_before_device_use(lib):
    assert lib.emd_ground_state(None, 10, 1e-8, 8, 0.5, None, None) == emd.EMD_EINVAL
    assert "NULL" in lib.emd_last_error().decode()


def test_binding_constants_match_the_header():
    text = open(HEADER).read()
    defs = dict(re.findall(r"#define\s+(EMD_[A-Z0-9_]+)\s+(-?\d+)", text))
    for name, value in defs.items():
        if hasattr(emd, name):
            assert getattr(emd, name) == int(value), name
    for name in ("EMD_OK", "EMD_EINVAL", "EMD_ESTATE", "EMD_EUNSTABLE", "EMD_ENOTCONV",
                 "EMD_ETIMEOUT", "EMD_FP64", "EMD_FP32_ORBITALS", "EMD_OPT_PROFILE",
                 "EMD_OPT_ZCHUNK", "EMD_OBS_DIPOLE_Z"):
        assert hasattr(emd, name) and name in defs, name


def test_binding_declares_argument_types(lib):
    """ctypes would pass Python floats and 64-bit pointers wrongly without
    argtypes: every declared function that takes arguments has them."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for name, args in re.findall(r"\b(emd_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        if args.strip() in ("", "void"):
            continue
        assert getattr(lib, name).argtypes is not None, name
