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


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of emd_species, emd_config, emd_energy and
    emd_gs_info have the C compiler's size and field offsets."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"emd_species": emd.emd_species, "emd_config": emd.emd_config,
               "emd_energy": emd.emd_energy, "emd_gs_info": emd.emd_gs_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "emd.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'  printf("{name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True,
                                                         capture_output=True, text=True).stdout.split("\n") if l)
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert int(out[f"{name}.{f[0]}"]) == getattr(cls, f[0]).offset, (name, f[0])


@pytest.mark.parametrize("lmax,prec,bo", [(3, 0, 0), (-1, 0, 0), (1, 1, 0), (2, 0, 4), (1, 0, 1)])
def test_projector_channels_rejected_before_device_use(lib, lmax, prec, bo):
    """lmax outside 0..2, or several projectors per atom outside the FP64 form
    with block width 2 (the double-float kernels that carry them)."""
    s = inputs.small_system(n=16, h=0.35, n_atoms=2, seed=1)
    cfg = emd.config_for(s, precision=prec, block_orbitals=bo)
    cfg.species.lmax = lmax
    with pytest.raises(emd.EmdError) as ei:
        emd.emd_init_system(cfg)
    assert ei.value.code == emd.EMD_EINVAL


def test_occupation_and_smeared_entry_points_reject_null(lib):
    import ctypes
    f = (ctypes.c_double * 4)(2.0, 2.0, 1.0, 1.0)
    assert lib.emd_set_occupations(None, f) == emd.EMD_EINVAL
    assert lib.emd_get_occupations(None, f) == emd.EMD_EINVAL
    assert lib.emd_ground_state_smeared(None, 10, 1e-8, 8, 0.5, 0.01, 6.0, 0.8,
                                        None, None, None) == emd.EMD_EINVAL
    assert "NULL" in lib.emd_last_error().decode()
