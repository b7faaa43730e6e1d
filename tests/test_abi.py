"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/dem.h declares; host-side validation and marshalling (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1301_1714_gb300 import _build, dem, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(dem_\w+)\s*\(", src, flags=re.M):
            syms.add(m.group(1))
    return sorted(syms)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ctypes.CDLL(_build.LIB)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["dem_create", "dem_set_particles", "dem_set_walls", "dem_step", "dem_get_state", "dem_destroy"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_has_same_names(lib):
    for s in declared_symbols():
        assert hasattr(dem, s), s


def test_config_validation_on_host(lib):
    """dem_create validates the configuration before it touches a device."""
    sc = scenes.box_lattice()
    h = ctypes.c_void_p()
    bad = dem.config_from_params(sc.params)
    bad.dt = -1.0
    assert dem.lib().dem_create(ctypes.byref(bad), 0, None, ctypes.byref(h)) == 1
    bad = dem.config_from_params(sc.params)
    bad.domain_hi[0] = bad.domain_lo[0]
    assert dem.lib().dem_create(ctypes.byref(bad), 0, None, ctypes.byref(h)) == 1
    bad = dem.config_from_params(sc.params)
    bad.block_size = 100
    assert dem.lib().dem_create(ctypes.byref(bad), 0, None, ctypes.byref(h)) == 1
    assert dem.lib().dem_create(None, 0, None, ctypes.byref(h)) == 1
    for field, value in (("terms", 16), ("mu_roll", -1.0), ("alpha_t", float("inf")), ("k_coh", float("nan")),
                         ("max_contacts", 65), ("resort_interval", 0)):
        bad = dem.config_from_params(sc.params)
        setattr(bad, field, value)
        if field == "resort_interval":
            bad.skin = 0.0                      # skin-driven sorting needs a skin
        assert dem.lib().dem_create(ctypes.byref(bad), 0, None, ctypes.byref(h)) == 1, field
    bad = dem.config_from_params(sc.params.copy(model="simple", terms=1))
    assert dem.lib().dem_create(ctypes.byref(bad), 0, None, ctypes.byref(h)) == 1
    assert h.value is None


def test_marshalling_of_config_and_walls():
    sc = scenes.drum(n=2000)
    c = dem.config_from_params(sc.params, block_size=64, max_contacts=24)
    assert c.precision == dem.DEM_FP32 and c.model == dem.DEM_PRACTICAL
    assert c.dt == sc.params.dt and tuple(c.domain_lo) == tuple(sc.params.domain_lo)
    assert c.block_size == 64 and c.max_contacts == 24
    w = dem.walls_array(sc.params.walls)
    assert w[0].kind == dem.DEM_CYLINDER_IN and w[0].radius == sc.params.walls[0]["radius"]
    assert tuple(w[0].omega) == (2.0, 0.0, 0.0)
    assert w[1].kind == dem.DEM_PLANE and tuple(w[2].n) == (-1.0, 0.0, 0.0)
    assert w[1].u[0] == 0.0


def test_ctypes_layouts_match_the_header(tmp_path):
    """sizeof and field offsets of dem_config and dem_wall as gcc lays out include/dem.h
    equal those of the ctypes mirrors in the binding."""
    fields = {"dem_config": [f[0] for f in dem.dem_config._fields_], "dem_wall": [f[0] for f in dem.dem_wall._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dem.h"', "int main(void) {"]
    for t, fs in fields.items():
        lines.append(f'printf("{t} %zu\\n", sizeof({t}));')
        for f in fs:
            lines.append(f'printf("{t}.{f} %zu\\n", offsetof({t}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    import subprocess
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for t, fs in fields.items():
        cls = getattr(dem, t)
        assert int(out[t]) == ctypes.sizeof(cls), t
        for f in fs:
            assert int(out[f"{t}.{f}"]) == getattr(cls, f).offset, (t, f)
