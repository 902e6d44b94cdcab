"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/heat.h declares (no compute calls: this machine may have no GPU)."""
import ctypes
import shutil

import pytest

from paper_1311_4627_gb300 import build, heat


@pytest.fixture(scope="module")
def libheat():
    if shutil.which("nvcc") is None and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    build.build_lib()
    return heat.lib()


def test_header_declares_the_boundary():
    syms = heat.declared_symbols()
    for name in ["heat_create_grid", "heat_set_grains", "heat_set_fields", "heat_solve", "heat_sync",
                 "heat_last_error", "heat_destroy", "heat_default_opts", "heat_get_cooling", "heat_band_elements"]:
        assert name in syms


def test_library_exports_every_declared_symbol(libheat):
    missing = [s for s in heat.declared_symbols() if not hasattr(libheat, s)]
    assert not missing, missing


def test_default_opts_and_null_handling(libheat):
    o = heat.heat_default_opts()
    assert (o.build, o.emis, o.j_dtype, o.size_integrate, o.host_io) == (0, 0, 0, 0, 0)
    assert (o.streams, o.heating, o.prune_eps) == (0, heat.HEAT_HEATING_INTEGRAL, 0.0)
    # the binding's struct ends where the library's does: the last field is written by
    # heat_default_opts, so a poisoned value there must be overwritten
    o.heating = 12345
    o.prune_eps = 0.5
    o.cooling = 777
    o.build_prefetch = 3
    libheat.heat_default_opts(ctypes.byref(o))
    assert o.heating == heat.HEAT_HEATING_INTEGRAL and o.prune_eps == 0.0
    assert o.cooling == heat.HEAT_COOLING_CONTINUOUS and o.build_prefetch == 0
    assert heat.heat_opts._fields_[-1][0] == "build_prefetch"
    # null contexts are rejected without touching a device
    assert libheat.heat_sync(None) == heat.HEAT_EINVAL
    assert libheat.heat_solve(None, ctypes.byref(o), None, None, None) == heat.HEAT_EINVAL
    assert heat.heat_last_error(None) == "null context"
    libheat.heat_destroy(None)


def test_create_grid_rejects_bad_grids(libheat):
    import numpy as np

    h = ctypes.c_void_p()
    bad = np.array([1.0, 1.0, 2.0])
    assert libheat.heat_create_grid(ctypes.byref(h), 0, 3, bad.ctypes.data) == heat.HEAT_EINVAL
    neg = np.array([-1.0, 2.0])
    assert libheat.heat_create_grid(ctypes.byref(h), 0, 2, neg.ctypes.data) == heat.HEAT_EINVAL
    assert libheat.heat_create_grid(ctypes.byref(h), 0, 1, neg.ctypes.data) == heat.HEAT_EINVAL


def _header_struct_fields(text, name):
    """Member names of `typedef struct name {...} name;` in declaration order (comments removed)."""
    import re

    m = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), text, re.S)
    assert m, name
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            decl = re.sub(r"^(const\s+)?(unsigned\s+)?(long long|int|double|float|void|char)\s*\**\s*", "", decl)
            fields += [f.strip().lstrip("*") for f in decl.split(",")]
    return fields


def test_binding_structs_mirror_the_header():
    """Every struct the header defines has a ctypes mirror with the same members in the same order."""
    import os
    import re

    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "heat.h")).read()
    defined = re.findall(r"typedef struct (\w+) \{", text)
    assert set(defined) == {"heat_opts", "heat_tuning"}
    for name in defined:
        assert [f for f, _ in getattr(heat, name)._fields_] == _header_struct_fields(text, name), name
