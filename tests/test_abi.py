"""The C ABI library loads and exports every entry point declared in include/evap.h (no GPU needed).

Only host-side argument validation is exercised here: calls that fail validation return before any CUDA work."""
import ctypes
import os
import re

import pytest

import paper_2401_07805_gb300 as evap
from paper_2401_07805_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "evap.h")


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(evap.library_path()):
        build.build()
    return evap.lib()


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(evap_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_api():
    names = declared()
    for required in ("evap_create_mesh", "evap_set_fields", "evap_apply_momentum", "evap_apply_levelset",
                     "evap_apply_adjoint", "evap_solve"):
        assert required in names


def test_every_declared_symbol_is_exported_and_bound(L):
    for name in declared():
        assert hasattr(L, name), name
        assert name in evap.SIGNATURES, name


def test_params_struct_matches_header():
    src = open(HEADER).read()
    body = src[src.index("typedef struct {") + len("typedef struct {"): src.index("} evap_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for line in body.splitlines():
        decl = line.strip().rstrip(";")
        if not decl:
            continue
        typ, names = decl.split(None, 1)
        fields += [(n.strip(), typ) for n in names.split(",")]
    assert [f for f, _ in fields] == [f for f, _ in evap.EvapParams._fields_]
    ct = {"double": ctypes.c_double, "int": ctypes.c_int, "unsigned": ctypes.c_uint}
    for (name, typ), (pname, ptyp) in zip(fields, evap.EvapParams._fields_):
        assert ct[typ] == ptyp, name


def test_status_strings(L):
    for code, name in evap.STATUS.items():
        assert L.evap_status_string(code).decode() == name


def test_invalid_arguments_are_rejected_on_the_host(L):
    prm = evap.make_params(4)
    h = ctypes.c_void_p()
    assert L.evap_create_mesh(0, 2, 1.0, ctypes.byref(prm), ctypes.byref(h)) == -1
    assert L.evap_create_mesh(4, 4, 1.0, ctypes.byref(prm), ctypes.byref(h)) == -1
    assert L.evap_create_mesh(4, 2, -1.0, ctypes.byref(prm), ctypes.byref(h)) == -1
    bad = evap.make_params(4, variant=7)
    assert L.evap_create_mesh(4, 2, 1.0, ctypes.byref(bad), ctypes.byref(h)) == -1
    assert L.evap_create_mesh(4, 2, 1.0, None, ctypes.byref(h)) == -1
    assert not h
    assert b"variant" in L.evap_last_error() or b"null" in L.evap_last_error()
    for fn, args in (("evap_apply_momentum", (None, 64, None, None, None, None)),
                     ("evap_apply_levelset", (None, 0, 64, None, None, None)),
                     ("evap_set_fields", (None, None, None, None, None)),
                     ("evap_apply_adjoint", (None,) * 9),
                     ("evap_jacobi_diagonal", (None, None, None)),
                     ("evap_projected_normal", (None, None, None, None, None)),
                     ("evap_curvature", (None, None, None, None, None, None)),
                     ("evap_set_levelset_normal", (None, None, None)),
                     ("evap_reinitialize", (None, None, 1, None, None, None)),
                     ("evap_surface_tension", (None, None, None, 1.0, None, None)),
                     ("evap_advect_levelset", (None, None, 1, 0.0, None, None, None, None)),
                     ("evap_set_checks", (None, 1)),
                     ("evap_time_step", (None,) * 7 + (0.0, 1, 0.0, 1, 1, 1e-8, None, None, None, None)),
                     ("evap_apply_saddle", (None,) * 6),
                     ("evap_solve_saddle", (None, None, None, None, 30, 1e-8, 10, None, None, None)),
                     ("evap_update_transport_velocity", (None, None)),
                     ("evap_transport_stats", (None, None, None, None, None))):
        assert getattr(L, fn)(*args) == -1, fn
    assert L.evap_destroy(None) == 0
