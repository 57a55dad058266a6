"""The C-ABI library builds, loads and exports every function include/trheed.h declares; argument
validation happens before any device work (no compute call here)."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from paper_2306_00271_gb300 import api, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(api.LIB_PATH):
        from paper_2306_00271_gb300 import build
        build.build()
    return api.load()


def test_header_lists_the_boundary():
    names = api.header_functions()
    for f in ("trh_create", "trh_set_structure", "trh_rocking_curve", "trh_query",
              "trh_strerror", "trh_last_error", "trh_destroy"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", api.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for f in api.header_functions():
        assert f in exported, f
        assert hasattr(lib, f)


def test_strerror_names_every_code(lib):
    for code in range(0, -8, -1):
        assert lib.trh_strerror(code) not in (None, b"")
    assert lib.trh_strerror(-99) == b"unknown status"


def _problem(wl, **over):
    keep = dict(beams=np.ascontiguousarray(wl.beams, np.int32),
                atoms=np.ascontiguousarray(wl.atoms), dw=np.ascontiguousarray(wl.dw),
                species=np.ascontiguousarray(wl.species, np.int32), sf=np.ascontiguousarray(wl.sf))
    p = api.TrhProblem()
    p.particle, p.energy_ev, p.absorption = wl.particle, wl.energy_ev, wl.absorption
    p.a1[0], p.a1[1], p.a2[0], p.a2[1] = *wl.a1, *wl.a2
    p.n_beams = wl.beams.shape[0]
    p.beams = keep["beams"].ctypes.data_as(C.POINTER(C.c_int))
    p.n_atoms = wl.atoms.shape[0]
    p.atoms = keep["atoms"].ctypes.data_as(C.POINTER(C.c_double))
    p.dw = keep["dw"].ctypes.data_as(C.POINTER(C.c_double))
    p.species = keep["species"].ctypes.data_as(C.POINTER(C.c_int))
    p.n_species = wl.sf.shape[0]
    p.sf = keep["sf"].ctypes.data_as(C.POINTER(C.c_double))
    p.z_e, p.n_steps, p.integrator, p.rhst_threshold, p.precision = wl.z_e, wl.n_steps, 0, 0.0, 0
    for k, v in over.items():
        setattr(p, k, v)
    return p, keep


@pytest.mark.parametrize("field,value", [("particle", 0), ("energy_ev", -1.0), ("z_e", 1.0),
                                         ("n_steps", 0), ("integrator", 7), ("precision", 5),
                                         ("n_beams", 0)])
def test_create_rejects_bad_problems(lib, field, value):
    p, keep = _problem(W.rheed_row(), **{field: value})
    ctx = C.c_void_p()
    rc = lib.trh_create(C.byref(ctx), C.byref(p))
    assert rc == api.TRH_EINVAL
    assert not ctx.value
    assert lib.trh_last_error() != b""


def test_create_rejects_nonzero_first_beam(lib):
    wl = W.rheed_row()
    wl.beams = wl.beams[::-1].copy()
    p, keep = _problem(wl)
    ctx = C.c_void_p()
    assert lib.trh_create(C.byref(ctx), C.byref(p)) == api.TRH_EINVAL


def test_large_beam_sets_are_unsupported_not_wrong(lib):
    """Both paths take N <= 256, and the mixed path above 128 beams a difference grid of at most
    1536 entries; these limits are checked before any device work, so they are reported here
    without a GPU."""
    a1, a2 = W.hex_lattice(3.84)
    wl = W.trhepd_n61()
    wl.beams = W.beam_disk(a1, a2, 257)
    p, keep = _problem(wl)
    ctx = C.c_void_p()
    assert lib.trh_create(C.byref(ctx), C.byref(p)) == api.TRH_EUNSUPPORTED
    p, keep = _problem(wl, precision=1)
    assert lib.trh_create(C.byref(ctx), C.byref(p)) == api.TRH_EUNSUPPORTED
    # 143 beams spread over a long row: the grid of their differences has 22,599 entries
    wl.beams = np.array([[0, 0], [1, 0], [0, 1]] + [[m, 40] for m in range(-70, 70)],
                        dtype=np.int32)
    p, keep = _problem(wl, precision=1)
    assert lib.trh_create(C.byref(ctx), C.byref(p)) == api.TRH_EUNSUPPORTED
    assert b"difference grid" in lib.trh_last_error()
    # RK4 runs on the FP64 path only
    p, keep = _problem(W.rheed_row(), precision=1, integrator=2)
    assert lib.trh_create(C.byref(ctx), C.byref(p)) == api.TRH_EUNSUPPORTED


def _header_struct_fields(name):
    import re
    text = open(api.HEADER).read()
    body = text[text.index(f"typedef struct {name} {{"):]
    body = body[body.index("{") + 1:body.index(f"}} {name};")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:  # one or more declarators after the type: "double a1[2], a2[2]"
            names += re.findall(r"([A-Za-z_][A-Za-z_0-9]*)\s*(?:\[[^]]*\])?\s*(?=,|$)", decl)
    return names


@pytest.mark.parametrize("name, cls", [("trh_stats", api.TrhStats),
                                       ("trh_problem", api.TrhProblem)])
def test_binding_structs_match_the_header(name, cls):
    assert [f[0] for f in cls._fields_] == _header_struct_fields(name)


def test_null_arguments(lib):
    assert lib.trh_set_column_split(None, 0) == api.TRH_EINVAL
    assert lib.trh_set_async(None, 1) == api.TRH_EINVAL
    assert lib.trh_create(None, None) == api.TRH_EINVAL
    assert lib.trh_query(None, None) == api.TRH_EINVAL
    assert lib.trh_rocking_curve(None, 1, None, None, None, None, None) == api.TRH_EINVAL
    lib.trh_destroy(None)
