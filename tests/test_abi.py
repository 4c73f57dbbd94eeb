"""The C-ABI library loads and exports every function include/es_dg.h declares
(CPU only: no kernel runs; argument validation happens before any CUDA call)."""
import ctypes as C
import os
import re

import pytest

from paper_2605_16684_gb300 import _build, _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(es_dg_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _lib.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "es_dg_create" in names and "es_dg_rhs" in names and len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    assert declared_functions() <= set(_lib.SIGNATURES)


def test_strerror(lib):
    assert lib.es_dg_strerror(0) == b"ok"
    assert lib.es_dg_strerror(-1) == b"invalid argument"
    assert lib.es_dg_strerror(12345) == b"unknown status"


# (1 << 28) + 1 elements along x (times 2 x 2): more than the 2^30 elements a handle admits
@pytest.mark.parametrize("kx,N,warp", [(0, 3, 0.0), (2, 0, 0.0), (2, 8, 0.0), (2, 3, 0.5),
                                       ((1 << 28) + 1, 3, 0.0)])
def test_create_rejects_bad_arguments_before_touching_cuda(lib, kx, N, warp):
    m = _lib.es_dg_mesh(kx, 2, 2, (C.c_double * 3)(0, 0, 0), (C.c_double * 3)(1, 1, 1),
                        (C.c_int * 3)(1, 1, 0), warp)
    h = C.c_void_p()
    assert lib.es_dg_create(C.byref(m), N, 0, None, None, None, C.byref(h)) == -1
    assert not h.value


def test_null_handle_rejected(lib):
    assert lib.es_dg_step(None, 1.0, 1) == -1
    assert lib.es_dg_rhs(None, None, None, 0) == -1


def test_create_rejects_gravity_with_z_periodic_box(lib):
    # phi = g z would jump across the periodic z faces
    m = _lib.es_dg_mesh(2, 2, 2, (C.c_double * 3)(0, 0, 0), (C.c_double * 3)(1, 1, 1),
                        (C.c_int * 3)(1, 1, 1), 0.0)
    h = C.c_void_p()
    assert lib.es_dg_create(C.byref(m), 3, 0, None, None, None, C.byref(h)) == -1
    assert not h.value


def test_server_rejects_bad_arguments_before_touching_cuda(lib):
    h = C.c_void_p()
    assert lib.es_dg_server_create(0, 4, None, C.byref(h)) == -1
    assert lib.es_dg_server_create(1 << 30, 0, None, C.byref(h)) == -1
    assert lib.es_dg_batch_submit(None, None, None) == -1


@pytest.mark.parametrize("xb,xe", [(0, 0), (2, 1), (-1, 2), (0, 5), (3, 3)])
def test_create_partition_rejects_bad_ranges_before_touching_cuda(lib, xb, xe):
    m = _lib.es_dg_mesh(4, 2, 2, (C.c_double * 3)(0, 0, 0), (C.c_double * 3)(1, 1, 1),
                        (C.c_int * 3)(1, 1, 0), 0.0)
    h = C.c_void_p()
    assert lib.es_dg_create_partition(C.byref(m), 3, 0, None, xb, xe, None, None, C.byref(h)) == -1
    assert not h.value


def test_partition_calls_reject_null_arguments(lib):
    assert lib.es_dg_partition_info(None, None, None, None, None) == -1
    assert lib.es_dg_set_traces(None, None, None, None, None) == -1
    assert lib.es_dg_pack_traces(None, 0) == -1
    assert lib.es_dg_accept_geometry_trace(None) == -1
    assert lib.es_dg_partitions_connect(None, 2) == -1
    assert lib.es_dg_partitions_exchange(None, 0) == -1
    assert lib.es_dg_partitions_step(None, 2, 1.0, 1) == -1
