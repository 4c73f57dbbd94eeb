"""Allocation-free integrals entry point (es_dg_integrals_noalloc).

This entry point serves callers that cannot allocate device memory -- for
example code running inside a memory pool it does not own, or inside a
framework that forbids cudaMalloc on its hot path.  It takes caller-owned
device arrays (state, Jacobian, coordinates, 3-double output), keeps its
per-element partial sums in a static device array, and must produce the same
mass, energy and entropy integrals as the handle-based es_dg_integrals.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone.
"""
import ctypes as C

import numpy as np
import pytest

CUBE = dict(lo=(0.0, 0.0, 0.0), hi=(1000.0, 1000.0, 1000.0))


def _mesh(lib_mod, K, periodic=(1, 1, 0), warp=0.0):
    return lib_mod.es_dg_mesh(*K, (C.c_double * 3)(*CUBE["lo"]), (C.c_double * 3)(*CUBE["hi"]),
                              (C.c_int * 3)(*periodic), float(warp))


@pytest.mark.gpu
def test_noalloc_integrals_match_handle_path_on_consecutive_calls():
    import torch

    import oracle as O
    from paper_2605_16684_gb300 import _build, _lib, inputs

    _build.build()
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    cases = [((6, 5, 4), 4, 0.05, "generic"), ((3, 3, 3), 3, 0.0, "bubble")]
    for K, N, warp, kind in cases:
        s = _lib.Solver(*K, N, warp=warp, **CUBE)
        if kind == "generic":
            o = O.Oracle(*K, N, warp=warp, **CUBE)
            x_o, _, _ = o.geometry()
            q = inputs.perturb_state(o.bubble(), x_o, CUBE["lo"], CUBE["hi"], seed=9)
            s.set_state(q)
        else:
            s.init_bubble()
        expected = s.integrals()
        E, np_ = s.E, s.np
        q_dev = torch.empty((E, 5, np_), dtype=torch.float64, device="cuda")
        J_dev = torch.empty((E, np_), dtype=torch.float64, device="cuda")
        x_dev = torch.empty((E, 3, np_), dtype=torch.float64, device="cuda")
        s.get_state(q_dev)
        assert lib.es_dg_geometry(s.h, C.c_void_p(x_dev.data_ptr()), C.c_void_p(J_dev.data_ptr()),
                                  None, 1) == 0
        torch.cuda.synchronize()
        mesh = _mesh(_lib, K, warp=warp)
        outs = []
        for _ in range(2):  # two calls in a row share the static scratch
            out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            rc = lib.es_dg_integrals_noalloc(C.byref(mesh), N, None, C.c_void_p(q_dev.data_ptr()),
                                             C.c_void_p(J_dev.data_ptr()),
                                             C.c_void_p(x_dev.data_ptr()),
                                             C.c_void_p(out.data_ptr()),
                                             C.c_void_p(stream.cuda_stream))
            assert rc == 0
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
        for got in outs:
            assert np.allclose(got, expected, rtol=1e-12, atol=0), (got, expected)
        assert np.array_equal(outs[0], outs[1])
        # the property the entry point exists for: a warm call takes no device memory
        out = torch.empty((3,), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = lib.es_dg_integrals_noalloc(C.byref(mesh), N, None, C.c_void_p(q_dev.data_ptr()),
                                         C.c_void_p(J_dev.data_ptr()), C.c_void_p(x_dev.data_ptr()),
                                         C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        torch.cuda.synchronize()
        assert rc == 0
        assert torch.cuda.mem_get_info()[0] == free_before
        assert np.array_equal(out.cpu().numpy(), outs[0])
        s.close()


def test_noalloc_rejects_meshes_beyond_the_static_scratch():
    from paper_2605_16684_gb300 import _build, _lib

    _build.build()
    lib = _lib.load()
    mesh = _mesh(_lib, (64, 64, 65))  # 266240 > ES_DG_NOALLOC_MAX_ELEMS elements
    dummy = C.c_void_p(16)
    rc = lib.es_dg_integrals_noalloc(C.byref(mesh), 3, None, dummy, dummy, dummy, dummy, None)
    assert rc == -1


def _cuda_device_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


@pytest.mark.skipif(_cuda_device_present(), reason="needs a machine without a CUDA device")
def test_noalloc_accepts_a_mesh_of_exactly_the_maximum_size():
    # 64 x 64 x 64 = ES_DG_NOALLOC_MAX_ELEMS elements passes the size check; with no
    # device present the call then fails at the device query (-ES_DG_ECUDA), not with
    # -ES_DG_EINVAL for its size
    from paper_2605_16684_gb300 import _build, _lib

    _build.build()
    lib = _lib.load()
    mesh = _mesh(_lib, (64, 64, 64))
    dummy = C.c_void_p(16)
    rc = lib.es_dg_integrals_noalloc(C.byref(mesh), 3, None, dummy, dummy, dummy, dummy, None)
    assert rc == -3  # ES_DG_ECUDA


def test_noalloc_rejects_physics_that_create_rejects():
    from paper_2605_16684_gb300 import _build, _lib

    _build.build()
    lib = _lib.load()
    mesh = _mesh(_lib, (2, 2, 2))
    dummy = C.c_void_p(16)
    for gamma, R, p0 in ((1.0, 287.0, 1e5), (1.4, 0.0, 1e5), (1.4, 287.0, -1.0),
                         (float("nan"), 287.0, 1e5)):
        ph = _lib.es_dg_physics(gamma, 9.81, R, p0, 0.0, 0.0, 0.0, 1)
        rc = lib.es_dg_integrals_noalloc(C.byref(mesh), 3, C.byref(ph), dummy, dummy, dummy,
                                         dummy, None)
        assert rc == -1  # ES_DG_EINVAL, before any CUDA call
