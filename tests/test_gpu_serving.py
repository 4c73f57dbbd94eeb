"""Batched ensembles and the continuous-batching server on the GPU.

* Every served result equals the CPU oracle's trajectory from the same initial
  state with the same time step (FP64 members to 1e-12 or the long-double
  floor, mixed members to 1e-4 per variable in the state and the flow), for
  orders 3, 4 and 7, bubbles, sharp bubbles and channels.
* A batched solve (persistent launches over work tables, CUDA graph) also gives
  the same state as the same solve through the single-handle path, bit for bit.
* A result is the same alone and in a mix of other requests (bit for bit: the
  members' arithmetic is independent), and both equal the oracle's.
* Admission respects the footprint budget; errors are reported per request.
"""
import numpy as np
import pytest

from oracle_checks import check_request_result

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2605_16684_gb300 import _build, _lib
    _build.build()
    return _lib


def single_handle(lib, req):
    kind = req.get("kind", "bubble")
    K, N = req["K"], req["N"]
    if kind in ("bubble", "sharp_bubble"):
        s = lib.Solver(*K, N, precision=req.get("precision", "fp64"), warp=req.get("warp", 0.0))
        s.init_bubble(300.0, req.get("amp", 0.5), req.get("centre", (500.0, 500.0, 350.0)), 250.0,
                      profile="sharp" if kind == "sharp_bubble" else "smooth")
    else:
        s = lib.Solver(*K, N, lo=(0, 0, 0), hi=(40000e3, 6000e3, 30e3), periodic=(1, 0, 0),
                       precision=req.get("precision", "fp64"), f0=1e-4)
        s.init_channel()
    dt = s.cfl_dt(req.get("cfl", 0.4))  # the server's default Courant number
    s.step(dt, req["nsteps"])
    q = s.get_state().reshape(-1)
    s.close()
    return q, dt


MIX = [
    dict(K=(4, 4, 4), N=3, precision="fp64", nsteps=4),
    dict(K=(3, 3, 3), N=4, precision="mixed", nsteps=5, warp=0.05, amp=0.8),
    dict(K=(2, 2, 2), N=7, precision="mixed", nsteps=3),
    dict(kind="channel", K=(6, 3, 2), N=3, precision="fp64", nsteps=2),
    dict(K=(5, 4, 3), N=4, precision="fp64", nsteps=6, centre=(450.0, 520.0, 300.0)),
    dict(K=(3, 2, 2), N=3, precision="mixed", nsteps=7),
    dict(kind="sharp_bubble", K=(3, 3, 3), N=4, precision="mixed", nsteps=4),
    dict(K=(2, 2, 2), N=7, precision="fp64", nsteps=3, warp=0.05, amp=0.9),
]


def test_batched_equals_single_handle_and_oracle(lib):
    srv = lib.Server()
    tickets = [srv.submit(**r) for r in MIX]
    for t, r in zip(tickets, MIX):
        res = srv.wait(t)
        assert res["status"] == 0, srv.stats()["error"]
        q_ref, dt = single_handle(lib, r)
        assert res["dt"] == pytest.approx(dt, rel=0, abs=0)
        assert res["nsteps"] == r["nsteps"]
        assert np.array_equal(res["q"], q_ref), np.abs(res["q"] - q_ref).max()
        check_request_result(r, res["q"], res["dt"])
    st = srv.stats()
    assert st["finished"] == len(MIX) and st["last_error"] == 0
    srv.close()


def test_result_same_alone_and_in_mix(lib):
    target = dict(K=(4, 3, 3), N=4, precision="mixed", nsteps=6, warp=0.05)
    alone = lib.Server()
    ra = alone.wait(alone.submit(**target))
    alone.close()
    mix = lib.Server()
    others = [mix.submit(**r) for r in MIX[:3]]
    t = mix.submit(**target)
    later = [mix.submit(**r) for r in MIX[3:]]
    rm = mix.wait(t)
    for o in others + later:
        assert mix.wait(o)["status"] == 0
    mix.close()
    assert ra["status"] == 0 and rm["status"] == 0
    assert np.array_equal(ra["q"], rm["q"])
    # and both are the oracle's trajectory within the mixed-precision bars
    check_request_result(target, ra["q"], ra["dt"])


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_every_batched_variant_equals_single_handle(lib, monkeypatch, variant):
    # the autotuner's candidates (pipelined table-driven kernel, per-tile kernel at two
    # tile shapes), each forced in turn: bitwise the single-handle result
    monkeypatch.setenv("ES_DG_BATCH_VARIANT", str(variant))
    reqs = [dict(K=(5, 4, 3), N=4, precision="fp64", nsteps=3, warp=0.05),
            dict(K=(4, 4, 3), N=4, precision="mixed", nsteps=4, warp=0.05, amp=0.7),
            dict(K=(3, 3, 3), N=3, precision="mixed", nsteps=3),
            dict(K=(2, 2, 2), N=7, precision="mixed", nsteps=2),
            dict(kind="channel", K=(6, 3, 2), N=4, precision="mixed", nsteps=2)]
    srv = lib.Server()
    tickets = [srv.submit(**r) for r in reqs]
    for t, r in zip(tickets, reqs):
        res = srv.wait(t)
        assert res["status"] == 0, srv.stats()["error"]
        assert np.array_equal(res["q"], single_handle(lib, r)[0]), r
        check_request_result(r, res["q"], res["dt"])
    srv.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_equals_single_handle_several_tiles_per_cta(lib, precision):
    # 15 x 16 x 13 elements at N = 4: the single-mesh kernels (the warp-specialised
    # mixed kernel, the pipelined FP64 kernel) walk several tiles per CTA through their
    # double-buffered hand-overs, with a partial last round; the batched kernels walk
    # the work table.  Bitwise the same state.
    r = dict(K=(15, 16, 13), N=4, precision=precision, nsteps=2, warp=0.05, amp=0.8)
    srv = lib.Server()
    res = srv.wait(srv.submit(**r))
    srv.close()
    assert res["status"] == 0
    q_ref, dt = single_handle(lib, r)
    assert res["dt"] == dt
    assert np.array_equal(res["q"], q_ref), np.abs(res["q"] - q_ref).max()


def test_twin_meshes_share_geometry_exactly(lib):
    # members with the same mesh and order copy the first one's geometry at
    # admission; every result still equals its own single-handle solve bit for bit
    reqs = [dict(K=(4, 4, 3), N=4, precision=p, nsteps=3, warp=0.05, amp=a)
            for p, a in (("mixed", 0.5), ("mixed", 0.9), ("fp64", 0.7))]
    srv = lib.Server()
    tickets = [srv.submit(**r) for r in reqs]
    for t, r in zip(tickets, reqs):
        res = srv.wait(t)
        assert res["status"] == 0, srv.stats()["error"]
        assert np.array_equal(res["q"], single_handle(lib, r)[0])
        check_request_result(r, res["q"], res["dt"])
    srv.close()


def test_admission_by_footprint_serialises_large_requests(lib):
    # budget for one 4^3 N=3 FP64 request at a time (estimated 1.7 MiB each)
    srv = lib.Server(hbm_budget_bytes=3 << 20, max_slots=8)
    reqs = [dict(K=(4, 4, 4), N=3, precision="fp64", nsteps=3) for _ in range(3)]
    ts = [srv.submit(**r) for r in reqs]
    res = [srv.wait(t) for t in ts]
    assert all(r["status"] == 0 for r in res)
    # FIFO: each admission waits for the previous request to finish
    for a, b in zip(res, res[1:]):
        assert b["t_admit"] >= a["t_finish"] - 1e-3
    srv.close()


def test_errors_and_cancel(lib):
    from paper_2605_16684_gb300._lib import EsDgError
    srv = lib.Server(hbm_budget_bytes=8 << 20)
    with pytest.raises(EsDgError):
        srv.submit(K=(4, 4, 4), N=9)
    with pytest.raises(EsDgError):  # can never fit the budget
        srv.submit(K=(32, 32, 32), N=4)
    t = srv.submit(K=(2, 2, 2), N=3, nsteps=100000)
    srv.cancel(t)
    assert srv.wait(t)["status"] in (0, -7)
    srv.close()


def test_diverging_member_finishes_alone_with_enan(lib):
    # host-side injection: one request's time step is far beyond the stability limit
    # (Courant number 40), so its state overflows within a few steps.  That member
    # is finished early with ES_DG_ENAN; the members around it are unaffected.
    good = [dict(K=(3, 3, 3), N=3, precision="fp64", nsteps=40),
            dict(K=(3, 3, 2), N=4, precision="mixed", nsteps=40, warp=0.05)]
    bad = dict(K=(3, 3, 3), N=3, precision="mixed", nsteps=400, cfl=40.0)
    srv = lib.Server()
    tg = [srv.submit(**good[0]), srv.submit(**bad), srv.submit(**good[1])]
    res = [srv.wait(t) for t in tg]
    srv.close()
    assert res[1]["status"] == -4 and res[1]["q"] is None
    assert res[1]["nsteps"] < bad["nsteps"]
    for r, req in zip((res[0], res[2]), good):
        assert r["status"] == 0
        assert np.array_equal(r["q"], single_handle(lib, req)[0])
        check_request_result(req, r["q"], r["dt"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_handle_reports_non_finite_state(lib, precision):
    s = lib.Solver(3, 3, 3, 3, precision=precision)
    s.init_bubble()
    q0 = s.get_state()
    dt = s.cfl_dt(0.5)
    s.step(80.0 * dt, 60)
    with pytest.raises(lib.EsDgError) as err:
        s.sync()
    assert err.value.code == -4  # ES_DG_ENAN
    s.set_state(q0)  # the flag was cleared by the failed sync
    s.step(dt, 2)
    s.sync()
    assert np.isfinite(s.get_state()).all()
    s.close()
