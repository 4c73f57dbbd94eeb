"""The benchmark's algorithmic flop counts are those of the oracle (CPU only).

bench.py computes the FP64 volume kernel's achieved FLOP/s from FLOPS_PER_PAIR
(per unordered node pair of the half sweep) and FLOPS_PER_NODE (per node and
stage).  The counting instantiation of the oracle (oracle/count_flops.cpp)
counts both from the oracle's own volume_pair(), primitives(), volume_value()
and lsrk_value(); the benchmark may not load the oracle, so it carries the
numbers as constants, held here to the counted ones for every order.
"""
import importlib.util
import os

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_bench_flop_constants_are_the_counted_ones(N):
    b = bench_module()
    c = O.count_flops(N)
    assert b.FLOPS_PER_PAIR == c["pair"]
    assert b.FLOPS_PER_NODE == c["node"]


def test_count_structure():
    c = O.count_flops(4)
    # the half sweep evaluates the symmetric flux once per pair: sharing saves work
    assert c["pair"] < c["pair_without_sharing"] < 2 * c["pair"]
    # one stage update per value: dq <- A dq + dt (vol + surf + src), q <- q + B dq
    assert c["stage_update"] == 7
    # per node: primitives, then for each of the five values its volume value
    # (one division) and its stage update
    assert c["node"] == c["primitives"] + 5 * (1 + c["stage_update"])


def test_memory_side_byte_counts():
    # the algorithmic bytes behind the bench's achieved-bandwidth figures: the mixed
    # volume kernel moves 240 B per node at N = 4 (29.3 KB per element: FP64 state in
    # and out, FP32 increment in and out, 11 FP32 geometry values, the background's
    # 3 FP64 + 4 FP32 values and 3 FP32 momentum right-hand-side values, and the FP32
    # fluxes of the element's six faces); a face node costs two 5-value traces, its
    # geometry and the flux write (FP64 160 B, mixed 140 B with an FP32 flux)
    b = bench_module()
    assert b.mixed_volume_bytes_per_node(4) == pytest.approx(240.0)
    assert b.mixed_volume_bytes_per_node(4) * 125 == pytest.approx(30000.0)
    assert b.FACE_BYTES_PER_NODE == {"fp64": 160, "mixed": 140}
    # pairs of the half sweep: N_q^2 pencils per direction, N_q (N_q - 1) / 2 pairs each
    for N in range(1, 8):
        nq = N + 1
        assert b.pairs_per_element(N) == 3 * nq * nq * nq * (nq - 1) // 2
