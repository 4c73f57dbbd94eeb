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
