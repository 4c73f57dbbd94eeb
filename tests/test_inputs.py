"""Seeded synthetic inputs (paper_2605_16684_gb300/inputs.py), CPU only.

The generators stand in for the paper's workloads; these tests check that the draws
follow the stated recipes and are reproducible from their seeds: the generic-state
perturbation (smooth, unit-maximum fields of the requested wavenumbers, periodic over
the box), the batched-ensemble members (K^3 grids with K in 8..24, N in {3, 4, 7},
amplitude in [0.25, 1] K, centre jitter of at most 100 m) and the Poisson serving
stream (exponential inter-arrival times at the requested rate, 70 % bubbles with
K in 8..32, 30 % channels of (40 s, 8 s, 4 s) elements, s in [1, 3]).
"""
import numpy as np
import pytest

from paper_2605_16684_gb300 import inputs

BOX = ((0.0, 0.0, 0.0), (1000.0, 1000.0, 1000.0))


def _nodes(n=2000, seed=1):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1000.0, size=(n, 3, 1))


def test_perturbation_fields_are_seeded_unit_and_periodic():
    x = _nodes()
    f1 = inputs.perturbation_factors(x, *BOX, 5, seed=7)
    f2 = inputs.perturbation_factors(x, *BOX, 5, seed=7)
    f3 = inputs.perturbation_factors(x, *BOX, 5, seed=8)
    assert f1.shape == (5, 2000, 1)
    assert np.array_equal(f1, f2) and not np.allclose(f1, f3)
    assert np.allclose(np.abs(f1).max(axis=(1, 2)), 1.0)
    # integer wavenumbers over the box: the fields repeat with the box period
    xs = x + np.array([1000.0, -1000.0, 2000.0]).reshape(1, 3, 1)
    fp = inputs.perturbation_factors(xs, *BOX, 5, seed=7)
    # the normalisation uses the maximum over the given nodes, which is the same set
    # of values up to the period shift
    assert np.allclose(f1, fp, atol=1e-9)


def test_perturbation_wavenumbers_follow_the_requested_band():
    # along a line in x only (y = z = const), a single-axis field of wavenumbers kmin..kmax
    # has no spectral content below kmin or above kmax
    n = 512
    x = np.zeros((n, 3, 1))
    x[:, 0, 0] = np.arange(n) * 1000.0 / n
    x[:, 1, 0] = 137.0
    x[:, 2, 0] = 611.0
    for kmin, kmax in ((1, 3), (8, 16)):
        f = inputs.perturbation_factors(x, *BOX, 1, seed=3, kmin=kmin, kmax=kmax)[0, :, 0]
        spec = np.abs(np.fft.rfft(f))
        band = np.zeros_like(spec, dtype=bool)
        band[kmin:kmax + 1] = True
        assert spec[~band].max() < 1e-9 * spec.max()


def test_perturb_state_recipe():
    rng = np.random.default_rng(2)
    E, npn = 40, 8
    x = rng.uniform(0.0, 1000.0, size=(E, 3, npn))
    q = np.zeros((E, 5, npn))
    q[:, 0] = rng.uniform(0.9, 1.2, size=(E, npn))
    q[:, 4] = rng.uniform(2.0e5, 2.6e5, size=(E, npn))
    out = inputs.perturb_state(q, x, *BOX, seed=5)
    f = inputs.perturbation_factors(x, *BOX, 5, seed=5)
    assert np.allclose(out[:, 0], q[:, 0] * (1 + 1e-2 * f[0]), rtol=1e-15)
    for k in range(3):
        assert np.allclose(out[:, 1 + k], out[:, 0] * 5.0 * f[1 + k], rtol=1e-15, atol=0)
    assert np.allclose(out[:, 4], q[:, 4] * (1 + 1e-2 * f[4]), rtol=1e-15)
    # the input is not modified
    assert np.all(q[:, 1:4] == 0)


def test_ensemble_members_recipe():
    m = inputs.ensemble_members(2000, seed=11)
    assert m == inputs.ensemble_members(2000, seed=11)
    K = np.array([x["K"] for x in m])
    N = np.array([x["N"] for x in m])
    amp = np.array([x["amp"] for x in m])
    c = np.array([x["centre"] for x in m])
    assert K.min() == 8 and K.max() == 24
    assert set(N.tolist()) == {3, 4, 7}
    for n in (3, 4, 7):  # uniform over the three orders
        assert abs(np.mean(N == n) - 1 / 3) < 0.05
    assert amp.min() >= 0.25 and amp.max() <= 1.0
    assert np.all(np.abs(c - np.array([500.0, 500.0, 350.0])) <= 100.0)
    assert inputs.ensemble_members(64)[0]["K"] >= 8


def test_request_stream_recipe():
    n, rate = 20000, 4.0
    r = inputs.request_stream(n, rate, seed=13, steps=200)
    assert r == inputs.request_stream(n, rate, seed=13, steps=200)
    t = np.array([x["arrival"] for x in r])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps: mean 1/rate and coefficient of variation 1 (within 5 sigma)
    assert abs(gaps.mean() * rate - 1) < 5 / np.sqrt(n)
    assert abs(gaps.std() / gaps.mean() - 1) < 0.05
    bub = [x for x in r if x["kind"] == "bubble"]
    chan = [x for x in r if x["kind"] == "channel"]
    assert abs(len(bub) / n - 0.7) < 5 * np.sqrt(0.21 / n)
    Kb = np.array([x["K"][0] for x in bub])
    assert Kb.min() == 8 and Kb.max() == 32
    assert all(x["K"][0] == x["K"][1] == x["K"][2] for x in bub)
    for x in chan:
        kx, ky, kz = x["K"]
        s = kx / 40.0
        assert 1.0 - 1 / 80 <= s <= 3.0 + 1 / 80
        assert abs(ky - 8 * s) <= 0.5 + 1e-9 + 8 / 80 and abs(kz - 4 * s) <= 0.5 + 1e-9 + 4 / 80
    assert all(x["steps"] == 200 and x["N"] in (3, 4, 7) for x in r)
    assert [x["id"] for x in r] == list(range(n))


@pytest.mark.parametrize("rate", [0.5, 8.0])
def test_request_stream_rate_scales_arrivals(rate):
    # the same seed at another rate gives the same requests, arrivals scaled by 1/rate
    a = inputs.request_stream(50, 1.0, seed=17)
    b = inputs.request_stream(50, rate, seed=17)
    for x, y in zip(a, b):
        assert y["arrival"] == pytest.approx(x["arrival"] / rate, rel=1e-12)
        assert (x["kind"], x["K"], x["N"]) == (y["kind"], y["K"], y["N"])
