"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module draws random numbers and nothing else: it holds none of the
solver's arithmetic (no equation of state, no fluxes, no geometry).  Fields are
smooth functions of coordinates that the caller passes in, so either side may
supply the coordinates.

Recipes
-------
* ``perturbation_factors``: a few random Fourier modes (integer wavenumbers
  kmin..kmax per axis over the box, 1..3 by default) evaluated at the given
  nodes; each returned field is scaled to unit maximum.  Fine meshes use
  wavenumbers that scale with the element count so every element sees O(1)
  variation and the right-hand side stays O(1) relative to its terms.
* ``perturb_state``: multiplies density and total energy by (1 + eps f) with
  eps = 1e-2 and adds momentum rho * u0 * f with u0 = 5 m/s, so every conserved
  variable's right-hand side is O(1) ("generic state").
* ``ensemble_members``: the batched-ensemble draw (grid K^3, K ~ U{8..24},
  N ~ U{3,4,7}, bubble amplitude ~ U(0.25, 1.0) K, centre jitter U(-100, 100) m).
* ``request_stream``: Poisson arrivals of solve requests, 70 % bubbles
  (K ~ U{8..32}) and 30 % channels (scale s ~ U[1,3]: (40 s, 8 s, 4 s)
  elements), N ~ U{3,4,7}.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20260516


def perturbation_factors(x: np.ndarray, lo, hi, nfields: int, seed: int = DEFAULT_SEED,
                         modes: int = 6, kmin: int = 1, kmax: int = 3) -> np.ndarray:
    """Smooth random fields at node coordinates x[E, 3, np] -> [nfields, E, np];
    integer wavenumbers per axis are drawn from [kmin, kmax] over the box."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64).reshape(3, 1, 1)
    hi = np.asarray(hi, dtype=np.float64).reshape(3, 1, 1)
    xs = (np.moveaxis(x, 1, 0) - lo) / (hi - lo)          # [3, E, np] in [0, 1]
    out = np.zeros((nfields,) + x[:, 0, :].shape)
    for f in range(nfields):
        acc = np.zeros_like(out[f])
        for _ in range(modes):
            k = rng.integers(kmin, kmax + 1, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            a = rng.uniform(0.5, 1.0)
            acc += a * np.sin(2 * np.pi * (k[0] * xs[0] + k[1] * xs[1] + k[2] * xs[2]) + ph)
        out[f] = acc / np.max(np.abs(acc))
    return out


def perturb_state(q: np.ndarray, x: np.ndarray, lo, hi, seed: int = DEFAULT_SEED,
                  eps: float = 1e-2, u0: float = 5.0, kmin: int = 1, kmax: int = 3) -> np.ndarray:
    """Generic state: q[E, 5, np] with smooth random perturbations of every variable."""
    f = perturbation_factors(x, lo, hi, 5, seed, kmin=kmin, kmax=kmax)
    out = np.array(q, dtype=np.float64, copy=True)
    out[:, 0, :] = q[:, 0, :] * (1 + eps * f[0])
    for k in range(3):
        out[:, 1 + k, :] = q[:, 1 + k, :] + out[:, 0, :] * u0 * f[1 + k]
    out[:, 4, :] = q[:, 4, :] * (1 + eps * f[4])
    return out


def ensemble_members(n: int = 64, seed: int = DEFAULT_SEED, kmin: int = 8, kmax: int = 24,
                     orders=(3, 4, 7)):
    """Batched-ensemble member draw, all from one seed."""
    rng = np.random.default_rng(seed)
    members = []
    for _ in range(n):
        K = int(rng.integers(kmin, kmax + 1))
        N = int(rng.choice(orders))
        amp = float(rng.uniform(0.25, 1.0))
        centre = (500.0 + rng.uniform(-100, 100), 500.0 + rng.uniform(-100, 100),
                  350.0 + rng.uniform(-100, 100))
        members.append(dict(K=K, N=N, amp=amp, centre=centre))
    return members


def request_stream(n: int, rate_hz: float, seed: int = DEFAULT_SEED, steps: int = 200,
                   orders=(3, 4, 7), bubble_frac: float = 0.7, kmin: int = 8, kmax: int = 32):
    """Poisson stream of solve requests: list of dicts with an arrival time (s)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate_hz))
        N = int(rng.choice(orders))
        if rng.uniform() < bubble_frac:
            K = int(rng.integers(kmin, kmax + 1))
            reqs.append(dict(id=i, arrival=t, kind="bubble", K=(K, K, K), N=N, steps=steps,
                             amp=float(rng.uniform(0.25, 1.0))))
        else:
            s = float(rng.uniform(1.0, 3.0))
            K = (int(round(40 * s)), int(round(8 * s)), int(round(4 * s)))
            reqs.append(dict(id=i, arrival=t, kind="channel", K=K, N=N, steps=steps))
    return reqs
