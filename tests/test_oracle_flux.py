"""Pins of the oracle's pointwise physics (CPU only).

What fixes each quantity outside the oracle:
* log mean: arbitrary-precision evaluation of its definition (Section 4.1);
* entropy variables: complex-step gradient of eta = -rho s/(gamma-1);
* two-point flux: consistency with the Euler flux of Section 2, symmetry, the
  gravity partner rule G -> -G b-/b+ (Section 4.1), and Tadmor's entropy
  conservation condition including the gravity term;
* matrix dissipation: at equal states R diag(lam) R^-1 is the Jacobian of the
  Euler normal flux and R diag(T) R^T is (dv/dq)^-1; D is symmetric PSD.
"""
import numpy as np
import pytest

import oracle as O

GAMMA = 1.4


def rand_state(rng, phi=None):
    rho = rng.uniform(0.3, 1.5)
    u = rng.normal(0, 30, size=3)
    p = rng.uniform(2e4, 1.2e5)
    if phi is None:
        phi = rng.uniform(0, 2e4)
    E = p / (GAMMA - 1) + 0.5 * rho * u @ u + rho * phi
    return np.array([rho, *(rho * u), E]), phi


def euler_flux(q, phi, n):
    """Normal Euler flux of Section 2: (rho u_n, rho u u_n + P n, (E + P) u_n)."""
    rho, U, E = q[0], q[1:4], q[4]
    u = U / rho
    P = (GAMMA - 1) * (E - 0.5 * U @ U / rho - rho * phi)
    un = u @ n
    return np.concatenate([[rho * un], rho * u * un + P * n, [(E + P) * un]])


def eta(q, phi):
    rho, U, E = q[0], q[1:4], q[4]
    P = (GAMMA - 1) * (E - 0.5 * (U @ U) / rho - rho * phi)
    s = np.log(P) - GAMMA * np.log(rho)
    return -rho * s / (GAMMA - 1)


def complex_grad(f, x, h=1e-30):
    g = np.zeros(len(x))
    for k in range(len(x)):
        xc = x.astype(complex)
        xc[k] += 1j * h
        g[k] = f(xc).imag / h
    return g


def complex_jac(f, x, h=1e-30):
    cols = []
    for k in range(len(x)):
        xc = x.astype(complex)
        xc[k] += 1j * h
        cols.append(f(xc).imag / h)
    return np.array(cols).T


def test_logmean_against_arbitrary_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(1)
    pairs = [(a, a * r) for a, r in zip(10 ** rng.uniform(-6, 2, 300), 10 ** rng.uniform(-1, 1, 300))]
    pairs += [(a, a * (1 + d)) for a, d in zip(10 ** rng.uniform(-6, 2, 300),
                                               rng.choice([-1, 1], 300) * 10 ** rng.uniform(-9, -1, 300))]
    pairs += [(1.0, 1.0), (2.5e-6, 2.5e-6)]
    for a, b in pairs:
        ma, mb = mp.mpf(a), mp.mpf(b)
        exact = ma if a == b else (mb - ma) / (mp.log(mb) - mp.log(ma))
        got = O.logmean(a, b)
        rel = abs((mp.mpf(got) - exact) / exact)
        # the log branch subtracts per-argument logarithms, so its error bound is
        # a few ulp times (|ln a| + |ln b|) / |ln a - ln b|; the series branch is
        # good to a few ulp
        cond = 1.0 if a == b else 1.0 + (abs(np.log(a)) + abs(np.log(b))) / abs(np.log(a / b))
        assert rel < 4 * 2.0 ** -53 * cond, (a, b, float(rel))
        got_ld = O.logmean(a, b, precision="long")
        assert abs((mp.mpf(got_ld) - exact) / exact) < 2.0 ** -53


def test_logmean_symmetric_and_bounds():
    rng = np.random.default_rng(2)
    for _ in range(200):
        a, b = 10 ** rng.uniform(-3, 3, 2)
        m = O.logmean(a, b)
        assert m == pytest.approx(O.logmean(b, a), rel=1e-15)
        assert np.sqrt(a * b) * (1 - 1e-14) <= m <= (a + b) / 2 * (1 + 1e-14)


def test_entropy_variables_are_gradient_of_entropy():
    rng = np.random.default_rng(3)
    for _ in range(20):
        q, phi = rand_state(rng)
        g = complex_grad(lambda x: eta(x, phi), q)
        v = O.entropy_vars(q, phi)
        assert np.allclose(v, g, rtol=1e-12, atol=1e-12 * np.abs(g).max())


def test_ec_flux_consistency_and_symmetry():
    rng = np.random.default_rng(4)
    for _ in range(50):
        q, phi = rand_state(rng)
        n = rng.normal(size=3)
        F, G = O.ec_flux(q, phi, q, phi, n)
        f = euler_flux(q, phi, n)
        assert np.allclose(F, f, rtol=1e-13, atol=1e-12 * np.abs(f).max())
        assert np.all(G == 0)
        qb, phib = rand_state(rng)
        Fab, _ = O.ec_flux(q, phi, qb, phib, n)
        Fba, _ = O.ec_flux(qb, phib, q, phi, n)
        assert np.allclose(Fab, Fba, rtol=1e-14, atol=1e-12 * np.abs(Fab).max())


def test_gravity_partner_rule():
    rng = np.random.default_rng(5)
    for _ in range(50):
        qa, pa = rand_state(rng)
        qb, pb = rand_state(rng)
        n = rng.normal(size=3)
        _, Gab = O.ec_flux(qa, pa, qb, pb, n)
        _, Gba = O.ec_flux(qb, pb, qa, pa, n)
        ba = qa[0] / (2 * (GAMMA - 1) * (qa[4] - 0.5 * qa[1:4] @ qa[1:4] / qa[0] - qa[0] * pa))
        bb = qb[0] / (2 * (GAMMA - 1) * (qb[4] - 0.5 * qb[1:4] @ qb[1:4] / qb[0] - qb[0] * pb))
        assert np.allclose(Gba, -Gab * ba / bb, rtol=1e-12, atol=1e-14 * np.abs(Gab).max())


@pytest.mark.parametrize("precision", ["double", "long"])
def test_tadmor_condition_with_gravity(precision):
    """v_a . H(a,b) - v_b . H(b,a) = psi_a - psi_b with H = F# + G, psi = rho u . n;
    without gravity this is [[v]] . F# = [[rho u_n]]."""
    rng = np.random.default_rng(6)
    tol = 1e-11 if precision == "double" else 1e-14
    for _ in range(100):
        qa, pa = rand_state(rng)
        qb, pb = rand_state(rng)
        # nearby states as well (series branch of the log mean)
        if rng.uniform() < 0.5:
            qb = qa * (1 + 1e-3 * rng.normal(size=5))
            pb = pa + rng.uniform(-50, 50)
        n = rng.normal(size=3)
        va = O.entropy_vars(qa, pa, precision=precision)
        vb = O.entropy_vars(qb, pb, precision=precision)
        Fab, Gab = O.ec_flux(qa, pa, qb, pb, n, precision=precision)
        Fba, Gba = O.ec_flux(qb, pb, qa, pa, n, precision=precision)
        Hab = Fab.copy(); Hab[1:4] += Gab
        Hba = Fba.copy(); Hba[1:4] += Gba
        lhs = va @ Hab - vb @ Hba
        rhs = qa[1:4] @ n - qb[1:4] @ n
        scale = np.abs(va * Hab).sum() + np.abs(vb * Hba).sum()
        assert abs(lhs - rhs) < tol * scale
        # no-gravity form: equal geopotential
        Fab0, G0 = O.ec_flux(qa, pa, qb, pa, n, precision=precision)
        assert np.all(G0 == 0)
        va0 = O.entropy_vars(qa, pa, precision=precision)
        vb0 = O.entropy_vars(qb, pa, precision=precision)
        lhs0 = (vb0 - va0) @ Fab0
        assert abs(lhs0 - (qb[1:4] - qa[1:4]) @ n) < tol * np.abs((vb0 - va0) * Fab0).sum() + 1e-9


def test_eigensystem_at_equal_states():
    rng = np.random.default_rng(7)
    for _ in range(20):
        q, phi = rand_state(rng)
        nh = rng.normal(size=3)
        nh /= np.linalg.norm(nh)
        R, lam, T = O.eigensystem(q, q, phi, nh)
        Jac = complex_jac(lambda x: euler_flux(x, phi, nh), q)
        A = R @ np.diag(lam) @ np.linalg.inv(R)
        assert np.allclose(A, Jac, rtol=1e-9, atol=1e-9 * np.abs(Jac).max())
        # dq/dv = (dv/dq)^-1; dv/dq by central differences of the oracle's v
        H = np.zeros((5, 5))
        for k in range(5):
            h = 1e-6 * abs(q[k]) + 1e-6
            e = np.zeros(5); e[k] = h
            H[:, k] = (O.entropy_vars(q + e, phi) - O.entropy_vars(q - e, phi)) / (2 * h)
        S = R @ np.diag(T) @ R.T
        Hinv = np.linalg.inv(H)
        assert np.allclose(S, Hinv, rtol=1e-6, atol=1e-6 * np.abs(Hinv).max())


def test_dissipation_symmetric_psd_and_zero_jump():
    rng = np.random.default_rng(8)
    for _ in range(30):
        qa, phi = rand_state(rng)
        qb = qa * (1 + 0.05 * rng.normal(size=5))
        nh = rng.normal(size=3)
        nh /= np.linalg.norm(nh)
        D = O.dissipation_matrix(qa, qb, phi, nh)
        assert np.allclose(D, D.T, rtol=1e-12, atol=1e-12 * np.abs(D).max())
        ev = np.linalg.eigvalsh(0.5 * (D + D.T))
        assert ev.min() > -1e-10 * ev.max()
        # F*(q, q) = Euler flux: no dissipation for equal states
        Fs = O.es_flux(qa, qa, phi, nh)
        assert np.allclose(Fs, euler_flux(qa, phi, nh), rtol=1e-12,
                           atol=1e-12 * np.abs(Fs).max())
        # F* = F# - 1/2 D [[v]]
        F, G = O.ec_flux(qa, phi, qb, phi, nh)
        jv = O.entropy_vars(qb, phi) - O.entropy_vars(qa, phi)
        Fs = O.es_flux(qa, qb, phi, nh)
        assert np.allclose(Fs, F - 0.5 * D @ jv, rtol=1e-12, atol=1e-10 * np.abs(F).max())
        # conservation: F*(b, a, -n) = -F*(a, b, n)
        Fr = O.es_flux(qb, qa, phi, -nh)
        assert np.allclose(Fr, -Fs, rtol=1e-11, atol=1e-11 * np.abs(Fs).max())
