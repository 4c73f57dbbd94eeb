"""Pin of the oracle's volume term against the matrix form of Eq. (nm:semi) (CPU only).

The oracle evaluates the volume term in the metric-averaged form
    vol_i = -(1/J_i) sum_d sum_l Dt_il H(q_i, q_l; {{Ja^d}}_il),   Dt = 2D - W^-1 B,
with H = F# + G (the EC flux plus the non-symmetric gravity term of Section 4.1).  The paper
prints the volume term of Eq. (nm:semi) as  G_jk (D_j o F_j) 1 - (F_j o D_j^T) G_jk 1, whose
mass factors were lost in the printed equation; with the collocated LGL mass matrix W put
back on the transposed operator (W^-1 D^T W, the form the summation-by-parts property
makes conservative) it reads, per node and reference direction,
    sum_l [ D_il H(q_i, q_l; Ja_i) - (w_l / w_i) D_li H(q_i, q_l; Ja_l) ].
The two forms agree exactly in exact arithmetic for any two-point flux, symmetric or not,
because W D + D^T W = B with B diagonal.  This test evaluates the matrix form here, in
numpy, with its own LGL nodes, weights and differentiation matrix (not the oracle's), and only
the pointwise two-point flux taken from the oracle; a wrong averaging, a transposed D, a
dropped boundary correction, a wrong 1/J or a wrong partner rule in the oracle's loop fails it.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as Lg

import oracle as O
from paper_2605_16684_gb300 import inputs

BOX = ((0.0, 0.0, 0.0), (1000.0, 1000.0, 1000.0))


def lgl_basis(N):
    """LGL nodes, weights and the Lagrange differentiation matrix (barycentric form)."""
    cN = np.zeros(N + 1)
    cN[N] = 1.0
    inner = np.sort(np.real(Lg.legroots(Lg.legder(cN)))) if N > 1 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (N * (N + 1) * Lg.legval(x, cN) ** 2)
    Nq = N + 1
    lam = np.array([1.0 / np.prod([x[j] - x[k] for k in range(Nq) if k != j]) for j in range(Nq)])
    D = np.zeros((Nq, Nq))
    for i in range(Nq):
        for l in range(Nq):
            if i != l:
                D[i, l] = lam[l] / (lam[i] * (x[i] - x[l]))
        D[i, i] = -D[i].sum()
    return x, w, D


def node(Nq, a, b, c):
    return a + Nq * (b + Nq * c)


def volume_matrix_form(q, x, J, Ja, N, g, gamma=1.4):
    """Matrix form of the volume term, node by node, for every element."""
    _, w, D = lgl_basis(N)
    Nq = N + 1
    E = q.shape[0]
    out = np.zeros_like(q)
    phi = g * x[:, 2, :]
    for e in range(E):
        for n in range(Nq ** 3):
            idx = [n % Nq, (n // Nq) % Nq, n // (Nq * Nq)]
            acc = np.zeros(5)
            for d in range(3):
                a = idx[d]
                for m in range(Nq):
                    t = list(idx)
                    t[d] = m
                    l = node(Nq, *t)
                    for coef, nvec in ((D[a, m], Ja[e, d, :, n]),
                                       (-(w[m] / w[a]) * D[m, a], Ja[e, d, :, l])):
                        F, G = O.ec_flux(q[e, :, n], phi[e, n], q[e, :, l], phi[e, l],
                                         np.ascontiguousarray(nvec), gamma)
                        H = F.copy()
                        H[1:4] += G
                        acc += coef * H
            out[e, :, n] = -acc / J[e, n]
    return out


@pytest.mark.parametrize("K,N,warp,periodic", [((2, 2, 2), 3, 0.05, (1, 1, 0)),
                                               ((2, 1, 2), 4, 0.05, (0, 1, 0)),
                                               ((1, 2, 1), 2, 0.0, (1, 1, 0))])
def test_volume_term_equals_matrix_form_of_semi_discretisation(K, N, warp, periodic):
    o = O.Oracle(*K, N, lo=BOX[0], hi=BOX[1], periodic=periodic, warp=warp)
    x, J, Ja = o.geometry()
    q = inputs.perturb_state(o.bubble(), x, *BOX, seed=3)
    vol, _, _ = o.rhs_parts(q)
    ref = volume_matrix_form(q, x, J, Ja, N, g=o.phys["g"])
    for v in range(5):
        err = np.linalg.norm(vol[:, v] - ref[:, v]) / np.linalg.norm(ref[:, v])
        assert err < 1e-12, (v, err)


def test_lgl_basis_here_is_the_oracles():
    # The matrix form above must not share its basis with the oracle; both must still be
    # the same textbook objects.
    for N in (2, 3, 4, 7):
        x, w, D = lgl_basis(N)
        xo, wo, Do, _ = O.lgl(N)
        assert np.allclose(x, xo, atol=1e-15) and np.allclose(w, wo, atol=1e-15)
        assert np.allclose(D, Do, atol=1e-12)
