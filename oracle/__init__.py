"""Python handle on the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It loads the C oracle built by
``oracle/build.py`` (double or long double) through ctypes; numpy arrays in
the layouts documented in ``oracle.h``.
"""
import ctypes as C
import threading

import numpy as np

from . import build as _build

_LOCK = threading.Lock()
_LIBS = {}

DEFAULT_PHYS = dict(gamma=1.4, g=9.81, R=287.0, p0=1.0e5, f0=0.0, beta=0.0, y0=0.0,
                    dissipation=1)


class _Mesh(C.Structure):
    _fields_ = [("kx", C.c_int), ("ky", C.c_int), ("kz", C.c_int),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("periodic", C.c_int * 3), ("warp", C.c_double)]


class _Phys(C.Structure):
    _fields_ = [("gamma", C.c_double), ("g", C.c_double), ("R", C.c_double),
                ("p0", C.c_double), ("f0", C.c_double), ("beta", C.c_double),
                ("y0", C.c_double), ("dissipation", C.c_int)]


_D = C.POINTER(C.c_double)


def _lib(precision: str = "double"):
    name = {"double": "liboracle.so", "long": "liboracle_ld.so"}[precision]
    with _LOCK:
        if name not in _LIBS:
            _build.build()
            lib = C.CDLL(_build.lib_path(name))
            lib.or_create.restype = C.c_void_p
            lib.or_create.argtypes = [C.POINTER(_Mesh), C.c_int, C.POINTER(_Phys)]
            lib.or_free.argtypes = [C.c_void_p]
            lib.or_nelem.argtypes = [C.c_void_p]
            for fn in ("or_geometry",):
                getattr(lib, fn).argtypes = [C.c_void_p, _D, _D, _D]
            lib.or_rhs.argtypes = [C.c_void_p, _D, _D]
            lib.or_rhs_parts.argtypes = [C.c_void_p, _D, _D, _D, _D]
            lib.or_rhs_scale.argtypes = [C.c_void_p, _D, _D]
            lib.or_lsrk_coeffs.argtypes = [_D, _D, _D]
            lib.or_lsrk_steps.argtypes = [C.c_void_p, _D, C.c_double, C.c_int]
            lib.or_init_bubble.argtypes = [C.c_void_p, C.c_double, C.c_double, _D, C.c_double, _D]
            lib.or_init_bubble_profile.argtypes = [C.c_void_p, C.c_double, C.c_double, _D,
                                                   C.c_double, C.c_int, _D]
            lib.or_init_isothermal.argtypes = [C.c_void_p, C.c_double, C.c_double, _D]
            lib.or_init_channel.argtypes = [C.c_void_p, _D]
            lib.or_integrals.argtypes = [C.c_void_p, _D, _D]
            lib.or_entropy_rate.argtypes = [C.c_void_p, _D, _D]
            lib.or_entropy_rate.restype = C.c_double
            lib.or_cfl_dt.argtypes = [C.c_void_p, _D, C.c_double]
            lib.or_cfl_dt.restype = C.c_double
            lib.or_lgl.argtypes = [C.c_int, _D, _D, _D, _D]
            lib.or_logmean.argtypes = [C.c_double, C.c_double]
            lib.or_logmean.restype = C.c_double
            lib.or_entropy_vars.argtypes = [_D, C.c_double, C.c_double, _D]
            lib.or_ec_flux.argtypes = [_D, C.c_double, _D, C.c_double, _D, C.c_double, _D, _D]
            lib.or_es_flux.argtypes = [_D, _D, C.c_double, _D, C.c_double, C.c_int, _D]
            lib.or_dissipation_matrix.argtypes = [_D, _D, C.c_double, _D, C.c_double, _D]
            lib.or_eigensystem.argtypes = [_D, _D, C.c_double, _D, C.c_double, _D, _D, _D]
            _LIBS[name] = lib
        return _LIBS[name]


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _vec(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


# ---------------------------------------------------------------- pointwise --

def lgl(N: int, precision="double"):
    Nq = N + 1
    xi, w = np.zeros(Nq), np.zeros(Nq)
    D, Dt = np.zeros((Nq, Nq)), np.zeros((Nq, Nq))
    if _lib(precision).or_lgl(N, _p(xi), _p(w), _p(D), _p(Dt)):
        raise ValueError("unsupported N")
    return xi, w, D, Dt


def logmean(a, b, precision="double"):
    return _lib(precision).or_logmean(float(a), float(b))


def entropy_vars(q, phi, gamma=1.4, precision="double"):
    v = np.zeros(5)
    _lib(precision).or_entropy_vars(_p(_vec(q, 5)), float(phi), float(gamma), _p(v))
    return v


def ec_flux(qa, phia, qb, phib, n, gamma=1.4, precision="double"):
    F, G = np.zeros(5), np.zeros(3)
    _lib(precision).or_ec_flux(_p(_vec(qa, 5)), float(phia), _p(_vec(qb, 5)), float(phib),
                               _p(_vec(n, 3)), float(gamma), _p(F), _p(G))
    return F, G


def es_flux(qm, qp, phi, nhat, gamma=1.4, dissipation=1, precision="double"):
    F = np.zeros(5)
    _lib(precision).or_es_flux(_p(_vec(qm, 5)), _p(_vec(qp, 5)), float(phi), _p(_vec(nhat, 3)),
                               float(gamma), int(dissipation), _p(F))
    return F


def dissipation_matrix(qm, qp, phi, nhat, gamma=1.4, precision="double"):
    D = np.zeros((5, 5))
    _lib(precision).or_dissipation_matrix(_p(_vec(qm, 5)), _p(_vec(qp, 5)), float(phi),
                                          _p(_vec(nhat, 3)), float(gamma), _p(D))
    return D


def eigensystem(qm, qp, phi, nhat, gamma=1.4, precision="double"):
    R, lam, T = np.zeros((5, 5)), np.zeros(5), np.zeros(5)
    _lib(precision).or_eigensystem(_p(_vec(qm, 5)), _p(_vec(qp, 5)), float(phi),
                                   _p(_vec(nhat, 3)), float(gamma), _p(R), _p(lam), _p(T))
    return R, lam, T


def count_flops(N: int) -> dict:
    """Algorithmic flops of the volume term counted from the oracle's own code by
    its counting instantiation (count_flops.cpp): per unordered node pair of the
    half sweep (both orderings, shared subexpressions once) and per node and stage
    (primitives, the volume values and the stage updates)."""
    with _LOCK:
        if "count" not in _LIBS:
            _build.build()
            lib = C.CDLL(_build.lib_path("liboracle_count.so"))
            lib.or_count_flops.argtypes = [C.c_int, _D]
            _LIBS["count"] = lib
    out = np.zeros(5)
    if _LIBS["count"].or_count_flops(int(N), _p(out)):
        raise ValueError("unsupported N")
    return dict(pair=int(out[0]), node=int(out[1]), primitives=int(out[2]),
                stage_update=int(out[3]), pair_without_sharing=int(out[4]))


def lsrk_coeffs():
    A, B, c = np.zeros(5), np.zeros(5), np.zeros(5)
    _lib().or_lsrk_coeffs(_p(A), _p(B), _p(c))
    return A, B, c


# ------------------------------------------------------------------- solver --

class Oracle:
    """One mesh + order + physics, evaluated on the CPU in double or long double."""

    def __init__(self, kx, ky, kz, N, lo=(0, 0, 0), hi=(1000, 1000, 1000),
                 periodic=(1, 1, 0), warp=0.0, precision="double", **phys):
        self.lib = _lib(precision)
        self.N, self.Nq, self.np = N, N + 1, (N + 1) ** 3
        self.K = (kx, ky, kz)
        self.E = kx * ky * kz
        self.mesh_args = dict(kx=kx, ky=ky, kz=kz, lo=tuple(lo), hi=tuple(hi),
                              periodic=tuple(periodic), warp=warp)
        m = _Mesh(kx, ky, kz, (C.c_double * 3)(*lo), (C.c_double * 3)(*hi),
                  (C.c_int * 3)(*periodic), float(warp))
        p = dict(DEFAULT_PHYS)
        p.update(phys)
        self.phys = p
        ph = _Phys(p["gamma"], p["g"], p["R"], p["p0"], p["f0"], p["beta"], p["y0"],
                   int(p["dissipation"]))
        self._h = self.lib.or_create(C.byref(m), N, C.byref(ph))
        if not self._h:
            raise ValueError("oracle: bad mesh or order")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self.lib.or_free(h)
            self._h = None

    def shape(self):
        return (self.E, 5, self.np)

    def geometry(self):
        x = np.zeros((self.E, 3, self.np))
        J = np.zeros((self.E, self.np))
        Ja = np.zeros((self.E, 3, 3, self.np))
        self.lib.or_geometry(self._h, _p(x), _p(J), _p(Ja))
        return x, J, Ja

    def rhs(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros(self.shape())
        self.lib.or_rhs(self._h, _p(q), _p(out))
        return out

    def rhs_parts(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        v, s, h = (np.zeros(self.shape()) for _ in range(3))
        self.lib.or_rhs_parts(self._h, _p(q), _p(v), _p(s), _p(h))
        return v, s, h

    def rhs_scale(self, q):
        """Per-node magnitude of the cancelling terms (see or_rhs_scale)."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros(self.shape())
        self.lib.or_rhs_scale(self._h, _p(q), _p(out))
        return out

    def steps(self, q, dt, nsteps):
        q = np.array(q, dtype=np.float64, order="C", copy=True)
        self.lib.or_lsrk_steps(self._h, _p(q), float(dt), int(nsteps))
        return q

    def bubble(self, theta0=300.0, amp=0.5, centre=(500.0, 500.0, 350.0), radius=250.0,
               profile="smooth"):
        """Rising-bubble state: profile "smooth" is Eq. (smooth-rb-ic), "sharp" Eq. (sharp-rb-ic)."""
        q = np.zeros(self.shape())
        k = {"smooth": 0, "sharp": 1}[profile]
        st = self.lib.or_init_bubble_profile(self._h, theta0, amp, _p(_vec(centre, 3)), radius,
                                             k, _p(q))
        assert st == 0
        return q

    def isothermal(self, T=280.0, rho_surface=1.2):
        q = np.zeros(self.shape())
        self.lib.or_init_isothermal(self._h, T, rho_surface, _p(q))
        return q

    def channel(self):
        q = np.zeros(self.shape())
        self.lib.or_init_channel(self._h, _p(q))
        return q

    def integrals(self, q):
        out = np.zeros(3)
        self.lib.or_integrals(self._h, _p(np.ascontiguousarray(q, dtype=np.float64)), _p(out))
        return out

    def entropy_rate(self, q, rhs):
        return self.lib.or_entropy_rate(self._h, _p(np.ascontiguousarray(q, dtype=np.float64)),
                                        _p(np.ascontiguousarray(rhs, dtype=np.float64)))

    def cfl_dt(self, q, C=0.5):
        return self.lib.or_cfl_dt(self._h, _p(np.ascontiguousarray(q, dtype=np.float64)), float(C))
