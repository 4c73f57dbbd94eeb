"""ctypes binding of include/es_dg.h (argument marshalling only).

Every computation happens in libesdg.so's CUDA kernels.  If the library has not
been built, loading raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

ES_DG_OK = 0
ES_DG_PENDING = 1
ES_DG_FP64 = 0
ES_DG_FP32_MIXED = 1

_lock = threading.Lock()
_lib = None


class es_dg_mesh(C.Structure):
    _fields_ = [("kx", C.c_int), ("ky", C.c_int), ("kz", C.c_int),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("periodic", C.c_int * 3), ("warp", C.c_double)]


class es_dg_physics(C.Structure):
    _fields_ = [("gamma", C.c_double), ("g", C.c_double), ("R", C.c_double),
                ("p0", C.c_double), ("f0", C.c_double), ("beta", C.c_double),
                ("y0", C.c_double), ("dissipation", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class es_dg_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class es_dg_info_t(C.Structure):
    _fields_ = [("N", C.c_int), ("Nq", C.c_int), ("np", C.c_int), ("nelem", C.c_int),
                ("ndof", C.c_longlong), ("nfaces", C.c_longlong),
                ("device_bytes", C.c_size_t), ("precision", C.c_int)]


class es_dg_request(C.Structure):
    _fields_ = [("kind", C.c_int), ("kx", C.c_int), ("ky", C.c_int), ("kz", C.c_int),
                ("N", C.c_int), ("precision", C.c_int), ("nsteps", C.c_int), ("cfl", C.c_double),
                ("amp", C.c_double), ("centre", C.c_double * 3), ("radius", C.c_double),
                ("theta0", C.c_double), ("warp", C.c_double)]


class es_dg_result(C.Structure):
    _fields_ = [("status", C.c_int), ("ticket", C.c_uint64), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_finish", C.c_double), ("ndof", C.c_longlong),
                ("nsteps", C.c_int), ("dt", C.c_double), ("integrals", C.c_double * 3),
                ("q", C.POINTER(C.c_double)), ("nq", C.c_size_t)]


class es_dg_server_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("admitted", C.c_longlong),
                ("finished", C.c_longlong), ("steps", C.c_longlong), ("active", C.c_int),
                ("pending", C.c_int), ("dof_updates", C.c_double), ("launch_seconds", C.c_double),
                ("bytes_in_use", C.c_size_t), ("last_error", C.c_int), ("error", C.c_char * 96)]


_VP = C.c_void_p
_DP = C.POINTER(C.c_double)

SIGNATURES = {
    "es_dg_create": (C.c_int, [C.POINTER(es_dg_mesh), C.c_int, C.c_int, C.POINTER(es_dg_physics),
                               C.POINTER(es_dg_allocator), _VP, C.POINTER(_VP)]),
    "es_dg_destroy": (None, [_VP]),
    "es_dg_get_info": (C.c_int, [_VP, C.POINTER(es_dg_info_t)]),
    "es_dg_set_state": (C.c_int, [_VP, _VP, C.c_int]),
    "es_dg_get_state": (C.c_int, [_VP, _VP, C.c_int]),
    "es_dg_init_bubble": (C.c_int, [_VP, C.c_double, C.c_double, _DP, C.c_double]),
    "es_dg_init_bubble_profile": (C.c_int, [_VP, C.c_double, C.c_double, _DP, C.c_double,
                                            C.c_int]),
    "es_dg_init_channel": (C.c_int, [_VP]),
    "es_dg_init_channel_ex": (C.c_int, [_VP, C.c_double, C.c_int]),
    "es_dg_rhs": (C.c_int, [_VP, _VP, _VP, C.c_int]),
    "es_dg_set_background": (C.c_int, [_VP, _VP, C.c_int]),
    "es_dg_set_moving_background": (C.c_int, [_VP, _VP, C.c_int]),
    "es_dg_clear_background": (C.c_int, [_VP]),
    "es_dg_cfl_dt": (C.c_int, [_VP, C.c_double, _DP]),
    "es_dg_step": (C.c_int, [_VP, C.c_double, C.c_int]),
    "es_dg_sync": (C.c_int, [_VP]),
    "es_dg_debug_inject_wait_timeout": (None, []),
    "es_dg_integrals": (C.c_int, [_VP, _DP]),
    "es_dg_geometry": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int]),
    "es_dg_launch": (C.c_int, [_VP, C.c_int, C.c_int, C.c_double]),
    "es_dg_create_partition": (C.c_int, [C.POINTER(es_dg_mesh), C.c_int, C.c_int,
                                         C.POINTER(es_dg_physics), C.c_int, C.c_int,
                                         C.POINTER(es_dg_allocator), _VP, C.POINTER(_VP)]),
    "es_dg_partition_info": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    "es_dg_set_traces": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "es_dg_pack_traces": (C.c_int, [_VP, C.c_int]),
    "es_dg_accept_geometry_trace": (C.c_int, [_VP]),
    "es_dg_partitions_connect": (C.c_int, [C.POINTER(_VP), C.c_int]),
    "es_dg_partitions_exchange": (C.c_int, [C.POINTER(_VP), C.c_int]),
    "es_dg_partitions_step": (C.c_int, [C.POINTER(_VP), C.c_int, C.c_double, C.c_int]),
    "es_dg_strerror": (C.c_char_p, [C.c_int]),
    "es_dg_integrals_noalloc": (C.c_int, [C.POINTER(es_dg_mesh), C.c_int, C.POINTER(es_dg_physics),
                                          _VP, _VP, _VP, _VP, _VP]),
    "es_dg_server_create": (C.c_int, [C.c_size_t, C.c_int, _VP, C.POINTER(_VP)]),
    "es_dg_server_warmup": (C.c_int, [_VP, C.POINTER(C.c_int), C.c_int, C.c_int]),
    "es_dg_debug_numeric": (C.c_int, [C.c_int, _VP, _VP, C.c_longlong, C.c_int, _VP]),
    "es_dg_batch_submit": (C.c_int, [_VP, C.POINTER(es_dg_request), C.POINTER(C.c_uint64)]),
    "es_dg_batch_poll": (C.c_int, [_VP, C.c_uint64, C.POINTER(es_dg_result)]),
    "es_dg_batch_wait": (C.c_int, [_VP, C.c_uint64, C.c_double, C.POINTER(es_dg_result)]),
    "es_dg_batch_cancel": (C.c_int, [_VP, C.c_uint64]),
    "es_dg_result_free": (None, [C.POINTER(es_dg_result)]),
    "es_dg_server_stats": (C.c_int, [_VP, C.POINTER(es_dg_server_stats_t)]),
    "es_dg_server_destroy": (None, [_VP]),
}


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libesdg.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build the CUDA library first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = lib
        return _lib


class EsDgError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().es_dg_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def check(code: int, where: str) -> int:
    if code < 0:
        raise EsDgError(code, where)
    return code


def _ptr(a) -> int:
    """Data pointer of a C-contiguous float64 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.dtype.is_floating_point and a.is_contiguous()
    return a.data_ptr()


def _on_device(a) -> int:
    return 0 if isinstance(a, np.ndarray) else int(a.is_cuda)


class _TorchAllocator:
    """Hands PyTorch's caching allocator to the library (es_dg_allocator)."""

    def __init__(self, stream_ptr: int):
        import torch
        self._torch = torch
        self._stream = stream_ptr
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = es_dg_allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, ctx):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), stream=self._stream)
        except Exception:
            return None

    def _do_free(self, ptr, ctx):
        self._torch.cuda.caching_allocator_delete(ptr)


class Solver:
    """One es_dg handle: a mesh, an order, a precision and the state on the GPU."""

    def __init__(self, kx, ky, kz, N, lo=(0.0, 0.0, 0.0), hi=(1000.0, 1000.0, 1000.0),
                 periodic=(1, 1, 0), warp=0.0, precision="fp64", stream=None,
                 torch_allocator=True, part=None, **phys):
        """part=(x_begin, x_end): the slab of x element layers [x_begin, x_end) of this
        mesh (es_dg_create_partition); K and E are then the slab's."""
        import torch
        self.lib = load()
        self.N, self.Nq, self.np = N, N + 1, (N + 1) ** 3
        self.part = tuple(part) if part is not None else None
        self.K = (kx if part is None else part[1] - part[0], ky, kz)
        self.E = self.K[0] * ky * kz
        self.precision = precision
        p = dict(gamma=1.4, g=9.81, R=287.0, p0=1.0e5, f0=0.0, beta=0.0, y0=0.0, dissipation=1)
        p.update(phys)
        self.phys = p
        self._mesh = es_dg_mesh(kx, ky, kz, (C.c_double * 3)(*lo), (C.c_double * 3)(*hi),
                                (C.c_int * 3)(*periodic), float(warp))
        self._phys = es_dg_physics(p["gamma"], p["g"], p["R"], p["p0"], p["f0"], p["beta"],
                                   p["y0"], int(p["dissipation"]))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sp = stream.cuda_stream
        self._alloc = _TorchAllocator(sp) if torch_allocator else None
        h = C.c_void_p()
        prec = {"fp64": ES_DG_FP64, "mixed": ES_DG_FP32_MIXED}[precision]
        alloc = C.byref(self._alloc.struct) if self._alloc else None
        if part is None:
            check(self.lib.es_dg_create(C.byref(self._mesh), N, prec, C.byref(self._phys), alloc,
                                        C.c_void_p(sp), C.byref(h)), "es_dg_create")
        else:
            check(self.lib.es_dg_create_partition(C.byref(self._mesh), N, prec, C.byref(self._phys),
                                                  int(part[0]), int(part[1]), alloc,
                                                  C.c_void_p(sp), C.byref(h)),
                  "es_dg_create_partition")
        self.h = h

    def partition_info(self):
        """(x_begin, x_end, (remote_lo, remote_hi), trace length in doubles)."""
        b, e, n = C.c_int(), C.c_int(), C.c_longlong()
        r = (C.c_int * 2)()
        check(self.lib.es_dg_partition_info(self.h, C.byref(b), C.byref(e), r, C.byref(n)),
              "es_dg_partition_info")
        return b.value, e.value, (r[0], r[1]), n.value

    def set_traces(self, send_lo, send_hi, recv_lo, recv_hi):
        """Register caller-owned CUDA float64 tensors (None for a plane that is not remote);
        keep them alive while the handle steps."""
        ptr = lambda t: C.c_void_p(None if t is None else _ptr(t))
        self._traces = (send_lo, send_hi, recv_lo, recv_hi)
        check(self.lib.es_dg_set_traces(self.h, ptr(send_lo), ptr(send_hi), ptr(recv_lo),
                                        ptr(recv_hi)), "es_dg_set_traces")

    def pack_traces(self, geometry=False):
        check(self.lib.es_dg_pack_traces(self.h, 1 if geometry else 0), "es_dg_pack_traces")

    def accept_geometry_trace(self):
        check(self.lib.es_dg_accept_geometry_trace(self.h), "es_dg_accept_geometry_trace")

    def close(self):
        if getattr(self, "h", None):
            self.lib.es_dg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self):
        return (self.E, 5, self.np)

    def info(self) -> es_dg_info_t:
        i = es_dg_info_t()
        check(self.lib.es_dg_get_info(self.h, C.byref(i)), "es_dg_get_info")
        return i

    def set_state(self, q):
        check(self.lib.es_dg_set_state(self.h, C.c_void_p(_ptr(q)), _on_device(q)), "es_dg_set_state")

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape())
        check(self.lib.es_dg_get_state(self.h, C.c_void_p(_ptr(out)), _on_device(out)), "es_dg_get_state")
        return out

    def init_bubble(self, theta0=300.0, amp=0.5, centre=(500.0, 500.0, 350.0), radius=250.0,
                    profile="smooth"):
        """Rising-bubble state: "smooth" (Eq. smooth-rb-ic) or "sharp" (Eq. sharp-rb-ic)."""
        c = (C.c_double * 3)(*centre)
        k = {"smooth": 0, "sharp": 1}[profile]
        check(self.lib.es_dg_init_bubble_profile(self.h, theta0, amp, c, radius, k),
              "es_dg_init_bubble_profile")

    def init_channel(self, amp=None, background=None):
        """The channel state; with amp (m/s) or background ("rest" or "jet") given,
        es_dg_init_channel_ex, else es_dg_init_channel (amp 1, background at rest)."""
        if amp is None and background is None:
            check(self.lib.es_dg_init_channel(self.h), "es_dg_init_channel")
            return
        kinds = {"rest": 0, "jet": 1}
        if (background or "rest") not in kinds:
            raise ValueError("background: 'rest' or 'jet'")
        check(self.lib.es_dg_init_channel_ex(self.h, float(1.0 if amp is None else amp),
                                             kinds[background or "rest"]),
              "es_dg_init_channel_ex")

    def set_background(self, q_bg):
        check(self.lib.es_dg_set_background(self.h, C.c_void_p(_ptr(q_bg)), _on_device(q_bg)),
              "es_dg_set_background")

    def set_moving_background(self, q_bg):
        check(self.lib.es_dg_set_moving_background(self.h, C.c_void_p(_ptr(q_bg)),
                                                   _on_device(q_bg)),
              "es_dg_set_moving_background")

    def clear_background(self):
        check(self.lib.es_dg_clear_background(self.h), "es_dg_clear_background")

    def rhs(self, q, out=None):
        if out is None:
            out = np.empty(self.shape()) if isinstance(q, np.ndarray) else q.new_empty(self.shape())
        check(self.lib.es_dg_rhs(self.h, C.c_void_p(_ptr(q)), C.c_void_p(_ptr(out)), _on_device(q)),
              "es_dg_rhs")
        return out

    def cfl_dt(self, C_=0.5) -> float:
        dt = C.c_double()
        check(self.lib.es_dg_cfl_dt(self.h, float(C_), C.byref(dt)), "es_dg_cfl_dt")
        return dt.value

    def step(self, dt, nsteps=1):
        check(self.lib.es_dg_step(self.h, float(dt), int(nsteps)), "es_dg_step")

    def sync(self):
        check(self.lib.es_dg_sync(self.h), "es_dg_sync")

    def integrals(self):
        out = (C.c_double * 3)()
        check(self.lib.es_dg_integrals(self.h, out), "es_dg_integrals")
        return np.array(out[:])

    def geometry(self, device=False):
        """Node positions x [E][3][np], J [E][np] and Ja [E][3][3][np]: numpy arrays, or
        CUDA torch tensors with device=True."""
        shapes = ((self.E, 3, self.np), (self.E, self.np), (self.E, 3, 3, self.np))
        if device:
            import torch
            x, J, Ja = (torch.empty(sh, dtype=torch.float64, device="cuda") for sh in shapes)
        else:
            x, J, Ja = (np.empty(sh) for sh in shapes)
        check(self.lib.es_dg_geometry(self.h, C.c_void_p(_ptr(x)), C.c_void_p(_ptr(J)),
                                      C.c_void_p(_ptr(Ja)), int(device)), "es_dg_geometry")
        return x, J, Ja

    def launch(self, which: int, stage: int = 0, dt: float = 0.0):
        check(self.lib.es_dg_launch(self.h, int(which), int(stage), float(dt)), "es_dg_launch")


class PartitionedSolver:
    """A mesh cut into P slabs of x element layers, each its own handle, all on one
    GPU and one stream; traces move by device copies (es_dg_partitions_*).  The
    state, RHS and time step are those of the whole mesh, bit for bit."""

    def __init__(self, kx, ky, kz, N, P=2, bounds=None, precision="fp64", stream=None, **kw):
        import torch
        from .decomp import split_layers
        self.lib = load()
        self.N, self.np, self.K = N, (N + 1) ** 3, (kx, ky, kz)
        self.E = kx * ky * kz
        self.bounds = list(bounds) if bounds is not None else split_layers(kx, P)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.parts = [Solver(kx, ky, kz, N, precision=precision, stream=stream, part=b, **kw)
                      for b in self.bounds]
        self.traces = []
        for s in self.parts:
            _, _, remote, n = s.partition_info()
            t = [torch.zeros(n, dtype=torch.float64, device="cuda") if remote[k % 2] else None
                 for k in range(4)]  # send_lo, send_hi, recv_lo, recv_hi
            s.set_traces(*t)
            self.traces.append(t)
        self._arr = (C.c_void_p * len(self.parts))(*[s.h.value for s in self.parts])
        check(self.lib.es_dg_partitions_connect(self._arr, len(self.parts)),
              "es_dg_partitions_connect")

    def shape(self):
        return (self.E, 5, self.np)

    def _split(self, q):
        kx, ky, kz = self.K
        g = q.reshape(kz, ky, kx, 5, self.np)
        return [np.ascontiguousarray(g[:, :, b:e]).reshape(-1, 5, self.np) for b, e in self.bounds]

    def _join(self, parts):
        kx, ky, kz = self.K
        g = [p.reshape(kz, ky, e - b, 5, self.np) for p, (b, e) in zip(parts, self.bounds)]
        return np.concatenate(g, axis=2).reshape(self.E, 5, self.np)

    def set_state(self, q):
        for s, qp in zip(self.parts, self._split(np.asarray(q, dtype=np.float64))):
            s.set_state(qp)

    def get_state(self):
        return self._join([s.get_state() for s in self.parts])

    def init_bubble(self, **kw):
        for s in self.parts:
            s.init_bubble(**kw)

    def init_channel(self, amp=None, background=None):
        for s in self.parts:
            s.init_channel(amp, background)

    def exchange(self):
        check(self.lib.es_dg_partitions_exchange(self._arr, len(self.parts)),
              "es_dg_partitions_exchange")

    def rhs(self, q):
        """Right-hand side of the whole-mesh state q (host arrays): slab states set,
        traces exchanged, one RHS per slab."""
        self.set_state(q)
        self.exchange()
        return self._join([s.rhs(qp) for s, qp in zip(self.parts, self._split(np.asarray(q)))])

    def cfl_dt(self, C_=0.5):
        return min(s.cfl_dt(C_) for s in self.parts)

    def step(self, dt, nsteps=1):
        check(self.lib.es_dg_partitions_step(self._arr, len(self.parts), float(dt), int(nsteps)),
              "es_dg_partitions_step")

    def sync(self):
        for s in self.parts:
            s.sync()

    def close(self):
        for s in self.parts:
            s.close()


class Server:
    """Continuous-batching server (es_dg_server_*): resident solves advanced
    together by persistent batched launches under a captured CUDA graph."""

    def __init__(self, hbm_budget_bytes=64 << 30, max_slots=256, stream=None):
        import torch
        torch.cuda.init()
        self.lib = load()
        self.stream = stream
        sp = stream.cuda_stream if stream is not None else None  # None: the server's own stream
        h = C.c_void_p()
        check(self.lib.es_dg_server_create(int(hbm_budget_bytes), int(max_slots),
                                           C.c_void_p(sp), C.byref(h)), "es_dg_server_create")
        self.h = h

    @staticmethod
    def request(kind="bubble", K=(4, 4, 4), N=3, precision="fp64", nsteps=10, cfl=0.4, amp=0.5,
                centre=(500.0, 500.0, 350.0), radius=250.0, theta0=300.0, warp=0.0):
        return es_dg_request({"bubble": 0, "channel": 1, "sharp_bubble": 2}[kind], *K, N,
                             {"fp64": ES_DG_FP64, "mixed": ES_DG_FP32_MIXED}[precision], nsteps,
                             cfl, amp, (C.c_double * 3)(*centre), radius, theta0, warp)

    def warmup(self, orders=(3, 4, 7), precision="mixed"):
        """Tune the batched kernels of these orders before requests arrive."""
        arr = (C.c_int * len(orders))(*orders)
        check(self.lib.es_dg_server_warmup(self.h, arr, len(orders),
                                           {"fp64": ES_DG_FP64, "mixed": ES_DG_FP32_MIXED}[precision]),
              "es_dg_server_warmup")

    def submit(self, **req) -> int:
        t = C.c_uint64()
        r = self.request(**req)
        check(self.lib.es_dg_batch_submit(self.h, C.byref(r), C.byref(t)), "es_dg_batch_submit")
        return t.value

    def _take(self, res):
        out = dict(status=res.status, ticket=res.ticket, t_submit=res.t_submit,
                   t_admit=res.t_admit, t_finish=res.t_finish, ndof=res.ndof, nsteps=res.nsteps,
                   dt=res.dt, integrals=np.array(res.integrals[:]), q=None)
        if res.q and res.nq:
            out["q"] = np.ctypeslib.as_array(res.q, shape=(res.nq,)).copy()
        self.lib.es_dg_result_free(C.byref(res))
        return out

    def poll(self, ticket):
        res = es_dg_result()
        rc = self.lib.es_dg_batch_poll(self.h, C.c_uint64(ticket), C.byref(res))
        if rc == ES_DG_PENDING:
            return None
        check(rc, "es_dg_batch_poll")
        return self._take(res)

    def wait(self, ticket, timeout=600.0):
        res = es_dg_result()
        check(self.lib.es_dg_batch_wait(self.h, C.c_uint64(ticket), float(timeout), C.byref(res)),
              "es_dg_batch_wait")
        return self._take(res)

    def cancel(self, ticket):
        check(self.lib.es_dg_batch_cancel(self.h, C.c_uint64(ticket)), "es_dg_batch_cancel")

    def stats(self):
        st = es_dg_server_stats_t()
        check(self.lib.es_dg_server_stats(self.h, C.byref(st)), "es_dg_server_stats")
        out = {k: getattr(st, k) for k, _ in es_dg_server_stats_t._fields_}
        out["error"] = st.error.decode(errors="replace")
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.es_dg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
