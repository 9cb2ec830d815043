"""Thin ctypes binding of libcoll.so, with the C ABI's names (include/coll.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libcoll.so.  Device buffers are torch CUDA tensors (PyTorch is used
for device memory and streams); host arrays are accepted only by the
end-to-end helper ``eval_host``, which copies them in and out around the same
C-ABI call.  If the shared library is missing this module raises on import:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libcoll.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "coll.h")
HEADERS = [HEADER, os.path.join(os.path.dirname(PKG), "include", "coll_debug.h")]

COLL_OK, COLL_EINVAL, COLL_EUNSUPPORTED, COLL_ENOMEM, COLL_ECUDA, COLL_ETIMEOUT, COLL_ENONFINITE = range(7)
COLL_F64, COLL_F32, COLL_MIXED_F16X2, COLL_MIXED_BF16X3, COLL_F32X2, COLL_MIXED_SLICED = range(6)
PREC = {"f64": COLL_F64, "f32": COLL_F32, "mixed_f16x2": COLL_MIXED_F16X2,
        "mixed_bf16x3": COLL_MIXED_BF16X3, "f32x2": COLL_F32X2, "mixed_sliced": COLL_MIXED_SLICED}


class CollError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed: %s" % (what, coll_status_string(status)))
        self.status = status


class coll_plan_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("L", ctypes.c_double), ("S", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("b0", ctypes.c_double), ("M", ctypes.c_int32),
                ("Mtheta", ctypes.c_int32), ("Mr", ctypes.c_int32), ("sphere_rule", ctypes.c_int32),
                ("dealias", ctypes.c_int32), ("prec", ctypes.c_int32), ("io_dtype", ctypes.c_int32),
                ("rank", ctypes.c_int32)]


class coll_m2d_plan_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("L", ctypes.c_double), ("S", ctypes.c_double), ("b0", ctypes.c_double),
                ("A", ctypes.c_int32), ("prec", ctypes.c_int32), ("io_dtype", ctypes.c_int32)]


class coll_cell_group(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("f", ctypes.c_void_p), ("Q", ctypes.c_void_p)]


class coll_regime_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("eps", "mu0", "kappa0", "dx", "dy", "eta0", "eta1", "delta0")]


MOMENT_DOUBLES = 40


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libcoll.so is not built (%s); run __graft_entry__.build() or "
                          "python -m paper_2505_03360_gb300.build" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    sig = {
        "coll_plan_create": (I32, [ctypes.POINTER(coll_plan_desc), ctypes.POINTER(P)]),
        "coll_plan_destroy": (I32, [P]),
        "coll_plan_terms": (I32, [P, ctypes.POINTER(I32)]),
        "coll_workspace_size": (I32, [P, I64, ctypes.POINTER(SZ)]),
        "coll_eval_batch": (I32, [P, P, P, I64, P, SZ, P]),
        "coll_eval_batch_static": (I32, [P, P, P, I64, P]),
        "coll_plan_autotune": (I32, [P, P, P, I64, P, SZ, P, ctypes.POINTER(I32)]),
        "coll_plan_set_variant": (I32, [P, I32]),
        "coll_advance": (I32, [P, P, I64, D, I32, P]),
        "coll_ragged_workspace_size": (I32, [ctypes.POINTER(coll_cell_group), ctypes.POINTER(I64), I32,
                                             ctypes.POINTER(SZ)]),
        "coll_eval_ragged": (I32, [ctypes.POINTER(coll_cell_group), ctypes.POINTER(I64), I32, P, SZ, P]),
        "moments_realizability": (I32, [P, I32, I32, D, I64, D, D, P, P, P]),
        "coll_conservation": (I32, [P, I32, I32, D, I64, P, P]),
        "regime_update": (I32, [P, P, P, I32, I32, ctypes.POINTER(coll_regime_params), P, P, P]),
        "coll_imex_stage": (I32, [I32, P, P, P, P, P, P, P, I32, I32, D, I64, D, D, P, P]),
        "coll_esbgk_step": (I32, [P, P, I32, I32, D, I64, D, D, D, D, P, P]),
        "coll_device_status": (I32, [P]),
        "coll_device_status_clear": (I32, [P]),
        "coll_status_string": (ctypes.c_char_p, [I32]),
        "coll_launch_count": (I64, []),
        "coll_plan_tables_host": (I32, [ctypes.POINTER(coll_plan_desc), P, SZ, ctypes.POINTER(I32),
                                        ctypes.POINTER(SZ)]),
        "coll_debug_mixed_drop_commit": (I32, [I32]),
        "coll_m2d_plan_create": (I32, [ctypes.POINTER(coll_m2d_plan_desc), ctypes.POINTER(P)]),
        "coll_m2d_plan_destroy": (I32, [P]),
        "coll_m2d_eval_batch": (I32, [P, P, P, I64, P]),
        "coll_m2d_device_status": (I32, [P]),
        "coll_m2d_device_status_clear": (I32, [P]),
        "coll_m2d_tables_host": (I32, [ctypes.POINTER(coll_m2d_plan_desc), P, SZ, ctypes.POINTER(I32),
                                       ctypes.POINTER(SZ)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def header_functions() -> list:
    """Names of every function the headers under include/ declare."""
    names = set()
    for h in HEADERS:
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(coll_\w+|moments_realizability|regime_update)\s*\(",
                                txt, re.M))
    return sorted(names)


def coll_debug_mixed_drop_commit(on: bool):
    """Failure injection for the tensor-core path's bounded waits (see coll_debug.h)."""
    _check(_lib.coll_debug_mixed_drop_commit(1 if on else 0), "coll_debug_mixed_drop_commit")


def coll_status_string(status: int) -> str:
    return _lib.coll_status_string(int(status)).decode()


def coll_launch_count() -> int:
    return int(_lib.coll_launch_count())


def _check(status: int, what: str):
    if status != COLL_OK:
        raise CollError(status, what)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def make_desc(N, L, S=0.0, lam=1.0, b0=-1.0, M=48, Mtheta=4, Mr=16, sphere_rule=0, dealias=0, prec="f64",
              io_dtype=None, rank=0) -> coll_plan_desc:
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    if io_dtype is None:
        io_dtype = 1 if p == COLL_F32 else 0
    return coll_plan_desc(int(N), float(L), float(S), float(lam), float(b0), int(M), int(Mtheta), int(Mr),
                          int(sphere_rule), int(dealias), p, int(io_dtype), int(rank))


def coll_plan_create(desc: coll_plan_desc) -> int:
    h = ctypes.c_void_p()
    _check(_lib.coll_plan_create(ctypes.byref(desc), ctypes.byref(h)), "coll_plan_create")
    return h.value


def coll_plan_destroy(plan: int):
    _check(_lib.coll_plan_destroy(ctypes.c_void_p(plan)), "coll_plan_destroy")


def coll_plan_terms(plan: int) -> int:
    n = ctypes.c_int32()
    _check(_lib.coll_plan_terms(ctypes.c_void_p(plan), ctypes.byref(n)), "coll_plan_terms")
    return n.value


def coll_workspace_size(plan: int, max_cells: int) -> int:
    b = ctypes.c_size_t()
    _check(_lib.coll_workspace_size(ctypes.c_void_p(plan), int(max_cells), ctypes.byref(b)), "coll_workspace_size")
    return b.value


def coll_eval_batch(plan: int, f, Q, n_cells: int, ws, ws_bytes: int = None, stream=None, check=True) -> int:
    nb = ws.numel() * ws.element_size() if (ws is not None and ws_bytes is None) else (ws_bytes or 0)
    st = _lib.coll_eval_batch(ctypes.c_void_p(plan), _ptr(f), _ptr(Q), int(n_cells), _ptr(ws), nb,
                              _stream_ptr(stream))
    if check:
        _check(st, "coll_eval_batch")
    return st


def coll_eval_batch_static(plan: int, f, Q, n_cells: int, stream=None, check=True) -> int:
    """coll_eval_batch with the library's fixed device scratch (no allocation)."""
    st = _lib.coll_eval_batch_static(ctypes.c_void_p(plan), _ptr(f), _ptr(Q), int(n_cells), _stream_ptr(stream))
    if check:
        _check(st, "coll_eval_batch_static")
    return st


def coll_plan_autotune(plan: int, f, Q, n_cells: int, ws, stream=None) -> int:
    """Time every slab-shape variant on this batch; the faster is kept in the plan."""
    ch = ctypes.c_int32(-1)
    _check(_lib.coll_plan_autotune(ctypes.c_void_p(plan), _ptr(f), _ptr(Q), int(n_cells), _ptr(ws),
                                   ws.numel() * ws.element_size(), _stream_ptr(stream), ctypes.byref(ch)),
           "coll_plan_autotune")
    return ch.value


def coll_plan_set_variant(plan: int, variant: int):
    _check(_lib.coll_plan_set_variant(ctypes.c_void_p(plan), int(variant)), "coll_plan_set_variant")


def coll_advance(f, Q, dt: float, stream=None, check=True) -> int:
    """f += dt * Q on the device (same dtype, same number of elements)."""
    import torch
    io = 0 if f.dtype == torch.float64 else 1
    st = _lib.coll_advance(_ptr(f), _ptr(Q), f.numel(), float(dt), io, _stream_ptr(stream))
    if check:
        _check(st, "coll_advance")
    return st


def coll_ragged_workspace_size(groups, cells) -> int:
    arr, cnt = _groups(groups, cells)
    b = ctypes.c_size_t()
    _check(_lib.coll_ragged_workspace_size(arr, cnt, len(groups), ctypes.byref(b)), "coll_ragged_workspace_size")
    return b.value


def _groups(groups, cells):
    arr = (coll_cell_group * len(groups))()
    for i, (plan, f, Q) in enumerate(groups):
        arr[i] = coll_cell_group(ctypes.c_void_p(plan), ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(Q.data_ptr()))
    cnt = (ctypes.c_int64 * len(groups))(*[int(c) for c in cells])
    return arr, cnt


def coll_eval_ragged(groups, cells, ws, stream=None, check=True) -> int:
    """groups: list of (plan, f_tensor, Q_tensor); cells: cells per group."""
    arr, cnt = _groups(groups, cells)
    st = _lib.coll_eval_ragged(arr, cnt, len(groups), _ptr(ws), ws.numel() * ws.element_size() if ws is not None else 0,
                               _stream_ptr(stream))
    if check:
        _check(st, "coll_eval_ragged")
    return st


def moments_realizability(f, io_dtype: int, N: int, L: float, n_cells: int, eta0: float, delta0: float,
                          mom_out, mask_out, stream=None, check=True) -> int:
    st = _lib.moments_realizability(_ptr(f), int(io_dtype), int(N), float(L), int(n_cells), float(eta0),
                                    float(delta0), _ptr(mom_out), _ptr(mask_out), _stream_ptr(stream))
    if check:
        _check(st, "moments_realizability")
    return st


def regime_update(fields, l1, r_in, nx: int, ny: int, params: "coll_regime_params", r_out, ind=None, stream=None,
                  check=True) -> int:
    st = _lib.regime_update(_ptr(fields), _ptr(l1), _ptr(r_in), int(nx), int(ny), ctypes.byref(params), _ptr(r_out),
                            _ptr(ind), _stream_ptr(stream))
    if check:
        _check(st, "regime_update")
    return st


IMEX_FIRST_ORDER, IMEX_PR_Y1, IMEX_PR_Y2, IMEX_PR_FINAL = range(4)


def coll_imex_stage(stage: int, f, Y, Q1, Q2, tr, mom0, mom1, io_dtype: int, N: int, L: float, n_cells: int,
                    dt: float, eps: float, out, stream=None, check=True) -> int:
    st = _lib.coll_imex_stage(int(stage), _ptr(f), _ptr(Y), _ptr(Q1), _ptr(Q2), _ptr(tr), _ptr(mom0), _ptr(mom1),
                              int(io_dtype), int(N), float(L), int(n_cells), float(dt), float(eps), _ptr(out),
                              _stream_ptr(stream))
    if check:
        _check(st, "coll_imex_stage")
    return st


def coll_esbgk_step(f, mom, io_dtype: int, N: int, L: float, n_cells: int, dt: float, eps: float, beta: float,
                    mu0: float, out, stream=None, check=True) -> int:
    st = _lib.coll_esbgk_step(_ptr(f), _ptr(mom), int(io_dtype), int(N), float(L), int(n_cells), float(dt),
                              float(eps), float(beta), float(mu0), _ptr(out), _stream_ptr(stream))
    if check:
        _check(st, "coll_esbgk_step")
    return st


def esbgk_step(f, L: float, dt: float, eps: float, beta: float = -0.5, mu0: float = 1.0, out=None, stream=None):
    """One ES-BGK IMEX step of f [n, N, N, N] on the device (moments, then the relaxation)."""
    import torch
    n, N = f.shape[0], f.shape[-1]
    mom, _ = moments(f, L, stream=stream)
    out = torch.empty_like(f) if out is None else out
    coll_esbgk_step(f, mom, 0 if f.dtype == torch.float64 else 1, N, L, n, dt, eps, beta, mu0, out, stream=stream)
    return out


def pr222_step(plan: "Plan", f, L: float, dt: float, eps: float, out=None, stream=None):
    """One PR(2,2,2) step of df/dt = Q(f)/eps for f [n, N, N, N] on the device:
    moments of f, Y1, Q(Y1), Y2, Q(Y2) through the plan, then the final stage."""
    import torch
    n, N = f.shape[0], f.shape[-1]
    io = 0 if f.dtype == torch.float64 else 1
    mom, _ = moments(f, L, stream=stream)
    Y1 = torch.empty_like(f)
    coll_imex_stage(IMEX_PR_Y1, f, None, None, None, None, mom, None, io, N, L, n, dt, eps, Y1, stream=stream)
    Q1 = plan.eval(Y1, stream=stream)
    Y2 = torch.empty_like(f)
    coll_imex_stage(IMEX_PR_Y2, f, Y1, Q1, None, None, mom, None, io, N, L, n, dt, eps, Y2, stream=stream)
    Q2 = plan.eval(Y2, stream=stream)
    out = torch.empty_like(f) if out is None else out
    coll_imex_stage(IMEX_PR_FINAL, f, None, Q1, Q2, None, None, None, io, N, L, n, dt, eps, out, stream=stream)
    return out


def regime(fields, l1, r, eps, mu0, kappa0, dx, dy, eta0, eta1, delta0, indicators=False, stream=None):
    """r^{n+1} [ny, nx] (uint8) and, if asked, the indicators [4, ny, nx] for
    fields [4, ny + 2, nx + 2] (float64, with halo), l1 [ny, nx], r [ny, nx] on the device."""
    import torch
    ny, nx = r.shape
    out = torch.empty_like(r)
    ind = torch.empty((4, ny, nx), dtype=torch.float64, device=r.device) if indicators else None
    p = coll_regime_params(eps, mu0, kappa0, dx, dy, eta0, eta1, delta0)
    regime_update(fields, l1, r, nx, ny, p, out, ind, stream=stream)
    return (out, ind) if indicators else out


def coll_plan_tables_host(desc: coll_plan_desc):
    """Host-built multiplier tables [n_terms, N, N, N/2, 2] (numpy, no GPU needed)."""
    import numpy as np
    nt, nd = ctypes.c_int32(), ctypes.c_size_t()
    _check(_lib.coll_plan_tables_host(ctypes.byref(desc), None, 0, ctypes.byref(nt), ctypes.byref(nd)),
           "coll_plan_tables_host")
    out = np.empty(nd.value, dtype=np.float64)
    _check(_lib.coll_plan_tables_host(ctypes.byref(desc), out.ctypes.data_as(ctypes.c_void_p), nd.value,
                                      ctypes.byref(nt), ctypes.byref(nd)), "coll_plan_tables_host")
    N = desc.N
    return out.reshape(nt.value, N, N, N // 2, 2)


def coll_device_status(plan: int) -> int:
    return int(_lib.coll_device_status(ctypes.c_void_p(plan)))


def coll_device_status_clear(plan: int):
    _check(_lib.coll_device_status_clear(ctypes.c_void_p(plan)), "coll_device_status_clear")


class Plan:
    """RAII wrapper: a plan, its workspace sized for max_cells, and eval helpers."""

    def __init__(self, N, L, S=0.0, lam=1.0, b0=-1.0, M=48, Mtheta=4, Mr=16, sphere_rule=0, prec="f64",
                 io_dtype=None, max_cells=1, device=None, rank=0, dealias=0):
        import torch
        self.desc = make_desc(N, L, S, lam, b0, M, Mtheta, Mr, sphere_rule, dealias, prec, io_dtype, rank)
        self.N = int(N)
        self.io_dtype = self.desc.io_dtype
        self.torch_dtype = torch.float64 if self.io_dtype == 0 else torch.float32
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.handle = coll_plan_create(self.desc)
        self.n_terms = coll_plan_terms(self.handle)
        self._ws = None
        self.reserve(max_cells)

    def reserve(self, max_cells):
        import torch
        nb = coll_workspace_size(self.handle, max(1, int(max_cells)))
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def eval(self, f, Q=None, stream=None):
        """Q = Q^R(f, f) for f [n, N, N, N] on the device (the plan's io dtype)."""
        import torch
        n = f.shape[0]
        if Q is None:
            Q = torch.empty_like(f)
        ws = self.reserve(n)
        coll_eval_batch(self.handle, f, Q, n, ws, stream=stream)
        return Q

    def eval_host(self, f_host, stream=None):
        """End-to-end: pinned host f -> device -> Q^R -> host (same C-ABI call)."""
        import torch
        fd = f_host.to(self.device, non_blocking=True)
        Q = self.eval(fd, stream=stream)
        return Q.to("cpu")

    def autotune(self, f, stream=None) -> int:
        """Pick the faster slab shape on batch f (device); returns the variant."""
        import torch
        Q = torch.empty_like(f)
        return coll_plan_autotune(self.handle, f, Q, f.shape[0], self.reserve(f.shape[0]), stream=stream)

    def status(self) -> int:
        return coll_device_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            coll_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_m2d_desc(N, L, S=0.0, b0=-1.0, A=16, prec="f64", io_dtype=None) -> coll_m2d_plan_desc:
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    if io_dtype is None:
        io_dtype = 1 if p == COLL_F32 else 0
    return coll_m2d_plan_desc(int(N), float(L), float(S), float(b0), int(A), p, int(io_dtype))


def coll_m2d_plan_create(desc: coll_m2d_plan_desc) -> int:
    h = ctypes.c_void_p()
    _check(_lib.coll_m2d_plan_create(ctypes.byref(desc), ctypes.byref(h)), "coll_m2d_plan_create")
    return h.value


def coll_m2d_plan_destroy(plan: int):
    _check(_lib.coll_m2d_plan_destroy(ctypes.c_void_p(plan)), "coll_m2d_plan_destroy")


def coll_m2d_eval_batch(plan: int, f, Q, n_cells: int, stream=None, check=True) -> int:
    rc = _lib.coll_m2d_eval_batch(ctypes.c_void_p(plan), _ptr(f), _ptr(Q), int(n_cells), _stream_ptr(stream))
    if check:
        _check(rc, "coll_m2d_eval_batch")
    return rc


def coll_m2d_device_status(plan: int) -> int:
    return int(_lib.coll_m2d_device_status(ctypes.c_void_p(plan)))


def coll_m2d_device_status_clear(plan: int):
    _check(_lib.coll_m2d_device_status_clear(ctypes.c_void_p(plan)), "coll_m2d_device_status_clear")


def coll_m2d_tables_host(desc: coll_m2d_plan_desc):
    """Host-built 2D table [A + 1, N, N/2, 2] (numpy, no GPU needed)."""
    import numpy as np
    nt, nd = ctypes.c_int32(), ctypes.c_size_t()
    _check(_lib.coll_m2d_tables_host(ctypes.byref(desc), None, 0, ctypes.byref(nt), ctypes.byref(nd)),
           "coll_m2d_tables_host")
    out = np.empty(nd.value, dtype=np.float64)
    _check(_lib.coll_m2d_tables_host(ctypes.byref(desc), out.ctypes.data_as(ctypes.c_void_p), nd.value,
                                     ctypes.byref(nt), ctypes.byref(nd)), "coll_m2d_tables_host")
    return out.reshape(nt.value, desc.N, desc.N // 2, 2)


class Plan2D:
    """RAII wrapper of a 2D Maxwell-molecule plan (coll_m2d_*)."""

    def __init__(self, N, L, S=0.0, b0=-1.0, A=16, prec="f64", io_dtype=None, device=None):
        import torch
        self.desc = make_m2d_desc(N, L, S, b0, A, prec, io_dtype)
        self.N = int(N)
        self.torch_dtype = torch.float64 if self.desc.io_dtype == 0 else torch.float32
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.handle = coll_m2d_plan_create(self.desc)

    def eval(self, f, Q=None, stream=None):
        """Q for f [n, N, N] on the device (the plan's io dtype)."""
        import torch
        if Q is None:
            Q = torch.empty_like(f)
        coll_m2d_eval_batch(self.handle, f, Q, f.shape[0], stream=stream)
        return Q

    def status(self) -> int:
        return coll_m2d_device_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            coll_m2d_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def moments(f, L, eta0=1e-3, delta0=1e-4, stream=None):
    """Moments records [n, 40] (float64) and mask bytes [n] for f [n, N, N, N] on the device."""
    import torch
    n, N = f.shape[0], f.shape[-1]
    io = 0 if f.dtype == torch.float64 else 1
    mom = torch.empty((n, MOMENT_DOUBLES), dtype=torch.float64, device=f.device)
    mask = torch.empty((n,), dtype=torch.uint8, device=f.device)
    moments_realizability(f, io, N, L, n, eta0, delta0, mom, mask, stream=stream)
    return mom, mask


def coll_conservation(Q, io_dtype: int, N: int, L: float, n_cells: int, out, stream=None, check=True) -> int:
    st = _lib.coll_conservation(_ptr(Q), int(io_dtype), int(N), float(L), int(n_cells), _ptr(out),
                                _stream_ptr(stream))
    if check:
        _check(st, "coll_conservation")
    return st


def conservation(Q, L, stream=None):
    """Collision invariants [n, 8] (m0, m1[3], m2, a0, a1, a2; float64) of Q [n, N, N, N] on the device."""
    import torch
    n, N = Q.shape[0], Q.shape[-1]
    io = 0 if Q.dtype == torch.float64 else 1
    out = torch.empty((n, 8), dtype=torch.float64, device=Q.device)
    coll_conservation(Q, io, N, L, n, out, stream=stream)
    return out


def conservation_errors(inv):
    """[n, 3] relative errors |m0|/a0, max_d |m1_d|/a1, |m2|/a2 of coll_conservation records (torch)."""
    import torch
    return torch.stack([inv[:, 0].abs() / inv[:, 5], inv[:, 1:4].abs().amax(1) / inv[:, 6],
                        inv[:, 4].abs() / inv[:, 7]], 1)
