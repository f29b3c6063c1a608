"""Thin ctypes binding of libibgb.so (include/ib.h): argument marshalling only.

Every step of the immersed-boundary path runs in the library's CUDA kernels;
this module converts Python objects to the C structs and pointers of the ABI
and raises ``IBError`` on any non-OK status.  With ``device=True`` (the
default) fields and marker arrays are torch CUDA tensors whose device
pointers are passed with IB_PTR_DEVICE; with ``device=False`` they are
numpy arrays passed as host pointers.

``load()`` fails loudly when the library has not been built; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build as _build

IB_OK, IB_ERR_ARG, IB_ERR_STATE, IB_ERR_CUDA, IB_ERR_NOMEM, IB_ERR_NONFINITE, IB_ERR_TIMEOUT, IB_ERR_UNSUPPORTED = \
    range(8)
IB_FP64, IB_FP32, IB_FP32_TCFFT = 0, 1, 2
IB_PTR_DEVICE, IB_NO_ADVECTION = 0x1, 0x2
IB_NSTAGES = 10
_STATUS = {0: "IB_OK", 1: "IB_ERR_ARG", 2: "IB_ERR_STATE", 3: "IB_ERR_CUDA", 4: "IB_ERR_NOMEM",
           5: "IB_ERR_NONFINITE", 6: "IB_ERR_TIMEOUT", 7: "IB_ERR_UNSUPPORTED"}


class IBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class ib_grid_desc(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("h", C.c_double), ("rho", C.c_double), ("mu", C.c_double),
                ("dt", C.c_double), ("prec", C.c_int), ("stream", C.c_void_p), ("flags", C.c_uint32)]


class ib_sheet(C.Structure):
    _fields_ = [("first", C.c_int64), ("n1", C.c_int32), ("n2", C.c_int32), ("ds", C.c_double),
                ("dw", C.POINTER(C.c_double)), ("seg_of_row", C.POINTER(C.c_int32))]


class ib_forcing(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("direction", C.c_double * 3), ("radius", C.c_double),
                ("half_len", C.c_double), ("amp", C.c_double), ("omega", C.c_double)]


class ib_structure_desc(C.Structure):
    _fields_ = [("m", C.c_int64), ("X0", C.POINTER(C.c_double)),
                ("n_spring", C.c_int64), ("spring_ij", C.POINTER(C.c_int32)),
                ("spring_k", C.POINTER(C.c_double)), ("spring_L0", C.POINTER(C.c_double)),
                ("n_tether", C.c_int64), ("tether_i", C.POINTER(C.c_int32)), ("tether_k", C.POINTER(C.c_double)),
                ("n_sheet", C.c_int32), ("sheets", C.POINTER(ib_sheet)),
                ("n_seg", C.c_int32), ("bend_b", C.POINTER(C.c_double)),
                ("forcing", ib_forcing),
                ("n_mforce", C.c_int64), ("mforce_i", C.POINTER(C.c_int32)), ("mforce_dir", C.POINTER(C.c_double)),
                ("mforce_amp", C.c_double), ("mforce_omega", C.c_double)]


class ib_tuning(C.Structure):
    _fields_ = [("fft_x", C.c_int32), ("fft_y", C.c_int32), ("fft_z", C.c_int32), ("marker_blocks", C.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def header_functions() -> list[str]:
    """Names of the functions declared in include/ib.h."""
    txt = open(os.path.join(_build.INCLUDE, "ib.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ib_\w+)\s*\(", txt, flags=re.M)


def load(path: str | None = None) -> C.CDLL:
    """Load libibgb.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build() first")
    lib = C.CDLL(path)
    vp, st = C.c_void_p, C.c_int
    pctx = C.c_void_p
    sig = {
        "ib_create": ([C.POINTER(ib_grid_desc), C.POINTER(C.c_void_p)], st),
        "ib_set_structure": ([pctx, C.POINTER(ib_structure_desc)], st),
        "ib_set_state": ([pctx, vp, vp, C.c_double], st),
        "ib_get_state": ([pctx, vp, vp, C.POINTER(C.c_double)], st),
        "ib_step": ([pctx, C.c_int64], st),
        "ib_set_displacement": ([pctx, vp], st),
        "ib_get_displacement": ([pctx, vp], st),
        "ib_spread": ([pctx, vp, vp, vp], st),
        "ib_interp": ([pctx, vp, vp, vp], st),
        "ib_fluid_solve": ([pctx, vp, vp, vp, vp], st),
        "ib_bin_sort": ([pctx, vp, vp, vp], st),
        "ib_get_bin_order": ([pctx, vp, vp, vp], st),
        "ib_get_mean_velocity": ([pctx, vp], st),
        "ib_adjoint_step": ([pctx, vp, vp, vp, vp, vp, vp], st),
        "ib_set_bend_stiffness": ([pctx, vp], st),
        "ib_snapshot_bytes": ([pctx], C.c_int64),
        "ib_set_tuning": ([pctx, C.POINTER(ib_tuning)], st),
        "ib_set_probe": ([pctx, C.c_int32, vp, vp, C.c_int32, C.c_int32], st),
        "ib_read_probe": ([pctx, vp, vp, vp, C.POINTER(C.c_int64)], st),
        "ib_get_tuning": ([pctx, C.POINTER(ib_tuning)], st),
        "ib_autotune": ([pctx, C.c_int32, C.POINTER(ib_tuning)], st),
        "ib_batch_create": ([C.POINTER(C.c_void_p), C.c_int32, C.c_int32, vp, C.POINTER(C.c_void_p)], st),
        "ib_batch_step": ([vp, C.c_int64], st),
        "ib_batch_autotune": ([vp, C.c_int32], st),
        "ib_batch_sync": ([vp], st),
        "ib_batch_destroy": ([vp], st),
        "ib_snapshot_save": ([pctx, vp], st),
        "ib_snapshot_load": ([pctx, vp], st),
        "ib_sync": ([pctx], st),
        "ib_check_bounded_wait": ([pctx, C.c_int32], st),
        "ib_destroy": ([pctx], st),
        "ib_last_error": ([], C.c_char_p),
        "ib_info": ([pctx, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32)], st),
        "ib_stage_name": ([C.c_int32], C.c_char_p),
        "ib_bin_sort_noalloc": ([C.POINTER(C.c_int32), C.c_double, C.c_int64, vp, vp, vp, vp], st),
        "ib_profile": ([pctx, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int64)], st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(status: int):
    if status != IB_OK:
        raise IBError(status, (_lib.ib_last_error() or b"").decode())


def _ptr(a):
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def bin_sort_noalloc(n, h: float, X, key, perm, stream=None):
    """ib_bin_sort_noalloc on caller-owned CUDA tensors X [3][m] float64, key/perm [m] int32.

    The tensors must sit on the current CUDA device; the call is enqueued on
    `stream` (default: torch's current stream)."""
    import torch
    lib = load()
    dev = torch.cuda.current_device()
    if X.dtype != torch.float64 or X.dim() != 2 or X.shape[0] != 3 or not X.is_contiguous():
        raise ValueError("bin_sort_noalloc: X must be a contiguous float64 tensor of shape (3, m)")
    m = int(X.shape[1])
    for name, t in (("key", key), ("perm", perm)):
        if t.dtype != torch.int32 or t.dim() != 1 or t.shape[0] != m or not t.is_contiguous():
            raise ValueError(f"bin_sort_noalloc: {name} must be a contiguous int32 tensor of length {m}")
    for name, t in (("X", X), ("key", key), ("perm", perm)):
        if not t.is_cuda or t.device.index != dev:
            raise ValueError(f"bin_sort_noalloc: {name} must be on the current CUDA device {dev}")
    if stream is None:
        stream = torch.cuda.current_stream()
    nn = (C.c_int32 * 3)(*[int(v) for v in n])
    sp = C.c_void_p(stream.cuda_stream)
    _check(lib.ib_bin_sort_noalloc(nn, float(h), int(X.shape[1]), _ptr(X), _ptr(key), _ptr(perm), sp))


class Context:
    """One IB problem (grid + markers) on the current CUDA device."""

    def __init__(self, grid, prec: str = "fp32", device: bool = True, no_advection: bool = False, stream=None):
        import torch
        self.lib = load()
        self.device = device
        self.fp64 = prec == "fp64"
        self.dtype_np = np.float64 if self.fp64 else np.float32
        self.dtype_t = torch.float64 if self.fp64 else torch.float32
        self.n = tuple(int(v) for v in grid.n)
        self.G = self.n[0] * self.n[1] * self.n[2]
        if stream is None and device:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sp = stream.cuda_stream if stream is not None else None
        flags = (IB_PTR_DEVICE if device else 0) | (IB_NO_ADVECTION if no_advection else 0)
        pc = {"fp64": IB_FP64, "fp32": IB_FP32, "fp32_tcfft": IB_FP32_TCFFT}
        if prec not in pc:
            raise ValueError(f"precision {prec!r} not in {sorted(pc)}")
        d = ib_grid_desc((C.c_int32 * 3)(*self.n), float(grid.h), float(grid.rho), float(grid.mu), float(grid.dt),
                         pc[prec], sp, flags)
        h = C.c_void_p()
        _check(self.lib.ib_create(C.byref(d), C.byref(h)))
        self.h = h
        self.m = 0
        self.n_seg = 0
        self._keep = None

    # -- helpers -------------------------------------------------------------
    # The C ABI takes bare pointers and sizes every array from the context, so
    # each array is checked here for the element count the call will touch.
    @staticmethod
    def _numel(a) -> int:
        return int(a.numel()) if hasattr(a, "numel") else int(np.size(a))

    def _expect(self, a, count: int, what: str):
        if self._numel(a) != count:
            raise ValueError(f"{what}: expected {count} elements, got {self._numel(a)}")

    def _field(self, a, count=None):
        """Coerce a real array (default: a (3, nz, ny, nx) field) to this
        context's real type and location."""
        import torch
        self._expect(a, 3 * self.G if count is None else count, "field")
        if self.device:
            t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.asarray(a))
            return t.to(device="cuda", dtype=self.dtype_t).contiguous()
        return np.ascontiguousarray(np.asarray(a), dtype=self.dtype_np)

    def _pos(self, X, count=None):
        """Coerce an FP64 array (default: marker positions [3][m]) to this context's location."""
        import torch
        self._expect(X, 3 * self.m if count is None else count, "marker array")
        if self.device:
            t = X if isinstance(X, torch.Tensor) else torch.from_numpy(np.asarray(X))
            return t.to(device="cuda", dtype=torch.float64).contiguous()
        return np.ascontiguousarray(np.asarray(X), dtype=np.float64)

    def _out(self, a, count: int, f64: bool, what: str):
        """A caller buffer the library writes: `count` contiguous elements of the
        context's real type (FP64 if f64) in the context's memory."""
        import torch
        if isinstance(a, torch.Tensor):
            want = torch.float64 if f64 else self.dtype_t
            ok = a.dtype == want and a.is_contiguous() and a.is_cuda == bool(self.device)
        else:
            want = np.float64 if f64 else self.dtype_np
            ok = (not self.device and isinstance(a, np.ndarray) and a.dtype == want
                  and a.flags.c_contiguous)
        if not ok:
            raise ValueError(f"{what}: expected a contiguous {want} buffer in "
                             f"{'device' if self.device else 'host'} memory")
        self._expect(a, count, what)
        return a

    def _empty(self, shape, dtype=None):
        import torch
        if self.device:
            return torch.empty(shape, device="cuda", dtype=dtype or self.dtype_t)
        return np.empty(shape, dtype=dtype or self.dtype_np)

    # -- ABI calls -------------------------------------------------------------
    def set_structure(self, st, bend_b=None):
        X0 = np.ascontiguousarray(st.X0, dtype=np.float64)
        m = X0.shape[1]
        sij = np.ascontiguousarray(st.spring_ij, dtype=np.int32).reshape(-1, 2)
        sk = np.ascontiguousarray(st.spring_k, dtype=np.float64)
        sL0 = np.ascontiguousarray(st.spring_L0, dtype=np.float64)
        ti = np.ascontiguousarray(st.tether_i, dtype=np.int32)
        tk = np.ascontiguousarray(st.tether_k, dtype=np.float64)
        bb = np.ascontiguousarray(st.bend_b if bend_b is None else bend_b, dtype=np.float64)
        keep = [X0, sij, sk, sL0, ti, tk, bb]
        sheets = (ib_sheet * max(1, len(st.sheets)))()
        for q, sh in enumerate(st.sheets):
            dw = np.ascontiguousarray(sh.dw, dtype=np.float64)
            seg = np.ascontiguousarray(sh.seg_of_row, dtype=np.int32)
            keep += [dw, seg]
            sheets[q] = ib_sheet(int(sh.first), int(sh.n1), int(sh.n2), float(sh.ds),
                                 dw.ctypes.data_as(C.POINTER(C.c_double)),
                                 seg.ctypes.data_as(C.POINTER(C.c_int32)))
        fo = st.forcing
        forcing = ib_forcing((C.c_double * 3)(*fo.center), (C.c_double * 3)(*fo.direction), float(fo.radius),
                             float(fo.half_len), float(fo.amp), float(fo.omega))
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
        mf = getattr(st, "marker_forcing", None)
        if mf is not None:
            mfi = np.ascontiguousarray(mf.index, dtype=np.int32)
            mfd = np.ascontiguousarray(mf.direction, dtype=np.float64)
            keep += [mfi, mfd]
            mfargs = (len(mfi), ip(mfi), dp(mfd), float(mf.amp), float(mf.omega))
        else:
            mfargs = (0, None, None, 0.0, 0.0)
        desc = ib_structure_desc(m, dp(X0), len(sk), ip(sij), dp(sk), dp(sL0), len(tk), ip(ti), dp(tk),
                                 len(st.sheets), sheets, len(bb), dp(bb), forcing, *mfargs)
        _check(self.lib.ib_set_structure(self.h, C.byref(desc)))
        self.m = m
        self.n_seg = len(bb)

    def set_state(self, u=None, X=None, t: float = 0.0):
        uu = self._field(u) if u is not None else None
        XX = self._pos(X) if X is not None else None
        _check(self.lib.ib_set_state(self.h, _ptr(uu), _ptr(XX), float(t)))

    def get_state(self):
        import torch
        u = self._empty((3,) + self.n[::-1])
        X = torch.empty((3, self.m), device="cuda", dtype=torch.float64) if self.device else \
            np.empty((3, self.m), dtype=np.float64)
        t = C.c_double()
        _check(self.lib.ib_get_state(self.h, _ptr(u), _ptr(X), C.byref(t)))
        return u, X, t.value

    def set_displacement(self, D):
        DD = self._pos(D)
        _check(self.lib.ib_set_displacement(self.h, _ptr(DD)))

    def get_displacement(self):
        import torch
        D = torch.empty((3, self.m), device="cuda", dtype=torch.float64) if self.device else \
            np.empty((3, self.m), dtype=np.float64)
        _check(self.lib.ib_get_displacement(self.h, _ptr(D)))
        return D

    def step(self, nsteps: int = 1):
        _check(self.lib.ib_step(self.h, int(nsteps)))

    def spread(self, X, f):
        XX, ff = self._pos(X), self._field(f, 3 * self.m)
        F = self._empty((3,) + self.n[::-1])
        _check(self.lib.ib_spread(self.h, _ptr(XX), _ptr(ff), _ptr(F)))
        return F

    def interp(self, X, u):
        XX, uu = self._pos(X), self._field(u)
        U = self._empty((3, self.m))
        _check(self.lib.ib_interp(self.h, _ptr(XX), _ptr(uu), _ptr(U)))
        return U

    def fluid_solve(self, u, F, want_p: bool = False):
        uu, FF = self._field(u), self._field(F)
        un = self._empty((3,) + self.n[::-1])
        p = self._empty(self.n[::-1]) if want_p else None
        _check(self.lib.ib_fluid_solve(self.h, _ptr(uu), _ptr(FF), _ptr(un), _ptr(p)))
        return (un, p) if want_p else un

    def bin_sort(self, X):
        import torch
        XX = self._pos(X)
        if self.device:
            key = torch.empty(self.m, device="cuda", dtype=torch.int32)
            perm = torch.empty(self.m, device="cuda", dtype=torch.int32)
        else:
            key = np.empty(self.m, np.int32)
            perm = np.empty(self.m, np.int32)
        _check(self.lib.ib_bin_sort(self.h, _ptr(XX), _ptr(key), _ptr(perm)))
        return key, perm

    def get_mean_velocity(self):
        """The state's mean velocity, FP64 (ib_get_mean_velocity)."""
        out = np.zeros(3)
        _check(self.lib.ib_get_mean_velocity(self.h, _ptr(out)))
        return out

    def get_bin_order(self):
        """(key, perm, internal) of the last step's bin sort, caller numbering (ib_get_bin_order)."""
        import torch
        if self.device:
            out = [torch.empty(self.m, device="cuda", dtype=torch.int32) for _ in range(3)]
        else:
            out = [np.empty(self.m, np.int32) for _ in range(3)]
        _check(self.lib.ib_get_bin_order(self.h, *[_ptr(o) for o in out]))
        return tuple(out)

    def set_bend_stiffness(self, bend_b):
        """Replace the per-segment bending stiffness (float64 [n_seg])."""
        b = self._pos(bend_b, self.n_seg)
        _check(self.lib.ib_set_bend_stiffness(self.h, _ptr(b)))

    def adjoint_step(self, lam_u, lam_D, u_np1=None, grad_b=None, out=None):
        """Reverse of one step about the current state: (lam_u^n, lam_D^n).

        lam_u: dJ/du^{n+1} field, lam_D: dJ/dD^{n+1} [3][m] float64; grad_b
        (float64 [n_seg], same location as the context's arrays) is
        accumulated in place.  out: optional (lam_u_out, lam_D_out) buffers,
        which may be lam_u and lam_D themselves."""
        lu = self._field(lam_u)
        lD = self._pos(lam_D)
        u1 = self._field(u_np1) if u_np1 is not None else None
        if out is None:
            luo = self._empty((3,) + self.n[::-1])
            lDo = self._empty((3, self.m), dtype=self._f64())
        else:
            luo = self._out(out[0], 3 * self.G, False, "lam_u_out")
            lDo = self._out(out[1], 3 * self.m, True, "lam_D_out")
        if grad_b is not None:
            self._out(grad_b, self.n_seg, True, "grad_b")
        _check(self.lib.ib_adjoint_step(self.h, _ptr(u1), _ptr(lu), _ptr(lD), _ptr(luo), _ptr(lDo), _ptr(grad_b)))
        return luo, lDo

    def set_probe(self, markers, direction, every: int = 10, capacity: int = 1024):
        """Record eta_i = D_i . direction_i of `markers` every `every` steps."""
        mk = np.ascontiguousarray(markers, dtype=np.int32)
        dr = np.ascontiguousarray(direction, dtype=np.float64).reshape(3, len(mk))
        self._probe = (len(mk), int(capacity))
        _check(self.lib.ib_set_probe(self.h, len(mk), mk.ctypes.data_as(C.c_void_p), dr.ctypes.data_as(C.c_void_p),
                                     int(every), int(capacity)))

    def read_probe(self):
        """(eta [k][n], times [k], envelope [n], produced) for the newest k records."""
        n, cap = self._probe
        eta = np.zeros((cap, n))
        times = np.zeros(cap)
        env = np.zeros(n)
        cnt = C.c_int64()
        _check(self.lib.ib_read_probe(self.h, eta.ctypes.data_as(C.c_void_p), times.ctypes.data_as(C.c_void_p),
                                      env.ctypes.data_as(C.c_void_p), C.byref(cnt)))
        k = min(cnt.value, cap)
        return eta[:k], times[:k], env, cnt.value

    def set_tuning(self, fft_x=0, fft_y=0, fft_z=0, marker_blocks=0):
        t = ib_tuning(int(fft_x), int(fft_y), int(fft_z), int(marker_blocks))
        _check(self.lib.ib_set_tuning(self.h, C.byref(t)))

    def get_tuning(self) -> dict:
        t = ib_tuning()
        _check(self.lib.ib_get_tuning(self.h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in ib_tuning._fields_}

    def autotune(self, reps: int = 10) -> dict:
        t = ib_tuning()
        _check(self.lib.ib_autotune(self.h, int(reps), C.byref(t)))
        return {f: getattr(t, f) for f, _ in ib_tuning._fields_}

    def snapshot_bytes(self) -> int:
        return int(self.lib.ib_snapshot_bytes(self.h))

    def new_snapshot(self):
        """A device buffer (uint8 tensor) for one state snapshot."""
        import torch
        return torch.empty(self.snapshot_bytes(), dtype=torch.uint8, device="cuda")

    def snapshot_save(self, buf):
        _check(self.lib.ib_snapshot_save(self.h, _ptr(buf)))

    def snapshot_load(self, buf):
        _check(self.lib.ib_snapshot_load(self.h, _ptr(buf)))

    def snapshot_velocity(self, buf):
        """The velocity field stored at the start of a snapshot buffer (a view)."""
        n = 3 * self.G
        return buf[: n * (8 if self.fp64 else 4)].view(self.dtype_t).view((3,) + self.n[::-1])

    def _f64(self):
        import torch
        return torch.float64 if self.device else np.float64

    def profile(self, nsteps: int):
        """Mean device ms per stage over nsteps eager steps, and the active tile count."""
        ms = (C.c_double * IB_NSTAGES)()
        tiles = C.c_int64()
        _check(self.lib.ib_profile(self.h, int(nsteps), ms, C.byref(tiles)))
        return {self.lib.ib_stage_name(i).decode(): ms[i] for i in range(IB_NSTAGES)}, tiles.value

    def sync(self):
        _check(self.lib.ib_sync(self.h))

    def check_bounded_wait(self, polls: int):
        """Enqueue the bounded-wait self-check; the next sync raises IB_ERR_TIMEOUT."""
        _check(self.lib.ib_check_bounded_wait(self.h, int(polls)))

    def close(self):
        if self.h:
            self.lib.ib_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many contexts stepped together by one CUDA graph (ib_batch_*)."""

    def __init__(self, contexts, steps_per_launch: int = 1, stream=None):
        import torch
        self.lib = load()
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.steps_per_launch = int(steps_per_launch)
        h = C.c_void_p()
        _check(self.lib.ib_batch_create(arr, len(self.contexts), self.steps_per_launch,
                                        C.c_void_p(stream.cuda_stream), C.byref(h)))
        self.h = h

    def step(self, nsteps: int):
        _check(self.lib.ib_batch_step(self.h, int(nsteps)))

    def autotune(self, reps: int = 3):
        _check(self.lib.ib_batch_autotune(self.h, int(reps)))

    def sync(self):
        _check(self.lib.ib_batch_sync(self.h))

    def close(self):
        if self.h:
            self.lib.ib_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
