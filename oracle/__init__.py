"""FP64 CPU oracle of the immersed-boundary time step (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``ib_oracle.c`` (plain C,
compiled with ``-ffp-contract=off``) through ctypes and shares no code with
the CUDA library or its Python binding; the two meet only in the seeded input
generator ``paper_math_0301321_gb300.synth``, which holds no arithmetic of the
method.

Each wrapper names the passage of the paper (Section 3.2) that its C function
follows; see ``ib_oracle.c`` for the transcription itself.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ib_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile ib_oracle.c into liboracle.so (plain gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-D_DEFAULT_SOURCE",
                        "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Sheet(C.Structure):
    _fields_ = [("first", C.c_int64), ("n1", C.c_int32), ("n2", C.c_int32), ("ds", C.c_double),
                ("dw", C.POINTER(C.c_double)), ("seg_of_row", C.POINTER(C.c_int32))]


class _Forcing(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("direction", C.c_double * 3), ("radius", C.c_double),
                ("half_len", C.c_double), ("amp", C.c_double), ("omega", C.c_double)]


class _Structure(C.Structure):
    _fields_ = [("m", C.c_int64), ("X0", C.POINTER(C.c_double)),
                ("n_spring", C.c_int64), ("spring_ij", C.POINTER(C.c_int32)),
                ("spring_k", C.POINTER(C.c_double)), ("spring_L0", C.POINTER(C.c_double)),
                ("n_tether", C.c_int64), ("tether_i", C.POINTER(C.c_int32)), ("tether_k", C.POINTER(C.c_double)),
                ("n_sheet", C.c_int32), ("sheets", C.POINTER(_Sheet)),
                ("n_seg", C.c_int32), ("bend_b", C.POINTER(C.c_double)),
                ("forcing", _Forcing),
                ("n_mforce", C.c_int64), ("mforce_i", C.POINTER(C.c_int32)),
                ("mforce_dir", C.POINTER(C.c_double)), ("mforce_amp", C.c_double), ("mforce_omega", C.c_double)]


class _Grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("h", C.c_double), ("rho", C.c_double), ("mu", C.c_double),
                ("dt", C.c_double), ("no_advection", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i64 = C.POINTER(C.c_double), C.c_int64
        g, s = C.POINTER(_Grid), C.POINTER(_Structure)
        _lib.or_phi.restype = C.c_double
        _lib.or_phi.argtypes = [C.c_double]
        _lib.or_spread.argtypes = [g, i64, d, d, d]
        _lib.or_interp.argtypes = [g, i64, d, d, d]
        _lib.or_bin_sort.argtypes = [g, i64, d, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        _lib.or_forces.argtypes = [s, d, d]
        _lib.or_energy.restype = C.c_double
        _lib.or_energy.argtypes = [s, d]
        _lib.or_body_force.argtypes = [g, C.POINTER(_Forcing), C.c_double, C.c_double, d]
        _lib.or_advection.argtypes = [g, d, d]
        _lib.or_rhs.argtypes = [g, d, d, d]
        _lib.or_dft3.argtypes = [g, d, d, C.c_int]
        _lib.or_dft1.argtypes = [C.c_int, d, d, C.c_int]
        _lib.or_solve.argtypes = [g, d, d, d]
        _lib.or_fluid_solve.argtypes = [g, d, d, d, d]
        _lib.or_step.argtypes = [g, s, d, d, d, i64]
        _lib.or_marker_forcing.argtypes = [s, C.c_double, d]
        _lib.or_phi_d.restype = C.c_double
        _lib.or_phi_d.argtypes = [C.c_double]
        _lib.or_interp_grad.argtypes = [g, i64, d, d, d, C.c_double, d]
        _lib.or_advection_adjoint.argtypes = [g, d, d, d]
        _lib.or_forces_lin.argtypes = [s, d, d, d]
        _lib.or_forces_dbend.argtypes = [s, d, d, d]
        _lib.or_adjoint_step.argtypes = [g, s, d, d, C.c_double, d, d, d, d, d]
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


def grid(g, no_advection: bool = False) -> _Grid:
    """ctypes grid from a synth.Grid (or anything with n, h, rho, mu, dt)."""
    return _Grid((C.c_int32 * 3)(*[int(v) for v in g.n]), float(g.h), float(g.rho), float(g.mu),
                 float(g.dt), int(bool(no_advection)))


class Structure:
    """Owns the numpy arrays behind a ctypes or_structure."""

    def __init__(self, st, bend_b=None):
        self.X0 = _f64(st.X0)
        self.m = self.X0.shape[1]
        self.sij = np.ascontiguousarray(st.spring_ij, dtype=np.int32).reshape(-1, 2)
        self.sk = _f64(st.spring_k)
        self.sL0 = _f64(st.spring_L0)
        self.ti = np.ascontiguousarray(st.tether_i, dtype=np.int32)
        self.tk = _f64(st.tether_k)
        self.bend_b = _f64(st.bend_b if bend_b is None else bend_b)
        self._keep = []
        sheets = (_Sheet * max(1, len(st.sheets)))()
        for q, sh in enumerate(st.sheets):
            dw = _f64(sh.dw)
            seg = np.ascontiguousarray(sh.seg_of_row, dtype=np.int32)
            self._keep += [dw, seg]
            sheets[q] = _Sheet(int(sh.first), int(sh.n1), int(sh.n2), float(sh.ds), _p(dw), _p(seg, C.c_int32))
        self._sheets = sheets
        fo = st.forcing
        self.forcing = _Forcing((C.c_double * 3)(*fo.center), (C.c_double * 3)(*fo.direction), float(fo.radius),
                                float(fo.half_len), float(fo.amp), float(fo.omega))
        mf = getattr(st, "marker_forcing", None)
        if mf is not None:
            self.mfi = np.ascontiguousarray(mf.index, dtype=np.int32)
            self.mfd = _f64(mf.direction)
            mf_n, mf_amp, mf_om = len(self.mfi), float(mf.amp), float(mf.omega)
        else:
            self.mfi = np.zeros(1, np.int32)
            self.mfd = np.zeros((3, 1))
            mf_n, mf_amp, mf_om = 0, 0.0, 0.0
        self.c = _Structure(self.m, _p(self.X0), len(self.sk), _p(self.sij, C.c_int32), _p(self.sk), _p(self.sL0),
                            len(self.tk), _p(self.ti, C.c_int32), _p(self.tk), len(st.sheets), sheets,
                            len(self.bend_b), _p(self.bend_b), self.forcing,
                            mf_n, _p(self.mfi, C.c_int32), _p(self.mfd), mf_amp, mf_om)


# ----------------------------------------------------------------------------
# numpy-level wrappers
# ----------------------------------------------------------------------------
def phi(r) -> np.ndarray:
    """The 4-point kernel phi of delta_h (Section 3.2)."""
    r = np.asarray(r, dtype=np.float64)
    return np.vectorize(lambda x: lib().or_phi(float(x)), otypes=[np.float64])(r)


def _shape(g):
    nx, ny, nz = (int(v) for v in g.n)
    return (3, nz, ny, nx)


def spread(g, X, f) -> np.ndarray:
    """Eq. (discreteF): F = sum_l f_l delta_h(x - X_l)  -> (3, nz, ny, nx)."""
    X, f = _f64(X), _f64(f)
    F = np.zeros(_shape(g))
    lib().or_spread(C.byref(grid(g)), X.shape[1], _p(X), _p(f), _p(F))
    return F


def interp(g, X, u) -> np.ndarray:
    """Eq. (discreteX): U_l = sum_x u(x) delta_h(x - X_l) h^3  -> (3, m)."""
    X, u = _f64(X), _f64(u)
    U = np.zeros((3, X.shape[1]))
    lib().or_interp(C.byref(grid(g)), X.shape[1], _p(X), _p(u), _p(U))
    return U


def bin_sort(g, X):
    """Cell key of floor(X/h) (wrapped) per marker and the stable key order."""
    X = _f64(X)
    m = X.shape[1]
    key = np.zeros(m, np.int32)
    perm = np.zeros(m, np.int32)
    lib().or_bin_sort(C.byref(grid(g)), m, _p(X), _p(key, C.c_int32), _p(perm, C.c_int32))
    return key, perm


def forces(st: Structure, D) -> np.ndarray:
    """Marker forces at positions X0 + D (D: displacement from the reference X0)."""
    D = _f64(D)
    f = np.zeros_like(D)
    lib().or_forces(C.byref(st.c), _p(D), _p(f))
    return f


def marker_forcing(st: Structure, t: float) -> np.ndarray:
    """The external marker force at time t alone (Section 4, oval window load)."""
    f = np.zeros((3, st.m))
    lib().or_marker_forcing(C.byref(st.c), float(t), _p(f))
    return f


def energy(st: Structure, D) -> float:
    """Elastic energy at positions X0 + D."""
    D = _f64(D)
    return lib().or_energy(C.byref(st.c), _p(D))


def body_force(g, st: Structure, t: float) -> np.ndarray:
    F = np.zeros(_shape(g))
    lib().or_body_force(C.byref(grid(g)), C.byref(st.forcing), float(g.rho), float(t), _p(F))
    return F


def advection(g, u) -> np.ndarray:
    u = _f64(u)
    A = np.zeros_like(u)
    lib().or_advection(C.byref(grid(g)), _p(u), _p(A))
    return A


def rhs(g, u, F, no_advection: bool = False) -> np.ndarray:
    u, F = _f64(u), _f64(F)
    w = np.zeros_like(u)
    lib().or_rhs(C.byref(grid(g, no_advection)), _p(u), _p(F), _p(w))
    return w


def dft3(g, a, sign: int = -1) -> np.ndarray:
    """Unscaled complex 3-D DFT of a (nz, ny, nx) array, sign -1 forward."""
    a = np.asarray(a, dtype=np.complex128)
    re, im = _f64(a.real), _f64(a.imag)
    lib().or_dft3(C.byref(grid(g)), _p(re), _p(im), int(sign))
    return re + 1j * im


def dft1(a, sign: int = -1) -> np.ndarray:
    a = np.asarray(a, dtype=np.complex128)
    re, im = _f64(a.real), _f64(a.imag)
    lib().or_dft1(len(a), _p(re), _p(im), int(sign))
    return re + 1j * im


def solve(g, w, want_p: bool = False):
    """Eqs. (discreteNS1)-(discreteNS2) given the known terms w."""
    w = _f64(w)
    un = np.zeros_like(w)
    p = np.zeros(w.shape[1:]) if want_p else None
    lib().or_solve(C.byref(grid(g)), _p(w), _p(un), _p(p) if want_p else None)
    return (un, p) if want_p else un


def fluid_solve(g, u, F, want_p: bool = False, no_advection: bool = False):
    """Step 3: u^{n+1} (and p^{n+1}) from u^n and F^n."""
    u, F = _f64(u), _f64(F)
    un = np.zeros_like(u)
    p = np.zeros(u.shape[1:]) if want_p else None
    lib().or_fluid_solve(C.byref(grid(g, no_advection)), _p(u), _p(F), _p(un), _p(p) if want_p else None)
    return (un, p) if want_p else un


def step(g, st: Structure, D, u, t: float = 0.0, nsteps: int = 1, no_advection: bool = False):
    """Steps 1-4 of the time step, nsteps times, on positions X0 + D.

    Returns (D, u, t) with D the new displacement from the reference X0."""
    D = _f64(D).copy()
    u = _f64(u).copy()
    tt = C.c_double(float(t))
    lib().or_step(C.byref(grid(g, no_advection)), C.byref(st.c), _p(D), _p(u), C.byref(tt), int(nsteps))
    return D, u, tt.value


# ----------------------------------------------------------------------------
# adjoint (reverse of one time step; see or_adjoint_step)
# ----------------------------------------------------------------------------
def phi_d(r) -> np.ndarray:
    """phi'(r), the derivative of the kernel of delta_h (Section 3.2)."""
    L = lib()
    r = np.asarray(r, dtype=np.float64)
    return np.vectorize(lambda x: L.or_phi_d(float(x)), otypes=[np.float64])(r)


def interp_grad(g, X, u, v, scale: float = 1.0) -> np.ndarray:
    """scale * sum_c v_c(l) d/dX_l [interp of u_c at X_l]  -> (3, m)."""
    X, u, v = _f64(X), _f64(u), _f64(v)
    out = np.zeros_like(X)
    lib().or_interp_grad(C.byref(grid(g)), X.shape[1], _p(X), _p(u), _p(v), float(scale), _p(out))
    return out


def advection_adjoint(g, u, lam) -> np.ndarray:
    """(dA/du)^T lam for the upwind term of Eq. (discreteNS1)."""
    u, lam = _f64(u), _f64(lam)
    out = np.zeros(_shape(g))
    lib().or_advection_adjoint(C.byref(grid(g)), _p(u), _p(lam), _p(out))
    return out


def forces_lin(st: Structure, D, lam) -> np.ndarray:
    """(df/dD) lam at displacement D (the negative elastic Hessian times lam)."""
    D, lam = _f64(D), _f64(lam)
    out = np.zeros((3, st.m))
    lib().or_forces_lin(C.byref(st.c), _p(D), _p(lam), _p(out))
    return out


def forces_dbend(st: Structure, D, lam) -> np.ndarray:
    """(df/db)^T lam: per-segment derivative of lam . f in the bending stiffness."""
    D, lam = _f64(D), _f64(lam)
    out = np.zeros(len(st.bend_b))
    lib().or_forces_dbend(C.byref(st.c), _p(D), _p(lam), _p(out))
    return out


def adjoint_step(g, st: Structure, D, u, t, lam_u, lam_D, no_advection: bool = False):
    """Reverse of one time step about (u^n, D^n, t^n): returns
    (lam_u^n, lam_D^n, grad_b) from lam_u^{n+1}, lam_D^{n+1}."""
    D, u, lam_u, lam_D = _f64(D), _f64(u), _f64(lam_u), _f64(lam_D)
    lu0 = np.zeros_like(u)
    lD0 = np.zeros_like(D)
    gb = np.zeros(len(st.bend_b))
    lib().or_adjoint_step(C.byref(grid(g, no_advection)), C.byref(st.c), _p(D), _p(u), float(t),
                                   _p(lam_u), _p(lam_D), _p(lu0), _p(lD0), _p(gb))
    return lu0, lD0, gb
