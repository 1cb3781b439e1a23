"""ctypes wrapper around the plain-C FP64 oracle, plus the paper's closed forms.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Closed forms restated from the paper:
  * lambda* of Eq. Lambda-Star with the integrals printed in Tab. 3
    (I = 2/3, K = (31 - 30 ln 2)/150, F = ln 2 / 4);
  * the one-sided Stefan root of Eq. Cartesian_Transcendental (Sec. 4.2);
  * the two-sided (Maugis) root of Eq. Transcendental_Eq with u_Phi of
    Eq. solution_u (Sec. 4.1).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbpf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblbpf_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over rows)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-std=c99",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.or_init.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp, dp]
        _lib.or_step.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, ctypes.c_int]
        _lib.or_gradient.argtypes = [ctypes.c_void_p, dp, dp]
        _lib.or_mu.argtypes = [ctypes.c_void_p, dp, dp, dp]
        _lib.or_lattice.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp,
                                    ctypes.POINTER(ctypes.c_int)]
        _lib.or_set_threads.argtypes = [ctypes.c_int]
        _lib.or_get_threads.restype = ctypes.c_int
    return _lib


class _CParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("bc", ctypes.c_int * 3),
                ("tau_g", ctypes.c_double), ("tau_h", ctypes.c_double),
                ("W", ctypes.c_double), ("lam", ctypes.c_double),
                ("D_l", ctypes.c_double), ("D_s", ctypes.c_double),
                ("c_s_co", ctypes.c_double), ("c_l_co", ctypes.c_double),
                ("mu_eq", ctypes.c_double), ("counter_term", ctypes.c_int),
                ("anti_trapping", ctypes.c_int), ("a_at", ctypes.c_double),
                ("eps_n", ctypes.c_double)]


@dataclass
class OracleParams:
    """Model parameters in lattice units (dx = dt = 1).

    M_phi = tau_g / 3 (Sec. 3.2) and gamma = 3 / tau_h (Sec. 3.3)."""
    nx: int
    ny: int
    nz: int = 1
    bc: tuple = (0, 0, 0)
    tau_g: float = 0.5
    tau_h: float = 0.5
    W: float = 3.0
    lam: float = 0.0
    D_l: float = 0.1
    D_s: float = 0.1
    c_s_co: float = 1.0
    c_l_co: float = 0.5
    mu_eq: float = 0.4
    counter_term: int = 1
    anti_trapping: int = 0
    a_at: float = 0.25
    eps_n: float = 1e-12

    @property
    def dim(self) -> int:
        return 3 if self.nz > 1 else 2

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def _c(self) -> _CParams:
        c = _CParams()
        c.dim, c.nx, c.ny, c.nz = self.dim, self.nx, self.ny, self.nz
        for a in range(3):
            c.bc[a] = int(self.bc[a])
        c.tau_g, c.tau_h, c.W, c.lam = self.tau_g, self.tau_h, self.W, self.lam
        c.D_l, c.D_s = self.D_l, self.D_s
        c.c_s_co, c.c_l_co, c.mu_eq = self.c_s_co, self.c_l_co, self.mu_eq
        c.counter_term, c.anti_trapping = int(self.counter_term), int(self.anti_trapping)
        c.a_at, c.eps_n = self.a_at, self.eps_n
        return c


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lattice_tables(dim: int):
    """(e [q,3] int, w [q], opp [q]) of the oracle's lattice."""
    lib = _load()
    e = (ctypes.c_int * 57)()
    w = np.zeros(19)
    opp = (ctypes.c_int * 19)()
    q = lib.or_lattice(dim, e, _dp(w), opp)
    return (np.array(e[:3 * q], dtype=np.int64).reshape(q, 3), w[:q].copy(),
            np.array(opp[:q], dtype=np.int64))


def gradient(p: OracleParams, phi: np.ndarray) -> np.ndarray:
    """Directional-derivative gradient of phi, shape (nz, ny, nx, 3)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(p.shape)
    out = np.zeros(p.shape + (3,))
    cp = p._c()
    _load().or_gradient(ctypes.byref(cp), _dp(phi), _dp(out))
    return out


class Oracle:
    """State of one oracle simulation: populations g, h [q, nz, ny, nx] and
    the fields phi, c [nz, ny, nx], all FP64."""

    def __init__(self, p: OracleParams, phi0: np.ndarray, c0: np.ndarray):
        self.p = p
        self._cp = p._c()
        q = 19 if p.dim == 3 else 9
        self.q = q
        shp = p.shape
        self.phi = np.zeros(shp)
        self.c = np.zeros(shp)
        self.g = np.zeros((q,) + shp)
        self.h = np.zeros((q,) + shp)
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(shp)
        c0 = np.ascontiguousarray(c0, dtype=np.float64).reshape(shp)
        rc = _load().or_init(ctypes.byref(self._cp), _dp(phi0), _dp(c0), _dp(self.g),
                             _dp(self.h), _dp(self.phi), _dp(self.c))
        if rc != 0:
            raise MemoryError("oracle init failed")
        self.t = 0

    @classmethod
    def from_state(cls, p: OracleParams, g: np.ndarray, h: np.ndarray, phi: np.ndarray,
                   c: np.ndarray) -> "Oracle":
        """An oracle whose state is given directly: populations g, h [q, nz, ny, nx]
        (after streaming, before the next collision) and the fields phi, c."""
        o = cls.__new__(cls)
        o.p = p
        o._cp = p._c()
        o.q = 19 if p.dim == 3 else 9
        o.g = np.ascontiguousarray(g, dtype=np.float64).reshape((o.q,) + p.shape).copy()
        o.h = np.ascontiguousarray(h, dtype=np.float64).reshape((o.q,) + p.shape).copy()
        o.phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(p.shape).copy()
        o.c = np.ascontiguousarray(c, dtype=np.float64).reshape(p.shape).copy()
        o.t = 0
        return o

    def step(self, n: int = 1) -> "Oracle":
        rc = _load().or_step(ctypes.byref(self._cp), _dp(self.g), _dp(self.h),
                             _dp(self.phi), _dp(self.c), int(n))
        if rc != 0:
            raise MemoryError("oracle step failed")
        self.t += n
        return self

    @property
    def mu(self) -> np.ndarray:
        out = np.zeros(self.p.shape)
        _load().or_mu(ctypes.byref(self._cp), _dp(self.phi), _dp(self.c), _dp(out))
        return out

    @staticmethod
    def set_threads(n: int) -> None:
        _load().or_set_threads(int(n))

    @staticmethod
    def threads() -> int:
        return _load().or_get_threads()


# ---- closed forms printed in, or defined by, the paper ---------------------

TAB3_I = 2.0 / 3.0
TAB3_K_PRINTED = (31.0 - 30.0 * math.log(2.0)) / 150.0
TAB3_F = math.log(2.0) / 4.0


def lambda_star_printed(D_l: float, M_phi: float, dc: float) -> float:
    """lambda* of Eq. Lambda-Star, with the integrals printed in Tab. 3."""
    return D_l / (M_phi * dc * dc) * TAB3_I / (TAB3_K_PRINTED + TAB3_F)


def _brent(f, a, b, tol=1e-15):
    from scipy.optimize import brentq
    return brentq(f, a, b, xtol=tol, rtol=4 * np.finfo(float).eps, maxiter=500)


def stefan_one_sided_root(mu_eq: float, mu_inf: float, dc: float) -> float:
    """Root alpha of alpha e^{alpha^2} erfc(alpha) + (mu_eq - mu_inf)/(dc sqrt(pi)) = 0
    (Eq. Cartesian_Transcendental).  The interface is at x_i = 2 alpha sqrt(D_l t)."""
    from scipy.special import erfcx
    rhs = (mu_eq - mu_inf) / (dc * math.sqrt(math.pi))
    return _brent(lambda a: a * erfcx(a) + rhs, -5.0, 5.0)


def stefan_two_sided_root(D_s, D_l, m_s, m_l, df_min, cs_inf, cl_inf) -> float:
    """Root alpha of Eq. Transcendental_Eq with u_Phi of Eq. solution_u; the
    interface is at x_i = alpha sqrt(t)."""
    from scipy.special import erfcx
    dm = m_s - m_l

    def u(D, a):  # sqrt(D/pi) e^{-a^2/4D} / erfc(a / 2 sqrt D) = sqrt(D/pi)/erfcx(a/2sqrtD)
        return math.sqrt(D / math.pi) / erfcx(a / (2.0 * math.sqrt(D)))

    def f(a):
        us, ul = u(D_s, -a), u(D_l, a)
        return (df_min * (us + ul) + dm * ((m_s - cs_inf) * us + (m_l - cl_inf) * ul)
                + 0.5 * a * dm * dm)

    return _brent(f, -2.0, 2.0)
