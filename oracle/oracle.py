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
_SRC_CS = os.path.join(_HERE, "tangent_cs.c")
_LIB_CS = os.path.join(_HERE, "_build", "liblbpf_oracle_cs.so")
_lib = None
_lib_cs = None


def _compile(src, lib, deps, force):
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    stale = (not os.path.exists(lib)) or any(os.path.getmtime(lib) < os.path.getmtime(d) for d in deps)
    if force or stale:
        tmp = lib + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-std=c99",
                               "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile the oracle and its complex-step build with gcc (no FMA
    contraction, OpenMP over rows)."""
    _compile(_SRC_CS, _LIB_CS, [_SRC, _SRC_CS], force)
    return _compile(_SRC, _LIB, [_SRC], force)


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
        _lib.or_step_adjoint.argtypes = [ctypes.c_void_p] + [dp] * 9
        _lib.or_init_adjoint.argtypes = [ctypes.c_void_p] + [dp] * 7
    return _lib


def _load_cs():
    global _lib_cs
    if _lib_cs is None:
        build()
        _lib_cs = ctypes.CDLL(_LIB_CS)
        vp = ctypes.c_void_p
        _lib_cs.or_init.argtypes = [vp] * 7
        _lib_cs.or_step.argtypes = [vp] * 5 + [ctypes.c_int]
    return _lib_cs


class _CParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("bc", ctypes.c_int * 3),
                ("tau_g", ctypes.c_double), ("tau_h", ctypes.c_double),
                ("W", ctypes.c_double), ("lam", ctypes.c_double),
                ("D_l", ctypes.c_double), ("D_s", ctypes.c_double),
                ("c_s_co", ctypes.c_double), ("c_l_co", ctypes.c_double),
                ("mu_eq", ctypes.c_double), ("counter_term", ctypes.c_int),
                ("anti_trapping", ctypes.c_int), ("a_at", ctypes.c_double),
                ("eps_n", ctypes.c_double), ("h_lattice", ctypes.c_int), ("h_eq_alt", ctypes.c_int),
                ("unequal_eps", ctypes.c_int), ("eps_ratio", ctypes.c_double)]


@dataclass
class OracleParams:
    """Model parameters in lattice units (dx = dt = 1).

    M_phi = tau_g / 3 (Sec. 3.2) and gamma = 3 / tau_h (Sec. 3.3).  h_lattice = 1
    puts h on D2Q5 / D3Q7 (xi_s^2 = 1/3); h_eq_alt = 1 uses the alternative
    equilibrium of Eq. Seq_Concent_Alt with H = 0 (Sec. 3.3).  unequal_eps = 1
    gives the parabolas the curvature ratio eps_ratio = eps_s / eps_l (Sec. 2.3:
    Eq. Closure, Eq. SourceTerm, Eq. Anti-Trapping_Quadratic)."""
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
    h_lattice: int = 0
    h_eq_alt: int = 0
    unequal_eps: int = 0
    eps_ratio: float = 1.0

    @property
    def dim(self) -> int:
        return 3 if self.nz > 1 else 2

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def q(self) -> int:
        return 19 if self.dim == 3 else 9

    @property
    def q_h(self) -> int:
        if self.h_lattice:
            return 7 if self.dim == 3 else 5
        return self.q

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
        c.h_lattice, c.h_eq_alt = int(self.h_lattice), int(self.h_eq_alt)
        c.unequal_eps, c.eps_ratio = int(self.unequal_eps), float(self.eps_ratio)
        return c


class _CParamsCS(ctypes.Structure):
    """or_params of the complex-step build: every double is a (re, im) pair."""
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("bc", ctypes.c_int * 3), ("pad", ctypes.c_int),
                ("tau_g", ctypes.c_double * 2), ("tau_h", ctypes.c_double * 2),
                ("W", ctypes.c_double * 2), ("lam", ctypes.c_double * 2),
                ("D_l", ctypes.c_double * 2), ("D_s", ctypes.c_double * 2),
                ("c_s_co", ctypes.c_double * 2), ("c_l_co", ctypes.c_double * 2),
                ("mu_eq", ctypes.c_double * 2), ("counter_term", ctypes.c_int),
                ("anti_trapping", ctypes.c_int), ("a_at", ctypes.c_double * 2),
                ("eps_n", ctypes.c_double * 2), ("h_lattice", ctypes.c_int), ("h_eq_alt", ctypes.c_int),
                ("unequal_eps", ctypes.c_int), ("pad2", ctypes.c_int), ("eps_ratio", ctypes.c_double * 2)]


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lattice_tables(code: int):
    """(e [q,3] int, w [q], opp [q]) of an oracle lattice: code 2 D2Q9, 3 D3Q19,
    5 D2Q5, 7 D3Q7."""
    lib = _load()
    e = (ctypes.c_int * 57)()
    w = np.zeros(19)
    opp = (ctypes.c_int * 19)()
    q = lib.or_lattice(code, e, _dp(w), opp)
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
        q = p.q
        self.q = q
        shp = p.shape
        self.phi = np.zeros(shp)
        self.c = np.zeros(shp)
        self.g = np.zeros((q,) + shp)
        self.h = np.zeros((p.q_h,) + shp)
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
        o.q = p.q
        o.g = np.ascontiguousarray(g, dtype=np.float64).reshape((o.q,) + p.shape).copy()
        o.h = np.ascontiguousarray(h, dtype=np.float64).reshape((p.q_h,) + p.shape).copy()
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


# ---- discrete adjoint and complex-step tangents -------------------------------

PARAM_NAMES = ("D_l", "tau_g", "tau_h", "lam")


def step_adjoint(p: OracleParams, g, h, phi, c, gb, hb, phib, cb):
    """Adjoint of one step at state (g, h, phi, c): maps the adjoints of the state
    at n+1 to those at n; returns (gb, hb, phib, cb, pb) with pb the adjoints of
    (D_l, tau_g, tau_h, lambda)."""
    cp = p._c()
    arrs = [np.ascontiguousarray(a, dtype=np.float64).copy() for a in (gb, hb, phib, cb)]
    st = [np.ascontiguousarray(a, dtype=np.float64) for a in (g, h, phi, c)]
    pb = np.zeros(4)
    rc = _load().or_step_adjoint(ctypes.byref(cp), *[_dp(a) for a in st], *[_dp(a) for a in arrs], _dp(pb))
    if rc != 0:
        raise MemoryError("oracle adjoint failed")
    return (*arrs, pb)


def init_adjoint(p: OracleParams, phi0, c0, gb, hb, phib, cb):
    """Adjoint of the initialisation: returns (adjoint of phi0, of c0, pb)."""
    cp = p._c()
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    c0 = np.ascontiguousarray(c0, dtype=np.float64)
    gb = np.ascontiguousarray(gb, dtype=np.float64)
    hb = np.ascontiguousarray(hb, dtype=np.float64)
    phib = np.ascontiguousarray(phib, dtype=np.float64).copy()
    cb = np.ascontiguousarray(cb, dtype=np.float64).copy()
    pb = np.zeros(4)
    rc = _load().or_init_adjoint(ctypes.byref(cp), _dp(phi0), _dp(c0), _dp(gb), _dp(hb), _dp(phib), _dp(cb),
                                 _dp(pb))
    if rc != 0:
        raise MemoryError("oracle adjoint failed")
    return phib, cb, pb


def trajectory_gradient(p: OracleParams, phi0, c0, nsteps, phib_final, cb_final):
    """Gradient of L(phi_n, c_n) given dL/dphi_n, dL/dc_n after nsteps steps from
    (phi0, c0): forward storing every state, then the adjoint steps in reverse and
    the adjoint of the initialisation.  Returns (dL/dphi0, dL/dc0, dL/dparams)."""
    o = Oracle(p, phi0, c0)
    states = [(o.g.copy(), o.h.copy(), o.phi.copy(), o.c.copy())]
    for _ in range(nsteps):
        o.step(1)
        states.append((o.g.copy(), o.h.copy(), o.phi.copy(), o.c.copy()))
    gb = np.zeros_like(o.g)
    hb = np.zeros_like(o.h)
    phib = np.ascontiguousarray(phib_final, dtype=np.float64).reshape(p.shape).copy()
    cb = np.ascontiguousarray(cb_final, dtype=np.float64).reshape(p.shape).copy()
    ptot = np.zeros(4)
    for n in range(nsteps - 1, -1, -1):
        gb, hb, phib, cb, pb = step_adjoint(p, *states[n], gb, hb, phib, cb)
        ptot += pb
    phi0b, c0b, pb = init_adjoint(p, phi0, c0, gb, hb, phib, cb)
    return phi0b, c0b, ptot + pb


def _cs_params(p: OracleParams, dparams, h):
    c = _CParamsCS()
    c.dim, c.nx, c.ny, c.nz = p.dim, p.nx, p.ny, p.nz
    for a in range(3):
        c.bc[a] = int(p.bc[a])
    d = dict(zip(PARAM_NAMES, dparams if dparams is not None else (0.0,) * 4))
    for name in ("tau_g", "tau_h", "W", "lam", "D_l", "D_s", "c_s_co", "c_l_co", "mu_eq", "a_at", "eps_n"):
        getattr(c, name)[0] = getattr(p, name)
        getattr(c, name)[1] = h * d.get(name, 0.0)
    c.counter_term, c.anti_trapping = int(p.counter_term), int(p.anti_trapping)
    c.h_lattice, c.h_eq_alt = int(p.h_lattice), int(p.h_eq_alt)
    c.unequal_eps = int(p.unequal_eps)
    c.eps_ratio[0] = p.eps_ratio
    return c


def tangent_trajectory(p: OracleParams, phi0, c0, nsteps, dphi0=None, dc0=None, dparams=None, h=1e-30):
    """Exact directional derivative (complex step) of the state after nsteps steps
    along (dphi0, dc0, dparams); returns (dg, dh, dphi, dc)."""
    lib = _load_cs()
    cp = _cs_params(p, dparams, h)
    shp = p.shape
    q = p.q
    z = lambda a: np.zeros(shp) if a is None else np.asarray(a, dtype=np.float64).reshape(shp)
    phi0c = np.ascontiguousarray(np.asarray(phi0, dtype=np.float64).reshape(shp) + 1j * h * z(dphi0))
    c0c = np.ascontiguousarray(np.asarray(c0, dtype=np.float64).reshape(shp) + 1j * h * z(dc0))
    g = np.zeros((q,) + shp, complex)
    hh = np.zeros((p.q_h,) + shp, complex)
    phi = np.zeros(shp, complex)
    c = np.zeros(shp, complex)
    P = lambda a: a.ctypes.data
    lib.or_init(ctypes.byref(cp), P(phi0c), P(c0c), P(g), P(hh), P(phi), P(c))
    if nsteps:
        lib.or_step(ctypes.byref(cp), P(g), P(hh), P(phi), P(c), int(nsteps))
    return g.imag / h, hh.imag / h, phi.imag / h, c.imag / h


def tangent_step(p: OracleParams, g, hpop, phi, c, dg, dh, dphi, dc, dparams=None, h=1e-30):
    """Exact directional derivative (complex step) of one step from state
    (g, h, phi, c) along (dg, dh, dphi, dc, dparams)."""
    lib = _load_cs()
    cp = _cs_params(p, dparams, h)
    G = np.ascontiguousarray(g + 1j * h * dg)
    H = np.ascontiguousarray(hpop + 1j * h * dh)
    F = np.ascontiguousarray(phi + 1j * h * dphi)
    C = np.ascontiguousarray(c + 1j * h * dc)
    lib.or_step(ctypes.byref(cp), G.ctypes.data, H.ctypes.data, F.ctypes.data, C.ctypes.data, 1)
    return G.imag / h, H.imag / h, F.imag / h, C.imag / h
