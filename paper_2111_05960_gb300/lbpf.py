"""Thin ctypes binding of libgb_lbpf (include/lbpf.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Host arrays are numpy float64 (C order); device arrays are anything
with ``data_ptr()`` (a CUDA torch tensor, float64, contiguous).  There is no CPU
fallback: if the library is missing, loading fails with an error that says how
to build it.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import fields as dc_fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgb_lbpf.so")

LBPF_OK, LBPF_EINVAL, LBPF_ENOMEM, LBPF_ECUDA, LBPF_EUNSTABLE = range(5)
LBPF_ESTATE, LBPF_EUNSUPPORTED = 6, 7          # 5 is unused (no call times out)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EUNSTABLE", "(unused)", "ESTATE", "EUNSUPPORTED"]
LBPF_D2Q9, LBPF_D3Q19, LBPF_D2Q5, LBPF_D3Q7 = 0, 1, 2, 3
LBPF_FP64, LBPF_FP32, LBPF_FP32_BF16DEV, LBPF_FP32_FP16DEV = 0, 1, 2, 3
PRECISIONS = {"fp64": LBPF_FP64, "fp32": LBPF_FP32, "bf16dev": LBPF_FP32_BF16DEV,
              "fp16dev": LBPF_FP32_FP16DEV}


class LbpfError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("LBPF_%s: %s" % (name, message))


class lbpf_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("lattice", ctypes.c_int32), ("bc", ctypes.c_int32 * 3),
                ("precision", ctypes.c_int32), ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("tau_g", ctypes.c_double), ("tau_h", ctypes.c_double), ("W", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("D_l", ctypes.c_double), ("D_s", ctypes.c_double),
                ("c_s_co", ctypes.c_double), ("c_l_co", ctypes.c_double),
                ("mu_eq", ctypes.c_double), ("counter_term", ctypes.c_int32),
                ("anti_trapping", ctypes.c_int32), ("a_at", ctypes.c_double),
                ("eps_n", ctypes.c_double), ("mass_every", ctypes.c_int32),
                ("checkpoint_every", ctypes.c_int32), ("h_lattice", ctypes.c_int32),
                ("h_eq_alt", ctypes.c_int32), ("unequal_eps", ctypes.c_int32),
                ("eps_ratio", ctypes.c_double)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


def load() -> ctypes.CDLL:
    """Load libgb_lbpf.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libgb_lbpf.so is not built (%s); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    sig = {
        "lbpf_default_params": [ctypes.POINTER(lbpf_params)],
        "lbpf_create": [ctypes.POINTER(lbpf_params), _vp, _vp, ctypes.c_int32, _vp,
                        ctypes.POINTER(_vp)],
        "lbpf_step": [_vp, ctypes.c_int64],
        "lbpf_step_timed": [_vp, ctypes.c_int64, _dp],
        "lbpf_mass": [_vp, _dp, _dp],
        "lbpf_get_fields": [_vp, _vp, _vp, _vp, ctypes.c_int32],
        "lbpf_get_populations": [_vp, _vp, _vp, ctypes.c_int32],
        "lbpf_get_step": [_vp, ctypes.POINTER(ctypes.c_int64)],
        "lbpf_destroy": [_vp],
        "lbpf_lattice_info": [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ctypes.c_int32), _dp],
        "lbpf_mass_noalloc": [_vp, _vp, ctypes.c_int64, ctypes.c_int32, _vp, _vp],
        "lbpf_solute_mass": [_vp, _dp, _dp],
        "lbpf_create_batch": [ctypes.POINTER(lbpf_params), ctypes.c_int32, ctypes.POINTER(_vp),
                              ctypes.POINTER(_vp), ctypes.c_int32, _vp, ctypes.POINTER(_vp)],
        "lbpf_batch_get_fields": [_vp, ctypes.c_int32, _vp, _vp, _vp, ctypes.c_int32],
        "lbpf_batch_solute_mass": [_vp, _dp],
        "lbpf_adjoint_step": [_vp, _vp, _vp, _vp, _vp, ctypes.c_int32, _dp],
        "lbpf_batch_tile": [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), _dp],
        "lbpf_batch_set_tile": [_vp, ctypes.c_int32, ctypes.c_int32],
        "lbpf_fp64_fma_rate": [_vp, _dp],
        "lbpf_pull_path": [_vp, ctypes.POINTER(ctypes.c_int32)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = st
    lib.lbpf_last_error.argtypes = [_vp]
    lib.lbpf_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def exported_symbols():
    """Names declared in include/lbpf.h that the loaded library must export."""
    return ["lbpf_default_params", "lbpf_create", "lbpf_step", "lbpf_step_timed", "lbpf_mass",
            "lbpf_get_fields", "lbpf_get_populations", "lbpf_get_step", "lbpf_destroy",
            "lbpf_last_error", "lbpf_lattice_info", "lbpf_mass_noalloc", "lbpf_solute_mass",
            "lbpf_create_batch", "lbpf_batch_get_fields", "lbpf_batch_solute_mass",
            "lbpf_adjoint_step", "lbpf_batch_tile", "lbpf_batch_set_tile", "lbpf_fp64_fma_rate",
            "lbpf_pull_path"]


def _check(status: int, ctx=None):
    if status != LBPF_OK:
        msg = load().lbpf_last_error(ctx)
        raise LbpfError(status, msg.decode() if msg else "")


def _ptr(a):
    """(address, is_device) of a numpy array or a CUDA tensor; None -> (None, None)."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):
        if a.dtype.__str__() != "torch.float64" or not a.is_contiguous():
            raise ValueError("device arrays must be contiguous float64")
        return a.data_ptr(), bool(a.is_cuda)
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError("host arrays must be C-contiguous float64 numpy arrays")
    return a.ctypes.data, False


# ---- the ABI, one function per C entry point ---------------------------------------

def lbpf_default_params() -> lbpf_params:
    p = lbpf_params()
    _check(load().lbpf_default_params(ctypes.byref(p)))
    return p


def lbpf_create(p: lbpf_params, phi0, c0, ptr_is_device: int, cuda_stream=None):
    ctx = _vp()
    a, _ = _ptr(phi0)
    b, _ = _ptr(c0)
    _check(load().lbpf_create(ctypes.byref(p), a, b, int(ptr_is_device), cuda_stream or None,
                              ctypes.byref(ctx)))
    return ctx


def lbpf_step(ctx, nsteps: int) -> None:
    _check(load().lbpf_step(ctx, int(nsteps)), ctx)


def lbpf_step_timed(ctx, nsteps: int):
    """(phi kernel, composition kernel, mass correction) milliseconds summed over nsteps."""
    ms = (ctypes.c_double * 3)()
    _check(load().lbpf_step_timed(ctx, int(nsteps), ms), ctx)
    return float(ms[0]), float(ms[1]), float(ms[2])


def lbpf_solute_mass(ctx):
    """(exact population mass, mass held by the correction or NaN)."""
    m, t = ctypes.c_double(), ctypes.c_double()
    _check(load().lbpf_solute_mass(ctx, ctypes.byref(m), ctypes.byref(t)), ctx)
    return m.value, t.value


def lbpf_mass(ctx):
    tc, tp = ctypes.c_double(), ctypes.c_double()
    _check(load().lbpf_mass(ctx, ctypes.byref(tc), ctypes.byref(tp)), ctx)
    return tc.value, tp.value


def lbpf_get_fields(ctx, phi=None, c=None, mu=None, ptr_is_device: int = 0) -> None:
    _check(load().lbpf_get_fields(ctx, _ptr(phi)[0], _ptr(c)[0], _ptr(mu)[0], int(ptr_is_device)), ctx)


def lbpf_get_populations(ctx, g=None, h=None, ptr_is_device: int = 0) -> None:
    _check(load().lbpf_get_populations(ctx, _ptr(g)[0], _ptr(h)[0], int(ptr_is_device)), ctx)


def lbpf_get_step(ctx) -> int:
    s = ctypes.c_int64()
    _check(load().lbpf_get_step(ctx, ctypes.byref(s)), ctx)
    return s.value


def lbpf_destroy(ctx) -> None:
    if ctx:
        load().lbpf_destroy(ctx)


def lbpf_last_error(ctx=None) -> str:
    m = load().lbpf_last_error(ctx)
    return m.decode() if m else ""


def lbpf_create_batch(params, phi0s, c0s, ptr_is_device: int = 0, cuda_stream=None):
    """params: sequence of lbpf_params; phi0s, c0s: sequences of per-instance fields."""
    n = len(params)
    arr = (lbpf_params * n)(*params)
    pp = (_vp * n)(*[_ptr(a)[0] for a in phi0s])
    cp = (_vp * n)(*[_ptr(a)[0] for a in c0s])
    ctx = _vp()
    _check(load().lbpf_create_batch(arr, n, pp, cp, int(ptr_is_device), cuda_stream or None, ctypes.byref(ctx)))
    return ctx


def lbpf_batch_get_fields(ctx, i: int, phi=None, c=None, mu=None, ptr_is_device: int = 0) -> None:
    _check(load().lbpf_batch_get_fields(ctx, int(i), _ptr(phi)[0], _ptr(c)[0], _ptr(mu)[0],
                                        int(ptr_is_device)), ctx)


def lbpf_batch_solute_mass(ctx, n: int) -> np.ndarray:
    out = np.zeros(n)
    _check(load().lbpf_batch_solute_mass(ctx, out.ctypes.data_as(_dp)), ctx)
    return out


BATCH_TILES = ((32, 32), (32, 64), (64, 32), (64, 64), (128, 32))


def lbpf_batch_tile(ctx):
    """((tile_x, tile_rows) in use, ms per step of each shape in BATCH_TILES)."""
    tx, tr = ctypes.c_int32(), ctypes.c_int32()
    ms = np.zeros(len(BATCH_TILES))
    _check(load().lbpf_batch_tile(ctx, ctypes.byref(tx), ctypes.byref(tr), ms.ctypes.data_as(_dp)))
    return (tx.value, tr.value), ms


def lbpf_batch_set_tile(ctx, tile_x: int, tile_rows: int) -> None:
    _check(load().lbpf_batch_set_tile(ctx, int(tile_x), int(tile_rows)), ctx)


NOALLOC_MAX_ELEMENTS = 67108864


def _stream_handle(cuda_stream):
    """A cudaStream_t address from None, an int or a torch.cuda.Stream."""
    if cuda_stream is None:
        return None
    if hasattr(cuda_stream, "cuda_stream"):
        return cuda_stream.cuda_stream or None
    return int(cuda_stream) or None


def lbpf_mass_noalloc(c_dev, phi_dev, n: int, precision: int, out_dev, cuda_stream=None) -> None:
    """Sums of c and phi over caller-owned device arrays into out_dev (3 doubles on
    the device), with no allocation; see include/lbpf.h.  Queued on cuda_stream
    (None, a cudaStream_t address or a torch.cuda.Stream).  c_dev, phi_dev: CUDA
    tensors, contiguous, float64 for LBPF_FP64 or float32 for LBPF_FP32, with at
    least n elements; out_dev: a contiguous CUDA float64 tensor of >= 3 elements."""
    import torch
    want = {LBPF_FP64: torch.float64, LBPF_FP32: torch.float32}.get(int(precision))
    for name, t in (("c", c_dev), ("phi", phi_dev)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise ValueError("%s must be a contiguous CUDA tensor" % name)
        if want is not None and t.dtype != want:
            raise ValueError("%s has dtype %s; precision %d needs %s" % (name, t.dtype, precision, want))
        if t.numel() < max(int(n), 0):
            raise ValueError("%s has %d elements, fewer than n = %d" % (name, t.numel(), n))
    if not (isinstance(out_dev, torch.Tensor) and out_dev.is_cuda and out_dev.is_contiguous()
            and out_dev.dtype == torch.float64 and out_dev.numel() >= 3):
        raise ValueError("out_dev must be a contiguous CUDA float64 tensor of at least 3 elements")
    _check(load().lbpf_mass_noalloc(c_dev.data_ptr(), phi_dev.data_ptr(), int(n), int(precision),
                                    out_dev.data_ptr(), _stream_handle(cuda_stream)))


ADJ_PARAM_NAMES = ("D_l", "tau_g", "tau_h", "lam", "a_at", "D_s")


def lbpf_adjoint_step(ctx, dL_dphi=None, dL_dc=None, dL_dphi0=None, dL_dc0=None,
                      ptr_is_device: int = 0) -> np.ndarray:
    """Reverse sweep over the trajectory since creation (see include/lbpf.h).
    Writes dL/dphi0, dL/dc0 into the given arrays (either may be None) and
    returns the parameter adjoints, ordered as ADJ_PARAM_NAMES."""
    out = np.zeros(len(ADJ_PARAM_NAMES))
    _check(load().lbpf_adjoint_step(ctx, _ptr(dL_dphi)[0], _ptr(dL_dc)[0], _ptr(dL_dphi0)[0],
                                    _ptr(dL_dc0)[0], int(ptr_is_device), out.ctypes.data_as(_dp)), ctx)
    return out


def lbpf_pull_path(ctx) -> int:
    """1 if the step kernels pull the populations through tensor maps, else 0."""
    v = ctypes.c_int32()
    _check(load().lbpf_pull_path(ctx, ctypes.byref(v)), ctx)
    return int(v.value)


def lbpf_fp64_fma_rate(cuda_stream=None) -> float:
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    t = ctypes.c_double()
    _check(load().lbpf_fp64_fma_rate(cuda_stream or None, ctypes.byref(t)))
    return t.value


def lbpf_lattice_info(lattice: int):
    q = ctypes.c_int32()
    e = (ctypes.c_int32 * 57)()
    w = np.zeros(19)
    _check(load().lbpf_lattice_info(int(lattice), ctypes.byref(q), e, w.ctypes.data_as(_dp)))
    n = q.value
    return np.array(e[:3 * n], dtype=np.int64).reshape(n, 3), w[:n].copy()


# ---- convenience wrapper -------------------------------------------------------------

def params_from(model, precision="fp64", dx=1.0, dt=1.0, mass_every=0, checkpoint_every=0) -> lbpf_params:
    """lbpf_params from a workloads.ModelParams (lattice units unless dx, dt given)."""
    p = lbpf_default_params()
    p.nx, p.ny, p.nz = model.nx, model.ny, model.nz
    p.lattice = LBPF_D3Q19 if model.nz > 1 else LBPF_D2Q9
    for a in range(3):
        p.bc[a] = int(model.bc[a])
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.dx, p.dt = dx, dt
    p.tau_g, p.tau_h, p.W, p.lambda_ = model.tau_g, model.tau_h, model.W, model.lam
    p.D_l, p.D_s = model.D_l, model.D_s
    p.c_s_co, p.c_l_co, p.mu_eq = model.c_s_co, model.c_l_co, model.mu_eq
    p.counter_term, p.anti_trapping = int(model.counter_term), int(model.anti_trapping)
    p.a_at, p.eps_n = model.a_at, model.eps_n
    p.mass_every = int(mass_every)
    p.checkpoint_every = int(checkpoint_every)
    p.h_lattice = int(getattr(model, "h_lattice", 0))
    p.h_eq_alt = int(getattr(model, "h_eq_alt", 0))
    p.unequal_eps = int(getattr(model, "unequal_eps", 0))
    p.eps_ratio = float(getattr(model, "eps_ratio", 1.0))
    return p


class Simulation:
    """One GPU simulation context.  Host fields in/out are numpy float64 arrays
    shaped (nz, ny, nx); device fields are CUDA float64 tensors."""

    def __init__(self, model, phi0, c0, precision="fp64", stream=None, lattice=None, mass_every=0,
                 checkpoint_every=0):
        self.model = model
        self.params = params_from(model, precision, mass_every=mass_every, checkpoint_every=checkpoint_every)
        if lattice is not None:
            self.params.lattice = int(lattice)
        is_dev = hasattr(phi0, "data_ptr")
        if not is_dev:
            phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
            c0 = np.ascontiguousarray(c0, dtype=np.float64)
        self.ctx = lbpf_create(self.params, phi0, c0, int(is_dev), stream)
        self.q = 19 if self.params.lattice == LBPF_D3Q19 else 9
        self.q_h = (7 if self.q == 19 else 5) if self.params.h_lattice else self.q
        self.shape = (model.nz, model.ny, model.nx)

    def step(self, n=1):
        lbpf_step(self.ctx, n)
        return self

    def step_timed(self, n):
        return lbpf_step_timed(self.ctx, n)

    def mass(self):
        return lbpf_mass(self.ctx)

    def solute_mass(self):
        return lbpf_solute_mass(self.ctx)

    def fields(self):
        phi, c, mu = (np.empty(self.shape) for _ in range(3))
        lbpf_get_fields(self.ctx, phi, c, mu, 0)
        return phi, c, mu

    def adjoint(self, dL_dphi=None, dL_dc=None):
        """(dL/dphi0, dL/dc0, parameter adjoints) of a loss of the current fields;
        needs checkpoint_every > 0 at construction."""
        as_np = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape)
        dphi0, dc0 = np.empty(self.shape), np.empty(self.shape)
        pv = lbpf_adjoint_step(self.ctx, as_np(dL_dphi), as_np(dL_dc), dphi0, dc0, 0)
        return dphi0, dc0, pv

    def populations(self):
        g = np.empty((self.q,) + self.shape)
        h = np.empty((self.q_h,) + self.shape)
        lbpf_get_populations(self.ctx, g, h, 0)
        return g, h

    @property
    def t(self):
        return lbpf_get_step(self.ctx)

    def close(self):
        if self.ctx:
            lbpf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSimulation:
    """Many 2-D instances stepped together (lbpf_create_batch).  models: sequence
    of workloads.ModelParams; phis, cs: their initial fields."""

    def __init__(self, models, phis, cs, precision="fp32", stream=None):
        self.models = list(models)
        self.n = len(self.models)
        params = [params_from(m, precision) for m in self.models]
        phis = [np.ascontiguousarray(a, dtype=np.float64) for a in phis]
        cs = [np.ascontiguousarray(a, dtype=np.float64) for a in cs]
        self.ctx = lbpf_create_batch(params, phis, cs, 0, stream)
        self.nodes = sum(m.nodes for m in self.models)

    def step(self, n=1):
        lbpf_step(self.ctx, n)
        return self

    def step_timed(self, n):
        return lbpf_step_timed(self.ctx, n)

    def fields(self, i):
        m = self.models[i]
        phi, c, mu = (np.empty((m.nz, m.ny, m.nx)) for _ in range(3))
        lbpf_batch_get_fields(self.ctx, i, phi, c, mu, 0)
        return phi, c, mu

    def solute_masses(self):
        return lbpf_batch_solute_mass(self.ctx, self.n)

    def tile(self):
        return lbpf_batch_tile(self.ctx)

    def set_tile(self, tile_x, tile_rows):
        lbpf_batch_set_tile(self.ctx, tile_x, tile_rows)

    def close(self):
        if self.ctx:
            lbpf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
