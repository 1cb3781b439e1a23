"""Seeded synthetic inputs for the coupled phi-mu LBM step.

This module only builds initial fields (phi0, c0) and parameter sets.  It
holds none of the time step's arithmetic, and both the CUDA path and the CPU
oracle take their inputs from it.  All sizes, widths and diffusivities are in
lattice units (dx = dt = 1).

Phase convention (Tab. 2): phi = 0 is the solid, phi = 1 the liquid.

Parameter recipe where a workload leaves values open:
  * M_phi = 1.2 D_l, the ratio of every run in Sec. 4 and Sec. 5;
  * gamma = 1 / M_phi (Sec. 3.3), so tau_g = tau_h = 3 M_phi;
  * lambda = lambda* of Eq. Lambda-Star with the integrals printed in Tab. 3;
  * c_s^co = 1.0, c_l^co = 0.5, mu_eq = 0.4;
  * anti-trapping coefficient a = (1 - D_s/D_l)/4 (Sec. 2.4.2).

Workloads:
  planar_1d   512x8 planar front, solid for x < 128 (Eq. C_init blend)
  disc_2d     512x512 periodic, disc of radius 60, solid inside, c = c^co(phi)
  porous_3d   256^3 periodic Gaussian-random-field medium, porosity 0.35, W = 3
  batch_2d    384 square instances, 64..768 a side, 1-8 solid discs each
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

# Tab. 3 as printed: I = 2/3, K = (31 - 30 ln 2)/150, F = ln 2 / 4.
_I = 2.0 / 3.0
_K = (31.0 - 30.0 * math.log(2.0)) / 150.0
_F = math.log(2.0) / 4.0


def lambda_star(D_l: float, M_phi: float, dc: float) -> float:
    """Coupling constant lambda* (Eq. Lambda-Star) with Tab. 3's printed integrals."""
    return D_l / (M_phi * dc * dc) * _I / (_K + _F)


@dataclass
class ModelParams:
    """Model parameters in lattice units; mirrors the C struct field by field."""
    nx: int
    ny: int
    nz: int = 1
    bc: tuple = (0, 0, 0)          # per axis: 0 periodic, 1 half-way bounce-back
    tau_g: float = 0.36
    tau_h: float = 0.36
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
    h_lattice: int = 0             # 1: h on D2Q5 / D3Q7 (Sec. 3.1)
    h_eq_alt: int = 0              # 1: alternative equilibrium with H = 0 (Sec. 3.3)
    unequal_eps: int = 0           # 1: parabolas of curvature ratio eps_ratio (Sec. 2.3)
    eps_ratio: float = 1.0         # eps_s / eps_l

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def M_phi(self) -> float:
        return self.tau_g / 3.0


def recipe(nx, ny, nz=1, *, D_l, D_s, W, ratio=1.2, counter_term=1, anti_trapping=None,
           c_s_co=1.0, c_l_co=0.5, mu_eq=0.4, bc=(0, 0, 0), lam=None) -> ModelParams:
    """Parameters from the recipe in the module docstring."""
    M = ratio * D_l
    tau = 3.0 * M
    if lam is None:
        lam = lambda_star(D_l, M, c_s_co - c_l_co)
    a = (1.0 - D_s / D_l) / 4.0
    if anti_trapping is None:
        anti_trapping = 1 if a > 0 else 0
    return ModelParams(nx=nx, ny=ny, nz=nz, bc=tuple(bc), tau_g=tau, tau_h=tau, W=W, lam=lam,
                       D_l=D_l, D_s=D_s, c_s_co=c_s_co, c_l_co=c_l_co, mu_eq=mu_eq,
                       counter_term=counter_term, anti_trapping=anti_trapping, a_at=a)


def tanh_profile(d: np.ndarray, W: float) -> np.ndarray:
    """phi = [1 + tanh(2 d / W)] / 2 (Eq. Sol_TanH) of a signed distance d (liquid > 0)."""
    return 0.5 * (1.0 + np.tanh(2.0 * d / W))


def blend(phi: np.ndarray, c_solid: float, c_liquid: float) -> np.ndarray:
    """c = (1 - phi) c_solid + phi c_liquid (the two-level tanh start of Eq. C_init)."""
    return (1.0 - phi) * c_solid + phi * c_liquid


# ---- planar front ----------------------------------------------------------

def planar_1d(nx=512, ny=8, x0=127.5, W=2.5, D_l=0.1, D_s=0.1, c_solid=1.0, c_liquid=0.2,
              counter_term=1, bc=(1, 0, 0)):
    """Planar dissolution front: solid for x < x0, liquid beyond; x walls bounce back."""
    p = recipe(nx, ny, D_l=D_l, D_s=D_s, W=W, counter_term=counter_term, bc=bc)
    x = np.arange(nx, dtype=np.float64)
    phi = np.broadcast_to(tanh_profile(x - x0, W), (1, ny, nx)).copy()
    c = blend(phi, c_solid, c_liquid)
    return p, phi, c


# ---- disc ------------------------------------------------------------------

def disc_2d(n=512, R=60.0, W=3.0, D_l=0.05, D_s=0.05, counter_term=1, equilibrium=True,
            c_liquid=0.2, lam=None):
    """Solid disc of radius R centred in an n x n periodic box.  With
    equilibrium=True the composition sits on the coexistence line, c = c^co(phi)."""
    p = recipe(n, n, D_l=D_l, D_s=D_s, W=W, counter_term=counter_term, lam=lam)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    r = np.hypot(x - (n - 1) / 2.0, y - (n - 1) / 2.0)
    phi = tanh_profile(r - R, W)[None]
    c = blend(phi, p.c_s_co, p.c_l_co if equilibrium else c_liquid)
    return p, phi, c


# ---- Gaussian-random-field porous medium -----------------------------------

def grf_mask(shape, corr=8.0, porosity=0.35, seed=0) -> np.ndarray:
    """Boolean pore mask: white noise (PCG64, seed) convolved periodically with a
    Gaussian of std `corr` cells, thresholded so that `porosity` of the cells are pore."""
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal(shape)
    k = [np.fft.fftfreq(n) for n in shape]
    if len(shape) == 3:
        kz, ky, kx = np.meshgrid(*k, indexing="ij")
        k2 = kx * kx + ky * ky + kz * kz
        field_k = np.fft.rfftn(noise)
        k2 = k2[..., : field_k.shape[-1]]
    else:
        ky, kx = np.meshgrid(*k, indexing="ij")
        k2 = kx * kx + ky * ky
        field_k = np.fft.rfftn(noise)
        k2 = k2[..., : field_k.shape[-1]]
    smooth = np.fft.irfftn(field_k * np.exp(-2.0 * math.pi ** 2 * corr ** 2 * k2), s=shape,
                           axes=tuple(range(len(shape))))
    thr = np.quantile(smooth, porosity)
    return smooth < thr


def signed_distance(mask: np.ndarray, clip=8.0) -> np.ndarray:
    """Signed Euclidean distance to the pore/solid boundary (pore > 0), periodic,
    through an exact EDT of a wrap-padded copy; |d| is clipped at `clip`."""
    from scipy.ndimage import distance_transform_edt
    pad = int(math.ceil(clip)) + 2
    m = np.pad(mask, pad, mode="wrap")
    inner = tuple(slice(pad, pad + n) for n in mask.shape)
    d_pore = distance_transform_edt(m)[inner]
    d_solid = distance_transform_edt(~m)[inner]
    d = np.where(mask, d_pore - 0.5, -(d_solid - 0.5))
    return np.clip(d, -clip, clip)


def porous_3d(n=256, porosity=0.35, seed=0, W=3.0, D_l=0.1, D_s=0.0, c_solid=1.0,
              c_liquid=0.1, corr=8.0, nz=None, counter_term=1, eps_n=1e-6):
    """Synthetic porous medium standing in for the tomography sample of Sec. 5:
    GRF pores (liquid), tanh-smoothed phi, undersaturated liquid.

    W = 3 lattice units: with the coupling lambda* and the counter term, a
    2-node interface (W = 2) diverges within ~150 steps in the FP64 oracle as
    well as on the GPU, while W = 3 stays bounded for thousands of steps.

    eps_n = 1e-6 regularises the unit normal n = grad phi / sqrt(|grad phi|^2 +
    eps_n^2).  The signed distance is clipped, so a sixth of the medium is
    exactly flat bulk where grad phi is nothing but rounding: with eps_n = 1e-12
    n points in an arbitrary unit direction there, a different one in FP32 than
    in FP64.  1e-6 lies above the rounding level of an FP32 gradient and moves n
    by less than 5e-5 (relative) wherever |grad phi| > 1e-4, i.e. on every
    interface node."""
    nz = n if nz is None else nz
    mask = grf_mask((nz, n, n), corr=corr, porosity=porosity, seed=seed)
    d = signed_distance(mask)
    phi = tanh_profile(d, W)
    c = blend(phi, c_solid, c_liquid)
    p = recipe(n, n, nz, D_l=D_l, D_s=D_s, W=W, counter_term=counter_term)
    p = replace(p, eps_n=eps_n)
    return p, phi, c


def differentiable_3d(n=128, porosity=0.4, seed=2, eps_n=1e-3):
    """The differentiable 3-D workload: the porous medium of porous_3d with the
    normal regularised by eps_n = 1e-3, and the seeded target of the slab
    solid-fraction loss (slab_loss): s*_z = s_z(0) - 0.05 u_z, u ~ U[0, 1]
    (PCG64 seed 3), s_z(0) the initial solid fraction of z-slab z.

    With eps_n = 1e-12 the step's Jacobian is ~ phi(1 - phi)/eps_n at nodes where
    grad phi vanishes inside a thin neck or gap (the counter term turns n freely
    there), so adjoints through such media reach 1e5..1e25 and no finite
    difference can follow them; eps_n = 1e-3 leaves interfaces (|grad phi| ~ 0.1)
    unchanged to ~1e-4 and bounds that factor."""
    p, phi, c = porous_3d(n, porosity=porosity, seed=seed)
    p = replace(p, eps_n=eps_n)
    s0 = (1.0 - phi).mean(axis=(1, 2))
    u = np.random.Generator(np.random.PCG64(3)).uniform(0.0, 1.0, p.nz)
    return p, phi, c, s0 - 0.05 * u


def slab_loss(phi, target):
    """L = sum_z (s_z - s*_z)^2 with s_z = mean_xy(1 - phi) the solid fraction of
    z-slab z (phi = 0 is the solid), and dL/dphi.  phi: (nz, ny, nx); works on
    numpy arrays and on torch tensors."""
    nz, ny, nx = phi.shape
    s = 1.0 - phi.mean(axis=(1, 2)) if isinstance(phi, np.ndarray) else 1.0 - phi.mean(dim=(1, 2))
    r = s - target
    loss = float((r * r).sum())
    g = (-2.0 / (nx * ny)) * r
    if isinstance(phi, np.ndarray):
        return loss, np.broadcast_to(g[:, None, None], phi.shape).copy()
    return loss, g[:, None, None].expand(phi.shape).contiguous()


# ---- the paper's porous-medium experiment (Sec. 5) on a synthetic slice -----

def paper_e4_2d(n=1024, counter_term=1, porosity=0.35, corr=16.0, seed=4):
    """The dissolution experiment of Sec. 5 on a synthetic 2-D porous slice.

    The paper's slice of a microtomography sample is not available; a Gaussian
    random field thresholded at `porosity` (pores = liquid, correlation length
    `corr` nodes, PCG64 `seed`) stands in for it.  Everything else follows
    Sec. 5: the unit square on n x n nodes (dx = 1/n), dt = 5e-7, zero-flux
    walls on all sides, M_phi = 1.2, W = 0.02, lambda* = 230, c_s^co = 0.6,
    c_l^co = 0.5, mu_eq = 0.4, D_s = 0, D_l = 1, the anti-trapping current on
    (a = 1/4), discontinuous start: phi = 0 and c = 0.6 in the solid, phi = 1
    and c = 0.4 in the liquid.  Returned in lattice units (gamma = 1/M_phi, so
    tau_g = tau_h = 3 M_phi dt/dx^2)."""
    dx, dt = 1.0 / n, 5e-7
    f = dt / (dx * dx)
    tau = 3.0 * 1.2 * f
    p = ModelParams(nx=n, ny=n, nz=1, bc=(1, 1, 0), tau_g=tau, tau_h=tau, W=0.02 / dx, lam=230.0,
                    D_l=1.0 * f, D_s=0.0, c_s_co=0.6, c_l_co=0.5, mu_eq=0.4,
                    counter_term=counter_term, anti_trapping=1, a_at=0.25)
    pore = grf_mask((n, n), corr=corr, porosity=porosity, seed=seed)
    phi = np.where(pore, 1.0, 0.0)[None, :, :]
    c = np.where(pore, 0.4, 0.6)[None, :, :]
    return p, phi, c


# ---- batch of 2-D instances ------------------------------------------------

@dataclass
class Instance:
    params: ModelParams
    phi: np.ndarray
    c: np.ndarray


def batch_2d(count=384, seed=1, nmin=64, nmax=768, W=3.0, c_liquid=0.2):
    """Uneven 2-D instances: side ~ U{nmin..nmax}, 1-8 solid discs of radius
    U[8, 40] at uniform (periodic) centres, D_l ~ U[0.02, 0.2],
    M_phi / D_l ~ U[0.5, 5], counter term on or off with probability 1/2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        ndisc = int(rng.integers(1, 9))
        radii = rng.uniform(8.0, 40.0, ndisc)
        centres = rng.uniform(0.0, n, (ndisc, 2))
        D_l = float(rng.uniform(0.02, 0.2))
        ratio = float(rng.uniform(0.5, 5.0))
        ct = int(rng.integers(0, 2))
        y, x = np.mgrid[0:n, 0:n].astype(np.float64)
        d = np.full((n, n), np.inf)
        for (cx, cy), r in zip(centres, radii):
            dx = np.abs(x - cx); dx = np.minimum(dx, n - dx)
            dy = np.abs(y - cy); dy = np.minimum(dy, n - dy)
            d = np.minimum(d, np.hypot(dx, dy) - r)
        phi = tanh_profile(d, W)[None]
        p = recipe(n, n, D_l=D_l, D_s=D_l, W=W, ratio=ratio, counter_term=ct)
        c = blend(phi, p.c_s_co, c_liquid)
        out.append(Instance(p, phi, c))
    return out


def random_fields(shape, seed, smooth=True):
    """Smooth random (phi, c) in (0, 1) for parity tests: every term of the step is
    exercised everywhere (no flat bulk)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.uniform(0.05, 0.95, shape)
    b = rng.uniform(0.1, 0.9, shape)
    if smooth:
        for arr in (a, b):
            for ax in range(len(shape)):
                if shape[ax] > 2:
                    arr[...] = 0.5 * arr + 0.25 * (np.roll(arr, 1, ax) + np.roll(arr, -1, ax))
    return a, b
