"""Pins of the oracle's two variants of the composition scheme (Sec. 3.3 and
Sec. 3.1): h on the small lattices D2Q5 / D3Q7 (h_lattice = 1) and the
alternative equilibrium h^eq,alt with H_k = 0 (h_eq_alt = 1, Eq. Seq_Concent_Alt).

Both must reproduce the same macroscopic composition equation as the main
scheme, so they are pinned by what fixes that equation: the lattice moments,
the decay rate of a diffusion mode, exact solute conservation, a stationary
flat front, and the analytic one-sided Stefan dissolution of Sec. 4.2 (whose
flux F = mu D' grad phi + j_at is the term the alternative equilibrium moves).
"""
import math

import numpy as np
import pytest
from scipy.special import erfc

import oracle as O
from paper_2111_05960_gb300 import workloads as WL
from conftest import to_oracle

VARIANTS = [(1, 0), (0, 1), (1, 1)]   # (h_lattice, h_eq_alt)


@pytest.mark.parametrize("code,dim", [(5, 2), (7, 3)])
def test_reduced_lattice_moments(code, dim):
    """sum w = 1, sum w e = 0, 3 sum w e e = I (xi_s^2 = 1/3, so tau_h = 3/gamma holds
    as for D2Q9), zero third moments, opposite pairs.  The directions are the rest
    and axis links of D2Q9 / D3Q19 in the same order.  Catches a weight chosen for
    another xi_s^2 (e.g. the D3Q7 set 1/4, 1/8, which would change the diffusivity)."""
    e, w, opp = O.lattice_tables(code)
    e_full, _, _ = O.lattice_tables(dim)
    assert len(w) == 1 + 2 * dim
    assert np.all(e == e_full[:len(w)])
    assert np.all(np.abs(e).sum(1)[1:] == 1)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.abs((w[:, None] * e).sum(0)).max() < 1e-15
    m2 = 3.0 * np.einsum("k,ka,kb->ab", w, e, e)
    eye = np.eye(3)
    if dim == 2:
        eye[2, 2] = 0.0
    assert np.abs(m2 - eye).max() < 1e-15
    assert np.abs(np.einsum("k,ka,kb,kc->abc", w, e, e, e)).max() < 1e-15
    for k in range(len(w)):
        assert np.all(e[opp[k]] == -e[k])


@pytest.mark.parametrize("dim", [2, 3])
def test_diffusion_mode_decay_on_reduced_lattice(dim):
    """Pure liquid: the composition equation is diffusion with D_l; a Fourier mode
    decays as exp(-D_l k^2 t) on D2Q5 / D3Q7 exactly as on the full lattice.  With
    phi = 1 the flux F vanishes, so the alternative equilibrium gives the same bits."""
    L = 32
    nz = 1 if dim == 2 else L
    D = 0.1
    k = 2 * math.pi / L
    shape = (nz, L, L)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(L), np.arange(L), indexing="ij")
    mode = np.sin(k * (x + y + (z if dim == 3 else 0)))
    kk = k * k * (3 if dim == 3 else 2)
    rates, states = [], []
    for alt in (0, 1):
        p = O.OracleParams(nx=L, ny=L, nz=nz, tau_g=0.36, tau_h=0.9, W=3.0, lam=5.0, D_l=D,
                           D_s=0.5 * D, counter_term=1, anti_trapping=1, h_lattice=1, h_eq_alt=alt)
        o = O.Oracle(p, np.ones(shape), 0.5 + 0.05 * mode)
        n = 600
        o.step(n)
        amp = float(((o.c - 0.5) * mode).sum() / (mode * mode).sum())
        rates.append(-math.log(amp / 0.05) / n)
        states.append(o.c.copy())
    assert rates[0] == pytest.approx(D * kk, rel=0.02)
    assert np.array_equal(states[0], states[1])


@pytest.mark.parametrize("hl,alt", VARIANTS)
@pytest.mark.parametrize("dim,bc", [(2, (0, 0, 0)), (2, (1, 1, 0)), (3, (1, 0, 1))])
def test_solute_mass_is_conserved_with_variants(hl, alt, dim, bc):
    """sum_x c is invariant: the zeroth moment of h^eq,alt is c (its flux part has
    sum_k w_k e_k = 0), and D2Q5 / D3Q7 streaming with bounce-back loses nothing."""
    shape = (6 if dim == 3 else 1, 10, 12)
    phi0, c0 = WL.random_fields(shape, seed=21 + dim)
    p = O.OracleParams(nx=12, ny=10, nz=shape[0], bc=bc, tau_g=0.7, tau_h=0.9, W=3.0, lam=4.0,
                       D_l=0.15, D_s=0.03, counter_term=1, anti_trapping=1, h_lattice=hl, h_eq_alt=alt)
    o = O.Oracle(p, phi0, c0)
    assert o.h.shape[0] == p.q_h
    m0 = o.c.sum()
    o.step(200)
    assert abs(o.c.sum() - m0) / m0 < 1e-13
    assert np.all(np.isfinite(o.phi))


@pytest.mark.parametrize("hl,alt", VARIANTS)
def test_initial_zeroth_moment_is_c(hl, alt):
    """The initial populations (h^eq - H/2, or h^eq,alt) sum to c0 at every node."""
    phi0, c0 = WL.random_fields((1, 9, 11), seed=5)
    p = O.OracleParams(nx=11, ny=9, tau_g=0.7, tau_h=0.9, lam=4.0, D_l=0.15, D_s=0.03,
                       anti_trapping=1, h_lattice=hl, h_eq_alt=alt)
    o = O.Oracle(p, phi0, c0)
    assert np.abs(o.h.sum(0) - c0).max() < 1e-15


@pytest.mark.parametrize("hl,alt", VARIANTS)
def test_flat_interface_at_equilibrium_stays_put_with_variants(hl, alt):
    """tanh front with c = c^co(phi): mu = mu_eq, S_phi = 0, F = 0 up to the
    relaxation onto the discrete profile; the front must not move."""
    nx, W = 96, 4.0
    p = WL.recipe(nx, 4, D_l=0.1, D_s=0.1, W=W, counter_term=1, bc=(1, 0, 0))
    p.h_lattice, p.h_eq_alt = hl, alt
    x = np.arange(nx, dtype=float)
    phi0 = np.tile(WL.tanh_profile(x - 47.5, W), (4, 1))[None]
    o = O.Oracle(to_oracle(p), phi0, WL.blend(phi0, p.c_s_co, p.c_l_co))
    pos = lambda ph: (1 - ph[0].mean(0)).sum()
    o.step(200)
    x1 = pos(o.phi)
    o.step(2000)
    assert abs(pos(o.phi) - x1) < 0.05
    assert abs(x1 - pos(phi0)) < 0.05


def _stefan(nx, ny, nz, hl, alt):
    """The one-sided dissolution of Sec. 4.2 in lattice units (W = 10, D_l = 0.5,
    D_s = 0 with j_at, lambda* = 230, tau = 1.8), walls at both x ends."""
    p = O.OracleParams(nx=nx, ny=ny, nz=nz, bc=(1, 0, 0), tau_g=1.8, tau_h=1.8, W=10.0, lam=230.0,
                       D_l=0.5, D_s=0.0, c_s_co=0.6, c_l_co=0.5, mu_eq=0.4, counter_term=1,
                       anti_trapping=1, a_at=0.25, h_lattice=hl, h_eq_alt=alt)
    x = np.arange(nx) + 0.5 - nx / 2
    phi = WL.tanh_profile(x, 10.0)
    c = 0.5 * (0.4 + 0.6 + (0.4 - 0.6) * np.tanh(2 * x / 10.0))
    o = O.Oracle(p, np.broadcast_to(phi, (nz, ny, nx)), np.broadcast_to(c, (nz, ny, nx)))
    return x, o


@pytest.mark.parametrize("hl,alt", VARIANTS)
def test_one_sided_stefan_dissolution_with_variants(hl, alt):
    """The front follows x_i = 2 alpha sqrt(D_l t) (Eq. x_i_Ds0) and mu the profile of
    Eq. Analytical_muL_Ds0, to the paper's L2 level, with h on D2Q5 and/or the
    alternative equilibrium.  F = mu D_l grad phi + j_at is non-zero here, so a
    wrong factor on the flux in h^eq,alt (gamma instead of 1/xi_s^2, a missing
    factor 3) moves the front or the mu profile."""
    x, o = _stefan(1000, 4, 1, hl, alt)
    alpha = O.stefan_one_sided_root(0.4, 0.3, 0.1)
    n = 6000
    o.step(n)
    xi = -500 + (1 - o.phi[0].mean(0)).sum()
    xa = 2 * alpha * math.sqrt(0.5 * n)
    assert abs(xi - xa) < 0.05 * abs(xa) + 0.5
    mua = 0.3 + 0.1 * erfc(x / (2 * math.sqrt(0.5 * n))) / erfc(alpha)
    sel = (x > xi + 20) & (x < 300)
    mu = o.mu[0].mean(0)
    assert np.linalg.norm(mu[sel] - mua[sel]) / np.linalg.norm(mua[sel]) < 1.6e-3


def test_one_sided_stefan_dissolution_3d_d3q7():
    """The same front in 3-D with h on D3Q7 (a 1-D problem on a 1000 x 2 x 2 grid)."""
    x, o = _stefan(1000, 2, 2, 1, 0)
    alpha = O.stefan_one_sided_root(0.4, 0.3, 0.1)
    n = 6000
    o.step(n)
    xi = -500 + (1 - o.phi.mean((0, 1))).sum()
    xa = 2 * alpha * math.sqrt(0.5 * n)
    assert abs(xi - xa) < 0.05 * abs(xa) + 0.5
