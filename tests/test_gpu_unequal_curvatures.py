"""GPU parity of the unequal-curvature model (Sec. 2.3: Eq. Closure, Eq. SourceTerm,
Eq. Anti-Trapping_Quadratic; unequal_eps = 1, eps_ratio = eps_s / eps_l) against
the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2111_05960_gb300 import lbpf as L
from paper_2111_05960_gb300 import workloads as WL
from conftest import rel_err, to_oracle

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2111_05960_gb300 import build as B
    B.build()
    L.load()


def _case(shape, seed, **kw):
    nz, ny, nx = shape
    base = dict(tau_g=0.7, tau_h=0.9, W=3.0, lam=4.0, D_l=0.15, D_s=0.03,
                counter_term=1, anti_trapping=1, a_at=0.2, unequal_eps=1)
    base.update(kw)
    m = WL.ModelParams(nx=nx, ny=ny, nz=nz, **base)
    phi0, c0 = WL.random_fields(shape, seed=seed)
    return m, phi0, c0


CASES = [
    ((1, 37, 300), (1, 1, 0), 2.0, 1, {}),
    ((1, 21, 130), (0, 0, 0), 0.5, 0, {}),
    ((1, 17, 33), (1, 0, 0), 3.0, 1, dict(h_lattice=1, h_eq_alt=1)),
    ((20, 10, 40), (1, 0, 1), 2.0, 1, {}),
    ((9, 12, 70), (0, 0, 0), 0.25, 0, dict(h_lattice=1)),
]


@pytest.mark.parametrize("shape,bc,rho,ct,extra", CASES)
def test_fp64_matches_oracle(shape, bc, rho, ct, extra):
    """Fields (mu by the general closure) and every population plane after 100 steps
    within 1e-11 of the oracle."""
    m, phi0, c0 = _case(shape, seed=sum(shape) + int(4 * rho), bc=bc, counter_term=ct, eps_ratio=rho, **extra)
    sim = L.Simulation(m, phi0, c0, precision="fp64")
    sim.step(100)
    phi, c, mu = sim.fields()
    g, h = sim.populations()
    sim.close()
    o = O.Oracle(to_oracle(m), phi0, c0).step(100)
    errs = dict(phi=rel_err(phi, o.phi), c=rel_err(c, o.c), mu=rel_err(mu, o.mu),
                g=max(rel_err(g[k], o.g[k]) for k in range(g.shape[0])),
                h=max(rel_err(h[k], o.h[k]) for k in range(h.shape[0])))
    assert max(errs.values()) < FP64_TOL, errs


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("fp16dev", 2e-5)])
def test_reduced_precision_on_porous_medium(precision, tol):
    """48^3 porous crop with eps_s / eps_l = 2, 100 steps with the mass correction,
    against the FP64 oracle (eps_n = 1e-3)."""
    m, phi0, c0 = WL.porous_3d(n=48)
    m = dataclasses.replace(m, eps_n=1e-3, unequal_eps=1, eps_ratio=2.0)
    o = O.Oracle(to_oracle(m), phi0, c0).step(100)
    sim = L.Simulation(m, phi0, c0, precision=precision, mass_every=1)
    sim.step(100)
    phi, c, _ = sim.fields()
    sim.close()
    errs = dict(phi=rel_err(phi, o.phi), c=rel_err(c, o.c))
    assert max(errs.values()) < tol, errs


def test_fp32_stefan_front_with_unequal_curvatures():
    """The one-sided dissolution of Sec. 4.2 with eps_s / eps_l = 2 in FP32: after
    3000 steps the front (moved ~23 cells) within 0.05 cell of the FP64 oracle and
    the solute mass held."""
    nx, ny = 1000, 4
    m = WL.ModelParams(nx=nx, ny=ny, bc=(1, 0, 0), tau_g=1.8, tau_h=1.8, W=10.0, lam=230.0,
                       D_l=0.5, D_s=0.0, c_s_co=0.6, c_l_co=0.5, mu_eq=0.4, counter_term=1,
                       anti_trapping=1, a_at=0.25, unequal_eps=1, eps_ratio=2.0)
    x = np.arange(nx) + 0.5 - nx / 2
    phi0 = np.broadcast_to(WL.tanh_profile(x, 10.0), (1, ny, nx)).copy()
    c0 = np.broadcast_to(0.5 * (1.0 - 0.2 * np.tanh(2 * x / 10.0)), (1, ny, nx)).copy()
    o = O.Oracle(to_oracle(m), phi0, c0).step(3000)
    sim = L.Simulation(m, phi0, c0, precision="fp32", mass_every=1)
    m0, _ = sim.solute_mass()
    sim.step(3000)
    m1, _ = sim.solute_mass()
    phi, c, _ = sim.fields()
    sim.close()
    front = lambda ph: (1 - ph[0].mean(0)).sum()
    assert abs(front(o.phi) - front(phi0)) > 15
    assert abs(front(phi) - front(o.phi)) < 0.05
    assert abs(m1 - m0) / m0 < 1e-10
