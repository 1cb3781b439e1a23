"""Pins of the oracle's hand-written discrete adjoint.

The adjoint (Jacobian transpose) is checked against exact Jacobian-vector
products from the complex-step build of the forward oracle (tangent_cs.c):
<u, J v> = <J^T u, v> for random u, v, on one step and on the initialisation,
over both lattices, periodic and walled boxes, both phi equations and the
anti-trapping current, and with the model's options (h on D2Q5 / D3Q7, h^eq,alt,
unequal curvatures); and, on whole trajectories, against the complex-step
directional derivative and central finite differences (h = 1e-4, FP64).
A wrong sign, index or missed term in any adjoint operation breaks an equality.
"""
import numpy as np
import pytest

import oracle as O
from paper_2111_05960_gb300 import workloads as WL


def _params(shape, bc, ct, at):
    nz, ny, nx = shape
    return O.OracleParams(nx=nx, ny=ny, nz=nz, bc=bc, tau_g=0.7, tau_h=0.9, W=3.0, lam=4.0,
                          D_l=0.15, D_s=0.03, counter_term=ct, anti_trapping=at, a_at=0.2)


CASES = [((1, 7, 9), (0, 0, 0), 1, 1), ((1, 7, 9), (1, 0, 0), 0, 1), ((1, 6, 8), (1, 1, 0), 1, 0),
         ((4, 4, 5), (0, 0, 0), 1, 1), ((4, 5, 4), (1, 0, 1), 0, 1)]


@pytest.mark.parametrize("shape,bc,ct,at", CASES)
def test_step_adjoint_dot_product(shape, bc, ct, at):
    p = _params(shape, bc, ct, at)
    rng = np.random.default_rng(sum(shape) + 7 * ct + at)
    phi0, c0 = WL.random_fields(shape, seed=3 + ct)
    o = O.Oracle(p, phi0, c0).step(3)           # a generic state with non-zero dphi/dt
    st = (o.g.copy(), o.h.copy(), o.phi.copy(), o.c.copy())
    v = [rng.standard_normal(a.shape) for a in st]
    vp = rng.standard_normal(4)
    Jv = O.tangent_step(p, *st, *v, dparams=vp)
    u = [rng.standard_normal(a.shape) for a in st]
    ub = O.step_adjoint(p, *st, *u)
    lhs = sum(float(np.vdot(a, b)) for a, b in zip(u, Jv))
    rhs = sum(float(np.vdot(a, b)) for a, b in zip(ub[:4], v)) + float(np.dot(ub[4], vp))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0), (lhs, rhs)


@pytest.mark.parametrize("shape,bc,ct,at", CASES[:4])
def test_init_adjoint_dot_product(shape, bc, ct, at):
    p = _params(shape, bc, ct, at)
    rng = np.random.default_rng(11 + sum(shape))
    phi0, c0 = WL.random_fields(shape, seed=9)
    dphi, dc, vp = rng.standard_normal(shape), rng.standard_normal(shape), rng.standard_normal(4)
    dg, dh, dph, dcc = O.tangent_trajectory(p, phi0, c0, 0, dphi, dc, vp)
    q = dg.shape[0]
    gb, hb = rng.standard_normal(dg.shape), rng.standard_normal(dh.shape)
    phib, cb = rng.standard_normal(shape), rng.standard_normal(shape)
    a0, c0b, pb = O.init_adjoint(p, phi0, c0, gb, hb, phib, cb)
    lhs = float(np.vdot(gb, dg) + np.vdot(hb, dh) + np.vdot(phib, dph) + np.vdot(cb, dcc))
    rhs = float(np.vdot(a0, dphi) + np.vdot(c0b, dc) + np.dot(pb, vp))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0), (lhs, rhs)


def _slab_loss(phi, target):
    """L = sum_z (s_z - s*_z)^2, s_z = mean over x, y of (1 - phi)."""
    s = (1.0 - phi).mean(axis=(1, 2))
    return float(((s - target) ** 2).sum())


def _slab_loss_grad(phi, target):
    s = (1.0 - phi).mean(axis=(1, 2))
    per = phi.shape[1] * phi.shape[2]
    return np.broadcast_to((-2.0 * (s - target) / per)[:, None, None], phi.shape).copy()


@pytest.mark.parametrize("dim", [2, 3])
def test_trajectory_gradient_against_complex_step_and_fd(dim):
    shape = (5, 6, 7) if dim == 3 else (1, 9, 12)
    bc = (1, 0, 0)
    p = _params(shape, bc, 1, 1)
    phi0, c0 = WL.random_fields(shape, seed=21)
    target = np.linspace(0.3, 0.5, shape[0])
    n = 12
    o = O.Oracle(p, phi0, c0).step(n)
    phib = _slab_loss_grad(o.phi, target)
    a0, c0b, pb = O.trajectory_gradient(p, phi0, c0, n, phib, np.zeros(shape))
    rng = np.random.default_rng(5)
    d = rng.standard_normal(shape)
    d /= np.linalg.norm(d)
    # complex step: exact directional derivative of the loss along d (phi0) and each parameter
    _, _, dphi, _ = O.tangent_trajectory(p, phi0, c0, n, dphi0=d)
    cs = float(np.vdot(phib, dphi))
    assert abs(cs - float(np.vdot(a0, d))) <= 1e-11 * max(abs(cs), 1e-14)
    for j in range(4):
        e = np.zeros(4)
        e[j] = 1.0
        _, _, dphi, _ = O.tangent_trajectory(p, phi0, c0, n, dparams=e)
        cs = float(np.vdot(phib, dphi))
        assert abs(cs - pb[j]) <= 1e-10 * max(abs(cs), 1e-12), (O.PARAM_NAMES[j], cs, pb[j])
    # central finite differences, h = 1e-4 (second-order truncation)
    hfd = 1e-4
    lp = _slab_loss(O.Oracle(p, phi0 + hfd * d, c0).step(n).phi, target)
    lm = _slab_loss(O.Oracle(p, phi0 - hfd * d, c0).step(n).phi, target)
    fd = (lp - lm) / (2 * hfd)
    assert abs(fd - float(np.vdot(a0, d))) <= 1e-6 * max(abs(fd), 1e-10)
    for j, name in enumerate(O.PARAM_NAMES):
        pp, pm = _params(shape, bc, 1, 1), _params(shape, bc, 1, 1)
        setattr(pp, name, getattr(pp, name) + hfd)
        setattr(pm, name, getattr(pm, name) - hfd)
        fd = (_slab_loss(O.Oracle(pp, phi0, c0).step(n).phi, target) -
              _slab_loss(O.Oracle(pm, phi0, c0).step(n).phi, target)) / (2 * hfd)
        assert abs(fd - pb[j]) <= 1e-5 * max(abs(fd), 1e-8), (name, fd, pb[j])


# The options of the model (h on D2Q5 / D3Q7, h^eq,alt, unequal curvatures): the
# same dot-product identity for one step and for the initialisation.
VARIANT_CASES = [
    ((1, 7, 9), (0, 0, 0), dict(h_lattice=1)),
    ((1, 7, 9), (1, 0, 0), dict(h_eq_alt=1)),
    ((1, 6, 8), (1, 1, 0), dict(unequal_eps=1, eps_ratio=2.5)),
    ((4, 4, 5), (0, 0, 0), dict(h_lattice=1, h_eq_alt=1)),
    ((4, 5, 4), (1, 0, 1), dict(h_lattice=1, h_eq_alt=1, unequal_eps=1, eps_ratio=0.4)),
]


def _vparams(shape, bc, opts, ct=1):
    p = _params(shape, bc, ct, 1)
    for k, v in opts.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("shape,bc,opts", VARIANT_CASES)
@pytest.mark.parametrize("ct", [1, 0])
def test_step_adjoint_dot_product_variants(shape, bc, opts, ct):
    p = _vparams(shape, bc, opts, ct)
    rng = np.random.default_rng(sum(shape) + len(opts) + 5 * ct)
    phi0, c0 = WL.random_fields(shape, seed=13)
    o = O.Oracle(p, phi0, c0).step(3)
    st = (o.g.copy(), o.h.copy(), o.phi.copy(), o.c.copy())
    assert st[1].shape[0] == p.q_h
    v = [rng.standard_normal(a.shape) for a in st]
    vp = rng.standard_normal(4)
    Jv = O.tangent_step(p, *st, *v, dparams=vp)
    u = [rng.standard_normal(a.shape) for a in st]
    ub = O.step_adjoint(p, *st, *u)
    lhs = sum(float(np.vdot(a, b)) for a, b in zip(u, Jv))
    rhs = sum(float(np.vdot(a, b)) for a, b in zip(ub[:4], v)) + float(np.dot(ub[4], vp))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0), (lhs, rhs)


@pytest.mark.parametrize("shape,bc,opts", VARIANT_CASES)
def test_init_adjoint_dot_product_variants(shape, bc, opts):
    p = _vparams(shape, bc, opts)
    rng = np.random.default_rng(17 + sum(shape) + len(opts))
    phi0, c0 = WL.random_fields(shape, seed=19)
    dphi, dc, vp = rng.standard_normal(shape), rng.standard_normal(shape), rng.standard_normal(4)
    dg, dh, dph, dcc = O.tangent_trajectory(p, phi0, c0, 0, dphi, dc, vp)
    gb, hb = rng.standard_normal(dg.shape), rng.standard_normal(dh.shape)
    phib, cb = rng.standard_normal(shape), rng.standard_normal(shape)
    a0, c0b, pb = O.init_adjoint(p, phi0, c0, gb, hb, phib, cb)
    lhs = float(np.vdot(gb, dg) + np.vdot(hb, dh) + np.vdot(phib, dph) + np.vdot(cb, dcc))
    rhs = float(np.vdot(a0, dphi) + np.vdot(c0b, dc) + np.dot(pb, vp))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0), (lhs, rhs)


@pytest.mark.parametrize("dim", [2, 3])
def test_trajectory_gradient_variants_against_complex_step(dim):
    """Whole trajectory with every option on (h on the small lattice, h^eq,alt,
    eps_s / eps_l = 2): gradients of the slab loss with respect to phi0 and the
    four parameters equal the complex-step directional derivatives."""
    shape = (5, 6, 7) if dim == 3 else (1, 9, 12)
    p = _vparams(shape, (1, 0, 0), dict(h_lattice=1, h_eq_alt=1, unequal_eps=1, eps_ratio=2.0))
    phi0, c0 = WL.random_fields(shape, seed=23)
    target = np.linspace(0.3, 0.5, shape[0])
    n = 12
    o = O.Oracle(p, phi0, c0).step(n)
    phib = _slab_loss_grad(o.phi, target)
    a0, c0b, pb = O.trajectory_gradient(p, phi0, c0, n, phib, np.zeros(shape))
    d = np.random.default_rng(6).standard_normal(shape)
    d /= np.linalg.norm(d)
    _, _, dphi, _ = O.tangent_trajectory(p, phi0, c0, n, dphi0=d)
    cs = float(np.vdot(phib, dphi))
    assert abs(cs - float(np.vdot(a0, d))) <= 1e-11 * max(abs(cs), 1e-14)
    for j in range(4):
        e = np.zeros(4)
        e[j] = 1.0
        _, _, dphi, _ = O.tangent_trajectory(p, phi0, c0, n, dparams=e)
        cs = float(np.vdot(phib, dphi))
        assert abs(cs - pb[j]) <= 1e-10 * max(abs(cs), 1e-12), (O.PARAM_NAMES[j], cs, pb[j])
