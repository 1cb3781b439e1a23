"""The seeded synthetic inputs: each generator produces the workload its
description states (sizes, fractions, parameter ranges, seeds), so that the
benchmark and the parity tests run on the configurations they name.  Host only."""
import math

import numpy as np
import pytest

from paper_2111_05960_gb300 import workloads as WL


def test_grf_mask_fraction_and_seed():
    m = WL.grf_mask((32, 40, 48), corr=4.0, porosity=0.35, seed=0)
    assert m.shape == (32, 40, 48) and m.dtype == bool
    assert abs(m.mean() - 0.35) <= 1.0 / m.size
    assert np.array_equal(m, WL.grf_mask((32, 40, 48), corr=4.0, porosity=0.35, seed=0))
    assert not np.array_equal(m, WL.grf_mask((32, 40, 48), corr=4.0, porosity=0.35, seed=1))


def test_grf_mask_correlation_grows_with_corr():
    """Longer correlation length: neighbouring cells agree more often (a smoother medium)."""
    agree = []
    for corr in (2.0, 8.0):
        m = WL.grf_mask((64, 64, 64), corr=corr, porosity=0.35, seed=5)
        agree.append(np.mean(m == np.roll(m, 4, axis=2)))
    assert agree[1] > agree[0] + 0.1


def test_signed_distance_of_a_slab():
    """Pores x < 10 on a periodic 32-wide axis: the boundary sits half-way between
    the last pore and the first solid node, d > 0 in the pore."""
    m = np.zeros((1, 4, 32), dtype=bool)
    m[..., :10] = True
    d = WL.signed_distance(m, clip=8.0)
    x = np.arange(32)
    # distance to the nearest boundary, either at x = 9.5 or (periodically) at x = -0.5
    dist = np.minimum(np.abs(x - 9.5), np.minimum(np.abs(x + 0.5), np.abs(x - 31.5)))
    expect = np.where(x < 10, dist, -dist).clip(-8, 8)
    assert np.allclose(d[0, 0], expect)


def test_porous_3d_workload():
    p, phi, c = WL.porous_3d(n=32)
    assert phi.shape == (32, 32, 32) and c.shape == phi.shape
    assert 0.0 < phi.min() and phi.max() < 1.0
    assert np.allclose(c, (1 - phi) * 1.0 + phi * 0.1)
    assert (p.D_l, p.D_s, p.W, p.counter_term, p.anti_trapping) == (0.1, 0.0, 3.0, 1, 1)
    assert p.a_at == pytest.approx(0.25)
    assert p.tau_g == pytest.approx(3 * 1.2 * 0.1) and p.tau_h == p.tau_g
    assert p.lam == pytest.approx(WL.lambda_star(0.1, 0.12, 0.5))
    # liquid fraction near the porosity (the tanh smoothing is symmetric about d = 0)
    assert abs(phi.mean() - 0.35) < 0.03


def test_differentiable_3d_target():
    p, phi, c, target = WL.differentiable_3d(n=32)
    s0 = (1 - phi).mean(axis=(1, 2))
    u = np.random.Generator(np.random.PCG64(3)).uniform(0.0, 1.0, 32)
    assert np.allclose(target, s0 - 0.05 * u)
    assert p.eps_n == 1e-3
    assert abs(phi.mean() - 0.4) < 0.03


def test_planar_and_disc_workloads():
    p, phi, c = WL.planar_1d()
    assert phi.shape == (1, 8, 512) and tuple(p.bc) == (1, 0, 0)
    assert (p.W, p.D_l, p.D_s) == (2.5, 0.1, 0.1)
    assert abs((1 - phi[0, 0]).sum() - 128.0) < 1e-9          # solid for x < 127.5 (+ 1/2 cell)
    assert c[0, 0, 0] == pytest.approx(1.0) and c[0, 0, -1] == pytest.approx(0.2)
    p, phi, c = WL.disc_2d()
    assert phi.shape == (1, 512, 512) and (p.W, p.D_l, p.D_s) == (3.0, 0.05, 0.05)
    assert math.sqrt((1 - phi).sum() / math.pi) == pytest.approx(60.0, abs=0.05)
    assert np.allclose(c, (1 - phi) * p.c_s_co + phi * p.c_l_co)   # on the coexistence line


def test_batch_sweep_workload():
    """The 384-instance sweep of the benchmark: sides in 64..768 (83,070,399 nodes for
    seed 1), D_l in [0.02, 0.2], M_phi / D_l in [0.5, 5], counter term on for about
    half, solid discs in every instance."""
    inst = WL.batch_2d(count=384, seed=1)
    assert len(inst) == 384
    sides = np.array([x.params.nx for x in inst])
    assert sides.min() >= 64 and sides.max() <= 768
    assert all(x.params.nx == x.params.ny and x.params.nz == 1 for x in inst)
    assert sum(x.params.nodes for x in inst) == 83_070_399
    D = np.array([x.params.D_l for x in inst])
    ratio = np.array([x.params.M_phi / x.params.D_l for x in inst])
    assert D.min() >= 0.02 and D.max() <= 0.2
    assert ratio.min() >= 0.5 - 1e-12 and ratio.max() <= 5.0 + 1e-12
    ct = np.array([x.params.counter_term for x in inst])
    assert 150 < ct.sum() < 234
    assert all((x.phi < 0.5).any() for x in inst)


def test_paper_e4_workload():
    """Sec. 5 on a synthetic slice: 1024^2, W = 0.02 / dx, lambda* = 230, zero-flux walls,
    tau = 3 M_phi dt / dx^2 with M_phi = 1.2 and dt = 5e-7, D_l = dt / dx^2, D_s = 0,
    discontinuous start (phi 0/1, c 0.6/0.4), pore fraction 0.35."""
    p, phi, c = WL.paper_e4_2d()
    f = 5e-7 * 1024 ** 2
    assert phi.shape == (1, 1024, 1024)
    assert p.W == pytest.approx(0.02 * 1024) and p.lam == 230.0
    assert p.tau_g == pytest.approx(3 * 1.2 * f) and p.D_l == pytest.approx(f) and p.D_s == 0.0
    assert tuple(p.bc) == (1, 1, 0) and p.anti_trapping == 1 and p.a_at == 0.25
    assert set(np.unique(phi)) == {0.0, 1.0}
    assert np.array_equal(c, np.where(phi > 0.5, 0.4, 0.6))
    assert abs(phi.mean() - 0.35) <= 1.0 / phi.size
