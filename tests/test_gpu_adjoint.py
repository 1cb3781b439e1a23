"""The GPU discrete adjoint (lbpf_adjoint_step) against the oracle's FP64 adjoint,
against central finite differences of the GPU forward, and through the torch
autograd Function.

Metric for fields: max_x |gpu - oracle| / max_x |oracle| (infinity norm).  FP64
must agree with the oracle to 1e-11; the FP32 adjoint (FP32 forward replay and
FP32 field adjoints, FP64 parameter sums) states its error against the FP64
oracle: 2e-4, from ~1e-7 rounding per operation compounded over the steps.
"""
import numpy as np
import pytest

import oracle as O
from paper_2111_05960_gb300 import lbpf as L
from paper_2111_05960_gb300 import workloads as WL
from conftest import rel_err, to_oracle

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 2e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2111_05960_gb300 import build as B
    B.build()
    L.load()


def _case(shape, seed, **kw):
    nz, ny, nx = shape
    base = dict(tau_g=0.7, tau_h=0.9, W=3.0, lam=4.0, D_l=0.15, D_s=0.03,
                counter_term=1, anti_trapping=1, a_at=0.2)
    base.update(kw)
    m = WL.ModelParams(nx=nx, ny=ny, nz=nz, **base)
    phi0, c0 = WL.random_fields(shape, seed=seed)
    return m, phi0, c0


def _seeds(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape), rng.standard_normal(shape)


def _gpu(m, phi0, c0, T, K, seeds, precision="fp64", mass_every=0):
    sim = L.Simulation(m, phi0, c0, precision=precision, checkpoint_every=K, mass_every=mass_every)
    sim.step(T)
    out = sim.adjoint(*seeds)
    sim.close()
    return out


def _param_err(pv, po):
    po = np.asarray(po)
    return float(np.max(np.abs(pv[:4] - po)) / max(np.max(np.abs(po)), 1e-300))


CASES = [
    ((1, 21, 70), (0, 0, 0), 1, 1),
    ((1, 17, 33), (1, 1, 0), 0, 1),
    ((1, 9, 40), (1, 0, 0), 1, 0),
    ((1, 1, 36), (0, 0, 0), 1, 1),
    ((6, 10, 33), (1, 0, 1), 0, 1),
    ((5, 11, 37), (0, 0, 0), 1, 1),
    ((3, 4, 9), (1, 1, 1), 1, 1),
]


@pytest.mark.parametrize("shape,bc,ct,at", CASES)
def test_fp64_adjoint_matches_oracle(shape, bc, ct, at):
    m, phi0, c0 = _case(shape, seed=5 * sum(shape) + ct, bc=bc, counter_term=ct, anti_trapping=at)
    T, K = 12, 5                         # segments [0, 5), [5, 10), [10, 12)
    seeds = _seeds(shape, sum(shape))
    d0, c0b, pv = _gpu(m, phi0, c0, T, K, seeds)
    od0, oc0, op = O.trajectory_gradient(to_oracle(m), phi0, c0, T, *seeds)
    errs = dict(phi0=rel_err(d0, od0), c0=rel_err(c0b, oc0), params=_param_err(pv, op))
    assert max(errs.values()) < FP64_TOL, errs
    if not at:
        assert pv[4] == 0.0


@pytest.mark.parametrize("T", [0, 1, 4])
def test_short_trajectories_match_oracle(T):
    m, phi0, c0 = _case((1, 13, 40), seed=31, bc=(1, 0, 0))
    seeds = _seeds(m.shape, 4)
    d0, c0b, pv = _gpu(m, phi0, c0, T, 3, seeds)
    od0, oc0, op = O.trajectory_gradient(to_oracle(m), phi0, c0, T, *seeds)
    assert rel_err(d0, od0) < FP64_TOL and rel_err(c0b, oc0) < FP64_TOL
    assert _param_err(pv, op) < FP64_TOL or np.max(np.abs(op)) == 0.0


def test_checkpoint_interval_does_not_change_the_result():
    # the replay is bitwise the forward run and the sweep the same kernels in
    # the same order, so every interval gives the same bits
    m, phi0, c0 = _case((1, 19, 45), seed=8, bc=(0, 1, 0))
    seeds = _seeds(m.shape, 9)
    ref = _gpu(m, phi0, c0, 9, 9, seeds)
    for K in (1, 2, 4, 50):
        out = _gpu(m, phi0, c0, 9, K, seeds)
        for a, b in zip(out, ref):
            assert np.array_equal(a, b), K


def test_forward_state_is_unchanged_and_can_continue():
    m, phi0, c0 = _case((4, 9, 34), seed=12, bc=(1, 0, 0))
    seeds = _seeds(m.shape, 13)
    sim = L.Simulation(m, phi0, c0, precision="fp64", checkpoint_every=3)
    sim.step(5)
    before = sim.fields() + sim.populations()
    sim.adjoint(*seeds)
    after = sim.fields() + sim.populations()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    sim.step(4)                                         # 9 steps in all, still recorded
    d0, c0b, pv = sim.adjoint(*seeds)
    sim.close()
    od0, oc0, op = O.trajectory_gradient(to_oracle(m), phi0, c0, 9, *seeds)
    assert max(rel_err(d0, od0), rel_err(c0b, oc0), _param_err(pv, op)) < FP64_TOL


def _slab_loss(phi, target):
    return WL.slab_loss(phi, target)


def _final_loss(m, phi0, c0, T, target):
    sim = L.Simulation(m, phi0, c0, precision="fp64")
    sim.step(T)
    phi, _, _ = sim.fields()
    sim.close()
    return _slab_loss(phi, target)[0]


def _richardson(f, h):
    """Central difference with its h^2 error term removed: (4 D(h/2) - D(h)) / 3."""
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3, d1


def _porous(n, **kw):
    import dataclasses
    m, phi0, c0, target = WL.differentiable_3d(n)
    return dataclasses.replace(m, **kw), phi0, c0, target


# Central differences (h = 1e-4, FP64 forward on the GPU) need a step that is
# smooth at the scale h: the differentiable workload (porous medium, slab
# solid-fraction loss, eps_n = 1e-3).  With eps_n = 1e-12 the exact Jacobian
# is ~ phi(1 - phi)/eps_n where grad phi vanishes inside thin necks (n turns
# freely there): the adjoint is then exact (it matches the oracle) but no
# finite difference can follow it.
@pytest.mark.parametrize("auto_a", [False, True])
def test_parameter_gradients_match_central_differences(auto_a):
    import dataclasses
    m, phi0, c0, target = _porous(20, D_s=0.02, anti_trapping=1, a_at=-1.0 if auto_a else 0.2)
    T = 30
    sim = L.Simulation(m, phi0, c0, precision="fp64", checkpoint_every=7)
    sim.step(T)
    _, seed = _slab_loss(sim.fields()[0], target)
    _, _, pv = sim.adjoint(seed, None)
    sim.close()
    for name in ("D_l", "tau_g", "tau_h", "lam", "D_s"):
        j = L.ADJ_PARAM_NAMES.index(name)
        x = getattr(m, name)
        f = lambda d: _final_loss(dataclasses.replace(m, **{name: x + d}), phi0, c0, T, target)
        rich, fd = _richardson(f, 1e-4)
        assert abs(pv[j] - rich) <= 1e-6 * abs(rich) + 1e-12, (name, pv[j], rich, fd)


def test_initial_field_gradient_matches_central_differences():
    m, phi0, c0, target = _porous(20)
    T = 30
    rng = np.random.default_rng(43)
    dphi = rng.standard_normal(m.shape) * phi0 * (1 - phi0)     # on the interfaces
    dc = rng.standard_normal(m.shape) * 0.1
    sim = L.Simulation(m, phi0, c0, precision="fp64", checkpoint_every=8)
    sim.step(T)
    _, seed = _slab_loss(sim.fields()[0], target)
    d0, c0b, _ = sim.adjoint(seed, None)
    sim.close()
    rich, fd = _richardson(lambda d: _final_loss(m, phi0 + d * dphi, c0 + d * dc, T, target), 1e-4)
    ad = float(np.vdot(d0, dphi) + np.vdot(c0b, dc))
    assert abs(ad - rich) <= 1e-6 * abs(rich), (ad, rich, fd)


@pytest.mark.parametrize("mass_every", [0, 1])
@pytest.mark.parametrize("shape,bc", [((1, 24, 64), (1, 0, 0)), ((6, 12, 40), (0, 0, 1))])
def test_fp32_adjoint_close_to_fp64_oracle(shape, bc, mass_every):
    m, phi0, c0 = _case(shape, seed=sum(shape), bc=bc)
    seeds = _seeds(shape, 3 + mass_every)
    T = 12
    d0, c0b, pv = _gpu(m, phi0, c0, T, 5, seeds, precision="fp32", mass_every=mass_every)
    od0, oc0, op = O.trajectory_gradient(to_oracle(m), phi0, c0, T, *seeds)
    errs = dict(phi0=rel_err(d0, od0), c0=rel_err(c0b, oc0), params=_param_err(pv, op))
    assert max(errs.values()) < FP32_TOL, errs


def test_full_size_128_cubed_directional_derivative():
    # the differentiable 3-D workload at its full size (128^3 porous medium,
    # porosity 0.4) and loss: the FP64 adjoint against central differences of the
    # FP64 forward along three random unit directions of phi0 and along D_l, and
    # the FP32 adjoint (with the mass correction) against the FP64 one
    import dataclasses
    m, phi0, c0, target = WL.differentiable_3d(128)
    T = 20
    res = {}
    for prec, me in (("fp64", 0), ("fp32", 1)):
        sim = L.Simulation(m, phi0, c0, precision=prec, checkpoint_every=8, mass_every=me)
        sim.step(T)
        _, seed = _slab_loss(sim.fields()[0], target)
        res[prec] = sim.adjoint(seed, None)
        sim.close()
    d64, _, p64 = res["fp64"]
    rng = np.random.default_rng(7)
    for _ in range(3):
        dphi = rng.standard_normal(m.shape)
        dphi /= np.linalg.norm(dphi)
        fd = (_final_loss(m, phi0 + 1e-4 * dphi, c0, T, target)
              - _final_loss(m, phi0 - 1e-4 * dphi, c0, T, target)) / 2e-4
        ad = float(np.vdot(d64, dphi))
        assert abs(ad - fd) <= 1e-5 * abs(fd), (ad, fd)
    rich, fd = _richardson(lambda d: _final_loss(dataclasses.replace(m, D_l=m.D_l + d), phi0, c0, T, target), 1e-4)
    assert abs(p64[0] - rich) <= 1e-6 * abs(rich), (p64[0], rich, fd)
    d32, _, p32 = res["fp32"]
    assert rel_err(d32, d64) < 1e-3
    assert np.max(np.abs(p32[:4] - p64[:4]) / np.maximum(np.abs(p64[:4]), 1e-12)) < 1e-3


def test_adjoint_needs_recording():
    m, phi0, c0 = _case((1, 8, 40), seed=1)
    sim = L.Simulation(m, phi0, c0, precision="fp64")
    sim.step(2)
    with pytest.raises(L.LbpfError) as ei:
        sim.adjoint(*_seeds(m.shape, 1))
    sim.close()
    assert ei.value.status == L.LBPF_EUNSUPPORTED


@pytest.mark.parametrize("theta_device", ["cpu", "cuda:0"])
def test_autograd_function_solid_fraction_loss(theta_device):
    import torch
    from paper_2111_05960_gb300 import autograd as AG
    m, phi0, c0, target_np = _porous(16)
    dev = torch.device("cuda:0")
    target = torch.tensor(target_np, dtype=torch.float64, device=dev)
    c0_t = torch.tensor(c0, device=dev)

    def loss_of(phi0_t, theta_t):
        phi, _ = AG.trajectory(phi0_t, c0_t, theta_t, m, 24, "fp64", 5)
        s = 1.0 - phi.mean(dim=(1, 2))                  # solid fraction per z-slab
        return ((s - target) ** 2).sum()

    phi0_t = torch.tensor(phi0, device=dev, requires_grad=True)
    theta = torch.tensor([m.D_l, m.tau_g, m.tau_h, m.lam], dtype=torch.float64, device=theta_device,
                         requires_grad=True)
    loss = loss_of(phi0_t, theta)
    loss.backward()
    assert theta.grad.device == theta.device
    base = theta.detach()
    for i in range(4):
        def f(d, i=i):
            t = base.clone()
            t[i] += d
            with torch.no_grad():
                return loss_of(phi0_t.detach(), t).item()
        rich, fd = _richardson(f, 1e-4)
        assert abs(theta.grad[i].item() - rich) <= 1e-6 * abs(rich), (i, theta.grad[i].item(), rich, fd)
    p0 = torch.tensor(phi0, device=dev)
    dphi = torch.randn(m.shape, dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(5))
    dphi /= dphi.norm()

    def g(d):
        with torch.no_grad():
            return loss_of(p0 + d * dphi, base).item()
    rich, fd = _richardson(g, 1e-4)
    ad = float((phi0_t.grad * dphi).sum())
    assert abs(ad - rich) <= 1e-6 * abs(rich), (ad, rich, fd)


def test_differentiable_workload_as_configured_2000_steps():
    """The differentiable 3-D workload as configured: 128^3 porous medium
    (porosity 0.4), 2000 FP32 steps with the FP64 mass correction, a checkpoint
    every 100 steps, the slab solid-fraction loss.  The same trajectory in FP64
    gives the reference: its adjoint is pinned to the oracle's FP64 discrete
    adjoint by the tests above, and here it is checked against central
    differences (h = 1e-4, Richardson-extrapolated) of the FP64 GPU forward over
    the same 2000 steps, for dL/dD_l, dL/dM_phi = 3 dL/dtau_g (tau_h held) and
    one unit direction of phi0.  The FP32 adjoint is then compared with the FP64
    one."""
    import dataclasses
    m, phi0, c0, target = WL.differentiable_3d(128)
    T, K = 2000, 100
    res = {}
    for prec, me in (("fp32", 1), ("fp64", 0)):
        sim = L.Simulation(m, phi0, c0, precision=prec, checkpoint_every=K, mass_every=me)
        sim.step(T)
        loss, seed = _slab_loss(sim.fields()[0], target)
        res[prec] = (loss,) + tuple(sim.adjoint(seed, None))
        sim.close()
    loss64, d64, _, p64 = res["fp64"]
    loss32, d32, _, p32 = res["fp32"]
    h = 1e-4
    rich_D, fd_D = _richardson(lambda d: _final_loss(dataclasses.replace(m, D_l=m.D_l + d), phi0, c0, T, target), h)
    rich_M, fd_M = _richardson(
        lambda d: _final_loss(dataclasses.replace(m, tau_g=m.tau_g + 3.0 * d), phi0, c0, T, target), h)
    dphi = np.random.default_rng(11).standard_normal(m.shape)
    dphi /= np.linalg.norm(dphi)
    rich_p, fd_p = _richardson(lambda d: _final_loss(m, phi0 + d * dphi, c0, T, target), h)
    ad_D, ad_M, ad_p = p64[0], 3.0 * p64[1], float(np.vdot(d64, dphi))
    print("loss fp64 %.10e fp32 %.10e" % (loss64, loss32))
    print("dL/dD_l   adjoint %.10e  richardson %.10e  central %.10e" % (ad_D, rich_D, fd_D))
    print("dL/dM_phi adjoint %.10e  richardson %.10e  central %.10e" % (ad_M, rich_M, fd_M))
    print("dphi0     adjoint %.10e  richardson %.10e  central %.10e" % (ad_p, rich_p, fd_p))
    assert abs(ad_D - rich_D) <= 1e-5 * abs(rich_D), (ad_D, rich_D, fd_D)
    assert abs(ad_M - rich_M) <= 1e-5 * abs(rich_M), (ad_M, rich_M, fd_M)
    assert abs(ad_p - rich_p) <= 1e-5 * abs(rich_p), (ad_p, rich_p, fd_p)
    e_field = rel_err(d32, d64)
    e_par = np.max(np.abs(p32[:4] - p64[:4]) / np.maximum(np.abs(p64[:4]), 1e-300))
    print("fp32 vs fp64 adjoint: dphi0 %.3e  params %.3e  loss %.3e" % (e_field, e_par, abs(loss32 - loss64) / loss64))
    assert e_field < 1e-2 and e_par < 1e-2, (e_field, e_par)
