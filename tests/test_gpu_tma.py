"""The step kernels' opt-in tensor-map pulls (LBPF_TMA=1; FP32 storage, D3Q19,
periodic domains): the copy engine brings each plane's rows of the links with
e_x = 0 into shared memory (the other links are loaded by the threads), and
the threads on the grid's y faces reload the rows that wrap.  The arithmetic
is that of the load path, so both must give the same bits; one case is also
held against the FP64 oracle."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2111_05960_gb300 import lbpf as L
from paper_2111_05960_gb300 import workloads as WL
from conftest import rel_err, to_oracle

pytestmark = pytest.mark.gpu


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


def _run(m, phi0, c0, steps, tma, mass_every=1):
    old = os.environ.get("LBPF_TMA")
    if tma:
        os.environ["LBPF_TMA"] = "1"
    else:
        os.environ.pop("LBPF_TMA", None)
    try:
        import torch
        stream = torch.cuda.Stream()
        sim = L.Simulation(m, phi0, c0, precision="fp32", stream=stream.cuda_stream, lattice=L.LBPF_D3Q19,
                           mass_every=mass_every)
    finally:
        if old is None:
            os.environ.pop("LBPF_TMA", None)
        else:
            os.environ["LBPF_TMA"] = old
    path = L.lbpf_pull_path(sim.ctx)
    # a single step, a graph-replayed run and a single step again
    sim.step(1)
    sim.step(steps - 2)
    sim.step(1)
    mc, mphi = sim.mass()
    phi, c, mu = sim.fields()
    g, h = sim.populations()
    sim.close()
    return path, dict(phi=phi, c=c, mu=mu, g=g, h=h, mass=np.array([mc, mphi]))


# (nz, ny, nx): full and partial 32 x 4 tiles, z-chunks with a ragged tail,
# x and y faces on every side
@pytest.mark.parametrize("shape,kw", [
    ((24, 40, 64), {}),
    ((9, 42, 72), dict(counter_term=0)),
    ((37, 8, 40), dict(h_lattice=1)),
    ((12, 13, 96), dict(h_eq_alt=1, anti_trapping=0)),
    ((5, 6, 44), dict(h_lattice=1, h_eq_alt=1)),
])
def test_tensor_map_pulls_match_load_pulls_bitwise(shape, kw):
    m, phi0, c0 = _case(shape, seed=sum(shape), **kw)
    p_tma, a = _run(m, phi0, c0, 41, tma=True)
    p_ld, b = _run(m, phi0, c0, 41, tma=False)
    assert p_tma == 1 and p_ld == 0
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_tensor_map_pulls_against_fp64_oracle():
    """FP32 with tensor-map pulls after 100 steps within the FP32 bound of the
    other FP32 parity tests (2e-5 of max |oracle|)."""
    m, phi0, c0 = _case((16, 40, 64), seed=5)
    path, a = _run(m, phi0, c0, 100, tma=True, mass_every=1)
    assert path == 1
    o = O.Oracle(to_oracle(m), phi0, c0).step(100)
    assert rel_err(a["phi"], o.phi) < 2e-5
    assert rel_err(a["c"], o.c) < 2e-5


@pytest.mark.parametrize("what", ["walls", "fp64", "narrow", "odd_nx", "default"])
def test_contexts_outside_the_tensor_map_path_pull_with_loads(what):
    kw, prec, shape = {}, "fp32", (8, 8, 64)
    if what == "walls":
        kw = dict(bc=(0, 1, 0))
    elif what == "fp64":
        prec = "fp64"
    elif what == "narrow":
        shape = (8, 8, 28)
    elif what == "odd_nx":
        shape = (8, 8, 66)
    m, phi0, c0 = _case(shape, seed=1, **kw)
    if what == "default":         # without LBPF_TMA=1 every context pulls with loads
        sim = L.Simulation(m, phi0, c0, precision=prec, lattice=L.LBPF_D3Q19)
        assert L.lbpf_pull_path(sim.ctx) == 0
        sim.close()
        return
    os.environ["LBPF_TMA"] = "1"
    try:
        sim = L.Simulation(m, phi0, c0, precision=prec, lattice=L.LBPF_D3Q19)
    finally:
        os.environ.pop("LBPF_TMA", None)
    assert L.lbpf_pull_path(sim.ctx) == 0
    sim.step(3)
    sim.close()
