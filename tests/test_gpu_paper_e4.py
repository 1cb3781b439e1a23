"""The dissolution experiment of Sec. 5 on a synthetic porous slice (1024^2,
W ~ 20 nodes, lambda* = 230, D_s = 0, anti-trapping, 10^4 steps), with and
without the counter term: the paper's qualitative findings, and FP64 parity
with the oracle over the first steps from the discontinuous start."""
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


def _measures(phi, c):
    from scipy import ndimage
    ph, cc = phi[0], c[0]
    solid, liquid = ph < 0.05, ph > 0.95
    return dict(pores=ndimage.label(ph > 0.5)[1], c_solid_mean=float(cc[solid].mean()),
                c_solid_std=float(cc[solid].std()), c_liquid_mean=float(cc[liquid].mean()),
                interface=int(((ph > 0.1) & (ph < 0.9)).sum()))


@pytest.fixture(scope="module")
def runs():
    pytest.importorskip("scipy")
    out = {}
    for ct in (1, 0):
        m, phi0, c0 = WL.paper_e4_2d(counter_term=ct)
        sim = L.Simulation(m, phi0, c0, precision="fp32", mass_every=1)
        m0, target = sim.solute_mass()
        sim.step(10000)
        phi, c, _ = sim.fields()
        m1, _ = sim.solute_mass()
        sim.close()
        out[ct] = dict(_measures(phi, c), drift=abs(m1 - target) / target, start=_measures(phi0, c0))
    return out


def test_counter_term_keeps_the_small_pores(runs):
    # without the counter term curvature-driven motion closes small pores
    # (71 at the start: 21 remain with it, 7 without)
    assert runs[1]["pores"] >= 2 * runs[0]["pores"], runs
    assert runs[0]["pores"] < runs[0]["start"]["pores"]


def test_counter_term_keeps_the_solid_at_coexistence(runs):
    # with the counter term the solid stays at c_s^co = 0.6; without it the solid
    # composition becomes heterogeneous (std 0.004 against 0.017)
    assert abs(runs[1]["c_solid_mean"] - 0.6) < 0.005
    assert runs[0]["c_solid_std"] > 3.0 * runs[1]["c_solid_std"], runs


def test_counter_term_leaves_an_irregular_interface(runs):
    # the interface keeps the medium's small-scale shape with the counter term
    # and is smoothed by curvature without it
    assert runs[1]["interface"] > 1.5 * runs[0]["interface"], runs


def test_liquid_reaches_coexistence_and_mass_is_held(runs):
    for ct in (1, 0):
        assert abs(runs[ct]["c_liquid_mean"] - 0.5) < 0.01, runs[ct]
        assert runs[ct]["drift"] < 1e-9, runs[ct]


@pytest.mark.parametrize("ct", [1, 0])
@pytest.mark.parametrize("eps_n,tol", [(1e-3, 1e-11), (1e-12, 1e-8)])
def test_fp64_matches_oracle_from_the_discontinuous_start(ct, eps_n, tol):
    """From the discontinuous start every node begins flat (phi = 0 or 1); with
    eps_n = 1e-12 the unit normal of the nodes that stay nearly flat turns with
    rounding-level changes of grad phi, so FMA contraction on the GPU (absent
    in the oracle) shows up after 40 steps at a few such nodes (measured 6e-10
    with the counter term, 3.5e-9 in c without it, where n enters through the
    anti-trapping current).  With eps_n = 1e-3 the step is well conditioned and
    the usual 1e-11 holds."""
    import dataclasses
    m, phi0, c0 = WL.paper_e4_2d(counter_term=ct)
    m = dataclasses.replace(m, eps_n=eps_n)
    sim = L.Simulation(m, phi0, c0, precision="fp64")
    sim.step(40)
    phi, c, _ = sim.fields()
    sim.close()
    o = O.Oracle(to_oracle(m), phi0, c0).step(40)
    errs = dict(phi=rel_err(phi, o.phi), c=rel_err(c, o.c))
    assert max(errs.values()) < tol, errs
