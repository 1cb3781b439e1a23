"""The unstable path of the C ABI, driven by a run that really blows up.

The porous workload with a two-node interface (W = 2) diverges within ~150
steps in the FP64 oracle (tests/test_oracle_interface_width.py), and so does
the GPU.  Non-finite values fault nothing on the device; lbpf_mass sees them,
returns LBPF_EUNSTABLE and poisons the context, after which every call but
lbpf_last_error, lbpf_get_step and lbpf_destroy returns LBPF_ESTATE.
"""
import numpy as np
import pytest

from paper_2111_05960_gb300 import lbpf as L
from paper_2111_05960_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2111_05960_gb300 import build as B
    B.build()
    L.load()


@pytest.mark.parametrize("precision,mass_every", [("fp64", 0), ("fp32", 1)])
def test_diverging_run_reports_unstable_then_poisons_the_context(precision, mass_every):
    m, phi0, c0 = WL.porous_3d(n=32, W=2.0)
    sim = L.Simulation(m, phi0, c0, precision=precision, mass_every=mass_every)
    status, at = None, None
    for s in range(10, 601, 10):
        sim.step(10)
        try:
            sim.mass()
        except L.LbpfError as e:
            status, at = e.status, s
            break
    assert status == L.LBPF_EUNSTABLE, status
    assert at <= 400, at
    assert "unstable" in L.lbpf_last_error(sim.ctx)
    for call in (lambda: sim.step(1), sim.fields, sim.mass, sim.solute_mass, sim.populations):
        with pytest.raises(L.LbpfError) as ei:
            call()
        assert ei.value.status == L.LBPF_ESTATE
    assert sim.t == at                  # the step counter still answers
    sim.close()                         # and destroy succeeds


def test_the_same_medium_with_three_node_interfaces_stays_stable():
    m, phi0, c0 = WL.porous_3d(n=32, W=3.0)
    sim = L.Simulation(m, phi0, c0, precision="fp32", mass_every=1)
    for _ in range(6):
        sim.step(100)
        sim.mass()
    phi, c, _ = sim.fields()
    sim.close()
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(c))
    assert phi.min() > -1e-3 and phi.max() < 1.0 + 1e-3


def test_injected_allocation_failure_reports_enomem_and_leaks_nothing(monkeypatch):
    """LBPF_FAULT=alloc makes the library's device allocations fail on the host
    side (no GPU fault): lbpf_create returns LBPF_ENOMEM, hands back no context
    and leaves device memory as it found it; without the variable the same call
    succeeds."""
    import torch
    m, phi0, c0 = WL.porous_3d(n=16)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("LBPF_FAULT", "alloc")
    with pytest.raises(L.LbpfError) as ei:
        L.Simulation(m, phi0, c0, precision="fp32", mass_every=1)
    assert ei.value.status == L.LBPF_ENOMEM
    assert "injected allocation failure" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    monkeypatch.delenv("LBPF_FAULT")
    sim = L.Simulation(m, phi0, c0, precision="fp32", mass_every=1)
    sim.step(3)
    sim.close()


def test_non_finite_initial_field_is_reported_on_the_first_mass_call():
    """A NaN seeded into phi0 on the host propagates through the initialisation;
    the first lbpf_mass reports LBPF_EUNSTABLE."""
    m, phi0, c0 = WL.porous_3d(n=16)
    phi0 = phi0.copy()
    phi0[3, 4, 5] = float("nan")
    sim = L.Simulation(m, phi0, c0, precision="fp64")
    with pytest.raises(L.LbpfError) as ei:
        sim.mass()
    assert ei.value.status == L.LBPF_EUNSTABLE
    with pytest.raises(L.LbpfError) as ei:
        sim.step(1)
    assert ei.value.status == L.LBPF_ESTATE
    sim.close()
