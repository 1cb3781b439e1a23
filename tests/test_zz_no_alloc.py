"""lbpf_mass_noalloc: the allocation-free field sums, for callers that cannot call
cudaMalloc (host callbacks, graph nodes, runtimes that own all device memory).

It must agree with lbpf_mass, the entry point that allocates its scratch per
context, on the same fields, on two calls in a row (the second call reuses the
shared scratch array the first one left behind).  This file is collected last
on purpose, and it passes alone in a fresh process or after the other tests.
"""
import numpy as np
import pytest

from paper_2111_05960_gb300 import lbpf as L
from paper_2111_05960_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

MASS_TOL = 1e-13   # the relative tolerance of the FP64 mass tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2111_05960_gb300 import build as B
    B.build()
    L.load()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_sums_match_lbpf_mass_on_two_calls(precision):
    import torch
    m = WL.recipe(96, 70, D_l=0.1, D_s=0.02, W=3.0, counter_term=1, bc=(1, 0, 0))
    phi0, c0 = WL.random_fields(m.shape, seed=21)
    sim = L.Simulation(m, phi0, c0, precision=precision)
    sim.step(30)
    mc, mphi = sim.mass()

    # the context's fields, exported in FP64 to caller-owned device memory
    phi = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    c = torch.empty(m.shape, dtype=torch.float64, device="cuda")
    L.lbpf_get_fields(sim.ctx, phi, c, None, 1)
    sim.close()
    if precision == "fp32":
        # the FP32 context holds FP32 fields; the FP64 export of them is exact
        phi, c = phi.float().contiguous(), c.float().contiguous()
    prec = L.LBPF_FP64 if precision == "fp64" else L.LBPF_FP32

    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    # two calls in a row on the legacy default stream, then two on a caller's
    # stream handed over as a torch.cuda.Stream
    for stream in (None, None, side, side):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        L.lbpf_mass_noalloc(c, phi, c.numel(), prec, out, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - mc) <= MASS_TOL * abs(mc)
        assert abs(got[1] - mphi) <= MASS_TOL * abs(mphi)
        assert got[2] == 0.0


def test_noalloc_rejects_oversize_and_bad_arguments():
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    a = torch.zeros(8, dtype=torch.float64, device="cuda")
    # the C entry point itself rejects n above its maximum before touching any
    # buffer (called raw: the binding would refuse n > numel first)
    st = L.load().lbpf_mass_noalloc(a.data_ptr(), a.data_ptr(), L.NOALLOC_MAX_ELEMENTS + 1, L.LBPF_FP64,
                                    out.data_ptr(), None)
    assert st == L.LBPF_EINVAL and "no-alloc maximum" in L.lbpf_last_error(None)
    with pytest.raises(L.LbpfError):
        L.lbpf_mass_noalloc(a, a, 8, L.LBPF_FP32_FP16DEV, out)
    with pytest.raises(L.LbpfError):
        L.lbpf_mass_noalloc(a, a, -1, L.LBPF_FP64, out)
    # n = 0 writes zero sums
    out.fill_(1.0)
    L.lbpf_mass_noalloc(a, a, 0, L.LBPF_FP64, out)
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0.0)


def test_noalloc_binding_checks_its_arguments():
    """The binding refuses buffers the kernels would misread: host tensors, a
    dtype other than the precision's, fewer than n elements, a short output."""
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    a64 = torch.zeros(8, dtype=torch.float64, device="cuda")
    a32 = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        L.lbpf_mass_noalloc(a32, a32, 8, L.LBPF_FP64, out)
    with pytest.raises(ValueError):
        L.lbpf_mass_noalloc(a64.cpu(), a64, 8, L.LBPF_FP64, out)
    with pytest.raises(ValueError):
        L.lbpf_mass_noalloc(a64, a64, 9, L.LBPF_FP64, out)
    with pytest.raises(ValueError):
        L.lbpf_mass_noalloc(a64, a64, 8, L.LBPF_FP64, out[:2])
    L.lbpf_mass_noalloc(a32, a32, 8, L.LBPF_FP32, out)
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0.0)
