"""Batched 2-D instances (lbpf_create_batch) and CUDA-graph replay of the step."""
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


def _mixed_instances():
    """Uneven sizes (ragged tiles, 1-wide and 2-wide axes), walls and periodic,
    both phi equations, anti-trapping on and off, different diffusivities."""
    specs = [((21, 70), (0, 0, 0), 1, 1, 0.15, 0.03), ((17, 33), (1, 1, 0), 0, 1, 0.1, 0.0),
             ((8, 64), (0, 1, 0), 1, 0, 0.05, 0.05), ((40, 40), (1, 0, 0), 0, 0, 0.2, 0.1),
             ((1, 40), (0, 0, 0), 1, 1, 0.12, 0.02), ((30, 100), (0, 0, 0), 1, 1, 0.02, 0.0)]
    out = []
    for j, ((ny, nx), bc, ct, at, Dl, Ds) in enumerate(specs):
        m = WL.ModelParams(nx=nx, ny=ny, bc=bc, tau_g=0.5 + 0.1 * j, tau_h=0.6 + 0.05 * j, W=3.0, lam=2.0 + j,
                           D_l=Dl, D_s=Ds, counter_term=ct, anti_trapping=at, a_at=0.25)
        phi0, c0 = WL.random_fields((1, ny, nx), seed=100 + j)
        out.append((m, phi0, c0))
    return out


def test_batch_fp64_matches_oracle_per_instance():
    inst = _mixed_instances()
    b = L.BatchSimulation([m for m, _, _ in inst], [p for _, p, _ in inst], [c for _, _, c in inst],
                          precision="fp64")
    b.step(40)
    for i, (m, phi0, c0) in enumerate(inst):
        phi, c, mu = b.fields(i)
        o = O.Oracle(to_oracle(m), phi0, c0).step(40)
        errs = (rel_err(phi, o.phi), rel_err(c, o.c), rel_err(mu, o.mu))
        assert max(errs) < FP64_TOL, (i, errs)
    masses = b.solute_masses()
    b.close()
    for i, (m, phi0, c0) in enumerate(inst):
        assert abs(masses[i] - c0.sum()) <= 1e-12 * c0.sum(), i


def test_batch_fp32_agrees_with_single_runs():
    inst = _mixed_instances()[:4]
    b = L.BatchSimulation([m for m, _, _ in inst], [p for _, p, _ in inst], [c for _, _, c in inst],
                          precision="fp32")
    b.step(30)
    for i, (m, phi0, c0) in enumerate(inst):
        phi_b, c_b, _ = b.fields(i)
        s = L.Simulation(m, phi0, c0, precision="fp32")
        s.step(30)
        phi_s, c_s, _ = s.fields()
        s.close()
        assert rel_err(phi_b, phi_s) < 1e-6 and rel_err(c_b, c_s) < 1e-6, i
    b.close()


def test_graph_replay_matches_plain_launches():
    """On a non-default stream lbpf_step replays a captured two-step graph; the
    result must be identical to launching the kernels one by one."""
    import torch
    m, phi0, c0 = WL.porous_3d(n=40)
    stream = torch.cuda.Stream()
    a = L.Simulation(m, phi0, c0, precision="fp32", stream=stream.cuda_stream, mass_every=1)
    b = L.Simulation(m, phi0, c0, precision="fp32", mass_every=1)   # default stream: no graph
    a.step(11)
    b.step(11)
    pa, ca, _ = a.fields()
    pb, cb, _ = b.fields()
    ma, _ = a.solute_mass()
    mb, _ = b.solute_mass()
    a.close()
    b.close()
    assert np.array_equal(pa, pb) and np.array_equal(ca, cb)
    assert ma == mb


def test_batch_of_the_sweep_workload_runs():
    """A slice of the 384-instance sweep (sizes 64..768, 1-8 discs, D_l and
    M_phi/D_l drawn at random, counter term on or off): finite and mass-conserving."""
    inst = WL.batch_2d(count=24, seed=1)
    b = L.BatchSimulation([x.params for x in inst], [x.phi for x in inst], [x.c for x in inst],
                          precision="fp32")
    m0 = b.solute_masses()
    b.step(200)
    m1 = b.solute_masses()
    for i in range(len(inst)):
        phi, c, _ = b.fields(i)
        assert np.all(np.isfinite(phi)) and np.all(np.isfinite(c))
    b.close()
    assert np.max(np.abs(m1 - m0) / m0) < 1e-5


def test_every_tile_shape_gives_the_same_bits():
    # the tile shape changes the schedule only: each node's arithmetic is the same
    inst = _mixed_instances()
    ref = None
    for tile in L.BATCH_TILES:
        b = L.BatchSimulation([m for m, _, _ in inst], [p for _, p, _ in inst], [c for _, _, c in inst],
                              precision="fp32")
        b.set_tile(*tile)
        assert b.tile()[0] == tile
        b.step(7)
        out = [b.fields(i)[:2] for i in range(b.n)]
        b.close()
        if ref is None:
            ref = out
        for (pa, ca), (pb, cb) in zip(out, ref):
            assert np.array_equal(pa, pb) and np.array_equal(ca, cb), tile


def test_autotuner_times_every_shape_and_keeps_the_fastest():
    inst = _mixed_instances()
    b = L.BatchSimulation([m for m, _, _ in inst], [p for _, p, _ in inst], [c for _, _, c in inst],
                          precision="fp32")
    tile, ms = b.tile()
    with pytest.raises(L.LbpfError) as ei:
        b.set_tile(48, 8)
    b.close()
    assert ei.value.status == L.LBPF_EINVAL
    assert tile in L.BATCH_TILES
    assert np.all(ms > 0)
    assert ms[L.BATCH_TILES.index(tile)] == ms.min()


def test_full_size_sweep_sampled_against_the_oracle():
    """The 384-instance sweep the benchmark times (83 M nodes, FP32, the
    autotuned tile, graphs): after 3 steps the smallest, the median and the
    largest instance agree with the FP64 oracle run from the same fields."""
    inst = WL.batch_2d(count=384, seed=1)
    b = L.BatchSimulation([x.params for x in inst], [x.phi for x in inst], [x.c for x in inst], precision="fp32")
    b.step(3)
    sizes = np.array([x.params.nodes for x in inst])
    order = np.argsort(sizes)
    for i in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        phi, c, _ = b.fields(i)
        o = O.Oracle(to_oracle(inst[i].params), inst[i].phi, inst[i].c).step(3)
        errs = dict(phi=rel_err(phi, o.phi), c=rel_err(c, o.c))
        assert max(errs.values()) < 2e-5, (i, inst[i].params.nx, errs)
    b.close()
