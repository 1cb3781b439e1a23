"""Brute-force pin of the oracle: one step of Sec. 3 written again, independently,
as whole-array NumPy (shifts with np.roll, mirror ghosts with np.pad, bounce-back
as a mask, instead of the oracle's per-node C loops and index maps), on tiny
grids (4 x 4, 5 x 3, 3 x 3 x 3, 4 x 3 x 5 periodic; 6 x 5, 7 x 4, 5 x 3 x 4 and
3 x 4 x 5 with bounce-back walls on one or two axes), for the main scheme and
every option: both phi equations, anti-trapping, h on D2Q5 / D3Q7, h^eq,alt and
unequal curvatures.

The initial populations and one step must agree with the oracle to rounding
(1e-13 relative; the two sum in different orders).  Catches an index, offset
or stream-direction mistake in the oracle's loops, which the invariants and
closed forms of the other pins could miss on symmetric inputs.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2111_05960_gb300 import workloads as WL

TOL = 1e-13


BC = (0, 0, 0)   # set per test: 0 periodic, 1 half-way bounce-back, per axis (x, y, z)


def _shift(a, e):
    """a(x + e) for every x on the phi stencil: periodic, or across a wall the mirror
    ghost a(-1) = a(0), a(-2) = a(1) (np.pad 'symmetric'); a has the grid as its
    last three axes (z, y, x)."""
    out = a
    for ax, (d, bc) in enumerate(zip((e[2], e[1], e[0]), (BC[2], BC[1], BC[0]))):
        axis = ax - 3
        if d == 0:
            continue
        if bc == 0:
            out = np.roll(out, -d, axis=axis)
        else:
            n = out.shape[axis]
            pad = [(0, 0)] * out.ndim
            pad[axis] = (2, 2)
            padded = np.pad(out, pad, mode="symmetric")
            out = np.take(padded, np.arange(n) + 2 + d, axis=axis)
    return out


def _stream(fs, e, opp):
    """f_k(x) = f*_k(x - e_k), or f*_{opp k}(x) when x - e_k lies beyond a wall."""
    out = np.empty_like(fs)
    for k in range(fs.shape[0]):
        src = np.roll(fs[k], shift=(e[k][2], e[k][1], e[k][0]), axis=(-3, -2, -1))
        nz, ny, nx = fs.shape[1:]
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        outside = np.zeros((nz, ny, nx), dtype=bool)
        for c, n, d, bc in ((x, nx, e[k][0], BC[0]), (y, ny, e[k][1], BC[1]), (z, nz, e[k][2], BC[2])):
            if bc:
                outside |= (c - d < 0) | (c - d >= n)
        out[k] = np.where(outside, fs[opp[k]], src)
    return out


def _parabolas(p):
    e_s = math.sqrt(p.eps_ratio)
    e_l = 1.0 / e_s
    m_l = p.c_l_co - e_s * p.mu_eq
    m_s = p.c_s_co - e_l * p.mu_eq
    df = 0.5 * (e_l - e_s) * p.mu_eq ** 2 - (m_l - m_s) * p.mu_eq
    return e_s, e_l, m_l, m_s, df


def _mu(p, phi, c):
    if p.unequal_eps:
        e_s, e_l, m_l, m_s, _ = _parabolas(p)
        return (c - phi * m_l - (1 - phi) * m_s) / (e_s * phi + e_l * (1 - phi))
    return p.mu_eq + c - (p.c_l_co * phi + p.c_s_co * (1 - phi))


def _tables(p):
    code = 3 if p.nz > 1 else 2
    e, w, _ = O.lattice_tables(code)
    if p.h_lattice:
        eh, wh, _ = O.lattice_tables(7 if p.nz > 1 else 5)
    else:
        eh, wh = e, w
    return e, w, eh, wh


def _opposite(e):
    return np.array([next(j for j in range(len(e)) if np.all(e[j] == -e[k])) for k in range(len(e))])


def _sources(p, e, w, eh, wh, phi, c, dphi):
    """Pointwise terms of a step (Sec. 3.2, 3.3) from the fields at time n."""
    mu = _mu(p, phi, c)
    grad = np.zeros((3,) + phi.shape)
    for k in range(1, len(w)):
        dk = 0.5 * (_shift(phi, e[k]) - _shift(phi, -e[k]))
        for a in range(3):
            grad[a] += 3.0 * w[k] * e[k][a] * dk
    nrm = grad / np.sqrt((grad ** 2).sum(0) + p.eps_n ** 2)
    M = p.tau_g / 3.0
    pq = phi * (1 - phi)
    if p.unequal_eps:
        e_s, e_l, m_l, m_s, df = _parabolas(p)
        S = 6 * pq * (0.5 * (e_l - e_s) * mu ** 2 - (m_l - m_s) * mu - df)
        jump = (e_l - e_s) * mu + m_s - m_l
    else:
        S = 6 * pq * (p.c_s_co - p.c_l_co) * (mu - p.mu_eq)
        jump = p.c_s_co - p.c_l_co
    Gst = -p.lam * M * S / p.W ** 2
    G = np.empty((len(w),) + phi.shape)
    for k in range(len(w)):
        en = sum(e[k][a] * nrm[a] for a in range(3))
        if p.counter_term:
            G[k] = w[k] * (Gst + (4.0 / p.W) * pq * en)
        else:
            G[k] = w[k] * (Gst - (8 * M / p.W ** 2) * 2 * pq * (1 - 2 * phi))
    D = p.D_l * phi + p.D_s * (1 - phi)
    at = p.a_at * p.W * jump * dphi if p.anti_trapping else 0.0 * phi
    F = np.stack([mu * (p.D_l - p.D_s) * grad[a] + at * nrm[a] for a in range(3)])
    gamma = 3.0 / p.tau_h
    heq = np.empty((len(wh),) + phi.shape)
    eF = np.empty_like(heq)
    for k in range(len(wh)):
        heq[k] = wh[k] * gamma * D * mu if k else c - (1 - wh[0]) * gamma * D * mu
        eF[k] = sum(eh[k][a] * F[a] for a in range(3))
    return G, heq, eF, gamma


def _h_target(p, wh, heq, eF, gamma):
    """(equilibrium the collision relaxes to, source added after it): h^eq - H/2 and H,
    or h^eq,alt and 0."""
    if p.h_eq_alt:
        alt = heq + 3.0 * wh[:, None, None, None] * eF
        alt[0] = heq[0]
        return alt, 0.0 * heq
    H = gamma * wh[:, None, None, None] * eF
    return heq - 0.5 * H, H


def np_init(p, phi0, c0):
    e, w, eh, wh = _tables(p)
    G, heq, eF, gamma = _sources(p, e, w, eh, wh, phi0, c0, 0.0 * phi0)
    g = w[:, None, None, None] * phi0 - 0.5 * G
    target, _ = _h_target(p, wh, heq, eF, gamma)
    return g, target


def np_step(p, g, h, phi, c):
    e, w, eh, wh = _tables(p)
    omg, omh = 1 / (p.tau_g + 0.5), 1 / (p.tau_h + 0.5)
    G, _, _, _ = _sources(p, e, w, eh, wh, phi, c, 0.0 * phi)
    gs = g - omg * (g - (w[:, None, None, None] * phi - 0.5 * G)) + G
    g1 = _stream(gs, e, _opposite(e))
    phi1 = g1.sum(0) + 0.5 * G.sum(0)
    _, heq, eF, gamma = _sources(p, e, w, eh, wh, phi, c, phi1 - phi)
    target, H = _h_target(p, wh, heq, eF, gamma)
    hs = h - omh * (h - target) + H
    h1 = _stream(hs, eh, _opposite(eh))
    return g1, h1, phi1, h1.sum(0)


OPTIONS = [
    dict(),
    dict(counter_term=0),
    dict(anti_trapping=0),
    dict(h_lattice=1),
    dict(h_eq_alt=1),
    dict(unequal_eps=1, eps_ratio=2.5),
    dict(h_lattice=1, h_eq_alt=1, unequal_eps=1, eps_ratio=0.4, counter_term=0),
]


@pytest.mark.parametrize("shape,bc", [((1, 4, 4), (0, 0, 0)), ((1, 3, 5), (0, 0, 0)), ((3, 3, 3), (0, 0, 0)),
                                      ((5, 3, 4), (0, 0, 0)), ((1, 5, 6), (1, 1, 0)), ((1, 4, 7), (1, 0, 0)),
                                      ((4, 3, 5), (1, 0, 1)), ((5, 4, 3), (0, 1, 1))])
@pytest.mark.parametrize("opts", OPTIONS)
def test_one_step_matches_independent_numpy(shape, bc, opts):
    global BC
    BC = bc
    nz, ny, nx = shape
    base = dict(tau_g=0.7, tau_h=0.9, W=3.0, lam=4.0, D_l=0.15, D_s=0.03, counter_term=1,
                anti_trapping=1, a_at=0.2, eps_n=1e-3)
    base.update(opts)
    p = O.OracleParams(nx=nx, ny=ny, nz=nz, bc=bc, **base)
    phi0, c0 = WL.random_fields(shape, seed=nx + 7 * ny + 31 * nz, smooth=False)
    o = O.Oracle(p, phi0, c0)
    g0, h0 = np_init(p, phi0, c0)
    scale = lambda a: np.abs(a).max()
    assert np.abs(o.g - g0).max() < TOL * scale(g0)
    assert np.abs(o.h - h0).max() < TOL * scale(h0)
    # one step from the oracle's own state, so that only the step is compared
    g1, h1, phi1, c1 = np_step(p, o.g.copy(), o.h.copy(), o.phi.copy(), o.c.copy())
    o.step(1)
    assert np.abs(o.phi - phi1).max() < TOL * scale(phi1)
    assert np.abs(o.c - c1).max() < TOL * scale(c1)
    assert np.abs(o.g - g1).max() < TOL * scale(g1)
    assert np.abs(o.h - h1).max() < TOL * scale(h1)
