"""Why the porous benchmark uses W = 3 instead of the workload's W = 2.

With the coupling lambda* of Eq. Lambda-Star (M_phi = 1.2 D_l, the ratio of
Sec. 4 and Sec. 5), the counter term (Eq. SourceG_CT) and the anti-trapping
current (Eq. Anti-trapping_Equilibrium), a tanh interface two nodes wide is
under-resolved: the FP64 oracle itself leaves the physical range of c and then
blows up within ~150 steps.  Three nodes keep the same medium bounded for
thousands of steps.  (Sec. 5 itself resolves its interface with about twenty
nodes, W = 0.02 on a 1024-node unit square.)  Both runs use the porous
generator of the benchmark at 32^3 (periodic), everything else unchanged.
"""
import numpy as np
import pytest

import oracle as O
from paper_2111_05960_gb300 import workloads as WL
from conftest import to_oracle


def _run(W, steps, every=10):
    m, phi0, c0 = WL.porous_3d(n=32, W=W)
    o = O.Oracle(to_oracle(m), phi0, c0)
    left_range, non_finite = None, None
    for s in range(every, steps + 1, every):
        o.step(every)
        finite = bool(np.all(np.isfinite(o.c)) and np.all(np.isfinite(o.phi)))
        if not finite:
            non_finite = s
            break
        if left_range is None and (o.c.max() > 1.5 or o.c.min() < 0.0):
            left_range = s
    return o, c0, left_range, non_finite


def test_two_node_interface_diverges_in_the_oracle():
    _, _, left_range, non_finite = _run(2.0, 400)
    assert left_range is not None and left_range <= 300, left_range
    assert non_finite is not None and non_finite <= 400, non_finite


@pytest.mark.slow
def test_three_node_interface_stays_bounded():
    o, c0, left_range, non_finite = _run(3.0, 1500, every=100)
    assert non_finite is None and left_range is None
    assert -1e-3 < o.phi.min() and o.phi.max() < 1.0 + 1e-3
    assert 0.0 <= o.c.min() and o.c.max() < 1.2
    # solute conservation (Eq. Moment0_LBM_Concent) holds all along
    assert abs(o.c.sum() - c0.sum()) <= 1e-12 * c0.sum()
