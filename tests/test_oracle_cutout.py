"""Pin of the sampled-node parity method: the oracle evaluated on a cut-out of the initial
fields around a node (half-width 3 steps + 1, periodic wrap in x/y, clipped at the real walls in
z) gives that node's moments exactly as the full-field oracle does, at nodes on the periodic
seams, next to both walls and in the interior; and the dependency radius it rests on is 2 k + 1
after k steps, exactly (a cut-out reaching 2 k + 1 nodes out is exact, one reaching 2 k is not)."""
import numpy as np
import pytest

from oracle import lbm
from paper_1111_0905_gb300 import config
from helpers import STEP_RADIUS, _cutout_centre, oracle_cutout_moments, oracle_run

NODES = [(0, 0, 0), (23, 20, 21), (0, 10, 1), (12, 0, 20), (23, 5, 11), (7, 13, 9),
         (1, 19, 2), (22, 1, 19)]


def _full(steps):
    w = config.boiling_cell(24, nz=22, ny=21)
    rho, T = w.fields()
    f, g, op, _ = oracle_run(w.params, rho, T, steps)
    r_o, u_o, T_o = lbm.moments_out(f, g, op)
    want = lambda x, y, z: [float(r_o[z, y, x]), float(u_o[0][z, y, x]), float(u_o[1][z, y, x]),
                            float(u_o[2][z, y, x]), float(T_o[z, y, x])]
    return w.params, rho, T, want


@pytest.mark.parametrize("steps", [1, 2])
def test_cutout_equals_full_field(steps):
    p, rho, T, want = _full(steps)
    got = oracle_cutout_moments(p, rho, T, steps, NODES)
    for k, (x, y, z) in enumerate(NODES):
        assert list(got[k]) == want(x, y, z), (x, y, z, got[k], want(x, y, z))


@pytest.mark.parametrize("steps", [1, 2, 3])
def test_dependency_radius(steps):
    p, rho, T, want = _full(steps)
    x, y, z = 12, 10, 11
    assert 2 * steps + 1 <= STEP_RADIUS * steps + 1
    tight = _cutout_centre(p, rho, T, steps, x, y, z, 2 * steps + 1)
    assert tight == want(x, y, z)
    short = _cutout_centre(p, rho, T, steps, x, y, z, 2 * steps)
    assert max(abs(a - b) for a, b in zip(short, want(x, y, z))) > 1e-9
