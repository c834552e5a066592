"""Parity at the benchmark's full sizes, in its launch configuration (default 32 x 8 tiles and
the chunking lb_init chooses), on sampled nodes: the GPU runs the whole cell, and each sampled
node's rho, u, T after 2 steps is compared with the FP64 oracle evaluated on a cut-out of the
initial fields around that node (exact for the node, pinned in test_oracle_cutout.py). Samples:
the corners, nodes on both walls and next to them, on the x/y tile seams and on the z-chunk
seams, and seeded random nodes.

Cells: the 128^3 single-phase cell in FP32 (the benchmark's headline form); the 256^3 boiling
cell in BF16 and FP16 deviation storage and FP16 against local references; the 512^3 boiling
cell in FP32, FP16 deviation storage and FP16 against local references (the sizes the bandwidth
figures are quoted at). Tolerances as for the small grids: FP32
1e-5 of each field's scale (u on a floor of 1e-2), 16-bit 2e-3 on rho and T.
"""
import numpy as np
import pytest
import torch

from paper_1111_0905_gb300 import config, lb
from helpers import oracle_cutout_moments

pytestmark = pytest.mark.gpu

STEPS = 2


def _nodes(p, nchunks, seed):
    nx, ny, nz = p.nx, p.ny, p.nz
    zc = -(-nz // nchunks)
    nodes = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, ny - 1, 1), (nx - 1, 0, nz - 2),
             (31, 7, nz // 2), (32, 8, nz // 2 + 1), (63, 0, 0), (64, ny - 1, nz - 1),
             (17, 3, zc - 1), (18, 4, zc), (nx // 2, ny // 2, min(2 * zc, nz - 1))]
    rng = np.random.default_rng(seed)
    nodes += [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(9)]
    return nodes


def _check(w, tol_field, tol_u, seed):
    p = w.params
    rho, T = w.fields()
    lat = lb.Lattice(p, torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
    info = lat.launch_info()
    assert info["threads_per_cta"] == 256 and info["grid"][0] == (p.nx // 32) * (p.ny // 8)
    lat.step(STEPS)
    r_g, u_g, T_g = lat.moments(device=True)
    nodes = _nodes(p, info["grid"][1], seed)
    idx = torch.tensor([(z * p.ny + y) * p.nx + x for x, y, z in nodes], device="cuda")
    gpu = torch.stack([r_g.reshape(-1)[idx], u_g[0].reshape(-1)[idx], u_g[1].reshape(-1)[idx],
                       u_g[2].reshape(-1)[idx], T_g.reshape(-1)[idx]], dim=1).cpu().numpy()
    lat.close()
    del r_g, u_g, T_g
    torch.cuda.empty_cache()
    ora = oracle_cutout_moments(p, rho, T, STEPS, nodes)
    e_rho = np.abs(gpu[:, 0] - ora[:, 0]).max() / np.abs(ora[:, 0]).max()
    e_T = np.abs(gpu[:, 4] - ora[:, 4]).max() / np.abs(ora[:, 4]).max()
    u_scale = max(float(np.abs(ora[:, 1:4]).max()), 1e-2)
    e_u = np.abs(gpu[:, 1:4] - ora[:, 1:4]).max() / u_scale
    print(f"{p.nx}^3 precision {p.precision}: rho {e_rho:.2e}, T {e_T:.2e}, u {e_u:.2e} "
          f"over {len(nodes)} nodes, grid {info['grid']}")
    assert e_rho < tol_field and e_T < tol_field, (e_rho, e_T)
    if tol_u is not None:
        assert e_u < tol_u, e_u


def test_fp32_single_phase_128(lblib, cuda):
    _check(config.single_phase_cell(128, precision=lb.LB_FP32), 1e-5, 1e-5, 128)


@pytest.mark.parametrize("prec", [lb.LB_BF16_DEV, lb.LB_FP16_DEV, lb.LB_FP16_LOC])
def test_16bit_boiling_256(lblib, cuda, prec):
    _check(config.paper_scale_cell(256, precision=prec), 2e-3, None, 256 + prec)


@pytest.mark.parametrize("prec,tol", [(lb.LB_FP32, 1e-5), (lb.LB_FP16_DEV, 2e-3), (lb.LB_FP16_LOC, 2e-3)])
def test_boiling_512(lblib, cuda, prec, tol):
    _check(config.paper_scale_cell(512, precision=prec), tol, 1e-5 if prec == lb.LB_FP32 else None,
           512 + prec)
