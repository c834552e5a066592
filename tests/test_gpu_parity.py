"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances: FP64 1e-12 of each field's scale after N steps; FP32 1e-5; 16-bit deviation
storage 2e-3 on rho and T. Grids span several 32 x BY tiles, ragged tails in x, y and z,
several z chunks, the degenerate nz = 1, 2 and the three tile heights.
"""
import math

import numpy as np
import pytest
import torch

from oracle import lbm
from paper_1111_0905_gb300 import config, lb, synthetic
from helpers import oracle_params, oracle_run, rel_err

pytestmark = pytest.mark.gpu


def _gpu_run(p, rho, T, steps):
    lat = lb.Lattice(p, rho, T)
    lat.step(steps)
    rho_g, u_g, T_g = lat.moments()
    f_g, g_g = lat.populations()
    nu = lat.nusselt()
    return lat, rho_g, u_g, T_g, f_g, g_g, nu


def _compare(p, rho, T, steps, tol, nu_tol=None, pops=True, u_floor=None):
    lat, rho_g, u_g, T_g, f_g, g_g, nu = _gpu_run(p, rho, T, steps)
    f, g, op, _ = oracle_run(p, rho, T, steps)
    r_o, u_o, T_o = lbm.moments_out(f, g, op)
    errs = {"rho": rel_err(rho_g, r_o), "T": rel_err(T_g, T_o)}
    # velocity errors on the velocity scale with a floor: u = (j + F/2)/rho is a difference of
    # O(rho) population sums and of the O(0.1)-term force sum of Eq. (9), so its rounding error is
    # absolute (~1e-16 in FP64, ~1e-8 in FP32). Floors: 1e-3 lattice units for FP64, 1e-2 (Mach
    # ~0.02, a typical convection velocity) for the FP32/16-bit forms.
    if u_floor is None:
        u_floor = 1e-3 if p.precision == lb.LB_FP64 else 1e-2
    u_scale = max(max(float(np.abs(u_o[a].numpy()).max()) for a in range(3)), u_floor)
    for a in range(3):
        errs[f"u{a}"] = float(np.abs(u_g[a] - u_o[a].numpy()).max()) / u_scale
    if pops:
        errs["f"] = rel_err(f_g, f)
        errs["g"] = rel_err(g_g, g)
    nu_o, nuz_o = lbm.nusselt(f, g, op)
    errs["nu_z"] = float(np.abs(nu[1] - nuz_o.numpy()).max() / max(1.0, np.abs(nuz_o.numpy()).max()))
    lat.close()
    bad = {k: v for k, v in errs.items() if v > (nu_tol if (k == "nu_z" and nu_tol) else tol)}
    assert not bad, f"errors above tolerance: {bad} (all: {errs})"
    return errs


GRIDS = [
    # (nx, ny, nz, tile_y, z_chunk)
    (4, 4, 4, 8, 0),
    (5, 6, 7, 4, 3),
    (33, 9, 7, 8, 2),       # two x tiles with a 1-wide tail, ragged y, chunks of 2
    (40, 17, 10, 4, 4),
    (8, 8, 1, 4, 0),        # single layer between the two walls
    (8, 5, 2, 8, 1),
]


@pytest.mark.parametrize("nx,ny,nz,by,zc", GRIDS)
def test_fp64_boiling_parity_small_grids(lblib, cuda, nx, ny, nz, by, zc):
    w = config.boiling_cell(nx, nz=nz, ny=ny)
    p = w.params
    p.tile_y, p.z_chunk = by, zc
    rho, T = w.fields()
    _compare(p, rho, T, 12, 1e-12, nu_tol=1e-9)


def test_init_state_is_the_equilibrium(lblib, cuda):
    w = config.boiling_cell(12, nz=9, ny=7)
    rho, T = w.fields()
    lat = lb.Lattice(w.params, rho, T)
    r, u, TT = lat.moments()
    f, g = lat.populations()
    op = oracle_params(w.params)
    f0, g0 = lbm.init_state(torch.from_numpy(rho), torch.from_numpy(T), op)
    assert rel_err(r, rho) < 1e-14 and rel_err(TT, T) < 1e-14
    assert rel_err(f, f0) < 1e-14 and rel_err(g, g0) < 1e-14
    lat.close()


def test_fp64_boiling_cell_32_200_steps(lblib, cuda):
    """The 32^3 boiling cell (phase separation inside the spinodal), 200 steps, 1e-12."""
    w = config.boiling_cell(32)
    rho, T = w.fields()
    errs = _compare(w.params, rho, T, 200, 1e-12, nu_tol=1e-9, pops=False)
    print("32^3 x 200 FP64 errors:", errs)


def test_fp64_single_phase_full_size_128(lblib, cuda):
    """Full 128^3 single-phase workload in the benchmark's launch configuration, 2 steps."""
    w = config.single_phase_cell(128)
    rho, T = w.fields()
    _compare(w.params, rho, T, 2, 1e-12, nu_tol=1e-9, pops=False)


def test_fp32_parity(lblib, cuda):
    w = config.single_phase_cell(32, precision=lb.LB_FP32)
    rho, T = w.fields()
    errs = _compare(w.params, rho, T, 50, 1e-5, nu_tol=1e-5, pops=True)
    print("FP32 errors:", errs)


@pytest.mark.parametrize("by,zc", [(16, 4), (8, 32), (4, 0)])
def test_fp32_ragged_tiles(lblib, cuda, by, zc):
    """FP32 form on a ragged grid with each tile height (the 16-row tile is FP32/16-bit only)."""
    w = config.boiling_cell(40, nz=11, ny=19, precision=lb.LB_FP32)
    p = w.params
    p.tile_y, p.z_chunk = by, zc
    rho, T = w.fields()
    _compare(p, rho, T, 20, 1e-5, nu_tol=1e-5, pops=True)


def test_fp64_rejects_the_16_row_tile(lblib, cuda):
    """The FP64 windows of a 32 x 16 tile exceed a CTA's shared memory: lb_init says LB_EINVAL."""
    w = config.boiling_cell(8)
    p = w.params
    p.tile_y = 16
    rho, T = w.fields()
    with pytest.raises(lb.LBError) as e:
        lb.Lattice(p, rho, T)
    assert e.value.code == -1


def test_fp32_boiling_parity(lblib, cuda):
    w = config.boiling_cell(24, precision=lb.LB_FP32)
    rho, T = w.fields()
    errs = _compare(w.params, rho, T, 30, 1e-5, nu_tol=1e-5, pops=True)
    print("FP32 boiling errors:", errs)


@pytest.mark.parametrize("prec", [lb.LB_BF16_DEV, lb.LB_FP16_DEV, lb.LB_FP16_LOC])
def test_16bit_deviation_storage(lblib, cuda, prec):
    """rho and T within 2e-3 of the FP64 oracle after 50 steps of the single-phase cell."""
    w = config.single_phase_cell(32, precision=prec)
    rho, T = w.fields()
    lat = lb.Lattice(w.params, rho, T)
    lat.step(50)
    r, u, TT = lat.moments()
    f, g, op, _ = oracle_run(w.params, rho, T, 50)
    r_o, u_o, T_o = lbm.moments_out(f, g, op)
    e_rho = float(np.abs(r - r_o.numpy()).max() / np.abs(r_o.numpy()).max())
    e_T = float(np.abs(TT - T_o.numpy()).max() / np.abs(T_o.numpy()).max())
    print("16-bit", prec, e_rho, e_T)
    assert e_rho < 2e-3 and e_T < 2e-3
    lat.close()


def test_nu_time_average_matches_oracle(lblib, cuda):
    w = config.boiling_cell(16)
    p = w.params
    p.nu_every = 2
    rho, T = w.fields()
    lat = lb.Lattice(p, rho, T)
    lat.step(10)
    nu_mean, nu_z, avg = lat.nusselt()
    _, _, _, samples = oracle_run(p, rho, T, 10, nu_every=2)
    assert len(samples) == 5
    assert abs(avg - np.mean(samples)) < 1e-9 * max(1.0, abs(np.mean(samples)))
    lat.close()


def test_mass_conserved_and_diagnostics(lblib, cuda):
    w = config.boiling_cell(24)
    rho, T = w.fields()
    lat = lb.Lattice(w.params, rho, T)
    d0 = lat.diagnostics()
    assert abs(d0["mass"] - rho.sum()) < 1e-12 * rho.sum()
    assert abs(d0["min_rho"] - rho.min()) < 1e-15 and d0["nonfinite"] == 0
    lat.step(100)
    d1 = lat.diagnostics()
    assert abs(d1["mass"] - d0["mass"]) < 1e-13 * d0["mass"]
    lat.close()


def test_checkpoint_roundtrip_is_bitwise(lblib, cuda, tmp_path):
    w = config.boiling_cell(16)
    rho, T = w.fields()
    a = lb.Lattice(w.params, rho, T)
    a.step(20)
    a.save(tmp_path / "c.bin")
    a.step(30)
    fa, ga = a.populations()
    b = lb.Lattice(w.params, rho, T)
    b.load(tmp_path / "c.bin")
    assert b.step_count == 20
    b.step(30)
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    # a corrupted file is rejected
    raw = bytearray((tmp_path / "c.bin").read_bytes())
    raw[-5] ^= 0xFF
    (tmp_path / "bad.bin").write_bytes(bytes(raw))
    with pytest.raises(lb.LBError) as e:
        b.load(tmp_path / "bad.bin")
    assert e.value.code == -5
    a.close(); b.close()


def test_health_check_reports_nonphysical_state(lblib, cuda):
    """tau_nu = 0.55 is linearly unstable for this scheme: the periodic health check returns
    LB_ENONPHYS (a host-side error code; nothing faults on the device)."""
    w = config.boiling_cell(8)
    p = w.params
    p.tau_nu, p.tau_kappa, p.kappa, p.check_every = 0.55, 0.6, 0.02, 25
    rho, T = w.fields()
    lat = lb.Lattice(p, rho, T)
    with pytest.raises(lb.LBError) as e:
        lat.step(3000)
    assert e.value.code == -4
    lat.close()


def test_invalid_arguments(lblib, cuda):
    w = config.boiling_cell(8)
    rho, T = w.fields()
    bad = rho.copy()
    bad[0, 0, 0] = -1.0
    with pytest.raises(lb.LBError):
        lb.Lattice(w.params, bad, T)
    lat = lb.Lattice(w.params, rho, T)
    with pytest.raises(lb.LBError):
        lat.step(-1)
    lat.close()


def test_device_pointers_and_stream(lblib, cuda):
    """Initial fields and outputs passed as device pointers give the same result as host ones."""
    w = config.boiling_cell(16)
    rho, T = w.fields()
    a = lb.Lattice(w.params, torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
    b = lb.Lattice(w.params, rho, T)
    a.step(5); b.step(5)
    ra, ua, Ta = a.moments(device=True)
    rb, ub, Tb = b.moments()
    assert np.array_equal(ra.cpu().numpy(), rb) and np.array_equal(Ta.cpu().numpy(), Tb)
    a.close(); b.close()


SHAPES = [(8, 0), (8, 5), (8, 23), (4, 7), (4, 1), (16, 23), (16, 3)]
CROSS_TILE_TOL = {lb.LB_FP64: 1e-12, lb.LB_FP32: 1e-5, lb.LB_BF16_DEV: 2e-3, lb.LB_FP16_DEV: 2e-3,
                  lb.LB_FP16_LOC: 2e-3}


@pytest.mark.parametrize("prec", [lb.LB_FP64, lb.LB_FP32, lb.LB_BF16_DEV, lb.LB_FP16_DEV, lb.LB_FP16_LOC])
def test_launch_shape_does_not_change_the_result(lblib, cuda, prec):
    """Chunk prologues recompute their planes with the same arithmetic: for one tile height the
    populations after 30 steps of a ragged boiling cell are bitwise equal whatever the z chunk.
    Different tile heights are different kernel instantiations, whose floating-point contractions
    may differ: those agree within the form's parity tolerance."""
    w = config.boiling_cell(40, nz=23, ny=19, precision=prec)
    rho, T = w.fields()
    by_tile = {}
    for by, zc in SHAPES:
        if by == 16 and prec == lb.LB_FP64:
            continue
        p = w.params
        p.tile_y, p.z_chunk = by, zc
        lat = lb.Lattice(p, rho, T)
        info = lat.launch_info()
        assert info["threads_per_cta"] == 32 * by
        if zc:
            assert info["grid"][1] == -(-23 // zc)
        lat.step(30)
        f, g = lat.populations()
        lat.close()
        assert np.isfinite(f).all() and np.isfinite(g).all()
        if by not in by_tile:
            by_tile[by] = (f, g)
        else:
            ref = by_tile[by]
            assert np.array_equal(f, ref[0]) and np.array_equal(g, ref[1]), (by, zc)
    f8, g8 = by_tile[8]
    for by, (f, g) in by_tile.items():
        assert rel_err(f, f8) <= CROSS_TILE_TOL[prec] and rel_err(g, g8) <= CROSS_TILE_TOL[prec], by


def test_chunk_choice_and_occupancy(lblib, cuda):
    """The default launch of the FP32 and 16-bit forms keeps two CTAs of 256 threads per SM with
    at most 128 registers a thread, and picks the chunk count that minimises the wave cost
    ceil(CTAs / slots) * (zc + 4) over zc = 8..128."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for prec in (lb.LB_FP32, lb.LB_FP16_DEV):
        for n in (64, 128):
            w = config.single_phase_cell(n, precision=prec)
            rho, T = w.fields()
            lat = lb.Lattice(w.params, rho, T)
            info = lat.launch_info()
            lat.close()
            assert info["threads_per_cta"] == 256 and info["ctas_per_sm"] == 2
            assert info["registers"] <= 128
            ntiles = (n // 32) * (n // 8)
            assert info["grid"][0] == ntiles
            slots = 2 * sms
            costs = {}
            for nch in range(1, n + 1):
                zc = -(-n // nch)
                if zc > 128:
                    continue
                if zc < 8 and nch > 1:
                    break
                ctas = ntiles * -(-n // zc)
                costs.setdefault(zc, -(-ctas // slots) * (zc + 4))
            best = min(costs.values())
            zc_used = -(-n // info["grid"][1])
            assert costs[zc_used] == best, (n, info, costs)


VARIANTS = [(lb.LB_FORCE_GUO, lb.LB_PSI_EXP), (lb.LB_FORCE_SHIFT, lb.LB_PSI_VDW),
            (lb.LB_FORCE_GUO, lb.LB_PSI_VDW)]


def _variant_cell(forcing, psi, precision, nx=20, ny=9, nz=11):
    """Boiling cell of the variant: the paper's psi at rho = 1.30 (1 + 0.01 xi); the van der Waals
    psi (a = 5/42, b = 2/21, T_v = T_m, critical point rho_c = 3.5, T_c = 10/27) at
    rho = 3.5 (1 + 0.05 xi), inside its spinodal at T_m."""
    w = config.boiling_cell(nx, nz=nz, ny=ny, precision=precision)
    p = w.params
    p.forcing, p.psi_kind = forcing, psi
    rho, T = w.fields()
    if psi == lb.LB_PSI_VDW:
        rho, _ = synthetic.boiling_fields(nx, ny, nz, 3.5, p.T_d, p.T_u, 0.05)
    return p, rho, T


@pytest.mark.parametrize("forcing,psi", VARIANTS)
def test_variant_parity_fp64(lblib, cuda, forcing, psi):
    """Scheme variants (Guo forcing, van der Waals psi) against the oracle's variants, 1e-12."""
    p, rho, T = _variant_cell(forcing, psi, lb.LB_FP64)
    p.tile_y, p.z_chunk = 4, 3
    _compare(p, rho, T, 15, 1e-12, nu_tol=1e-9)


@pytest.mark.parametrize("forcing,psi", VARIANTS)
def test_variant_parity_fp32(lblib, cuda, forcing, psi):
    p, rho, T = _variant_cell(forcing, psi, lb.LB_FP32)
    _compare(p, rho, T, 15, 1e-5, nu_tol=1e-5)


@pytest.mark.parametrize("prec", [lb.LB_FP16_DEV, lb.LB_FP16_LOC])
def test_variant_parity_16bit(lblib, cuda, prec):
    """Guo forcing with the van der Waals psi in FP16 storage (deviations, and against local
    references): rho and T within 2e-3."""
    p, rho, T = _variant_cell(lb.LB_FORCE_GUO, lb.LB_PSI_VDW, prec)
    lat = lb.Lattice(p, rho, T)
    lat.step(15)
    r, u, TT = lat.moments()
    lat.close()
    f, g, op, _ = oracle_run(p, rho, T, 15)
    r_o, u_o, T_o = lbm.moments_out(f, g, op)
    assert rel_err(r, r_o) < 2e-3 and rel_err(TT, T_o) < 2e-3


def test_variant_arguments(lblib, cuda):
    """Unknown variants, a van der Waals psi that is not real at an initial density, and the
    adjoint of a variant are rejected with error codes."""
    p, rho, T = _variant_cell(lb.LB_FORCE_SHIFT, lb.LB_PSI_VDW, lb.LB_FP64)
    for field, value in (("forcing", 2), ("psi_kind", 7)):
        q = lb.Params(**{**p.__dict__, field: value})
        with pytest.raises(lb.LBError) as e:
            lb.Lattice(q, rho, T)
        assert e.value.code == -1
    too_dense = rho.copy()
    too_dense[0, 0, 0] = 0.999 * (1 - p.vdw_b * p.vdw_T / p.vdw_a) / p.vdw_b + 0.01
    with pytest.raises(lb.LBError) as e:
        lb.Lattice(p, too_dense, T)
    assert e.value.code == -1
    q = lb.Params(**{**p.__dict__, "G": 1.0})       # the van der Waals psi needs G < 0
    with pytest.raises(lb.LBError):
        lb.Lattice(q, rho, T)
    lat = lb.Lattice(p, rho, T)
    with pytest.raises(lb.LBError) as e:
        lat.adjoint(4, 2)
    assert e.value.code == -6
    lat.close()


@pytest.mark.parametrize("prec,tol", [(lb.LB_FP64, 1e-12), (lb.LB_FP32, 1e-6), (lb.LB_FP16_DEV, 1e-6),
                                      (lb.LB_FP16_LOC, 1e-6)])
def test_fused_nu_samples_equal_separate_passes(lblib, cuda, prec, tol):
    """With nu_every the Nu sample of state n is taken by the launch of step n -> n+1 (fused); the
    time average equals the mean of lb_nusselt called after every step (separate moments
    passes), and a checkpoint taken mid-run carries the samples due so far."""
    w = config.boiling_cell(20, nz=14, ny=9, precision=prec)
    rho, T = w.fields()
    p = w.params
    p.nu_every = 1
    a = lb.Lattice(p, rho, T)
    a.step(7)
    q = lb.Params(**{**p.__dict__, "nu_every": 0})
    b = lb.Lattice(q, rho, T)
    samples = []
    for _ in range(7):
        b.step(1)
        samples.append(b.nusselt()[0])
    avg = a.nusselt()[2]
    assert abs(avg - np.mean(samples)) <= tol * abs(np.mean(samples)), (avg, np.mean(samples))
    a.step(5)
    for _ in range(5):
        b.step(1)
        samples.append(b.nusselt()[0])
    assert abs(a.nusselt()[2] - np.mean(samples)) <= tol * abs(np.mean(samples))
    a.close(); b.close()


def test_nu_sampling_with_health_checks_and_checkpoints(lblib, cuda, tmp_path):
    """Nu samples due at a health check or a checkpoint are taken there (not lost or doubled):
    nu_every = 3 with check_every = 2 over 12 steps averages the samples of states 3, 6, 9, 12;
    a checkpoint saved at step 5 with nu_every = 1 and resumed gives the same time average as the
    uninterrupted run, bitwise."""
    w = config.boiling_cell(16, nz=12, ny=8)
    rho, T = w.fields()
    p = w.params
    q = lb.Params(**{**p.__dict__, "nu_every": 3, "check_every": 2})
    a = lb.Lattice(q, rho, T)
    b = lb.Lattice(p, rho, T)
    samples = []
    for n in range(1, 13):
        a.step(1)
        b.step(1)
        if n % 3 == 0:
            samples.append(b.nusselt()[0])
    assert abs(a.nusselt()[2] - np.mean(samples)) <= 1e-12 * abs(np.mean(samples))
    a.close(); b.close()
    r = lb.Params(**{**p.__dict__, "nu_every": 1})
    c = lb.Lattice(r, rho, T)
    c.step(5)
    c.save(tmp_path / "nu.bin")
    c.step(5)
    full = c.nusselt()[2]
    c.close()
    d = lb.Lattice(r, rho, T)
    d.load(tmp_path / "nu.bin")
    d.step(5)
    assert d.nusselt()[2] == full
    d.close()


@pytest.mark.parametrize("prec,tol", [(lb.LB_FP64, 1e-12), (lb.LB_FP32, 1e-5)])
def test_wall_force_of_a_z_profile_on_the_gpu(lblib, cuda, prec, tol):
    """The neutral-wetting wall ghosts on the GPU against the closed form (not the oracle): for a
    density that varies in z only, at the initial state (j = 0, no gravity) the exported physical
    velocity is u = F/(2 rho) with F_x = F_y = 0 and F_z(z) = -(G/2) psi(z) [psi(z+1) - psi(z-1)],
    the plane beyond each halfway wall carrying the density of its mirror image (psi(-1) = psi(0),
    psi(nz) = psi(nz-1)). Ragged tiles (40 x 9) and several z chunks."""
    nx, ny, nz = 40, 9, 7
    z = np.arange(nz, dtype=np.float64)
    prof = 1.3 + 0.4 * np.tanh(z - 1.0) - 0.3 * np.exp(-(nz - 1 - z))
    rho = np.broadcast_to(prof[:, None, None], (nz, ny, nx)).copy()
    T = np.full((nz, ny, nx), config.T_M)
    p = lb.Params(nx=nx, ny=ny, nz=nz, tau_nu=1.0, tau_kappa=1.0, G=config.G_DEFAULT, kappa=0.05,
                  g_z=0.0, T_d=config.T_M, T_u=config.T_M, precision=prec, tile_y=4, z_chunk=3)
    lat = lb.Lattice(p, rho, T)
    r, u, TT = lat.moments()
    lat.close()
    ps = np.exp(-1.0 / prof)
    ext = np.concatenate([[ps[0]], ps, [ps[-1]]])          # planes -1 .. nz
    Fz = -(p.G / 2.0) * ps * (ext[2:] - ext[:-2])
    want = Fz / (2.0 * prof)
    scale = np.abs(want).max()
    assert scale > 1e-3
    got = u[2][:, 0, 0]
    assert np.abs(u[2] - want[:, None, None]).max() <= tol * scale, (got, want)
    assert np.abs(u[0]).max() <= tol * scale and np.abs(u[1]).max() <= tol * scale


def _evolved_state(steps: int = 300):
    """Pre-collision populations of the 32 x 24 x 20 boiling cell (tau_nu = 1.25, kappa = 0.15)
    after `steps` FP64 GPU steps: phase separation under way, with flow at the interfaces."""
    w = config.boiling_cell(32, nz=20, ny=24, kappa=0.15, tau_nu=1.25)
    p = w.params
    rho, T = w.fields()
    lat = lb.Lattice(p, rho, T)
    lat.step(steps)
    f, g = lat.populations()
    lat.close()
    return p, rho, T, f, g


def _oracle_from(p, f, g, steps):
    op = oracle_params(p)
    ft, gt = torch.from_numpy(f), torch.from_numpy(g)
    for _ in range(steps):
        ft, gt = lbm.step(ft, gt, op)
    return ft, gt, op


def _conv_scale(f, g, op):
    """Scale of the convective term of Nu(z): max over z of <|rho U u_z|>_{x,y} / (kappa dT/nz)."""
    r, j, T, F, v, u = lbm.macroscopic(f, g, op)
    U = lbm.internal_energy(r, T, op)
    q = (r * U * u[2]).abs().mean(dim=(1, 2)) / (op.kappa * (op.T_d - op.T_u) / op.nz)
    return float(q.max())


def test_set_populations_continues_the_run_exactly(lblib, cuda):
    """lb_set_populations stores a given pre-collision state so that the next steps continue it:
    an FP64 context seeded with the state after 300 steps equals the oracle started from it
    (1e-12), and its populations read back unchanged."""
    p, rho, T, f, g = _evolved_state()
    lat = lb.Lattice(p, rho, T)
    lat.set_populations(f, g)
    assert lat.step_count == 0
    with pytest.raises(lb.LBError) as e:
        lat.adjoint(2, 1, grad_T0=True)      # no longer lb_init's equilibrium
    assert e.value.code == -1
    f1, g1 = lat.populations()
    assert rel_err(f1, f) < 1e-15 and rel_err(g1, g) < 1e-15
    lat.step(10)
    r, u, TT = lat.moments()
    ft, gt, op = _oracle_from(p, f, g, 10)
    r_o, u_o, T_o = lbm.moments_out(ft, gt, op)
    assert rel_err(r, r_o) < 1e-12 and rel_err(TT, T_o) < 1e-12
    us = max(float(np.abs(u_o[a].numpy()).max()) for a in range(3))
    assert max(float(np.abs(u[a] - u_o[a].numpy()).max()) for a in range(3)) < 1e-12 * us
    lat.close()


def _fp32_from(p, rho, T, f, g, steps):
    """FP32 form and oracle from the same FP64 pre-collision state (the FP32 context created from
    the run's initial fields, so that its deviation reference is the run's); errors as in the
    parity tests, u on the largest |u| of the oracle (no floor), Nu(z) on its convective scale."""
    q = lb.Params(**{**p.__dict__, "precision": lb.LB_FP32})
    lat = lb.Lattice(q, rho, T)
    lat.set_populations(f, g)
    lat.step(steps)
    r, u, TT = lat.moments()
    nu = lat.nusselt()[1]
    lat.close()
    ft, gt, op = _oracle_from(p, f, g, steps)
    r_o, u_o, T_o = lbm.moments_out(ft, gt, op)
    us = max(float(np.abs(u_o[a].numpy()).max()) for a in range(3))
    errs = {"rho": rel_err(r, r_o), "T": rel_err(TT, T_o), "u_max": us}
    errs["u"] = max(float(np.abs(u[a] - u_o[a].numpy()).max()) for a in range(3)) / us
    nu_o = lbm.nusselt(ft, gt, op)[1].numpy()
    cs = _conv_scale(ft, gt, op)
    errs["nu_z_on_conv"] = float(np.abs(nu - nu_o).max()) / cs
    errs["conv_scale"] = cs
    return errs


def test_fp32_parity_on_a_convecting_state(lblib, cuda):
    """FP32 form against the oracle from a flowing state, element by element at the FP32
    tolerance of 1e-5 relative with no velocity floor: the 96^3 single-phase cell after 1000 FP64
    GPU steps (the buoyancy-driven adjustment of the initial state, |u| up to 6e-3), then 10 steps
    of each. rho, T, every velocity component on the largest |u|, and Nu(z) on the scale of its
    convective term <|rho U u_z|>/(kappa dT/nz)."""
    w = config.single_phase_cell(96)
    p = w.params
    rho, T = w.fields()
    lat = lb.Lattice(p, rho, T)
    lat.step(1000)
    f, g = lat.populations()
    lat.close()
    errs = _fp32_from(p, rho, T, f, g, 10)
    print("FP32 convecting-state errors:", errs)
    assert errs["u_max"] > 3e-3, errs
    assert max(errs["rho"], errs["T"], errs["u"]) < 1e-5, errs
    assert errs["nu_z_on_conv"] < 1e-5, errs


def test_fp32_parity_on_a_phase_separating_state(lblib, cuda):
    """FP32 form against the oracle from a phase-separating state (the 32 x 24 x 20 boiling cell
    after 300 FP64 GPU steps, interface flow |u| ~ 3e-3), 20 steps: rho and T within 1e-5. The
    velocity and the convective Nu term are compared relative (no floor) with the bound the
    arithmetic gives here: the spinodal dynamics amplify the FP32 rounding of the O(0.1) force
    sum of Eq. (9) over the 20 steps to an absolute velocity error ~1e-7 (measured 4.1e-5 of the
    largest |u|, 1.4e-5 of the convective Nu scale), so 1e-4 and 5e-5."""
    p, rho, T, f, g = _evolved_state()
    errs = _fp32_from(p, rho, T, f, g, 20)
    print("FP32 phase-separating-state errors:", errs)
    assert errs["u_max"] > 3e-3, errs
    assert max(errs["rho"], errs["T"]) < 1e-5, errs
    assert errs["u"] < 1e-4, errs
    assert errs["nu_z_on_conv"] < 5e-5, errs


def test_checkpoint_of_other_physics_parameters_is_refused(lblib, cuda, tmp_path):
    """lb_load refuses a checkpoint saved under other physics parameters (here tau_nu, then the
    wall temperature); other launch shapes and sampling periods load."""
    w = config.boiling_cell(12, nz=8, ny=8)
    rho, T = w.fields()
    a = lb.Lattice(w.params, rho, T)
    a.step(3)
    a.save(tmp_path / "a.bin")
    a.close()
    for field, value in (("tau_nu", 1.1), ("T_d", w.params.T_d * 1.01), ("forcing", lb.LB_FORCE_GUO)):
        q = lb.Params(**{**w.params.__dict__, field: value})
        b = lb.Lattice(q, rho, T)
        with pytest.raises(lb.LBError) as e:
            b.load(tmp_path / "a.bin")
        assert e.value.code == -5 and b.step_count == 0
        b.close()
    q = lb.Params(**{**w.params.__dict__, "tile_y": 4, "z_chunk": 3, "nu_every": 2})
    b = lb.Lattice(q, rho, T)
    b.load(tmp_path / "a.bin")
    assert b.step_count == 3
    b.close()


def test_fp16_local_references_against_the_oracle(lblib, cuda):
    """FP16 storage against local references on the boiling cell (phase separation, ragged tiles,
    several z chunks): rho, T and the populations within 2e-3 of the oracle after 30 steps, and
    Nu(z) within 2e-3 of its convective scale. Its rounding is of the non-equilibrium and
    velocity parts only, so it also stays within 1e-4 here (FP16 deviations from the global
    reference: ~1e-3)."""
    w = config.boiling_cell(40, nz=11, ny=19, precision=lb.LB_FP16_LOC)
    p = w.params
    p.tile_y, p.z_chunk = 8, 4
    rho, T = w.fields()
    lat = lb.Lattice(p, rho, T)
    lat.step(30)
    r, u, TT = lat.moments()
    f_g, g_g = lat.populations()
    nu = lat.nusselt()[1]
    lat.close()
    f, g, op, _ = oracle_run(p, rho, T, 30)
    r_o, u_o, T_o = lbm.moments_out(f, g, op)
    errs = {"rho": rel_err(r, r_o), "T": rel_err(TT, T_o), "f": rel_err(f_g, f), "g": rel_err(g_g, g),
            "nu_on_conv": float(np.abs(nu - lbm.nusselt(f, g, op)[1].numpy()).max()) / _conv_scale(f, g, op)}
    print("FP16 local-reference errors:", errs)
    assert max(errs["rho"], errs["T"], errs["f"], errs["g"]) < 1e-4, errs
    assert errs["nu_on_conv"] < 2e-3, errs


@pytest.mark.parametrize("prec", [lb.LB_FP16_LOC, lb.LB_FP32])
def test_set_populations_and_checkpoints_carry_the_references(lblib, cuda, prec, tmp_path):
    """With the local-reference storage the two reference slots are part of the state: a
    checkpoint round trip continues bitwise, and lb_set_populations of an exported state
    continues within the storage's rounding."""
    w = config.boiling_cell(20, nz=12, ny=10, precision=prec)
    rho, T = w.fields()
    a = lb.Lattice(w.params, rho, T)
    a.step(15)
    a.save(tmp_path / "c.bin")
    f, g = a.populations()
    a.step(10)
    fa, ga = a.populations()
    b = lb.Lattice(w.params, rho, T)
    b.load(tmp_path / "c.bin")
    b.step(10)
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    c = lb.Lattice(w.params, rho, T)
    c.set_populations(f, g)
    f1, g1 = c.populations()
    tol = 1e-6 if prec == lb.LB_FP32 else 2e-4
    assert rel_err(f1, f) < tol and rel_err(g1, g) < tol, (rel_err(f1, f), rel_err(g1, g))
    c.step(10)
    fc, gc = c.populations()
    assert rel_err(fc, fa) < 10 * tol and rel_err(gc, ga) < 10 * tol
    a.close(); b.close(); c.close()
