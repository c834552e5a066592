"""Parity of the statistics entry points (lb_profiles, lb_histogram_T_rho, lb_heat_flux_pdf,
lb_structure_functions) with the oracle's, on the same evolved boiling cell."""
import numpy as np
import pytest
import torch

from oracle import analysis, lbm
from paper_1111_0905_gb300 import config, lb
from helpers import oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def evolved(lblib, cuda):
    w = config.boiling_cell(24, nz=20, ny=16)
    rho, T = w.fields()
    lat = lb.Lattice(w.params, rho, T)
    lat.step(60)
    f, g, op, _ = oracle_run(w.params, rho, T, 60)
    yield lat, f, g, op
    lat.close()


def test_profiles_match_oracle(evolved):
    lat, f, g, op = evolved
    r_z, T_z, PD_z = lat.profiles()
    r_o, T_o, PD_o = (t.numpy() for t in analysis.profiles(f, g, op))
    assert np.abs(r_z - r_o).max() <= 1e-12 * np.abs(r_o).max()
    assert np.abs(T_z - T_o).max() <= 1e-12 * np.abs(T_o).max()
    assert np.abs(PD_z - PD_o).max() <= 1e-10 * max(np.abs(PD_o).max(), 1e-12)


def test_histogram_matches_oracle(evolved):
    lat, f, g, op = evolved
    rho_o, u_o, T_o = (x.numpy() if hasattr(x, "numpy") else x for x in lbm.moments_out(f, g, op))
    rng_T, rng_r, nT, nr = (0.30, 0.38), (0.4, 2.0), 16, 24
    got = lat.histogram_T_rho(2, 18, nT, rng_T, nr, rng_r)
    ref = analysis.histogram_T_rho(rho_o, T_o, 2, 18, nT, rng_T, nr, rng_r)
    # values within 1e-10 (relative) of a bin edge may fall on either side between the two codes
    Tn = (T_o[2:18] - rng_T[0]) / (rng_T[1] - rng_T[0]) * nT
    rn = (rho_o[2:18] - rng_r[0]) / (rng_r[1] - rng_r[0]) * nr
    near = int(np.sum((np.abs(Tn - np.round(Tn)) < 1e-9) | (np.abs(rn - np.round(rn)) < 1e-9)))
    assert got.sum() == ref.sum() or near > 0
    assert int(np.abs(got.astype(np.int64) - ref.astype(np.int64)).sum()) <= 2 * near
    assert ref.sum() > 0.9 * 16 * 16 * 24


def test_structure_functions_match_oracle(evolved):
    lat, f, g, op = evolved
    rho_o, u_o, T_o = lbm.moments_out(f, g, op)
    got = lat.structure_functions(10, 3, 17)
    ref = analysis.structure_functions(u_o[2].numpy(), T_o.numpy(), 10, 3, 17)
    for k in ref:
        assert np.abs(got[k] - ref[k]).max() <= 1e-10 * np.abs(ref[k]).max(), k


def test_heat_flux_pdf_matches_oracle(evolved):
    """lb_heat_flux_pdf: counts of q = rho U u_z in 20 bins over the bulk planes and its mean and
    variance, against the oracle's."""
    lat, f, g, op = evolved
    _, (n_o, mean_o, var_o) = analysis.heat_flux_pdf(f, g, op, 3, 17, 1, (-1.0, 1.0))
    sd = var_o ** 0.5
    rng = (mean_o - 3 * sd, mean_o + 3 * sd)
    got, (n, mean, var) = lat.heat_flux_pdf(3, 17, 20, rng)
    ref, _ = analysis.heat_flux_pdf(f, g, op, 3, 17, 20, rng)
    assert n == n_o == 14 * 16 * 24
    assert abs(mean - mean_o) <= 1e-10 * sd and abs(var / var_o - 1) <= 1e-10
    diff = int(np.abs(got.astype(np.int64) - ref.astype(np.int64)).sum())
    assert diff <= 2 and ref.sum() > 0.8 * n, (got, ref)


def test_statistics_of_the_local_reference_storage(lblib, cuda):
    """The statistics entry points read the state through the same moments pass in every storage
    form: on the FP16 local-reference form of the evolved cell the rho(z) and T(z) profiles equal
    the FP64 form's within 5e-5 of their scale (measured 2.3e-6 and 1.2e-6), and the P div(u)
    profile within 5e-4 (measured 3.7e-5)."""
    w = config.boiling_cell(24, nz=20, ny=16)
    rho, T = w.fields()
    out = {}
    for prec in (lb.LB_FP64, lb.LB_FP16_LOC):
        q = lb.Params(**{**w.params.__dict__, "precision": prec})
        lat = lb.Lattice(q, rho, T)
        lat.step(60)
        out[prec] = lat.profiles()
        lat.close()
    errs = [float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-12))
            for a, b in zip(out[lb.LB_FP16_LOC], out[lb.LB_FP64])]
    print("local-reference profiles (rho, T, P div u):", errs)
    assert errs[0] <= 5e-5 and errs[1] <= 5e-5
    # P div(u) is a difference of velocities whose FP16 rounding is absolute: its own bound
    assert errs[2] <= 5e-4
