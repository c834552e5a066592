"""The 16-bit storage forms over long horizons of the paper-geometry boiling cell, against the
FP64 GPU step of the same cell (max over the field relative to the field's scale). FP16 against
local references holds rho and T within 2e-3; the forms that store deviations from the global
reference state are recorded beside it, with the bound each meets on that horizon."""
import numpy as np
import pytest
import torch

from paper_1111_0905_gb300 import config, lb

pytestmark = pytest.mark.gpu


def _run(w, prec, steps):
    p = lb.Params(**{**w.params.__dict__, "precision": prec})
    rho, T = w.fields()
    lat = lb.Lattice(p, torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
    m0 = lat.diagnostics()["mass"]
    lat.step(steps)
    r, u, TT = lat.moments(device=True)
    nu = lat.nusselt()[0]
    d = lat.diagnostics()
    lat.close()
    return r, u, TT, nu, d["mass"] / m0 - 1.0, d["nonfinite"]


@pytest.mark.parametrize("n,steps", [(64, 2000), (128, 3000)])
def test_16bit_storage_over_a_boiling_horizon(lblib, cuda, n, steps):
    w = config.paper_scale_cell(n)
    r0, u0, T0, nu0, dm0, _ = _run(w, lb.LB_FP64, steps)
    res = {}
    for name, prec in (("fp16loc", lb.LB_FP16_LOC), ("fp16dev", lb.LB_FP16_DEV), ("bf16dev", lb.LB_BF16_DEV),
                       ("f32", lb.LB_FP32)):
        r, u, TT, nu, dm, bad = _run(w, prec, steps)
        res[name] = {"rho": float((r - r0).abs().max() / r0.abs().max()),
                     "T": float((TT - T0).abs().max() / T0.abs().max()),
                     "nu": nu, "nu64": nu0, "mass_change": dm, "nonfinite": bad}
        print(f"{n}^3 x {steps} {name}: {res[name]}")
    assert res["fp16loc"]["nonfinite"] == 0
    assert res["fp16loc"]["rho"] < 2e-3 and res["fp16loc"]["T"] < 2e-3, res
    assert res["f32"]["rho"] < 1e-4 and res["f32"]["T"] < 1e-5, res
    # the documented boundary of the global-reference 16-bit forms: over these boiling horizons
    # neither holds 2e-3 on rho (measured 6.6e-3 / 8.2e-3 for FP16, 0.22 / 0.29 for BF16)
    assert res["fp16dev"]["rho"] > 2e-3 and res["bf16dev"]["rho"] > 2e-3, res


def test_16bit_storage_over_the_single_phase_horizon(lblib, cuda):
    """The 64^3 single-phase convection cell over 2000 steps: FP16 deviations and FP16 against
    local references both hold rho and T within 2e-3 of the FP64 step (the other side of the
    FP16 deviations' boundary); BF16 deviations do not."""
    w = config.single_phase_cell(64)
    r0, u0, T0, nu0, dm0, _ = _run(w, lb.LB_FP64, 2000)
    res = {}
    for name, prec in (("fp16loc", lb.LB_FP16_LOC), ("fp16dev", lb.LB_FP16_DEV), ("bf16dev", lb.LB_BF16_DEV)):
        r, u, TT, nu, dm, bad = _run(w, prec, 2000)
        res[name] = {"rho": float((r - r0).abs().max() / r0.abs().max()),
                     "T": float((TT - T0).abs().max() / T0.abs().max()), "nu": nu, "nu64": nu0}
        print(f"single-phase 64^3 x 2000 {name}: {res[name]}")
    for name in ("fp16loc", "fp16dev"):
        assert res[name]["rho"] < 2e-3 and res[name]["T"] < 2e-3, res
    assert res["bf16dev"]["rho"] > 2e-3 or res["bf16dev"]["T"] > 2e-3, res
