"""lb_nusselt_fields_noalloc: the Nusselt profile for callers that cannot allocate device memory
(an application whose own pool allocator owns all device memory, or a latency-critical loop that
cannot take cudaMalloc's implicit synchronisation). It must match lb_nusselt on the same state,
call after call, while using only its fixed file-scope device array."""
import numpy as np
import pytest
import torch

from paper_1111_0905_gb300 import config, lb

pytestmark = pytest.mark.gpu


def test_noalloc_nusselt_matches_lb_nusselt_on_two_calls(lblib, cuda):
    w = config.boiling_cell(24, nz=20, ny=16)
    p = w.params
    rho, T = w.fields()
    lat = lb.Lattice(p, rho, T)
    shape = (p.nz, p.ny, p.nx)
    for call in range(2):
        lat.step(7)
        r = torch.empty(shape, dtype=torch.float64, device="cuda")
        uz = torch.empty(shape, dtype=torch.float64, device="cuda")
        TT = torch.empty(shape, dtype=torch.float64, device="cuda")
        lat.moments_into(rho=r, uz=uz, T=TT, device=True)
        out = torch.full((p.nz + 1,), float("nan"), dtype=torch.float64, device="cuda")
        lb.nusselt_fields_noalloc(p, r, uz, TT, out)
        torch.cuda.synchronize()
        nu_mean, nu_z, _ = lat.nusselt()
        got = out.cpu().numpy()
        scale = max(1.0, float(np.abs(nu_z).max()))
        assert np.all(np.isfinite(got))
        assert np.abs(got[: p.nz] - nu_z).max() <= 1e-12 * scale, (call, got[: p.nz], nu_z)
        assert abs(got[p.nz] - nu_mean) <= 1e-12 * scale
    lat.close()


def test_noalloc_rejects_sizes_beyond_its_array(lblib, cuda):
    p = config.boiling_cell(4).params
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    big = lb.Params(**{**p.__dict__, "nz": lb.NOALLOC_MAX_NZ + 1})
    with pytest.raises(lb.LBError) as e:
        lb.nusselt_fields_noalloc(big, x, x, x, x)
    assert e.value.code == -1
    with pytest.raises(lb.LBError):
        lb.nusselt_fields_noalloc(p, None, x, x, x)
