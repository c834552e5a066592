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
    # a null pointer is refused by the entry point itself (the binding refuses it earlier)
    n = p.nx * p.ny * p.nz
    f = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(p.nz + 1, dtype=torch.float64, device="cuda")
    rc = lblib.lb_nusselt_fields_noalloc(None, f.data_ptr(), f.data_ptr(), p.nx, p.ny, p.nz, p.kappa,
                                         p.G, p.c_v, p.T_d, p.T_u, out.data_ptr(), None)
    assert rc == -1
    with pytest.raises(ValueError):
        lb.nusselt_fields_noalloc(p, None, f, f, out)


def test_noalloc_binding_refuses_tensors_the_kernels_would_misread(lblib, cuda):
    """Wrong dtype, a transposed view, short inputs or a short output never reach the device."""
    p = config.boiling_cell(8, nz=6, ny=5).params
    shape = (p.nz, p.ny, p.nx)
    good = torch.ones(shape, dtype=torch.float64, device="cuda")
    out = torch.zeros(p.nz + 1, dtype=torch.float64, device="cuda")
    bad_inputs = [good.float(), good.transpose(1, 2), good.reshape(-1)[:-1], good.cpu()]
    for b in bad_inputs:
        with pytest.raises(ValueError):
            lb.nusselt_fields_noalloc(p, b, good, good, out)
        with pytest.raises(ValueError):
            lb.nusselt_fields_noalloc(p, good, good, b, out)
    with pytest.raises(ValueError):
        lb.nusselt_fields_noalloc(p, good, good, good, out[:-1])
    vdw = lb.Params(**{**p.__dict__, "psi_kind": lb.LB_PSI_VDW})
    with pytest.raises(ValueError):
        lb.nusselt_fields_noalloc(vdw, good, good, good, out)
    torch.cuda.synchronize()
