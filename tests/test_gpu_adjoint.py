"""Discrete adjoint (lb_adjoint_step) against the oracle's exact gradient (PyTorch autograd
through the plain FP64 steps) and against central finite differences on the GPU."""
import time

import numpy as np
import pytest
import torch

from oracle import lbm
from paper_1111_0905_gb300 import config, lb
from helpers import oracle_params

pytestmark = pytest.mark.gpu
DT = torch.float64


def _oracle_grad(p, rho, T, nsteps):
    op = oracle_params(p)
    Td = torch.tensor(p.T_d, dtype=DT, requires_grad=True)
    Tu = torch.tensor(p.T_u, dtype=DT, requires_grad=True)
    G = torch.tensor(p.G, dtype=DT, requires_grad=True)
    T0 = torch.from_numpy(T).clone().requires_grad_(True)
    q = lbm.Params(op.nx, op.ny, op.nz, op.tau_nu, op.tau_kappa, G, op.kappa, op.c_v, op.g_z, Td, Tu)
    J = lbm.time_averaged_nusselt(torch.from_numpy(rho), T0, q, nsteps)
    J.backward()
    return {"J": J.item(), "T_d": Td.grad.item(), "T_u": Tu.grad.item(), "G": G.grad.item(),
            "T0": T0.grad.numpy()}


@pytest.mark.parametrize("shape,nsteps,K", [((8, 6, 7), 12, 5), ((5, 4, 3), 9, 9), ((33, 3, 4), 6, 2)])
def test_adjoint_matches_oracle_gradient(lblib, cuda, shape, nsteps, K):
    nx, ny, nz = shape
    w = config.boiling_cell(nx, nz=nz, ny=ny)
    rho, T = w.fields()
    lat = lb.Lattice(w.params, rho, T)
    got = lat.adjoint(nsteps, K, grad_T0=True)
    lat.close()
    ref = _oracle_grad(w.params, rho, T, nsteps)
    assert abs(got["J"] - ref["J"]) <= 1e-11 * max(1.0, abs(ref["J"]))
    for k in ("T_d", "T_u", "G"):
        assert abs(got[k] - ref[k]) <= 1e-9 * max(1.0, abs(ref[k])), (k, got[k], ref[k])
    scale = np.abs(ref["T0"]).max()
    assert np.abs(got["T0"] - ref["T0"]).max() <= 1e-9 * scale


def _J_gpu(p, rho, T, nsteps):
    q = lb.Params(**{**p.__dict__, "nu_every": 1})
    lat = lb.Lattice(q, rho, T)
    lat.step(nsteps)
    J = lat.nusselt()[2]
    lat.close()
    return J


def test_adjoint_matches_central_differences_boiling_32(lblib, cuda):
    """The 32^3 boiling cell over 200 steps (checkpoints every 50): dJ/d(T_d, T_u, G) and a
    random direction of dJ/dT0 against central differences (h = 1e-6) within 1e-4."""
    w = config.boiling_cell(32)
    p = w.params
    rho, T = w.fields()
    N, K = 200, 50
    lat = lb.Lattice(p, rho, T)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    got = lat.adjoint(N, K, grad_T0=True)
    t_adj = time.perf_counter() - t0
    lat.close()
    lat = lb.Lattice(p, rho, T)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.step(N)
    lat.nusselt()
    t_fwd = time.perf_counter() - t0
    lat.close()
    print(f"adjoint {t_adj:.3f} s vs forward {t_fwd:.3f} s ({t_adj / t_fwd:.2f}x)")
    assert abs(got["J"] - _J_gpu(p, rho, T, N)) <= 1e-12 * abs(got["J"])
    h = 1e-6
    for k in ("T_d", "T_u", "G"):
        base = getattr(p, k)
        Jp = _J_gpu(lb.Params(**{**p.__dict__, k: base + h}), rho, T, N)
        Jm = _J_gpu(lb.Params(**{**p.__dict__, k: base - h}), rho, T, N)
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - got[k]) <= 1e-4 * max(abs(fd), 1e-3), (k, fd, got[k])
    v = np.random.default_rng(5).standard_normal(T.shape)
    fd = (_J_gpu(p, rho, T + h * v, N) - _J_gpu(p, rho, T - h * v, N)) / (2 * h)
    ad = float((got["T0"] * v).sum())
    assert abs(fd - ad) <= 1e-4 * max(abs(fd), 1e-3), (fd, ad)


def test_adjoint_of_the_fp32_form_matches_fp64(lblib, cuda):
    """The FP32 form (FP32 forward states, FP64 adjoint arithmetic and accumulation) gives the
    gradients of the FP64 form to the FP32 state error (1e-4 relative)."""
    w = config.boiling_cell(24)
    rho, T = w.fields()
    g64 = lb.Lattice(w.params, rho, T).adjoint(100, 25, grad_T0=True)
    p32 = lb.Params(**{**w.params.__dict__, "precision": lb.LB_FP32})
    g32 = lb.Lattice(p32, rho, T).adjoint(100, 25, grad_T0=True)
    assert abs(g32["J"] - g64["J"]) <= 1e-5 * abs(g64["J"])
    for k in ("T_d", "T_u", "G"):
        assert abs(g32[k] - g64[k]) <= 1e-4 * max(abs(g64[k]), 1e-3), (k, g32[k], g64[k])
    assert np.abs(g32["T0"] - g64["T0"]).max() <= 1e-4 * np.abs(g64["T0"]).max()


def test_adjoint_boiling_64_over_1000_steps(lblib, cuda):
    """The 64^3 adjoint configuration: 1000 steps, checkpoints every 50; dJ/d(T_d, T_u, G) and
    two random directions of dJ/dT0 (the initial temperature field) against central differences
    (h = 1e-6) within 1e-4, and the cost against the forward run.
    tau_nu = 1.25 and kappa = 0.15 (lambda = 0.3 in the g^eq positivity window) keep the
    phase-separating cell bounded for the whole run (tau_nu = 1 breaks down after ~500 steps)."""
    w = config.boiling_cell(64, kappa=0.15, tau_nu=1.25)
    p = w.params
    rho, T = w.fields()
    N, K = 1000, 50
    lat = lb.Lattice(p, rho, T)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    got = lat.adjoint(N, K, grad_T0=True)
    t_adj = time.perf_counter() - t0
    lat.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = _J_gpu(p, rho, T, N)
    t_fwd = time.perf_counter() - t0
    print(f"64^3 x 1000: J = {got['J']:.6f}, adjoint {t_adj:.2f} s vs forward {t_fwd:.2f} s "
          f"({t_adj / t_fwd:.2f}x), grads {got['T_d']:.6e} {got['T_u']:.6e} {got['G']:.6e}")
    assert abs(got["J"] - J) <= 1e-12 * abs(J)
    h = 1e-6
    for k in ("T_d", "T_u", "G"):
        base = getattr(p, k)
        fd = (_J_gpu(lb.Params(**{**p.__dict__, k: base + h}), rho, T, N)
              - _J_gpu(lb.Params(**{**p.__dict__, k: base - h}), rho, T, N)) / (2 * h)
        print(f"  {k}: adjoint {got[k]:.8e}, central difference {fd:.8e}")
        assert abs(fd - got[k]) <= 1e-4 * max(abs(fd), 1e-3), (k, fd, got[k])
    for seed in (64, 1000):
        v = np.random.default_rng(seed).standard_normal(T.shape)
        fd = (_J_gpu(p, rho, T + h * v, N) - _J_gpu(p, rho, T - h * v, N)) / (2 * h)
        ad = float((got["T0"] * v).sum())
        print(f"  T0 direction {seed}: adjoint {ad:.8e}, central difference {fd:.8e}")
        assert abs(fd - ad) <= 1e-4 * max(abs(fd), 1e-3), (seed, fd, ad)


@pytest.mark.parametrize("device", ["cpu", "cuda"])
def test_autograd_function_matches_the_oracle_gradient(lblib, cuda, device):
    """torch.autograd binding: J.backward() through NusseltObjective gives the oracle's exact
    gradient (PyTorch autograd through the plain FP64 steps) in T_d, T_u, G and T0, with the
    initial fields on the host or on the GPU; without gradients the forward pass (lb_step with
    a Nu sample per step) gives the same J."""
    from paper_1111_0905_gb300.autograd import nusselt_objective
    w = config.boiling_cell(8, nz=7, ny=6)
    rho, T = w.fields()
    nsteps, K = 12, 5
    Td = torch.tensor(w.params.T_d, dtype=DT, requires_grad=True)
    Tu = torch.tensor(w.params.T_u, dtype=DT, requires_grad=True)
    G = torch.tensor(w.params.G, dtype=DT, requires_grad=True)
    T0 = torch.from_numpy(T).to(device).requires_grad_(True)
    J = nusselt_objective(Td, Tu, G, T0, rho, w.params, nsteps, K)
    (2.0 * J).backward()
    ref = _oracle_grad(w.params, rho, T, nsteps)
    assert abs(J.item() - ref["J"]) <= 1e-11 * max(1.0, abs(ref["J"]))
    for k, t in (("T_d", Td), ("T_u", Tu), ("G", G)):
        assert abs(t.grad.item() - 2.0 * ref[k]) <= 1e-9 * max(1.0, abs(ref[k])), k
    assert T0.grad.device.type == device
    scale = np.abs(ref["T0"]).max()
    assert np.abs(T0.grad.cpu().numpy() - 2.0 * ref["T0"]).max() <= 2e-9 * scale
    J0 = nusselt_objective(Td.detach(), Tu.detach(), G.detach(), T0.detach(), rho, w.params, nsteps, K)
    assert not J0.requires_grad
    assert abs(J0.item() - J.item()) <= 1e-12 * max(1.0, abs(J.item()))


def test_adjoint_of_the_fp32_form_matches_its_central_differences(lblib, cuda):
    """The 64^3 adjoint configuration in the FP32 form (FP32 forward states, FP64 reverse sweep):
    dJ/d(T_d, T_u, G) against central differences of the FP32 form's own J within 1e-4, and a
    random direction of dJ/dT0 within 1e-2.
    Step sizes come from the FP32 noise floor. J of 1000 FP32 steps carries rounding noise of
    about 1e-7 of J, which a central difference divides by 2h. Measured on this cell, the
    difference at h = 1e-6 |p| is off by 3e-3 to 1e-2 (noise), at 1e-4 |p| by 3e-5 to 6e-5,
    and at 1e-3 |p| by 1e-4 (truncation: the FP64 form's own difference is off by 8.7e-5 there).
    So h = 3e-4 |p| for the scalars. For the T0 direction (unit normal entries on every node) the
    noise is larger: at h = 1e-3 the difference is off by 3.5e-3, against 6e-5 truncation in FP64."""
    w = config.boiling_cell(64, kappa=0.15, tau_nu=1.25)
    p = lb.Params(**{**w.params.__dict__, "precision": lb.LB_FP32})
    rho, T = w.fields()
    N, K = 1000, 50
    lat = lb.Lattice(p, rho, T)
    got = lat.adjoint(N, K, grad_T0=True)
    lat.close()
    # J of the reverse sweep sums the FP64 images of the FP32 states; the forward run's J sums
    # the same states with FP32 warp sums: equal to the FP32 rounding of the sums
    assert abs(got["J"] - _J_gpu(p, rho, T, N)) <= 1e-6 * abs(got["J"])
    for k in ("T_d", "T_u", "G"):
        base = getattr(p, k)
        h = 3e-4 * abs(base)
        fd = (_J_gpu(lb.Params(**{**p.__dict__, k: base + h}), rho, T, N)
              - _J_gpu(lb.Params(**{**p.__dict__, k: base - h}), rho, T, N)) / (2 * h)
        print(f"  FP32 {k}: adjoint {got[k]:.8e}, central difference {fd:.8e} ({fd / got[k] - 1:+.2e})")
        assert abs(fd - got[k]) <= 1e-4 * abs(fd), (k, fd, got[k])
    v = np.random.default_rng(64).standard_normal(T.shape)
    h = 1e-3
    fd = (_J_gpu(p, rho, T + h * v, N) - _J_gpu(p, rho, T - h * v, N)) / (2 * h)
    ad = float((got["T0"] * v).sum())
    print(f"  FP32 T0 direction: adjoint {ad:.8e}, central difference {fd:.8e} ({fd / ad - 1:+.2e})")
    assert abs(fd - ad) <= 1e-2 * abs(fd), (fd, ad)


@pytest.mark.parametrize("prec,tol", [(lb.LB_FP16_LOC, 2e-4), (lb.LB_FP16_DEV, 5e-3)])
def test_adjoint_of_the_16bit_forms_against_fp64(lblib, cuda, prec, tol):
    """The 16-bit storage forms' adjoint (FP64 reverse sweep around their own forward states,
    checkpoints holding every stored slot, the local-reference form's two reference slots included)
    gives the FP64 form's gradients within its state error: J and dJ/d(T_d, T_u, G) over 100 steps
    of the 24^3 boiling cell, checkpoints every 25. Measured largest relative differences: 1.2e-5
    (local references) and 5.2e-4 (deviations from the global reference), both on dJ/dT_d."""
    w = config.boiling_cell(24)
    rho, T = w.fields()
    g64 = lb.Lattice(w.params, rho, T).adjoint(100, 25)
    q = lb.Params(**{**w.params.__dict__, "precision": prec})
    g16 = lb.Lattice(q, rho, T).adjoint(100, 25)
    errs = {k: abs(g16[k] - g64[k]) / max(abs(g64[k]), 1e-3) for k in ("J", "T_d", "T_u", "G")}
    print("16-bit adjoint", prec, errs)
    assert max(errs.values()) <= tol, errs


@pytest.mark.parametrize("prec", [lb.LB_FP64, lb.LB_FP32])
def test_adjoint_segment_length_from_free_memory(lblib, cuda, prec):
    """checkpoint_every = 0 keeps every state's fields when they fit (they do for 100 steps of the
    24^3 cell): the same J and gradients as checkpoint_every = nsteps, bit for bit, and as the
    checkpointed run with segments of 25 steps to rounding; a negative length is refused."""
    w = config.boiling_cell(24)
    rho, T = w.fields()
    q = lb.Params(**{**w.params.__dict__, "precision": prec})
    auto = lb.Lattice(q, rho, T).adjoint(100, 0, grad_T0=True)
    full = lb.Lattice(q, rho, T).adjoint(100, 100, grad_T0=True)
    seg = lb.Lattice(q, rho, T).adjoint(100, 25, grad_T0=True)
    for k in ("J", "T_d", "T_u", "G"):
        assert auto[k] == full[k], (k, auto[k], full[k])
        assert abs(auto[k] - seg[k]) <= 1e-12 * max(abs(seg[k]), 1e-3), (k, auto[k], seg[k])
    assert np.array_equal(auto["T0"], full["T0"])
    lat = lb.Lattice(q, rho, T)
    with pytest.raises(lb.LBError) as e:
        lat.adjoint(10, -1)
    assert e.value.code == -1
    lat.close()
