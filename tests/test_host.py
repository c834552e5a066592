"""Host-side checks that need no GPU: the seeded generator, the workload helper against the
oracle's EOS, the C-ABI library's exports and the binding's struct layout."""
import ctypes
import math
import subprocess
import sys
import textwrap
from pathlib import Path

import numpy as np
import pytest

from paper_1111_0905_gb300 import config, lb, synthetic
from oracle import eos

ROOT = Path(__file__).resolve().parent.parent


def test_splitmix64_reference_outputs():
    """First outputs of SplitMix64 with seed 0 (the published reference sequence)."""
    got = [int(x) for x in synthetic.splitmix64(5, seed=0)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
                   0xF88BB8A8724C81EC, 0x1B39896A51A8749B]


def test_uniform_noise_range_and_order():
    u = synthetic.uniform_pm1(100000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01
    f = synthetic.noise_field(4, 3, 2)
    assert f.shape == (2, 3, 4)
    assert np.array_equal(f.reshape(-1), synthetic.uniform_pm1(24))
    assert np.array_equal(synthetic.uniform_pm1(5, offset=3), synthetic.uniform_pm1(8)[3:])


def test_workload_helper_matches_oracle_thermodynamics():
    for rho in (0.57, 1.5, 1.789, 2.3):
        b, cp = config.beta_cp(rho, config.T_M)
        assert abs(b - eos.beta(rho, config.T_M, config.G_DEFAULT)) < 1e-12 * abs(b)
        assert abs(cp - eos.c_p(rho, config.T_M, config.G_DEFAULT)) < 1e-12 * cp
    _, Tc, _ = eos.critical_point(config.G_DEFAULT)
    assert abs(Tc - config.T_C) < 1e-15 and abs(config.T_M - 1.0 / 3.0) < 1e-15
    w = config.single_phase_cell(128)
    p = w.params
    nu = config.T_M * (p.tau_nu - 0.5)
    Ra = eos.rayleigh(-p.g_z, 2.30, config.T_M, config.G_DEFAULT, 128, p.T_d - p.T_u, p.kappa, nu)
    Ra_max = config.max_rayleigh(128, p.T_d - p.T_u, p.kappa, nu, 2.30, config.T_M)
    assert abs(Ra / (0.5 * Ra_max) - 1) < 1e-9
    chi = p.kappa / (2.30 * eos.c_p(2.30, config.T_M, config.G_DEFAULT))
    assert abs(nu / chi - 9.0) < 1e-9


def test_library_builds_and_exports_every_declared_symbol(lblib):
    header = (ROOT / "include" / "lb.h").read_text()
    declared = set()
    for name in lb.EXPORTS:
        assert f"{name}(" in header
        declared.add(name)
    import re
    in_header = set(re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(lb_\w+)\(", header, re.M))
    assert in_header == declared
    out = subprocess.run(["nm", "-D", "--defined-only", str(lb.library_path())], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert declared <= exported
    for name in declared:
        assert hasattr(lblib, name)
    assert lblib.lb_strerror(-4).decode().startswith("non-physical")
    assert lblib.lb_step_count(None) == -1
    assert lblib.lb_launch_info(None, None) == -1   # LB_EINVAL, no device needed


def test_lb_params_layout_matches_the_c_header(tmp_path):
    """Offsets and size of lb_params as the C compiler lays it out equal the ctypes mirror."""
    fields = [f[0] for f in lb.LbParams._fields_]
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"lb.h\"\nint main(void){\n"
    src += f'printf("%zu\\n", sizeof(lb_params));\n'
    for f in fields:
        src += f'printf("%zu\\n", offsetof(lb_params, {f}));\n'
    src += "return 0;}\n"
    c = tmp_path / "layout.c"
    c.write_text(src)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), str(c), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(lb.LbParams)
    for f, off in zip(fields, vals[1:]):
        assert getattr(lb.LbParams, f).offset == off, f


def test_init_rejects_invalid_parameters_without_a_gpu(lblib):
    """Parameter validation happens before any device call."""
    w = config.boiling_cell(4)
    rho, T = w.fields()
    bad = dict(tau_nu=0.5)
    p = w.params
    for field, val in [("tau_nu", 0.5), ("tau_kappa", 0.4), ("kappa", 0.0), ("tile_y", 5), ("precision", 7)]:
        q = lb.Params(**{**p.__dict__, field: val})
        with pytest.raises(lb.LBError) as e:
            lb.Lattice(q, rho, T, stream=None)
        assert e.value.code == -1


def test_init_rejects_degenerate_and_oversized_grids_without_a_gpu(lblib):
    """lb_init's own checks, called through the C ABI with small dummy arrays (every check runs
    before the fields are read or any device call is made): empty grids, grids whose 19 N
    population offsets overflow 32 bits (the 512^3 workload is inside), the 16-row tile for FP64,
    negative chunk/sampling/check periods, unknown variants, a van der Waals psi without an
    attractive coupling, non-positive wall temperatures and a non-finite coupling."""
    import ctypes
    import dataclasses
    import math
    w = config.boiling_cell(4)
    p = w.params
    rho, T = w.fields()
    cases = [dict(nx=0), dict(ny=0), dict(nz=0), dict(nx=700, ny=700, nz=700),
             dict(nx=1024, ny=1024, nz=230), dict(precision=lb.LB_FP64, tile_y=16),
             dict(z_chunk=-1), dict(nu_every=-2), dict(check_every=-1), dict(forcing=2),
             dict(psi_kind=3), dict(psi_kind=lb.LB_PSI_VDW, G=0.5), dict(T_d=0.0), dict(T_u=-1.0),
             dict(G=math.inf), dict(c_v=0.0)]
    for kw in cases:
        cp = dataclasses.replace(p, **kw).to_c()
        out = ctypes.c_void_p()
        rc = lblib.lb_init(ctypes.byref(cp), rho.ctypes.data_as(ctypes.c_void_p),
                           T.ctypes.data_as(ctypes.c_void_p), 0, None, ctypes.byref(out))
        assert rc == -1, (kw, rc)
        assert not out.value
    # the 512^3 workload itself passes the size checks (19 N < 2^32)
    assert 19 * 512 ** 3 < 2 ** 32 <= 19 * 700 ** 3


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the FP64 oracle as the reference arm) prints one JSON line
    with the benchmark's metric, unit and config, impl = reference, a cpu_baseline and an e2e
    entry with no host-device bytes."""
    import json
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, check=True, cwd=ROOT,
                         timeout=600).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_noalloc_binding_refuses_host_tensors_and_the_vdw_psi_without_a_gpu(lblib):
    """The binding of lb_nusselt_fields_noalloc refuses, before any call into the library,
    numpy arrays, CPU tensors, float32 tensors and a context of the van der Waals psi (whose
    internal energy the entry point does not implement)."""
    import torch
    p = config.boiling_cell(4).params
    n = p.nx * p.ny * p.nz
    host = torch.zeros(n, dtype=torch.float64)
    out = torch.zeros(p.nz + 1, dtype=torch.float64)
    for bad in (np.zeros(n), host, host.float()):
        with pytest.raises(ValueError):
            lb.nusselt_fields_noalloc(p, bad, host, host, out)
    vdw = lb.Params(**{**p.__dict__, "psi_kind": lb.LB_PSI_VDW})
    with pytest.raises(ValueError, match="exp"):
        lb.nusselt_fields_noalloc(vdw, host, host, host, out)


def test_boiling_block_equals_the_same_block_of_the_full_cell():
    """The block generator (used for the oracle's samples of the 512^3 cell) draws the same values
    as the full-cell recipe at those nodes, including blocks that touch the grid's far corner."""
    r, T = synthetic.boiling_fields(20, 12, 9, 1.5, 0.35, 0.31)
    for (x0, y0, z0, sx, sy, sz) in ((3, 2, 4, 7, 5, 3), (0, 0, 0, 20, 12, 9), (13, 7, 6, 7, 5, 3)):
        b, Tb = synthetic.boiling_block(20, 12, 9, x0, y0, z0, sx, sy, sz, 1.5, 0.35, 0.31)
        assert np.array_equal(b, r[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx])
        assert np.array_equal(Tb, T[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx])


def test_stream_bound_rejects_invalid_arguments_without_a_gpu(lblib):
    """lb_stream_bound checks its arguments before any device call: null lattices, element sizes
    other than 2 and 4, empty grids, 19 N offsets beyond 32 bits, a negative CTA count; the binding
    refuses host tensors."""
    import ctypes
    import torch
    fake = ctypes.c_void_p(256)
    ok = (4, fake, fake, fake, fake, 8, 8, 8, 1, None, None)
    for i, bad in [(0, 3), (0, 8), (1, None), (4, None), (5, 0), (7, -1), (8, -1)]:
        args = list(ok)
        args[i] = bad
        assert lblib.lb_stream_bound(*args) == -1, (i, bad)
    assert lblib.lb_stream_bound(4, fake, fake, fake, fake, 1024, 1024, 1024, 0, None, None) == -1
    host = torch.zeros(19 * 8, dtype=torch.float32)
    with pytest.raises(ValueError):
        lb.stream_bound(host, host, host, host, (2, 2, 2))
