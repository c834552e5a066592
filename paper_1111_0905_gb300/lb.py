"""Python binding of the C ABI in include/lb.h (ctypes; argument marshalling only).

Every step of the method runs in the sm_103a kernels of libthermal_lbm.so. PyTorch is used
only for device memory (CUDA tensors whose pointers are passed through) and for the current
CUDA stream. There is no CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field, fields
from pathlib import Path

import numpy as np

LB_FP64, LB_FP32, LB_BF16_DEV, LB_FP16_DEV, LB_FP16_LOC = 0, 1, 2, 3, 4
PRECISIONS = {"f64": LB_FP64, "f32": LB_FP32, "bf16dev": LB_BF16_DEV, "fp16dev": LB_FP16_DEV,
              "fp16loc": LB_FP16_LOC}
STORAGE_BYTES = {LB_FP64: 8, LB_FP32: 4, LB_BF16_DEV: 2, LB_FP16_DEV: 2, LB_FP16_LOC: 2}
# stored values per lattice and node (the local-reference storage adds two reference slots)
STORED_SLOTS = {LB_FP64: 19, LB_FP32: 19, LB_BF16_DEV: 19, LB_FP16_DEV: 19, LB_FP16_LOC: 21}
LB_FORCE_SHIFT, LB_FORCE_GUO = 0, 1     # scheme variants (include/lb.h); 0 = the paper's
LB_PSI_EXP, LB_PSI_VDW = 0, 1
Q = 19

_LIB_PATH = Path(__file__).resolve().parent / "libthermal_lbm.so"
_lib = None

# Names declared in include/lb.h.
EXPORTS = ("lb_init", "lb_step", "lb_adjoint_step", "lb_profiles", "lb_histogram_T_rho",
           "lb_structure_functions", "lb_moments", "lb_nusselt", "lb_populations", "lb_diagnostics",
           "lb_save", "lb_load", "lb_step_count", "lb_free", "lb_strerror", "lb_last_error",
           "lb_nusselt_fields_noalloc", "lb_launch_info", "lb_heat_flux_pdf", "lb_set_populations",
           "lb_stream_bound")
NOALLOC_MAX_NZ = 8192


class LbParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("tau_nu", ctypes.c_double), ("tau_kappa", ctypes.c_double), ("G", ctypes.c_double),
        ("kappa", ctypes.c_double), ("c_v", ctypes.c_double), ("g_z", ctypes.c_double),
        ("T_d", ctypes.c_double), ("T_u", ctypes.c_double),
        ("rho0", ctypes.c_double), ("T0", ctypes.c_double),
        ("precision", ctypes.c_int), ("nu_every", ctypes.c_int), ("check_every", ctypes.c_int),
        ("tile_y", ctypes.c_int), ("z_chunk", ctypes.c_int),
        ("forcing", ctypes.c_int), ("psi_kind", ctypes.c_int),
        ("vdw_a", ctypes.c_double), ("vdw_b", ctypes.c_double), ("vdw_T", ctypes.c_double),
    ]


@dataclass
class Params:
    """Mirror of lb_params (include/lb.h)."""
    nx: int
    ny: int
    nz: int
    tau_nu: float
    tau_kappa: float
    G: float
    kappa: float
    c_v: float = 1.0
    g_z: float = 0.0
    T_d: float = 1.0 / 3.0
    T_u: float = 1.0 / 3.0
    rho0: float = 0.0
    T0: float = 0.0
    precision: int = LB_FP64
    nu_every: int = 0
    check_every: int = 0
    tile_y: int = 0
    z_chunk: int = 0
    forcing: int = 0          # LB_FORCE_SHIFT (the paper) or LB_FORCE_GUO
    psi_kind: int = 0         # LB_PSI_EXP (the paper) or LB_PSI_VDW
    vdw_a: float = 5.0 / 42.0
    vdw_b: float = 2.0 / 21.0
    vdw_T: float = 1.0 / 3.0

    def to_c(self) -> LbParams:
        return LbParams(*[getattr(self, f.name) for f in fields(self)])

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz


class LBError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def library_path() -> Path:
    return _LIB_PATH


def load_library():
    """Load libthermal_lbm.so (built by paper_1111_0905_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_1111_0905_gb300.build.build()")
    lib = ctypes.CDLL(str(_LIB_PATH))
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    DP = ctypes.POINTER(ctypes.c_double)
    lib.lb_init.argtypes = [ctypes.POINTER(LbParams), P, P, I, P, ctypes.POINTER(P)]
    lib.lb_init.restype = I
    lib.lb_step.argtypes = [P, LL]
    lib.lb_step.restype = I
    lib.lb_moments.argtypes = [P, P, P, P, P, P, I]
    lib.lb_moments.restype = I
    lib.lb_nusselt.argtypes = [P, DP, P, DP]
    lib.lb_nusselt.restype = I
    lib.lb_populations.argtypes = [P, P, P, I]
    lib.lb_populations.restype = I
    lib.lb_set_populations.argtypes = [P, P, P, I]
    lib.lb_set_populations.restype = I
    lib.lb_diagnostics.argtypes = [P, P]
    lib.lb_diagnostics.restype = I
    lib.lb_save.argtypes = [P, ctypes.c_char_p]
    lib.lb_save.restype = I
    lib.lb_load.argtypes = [P, ctypes.c_char_p]
    lib.lb_load.restype = I
    lib.lb_step_count.argtypes = [P]
    lib.lb_step_count.restype = LL
    lib.lb_free.argtypes = [P]
    lib.lb_free.restype = None
    lib.lb_strerror.argtypes = [I]
    lib.lb_strerror.restype = ctypes.c_char_p
    lib.lb_last_error.argtypes = [P]
    lib.lb_last_error.restype = ctypes.c_char_p
    lib.lb_profiles.argtypes = [P, P, P, P]
    lib.lb_profiles.restype = I
    lib.lb_histogram_T_rho.argtypes = [P, I, I, I, D, D, I, D, D, P]
    lib.lb_histogram_T_rho.restype = I
    lib.lb_structure_functions.argtypes = [P, I, I, I, P, P, P, P]
    lib.lb_structure_functions.restype = I
    lib.lb_adjoint_step.argtypes = [P, LL, I, DP, DP, DP, DP, P]
    lib.lb_adjoint_step.restype = I
    lib.lb_nusselt_fields_noalloc.argtypes = [P, P, P, I, I, I, D, D, D, D, D, P, P]
    lib.lb_nusselt_fields_noalloc.restype = I
    lib.lb_launch_info.argtypes = [P, P]
    lib.lb_launch_info.restype = I
    lib.lb_heat_flux_pdf.argtypes = [P, I, I, I, D, D, P, P]
    lib.lb_heat_flux_pdf.restype = I
    lib.lb_stream_bound.argtypes = [I, P, P, P, P, I, I, I, I, ctypes.POINTER(I), P]
    lib.lb_stream_bound.restype = I
    _lib = lib
    return lib


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _host_f64(a, n: int) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)
    if a.size != n:
        raise ValueError(f"field has {a.size} entries, grid has {n}")
    return a


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:  # pragma: no cover
        pass
    return None


def _check_device_f64(name: str, t, min_numel: int, exact: bool) -> None:
    """A CUDA float64 contiguous tensor of (at least, unless exact) min_numel elements."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a CUDA float64 tensor, got {type(t).__name__}")
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA float64 tensor "
                         f"(dtype {t.dtype}, device {t.device}, contiguous {t.is_contiguous()})")
    if (t.numel() != min_numel) if exact else (t.numel() < min_numel):
        raise ValueError(f"{name} has {t.numel()} elements, needs {'' if exact else 'at least '}{min_numel}")


def nusselt_fields_noalloc(params: Params, rho, uz, T, nu_out, stream=None) -> None:
    """lb_nusselt_fields_noalloc on CUDA tensors (inputs [nz, ny, nx] float64; nu_out nz + 1
    float64); enqueued on the current stream, allocates no device memory. The tensors are checked
    here (dtype, device, contiguity, sizes) before any pointer reaches the device; the call
    supports the paper's pseudopotential only (params.psi_kind = LB_PSI_EXP)."""
    if params.psi_kind != LB_PSI_EXP:
        raise ValueError("lb_nusselt_fields_noalloc uses the internal energy of psi = exp(-1/rho) only")
    lib = load_library()
    if params.nx >= 1 and params.ny >= 1 and 1 <= params.nz <= NOALLOC_MAX_NZ:
        n = params.nx * params.ny * params.nz
        for name, t in (("rho", rho), ("uz", uz), ("T", T)):
            _check_device_f64(name, t, n, exact=True)
        _check_device_f64("nu_out", nu_out, params.nz + 1, exact=False)
    # sizes outside the entry point's limits go through unchecked: it rejects them (LB_EINVAL)
    # before touching any pointer
    st = _current_stream() if stream is None else stream
    rc = lib.lb_nusselt_fields_noalloc(_ptr(rho), _ptr(uz), _ptr(T), params.nx, params.ny, params.nz,
                                       params.kappa, params.G, params.c_v, params.T_d, params.T_u,
                                       _ptr(nu_out), st)
    if rc != 0:
        raise LBError(rc, "lb_nusselt_fields_noalloc", lib.lb_strerror(rc).decode())


def stream_bound(f_in, g_in, f_out, g_out, shape, ctas_per_sm: int = 0, stream=None) -> int:
    """lb_stream_bound on four contiguous CUDA tensors of one 4- or 2-byte dtype and 19 * nx*ny*nz
    elements each (shape = (nz, ny, nx)): the step's streaming loads and stores without its
    arithmetic, a bandwidth yardstick. Enqueued on the current stream; returns the kernel's
    occupancy limit in CTAs per SM."""
    import torch
    lib = load_library()
    nz, ny, nx = shape
    n = 19 * nx * ny * nz
    ts = (f_in, g_in, f_out, g_out)
    for t in ts:
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise ValueError("stream_bound takes contiguous CUDA tensors")
        if t.dtype != f_in.dtype or t.element_size() not in (2, 4) or t.numel() != n:
            raise ValueError(f"stream_bound: tensors of one 2- or 4-byte dtype with {n} elements each")
    out = ctypes.c_int(0)
    st = _current_stream() if stream is None else stream
    rc = lib.lb_stream_bound(f_in.element_size(), *[_ptr(t) for t in ts], nx, ny, nz, int(ctas_per_sm),
                             ctypes.byref(out), st)
    if rc != 0:
        raise LBError(rc, "lb_stream_bound", lib.lb_strerror(rc).decode())
    return out.value


class Lattice:
    """A context of the C ABI: lb_init on construction, lb_free on close()."""

    def __init__(self, params: Params, rho, T, stream=None):
        self.lib = load_library()
        self.params = params
        self.shape = (params.nz, params.ny, params.nx)
        self._ctx = ctypes.c_void_p()
        n = params.N
        on_device = (not isinstance(rho, np.ndarray)) and bool(rho.is_cuda)
        if not isinstance(rho, np.ndarray):
            import torch
            if rho.dtype != torch.float64 or T.dtype != torch.float64:
                raise ValueError("fields must be float64")
            rho, T = rho.contiguous(), T.contiguous()
            if rho.numel() != n or T.numel() != n or bool(T.is_cuda) != on_device:
                raise ValueError("field size or placement does not match")
            self._keep = (rho, T)
        else:
            rho, T = _host_f64(rho, n), _host_f64(T, n)
        self.stream = _current_stream() if stream is None else stream
        cp = params.to_c()
        rc = self.lib.lb_init(ctypes.byref(cp), _ptr(rho), _ptr(T), int(on_device), self.stream,
                              ctypes.byref(self._ctx))
        if rc != 0:
            raise LBError(rc, "lb_init", self.lib.lb_strerror(rc).decode())
        self._keep = None

    # -- helpers ----------------------------------------------------------------------------
    def _check(self, rc: int, where: str):
        if rc != 0:
            msg = self.lib.lb_last_error(self._ctx).decode() or self.lib.lb_strerror(rc).decode()
            raise LBError(rc, where, msg)

    @property
    def ctx(self):
        if not self._ctx:
            raise RuntimeError("lattice is closed")
        return self._ctx

    # -- C ABI ------------------------------------------------------------------------------
    def step(self, n: int = 1):
        self._check(self.lib.lb_step(self.ctx, int(n)), "lb_step")

    @property
    def step_count(self) -> int:
        return int(self.lib.lb_step_count(self.ctx))

    def launch_info(self) -> dict:
        """lb_launch_info: grid, threads and shared memory per CTA, resident CTAs per SM, registers."""
        out = (ctypes.c_int * 6)()
        self._check(self.lib.lb_launch_info(self.ctx, out), "lb_launch_info")
        return {"grid": [out[0], out[1]], "threads_per_cta": out[2], "smem_bytes": out[3],
                "ctas_per_sm": out[4], "registers": out[5]}

    def adjoint(self, nsteps: int, checkpoint_every: int = 50, grad_T0: bool = False) -> dict:
        """lb_adjoint_step: J = time-averaged Nu over the next nsteps steps and dJ/d(T_d, T_u, G)
        (and dJ/dT0 as [nz, ny, nx] if grad_T0; requires step 0). checkpoint_every = 0: the longest
        segment that fits in free device memory (every state's fields when they fit)."""
        J, dTd, dTu, dG = (ctypes.c_double() for _ in range(4))
        dT0 = np.empty(self.shape, dtype=np.float64) if grad_T0 else None
        self._check(self.lib.lb_adjoint_step(self.ctx, int(nsteps), int(checkpoint_every),
                                             ctypes.byref(J), ctypes.byref(dTd), ctypes.byref(dTu),
                                             ctypes.byref(dG), _ptr(dT0)), "lb_adjoint_step")
        return {"J": J.value, "T_d": dTd.value, "T_u": dTu.value, "G": dG.value, "T0": dT0}

    def profiles(self):
        """(rho_z, T_z, PdivU_z): per-plane means of rho, T and P div(u)."""
        out = [np.empty(self.params.nz, dtype=np.float64) for _ in range(3)]
        self._check(self.lib.lb_profiles(self.ctx, *[_ptr(o) for o in out]), "lb_profiles")
        return tuple(out)

    def histogram_T_rho(self, z_lo, z_hi, nT, T_range, nrho, rho_range):
        """uint64 counts [nT, nrho] of (T, rho) over planes [z_lo, z_hi)."""
        counts = np.zeros((nT, nrho), dtype=np.uint64)
        self._check(self.lib.lb_histogram_T_rho(self.ctx, z_lo, z_hi, nT, T_range[0], T_range[1],
                                                nrho, rho_range[0], rho_range[1], _ptr(counts)),
                    "lb_histogram_T_rho")
        return counts

    def heat_flux_pdf(self, z_lo, z_hi, nbins, q_range):
        """(uint64 counts [nbins], (n, mean, variance)) of q = rho U u_z over planes [z_lo, z_hi)."""
        counts = np.zeros(nbins, dtype=np.uint64)
        stats = np.zeros(3, dtype=np.float64)
        self._check(self.lib.lb_heat_flux_pdf(self.ctx, z_lo, z_hi, nbins, q_range[0], q_range[1],
                                              _ptr(counts), _ptr(stats)), "lb_heat_flux_pdf")
        return counts, (float(stats[0]), float(stats[1]), float(stats[2]))

    def structure_functions(self, rmax, z_lo, z_hi):
        """dict of S2/S4 of u_z and T for horizontal increments r = 1..rmax."""
        out = [np.empty(rmax, dtype=np.float64) for _ in range(4)]
        self._check(self.lib.lb_structure_functions(self.ctx, rmax, z_lo, z_hi, *[_ptr(o) for o in out]),
                    "lb_structure_functions")
        return {"S2_uz": out[0], "S4_uz": out[1], "S2_T": out[2], "S4_T": out[3]}

    def moments(self, device: bool = False):
        """(rho, (ux, uy, uz), T) as numpy [nz, ny, nx] arrays, or torch CUDA tensors if device."""
        if device:
            import torch
            outs = [torch.empty(self.shape, dtype=torch.float64, device="cuda") for _ in range(5)]
        else:
            outs = [np.empty(self.shape, dtype=np.float64) for _ in range(5)]
        self._check(self.lib.lb_moments(self.ctx, *[_ptr(o) for o in outs], int(device)), "lb_moments")
        return outs[0], (outs[1], outs[2], outs[3]), outs[4]

    def moments_into(self, rho=None, ux=None, uy=None, uz=None, T=None, device: bool = False):
        """lb_moments into caller-owned buffers (numpy/pinned host tensors, or CUDA tensors)."""
        self._check(self.lib.lb_moments(self.ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(uz), _ptr(T),
                                        int(device)), "lb_moments")

    def nusselt(self):
        """(Nu_mean, Nu(z) [nz], time average of the accumulated Nu_mean samples or NaN)."""
        mean = ctypes.c_double()
        avg = ctypes.c_double()
        nu_z = np.empty(self.params.nz, dtype=np.float64)
        self._check(self.lib.lb_nusselt(self.ctx, ctypes.byref(mean), _ptr(nu_z), ctypes.byref(avg)),
                    "lb_nusselt")
        return mean.value, nu_z, avg.value

    def populations(self, device: bool = False):
        """Pre-collision (f, g), each [19, nz, ny, nx] float64."""
        shape = (Q,) + self.shape
        if device:
            import torch
            f = torch.empty(shape, dtype=torch.float64, device="cuda")
            g = torch.empty(shape, dtype=torch.float64, device="cuda")
        else:
            f = np.empty(shape, dtype=np.float64)
            g = np.empty(shape, dtype=np.float64)
        self._check(self.lib.lb_populations(self.ctx, _ptr(f), _ptr(g), int(device)), "lb_populations")
        return f, g

    def set_populations(self, f, g) -> None:
        """lb_set_populations: replace the state by pre-collision (f, g), each [19, nz, ny, nx]
        float64 (numpy / host tensors, or CUDA tensors)."""
        n = Q * self.params.N
        if isinstance(f, np.ndarray) or isinstance(g, np.ndarray):
            f, g = _host_f64(f, n), _host_f64(g, n)
            on_device = False
        else:
            import torch
            if f.dtype != torch.float64 or g.dtype != torch.float64:
                raise ValueError("populations must be float64")
            if f.numel() != n or g.numel() != n or bool(f.is_cuda) != bool(g.is_cuda):
                raise ValueError("population size or placement does not match")
            f, g = f.contiguous(), g.contiguous()
            on_device = bool(f.is_cuda)
        self._check(self.lib.lb_set_populations(self.ctx, _ptr(f), _ptr(g), int(on_device)),
                    "lb_set_populations")

    def diagnostics(self) -> dict:
        out = np.empty(5, dtype=np.float64)
        self._check(self.lib.lb_diagnostics(self.ctx, _ptr(out)), "lb_diagnostics")
        return {"min_rho": out[0], "min_T": out[1], "nonfinite": int(out[2]), "mass": out[3],
                "energy": out[4]}

    def save(self, path):
        self._check(self.lib.lb_save(self.ctx, str(path).encode()), "lb_save")

    def load(self, path):
        self._check(self.lib.lb_load(self.ctx, str(path).encode()), "lb_load")

    def close(self):
        if self._ctx:
            self.lib.lb_free(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
