"""Python binding of libnufft3d: argument marshalling over the C ABI only.

Every step of the projector runs in the library's CUDA kernels; this module
checks shapes, dtypes and devices of torch tensors, passes their device
pointers and the current CUDA stream to the C entry points, and turns status
codes into exceptions.  There is no CPU fallback: without the built library
every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libnufft3d.so")

EXPORTS = (
    "nufft3d_plan_create",
    "nufft3d_forward",
    "nufft3d_adjoint",
    "nufft3d_workspace_bytes",
    "nufft3d_plan_sync_status",
    "nufft3d_plan_destroy",
    "nufft3d_error_string",
    "nufft3d_plan_info",
    "nufft3d_plan_tune",
    "nufft3d_plan_set_timing",
    "nufft3d_plan_set_wait_limit",
    "nufft3d_plan_stage_times",
    "nufft3d_adjoint_noalloc",
    "nufft3d_batch_create",
    "nufft3d_batch_size",
    "nufft3d_batch_item",
    "nufft3d_batch_forward_adjoint",
    "nufft3d_batch_invalidate",
    "nufft3d_batch_set_grouping",
    "nufft3d_batch_destroy",
    "nufft3d_fourier_slice_weights",
    "nufft3d_polar_resample",
    "nufft3d_polar_nufft_create",
    "nufft3d_polar_nufft_info",
    "nufft3d_polar_nufft_prepare",
    "nufft3d_polar_nufft_gather",
    "nufft3d_polar_nufft_resample",
    "nufft3d_polar_nufft_destroy",
    "nufft3d_grangeat_create",
    "nufft3d_grangeat_info",
    "nufft3d_grangeat_run",
    "nufft3d_grangeat_destroy",
    "nufft3d_fp32_fma_peak",
    "nufft3d_host_pipeline_create",
    "nufft3d_host_forward_adjoint",
    "nufft3d_host_pipeline_sync",
    "nufft3d_host_pipeline_destroy",
)

FWD_STAGES = ("x_pass", "y_pass", "z_pass", "gather", "line_dft")
ADJ_STAGES = ("line_dft", "grid_clear", "spread", "z_pass", "y_pass", "x_pass")

GRID_DTYPES = {"c64": 0, "complex64": 0, "bf16": 1, "fp16": 2, "f16": 2}


class Params(ctypes.Structure):
    """Mirror of nufft3d_params (include/nufft3d.h)."""

    _fields_ = [
        ("n", ctypes.c_int),
        ("k", ctypes.c_int),
        ("j", ctypes.c_int),
        ("table_oversamp", ctypes.c_int),
        ("n_dirs", ctypes.c_int),
        ("dirs", ctypes.POINTER(ctypes.c_double)),
        ("m", ctypes.c_int),
        ("omega", ctypes.POINTER(ctypes.c_double)),
        ("weight", ctypes.POINTER(ctypes.c_float)),
        ("grid_dtype", ctypes.c_int),
        ("complex_volume", ctypes.c_int),
        ("do_line_fft", ctypes.c_int),
        ("keep_duplicates", ctypes.c_int),
        ("exact_coeffs", ctypes.c_int),
        ("line_weight", ctypes.POINTER(ctypes.c_float)),
    ]


class NufftError(RuntimeError):
    def __init__(self, what: str, status: int):
        super().__init__(f"{what}: {error_string(status)} (status {status})")
        self.status = status


_LIB = None


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libnufft3d.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(the projector has no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, ip, i = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int
    lib.nufft3d_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params), vp]
    lib.nufft3d_forward.argtypes = [vp, vp, vp, vp]
    lib.nufft3d_adjoint.argtypes = [vp, vp, vp, vp]
    lib.nufft3d_adjoint_noalloc.argtypes = [vp, vp, vp, vp]
    lib.nufft3d_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params), i, vp]
    lib.nufft3d_batch_size.argtypes = [vp, ip]
    lib.nufft3d_batch_item.argtypes = [vp, i, ctypes.POINTER(vp)]
    lib.nufft3d_batch_forward_adjoint.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.nufft3d_batch_invalidate.argtypes = [vp]
    lib.nufft3d_batch_set_grouping.argtypes = [vp, i]
    lib.nufft3d_batch_destroy.argtypes = [vp]
    lib.nufft3d_workspace_bytes.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)]
    lib.nufft3d_plan_sync_status.argtypes = [vp, ip]
    lib.nufft3d_plan_destroy.argtypes = [vp]
    lib.nufft3d_error_string.argtypes = [i]
    lib.nufft3d_error_string.restype = ctypes.c_char_p
    lib.nufft3d_plan_info.argtypes = [vp, ip]
    lib.nufft3d_plan_tune.argtypes = [vp, i, i, i, i, vp]
    fp = ctypes.POINTER(ctypes.c_float)
    lib.nufft3d_plan_set_timing.argtypes = [vp, i]
    lib.nufft3d_plan_set_wait_limit.argtypes = [vp, i]
    lib.nufft3d_plan_stage_times.argtypes = [vp, fp, fp, ip]
    lib.nufft3d_fourier_slice_weights.argtypes = [i, i, ctypes.c_double, i, fp, fp]
    lib.nufft3d_polar_resample.argtypes = [vp, i, i, i, vp, ctypes.c_longlong, i, vp, vp]
    lib.nufft3d_polar_nufft_create.argtypes = [ctypes.POINTER(vp), i, i, i, i]
    lib.nufft3d_polar_nufft_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]
    lib.nufft3d_polar_nufft_prepare.argtypes = [vp, vp, vp]
    lib.nufft3d_polar_nufft_gather.argtypes = [vp, vp, ctypes.c_longlong, vp, vp]
    lib.nufft3d_polar_nufft_resample.argtypes = [vp, vp, vp, ctypes.c_longlong, vp, vp]
    lib.nufft3d_polar_nufft_destroy.argtypes = [vp]
    lib.nufft3d_grangeat_create.argtypes = [ctypes.POINTER(vp), i, i, i, i, ctypes.POINTER(ctypes.c_double), i]
    lib.nufft3d_grangeat_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.POINTER(ctypes.c_double)]
    lib.nufft3d_grangeat_run.argtypes = [vp, vp, vp, vp, i, vp, vp]
    lib.nufft3d_grangeat_destroy.argtypes = [vp]
    lib.nufft3d_fp32_fma_peak.argtypes = [ctypes.POINTER(ctypes.c_double), ip, vp]
    lib.nufft3d_host_pipeline_create.argtypes = [vp, ctypes.POINTER(vp)]
    lib.nufft3d_host_forward_adjoint.argtypes = [vp, vp, vp, vp]
    lib.nufft3d_host_pipeline_sync.argtypes = [vp]
    lib.nufft3d_host_pipeline_destroy.argtypes = [vp]
    for name in EXPORTS:
        if name != "nufft3d_error_string":
            getattr(lib, name).restype = ctypes.c_int
    if path == LIB_PATH:
        _LIB = lib
    return lib


def error_string(status: int) -> str:
    try:
        return load_library().nufft3d_error_string(int(status)).decode()
    except Exception:
        return "unknown"


def _check(rc: int, what: str):
    if rc != 0:
        raise NufftError(what, rc)


def make_params(n, dirs, m=0, k=0, j=6, table_oversamp=1024, omega=None, weight=None, grid_dtype="c64",
                complex_volume=False, do_line_fft=True, keep_duplicates=False, exact_coeffs=False,
                line_weight=None):
    """Build a Params struct plus the host arrays it points to (kept alive by the caller)."""
    dirs = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    keep = [dirs]
    p = Params()
    p.n = int(n)
    p.k = int(k)
    p.j = int(j)
    p.table_oversamp = int(table_oversamp)
    p.n_dirs = int(dirs.shape[0])
    p.dirs = dirs.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.m = int(m)
    if omega is not None:
        om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
        keep.append(om)
        p.omega = om.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if weight is not None:
        w = np.asarray(weight, dtype=np.complex64)
        wf = np.ascontiguousarray(np.stack([w.real, w.imag], axis=-1).astype(np.float32))
        keep.append(wf)
        p.weight = wf.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    p.grid_dtype = GRID_DTYPES[grid_dtype] if isinstance(grid_dtype, str) else int(grid_dtype)
    p.complex_volume = 1 if complex_volume else 0
    p.do_line_fft = 1 if do_line_fft else 0
    p.keep_duplicates = 1 if keep_duplicates else 0
    p.exact_coeffs = int(exact_coeffs)
    if line_weight is not None:
        lw = np.ascontiguousarray(np.asarray(line_weight, dtype=np.float32).reshape(-1))
        if lw.shape[0] != p.n_dirs:
            raise ValueError(f"line_weight needs {p.n_dirs} values, got {lw.shape[0]}")
        keep.append(lw)
        p.line_weight = lw.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    return p, keep


def fourier_slice_weights(n_az: int, n_pol: int, cone_half_angle: float, m: int):
    """Radial (M,) complex64 and per-line (n_az n_pol,) float32 weights with which
    the adjoint of plane integrals over the umbrella directions of Eq. 2.1 is the
    direct Fourier-slice reconstruction (nufft3d_fourier_slice_weights).
    cone_half_angle in radians."""
    rw = np.zeros(2 * int(m), dtype=np.float32)
    lw = np.zeros(int(n_az) * int(n_pol), dtype=np.float32)
    _check(load_library().nufft3d_fourier_slice_weights(
        int(n_az), int(n_pol), float(cone_half_angle), int(m),
        rw.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), lw.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
        "nufft3d_fourier_slice_weights")
    return (rw[0::2] + 1j * rw[1::2]).astype(np.complex64), lw


def polar_resample(grid, targets, J: int = 3, out=None, stream=None):
    """Direct resampling of the polar Radon grid (Eq. 2.15; nufft3d_polar_resample).
    grid: complex64 CUDA tensor (n_phi, n_theta, n_s), e.g. a plan's (D, M)
    lines viewed as (n_az, n_pol, M); targets: float32 CUDA tensor (P, 3) of
    (u_s, u_theta, u_phi) in grid-index units.  Returns complex64 (P,)."""
    import torch

    if grid.dtype != torch.complex64 or grid.dim() != 3 or not grid.is_cuda or not grid.is_contiguous():
        raise ValueError("grid must be a contiguous complex64 CUDA tensor (n_phi, n_theta, n_s)")
    if targets.dtype != torch.float32 or targets.dim() != 2 or targets.shape[1] != 3 or not targets.is_cuda \
            or not targets.is_contiguous() or targets.device != grid.device:
        raise ValueError("targets must be a contiguous float32 (P, 3) tensor on the grid's device")
    n = targets.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.complex64, device=grid.device)
    elif out.dtype != torch.complex64 or out.shape != (n,) or not out.is_contiguous() or out.device != grid.device:
        raise ValueError("out must be a contiguous complex64 (P,) tensor on the grid's device")
    n_phi, n_theta, n_s = grid.shape
    _check(load_library().nufft3d_polar_resample(
        ctypes.c_void_p(grid.data_ptr()), int(n_phi), int(n_theta), int(n_s), ctypes.c_void_p(targets.data_ptr()),
        int(n), int(J), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream, grid.device)), "nufft3d_polar_resample")
    return out


class PolarNufft:
    """NUFFT-based resampling of the polar Radon grid (Eqs. 2.8-2.11;
    nufft3d_polar_nufft_*): x~ ~= T_sparse F P F^-1 x on a (n_phi, n_theta,
    n_s) complex64 grid, all axes periodic, K = 2n per axis, J taps.  The
    plan holds the oversampled spectrum of the last prepared grid."""

    def __init__(self, n_phi: int, n_theta: int, n_s: int, J: int = 6):
        self.lib = load_library()
        h = ctypes.c_void_p()
        _check(self.lib.nufft3d_polar_nufft_create(ctypes.byref(h), int(n_phi), int(n_theta), int(n_s), int(J)),
               "nufft3d_polar_nufft_create")
        self._handle = h
        self.shape = (int(n_phi), int(n_theta), int(n_s))
        self.J = int(J)

    def info(self):
        wb = ctypes.c_longlong(0)
        fe = ctypes.c_double(0.0)
        _check(self.lib.nufft3d_polar_nufft_info(self._handle, ctypes.byref(wb), ctypes.byref(fe)),
               "nufft3d_polar_nufft_info")
        return {"workspace_bytes": int(wb.value), "fit_error": float(fe.value)}

    def _grid(self, grid):
        import torch

        if grid.dtype != torch.complex64 or tuple(grid.shape) != self.shape or not grid.is_cuda \
                or not grid.is_contiguous():
            raise ValueError(f"grid must be a contiguous complex64 CUDA tensor of shape {self.shape}")
        return grid

    def _targets_out(self, targets, out, device):
        import torch

        if targets.dtype != torch.float32 or targets.dim() != 2 or targets.shape[1] != 3 or not targets.is_cuda \
                or not targets.is_contiguous() or targets.device != device:
            raise ValueError("targets must be a contiguous float32 (P, 3) CUDA tensor on the grid's device")
        n = targets.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.complex64, device=device)
        elif out.dtype != torch.complex64 or tuple(out.shape) != (n,) or not out.is_contiguous() \
                or out.device != device:
            raise ValueError("out must be a contiguous complex64 (P,) tensor on the targets' device")
        return n, out

    def prepare(self, grid, stream=None):
        """F P F^-1 of grid into the plan's oversampled spectrum."""
        g = self._grid(grid)
        _check(self.lib.nufft3d_polar_nufft_prepare(self._handle, ctypes.c_void_p(g.data_ptr()),
                                                    _stream_ptr(stream, g.device)), "nufft3d_polar_nufft_prepare")

    def gather(self, targets, out=None, stream=None):
        """T_sparse of the last prepared spectrum at targets (P, 3) = (u_s, u_theta, u_phi)."""
        n, out = self._targets_out(targets, out, targets.device)
        _check(self.lib.nufft3d_polar_nufft_gather(self._handle, ctypes.c_void_p(targets.data_ptr()), int(n),
                                                   ctypes.c_void_p(out.data_ptr()),
                                                   _stream_ptr(stream, targets.device)), "nufft3d_polar_nufft_gather")
        return out

    def resample(self, grid, targets, out=None, stream=None):
        g = self._grid(grid)
        n, out = self._targets_out(targets, out, g.device)
        _check(self.lib.nufft3d_polar_nufft_resample(self._handle, ctypes.c_void_p(g.data_ptr()),
                                                     ctypes.c_void_p(targets.data_ptr()), int(n),
                                                     ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream, g.device)),
               "nufft3d_polar_nufft_resample")
        return out

    def close(self):
        if getattr(self, "_handle", None):
            self.lib.nufft3d_polar_nufft_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ReverseGrangeat:
    """Per-view reverse Grangeat step (Sec. 2.2.2, C3a-C3d; nufft3d_grangeat_*):
    umbrella subsets y (V, L, M) with post-weights (V, L, M) and pre-weights
    (V, N, N) to detector images (V, N, N), complex64, on the GPU."""

    def __init__(self, N: int, angles, M: int, J: int = 5, max_views: int = 64):
        self.lib = load_library()
        a = np.ascontiguousarray(np.asarray(angles, dtype=np.float64).reshape(-1))
        h = ctypes.c_void_p()
        _check(self.lib.nufft3d_grangeat_create(ctypes.byref(h), int(N), int(a.size), int(M), int(J),
                                                a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(max_views)),
               "nufft3d_grangeat_create")
        self._handle = h
        self.N, self.L, self.M, self.J = int(N), int(a.size), int(M), int(J)

    def info(self):
        wb = ctypes.c_longlong(0)
        nnz = ctypes.c_longlong(0)
        fe = ctypes.c_double(0.0)
        _check(self.lib.nufft3d_grangeat_info(self._handle, ctypes.byref(wb), ctypes.byref(nnz), ctypes.byref(fe)),
               "nufft3d_grangeat_info")
        return {"workspace_bytes": int(wb.value), "nnz": int(nnz.value), "fit_error": float(fe.value)}

    def run(self, y, w_post, w_pre, out=None, stream=None):
        import torch

        V = y.shape[0] if y.dim() == 3 else -1
        if y.dtype != torch.complex64 or tuple(y.shape) != (V, self.L, self.M) or not y.is_cuda \
                or not y.is_contiguous():
            raise ValueError(f"y must be a contiguous complex64 CUDA tensor (V, {self.L}, {self.M})")
        dev = y.device
        if w_post.dtype != torch.float32 or tuple(w_post.shape) != (V, self.L, self.M) or \
                not w_post.is_contiguous() or w_post.device != dev:
            raise ValueError("w_post must be a contiguous float32 tensor shaped like y on its device")
        if w_pre.dtype != torch.float32 or tuple(w_pre.shape) != (V, self.N, self.N) or \
                not w_pre.is_contiguous() or w_pre.device != dev:
            raise ValueError(f"w_pre must be a contiguous float32 (V, {self.N}, {self.N}) tensor on y's device")
        if out is None:
            out = torch.empty((V, self.N, self.N), dtype=torch.complex64, device=dev)
        elif out.dtype != torch.complex64 or tuple(out.shape) != (V, self.N, self.N) or not out.is_contiguous() \
                or out.device != dev:
            raise ValueError(f"out must be a contiguous complex64 (V, {self.N}, {self.N}) tensor on y's device")
        _check(self.lib.nufft3d_grangeat_run(self._handle, ctypes.c_void_p(y.data_ptr()),
                                             ctypes.c_void_p(w_post.data_ptr()), ctypes.c_void_p(w_pre.data_ptr()),
                                             int(V), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream, dev)),
               "nufft3d_grangeat_run")
        return out

    def close(self):
        if getattr(self, "_handle", None):
            self.lib.nufft3d_grangeat_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workspace_bytes(**kw) -> int:
    p, keep = make_params(**kw)
    out = ctypes.c_size_t(0)
    _check(load_library().nufft3d_workspace_bytes(ctypes.byref(p), ctypes.byref(out)), "nufft3d_workspace_bytes")
    return int(out.value)


def _stream_ptr(stream, device):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """A projector plan: N^3 volume <-> D radial lines of M samples.

    forward(x): x (N, N, N) float32 (or complex64 with complex_volume) on the
    plan's CUDA device -> (D, M) complex64 plane integrals (or raw Fourier
    samples with do_line_fft=False).  adjoint(y): the transpose.
    """

    def __init__(self, n, dirs, m=0, k=0, j=6, table_oversamp=1024, omega=None, weight=None,
                 grid_dtype="c64", complex_volume=False, do_line_fft=True, keep_duplicates=False,
                 exact_coeffs=False, line_weight=None, device=None, stream=None, _handle=None):
        import torch

        self.lib = load_library()
        self._owned = _handle is None
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        p, keep = make_params(n, dirs, m, k, j, table_oversamp, omega, weight, grid_dtype, complex_volume,
                              do_line_fft, keep_duplicates, exact_coeffs, line_weight)
        self.n = int(n)
        self.n_dirs = p.n_dirs
        self.m = int(m) if m else 2 * int(n)
        self.k = int(k) if k else 2 * int(n)
        self.j = int(j)
        self.complex_volume = bool(complex_volume)
        self.do_line_fft = bool(do_line_fft)
        self.grid_dtype = str(grid_dtype)
        self.exact_coeffs = bool(exact_coeffs)
        self._handle = ctypes.c_void_p()
        if _handle is not None:
            self._handle = _handle
        else:
            with torch.cuda.device(self.device):
                _check(self.lib.nufft3d_plan_create(ctypes.byref(self._handle), ctypes.byref(p),
                                                    _stream_ptr(stream, self.device)), "nufft3d_plan_create")
        del keep

    # -- shapes ------------------------------------------------------------
    @property
    def n_points(self) -> int:
        return self.n_dirs * self.m

    @property
    def vol_dtype(self):
        import torch

        return torch.complex64 if self.complex_volume else torch.float32

    def _check_tensor(self, t, shape, dtype, name):
        import torch

        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if t.device != self.device:
            raise ValueError(f"{name} must be on {self.device}, got {t.device}")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")

    # -- operators ---------------------------------------------------------
    def forward(self, vol, out=None, stream=None):
        import torch

        self._check_tensor(vol, (self.n,) * 3, self.vol_dtype, "vol")
        if out is None:
            out = torch.empty((self.n_dirs, self.m), dtype=torch.complex64, device=self.device)
        self._check_tensor(out, (self.n_dirs, self.m), torch.complex64, "out")
        _check(self.lib.nufft3d_forward(self._handle, ctypes.c_void_p(vol.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream, self.device)),
               "nufft3d_forward")
        return out

    def adjoint(self, lines, out=None, stream=None):
        import torch

        self._check_tensor(lines, (self.n_dirs, self.m), torch.complex64, "lines")
        if out is None:
            out = torch.empty((self.n,) * 3, dtype=self.vol_dtype, device=self.device)
        self._check_tensor(out, (self.n,) * 3, self.vol_dtype, "out")
        _check(self.lib.nufft3d_adjoint(self._handle, ctypes.c_void_p(lines.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream, self.device)),
               "nufft3d_adjoint")
        return out

    def sync_status(self) -> int:
        v = ctypes.c_int(0)
        _check(self.lib.nufft3d_plan_sync_status(self._handle, ctypes.byref(v)), "nufft3d_plan_sync_status")
        return int(v.value)

    def info(self) -> dict:
        a = (ctypes.c_int * 12)()
        _check(self.lib.nufft3d_plan_info(self._handle, a), "nufft3d_plan_info")
        keys = ("tile", "tiles_per_axis", "subproblems", "gather_variant", "spread_variant",
                "points_per_subproblem", "nonempty_tiles", "max_tile_points", "evaluated_points",
                "merged_line_pairs", "exact_coeffs")
        d = dict(zip(keys, list(a)))
        d["coeff_fit_error"] = a[11] * 1e-12
        return d

    def tune(self, gather_variant=-1, spread_variant=-1, points_per_subproblem=0, tile_edge=0, stream=None):
        """Pick the gather (0-7) and spread (0-4) variants, points per subproblem and tile edge (-1 / 0 keep)."""
        _check(self.lib.nufft3d_plan_tune(self._handle, int(gather_variant), int(spread_variant),
                                          int(points_per_subproblem), int(tile_edge),
                                          _stream_ptr(stream, self.device)), "nufft3d_plan_tune")

    def set_wait_limit(self, first_wait_polls: int):
        """Testing hook: cap the first wait on each TMA tile copy (variant 8) at
        this many polls (0 gives up at once); a negative value restores the default."""
        _check(self.lib.nufft3d_plan_set_wait_limit(self._handle, int(first_wait_polls)),
               "nufft3d_plan_set_wait_limit")

    def set_timing(self, max_calls: int):
        """Arm per-stage CUDA-event timing of the next max_calls calls."""
        _check(self.lib.nufft3d_plan_set_timing(self._handle, int(max_calls)), "nufft3d_plan_set_timing")

    def stage_times(self) -> dict:
        """Summed per-stage milliseconds of the recorded calls (synchronises)."""
        f = (ctypes.c_float * len(FWD_STAGES))()
        a = (ctypes.c_float * len(ADJ_STAGES))()
        c = (ctypes.c_int * 2)()
        _check(self.lib.nufft3d_plan_stage_times(self._handle, f, a, c), "nufft3d_plan_stage_times")
        return {"forward": dict(zip(FWD_STAGES, list(f))), "adjoint": dict(zip(ADJ_STAGES, list(a))),
                "forward_calls": c[0], "adjoint_calls": c[1]}

    def close(self):
        if getattr(self, "_handle", None) is not None and self._handle.value:
            if getattr(self, "_owned", True):
                self.lib.nufft3d_plan_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class _Project(torch.autograd.Function):
        """y = A x with the hand-written adjoint kernel as backward: dL/dx = A^H g
        (real part for a real volume)."""

        @staticmethod
        def forward(ctx, x, plan):
            ctx.plan = plan
            return plan.forward(x.contiguous())

        @staticmethod
        def backward(ctx, g):
            gx = ctx.plan.adjoint(g.contiguous().to(torch.complex64))
            return gx, None

    return _Project


_PROJECT = None


def project(x, plan: Plan):
    """Differentiable forward projection: plan.forward with plan.adjoint as backward."""
    global _PROJECT
    if _PROJECT is None:
        _PROJECT = _autograd_function()
    return _PROJECT.apply(x, plan)


class Batch:
    """Many independent problems of mixed sizes: one plan per item, forward +
    adjoint of every item replayed as one CUDA graph launch.

    items: list of dicts with the Plan keyword arguments (n, dirs, m, k, j,
    table_oversamp, grid_dtype, complex_volume, ...).
    """

    def __init__(self, items, stream=None, device=None):
        import torch

        self.lib = load_library()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        built = [make_params(**it) for it in items]
        arr = (Params * len(items))(*[b[0] for b in built])
        self._handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.nufft3d_batch_create(ctypes.byref(self._handle), arr, len(items),
                                                 _stream_ptr(stream, self.device)), "nufft3d_batch_create")
        self.items = []
        for idx, it in enumerate(items):
            h = ctypes.c_void_p()
            _check(self.lib.nufft3d_batch_item(self._handle, idx, ctypes.byref(h)), "nufft3d_batch_item")
            kw = dict(it)
            self.items.append(Plan(device=self.device, _handle=h, **kw))
        del built

    def __len__(self):
        return len(self.items)

    def invalidate(self):
        """Capture the graph again on the next call (after re-tuning item plans)."""
        _check(self.lib.nufft3d_batch_invalidate(self._handle), "nufft3d_batch_invalidate")

    def set_grouping(self, on: bool):
        """Grouped interpolation launches across items of equal N, K, J (default on)."""
        _check(self.lib.nufft3d_batch_set_grouping(self._handle, int(bool(on))), "nufft3d_batch_set_grouping")

    def forward_adjoint(self, vols, lines, vols_out, stream=None):
        n = len(self.items)
        if not (len(vols) == len(lines) == len(vols_out) == n):
            raise ValueError("one volume, line buffer and output volume per item")
        for it, v, l, o in zip(self.items, vols, lines, vols_out):
            it._check_tensor(v, (it.n,) * 3, it.vol_dtype, "vol")
            it._check_tensor(l, (it.n_dirs, it.m), __import__("torch").complex64, "lines")
            it._check_tensor(o, (it.n,) * 3, it.vol_dtype, "vol_out")
        P = ctypes.c_void_p * n
        _check(self.lib.nufft3d_batch_forward_adjoint(
            self._handle, P(*[v.data_ptr() for v in vols]), P(*[l.data_ptr() for l in lines]),
            P(*[o.data_ptr() for o in vols_out]), _stream_ptr(stream, self.device)), "nufft3d_batch_forward_adjoint")

    def close(self):
        if getattr(self, "_handle", None) is not None and self._handle.value:
            for it in self.items:
                it._handle = ctypes.c_void_p()
            self.lib.nufft3d_batch_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostPipeline:
    """Forward + adjoint of volumes that live in host memory, through the
    library's host pipeline (nufft3d_host_pipeline_*): the library copies the
    volume in, runs the plan's forward and adjoint and copies the lines and the
    output volume out on its own streams, overlapping the copies of one call
    with the kernels of its neighbours.  Host tensors should be pinned
    (``tensor.pin_memory()``).  run() returns immediately; results are valid
    after synchronize().
    """

    def __init__(self, plan: "Plan"):
        self.plan = plan
        self.lib = plan.lib
        h = ctypes.c_void_p()
        _check(self.lib.nufft3d_host_pipeline_create(plan._handle, ctypes.byref(h)), "nufft3d_host_pipeline_create")
        self._handle = h
        self._inflight = []

    def run(self, vol_host, lines_host, vout_host):
        """Enqueue one forward + adjoint: vol_host -> lines_host, vout_host (host tensors)."""
        import torch

        p = self.plan
        for t, shape, dt in ((vol_host, (p.n,) * 3, p.vol_dtype), (lines_host, (p.n_dirs, p.m), torch.complex64),
                             (vout_host, (p.n,) * 3, p.vol_dtype)):
            if t.device.type != "cpu" or tuple(t.shape) != shape or t.dtype != dt or not t.is_contiguous():
                raise ValueError(f"host tensor must be a contiguous CPU {dt} of shape {shape}")
        _check(self.lib.nufft3d_host_forward_adjoint(self._handle, ctypes.c_void_p(vol_host.data_ptr()),
                                                     ctypes.c_void_p(lines_host.data_ptr()),
                                                     ctypes.c_void_p(vout_host.data_ptr())),
               "nufft3d_host_forward_adjoint")
        self._inflight.append((vol_host, lines_host, vout_host))
        del self._inflight[:-2]

    def synchronize(self):
        _check(self.lib.nufft3d_host_pipeline_sync(self._handle), "nufft3d_host_pipeline_sync")
        self._inflight.clear()

    def close(self):
        if getattr(self, "_handle", None):
            self.lib.nufft3d_host_pipeline_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp32_fma_peak(stream=None):
    """Measured FP32 FMA throughput (TFLOP/s) and SM count of the current device."""
    import torch

    t = ctypes.c_double(0.0)
    n = ctypes.c_int(0)
    dev = torch.cuda.current_device()
    _check(load_library().nufft3d_fp32_fma_peak(ctypes.byref(t), ctypes.byref(n), _stream_ptr(stream, dev)),
           "nufft3d_fp32_fma_peak")
    return float(t.value), int(n.value)
