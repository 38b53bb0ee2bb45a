"""Thin Python binding of libcaxsi (ctypes).  Argument marshalling only: every
step of the forward model, the adjoint and the reconstruction update runs in
the library's CUDA kernels.  PyTorch supplies device memory and streams.

There is no fallback: if the shared library is missing or fails to load, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

PATH_DIRECT = 0
PATH_TABLE_FP32 = 1
PATH_TABLE_BF16 = 2
PATH_TABLE_FP16 = 3
PATHS = {"direct": PATH_DIRECT, "table_fp32": PATH_TABLE_FP32,
         "table_bf16": PATH_TABLE_BF16, "table_fp16": PATH_TABLE_FP16}

STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory",
          4: "positive count with non-positive mean", 5: "internal check failed",
          6: "unsupported option", 7: "problem exceeds the static scratch array"}


class CaxsiError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


class CGeometry(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in
                ("X", "J", "Q", "M", "N", "K", "rho_y", "mask_rows", "mask_cols")] + \
               [(k, ctypes.c_double) for k in
                ("x_center", "dx", "p_y", "p_z", "X_det", "X_mask", "q_min", "q_max",
                 "E_min", "E_max", "hc", "C", "mask_cell", "mask_y0", "mask_z0")]


class CPlanInfo(ctypes.Structure):
    _fields_ = [("n_offsets", ctypes.c_int64), ("table_bytes", ctypes.c_int64),
                ("n_breakpoints", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("n_open_pairs", ctypes.c_int64), ("n_records", ctypes.c_int64),
                ("device_error", ctypes.c_int64), ("n_sym_records", ctypes.c_int64),
                ("mask_symmetric", ctypes.c_int64)]


class CKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load():
    """Load libcaxsi.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with "
                                   "paper_1603_06400_gb300.build.build()")
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            F = ctypes.POINTER(ctypes.c_float)
            I64 = ctypes.c_int64
            lib.caxsi_plan_create.argtypes = [ctypes.POINTER(CGeometry),
                                              ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_uint8),
                                              ctypes.POINTER(P)]
            lib.caxsi_plan_destroy.argtypes = [P]
            lib.caxsi_plan_destroy.restype = None
            lib.caxsi_forward.argtypes = [P, P, I64, P, I64, ctypes.c_int, P]
            lib.caxsi_adjoint.argtypes = [P, P, I64, P, I64, ctypes.c_int, P]
            lib.caxsi_recon_step.argtypes = [P, P, P, P, I64, ctypes.c_float, ctypes.c_float,
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_double), P]
            lib.caxsi_forward_host.argtypes = [P, F, I64, F, I64, ctypes.c_int]
            lib.caxsi_adjoint_host.argtypes = [P, F, I64, F, I64, ctypes.c_int]
            lib.caxsi_plan_info.argtypes = [P, ctypes.POINTER(CPlanInfo)]
            lib.caxsi_forward_static_scratch.argtypes = [P, P, I64, P, I64, P]
            lib.caxsi_forward_static_scratch.restype = ctypes.c_int
            lib.caxsi_plan_set_option.argtypes = [P, ctypes.c_int, ctypes.c_int]
            lib.caxsi_plan_set_option.restype = ctypes.c_int
            lib.caxsi_profile_enable.argtypes = [P, ctypes.c_int]
            lib.caxsi_profile_read.argtypes = [P, ctypes.POINTER(CKernelStat), ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)]
            lib.caxsi_plan_set_subsets.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]
            lib.caxsi_forward_subset.argtypes = [P, ctypes.c_int, P, I64, P, I64, ctypes.c_int, P]
            lib.caxsi_adjoint_subset.argtypes = [P, ctypes.c_int, P, I64, P, I64, ctypes.c_int, P]
            lib.caxsi_recon_step_subset.argtypes = [P, ctypes.c_int, P, P, P, I64, ctypes.c_float,
                                                    ctypes.c_float, ctypes.c_int,
                                                    ctypes.POINTER(ctypes.c_double), P]
            I32P = ctypes.POINTER(ctypes.c_int32)
            lib.caxsi_forward_batch.argtypes = [P, ctypes.c_int, I32P, P, I64, P, I64, ctypes.c_int, P]
            lib.caxsi_adjoint_batch.argtypes = [P, ctypes.c_int, I32P, P, I64, P, I64, ctypes.c_int, P]
            lib.caxsi_em_update.argtypes = [P, P, P, P, ctypes.c_float, ctypes.c_float, P, I64, P]
            lib.caxsi_em_update_vjp.argtypes = [P, P, P, P, ctypes.c_float, ctypes.c_float, P, P, P, I64, P]
            V, U16 = ctypes.c_void_p, ctypes.c_void_p
            I, F32, I64_ = ctypes.c_int, ctypes.c_float, ctypes.c_int64
            nn = {
                "caxsi_nn_im2col3x3": [V, I, I, I, I, U16, V],
                "caxsi_nn_col2im3x3": [V, I, I, I, I, V, V],
                "caxsi_nn_gemm_bf16": [I, I, I, U16, U16, V, V, V],
                "caxsi_nn_to_bf16": [V, U16, I64_, V],
                "caxsi_nn_transpose_bf16": [V, I, I, I, U16, V],
                "caxsi_nn_bias_act": [V, V, I64_, I, I, V],
                "caxsi_nn_relu_bwd": [V, V, I64_, V],
                "caxsi_nn_bias_grad": [V, I64_, I, V, V],
                "caxsi_nn_pool2": [V, I, I, I, I, V, V],
                "caxsi_nn_pool2_bwd": [V, I, I, I, I, V, V],
                "caxsi_nn_up2": [V, I, I, I, I, V, V],
                "caxsi_nn_up2_bwd": [V, I, I, I, I, V, V],
                "caxsi_nn_copy_channels": [V, I64_, I, I, I, V, I, I, V],
                "caxsi_nn_scale_clamp": [V, F32, F32, V, I64_, V],
                "caxsi_nn_adam": [V, V, V, V, I64_, F32, F32, F32, F32, I, V],
                "caxsi_nn_axpy": [F32, V, V, I64_, V],
                "caxsi_nn_mse": [V, V, I64_, V, V, V],
                "caxsi_nn_poisson": [V, F32, I64_, ctypes.c_uint64, V, V],
            }
            for name, at in nn.items():
                getattr(lib, name).argtypes = at
                getattr(lib, name).restype = ctypes.c_int
            lib.caxsi_os_partition.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, I32P]
            lib.caxsi_ratio.argtypes = [P, P, P, P, P, I64, P]
            lib.caxsi_ratio_vjp.argtypes = [P, P, P, P, P, P, I64, P]
            I64P = ctypes.POINTER(ctypes.c_int64)
            lib.caxsi_multi_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(P)]
            lib.caxsi_multi_destroy.argtypes = [P]
            lib.caxsi_multi_destroy.restype = None
            lib.caxsi_multi_layout.argtypes = [P, I64P, I64P]
            lib.caxsi_multi_forward.argtypes = [P, P, I64, P, I64, ctypes.c_int, P]
            lib.caxsi_multi_adjoint.argtypes = [P, P, I64, P, I64, ctypes.c_int, P]
            lib.caxsi_multi_em_update.argtypes = [P, P, P, P, ctypes.c_float, ctypes.c_float, P, I64, P]
            lib.caxsi_multi_em_update_vjp.argtypes = [P, P, P, P, ctypes.c_float, ctypes.c_float, P, P, P, I64, P]
            lib.caxsi_status_string.argtypes = [ctypes.c_int]
            lib.caxsi_status_string.restype = ctypes.c_char_p
            for name in ("caxsi_plan_create", "caxsi_forward", "caxsi_adjoint",
                         "caxsi_recon_step", "caxsi_forward_host", "caxsi_adjoint_host",
                         "caxsi_plan_info", "caxsi_profile_enable", "caxsi_profile_read",
                         "caxsi_plan_set_subsets", "caxsi_forward_subset", "caxsi_adjoint_subset",
                         "caxsi_recon_step_subset", "caxsi_forward_batch", "caxsi_adjoint_batch",
                         "caxsi_em_update", "caxsi_em_update_vjp", "caxsi_os_partition", "caxsi_ratio",
                         "caxsi_ratio_vjp", "caxsi_multi_create", "caxsi_multi_layout", "caxsi_multi_forward",
                         "caxsi_multi_adjoint", "caxsi_multi_em_update", "caxsi_multi_em_update_vjp"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


def geometry_struct(g) -> CGeometry:
    d = g.as_dict() if hasattr(g, "as_dict") else dict(g)
    return CGeometry(**{k: d[k] for k, _ in CGeometry._fields_})


def _check(status: int, where: str):
    if status != 0:
        raise CaxsiError(status, where)


def _dev(t, n, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return ctypes.c_void_p(t.data_ptr())


def os_partition(M: int, N: int, rho_y: int, rho_z: int, sigma_y: int | None = None) -> np.ndarray:
    """Subset index of every detector pixel (int32 [M*N], row-major in (m, n)) for
    the symmetry-preserving ordered-subset partition of Sec. VI, computed by the
    library (caxsi_os_partition: rows in rho_z classes joined with their up-down
    mirrors, columns in sigma_y / 2 classes of step sigma_y joined with their
    left-right mirrors).  sigma_y defaults to rho_y when rho_y is even and to
    16 * rho_y otherwise.  Raises ValueError for steps the library rejects."""
    out = np.empty(M * N, dtype=np.int32)
    st = load().caxsi_os_partition(int(M), int(N), int(rho_y), int(rho_z),
                                   0 if sigma_y is None else int(sigma_y),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if st != 0:
        raise ValueError(f"os_partition: M={M}, N={N}, rho_y={rho_y}, rho_z={rho_z}, sigma_y={sigma_y} "
                         f"rejected ({STATUS.get(st, st)}): rho_z must divide M / 2 (M even), sigma_y must be "
                         "even, divide N and be a multiple of rho_y")
    return out


class Plan:
    """A device plan for one geometry, spectrum and mask (see include/caxsi.h)."""

    def __init__(self, geom, phi, mask):
        self.lib = load()
        self.geom = geom
        self.X, self.J, self.Q = geom.X, geom.J, geom.Q
        self.M, self.N = geom.M, geom.N
        self.f_len = self.X * self.J * self.Q
        self.g_len = self.M * self.N
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        if phi.size != geom.K or mask.size != geom.mask_rows * geom.mask_cols:
            raise ValueError("spectrum or mask has the wrong size")
        self._g = geometry_struct(geom)
        h = ctypes.c_void_p()
        _check(self.lib.caxsi_plan_create(
            ctypes.byref(self._g), phi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.byref(h)),
            "caxsi_plan_create")
        self.handle = h
        import torch
        self.device = torch.cuda.current_device()   # the library builds the plan there

    def _dev(self, t, n, name):
        ptr = _dev(t, n, name)
        if t.device.index != self.device:
            raise ValueError(f"{name} is on {t.device}, the plan on cuda:{self.device}")
        return ptr

    def _stream(self, stream):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(stream.cuda_stream)

    # -- device-pointer calls -------------------------------------------------
    def forward(self, f, out=None, path=PATH_DIRECT, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.M, self.N), device=f.device, dtype=torch.float32)
        _check(self.lib.caxsi_forward(self.handle, self._dev(f, self.f_len, "f"), self.f_len,
                                      self._dev(out, self.g_len, "g"), self.g_len, int(path),
                                      self._stream(stream)), "caxsi_forward")
        return out

    def adjoint(self, w, out=None, path=PATH_DIRECT, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.X, self.J, self.Q), device=w.device, dtype=torch.float32)
        _check(self.lib.caxsi_adjoint(self.handle, self._dev(w, self.g_len, "w"), self.g_len,
                                      self._dev(out, self.f_len, "f"), self.f_len, int(path),
                                      self._stream(stream)), "caxsi_adjoint")
        return out

    def recon_step(self, y, f, r=None, beta=0.0, delta=0.0, path=PATH_DIRECT,
                   want_nll=False, stream=None):
        nll = ctypes.c_double(0.0)
        rp = self._dev(r, self.g_len, "r") if r is not None else ctypes.c_void_p(None)
        _check(self.lib.caxsi_recon_step(
            self.handle, self._dev(y, self.g_len, "y"), rp, self._dev(f, self.f_len, "f"), self.f_len,
            float(beta), float(delta), int(path),
            ctypes.byref(nll) if want_nll else None, self._stream(stream)), "caxsi_recon_step")
        return nll.value if want_nll else None

    # -- ordered subsets (Sec. VI, Algorithm 5) --------------------------------
    def set_subsets(self, subset_of_pixel):
        """Set the detector partition (M*N subset indexes, e.g. from os_partition)."""
        sub = np.ascontiguousarray(np.asarray(subset_of_pixel).reshape(-1), dtype=np.int32)
        if sub.size != self.g_len:
            raise ValueError("subset_of_pixel must have M*N entries")
        n = int(sub.max()) + 1 if sub.size else 0
        _check(self.lib.caxsi_plan_set_subsets(self.handle, n, sub.ctypes.data_as(
            ctypes.POINTER(ctypes.c_int32))), "caxsi_plan_set_subsets")
        self.n_subsets = n

    def forward_subset(self, subset, f, out=None, path=PATH_TABLE_FP32, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.M, self.N), device=f.device, dtype=torch.float32)
        _check(self.lib.caxsi_forward_subset(self.handle, int(subset), self._dev(f, self.f_len, "f"), self.f_len,
                                             self._dev(out, self.g_len, "g"), self.g_len, int(path),
                                             self._stream(stream)), "caxsi_forward_subset")
        return out

    def adjoint_subset(self, subset, w, out=None, path=PATH_TABLE_FP32, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.X, self.J, self.Q), device=w.device, dtype=torch.float32)
        _check(self.lib.caxsi_adjoint_subset(self.handle, int(subset), self._dev(w, self.g_len, "w"), self.g_len,
                                             self._dev(out, self.f_len, "f"), self.f_len, int(path),
                                             self._stream(stream)), "caxsi_adjoint_subset")
        return out

    def recon_step_subset(self, subset, y, f, r=None, beta=0.0, delta=0.0, path=PATH_TABLE_FP32,
                          want_nll=False, stream=None):
        nll = ctypes.c_double(0.0)
        rp = self._dev(r, self.g_len, "r") if r is not None else ctypes.c_void_p(None)
        _check(self.lib.caxsi_recon_step_subset(
            self.handle, int(subset), self._dev(y, self.g_len, "y"), rp, self._dev(f, self.f_len, "f"), self.f_len,
            float(beta), float(delta), int(path), ctypes.byref(nll) if want_nll else None,
            self._stream(stream)), "caxsi_recon_step_subset")
        return nll.value if want_nll else None

    def os_pass(self, y, f, r=None, beta=0.0, delta=0.0, path=PATH_TABLE_FP32, stream=None):
        """One pass of Algorithm 5 over the subsets in order, in place on f; each
        step uses the penalty weight beta / P (the subset's data term stands for
        1/P of the full one)."""
        P = getattr(self, "n_subsets", 0)
        if P < 1:
            raise CaxsiError("set_subsets has not been called")
        for p in range(P):
            self.recon_step_subset(p, y, f, r=r, beta=beta / P, delta=delta, path=path, stream=stream)
        return f

    # -- batches of objects (voxel ranges of this geometry) ---------------------
    def _ranges(self, nb, ranges):
        R = self.X * self.J
        if ranges is None:
            ranges = [(0, R)] * nb
        r = np.ascontiguousarray(np.asarray(ranges, dtype=np.int32).reshape(nb, 2))
        return r

    def forward_batch(self, f, ranges=None, out=None, path=PATH_TABLE_FP32, stream=None):
        """g[b] = A f[b] over object b's voxel range (f: [nb, X, J, Q] device)."""
        import torch
        nb = f.shape[0]
        r = self._ranges(nb, ranges)
        if out is None:
            out = torch.empty((nb, self.M, self.N), device=f.device, dtype=torch.float32)
        _check(self.lib.caxsi_forward_batch(self.handle, nb, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                            self._dev(f, nb * self.f_len, "f"), nb * self.f_len,
                                            self._dev(out, nb * self.g_len, "g"), nb * self.g_len, int(path),
                                            self._stream(stream)), "caxsi_forward_batch")
        return out

    def adjoint_batch(self, w, ranges=None, out=None, path=PATH_TABLE_FP32, stream=None):
        """f[b] = A^T w[b] on object b's voxel range, 0 elsewhere (w: [nb, M, N] device)."""
        import torch
        nb = w.shape[0]
        r = self._ranges(nb, ranges)
        if out is None:
            out = torch.empty((nb, self.X, self.J, self.Q), device=w.device, dtype=torch.float32)
        _check(self.lib.caxsi_adjoint_batch(self.handle, nb, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                            self._dev(w, nb * self.g_len, "w"), nb * self.g_len,
                                            self._dev(out, nb * self.f_len, "f"), nb * self.f_len, int(path),
                                            self._stream(stream)), "caxsi_adjoint_batch")
        return out

    # -- the update step and its reverse mode -------------------------------------
    def em_update(self, f, b1, b2, beta=0.0, delta=0.0, out=None, stream=None):
        import torch
        n = f.numel()
        if out is None:
            out = torch.empty_like(f)
        _check(self.lib.caxsi_em_update(self.handle, self._dev(f, n, "f"), self._dev(b1, n, "b1"), self._dev(b2, n, "b2"),
                                        float(beta), float(delta), self._dev(out, n, "out"), n,
                                        self._stream(stream)), "caxsi_em_update")
        return out

    def em_update_vjp(self, f, b1, b2, grad_out, beta=0.0, delta=0.0, stream=None):
        import torch
        n = f.numel()
        gf, gb2 = torch.empty_like(f), torch.empty_like(f)
        _check(self.lib.caxsi_em_update_vjp(self.handle, self._dev(f, n, "f"), self._dev(b1, n, "b1"), self._dev(b2, n, "b2"),
                                            float(beta), float(delta), self._dev(grad_out, n, "grad_out"),
                                            self._dev(gf, n, "grad_f"), self._dev(gb2, n, "grad_b2"), n,
                                            self._stream(stream)), "caxsi_em_update_vjp")
        return gf, gb2

    # -- the likelihood ratio and its reverse mode ---------------------------------
    def ratio(self, g, y, r=None, out=None, stream=None):
        """y / (g + r) elementwise (0 where g + r <= 0); g, y, r of any equal size."""
        import torch
        n = g.numel()
        if out is None:
            out = torch.empty_like(g)
        rp = self._dev(r, n, "r") if r is not None else ctypes.c_void_p(None)
        _check(self.lib.caxsi_ratio(self.handle, self._dev(g, n, "g"), self._dev(y, n, "y"), rp,
                                    self._dev(out, n, "ratio"), n, self._stream(stream)), "caxsi_ratio")
        return out

    def ratio_vjp(self, g, y, grad_ratio, r=None, stream=None):
        """d(sum grad_ratio * ratio) / dg = -grad_ratio y / (g + r)^2 where g + r > 0."""
        import torch
        n = g.numel()
        out = torch.empty_like(g)
        rp = self._dev(r, n, "r") if r is not None else ctypes.c_void_p(None)
        _check(self.lib.caxsi_ratio_vjp(self.handle, self._dev(g, n, "g"), self._dev(y, n, "y"), rp,
                                        self._dev(grad_ratio, n, "grad_ratio"), self._dev(out, n, "grad_g"), n,
                                        self._stream(stream)), "caxsi_ratio_vjp")
        return out

    # -- host-buffer calls ----------------------------------------------------
    def forward_host(self, f, out=None, path=PATH_DIRECT):
        f = np.ascontiguousarray(f, dtype=np.float32)
        out = np.empty((self.M, self.N), np.float32) if out is None else out
        FP = ctypes.POINTER(ctypes.c_float)
        _check(self.lib.caxsi_forward_host(self.handle, f.ctypes.data_as(FP), f.size,
                                           out.ctypes.data_as(FP), out.size, int(path)),
               "caxsi_forward_host")
        return out

    def adjoint_host(self, w, out=None, path=PATH_DIRECT):
        w = np.ascontiguousarray(w, dtype=np.float32)
        out = np.empty((self.X, self.J, self.Q), np.float32) if out is None else out
        FP = ctypes.POINTER(ctypes.c_float)
        _check(self.lib.caxsi_adjoint_host(self.handle, w.ctypes.data_as(FP), w.size,
                                           out.ctypes.data_as(FP), out.size, int(path)),
               "caxsi_adjoint_host")
        return out

    def info(self) -> dict:
        i = CPlanInfo()
        _check(self.lib.caxsi_plan_info(self.handle, ctypes.byref(i)), "caxsi_plan_info")
        return {k: getattr(i, k) for k, _ in CPlanInfo._fields_}

    def set_u_samples(self, n: int = 0):
        """Table paths: 0 (default) interpolates W between the exact knots; n >= 2
        samples it at n uniform u and interpolates between them (an approximation
        of A, cheaper by B/n).  Set it before the first table-path call."""
        _check(self.lib.caxsi_plan_set_option(self.handle, 3, int(n)), "caxsi_plan_set_option")

    def set_sparse_subsets(self, on: bool = True):
        """FP32 subset operators contracted per record at the subset's knots only
        (default on) instead of by the whole-object contractions."""
        _check(self.lib.caxsi_plan_set_option(self.handle, 5, int(bool(on))), "caxsi_plan_set_option")

    def set_gemm_bands(self, on: bool = True):
        """Skip the product blocks of the tcgen05 contractions that meet only
        zeros of the band-limited spectral matrix (default on; results unchanged)."""
        _check(self.lib.caxsi_plan_set_option(self.handle, 4, int(bool(on))), "caxsi_plan_set_option")

    def set_symmetry(self, on: bool = True):
        """Mirror-symmetric records for the table paths' full forward and adjoint
        (default on when the geometry allows)."""
        _check(self.lib.caxsi_plan_set_option(self.handle, 2, int(bool(on))), "caxsi_plan_set_option")

    def set_online_mask(self, on: bool = True):
        """Direct path: exploit a mirror-symmetric mask (shared mask factor of the
        four mirror pairs, computed online); raises for a mask without the symmetry."""
        _check(self.lib.caxsi_plan_set_option(self.handle, 8, int(bool(on))), "caxsi_plan_set_option")

    def set_gemm_engine(self, engine: str):
        """'tcgen05' (default) or 'cublas' for the table paths' contractions."""
        _check(self.lib.caxsi_plan_set_option(self.handle, 1, {"tcgen05": 0, "cublas": 1}[engine]),
               "caxsi_plan_set_option")

    def profile(self, enable: bool = True):
        _check(self.lib.caxsi_profile_enable(self.handle, int(bool(enable))), "caxsi_profile_enable")

    def profile_read(self) -> dict:
        """{kernel name: (launches, total device ms)} since the last read/enable."""
        cap = 64
        arr = (CKernelStat * cap)()
        n = ctypes.c_int(0)
        _check(self.lib.caxsi_profile_read(self.handle, arr, cap, ctypes.byref(n)),
               "caxsi_profile_read")
        return {arr[k].name.decode(): (arr[k].launches, arr[k].total_ms) for k in range(n.value)}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.caxsi_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """Objects of different geometries, one Plan each, whose forward models and
    adjoints run as one persistent kernel launch per call (caxsi_multi_*, direct
    FP32 path).  Arrays are packed: object b's f occupies f_offsets[b] ..
    f_offsets[b+1] of a flat float32 tensor, its detector image g_offsets[b] ..
    g_offsets[b+1].  Each object's result is bit-identical to its own plan's call."""

    def __init__(self, plans):
        self.lib = load()
        self.plans = list(plans)
        n = len(self.plans)
        arr = (ctypes.c_void_p * n)(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(self.lib.caxsi_multi_create(arr, n, ctypes.byref(h)), "caxsi_multi_create")
        self.handle = h
        fo = np.zeros(n + 1, np.int64)
        go = np.zeros(n + 1, np.int64)
        I64P = ctypes.POINTER(ctypes.c_int64)
        _check(self.lib.caxsi_multi_layout(self.handle, fo.ctypes.data_as(I64P), go.ctypes.data_as(I64P)),
               "caxsi_multi_layout")
        self.f_offsets, self.g_offsets = fo, go
        self.f_len, self.g_len = int(fo[-1]), int(go[-1])
        self.device = self.plans[0].device

    def _dev(self, t, n, name):
        ptr = _dev(t, n, name)
        if t.device.index != self.device:
            raise ValueError(f"{name} is on {t.device}, the plans on cuda:{self.device}")
        return ptr

    def _stream(self, stream):
        return self.plans[0]._stream(stream)

    # packing helpers (views, no arithmetic)
    def pack_f(self, objs):
        import torch
        return torch.cat([o.reshape(-1) for o in objs]).contiguous()

    def pack_g(self, imgs):
        import torch
        return torch.cat([o.reshape(-1) for o in imgs]).contiguous()

    def unpack_f(self, flat):
        return [flat[self.f_offsets[b]:self.f_offsets[b + 1]].view(p.X, p.J, p.Q)
                for b, p in enumerate(self.plans)]

    def unpack_g(self, flat):
        return [flat[self.g_offsets[b]:self.g_offsets[b + 1]].view(p.M, p.N) for b, p in enumerate(self.plans)]

    def forward(self, f, out=None, path=PATH_DIRECT, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.g_len, device=f.device, dtype=torch.float32)
        _check(self.lib.caxsi_multi_forward(self.handle, self._dev(f, self.f_len, "f"), self.f_len,
                                            self._dev(out, self.g_len, "g"), self.g_len, int(path),
                                            self._stream(stream)), "caxsi_multi_forward")
        return out

    def adjoint(self, w, out=None, path=PATH_DIRECT, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.f_len, device=w.device, dtype=torch.float32)
        _check(self.lib.caxsi_multi_adjoint(self.handle, self._dev(w, self.g_len, "w"), self.g_len,
                                            self._dev(out, self.f_len, "f"), self.f_len, int(path),
                                            self._stream(stream)), "caxsi_multi_adjoint")
        return out

    def em_update(self, f, b1, b2, beta=0.0, delta=0.0, out=None, stream=None):
        import torch
        n = self.f_len
        if out is None:
            out = torch.empty_like(f)
        _check(self.lib.caxsi_multi_em_update(self.handle, self._dev(f, n, "f"), self._dev(b1, n, "b1"),
                                              self._dev(b2, n, "b2"), float(beta), float(delta),
                                              self._dev(out, n, "out"), n, self._stream(stream)),
               "caxsi_multi_em_update")
        return out

    def em_update_vjp(self, f, b1, b2, grad_out, beta=0.0, delta=0.0, stream=None):
        import torch
        n = self.f_len
        gf, gb2 = torch.empty_like(f), torch.empty_like(f)
        _check(self.lib.caxsi_multi_em_update_vjp(self.handle, self._dev(f, n, "f"), self._dev(b1, n, "b1"),
                                                  self._dev(b2, n, "b2"), float(beta), float(delta),
                                                  self._dev(grad_out, n, "grad_out"), self._dev(gf, n, "grad_f"),
                                                  self._dev(gb2, n, "grad_b2"), n, self._stream(stream)),
               "caxsi_multi_em_update_vjp")
        return gf, gb2

    def close(self):
        if getattr(self, "handle", None):
            self.lib.caxsi_multi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
