"""FP64 CPU oracle for the fan-beam coded-aperture coherent-scatter operators.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  It shares no code with
the CUDA library in ``paper_1603_06400_gb300`` and never imports it.

* ``forward`` / ``adjoint`` (and their pixel- / voxel-sampled forms) wrap the
  plain C direct summation in ``caxsi_oracle.c`` (Eq. 1-4, Algorithms 1 and 3,
  Appendix A), which the module compiles with gcc on first use.
* ``spectral_factor`` is the paper's S(theta, q) (Eq. 2 / Appendix A) used by
  the change-of-variables pin.
* ``nll``, ``penalty``, ``em_update`` restate Sec. V and Appendices B-C
  (penalised Poisson negative log-likelihood, Huber edge-preserving penalty on
  the 4 spatial neighbours, separable surrogate and its closed-form minimiser
  from the Lemma).
* ``os_subsets`` restates the symmetry-preserving ordered-subset partition of
  Sec. VI.
"""
from __future__ import annotations

import ctypes
import math
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "caxsi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
# one library per machine type: a build made on another architecture is never loaded
_LIB_PATH = os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OGeom(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in
                ("X", "J", "Q", "M", "N", "K", "rho_y", "mask_rows", "mask_cols")] + \
               [(k, ctypes.c_double) for k in
                ("x_center", "dx", "p_y", "p_z", "X_det", "X_mask", "q_min", "q_max",
                 "E_min", "E_max", "hc", "C", "mask_cell", "mask_y0", "mask_z0")]


class OPair(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("x", "y", "yp", "zp", "Gso", "God", "dtheta", "theta", "u", "T",
                 "mask_y", "mask_z", "angular")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            L = ctypes.POINTER(ctypes.c_long)
            U8 = ctypes.POINTER(ctypes.c_uint8)
            G = ctypes.POINTER(OGeom)
            lib.oracle_forward_pixels.argtypes = [G, D, U8, D, L, ctypes.c_long, D, ctypes.c_int]
            lib.oracle_adjoint_voxels.argtypes = [G, D, U8, D, L, ctypes.c_long, D, ctypes.c_int]
            lib.oracle_forward.argtypes = [G, D, U8, D, D, ctypes.c_int]
            lib.oracle_adjoint.argtypes = [G, D, U8, D, D, ctypes.c_int]
            lib.oracle_assemble_H.argtypes = [G, D, U8, D]
            lib.oracle_pair.argtypes = [G, U8] + [ctypes.c_int] * 4 + [ctypes.POINTER(OPair)]
            lib.oracle_w_energy.argtypes = [G, D, U8, D] + [ctypes.c_int] * 4
            lib.oracle_w_energy.restype = ctypes.c_double
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _geom(g) -> OGeom:
    d = g.as_dict() if hasattr(g, "as_dict") else dict(g)
    return OGeom(**{k: d[k] for k, _ in OGeom._fields_})


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _mask(g, mask):
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    assert mask.shape == (g.mask_rows, g.mask_cols)
    return mask


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def forward(g, phi, mask, f, nthreads: int = 0) -> np.ndarray:
    """g = A f over the whole detector, [M][N] float64."""
    lib = _load()
    f = _f64(f).reshape(-1)
    assert f.size == g.X * g.J * g.Q
    phi = _f64(phi)
    assert phi.size == g.K
    out = np.empty(g.M * g.N)
    lib.oracle_forward(ctypes.byref(_geom(g)), _dptr(phi), _mask(g, mask).ctypes.data_as(
        ctypes.POINTER(ctypes.c_uint8)), _dptr(f), _dptr(out), int(nthreads))
    return out.reshape(g.M, g.N)


def forward_pixels(g, phi, mask, f, pixels, nthreads: int = 0) -> np.ndarray:
    """(A f)[p] for flat pixel indices p = m*N + n."""
    lib = _load()
    f = _f64(f).reshape(-1)
    pix = np.ascontiguousarray(pixels, dtype=np.int64).reshape(-1)
    out = np.empty(pix.size)
    lib.oracle_forward_pixels(ctypes.byref(_geom(g)), _dptr(_f64(phi)),
                              _mask(g, mask).ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              _dptr(f), pix.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                              pix.size, _dptr(out), int(nthreads))
    return out


def adjoint(g, phi, mask, w, nthreads: int = 0) -> np.ndarray:
    """f = A^T w, [X][J][Q] float64."""
    lib = _load()
    w = _f64(w).reshape(-1)
    assert w.size == g.M * g.N
    out = np.empty(g.X * g.J * g.Q)
    lib.oracle_adjoint(ctypes.byref(_geom(g)), _dptr(_f64(phi)),
                       _mask(g, mask).ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                       _dptr(w), _dptr(out), int(nthreads))
    return out.reshape(g.X, g.J, g.Q)


def adjoint_voxels(g, phi, mask, w, voxels, nthreads: int = 0) -> np.ndarray:
    """(A^T w)[v, :] for flat voxel indices v = i*J + j, [len][Q]."""
    lib = _load()
    w = _f64(w).reshape(-1)
    vox = np.ascontiguousarray(voxels, dtype=np.int64).reshape(-1)
    out = np.empty(vox.size * g.Q)
    lib.oracle_adjoint_voxels(ctypes.byref(_geom(g)), _dptr(_f64(phi)),
                              _mask(g, mask).ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              _dptr(w), vox.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                              vox.size, _dptr(out), int(nthreads))
    return out.reshape(vox.size, g.Q)


def assemble_H(g, phi, mask) -> np.ndarray:
    """Dense system matrix [M*N][X*J*Q] (tiny instances only)."""
    lib = _load()
    P, V = g.M * g.N, g.X * g.J * g.Q
    assert P * V <= 5_000_000, "dense H only for tiny instances"
    H = np.empty(P * V)
    lib.oracle_assemble_H(ctypes.byref(_geom(g)), _dptr(_f64(phi)),
                          _mask(g, mask).ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                          _dptr(H))
    return H.reshape(P, V)


def pair(g, mask, i, j, m, n) -> dict:
    """Per-pair factors: G_so, G_od, dtheta, theta, u, T, crossing point, angular."""
    lib = _load()
    o = OPair()
    lib.oracle_pair(ctypes.byref(_geom(g)), _mask(g, mask).ctypes.data_as(
        ctypes.POINTER(ctypes.c_uint8)), int(i), int(j), int(m), int(n), ctypes.byref(o))
    return {k: getattr(o, k) for k, _ in OPair._fields_}


def w_energy(g, phi, mask, frow, i, j, m, n) -> float:
    """Effective spectral factor W(r, theta) (Eq. 4, energy form) for one pair."""
    lib = _load()
    frow = _f64(frow)
    assert frow.size == g.Q
    return float(lib.oracle_w_energy(ctypes.byref(_geom(g)), _dptr(_f64(phi)),
                                     _mask(g, mask).ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                     _dptr(frow), int(i), int(j), int(m), int(n)))


# ---------------------------------------------------------------------------
# Spectral factor in the paper's q form (Eq. 2 / Appendix A)
# ---------------------------------------------------------------------------

def spectral_factor(theta, q, phi_fn, hc):
    """S(theta, q) = q (1 + cos^2 theta) cos(theta/2) / sin^2(theta/2) * Phi(hc q / sin(theta/2))."""
    s2 = np.sin(0.5 * theta)
    return q * (1.0 + np.cos(theta) ** 2) * np.cos(0.5 * theta) / s2 ** 2 * phi_fn(hc * q / s2)


# ---------------------------------------------------------------------------
# Reconstruction (Sec. V, Sec. VI, Appendices B and C)
# ---------------------------------------------------------------------------

def _lgamma1(y):
    return np.array([math.lgamma(v + 1.0) for v in np.asarray(y, dtype=np.float64).ravel()]
                    ).reshape(np.shape(y))


def nll(y, z) -> float:
    """L = sum_i z_i - y_i ln z_i + ln y_i!  (z_i = l_i + r_i), with 0 ln 0 = 0."""
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    if np.any((y > 0) & (z <= 0)):
        raise ValueError("positive count with non-positive mean")
    ylogz = np.where(y > 0, y * np.log(np.where(z > 0, z, 1.0)), 0.0)
    return float(np.sum(z - ylogz + _lgamma1(y)))


def huber(t, delta):
    """psi_delta(t): t^2/2 for |t| <= delta, delta|t| - delta^2/2 otherwise."""
    a = np.abs(t)
    return np.where(a <= delta, 0.5 * t * t, delta * a - 0.5 * delta * delta)


def huber_grad(t, delta):
    """psi_dot_delta(t) = clamp(t, -delta, delta)."""
    return np.clip(t, -delta, delta)


def huber_curv(t, delta):
    """omega(t) = psi_dot(t)/t, equal to 1 on |t| <= delta (including t = 0)."""
    a = np.abs(t)
    return np.where(a <= delta, 1.0, delta / np.where(a > 0, a, 1.0))


def _neighbours(f):
    """The 4 spatial neighbours of every voxel in (i, j), each q channel
    independent; yields (neighbour values, valid) for each direction."""
    X, J, Q = f.shape
    for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        nb = np.zeros_like(f)
        ok = np.zeros((X, J, 1), dtype=bool)
        i0, i1 = max(0, -di), X - max(0, di)
        j0, j1 = max(0, -dj), J - max(0, dj)
        nb[i0:i1, j0:j1] = f[i0 + di:i1 + di, j0 + dj:j1 + dj]
        ok[i0:i1, j0:j1] = True
        yield nb, ok


def penalty(f, delta) -> float:
    """R(f) = sum_j sum_{k in N_j} w_jk psi_delta(f_j - f_k), w_jk = 1 (Eq. 7)."""
    f = np.asarray(f, dtype=np.float64)
    tot = 0.0
    for nb, ok in _neighbours(f):
        tot += float(np.sum(np.where(ok, huber(f - nb, delta), 0.0)))
    return tot


def b_terms(f_hat, delta):
    """b3 = b4 = 2 sum_k omega(f_j - f_k); b5 = b6 = sum_k psi_dot(f_j - f_k)
    over the symmetric 4-neighbourhood (Appendix B, w_jk = w_kj = 1)."""
    f_hat = np.asarray(f_hat, dtype=np.float64)
    b3 = np.zeros_like(f_hat)
    b5 = np.zeros_like(f_hat)
    for nb, ok in _neighbours(f_hat):
        d = f_hat - nb
        b3 += np.where(ok, 2.0 * huber_curv(d, delta), 0.0)
        b5 += np.where(ok, huber_grad(d, delta), 0.0)
    return b3, b3.copy(), b5, b5.copy()


def lemma_minimiser(a, b, c):
    """Unique minimiser over x >= 0 of a x^2/2 + b x - c ln x (Lemma, Appendix C):
    (-b + sqrt(b^2 + 4ac)) / (2a) for a > 0, c/b for a = 0 < b, +inf for a = 0 >= b."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        root = (-b + np.sqrt(b * b + 4.0 * a * c)) / (2.0 * a)
        lin = np.where(b > 0, c / b, np.inf)
    return np.where(a > 0, root, lin)


def em_update(f_hat, b1, b2, beta, delta):
    """Closed-form update of Eq. 10 (chi1 f^2 + chi2 f - chi3 = 0, positive root).

    Voxels with chi1 = 0 and chi2 <= 0 (never seen by any pixel and without a
    penalty) keep their value.
    """
    f_hat = np.asarray(f_hat, dtype=np.float64)
    b3, b4, b5, b6 = b_terms(f_hat, delta) if beta != 0 else (0.0, 0.0, 0.0, 0.0)
    chi1 = beta * (b3 + b4) * np.ones_like(f_hat)
    chi2 = b1 + beta * (-f_hat * (b3 + b4) + b5 + b6)
    chi3 = f_hat * b2
    x = lemma_minimiser(chi1, chi2, chi3)
    return np.where(np.isfinite(x), x, f_hat)


def em_iteration(A, At, y, r, f_hat, b1, beta, delta):
    """One iteration of the EM-type algorithm (Algorithm 4): z = A f + r,
    b2 = A^T (y / z), closed-form update.  Returns (f_next, L(f_hat))."""
    z = A(f_hat) + r
    if np.any((y > 0) & (z <= 0)):
        raise ValueError("positive count with non-positive mean")
    ratio = np.where(z > 0, y / np.where(z > 0, z, 1.0), 0.0)
    b2 = At(ratio)
    return em_update(f_hat, b1, b2, beta, delta), nll(y, z)


# ---------------------------------------------------------------------------
# Ordered subsets (Sec. VI)
# ---------------------------------------------------------------------------

def os_pixel_mask(M, N, rows, cols):
    """Boolean [M, N] mask of one subset from its 1-based row and column lists."""
    m = np.zeros((M, N), dtype=bool)
    m[np.ix_(np.asarray(rows) - 1, np.asarray(cols) - 1)] = True
    return m


def os_b1(At, in_subset):
    """b1_p = A_p^T 1 = A^T (indicator of the subset's pixels) (Algorithm 5)."""
    return At(np.asarray(in_subset, dtype=np.float64))


def os_sub_iteration(A, At, y, r, f_hat, in_subset, b1_p, beta_p, delta):
    """One inner step of the ordered-subset EM-type algorithm (Algorithm 5, Sec. VI).

    A_p is A restricted to the rows (pixels) of subset p, so z_p = (A f + r) on
    the subset, b2_p = A_p^T (y_p / z_p) = A^T of the ratio with zeros outside
    the subset, and f is updated by Eq. 10 with b1_p = A_p^T 1 in place of b1.
    beta_p is the penalty weight used in this step (the OS passes use beta / P:
    the subset data term stands for 1/P of the full one).  Returns
    (f_next, L_p(f_hat)) with L_p the likelihood of the subset's counts.
    """
    in_subset = np.asarray(in_subset, dtype=bool)
    z = A(f_hat) + r
    if np.any(in_subset & (y > 0) & (z <= 0)):
        raise ValueError("positive count with non-positive mean")
    ok = in_subset & (z > 0)
    ratio = np.where(ok, y / np.where(ok, z, 1.0), 0.0)
    b2 = At(ratio)
    return em_update(f_hat, b1_p, b2, beta_p, delta), nll(y[in_subset], z[in_subset])


def os_em_pass(A, At, y, r, f_hat, masks, b1s, beta, delta):
    """One pass t -> t+1 of Algorithm 5 over the P subsets in order, each step
    with penalty weight beta / P."""
    P = len(masks)
    f = f_hat
    for m, b1_p in zip(masks, b1s):
        f, _ = os_sub_iteration(A, At, y, r, f, m, b1_p, beta / P, delta)
    return f


def os_subsets(M, N, rho_y, rho_z):
    """Symmetry-preserving detector partition of Sec. VI, 1-based as in the paper.

    Rows: for 1 <= m <= rho_z, rows m:rho_z:M/2 together with M-m+1:-rho_z:M/2+1.
    Columns: for 1 <= n <= rho_y/2, columns n:rho_y:N with N-n+1:-rho_y:1.
    Returns a list of (rows, cols) index arrays (1-based), one per subset,
    in the order (row class, column class).
    """
    assert M % 2 == 0 and (M // 2) % rho_z == 0 and rho_y % 2 == 0 and N % rho_y == 0
    out = []
    for m in range(1, rho_z + 1):
        rows = list(range(m, M // 2 + 1, rho_z)) + list(range(M - m + 1, M // 2, -rho_z))
        for n in range(1, rho_y // 2 + 1):
            cols = list(range(n, N + 1, rho_y)) + list(range(N - n + 1, 0, -rho_y))
            out.append((np.array(rows), np.array(cols)))
    return out
