"""Seeded synthetic inputs for the fan-beam coded-aperture coherent-scatter operators.

This module is shared by the FP64 oracle (``oracle/``) and the CUDA path
(``paper_1603_06400_gb300``).  It only produces *inputs*: geometry parameters,
the binned source spectrum, the binary secondary mask, phantom scatter
densities and Poisson draws.  It holds none of the operator arithmetic
(no coordinates, angles, geometric factors or interpolation): both sides
derive those themselves from the parameters returned here.

Workload recipe (stand-ins for the paper's measured NaCl/Al momentum-transfer
profiles and its Monte Carlo graphite data, which are not available):

* geometry: the distances of Sec. VII (source at the origin, object centre
  1035 mm, secondary mask 1446.5 mm, detector 1546.5 mm); the detector spans
  194.56 mm (y) x 97.28 mm (z) and the object 70 mm (x) x 194.56 mm (y);
* spectrum: tungsten-like bremsstrahlung -- Kramers continuum (E_max/E - 1)
  with soft filtration exp(-(25/E)^3) plus W K-lines (59.3 keV, 67.2 keV,
  sigma 0.5 keV), averaged over each energy bin and normalised to unit
  integral;
* mask: Bernoulli(0.5) cells two detector pixels wide (the "2-pixel
  feature"), centred on the central ray;
* phantoms: ellipses in the (x, y) field whose momentum-transfer profiles are
  1-4 Gaussian Bragg peaks (sigma 0.02-0.05 nm^-1) plus an amorphous hump;
* counts: Poisson draws around a mean scaled to a chosen peak.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict, replace

import numpy as np

HC_KEV_NM = 1.23984193  # h*c in keV*nm (Eq. for Bragg's law gives 12.3984193 keV*Angstrom)


@dataclass(frozen=True)
class Geometry:
    """Plain numbers describing one system; units mm, keV, nm^-1.

    Index conventions: object voxel (i, j) with i along the central ray (the
    paper's x, X voxels) and j across the fan (the paper's y, J voxels);
    detector pixel (m, n) with m along z (M rows) and n along y (N columns);
    q bin l (Q bins, endpoints q_min and q_max inclusive); energy bin k
    (K bins between E_min and E_max).
    """

    X: int
    J: int
    Q: int
    M: int
    N: int
    K: int
    rho_y: int
    x_center: float
    dx: float
    p_y: float
    p_z: float
    X_det: float
    X_mask: float
    q_min: float
    q_max: float
    E_min: float
    E_max: float
    hc: float
    C: float
    mask_rows: int
    mask_cols: int
    mask_cell: float
    mask_y0: float
    mask_z0: float

    def as_dict(self) -> dict:
        return asdict(self)

    def with_(self, **kw) -> "Geometry":
        return replace(self, **kw)

    @property
    def n_voxels(self) -> int:
        return self.X * self.J

    @property
    def f_len(self) -> int:
        return self.X * self.J * self.Q

    @property
    def g_len(self) -> int:
        return self.M * self.N


def make_geometry(X, J, Q, M, N, K, rho_y, p_y, p_z, dx, *, x_center=1035.0,
                  X_det=1546.5, X_mask=1446.5, q_min=0.1, q_max=3.5,
                  E_min=20.0, E_max=100.0, hc=HC_KEV_NM, C=None,
                  mask_half_y=120.0, mask_half_z=60.0, mask_cell=None) -> Geometry:
    """Build a geometry; the mask grid is centred on the central ray.

    C (the paper's calibration constant) is an input.  When not given it is set
    to a dimensional scale x_c^2 (X_d - x_c)^3 / (p_z X J) that keeps detector
    values of order one for order-one densities.
    """
    cell = float(mask_cell if mask_cell is not None else 2.0 * p_y)
    cols = 2 * int(math.ceil(mask_half_y / cell))
    rows = 2 * int(math.ceil(mask_half_z / cell))
    if C is None:
        L = X_det - x_center
        C = x_center ** 2 * L ** 3 / (p_z * X * J)
    return Geometry(X=int(X), J=int(J), Q=int(Q), M=int(M), N=int(N), K=int(K),
                    rho_y=int(rho_y), x_center=float(x_center), dx=float(dx),
                    p_y=float(p_y), p_z=float(p_z), X_det=float(X_det),
                    X_mask=float(X_mask), q_min=float(q_min), q_max=float(q_max),
                    E_min=float(E_min), E_max=float(E_max), hc=float(hc),
                    C=float(C), mask_rows=rows, mask_cols=cols, mask_cell=cell,
                    mask_y0=-0.5 * cols * cell, mask_z0=-0.5 * rows * cell)


# The two single-GPU workloads: a tiny one (32x32 voxels x 64 q, detector
# 64x16, 32 energies) and the paper-scale one (256x128 voxels x 128 q,
# detector 256x64, 64 energies).  Both cover a 70 mm x 194.56 mm object and a
# 194.56 mm x 97.28 mm detector.
def tiny_geometry(**kw) -> Geometry:
    return make_geometry(X=32, J=32, Q=64, M=16, N=64, K=32, rho_y=2,
                         p_y=3.04, p_z=6.08, dx=2.1875, **kw)


def paper_geometry(**kw) -> Geometry:
    return make_geometry(X=128, J=256, Q=128, M=64, N=256, K=64, rho_y=1,
                         p_y=0.76, p_z=1.52, dx=0.546875, **kw)


def paper_table1_geometry(**kw) -> Geometry:
    """The geometry of the paper's timing study (Sec. VII, Table I): detector
    2048 (y) x 1536 (z) pixels at 0.19 mm, object 28 x 28 voxels of 2.5 mm (x) x
    3.04 mm (y, 16 detector pitches: translation step 16), 79 q bins over
    0.01-0.4 A^-1 (0.1-4 nm^-1), 125 kVp source (64 energy bins 15-125 keV here),
    the paper's distances, and a mask grid wide enough to cover every detector
    ray.  The paper's own mask and spectrum are not available: the mask and
    spectrum recipes of this module stand in for them."""
    return make_geometry(X=28, J=28, Q=79, M=1536, N=2048, K=64, rho_y=16, p_y=0.19, p_z=0.19, dx=2.5,
                         q_min=0.1, q_max=4.0, E_min=15.0, E_max=125.0, mask_half_y=200.0, mask_half_z=150.0,
                         **kw)


def energy_bin_edges(g: Geometry) -> np.ndarray:
    return np.linspace(g.E_min, g.E_max, g.K + 1)


def tungsten_spectrum(g: Geometry, *, lines: bool = True, sub: int = 64) -> np.ndarray:
    """Bin-averaged tungsten-like spectrum Phi_k (K values), unit integral.

    Phi(E) = (E_max/E - 1) exp(-(25/E)^3) + K-lines, averaged over each bin by
    ``sub``-point midpoint sampling, then scaled so sum_k Phi_k dE = 1.
    """
    edges = energy_bin_edges(g)
    dE = (g.E_max - g.E_min) / g.K
    out = np.empty(g.K)
    Ef = np.linspace(1.0, g.E_max, 4000)
    cont_max = np.max(np.clip(g.E_max / Ef - 1.0, 0, None) * np.exp(-(25.0 / Ef) ** 3))
    for k in range(g.K):
        E = edges[k] + (np.arange(sub) + 0.5) * (dE / sub)
        v = np.clip(g.E_max / E - 1.0, 0.0, None) * np.exp(-(25.0 / E) ** 3)
        if lines:
            v = v + 0.35 * cont_max * np.exp(-0.5 * ((E - 59.3) / 0.5) ** 2)
            v = v + 0.10 * cont_max * np.exp(-0.5 * ((E - 67.2) / 0.5) ** 2)
        out[k] = v.mean()
    out /= out.sum() * dE
    return out


def random_mask(g: Geometry, seed: int, open_fraction: float = 0.5) -> np.ndarray:
    """Binary secondary mask, uint8 [mask_rows][mask_cols], row = z cell, col = y cell."""
    rng = np.random.default_rng(seed)
    return (rng.random((g.mask_rows, g.mask_cols)) < open_fraction).astype(np.uint8)


def symmetric_mask(g: Geometry, seed: int, open_fraction: float = 0.5) -> np.ndarray:
    """A mask designed for the mirror symmetries: Bernoulli cells drawn for the
    upper-left quarter of the (centred, even-sized) cell grid and mirrored left-right
    and up-down, so the pattern is symmetric about the central ray in y and z."""
    rows, cols = g.mask_rows, g.mask_cols
    assert rows % 2 == 0 and cols % 2 == 0
    rng = np.random.default_rng(seed)
    q = (rng.random((rows // 2, cols // 2)) < open_fraction).astype(np.uint8)
    top = np.concatenate([q, q[:, ::-1]], axis=1)
    return np.ascontiguousarray(np.concatenate([top, top[::-1, :]], axis=0))


def _profile(rng, q, n_peaks_max=4):
    prof = np.zeros_like(q)
    lo, hi = q[0] + 0.2, q[-1] - 0.2
    for _ in range(int(rng.integers(1, n_peaks_max + 1))):
        c = rng.uniform(lo, hi)
        s = rng.uniform(0.02, 0.05)
        a = rng.uniform(0.3, 1.0)
        prof += a * np.exp(-0.5 * ((q - c) / s) ** 2)
    c = rng.uniform(1.0, 2.5)
    w = rng.uniform(0.4, 0.8)
    a = rng.uniform(0.1, 0.3)
    prof += a * np.exp(-0.5 * ((q - c) / w) ** 2)
    return prof


def phantom(g: Geometry, seed: int, n_ellipses: int | None = None,
            max_ellipses: int = 8) -> np.ndarray:
    """Scatter density f [X][J][Q] (float64): ellipses with Bragg-peak profiles.

    Centres uniform in the inner 60 % of the (i, j) field, semi-axes 10-30 % of
    the extent, rotation U[0, pi); later ellipses overwrite earlier ones and
    the background is zero.  Peaks are point-sampled on the q grid.
    """
    rng = np.random.default_rng(seed)
    if n_ellipses is None:
        n_ellipses = int(rng.integers(1, max_ellipses + 1))
    q = np.linspace(g.q_min, g.q_max, g.Q)
    f = np.zeros((g.X, g.J, g.Q))
    ii, jj = np.meshgrid((np.arange(g.X) + 0.5) / g.X, (np.arange(g.J) + 0.5) / g.J,
                         indexing="ij")
    for _ in range(n_ellipses):
        ci, cj = rng.uniform(0.2, 0.8, size=2)
        ai, aj = rng.uniform(0.1, 0.3, size=2)
        rot = rng.uniform(0.0, math.pi)
        di, dj = ii - ci, jj - cj
        u = (math.cos(rot) * di + math.sin(rot) * dj) / ai
        v = (-math.sin(rot) * di + math.cos(rot) * dj) / aj
        inside = u * u + v * v <= 1.0
        f[inside] = _profile(rng, q)
    return f


def phantom_torch(g: Geometry, seed: int, device, n_ellipses: int | None = None, max_ellipses: int = 8):
    """The phantom of `phantom` (the same random draws, ellipse tests in float64)
    rasterised on a torch device as float32 [X][J][Q], for generating many
    training objects quickly."""
    import torch
    rng = np.random.default_rng(seed)
    if n_ellipses is None:
        n_ellipses = int(rng.integers(1, max_ellipses + 1))
    q = np.linspace(g.q_min, g.q_max, g.Q)
    f = torch.zeros((g.X, g.J, g.Q), dtype=torch.float32, device=device)
    ii = ((torch.arange(g.X, dtype=torch.float64, device=device) + 0.5) / g.X)[:, None]
    jj = ((torch.arange(g.J, dtype=torch.float64, device=device) + 0.5) / g.J)[None, :]
    for _ in range(n_ellipses):
        ci, cj = rng.uniform(0.2, 0.8, size=2)
        ai, aj = rng.uniform(0.1, 0.3, size=2)
        rot = rng.uniform(0.0, math.pi)
        di, dj = ii - ci, jj - cj
        u = (math.cos(rot) * di + math.sin(rot) * dj) / ai
        v = (-math.sin(rot) * di + math.cos(rot) * dj) / aj
        inside = u * u + v * v <= 1.0
        prof = torch.tensor(_profile(rng, q), dtype=torch.float32, device=device)
        f[inside] = prof
    return f


def uniform_random(shape, seed: int, lo=0.0, hi=1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape)


def normal_random(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=shape)


def poisson_counts(mean: np.ndarray, seed: int) -> np.ndarray:
    """Poisson draws y ~ Poisson(mean) (float64 array of integers)."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.clip(mean, 0.0, None)).astype(np.float64)


def log_uniform_peak(seed: int, lo=1e2, hi=1e4) -> float:
    rng = np.random.default_rng(seed + 7919)
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


TINY_MASK_SEED = 1001
PAPER_MASK_SEED = 1002


# Objects of uneven size sharing the paper-scale detector, spectrum model and
# mask: extents uniform in x across the fan J in [64, 256], z along the beam
# X in [32, 128] and q bins Q in [64, 128] (same q range), at the paper-scale
# voxel pitches, centred where the paper-scale object is.
UNEVEN_J = (64, 256)
UNEVEN_X = (32, 128)
UNEVEN_Q = (64, 128)


def uneven_sizes(n: int, seed: int, X=UNEVEN_X, J=UNEVEN_J, Q=UNEVEN_Q) -> list:
    """n seeded (X, J, Q) extents, each uniform in its closed range; the first two
    objects take the range ends (smallest and largest) so that both occur."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n):
        if b == 0:
            out.append((X[0], J[0], Q[0]))
        elif b == 1:
            out.append((X[1], J[1], Q[1]))
        else:
            out.append((int(rng.integers(X[0], X[1] + 1)), int(rng.integers(J[0], J[1] + 1)),
                        int(rng.integers(Q[0], Q[1] + 1))))
    return out


def uneven_object_geometry(X: int, J: int, Q: int, base: Geometry | None = None) -> Geometry:
    """The geometry of one uneven object: `base` (default the paper-scale
    geometry) with X, J and Q replaced, and C rescaled as make_geometry sets it."""
    b = base if base is not None else paper_geometry()
    L = b.X_det - b.x_center
    return replace(b, X=int(X), J=int(J), Q=int(Q), C=b.x_center ** 2 * L ** 3 / (b.p_z * X * J))
