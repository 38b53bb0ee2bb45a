"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
evaluated by a different route, the Bragg-law support of a point scatterer,
the paper's printed constants and worked example, exact symmetries and
algebraic identities of the model, and a brute-force dense system matrix.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def small_geometry(**kw):
    base = dict(X=4, J=5, Q=12, M=6, N=10, K=7, rho_y=2, p_y=3.04, p_z=6.08, dx=2.5)
    base.update(kw)
    return synth.make_geometry(**base)


# --------------------------------------------------------------------------
# Constants printed in the paper
# --------------------------------------------------------------------------

def test_hc_matches_paper():
    gold = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    # the paper prints hc in keV*Angstrom; the q grid here is in nm^-1
    assert synth.HC_KEV_NM * 10.0 == pytest.approx(gold["hc_keV_angstrom"], rel=1e-15)
    g = synth.tiny_geometry()
    assert g.X_det == gold["X_det_mm"]
    assert g.X_det - g.X_mask == gold["mask_to_detector_mm"]
    assert g.x_center == gold["object_centre_mm"]


# --------------------------------------------------------------------------
# Geometric factors by a second route
# --------------------------------------------------------------------------

def _law_of_cosines_angle(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    la, lb, lc = np.linalg.norm(a), np.linalg.norm(b), np.linalg.norm(a - b)
    return math.acos((la * la + lb * lb - lc * lc) / (2 * la * lb))


@pytest.mark.parametrize("m,n", [(0, 0), (2, 3), (5, 9), (3, 4)])
def test_on_axis_voxel_closed_forms(m, n):
    # J = 1 puts the single object column on the central ray (y = 0): r_hat = x_hat,
    # so theta = atan(R/L) with R the radial distance of the pixel on the detector.
    g = small_geometry(J=1, X=3)
    mask = np.ones((g.mask_rows, g.mask_cols), np.uint8)
    for i in range(g.X):
        p = oracle.pair(g, mask, i, 0, m, n)
        x = g.x_center + (i - 1) * g.dx
        L = g.X_det - x
        yp = (n - (g.N - 1) / 2) * g.p_y
        zp = (m - (g.M - 1) / 2) * g.p_z
        R = math.hypot(yp, zp)
        assert p["y"] == 0.0
        assert p["theta"] == pytest.approx(math.atan(R / L), rel=1e-13)
        assert p["Gso"] == pytest.approx(1.0 / x ** 2, rel=1e-14)
        assert p["God"] == pytest.approx(L / (L * L + R * R) ** 1.5, rel=1e-13)
        h = g.p_z / 2
        dth = _law_of_cosines_angle([L, yp, zp + h], [L, yp, zp - h])
        assert p["dtheta"] == pytest.approx(dth, rel=1e-9)
        assert p["u"] == pytest.approx(math.sin(math.atan(R / L) / 2), rel=1e-13)
        c = math.cos(math.atan(R / L))
        assert p["angular"] == pytest.approx((1 + c * c) * math.sqrt((1 + c) / 2), rel=1e-13)


def test_off_axis_theta_by_dot_product():
    g = small_geometry()
    mask = np.ones((g.mask_rows, g.mask_cols), np.uint8)
    rng = np.random.default_rng(3)
    for _ in range(40):
        i, j, m, n = (int(rng.integers(0, s)) for s in (g.X, g.J, g.M, g.N))
        p = oracle.pair(g, mask, i, j, m, n)
        r = np.array([p["x"], p["y"], 0.0])
        s = np.array([g.X_det - p["x"], p["yp"] - p["y"], p["zp"]])
        th = _law_of_cosines_angle(r / np.linalg.norm(r) * np.linalg.norm(s), s)
        assert p["theta"] == pytest.approx(th, rel=1e-7)
        assert p["Gso"] == pytest.approx(np.dot(r, [1, 0, 0]) / np.linalg.norm(r) ** 3, rel=1e-14)


def test_translation_symmetry_of_scatter_vector():
    # Sec. III-A: with the object pitch along y equal to rho_y detector pitches,
    # s(r + v, r' + v) = s(r, r'): G_od and dtheta are unchanged when the voxel
    # moves by one column and the pixel by rho_y columns.
    g = small_geometry(J=5, N=14, rho_y=2)
    mask = np.ones((g.mask_rows, g.mask_cols), np.uint8)
    for i in range(g.X):
        for j in range(g.J - 1):
            for m in range(g.M):
                for n in range(g.N - g.rho_y):
                    a = oracle.pair(g, mask, i, j, m, n)
                    b = oracle.pair(g, mask, i, j + 1, m, n + g.rho_y)
                    assert b["God"] == pytest.approx(a["God"], rel=1e-13)
                    assert b["dtheta"] == pytest.approx(a["dtheta"], rel=1e-12)


# --------------------------------------------------------------------------
# Mask geometry: a single open cell is seen exactly along rays through it
# --------------------------------------------------------------------------

def test_single_open_cell_ray_trace():
    g = small_geometry(M=40, N=60, p_y=1.0, p_z=1.0, J=3, rho_y=2)
    rows, cols = g.mask_rows, g.mask_cols
    mask = np.zeros((rows, cols), np.uint8)
    rc, cc = rows // 2 + 3, cols // 2 - 4
    mask[rc, cc] = 1
    yc = g.mask_y0 + (cc + 0.5) * g.mask_cell
    zc = g.mask_z0 + (rc + 0.5) * g.mask_cell
    for i in range(g.X):
        for j in range(g.J):
            x = g.x_center + (i - (g.X - 1) / 2) * g.dx
            y = (j - (g.J - 1) / 2) * g.rho_y * g.p_y
            # extend the ray from (x, y, 0) through the cell centre to the detector plane
            s = (g.X_det - x) / (g.X_mask - x)
            yd, zd = y + (yc - y) * s, zc * s
            n = int(round(yd / g.p_y + (g.N - 1) / 2))
            m = int(round(zd / g.p_z + (g.M - 1) / 2))
            assert 0 <= n < g.N and 0 <= m < g.M
            assert oracle.pair(g, mask, i, j, m, n)["T"] == 1.0
            # a pixel whose ray lands more than one cell away is blocked
            far = oracle.pair(g, mask, i, j, min(g.M - 1, m + 8), n)
            assert far["T"] == 0.0
    # total open pairs: the footprint of one cell, magnified by 1/t, covers about
    # (cell / t / pitch)^2 pixels per voxel
    f = np.ones((g.X, g.J, g.Q))
    assert np.count_nonzero(oracle.forward(g, synth.tungsten_spectrum(g), mask, f)) > 0


def test_open_cell_seen_from_off_axis_voxels():
    # Voxels up to 16 mm off the central plane: the mask crossing of a ray moves by
    # (1 - t) y with the voxel's y (t = (X_mask - x)/(X_det - x)), several cells here.
    # From each voxel, the ray through the open cell's centre, extended to the
    # detector, lands on a pixel that sees the cell; pixels 4 steps away in y or z
    # (3.2 mm at the mask plane, past the 1 mm half-cell) do not.
    g = small_geometry(X=3, J=5, M=24, N=40, p_y=1.0, p_z=1.0, rho_y=8)
    rows, cols = g.mask_rows, g.mask_cols
    mask = np.zeros((rows, cols), np.uint8)
    rc, cc = rows // 2, cols // 2 - 1
    mask[rc, cc] = 1
    yc = g.mask_y0 + (cc + 0.5) * g.mask_cell
    zc = g.mask_z0 + (rc + 0.5) * g.mask_cell
    seen = 0
    for i in range(g.X):
        x = g.x_center + (i - (g.X - 1) / 2) * g.dx
        for j in range(g.J):
            y = (j - (g.J - 1) / 2) * g.rho_y * g.p_y
            s = (g.X_det - x) / (g.X_mask - x)
            yd, zd = y + (yc - y) * s, zc * s
            n = int(round(yd / g.p_y + (g.N - 1) / 2))
            m = int(round(zd / g.p_z + (g.M - 1) / 2))
            assert 0 <= n < g.N and 0 <= m < g.M
            assert oracle.pair(g, mask, i, j, m, n)["T"] == 1.0, (i, j)
            seen += 1
            for dm, dn in ((4, 0), (-4, 0), (0, 4), (0, -4)):
                if 0 <= m + dm < g.M and 0 <= n + dn < g.N:
                    assert oracle.pair(g, mask, i, j, m + dm, n + dn)["T"] == 0.0, (i, j, dm, dn)
    assert seen == g.X * g.J
    assert max(abs((j - (g.J - 1) / 2) * g.rho_y * g.p_y) for j in range(g.J)) == 16.0


# --------------------------------------------------------------------------
# Point scatterer: Bragg-law annulus and its values, by polar coordinates
# --------------------------------------------------------------------------

@pytest.mark.parametrize("l", [0, 17])
def test_point_scatterer_footprint(l):
    # One voxel on the central ray, one q bin, one energy bin (a narrow spectrum):
    # the detector sees a ring where E sin(theta/2)/hc is within one q step of q_l.
    # For the first bin the ring includes the half step below q_0: the q samples
    # are hat functions, the grid extended by a zero sample at each end.
    g = synth.make_geometry(X=1, J=1, Q=40, M=64, N=128, K=1, rho_y=1, p_y=0.76,
                            p_z=0.76, dx=2.0, E_min=59.0, E_max=61.0, q_min=0.1,
                            q_max=3.5, C=2.5)
    mask = np.ones((g.mask_rows, g.mask_cols), np.uint8)
    phi = np.array([1.0])
    f = np.zeros((1, 1, g.Q))
    f[0, 0, l] = 1.0
    out = oracle.forward(g, phi, mask, f)
    E = 60.0
    dE = 2.0
    dq = (g.q_max - g.q_min) / (g.Q - 1)
    ql = g.q_min + l * dq
    L = g.X_det - g.x_center
    x = g.x_center

    def radius(q):
        return L * math.tan(2 * math.asin(q * g.hc / E))

    R_lo, R_hi = radius(ql - dq), radius(ql + dq)
    nz = 0
    for m in range(g.M):
        for n in range(g.N):
            yp = (n - (g.N - 1) / 2) * g.p_y
            zp = (m - (g.M - 1) / 2) * g.p_z
            R = math.hypot(yp, zp)
            theta = math.atan2(R, L)
            q = E * math.sin(theta / 2) / g.hc
            tau = (q - g.q_min) / dq
            hat = max(0.0, 1.0 - abs(tau - l))
            Gso = 1.0 / x ** 2
            God = L / (L * L + R * R) ** 1.5
            h = g.p_z / 2
            dth = _law_of_cosines_angle([L, yp, zp + h], [L, yp, zp - h])
            ang = (1 + math.cos(theta) ** 2) * math.cos(theta / 2)
            expect = g.C * Gso * God * dth * ang * E * dE / g.hc ** 2 * hat
            assert out[m, n] == pytest.approx(expect, rel=1e-8, abs=1e-300)
            inside = R_lo < R < R_hi
            assert (out[m, n] > 0) == inside
            nz += inside
    assert nz > 50


# --------------------------------------------------------------------------
# Change of variables: energy form against the paper's q form of S(theta, q)
# --------------------------------------------------------------------------

def test_energy_form_matches_q_form_of_spectral_factor():
    # W(theta) = int S(theta, q) f(q) dq with S from Eq. 2.  The oracle evaluates
    # it as an energy sum of K midpoint bins with f linearly interpolated on a
    # q grid; both discretisations converge to the same integral, which pins
    # the Jacobian E/(hc)^2 dE and the angular factor.
    E_min, E_max = 20.0, 100.0

    def phi_fn(E):
        E = np.asarray(E, float)
        Es = np.where(E > 0, E, 1.0)
        # Kramers continuum with a taper that vanishes smoothly at E_min
        v = (E_max / Es - 1) * (Es / E_min - 1) ** 2 * np.exp(-(25 / Es) ** 3)
        return np.where((E > E_min) & (E < E_max), v, 0.0)

    def f_fn(q):
        return np.exp(-0.5 * ((q - 1.3) / 0.35) ** 2) + 0.4 * np.exp(-0.5 * ((q - 2.2) / 0.5) ** 2)

    errs = []
    for K, Q in ((200, 400), (800, 1600)):
        g = synth.make_geometry(X=1, J=3, Q=Q, M=4, N=8, K=K, rho_y=4, p_y=6.0, p_z=6.0,
                                dx=2.0, q_min=0.05, q_max=5.0, E_min=E_min, E_max=E_max, C=1.0)
        dE = (E_max - E_min) / K
        Ek = E_min + (np.arange(K) + 0.5) * dE
        phi = phi_fn(Ek)
        qg = np.linspace(g.q_min, g.q_max, g.Q)
        frow = f_fn(qg)
        mask = np.ones((g.mask_rows, g.mask_cols), np.uint8)
        rel = []
        for (j, m, n) in ((0, 0, 0), (2, 3, 7), (1, 1, 5), (0, 2, 6)):
            p = oracle.pair(g, mask, 0, j, m, n)
            W = oracle.w_energy(g, phi, mask, frow, 0, j, m, n)
            qq = np.linspace(E_min * p["u"] / g.hc, E_max * p["u"] / g.hc, 200001)
            S = oracle.spectral_factor(p["theta"], qq, phi_fn, g.hc)
            ref = np.trapezoid(S * f_fn(qq), qq)
            rel.append(abs(W - ref) / abs(ref))
        errs.append(max(rel))
    # second-order convergence (midpoint rule in E, linear interpolation in q):
    # quadrupling K and Q divides the error by about 16; any dropped or wrong
    # factor would leave an O(1) discrepancy that does not shrink
    assert errs[-1] < 5e-5
    assert errs[-1] < errs[0] / 12


# --------------------------------------------------------------------------
# Exact identities of the linear model
# --------------------------------------------------------------------------

def test_adjoint_identity():
    g = small_geometry(X=5, J=6, Q=16, M=8, N=14, K=9, rho_y=2)
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 5)
    f = synth.uniform_random((g.X, g.J, g.Q), 11)
    w = synth.normal_random((g.M, g.N), 12)
    lhs = float(np.sum(oracle.forward(g, phi, mask, f) * w))
    rhs = float(np.sum(f * oracle.adjoint(g, phi, mask, w)))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


def test_dense_matrix_brute_force():
    g = small_geometry(X=4, J=4, Q=8, M=4, N=4, K=4, rho_y=1, p_y=12.0, p_z=12.0)
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 6)
    H = oracle.assemble_H(g, phi, mask)
    assert np.count_nonzero(H) > 0.05 * H.size
    f = synth.uniform_random((g.X, g.J, g.Q), 21)
    w = synth.uniform_random((g.M, g.N), 22)
    np.testing.assert_allclose(oracle.forward(g, phi, mask, f).ravel(), H @ f.ravel(), rtol=1e-12)
    np.testing.assert_allclose(oracle.adjoint(g, phi, mask, w).ravel(), H.T @ w.ravel(), rtol=1e-12,
                               atol=1e-14 * np.abs(H.T @ w.ravel()).max())


def test_linearity_and_positivity():
    g = small_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 7)
    f1 = synth.uniform_random((g.X, g.J, g.Q), 1)
    f2 = synth.uniform_random((g.X, g.J, g.Q), 2)
    a, b = 0.7, -1.9
    lhs = oracle.forward(g, phi, mask, a * f1 + b * f2)
    rhs = a * oracle.forward(g, phi, mask, f1) + b * oracle.forward(g, phi, mask, f2)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-11, atol=1e-13 * np.abs(rhs).max())
    assert np.all(oracle.forward(g, phi, mask, f1) >= 0)
    assert np.all(oracle.adjoint(g, phi, mask, synth.uniform_random((g.M, g.N), 3)) >= 0)
    assert not np.any(oracle.forward(g, phi, mask, np.zeros_like(f1)))


def test_left_right_mirror_symmetry():
    # Sec. III-A: mirroring the object about y = 0 and the mask about the central
    # ray mirrors the detector image left-right.
    g = small_geometry(J=6, N=12)
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 8)
    f = synth.uniform_random((g.X, g.J, g.Q), 9)
    a = oracle.forward(g, phi, mask, f)
    b = oracle.forward(g, phi, mask[:, ::-1], f[:, ::-1, :])
    np.testing.assert_allclose(b, a[:, ::-1], rtol=1e-12)
    w = synth.uniform_random((g.M, g.N), 10)
    fa = oracle.adjoint(g, phi, mask, w)
    fb = oracle.adjoint(g, phi, mask[:, ::-1], w[:, ::-1])
    np.testing.assert_allclose(fb, fa[:, ::-1, :], rtol=1e-12)


def test_up_down_mirror_symmetry():
    # Sec. III-A: the fan lies in z = 0, so mirroring the mask in z mirrors the
    # detector image up-down.
    g = small_geometry(M=8)
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 13)
    f = synth.uniform_random((g.X, g.J, g.Q), 14)
    a = oracle.forward(g, phi, mask, f)
    b = oracle.forward(g, phi, mask[::-1, :], f)
    np.testing.assert_allclose(b, a[::-1, :], rtol=1e-12)


def test_mask_complement_adds_up():
    # T enters linearly: an all-open mask equals mask + complement.
    g = small_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 15)
    f = synth.uniform_random((g.X, g.J, g.Q), 16)
    full = oracle.forward(g, phi, np.ones_like(mask), f)
    parts = oracle.forward(g, phi, mask, f) + oracle.forward(g, phi, 1 - mask, f)
    np.testing.assert_allclose(parts, full, rtol=1e-12)


def test_sampled_entry_points_agree_with_full():
    g = small_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 17)
    f = synth.uniform_random((g.X, g.J, g.Q), 18)
    w = synth.uniform_random((g.M, g.N), 19)
    full = oracle.forward(g, phi, mask, f).ravel()
    pix = np.array([0, 7, g.M * g.N - 1, 13])
    np.testing.assert_array_equal(oracle.forward_pixels(g, phi, mask, f, pix), full[pix])
    fa = oracle.adjoint(g, phi, mask, w).reshape(g.X * g.J, g.Q)
    vox = np.array([g.X * g.J - 1, 0, 5])
    np.testing.assert_array_equal(oracle.adjoint_voxels(g, phi, mask, w, vox), fa[vox])
