"""Pins for the reconstruction part of the oracle (Sec. V-VI, Appendices B-C)."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_section(fun, lo, hi, iters=200):
    g = (np.sqrt(5) - 1) / 2
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    for _ in range(iters):
        if fun(c) < fun(d):
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    return 0.5 * (a + b)


def test_lemma_against_golden_section():
    rng = np.random.default_rng(0)
    for _ in range(60):
        a = rng.uniform(0.01, 5)
        b = rng.uniform(-5, 5)
        c = rng.uniform(0.01, 5)
        x = float(oracle.lemma_minimiser(a, b, c))
        obj = lambda t: 0.5 * a * t * t + b * t - c * np.log(t)
        hi = 10 * (abs(b) / a + np.sqrt(c / a) + 1)
        xs = _golden_section(obj, 1e-12, hi)
        assert x == pytest.approx(xs, rel=1e-7)
        # the stationarity condition a x + b - c/x = 0
        assert a * x + b - c / x == pytest.approx(0.0, abs=1e-9 * (abs(b) + c / x + a * x))


def test_lemma_cases():
    # case a = 0, b > 0 gives c/b; a = 0, b <= 0 gives +inf; a > 0, c = 0 gives
    # -b/a for b <= 0 and 0 for b > 0 (Appendix C)
    assert float(oracle.lemma_minimiser(0.0, 2.0, 3.0)) == 1.5
    assert np.isinf(oracle.lemma_minimiser(0.0, -1.0, 3.0))
    assert np.isinf(oracle.lemma_minimiser(0.0, 0.0, 3.0))
    assert float(oracle.lemma_minimiser(2.0, -3.0, 0.0)) == pytest.approx(1.5)
    assert float(oracle.lemma_minimiser(2.0, 3.0, 0.0)) == 0.0


def test_huber_derivatives():
    t = np.linspace(-3, 3, 601)
    d = 0.7
    h = 1e-6
    fd = (oracle.huber(t + h, d) - oracle.huber(t - h, d)) / (2 * h)
    np.testing.assert_allclose(oracle.huber_grad(t, d), fd, atol=1e-6)
    nz = np.abs(t) > 1e-9
    np.testing.assert_allclose(oracle.huber_curv(t, d)[nz] * t[nz], oracle.huber_grad(t, d)[nz],
                               atol=1e-12)
    assert oracle.huber_curv(0.0, d) == 1.0
    # Huber's quadratic surrogate (curvature omega) majorises psi and touches at the expansion point
    for xh in (-2.0, -0.3, 0.0, 0.5, 1.7):
        sur = oracle.huber(xh, d) + oracle.huber_grad(xh, d) * (t - xh) + \
            0.5 * oracle.huber_curv(xh, d) * (t - xh) ** 2
        assert np.all(sur >= oracle.huber(t, d) - 1e-12)


def test_penalty_gradient_is_b5_plus_b6():
    # dR/df_j = sum_{k in N_j} psi_dot(f_j - f_k) + sum_{m: j in N_m} psi_dot(f_j - f_m) = b5 + b6
    rng = np.random.default_rng(1)
    f = rng.uniform(0, 1, size=(4, 5, 3))
    d = 0.2
    b3, b4, b5, b6 = oracle.b_terms(f, d)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 1), (3, 4, 2), (2, 0, 1)]:
        fp, fm = f.copy(), f.copy()
        fp[idx] += h
        fm[idx] -= h
        fd = (oracle.penalty(fp, d) - oracle.penalty(fm, d)) / (2 * h)
        assert fd == pytest.approx(b5[idx] + b6[idx], abs=1e-6)


def test_separable_surrogate_majorises_the_penalty():
    # Appendix B: with b3..b6 taken at f_hat, the separable surrogate
    #   P(f) = R(f_hat) + sum_j (b5 + b6)_j (f_j - f_hat_j) + 1/2 sum_j (b3 + b4)_j (f_j - f_hat_j)^2
    # lies above R everywhere and touches it at f_hat (Huber's quadratic majoriser
    # of each psi, then (a - b)^2 <= 2 a^2 + 2 b^2 to separate the voxels).  The
    # curvature is tight: along a checkerboard perturbation in the quadratic zone
    # R curves as 16 per voxel (the largest eigenvalue of twice the 4-neighbour
    # Laplacian) and so does P.
    rng = np.random.default_rng(3)
    f_hat = rng.uniform(0.5, 1.0, size=(6, 7, 3))
    d = 0.15
    b3, b4, b5, b6 = oracle.b_terms(f_hat, d)
    R0 = oracle.penalty(f_hat, d)

    def sur(f):
        e = f - f_hat
        return R0 + float(np.sum((b5 + b6) * e)) + 0.5 * float(np.sum((b3 + b4) * e * e))

    assert sur(f_hat) == pytest.approx(R0, rel=1e-15)
    ii, jj = np.meshgrid(np.arange(6), np.arange(7), indexing="ij")
    checker = ((-1.0) ** (ii + jj))[:, :, None] * np.ones((1, 1, 3))
    for scale in (1e-3, 1e-2, 0.1, 1.0):
        for trial in range(20):
            e = scale * rng.standard_normal(f_hat.shape)
            f = f_hat + e
            assert sur(f) >= oracle.penalty(f, d) - 1e-12 * (1.0 + abs(R0)), (scale, trial)
        f = f_hat + scale * checker
        assert sur(f) >= oracle.penalty(f, d) - 1e-12 * (1.0 + abs(R0)), scale
    # flat image, checkerboard of amplitude well inside delta: both sides gain
    # 4 eps^2 per neighbour edge (R: (2 eps)^2 per edge; P: 2 eps^2 times the
    # voxel's degree, summed over voxels), so the bound is attained
    flat = np.full((6, 7, 3), 0.7)
    c3, c4, c5, c6 = oracle.b_terms(flat, d)
    eps = 0.01
    e = eps * checker
    R_pert = oracle.penalty(flat + e, d) - oracle.penalty(flat, d)
    P_pert = 0.5 * float(np.sum((c3 + c4) * e * e)) + float(np.sum((c5 + c6) * e))
    edges = 3 * ((6 - 1) * 7 + 6 * (7 - 1))
    assert R_pert == pytest.approx(4 * eps ** 2 * edges, rel=1e-9)
    assert P_pert == pytest.approx(R_pert, rel=1e-12)


def test_beta_zero_is_mlem():
    rng = np.random.default_rng(2)
    f = rng.uniform(0.1, 1, size=(3, 4, 5))
    b1 = rng.uniform(0.5, 2, size=f.shape)
    b2 = rng.uniform(0.5, 2, size=f.shape)
    np.testing.assert_allclose(oracle.em_update(f, b1, b2, 0.0, 0.1), f * b2 / b1, rtol=1e-14)
    # a voxel no pixel sees (b1 = b2 = 0) keeps its value
    b1[0, 0, 0] = b2[0, 0, 0] = 0.0
    assert oracle.em_update(f, b1, b2, 0.0, 0.1)[0, 0, 0] == f[0, 0, 0]


def _small_problem(seed=0):
    g = synth.make_geometry(X=6, J=8, Q=16, M=8, N=16, K=8, rho_y=2, p_y=6.08, p_z=6.08, dx=8.0)
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 40 + seed)
    f_true = synth.phantom(g, seed, n_ellipses=3)
    A = lambda f: oracle.forward(g, phi, mask, f)
    At = lambda w: oracle.adjoint(g, phi, mask, w)
    mean = A(f_true)
    y = synth.poisson_counts(mean * (200.0 / mean.max()), seed + 100)
    return g, A, At, y, f_true


def test_em_count_preservation_and_monotone_nll():
    g, A, At, y, _ = _small_problem(0)
    r = np.zeros_like(y)
    b1 = At(np.ones_like(y))
    f = np.full((g.X, g.J, g.Q), y.sum() / b1.sum())
    prev = np.inf
    for _ in range(8):
        f_new, L = oracle.em_iteration(A, At, y, r, f, b1, 0.0, 0.1)
        assert L <= prev + 1e-9 * abs(prev if np.isfinite(prev) else 1)
        prev = L
        # sum_i (A f^{t+1})_i = sum_j b1_j f_j b2_j / b1_j = sum_i y_i (exact algebra)
        seen = b1 > 0
        assert A(np.where(seen, f_new, 0.0)).sum() == pytest.approx(y.sum(), rel=1e-10)
        f = f_new


def test_penalised_objective_monotone():
    g, A, At, y, _ = _small_problem(1)
    r = np.full_like(y, 0.5)
    b1 = At(np.ones_like(y))
    f = np.full((g.X, g.J, g.Q), y.sum() / b1.sum())
    beta, delta = 2.0, 0.05
    prev = np.inf
    for _ in range(8):
        z = A(f) + r
        J = oracle.nll(y, z) + beta * oracle.penalty(f, delta)
        assert J <= prev + 1e-9 * abs(J)
        prev = J
        f, _ = oracle.em_iteration(A, At, y, r, f, b1, beta, delta)
        assert np.all(f >= 0)


def test_nll_value():
    y = np.array([0.0, 1.0, 3.0])
    z = np.array([0.5, 2.0, 3.0])
    from math import lgamma, log
    ref = sum(zz - (yy * log(zz) if yy > 0 else 0.0) + lgamma(yy + 1) for yy, zz in zip(y, z))
    assert oracle.nll(y, z) == pytest.approx(ref, rel=1e-15)
    with pytest.raises(ValueError):
        oracle.nll(np.array([1.0]), np.array([0.0]))


def test_os_partition_matches_worked_example():
    txt = [ln.split() for ln in open(os.path.join(GOLD, "os_partition_32x64.txt"))
           if ln.strip() and not ln.startswith("#")]
    kv = {t[0]: [int(v) for v in t[1:]] for t in txt}
    M, N, ry, rz = kv["M"][0], kv["N"][0], kv["rho_y"][0], kv["rho_z"][0]
    subs = oracle.os_subsets(M, N, ry, rz)
    assert len(subs) == kv["n_subsets"][0]
    # the example subset is the first row class and first column class
    rows, cols = subs[0]
    assert list(cols) == kv["cols"]
    assert list(rows) == kv["rows"]
    # a partition of the detector: every pixel exactly once
    cover = np.zeros((M, N), int)
    for rws, cls in subs:
        cover[np.ix_(rws - 1, cls - 1)] += 1
    assert np.all(cover == 1)


# ---------------------------------------------------------------------------
# Ordered subsets (Algorithm 5, Sec. VI)
# ---------------------------------------------------------------------------

def _os_masks(g, rho_z, sigma_y):
    return [oracle.os_pixel_mask(g.M, g.N, rows, cols)
            for rows, cols in oracle.os_subsets(g.M, g.N, sigma_y, rho_z)]


def test_os_single_subset_is_the_em_iteration():
    g, A, At, y, _ = _small_problem(2)
    r = np.full_like(y, 0.25)
    b1 = At(np.ones_like(y))
    f = np.full((g.X, g.J, g.Q), y.sum() / b1.sum())
    every = np.ones((g.M, g.N), bool)
    f1, L1 = oracle.os_sub_iteration(A, At, y, r, f, every, oracle.os_b1(At, every), 0.3, 0.05)
    f2, L2 = oracle.em_iteration(A, At, y, r, f, b1, 0.3, 0.05)
    np.testing.assert_array_equal(f1, f2)
    assert L1 == L2


def test_os_subset_sensitivities_sum_to_b1():
    g, A, At, y, _ = _small_problem(3)
    masks = _os_masks(g, 2, 4)
    assert len(masks) == 4
    np.testing.assert_allclose(sum(oracle.os_b1(At, m) for m in masks), At(np.ones_like(y)),
                               rtol=1e-12, atol=1e-300)


def test_os_step_preserves_the_subset_counts():
    # with beta = 0 and r = 0 each step is MLEM on its subset:
    # sum_{i in S_p} (A f')_i = sum_j f_j b2_pj = sum_{i in S_p} y_i (exact algebra)
    g, A, At, y, _ = _small_problem(4)
    r = np.zeros_like(y)
    masks = _os_masks(g, 2, 4)
    b1s = [oracle.os_b1(At, m) for m in masks]
    f = np.full((g.X, g.J, g.Q), y.sum() / sum(b.sum() for b in b1s))
    for m, b1p in zip(masks, b1s):
        f_new, _ = oracle.os_sub_iteration(A, At, y, r, f, m, b1p, 0.0, 0.1)
        assert A(f_new)[m].sum() == pytest.approx(y[m].sum(), rel=1e-10)
        # pixels outside the subset do not enter the step
        y_other = np.where(m, y, y + 7.0)
        f_alt, _ = oracle.os_sub_iteration(A, At, y_other, r, f, m, b1p, 0.0, 0.1)
        np.testing.assert_array_equal(f_alt, f_new)
        f = f_new


def test_os_pass_reduces_the_likelihood_from_a_flat_start():
    g, A, At, y, f_true = _small_problem(5)
    r = np.zeros_like(y)
    masks = _os_masks(g, 2, 4)
    b1s = [oracle.os_b1(At, m) for m in masks]
    f0 = np.full((g.X, g.J, g.Q), y.sum() / sum(b.sum() for b in b1s))
    f1 = oracle.os_em_pass(A, At, y, r, f0, masks, b1s, 0.0, 0.1)
    assert oracle.nll(y, A(f1)) < oracle.nll(y, A(f0))
