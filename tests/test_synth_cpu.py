"""The seeded input recipe: the workload sizes and spans, the tungsten-like
spectrum, the mask, the phantoms and the count draws have the properties the
recipe states, and the on-device phantom generator used for training data
rasterises the same phantoms as the reference generator."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("make", [synth.tiny_geometry, synth.paper_geometry])
def test_workload_spans_and_distances(make):
    g = make()
    # both workloads cover the same object and detector (mm)
    assert g.N * g.p_y == pytest.approx(194.56)
    assert g.M * g.p_z == pytest.approx(97.28)
    assert g.X * g.dx == pytest.approx(70.0)
    assert g.J * g.rho_y * g.p_y == pytest.approx(194.56)
    assert (g.x_center, g.X_mask, g.X_det) == (1035.0, 1446.5, 1546.5)
    assert (g.q_min, g.q_max, g.E_min, g.E_max) == (0.1, 3.5, 20.0, 100.0)
    # the object lies between the source and the mask
    assert g.x_center - 0.5 * (g.X - 1) * g.dx > 0
    assert g.x_center + 0.5 * (g.X - 1) * g.dx < g.X_mask


def test_paper_workload_sizes():
    g = synth.paper_geometry()
    assert (g.X, g.J, g.Q, g.M, g.N, g.K, g.rho_y) == (128, 256, 128, 64, 256, 64, 1)
    t = synth.tiny_geometry()
    assert (t.X, t.J, t.Q, t.M, t.N, t.K, t.rho_y) == (32, 32, 64, 16, 64, 32, 2)


def test_spectrum_normalised_with_tungsten_lines():
    g = synth.paper_geometry()
    phi = synth.tungsten_spectrum(g)
    dE = (g.E_max - g.E_min) / g.K
    assert phi.shape == (g.K,) and np.all(phi > 0)
    assert float(np.sum(phi) * dE) == pytest.approx(1.0, rel=1e-12)
    edges = synth.energy_bin_edges(g)
    for line in (59.3, 67.2):
        k = int(np.searchsorted(edges, line) - 1)
        # the line's bin stands above both neighbours
        assert phi[k] > phi[k - 1] and phi[k] > phi[k + 1], line
    # without the lines the continuum is smooth: a single maximum
    cont = synth.tungsten_spectrum(g, lines=False)
    d = np.sign(np.diff(cont))
    assert np.count_nonzero(d[1:] != d[:-1]) == 1
    # the Kramers continuum vanishes at E_max: the last bin is small
    assert cont[-1] < 0.02 * cont.max()


def test_mask_cells_centred_and_half_open():
    g = synth.paper_geometry()
    m = synth.random_mask(g, synth.PAPER_MASK_SEED)
    assert m.shape == (g.mask_rows, g.mask_cols) and m.dtype == np.uint8
    assert set(np.unique(m)) <= {0, 1}
    assert g.mask_cell == pytest.approx(2 * g.p_y)                  # two detector pixels wide
    assert g.mask_y0 == pytest.approx(-0.5 * g.mask_cols * g.mask_cell)
    assert g.mask_z0 == pytest.approx(-0.5 * g.mask_rows * g.mask_cell)
    n = m.size
    assert abs(m.mean() - 0.5) < 5 * np.sqrt(0.25 / n)               # Bernoulli(0.5)
    assert np.array_equal(m, synth.random_mask(g, synth.PAPER_MASK_SEED))
    assert not np.array_equal(m, synth.random_mask(g, synth.PAPER_MASK_SEED + 1))


def test_phantom_structure():
    g = synth.tiny_geometry()
    for seed in range(6):
        f = synth.phantom(g, seed)
        assert f.shape == (g.X, g.J, g.Q) and np.all(f >= 0)
        rows = f.reshape(-1, g.Q)
        nonzero = rows[np.any(rows > 0, axis=1)]
        assert len(nonzero) > 0
        # distinct profiles, at most one per ellipse (at most 8)
        assert 1 <= len(np.unique(nonzero, axis=0)) <= 8
        for prof in np.unique(nonzero, axis=0):
            # at least one Bragg peak of amplitude >= 0.3 on top of a hump of <= 0.3
            assert prof.max() >= 0.3
            # the hump keeps every bin of a profile positive
            assert np.all(prof > 0)
        # the voxels outside every ellipse are exactly zero
        assert np.all(rows[~np.any(rows > 0, axis=1)] == 0)
    assert np.array_equal(synth.phantom(g, 3), synth.phantom(g, 3))
    assert len(np.unique(synth.phantom(g, 4, n_ellipses=1).reshape(-1, g.Q), axis=0)) <= 2


def test_device_phantom_generator_matches_the_reference():
    torch = pytest.importorskip("torch")
    g = synth.tiny_geometry()
    for seed in (0, 5, 11):
        ref = synth.phantom(g, seed).astype(np.float32)
        got = synth.phantom_torch(g, seed, "cpu").numpy()
        assert np.array_equal(got, ref), seed


def test_count_draws():
    mean = np.full((64, 64), 37.5)
    y = synth.poisson_counts(mean, 9)
    assert np.all(y >= 0) and np.all(y == np.round(y))
    assert y.mean() == pytest.approx(37.5, rel=0.03)
    assert y.var() == pytest.approx(37.5, rel=0.1)                   # Poisson: variance = mean
    assert np.array_equal(y, synth.poisson_counts(mean, 9))
    assert np.all(synth.poisson_counts(np.array([-1.0, 0.0]), 1) == 0)   # negative means clip to 0
    peaks = [synth.log_uniform_peak(s) for s in range(200)]
    assert min(peaks) >= 1e2 and max(peaks) <= 1e4
    # log-uniform: the median is near the geometric mean 1e3
    assert 3e2 < float(np.median(peaks)) < 3e3


def test_symmetric_mask_is_mirror_symmetric_and_seeded():
    for g in (synth.tiny_geometry(), synth.paper_geometry()):
        m = synth.symmetric_mask(g, 5)
        assert m.shape == (g.mask_rows, g.mask_cols) and m.dtype == np.uint8
        np.testing.assert_array_equal(m, m[:, ::-1])      # left-right about y = 0
        np.testing.assert_array_equal(m, m[::-1, :])      # up-down about z = 0
        assert 0.4 < m.mean() < 0.6
        # the grid is centred on the central ray, as the symmetry needs
        assert g.mask_y0 == -0.5 * g.mask_cols * g.mask_cell and g.mask_z0 == -0.5 * g.mask_rows * g.mask_cell
        np.testing.assert_array_equal(m, synth.symmetric_mask(g, 5))
        assert not np.array_equal(m, synth.symmetric_mask(g, 6))


def test_uneven_sizes_cover_their_ranges():
    sizes = synth.uneven_sizes(32, 2024)
    assert len(sizes) == 32 and sizes[0] == (32, 64, 64) and sizes[1] == (128, 256, 128)
    X, J, Q = map(np.array, zip(*sizes))
    assert X.min() == 32 and X.max() == 128 and J.min() == 64 and J.max() == 256
    assert Q.min() == 64 and Q.max() == 128
    assert len(set(sizes)) == 32                         # sizes differ in every dimension
    g = synth.uneven_object_geometry(77, 162, 113)
    base = synth.paper_geometry()
    assert (g.X, g.J, g.Q) == (77, 162, 113)
    assert (g.M, g.N, g.K, g.p_y, g.dx, g.q_min, g.q_max) == (base.M, base.N, base.K, base.p_y, base.dx,
                                                              base.q_min, base.q_max)
    # C scales like the recipe's dimensional constant (inversely with X J)
    assert g.C * 77 * 162 == pytest.approx(base.C * base.X * base.J)


def test_paper_table1_geometry_matches_the_timing_study():
    g = synth.paper_table1_geometry()
    assert (g.N, g.M) == (2048, 1536) and g.p_y == g.p_z == 0.19          # 0.19 mm pixels
    assert (g.X, g.J) == (28, 28) and g.dx == 2.5
    assert g.rho_y == 16 and g.rho_y * g.p_y == pytest.approx(3.04)          # 3.04 mm object pitch
    assert g.Q == 79 and (g.q_min, g.q_max) == (0.1, 4.0)                   # 0.01-0.4 per Angstrom
    assert g.E_max == 125.0
    # the mask grid covers every ray from the object to the detector edges
    t = (g.X_mask - (g.x_center - 0.5 * (g.X - 1) * g.dx)) / (g.X_det - (g.x_center - 0.5 * (g.X - 1) * g.dx))
    y_obj, y_det = 0.5 * g.J * g.rho_y * g.p_y, 0.5 * g.N * g.p_y
    assert (1 - t) * y_obj + t * y_det < -g.mask_y0        # the widest crossing, object and detector edges
    assert t * 0.5 * g.M * g.p_z < -g.mask_z0
