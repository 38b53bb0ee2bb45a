"""GPU parity of the ordered-subset operators (Sec. VI, Algorithm 5) through the
C ABI against the FP64 oracle: A_p f, A_p^T w and one ordered-subset EM step.

Tolerance: relative L2 error <= 1e-5 on the subset's pixels (forward) and on the
whole object (adjoint), as for the full FP32 operators; exact zeros outside the
subset.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

REL_L2_TOL = 1e-5
OS_PATHS = ["direct", "table_fp32", "table_fp32@cublas"]


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def cx():
    import torch
    from paper_1603_06400_gb300 import build, caxsi
    build.build()
    return caxsi, torch


def _t(torch, a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda:0")


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _plan(caxsi, g, phi, mask, path):
    plan = caxsi.Plan(g, phi, mask)
    name, _, engine = path.partition("@")
    if engine:
        plan.set_gemm_engine(engine)
    return plan, caxsi.PATHS[name]


def _partitions(caxsi, g):
    """The paper's symmetry-preserving partition where the detector allows it, and
    an arbitrary (random) one: the operators accept any partition."""
    out = {"random3": synth.uniform_random((g.M * g.N,), 11) * 3}
    out["random3"] = np.minimum(out["random3"].astype(np.int32), 2)
    if g.M % 2 == 0 and (g.M // 2) % 2 == 0 and g.N % 4 == 0:
        out["paper"] = caxsi.os_partition(g.M, g.N, g.rho_y, 2, 4 if 4 % g.rho_y == 0 else 2 * g.rho_y)
    return out


GEOMS = {
    "tiny": lambda: synth.tiny_geometry(),
    "ragged": lambda: synth.make_geometry(X=5, J=7, Q=37, M=9, N=45, K=13, rho_y=3,
                                          p_y=2.5, p_z=4.0, dx=6.0),
}


@pytest.mark.parametrize("name", sorted(GEOMS))
@pytest.mark.parametrize("path", OS_PATHS)
def test_subset_forward_adjoint_parity(cx, name, path):
    caxsi, torch = cx
    g = GEOMS[name]()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 77)
    f = synth.phantom(g, 3, n_ellipses=3) + 0.05 * synth.uniform_random((g.X, g.J, g.Q), 4)
    w = synth.uniform_random((g.M, g.N), 5) + 0.1
    plan, p = _plan(caxsi, g, phi, mask, path)
    ref_g = oracle.forward(g, phi, mask, _f32(f))
    full = plan.forward(_t(torch, f), path=p).cpu().numpy()
    for pname, sub in _partitions(caxsi, g).items():
        plan.set_subsets(sub)
        P = int(sub.max()) + 1
        total = np.zeros((g.M, g.N))
        for s in range(P):
            inside = (sub == s).reshape(g.M, g.N)
            gp = plan.forward_subset(s, _t(torch, f), path=p).cpu().numpy()
            assert np.all(gp[~inside] == 0.0), (pname, s)
            assert rel_l2(gp[inside], ref_g[inside]) <= REL_L2_TOL, (pname, s)
            total += gp
            fp = plan.adjoint_subset(s, _t(torch, w), path=p).cpu().numpy()
            ref_f = oracle.adjoint(g, phi, mask, np.where(inside, _f32(w), 0.0))
            assert rel_l2(fp, ref_f) <= REL_L2_TOL, (pname, s)
        # the subsets partition the rows of A
        assert rel_l2(total, full) <= 1e-6
    plan.close()


@pytest.mark.parametrize("beta", [0.0, 5e-3])
@pytest.mark.parametrize("path", OS_PATHS)
def test_os_step_parity(cx, beta, path):
    caxsi, torch = cx
    g = synth.tiny_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, synth.TINY_MASK_SEED)
    f_true = synth.phantom(g, 1, n_ellipses=3)
    mean = oracle.forward(g, phi, mask, f_true)
    y = synth.poisson_counts(mean * (1e3 / mean.max()), 2)
    r = np.full_like(y, 0.25)
    plan, p = _plan(caxsi, g, phi, mask, path)
    sub = caxsi.os_partition(g.M, g.N, g.rho_y, 2, 4)
    plan.set_subsets(sub)
    P = int(sub.max()) + 1
    A = lambda x: oracle.forward(g, phi, mask, x)
    At = lambda x: oracle.adjoint(g, phi, mask, x)
    masks = [(sub == s).reshape(g.M, g.N) for s in range(P)]
    b1s = [oracle.os_b1(At, m) for m in masks]
    f0 = np.full((g.X, g.J, g.Q), y.sum() / sum(b.sum() for b in b1s))
    delta = 0.02
    ft = _t(torch, f0)
    yt, rt = _t(torch, y), _t(torch, r)
    f = _f32(f0)
    for s in range(P):
        nll_gpu = plan.recon_step_subset(s, yt, ft, r=rt, beta=beta / P, delta=delta, want_nll=True, path=p)
        f_next, nll_ref = oracle.os_sub_iteration(A, At, y, r, f, masks[s], b1s[s], beta / P, delta)
        assert nll_gpu == pytest.approx(nll_ref, rel=1e-6)
        got = ft.cpu().numpy()
        # only channels the subset observes are compared (as for the full step)
        seen = b1s[s] > 1e-6 * b1s[s].max()
        assert rel_l2(got[seen], f_next[seen]) <= 5 * REL_L2_TOL, s
        assert np.all(np.isfinite(got)) and np.all(got >= 0)
        f = _f32(got)
    plan.close()


def test_os_pass_matches_the_steps(cx):
    caxsi, torch = cx
    g = synth.tiny_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, synth.TINY_MASK_SEED)
    y = synth.poisson_counts(oracle.forward(g, phi, mask, synth.phantom(g, 4, n_ellipses=2)) * 50.0, 3)
    plan = caxsi.Plan(g, phi, mask)
    plan.set_subsets(caxsi.os_partition(g.M, g.N, g.rho_y, 2, 4))
    yt = _t(torch, y)
    f1 = torch.full((g.X, g.J, g.Q), 0.5, device="cuda:0")
    f2 = f1.clone()
    plan.os_pass(yt, f1, beta=0.01, delta=0.05)
    for s in range(plan.n_subsets):
        plan.recon_step_subset(s, yt, f2, beta=0.01 / plan.n_subsets, delta=0.05)
    assert torch.equal(f1, f2)   # deterministic kernels: bit-identical
    plan.close()


def test_subset_errors(cx):
    caxsi, torch = cx
    g = synth.tiny_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, synth.TINY_MASK_SEED)
    plan = caxsi.Plan(g, phi, mask)
    f = torch.ones(g.f_len, device="cuda:0")
    with pytest.raises(caxsi.CaxsiError) as e:      # no partition yet
        plan.forward_subset(0, f)
    assert e.value.status == 1
    sub = caxsi.os_partition(g.M, g.N, g.rho_y, 2, 4)
    bad = sub.copy()
    bad[5] = -1
    with pytest.raises(caxsi.CaxsiError) as e:
        plan.set_subsets(bad)
    assert e.value.status == 1
    plan.set_subsets(sub)
    with pytest.raises(caxsi.CaxsiError) as e:      # subset out of range
        plan.forward_subset(plan.n_subsets, f)
    assert e.value.status == 1
    with pytest.raises(caxsi.CaxsiError) as e:      # out of range on the direct path too
        plan.forward_subset(plan.n_subsets, f, path=caxsi.PATHS["direct"])
    assert e.value.status == 1
    assert plan.info()["device_error"] == 0
    plan.close()


def test_direct_and_table_subsets_agree_and_replace_partitions(cx):
    """The direct subset operators (pixel lists) and the table ones (records
    grouped by subset) compute the same A_p; a new partition replaces the old
    one for both (the table records are rebuilt on first use)."""
    caxsi, torch = cx
    g = synth.tiny_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 41)
    plan = caxsi.Plan(g, phi, mask)
    f = _t(torch, synth.uniform_random((g.X, g.J, g.Q), 42))
    w = _t(torch, synth.uniform_random((g.M, g.N), 43) + 0.1)
    D, T = caxsi.PATHS["direct"], caxsi.PATHS["table_fp32"]
    for part in _partitions(caxsi, g).values():
        plan.set_subsets(part)
        for s in range(plan.n_subsets):
            gd = plan.forward_subset(s, f, path=D).cpu().numpy()
            gt = plan.forward_subset(s, f, path=T).cpu().numpy()
            assert rel_l2(gd, gt) <= 1e-5
            assert np.all(gd.ravel()[part != s] == 0)
            fd = plan.adjoint_subset(s, w, path=D).cpu().numpy()
            ft = plan.adjoint_subset(s, w, path=T).cpu().numpy()
            assert rel_l2(fd, ft) <= 1e-5
    assert plan.info()["device_error"] == 0
    plan.close()


def test_paper_scale_subsets_sampled(cx):
    caxsi, torch = cx
    g = synth.paper_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, synth.PAPER_MASK_SEED)
    f = synth.phantom(g, 0)
    w = synth.uniform_random((g.M, g.N), 1) + 0.5
    plan = caxsi.Plan(g, phi, mask)
    sub = caxsi.os_partition(g.M, g.N, g.rho_y, 8, 16)     # 64 subsets, as in the paper
    plan.set_subsets(sub)
    rng = np.random.default_rng(7)
    for s in (0, 27, 63):
        inside = np.flatnonzero(sub == s)
        gp = plan.forward_subset(s, _t(torch, f)).cpu().numpy().ravel()
        pix = rng.choice(inside, 12, replace=False)
        assert rel_l2(gp[pix], oracle.forward_pixels(g, phi, mask, _f32(f), pix)) <= REL_L2_TOL
        assert np.all(np.delete(gp, inside) == 0.0)
        fp = plan.adjoint_subset(s, _t(torch, w)).cpu().numpy().reshape(g.X * g.J, g.Q)
        vox = rng.choice(g.X * g.J, 8, replace=False)
        wm = np.where((sub == s).reshape(g.M, g.N), _f32(w), 0.0)
        assert rel_l2(fp[vox], oracle.adjoint_voxels(g, phi, mask, wm, vox)) <= REL_L2_TOL
    assert plan.info()["device_error"] == 0
    plan.close()


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_sparse_subset_operators_equal_the_contracted_ones(cx, name):
    """The FP32 subset operators contracted per record at the subset's knots
    (default) against the whole-object contractions (CAXSI_OPT_SPARSE_SUBSETS 0),
    for every subset of each partition, and the sensitivities b1_p.  The
    16-subset partition is sparse enough for both sparse operators to be used."""
    caxsi, torch = cx
    g = GEOMS[name]()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 51)
    plan = caxsi.Plan(g, phi, mask)
    P = caxsi.PATHS["table_fp32"]
    f = _t(torch, synth.phantom(g, 5, n_ellipses=3) + 0.05 * synth.uniform_random((g.X, g.J, g.Q), 52))
    w = _t(torch, synth.uniform_random((g.M, g.N), 53) + 0.1)
    ones = torch.ones((g.M, g.N), device="cuda:0")
    parts = list(_partitions(caxsi, g).values())
    parts.append(np.minimum((synth.uniform_random((g.M * g.N,), 54) * 16).astype(np.int32), 15))
    for part in parts:
        plan.set_subsets(part)
        for s in range(plan.n_subsets):
            out = []
            for sparse in (True, False):
                plan.set_sparse_subsets(sparse)
                out.append((plan.forward_subset(s, f, path=P).cpu().numpy(),
                            plan.adjoint_subset(s, w, path=P).cpu().numpy(),
                            plan.adjoint_subset(s, ones, path=P).cpu().numpy()))
            for a, b in zip(*out):
                assert rel_l2(a, b) <= 1e-6
    assert plan.info()["device_error"] == 0
    plan.close()
