"""Failure detection without a GPU fault: a bounded wait for a bulk copy runs
out because the copy was never issued (a test hook of the record forward), the
kernel reports it through the plan's error word and returns, and the plan keeps
working: the next normal call is bit-identical to one made before."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

OPT_SYMMETRY, OPT_TEST_WAIT_LIMIT, OPT_TEST_WITHHOLD_COPY = 2, 6, 7


@pytest.fixture(scope="module")
def cx():
    import torch
    from paper_1603_06400_gb300 import build, caxsi
    build.build()
    return caxsi, torch


def test_a_copy_wait_that_runs_out_is_reported_and_the_plan_recovers(cx, tiny):
    caxsi, torch = cx
    g, phi, mask = tiny
    plan = caxsi.Plan(g, phi, mask)
    plan.set_symmetry(False)          # the forward streams one record per pair (k_fwd_rec)
    T = caxsi.PATHS["table_fp32"]
    f = synth.phantom(g, 3, n_ellipses=3)
    ft = torch.tensor(f, dtype=torch.float32, device="cuda:0")
    good = plan.forward(ft, path=T)
    ref = oracle.forward(g, phi, mask, np.asarray(f, np.float32).astype(np.float64))
    assert np.linalg.norm(good.double().cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)
    assert plan.info()["device_error"] == 0
    y = torch.tensor(synth.poisson_counts(ref * 50.0 / ref.max(), 4), dtype=torch.float32, device="cuda:0")

    set_opt = lambda k, v: caxsi._check(plan.lib.caxsi_plan_set_option(plan.handle, k, v), "set_option")
    set_opt(OPT_TEST_WAIT_LIMIT, 4096)
    set_opt(OPT_TEST_WITHHOLD_COPY, 1)
    plan.forward(ft, path=T)          # launches and returns; the kernel gives up its first wait
    torch.cuda.synchronize()
    assert plan.info()["device_error"] == 1       # reported once, then cleared
    assert plan.info()["device_error"] == 0
    f_rec = ft.clone()
    with pytest.raises(caxsi.CaxsiError) as e:
        plan.recon_step(y, f_rec, path=T, want_nll=True)
    assert e.value.status == 5
    assert torch.equal(f_rec, ft)     # the step stopped before the update

    set_opt(OPT_TEST_WITHHOLD_COPY, 0)
    set_opt(OPT_TEST_WAIT_LIMIT, 0)
    assert torch.equal(plan.forward(ft, path=T), good)
    assert plan.info()["device_error"] == 0
    nll = plan.recon_step(y, f_rec, path=T, want_nll=True)
    assert np.isfinite(nll) and bool(torch.isfinite(f_rec).all())
    plan.close()
