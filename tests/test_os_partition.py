"""The package's ordered-subset partition (host logic) against the oracle's
loop-by-loop restatement of Sec. VI and the paper's worked example."""
import os

import numpy as np
import pytest

import oracle
from paper_1603_06400_gb300 import caxsi

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _oracle_ids(M, N, sigma_y, rho_z):
    ids = np.full((M, N), -1, dtype=np.int64)
    for k, (rows, cols) in enumerate(oracle.os_subsets(M, N, sigma_y, rho_z)):
        ids[np.ix_(rows - 1, cols - 1)] = k
    return ids.reshape(-1)


@pytest.mark.parametrize("M,N,rho_y,rho_z,sigma_y", [
    (32, 64, 16, 8, 16),     # the worked example
    (64, 256, 1, 8, 16),     # paper-scale detector, translation step 1
    (16, 64, 2, 2, 4),
    (16, 64, 2, 8, 2),
    (8, 16, 2, 1, 16),
])
def test_partition_matches_oracle(M, N, rho_y, rho_z, sigma_y):
    got = caxsi.os_partition(M, N, rho_y, rho_z, sigma_y)
    np.testing.assert_array_equal(got, _oracle_ids(M, N, sigma_y, rho_z))
    assert got.dtype == np.int32 and got.min() == 0 and got.max() == rho_z * sigma_y // 2 - 1


def test_partition_worked_example_first_subset():
    txt = [ln.split() for ln in open(os.path.join(GOLD, "os_partition_32x64.txt"))
           if ln.strip() and not ln.startswith("#")]
    kv = {t[0]: [int(v) for v in t[1:]] for t in txt}
    M, N = kv["M"][0], kv["N"][0]
    ids = caxsi.os_partition(M, N, kv["rho_y"][0], kv["rho_z"][0]).reshape(M, N)
    assert ids.max() + 1 == kv["n_subsets"][0]
    rows, cols = np.nonzero(ids == 0)
    assert sorted(set(cols + 1)) == sorted(kv["cols"])
    assert sorted(set(rows + 1)) == sorted(kv["rows"])


def test_partition_keeps_the_mirror_and_translation_classes():
    M, N, rho_y = 16, 64, 4
    ids = caxsi.os_partition(M, N, rho_y, 4, 8).reshape(M, N)
    np.testing.assert_array_equal(ids, ids[::-1, :])              # up-down mirror
    np.testing.assert_array_equal(ids, ids[:, ::-1])              # left-right mirror
    np.testing.assert_array_equal(ids[:, 8:], ids[:, :-8])        # the column step


def test_partition_rejects_bad_steps():
    with pytest.raises(ValueError):
        caxsi.os_partition(16, 64, 2, 3)        # rho_z does not divide M/2
    with pytest.raises(ValueError):
        caxsi.os_partition(16, 64, 4, 2, 6)     # sigma_y not a multiple of rho_y
    with pytest.raises(ValueError):
        caxsi.os_partition(16, 60, 2, 2, 8)     # sigma_y does not divide N
