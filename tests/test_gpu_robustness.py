"""Failure paths that are safe to exercise on a GPU, by injection on the host.

* Out of memory: SOFA_TEST_MEM_CAP makes every device allocation larger
  than the cap fail as if the device were full.  Each call then returns
  SOFA_ERR_OOM (a constructor NULL), and the index is left as it was: once
  the cap is lifted it answers the oracle's k-NN, and it can still grow.
* A bounded device wait: sofa_wait_selftest waits on a barrier that nothing
  completes; the wait gives up after its limit, the call reports
  SOFA_ERR_TIMEOUT, and the context stays usable.  No copy, MMA or tensor
  memory is in flight when it gives up.
"""
import time

import numpy as np
import pytest
import torch

from oracle import sofa_oracle as orc
from paper_2411_17483_gb300 import datagen

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
OOM = -2


@pytest.fixture(scope="module")
def sofa():
    from paper_2411_17483_gb300 import sofa as s
    s.load()
    return s


def assert_knn_equal(gi, gd, oi, od):
    gi = gi.cpu().numpy()
    gd = gd.cpu().numpy().astype(np.float64)
    assert np.array_equal(gi, oi)
    assert np.array_equal(gd.astype(np.float32), od.astype(np.float32))


def test_allocation_cap_gives_oom_and_keeps_the_index(sofa, monkeypatch):
    n = 128
    x = datagen.random_walks(40000, n, seed=701, device=DEV)
    extra = datagen.random_walks(2000, n, seed=702, device=DEV)
    q = datagen.half_perturbed_queries(x, 32, seed=703)
    ix = sofa.Index(x, 16, 256, precision=1)
    ix.set_tuning(series_bound=1, refine_filter=1)
    z, _, _ = orc.znorm(x.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    oi, od = orc.knn(z, zq, 3)
    gi, gd = ix.query(q, 3)
    assert_knn_equal(gi, gd, oi, od)

    # a cap below the insert's temporaries: refused before any change
    monkeypatch.setenv("SOFA_TEST_MEM_CAP", str(1 << 19))
    with pytest.raises(sofa.SofaError) as e:
        ix.insert(extra)
    assert e.value.code == OOM
    assert ix.info()["N"] == x.shape[0] and ix.info()["appended"] == 0
    # a cap above the temporaries but below the grown arrays: the allocate-all
    # phase fails and the index is unchanged
    monkeypatch.setenv("SOFA_TEST_MEM_CAP", str(4 << 20))
    with pytest.raises(sofa.SofaError) as e:
        ix.insert(extra[:500])
    assert e.value.code == OOM and "unchanged" in str(e.value)
    assert ix.info()["N"] == x.shape[0]
    # the query scratch cannot be regrown under a tight cap either
    monkeypatch.setenv("SOFA_TEST_MEM_CAP", str(1 << 10))
    with pytest.raises(sofa.SofaError) as e:
        ix.query(q, 3)
    assert e.value.code == OOM
    with pytest.raises(sofa.SofaError):
        sofa.Index(x[:5000].contiguous(), 8, 256)

    # lifted: the same exact answers, and the index still grows
    monkeypatch.delenv("SOFA_TEST_MEM_CAP")
    gi, gd = ix.query(q, 3)
    torch.cuda.synchronize()
    assert ix.status() == 0
    assert_knn_equal(gi, gd, oi, od)
    ix.insert(extra)
    X = torch.cat([x, extra])
    zx, _, _ = orc.znorm(X.cpu().numpy())
    oi2, od2 = orc.knn(zx, zq, 3)
    gi, gd = ix.query(q, 3)
    assert_knn_equal(gi, gd, oi2, od2)
    ix.close()


def test_bounded_wait_runs_out_and_the_context_survives(sofa):
    lib = sofa.load()
    t0 = time.perf_counter()
    rc = lib.sofa_wait_selftest(50, None)
    el = time.perf_counter() - t0
    assert rc == -4 and "ran out" in lib.sofa_last_error().decode()
    assert el >= 0.05
    assert lib.sofa_wait_selftest(0, None) == -1 and lib.sofa_wait_selftest(5000, None) == -1
    # the context is fine: a query right after answers exactly
    x = datagen.random_walks(5000, 64, seed=711, device=DEV)
    q = datagen.random_walks(8, 64, seed=712, device=DEV)
    ix = sofa.Index(x, 8, 256, precision=1)
    ix.set_tuning(series_bound=1)
    gi, gd = ix.query(q, 2)
    torch.cuda.synchronize()
    assert ix.status() == 0
    z, _, _ = orc.znorm(x.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    oi, od = orc.knn(z, zq, 2)
    assert_knn_equal(gi, gd, oi, od)
    ix.close()
