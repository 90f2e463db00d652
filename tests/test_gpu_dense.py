"""Dense tensor-core form of the query: its approximate squared distances
stay within the derived bound M of the FP64 distances, and the answers it
leads to are the oracle's."""
import numpy as np
import pytest
import torch

from oracle import sofa_oracle as orc
from paper_2411_17483_gb300 import datagen

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def sofa():
    from paper_2411_17483_gb300 import sofa as s
    s.load()
    return s


def oracle_knn(x, q, k):
    z, _, _ = orc.znorm(x.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    return orc.knn(z, zq, k)


def tf32_margin(n):
    """The margin the library states for the dense contraction with TF32
    operands; a smaller returned margin shows that FP16 operands were used."""
    u = 2.0 ** -24
    n1 = n * (1 + 4 * u)
    dot = n1 * (2.0 ** -9 + 2.0 ** -20 + n * 2.0 ** -22 * (1 + 2.0 ** -9))
    return (2 * dot + 8.2 * u * n1) * 1.01


# N not a multiple of the 256-series tile, Q not a multiple of the 128-query
# block, n not a multiple of the 32-value k-block (zero-filled tails)
@pytest.mark.parametrize("N,n,Q,gen,precision", [(3000, 256, 200, "rw", 0), (1000, 100, 130, "sin", 0),
                                                 (700, 1024, 64, "sin", 0), (257, 32, 1, "rw", 0),
                                                 (3000, 256, 200, "rw", 2), (700, 1024, 64, "sin", 2),
                                                 (257, 32, 1, "rw", 2), (1500, 96, 129, "sin", 2),
                                                 (900, 100, 70, "sin", 2)])     # n % 8 != 0: TF32
def test_dense_sqdist_within_margin(sofa, N, n, Q, gen, precision):
    """TF32 operands (precision 0) or FP16 operands (precision 2)."""
    x = datagen.random_walks(N, n, seed=N, device=DEV) if gen == "rw" else \
        datagen.sinusoid_mix(N, n, seed=N, device=DEV)
    q = datagen.random_walks(Q, n, seed=N + 1, device=DEV) if gen == "rw" else \
        datagen.sinusoid_mix(Q, n, seed=N + 1, device=DEV)
    ix = sofa.Index(x, 8 if n <= 64 else 16, 256, precision=precision)
    out, margin = sofa.dense_sqdist(ix, q)
    f16 = precision == 2 and n % 8 == 0
    assert (margin < 0.9 * tf32_margin(n)) == f16         # the FP16 bound is the tighter one
    torch.cuda.synchronize()
    perm = ix.perm().numpy().astype(np.int64)         # sorted position -> original row
    z, _, _ = orc.znorm(x.cpu().numpy())
    zq, _, _ = orc.znorm(q.cpu().numpy())
    exact = np.stack([orc.sqdist(z, zq[i]) for i in range(Q)])    # Q x N, original order
    approx = np.empty_like(exact)
    approx[:, perm] = out.cpu().numpy().astype(np.float64)
    err = np.abs(approx - exact)
    assert np.all(np.isfinite(approx))
    assert err.max() <= margin, (err.max(), margin)
    # the bound is not vacuous: TF32 errors are a visible part of it
    assert err.max() > 1e-6 * margin
    ix.close()


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("N,n,l,k,Q,gen", [(20000, 128, 16, 1, 64, "rw"), (20000, 256, 16, 5, 48, "mixed"),
                                           (9000, 96, 16, 16, 16, "sin"), (12000, 1024, 32, 1, 40, "sin"),
                                           (100, 16, 6, 4, 3, "rw")])
def test_dense_knn_matches_oracle(sofa, N, n, l, k, Q, gen, precision):
    if gen == "rw":
        x = datagen.random_walks(N, n, seed=N + n, device=DEV)
    elif gen == "mixed":
        x = datagen.mixed_walks(N, n, seed=N + n, device=DEV)
    else:
        x = datagen.sinusoid_mix(N, n, seed=N + n, device=DEV)
    q = datagen.half_perturbed_queries(x, Q, seed=5)
    ix = sofa.Index(x, l, 256, precision=precision)
    ix.set_tuning(dense=2)
    ix.stats(reset=True)
    gi, gd = ix.query(q, k)
    torch.cuda.synchronize()
    assert ix.status() == 0
    st = ix.stats()
    assert st["dense_passes"] >= 1 and st["dense_pairs"] > 0
    oi, od = oracle_knn(x, q, k)
    gi = gi.cpu().numpy()
    gdv = gd.cpu().numpy().astype(np.float64)
    assert np.array_equal(gi, oi)
    assert np.array_equal(gdv.astype(np.float32), od.astype(np.float32))
    # the scan form gives the same answers
    ix.set_tuning(dense=1)
    gi2, gd2 = ix.query(q, k)
    assert np.array_equal(gi2.cpu().numpy(), gi) and torch.equal(gd2, gd)
    ix.close()


def test_dense_chosen_when_bounds_fail(sofa):
    """High-frequency data: the SFA bound passes nearly every leaf, so the
    automatic mode takes the dense form; answers stay exact."""
    N, n, Q = 40000, 512, 32
    x = datagen.sinusoid_mix(N, n, seed=77, device=DEV)
    q = datagen.sinusoid_mix(Q, n, seed=78, device=DEV)
    ix = sofa.Index(x, 16, 256)
    ix.stats(reset=True)
    gi, gd = ix.query(q, 1)
    torch.cuda.synchronize()
    assert ix.status() == 0
    assert ix.stats()["dense_passes"] >= 1
    oi, od = oracle_knn(x, q, 1)
    assert np.array_equal(gi.cpu().numpy(), oi)
    ix.close()


def test_graph_recording_takes_the_dense_decision(sofa):
    """A recorded graph replays the decision of its shape's eager batch: on
    high-frequency data that batch takes the dense form, so the replays do too
    (the device counters see Q x N dense pairs per execution and no scanned
    tile), with the same exact answers as the eager batches."""
    N, n, Q = 40000, 512, 32
    x = datagen.sinusoid_mix(N, n, seed=79, device=DEV)
    batches = [datagen.sinusoid_mix(Q, n, seed=80 + i, device=DEV) for i in range(3)]
    ix = sofa.Index(x, 16, 256)
    eager = [ix.query(q, 2) for q in batches]
    ix.set_tuning(use_graph=1)
    ix.stats(reset=True)
    for _ in range(2):                      # first call records, later calls replay
        for q, (ei, ed) in zip(batches, eager):
            gi, gd = ix.query(q, 2)
            torch.cuda.synchronize()
            assert torch.equal(gi, ei) and torch.equal(gd, ed)
    assert ix.status() == 0
    st = ix.stats()
    assert st["graphs_recorded"] == 1 and st["graph_replays"] == 5
    # executions: the recording's eager batch and 5 replays (a capture runs nothing)
    assert st["dense_pairs"] == 6 * Q * N and st["tile_pairs"] == 0, st
    oi, od = oracle_knn(x, batches[0], 2)
    assert np.array_equal(eager[0][0].cpu().numpy(), oi)
    ix.close()
