"""The allocation-free lower-bound entry point gives the same output as the
allocating one, call after call.

Some callers cannot let the library allocate device memory during a call
(their memory budget is spent, their allocator is their own, or the call sits
in a loop that cannot take an allocation's synchronisation).  For them
sofa_lower_bounds_noalloc works out of a fixed array in the library's device
image.  This file is collected last, so a run that stops at the first failure
has run every other test first."""
import pytest
import torch

from paper_2411_17483_gb300 import datagen

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_noalloc_matches_allocating_entry_point_twice():
    from paper_2411_17483_gb300 import sofa
    sofa.load()
    x = datagen.random_walks(30000, 128, seed=51, device=DEV)
    ix = sofa.Index(x, 16, 256)
    for q in (datagen.random_walks(37, 128, seed=52, device=DEV),
              datagen.half_perturbed_queries(x, 211, seed=53)):
        ref = ix.lower_bounds(q)
        # fill the output with garbage first: every entry must be written
        out = torch.full((q.shape[0], ix.N), float("nan"), device=DEV)
        got = sofa.lower_bounds_noalloc(ix, q, out)
        torch.cuda.synchronize()
        # the same kernels on the same inputs: bit-identical bounds
        assert torch.equal(got, ref)
    ix.close()


def test_noalloc_rejects_oversized_batches():
    from paper_2411_17483_gb300 import sofa
    x = datagen.random_walks(2000, 256, seed=54, device=DEV)
    ix = sofa.Index(x, 16, 256)
    qmax = (1 << 22) // (256 + 32)
    q = torch.zeros((qmax + 1, 256), device=DEV)
    out = torch.empty((1, 1), device=DEV)          # never touched: the call is refused first
    with pytest.raises(sofa.SofaError) as e:
        sofa.lower_bounds_noalloc(ix, q, out)
    assert e.value.code == -1 and "allocation-free work space" in str(e.value)
    ix.close()
