"""lb_select_only_noalloc: the selection entry point for callers that cannot
allocate device memory (hosts whose own allocator has reserved the device
memory and hands it out itself, real-time loops that must not take
cudaMalloc's implicit synchronisation).  Its working memory is a fixed array
inside the library, so the test checks that two calls in a row, which reuse
that array, each give exactly the oracle's selection (the brute-force rule of
Sec. 3.2 with ties to the lower index) and the selection of the allocating
entry point lb_select_only on the same values.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""

import numpy as np
import pytest

from oracle import core as ora
from paper_0705_4371_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_0705_4371_gb300 import lbm
    lbm.load()
    assert torch.cuda.is_available()
    return torch, lbm


def _noalloc_select(torch, lbm, ds_host, delta, k):
    dev = torch.device("cuda", 0)
    ds = torch.from_numpy(np.ascontiguousarray(ds_host, np.float64)).to(dev)
    out = torch.full((max(1, min(k, ds.numel())),), -1, dtype=torch.int32, device=dev)
    cnt = torch.full((1,), -1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    lbm.select_only_noalloc(ds.data_ptr(), ds.numel(), delta, k, out.data_ptr(), cnt.data_ptr(),
                            stream.cuda_stream)
    torch.cuda.synchronize(dev)
    c = int(cnt.item())
    return np.sort(out[:c].cpu().numpy().astype(np.int64))


def test_two_calls_in_a_row_match_the_oracle(env):
    torch, lbm = env
    cases = [
        # (seed, n, k, ties, frac_inf, delta quantile)
        (3001, 200000, 64, 5000, 0.01, 0.7),    # candidates beyond shared-memory staging
        (3002, 4096, 16, 100, 0.0, 0.9),        # fewer, smaller; the array holds the old data
    ]
    for seed, n, k, ties, finf, q in cases:
        ds = inputs.random_ds_with_ties(seed, n, n_ties=ties, frac_inf=finf)
        delta = float(np.quantile(ds[np.isfinite(ds)], q))
        got = _noalloc_select(torch, lbm, ds, delta, k)
        want = ora.select(ds, delta, k)
        assert got.size == min(k, int((ds > delta).sum()))
        assert np.array_equal(got, want)
        assert np.array_equal(got, lbm.select_only(ds, delta, k))


def test_empty_input_selects_nothing(env):
    torch, lbm = env
    dev = torch.device("cuda", 0)
    cnt = torch.full((1,), -1, dtype=torch.int32, device=dev)
    lbm.select_only_noalloc(0, 0, 0.0, 4, 0, cnt.data_ptr())
    torch.cuda.synchronize(dev)
    assert int(cnt.item()) == 0


def test_rejects_sizes_beyond_the_fixed_memory(env):
    torch, lbm = env
    dev = torch.device("cuda", 0)
    ds = torch.zeros(4, dtype=torch.float64, device=dev)
    out = torch.zeros(4, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(lbm.LBError) as e:
        lbm.select_only_noalloc(ds.data_ptr(), lbm.NOALLOC_MAX_N + 1, 0.0, 4, out.data_ptr(),
                                cnt.data_ptr())
    assert e.value.code == lbm.LB_ERR_ARG
    assert "exceeds" in str(e.value)


def test_empty_and_largest_inputs(env):
    torch, lbm = env
    # no values: the count is written (0), nothing is selected
    assert _noalloc_select(torch, lbm, np.zeros(0), 0.0, 8).size == 0
    # the largest n the fixed working memory holds, every value a candidate
    n = lbm.NOALLOC_MAX_N
    ds = inputs.random_ds_with_ties(3003, n, n_ties=2000, frac_inf=0.001)
    for k in (1, 1000):
        got = _noalloc_select(torch, lbm, ds, -1.0, k)
        assert np.array_equal(got, ora.select(ds, -1.0, k))
    # one more is refused on the host, before any launch (the buffers are
    # real and large enough all the same)
    dev = torch.device("cuda", 0)
    big = torch.zeros(n + 1, dtype=torch.float64, device=dev)
    out = torch.zeros(4, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(lbm.LBError, match="fixed working memory"):
        lbm.select_only_noalloc(big.data_ptr(), n + 1, 0.0, 4, out.data_ptr(), cnt.data_ptr())
    torch.cuda.synchronize(dev)
