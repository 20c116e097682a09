"""are_risk_measures_static: PML/TVaR without a context and without any
allocation, for callers that cannot allocate device memory (a service whose
memory is reserved up front, or code running under another framework's
memory pool).  Its results must equal those of are_risk_measures, call after
call, although every call reuses the same fixed device scratch array.

This file is collected last on purpose: it passes alone in a fresh process
(where its first call sets the scratch up) and after every other test."""
import numpy as np
import pytest

from gpu_support import rel_close

pytestmark = pytest.mark.gpu

RPS = [100.0, 250.0, 10.0, 1.0]
LEVELS = [0.99, 0.9]


def ylt(seed, n):
    g = np.random.default_rng(seed)
    y = np.round(g.lognormal(14, 2.0, n), 2)
    y[g.random(n) < 0.25] = 0.0
    y[g.random(n) < 0.02] = 1e8          # ties at an aggregate limit
    return y


@pytest.fixture(scope="module")
def are():
    import torch
    assert torch.cuda.is_available()
    import paper_1308_2066_gb300 as are
    are.lib()
    return are


def test_static_matches_context_entry_on_consecutive_calls(are):
    import torch
    ctx = are.are_create(0)
    try:
        cases = [(11, 1_000_000), (12, 4097), (11, 1_000_000)]
        for seed, n in cases:                  # three calls in a row, shared scratch
            d = torch.from_numpy(ylt(seed, n)).cuda()
            p_ref, t_ref = are.are_risk_measures(ctx, d, n, RPS, LEVELS)
            p, t = are.are_risk_measures_static(d, n, RPS, LEVELS)
            np.testing.assert_array_equal(p, p_ref)
            assert rel_close(t, t_ref, 1e-13), (t, t_ref)
            stream = torch.cuda.Stream()
            p2, t2 = are.are_risk_measures_static(d, n, RPS, LEVELS, stream=stream)
            np.testing.assert_array_equal(p2, p)
            np.testing.assert_array_equal(t2, t)
    finally:
        are.are_destroy(ctx)


def test_static_rejects_what_it_cannot_hold(are):
    import torch
    d = torch.from_numpy(ylt(5, 1000)).cuda()
    with pytest.raises(are.AreError) as e:
        are.are_risk_measures_static(d, 1000, [2.0] * 5, [0.9] * 4)
    assert e.value.status == are.ARE_EINVAL and "at most 8" in e.value.message
    with pytest.raises(are.AreError) as e:
        are.are_risk_measures_static(ylt(5, 1000), 1000, [2.0], [])
    assert e.value.status == are.ARE_EINVAL and "device memory" in e.value.message
    with pytest.raises(are.AreError) as e:
        are.are_risk_measures_static(d, 1000, [0.5], [])
    assert e.value.status == are.ARE_EINVAL
    p, t = are.are_risk_measures_static(d, 1000, [2.0], [0.5])   # still usable afterwards
    assert p[0] >= 0 and t[0] >= p[0]
