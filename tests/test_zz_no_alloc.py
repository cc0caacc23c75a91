"""The allocation-free sketch entry point against the allocating one.

Collected last on purpose (file name), so that a run stopping at its first
failure has already run every other test.  It must also pass alone in a fresh
process: the first call on the device performs the scratch look-up.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from paper_2605_22281_gb300 import api as G  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(autouse=True)
def _needs_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test selected but no CUDA device is available")


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    cases = [(42, 600, 8, 70001, 1), (7, 200, 3, 5460, 2), (42, 600, 8, 70001, 3), (9, 1024, 16, 4097, 4)]
    for seed, s, zeta, n, vseed in cases:       # consecutive calls share the scratch
        v = torch.as_tensor(np.random.default_rng(vseed).standard_normal(n), device="cuda")
        want = G.sketch_apply(seed, s, zeta, v).cpu().numpy()
        got1 = G.sketch_apply_noalloc(seed, s, zeta, v).cpu().numpy()
        got2 = G.sketch_apply_noalloc(seed, s, zeta, v).cpu().numpy()
        assert _rel(got1, want) <= 1e-14
        assert np.array_equal(got1, got2)


def test_noalloc_writes_into_a_preallocated_output():
    """With `out` given, neither the C entry point nor the wrapper allocates;
    the result lands in the caller's buffer (longer than s is allowed), on two
    calls in a row."""
    seed, s, zeta, n = 5, 333, 8, 20011
    v = torch.as_tensor(np.random.default_rng(6).standard_normal(n), device="cuda")
    want = G.sketch_apply(seed, s, zeta, v).cpu().numpy()
    out = torch.full((s + 7,), 7.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        got = G.sketch_apply_noalloc(seed, s, zeta, v, out=out)
        assert got.data_ptr() == out.data_ptr()
        assert _rel(out[:s].cpu().numpy(), want) <= 1e-14
    assert torch.all(out[s:] == 7.0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    v = torch.ones(100, dtype=torch.float64, device="cuda")
    with pytest.raises(G.N.SflError) as e:
        G.sketch_apply_noalloc(1, 1025, 8, v)
    assert e.value.status == G.N.SFL_EINVAL
