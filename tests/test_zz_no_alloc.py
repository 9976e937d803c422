"""psi_sort_keys_noalloc: the sort for callers that cannot allocate device
memory (needs a GPU).

Some callers cannot hand the library a workspace: a real-time control thread
that must not wait on an allocator, or a plug-in whose host framework owns all
device memory and passes it only inputs and outputs. For them the sort has an entry point whose scratch is a fixed array
inside the library. Its results must equal those of psi_sort_keys with a
caller workspace, call after call, since every call reuses the same array.

The file name sorts last so that a run stopping at the first failure has run
every other test first; the test also passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import _build, psi
    _build.build()
    return psi.Context(0)


def _sort_both(ctx, keys, vals, cap, bits, n_tiles):
    """Sort the same pairs through both entry points; return both results."""
    from paper_2604_10982_gb300 import psi
    n = len(keys)
    out = []
    for noalloc in (False, True):
        kk = torch.zeros(cap, dtype=torch.int64, device="cuda")
        vv = torch.zeros(cap, dtype=torch.int32, device="cuda")
        kk[:n] = torch.from_numpy(keys.view(np.int64)).cuda()
        vv[:n] = torch.from_numpy(vals.view(np.int32)).cuda()
        npairs = torch.tensor([n], dtype=torch.int64, device="cuda")
        ranges = torch.full((n_tiles * 3,), -1, dtype=torch.int32, device="cuda")
        if noalloc:
            psi.psi_sort_keys_noalloc(ctx, kk, vv, npairs, cap, 0, bits, ranges, n_tiles)
        else:
            ws = torch.empty(psi.sort_workspace_size(cap), dtype=torch.uint8, device="cuda")
            psi.psi_sort_keys(ctx, kk, vv, npairs, cap, 0, bits, ranges, n_tiles, ws)
        torch.cuda.synchronize()
        # tile ranges; the launch-order tail is a schedule (arbitrary among
        # tiles of similar length), so only its being a permutation is checked
        rr = ranges.cpu().numpy()
        assert np.array_equal(np.sort(rr[2 * n_tiles:]), np.arange(n_tiles))
        out.append((kk[:n].cpu().numpy().view(np.uint64), vv[:n].cpu().numpy().view(np.uint32), rr[: 2 * n_tiles]))
    return out


def test_noalloc_sort_matches_workspace_sort_on_consecutive_calls(ctx):
    from paper_2604_10982_gb300 import psi
    rng = np.random.default_rng(2024)
    # two calls in a row with different sizes and key widths: the second call
    # runs on scratch that still holds the first call's contents
    for n, bits, cap in [(700_001, 45, 1 << 20), (123_457, 41, 300_000)]:
        hi = rng.integers(0, 1 << (bits - 32), n, dtype=np.uint64)
        lo = rng.integers(0, 512, n, dtype=np.uint64)  # many equal keys: stability matters
        keys = (hi << np.uint64(32)) | lo
        vals = rng.permutation(n).astype(np.uint32)
        n_tiles = 1 << (bits - 32)
        (k0, v0, r0), (k1, v1, r1) = _sort_both(ctx, keys, vals, cap, bits, n_tiles)
        # the sort is exact: identical keys, values (stable order) and ranges
        assert np.array_equal(k1, k0) and np.array_equal(v1, v0) and np.array_equal(r1, r0)
        perm = np.argsort(keys, kind="stable")
        assert np.array_equal(k1, keys[perm]) and np.array_equal(v1, vals[perm])
    st, _ = ctx.status_fetch()
    assert st == 0


def test_noalloc_sort_rejects_capacity_beyond_limit(ctx):
    from paper_2604_10982_gb300 import psi
    cap = (1 << 20) + 1
    kk = torch.zeros(cap, dtype=torch.int64, device="cuda")
    vv = torch.zeros(cap, dtype=torch.int32, device="cuda")
    npairs = torch.tensor([10], dtype=torch.int64, device="cuda")
    ranges = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(psi.PsiError) as e:
        psi.psi_sort_keys_noalloc(ctx, kk, vv, npairs, cap, 0, 33, ranges, 1)
    assert e.value.code == psi.PSI_ERR_INVALID_ARG
    assert "capacity" in str(e.value)
