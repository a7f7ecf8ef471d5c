"""The allocation-free sort entry point (nvgs_sort_pairs_noalloc), for callers that cannot call
cudaMalloc -- for example a plugin whose host application owns all device memory, or a real-time
loop that cannot take cudaMalloc's implicit synchronisation.  Its output must equal that of the
regular, context-owned sort (nvgs_sort_pairs) bit for bit, call after call, even though every call
reuses the same fixed scratch array.  This file is named to be collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def N():
    from paper_2511_19202_b300 import build
    build.build()
    from paper_2511_19202_b300 import nvgs
    return nvgs


def _pairs(n, bits, seed, high_bits=False):
    """n keys below 2^bits with many repeats; with high_bits, random bits above key_bits too
    (the sort must ignore them)."""
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 1 << min(bits, 62), n, dtype=np.uint64)
    if bits > 62:
        keys |= rng.integers(0, 4, n, dtype=np.uint64) << np.uint64(62)
    keys[: n // 3] = keys[n // 3: 2 * (n // 3)]          # plenty of equal keys: stability matters
    if high_bits:
        assert 1 <= bits < 64
        keys |= rng.integers(0, 1 << (63 - bits), n, dtype=np.uint64) << np.uint64(bits)
    return keys, np.arange(n, dtype=np.uint32)[::-1].copy()


# (n, key bits, random bits above key_bits): 6, 8 and 2 passes (even), 1 and 3 passes (odd: the
# result comes back from the shared scratch array), and keys with bits set above key_bits
CASES = [(N_MAX := 1 << 20, 45, False), (77_777, 64, False), (8193, 13, False),
         (100_003, 8, False), (300_001, 20, False), (65_537, 13, True), (4097, 20, True)]


def test_noalloc_sort_matches_the_regular_sort_on_consecutive_calls(N):
    assert N.NVGS_SORT_NOALLOC_MAX_PAIRS == N_MAX
    ctx = N.nvgs_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        stream = torch.cuda.current_stream()
        for call, (n, bits, high) in enumerate(CASES):
            keys, vals = _pairs(n, bits, call, high)
            k_ref = torch.from_numpy(keys.view(np.int64)).cuda()
            v_ref = torch.from_numpy(vals.view(np.int32)).cuda()
            k_new, v_new = k_ref.clone(), v_ref.clone()
            N.nvgs_sort_pairs(ctx, k_ref, v_ref, n, bits)
            st = N.nvgs_sort_pairs_noalloc(k_new, v_new, n, bits, stream)
            assert st == N.NVGS_OK
            torch.cuda.synchronize()
            assert torch.equal(k_new, k_ref) and torch.equal(v_new, v_ref), f"call {call}"
            low = keys & np.uint64((1 << bits) - 1) if bits < 64 else keys
            order = np.argsort(low, kind="stable")
            np.testing.assert_array_equal(v_new.cpu().numpy().view(np.uint32), vals[order])
            np.testing.assert_array_equal(k_new.cpu().numpy().view(np.uint64), keys[order])
    finally:
        N.nvgs_destroy(ctx)


def test_noalloc_sort_rejects_oversized_input(N):
    n = N.NVGS_SORT_NOALLOC_MAX_PAIRS + 1
    k = torch.zeros(n, dtype=torch.int64, device="cuda")
    v = torch.arange(n, dtype=torch.int32, device="cuda")
    assert N.nvgs_sort_pairs_noalloc(k, v, n, 32, None) == N.NVGS_ERR_CAPACITY
    assert N.nvgs_sort_pairs_noalloc(k, v, 5, 65, None) == N.NVGS_ERR_INVALID_ARG
