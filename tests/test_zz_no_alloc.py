"""art_sort_pairs_static: the radix sort for callers that may not allocate
device memory while they run (a VR or engine frame loop that cannot absorb
the synchronisation of a cudaMalloc mid-frame; a host whose device memory
belongs to a pool allocator).  Its scratch is a fixed array inside the
library; its results must equal those of art_sort_pairs, which allocates its
scratch through the context.

This file is collected last (tests/conftest.py orders it after every other
test) and also runs alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pairs(n, seed):
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    k[: n // 4] = k[n // 4: 2 * (n // 4)]  # repeated keys: the sort must be stable
    v = rng.permutation(n).astype(np.uint32)
    return k, v


def test_static_sort_equals_context_sort_on_two_calls_in_a_row():
    import torch
    import paper_2202_05628_gb300 as art
    r = art.Renderer()
    # two calls in a row with different data, sizes and key widths (24 bits
    # ends on the scratch side of the ping-pong and copies back)
    for call, (n, bits) in enumerate([(300001, 32), (art.SORT_STATIC_MAX_PAIRS, 24)]):
        k, v = _pairs(n, seed=call)
        k_ref = torch.from_numpy(k.view(np.int32)).cuda()
        v_ref = torch.from_numpy(v.view(np.int32)).cuda()
        k_st, v_st = k_ref.clone(), v_ref.clone()
        r.sort_pairs(k_ref, v_ref, bits)
        st = art.sort_pairs_static(k_st, v_st, bits)
        assert st == 0, f"art_sort_pairs_static returned {st}"
        torch.cuda.synchronize()
        assert torch.equal(k_st, k_ref), f"call {call}: keys differ"
        assert torch.equal(v_st, v_ref), f"call {call}: values differ"
        # and both are the stable sort by the low key_bits bits
        order = np.argsort(k.astype(np.uint64) & np.uint64((1 << bits) - 1), kind="stable")
        np.testing.assert_array_equal(k_st.cpu().numpy().view(np.uint32), k[order])
        np.testing.assert_array_equal(v_st.cpu().numpy().view(np.uint32), v[order])


def test_static_sort_rejects_more_than_its_maximum():
    import torch
    import paper_2202_05628_gb300 as art
    n = art.SORT_STATIC_MAX_PAIRS + 1
    k = torch.zeros(n, dtype=torch.int32, device="cuda")
    v = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert art.sort_pairs_static(k, v, 32) == 1  # ART_ERR_INVALID_ARG, nothing launched
    assert art.sort_pairs_static(k[:10], v[:10], 12) == 1  # key_bits not a multiple of 8


def test_static_sort_rejects_host_memory_and_mismatched_arrays():
    import ctypes

    import torch
    import paper_2202_05628_gb300 as art
    # host arrays: refused by the library's pointer check before any launch
    k = np.zeros(64, np.uint32)
    v = np.zeros(64, np.uint32)
    st = art.library().art_sort_pairs_static(k.ctypes.data, v.ctypes.data, 64, 32,
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1  # ART_ERR_INVALID_ARG
    # the binding refuses arrays of different lengths or widths
    kd = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        art.sort_pairs_static(kd, torch.zeros(63, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        art.sort_pairs_static(kd, torch.zeros(64, dtype=torch.int64, device="cuda"))
    # and a valid call still works afterwards
    assert art.sort_pairs_static(kd, torch.arange(64, dtype=torch.int32, device="cuda"), 32) == 0
    torch.cuda.synchronize()
