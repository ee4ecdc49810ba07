"""bh_sort_keys_static, the sort entry point that allocates nothing, against
the sort inside bh_build_tree (read back with bh_get_keys).  Keys are integers,
so the tolerance is zero: both calls must agree bit for bit.

The file name makes it collect last, so it runs both alone and after every
other GPU test in the same process."""
import numpy as np
import pytest

import oracle as orc
from paper_1907_02289_gb300 import synth

pytestmark = pytest.mark.gpu


def _existing_entry_point(P):
    """Sorted keys and permutation from bh_build_tree + bh_get_keys."""
    from paper_1907_02289_gb300 import bh
    ctx = bh.Context(theta=0.5, n_g=64, n_leaf=8)
    D = bh.Particles(P)
    ctx.bh_build_tree(D)
    k, perm = ctx.bh_get_keys(len(P["x"]))
    ctx.close()
    return k, perm


def _unsorted_keys(P):
    lo, L = orc.root_box(P["x"], P["y"], P["z"])
    return orc.keys(P["x"], P["y"], P["z"], lo, L)


def _static_sort(keys_u64):
    import torch
    from paper_1907_02289_gb300 import bh
    n = len(keys_u64)
    k = torch.from_numpy(keys_u64.view(np.int64).copy()).cuda()
    i = torch.empty(n, dtype=torch.int32, device="cuda")
    kt = torch.empty_like(k)
    it = torch.empty_like(i)
    bh.bh_sort_keys_static(k, i, kt, it)
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint64), i.cpu().numpy().view(np.uint32)


@pytest.fixture(scope="module")
def cases():
    """Two inputs of different sizes (both several tiles with a ragged tail)."""
    out = []
    for n, seed in ((300001, 5), (65537, 6)):
        P = synth.ring(n, seed)
        out.append((_unsorted_keys(P), _existing_entry_point(P)))
    return out


def test_two_consecutive_calls_match_existing_entry_point(cases):
    for keys_u64, (k_ref, perm_ref) in cases:
        k, perm = _static_sort(keys_u64)
        assert np.array_equal(k, k_ref)
        assert np.array_equal(perm, perm_ref)


def test_repeat_call_same_input(cases):
    keys_u64, (k_ref, perm_ref) = cases[0]
    for _ in range(2):
        k, perm = _static_sort(keys_u64)
        assert np.array_equal(k, k_ref) and np.array_equal(perm, perm_ref)


def test_all_bits_and_ties_at_max_size():
    """n = the largest accepted size; keys use all 64 bits and have many ties,
    checked against a stable argsort."""
    from paper_1907_02289_gb300 import bh
    n = bh.BH_SORT_STATIC_MAX_N
    rng = np.random.default_rng(11)
    keys = rng.integers(0, 1 << 12, n, dtype=np.uint64) << np.uint64(52)
    keys |= rng.integers(0, 4, n, dtype=np.uint64)
    k, perm = _static_sort(keys)
    ref = np.argsort(keys, kind="stable").astype(np.uint32)
    assert np.array_equal(perm, ref)
    assert np.array_equal(k, keys[ref])


def test_no_device_memory_taken_after_first_call(cases):
    import torch
    from paper_1907_02289_gb300 import bh
    keys_u64 = cases[1][0]
    n = len(keys_u64)
    k = torch.from_numpy(keys_u64.view(np.int64).copy()).cuda()
    i = torch.empty(n, dtype=torch.int32, device="cuda")
    kt, it = torch.empty_like(k), torch.empty_like(i)
    bh.bh_sort_keys_static(k, i, kt, it)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        bh.bh_sort_keys_static(k, i, kt, it)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_rejects_size_over_max_and_bad_buffers():
    import torch
    from paper_1907_02289_gb300 import bh
    n = bh.BH_SORT_STATIC_MAX_N + 1
    k = torch.zeros(n, dtype=torch.int64, device="cuda")
    i = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(bh.BHError) as e:
        bh.bh_sort_keys_static(k, i, k.clone(), i.clone())
    assert e.value.code == bh.BH_E_INVAL and "largest sort" in str(e.value)
    k1 = torch.zeros(10, dtype=torch.int64, device="cuda")
    i1 = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(bh.BHError) as e:
        bh.bh_sort_keys_static(k1, i1, k1, i1.clone())
    assert e.value.code == bh.BH_E_INVAL
    # partial overlaps: keys_tmp starting inside keys, idx sharing keys' bytes
    big = torch.zeros(20, dtype=torch.int64, device="cuda")
    for args in ((big[0:10], i1, big[5:15], i1.clone()),
                 (big[0:10], big[0:10].view(torch.int32)[0:10], big[10:20], i1.clone())):
        with pytest.raises(bh.BHError) as e:
            bh.bh_sort_keys_static(*args)
        assert e.value.code == bh.BH_E_INVAL and "overlap" in str(e.value)
    k0 = torch.zeros(0, dtype=torch.int64, device="cuda")
    i0 = torch.zeros(0, dtype=torch.int32, device="cuda")
    assert bh.bh_sort_keys_static(k0, i0, k0.clone(), i0.clone()) == bh.BH_OK
