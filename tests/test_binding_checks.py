"""The Python binding rejects buffers the C entry points cannot check (their
lengths, dtypes, layout and device) before anything is launched.  Runs on the
CPU: every case here fails in the binding's checks, so no kernel starts."""
import pytest
import torch

from paper_1907_02289_gb300 import bh


def _sort_args(n=16):
    return [torch.zeros(n, dtype=torch.int64), torch.zeros(n, dtype=torch.int32),
            torch.zeros(n, dtype=torch.int64), torch.zeros(n, dtype=torch.int32)]


@pytest.mark.parametrize("pos,bad,msg", [
    (1, torch.zeros(15, dtype=torch.int32), "elements"),       # short idx
    (2, torch.zeros(15, dtype=torch.int64), "elements"),       # short keys_tmp
    (3, torch.zeros(16, dtype=torch.int64), "dtype"),          # idx_tmp of the wrong dtype
    (0, torch.zeros(16, dtype=torch.float64), "dtype"),        # keys of the wrong dtype
    (2, torch.zeros(32, dtype=torch.int64)[::2], "contiguous"),  # strided keys_tmp
    (1, [0] * 16, "torch tensor"),
])
def test_sort_rejects_bad_buffers(pos, bad, msg):
    args = _sort_args()
    args[pos] = bad
    with pytest.raises(ValueError, match=msg):
        bh.bh_sort_keys_static(*args)


def test_sort_rejects_host_tensors():
    with pytest.raises(ValueError, match="CUDA tensor"):
        bh.bh_sort_keys_static(*_sort_args())


@pytest.mark.parametrize("which,bad,msg", [
    ("hi", torch.zeros(7, dtype=torch.float32), "elements"),
    ("lo", torch.zeros(8, dtype=torch.float64), "dtype"),
    ("v", torch.zeros(8, dtype=torch.float32), "dtype"),
    ("hi", torch.zeros(16, dtype=torch.float32)[::2], "contiguous"),
])
def test_split_rejects_bad_buffers(which, bad, msg):
    a = {"v": torch.zeros(8, dtype=torch.float64), "hi": torch.zeros(8, dtype=torch.float32),
         "lo": torch.zeros(8, dtype=torch.float32)}
    a[which] = bad
    with pytest.raises(ValueError, match=msg):
        bh.bh_split_f32(a["v"], a["hi"], a["lo"])


def test_split_rejects_host_tensors():
    with pytest.raises(ValueError, match="CUDA tensor"):
        bh.bh_split_f32(torch.zeros(8, dtype=torch.float64), torch.zeros(8), torch.zeros(8))
