"""Helpers shared by the GPU parity tests (no sorting arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t) -> np.ndarray:
    return t.cpu().numpy()


_M1 = 0xBF58476D1CE4E5B9


def multiset_hash(t):
    """Order-independent hash of a device key array (sum of a 64-bit mix)."""
    x = t.to(torch.int64) if t.dtype in (torch.uint32, torch.int32) else t.view(torch.int64)
    x = x * _M1 ^ (x >> 29 & 0x7FFFFFFFF)
    x = x * 0x94D049BB133111EB
    return int(x.sum().item())


def is_sorted_dev(t) -> bool:
    if t.numel() < 2:
        return True
    if t.dtype == torch.uint32:
        x = t.to(torch.int64)
        return bool((x[1:] >= x[:-1]).all().item())
    # uint64: compare as unsigned via the sign-flipped int64 view
    x = t.view(torch.int64) ^ torch.iinfo(torch.int64).min
    return bool((x[1:] >= x[:-1]).all().item())
