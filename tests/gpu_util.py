"""Helpers for the GPU parity tests: numpy <-> torch limb arrays."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def to_dev(x: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32).view(np.int32)).cuda()


def to_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def assert_limbs_equal(got: np.ndarray, want: np.ndarray, what: str = ""):
    assert got.shape == want.shape, (what, got.shape, want.shape)
    if not np.array_equal(got, want):
        rows = np.unique(np.argwhere(got != want)[:, 0])
        r = int(rows[0])
        cols = np.argwhere(got[r] != want[r])[:5, 0].tolist()
        raise AssertionError(f"{what}: {rows.size} rows differ; first row {r}, limbs {cols}")
