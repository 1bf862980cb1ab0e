"""Helpers shared by the GPU tests: host <-> device transfers of uint32 data
(carried in int32 tensors, bit-identical) and the seeded input recipes."""
import numpy as np
import torch


def dev(a: np.ndarray, pad_front: int = 0) -> torch.Tensor:
    """Copy a uint32 numpy array to the GPU (optionally at an element offset,
    to exercise unaligned operands); returns a view of exactly len(a)."""
    a = np.ascontiguousarray(a, dtype=np.uint32)
    t = torch.zeros(a.shape[0] + pad_front + 4, dtype=torch.int32, device="cuda")
    if a.size:
        t[pad_front:pad_front + a.shape[0]].copy_(torch.from_numpy(a.view(np.int32)))
    return t[pad_front:pad_front + a.shape[0]]


def dev2(a: np.ndarray, ld: int | None = None) -> torch.Tensor:
    """Row-major uint32 matrix on the GPU with leading dimension ld >= cols."""
    a = np.ascontiguousarray(a, dtype=np.uint32)
    m, k = a.shape
    ld = k if ld is None else ld
    t = torch.zeros((m, ld), dtype=torch.int32, device="cuda")
    if a.size:
        t[:, :k].copy_(torch.from_numpy(a.view(np.int32)))
    return t[:, :k]


def host(t: torch.Tensor) -> np.ndarray:
    return t.contiguous().cpu().numpy().view(np.uint32)


def empty(n: int) -> torch.Tensor:
    return torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
