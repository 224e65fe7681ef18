"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs."""
import numpy as np
import pytest

BAND_F32 = float(np.float32(1e-5))   # the library's default band, as the kernels see it
BAND_BF16 = float(np.float32(1e-3))


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_06743_gb300 as sng
    sng.lib()
    return torch, sng


def padded(torch, x: np.ndarray, ld: int, dtype=None):
    """Device copy of x with row stride ld (>= d); padding columns hold 7.0
    so that any read past d shows up as a wrong distance."""
    n, d = x.shape
    buf = torch.full((n, ld), 7.0, dtype=torch.float32, device="cuda")
    buf[:, :d] = torch.from_numpy(x).cuda()
    v = buf[:, :d]
    if dtype is not None:
        v = v.to(dtype)
    return v, buf
