"""Helpers of the GPU parity tests: numpy <-> CUDA tensors, a context with keys loaded."""
import numpy as np


def to_dev(a: np.ndarray):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def to_host(t) -> np.ndarray:
    a = t.detach().cpu().numpy()
    return a.view(np.uint32) if a.dtype == np.int32 else a


def empty_dev(*shape):
    import torch
    return torch.empty(shape, dtype=torch.int32, device="cuda")


def make_context(keys, device: int = 0):
    from paper_2407_19871_gb300 import build
    from paper_2407_19871_gb300.locpir import Context
    build.build()
    ctx = Context(device)
    ctx.lp_load_bsk(np.ascontiguousarray(keys.bsk.reshape(-1)))
    ctx.lp_load_ksk(np.ascontiguousarray(keys.ksk.reshape(-1)))
    return ctx


def assert_same(got: np.ndarray, want: np.ndarray, what: str = ""):
    got = np.asarray(got, dtype=np.uint32)
    want = np.asarray(want, dtype=np.uint32)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{what}: {len(bad)} words differ, first at {bad[:5].tolist()}"
