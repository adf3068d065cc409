"""Helpers for the GPU parity tests: move uint32 limb arrays to and from the
device (int32 tensors carry the same 32 bits) and report the first mismatch."""
import numpy as np


def dev(x):
    import torch
    x = np.ascontiguousarray(x)
    if x.dtype == np.uint32:
        x = x.view(np.int32)
    elif x.dtype == np.uint64:
        x = x.view(np.int64)
    return torch.from_numpy(x).cuda()


def host(t):
    x = t.cpu().numpy()
    if x.dtype == np.int32:
        return x.view(np.uint32)
    if x.dtype == np.int64:
        return x.view(np.uint64)
    return x


def assert_same(got, want, what=""):
    got = np.asarray(got)
    want = np.asarray(want)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        idx = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} mismatches; first at {idx}: "
                             f"got {got[idx]:#x} want {want[idx]:#x}")
