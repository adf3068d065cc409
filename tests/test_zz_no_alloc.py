"""dot_add_noalloc, the addition entry point that performs no device
allocation (for callers that may not call cudaMalloc), against the CPU oracle
and against dot_add.

Kept in a file of its own that pytest collects last.  It must pass both in a
fresh process and after every other test: each call clears the part of the
library's fixed scratch array it uses, so nothing left there by earlier calls
(of either entry point) can change its results.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, dev, host
from paper_2604_21566_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_21566_gb300 import dot
    dot.lib()
    return dot


CASES = [
    # (limbs, batch, class): tiled look-back path (long ops) and whole-op-in-a-warp path
    (1 << 16, 5, "ones"),     # 16 tiles per op, carry ripples across every tile
    (1 << 14, 9, "runs"),
    (8191, 3, "runs"),        # odd length: 1-limb segments, 1024-limb tiles
    (128, 3000, "uniform"),   # no scratch needed
]


@pytest.mark.parametrize("m,batch,cls", CASES)
def test_matches_dot_add_two_calls_in_a_row(D, m, batch, cls):
    import torch
    g = W.rng(77 + m)
    for call in range(2):
        x, y = W.class_operands(g, cls, batch, m)
        a, b = dev(x), dev(y)
        s_ref, c_ref = D.add(a, b)
        s, c = D.add_noalloc(a, b)
        torch.cuda.synchronize()
        ws, wc = oracle.add(x, y)
        assert_same(host(s), ws, f"sum vs oracle, call {call}, m={m}")
        assert_same(host(c), wc, f"carry vs oracle, call {call}, m={m}")
        assert_same(host(s), host(s_ref), f"sum vs dot_add, call {call}, m={m}")
        assert_same(host(c), host(c_ref), f"carry vs dot_add, call {call}, m={m}")


def test_in_place_and_limit(D):
    import torch
    g = W.rng(5)
    x, y = W.class_operands(g, "runs", 4, 1 << 13)
    a, b = dev(x), dev(y)
    ws, wc = oracle.add(x, y)
    c = torch.empty(4, dtype=torch.int32, device="cuda")
    D.add_noalloc(a, b, out=a, carry=c)  # result over operand a
    torch.cuda.synchronize()
    assert_same(host(a), ws, "in place")
    assert_same(host(c), wc, "in place, carry")
    # more tiles than the fixed scratch holds: rejected before any launch
    big = torch.zeros((16385, 4096), dtype=torch.int32, device="cuda")
    with pytest.raises(D.DotError) as e:
        D.add_noalloc(big, big, out=big)
    assert e.value.status == D.EUNSUPPORTED
    del big
    # and a call right after still works
    s, c = D.add_noalloc(dev(x), dev(y))
    torch.cuda.synchronize()
    assert_same(host(s), ws, "after rejection")
    assert_same(host(c), wc, "carry after rejection")


def test_caller_device_kept(D):
    """The call makes its device current only for its own duration."""
    import torch
    g = W.rng(9)
    x, y = W.class_operands(g, "runs", 3, 1 << 13)
    torch.cuda.set_device(0)
    before = torch.cuda.current_device()
    s, c = D.add_noalloc(dev(x), dev(y))
    assert torch.cuda.current_device() == before
    torch.cuda.synchronize()
    ws, wc = oracle.add(x, y)
    assert_same(host(s), ws, "sum")
    assert_same(host(c), wc, "carry")
