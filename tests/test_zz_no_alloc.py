"""The allocation-free convolution entry point, nvisr_conv2d_static.

Some callers cannot allocate device memory while they run: a process whose
memory is handed out in advance, or real-time work that cannot let cudaFree
synchronise the device.  nvisr_conv2d_static serves them from a fixed device
area.  It runs the same kernels as the allocating nvisr_conv2d on the same
inputs, so its output must be bit-identical to nvisr_conv2d's; it is also held
to the FP64 oracle within the convolution tests' tolerance.  Two calls in a
row (different shapes, with and without a residual) check that the second
call does not see what the first left in the shared area.  This file is
collected last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2308_03121_gb300 as nv

CASES = [
    # cin, cout, H, W, k, act, residual
    (64, 64, 37, 150, 3, 1, True),    # 64 -> 64 3x3: the row-streaming tensor-core kernel
    (16, 48, 17, 70, 3, 0, False),    # ragged channel counts, no residual
]


def _inputs(cin, cout, H, W, k, seed):
    rs = np.random.default_rng(seed)
    x = rs.uniform(-1, 1, size=(cin, H, W)).astype(np.float32)
    w = (rs.normal(size=(cout, cin, k, k)) * np.sqrt(2.0 / (cin * k * k))).astype(np.float32)
    b = rs.uniform(-0.1, 0.1, size=cout).astype(np.float32)
    r = rs.uniform(-1, 1, size=(cout, H, W)).astype(np.float32)
    return x, w, b, r


def _round16(a, prec):
    t = torch.from_numpy(np.asarray(a, np.float32))
    return t.to(torch.bfloat16 if prec == "bf16" else torch.float16).double().numpy()


def _oracle(prec, x, w, b, act, r):
    """FP64 oracle on the operands rounded as the kernel stores them, with its tolerance."""
    if prec == "fp32":
        y = oracle.conv2d_direct(x.astype(np.float64), w.astype(np.float64), b)
    else:
        y = oracle.conv2d_direct(_round16(x, prec), _round16(w, prec), b)
    if act:
        y = oracle.leaky_relu(y)
    if r is not None:
        y = y + r
    ulp = {"fp32": 0.0, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}[prec]
    return y, 2e-5 + ulp * np.abs(y).max()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_conv2d_static_matches_conv2d_on_two_calls_in_a_row(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nv.load()
    for i, (cin, cout, H, W, k, act, res) in enumerate(CASES):
        x, w, b, r = _inputs(cin, cout, H, W, k, 1000 * i + cin)
        xd, wd, bd, rd = (torch.from_numpy(a).cuda() for a in (x, w, b, r))
        rr = rd if res else None
        want = nv.nvisr_conv2d(prec, xd, wd, bd, act, rr)
        got = nv.nvisr_conv2d_static(prec, xd, wd, bd, act, rr)
        torch.cuda.synchronize()
        want = want.cpu().numpy()
        got = got.cpu().numpy()
        # same kernels, same inputs: the same bits
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), (prec, i)
        ref, tol = _oracle(prec, x, w, b, act, r if res else None)
        err = np.abs(got.astype(np.float64) - ref).max()
        assert err < tol, (prec, i, err, tol)


@pytest.mark.skipif(torch.cuda.is_available(), reason="host-side argument checks; run where no GPU is present")
def test_conv2d_static_rejects_oversize_and_bad_precision_before_device_work():
    lib = nv.load()
    fake = ctypes.c_void_p(256)  # never dereferenced: every check returns before any CUDA call
    big = lib.nvisr_conv2d_static(1, fake, 64, 2048, 2048, fake, None, 64, 3, 0, None, fake, None)
    assert big == nv.Status.OVER_BUDGET
    assert b"static scratch area" in lib.nvisr_last_error(None)
    fp8 = lib.nvisr_conv2d_static(3, fake, 64, 8, 8, fake, None, 64, 3, 0, None, fake, None)
    assert fp8 == nv.Status.UNSUPPORTED_FORMAT
    for p in (-1, 4):
        assert lib.nvisr_conv2d_static(p, fake, 64, 8, 8, fake, None, 64, 3, 0, None, fake, None) == \
            nv.Status.INVALID_ARG
