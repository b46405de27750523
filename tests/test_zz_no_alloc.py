"""The allocation-free convolution entry point, nvisr_conv2d_static, against the
allocating nvisr_conv2d: the same kernels run on buffers carved from a fixed
device area, so the outputs agree within the convolution tests' tolerance.
Two calls in a row (different shapes, with and without a residual) check that
the second call does not see what the first left in the area."""
import ctypes

import numpy as np
import pytest
import torch

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
    return [torch.from_numpy(a).cuda() for a in (x, w, b, r)]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_conv2d_static_matches_conv2d_on_two_calls_in_a_row(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nv.load()
    for i, (cin, cout, H, W, k, act, res) in enumerate(CASES):
        x, w, b, r = _inputs(cin, cout, H, W, k, 1000 * i + cin)
        rr = r if res else None
        want = nv.nvisr_conv2d(prec, x, w, b, act, rr)
        got = nv.nvisr_conv2d_static(prec, x, w, b, act, rr)
        torch.cuda.synchronize()
        want = want.double().cpu().numpy()
        got = got.double().cpu().numpy()
        ulp = {"fp32": 0.0, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}[prec]
        tol = 2e-5 + ulp * np.abs(want).max()
        err = np.abs(got - want).max()
        assert err <= tol, (prec, i, err, tol)


@pytest.mark.skipif(torch.cuda.is_available(), reason="host-side argument checks; run where no GPU is present")
def test_conv2d_static_rejects_oversize_and_fp8_before_device_work():
    lib = nv.load()
    fake = ctypes.c_void_p(256)  # never dereferenced: both checks return before any CUDA call
    big = lib.nvisr_conv2d_static(1, fake, 64, 2048, 2048, fake, None, 64, 3, 0, None, fake, None)
    assert big == nv.Status.OVER_BUDGET
    assert b"static scratch area" in lib.nvisr_last_error()
    fp8 = lib.nvisr_conv2d_static(3, fake, 64, 8, 8, fake, None, 64, 3, 0, None, fake, None)
    assert fp8 == nv.Status.UNSUPPORTED_FORMAT
