"""Residual block of a trunk fused into one launch of 2-CTA clusters (nvisr_resblock2d and the
filters' default path): the same values as two single-layer launches, bit for bit, and the FP64
oracle's block within the rounding of the 16-bit activations (Section 3.1's 3x3 residual blocks)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2308_03121_gb300 as nv
import synth
from gpu_util import fmt_dict, prequant
from test_gpu_filter import lsb_stats, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nv.load()


def _block_inputs(H, W, seed):
    rs = np.random.default_rng(seed)
    x = rs.uniform(-1, 1, size=(64, H, W)).astype(np.float32)
    std = np.sqrt(2.0 / (64 * 9))
    w1 = (rs.normal(size=(64, 64, 3, 3)) * std).astype(np.float32)
    w2 = (rs.normal(size=(64, 64, 3, 3)) * std).astype(np.float32)
    b1 = rs.uniform(-0.1, 0.1, size=64).astype(np.float32)
    b2 = rs.uniform(-0.1, 0.1, size=64).astype(np.float32)
    return x, w1, b1, w2, b2


def _q(prec, a):
    t = torch.from_numpy(np.asarray(a, np.float32))
    return (t.to(torch.bfloat16) if prec == "bf16" else t.half()).double().numpy()


def _run(prec, x, w1, b1, w2, b2, fused):
    c = lambda a: torch.from_numpy(a).cuda()
    y = nv.nvisr_resblock2d(prec, c(x), c(w1), c(b1), c(w2), c(b2), fused=fused)
    torch.cuda.synchronize()
    return y.cpu().numpy()


# (H, W): one, two, three column tiles of 126 pixels with ragged last tiles; a single row; a
# single column; 1080p (76 clusters, strips crossing column tiles)
SIZES = [(70, 136), (37, 300), (130, 126), (200, 253), (1, 5), (9, 1), (1080, 1920)]


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("H,W", SIZES)
def test_fused_block_equals_two_launches(prec, H, W):
    x, w1, b1, w2, b2 = _block_inputs(H, W, 7 * W + H)
    fused = _run(prec, x, w1, b1, w2, b2, True)
    plain = _run(prec, x, w1, b1, w2, b2, False)
    assert np.isfinite(fused).all()
    bad = np.argwhere(fused != plain)
    assert bad.size == 0, (len(bad), bad[:5])


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("H,W", [(37, 300), (70, 136)])
def test_fused_block_matches_oracle(prec, H, W):
    x, w1, b1, w2, b2 = _block_inputs(H, W, 11 * W + H)
    got = _run(prec, x, w1, b1, w2, b2, True).astype(np.float64)
    # operands rounded as the kernel stores them, h rounded to the activation type, FP64 sums
    xq = _q(prec, x)
    h = _q(prec, oracle.leaky_relu(oracle.conv2d_direct(xq, _q(prec, w1), b1)))
    ref = oracle.conv2d_direct(h, _q(prec, w2), b2) + xq
    ulp = 2.0 ** -8 if prec == "bf16" else 2.0 ** -11
    tol = 2e-5 + ulp * np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err < tol, (err, tol)


def test_fused_block_timeout_drill_leaves_context_usable():
    """A fused block whose input never arrives: rank 0's wait runs out, both CTAs of each cluster
    give up and the call reports NVISR_DEVICE_TIMEOUT; the next call runs normally."""
    x, w1, b1, w2, b2 = _block_inputs(20, 140, 5)
    nv.nvisr_test_starve(1)
    try:
        with pytest.raises(nv.NvisrError) as ei:
            _run("bf16", x, w1, b1, w2, b2, True)
    finally:
        nv.nvisr_test_starve(0)
    assert ei.value.status == nv.Status.DEVICE_TIMEOUT
    fused = _run("bf16", x, w1, b1, w2, b2, True)
    plain = _run("bf16", x, w1, b1, w2, b2, False)
    assert np.array_equal(fused, plain)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_filter_fused_blocks_equal_unfused(prec):
    """A tuple network's trunk (10-bit 4:2:0, 300 x 38, a cut before frame 3) with its residual
    blocks fused (the default) and as two launches each (NVISR_OPT_UNFUSED_BLOCKS): the same
    codes, and the oracle within 1 LSB."""
    W, H, N = 300, 38, 5
    frames = synth.frames_textured(synth.BASE_SEED + 91, N, W, H, 10, "420", "limited")
    flags = np.zeros(N, bool)
    flags[3] = True
    text, blob = synth.net_tuple(synth.BASE_SEED + 92, frames=5, channels=64, nres=3, scale=2)
    fi = nv.fmt(W, H, 10, "420", "limited")
    fo = nv.fmt(2 * W, 2 * H, 10, "420", "limited")
    fused, _ = run_gpu(text, blob, frames, flags, fi, fo, prec)
    plain, _ = run_gpu(text, blob, frames, flags, fi, fo, prec, options=nv.OPT_UNFUSED_BLOCKS)
    assert len(fused) == len(plain) == N
    for a, b in zip(fused, plain):
        for k in "YUV":
            assert np.array_equal(a[k], b[k]), (k, np.argwhere(a[k] != b[k])[:5])
    fdo = fmt_dict(2 * W, 2 * H, 10, "420", "limited")
    ref = oracle.run_filter(frames, flags, text, blob, fmt_dict(W, H, 10, "420", "limited"), fdo, keep_float=True)
    for got, r in zip(fused, ref):
        pq = prequant(r, fdo)
        mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], 10) for k in "YUV"})
        assert mx <= 1, mx


def test_group_filter_fused_blocks_equal_unfused():
    """A space-time group network (deformable alignment, then trunks of residual blocks on two
    feature maps): fused blocks give the same codes as two launches per block."""
    W, H, N = 96, 48, 5
    frames = synth.frames_textured(synth.BASE_SEED + 93, N, W, H, 8, "420", "limited")
    flags = np.zeros(N, bool)
    flags[2] = True
    text, blob = synth.net_group_stvsr(synth.BASE_SEED + 94, nres=2)
    fi, fo = nv.fmt(W, H, 8), nv.fmt(4 * W, 4 * H, 8)
    fused, _ = run_gpu(text, blob, frames, flags, fi, fo, "bf16", scale=4)
    plain, _ = run_gpu(text, blob, frames, flags, fi, fo, "bf16", scale=4, options=nv.OPT_UNFUSED_BLOCKS)
    assert len(fused) == len(plain) > 0
    for a, b in zip(fused, plain):
        for k in "YUV":
            assert np.array_equal(a[k], b[k]), (k, np.argwhere(a[k] != b[k])[:5])
