"""Every kernel of the path writes inside its buffers.

A filter created with OPT_GUARD_BANDS surrounds each of its device buffers
(ring, staging planes, weights, activations, DCN and calibration scratch) with
4 KB bands of a known byte pattern; check_guards reads them back after the
run.  The cases cover every kernel family on sizes that leave ragged tiles:
ingest and requantise in several formats, the tuple head, fused residual
blocks, the fused requantise tail, the FP32 SIMT convolutions, FP8 layers, the
generic conv, the 1 x 1 and 1 x 2 output layers with their shuffle, and the
deformable space-time networks (offset head, DCN gather, blend, upsampler
slices, pyramid resampling).
"""
import numpy as np
import pytest
import torch

import paper_2308_03121_gb300 as nv
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nv.load()


def _run_and_check(text, blob, frames, flags, fin, fout, prec, scale):
    """Push every frame, pull every output, then check the guard bands; returns the
    number of outputs and of overwritten buffers."""
    eng = nv.Engine()
    try:
        flt = eng.filter(text, blob, fin, fout, prec, scale, options=nv.OPT_GUARD_BANDS)
        n = 0
        out = flt.alloc_out_host()
        for i, fr in enumerate(frames):
            while flt.push((fr["Y"], fr["U"], fr["V"]), cut=bool(flags[i])) == nv.Status.FULL:
                assert flt.pull(out)[0] == nv.Status.OK
                n += 1
            while flt.ready() > 0:
                assert flt.pull(out)[0] == nv.Status.OK
                n += 1
        flt.flush()
        while flt.pull(out)[0] == nv.Status.OK:
            n += 1
        return n, flt.check_guards()
    finally:
        eng.close()


TUPLE_CASES = [
    # prec, W, H, bits, sub, scale (sx, sy)
    ("bf16", 300, 38, 10, "420", (2, 2)),   # fused blocks, fused requantise tail, 3 column tiles
    ("fp32", 70, 24, 8, "420", (2, 2)),     # SIMT convolutions, pack, separate requantise
    ("fp8", 136, 40, 10, "420", (2, 2)),    # FP8 trunk layers and copies, calibration
    ("bf16", 70, 24, 8, "444", (2, 2)),     # 4:4:4 ingest and requantise
    ("bf16", 96, 20, 10, "420", (1, 1)),    # same-size output layer (generic conv, planar shuffle)
    ("bf16", 96, 20, 10, "420", (1, 2)),    # one-axis 2x output layer
]


@pytest.mark.parametrize("prec,W,H,bits,sub,scale", TUPLE_CASES)
def test_tuple_filter_stays_inside_its_buffers(prec, W, H, bits, sub, scale):
    sx, sy = scale
    n_in = 8
    frames = synth.frames_textured(synth.BASE_SEED + 70 + W, n_in, W, H, bits, sub, "limited")
    flags = np.zeros(n_in, bool)
    flags[5] = True
    text, blob = synth.net_tuple(synth.BASE_SEED + 71, frames=5, channels=64, nres=3, scale=(sx, sy))
    fin = nv.fmt(W, H, bits, sub, "limited")
    fout = nv.fmt(W * sx, H * sy, bits, sub, "limited")
    n, bad = _run_and_check(text, blob, frames, flags, fin, fout, prec, (sx, sy))
    assert n == n_in
    assert bad == 0


@pytest.mark.parametrize("net", ["stvsr4x", "pyramid"])
def test_space_time_filter_stays_inside_its_buffers(net):
    W, H, n_in = 144, 72, 5
    frames = synth.frames_textured(synth.BASE_SEED + 72, n_in, W, H, 8, "420", "limited")
    flags = np.zeros(n_in, bool)
    flags[3] = True
    text, blob = synth.net_stvsr4x() if net == "stvsr4x" else synth.net_group_pyramid(synth.BASE_SEED + 73)
    n, bad = _run_and_check(text, blob, frames, flags, nv.fmt(W, H, 8), nv.fmt(4 * W, 4 * H, 8), "bf16", 4)
    assert n == 2 * n_in
    assert bad == 0


def test_guard_check_reports_an_overwritten_band():
    """The check itself: a byte written into a band from the host is reported."""
    W, H = 64, 16
    text, blob = synth.net_tuple(synth.BASE_SEED + 74, frames=3, channels=32, nres=1, scale=2)
    eng = nv.Engine()
    try:
        flt = eng.filter(text, blob, nv.fmt(W, H, 8), nv.fmt(2 * W, 2 * H, 8), "bf16", 2,
                         options=nv.OPT_GUARD_BANDS)
        assert flt.check_guards() == 0
        flt.poke_guard(2)
        assert flt.check_guards() == 1
        assert b"guard bands overwritten" in nv.load().nvisr_last_error(None)
    finally:
        eng.close()
