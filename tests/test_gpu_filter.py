"""End-to-end parity of the filter (push / pull through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2308_03121_gb300 as nv
import synth
from gpu_util import (assert_codes_match, crop_codes, fmt_dict, lsb_stats, oracle_window, prequant,
                      stvsr_window, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nv.load()


def run_gpu(text, blob, frames, flags, fin, fout, prec, scale=2, device_io=False, limit=None, options=0):
    """Push every frame (pulling whenever the ring is full) and pull all outputs."""
    eng = nv.Engine()
    flt = eng.filter(text, blob, fin, fout, prec, scale, options=options)
    outs, infos = [], []

    def pull_one():
        if device_io:
            h = flt.alloc_out_host()
            buf = tuple(to_dev(a) for a in h)
            st, info = flt.pull(buf)
            torch.cuda.synchronize()  # the pull is enqueued on the engine's stream
            res = tuple(b.cpu().numpy() for b in buf)
            res = tuple(r.view(np.uint16) if r.dtype == np.int16 else r for r in res)
        else:
            res = flt.alloc_out_host()
            st, info = flt.pull(res)
        if st == nv.Status.OK:
            outs.append({k: r.astype(np.int64) for k, r in zip("YUV", res)})
            infos.append((info.index, info.src_first, info.src_last, info.kind))
        return st

    for i, fr in enumerate(frames):
        planes = (fr["Y"], fr["U"], fr["V"])
        if device_io:
            planes = tuple(to_dev(p) for p in planes)
        while flt.push(planes, cut=bool(flags[i])) == nv.Status.FULL:
            assert pull_one() == nv.Status.OK
        while flt.ready() > 0 and (limit is None or len(outs) < limit):
            assert pull_one() == nv.Status.OK
    flt.flush()
    while limit is None or len(outs) < limit:
        st = pull_one()
        if st == nv.Status.EOS:
            break
        assert st == nv.Status.OK
    eng.close()
    return outs, infos


def _clip64_t3():
    frames = synth.frames_gradient(synth.BASE_SEED + 1, 16, 64, 64, 8, "420", "full")
    flags = np.zeros(16, bool)
    flags[9] = True
    fd_in = fmt_dict(64, 64, 8, "420", "full")
    fd_out = fmt_dict(128, 128, 8, "420", "full")
    return frames, flags, fd_in, fd_out


@pytest.fixture(scope="module")
def clip64_oracle():
    frames, flags, fdi, fdo = _clip64_t3()
    text, blob = synth.net_sr2x_t3()
    flt = oracle.run_filter(frames, flags, text, blob, fdi, fdo, keep_float=True)
    return [prequant(o, fdo) for o in flt]


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_sr2x_t3_filter_within_1lsb(prec, clip64_oracle):
    frames, flags, fdi, fdo = _clip64_t3()
    text, blob = synth.net_sr2x_t3()
    outs, infos = run_gpu(text, blob, frames, flags, nv.fmt(64, 64, 8, "420", "full"),
                          nv.fmt(128, 128, 8, "420", "full"), prec)
    assert len(outs) == 16
    assert [i[0] for i in infos] == list(range(16))
    assert infos[8][1:3] == (7, 8) and infos[9][1:3] == (9, 10)    # scene cut on frame 9
    for got, pq in zip(outs, clip64_oracle):
        if prec == "fp32":
            assert_codes_match(got, pq, 8)
        else:
            exp = {k: oracle.quantise(pq[k], 8) for k in "YUV"}
            mx, _ = lsb_stats(got, exp)
            assert mx <= 1, mx


def test_sr2x_t3_device_io_matches_host_io():
    frames, flags, _, _ = _clip64_t3()
    text, blob = synth.net_sr2x_t3()
    fi, fo = nv.fmt(64, 64, 8, "420", "full"), nv.fmt(128, 128, 8, "420", "full")
    a, _ = run_gpu(text, blob, frames, flags, fi, fo, "bf16")
    b, _ = run_gpu(text, blob, frames, flags, fi, fo, "bf16", device_io=True)
    for x, y in zip(a, b):
        for k in "YUV":
            assert np.array_equal(x[k], y[k])


def test_scene_cut_poisoning_on_gpu():
    """Frames outside an output's scene never change it (bit-identical)."""
    frames, flags, _, _ = _clip64_t3()
    text, blob = synth.net_sr2x_t3()
    fi, fo = nv.fmt(64, 64, 8, "420", "full"), nv.fmt(128, 128, 8, "420", "full")
    base, _ = run_gpu(text, blob, frames, flags, fi, fo, "bf16")
    poisoned = [dict(f) for f in frames]
    for i in range(9, 16):
        poisoned[i] = {k: np.full_like(v, 255 if k == "Y" else 0) for k, v in frames[i].items()}
    pz, _ = run_gpu(text, blob, poisoned, flags, fi, fo, "bf16")
    for t in range(9):
        for k in "YUV":
            assert np.array_equal(base[t][k], pz[t][k]), (t, k)


def _clip_sr2x_t5_small(W=136, H=70, n=6):
    frames = synth.frames_textured(synth.BASE_SEED + 2, n, W, H, 10, "420", "limited")
    flags = np.zeros(n, bool)
    flags[3] = True
    return frames, flags


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_sr2x_t5_network_ragged_size_full_frames(prec):
    """The 2x SR network (T=5, 10 residual blocks of 64) at 136x70 (ragged 128-pixel tiles, a cut on frame 3), every output."""
    W, H = 136, 70
    frames, flags = _clip_sr2x_t5_small(W, H)
    text, blob = synth.net_sr2x_t5()
    fdi, fdo = fmt_dict(W, H, 10), fmt_dict(2 * W, 2 * H, 10)
    ref = oracle.run_filter(frames, flags, text, blob, fdi, fdo, keep_float=True)
    outs, _ = run_gpu(text, blob, frames, flags, nv.fmt(W, H, 10), nv.fmt(2 * W, 2 * H, 10), prec)
    assert len(outs) == len(frames)
    for got, r in zip(outs, ref):
        pq = prequant(r, fdo)
        if prec == "fp32":
            assert_codes_match(got, pq, 10)
        else:
            mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], 10) for k in "YUV"})
            assert mx <= 1, mx


FULL_WINDOWS = [(0, 16, 0, 16), (0, 16, 1904, 1920), (1064, 1080, 960, 976), (540, 556, 900, 916),
                (200, 216, 120, 136)]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_sr2x_t5_1080p_sampled_windows(prec):
    """1920x1080 10-bit, T = 5: outputs 0 (scene start, edge replication) and 3 on sampled windows."""
    W, H = 1920, 1080
    frames = synth.frames_textured(synth.BASE_SEED + 2, 6, W, H, 10, "420", "limited")
    flags = np.zeros(6, bool)
    text, blob = synth.net_sr2x_t5()
    outs, _ = run_gpu(text, blob, frames, flags, nv.fmt(W, H, 10), nv.fmt(2 * W, 2 * H, 10), prec, limit=4)
    fdi, fdo = fmt_dict(W, H, 10), fmt_dict(2 * W, 2 * H, 10)
    net = oracle.Net(text, blob)
    rgb = [oracle.ingest(f, fdi) for f in frames]
    for t in (0, 3):
        idx = oracle.tuple_indices(t, 5, 0, 5)
        for (y0, y1, x0, x1) in FULL_WINDOWS:
            pq = oracle_window(net, [rgb[i] for i in idx], y0, y1, x0, x1, fdo)
            got = crop_codes(outs[t], y0, y1, x0, x1, 2, "420")
            if prec == "fp32":
                assert_codes_match(got, pq, 10)
            else:
                mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], 10) for k in "YUV"})
                assert mx <= 1, (t, (y0, x0), mx)


# windows of a 3840 x 2160 input: the four corners (the last column tile of the 126-pixel
# fused-block tiles is 60 pixels wide), a tile boundary (126 * 15 = 1890) and the interior
UHD_WINDOWS = [(0, 16, 0, 16), (0, 16, 3824, 3840), (2144, 2160, 0, 16), (2144, 2160, 3824, 3840),
               (1080, 1096, 1882, 1898), (700, 716, 3776, 3792)]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_sr2x_t5_4k_input_sampled_windows(prec):
    """The largest frames of the 2x SR class: 3840x2160 10-bit in, 7680x4320 out (every
    activation over 1 GB), outputs 0 and 2 on sampled windows."""
    W, H = 3840, 2160
    frames = synth.frames_textured(synth.BASE_SEED + 80, 5, W, H, 10, "420", "limited")
    flags = np.zeros(5, bool)
    text, blob = synth.net_sr2x_t5()
    outs, _ = run_gpu(text, blob, frames, flags, nv.fmt(W, H, 10), nv.fmt(2 * W, 2 * H, 10), prec, limit=3)
    fdi, fdo = fmt_dict(W, H, 10), fmt_dict(2 * W, 2 * H, 10)
    net = oracle.Net(text, blob)
    rgb = [oracle.ingest(f, fdi) for f in frames]
    for t in (0, 2):
        idx = oracle.tuple_indices(t, 5, 0, 4)
        for (y0, y1, x0, x1) in UHD_WINDOWS:
            pq = oracle_window(net, [rgb[i] for i in idx], y0, y1, x0, x1, fdo)
            got = crop_codes(outs[t], y0, y1, x0, x1, 2, "420")
            if prec == "fp32":
                assert_codes_match(got, pq, 10)
            else:
                mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], 10) for k in "YUV"})
                assert mx <= 1, (t, (y0, x0), mx)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_seven_frame_tuple_with_one_frame_scenes(prec):
    """The largest tuple (T = 7, 21 input channels) on a ragged size, with scenes of 3, 1,
    1 and 4 frames: every tuple slot of a one-frame scene is that frame."""
    W, H = 136, 38
    n = 9
    frames = synth.frames_textured(synth.BASE_SEED + 81, n, W, H, 10, "420", "limited")
    flags = np.zeros(n, bool)
    flags[[3, 4, 5]] = True
    text, blob = synth.net_tuple(synth.BASE_SEED + 82, frames=7, channels=64, nres=2, scale=2)
    fdi, fdo = fmt_dict(W, H, 10), fmt_dict(2 * W, 2 * H, 10)
    ref = oracle.run_filter(frames, flags, text, blob, fdi, fdo, keep_float=True)
    outs, infos = run_gpu(text, blob, frames, flags, nv.fmt(W, H, 10), nv.fmt(2 * W, 2 * H, 10), prec)
    assert len(outs) == n
    assert [(i[1], i[2]) for i in infos[3:6]] == [(3, 3), (4, 4), (5, 8)]
    for got, r in zip(outs, ref):
        pq = prequant(r, fdo)
        if prec == "fp32":
            assert_codes_match(got, pq, 10)
        else:
            mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], 10) for k in "YUV"})
            assert mx <= 1, mx


STVSR_WINDOWS = [(0, 16, 0, 16), (0, 16, 944, 960), (524, 540, 944, 960), (270, 286, 480, 496),
                 (100, 116, 120, 136)]


@pytest.mark.parametrize("bits,sub,loc,prec,device_io", [
    (10, "420", "left", "bf16", False), (10, "420", "left", "fp16", True), (8, "420", "center", "bf16", False),
    (8, "420", "point", "bf16", True), (8, "444", "left", "bf16", False), (10, "444", "center", "fp16", False)])
def test_fused_requantise_equals_separate_kernel(bits, sub, loc, prec, device_io):
    """Requantise fused into the 2x2 shuffle tail's epilogue (the default for tensor-core tuple
    networks) gives the same codes as the separate requantise kernel (NVISR_OPT_UNFUSED_OUTPUT),
    sample for sample: 300 px wide (three 128-pixel tiles, so LEFT-sited 4:2:0 chroma at two tile
    edges goes through the fix-up), a cut before frame 3; and the oracle within 1 LSB."""
    W, H, N = 300, 38, 5
    frames = synth.frames_textured(synth.BASE_SEED + 83, N, W, H, bits, sub, "limited")
    flags = np.zeros(N, bool)
    flags[3] = True
    text, blob = synth.net_tuple(synth.BASE_SEED + 84, frames=5, channels=64, nres=2, scale=2)
    fi = nv.fmt(W, H, bits, sub, "limited", loc)
    fo = nv.fmt(2 * W, 2 * H, bits, sub, "limited", loc)
    fused, _ = run_gpu(text, blob, frames, flags, fi, fo, prec, device_io=device_io)
    plain, _ = run_gpu(text, blob, frames, flags, fi, fo, prec, device_io=device_io,
                       options=nv.OPT_UNFUSED_OUTPUT)
    assert len(fused) == len(plain) == N
    for a, b in zip(fused, plain):
        for k in "YUV":
            assert np.array_equal(a[k], b[k]), (k, np.argwhere(a[k] != b[k])[:5])
    fdo = fmt_dict(2 * W, 2 * H, bits, sub, "limited", loc)
    ref = oracle.run_filter(frames, flags, text, blob, fmt_dict(W, H, bits, sub, "limited", loc), fdo,
                            keep_float=True)
    for got, r in zip(fused, ref):
        pq = prequant(r, fdo)
        mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], bits) for k in "YUV"})
        assert mx <= 1, mx


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_pyramid_extract_network_matches_oracle(prec):
    """A two-frame space-time network whose extract stage is a three-level feature pyramid
    (Section 3.1), aligned by deformable convs at every level: 96x48 8-bit 4:2:0 -> 4x,
    6 frames with a cut before frame 3, every output against the oracle."""
    W, H, N = 96, 48, 6
    frames = synth.frames_textured(synth.BASE_SEED + 80, N, W, H, 8, "420", "limited")
    flags = np.zeros(N, bool)
    flags[3] = True
    text, blob = synth.net_group_pyramid(synth.BASE_SEED + 81, nres=2)
    fdo = fmt_dict(4 * W, 4 * H, 8)
    ref = oracle.run_filter(frames, flags, text, blob, fmt_dict(W, H, 8), fdo, keep_float=True)
    outs, infos = run_gpu(text, blob, frames, flags, nv.fmt(W, H, 8), nv.fmt(4 * W, 4 * H, 8), prec, scale=4)
    assert len(outs) == len(ref) == 2 * N
    assert [i[1:3] for i in infos] == [(0, 1), (0, 1), (1, 2), (1, 2), (2, 2), (2, 2),
                                       (3, 4), (3, 4), (4, 5), (4, 5), (5, 5), (5, 5)]
    for got, r in zip(outs, ref):
        pq = prequant(r, fdo)
        if prec == "fp32":
            assert_codes_match(got, pq, 8)
        else:
            mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], 8) for k in "YUV"})
            assert mx <= 1, mx


@pytest.mark.parametrize("net", ["pyramid", "stvsr4x"])
def test_extract_cache_reuses_each_frames_features(net):
    """The extract stage's features of a frame are computed once and reused by the next run
    that takes the frame: 6 frames, a cut before frame 3, runs (0,1) (1,2) (2,2) (3,4) (4,5)
    (5,5) compute 2, 1, 1, 2, 1, 1 frames' features (4 hits, 8 misses).  The reused
    features' correctness is what the parity tests of these networks check."""
    W, H, N = 64, 32, 6
    frames = synth.frames_textured(synth.BASE_SEED + 82, N, W, H, 8, "420", "limited")
    flags = np.zeros(N, bool)
    flags[3] = True
    text, blob = (synth.net_group_pyramid(synth.BASE_SEED + 81, nres=1) if net == "pyramid"
                  else synth.net_stvsr4x())
    eng = nv.Engine()
    flt = eng.filter(text, blob, nv.fmt(W, H, 8), nv.fmt(4 * W, 4 * H, 8), "bf16", 4)
    for i, fr in enumerate(frames):
        assert flt.push((fr["Y"], fr["U"], fr["V"]), cut=bool(flags[i])) == nv.Status.OK
    flt.flush()
    outs = []
    while True:
        o = flt.alloc_out_host()
        st, _ = flt.pull(o)
        if st == nv.Status.EOS:
            break
        outs.append(o)
    assert len(outs) == 2 * N
    assert flt.cache_stats() == (4, 8)
    eng.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_stvsr4x_540p_sampled_windows(prec):
    """960x540 8-bit, the deformable ST-SR network in the bench's launch shapes: both outputs
    of the first run on sampled windows (corners, the ragged last column tile, interior)."""
    W, H = 960, 540
    frames = synth.frames_textured(synth.BASE_SEED + 3, 2, W, H, 8, "420", "limited")
    flags = np.zeros(2, bool)
    text, blob = synth.net_stvsr4x()
    outs, _ = run_gpu(text, blob, frames, flags, nv.fmt(W, H, 8), nv.fmt(4 * W, 4 * H, 8), prec, scale=4,
                      limit=2)
    fdi, fdo = fmt_dict(W, H, 8), fmt_dict(4 * W, 4 * H, 8)
    net = oracle.Net(text, blob)
    rgb = [oracle.ingest(f, fdi) for f in frames]
    for (y0, y1, x0, x1) in STVSR_WINDOWS:
        exp = stvsr_window(net, rgb, y0, y1, x0, x1, fdo)
        for k in range(2):
            got = crop_codes(outs[k], y0, y1, x0, x1, 4, "420")
            if prec == "fp32":
                assert_codes_match(got, exp[k], 8)
            else:
                mx, _ = lsb_stats(got, {p: oracle.quantise(exp[k][p], 8) for p in "YUV"})
                assert mx <= 1, ((y0, x0), k, mx)


def test_fp8_filter_reports_error_vs_oracle():
    """FP8 E4M3 (per-tensor scales from frames 0-3) on the ragged 136x70 case of the 2x SR network: within the
    2 LSB it measures (the 1 LSB target is not met by FP8; see test_gpu_accuracy)."""
    W, H = 136, 70
    frames, flags = _clip_sr2x_t5_small(W, H)
    text, blob = synth.net_sr2x_t5()
    fdi, fdo = fmt_dict(W, H, 10), fmt_dict(2 * W, 2 * H, 10)
    ref = oracle.run_filter(frames, flags, text, blob, fdi, fdo)
    outs, _ = run_gpu(text, blob, frames, flags, nv.fmt(W, H, 10), nv.fmt(2 * W, 2 * H, 10), "fp8")
    worst = 0
    for got, r in zip(outs, ref):
        mx, frac = lsb_stats(got, r)
        worst = max(worst, mx)
    print("fp8 max LSB", worst)
    assert worst <= 2


def test_backpressure_full_then_pull():
    frames, flags, _, _ = _clip64_t3()
    text, blob = synth.net_sr2x_t3()
    eng = nv.Engine()
    flt = eng.filter(text, blob, nv.fmt(64, 64, 8, "420", "full"), nv.fmt(128, 128, 8, "420", "full"), "fp32")
    n = 0
    for fr in frames:
        st = flt.push((fr["Y"], fr["U"], fr["V"]))
        if st == nv.Status.FULL:
            break
        n += 1
    assert n == 5  # ring of T + 2 = 5 slots with no output pulled
    out = flt.alloc_out_host()
    # output 1 still needs frame 0 (its tuple is [0, 1, 2]): two pulls free the slot
    assert flt.pull(out)[0] == nv.Status.OK
    assert flt.push((frames[n]["Y"], frames[n]["U"], frames[n]["V"])) == nv.Status.FULL
    assert flt.pull(out)[0] == nv.Status.OK
    assert flt.push((frames[n]["Y"], frames[n]["U"], frames[n]["V"])) == nv.Status.OK
    eng.close()


def test_budget_rejects_filter():
    text, blob = synth.net_sr2x_t3()
    eng = nv.Engine(hbm_budget_bytes=1 << 20)
    with pytest.raises(nv.NvisrError) as e:
        eng.filter(text, blob, nv.fmt(64, 64, 8, "420", "full"), nv.fmt(128, 128, 8, "420", "full"), "bf16")
    assert e.value.status == nv.Status.OVER_BUDGET
    assert eng.bytes_in_use() == 0
    eng.close()


def _clip_stvsr_small(W=144, H=72, n=4):
    frames = synth.frames_textured(synth.BASE_SEED + 3, n, W, H, 8, "420", "limited")
    flags = np.zeros(n, bool)
    flags[2] = True
    return frames, flags


@pytest.fixture(scope="module")
def stvsr_oracle():
    W, H = 144, 72
    frames, flags = _clip_stvsr_small(W, H)
    text, blob = synth.net_stvsr4x()
    fdi, fdo = fmt_dict(W, H, 8), fmt_dict(4 * W, 4 * H, 8)
    outs = oracle.run_filter(frames, flags, text, blob, fdi, fdo, keep_float=True)
    return [prequant(o, fdo) for o in outs]


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_stvsr4x_dcn_filter(prec, stvsr_oracle):
    """Two-frame ST-VSR with deformable alignment, 4x space, 2x frame rate, a cut on frame 2:
    2 outputs per input (SR of frame i, midpoint i+1/2), the scene's last pair (s1, s1)."""
    W, H = 144, 72
    frames, flags = _clip_stvsr_small(W, H)
    text, blob = synth.net_stvsr4x()
    outs, infos = run_gpu(text, blob, frames, flags, nv.fmt(W, H, 8), nv.fmt(4 * W, 4 * H, 8), prec, scale=4)
    assert len(outs) == 2 * len(frames)
    assert [i[0] for i in infos] == list(range(8))
    assert [i[1:3] for i in infos] == [(0, 1), (0, 1), (1, 1), (1, 1), (2, 3), (2, 3), (3, 3), (3, 3)]
    worst = 0
    for got, pq in zip(outs, stvsr_oracle):
        if prec == "fp32":
            assert_codes_match(got, pq, 8)
        else:
            mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], 8) for k in "YUV"})
            worst = max(worst, mx)
    print(prec, "space-time SR max LSB vs oracle:", worst)
    assert worst <= 1


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("n,extra,interp,double", [(2, True, True, True), (3, False, False, False),
                                                   (2, False, False, True), (1, True, True, False),
                                                   (2, True, True, False), (3, True, False, False)])
def test_group_model_general_n(n, extra, interp, double, prec):
    """Group family with n > 1 and each flag set (Section 3.1 / 3.3): runs of n (+1) frames,
    2n network outputs with Double frame, a scene's last run moved back inside the scene
    with the outputs of already covered frames dropped, 2 outputs per frame with
    Interpolation; without Double frame the input frames themselves are outputs (scale 1,
    copied unchanged).  9 frames, a cut before frame 5."""
    W, H, N = 48, 32, 9
    frames = synth.frames_textured(synth.BASE_SEED + 61, N, W, H, 8, "420", "limited")
    flags = np.zeros(N, bool)
    flags[5] = True
    s = 1 if (interp and not double) else 2
    text, blob = synth.net_group_general(synth.BASE_SEED + 60, n, extra, interp, double, scale=s)
    fdi, fdo = fmt_dict(W, H, 8), fmt_dict(s * W, s * H, 8)
    ref = oracle.run_filter(frames, flags, text, blob, fdi, fdo, keep_float=True)
    # expected source range and kind of every output, from the oracle's presentation order
    src = [(e[1], e[1], nv.OUT_PASSTHROUGH) if e[0] == "pass" else (e[1][0], e[1][-1], nv.OUT_NETWORK)
           for e in oracle.group_outputs(flags, N, n, extra, interp, double)]
    outs, infos = run_gpu(text, blob, frames, flags, nv.fmt(W, H, 8), nv.fmt(s * W, s * H, 8), prec, scale=s)
    assert len(outs) == len(ref) == len(src) == N * (2 if (interp or double) else 1)
    assert [i[0] for i in infos] == list(range(len(ref)))
    assert [i[1:] for i in infos] == src
    for got, r in zip(outs, ref):
        if isinstance(r, dict):  # an input frame passed through: its planes, unchanged
            for k in "YUV":
                assert np.array_equal(got[k], r[k].astype(np.int64)), k
            continue
        pq = prequant(r, fdo)
        if prec == "fp32":
            assert_codes_match(got, pq, 8)
        else:
            mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], 8) for k in "YUV"})
            assert mx <= 1, mx


@pytest.mark.parametrize("device_io", [False, True])
def test_interpolation_passthrough_into_another_format(device_io):
    """Interpolation without Double frame with 8-bit 4:2:0 in and 10-bit 4:4:4 out: the
    passed-through input frames are converted to the output format (ingest, then
    requantise, no network), the network outputs go between them; FP32, a cut on frame 3."""
    W, H, N = 40, 24, 6
    frames = synth.frames_textured(synth.BASE_SEED + 62, N, W, H, 8, "420", "limited")
    flags = np.zeros(N, bool)
    flags[3] = True
    text, blob = synth.net_group_general(synth.BASE_SEED + 63, 1, True, True, False, scale=1)
    fdi, fdo = fmt_dict(W, H, 8), fmt_dict(W, H, 10, "444")
    ref = oracle.run_filter(frames, flags, text, blob, fdi, fdo, keep_float=True)
    outs, infos = run_gpu(text, blob, frames, flags, nv.fmt(W, H, 8), nv.fmt(W, H, 10, "444"), "fp32", scale=1,
                          device_io=device_io)
    assert len(outs) == len(ref) == 2 * N
    assert [i[3] for i in infos] == [nv.OUT_PASSTHROUGH, nv.OUT_NETWORK] * N
    assert [i[1] for i in infos[0::2]] == list(range(N))
    for got, r in zip(outs, ref):
        assert_codes_match(got, prequant(r, fdo), 10)


def test_interpolation_without_double_needs_scale_1():
    """An input frame passed through cannot be an output of another size: such a filter
    with spatial scale 2 is rejected."""
    text, blob = synth.net_group_general(synth.BASE_SEED + 64, 1, True, True, False, scale=2)
    eng = nv.Engine()
    with pytest.raises(nv.NvisrError) as ei:
        eng.filter(text, blob, nv.fmt(32, 32, 8), nv.fmt(64, 64, 8), "fp32", 2)
    assert ei.value.status == nv.Status.UNSUPPORTED_FORMAT
    assert "scale must be 1" in eng.last_error()
    eng.close()


def test_last_error_is_kept_per_engine():
    """nvisr_last_error(engine): a failure on one engine leaves another engine's message."""
    text, blob = synth.net_group_general(synth.BASE_SEED + 64, 1, True, True, False, scale=2)
    a, b = nv.Engine(), nv.Engine()
    with pytest.raises(nv.NvisrError):
        a.filter(text, blob, nv.fmt(32, 32, 8), nv.fmt(64, 64, 8), "fp32", 2)
    with pytest.raises(nv.NvisrError):
        b.filter(text, blob, nv.fmt(32, 32, 8), nv.fmt(32, 32, 8), "fp32", 1)
    assert "scale must be 1" in a.last_error()
    assert "scale does not match" in b.last_error()
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_filter_bt2020_12bit(prec):
    """The whole filter on 12-bit BT.2020 4:2:0 in and out (the 3-frame 32-channel 2x network, a cut on frame 5)."""
    frames = synth.frames_textured(synth.BASE_SEED + 71, 8, 64, 48, 12, "420", "limited")
    flags = np.zeros(8, bool)
    flags[5] = True
    fdi = fmt_dict(64, 48, 12, "420", "limited", "left", "bt2020")
    fdo = fmt_dict(128, 96, 12, "420", "limited", "left", "bt2020")
    text, blob = synth.net_sr2x_t3()
    ref = [prequant(o, fdo) for o in oracle.run_filter(frames, flags, text, blob, fdi, fdo, keep_float=True)]
    outs, _ = run_gpu(text, blob, frames, flags, nv.fmt(64, 48, 12, "420", "limited", "left", "bt2020"),
                      nv.fmt(128, 96, 12, "420", "limited", "left", "bt2020"), prec)
    assert len(outs) == len(ref) == 8
    for got, pq in zip(outs, ref):
        if prec == "fp32":
            assert_codes_match(got, pq, 12)
        else:
            mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], 12) for k in "YUV"})
            assert mx <= 4, mx  # 12-bit codes: the 10-bit +-1 LSB bound, scaled by 4


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_filter_yuv_domain_network(prec):
    """A network that works on Y'Cb'Cr' (Section 3.1): ingest and requantise skip the colour
    matrix; 10-bit 4:2:0 in and out, the 3-frame 32-channel 2x network, a cut on frame 4."""
    frames = synth.frames_textured(synth.BASE_SEED + 72, 7, 64, 48, 10, "420", "limited")
    flags = np.zeros(7, bool)
    flags[4] = True
    fdi, fdo = fmt_dict(64, 48, 10), fmt_dict(128, 96, 10)
    text, blob = synth.net_tuple(synth.BASE_SEED + 73, frames=3, channels=32, nres=2, scale=2, domain="yuv")
    ref = oracle.run_filter(frames, flags, text, blob, fdi, fdo, keep_float=True)
    outs, _ = run_gpu(text, blob, frames, flags, nv.fmt(64, 48, 10), nv.fmt(128, 96, 10), prec)
    assert len(outs) == len(ref) == 7
    for got, r in zip(outs, ref):
        # a YUV-domain output is requantised without the matrix
        b = 10
        pq = {"Y": oracle.scale_luma(r[0], b, "limited"),
              "U": oracle.scale_chroma(oracle.downsample_chroma(r[1], "420", "left"), b, "limited"),
              "V": oracle.scale_chroma(oracle.downsample_chroma(r[2], "420", "left"), b, "limited")}
        if prec == "fp32":
            assert_codes_match(got, pq, b)
        else:
            mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], b) for k in "YUV"})
            assert mx <= 1, mx


@pytest.mark.parametrize("sx,sy", [(1, 1), (1, 2)])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_filter_separate_scales(sx, sy, prec):
    """Section 3.2's horizontal and vertical scale: a same-size enhancement (denoise) network
    (1 x 1) and a vertical 2x (deinterlace) network (1 x 2), 64 channels, 10-bit 4:2:0 in and
    out, a cut on frame 3.  The output layer writes float32, shuffled into the planar output
    by its own kernel."""
    frames = synth.frames_textured(synth.BASE_SEED + 74, 6, 64, 48, 10, "420", "limited")
    flags = np.zeros(6, bool)
    flags[3] = True
    fdi, fdo = fmt_dict(64, 48, 10), fmt_dict(64 * sx, 48 * sy, 10)
    text, blob = synth.net_tuple(synth.BASE_SEED + 75, frames=3, channels=64, nres=1, scale=(sx, sy))
    ref = [prequant(o, fdo) for o in oracle.run_filter(frames, flags, text, blob, fdi, fdo, keep_float=True)]
    outs, _ = run_gpu(text, blob, frames, flags, nv.fmt(64, 48, 10), nv.fmt(64 * sx, 48 * sy, 10), prec,
                      scale=(sx, sy))
    assert len(outs) == len(ref) == 6
    for got, pq in zip(outs, ref):
        assert got["Y"].shape == (48 * sy, 64 * sx)
        if prec == "fp32":
            assert_codes_match(got, pq, 10)
        else:
            mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], 10) for k in "YUV"})
            assert mx <= 1, mx


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_filter_rgb_planes(prec):
    """RGB planes in and out (Section 3.1: RGB or YUV I/O): 8-bit full-range 4:4:4 R, G, B,
    3-frame 32-channel 2x network, a cut on frame 4."""
    frames = synth.frames_textured(synth.BASE_SEED + 76, 6, 48, 32, 8, "444", "full")
    flags = np.zeros(6, bool)
    flags[4] = True
    fdi = fmt_dict(48, 32, 8, "444", "full", "left", "rgb")
    fdo = fmt_dict(96, 64, 8, "444", "full", "left", "rgb")
    text, blob = synth.net_sr2x_t3()
    ref = [prequant(o, fdo) for o in oracle.run_filter(frames, flags, text, blob, fdi, fdo, keep_float=True)]
    outs, _ = run_gpu(text, blob, frames, flags, nv.fmt(48, 32, 8, "444", "full", "left", "rgb"),
                      nv.fmt(96, 64, 8, "444", "full", "left", "rgb"), prec)
    assert len(outs) == len(ref) == 6
    for got, pq in zip(outs, ref):
        if prec == "fp32":
            assert_codes_match(got, pq, 8)
        else:
            mx, _ = lsb_stats(got, {k: oracle.quantise(pq[k], 8) for k in "YUV"})
            assert mx <= 1, mx


def test_rgb_format_checks():
    """RGB planes need 4:4:4 and an RGB-domain network."""
    eng = nv.Engine()
    text, blob = synth.net_sr2x_t3()
    with pytest.raises(Exception, match="UNSUPPORTED_FORMAT|unsupported"):
        eng.filter(text, blob, nv.fmt(48, 32, 8, "420", "full", "left", "rgb"),
                   nv.fmt(96, 64, 8, "420", "full", "left", "rgb"), "bf16")
    ytext, yblob = synth.net_tuple(3, frames=3, channels=16, nres=1, scale=2, domain="yuv")
    with pytest.raises(Exception, match="UNSUPPORTED_FORMAT|YUV-domain"):
        eng.filter(ytext, yblob, nv.fmt(48, 32, 8, "444", "full", "left", "rgb"),
                   nv.fmt(96, 64, 8, "444", "full", "left", "rgb"), "bf16")
    eng.close()


def test_filter_hdr10_pq_fp32():
    """HDR10 in and out (PQ, BT.2020, 10-bit 4:2:0 limited): the network runs on linear light.
    FP32 only: a 16-bit network in linear light moves dark PQ codes by more than 1 (the
    PQ curve is steep near black)."""
    frames = synth.frames_textured(synth.BASE_SEED + 77, 5, 48, 32, 10, "420", "limited")
    flags = np.zeros(5, bool)
    fdi = fmt_dict(48, 32, 10, "420", "limited", "left", "bt2020", "pq")
    fdo = fmt_dict(96, 64, 10, "420", "limited", "left", "bt2020", "pq")
    text, blob = synth.net_sr2x_t3()
    ref = oracle.run_filter(frames, flags, text, blob, fdi, fdo)
    outs, _ = run_gpu(text, blob, frames, flags, nv.fmt(48, 32, 10, "420", "limited", "left", "bt2020", "pq"),
                      nv.fmt(96, 64, 10, "420", "limited", "left", "bt2020", "pq"), "fp32")
    assert len(outs) == len(ref) == 5
    for got, r in zip(outs, ref):
        for k in "YUV":
            d = np.abs(got[k] - r[k])
            assert d.max() <= 1, (k, d.max())
            assert (d > 0).mean() < 0.01, (k, (d > 0).mean())
