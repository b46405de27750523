"""Pins for the FP64 oracle, against things other than the oracle itself.

Each test ties one oracle function to a textbook value, a library routine,
a brute-force evaluation, a closed form, or an invariant of the method, so a
dropped term, a wrong sign/index or a transposed operand fails somewhere.
"""
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F
from scipy import ndimage, signal

import oracle
import synth
from oracle import grouping

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _fmt(bits, sub="444", rng="limited", loc="left"):
    return dict(bit_depth=bits, subsampling=sub, range=rng, chroma_loc=loc)


# ------------------------------------------------------------------ C1 range

def test_range_closed_forms():
    assert oracle.normalise_luma(64, 10, "limited") == 0.0
    assert oracle.normalise_luma(940, 10, "limited") == 1.0
    assert oracle.normalise_chroma(512, 10, "limited") == 0.0
    assert oracle.normalise_chroma(960, 10, "limited") == 0.5
    assert oracle.normalise_chroma(64, 10, "limited") == -0.5
    assert oracle.normalise_luma(255, 8, "full") == 1.0
    assert oracle.normalise_luma(0, 8, "full") == 0.0
    assert oracle.normalise_chroma(128, 8, "full") == 0.0
    assert oracle.normalise_luma(16, 8, "limited") == 0.0
    assert oracle.normalise_luma(235, 8, "limited") == 1.0


# ------------------------------------------------------------------ C2 matrix

def _bars():
    rows = []
    with open(os.path.join(GOLD, "bt709_colour_bars.txt")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            t = ln.split()
            rows.append((t[0], [float(v) for v in t[1:4]], [int(v) for v in t[4:10]]))
    return rows


@pytest.mark.parametrize("bits", [8, 10])
def test_bt709_colour_bars_encode(bits):
    for name, rgb, codes in _bars():
        img = np.array(rgb, np.float64).reshape(3, 1, 1) * np.ones((3, 2, 2))
        out = oracle.requantise(img, _fmt(bits))
        exp = codes[0:3] if bits == 8 else codes[3:6]
        got = [int(out["Y"][0, 0]), int(out["U"][0, 0]), int(out["V"][0, 0])]
        assert got == exp, (name, got, exp)


@pytest.mark.parametrize("bits", [8, 10])
def test_bt709_colour_bars_decode(bits):
    lsb = 1.0 / (219 * 2 ** (bits - 8))
    for name, rgb, codes in _bars():
        c = codes[0:3] if bits == 8 else codes[3:6]
        planes = {"Y": np.full((2, 2), c[0]), "U": np.full((2, 2), c[1]), "V": np.full((2, 2), c[2])}
        out = oracle.ingest(planes, _fmt(bits))
        # each code is within half an LSB of the exact signal; the matrix rows
        # have sum |coef| <= 2.9, so the decoded RGB is within ~1.5 LSB
        assert np.allclose(out[:, 0, 0], rgb, atol=3 * lsb), (name, out[:, 0, 0])


def test_matrix_fp64_round_trip():
    rng = np.random.default_rng(1)
    y, cb, cr = rng.uniform(-0.5, 1.5, (3, 64))
    r, g, b = oracle.ycbcr_to_rgb(y, cb, cr)
    y2, cb2, cr2 = oracle.rgb_to_ycbcr(r, g, b)
    assert max(abs(y - y2).max(), abs(cb - cb2).max(), abs(cr - cr2).max()) < 1e-12


def test_matrix_rows_luma_weights():
    # grey maps to zero chroma, and Y' of a pure primary is its weight
    y, cb, cr = oracle.rgb_to_ycbcr(np.array(0.3), np.array(0.3), np.array(0.3))
    assert abs(cb) < 1e-15 and abs(cr) < 1e-15 and abs(y - 0.3) < 1e-15
    assert oracle.rgb_to_ycbcr(1.0, 0.0, 0.0)[0] == pytest.approx(0.2126)
    assert oracle.rgb_to_ycbcr(0.0, 0.0, 1.0)[0] == pytest.approx(0.0722)
    assert oracle.rgb_to_ycbcr(1.0, 0.0, 0.0)[2] == pytest.approx(0.5)
    assert oracle.rgb_to_ycbcr(0.0, 0.0, 1.0)[1] == pytest.approx(0.5)


@pytest.mark.parametrize("matrix", ["bt709", "bt2020"])
def test_matrix_fp64_round_trip_each_matrix(matrix):
    rng = np.random.default_rng(2)
    y, cb, cr = rng.uniform(-0.5, 1.5, (3, 64))
    r, g, b = oracle.ycbcr_to_rgb(y, cb, cr, matrix)
    y2, cb2, cr2 = oracle.rgb_to_ycbcr(r, g, b, matrix)
    assert max(abs(y - y2).max(), abs(cb - cb2).max(), abs(cr - cr2).max()) < 1e-12


def test_bt2020_luma_weights():
    """BT.2020 (non-constant luminance): Y' of a pure primary is its weight (Kr 0.2627,
    Kb 0.0593, Kg 0.6780), grey has zero chroma and a primary's own chroma is +-0.5."""
    r = oracle.rgb_to_ycbcr(1.0, 0.0, 0.0, "bt2020")
    g = oracle.rgb_to_ycbcr(0.0, 1.0, 0.0, "bt2020")
    b = oracle.rgb_to_ycbcr(0.0, 0.0, 1.0, "bt2020")
    assert r[0] == pytest.approx(0.2627) and g[0] == pytest.approx(0.6780) and b[0] == pytest.approx(0.0593)
    assert r[2] == pytest.approx(0.5) and b[1] == pytest.approx(0.5)
    y, cb, cr = oracle.rgb_to_ycbcr(np.array(0.4), np.array(0.4), np.array(0.4), "bt2020")
    assert abs(cb) < 1e-15 and abs(cr) < 1e-15 and abs(y - 0.4) < 1e-15


@pytest.mark.parametrize("bits", [12, 16])
def test_range_pins_high_bit_depths(bits):
    """Limited range at b bits scales the 8-bit anchors by 2^(b-8); full range spans the codes."""
    m = 2 ** (bits - 8)
    assert oracle.normalise_luma(16 * m, bits, "limited") == 0.0
    assert oracle.normalise_luma(235 * m, bits, "limited") == pytest.approx(1.0)
    assert oracle.normalise_chroma(128 * m, bits, "limited") == 0.0
    assert oracle.normalise_chroma(240 * m, bits, "limited") == pytest.approx(0.5)
    assert oracle.normalise_luma(2 ** bits - 1, bits, "full") == 1.0
    assert oracle.quantise(oracle.scale_luma(1.0, bits, "limited"), bits) == 235 * m


def test_pq_published_anchors_and_round_trip():
    """SMPTE ST 2084: 100 cd/m^2 (0.01 of the 10000 cd/m^2 range) codes to 0.508078 and
    1000 cd/m^2 to 0.751827 (the values HDR10 tables give), 10000 cd/m^2 to 1; the EOTF
    inverts the inverse EOTF."""
    assert abs(oracle.pq_inverse_eotf(0.01) - 0.508078) < 1e-6
    assert abs(oracle.pq_inverse_eotf(0.1) - 0.751827) < 1e-6
    assert abs(oracle.pq_inverse_eotf(1.0) - 1.0) < 1e-15
    y = np.geomspace(1e-6, 1.0, 200)
    assert np.abs(oracle.pq_eotf(oracle.pq_inverse_eotf(y)) / y - 1.0).max() < 1e-10
    e = np.linspace(0.0, 1.0, 101)
    assert np.all(np.diff(oracle.pq_eotf(e)) >= 0.0)


def test_hlg_knee_and_round_trip():
    """BT.2100 HLG OETF: sqrt(3E) up to E = 1/12 (code 0.5), a ln(12E - b) + c above, the two
    branches meeting at the knee; E = 1 codes to 1 (to the rounding of a); the inverse
    inverts it."""
    assert oracle.hlg_oetf(1.0 / 12.0) == 0.5
    knee_log = oracle.HLG_A * np.log(12.0 / 12.0 - oracle.HLG_B) + oracle.HLG_C
    assert abs(knee_log - 0.5) < 1e-12
    assert abs(oracle.hlg_oetf(1.0) - 1.0) < 1e-7
    e = np.linspace(0.0, 1.0, 301)
    assert np.abs(oracle.hlg_inverse_oetf(oracle.hlg_oetf(e)) - e).max() < 1e-12


@pytest.mark.parametrize("transfer", ["pq", "hlg"])
def test_transfer_zero_residual_nearest_reproduces_input(transfer):
    """A network in linear light (PQ or HLG in and out) with zero residual and nearest skip
    returns its input codes: ingest's transfer and requantise's inverse cancel."""
    text, blob = _identity_net()
    rng = np.random.default_rng(11)
    frames = [{k: rng.integers(64, 941, (12, 16)) for k in "YUV"} for _ in range(4)]
    fmt = _fmt(10, "444", "limited", "left")
    fmt["matrix"], fmt["transfer"] = "rgb", transfer
    outs = oracle.run_filter(frames, np.zeros(4, bool), text, blob, fmt, fmt)
    for f, o in zip(frames, outs):
        for k in "YUV":
            assert np.array_equal(o[k], np.repeat(np.repeat(f[k].astype(np.int64), 2, 0), 2, 1)), k


@pytest.mark.parametrize("bits,rng_name", [(8, "full"), (10, "limited"), (12, "full"), (16, "limited")])
def test_rgb_io_range_anchors_and_exact_round_trip(bits, rng_name):
    """RGB planes (Section 3.1: RGB or YUV I/O) take the luma range equations: the range
    ends map to 0 and 1, and every code comes back unchanged through ingest and
    requantise (no matrix, no resampling)."""
    fmt = {"bit_depth": bits, "subsampling": "444", "range": rng_name, "chroma_loc": "left", "matrix": "rgb"}
    m = 2 ** (bits - 8)
    lo, hi = (0, 2 ** bits - 1) if rng_name == "full" else (16 * m, 235 * m)
    codes = np.arange(0, 2 ** bits, max(1, 2 ** bits // 4096), dtype=np.int64)
    codes = np.concatenate([codes, [lo, hi, 2 ** bits - 1]])
    planes = {k: np.roll(codes, i).reshape(1, -1) for i, k in enumerate("YUV")}
    rgb = oracle.ingest(planes, fmt)
    assert rgb[0][0, -3] == 0.0 and rgb[0][0, -2] == 1.0
    back = oracle.requantise(rgb, fmt)
    for k in "YUV":
        assert np.array_equal(back[k], planes[k]), k


@pytest.mark.parametrize("rng_name", ["limited", "full"])
def test_8bit_round_trip_within_1lsb(rng_name):
    """8-bit YUV -> RGB -> 8-bit RGB -> YUV stays within +-1 LSB for in-gamut colours."""
    rng = np.random.default_rng(7)
    rgb8 = rng.integers(0, 256, size=(3, 32, 32)).astype(np.float64)
    fmt = _fmt(8, "444", rng_name)
    yuv = oracle.requantise(rgb8 / 255.0, fmt)          # in-gamut 8-bit YUV
    rgb = oracle.ingest(yuv, fmt)
    rgb_q = np.clip(np.rint(rgb * 255.0), 0, 255) / 255.0
    back = oracle.requantise(rgb_q, fmt)
    for k in "YUV":
        assert np.abs(back[k] - yuv[k]).max() <= 1, k


# ------------------------------------------------------------------ C3 chroma

def _read_blocks(path):
    blocks, cur = {}, None
    with open(path) as f:
        for ln in f:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            if ln[0].isalpha():
                cur = ln
                blocks[cur] = []
            else:
                blocks[cur].append([float(v) for v in ln.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def test_chroma_left_hand_example():
    b = _read_blocks(os.path.join(GOLD, "chroma_left_4x4.txt"))
    assert np.array_equal(oracle.upsample_chroma(b["upsample_in"], "420", "left"), b["upsample_out"])
    assert np.array_equal(oracle.downsample_chroma(b["downsample_in"], "420", "left"), b["downsample_out"])


@pytest.mark.parametrize("loc", ["left", "center", "point"])
def test_chroma_constant_stays_constant(loc):
    c = np.full((5, 7), 0.3125)
    assert np.array_equal(oracle.upsample_chroma(c, "420", loc), np.full((10, 14), 0.3125))
    assert np.array_equal(oracle.downsample_chroma(np.full((10, 14), 0.3125), "420", loc),
                          np.full((5, 7), 0.3125))


def test_chroma_ramp_interior():
    # chroma sample (j, i) of a 4:2:0 plane sits at luma (2j + 0.5, 2i) under 'left'
    j, i = np.mgrid[0:8, 0:8]
    a, by, bx = 0.1, 0.02, 0.03
    c = a + by * (2 * j + 0.5) + bx * (2 * i)
    up = oracle.upsample_chroma(c, "420", "left")
    y, x = np.mgrid[0:16, 0:16]
    ref = a + by * y + bx * x
    assert np.allclose(up[1:-1, 0:-2], ref[1:-1, 0:-2], atol=1e-14)
    # 'center': chroma at (2j + 0.5, 2i + 0.5)
    c2 = a + by * (2 * j + 0.5) + bx * (2 * i + 0.5)
    up2 = oracle.upsample_chroma(c2, "420", "center")
    assert np.allclose(up2[1:-1, 1:-1], ref[1:-1, 1:-1], atol=1e-14)
    # downsampling a full-resolution ramp returns the ramp at the chroma sites
    down = oracle.downsample_chroma(ref, "420", "left")
    assert np.allclose(down[:, 1:], c[:, 1:], atol=1e-14)


def test_chroma_point_round_trip_identity():
    c = np.random.default_rng(3).uniform(size=(6, 9))
    assert np.array_equal(oracle.downsample_chroma(oracle.upsample_chroma(c, "420", "point"), "420", "point"), c)


# ------------------------------------------------------------------ C15 requant

def test_round_half_even_and_code_clamp():
    assert list(oracle.quantise([2.5, 3.5, 0.5, 1.5, -0.4, -3.0, 1023.6, 255.5], 10)) == \
        [2, 4, 0, 2, 0, 0, 1023, 256]
    assert list(oracle.quantise([254.5, 255.5, 300.0], 8)) == [254, 255, 255]
    # clamp is to the code range, not the legal limited range
    out = oracle.requantise(np.full((3, 2, 2), 1.05), _fmt(8))
    assert int(out["Y"][0, 0]) == 246


# ------------------------------------------------------------------ C8 conv

def test_conv_direct_matches_im2col_and_torch():
    rng = np.random.default_rng(11)
    x = rng.normal(size=(5, 9, 7))
    w = rng.normal(size=(4, 5, 3, 3))
    b = rng.normal(size=4)
    d = oracle.conv2d_direct(x, w, b)
    i = oracle.conv2d_im2col(x, w, b)
    t = F.conv2d(torch.from_numpy(x)[None], torch.from_numpy(w), torch.from_numpy(b), padding=1)[0].numpy()
    assert np.abs(d - i).max() < 1e-12
    assert np.abs(d - t).max() < 1e-12
    w1 = rng.normal(size=(3, 5, 1, 1))
    t1 = F.conv2d(torch.from_numpy(x)[None], torch.from_numpy(w1))[0].numpy()
    assert np.abs(oracle.conv2d_direct(x, w1) - t1).max() < 1e-12


def test_conv_single_channel_is_scipy_correlate():
    rng = np.random.default_rng(12)
    x = rng.normal(size=(1, 6, 8))
    w = rng.normal(size=(1, 1, 3, 3))
    ref = signal.correlate2d(x[0], w[0, 0], mode="same", boundary="fill", fillvalue=0.0)
    assert np.abs(oracle.conv2d_direct(x, w)[0] - ref).max() < 1e-12


def test_conv_delta_kernel_and_linearity():
    rng = np.random.default_rng(13)
    x = rng.normal(size=(3, 5, 6))
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1] = 1.0
    assert np.array_equal(oracle.conv2d_direct(x, w), x)
    w2 = rng.normal(size=(2, 3, 3, 3))
    x2 = rng.normal(size=(3, 5, 6))
    lhs = oracle.conv2d_direct(2.0 * x + x2, w2)
    rhs = 2.0 * oracle.conv2d_direct(x, w2) + oracle.conv2d_direct(x2, w2)
    assert np.abs(lhs - rhs).max() < 1e-12


def test_conv_window_matches_full():
    rng = np.random.default_rng(14)
    x = rng.normal(size=(2, 10, 12))
    w = rng.normal(size=(3, 2, 3, 3))
    full = oracle.conv2d_direct(x, w)
    part = oracle.conv2d_direct(x, w, window=(2, 7, 3, 11))
    assert np.array_equal(part[:, 2:7, 3:11], full[:, 2:7, 3:11])
    assert not part[:, :2].any()


# ------------------------------------------------------------------ C9/C10/C11 layers

def test_pixel_shuffle_matches_torch_and_brute_force():
    x = np.random.default_rng(15).normal(size=(12, 3, 4))
    t = F.pixel_shuffle(torch.from_numpy(x)[None], 2)[0].numpy()
    ps = oracle.pixel_shuffle(x, 2)
    assert np.array_equal(ps, t)
    for c in range(3):
        for i in range(2):
            for j in range(2):
                assert np.array_equal(ps[c, i::2, j::2], x[c * 4 + i * 2 + j])
    # inverse
    assert np.array_equal(F.pixel_unshuffle(torch.from_numpy(ps)[None], 2)[0].numpy(), x)


@pytest.mark.parametrize("s", [2, 4])
def test_upsample_matches_torch(s):
    x = np.random.default_rng(16).normal(size=(3, 5, 7))
    tb = F.interpolate(torch.from_numpy(x)[None], scale_factor=s, mode="bilinear", align_corners=False)[0].numpy()
    assert np.abs(oracle.upsample_bilinear(x, s) - tb).max() < 1e-12
    tn = F.interpolate(torch.from_numpy(x)[None], scale_factor=s, mode="nearest")[0].numpy()
    assert np.array_equal(oracle.upsample_nearest(x, s), tn)


@pytest.mark.parametrize("ry,rx", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_pixel_shuffle_separate_factors_inverts_slicing(ry, rx):
    """PixelShuffle with row factor ry and column factor rx (Section 3.2's separate
    horizontal / vertical scales): cutting an image into its ry x rx phase images by
    slicing and stacking them channel-major (c, i, j) must be undone exactly."""
    img = np.random.default_rng(21 + 3 * ry + rx).normal(size=(3, 4 * ry, 5 * rx))
    phases = np.stack([img[c, i::ry, j::rx] for c in range(3) for i in range(ry) for j in range(rx)])
    assert np.array_equal(oracle.pixel_shuffle(phases, ry, rx), img)
    if ry == rx:
        assert np.array_equal(oracle.pixel_shuffle(phases, ry), img)


@pytest.mark.parametrize("sx,sy", [(1, 1), (1, 2), (2, 1), (2, 4)])
def test_upsample_separate_scales_match_torch(sx, sy):
    x = np.random.default_rng(17).normal(size=(3, 5, 7))
    tb = F.interpolate(torch.from_numpy(x)[None], scale_factor=(sy, sx), mode="bilinear",
                       align_corners=False)[0].numpy()
    assert np.abs(oracle.upsample_bilinear(x, sx, sy) - tb).max() < 1e-12
    tn = F.interpolate(torch.from_numpy(x)[None], scale_factor=(sy, sx), mode="nearest")[0].numpy()
    assert np.array_equal(oracle.upsample_nearest(x, sx, sy), tn)
    if (sx, sy) == (1, 1):
        assert np.array_equal(oracle.upsample_bilinear(x, 1), x)


def test_leaky_relu_matches_torch():
    x = np.linspace(-3, 3, 61)
    assert np.array_equal(oracle.leaky_relu(x), F.leaky_relu(torch.from_numpy(x), 0.1).numpy())


# ------------------------------------------------------------------ C13 DCN

def _dcn_case(seed, cin=4, h=6, w=7, groups=2, cout=3):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(cin, h, w))
    wt = rng.normal(size=(cout, cin, 3, 3))
    b = rng.normal(size=cout)
    return x, wt, b


def test_dcn_zero_offset_unit_mask_is_conv():
    x, wt, b = _dcn_case(21)
    off = np.zeros((2 * 2 * 9,) + x.shape[1:])
    m = np.ones((2 * 9,) + x.shape[1:])
    assert np.abs(oracle.dcn2d(x, off, m, wt, b, 2) - oracle.conv2d_im2col(x, wt, b)).max() < 1e-12


def test_dcn_zero_mask_is_bias():
    x, wt, b = _dcn_case(22)
    off = np.random.default_rng(0).normal(size=(36,) + x.shape[1:])
    m = np.zeros((18,) + x.shape[1:])
    assert np.array_equal(oracle.dcn2d(x, off, m, wt, b, 2), np.broadcast_to(b[:, None, None], (3,) + x.shape[1:]))


def _shift_on_canvas(plane, dy, dx, pad=4):
    """Zero-extended plane shifted so out[y, x] = plane[y + dy, x + dx] (zero outside)."""
    h, w = plane.shape
    canvas = np.zeros((h + 2 * pad, w + 2 * pad))
    canvas[pad:pad + h, pad:pad + w] = plane
    return np.roll(canvas, (-dy, -dx), axis=(0, 1))


def test_dcn_integer_offsets_per_group_are_shifted_conv():
    """Group g's offsets (dy_g, dx_g) on every tap = conv of x_g shifted by (dy_g, dx_g).

    Different, asymmetric shifts per group pin the offset channel order
    2*(g*9 + k) + {0: dy, 1: dx}.
    """
    x, wt, b = _dcn_case(23)
    shifts = [(1, -2), (-1, 0)]
    off = np.zeros((36,) + x.shape[1:])
    for g, (dy, dx) in enumerate(shifts):
        for k in range(9):
            off[2 * (g * 9 + k)] = dy
            off[2 * (g * 9 + k) + 1] = dx
    m = np.ones((18,) + x.shape[1:])
    pad = 4
    xs = np.stack([_shift_on_canvas(x[c], *shifts[c // 2], pad=pad) for c in range(4)])
    ref = F.conv2d(torch.from_numpy(xs)[None], torch.from_numpy(wt), torch.from_numpy(b), padding=1)[0].numpy()
    ref = ref[:, pad:-pad, pad:-pad]
    assert np.abs(oracle.dcn2d(x, off, m, wt, b, 2) - ref).max() < 1e-12


def test_dcn_mask_channel_order():
    """A per-(group, tap) constant mask m[g,k] equals conv with w[o,c,k] * m[g(c),k]."""
    x, wt, b = _dcn_case(24)
    mk = np.random.default_rng(5).uniform(size=(2, 9))
    m = np.broadcast_to(mk.reshape(18, 1, 1), (18,) + x.shape[1:]).copy()
    off = np.zeros((36,) + x.shape[1:])
    w2 = wt.copy()
    for c in range(4):
        w2[:, c] *= mk[c // 2].reshape(3, 3)
    assert np.abs(oracle.dcn2d(x, off, m, wt, b, 2) - oracle.conv2d_im2col(x, w2, b)).max() < 1e-12


def test_dcn_fractional_offsets_match_scipy_bilinear():
    """Fractional offsets: each sample equals scipy's order-1 interpolation with zero fill."""
    x, wt, b = _dcn_case(25, cin=2, h=5, w=5, groups=1, cout=1)
    rng = np.random.default_rng(6)
    off = rng.normal(0, 2.0, size=(18, 5, 5))
    m = rng.uniform(size=(9, 5, 5))
    got = oracle.dcn2d(x, off, m, wt, b, 1)
    ref = np.full((5, 5), b[0])
    for py in range(5):
        for px in range(5):
            for ky in range(3):
                for kx in range(3):
                    k = ky * 3 + kx
                    sy = py + ky - 1 + off[2 * k, py, px]
                    sx = px + kx - 1 + off[2 * k + 1, py, px]
                    for c in range(2):
                        v = ndimage.map_coordinates(x[c], [[sy], [sx]], order=1,
                                                    mode="grid-constant", cval=0.0)[0]
                        ref[py, px] += wt[0, c, ky, kx] * m[k, py, px] * v
    assert np.abs(got[0] - ref).max() < 1e-12


def test_pool2_is_torch_avg_pool():
    """The extract pyramid's 2x2 mean equals torch's avg_pool2d (kernel 2, stride 2)."""
    x = np.random.default_rng(31).normal(size=(5, 6, 10))
    ref = torch.nn.functional.avg_pool2d(torch.from_numpy(x)[None], 2)[0].numpy()
    assert np.abs(oracle.pool2(x) - ref).max() < 1e-15


# ------------------------------------------------------------------ C4/C5 grouping

def test_scenes_and_tuple_map_clip64_t3():
    flags = np.zeros(16, bool)
    flags[9] = True
    assert oracle.scenes_from_flags(flags, 16) == [(0, 8), (9, 15)]
    tm = oracle.tuple_map(flags, 16, 3)
    assert tm[0] == [0, 0, 1] and tm[8] == [7, 8, 8] and tm[9] == [9, 9, 10] and tm[15] == [14, 15, 15]


def test_tuple_map_brute_force_invariants():
    rng = np.random.default_rng(9)
    for trial in range(50):
        n = int(rng.integers(1, 30))
        T = int(rng.choice([1, 3, 5, 7]))
        flags = rng.uniform(size=n) < 0.2
        tm = oracle.tuple_map(flags, n, T)
        for t, idx in enumerate(tm):
            scene = [u for u in range(n) if all(not flags[v] for v in range(min(t, u) + 1, max(t, u) + 1))]
            assert all(i in scene for i in idx)          # never leaves the scene
            assert idx[(T - 1) // 2] == t                # centre frame
            assert idx == sorted(idx)
            for k, i in enumerate(idx):                  # unclamped entries are t-r+k
                if i == t - (T - 1) // 2 + k:
                    continue
                assert i in (min(scene), max(scene))


def test_group_runs_stvsr_pairs():
    runs = oracle.group_runs(0, 39, 1, extra=True)
    assert len(runs) == 40
    assert runs[0] == ([0, 1], 0, 1) and runs[38] == ([38, 39], 0, 1) and runs[39] == ([39, 39], 0, 1)
    assert oracle.group_output_count(1, True, True) == 2


def test_group_runs_recycle_and_duplicate():
    # n = 3 network, scene of 7 frames: the last group recycles 4, 5 and covers frame 6 only
    assert oracle.group_runs(0, 6, 3, extra=False) == \
        [([0, 1, 2], 0, 3), ([3, 4, 5], 0, 3), ([4, 5, 6], 2, 1)]
    # scene of 2 frames for a 3-frame network: last frame duplicated, 2 frames covered
    assert oracle.group_runs(10, 11, 3, extra=False) == [([10, 11, 11], 0, 2)]
    # interpolation network (n = 2, Extra frame), scene of 5: the last group recycles
    # frame 3 and its extra frame duplicates the scene's last frame
    assert oracle.group_runs(0, 4, 2, extra=True)[-1] == ([3, 4, 4], 1, 1)
    # n = 2 with Extra frame over 2 frames: one run, the extra frame duplicated
    assert oracle.group_runs(0, 1, 2, extra=True) == [([0, 1, 1], 0, 2)]


def test_group_runs_cover_each_scene_frame_once():
    """Brute force: the frames a scene's runs cover for the first time are s0..s1 in
    order, each once, and no run reads outside the scene."""
    for n in range(1, 6):
        for extra in (False, True):
            for s0 in (0, 3):
                for length in range(1, 14):
                    s1 = s0 + length - 1
                    covered = []
                    for inputs, skip, count in oracle.group_runs(s0, s1, n, extra):
                        assert len(inputs) == n + extra
                        assert all(s0 <= i <= s1 for i in inputs)
                        assert count >= 1 and skip + count <= n
                        covered += inputs[skip:skip + count]
                    assert covered == list(range(s0, s1 + 1)), (n, extra, s0, s1)


def _plan(flags, n, extra, interp, double):
    return [("P", e[1]) if e[0] == "pass" else ("N", e[1], e[2])
            for e in oracle.group_outputs(np.asarray(flags, bool), len(flags), n, extra, interp, double)]


def test_group_outputs_interpolation_passes_input_frames_through():
    """Section 3.1: Interpolation doubles the frame rate; without Double frame the input
    frames are output as they are and the network's n outputs are the intermediate frames.
    Written out by hand for n = 1 and n = 2 (Extra frame), one scene."""
    assert _plan([0, 0, 0, 0], 1, True, True, False) == [
        ("P", 0), ("N", (0, 1), 0), ("P", 1), ("N", (1, 2), 0),
        ("P", 2), ("N", (2, 3), 0), ("P", 3), ("N", (3, 3), 0)]
    assert _plan([0, 0, 0, 0, 0], 2, True, True, False) == [
        ("P", 0), ("N", (0, 1, 2), 0), ("P", 1), ("N", (0, 1, 2), 1),
        ("P", 2), ("N", (2, 3, 4), 0), ("P", 3), ("N", (2, 3, 4), 1),
        ("P", 4), ("N", (3, 4, 4), 1)]
    # a cut before frame 2: no pair crosses it, the scene's last frame is duplicated
    assert _plan([0, 0, 1, 0], 1, True, True, False) == [
        ("P", 0), ("N", (0, 1), 0), ("P", 1), ("N", (1, 1), 0),
        ("P", 2), ("N", (2, 3), 0), ("P", 3), ("N", (3, 3), 0)]


def test_group_outputs_double_and_plain_counts():
    """Double frame: 2n network outputs per run (2 per consumed frame); neither flag: n.
    Every stream gives 2 (Interpolation or Double frame) or 1 outputs per input frame."""
    assert _plan([0, 0, 0], 1, True, True, True) == [
        ("N", (0, 1), 0), ("N", (0, 1), 1), ("N", (1, 2), 0), ("N", (1, 2), 1),
        ("N", (2, 2), 0), ("N", (2, 2), 1)]
    assert _plan([0] * 7, 3, False, False, False) == [
        ("N", (0, 1, 2), 0), ("N", (0, 1, 2), 1), ("N", (0, 1, 2), 2),
        ("N", (3, 4, 5), 0), ("N", (3, 4, 5), 1), ("N", (3, 4, 5), 2), ("N", (4, 5, 6), 2)]
    assert _plan([0, 0, 0], 2, False, False, True) == [
        ("N", (0, 1), 0), ("N", (0, 1), 1), ("N", (0, 1), 2), ("N", (0, 1), 3),
        ("N", (1, 2), 2), ("N", (1, 2), 3)]
    rng = np.random.default_rng(4)
    for _ in range(40):
        nf = int(rng.integers(1, 20))
        flags = rng.uniform(size=nf) < 0.25
        n = int(rng.integers(1, 4))
        extra, interp, double = (bool(v) for v in rng.integers(0, 2, size=3))
        assert len(_plan(flags, n, extra, interp, double)) == nf * (2 if (interp or double) else 1)


def test_passthrough_copies_or_converts():
    """A passed-through frame in the input's own format is the input unchanged; into
    another format it is converted without a network: 8-bit full range to 10-bit full
    range is code * 1023 / 255 rounded (closed form), on 4:4:4 planes."""
    rng = np.random.default_rng(5)
    fr = {k: rng.integers(0, 256, size=(4, 6)).astype(np.uint8) for k in "YUV"}
    f8 = dict(width=6, height=4, bit_depth=8, subsampling="444", range="full", chroma_loc="left")
    same = oracle.passthrough(fr, f8, dict(f8))
    assert all(np.array_equal(same[k], fr[k]) for k in "YUV")
    f10 = dict(f8, bit_depth=10)
    conv = oracle.passthrough(fr, f8, f10)
    for k in "YUV":
        if k == "Y":
            exp = np.rint(fr[k].astype(np.float64) * 1023 / 255)
        else:  # chroma: C' = (C - 128) / 255 -> C' * 1023 + 512, clamped to the code range
            exp = np.clip(np.rint((fr[k].astype(np.float64) - 128) * 1023 / 255 + 512), 0, 1023)
        assert np.array_equal(conv[k], exp.astype(np.int64)), k


# ------------------------------------------------------------------ C7 Figure 1

def _fig1_rows():
    rows = []
    with open(os.path.join(GOLD, "fig1_layout_n3_b2.txt")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            rows.append([None if t == "_" else int(t) for t in ln.split() if t != "|"])
    return rows


def test_fig1_layout_reproduces_figure():
    rows = _fig1_rows()
    n, b = 3, 2
    grid, slot_start = oracle.fig1_layout(n, b)
    # the first block (leading column + n columns) is the layout of batch 0
    for r in range(b):
        assert rows[r][: n + 1] == grid[r]
    # every input slot is b contiguous cells of the column-first store
    slots = oracle.fig1_slot_frames(grid, slot_start, n, b)
    for k in range(n + 1):
        assert slots[k] == [r * n + k for r in range(b)]
    # b n + 1 cells used
    assert sum(v is not None for row in grid for v in row) == b * n + 1
    # rolling store: the next batch's block begins at the copy destination and
    # holds frames offset by b n; it is the figure's second block
    src, dst = oracle.fig1_next_batch_copy(n, b)
    flat = [grid[a % b][a // b] for a in range(b * (n + 1))]
    assert flat[src] == b * n and flat[dst] == 5            # "6 to 5"
    nxt = [[None if v is None else v + b * n for v in row] for row in grid]
    for r in range(b):
        assert rows[r][n + 1:] == nxt[r][1:]


@pytest.mark.parametrize("n,b", [(1, 1), (1, 4), (2, 3), (3, 2), (4, 5)])
def test_fig1_layout_general(n, b):
    grid, slot_start = oracle.fig1_layout(n, b)
    slots = oracle.fig1_slot_frames(grid, slot_start, n, b)
    for k in range(n + 1):
        assert slots[k] == [r * n + k for r in range(b)]
    assert sum(v is not None for row in grid for v in row) == b * n + 1


# ------------------------------------------------------------------ method invariants

def _identity_net(frames=3):
    """Tuple net whose residual is exactly zero (tail weights and bias 0), nearest skip."""
    text, blob = synth.net_tuple(5, frames=frames, channels=8, nres=1, scale=2, skip="nearest")
    blob = blob.copy()
    tail = 12 * 8 * 9 + 12
    blob[-tail:] = 0.0
    return text, blob


@pytest.mark.parametrize("sub,loc", [("444", "left"), ("420", "point")])
def test_zero_residual_nearest_reproduces_input(sub, loc):
    frames = synth.frames_gradient(3, 4, 16, 12, 8, sub, "full")
    fmt = _fmt(8, sub, "full", loc)
    text, blob = _identity_net()
    outs = oracle.run_filter(frames, np.zeros(4, bool), text, blob, fmt, fmt)
    for f, o in zip(frames, outs):
        for k in "YUV":
            exp = np.repeat(np.repeat(f[k].astype(np.int64), 2, 0), 2, 1)
            assert np.array_equal(o[k], exp), k


@pytest.mark.parametrize("sx,sy", [(1, 1), (1, 2), (2, 1)])
@pytest.mark.parametrize("sub,loc", [("444", "left"), ("420", "point")])
def test_zero_residual_nearest_separate_scales_reproduce_input(sx, sy, sub, loc):
    """Same-size (1 x 1, denoise) and one-axis (1 x 2 deinterlace, 2 x 1) networks with zero
    residual and nearest skip return their input codes, repeated along the scaled axis."""
    text, blob = synth.net_tuple(9, frames=3, channels=8, nres=1, scale=(sx, sy), skip="nearest")
    blob = blob.copy()
    tail = 3 * sx * sy * (8 * 9 + 1)
    blob[-tail:] = 0.0
    frames = synth.frames_gradient(3, 4, 16, 12, 8, sub, "full")
    fmt_in = _fmt(8, sub, "full", loc)
    outs = oracle.run_filter(frames, np.zeros(4, bool), text, blob, fmt_in, fmt_in)
    for f, o in zip(frames, outs):
        for k in "YUV":
            exp = np.repeat(np.repeat(f[k].astype(np.int64), sy, 0), sx, 1)
            assert np.array_equal(o[k], exp), k


def test_rgb_io_zero_residual_nearest_reproduces_input():
    """RGB planes in and out, zero residual and nearest skip: the output codes are the
    input codes repeated 2 x 2, for any code values."""
    text, blob = _identity_net()
    rng = np.random.default_rng(8)
    frames = [{k: rng.integers(0, 1024, (12, 16)) for k in "YUV"} for _ in range(4)]
    fmt = _fmt(10, "444", "limited", "left")
    fmt["matrix"] = "rgb"
    outs = oracle.run_filter(frames, np.zeros(4, bool), text, blob, fmt, fmt)
    for f, o in zip(frames, outs):
        for k in "YUV":
            assert np.array_equal(o[k], np.repeat(np.repeat(f[k].astype(np.int64), 2, 0), 2, 1)), k


@pytest.mark.parametrize("sub,loc", [("444", "left"), ("420", "point")])
def test_yuv_domain_zero_residual_reproduces_input(sub, loc):
    """A YUV-domain network (Section 3.1: networks may work on YUV) with zero residual and
    nearest skip returns its input codes, for any code values (no colour matrix either way)."""
    text, blob = synth.net_tuple(5, frames=3, channels=8, nres=1, scale=2, skip="nearest", domain="yuv")
    blob = blob.copy()
    blob[-(12 * 8 * 9 + 12):] = 0.0
    rng = np.random.default_rng(3)
    cw, ch = (16, 12) if sub == "444" else (8, 6)
    frames = [{"Y": rng.integers(0, 1024, (12, 16)), "U": rng.integers(0, 1024, (ch, cw)),
               "V": rng.integers(0, 1024, (ch, cw))} for _ in range(4)]
    fmt = _fmt(10, sub, "full", loc)
    outs = oracle.run_filter(frames, np.zeros(4, bool), text, blob, fmt, fmt)
    for f, o in zip(frames, outs):
        for k in "YUV":
            assert np.array_equal(o[k], np.repeat(np.repeat(f[k].astype(np.int64), 2, 0), 2, 1)), k


def test_scene_cut_never_leaks():
    """Poison every frame outside output t's scene: output t is bit-identical."""
    frames = synth.frames_gradient(synth.BASE_SEED + 1, 8, 16, 16, 8, "420", "full")
    flags = np.zeros(8, bool)
    flags[4] = True
    fmt = _fmt(8, "420", "full")
    text, blob = synth.net_tuple(3, frames=3, channels=8, nres=1, scale=2)
    base = oracle.run_filter(frames, flags, text, blob, fmt, fmt, keep_float=True)
    poisoned = [dict(f) for f in frames]
    for i in range(4, 8):
        poisoned[i] = {k: np.full_like(v, 255 if k == "Y" else 0) for k, v in frames[i].items()}
    pz = oracle.run_filter(poisoned, flags, text, blob, fmt, fmt, keep_float=True)
    for t in range(4):
        assert np.array_equal(base[t], pz[t])
    assert not np.array_equal(base[4], pz[4])


def test_crop_window_forward_is_exact_in_interior():
    """Forward on a crop with margin >= the receptive radius equals the full forward."""
    text, blob = synth.net_tuple(4, frames=3, channels=8, nres=2, scale=2)
    net = oracle.Net(text, blob)
    rng = np.random.default_rng(2)
    frames = [rng.uniform(size=(3, 30, 34)) for _ in range(3)]
    full = net.forward(frames)[0]
    R = net.receptive_radius()
    y0, y1, x0, x1 = 12, 16, 14, 20
    cy0, cx0 = max(y0 - R, 0), max(x0 - R, 0)
    crop = [f[:, cy0:y1 + R, cx0:x1 + R] for f in frames]
    part = net.forward(crop)[0]
    s = net.scale
    assert np.abs(part[:, (y0 - cy0) * s:(y1 - cy0) * s, (x0 - cx0) * s:(x1 - cx0) * s]
                  - full[:, y0 * s:y1 * s, x0 * s:x1 * s]).max() < 1e-12


def test_net_description_rejects_blob_mismatch():
    text, blob = synth.net_sr2x_t3()
    with pytest.raises(ValueError):
        oracle.Net(text, blob[:-1])
