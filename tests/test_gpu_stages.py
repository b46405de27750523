"""Per-stage parity of the CUDA kernels against the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2308_03121_gb300 as nv
import synth
from gpu_util import assert_codes_match, fmt_dict, from_dev, prequant, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nv.load()


def test_tensor_core_selftest():
    bf16, fp8 = nv.nvisr_selftest()
    assert bf16 == 0 and fp8 == 0, (bf16, fp8)


def test_swizzle128_descriptor_probe():
    """Reports which base-offset convention reads rows from inside a 128-byte swizzle atom."""
    out = nv.nvisr_selftest_swizzle()
    print("sw128 probe: base offset 0 ->", out[:8].tolist(), " base offset (start>>7)&7 ->", out[8:].tolist())
    # the conv kernels start A operands at any 128-byte row inside an atom with base offset 0
    assert (out[:8] == 0).all(), out


INGEST_CASES = [
    (64, 64, 8, "420", "full", "left"),
    (1920, 1080, 10, "420", "limited", "left"),
    (854, 480, 8, "420", "limited", "left"),
    (130, 66, 10, "420", "limited", "center"),
    (96, 40, 8, "420", "full", "point"),
    (70, 34, 8, "444", "limited", "left"),
    (6, 2, 10, "420", "full", "left"),
]


@pytest.mark.parametrize("W,H,bits,sub,rng,loc", INGEST_CASES)
def test_ingest_matches_oracle(W, H, bits, sub, rng, loc):
    fr = synth.frames_textured(11, 1, W, H, bits, sub, rng)[0]
    fd = fmt_dict(W, H, bits, sub, rng, loc)
    f = nv.fmt(W, H, bits, sub, rng, loc)
    pitch = (W + 3) // 4 * 4
    out = torch.full((3, H, pitch), float("nan"), device="cuda")
    nv.nvisr_ingest(f, to_dev(fr["Y"]), to_dev(fr["U"]), to_dev(fr["V"]), out)
    torch.cuda.synchronize()
    got = out[:, :, :W].double().cpu().numpy()
    ref = oracle.ingest(fr, fd)
    err = np.abs(got - ref).max()
    assert err < 4e-6, err


@pytest.mark.parametrize("W,H,bits,sub,loc", [(136, 70, 10, "420", "left"), (64, 32, 8, "444", "center"),
                                               (70, 34, 12, "420", "point")])
def test_ingest_full_code_range_under_limited_range(W, H, bits, sub, loc):
    """Limited-range formats still carry codes outside [16, 235] / [16, 240] (scaled):
    sub-black, super-white and the extreme codes 0 and 2^b - 1.  Uniform codes over the
    whole range, plus both extremes, against the oracle."""
    rs = np.random.default_rng(W + bits)
    top = (1 << bits) - 1
    dt = np.uint8 if bits <= 8 else np.uint16
    cw, ch = (W // 2, H // 2) if sub == "420" else (W, H)
    fr = {"Y": rs.integers(0, top + 1, size=(H, W)).astype(dt),
          "U": rs.integers(0, top + 1, size=(ch, cw)).astype(dt),
          "V": rs.integers(0, top + 1, size=(ch, cw)).astype(dt)}
    for k in "YUV":
        fr[k][0, 0], fr[k][-1, -1] = 0, top
    fd = fmt_dict(W, H, bits, sub, "limited", loc)
    pitch = (W + 3) // 4 * 4
    out = torch.full((3, H, pitch), float("nan"), device="cuda")
    nv.nvisr_ingest(nv.fmt(W, H, bits, sub, "limited", loc), to_dev(fr["Y"]), to_dev(fr["U"]), to_dev(fr["V"]), out)
    torch.cuda.synchronize()
    ref = oracle.ingest(fr, fd)
    # values reach about [-1.3, 2.3] here: FP32 arithmetic, relative 1e-6 of that
    err = np.abs(out[:, :, :W].double().cpu().numpy() - ref).max()
    assert err < 8e-6, err


@pytest.mark.parametrize("W,H,bits,sub,rng,loc", INGEST_CASES)
def test_requant_matches_oracle(W, H, bits, sub, rng, loc):
    rs = np.random.default_rng(W * H + bits)
    rgb = rs.uniform(-0.08, 1.08, size=(3, H, W)).astype(np.float32)
    fd = fmt_dict(W, H, bits, sub, rng, loc)
    f = nv.fmt(W, H, bits, sub, rng, loc)
    pitch = (W + 3) // 4 * 4
    dev = torch.zeros((3, H, pitch), device="cuda")
    dev[:, :, :W] = torch.from_numpy(rgb).cuda()
    dt = torch.uint8 if bits <= 8 else torch.int16
    cw, ch = (W // 2, H // 2) if sub == "420" else (W, H)
    y = torch.zeros((H, W), dtype=dt, device="cuda")
    u = torch.zeros((ch, cw), dtype=dt, device="cuda")
    v = torch.zeros((ch, cw), dtype=dt, device="cuda")
    nv.nvisr_requant(f, dev, y, u, v)
    torch.cuda.synchronize()
    got = {"Y": from_dev(y, bits), "U": from_dev(u, bits), "V": from_dev(v, bits)}
    assert_codes_match(got, prequant(rgb.astype(np.float64), fd), bits)


FORMAT_CASES = [  # BT.2020, RGB, and 12 / 16-bit samples (W, H, bits, subsampling, range, siting, matrix)
    (96, 40, 12, "420", "limited", "left", "bt2020"),
    (70, 34, 16, "444", "full", "center", "bt2020"),
    (64, 32, 12, "420", "full", "left", "bt709"),
    (130, 66, 16, "420", "limited", "center", "bt709"),
    (64, 32, 8, "444", "full", "left", "rgb"),       # RGB planes (luma range equations, no matrix)
    (70, 34, 10, "444", "limited", "center", "rgb"),
]


@pytest.mark.parametrize("W,H,bits,sub,rng,loc,matrix", FORMAT_CASES)
def test_ingest_matrix_and_depth_match_oracle(W, H, bits, sub, rng, loc, matrix):
    fr = synth.frames_textured(12, 1, W, H, bits, sub, rng)[0]
    fd = fmt_dict(W, H, bits, sub, rng, loc, matrix)
    f = nv.fmt(W, H, bits, sub, rng, loc, matrix)
    pitch = (W + 3) // 4 * 4
    out = torch.full((3, H, pitch), float("nan"), device="cuda")
    nv.nvisr_ingest(f, to_dev(fr["Y"]), to_dev(fr["U"]), to_dev(fr["V"]), out)
    torch.cuda.synchronize()
    err = np.abs(out[:, :, :W].double().cpu().numpy() - oracle.ingest(fr, fd)).max()
    assert err < 4e-6, err


@pytest.mark.parametrize("W,H,bits,sub,rng,loc,matrix", FORMAT_CASES)
def test_requant_matrix_and_depth_match_oracle(W, H, bits, sub, rng, loc, matrix):
    rs = np.random.default_rng(W * H + bits + 1)
    rgb = rs.uniform(-0.08, 1.08, size=(3, H, W)).astype(np.float32)
    fd = fmt_dict(W, H, bits, sub, rng, loc, matrix)
    f = nv.fmt(W, H, bits, sub, rng, loc, matrix)
    pitch = (W + 3) // 4 * 4
    dev = torch.zeros((3, H, pitch), device="cuda")
    dev[:, :, :W] = torch.from_numpy(rgb).cuda()
    dt = torch.uint8 if bits <= 8 else torch.int16
    cw, ch = (W // 2, H // 2) if sub == "420" else (W, H)
    y = torch.zeros((H, W), dtype=dt, device="cuda")
    u = torch.zeros((ch, cw), dtype=dt, device="cuda")
    v = torch.zeros((ch, cw), dtype=dt, device="cuda")
    nv.nvisr_requant(f, dev, y, u, v)
    torch.cuda.synchronize()
    got = {"Y": from_dev(y, bits), "U": from_dev(u, bits), "V": from_dev(v, bits)}
    assert_codes_match(got, prequant(rgb.astype(np.float64), fd), bits)


TRANSFER_CASES = [  # HDR transfer (W, H, bits, subsampling, range, siting, matrix, transfer)
    (64, 32, 10, "420", "limited", "left", "bt2020", "pq"),   # HDR10
    (70, 34, 10, "444", "full", "center", "bt2020", "hlg"),
    (48, 32, 12, "444", "full", "left", "rgb", "pq"),
]


@pytest.mark.parametrize("W,H,bits,sub,rng,loc,matrix,transfer", TRANSFER_CASES)
def test_ingest_transfer_matches_oracle(W, H, bits, sub, rng, loc, matrix, transfer):
    """Ingest to linear light (PQ EOTF / inverse HLG OETF after the matrix), float32 vs FP64."""
    fr = synth.frames_textured(13, 1, W, H, bits, sub, rng)[0]
    fd = fmt_dict(W, H, bits, sub, rng, loc, matrix, transfer)
    f = nv.fmt(W, H, bits, sub, rng, loc, matrix, transfer)
    pitch = (W + 3) // 4 * 4
    out = torch.full((3, H, pitch), float("nan"), device="cuda")
    nv.nvisr_ingest(f, to_dev(fr["Y"]), to_dev(fr["U"]), to_dev(fr["V"]), out)
    torch.cuda.synchronize()
    ref = oracle.ingest(fr, fd)
    err = np.abs(out[:, :, :W].double().cpu().numpy() - ref)
    # float32 powers: a few ulp of relative error, amplified by the PQ exponents
    assert (err <= 2e-5 * (1.0 + np.abs(ref))).all(), err.max()


@pytest.mark.parametrize("W,H,bits,sub,rng,loc,matrix,transfer", TRANSFER_CASES)
def test_requant_transfer_matches_oracle(W, H, bits, sub, rng, loc, matrix, transfer):
    """Requantise from linear light: clamp to [0, 1], inverse transfer, matrix.  The PQ
    inverse raises to the power 78.84, so float32 codes may round apart from FP64 ones by
    one code a little away from ties: every code within 1, nearly all equal."""
    rs = np.random.default_rng(W * H + bits + 2)
    lin = (rs.uniform(0.0, 1.0, size=(3, H, W)) ** 3 * 1.05 - 0.02).astype(np.float32)
    fd = fmt_dict(W, H, bits, sub, rng, loc, matrix, transfer)
    f = nv.fmt(W, H, bits, sub, rng, loc, matrix, transfer)
    pitch = (W + 3) // 4 * 4
    dev = torch.zeros((3, H, pitch), device="cuda")
    dev[:, :, :W] = torch.from_numpy(lin).cuda()
    dt = torch.uint8 if bits <= 8 else torch.int16
    cw, ch = (W // 2, H // 2) if sub == "420" else (W, H)
    y = torch.zeros((H, W), dtype=dt, device="cuda")
    u = torch.zeros((ch, cw), dtype=dt, device="cuda")
    v = torch.zeros((ch, cw), dtype=dt, device="cuda")
    nv.nvisr_requant(f, dev, y, u, v)
    torch.cuda.synchronize()
    got = {"Y": from_dev(y, bits), "U": from_dev(u, bits), "V": from_dev(v, bits)}
    ref = oracle.requantise(lin.astype(np.float64), fd)
    for k in "YUV":
        d = np.abs(got[k] - ref[k])
        assert d.max() <= 1, (k, d.max())
        assert (d > 0).mean() < 0.01, (k, (d > 0).mean())


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).double().numpy()


def _f16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).half().double().numpy()


def _e4m3(a, scale):
    inv = np.float32(1.0) / np.float32(scale)
    return torch.from_numpy(np.asarray(a, np.float32) * inv).to(torch.float8_e4m3fn).double().numpy() * float(scale)


CONV_CASES = [
    # cin, cout, H, W, k, act, residual
    (16, 64, 9, 200, 3, 0, False),
    (64, 64, 7, 300, 3, 1, False),
    (64, 64, 5, 129, 3, 0, True),
    (32, 32, 6, 64, 3, 1, False),
    (64, 16, 4, 257, 3, 0, False),
    (128, 64, 3, 130, 1, 0, False),
    (15, 64, 4, 70, 3, 0, False),
]


def _conv_inputs(cin, cout, H, W, k, seed):
    rs = np.random.default_rng(seed)
    x = rs.uniform(-1, 1, size=(cin, H, W)).astype(np.float32)
    w = (rs.normal(size=(cout, cin, k, k)) * np.sqrt(2.0 / (cin * k * k))).astype(np.float32)
    b = rs.uniform(-0.1, 0.1, size=cout).astype(np.float32)
    r = rs.uniform(-1, 1, size=(cout, H, W)).astype(np.float32)
    return x, w, b, r


def _ref_conv(x, w, b, act, r):
    y = oracle.conv2d_direct(x, w, b)
    if act:
        y = oracle.leaky_relu(y)
    if r is not None:
        y = y + r
    return y


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("cin,cout,H,W,k,act,res", CONV_CASES)
def test_conv2d_matches_oracle(prec, cin, cout, H, W, k, act, res):
    x, w, b, r = _conv_inputs(cin, cout, H, W, k, cin * 7 + W)
    rr = r if res else None
    got = nv.nvisr_conv2d(prec, torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda(),
                          torch.from_numpy(b).cuda(), act, torch.from_numpy(r).cuda() if res else None)
    torch.cuda.synchronize()
    got = got.double().cpu().numpy()
    if prec == "fp32":
        ref = _ref_conv(x.astype(np.float64), w.astype(np.float64), b, act, rr)
        tol = 2e-5
    else:
        q = _bf16 if prec == "bf16" else _f16
        # operands rounded exactly as the kernel stores them; FP32 accumulation
        ref = _ref_conv(q(x), q(w), b, act, None)
        if rr is not None:
            ref = ref + rr
        # 16-bit output rounding of the stored activation: half an ulp
        ulp = 2.0 ** -8 if prec == "bf16" else 2.0 ** -11
        tol = 2e-5 + ulp * np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err < tol, (err, tol)


@pytest.mark.parametrize("H,W,res", [(6, 200, False), (5, 131, True)])
def test_conv2d_fp8_matches_quantised_oracle(H, W, res):
    cin = cout = 64
    x, w, b, r = _conv_inputs(cin, cout, H, W, 3, 99 + W)
    got = nv.nvisr_conv2d("fp8", torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda(),
                          torch.from_numpy(b).cuda(), 0, torch.from_numpy(r).cuda() if res else None)
    torch.cuda.synchronize()
    got = got.double().cpu().numpy()
    sx = np.float32(np.abs(x).max()) / np.float32(448.0)
    sw = np.float32(np.abs(w).max()) / np.float32(448.0)
    ref = _ref_conv(_e4m3(x, sx), _e4m3(w, sw), b, 0, None)
    if res:
        ref = ref + _bf16(r)
    tol = 2e-4 + 2.0 ** -8 * np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err < tol, (err, tol)


@pytest.mark.parametrize("cin,groups,H,W", [(64, 8, 12, 140), (16, 2, 9, 33), (8, 1, 5, 7)])
def test_dcn2d_fp32_matches_oracle(cin, groups, H, W):
    x, off, m = synth.dcn_operands(cin + W, cin, H, W, groups)
    rs = np.random.default_rng(cin)
    cout = 64 if cin == 64 else 16
    w = (rs.normal(size=(cout, cin, 3, 3)) * np.sqrt(2.0 / (9 * cin))).astype(np.float32)
    b = rs.uniform(-0.1, 0.1, size=cout).astype(np.float32)
    got = nv.nvisr_dcn2d("fp32", torch.from_numpy(x).cuda(), torch.from_numpy(off).cuda(),
                         torch.from_numpy(m).cuda(), torch.from_numpy(w).cuda(), torch.from_numpy(b).cuda(), groups)
    torch.cuda.synchronize()
    ref = oracle.dcn2d(x, off, m, w, b, groups)
    err = np.abs(got.double().cpu().numpy() - ref).max()
    assert err < 5e-5, err


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("groups,H,W", [(8, 12, 140), (8, 5, 64), (2, 3, 257)])
def test_dcn2d_tensor_core_matches_oracle(prec, groups, H, W):
    """Tensor-core DCN: operands rounded as the kernel stores them; the sampled
    im2col values and the output are rounded once more to 16 bits, so the
    tolerance is two half-ulps of the magnitude sum |w| |sample|."""
    cin = cout = 64
    x, off, m = synth.dcn_operands(7 * W + groups, cin, H, W, groups)
    rs = np.random.default_rng(groups + W)
    w = (rs.normal(size=(cout, cin, 3, 3)) * np.sqrt(2.0 / (9 * cin))).astype(np.float32)
    b = rs.uniform(-0.1, 0.1, size=cout).astype(np.float32)
    got = nv.nvisr_dcn2d(prec, torch.from_numpy(x).cuda(), torch.from_numpy(off).cuda(), torch.from_numpy(m).cuda(),
                         torch.from_numpy(w).cuda(), torch.from_numpy(b).cuda(), groups)
    torch.cuda.synchronize()
    q = _bf16 if prec == "bf16" else _f16
    xq, wq = q(x), q(w)
    ref = oracle.dcn2d(xq, off, m, wq, b, groups)
    mag = oracle.dcn2d(np.abs(xq), off, m, np.abs(wq), None, groups)
    ulp = 2.0 ** -8 if prec == "bf16" else 2.0 ** -11
    tol = ulp * (mag + np.abs(ref)) + 1e-5
    err = np.abs(got.double().cpu().numpy() - ref)
    assert (err <= tol).all(), (err.max(), np.argwhere(err > tol)[:3])
