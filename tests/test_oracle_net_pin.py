"""Pins of the oracle's network forward (oracle.Net.forward) against independent models.

Each network is written out here a second time, by hand, as an FP64 torch
composition (F.conv2d, F.leaky_relu, F.pixel_shuffle, F.interpolate and, for
the deformable layer, F.grid_sample), reading the weight blob in the order
the description lists its non-shared layers.  No code is shared with the
oracle's parser or forward: a swapped activation / residual order, a
mis-ordered blob, a wrong concatenation order, a dropped skip or a wrong
weight sharing in the oracle fails here.  The deformable convolution follows
torchvision's modulated deform_conv2d (Section 3.1: the paper's DCN is
compatible with it): each of the four bilinear corners outside the image
contributes zero, which is grid_sample's zero padding with align_corners=True
on pixel-centre coordinates.  Weights are random and non-zero everywhere, so
every residual branch contributes.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
import synth

F64 = torch.float64  # every tensor here is FP64 (no process-wide default is changed)


class Blob:
    """Sequential reader of a weight blob: weight [cout][cin][k][k] then bias [cout]."""

    def __init__(self, blob):
        self.b = torch.from_numpy(np.asarray(blob, np.float32).astype(np.float64))
        self.pos = 0

    def take(self, cout, cin, k):
        n = cout * cin * k * k
        w = self.b[self.pos:self.pos + n].reshape(cout, cin, k, k)
        b = self.b[self.pos + n:self.pos + n + cout]
        self.pos += n + cout
        return w, b

    def done(self):
        return self.pos == self.b.numel()


def conv(x, wb):
    w, b = wb
    return F.conv2d(x, w, b, padding=w.shape[-1] // 2)


def lrelu(x):
    return F.leaky_relu(x, 0.1)


def up(x, s):
    return F.interpolate(x, scale_factor=s, mode="bilinear", align_corners=False)


def _frames(seed, n, h, w):
    rs = np.random.default_rng(seed)
    return [rs.uniform(-0.2, 1.2, size=(3, h, w)) for _ in range(n)]


def _t(a):
    return torch.from_numpy(np.asarray(a, np.float64))[None]


def _cmp(got, want):
    want = want[0].numpy()
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-10 * max(scale, 1.0), np.abs(got - want).max()


def _random_blob(text, blob, seed):
    """The same network with every weight and bias drawn at unit scale (no zero gains)."""
    rs = np.random.default_rng(seed)
    return (rs.normal(0.0, 0.3, size=np.asarray(blob).size)).astype(np.float32)


# ------------------------------------------------------------------ tuple networks

def torch_tuple_net(frames, blob, T, C, nres, s):
    """head conv (3T -> C, frame-major concatenation), nres blocks x + conv(lrelu(conv(x))),
    tail conv (C -> 3 s^2) + PixelShuffle(s), + bilinear x s of the centre frame."""
    rd = Blob(blob)
    x = torch.cat([_t(f) for f in frames], dim=1)
    h = conv(x, rd.take(C, 3 * T, 3))
    for _ in range(nres):
        a = lrelu(conv(h, rd.take(C, C, 3)))
        h = h + conv(a, rd.take(C, C, 3))
    y = conv(h, rd.take(3 * s * s, C, 3))
    if s > 1:
        y = F.pixel_shuffle(y, s)
    assert rd.done()
    return y + up(_t(frames[(T - 1) // 2]), s)


@pytest.mark.parametrize("T,C,nres", [(3, 32, 4), (5, 64, 10)])   # the 3-frame 32-channel and 5-frame 64-channel 2x networks
def test_tuple_network_forward_matches_torch_model(T, C, nres):
    text, blob = synth.net_tuple(synth.BASE_SEED + 90 + T, frames=T, channels=C, nres=nres, scale=2)
    blob = _random_blob(text, blob, T)
    frames = _frames(T, T, 14, 18)
    got = oracle.Net(text, blob).forward(frames)[0]
    _cmp(got, torch_tuple_net(frames, blob, T, C, nres, 2))


def test_tuple_network_same_size_forward_matches_torch_model():
    text, blob = synth.net_tuple(synth.BASE_SEED + 95, frames=3, channels=16, nres=2, scale=(1, 1))
    blob = _random_blob(text, blob, 95)
    frames = _frames(95, 3, 12, 10)
    got = oracle.Net(text, blob).forward(frames)[0]
    _cmp(got, torch_tuple_net(frames, blob, 3, 16, 2, 1))


# ------------------------------------------------------------------ deformable convolution

def torch_dcn(x, om, wb, G):
    """Modulated deformable 3x3 conv: for output p, tap k = (ky, kx), group g, sample
    x_c at p + (ky - 1, kx - 1) + (dy, dx) bilinearly (out-of-image corners 0), times
    sigmoid(mask logit), then sum W[o, c, k] * sample over c and k, plus bias.
    om: [1][27G][H][W], channels 2(g*9+k) = dy, 2(g*9+k)+1 = dx, 18G + g*9+k = logit."""
    w, b = wb
    _, C, H, W = x.shape
    cg = C // G
    yy, xx = torch.meshgrid(torch.arange(H, dtype=F64), torch.arange(W, dtype=F64), indexing="ij")
    cols = torch.zeros(C, 9, H, W, dtype=F64)
    for g in range(G):
        for k in range(9):
            ky, kx = divmod(k, 3)
            sy = yy + (ky - 1) + om[0, 2 * (g * 9 + k)]
            sx = xx + (kx - 1) + om[0, 2 * (g * 9 + k) + 1]
            grid = torch.stack([2 * sx / (W - 1) - 1, 2 * sy / (H - 1) - 1], dim=-1)[None]
            smp = F.grid_sample(x[:, g * cg:(g + 1) * cg], grid, mode="bilinear", padding_mode="zeros",
                                align_corners=True)[0]
            cols[g * cg:(g + 1) * cg, k] = smp * torch.sigmoid(om[0, 18 * G + g * 9 + k])
    y = torch.einsum("ock,ckhw->ohw", w.reshape(w.shape[0], C, 9), cols) + b[:, None, None]
    return y[None]


def test_dcn_torch_model_matches_oracle_dcn2d():
    """The grid_sample form above agrees with the oracle's direct DCN loops (which are
    pinned to scipy's map_coordinates): the model's DCN is itself a checked reading."""
    G, C, H, W = 2, 4, 7, 9
    x, off, m = synth.dcn_operands(3, C, H, W, G, offset_sigma=2.0)
    rs = np.random.default_rng(3)
    w = rs.normal(size=(5, C, 3, 3))
    b = rs.normal(size=5)
    logit = np.log(m / (1 - m))
    om = torch.from_numpy(np.concatenate([off, logit]).astype(np.float64))[None]
    got = oracle.dcn2d(x, off, oracle.sigmoid(logit), w, b, G)
    _cmp(got, torch_dcn(_t(x), om, (torch.from_numpy(w), torch.from_numpy(b)), G))


# ------------------------------------------------------------------ group networks

def torch_stvsr(frames, blob, C=64, G=8, nres=6):
    """Two-frame space-time SR network: shared extract, shared offset/mask head on both
    concatenation orders, shared DCN, 1x1 blend, shared residual trunk and upsampler."""
    rd = Blob(blob)
    f0w = rd.take(C, 3, 3)
    omw = rd.take(27 * G, 2 * C, 3)
    dw = rd.take(C, C, 3)
    midw = rd.take(C, 2 * C, 1)
    blocks = [(rd.take(C, C, 3), rd.take(C, C, 3)) for _ in range(nres)]
    u1 = rd.take(4 * C, C, 3)
    u2 = rd.take(12, C, 3)
    assert rd.done()
    x0, x1 = _t(frames[0]), _t(frames[1])
    f0, f1 = lrelu(conv(x0, f0w)), lrelu(conv(x1, f0w))
    a0 = torch_dcn(f0, conv(torch.cat([f0, f1], 1), omw), dw, G)
    a1 = torch_dcn(f1, conv(torch.cat([f1, f0], 1), omw), dw, G)
    mid = conv(torch.cat([a0, a1], 1), midw)

    def trunk(h):
        for wa, wb in blocks:
            h = h + conv(lrelu(conv(h, wa)), wb)
        h = lrelu(F.pixel_shuffle(conv(h, u1), 2))
        return F.pixel_shuffle(conv(h, u2), 2)

    return [trunk(f0) + up(x0, 4), trunk(mid) + (up(x0, 4) + up(x1, 4)) / 2]


def test_stvsr_network_forward_matches_torch_model():
    text, blob = synth.net_group_stvsr(synth.BASE_SEED + 96, channels=16, groups=2, nres=2)
    blob = _random_blob(text, blob, 96)
    frames = _frames(96, 2, 8, 10)
    got = oracle.Net(text, blob).forward(frames)
    # the model is written for the generator's shapes: 16 channels, 2 groups, 2 blocks
    want = torch_stvsr(frames, blob, C=16, G=2, nres=2)
    assert len(got) == 2
    for g, w in zip(got, want):
        _cmp(g, w)


@pytest.mark.parametrize("n,extra,double,scale", [(2, True, True, 2), (1, True, False, 1), (3, False, False, 2)])
def test_group_general_network_forward_matches_torch_model(n, extra, double, scale):
    text, blob = synth.net_group_general(synth.BASE_SEED + 97, n, extra, True, double, scale=scale)
    blob = _random_blob(text, blob, 97 + n)
    need = n + (1 if extra else 0)
    nout = 2 * n if double else n
    frames = _frames(97, need, 10, 12)
    rd = Blob(blob)
    ew = rd.take(16, 3, 3)
    fw = rd.take(32, need * 16, 3)
    ow = [rd.take(12 if scale == 2 else 3, 32, 3) for _ in range(nout)]
    assert rd.done()
    e = [lrelu(conv(_t(f), ew)) for f in frames]
    fu = lrelu(conv(torch.cat(e, 1), fw))
    want = []
    for k in range(nout):
        y = conv(fu, ow[k])
        if scale == 2:
            y = F.pixel_shuffle(y, 2)
        want.append(y + up(_t(frames[k % need]), scale))
    got = oracle.Net(text, blob).forward(frames)
    assert len(got) == nout
    for g, w in zip(got, want):
        _cmp(g, w)


def test_activation_comes_before_the_residual_add():
    """A layer with both an activation and a residual source: y = lrelu(conv(x)) + r (the
    description's order; the generated networks never combine the two, so this one does)."""
    rng = np.random.default_rng(98)
    spec = synth.NetSpec("tuple", 3, 2, "bilinear")
    spec.conv(rng, "head", "tuple", 9, 16)
    spec.conv(rng, "r", "head", 16, 16, act="lrelu", add="head")
    spec.conv(rng, "tail", "r", 16, 12, ps=2)
    spec.out("tail")
    text, blob = spec.build()
    frames = _frames(98, 3, 9, 11)
    rd = Blob(blob)
    h = conv(torch.cat([_t(f) for f in frames], 1), rd.take(16, 9, 3))
    r = lrelu(conv(h, rd.take(16, 16, 3))) + h
    want = F.pixel_shuffle(conv(r, rd.take(12, 16, 3)), 2) + up(_t(frames[1]), 2)
    assert rd.done()
    _cmp(oracle.Net(text, blob).forward(frames)[0], want)


def torch_pyramid(frames, blob, C, G, nres, levels):
    """The feature-pyramid space-time network: per-frame extract e1 = lrelu(conv(frame)),
    e_l = lrelu(conv(avg_pool2x2(e_{l-1}))); per frame a, coarse to fine: offsets from
    cat(e_l[a], e_l[other]), DCN of e_l[a], and below the coarsest level a 1x1 blend with
    the bilinear x2 of the coarser alignment; midpoint = 1x1 blend of both; trunk and
    upsampler as the two-frame network."""
    rd = Blob(blob)
    ew = [rd.take(C, 3, 3)] + [rd.take(C, C, 3) for _ in range(levels - 1)]
    lw = {}
    for lv in range(levels, 0, -1):
        lw[lv] = {"om": rd.take(27 * G, 2 * C, 3), "dcn": rd.take(C, C, 3)}
        if lv < levels:
            lw[lv]["d"] = rd.take(C, 2 * C, 1)
    midw = rd.take(C, 2 * C, 1)
    blocks = [(rd.take(C, C, 3), rd.take(C, C, 3)) for _ in range(nres)]
    u1 = rd.take(4 * C, C, 3)
    u2 = rd.take(12, C, 3)
    assert rd.done()
    x = [_t(f) for f in frames]
    e = []
    for k in range(2):
        lv = [lrelu(conv(x[k], ew[0]))]
        for i in range(1, levels):
            lv.append(lrelu(conv(F.avg_pool2d(lv[-1], 2), ew[i])))
        e.append(lv)
    fin = []
    for a in range(2):
        b = 1 - a
        d = None
        for lv in range(levels, 0, -1):
            om = conv(torch.cat([e[a][lv - 1], e[b][lv - 1]], 1), lw[lv]["om"])
            al = torch_dcn(e[a][lv - 1], om, lw[lv]["dcn"], G)
            d = al if d is None else conv(torch.cat([al, up(d, 2)], 1), lw[lv]["d"])
        fin.append(d)
    mid = conv(torch.cat(fin, 1), midw)

    def trunk(h):
        for wa, wb in blocks:
            h = h + conv(lrelu(conv(h, wa)), wb)
        h = lrelu(F.pixel_shuffle(conv(h, u1), 2))
        return F.pixel_shuffle(conv(h, u2), 2)

    return [trunk(e[0][0]) + up(x[0], 4), trunk(mid) + (up(x[0], 4) + up(x[1], 4)) / 2]


def test_pyramid_network_forward_matches_torch_model():
    text, blob = synth.net_group_pyramid(synth.BASE_SEED + 99, channels=16, groups=2, nres=2, levels=3)
    blob = _random_blob(text, blob, 99)
    frames = _frames(99, 2, 12, 16)
    got = oracle.Net(text, blob).forward(frames)
    want = torch_pyramid(frames, blob, 16, 2, 2, 3)
    assert len(got) == 2
    for g, w in zip(got, want):
        _cmp(g, w)
