"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds random numbers and test content only: integer video planes,
scene-cut flags, network descriptions with random-init FP32 weights, and DCN
offset/mask draws.  It holds none of the method's arithmetic (no range
normalisation, colour matrix, resampling, convolution or quantisation), so the
oracle and the CUDA path can both consume it without sharing any code with one
another.

Workload recipes follow the shapes the paper's use cases imply (Section 3.2:
super resolution, spatio-temporal SR; Section 3.3: scene-aware grouping):

* ``frames_gradient``   -- small 8-bit 4:2:0 clip: uniform noise + smooth ramp.
* ``frames_textured``   -- multi-octave value noise + random rectangles on a
  larger canvas, cropped with a global integer translation of 0..4 px per axis
  per frame (camera pan), at any size / bit depth / subsampling / range.
* ``scene_cuts_geometric`` -- per-frame cut flags with geometric gaps.
* ``net_tuple`` / ``net_group`` -- network descriptions (text) + weight blobs.

Base seed: 20230806; each generator takes an explicit integer seed.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20230806


# --------------------------------------------------------------------------
# video planes
# --------------------------------------------------------------------------

def _code_limits(bit_depth: int, range_: str):
    """Legal integer code ranges for synthetic content (luma lo/hi, chroma lo/hi)."""
    m = 1 << (bit_depth - 8)
    if range_ == "limited":
        return 16 * m, 235 * m, 16 * m, 240 * m
    top = (1 << bit_depth) - 1
    return 0, top, 0, top


def _plane_dtype(bit_depth: int):
    return np.uint8 if bit_depth <= 8 else np.uint16


def frames_gradient(seed: int, nframes: int, width: int, height: int,
                    bit_depth: int = 8, subsampling: str = "420",
                    range_: str = "full"):
    """Uniform-noise-plus-ramp clip.

    Luma: clamp(round(U[0, top] * 0.5 + 0.5 * (x + y) * top / (W + H - 2))).
    Chroma: U[lo, hi] blended with a horizontal/vertical gradient.
    Returns a list of dicts {"Y", "U", "V"} of integer planes.
    """
    rng = np.random.default_rng(seed)
    top = (1 << bit_depth) - 1
    ylo, yhi, clo, chi = _code_limits(bit_depth, range_)
    cw, ch = (width // 2, height // 2) if subsampling == "420" else (width, height)
    dt = _plane_dtype(bit_depth)
    yy, xx = np.mgrid[0:height, 0:width]
    ramp = 0.5 * (xx + yy) * top / max(width + height - 2, 1)
    cyy, cxx = np.mgrid[0:ch, 0:cw]
    out = []
    for f in range(nframes):
        y = np.rint(rng.uniform(0, top, size=(height, width)) * 0.5 + ramp)
        y = np.clip(y, ylo, yhi).astype(dt)
        planes = {"Y": y}
        for k, name in enumerate(("U", "V")):
            noise = rng.uniform(clo, chi, size=(ch, cw))
            grad = (cxx if k == 0 else cyy) / max((cw if k == 0 else ch) - 1, 1)
            c = 0.6 * noise + 0.4 * (clo + grad * (chi - clo))
            planes[name] = np.clip(np.rint(c), clo, chi).astype(dt)
        out.append(planes)
    return out


def _value_noise(rng, h: int, w: int, octaves: int = 5, base_cell: int = 64):
    """Multi-octave value noise in [0, 1] (bilinear-interpolated lattices)."""
    acc = np.zeros((h, w), np.float64)
    amp, total = 1.0, 0.0
    cell = base_cell
    for _ in range(octaves):
        gh, gw = h // cell + 2, w // cell + 2
        lattice = rng.uniform(0.0, 1.0, size=(gh, gw))
        ys = np.arange(h) / cell
        xs = np.arange(w) / cell
        y0 = np.floor(ys).astype(int)
        x0 = np.floor(xs).astype(int)
        fy = (ys - y0)[:, None]
        fx = (xs - x0)[None, :]
        a = lattice[y0][:, x0]
        b = lattice[y0][:, x0 + 1]
        c = lattice[y0 + 1][:, x0]
        d = lattice[y0 + 1][:, x0 + 1]
        acc += amp * ((a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + d * fx) * fy)
        total += amp
        amp *= 0.55
        cell = max(cell // 2, 2)
    return acc / total


def texture_canvas(rng, h: int, w: int, nrect: int = 24):
    """Value noise plus random axis-aligned rectangles, values in [0, 1]."""
    t = _value_noise(rng, h, w)
    for _ in range(nrect):
        rh = int(rng.integers(8, max(h // 4, 9)))
        rw = int(rng.integers(8, max(w // 4, 9)))
        y0 = int(rng.integers(0, max(h - rh, 1)))
        x0 = int(rng.integers(0, max(w - rw, 1)))
        t[y0:y0 + rh, x0:x0 + rw] = 0.5 * t[y0:y0 + rh, x0:x0 + rw] + 0.5 * rng.uniform()
    return t


def frames_textured(seed: int, nframes: int, width: int, height: int,
                    bit_depth: int = 10, subsampling: str = "420",
                    range_: str = "limited", max_step: int = 4):
    """Textured clip under a global integer translation (camera pan).

    Each axis moves by an integer step drawn from {0..max_step} per frame.
    The canvas is large enough for the whole pan.  Chroma of 4:2:0 clips is
    taken from its own canvas at half resolution (every other sample).
    """
    rng = np.random.default_rng(seed)
    steps = rng.integers(0, max_step + 1, size=(max(nframes - 1, 0), 2))
    span_y = int(steps[:, 0].sum()) if nframes > 1 else 0
    span_x = int(steps[:, 1].sum()) if nframes > 1 else 0
    ch_h, ch_w = height + span_y + 2, width + span_x + 2
    canv = [texture_canvas(rng, ch_h, ch_w) for _ in range(3)]
    ylo, yhi, clo, chi = _code_limits(bit_depth, range_)
    dt = _plane_dtype(bit_depth)
    out = []
    oy = ox = 0
    for f in range(nframes):
        if f > 0:
            oy += int(steps[f - 1, 0])
            ox += int(steps[f - 1, 1])
        y = canv[0][oy:oy + height, ox:ox + width]
        planes = {"Y": np.rint(ylo + y * (yhi - ylo)).astype(dt)}
        for k, name in enumerate(("U", "V")):
            c = canv[1 + k][oy:oy + height, ox:ox + width]
            if subsampling == "420":
                c = c[0::2, 0::2][: height // 2, : width // 2]
            planes[name] = np.rint(clo + c * (chi - clo)).astype(dt)
        out.append(planes)
    return out


def scene_cuts_geometric(seed: int, nframes: int, mean_spacing: float = 40.0):
    """Per-frame cut flags: frame k starts a new scene with probability 1/mean_spacing.

    Frame 0 never carries a flag (the clip start is always a scene start).
    """
    rng = np.random.default_rng(seed)
    flags = rng.uniform(size=nframes) < (1.0 / mean_spacing)
    flags[0] = False
    return flags.astype(bool)


# --------------------------------------------------------------------------
# network descriptions + weights
# --------------------------------------------------------------------------

class NetSpec:
    """A network description under construction: text lines + FP32 weight blob.

    Text format ("nvisr-net 1"), one statement per line::

        nvisr-net 1
        family tuple|group
        frames <T>
        scale <s> | <sx> <sy>               (horizontal and vertical scale)
        flags interp,extra,double          (group family)
        domain rgb|yuv                     (network colour domain, default rgb)
        skip none|nearest|bilinear
        conv <name> in=<a>[,<b>] cin=<C> cout=<N> k=<1|3> act=none|lrelu
             [add=<name>] [ps=<r> | psx=<rx> psy=<ry>] [share=<name>]
        dcn  <name> in=<x> om=<head> cin=<C> cout=<N> groups=<G> [share=<name>]
        pool <name> in=<x> cin=<C>         (2x2 mean: half the height and width)
        up   <name> in=<x> cin=<C>         (bilinear x2: twice the height and width)
        out  <name> [skip=<frame>[,<frame>]]

    Weights of every non-shared layer are appended to the blob in statement
    order: weight [cout][cin][k][k] then bias [cout], float32 little endian.
    """

    def __init__(self, family: str, frames: int, scale, skip: str, flags: str = "", domain: str = "rgb"):
        sc = f"{scale[0]} {scale[1]}" if isinstance(scale, tuple) else f"{scale}"
        self.lines = ["nvisr-net 1", f"family {family}", f"frames {frames}", f"scale {sc}"]
        if flags:
            self.lines.append(f"flags {flags}")
        if domain != "rgb":
            self.lines.append(f"domain {domain}")
        self.lines.append(f"skip {skip}")
        self.blobs = []

    def conv(self, rng, name, src, cin, cout, k=3, act="none", add=None, ps=None,
             share=None, gain=1.0, row_gains=None, psx=None, psy=None):
        line = f"conv {name} in={src} cin={cin} cout={cout} k={k} act={act}"
        if add:
            line += f" add={add}"
        if ps:
            line += f" ps={ps}"
        if psx:
            line += f" psx={psx}"
        if psy:
            line += f" psy={psy}"
        if share:
            line += f" share={share}"
        else:
            self.blobs.append(_he_normal(rng, cout, cin, k, gain, row_gains))
        self.lines.append(line)

    def dcn(self, rng, name, src, om, cin, cout, groups, share=None, gain=1.0):
        line = f"dcn {name} in={src} om={om} cin={cin} cout={cout} groups={groups}"
        if share:
            line += f" share={share}"
        else:
            self.blobs.append(_he_normal(rng, cout, cin, 3, gain, None))
        self.lines.append(line)

    def pool(self, name, src, cin):
        self.lines.append(f"pool {name} in={src} cin={cin}")

    def up(self, name, src, cin):
        self.lines.append(f"up {name} in={src} cin={cin}")

    def out(self, name, skip=None):
        self.lines.append(f"out {name}" + (f" skip={skip}" if skip else ""))

    def build(self):
        text = "\n".join(self.lines) + "\n"
        blob = np.concatenate(self.blobs).astype("<f4") if self.blobs else np.zeros(0, "<f4")
        return text, blob


def _he_normal(rng, cout, cin, k, gain, row_gains):
    """He-normal weights std sqrt(2 / (k*k*cin)) times gain; bias U(+-1/sqrt(fan_in))."""
    fan_in = cin * k * k
    w = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(cout, cin, k, k)) * gain
    if row_gains is not None:
        w = w * np.asarray(row_gains, np.float64)[:, None, None, None]
    b = rng.uniform(-1.0, 1.0, size=cout) / np.sqrt(fan_in) * gain
    if row_gains is not None:
        b = b * np.asarray(row_gains, np.float64)
    return np.concatenate([w.ravel(), b]).astype(np.float32)


# Gains baked into the random-init blobs (the residual-branch scale keeps the
# trunk's variance bounded over many blocks; the tail gain makes the network's
# residual about 0.02 of full scale so outputs stay in range and rounding stays
# sensitive to arithmetic error).
RES_GAIN = 0.1
TAIL_GAIN = 0.02
OFFSET_GAIN = 2.0


def net_tuple(seed: int, frames: int, channels: int, nres: int, scale=2,
              skip: str = "bilinear", tail_gain: float = TAIL_GAIN, res_gain: float = RES_GAIN,
              domain: str = "rgb"):
    """Sliding-window SR network: conv(3T->C), nres residual blocks, conv(C->3 s^2), PixelShuffle(s).

    scale is an int, or (sx, sy) with factors 1 or 2: (1, 1) is a same-size enhancement
    (denoise) network without a shuffle, (1, 2) a vertical 2x (deinterlace) network.
    """
    rng = np.random.default_rng(seed)
    sx, sy = scale if isinstance(scale, tuple) else (scale, scale)
    spec = NetSpec("tuple", frames, scale if sx != sy else sx, skip, domain=domain)
    spec.conv(rng, "head", "tuple", 3 * frames, channels, act="none")
    prev = "head"
    for i in range(nres):
        spec.conv(rng, f"r{i}a", prev, channels, channels, act="lrelu")
        spec.conv(rng, f"r{i}b", f"r{i}a", channels, channels, act="none", add=prev, gain=res_gain)
        prev = f"r{i}b"
    if sx == sy and sx > 1:
        spec.conv(rng, "tail", prev, channels, 3 * sx * sy, act="none", ps=sx, gain=tail_gain)
    else:
        spec.conv(rng, "tail", prev, channels, 3 * sx * sy, act="none", gain=tail_gain,
                  psx=sx if sx > 1 else None, psy=sy if sy > 1 else None)
    spec.out("tail")
    return spec.build()


def net_sr2x_t3(seed: int = BASE_SEED + 1):
    """9->32, 4 residual blocks of 32, 32->12, PixelShuffle(2), bilinear skip (T=3)."""
    return net_tuple(seed, frames=3, channels=32, nres=4, scale=2, skip="bilinear")


def net_sr2x_t5(seed: int = BASE_SEED + 2, skip: str = "bilinear"):
    """15->64, 10 residual blocks of 64, 64->12, PixelShuffle(2) (T=5)."""
    return net_tuple(seed, frames=5, channels=64, nres=10, scale=2, skip=skip)


def net_group_stvsr(seed: int, channels: int = 64, groups: int = 8, nres: int = 6,
                    tail_gain: float = TAIL_GAIN, res_gain: float = RES_GAIN,
                    offset_gain: float = OFFSET_GAIN):
    """Two-frame space-time SR network with deformable alignment (4x, 2x frame rate).

    extract conv 3->C per frame (shared), offset/mask head conv 2C->27G on both
    concatenation orders (shared), modulated deformable conv C->C per direction
    (shared), 1x1 blend 2C->C (midpoint features), nres residual blocks applied
    to the first frame's and the midpoint's features (shared), and an upsampler
    conv C->4C, PixelShuffle(2), LeakyReLU, conv C->12, PixelShuffle(2) per
    emitted output.  The head's offset rows are scaled so its offsets are a few
    pixels; its mask rows produce logits (sigmoid inside the DCN).
    """
    rng = np.random.default_rng(seed)
    C, G = channels, groups
    spec = NetSpec("group", 2, 4, "bilinear", flags="interp,extra,double")
    spec.conv(rng, "f0", "frame0", 3, C, act="lrelu")
    spec.conv(rng, "f1", "frame1", 3, C, act="lrelu", share="f0")
    head_rows = np.ones(27 * G)
    head_rows[: 18 * G] = offset_gain
    spec.conv(rng, "om01", "f0,f1", 2 * C, 27 * G, act="none", row_gains=head_rows)
    spec.conv(rng, "om10", "f1,f0", 2 * C, 27 * G, act="none", share="om01")
    spec.dcn(rng, "a0", "f0", "om01", C, C, G)
    spec.dcn(rng, "a1", "f1", "om10", C, C, G, share="a0")
    spec.conv(rng, "mid", "a0,a1", 2 * C, C, k=1, act="none")
    for trunk, src in (("t", "f0"), ("m", "mid")):
        prev = src
        for i in range(nres):
            sa = None if trunk == "t" else f"t{i}a"
            sb = None if trunk == "t" else f"t{i}b"
            spec.conv(rng, f"{trunk}{i}a", prev, C, C, act="lrelu", share=sa)
            spec.conv(rng, f"{trunk}{i}b", f"{trunk}{i}a", C, C, act="none", add=prev,
                      share=sb, gain=res_gain)
            prev = f"{trunk}{i}b"
        su = None if trunk == "t" else "tu1"
        sv = None if trunk == "t" else "tu2"
        spec.conv(rng, f"{trunk}u1", prev, C, 4 * C, act="lrelu", ps=2, share=su)
        spec.conv(rng, f"{trunk}u2", f"{trunk}u1", C, 12, act="none", ps=2, share=sv,
                  gain=tail_gain)
    spec.out("tu2", skip="frame0")
    spec.out("mu2", skip="frame0,frame1")
    return spec.build()


def net_stvsr4x(seed: int = BASE_SEED + 3):
    return net_group_stvsr(seed)


def net_group_pyramid(seed: int, channels: int = 64, groups: int = 8, nres: int = 6, levels: int = 3,
                      tail_gain: float = TAIL_GAIN, res_gain: float = RES_GAIN,
                      offset_gain: float = OFFSET_GAIN):
    """Two-frame space-time SR network whose extract stage is a feature pyramid (4x, 2x frame rate).

    Extract, per frame (shared weights): e1 = lrelu(conv 3->C), and for each coarser level
    l, e_l = lrelu(conv C->C (pool(e_{l-1}))) at half the previous height and width.
    Alignment of frame a (a = 0, 1; shared weights for both) at every level l, coarse to
    fine: an offset/mask head conv 2C->27G over cat(e_l of a, e_l of the other frame), a
    modulated deformable conv C->C of e_l of a, and below the coarsest level a 1x1 blend
    2C->C of that with the upsampled (bilinear x2) alignment of the level below.  Then
    the midpoint features are a 1x1 blend 2C->C of both frames' finest alignments, and
    the residual trunk and upsampler of net_group_stvsr run on frame 0's finest
    features and on the midpoint.  Frame sizes must be multiples of 2^(levels-1).
    """
    rng = np.random.default_rng(seed)
    C, G = channels, groups
    spec = NetSpec("group", 2, 4, "bilinear", flags="interp,extra,double")
    head_rows = np.ones(27 * G)
    head_rows[: 18 * G] = offset_gain
    for k in range(2):
        spec.conv(rng, f"e1f{k}", f"frame{k}", 3, C, act="lrelu", share="e1f0" if k else None)
        for lv in range(2, levels + 1):
            spec.pool(f"p{lv - 1}f{k}", f"e{lv - 1}f{k}", C)
            spec.conv(rng, f"e{lv}f{k}", f"p{lv - 1}f{k}", C, C, act="lrelu", share=f"e{lv}f0" if k else None)
    for a in range(2):
        b = 1 - a
        for lv in range(levels, 0, -1):
            sh = (lambda n: f"{n}a0") if a else (lambda n: None)
            spec.conv(rng, f"om{lv}a{a}", f"e{lv}f{a},e{lv}f{b}", 2 * C, 27 * G, act="none",
                      row_gains=head_rows, share=sh(f"om{lv}"))
            spec.dcn(rng, f"al{lv}a{a}", f"e{lv}f{a}", f"om{lv}a{a}", C, C, G, share=sh(f"al{lv}"))
            if lv == levels:
                continue
            spec.up(f"u{lv}a{a}", f"d{lv + 1}a{a}" if lv + 1 < levels else f"al{lv + 1}a{a}", C)
            spec.conv(rng, f"d{lv}a{a}", f"al{lv}a{a},u{lv}a{a}", 2 * C, C, k=1, act="none", share=sh(f"d{lv}"))
    fin = [f"d1a{a}" if levels > 1 else f"al1a{a}" for a in range(2)]
    spec.conv(rng, "mid", ",".join(fin), 2 * C, C, k=1, act="none")
    for trunk, src in (("t", "e1f0"), ("m", "mid")):
        prev = src
        for i in range(nres):
            sa = None if trunk == "t" else f"t{i}a"
            sb = None if trunk == "t" else f"t{i}b"
            spec.conv(rng, f"{trunk}{i}a", prev, C, C, act="lrelu", share=sa)
            spec.conv(rng, f"{trunk}{i}b", f"{trunk}{i}a", C, C, act="none", add=prev, share=sb, gain=res_gain)
            prev = f"{trunk}{i}b"
        su = None if trunk == "t" else "tu1"
        sv = None if trunk == "t" else "tu2"
        spec.conv(rng, f"{trunk}u1", prev, C, 4 * C, act="lrelu", ps=2, share=su)
        spec.conv(rng, f"{trunk}u2", f"{trunk}u1", C, 12, act="none", ps=2, share=sv, gain=tail_gain)
    spec.out("tu2", skip="frame0")
    spec.out("mu2", skip="frame0,frame1")
    return spec.build()


def net_group_general(seed: int, n: int, extra: bool, interp: bool, double: bool, feat: int = 16,
                      tail_gain: float = TAIL_GAIN, scale: int = 2):
    """Small group-model network for any n and flag set (2x space, or same size with scale=1).

    need = n (+1 with Extra frame) input frames: a shared extract conv 3->feat per
    frame, a fusion conv over their concatenation (need*feat -> 32, LeakyReLU),
    and one output conv per output (n, or 2n with Double frame): 32->12 +
    PixelShuffle(2), or 32->3 at scale 1; output k adds the skip of input frame
    k mod need.
    """
    rng = np.random.default_rng(seed)
    need = n + (1 if extra else 0)
    flags = ",".join(f for f, on in (("interp", interp), ("extra", extra), ("double", double)) if on)
    spec = NetSpec("group", need, scale, "bilinear", flags=flags)
    for i in range(need):
        spec.conv(rng, f"e{i}", f"frame{i}", 3, feat, act="lrelu", share="e0" if i else None)
    spec.conv(rng, "fuse", ",".join(f"e{i}" for i in range(need)), need * feat, 32, act="lrelu")
    nout = 2 * n if double else n
    for k in range(nout):
        if scale == 2:
            spec.conv(rng, f"o{k}", "fuse", 32, 12, act="none", ps=2, gain=tail_gain)
        else:
            spec.conv(rng, f"o{k}", "fuse", 32, 3, act="none", gain=tail_gain)
    for k in range(nout):
        spec.out(f"o{k}", skip=f"frame{k % need}")
    return spec.build()


# --------------------------------------------------------------------------
# DCN operands drawn directly (kernel-level tests bypass the offset head)
# --------------------------------------------------------------------------

def dcn_operands(seed: int, cin: int, height: int, width: int, groups: int,
                 offset_sigma: float = 2.0):
    """Features U(-1,1) [cin][H][W], offsets N(0, sigma^2) [2*G*9][H][W], mask U(0,1) [G*9][H][W]."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.0, 1.0, size=(cin, height, width))
    off = rng.normal(0.0, offset_sigma, size=(2 * groups * 9, height, width))
    mask = rng.uniform(0.0, 1.0, size=(groups * 9, height, width))
    return x.astype(np.float32), off.astype(np.float32), mask.astype(np.float32)


def activations(seed: int, channels: int, height: int, width: int, scale: float = 1.0):
    """Random activation tensor U(-scale, scale) [C][H][W] as float32."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1.0, 1.0, size=(channels, height, width)) * scale).astype(np.float32)
