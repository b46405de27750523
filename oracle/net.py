"""Oracle, network side: description parser, conv / DCN / PixelShuffle / skip, forward pass.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  FP64 throughout.

NNVISR runs any network that maps a frame group to enhanced frames, split into
a per-frame *extract* stage and a group *fusion* stage (Section 3.1, "Network
Integration"), and ships a modulated deformable convolution (DCN v2)
compatible with torchvision's (Section 3.1).  The layers here are the plain
definitions:

* conv:  2-D cross-correlation, OIHW weights, stride 1, zero padding (k-1)/2,
  + bias (``conv2d_direct`` in C; ``conv2d_im2col`` in numpy is the second,
  independent implementation used to pin the first).
* LeakyReLU(0.1): x >= 0 ? x : 0.1 x.
* residual add after the activation (no activation after the add).
* PixelShuffle(r): out[c, r*h+i, r*w+j] = in[c*r*r + i*r + j, h, w]; with separate
  row / column factors (ry, rx): out[c, ry*h+i, rx*w+j] = in[c*ry*rx + i*rx + j, h, w]
  (the final layer of a network whose horizontal and vertical scales differ,
  Section 3.2; ry = rx gives PyTorch's order).
* skip: upsample of the input frame in the network domain, 'bilinear'
  (align_corners = False per axis: src = (dst + 0.5)/s - 0.5 with that axis's
  scale, edge clamp) or 'nearest'.
* DCN v2: see oracle_conv.c; the head's output channels [0, 18G) are offsets
  (dy, dx interleaved per (group, tap)), [18G, 27G) are mask logits and the
  mask is their logistic sigmoid.
* pool: the 2x2 mean, out[c, y, x] = mean of in[c, 2y + i, 2x + j] (i, j in {0, 1});
  with up (bilinear x2, align_corners = False, edge clamp) it builds the extract
  stage's feature pyramid "in different spatial dimensions" (Section 3.1).
  Reading: both need even sizes (the engine rejects other frame sizes).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        lib.nvo_conv2d.argtypes = [dp, i, i, i, dp, dp, i, i, dp, i, i, i, i]
        lib.nvo_dcn2d.argtypes = [dp, i, i, i, dp, dp, i, dp, dp, i, dp, i, i, i, i]
        lib.nvo_threads.restype = i
        _LIB = lib
    return _LIB


def oracle_threads() -> int:
    return int(_lib().nvo_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------- layers

def conv2d_direct(x, w, b=None, window=None):
    """Direct FP64 cross-correlation (C loops).  x [C][H][W], w [O][C][k][k]."""
    x = np.ascontiguousarray(x, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    cin, h, wd = x.shape
    cout, cin2, k, k2 = w.shape
    assert cin == cin2 and k == k2 and k % 2 == 1
    y = np.zeros((cout, h, wd), np.float64)
    bb = None if b is None else np.ascontiguousarray(b, np.float64)
    r0, r1, c0, c1 = window if window is not None else (0, h, 0, wd)
    _lib().nvo_conv2d(_ptr(x), cin, h, wd, _ptr(w), _ptr(bb) if bb is not None else None,
                      cout, k, _ptr(y), r0, r1, c0, c1)
    return y


def conv2d_im2col(x, w, b=None):
    """im2col + GEMM FP64 cross-correlation (numpy), independent of conv2d_direct."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    cin, h, wd = x.shape
    cout, _, k, _ = w.shape
    p = (k - 1) // 2
    xp = np.zeros((cin, h + 2 * p, wd + 2 * p))
    xp[:, p:p + h, p:p + wd] = x
    cols = np.empty((cin, k, k, h, wd))
    for ky in range(k):
        for kx in range(k):
            cols[:, ky, kx] = xp[:, ky:ky + h, kx:kx + wd]
    y = w.reshape(cout, cin * k * k) @ cols.reshape(cin * k * k, h * wd)
    if b is not None:
        y = y + np.asarray(b, np.float64)[:, None]
    return y.reshape(cout, h, wd)


def dcn2d(x, offsets, mask, w, b, groups: int, window=None):
    """Modulated deformable conv 3x3 (DCN v2), FP64 C loops.  mask is already in [0, 1]."""
    x = np.ascontiguousarray(x, np.float64)
    off = np.ascontiguousarray(offsets, np.float64)
    m = np.ascontiguousarray(mask, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    cin, h, wd = x.shape
    cout = w.shape[0]
    assert w.shape == (cout, cin, 3, 3)
    assert off.shape == (2 * groups * 9, h, wd) and m.shape == (groups * 9, h, wd)
    assert cin % groups == 0
    y = np.zeros((cout, h, wd), np.float64)
    bb = None if b is None else np.ascontiguousarray(b, np.float64)
    r0, r1, c0, c1 = window if window is not None else (0, h, 0, wd)
    _lib().nvo_dcn2d(_ptr(x), cin, h, wd, _ptr(off), _ptr(m), groups, _ptr(w),
                     _ptr(bb) if bb is not None else None, cout, _ptr(y), r0, r1, c0, c1)
    return y


def leaky_relu(x, slope: float = 0.1):
    return np.where(x >= 0.0, x, slope * x)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-np.asarray(x, np.float64)))


def pixel_shuffle(x, r: int, rx: int | None = None):
    """[C*r*rx][H][W] -> [C][H*r][W*rx]: PyTorch channel order for rx = r (the default);
    row factor r, column factor rx otherwise."""
    ry = r
    rx = r if rx is None else rx
    crr, h, w = x.shape
    c = crr // (ry * rx)
    return x.reshape(c, ry, rx, h, w).transpose(0, 3, 1, 4, 2).reshape(c, h * ry, w * rx)


def upsample_bilinear(x, s: int, sy: int | None = None):
    """align_corners=False bilinear upsample with edge clamp, x [C][H][W]: by integer s
    along both axes, or s along columns and sy along rows."""
    x = np.asarray(x, np.float64)
    _, h, w = x.shape
    sy = s if sy is None else sy

    def coords(n, f):
        src = (np.arange(n * f) + 0.5) / f - 0.5
        src = np.maximum(src, 0.0)
        i0 = np.floor(src).astype(int)
        i0 = np.minimum(i0, n - 1)
        i1 = np.minimum(i0 + 1, n - 1)
        return i0, i1, src - i0

    y0, y1, fy = coords(h, sy)
    x0, x1, fx = coords(w, s)
    top = x[:, y0][:, :, x0] * (1 - fx) + x[:, y0][:, :, x1] * fx
    bot = x[:, y1][:, :, x0] * (1 - fx) + x[:, y1][:, :, x1] * fx
    return top * (1 - fy)[None, :, None] + bot * fy[None, :, None]


def pool2(x):
    """2x2 mean of [C][H][W] (H, W even) -> [C][H/2][W/2]."""
    x = np.asarray(x, np.float64)
    c, h, w = x.shape
    assert h % 2 == 0 and w % 2 == 0
    return x.reshape(c, h // 2, 2, w // 2, 2).mean(axis=(2, 4))


def upsample_nearest(x, s: int, sy: int | None = None):
    sy = s if sy is None else sy
    return np.repeat(np.repeat(np.asarray(x, np.float64), sy, axis=1), s, axis=2)


# ---------------------------------------------------------------- description

class Layer:
    def __init__(self, op, name, attrs):
        self.op, self.name, self.attrs = op, name, attrs
        self.w = None
        self.b = None

    def get(self, key, default=None):
        return self.attrs.get(key, default)


class Net:
    """Parsed network description + FP64 weights."""

    def __init__(self, text: str, blob):
        blob = np.asarray(blob, np.float32).astype(np.float64)
        self.family = "tuple"
        self.frames = 1
        self.scale = 1    # horizontal scale
        self.scale_y = 1  # vertical scale
        self.skip = "none"
        self.flags = set()
        self.domain = "rgb"
        self.align = 1
        self.layers = []
        self.outputs = []
        by_name = {}
        pos = 0
        lines = [ln.split("#", 1)[0].strip() for ln in text.splitlines()]
        lines = [ln for ln in lines if ln]
        if not lines or lines[0] != "nvisr-net 1":
            raise ValueError("not an nvisr-net 1 description")
        for ln in lines[1:]:
            tok = ln.split()
            key = tok[0]
            if key == "family":
                self.family = tok[1]
            elif key == "frames":
                self.frames = int(tok[1])
            elif key == "scale":  # "scale s", or "scale sx sy" (horizontal, vertical)
                self.scale = int(tok[1])
                self.scale_y = int(tok[2]) if len(tok) > 2 else self.scale
            elif key == "skip":
                self.skip = tok[1]
            elif key == "align":
                self.align = int(tok[1])
            elif key == "flags":
                self.flags = set(tok[1].split(","))
            elif key == "domain":
                self.domain = tok[1]
            elif key in ("conv", "dcn"):
                attrs = dict(t.split("=", 1) for t in tok[2:])
                for k in ("cin", "cout", "k", "groups", "ps", "psx", "psy"):
                    if k in attrs:
                        attrs[k] = int(attrs[k])
                if key == "dcn":
                    attrs["k"] = 3
                layer = Layer(key, tok[1], attrs)
                if "share" in attrs:
                    src = by_name[attrs["share"]]
                    assert (src.get("cin"), src.get("cout"), src.get("k")) == \
                        (attrs["cin"], attrs["cout"], attrs["k"])
                    layer.w, layer.b = src.w, src.b
                else:
                    co, ci, k = attrs["cout"], attrs["cin"], attrs["k"]
                    nw = co * ci * k * k
                    layer.w = blob[pos:pos + nw].reshape(co, ci, k, k)
                    layer.b = blob[pos + nw:pos + nw + co]
                    pos += nw + co
                by_name[layer.name] = layer
                self.layers.append(layer)
            elif key in ("pool", "up"):
                attrs = dict(t.split("=", 1) for t in tok[2:])
                attrs["cin"] = attrs["cout"] = int(attrs["cin"])
                layer = Layer(key, tok[1], attrs)
                by_name[layer.name] = layer
                self.layers.append(layer)
            elif key == "out":
                attrs = dict(t.split("=", 1) for t in tok[2:])
                self.outputs.append((tok[1], attrs.get("skip")))
            else:
                raise ValueError(f"unknown statement {key!r}")
        if pos != blob.size:
            raise ValueError(f"weight blob has {blob.size} values, description uses {pos}")

    # ------------------------------------------------------------ forward

    def _skip(self, frame_rgb):
        if self.skip == "bilinear":
            return upsample_bilinear(frame_rgb, self.scale, self.scale_y)
        if self.skip == "nearest":
            return upsample_nearest(frame_rgb, self.scale, self.scale_y)
        return np.zeros((3, frame_rgb.shape[1] * self.scale_y, frame_rgb.shape[2] * self.scale))

    def forward(self, frames_rgb, window=None, keep=False):
        """Run the graph on a list of float64 RGB frames [3][H][W].

        Tuple family: frames = the T frames of the tuple; the input tensor
        'tuple' is their channel concatenation (frame-major) and the skip comes
        from the centre frame (index (T-1)/2).  Group family: 'frame0',
        'frame1', ...; each output names its skip frames (mean of their skips).
        Returns the list of output images [3][sH][sW] in 'out' order (and the
        dict of all tensors if keep=True).
        """
        env = {}
        for i, f in enumerate(frames_rgb):
            env[f"frame{i}"] = np.asarray(f, np.float64)
        if self.family == "tuple":
            env["tuple"] = np.concatenate([env[f"frame{i}"] for i in range(len(frames_rgb))])
        for layer in self.layers:
            srcs = layer.get("in").split(",")
            x = np.concatenate([env[s] for s in srcs]) if len(srcs) > 1 else env[srcs[0]]
            if layer.op == "pool":
                env[layer.name] = pool2(x)
                continue
            if layer.op == "up":
                env[layer.name] = upsample_bilinear(x, 2)
                continue
            if layer.op == "conv":
                y = conv2d_direct(x, layer.w, layer.b)
            else:
                om = env[layer.get("om")]
                g = layer.get("groups")
                y = dcn2d(x, om[:18 * g], sigmoid(om[18 * g:27 * g]), layer.w, layer.b, g)
            if layer.get("act") == "lrelu":
                y = leaky_relu(y)
            if layer.get("add"):
                y = y + env[layer.get("add")]
            if layer.get("ps"):
                y = pixel_shuffle(y, layer.get("ps"))
            elif layer.get("psx", 1) != 1 or layer.get("psy", 1) != 1:
                y = pixel_shuffle(y, layer.get("psy", 1), layer.get("psx", 1))
            env[layer.name] = y
        outs = []
        for name, skip in self.outputs:
            res = env[name]
            if self.family == "tuple":
                sk = self._skip(env[f"frame{(len(frames_rgb) - 1) // 2}"])
            else:
                names = (skip or "").split(",") if skip else []
                sk = sum(self._skip(env[n]) for n in names) / len(names) if names else 0.0
            outs.append(res + sk)
        return (outs, env) if keep else outs

    def receptive_radius(self) -> int:
        """Input pixels of margin an output pixel depends on (sum of conv radii + DCN reach).

        Used to crop exact sub-windows for sampled full-size checks; DCN layers
        are not croppable (their reach is data dependent) and raise.
        """
        r = 0
        for layer in self.layers:
            if layer.op in ("dcn", "pool", "up"):
                raise ValueError("DCN reach is data dependent; pyramids change the scale")
            r += (layer.get("k") - 1) // 2
        return r + 1  # +1 for the bilinear skip's neighbours
