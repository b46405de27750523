"""Oracle, format side: range normalisation, BT.709 matrix, chroma resampling, requantisation.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  FP64 numpy, written as
the plain per-sample definitions.

The paper lets a network take and emit RGB or YUV and loads a network per
colour space (Section 3.1, "Network Integration": RGB/YUV I/O, YUV420 halves
two of the three channels' dimensions, colour-space-aware loading).  It fixes
none of the numeric conventions, so these follow ITU-T H.273 / BT.709 as read
in the design notes:

* range (limited): Y' = (Y - 16*2^(b-8)) / (219*2^(b-8)),
                   C' = (C - 128*2^(b-8)) / (224*2^(b-8));
  range (full):    Y' = Y / (2^b - 1),  C' = (C - 2^(b-1)) / (2^b - 1).
* BT.709: Kr = 0.2126, Kb = 0.0722, Kg = 1 - Kr - Kb; BT.2020 (non-constant
  luminance): Kr = 0.2627, Kb = 0.0593 (the same equations with its weights).
  Bit depths 8 to 16 use the same range equations.
* chroma siting: LEFT (H.273 type 0: co-sited horizontally, centred between
  rows vertically), CENTER (centred both ways), POINT (replicate; a test mode).
  Edges clamp to the nearest sample.
* requantisation: round half to even, clamp to the code range [0, 2^b - 1].
* RGB integer I/O (matrix 'rgb', 4:4:4): the three planes are R, G, B, each with
  the luma range equations, and no matrix.
* HDR transfer (transfer 'pq' or 'hlg'): the network sees linear light.  Ingest
  takes the coded R'G'B' through the SMPTE ST 2084 EOTF (1.0 = 10000 cd/m^2) or
  the inverse of the BT.2100 HLG OETF (scene light), after clamping the coded
  value to [0, 1]; requantise clamps the network's output to [0, 1] and
  applies the inverse functions before the matrix.
"""
from __future__ import annotations

import numpy as np

KR = 0.2126
KB = 0.0722
KG = 1.0 - KR - KB

# (Kr, Kb) of each supported matrix; Kg = 1 - Kr - Kb
MATRICES = {"bt709": (0.2126, 0.0722), "bt2020": (0.2627, 0.0593)}


# ---------------------------------------------------------------- range (C1)

def normalise_luma(y, bit_depth: int, range_: str):
    y = np.asarray(y, np.float64)
    if range_ == "limited":
        m = 2.0 ** (bit_depth - 8)
        return (y - 16.0 * m) / (219.0 * m)
    return y / (2.0 ** bit_depth - 1.0)


def normalise_chroma(c, bit_depth: int, range_: str):
    c = np.asarray(c, np.float64)
    if range_ == "limited":
        m = 2.0 ** (bit_depth - 8)
        return (c - 128.0 * m) / (224.0 * m)
    return (c - 2.0 ** (bit_depth - 1)) / (2.0 ** bit_depth - 1.0)


def scale_luma(yp, bit_depth: int, range_: str):
    """Inverse of normalise_luma, before rounding."""
    if range_ == "limited":
        m = 2.0 ** (bit_depth - 8)
        return yp * 219.0 * m + 16.0 * m
    return yp * (2.0 ** bit_depth - 1.0)


def scale_chroma(cp, bit_depth: int, range_: str):
    """Inverse of normalise_chroma, before rounding."""
    if range_ == "limited":
        m = 2.0 ** (bit_depth - 8)
        return cp * 224.0 * m + 128.0 * m
    return cp * (2.0 ** bit_depth - 1.0) + 2.0 ** (bit_depth - 1)


def quantise(v, bit_depth: int):
    """Round half to even (numpy rint), then clamp to [0, 2^b - 1]."""
    q = np.rint(np.asarray(v, np.float64))
    return np.clip(q, 0.0, 2.0 ** bit_depth - 1.0).astype(np.int64)


# ---------------------------------------------------------------- matrix (C2)

def ycbcr_to_rgb(yp, cb, cr, matrix: str = "bt709"):
    """Y'CbCr (normalised) -> R'G'B' with the matrix's weights.  No clamping."""
    kr, kb = MATRICES[matrix]
    kg = 1.0 - kr - kb
    r = yp + 2.0 * (1.0 - kr) * cr
    b = yp + 2.0 * (1.0 - kb) * cb
    g = (yp - kr * r - kb * b) / kg
    return r, g, b


def rgb_to_ycbcr(r, g, b, matrix: str = "bt709"):
    """R'G'B' -> Y'CbCr (normalised) with the matrix's weights."""
    kr, kb = MATRICES[matrix]
    kg = 1.0 - kr - kb
    yp = kr * r + kg * g + kb * b
    cb = (b - yp) / (2.0 * (1.0 - kb))
    cr = (r - yp) / (2.0 * (1.0 - kr))
    return yp, cb, cr


# ---------------------------------------------------------------- HDR transfer

# SMPTE ST 2084 (PQ) constants, as the standard defines them (exact rationals)
PQ_M1 = 2610.0 / 16384.0
PQ_M2 = 2523.0 / 4096.0 * 128.0
PQ_C1 = 3424.0 / 4096.0
PQ_C2 = 2413.0 / 4096.0 * 32.0
PQ_C3 = 2392.0 / 4096.0 * 32.0
# BT.2100 HLG OETF constants
HLG_A = 0.17883277
HLG_B = 1.0 - 4.0 * HLG_A
HLG_C = 0.5 - HLG_A * np.log(4.0 * HLG_A)


def pq_eotf(e):
    """PQ code value in [0, 1] -> linear light in [0, 1] (1 = 10000 cd/m^2)."""
    ep = np.power(np.maximum(np.asarray(e, np.float64), 0.0), 1.0 / PQ_M2)
    return np.power(np.maximum(ep - PQ_C1, 0.0) / (PQ_C2 - PQ_C3 * ep), 1.0 / PQ_M1)


def pq_inverse_eotf(y):
    """Linear light in [0, 1] -> PQ code value."""
    ym = np.power(np.clip(np.asarray(y, np.float64), 0.0, 1.0), PQ_M1)
    return np.power((PQ_C1 + PQ_C2 * ym) / (1.0 + PQ_C3 * ym), PQ_M2)


def hlg_oetf(e):
    """Scene light in [0, 1] -> HLG code value."""
    e = np.clip(np.asarray(e, np.float64), 0.0, 1.0)
    lo = np.sqrt(3.0 * e)
    hi = HLG_A * np.log(np.maximum(12.0 * e - HLG_B, 1e-300)) + HLG_C
    return np.where(e <= 1.0 / 12.0, lo, hi)


def hlg_inverse_oetf(ep):
    """HLG code value -> scene light."""
    ep = np.maximum(np.asarray(ep, np.float64), 0.0)
    return np.where(ep <= 0.5, ep * ep / 3.0, (np.exp((ep - HLG_C) / HLG_A) + HLG_B) / 12.0)


def to_linear(rgb, transfer: str):
    """Coded R'G'B' -> the network's linear light (identity for 'none').  The coded value is
    clamped to [0, 1], where the transfer functions are defined (an out-of-gamut Y'CbCr
    combination can give R' > 1, where the PQ EOTF has a pole)."""
    if transfer == "pq":
        return pq_eotf(np.clip(rgb, 0.0, 1.0))
    if transfer == "hlg":
        return hlg_inverse_oetf(np.clip(rgb, 0.0, 1.0))
    return rgb


def from_linear(rgb, transfer: str):
    """The network's linear light -> coded R'G'B' (clamped to [0, 1] first; identity for 'none')."""
    if transfer == "pq":
        return pq_inverse_eotf(rgb)
    if transfer == "hlg":
        return hlg_oetf(rgb)
    return rgb


# ---------------------------------------------------------------- chroma (C3)

def _clamp_idx(i, n):
    return np.clip(i, 0, n - 1)


def _up_axis(c, axis: int, mode: str):
    """Double the length of one axis.

    mode 'cosited': even output 2i = c_i, odd 2i+1 = (c_i + c_{i+1}) / 2.
    mode 'centred': output 2i = 3/4 c_i + 1/4 c_{i-1}, 2i+1 = 3/4 c_i + 1/4 c_{i+1}.
    mode 'replicate': output 2i = 2i+1 = c_i.
    Indices outside the plane clamp to the nearest sample.
    """
    c = np.moveaxis(np.asarray(c, np.float64), axis, -1)
    n = c.shape[-1]
    i = np.arange(n)
    out = np.empty(c.shape[:-1] + (2 * n,), np.float64)
    if mode == "cosited":
        out[..., 0::2] = c
        out[..., 1::2] = 0.5 * (c + c[..., _clamp_idx(i + 1, n)])
    elif mode == "centred":
        out[..., 0::2] = 0.75 * c + 0.25 * c[..., _clamp_idx(i - 1, n)]
        out[..., 1::2] = 0.75 * c + 0.25 * c[..., _clamp_idx(i + 1, n)]
    elif mode == "replicate":
        out[..., 0::2] = c
        out[..., 1::2] = c
    else:
        raise ValueError(mode)
    return np.moveaxis(out, -1, axis)


def _down_axis(c, axis: int, mode: str):
    """Halve the length of one (even-length) axis.

    mode 'cosited': out_i = (c_{2i-1} + 2 c_{2i} + c_{2i+1}) / 4 (edge clamp).
    mode 'pair':    out_i = (c_{2i} + c_{2i+1}) / 2.
    """
    c = np.moveaxis(np.asarray(c, np.float64), axis, -1)
    n = c.shape[-1]
    i = np.arange(n // 2)
    if mode == "cosited":
        out = 0.25 * (c[..., _clamp_idx(2 * i - 1, n)] + 2.0 * c[..., 2 * i]
                      + c[..., _clamp_idx(2 * i + 1, n)])
    elif mode == "pair":
        out = 0.5 * (c[..., 2 * i] + c[..., 2 * i + 1])
    else:
        raise ValueError(mode)
    return np.moveaxis(out, -1, axis)


_UP = {"left": ("centred", "cosited"), "center": ("centred", "centred"),
       "point": ("replicate", "replicate")}
_DOWN = {"left": ("pair", "cosited"), "center": ("pair", "pair"),
         "point": ("pair", "pair")}


def upsample_chroma(c, subsampling: str, loc: str):
    """4:2:0 -> 4:4:4 (vertical then horizontal); 4:4:4 passes through."""
    if subsampling == "444":
        return np.asarray(c, np.float64)
    v, h = _UP[loc]
    return _up_axis(_up_axis(c, 0, v), 1, h)


def downsample_chroma(c, subsampling: str, loc: str):
    """4:4:4 -> 4:2:0 (vertical then horizontal); 4:4:4 passes through."""
    if subsampling == "444":
        return np.asarray(c, np.float64)
    v, h = _DOWN[loc]
    return _down_axis(_down_axis(c, 0, v), 1, h)


# ---------------------------------------------------------------- ingest / requantise

def ingest(planes, fmt, domain: str = "rgb"):
    """Integer planes -> float64 network-domain planes [3][H][W]: RGB planes, or Y'CbCr
    planes through the matrix (or without it for a YUV-domain network)."""
    if fmt.get("matrix") == "rgb":
        return ingest_rgb(planes, fmt, domain)
    return _ingest_ycbcr(planes, fmt, domain)


def ingest_rgb(planes, fmt, domain: str = "rgb"):
    """Integer R'G'B' planes (positions Y, U, V hold R, G, B; 4:4:4) -> float64 R'G'B'.

    Section 3.1 allows RGB as well as YUV I/O.  Reading: each channel takes the
    luma range equations (limited: (v - 16m) / 219m; full: v / (2^b - 1)), as
    R'G'B' video does in H.273 / BT.709; no matrix.  Only an RGB-domain network
    takes RGB planes.
    """
    assert fmt["subsampling"] == "444" and domain == "rgb"
    b, rg = fmt["bit_depth"], fmt["range"]
    rgb = np.stack([normalise_luma(planes[k], b, rg) for k in "YUV"])
    return to_linear(rgb, fmt.get("transfer", "none"))


def _ingest_ycbcr(planes, fmt, domain: str = "rgb"):
    """Integer Y/U/V planes -> float64 R'G'B' [3][H][W] (network domain RGB, unclamped), or
    the normalised Y'Cb'Cr' planes (chroma upsampled, no matrix) for a YUV-domain network.

    fmt: dict with bit_depth, subsampling ('420'|'444'), range ('limited'|'full'),
    chroma_loc ('left'|'center'|'point') and optionally matrix ('bt709' default, 'bt2020').
    """
    b, rg = fmt["bit_depth"], fmt["range"]
    yp = normalise_luma(planes["Y"], b, rg)
    cb = upsample_chroma(normalise_chroma(planes["U"], b, rg), fmt["subsampling"], fmt["chroma_loc"])
    cr = upsample_chroma(normalise_chroma(planes["V"], b, rg), fmt["subsampling"], fmt["chroma_loc"])
    if domain == "yuv":
        return np.stack([yp, cb, cr])
    r, g, bb = ycbcr_to_rgb(yp, cb, cr, fmt.get("matrix", "bt709"))
    return to_linear(np.stack([r, g, bb]), fmt.get("transfer", "none"))


def requantise(rgb, fmt, domain: str = "rgb"):
    """float network-domain planes [3][H][W] -> integer planes {"Y","U","V"} (int64)."""
    if fmt.get("matrix") == "rgb":
        return requantise_rgb(rgb, fmt, domain)
    return _requantise_ycbcr(rgb, fmt, domain)


def requantise_rgb(rgb, fmt, domain: str = "rgb"):
    """float R'G'B' [3][H][W] -> integer planes {"Y","U","V"} holding R, G, B (4:4:4):
    each channel scaled with the luma range equations, rounded half to even and
    clamped to [0, 2^b - 1]."""
    assert fmt["subsampling"] == "444" and domain == "rgb"
    b, rg = fmt["bit_depth"], fmt["range"]
    rgb = from_linear(np.asarray(rgb, np.float64), fmt.get("transfer", "none"))
    return {k: quantise(scale_luma(rgb[i], b, rg), b) for i, k in enumerate("YUV")}


def _requantise_ycbcr(rgb, fmt, domain: str = "rgb"):
    """float R'G'B' [3][H][W] -> integer planes {"Y","U","V"} (int64 arrays).

    Y'CbCr from RGB, chroma downsampled in float, scaled to the code range,
    rounded half to even and clamped to [0, 2^b - 1].
    """
    b, rg = fmt["bit_depth"], fmt["range"]
    if domain == "yuv":  # a YUV-domain network's planes are Y'Cb'Cr' already
        yp, cb, cr = rgb[0], rgb[1], rgb[2]
    else:
        rgb = from_linear(np.asarray(rgb, np.float64), fmt.get("transfer", "none"))
        yp, cb, cr = rgb_to_ycbcr(rgb[0], rgb[1], rgb[2], fmt.get("matrix", "bt709"))
    cb = downsample_chroma(cb, fmt["subsampling"], fmt["chroma_loc"])
    cr = downsample_chroma(cr, fmt["subsampling"], fmt["chroma_loc"])
    return {"Y": quantise(scale_luma(yp, b, rg), b),
            "U": quantise(scale_chroma(cb, b, rg), b),
            "V": quantise(scale_chroma(cr, b, rg), b)}
