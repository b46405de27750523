"""FP64 CPU oracle for the NNVISR frame-group enhancement path.

TEST INFRASTRUCTURE -- NOT PART OF THE PRODUCT.  Only ``tests/``, the package's
``__graft_entry__.smoke()`` check and ``bench.py``'s CPU-baseline / reference
leg may import, call, link or run anything under ``oracle/``.  The CUDA path
never routes through it and shares no code with it (the two only read the same
seeded inputs from ``synth``).

What it computes (plain definitions, FP64):

* ingest: integer planes -> range normalise -> chroma upsample -> BT.709
  Y'CbCr->R'G'B' (``colour.py``);
* grouping: scenes from per-frame cut flags, sliding-window tuples, group-model
  runs, the Figure 1 frame-store layout (``grouping.py``, Section 3.3);
* network: direct convolution, LeakyReLU, residual add, PixelShuffle, skip,
  modulated deformable convolution (``net.py`` + ``oracle_conv.c``,
  Section 3.1);
* requantise: R'G'B'->Y'CbCr, chroma downsample, range scale, round half to
  even, clamp (``colour.py``);
* ``run_filter``: the whole filter over a clip, outputs in presentation order.

Pins (tests marked "not gpu"): textbook BT.709 colour-bar codes, closed-form
range values, library routines (torch conv2d / pixel_shuffle / interpolate,
scipy correlate), brute force on tiny inputs, the invariants of the method
(zero residual + nearest skip reproduces the input, no leak across a cut,
8-bit round trip within 1 LSB), and the Figure 1 layout as printed.
"""
from __future__ import annotations

import numpy as np

from .colour import (HLG_A, HLG_B, HLG_C, KB, KG, KR, downsample_chroma, hlg_inverse_oetf,
                     from_linear, hlg_oetf, ingest, normalise_chroma, normalise_luma, pq_eotf,
                     pq_inverse_eotf, quantise, requantise, rgb_to_ycbcr, scale_chroma,
                     scale_luma, to_linear, upsample_chroma, ycbcr_to_rgb)
from .grouping import (fig1_layout, fig1_next_batch_copy, fig1_slot_frames,
                       group_output_count, group_outputs, group_runs, outputs_per_frame,
                       scene_of, scenes_from_flags, tuple_indices, tuple_map)
from .net import (Net, conv2d_direct, conv2d_im2col, dcn2d, leaky_relu,
                  oracle_threads, pixel_shuffle, pool2, sigmoid, upsample_bilinear,
                  upsample_nearest)

__all__ = [
    "HLG_A", "HLG_B", "HLG_C", "KB", "KG", "KR", "Net", "conv2d_direct", "conv2d_im2col", "dcn2d",
    "from_linear", "hlg_inverse_oetf", "hlg_oetf", "pq_eotf", "pq_inverse_eotf", "to_linear",
    "downsample_chroma", "fig1_layout", "fig1_next_batch_copy", "fig1_slot_frames",
    "group_output_count", "group_outputs", "group_runs", "ingest", "outputs_per_frame",
    "passthrough", "leaky_relu", "normalise_chroma",
    "normalise_luma", "oracle_threads", "pad_to_align", "pixel_shuffle", "pool2", "quantise",
    "requantise", "rgb_to_ycbcr", "run_filter", "scale_chroma", "scale_luma",
    "scene_of", "scenes_from_flags", "sigmoid", "tuple_indices", "tuple_map",
    "upsample_bilinear", "upsample_chroma", "upsample_nearest", "ycbcr_to_rgb",
]


def pad_to_align(rgb, align: int):
    """Edge-replicate a [3][H][W] frame up to multiples of ``align`` (network stride)."""
    _, h, w = rgb.shape
    ph = (-h) % align
    pw = (-w) % align
    if ph == 0 and pw == 0:
        return rgb
    return np.pad(rgb, ((0, 0), (0, ph), (0, pw)), mode="edge")


def _same_format(a, b):
    keys = ("width", "height", "bit_depth", "subsampling", "range", "chroma_loc", "matrix", "transfer")
    dflt = {"matrix": "bt709", "transfer": "none"}
    return all(a.get(k, dflt.get(k)) == b.get(k, dflt.get(k)) for k in keys)


def passthrough(frame, in_fmt, out_fmt, domain="rgb", keep_float=False):
    """An input frame output as it is (Interpolation without Double frame, Section 3.1).

    Reading: with equal input and output formats the frame's planes are copied
    unchanged; otherwise the frame is converted to the output format by the
    filter's own format path with no network (ingest, then requantise).  With
    keep_float the converted frame is returned before requantisation.
    """
    if _same_format(in_fmt, out_fmt):
        return {k: np.array(frame[k]) for k in ("Y", "U", "V")}
    rgb = ingest(frame, in_fmt, domain)
    return rgb if keep_float else requantise(rgb, out_fmt, domain)


def run_filter(frames, flags, net_text, blob, in_fmt, out_fmt, outputs=None, keep_float=False):
    """Run the whole filter over a clip.

    frames: list of {"Y","U","V"} integer planes; flags: per-frame scene-start
    flags; in_fmt/out_fmt: dicts (bit_depth, subsampling, range, chroma_loc).
    outputs: optional iterable of output indices to compute (others skipped).
    Returns a list (presentation order) of output planes, or of float RGB
    images when keep_float is set; skipped outputs are None.  An input frame
    passed through (Interpolation without Double frame) is a dict of integer
    planes when it is copied unchanged, whatever keep_float says.
    """
    net = Net(net_text, blob)
    nframes = len(frames)
    scenes = scenes_from_flags(flags, nframes)
    cache = {}

    def rgb(i):
        if i not in cache:
            cache[i] = pad_to_align(ingest(frames[i], in_fmt, net.domain), net.align)
        return cache[i]

    h, w = frames[0]["Y"].shape
    oh, ow = h * net.scale_y, w * net.scale
    want = None if outputs is None else set(outputs)
    results = []

    def finish(img):
        img = img[:, :oh, :ow]
        return img if keep_float else requantise(img, out_fmt, net.domain)

    if net.family == "tuple":
        for t in range(nframes):
            if want is not None and t not in want:
                results.append(None)
                continue
            idx = tuple_indices(t, net.frames, *scene_of(t, scenes))
            results.append(finish(net.forward([rgb(i) for i in idx])[0]))
        return results
    extra = "extra" in net.flags
    n = net.frames - (1 if extra else 0)
    plan = group_outputs(flags, nframes, n, extra, "interp" in net.flags, "double" in net.flags)
    run_cache = {}
    for o, entry in enumerate(plan):
        if want is not None and o not in want:
            results.append(None)
        elif entry[0] == "pass":
            results.append(passthrough(frames[entry[1]], in_fmt, out_fmt, net.domain, keep_float))
        else:
            _, inputs, k = entry
            if inputs not in run_cache:
                run_cache.clear()
                run_cache[inputs] = net.forward([rgb(i) for i in inputs])
            results.append(finish(run_cache[inputs][k]))
    return results
