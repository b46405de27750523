"""Helpers shared by the GPU parity tests (inputs, oracle windows, tolerances)."""
import numpy as np
import torch

import oracle


def fmt_dict(width, height, bits, sub="420", rng="limited", loc="left", matrix="bt709", transfer="none"):
    return dict(width=width, height=height, bit_depth=bits, subsampling=sub, range=rng, chroma_loc=loc,
                matrix=matrix, transfer=transfer)


def to_dev(arr):
    """numpy uint8/uint16 plane -> torch cuda tensor of the same bytes."""
    a = np.ascontiguousarray(arr)
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda()
    return torch.from_numpy(a).cuda()


def from_dev(t, bits):
    a = t.cpu().numpy()
    return a.view(np.uint16).astype(np.int64) if bits > 8 else a.astype(np.int64)


def prequant(rgb, fmt):
    """Oracle requantisation values before rounding (to locate round-half ties)."""
    b, rg = fmt["bit_depth"], fmt["range"]
    rgb = oracle.from_linear(np.asarray(rgb, np.float64), fmt.get("transfer", "none"))  # PQ / HLG
    if fmt.get("matrix") == "rgb":  # R'G'B' planes, luma range equations
        return {k: oracle.scale_luma(rgb[i], b, rg) for i, k in enumerate("YUV")}
    yp, cb, cr = oracle.rgb_to_ycbcr(rgb[0], rgb[1], rgb[2], fmt.get("matrix", "bt709"))
    cb = oracle.downsample_chroma(cb, fmt["subsampling"], fmt["chroma_loc"])
    cr = oracle.downsample_chroma(cr, fmt["subsampling"], fmt["chroma_loc"])
    return {"Y": oracle.scale_luma(yp, b, rg), "U": oracle.scale_chroma(cb, b, rg),
            "V": oracle.scale_chroma(cr, b, rg)}


def assert_codes_match(got, exp_float, bits, tie_band=2e-3):
    """Integer codes equal the oracle's except at rounding near-ties (|frac - 0.5| < tie_band),
    where the FP32 kernel and the FP64 oracle may round apart by one code.  FP32 values
    carry ~1e-7 relative error, so above 10 bits the band grows with the code range."""
    if bits > 10:
        tie_band *= 2.0 ** (bits - 10)
    for k in "YUV":
        g = got[k]
        v = np.clip(exp_float[k], 0, 2 ** bits - 1)
        e = oracle.quantise(exp_float[k], bits)
        diff = np.abs(g - e)
        near_tie = np.abs(np.abs(v - np.floor(v)) - 0.5) < tie_band
        assert diff.max() <= 1, (k, diff.max())
        bad = (diff > 0) & ~near_tie
        assert not bad.any(), (k, int(bad.sum()), np.argwhere(bad)[:5])


def lsb_stats(got, exp):
    """max |diff| and fraction of exact codes over the three planes."""
    d = [np.abs(got[k].astype(np.int64) - exp[k].astype(np.int64)) for k in "YUV"]
    n = sum(x.size for x in d)
    return max(int(x.max()) for x in d), sum(int((x == 0).sum()) for x in d) / n


def oracle_window(net, frames_rgb, y0, y1, x0, x1, out_fmt):
    """Oracle output codes of the LR window [y0,y1) x [x0,x1) (even-aligned) of one frame.

    Runs the network on a crop with margin >= the receptive radius (+1 so the
    chroma downsampling's left neighbour is exact) and requantises the crop;
    entries away from the crop's artificial borders equal the full-frame result.
    """
    R = net.receptive_radius() + 2
    H, W = frames_rgb[0].shape[1:]
    cy0, cy1 = max(y0 - R, 0), min(y1 + R, H)
    cx0, cx1 = max(x0 - R, 0), min(x1 + R, W)
    cy0 -= cy0 % 2
    cx0 -= cx0 % 2
    crop = [f[:, cy0:cy1, cx0:cx1] for f in frames_rgb]
    out = net.forward(crop)[0]
    s = net.scale
    pq = prequant(out, out_fmt)
    oy, ox = (y0 - cy0) * s, (x0 - cx0) * s
    hy, hx = (y1 - y0) * s, (x1 - x0) * s
    res = {"Y": pq["Y"][oy:oy + hy, ox:ox + hx]}
    if out_fmt["subsampling"] == "420":
        res["U"] = pq["U"][oy // 2:(oy + hy) // 2, ox // 2:(ox + hx) // 2]
        res["V"] = pq["V"][oy // 2:(oy + hy) // 2, ox // 2:(ox + hx) // 2]
    else:
        res["U"] = pq["U"][oy:oy + hy, ox:ox + hx]
        res["V"] = pq["V"][oy:oy + hy, ox:ox + hx]
    return res


def crop_codes(planes, y0, y1, x0, x1, s, sub):
    out = {"Y": planes["Y"][y0 * s:y1 * s, x0 * s:x1 * s]}
    if sub == "420":
        out["U"] = planes["U"][y0 * s // 2:y1 * s // 2, x0 * s // 2:x1 * s // 2]
        out["V"] = planes["V"][y0 * s // 2:y1 * s // 2, x0 * s // 2:x1 * s // 2]
    else:
        out["U"] = planes["U"][y0 * s:y1 * s, x0 * s:x1 * s]
        out["V"] = planes["V"][y0 * s:y1 * s, x0 * s:x1 * s]
    return out


def _run_layer(layer, env):
    """One layer of the oracle graph on the tensors of env (as oracle.Net.forward does)."""
    srcs = layer.get("in").split(",")
    x = np.concatenate([env[s] for s in srcs]) if len(srcs) > 1 else env[srcs[0]]
    y = oracle.conv2d_direct(x, layer.w, layer.b)
    if layer.get("act") == "lrelu":
        y = oracle.leaky_relu(y)
    if layer.get("add"):
        y = y + env[layer.get("add")]
    if layer.get("ps"):
        y = oracle.pixel_shuffle(y, layer.get("ps"))
    return y


def stvsr_window(net, rgb, y0, y1, x0, x1, out_fmt, margin=16):
    """Oracle codes of the LR window [y0,y1) x [x0,x1) of both outputs of the first run
    of the deformable space-time SR network (synth.net_group_stvsr), at full size.

    The DCN's reach is data dependent, so it cannot be cropped like a plain conv
    stack.  Instead: the extract convs run on the whole frames; the offset/mask
    heads and everything after the DCNs run on a crop of `margin` LR pixels around
    the window (the radius of the layers after the DCN, plus the head's); the DCNs
    sample the whole-frame features at the crop's pixels.  Entries away from the
    crop's artificial borders equal the whole-frame result.
    """
    L = {layer.name: layer for layer in net.layers}
    H, W = rgb[0].shape[1:]
    s = net.scale
    cy0, cy1 = max(y0 - margin, 0), min(y1 + margin, H)
    cx0, cx1 = max(x0 - margin, 0), min(x1 + margin, W)
    cy0 -= cy0 % 2
    cx0 -= cx0 % 2
    full = {"frame0": rgb[0], "frame1": rgb[1]}
    full["f0"] = _run_layer(L["f0"], full)
    full["f1"] = _run_layer(L["f1"], full)
    crop = {k: v[:, cy0:cy1, cx0:cx1] for k, v in full.items()}
    for a, head in (("a0", "om01"), ("a1", "om10")):
        om_c = _run_layer(L[head], crop)  # exact inside the crop's interior
        om = np.zeros((om_c.shape[0], H, W))
        om[:, cy0:cy1, cx0:cx1] = om_c
        d = L[a]
        g = d.get("groups")
        y = oracle.dcn2d(full[d.get("in")], om[:18 * g], oracle.sigmoid(om[18 * g:27 * g]), d.w, d.b, g,
                         window=(cy0, cy1, cx0, cx1))
        crop[a] = y[:, cy0:cy1, cx0:cx1]
    names = [layer.name for layer in net.layers if layer.name not in ("f0", "f1", "om01", "om10", "a0", "a1")]
    for name in names:
        crop[name] = _run_layer(L[name], crop)
    res = []
    for name, skip in net.outputs:
        frames = (skip or "").split(",")
        sk = sum(net._skip(crop[f]) for f in frames) / len(frames)
        pq = prequant(crop[name] + sk, out_fmt)
        oy, ox = (y0 - cy0) * s, (x0 - cx0) * s
        hy, hx = (y1 - y0) * s, (x1 - x0) * s
        res.append({"Y": pq["Y"][oy:oy + hy, ox:ox + hx],
                    "U": pq["U"][oy // 2:(oy + hy) // 2, ox // 2:(ox + hx) // 2],
                    "V": pq["V"][oy // 2:(oy + hy) // 2, ox // 2:(ox + hx) // 2]})
    return res
