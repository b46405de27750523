"""The windowed oracle of the deformable ST-SR network (tests/gpu_util.stvsr_window), used
for sampled full-size checks, equals the oracle's whole-frame forward on a small clip."""
import numpy as np

import oracle
import synth
from gpu_util import fmt_dict, prequant, stvsr_window


def test_stvsr_window_equals_full_forward():
    W, H = 144, 72
    frames = synth.frames_textured(synth.BASE_SEED + 3, 2, W, H, 8, "420", "limited")
    text, blob = synth.net_stvsr4x()
    net = oracle.Net(text, blob)
    fdi, fdo = fmt_dict(W, H, 8), fmt_dict(4 * W, 4 * H, 8)
    rgb = [oracle.ingest(f, fdi) for f in frames]
    full = [prequant(o, fdo) for o in net.forward(rgb)]
    for (y0, y1, x0, x1) in [(0, 8, 0, 8), (30, 38, 60, 68), (64, 72, 136, 144)]:
        res = stvsr_window(net, rgb, y0, y1, x0, x1, fdo)
        for k in range(2):
            for p in "YUV":
                s = 4 if p == "Y" else 2
                ref = full[k][p][y0 * s:y1 * s, x0 * s:x1 * s]
                assert np.abs(res[k][p] - ref).max() < 1e-9, (y0, x0, k, p)
