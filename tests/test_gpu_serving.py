"""Serving runtime through the C ABI (continuous batching): clips arrive while
others are on the GPU, are admitted as memory frees up, run in shared batched
steps, and each clip's output equals the clip run alone on its own engine."""
import numpy as np
import pytest
import torch

import paper_2308_03121_gb300 as nv
import synth

pytestmark = pytest.mark.gpu

# (network, width, height, bits, frames, cut-before, arrival step)
CLIPS = [
    ("sr2x", 96, 64, 10, 7, 3, 0),
    ("stvsr", 64, 48, 8, 4, 2, 0),
    ("sr2x", 70, 40, 8, 5, None, 2),
    ("sr2x", 96, 64, 10, 6, None, 4),
    ("stvsr", 48, 32, 8, 3, None, 5),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nv.load()


@pytest.fixture(scope="module")
def nets():
    return {"sr2x": (synth.net_sr2x_t5(), 2), "stvsr": (synth.net_stvsr4x(), 4)}


def _frames(k, W, H, bits, n):
    return synth.frames_textured(synth.BASE_SEED + 50 + k, n, W, H, bits, "420", "limited")


def _alone(text, blob, scale, frames, cut, W, H, bits):
    eng = nv.Engine()
    flt = eng.filter(text, blob, nv.fmt(W, H, bits), nv.fmt(scale * W, scale * H, bits), "bf16", scale)
    outs = []

    def pull():
        res = flt.alloc_out_host()
        st, _ = flt.pull(res)
        if st == nv.Status.OK:
            outs.append([r.copy() for r in res])
        return st

    for i, fr in enumerate(frames):
        while flt.push((fr["Y"], fr["U"], fr["V"]), cut=(i == cut)) == nv.Status.FULL:
            assert pull() == nv.Status.OK
    flt.flush()
    while pull() == nv.Status.OK:
        pass
    eng.close()
    return outs


def _serve(nets, clips, budget=0, max_active=0):
    eng = nv.Engine(hbm_budget_bytes=budget)
    srv = nv.Server(eng, max_active)
    state = {}
    outs = {k: [] for k in range(len(clips))}
    peak_pending = 0
    for step in range(400):
        for k, (net, W, H, bits, n, cut, arrive) in enumerate(clips):
            if arrive == step:
                (text, blob), scale = nets[net]
                cid = srv.submit(text, blob, nv.fmt(W, H, bits), nv.fmt(scale * W, scale * H, bits), "bf16", scale)
                state[k] = {"id": cid, "frames": _frames(k, W, H, bits, n), "next": 0, "flushed": False,
                            "done": False}
        for k, s in state.items():
            if s["done"]:
                continue
            frames = s["frames"]
            if s["next"] < len(frames):
                fr = frames[s["next"]]
                if srv.push(s["id"], (fr["Y"], fr["U"], fr["V"]), cut=(s["next"] == clips[k][5])) == nv.Status.OK:
                    s["next"] += 1
            elif not s["flushed"]:
                if srv.flush(s["id"]) == nv.Status.OK:
                    s["flushed"] = True
        peak_pending = max(peak_pending, srv.stats()["pending"])
        srv.step()
        for k, s in state.items():
            if s["done"]:
                continue
            while True:
                res = srv.alloc_out_host(s["id"])
                st, _ = srv.pull(s["id"], res)
                if st == nv.Status.OK:
                    outs[k].append([r.copy() for r in res])
                    continue
                if st == nv.Status.EOS:
                    srv.close_clip(s["id"])
                    s["done"] = True
                break
        if len(state) == len(clips) and all(s["done"] for s in state.values()):
            break
    stats = srv.stats()
    srv.close()
    eng.close()
    return outs, stats, peak_pending


def _check_against_alone(nets, outs):
    for k, (net, W, H, bits, n, cut, _) in enumerate(CLIPS):
        (text, blob), scale = nets[net]
        want = _alone(text, blob, scale, _frames(k, W, H, bits, n), cut, W, H, bits)
        assert len(outs[k]) == len(want) > 0, (k, len(outs[k]), len(want))
        for t, (g, w) in enumerate(zip(outs[k], want)):
            for p in range(3):
                assert np.array_equal(g[p], w[p]), (k, t, p)


def test_each_clip_same_alone_and_in_the_mix(nets):
    outs, stats, _ = _serve(nets, CLIPS)
    assert stats["admitted"] == len(CLIPS) and stats["completed"] == len(CLIPS)
    assert stats["outputs"] == sum(len(o) for o in outs.values())
    assert stats["latency_p99_ms"] >= stats["latency_p50_ms"] > 0
    _check_against_alone(nets, outs)


def test_admission_waits_for_memory_then_admits(nets):
    # a budget that holds the two first clips together, but not a third one until
    # one of them finishes (and any single clip on its own)
    sizes = []
    for net, W, H, bits, n, cut, _ in CLIPS:
        (text, blob), scale = nets[net]
        eng = nv.Engine()
        eng.filter(text, blob, nv.fmt(W, H, bits), nv.fmt(scale * W, scale * H, bits), "bf16", scale)
        sizes.append(eng.bytes_in_use())
        eng.close()
    budget = max(sizes[0] + sizes[1], max(sizes)) + min(sizes) // 2
    outs, stats, peak_pending = _serve(nets, CLIPS, budget=budget)
    assert peak_pending >= 1 and stats["deferred_steps"] >= 1, stats
    assert stats["admitted"] == len(CLIPS) and stats["completed"] == len(CLIPS)
    _check_against_alone(nets, outs)
