"""Batched multi-stream stepping through the C ABI: every stream's outputs from a
shared batch (one launch per 64->64 layer over all streams, CUDA graph replay,
autotuned strip height) equal the same stream run alone, bit for bit, for
streams of different sizes, bit depths and chroma layouts, across a scene cut
and the end of each stream."""
import numpy as np
import pytest
import torch

import paper_2308_03121_gb300 as nv
import synth

pytestmark = pytest.mark.gpu

STREAMS = [  # width, height, bits, subsampling, frames, cut before frame
    (96, 64, 10, "420", 7, 3),
    (70, 40, 8, "420", 6, None),
    (64, 48, 8, "444", 5, None),
    (130, 66, 10, "420", 8, 5),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nv.load()


def _frames(k, W, H, bits, sub, n):
    return synth.frames_textured(synth.BASE_SEED + 40 + k, n, W, H, bits, sub, "limited")


def _fmts(W, H, bits, sub):
    return nv.fmt(W, H, bits, sub), nv.fmt(2 * W, 2 * H, bits, sub)


def _alone(text, blob, frames, cut, W, H, bits, sub, prec):
    eng = nv.Engine()
    fi, fo = _fmts(W, H, bits, sub)
    flt = eng.filter(text, blob, fi, fo, prec, 2)
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


def _batched(text, blob, clips, precs):
    eng = nv.Engine()
    flts = []
    for (W, H, bits, sub, n, cut), prec in zip(STREAMS, precs):
        fi, fo = _fmts(W, H, bits, sub)
        flts.append(eng.filter(text, blob, fi, fo, prec, 2))
    b = eng.batch(flts)
    outs = [[] for _ in flts]
    nxt = [0] * len(flts)
    done = [False] * len(flts)
    flushed = [False] * len(flts)
    for _ in range(200):
        for k, f in enumerate(flts):
            frames, cut = clips[k]
            if nxt[k] < len(frames):
                fr = frames[nxt[k]]
                if f.push((fr["Y"], fr["U"], fr["V"]), cut=(nxt[k] == cut)) == nv.Status.OK:
                    nxt[k] += 1
            elif not flushed[k]:
                f.flush()
                flushed[k] = True
        ready = sum(1 for k, f in enumerate(flts) if not done[k] and f.ready() > 0)
        assert b.step() == ready  # every stream with a ready output is computed by the batch
        for k, f in enumerate(flts):
            if done[k] or f.ready() == 0:
                if flushed[k] and f.ready() == 0:
                    res = f.alloc_out_host()
                    st, _ = f.pull(res)
                    if st == nv.Status.EOS:
                        done[k] = True
                    else:
                        assert st == nv.Status.AGAIN
                continue
            res = f.alloc_out_host()
            st, _ = f.pull(res)  # exactly one output per stream per step: the batched one
            assert st == nv.Status.OK
            outs[k].append([r.copy() for r in res])
        if all(done):
            break
    info = b.info()
    b.close()
    eng.close()
    return outs, info


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_batch_equals_each_stream_alone(prec):
    text, blob = synth.net_sr2x_t5()
    clips = [(_frames(k, W, H, bits, sub, n), cut) for k, (W, H, bits, sub, n, cut) in enumerate(STREAMS)]
    got, info = _batched(text, blob, clips, [prec] * len(STREAMS))
    assert info["shared"] and info["graphs"] >= 1 and info["rows_per_strip"] > 0, info
    for k, (W, H, bits, sub, n, cut) in enumerate(STREAMS):
        want = _alone(text, blob, clips[k][0], cut, W, H, bits, sub, prec)
        assert len(got[k]) == len(want) == n, (k, len(got[k]), len(want))
        for t, (g, w) in enumerate(zip(got[k], want)):
            for p in range(3):
                assert np.array_equal(g[p], w[p]), (k, t, p, int(np.abs(g[p].astype(np.int64) - w[p]).max()))


def test_mixed_precision_batch_steps_members_one_by_one():
    text, blob = synth.net_sr2x_t5()
    clips = [(_frames(k, W, H, bits, sub, n), cut) for k, (W, H, bits, sub, n, cut) in enumerate(STREAMS)]
    precs = ["bf16", "fp32", "bf16", "bf16"]
    got, info = _batched(text, blob, clips, precs)
    assert not info["shared"]
    for k in (0, 1):
        W, H, bits, sub, n, cut = STREAMS[k]
        want = _alone(text, blob, clips[k][0], cut, W, H, bits, sub, precs[k])
        assert len(got[k]) == len(want) == n
        for g, w in zip(got[k], want):
            for p in range(3):
                assert np.array_equal(g[p], w[p])
