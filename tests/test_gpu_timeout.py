"""The DEVICE_TIMEOUT path of the C ABI, driven without a GPU fault.

Every pipeline wait of the tensor-core kernels is bounded (2 s).  A CTA whose
wait runs out raises an abort flag seen by its other roles, records the
timeout in the error word, lets its own copies and MMAs finish, frees its
TMEM and returns; the host call then returns NVISR_DEVICE_TIMEOUT.  The fault
drill (nvisr_test_starve) makes the producers load nothing, so the first
pipeline wait runs out on every run.  Each test then switches the drill off
and checks that the next call on the same context succeeds and is correct,
which needs the aborted CTAs to have released their TMEM.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2308_03121_gb300 as nv
import synth
from gpu_util import fmt_dict, lsb_stats, prequant

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nv.load()
    yield
    nv.nvisr_test_starve(False)


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).double().numpy()


@pytest.mark.parametrize("cin,cout,H,W", [(16, 48, 17, 70),     # the generic tensor-core conv
                                          (64, 64, 37, 150)])   # the row-streaming kernel
def test_conv_wait_runs_out_then_next_call_succeeds(cin, cout, H, W):
    rs = np.random.default_rng(cin + W)
    x = rs.uniform(-1, 1, size=(cin, H, W)).astype(np.float32)
    w = (rs.normal(size=(cout, cin, 3, 3)) * np.sqrt(2.0 / (9 * cin))).astype(np.float32)
    b = rs.uniform(-0.1, 0.1, size=cout).astype(np.float32)
    xd, wd, bd = (torch.from_numpy(a).cuda() for a in (x, w, b))
    nv.nvisr_test_starve(True)
    try:
        with pytest.raises(nv.NvisrError) as ei:
            nv.nvisr_conv2d("bf16", xd, wd, bd, 1)
    finally:
        nv.nvisr_test_starve(False)
    assert ei.value.status == nv.Status.DEVICE_TIMEOUT
    got = nv.nvisr_conv2d("bf16", xd, wd, bd, 1)
    torch.cuda.synchronize()
    ref = oracle.leaky_relu(oracle.conv2d_direct(_bf16(x), _bf16(w), b))
    err = np.abs(got.double().cpu().numpy() - ref).max()
    assert err < 2e-5 + 2.0 ** -8 * np.abs(ref).max(), err


def test_dcn_wait_runs_out_then_next_call_succeeds():
    cin = cout = 64
    groups, H, W = 8, 6, 140
    x, off, m = synth.dcn_operands(5, cin, H, W, groups)
    rs = np.random.default_rng(6)
    w = (rs.normal(size=(cout, cin, 3, 3)) * np.sqrt(2.0 / (9 * cin))).astype(np.float32)
    b = rs.uniform(-0.1, 0.1, size=cout).astype(np.float32)
    args = [torch.from_numpy(a).cuda() for a in (x, off, m, w, b)]
    nv.nvisr_test_starve(True)
    try:
        with pytest.raises(nv.NvisrError) as ei:
            nv.nvisr_dcn2d("bf16", *args, groups)
    finally:
        nv.nvisr_test_starve(False)
    assert ei.value.status == nv.Status.DEVICE_TIMEOUT
    got = nv.nvisr_dcn2d("bf16", *args, groups)
    torch.cuda.synchronize()
    ref = oracle.dcn2d(_bf16(x), off, m, _bf16(w), b, groups)
    mag = oracle.dcn2d(np.abs(_bf16(x)), off, m, np.abs(_bf16(w)), None, groups)
    tol = 2.0 ** -8 * (mag + np.abs(ref)) + 1e-5
    assert (np.abs(got.double().cpu().numpy() - ref) <= tol).all()


def test_filter_pull_reports_timeout_then_recovers():
    """A pull whose network launches time out returns DEVICE_TIMEOUT; outputs the filter
    computed ahead in the same state are dropped, and pulling again gives every output
    within 1 LSB of the oracle (BF16, the 3-frame 32-channel 2x network, 8 frames, a cut on frame 5)."""
    W = H = 48
    frames = synth.frames_gradient(11, 8, W, H, 8, "420", "full")
    flags = np.zeros(8, bool)
    flags[5] = True
    text, blob = synth.net_sr2x_t3()
    fd_in, fd_out = fmt_dict(W, H, 8, rng="full"), fmt_dict(2 * W, 2 * H, 8, rng="full")
    ref = oracle.run_filter(frames, flags, text, blob, fd_in, fd_out, keep_float=True)
    eng = nv.Engine()
    flt = eng.filter(text, blob, nv.fmt(W, H, 8, "420", "full"), nv.fmt(2 * W, 2 * H, 8, "420", "full"), "bf16")
    got = []

    def pull_one():
        out = flt.alloc_out_host()
        st, info = flt.pull(out)
        if st == nv.Status.OK:
            assert info.index == len(got)
            got.append({k: p.astype(np.int64) for k, p in zip("YUV", out)})
        return st

    k = 0
    while flt.ready() < 2:  # outputs 0 and 1 known: the pull runs 1 ahead
        assert flt.push((frames[k]["Y"], frames[k]["U"], frames[k]["V"]), cut=bool(flags[k])) == nv.Status.OK
        k += 1
    nv.nvisr_test_starve(True)
    try:
        with pytest.raises(nv.NvisrError) as ei:
            pull_one()
    finally:
        nv.nvisr_test_starve(False)
    assert ei.value.status == nv.Status.DEVICE_TIMEOUT
    assert "time bound" in eng.last_error()
    for i in range(k, len(frames)):
        while flt.push((frames[i]["Y"], frames[i]["U"], frames[i]["V"]), cut=bool(flags[i])) == nv.Status.FULL:
            assert pull_one() == nv.Status.OK
    flt.flush()
    while pull_one() != nv.Status.EOS:
        pass
    eng.close()
    assert len(got) == 8
    for g, r in zip(got, ref):
        pq = prequant(r, fd_out)
        mx, _ = lsb_stats(g, {k: oracle.quantise(pq[k], 8) for k in "YUV"})
        assert mx <= 1, mx
