"""C-ABI library checks that need no GPU: exports, host-side grouping logic
(bit-exact against the oracle), and network-description validation."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2308_03121_gb300 as nv
import synth

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "nvisr.h")


def _declared():
    text = open(HDR).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nvisr_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = nv.load()
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.nvisr_abi_version() == 2


def test_binding_covers_every_declared_symbol():
    assert set(_declared()) <= set(nv._SIGS)


@pytest.mark.parametrize("T", [1, 3, 5, 7])
def test_tuple_map_matches_oracle(T):
    rng = np.random.default_rng(T)
    for trial in range(40):
        n = int(rng.integers(1, 40))
        flags = rng.uniform(size=n) < 0.15
        got = nv.nvisr_tuple_map(flags, T)
        exp = np.array(oracle.tuple_map(flags, n, T), np.int32).reshape(n, T)
        assert np.array_equal(got, exp)


def test_tuple_map_t3_cut_on_frame_9():
    flags = np.zeros(16, bool)
    flags[9] = True
    got = nv.nvisr_tuple_map(flags, 3)
    assert got[8].tolist() == [7, 8, 8] and got[9].tolist() == [9, 9, 10]


@pytest.mark.parametrize("n,extra", [(1, True), (3, False), (2, True), (3, True), (4, False)])
def test_group_runs_match_oracle(n, extra):
    for s0, s1 in [(0, 0), (0, 1), (5, 11), (0, 39), (3, 4), (10, 16)]:
        assert nv.nvisr_group_runs(s0, s1, n, extra) == oracle.group_runs(s0, s1, n, extra)


@pytest.mark.parametrize("n,extra,interp,double", [
    (1, True, True, True), (1, True, True, False), (2, True, True, False), (3, False, False, False),
    (2, False, False, True), (2, True, True, True), (3, True, False, False), (1, False, True, False)])
def test_group_outputs_match_oracle(n, extra, interp, double):
    """The filter's own output bookkeeping (what nvisr_pull reports, run without a device)
    equals the oracle's presentation order for every flag set, with cuts and short scenes."""
    rng = np.random.default_rng(n * 16 + extra * 8 + interp * 4 + double * 2)
    for trial in range(25):
        nf = int(rng.integers(1, 24))
        flags = rng.uniform(size=nf) < 0.2
        got = nv.nvisr_group_outputs(flags, n, extra, interp, double)
        exp = []
        for e in oracle.group_outputs(flags, nf, n, extra, interp, double):
            if e[0] == "pass":
                exp.append((nv.OUT_PASSTHROUGH, e[1], e[1], -1))
            else:
                exp.append((nv.OUT_NETWORK, e[1][0], e[1][-1], e[2]))
        assert got == exp, (trial, flags)


@pytest.mark.parametrize("n,b", [(1, 1), (1, 4), (2, 3), (3, 2), (4, 5), (7, 3)])
def test_fig1_layout_matches_oracle(n, b):
    cells, slots, copy = nv.nvisr_fig1_layout(n, b)
    grid, slot_start = oracle.fig1_layout(n, b)
    flat = [grid[a % b][a // b] for a in range((n + 1) * b)]
    assert cells.tolist() == [-1 if v is None else v for v in flat]
    assert slots.tolist() == slot_start
    assert tuple(copy.tolist()) == oracle.fig1_next_batch_copy(n, b, rolling=False)


def test_network_check_accepts_the_workload_networks():
    for text, blob in (synth.net_sr2x_t3(), synth.net_sr2x_t5(), synth.net_stvsr4x()):
        st, msg = nv.nvisr_network_check(text, blob.size)
        assert st == 0, msg


@pytest.mark.parametrize("mutate,needle", [
    (lambda t: t.replace("nvisr-net 1", "nvisr-net 2"), "nvisr-net"),
    (lambda t: t.replace("k=3", "k=5", 1), "k must be"),
    (lambda t: t.replace("in=r0a", "in=nosuch", 1), "unknown source"),
    (lambda t: t.replace("act=lrelu", "act=gelu", 1), "unknown act"),
    (lambda t: t + "bogus line\n", "unknown statement"),
])
def test_network_check_rejects_malformed(mutate, needle):
    text, blob = synth.net_sr2x_t3()
    st, msg = nv.nvisr_network_check(mutate(text), blob.size)
    assert st == nv.Status.BAD_NETWORK and needle in msg


@pytest.mark.parametrize("scale", [(1, 1), (1, 2), (2, 1)])
def test_network_check_accepts_separate_scales(scale):
    text, blob = synth.net_tuple(3, frames=3, channels=16, nres=1, scale=scale)
    st, msg = nv.nvisr_network_check(text, blob.size)
    assert st == 0, msg


@pytest.mark.parametrize("attr,needle", [("psx=3", "psx / psy"), ("ps=2 psx=2", "ps with psx"),
                                         ("psx=2", "divisible by psx")])
def test_network_check_rejects_bad_shuffle_factors(attr, needle):
    text, blob = synth.net_tuple(3, frames=3, channels=16, nres=1, scale=(1, 1))
    bad = text.replace("conv tail in=r0b cin=16 cout=3 k=3 act=none", "conv tail in=r0b cin=16 cout=3 k=3 act=none " + attr)
    assert bad != text
    st, msg = nv.nvisr_network_check(bad, blob.size)
    assert st == nv.Status.BAD_NETWORK and needle in msg, msg


def test_network_check_rejects_blob_size():
    text, blob = synth.net_sr2x_t3()
    st, msg = nv.nvisr_network_check(text, blob.size + 1)
    assert st == nv.Status.BAD_NETWORK and "weight blob" in msg
