"""GPU parity of general cells -- the full delay matrix with its input-edge
dimension, cells with several outputs, user-defined tables (UDP), pins
without arcs -- against the CPU oracle (oracle.sim_cells), transition by
transition."""
import numpy as np
import pytest

import oracle
import paper_2304_13398_gb300 as gls
import synth
from gpu_util import assert_same

pytestmark = pytest.mark.gpu


def run_cells(ctx, cn, st, sliced=0):
    nid = ctx.load_cell_netlist(cn)
    sid = ctx.load_stimulus(st)
    if sliced:
        rid = ctx.simulate_sliced(nid, sid, sliced)
        off, t, v = ctx.read_all64(rid)
    else:
        rid = ctx.simulate(nid, sid)
        ctx.run_stats(rid)
        off, packed = ctx.read_all(rid)
        t, v = gls.unpack(packed)
    return off, t, v


@pytest.mark.parametrize("kernel,schedule", [("windowed", "dependency"), ("windowed", "levels"),
                                             ("wide", "dependency")])
@pytest.mark.parametrize("fr", [dict(multi_frac=0.4, edge_frac=0.5, noarc_frac=0.15, x_frac=0.6),
                                dict(multi_frac=0.0, edge_frac=1.0, noarc_frac=0.0, x_frac=0.3),
                                dict(multi_frac=1.0, edge_frac=0.0, noarc_frac=0.3, x_frac=0.8)])
def test_cells_equal_oracle(kernel, schedule, fr):
    cn = synth.make_cell_netlist(14, 2500, 12, seed=21, shuffle=True, **fr)
    st = synth.make_stimulus(14, mean=120, window=50_000, seed=22)
    ref = oracle.sim_cells(cn, st)
    with gls.Context(0) as ctx:
        ctx.set_kernel(kernel)
        ctx.set_schedule(schedule)
        off, t, v = run_cells(ctx, cn, st)
    assert_same(ref, off, t, v, f"{kernel}/{schedule}")
    assert ref.off[-1] - ref.off[cn.n_pi] > 10_000


def test_builtin_cells_through_the_cell_loader():
    """Built-in cell ids in the general loader, rise/fall for both edges:
    the same waveforms as the classic loader and the oracle."""
    nl = synth.make_netlist(12, 2000, 11, fanout="pareto", d_min=5, d_max=200, seed=33)
    st = synth.make_stimulus(12, mean=100, window=40_000, seed=34)
    ref = oracle.sim_event(nl, st)
    k = np.diff(nl.fanin_off)
    d = np.zeros(4 * len(nl.fanin_net), np.int32)
    d[0::4] = d[2::4] = nl.d_fall
    d[1::4] = d[3::4] = nl.d_rise
    with gls.Context(0) as ctx:
        nid = ctx.load_netlist_cells(nl.n_pi, nl.type.astype(np.int32), nl.fanin_off, nl.fanin_net, d)
        sid = ctx.load_stimulus(st)
        rid = ctx.simulate(nid, sid)
        ctx.run_stats(rid)
        off, packed = ctx.read_all(rid)
        t, v = gls.unpack(packed)
        assert_same(ref, off, t, v, "built-in cells, general loader")
        ctx.set_kernel("segmented")      # no general feature: the segmented kernel applies too
        rid = ctx.simulate(nid, sid)
        ctx.run_stats(rid)
        off, packed = ctx.read_all(rid)
        t, v = gls.unpack(packed)
        assert_same(ref, off, t, v, "built-in cells, general loader, segmented")
    assert k.max() == 3


def test_edge_delay_xor_golden_on_gpu():
    from golden_io import waveform_cases
    cases = waveform_cases("edge_delay_xor.txt")
    xor = gls.cell_table(6)            # XOR2
    d = np.array([9, 7, 11, 13,        # pin a: rising (to 0, to 1), falling (to 0, to 1)
                  22, 20, 26, 24], np.int32)
    for name in ("edges", "pulse_eaten"):
        pins, want = cases[name]
        off = np.array([0, len(pins["a"]), len(pins["a"]) + len(pins["b"])], np.int64)
        t = np.array([x for x, _ in pins["a"]] + [x for x, _ in pins["b"]], np.int32)
        v = np.array([y for _, y in pins["a"]] + [y for _, y in pins["b"]], np.uint8)
        with gls.Context(0) as ctx:
            ct = ctx.define_cell(2, xor)
            nid = ctx.load_netlist_cells(2, [ct], [0, 2], [0, 1], d)
            sid = ctx.load_stimulus(synth.Stimulus(off, t, v))
            rid = ctx.simulate(nid, sid)
            ctx.run_stats(rid)
            tz, vz = ctx.read_waveform(rid, 2)
            assert list(zip(tz.tolist(), vz.tolist())) == want, name


def test_cells_sliced_equal_oracle():
    cn = synth.make_cell_netlist(12, 1500, 10, seed=41, multi_frac=0.4, edge_frac=0.6, noarc_frac=0.2)
    st = synth.make_stimulus(12, mean=90, window=40_000, seed=42)
    ref = oracle.sim_cells(cn, st)
    with gls.Context(0) as ctx:
        for sl in (173, 5_000):
            off, t, v = run_cells(ctx, cn, st, sliced=sl)
            assert_same(ref, off, t, v, f"sliced {sl}")


def test_general_cells_reject_segmented():
    cn = synth.make_cell_netlist(6, 100, 5, seed=51, edge_frac=1.0)
    st = synth.make_stimulus(6, mean=20, window=5_000, seed=52)
    with gls.Context(0) as ctx:
        nid = ctx.load_cell_netlist(cn)
        sid = ctx.load_stimulus(st)
        ctx.set_kernel("segmented")
        with pytest.raises(gls.GlsError):
            ctx.simulate(nid, sid)


def test_cell_definition_errors():
    with gls.Context(0) as ctx:
        with pytest.raises(gls.GlsError):
            ctx.define_cell(2, np.full(16, 3, np.uint8))        # value 3 (Z) is not an output
        with pytest.raises(gls.GlsError):
            ctx.define_cell(4, np.zeros(256, np.uint8))         # 4 inputs
        ct = ctx.define_cell(1, [0, 1, 2, 2])
        with pytest.raises(gls.GlsError):                      # no arc at all
            ctx.load_netlist_cells(1, [ct], [0, 1], [0], [-1, -1, -1, -1])
        with pytest.raises(gls.GlsError):                      # half an arc
            ctx.load_netlist_cells(1, [ct], [0, 1], [0], [5, -1, 5, 5])
        with pytest.raises(gls.GlsError):                      # fanin count
            ctx.load_netlist_cells(2, [ct], [0, 2], [0, 1], [5] * 8)
