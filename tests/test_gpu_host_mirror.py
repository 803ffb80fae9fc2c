"""Host-mirrored results (GLS_OPT_HOST_MIRROR): the kernels also store every
output transition into pinned host memory, and gls_read_host hands the
waveforms over without a device-to-host copy of them.  They must equal
gls_read_all and the oracle, after a rerun with new inputs, and per item of
a batch."""
import numpy as np
import pytest

import oracle
import paper_2304_13398_gb300 as gls
import synth
from gpu_util import assert_same

pytestmark = pytest.mark.gpu


def from_host(ctx, rid, item, n_pi, stim):
    arena, off, ln = ctx.read_host(rid, item)
    G = len(off)
    offs = np.zeros(n_pi + G + 1, np.int64)
    offs[1:n_pi + 1] = np.cumsum(np.diff(stim.off))
    offs[n_pi + 1:] = offs[n_pi] + np.cumsum(ln.astype(np.int64))
    parts = [((stim.t.astype(np.int64) << 2) | stim.v).astype(np.uint32)]
    parts += [arena[o:o + l] for o, l in zip(off, ln)]
    packed = np.concatenate(parts) if parts else np.zeros(0, np.uint32)
    t, v = gls.unpack(packed)
    return offs, t, v


@pytest.mark.parametrize("kernel,schedule", [("wide", "dependency"), ("windowed", "levels")])
def test_host_mirror_equals_oracle(kernel, schedule):
    nl = synth.make_netlist(16, 3000, 12, fanout="pareto", d_min=5, d_max=200, seed=91)
    st = synth.make_stimulus(16, mean=150, window=60_000, seed=92)
    st2 = synth.make_stimulus(16, mean=150, window=60_000, seed=93)
    with gls.Context(0) as ctx:
        ctx.set_kernel(kernel)
        ctx.set_schedule(schedule)
        ctx.set_option(gls.gls.GLS_OPT_HOST_MIRROR, 1)
        nid = ctx.load_netlist(nl)
        sid = ctx.load_stimulus(st)
        rid = ctx.simulate(nid, sid)
        ref = oracle.sim_event(nl, st)
        off, t, v = from_host(ctx, rid, 0, nl.n_pi, st)
        assert_same(ref, off, t, v, "host mirror")
        off2, packed = ctx.read_all(rid)
        np.testing.assert_array_equal(off2, off)
        # new inputs in place, evaluated again: the mirror follows
        ctx.update_stimulus(sid, st2.off, st2.t, st2.v)
        ctx.rerun(rid)
        off, t, v = from_host(ctx, rid, 0, nl.n_pi, st2)
        assert_same(oracle.sim_event(nl, st2), off, t, v, "host mirror after rerun")


def test_host_mirror_batch_items_and_errors():
    nl = synth.make_netlist(8, 800, 9, d_min=5, d_max=100, seed=95)
    sts = [synth.make_stimulus(8, mean=60, window=20_000, seed=96 + k) for k in range(3)]
    with gls.Context(0) as ctx:
        nid = ctx.load_netlist(nl)
        sids = [ctx.load_stimulus(s) for s in sts]
        rid0 = ctx.simulate(nid, sids[0])
        ctx.run_stats(rid0)
        with pytest.raises(gls.GlsError):
            ctx.read_host(rid0)                      # created without the mirror
        ctx.set_option(gls.gls.GLS_OPT_HOST_MIRROR, 1)
        rid = ctx.simulate_batch([nid] * 3, sids)
        for i, s in enumerate(sts):
            off, t, v = from_host(ctx, rid, i, nl.n_pi, s)
            assert_same(oracle.sim_event(nl, s), off, t, v, f"item {i}")
        ctx.set_kernel("segmented")
        with pytest.raises(gls.GlsError):
            ctx.simulate(nid, sids[0])              # the mirror needs the windowed kernels
