"""Helpers shared by the GPU tests: run a workload through the C-ABI and
compare with an oracle result transition by transition."""
import numpy as np

import paper_2304_13398_gb300 as gls


def run_gpu(ctx, nl, st, arena_events=0, keep=False):
    """Load, simulate, read back; release the device objects unless keep."""
    nid = ctx.load_netlist(nl)
    sid = ctx.load_stimulus(st, n_pi=nl.n_pi)
    rid = ctx.simulate(nid, sid, arena_events=arena_events)
    stats = ctx.run_stats(rid)
    off, packed = ctx.read_all(rid)
    t, v = gls.unpack(packed)
    if not keep:
        for i in (rid, sid, nid):
            ctx.release(i)
        return None, stats, off, t, v
    return (nid, sid, rid), stats, off, t, v


def assert_same(ref, off, t, v, what=""):
    assert np.array_equal(off, ref.off), f"{what}: waveform lengths differ at nets " \
        f"{np.nonzero(np.diff(off) != np.diff(ref.off))[0][:10]}"
    bad = np.nonzero((t.astype(np.int64) != ref.t) | (v != ref.v))[0]
    if len(bad):
        e = int(bad[0])
        net = int(np.searchsorted(ref.off, e, side="right") - 1)
        raise AssertionError(f"{what}: {len(bad)} transitions differ; first at net {net}, "
                             f"index {e - int(ref.off[net])}: gpu ({t[e]}, {v[e]}) vs oracle ({ref.t[e]}, {ref.v[e]})")
