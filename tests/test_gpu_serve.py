"""GPU tests of the serving layer and the device memory pool: every request
served in a continuously batched mix equals the same request simulated
alone and the CPU oracle."""
import numpy as np
import pytest

import oracle
import paper_2304_13398_gb300 as gls
import synth
from gpu_util import assert_same
from paper_2304_13398_gb300.serve import Request, Server, poisson_trace

pytestmark = pytest.mark.gpu

WINDOW = 50_000


def _cut(st, t_limit):
    keep = st.t < t_limit
    per = np.array([int(keep[st.off[i]:st.off[i + 1]].sum()) for i in range(len(st.off) - 1)], np.int64)
    off = np.zeros(len(per) + 1, np.int64)
    np.cumsum(per, out=off[1:])
    return synth.Stimulus(off, st.t[keep], st.v[keep])


def residents():
    out = {}
    for k, (G, D, n_pi) in enumerate([(120, 6, 8), (900, 14, 20), (2500, 20, 40)]):
        nl = synth.make_netlist(n_pi, G, D, fanout="pareto", d_min=5, d_max=200, seed=500 + k)
        st = synth.make_stimulus(n_pi, mean=400, window=WINDOW, probs=(0.45, 0.45, 0.07, 0.03), seed=600 + k)
        out[f"n{k}"] = (nl, st)
    return out


@pytest.mark.parametrize("batching,streams,policy", [(True, 3, "sjf"), (True, 3, "fifo"), (False, 1, "fifo")])
def test_served_results_equal_alone_and_oracle(batching, streams, policy):
    res = residents()
    with gls.Context(0) as ctx:
        ctx.set_option(gls.gls.GLS_OPT_POOL_BYTES, 8 << 30)
        ctx.set_option(gls.gls.GLS_OPT_HOST_POOL_BYTES, 4 << 30)
        srv = Server(ctx, budget_bytes=4 << 30, max_batch=8, streams=streams, batching=batching,
                     keep_results=True, policy=policy)
        for k, (nl, st) in res.items():
            srv.add_resident(k, nl, st, WINDOW)
        srv.calibrate()
        trace = poisson_trace(0.3, 200.0, list(res), 1000, WINDOW, seed=7)
        # half of the requests arrive in one burst, so that several wait together
        for q in trace[: len(trace) // 2]:
            q.arrival = 0.0
        stats = srv.serve(trace)
        assert stats.requests == len(trace) and stats.p50_ms <= stats.p99_ms
        if batching:
            assert stats.mean_batch > 1.0
        else:
            assert stats.mean_batch == 1.0
        for q in trace:
            nl, st = res[q.netlist]
            off, packed = q.result
            t, v = gls.unpack(packed)
            assert_same(oracle.sim_event(nl, _cut(st, q.t_limit)), off, t, v, f"request {q.rid}")
            # the waveforms the kernels wrote to host memory are the same
            np.testing.assert_array_equal(q.host_gates, packed[off[nl.n_pi]:])
        # a few requests alone, outside the mix
        for q in trace[:5]:
            r = srv.res[q.netlist]
            rid = ctx.simulate_batch([r.nid], [r.sid], t_limits=[q.t_limit])
            ctx.run_stats(rid)
            off, packed = ctx.read_item(rid, 0)
            assert np.array_equal(off, q.result[0]) and np.array_equal(packed, q.result[1])
            ctx.release(rid)


def test_pool_reuse_and_coalescing():
    w = synth.make_workload("tiny200", seed=3)
    ref = oracle.sim_event(w.netlist, w.stimulus)
    with gls.Context(0) as ctx:
        ctx.set_option(gls.gls.GLS_OPT_POOL_BYTES, 256 << 20)
        nid = ctx.load_netlist(w.netlist)
        sid = ctx.load_stimulus(w.stimulus)
        # many runs created and released out of order reuse the same region
        for rnd in range(3):
            rids = [ctx.simulate(nid, sid, arena_events=1 << 20) for _ in range(6)]
            for rid in rids[::2] + rids[1::2]:
                ctx.run_stats(rid)
                off, packed = ctx.read_all(rid)
                t, v = gls.unpack(packed)
                assert_same(ref, off, t, v, "pool run")
                ctx.release(rid)
        # after coalescing, one run can take most of the pool
        rid = ctx.simulate(nid, sid, arena_events=(200 << 20) // 4)
        ctx.run_stats(rid)
        ctx.release(rid)
        # a run beyond the pool is refused, not faulted
        with pytest.raises(gls.GlsError) as ei:
            ctx.simulate(nid, sid, arena_events=(300 << 20) // 4)
        assert ei.value.code == gls.gls.GLS_ENOMEM
        # the pool cannot be dropped while blocks are in use
        with pytest.raises(gls.GlsError):
            ctx.set_option(gls.gls.GLS_OPT_POOL_BYTES, 0)
        ctx.release(sid)
        ctx.release(nid)
        ctx.set_option(gls.gls.GLS_OPT_POOL_BYTES, 0)


def test_host_pool_mirrors():
    w = synth.make_workload("tiny200", seed=5)
    ref = oracle.sim_event(w.netlist, w.stimulus)
    P = w.netlist.n_pi
    with gls.Context(0) as ctx:
        ctx.set_option(gls.gls.GLS_OPT_HOST_POOL_BYTES, 64 << 20)
        ctx.set_option(gls.gls.GLS_OPT_HOST_MIRROR, 1)
        nid = ctx.load_netlist(w.netlist)
        sid = ctx.load_stimulus(w.stimulus)
        # mirrors carved from the pinned pool, released out of order and reused
        for rnd in range(2):
            rids = [ctx.simulate(nid, sid, arena_events=1 << 20) for _ in range(4)]
            for rid in rids[1::2] + rids[::2]:
                arena, goff, glen = ctx.read_host(rid)
                gates = np.concatenate([arena[o:o + n] for o, n in zip(goff.tolist(), glen.tolist())])
                t, v = gls.unpack(gates)
                np.testing.assert_array_equal(t.astype(np.int64), ref.t[ref.off[P]:])
                np.testing.assert_array_equal(v, ref.v[ref.off[P]:])
                ctx.release(rid)
        # a mirror larger than the pool is refused at run creation
        with pytest.raises(gls.GlsError) as ei:
            ctx.simulate(nid, sid, arena_events=(80 << 20) // 4)
        assert ei.value.code == gls.gls.GLS_ENOMEM
        # the pool cannot be dropped while a mirror is in use
        rid = ctx.simulate(nid, sid, arena_events=1 << 20)
        with pytest.raises(gls.GlsError):
            ctx.set_option(gls.gls.GLS_OPT_HOST_POOL_BYTES, 0)
        ctx.release(rid)
        ctx.set_option(gls.gls.GLS_OPT_HOST_MIRROR, 0)
        ctx.set_option(gls.gls.GLS_OPT_HOST_POOL_BYTES, 0)
