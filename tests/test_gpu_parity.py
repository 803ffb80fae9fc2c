"""GPU parity: waveforms from libgls.so (through the C-ABI) must equal the CPU
oracle's transition by transition (integer work: bit-exact)."""
import numpy as np
import pytest

import oracle
import paper_2304_13398_gb300 as gls
import synth
from gpu_util import assert_same, run_gpu

pytestmark = pytest.mark.gpu

X, Z = 2, 3


@pytest.fixture(scope="module", params=[("windowed", "dependency"), ("windowed", "levels"),
                                        ("wide", "dependency"), ("wide", "levels"),
                                        ("segmented", "dependency"), ("segmented", "levels")],
                ids=lambda p: f"{p[0]}-{p[1]}")
def ctx(request):
    c = gls.Context(0)
    c.set_kernel(request.param[0])
    c.set_schedule(request.param[1])
    yield c
    c.close()


def test_tiny200_three_seeds(ctx):
    for seed in (1, 2, 3):
        w = synth.make_workload("tiny200", seed=seed)
        ref = oracle.sim_event(w.netlist, w.stimulus)
        _, stats, off, t, v = run_gpu(ctx, w.netlist, w.stimulus)
        assert_same(ref, off, t, v, f"tiny200 seed {seed}")
        assert stats.total_events == int(ref.off[-1] - ref.off[w.netlist.n_pi])


def test_random_small_netlists(ctx):
    for seed in range(1, 61):
        rng = np.random.default_rng(1000 + seed)
        n_pi = int(rng.integers(1, 7))
        depth = int(rng.integers(1, 9))
        G = int(rng.integers(depth, 80))
        mask = int(rng.integers(1, synth.ALL_CELLS + 1))
        dmin = int(rng.integers(1, 40))
        nl = synth.make_netlist(n_pi, G, depth, fanout="geometric" if seed % 2 else "pareto",
                                d_min=dmin, d_max=dmin + int(rng.integers(0, 200)), cells=mask, seed=seed,
                                shuffle=bool(seed % 3 == 0))
        st = synth.make_stimulus(n_pi, mean=float(rng.integers(1, 600)), window=int(rng.integers(50, 20000)),
                                 probs=(0.4, 0.4, 0.12, 0.08), seed=seed)
        ref = oracle.sim_event(nl, st)
        _, _, off, t, v = run_gpu(ctx, nl, st)
        assert_same(ref, off, t, v, f"random case {seed}")


def test_long_waveforms_many_chunks(ctx):
    # waveforms far longer than one shared-memory window, including exact
    # multiples of the window and one-off sizes, dense (1-3 ps apart) and sparse
    for seed, (n_pi, mean, window) in enumerate([(3, 5000, 20000), (3, 128, 10**6), (4, 129, 10**6),
                                                 (2, 256, 300), (3, 20000, 10**7)]):
        nl = synth.make_netlist(n_pi, 60, 6, d_min=1, d_max=200, seed=seed + 7)
        st = synth.make_stimulus(n_pi, mean=mean, window=window, probs=(0.45, 0.45, 0.07, 0.03), seed=seed)
        ref = oracle.sim_levelized(nl, st, nthreads=4)
        _, _, off, t, v = run_gpu(ctx, nl, st)
        assert_same(ref, off, t, v, f"long case {seed}")


def _exact_lengths(n, lens, seed):
    rng = np.random.default_rng(seed)
    ts, vs, off = [], [], [0]
    for L in lens:
        t = np.sort(rng.choice(np.arange(0, 4 * L + 10), size=L, replace=False)).astype(np.int32)
        v, prev = [], X
        for _ in range(L):
            x = int(rng.choice([c for c in (0, 1, X, Z) if c != prev]))
            v.append(x)
            prev = x
        ts.append(t)
        vs.append(np.array(v, np.uint8))
        off.append(off[-1] + L)
    return synth.Stimulus(np.array(off, np.int64), np.concatenate(ts) if ts else np.zeros(0, np.int32),
                          np.concatenate(vs) if vs else np.zeros(0, np.uint8))


def test_window_boundary_lengths(ctx):
    # every cell on PI waveforms whose lengths straddle the per-pin window
    # sizes of both windowed variants (3-, 2- and 1-input cells: 128 / 192 /
    # 384 and 352 / 528 / 1056 transitions), other sizes, and the 32-lane split
    lens_sets = [[127, 128, 129], [1, 128, 256], [255, 256, 257], [31, 32, 33], [0, 129, 64], [0, 0, 5],
                 [63, 64, 65], [159, 160, 161], [191, 192, 193], [383, 384, 385], [527, 528, 529],
                 [1055, 1056, 1057], [161, 529, 1057], [351, 352, 353], [353, 705, 1057]]
    for cell in range(11):
        k = oracle.ARITY[cell]
        for li, lens in enumerate(lens_sets):
            from synth import Netlist
            rng = np.random.default_rng(cell * 10 + li)
            nl = Netlist(3, np.array([cell], np.uint8), np.array([0, k], np.int32),
                         np.array([0, 1, 2][:k], np.int32), rng.integers(1, 50, k).astype(np.int32),
                         rng.integers(1, 50, k).astype(np.int32))
            st = _exact_lengths(3, lens, seed=cell * 100 + li)
            ref = oracle.sim_event(nl, st)
            _, _, off, t, v = run_gpu(ctx, nl, st)
            assert_same(ref, off, t, v, f"cell {cell} lens {lens}")


def test_degenerate_inputs(ctx):
    from synth import Netlist
    nl = synth.make_netlist(4, 40, 5, seed=3)
    # no transitions at all: every waveform empty
    st = synth.Stimulus(np.zeros(5, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint8))
    _, stats, off, t, v = run_gpu(ctx, nl, st)
    assert stats.total_events == 0 and int(off[-1]) == 0
    # only X/Z on the inputs: gates stay X, no gate transitions
    st = synth.make_stimulus(4, mean=50, window=1000, probs=(0, 0, 0.5, 0.5), seed=2)
    ref = oracle.sim_event(nl, st)
    _, stats, off, t, v = run_gpu(ctx, nl, st)
    assert_same(ref, off, t, v, "xz only")
    # same net on every pin, and a chain reading one PI everywhere
    nl2 = Netlist(1, np.array([2, 6, 8, 9], np.uint8), np.array([0, 2, 4, 7, 10], np.int32),
                  np.array([0, 0, 1, 1, 0, 1, 2, 3, 3, 0], np.int32), np.arange(1, 11, dtype=np.int32),
                  np.arange(11, 1, -1, dtype=np.int32))
    st = synth.make_stimulus(1, mean=300, window=5000, seed=9)
    ref = oracle.sim_event(nl2, st)
    _, _, off, t, v = run_gpu(ctx, nl2, st)
    assert_same(ref, off, t, v, "shared nets")
    # a netlist of primary inputs only
    nl3 = Netlist(3, np.zeros(0, np.uint8), np.zeros(1, np.int32), np.zeros(0, np.int32),
                  np.zeros(0, np.int32), np.zeros(0, np.int32))
    st = synth.make_stimulus(3, mean=20, window=1000, seed=1)
    _, _, off, t, v = run_gpu(ctx, nl3, st)
    assert np.array_equal(off, st.off) and np.array_equal(t, st.t) and np.array_equal(v, st.v)


def test_max_delay_spread_and_dense_pulses(ctx):
    # delay spread at the device limit (255) with transitions 1 ps apart keeps
    # the most transitions pending between chunks
    nl = synth.make_netlist(6, 200, 8, d_min=1, d_max=1 + gls.gls.GLS_MAX_DELAY_SPREAD, seed=11)
    st = synth.make_stimulus(6, mean=3000, window=4000, probs=(0.45, 0.45, 0.05, 0.05), seed=11)
    ref = oracle.sim_levelized(nl, st, nthreads=4)
    _, _, off, t, v = run_gpu(ctx, nl, st)
    assert_same(ref, off, t, v, "max spread")


def test_mid_size_industrial_shape(ctx):
    # the 1M-gate recipe's shape (Pareto fanout, depth 60, delays 5-200,
    # 2000 transitions per input) at 20k gates
    w = synth.make_workload("ind1m", seed=4, net_n_pi=400, net_n_gates=20_000)
    ref = oracle.sim_levelized(w.netlist, w.stimulus, nthreads=8)
    _, stats, off, t, v = run_gpu(ctx, w.netlist, w.stimulus)
    assert_same(ref, off, t, v, "ind1m-shape 20k")


def test_rerun_and_update_stimulus(ctx):
    w = synth.make_workload("tiny200", seed=7)
    (nid, sid, rid), _, off, t, v = run_gpu(ctx, w.netlist, w.stimulus, keep=True)
    ctx.rerun(rid)
    ctx.run_stats(rid)
    off2, p2 = ctx.read_all(rid)
    t2, v2 = gls.unpack(p2)
    assert np.array_equal(off, off2) and np.array_equal(t, t2) and np.array_equal(v, v2)
    # new waveforms of the same shape, then rerun == oracle on the new stimulus
    st2 = synth.make_stimulus(16, mean=80, window=100_000, seed=99)
    assert st2.n_events <= w.stimulus.n_events
    ctx.update_stimulus(sid, st2.off, st2.t, st2.v)
    ctx.rerun(rid)
    ctx.run_stats(rid)
    off3, p3 = ctx.read_all(rid)
    t3, v3 = gls.unpack(p3)
    assert_same(oracle.sim_event(w.netlist, st2), off3, t3, v3, "after update")
    for i in (rid, sid, nid):
        ctx.release(i)


def test_read_waveform_matches_read_all(ctx):
    w = synth.make_workload("tiny200", seed=2)
    (nid, sid, rid), _, off, t, v = run_gpu(ctx, w.netlist, w.stimulus, keep=True)
    for net in (0, 5, 16, 17, 100, 215):
        tt, vv = ctx.read_waveform(rid, net)
        a, b = off[net], off[net + 1]
        assert np.array_equal(tt, t[a:b]) and np.array_equal(vv, v[a:b])


def test_error_paths(ctx):
    E = gls.gls
    w = synth.make_workload("tiny200", seed=1)
    nid = ctx.load_netlist(w.netlist)
    # malformed stimulus is caught on the device and reported as GLS_ESTIM
    bad_t = w.stimulus.t.copy()
    bad_t[5] = bad_t[4]
    with pytest.raises(gls.GlsError) as ei:
        ctx.load_stimulus(synth.Stimulus(w.stimulus.off, bad_t, w.stimulus.v))
    assert ei.value.code == E.GLS_ESTIM
    # times close to 2^30: simulate refuses with GLS_ERANGE
    shift = (1 << 30) - 302 - int(w.stimulus.t.max())
    late = synth.Stimulus(w.stimulus.off, (w.stimulus.t + shift).astype(np.int32), w.stimulus.v)
    sid = ctx.load_stimulus(late)
    with pytest.raises(gls.GlsError) as ei:
        ctx.simulate(nid, sid)
    assert ei.value.code == E.GLS_ERANGE
    # an arena that is too small: GLS_EOVERFLOW with the demand
    sid = ctx.load_stimulus(w.stimulus)
    rid = ctx.simulate(nid, sid, arena_events=64)
    rc, demand, _ = ctx.run_stats_raw(rid)
    assert rc == E.GLS_EOVERFLOW and demand > 64
    # the demand is a lower bound (skipped gates shrink later bounds): grow until it fits
    for _ in range(20):
        rid2 = ctx.simulate(nid, sid, arena_events=demand)
        rc, demand2, _ = ctx.run_stats_raw(rid2)
        if rc == E.GLS_OK:
            break
        assert rc == E.GLS_EOVERFLOW and demand2 > demand
        ctx.release(rid2)
        demand = demand2
    assert rc == E.GLS_OK
    # read_waveform with a short buffer
    import ctypes
    cnt = ctypes.c_int64(0)
    t = np.zeros(1, np.int32)
    v = np.zeros(1, np.uint8)
    net = int(np.argmax(np.diff(ctx.read_all(rid2)[0])))
    rc = E.gls_read_waveform(ctx.h, rid2, net, t.ctypes.data_as(ctypes.c_void_p), v.ctypes.data_as(ctypes.c_void_p),
                             1, ctypes.byref(cnt))
    assert rc == E.GLS_EOVERFLOW and cnt.value > 1
    # unknown ids and ids still in use
    with pytest.raises(gls.GlsError):
        ctx.simulate(12345, sid)
    with pytest.raises(gls.GlsError):
        ctx.release(nid)          # run still uses it


def test_bounded_wait_reports_timeout():
    # a gate that never signals completion: its readers give up after the
    # wait limit, the kernel finishes and the host reads GLS_ETIMEOUT
    E = gls.gls
    w = synth.make_workload("tiny200", seed=3)
    with gls.Context(0) as c:
        c.set_schedule("dependency")
        c.set_option(E.GLS_OPT_WAIT_LIMIT_MS, 50)
        c.set_option(E.GLS_OPT_TEST_WITHHOLD_GATE, 0)   # first gate of level 1 has readers
        nid = c.load_netlist(w.netlist)
        sid = c.load_stimulus(w.stimulus)
        rid = c.simulate(nid, sid)
        rc, _, _ = c.run_stats_raw(rid)
        assert rc == E.GLS_ETIMEOUT
        # the context stays usable: the same netlist without the hook is exact
        c.set_option(E.GLS_OPT_TEST_WITHHOLD_GATE, -1)
        rid = c.simulate(nid, sid)
        c.run_stats(rid)
        off, packed = c.read_all(rid)
        t, v = gls.unpack(packed)
        assert_same(oracle.sim_event(w.netlist, w.stimulus), off, t, v, "after timeout")
