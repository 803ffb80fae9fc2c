"""GPU test of gls_simulate_noalloc, the entry point that allocates no device
memory (for callers that cannot call cudaMalloc while they simulate, such as
code under CUDA-graph capture or inside a framework that owns all device
memory).  Its waveforms must equal those of the allocating gls_simulate, on
two calls in a row that share the statically allocated scratch.  This file is
collected last so that a stop at the first failure has run every other test;
it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import paper_2304_13398_gb300 as gls
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def device_order(nl):
    """caller net id -> device net id (PIs first, gates stable-sorted by level)"""
    _, level = gls.check_netlist(nl.n_pi, nl.type, nl.fanin_off, nl.fanin_net, nl.d_rise, nl.d_fall)
    order = np.argsort(level, kind="stable")
    ext2int = np.arange(nl.n_pi + nl.n_gates)
    ext2int[nl.n_pi + order] = nl.n_pi + np.arange(nl.n_gates)
    return ext2int


def vp(t):
    return ctypes.c_void_p(t.data_ptr())


def run_noalloc(ctx, nid, sid, n_nets, arena_words):
    net_ptr = torch.zeros(n_nets, dtype=torch.int64, device="cuda")
    net_len = torch.zeros(n_nets, dtype=torch.int32, device="cuda")
    arena = torch.zeros(arena_words, dtype=torch.int32, device="cuda")
    report = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = gls.gls.gls_simulate_noalloc(ctx.h, nid, sid, vp(net_ptr), vp(net_len), vp(arena), arena_words,
                                      vp(report), ctypes.c_void_p(stream.cuda_stream))
    assert rc == gls.gls.GLS_OK, ctx.lib.gls_last_error(ctx.h)
    torch.cuda.synchronize()
    return net_ptr.cpu().numpy(), net_len.cpu().numpy(), arena, report.cpu().numpy().view(np.uint32)


def check_against_simulate(ctx, w, arena_words, calls=2):
    nl, st = w.netlist, w.stimulus
    nid = ctx.load_netlist(nl)
    sid = ctx.load_stimulus(st)
    rid = ctx.simulate(nid, sid)
    ref_total = ctx.run_stats(rid).total_events
    off, packed = ctx.read_all(rid)
    ext2int = device_order(nl)
    N = nl.n_pi + nl.n_gates
    for call in range(calls):
        ptr, ln, arena, rep = run_noalloc(ctx, nid, sid, N, arena_words)
        assert rep[0] == 0, f"call {call}: status {rep[0]}"
        ln = ln.astype(np.int64)
        base = arena.data_ptr()
        host_arena = arena.cpu().numpy().view(np.uint32)
        assert int(ln[ext2int[nl.n_pi:]].sum()) == ref_total
        assert np.array_equal(ln[ext2int], np.diff(off))   # PI and gate lengths
        for g in range(nl.n_gates):
            i = ext2int[nl.n_pi + g]
            n = int(ln[i])
            want = packed[off[nl.n_pi + g]:off[nl.n_pi + g + 1]]
            if n == 0:
                assert len(want) == 0
                continue
            s0 = (int(ptr[i]) - base) // 4
            assert 0 <= s0 and s0 + n <= arena_words
            assert np.array_equal(host_arena[s0:s0 + n], want), f"call {call}, gate {g}"
    for i in (rid, sid, nid):
        ctx.release(i)


def test_noalloc_equals_simulate_two_calls():
    with gls.Context(0) as ctx:
        check_against_simulate(ctx, synth.make_workload("tiny200", seed=4), arena_words=1 << 20)
        check_against_simulate(ctx, synth.make_workload("ind1m", seed=2, net_n_pi=64, net_n_gates=3000),
                               arena_words=1 << 25)


def test_noalloc_limits():
    E = gls.gls
    with gls.Context(0) as ctx:
        # a chain deeper than the scratch holds is refused before any launch
        depth = E.GLS_NOALLOC_MAX_LEVELS + 1
        nl = synth.Netlist(1, np.ones(depth, np.uint8), np.arange(depth + 1, dtype=np.int32),
                           np.arange(depth, dtype=np.int32), np.ones(depth, np.int32), np.ones(depth, np.int32))
        nid = ctx.load_netlist(nl)
        sid = ctx.load_stimulus(synth.Stimulus(np.array([0, 2], np.int64), np.array([3, 9], np.int32),
                                               np.array([1, 0], np.uint8)))
        d = torch.zeros(depth + 1, dtype=torch.int64, device="cuda")
        rc = E.gls_simulate_noalloc(ctx.h, nid, sid, vp(d), vp(d), vp(d), 4096, vp(d), None)
        assert rc == E.GLS_ERANGE and b"levels" in ctx.lib.gls_last_error(ctx.h)
        # an arena that is too small is reported in the status word, not by a fault
        w = synth.make_workload("tiny200", seed=5)
        nid = ctx.load_netlist(w.netlist)
        sid = ctx.load_stimulus(w.stimulus)
        _, _, _, rep = run_noalloc(ctx, nid, sid, w.netlist.n_pi + w.netlist.n_gates, 128)
        assert rep[0] & 1 and (int(rep[1]) | (int(rep[2]) << 32)) > 64
