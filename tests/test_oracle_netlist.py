"""Whole-netlist pins of the oracle.

- The global event-driven simulator and the levelized Algorithm 2 evaluator
  are independent code and must agree exactly (processing order is
  irrelevant for a DAG, Sec. 4.1).
- Settle values: the last value of every waveform equals a static 4-value
  evaluation with the final primary-input values.
- Invariants: strictly increasing times, no repeated consecutive values, the
  first value is never X, and Eq. 2: |out| <= distinct fanin timestamps
  <= sum of fanin lengths.
- Closed form: a chain of BUF/INV cells with rise = fall = d shifts the
  input by k*d, reads Z as X, inverts for odd INV count and drops repeats.
- A cyclic netlist is rejected.
"""
import numpy as np
import pytest

import oracle
import synth

X, Z = 2, 3


def small_cases():
    cases = []
    for seed in range(1, 41):
        rng = np.random.default_rng(seed)
        n_pi = int(rng.integers(1, 6))
        depth = int(rng.integers(1, 7))
        G = int(rng.integers(depth, 40))
        mask = int(rng.integers(1, synth.ALL_CELLS + 1))
        nl = synth.make_netlist(n_pi, G, depth, fanout="geometric" if seed % 2 else "pareto",
                                d_min=1, d_max=int(rng.integers(1, 30)), cells=mask, seed=seed,
                                shuffle=bool(seed % 3 == 0))
        st = synth.make_stimulus(n_pi, mean=float(rng.integers(1, 40)), window=int(rng.integers(20, 400)),
                                 probs=(0.4, 0.4, 0.1, 0.1), seed=seed)
        cases.append((nl, st))
    return cases


def test_event_driven_equals_levelized():
    for nl, st in small_cases() + [(w.netlist, w.stimulus) for w in [synth.make_workload("tiny200", seed=s) for s in (1, 2, 3)]]:
        a = oracle.sim_event(nl, st)
        b = oracle.sim_levelized(nl, st, nthreads=2)
        assert np.array_equal(a.off, b.off)
        assert np.array_equal(a.t, b.t)
        assert np.array_equal(a.v, b.v)


def test_settle_values_equal_static_eval():
    for nl, st in small_cases():
        r = oracle.sim_levelized(nl, st)
        lens = np.diff(st.off)
        pi_final = np.where(lens > 0, st.v[np.maximum(st.off[1:] - 1, 0)], X).astype(np.uint8)
        want = oracle.static_eval(nl, pi_final)
        lens_r = np.diff(r.off)
        got = np.where(lens_r > 0, r.v[np.maximum(r.off[1:] - 1, 0)], X)
        assert np.array_equal(got, want)


def test_invariants_and_eq2_bound():
    for nl, st in small_cases():
        r = oracle.sim_levelized(nl, st)
        for n in range(nl.n_nets):
            t, v = r.net(n)
            assert np.all(np.diff(t) > 0)
            assert np.all(v[1:] != v[:-1])
            if n >= nl.n_pi and len(v):
                assert v[0] != X
                assert np.all(v != Z)
        for g in range(nl.n_gates):
            fins = nl.fanin_net[nl.fanin_off[g]:nl.fanin_off[g + 1]]
            ts = [r.net(int(f))[0] for f in fins]
            distinct = len(np.unique(np.concatenate(ts))) if ts else 0
            out = len(r.net(nl.n_pi + g)[0])
            assert out <= distinct <= sum(len(t) for t in ts)


def _chain(cells, d):
    from synth import Netlist
    G = len(cells)
    typ = np.array(cells, np.uint8)
    off = np.arange(G + 1, dtype=np.int32)
    net = np.arange(G, dtype=np.int32)     # gate g reads net g (PI 0, then gate g-1)
    dd = np.full(G, d, np.int32)
    return Netlist(1, typ, off, net, dd, dd.copy())


def test_buf_inv_chain_closed_form():
    rng = np.random.default_rng(3)
    for trial in range(50):
        cells = rng.choice([oracle.INV, oracle.BUF], size=int(rng.integers(1, 8))).tolist()
        d = int(rng.integers(1, 20))
        nl = _chain(cells, d)
        n = int(rng.integers(0, 30))
        ts = np.sort(rng.choice(np.arange(0, 500), size=n, replace=False)).astype(np.int32)
        vs, prev = [], X
        for _ in range(n):
            v = int(rng.choice([x for x in (0, 1, X, Z) if x != prev]))
            vs.append(v)
            prev = v
        st = synth.Stimulus(np.array([0, n], np.int64), ts, np.array(vs, np.uint8))
        r = oracle.sim_levelized(nl, st)
        k = len(cells)
        inv = sum(c == oracle.INV for c in cells) % 2
        want, prev = [], X
        for t, v in zip(ts.tolist(), vs):
            v = X if v == Z else v
            if inv and v != X:
                v = 1 - v
            if v != prev:
                want.append((t + k * d, v))
                prev = v
        t, v = r.net(k)
        assert list(zip(t.tolist(), v.tolist())) == want


def test_cycle_rejected():
    from synth import Netlist
    # gate 0 reads gate 1, gate 1 reads gate 0
    nl = Netlist(1, np.array([oracle.AND2, oracle.BUF], np.uint8), np.array([0, 2, 3], np.int32),
                 np.array([0, 2, 1], np.int32), np.ones(3, np.int32), np.ones(3, np.int32))
    st = synth.Stimulus(np.array([0, 1], np.int64), np.array([5], np.int32), np.array([1], np.uint8))
    with pytest.raises(oracle.OracleError):
        oracle.sim_levelized(nl, st)
    with pytest.raises(oracle.OracleError):
        oracle.sim_event(nl, st)


def test_check_gates_detects_planted_mistakes():
    w = synth.make_workload("tiny200", seed=5)
    nl, st = w.netlist, w.stimulus
    r = oracle.sim_levelized(nl, st)
    t32 = r.t.astype(np.int32)
    assert oracle.check_gates(nl, r.off, t32, r.v) == (0, -1)
    # shift one output transition of a gate with events: exactly that gate (and
    # its readers) stop matching
    lens = np.diff(r.off)
    g = int(np.nonzero(lens[nl.n_pi:] > 2)[0][0])
    e = int(r.off[nl.n_pi + g] + 1)
    t_bad = t32.copy()
    t_bad[e] += 1 if t_bad[e] + 1 < t_bad[e + 1] else 0
    v_bad = r.v.copy()
    v_bad[e] = 1 - v_bad[e] if v_bad[e] in (0, 1) else 0
    bad, first = oracle.check_gates(nl, r.off, t_bad, v_bad)
    assert bad >= 1 and first <= g


def test_time_translation_beyond_32_bits():
    """The method depends on time differences only (every net is X before its
    first transition, delays add to event times, Eq. 1 compares times), so
    shifting the whole stimulus by D shifts every waveform by D.  With D past
    2^32 this pins the oracle's 64-bit time path, which the long-duration
    (time-sliced) runs are checked against."""
    nl = synth.make_netlist(10, 300, 9, fanout="pareto", d_min=5, d_max=200, seed=13)
    st = synth.make_stimulus(10, mean=60, window=30_000, seed=14)
    D = 3 * (1 << 31) + 12345
    st64 = synth.Stimulus(st.off.copy(), st.t.astype(np.int64) + D, st.v.copy())
    for sim in (oracle.sim_event, lambda a, b: oracle.sim_levelized(a, b, nthreads=2)):
        base, far = sim(nl, st), sim(nl, st64)
        np.testing.assert_array_equal(base.off, far.off)
        np.testing.assert_array_equal(base.t + D, far.t)
        np.testing.assert_array_equal(base.v, far.v)
    assert oracle.check_gates(nl, far.off, far.t, far.v) == (0, -1)


def test_same_net_on_both_pins_closed_forms():
    """One net on both pins of a cell: both pins change at the same time, so
    the delay is the smaller of the two arcs (Sec. 2.3, all changed pins),
    and each pin's X is completed on its own (Sec. 2.2).  AND2(a, a) is then
    a with Z read as X, shifted by min(d0, d1); XOR2(a, a) is 0 while a is
    0 or 1 and X while it is X or Z, shifted by the arc delay."""
    from synth import Netlist
    rng = np.random.default_rng(21)
    for trial in range(60):
        d0, d1, dx = (int(x) for x in rng.integers(1, 25, size=3))
        typ = np.array([oracle.AND2, oracle.XOR2], np.uint8)
        off = np.array([0, 2, 4], np.int32)
        net = np.zeros(4, np.int32)                       # every pin reads PI 0
        dly = np.array([d0, d1, dx, dx], np.int32)
        nl = Netlist(1, typ, off, net, dly, dly.copy())
        n = int(rng.integers(0, 25))
        ts = np.sort(rng.choice(np.arange(0, 400), size=n, replace=False)).astype(np.int32)
        vs, prev = [], X
        for _ in range(n):
            v = int(rng.choice([x for x in (0, 1, X, Z) if x != prev]))
            vs.append(v)
            prev = v
        st = synth.Stimulus(np.array([0, n], np.int64), ts, np.array(vs, np.uint8))

        def shifted(f, d):
            out, last = [], X
            for t, v in zip(ts.tolist(), vs):
                y = f(v)
                if y != last:
                    out.append((t + d, y))
                    last = y
            return out

        want_and = shifted(lambda v: X if v == Z else v, min(d0, d1))
        want_xor = shifted(lambda v: 0 if v in (0, 1) else X, dx)
        for sim in (oracle.sim_event, oracle.sim_levelized):
            r = sim(nl, st)
            for g, want in ((0, want_and), (1, want_xor)):
                t, v = r.net(1 + g)
                assert list(zip(t.tolist(), v.tolist())) == want, (g, ts, vs, d0, d1, dx)


def test_event_driven_equals_levelized_fuzz():
    """The two independent simulators on many tiny random netlists with
    extreme settings: unit or wide delay ranges, dense pulses, X/Z-heavy
    stimuli, single cell types and shuffled gate numbering."""
    rng = np.random.default_rng(2024)
    for trial in range(400):
        n_pi = int(rng.integers(1, 4))
        depth = int(rng.integers(1, 5))
        G = int(rng.integers(depth, 12))
        d_min = int(rng.integers(1, 4))
        d_max = d_min + int(rng.choice([0, 1, 3, 40]))
        cells = int(rng.choice([synth.ALL_CELLS, 1 << int(rng.integers(0, 11)), int(rng.integers(1, synth.ALL_CELLS + 1))]))
        nl = synth.make_netlist(n_pi, G, depth, fanout="geometric" if trial % 2 else "pareto", d_min=d_min,
                                d_max=d_max, cells=cells, seed=1000 + trial, shuffle=bool(trial % 3 == 0))
        probs = [(0.45, 0.45, 0.07, 0.03), (0.25, 0.25, 0.25, 0.25), (0.5, 0.5, 0.0, 0.0)][trial % 3]
        st = synth.make_stimulus(n_pi, mean=float(rng.integers(1, 30)), window=int(rng.integers(5, 80)),
                                 probs=probs, seed=2000 + trial)
        a = oracle.sim_event(nl, st)
        b = oracle.sim_levelized(nl, st)
        assert np.array_equal(a.off, b.off) and np.array_equal(a.t, b.t) and np.array_equal(a.v, b.v), trial
