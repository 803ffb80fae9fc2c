"""Pins of the oracle's general cells: the full delay matrix (input-edge
dimension), several outputs per cell and user tables (Sec. 3 "Delay" and
"Module Function", Algorithm 2).  Each test ties the general code to
something other than itself: hand-written fixtures, or the already pinned
built-in-cell oracle."""
import numpy as np
import pytest

import oracle
import synth
from golden_io import SYM, _lines, waveform_cases

X, Z = 2, 3


def test_edge_classes_golden():
    seen = 0
    for ln in _lines("edge_classes.txt"):
        o, n, c = ln.split()
        assert oracle.edge_class(SYM[o], SYM[n]) == {"R": 0, "F": 1, "N": 2}[c], ln
        seen += 1
    assert seen == 12
    for v in range(4):
        assert oracle.edge_class(v, v) == -1


def test_arc_delay4_cases():
    D4 = [7, 9, 13, 11]      # index edge * 2 + value: rising to 0 = 7, to 1 = 9; falling to 0 = 13, to 1 = 11
    assert oracle.arc_delay4(D4, 0, 0) == 7
    assert oracle.arc_delay4(D4, 0, 1) == 9
    assert oracle.arc_delay4(D4, 1, 0) == 13
    assert oracle.arc_delay4(D4, 1, 1) == 11
    assert oracle.arc_delay4(D4, 0, X) == 7          # X: smaller of both values
    assert oracle.arc_delay4(D4, 2, 1) == 9          # neither edge: smaller of both edges
    assert oracle.arc_delay4(D4, 2, X) == 7
    assert oracle.arc_delay4([-1, -1, -1, -1], 0, 1) == oracle.INF


def _xor_table():
    t = np.zeros(16, np.uint8)
    for a in range(4):
        for b in range(4):
            t[a + 4 * b] = (a ^ b) if a < 2 and b < 2 else X
    return t


def _ins(pins, names):
    return [(np.array([t for t, _ in pins.get(n, [])], np.int64),
             np.array([v for _, v in pins.get(n, [])], np.uint8)) for n in names]


def test_edge_delay_golden():
    cases = waveform_cases("edge_delay_xor.txt")
    Dx = np.zeros((2, 2, 2), np.int64)   # [pin][edge][value]
    Dx[0, 0, 1], Dx[0, 0, 0], Dx[0, 1, 1], Dx[0, 1, 0] = 7, 9, 13, 11
    Dx[1, 0, 1], Dx[1, 0, 0], Dx[1, 1, 1], Dx[1, 1, 0] = 20, 22, 24, 26
    for name in ("edges", "pulse_eaten"):
        pins, want = cases[name]
        t, v = oracle.eval_cell_output(_xor_table(), Dx, _ins(pins, "ab"))
        assert list(zip(t.tolist(), v.tolist())) == want, name
    pins, want = cases["noarc"]
    tab = np.zeros(16, np.uint8)
    for a in range(4):
        for b in range(4):
            tab[a + 4 * b] = a if a < 2 else 0
    Dn = np.full((2, 2, 2), -1, np.int64)
    Dn[0, 0, 1], Dn[0, 0, 0], Dn[0, 1, 1], Dn[0, 1, 0] = 5, 6, 4, 8
    t, v = oracle.eval_cell_output(tab, Dn, _ins(pins, "ab"))
    assert list(zip(t.tolist(), v.tolist())) == want


def as_cells(nl):
    """A built-in-cell netlist as general cells: the oracle's own (pinned)
    tables, one output, rise/fall delays for both input edges."""
    C = nl.n_gates
    k = np.diff(nl.fanin_off).astype(np.int64)
    n_out = np.ones(C, np.int32)
    lut_off = np.zeros(C + 1, np.int64)
    np.cumsum(4 ** k, out=lut_off[1:])
    delay_off = np.zeros(C + 1, np.int64)
    np.cumsum(4 * k, out=delay_off[1:])
    luts = np.concatenate([oracle.cell_lut(int(t)) for t in nl.type]) if C else np.zeros(0, np.uint8)
    delays = np.zeros(int(delay_off[-1]), np.int32)
    for c in range(C):
        for p in range(int(k[c])):
            a = nl.fanin_off[c] + p
            for e in (0, 1):
                delays[delay_off[c] + (p * 2 + e) * 2 + 0] = nl.d_fall[a]
                delays[delay_off[c] + (p * 2 + e) * 2 + 1] = nl.d_rise[a]
    return synth.CellNetlist(nl.n_pi, n_out, nl.fanin_off.astype(np.int32), nl.fanin_net.astype(np.int32),
                             luts, lut_off, delays, delay_off)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_reduces_to_builtin_cells(seed):
    nl = synth.make_netlist(12, 500, 10, fanout="pareto", d_min=5, d_max=200, seed=seed, shuffle=seed == 2)
    st = synth.make_stimulus(12, mean=70, window=30_000, seed=seed + 10)
    ref = oracle.sim_event(nl, st)
    got = oracle.sim_cells(as_cells(nl), st)
    np.testing.assert_array_equal(got.off, ref.off)
    np.testing.assert_array_equal(got.t, ref.t)
    np.testing.assert_array_equal(got.v, ref.v)


def test_cell_candidates_equal_gate_candidates():
    rng = np.random.default_rng(5)
    for trial in range(200):
        cell = int(rng.integers(0, 11))
        k = oracle.ARITY[cell]
        ins = []
        for _ in range(k):
            n = int(rng.integers(0, 12))
            t = np.sort(rng.choice(60, n, replace=False)).astype(np.int64)
            v = np.zeros(n, np.uint8)
            prev = X
            for i in range(n):
                c = [x for x in range(4) if x != prev]
                v[i] = c[int(rng.integers(0, 3))]
                prev = v[i]
            ins.append((t, v))
        rise = rng.integers(1, 30, k)
        fall = rng.integers(1, 30, k)
        D = np.zeros((k, 2, 2), np.int64)
        D[:, :, 1] = rise[:, None]
        D[:, :, 0] = fall[:, None]
        a = oracle.gate_candidates(cell, ins, rise, fall)
        b = oracle.cell_candidates(oracle.cell_lut(cell), D, ins)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_outputs_are_independent():
    """A 2-output cell equals two 1-output cells with the same inputs,
    tables and delays (one waveform per output pin, Algorithm 2)."""
    cn = synth.make_cell_netlist(10, 600, 9, seed=8, multi_frac=0.6)
    st = synth.make_stimulus(10, mean=60, window=25_000, seed=9)
    ref = oracle.sim_cells(cn, st)
    # split: every output its own cell; net numbering is unchanged
    C = cn.n_cells
    n_out, fo, fn, luts, lut_off, dl, doff = [], [0], [], [], [0], [], [0]
    for c in range(C):
        k = cn.n_in(c)
        ins = cn.fanin_net[cn.fanin_off[c]:cn.fanin_off[c + 1]]
        for o in range(int(cn.n_out[c])):
            n_out.append(1)
            fn.extend(ins.tolist())
            fo.append(len(fn))
            tab = cn.luts[cn.lut_off[c] + o * 4 ** k: cn.lut_off[c] + (o + 1) * 4 ** k]
            luts.extend(tab.tolist())
            lut_off.append(len(luts))
            for p in range(k):
                at = cn.delay_off[c] + (p * int(cn.n_out[c]) + o) * 4
                dl.extend(cn.delays[at:at + 4].tolist())
            doff.append(len(dl))
    split = synth.CellNetlist(cn.n_pi, np.array(n_out, np.int32), np.array(fo, np.int32), np.array(fn, np.int32),
                              np.array(luts, np.uint8), np.array(lut_off, np.int64), np.array(dl, np.int32),
                              np.array(doff, np.int64))
    got = oracle.sim_cells(split, st)
    np.testing.assert_array_equal(got.off, ref.off)
    np.testing.assert_array_equal(got.t, ref.t)
    np.testing.assert_array_equal(got.v, ref.v)
    assert ref.off[-1] > 1000


def test_general_invariants():
    cn = synth.make_cell_netlist(10, 800, 10, seed=11)
    st = synth.make_stimulus(10, mean=80, window=25_000, seed=12)
    r = oracle.sim_cells(cn, st)
    for n in range(cn.n_pi, cn.n_nets):
        t, v = r.net(n)
        assert np.all(np.diff(t) > 0)
        assert np.all(v <= 2)
        if len(v):
            assert v[0] != X and np.all(v[1:] != v[:-1])


def test_cell_candidates_against_time_stepping():
    """Algorithm 2 for general cells against a time-stepped brute force on
    random user tables, edge-dependent delays and pins without arcs: at every
    integer time the pins with a transition there are applied together, the
    table gives the new value, and a change takes the smallest delay entry
    over those pins' arcs for their edge class (read from the hand-listed
    classes of tests/golden/edge_classes.txt; neither edge: both) toward the
    new value (X: both values), or the output's fastest arc toward it when
    none of them has an arc."""
    cls = {}
    for ln in _lines("edge_classes.txt"):
        o, n, c = ln.split()
        cls[(SYM[o], SYM[n])] = {"R": (0,), "F": (1,), "N": (0, 1)}[c]
    rng = np.random.default_rng(17)
    for trial in range(300):
        k = int(rng.integers(1, 4))
        n4 = 4 ** k
        lut = rng.integers(0, 3, n4).astype(np.uint8)
        D = rng.integers(1, 30, (k, 2, 2)).astype(np.int64)
        for p in range(1, k):
            if rng.random() < 0.3:
                D[p] = -1                                   # pin p has no arc
        ins = []
        for _ in range(k):
            n = int(rng.integers(0, 7))
            ts = np.sort(rng.choice(np.arange(0, 15), size=n, replace=False))
            vs, prev = [], X
            for _ in range(n):
                v = int(rng.choice([x for x in (0, 1, X, Z) if x != prev]))
                vs.append(v)
                prev = v
            ins.append((ts.astype(np.int64), np.array(vs, np.uint8)))
        vals = lambda F: (0, 1) if F == X else (F,)
        want, F, cur = [], X, [X] * k
        for t in range(0, 16):
            changed = {}
            for p, (ts, vs) in enumerate(ins):
                hit = np.nonzero(ts == t)[0]
                if len(hit):
                    changed[p] = cls[(cur[p], int(vs[hit[0]]))]
                    cur[p] = int(vs[hit[0]])
            if not changed:
                continue
            nF = int(lut[sum(v * 4 ** p for p, v in enumerate(cur))])
            if nF != F:
                ds = [D[p, e, v] for p, es in changed.items() for e in es for v in vals(nF) if D[p, e, v] > 0]
                if not ds:
                    ds = [D[p, e, v] for p in range(k) for e in (0, 1) for v in vals(nF) if D[p, e, v] > 0]
                want.append((t, t + min(ds), nF))
            F = nF
        td, tr, cv = oracle.cell_candidates(lut, D, ins)
        assert list(zip(td.tolist(), tr.tolist(), cv.tolist())) == want, (trial, lut, D, ins)
