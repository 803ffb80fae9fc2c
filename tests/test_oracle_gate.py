"""Pins of the oracle's per-gate evaluation (Algorithm 2) and of the
pulse-filtering rule (Eq. 1).

- Fig. 5 worked example (minimum delay over simultaneously changed pins).
- Fig. 6 worked example (a later-determined, earlier-appearing transition
  denies the scheduled one; the replacement equals z's value, so z holds).
- Eq. 1 characterised without any list manipulation: the output value at
  time tau is the value of the most recently determined transition among
  those with t_r <= tau (a transition with t_r <= tau can only have been
  denied by a later-determined one with an even smaller t_r).  Checked by
  brute force over every short candidate sequence, for both the stack form
  and the suffix-minimum scan form.
- Algorithm 2's candidates against a time-stepped brute force (step every
  integer time, recompute the cell value, take the minimum delay over pins
  with a transition at that time).
- Closed form: a single 0->1->0 pulse of width w through BUF survives iff
  w > rise - fall.
"""
import itertools

import numpy as np

import oracle
from golden_io import waveform_cases

X, Z = 2, 3


def _gate_from_case(pins, names):
    return [([t for t, _ in pins.get(n, [])], [v for _, v in pins.get(n, [])]) for n in names]


def test_fig5_min_delay():
    for name, (pins, expect) in waveform_cases("fig5_min_delay.txt").items():
        ins = _gate_from_case(pins, "ab")
        t, v = oracle.eval_gate(oracle.AND2, ins, rise=[7, 9], fall=[5, 10])
        assert list(zip(t.tolist(), v.tolist())) == expect, name


def test_fig6_glitch_eaten():
    for name, (pins, expect) in waveform_cases("fig6_glitch_eaten.txt").items():
        ins = _gate_from_case(pins, "ab")
        t, v = oracle.eval_gate(oracle.AND2, ins, rise=[15, 12], fall=[8, 5])
        assert list(zip(t.tolist(), v.tolist())) == expect, name
    # the denied transition is really produced as a candidate first
    ins = _gate_from_case(waveform_cases("fig6_glitch_eaten.txt")["glitch_eaten"][0], "ab")
    td, tr, cv = oracle.gate_candidates(oracle.AND2, ins, rise=[15, 12], fall=[8, 5])
    assert list(zip(td.tolist(), tr.tolist(), cv.tolist())) == [(0, 5, 0), (5, 20, 1), (10, 15, 0)]


def _wave_from_value_function(tr, v, lo, hi):
    """Output waveform implied by 'z(tau) = value of the latest-determined
    transition with t_r <= tau' (X when there is none)."""
    out, prev = [], X
    for tau in range(lo, hi + 1):
        z = X
        for i in range(len(tr)):
            if tr[i] <= tau:
                z = v[i]          # later i overrides: most recently determined
        if z != prev:
            out.append((tau, z))
            prev = z
    return out


def test_eq1_bruteforce_all_short_sequences():
    n_checked = 0
    for n in range(0, 6):
        for trs in itertools.product(range(0, 5), repeat=n):
            for vs in itertools.product((0, 1, X), repeat=n):
                # candidates never repeat the previous cell value
                if any(vs[i] == vs[i - 1] for i in range(1, n)) or (n and vs[0] == X):
                    continue
                want = _wave_from_value_function(trs, vs, -1, 6)
                td = list(range(n))
                t1, v1 = oracle.cancel_stack(td, trs, vs)
                t2, v2 = oracle.cancel_scan(trs, vs)
                assert list(zip(t1.tolist(), v1.tolist())) == want, (trs, vs)
                assert list(zip(t2.tolist(), v2.tolist())) == want, (trs, vs)
                n_checked += 1
    assert n_checked > 5000


def _value_at(ts, vs, tau):
    z = X
    for t, v in zip(ts, vs):
        if t <= tau:
            z = v
    return z


def test_candidates_against_time_stepping():
    rng = np.random.default_rng(7)
    for trial in range(400):
        cell = int(rng.integers(0, 11))
        k = oracle.ARITY[cell]
        ins = []
        for p in range(k):
            n = int(rng.integers(0, 6))
            ts = sorted(rng.choice(np.arange(0, 12), size=n, replace=False).tolist())
            vs, prev = [], X
            for _ in ts:
                v = int(rng.choice([x for x in (0, 1, X, Z) if x != prev]))
                vs.append(v)
                prev = v
            ins.append((ts, vs))
        rise = rng.integers(1, 9, size=k).tolist()
        fall = rng.integers(1, 9, size=k).tolist()
        want, F = [], X
        for t in range(0, 13):
            cur = [_value_at(ts, vs, t) for ts, vs in ins]
            nF = oracle.cell_eval(cell, cur)
            if nF != F:
                ds = [(rise[p] if nF == 1 else fall[p] if nF == 0 else min(rise[p], fall[p]))
                      for p in range(k) if t in ins[p][0]]
                want.append((t, t + min(ds), nF))
            F = nF
        td, tr, cv = oracle.gate_candidates(cell, ins, rise, fall)
        assert list(zip(td.tolist(), tr.tolist(), cv.tolist())) == want, (cell, ins, rise, fall)


def test_single_pulse_through_buf():
    for rise in range(1, 12):
        for fall in range(1, 12):
            for w in range(1, 15):
                ins = [([0, 100, 100 + w], [0, 1, 0])]
                t, v = oracle.eval_gate(oracle.BUF, ins, [rise], [fall])
                got = list(zip(t.tolist(), v.tolist()))
                if w > rise - fall:
                    assert got == [(fall, 0), (100 + rise, 1), (100 + w + fall, 0)]
                else:
                    assert got == [(fall, 0)]


def test_x_start_and_no_event_gate():
    # Algorithm 2 starts every signal at X: a gate without input events has no output events
    t, v = oracle.eval_gate(oracle.NAND2, [([], []), ([], [])], [3, 3], [4, 4])
    assert len(t) == 0
    # a controlling value on one pin settles the output while the other stays X
    t, v = oracle.eval_gate(oracle.NAND2, [([10], [0]), ([], [])], [3, 3], [4, 4])
    assert list(zip(t.tolist(), v.tolist())) == [(13, 1)]
    # X <-> Z changes on an input do not change the cell value
    t, v = oracle.eval_gate(oracle.BUF, [([1, 2, 3, 4], [1, Z, X, 0])], [2], [5])
    assert list(zip(t.tolist(), v.tolist())) == [(3, 1), (4, X), (9, 0)]


def test_eq1_random_long_sequences():
    """Beyond the exhaustive short cases: long random candidate sequences
    (many ties, deep cancellation chains) give the same waveform in the
    stack form, the scan form and the value-function characterisation."""
    rng = np.random.default_rng(11)
    for trial in range(300):
        n = int(rng.integers(6, 60))
        trs = rng.integers(0, max(2, n // 2), size=n).tolist()
        vs, prev = [], X
        for _ in range(n):
            v = int(rng.choice([x for x in (0, 1, X) if x != prev]))
            vs.append(v)
            prev = v
        want = _wave_from_value_function(trs, vs, -1, max(trs) + 1)
        t1, v1 = oracle.cancel_stack(list(range(n)), trs, vs)
        t2, v2 = oracle.cancel_scan(trs, vs)
        assert list(zip(t1.tolist(), v1.tolist())) == want, (trs, vs)
        assert list(zip(t2.tolist(), v2.tolist())) == want, (trs, vs)
