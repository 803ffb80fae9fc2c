"""The seeded input generators produce the workloads their recipes state.

The synthetic inputs stand in for the paper's re-simulation benchmarks
(Sec. 5, Table 2), so their shape is part of what is measured.  Checked
here on the CPU: sizes and depth with every level present and one fanin
from the level below (the levelized structure Algorithm 1 schedules),
delay ranges, the cell mix, the heavy-tailed (Pareto) fanout of the
industrial recipe, Poisson transition counts, the value process (a value
is redrawn while it equals the previous one, a reversible Markov chain
whose stationary law is proportional to p_i (1 - p_i)), clock primary
inputs, and the 1M-gate benchmark's own figures for seed 1 (stimulus
transitions and the waveform-length CV of Eq. 5), so the numbers quoted
for it are reproducible.
"""
import numpy as np

import synth


def _fanin_levels(nl):
    lv = np.concatenate([np.zeros(nl.n_pi, np.int32), nl.level])
    gate = np.repeat(np.arange(nl.n_gates), np.diff(nl.fanin_off))
    return lv[nl.fanin_net], gate


def _check_levels(nl, depth):
    assert nl.level.min() == 1 and nl.level.max() == depth
    assert np.all(np.bincount(nl.level, minlength=depth + 1)[1:] > 0)   # every level non-empty
    src, gate = _fanin_levels(nl)
    assert np.all(src < nl.level[gate])                                # a DAG, in level order
    deepest = np.zeros(nl.n_gates, np.int32)
    np.maximum.at(deepest, gate, src)
    assert np.all(deepest == nl.level - 1)                             # one fanin from the level below


def test_tiny200_netlist():
    nl = synth.make_workload("tiny200", seed=1).netlist
    assert (nl.n_pi, nl.n_gates) == (16, 200)
    _check_levels(nl, 12)
    assert np.array_equal(np.diff(nl.fanin_off), synth.ARITY[nl.type])
    for d in (nl.d_rise, nl.d_fall):
        assert d.min() >= 5 and d.max() <= 50
    counts = np.bincount(nl.type, minlength=11)
    assert counts.min() >= 5 and counts.max() <= 40                    # uniform over the 11 cells


def test_poisson_counts_and_value_process():
    p = np.array([0.45, 0.45, 0.07, 0.03])
    st = synth.make_stimulus(4000, mean=100, window=100_000, probs=tuple(p), seed=3)
    c = np.diff(st.off)
    assert abs(c.mean() - 100) < 1.0
    assert 0.9 < c.var() / c.mean() < 1.1                              # Poisson: variance = mean
    for i in range(0, 4000, 97):
        t, v = st.t[st.off[i]:st.off[i + 1]], st.v[st.off[i]:st.off[i + 1]]
        assert np.all(np.diff(t) > 0) and t.min() >= 0 and t.max() < 100_000
        assert np.all(v[1:] != v[:-1])
        assert len(v) == 0 or v[0] != 2                                # the value before the first is X
    pi = p * (1 - p)
    pi /= pi.sum()
    freq = np.bincount(st.v, minlength=4) / len(st.v)
    assert np.max(np.abs(freq - pi)) < 0.005, (freq, pi)


def test_clock_inputs():
    st = synth.make_stimulus(200, mean=200, window=25_000_000, probs=(0.49, 0.49, 0.015, 0.005), seed=5,
                             n_clock=10, clock_period=1000, clock_trans=50_000)
    c = np.diff(st.off)
    clocks = np.nonzero(c == 50_000)[0]
    assert len(clocks) == 10
    for i in clocks:
        t, v = st.t[st.off[i]:st.off[i + 1]], st.v[st.off[i]:st.off[i + 1]]
        assert np.all(np.diff(t) == 500) and 0 <= t[0] < 1000      # half-period steps, phase in [0, period)
        assert set(v[:2].tolist()) == {0, 1} and np.all(v[2:] == v[:-2])
    others = np.delete(c, clocks)
    assert abs(others.mean() - 200) < 5


def test_ind1m_benchmark_figures():
    w = synth.make_workload("ind1m", seed=1)
    nl, st = w.netlist, w.stimulus
    assert (nl.n_pi, nl.n_gates) == (20_000, 1_000_000)
    _check_levels(nl, 60)
    for d in (nl.d_rise, nl.d_fall):
        assert d.min() >= 5 and d.max() <= 200
    # fanout: Pareto(alpha 2) quotas, P(F >= k) ~ k^-2 -- a tail a geometric law does not have
    fo = np.bincount(nl.fanin_net, minlength=nl.n_nets)
    assert 1.9 < fo.mean() < 2.2
    n = nl.n_nets
    assert 0.5 * n / 32 ** 2 < (fo >= 32).sum() < 2.0 * n / 32 ** 2
    assert 0.4 * n / 128 ** 2 < (fo >= 128).sum() < 2.5 * n / 128 ** 2
    # the figures quoted for the benchmark (seed 1)
    assert st.n_events == 39_994_919
    assert round(st.wcv(), 3) == 0.022
    c = np.diff(st.off)
    assert abs(c.mean() - 2000) < 5


def test_cell_library_option():
    """Shared cell library: tables come from a few prototypes and a pin
    without an arc (all four delays -1) never matters to its output's table;
    without the option every instance draws its own tables."""
    cn = synth.make_cell_netlist(8, 3000, 9, seed=8, library=16, noarc_frac=0.2)
    k = np.diff(cn.fanin_off)
    sets = {(int(k[c]), cn.luts[cn.lut_off[c]:cn.lut_off[c + 1]].tobytes()) for c in range(cn.n_cells)}
    assert len(sets) <= 3 * (16 + 16 * 16)
    for c in range(0, cn.n_cells, 7):
        kk, no = int(k[c]), int(cn.n_out[c])
        n4 = 4 ** kk
        for o in range(no):
            tab = cn.luts[cn.lut_off[c] + o * n4: cn.lut_off[c] + (o + 1) * n4]
            for p in range(kk):
                d = cn.delays[cn.delay_off[c] + (p * no + o) * 4: cn.delay_off[c] + (p * no + o) * 4 + 4]
                assert np.all(d == -1) or np.all(d >= 5)
                if np.all(d == -1):
                    idx = np.arange(n4)
                    assert np.array_equal(tab, tab[idx & ~(3 << (2 * p))])
    plain = synth.make_cell_netlist(8, 300, 6, seed=3)
    assert len({plain.luts[plain.lut_off[c]:plain.lut_off[c + 1]].tobytes() for c in range(plain.n_cells)}) > 250
