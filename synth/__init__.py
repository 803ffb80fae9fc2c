"""Seeded synthetic netlists and primary-input stimuli.

This package draws inputs only; it holds none of the simulation arithmetic.
The CPU oracle (``oracle/``) and the CUDA path (``paper_2304_13398_gb300``)
both consume what it produces and neither depends on the other.

Workload shapes stand in for the paper's re-simulation benchmarks (Sec. 5,
Table 2: 10^4-10^6 cells, 10^7-10^8 given transitions, skewed waveform
lengths), which are not available here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")

CELLS = ["INV", "BUF", "AND2", "OR2", "NAND2", "NOR2", "XOR2", "XNOR2", "MUX2", "AOI21", "OAI21"]
ARITY = np.array([1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3], dtype=np.int32)
ALL_CELLS = (1 << len(CELLS)) - 1


def build(force: bool = False) -> str:
    """Compile libsynth.so in place (plain gcc, no GPU needed)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-o", _LIB + ".tmp", _SRC, "-lm"])
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.synth_netlist.restype = ctypes.c_int64
        lib.synth_netlist.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32,
                                      P, P, P, P, P, P]
        stim_args = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int64,
                     ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                     ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        lib.synth_stim_counts.restype = ctypes.c_int64
        lib.synth_stim_counts.argtypes = stim_args + [P]
        lib.synth_stim_fill.restype = ctypes.c_int
        lib.synth_stim_fill.argtypes = stim_args + [P, P, P]
        lib.synth_stim_fill64.restype = ctypes.c_int
        lib.synth_stim_fill64.argtypes = stim_args + [P, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Netlist:
    """Gate-level netlist.  Nets 0..n_pi-1 are primary inputs; net n_pi+g is
    the output of gate g.  Gate g reads nets fanin_net[fanin_off[g]:fanin_off[g+1]]
    (pin order a, b, c) with per-arc rise/fall delays in ps."""
    n_pi: int
    type: np.ndarray        # uint8[G]
    fanin_off: np.ndarray   # int32[G+1]
    fanin_net: np.ndarray   # int32[A]
    d_rise: np.ndarray      # int32[A]
    d_fall: np.ndarray      # int32[A]
    level: np.ndarray | None = None  # int32[G], generator's level (1..depth)

    @property
    def n_gates(self) -> int:
        return int(self.type.shape[0])

    @property
    def n_nets(self) -> int:
        return self.n_pi + self.n_gates


@dataclass
class Stimulus:
    """Given waveforms of the primary inputs: PI i owns transitions
    [off[i], off[i+1]) with strictly increasing times t and values v in
    {0, 1, 2=X, 3=Z}; before its first transition a PI is X."""
    off: np.ndarray   # int64[n_pi+1]
    t: np.ndarray     # int32[E]
    v: np.ndarray     # uint8[E]

    @property
    def n_events(self) -> int:
        return int(self.t.shape[0])

    def wcv(self) -> float:
        """Coefficient of variation of the given waveform lengths (Eq. 5)."""
        lens = np.diff(self.off).astype(np.float64)
        m = lens.mean()
        return float(lens.std() / m) if m > 0 else 0.0


def make_netlist(n_pi: int, n_gates: int, depth: int, *, fanout: str = "geometric",
                 pareto_alpha: float = 2.0, fanout_cap: int = 256, d_min: int = 5, d_max: int = 50,
                 cells: int = ALL_CELLS, seed: int = 1, shuffle: bool = False) -> Netlist:
    lib = _load()
    G = int(n_gates)
    typ = np.zeros(G, np.uint8)
    off = np.zeros(G + 1, np.int32)
    net = np.zeros(3 * G, np.int32)
    dr = np.zeros(3 * G, np.int32)
    df = np.zeros(3 * G, np.int32)
    lvl = np.zeros(G, np.int32)
    A = lib.synth_netlist(n_pi, G, depth, 0 if fanout == "geometric" else 1, pareto_alpha, fanout_cap,
                          d_min, d_max, cells, seed, 1 if shuffle else 0,
                          _p(typ), _p(off), _p(net), _p(dr), _p(df), _p(lvl))
    if A < 0:
        raise ValueError(f"synth_netlist failed ({A})")
    return Netlist(n_pi, typ, off, net[:A].copy(), dr[:A].copy(), df[:A].copy(), lvl)


def make_stimulus(n_pi: int, *, mean: float, window: int, probs=(0.45, 0.45, 0.07, 0.03), seed: int = 1,
                  n_clock: int = 0, clock_period: int = 1000, clock_trans: int = 0) -> Stimulus:
    lib = _load()
    args = (n_pi, seed, float(mean), int(window), *map(float, probs), n_clock, clock_period, clock_trans)
    counts = np.zeros(n_pi, np.int64)
    tot = lib.synth_stim_counts(*args, _p(counts))
    off = np.zeros(n_pi + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    v = np.zeros(tot, np.uint8)
    if window > 2**31 - 1 or n_clock and clock_period * clock_trans > 2**31 - 1:   # 64-bit times
        t = np.zeros(tot, np.int64)
        rc = lib.synth_stim_fill64(*args, _p(off), _p(t), _p(v))
    else:
        t = np.zeros(tot, np.int32)
        rc = lib.synth_stim_fill(*args, _p(off), _p(t), _p(v))
    if rc != 0:
        raise RuntimeError("synth_stim_fill mismatch")
    return Stimulus(off, t, v)


@dataclass
class CellNetlist:
    """Netlist of general cells: cell c reads nets fanin_net[fanin_off[c]:
    fanin_off[c+1]] (n_in = that count, 1..3) and drives n_out[c] nets.  Nets
    0..n_pi-1 are primary inputs, then the outputs of cell 0, cell 1, ... in
    order.  Output o of cell c has the 4-value table luts[lut_off[c] + o *
    4^n_in + sum v_p 4^p] (0, 1, 2 = X) and delays delays[delay_off[c] +
    ((p * n_out + o) * 2 + edge) * 2 + value] (edge 0 rising, 1 falling;
    value 0 = falling to 0, 1 = rising to 1; -1 = no arc from pin p)."""
    n_pi: int
    n_out: np.ndarray       # int32[C]
    fanin_off: np.ndarray   # int32[C+1]
    fanin_net: np.ndarray   # int32[A]
    luts: np.ndarray        # uint8
    lut_off: np.ndarray     # int64[C+1]
    delays: np.ndarray      # int32
    delay_off: np.ndarray   # int64[C+1]

    @property
    def n_cells(self) -> int:
        return int(self.n_out.shape[0])

    @property
    def n_nets(self) -> int:
        return int(self.n_pi + self.n_out.sum())

    def n_in(self, c: int) -> int:
        return int(self.fanin_off[c + 1] - self.fanin_off[c])


def make_cell_netlist(n_pi: int, n_cells: int, depth: int, *, seed: int = 1, multi_frac: float = 0.3,
                      edge_frac: float = 0.5, noarc_frac: float = 0.1, x_frac: float = 0.6, d_min: int = 5,
                      d_max: int = 200, fanout: str = "pareto", shuffle: bool = False,
                      library: int = 0) -> CellNetlist:
    """Seeded general-cell netlist on the structure of make_netlist: each cell
    has 1 or 2 outputs (multi_frac), user tables drawn at random (0/1 inputs
    give a random 0/1; inputs with X/Z give X with probability x_frac, else a
    random 0/1), delays uniform in [d_min, d_max] that depend on the input
    edge for a fraction edge_frac of the outputs, and, for a fraction
    noarc_frac of (pin, output) pairs of multi-input cells, no arc -- the
    output's table is then made independent of that pin.  About half of the
    reads of a 2-output cell use its second output.  With library > 0 the
    tables and the pins without an arc come from `library` prototype cells
    per input count and output (a cell library shared by many instances);
    the delays stay per instance."""
    base = make_netlist(n_pi, n_cells, depth, fanout=fanout, d_min=d_min, d_max=d_max, seed=seed, shuffle=shuffle)
    rng = np.random.default_rng(seed * 7919 + 17)
    C = base.n_gates
    k = np.diff(base.fanin_off).astype(np.int64)
    n_out = np.where(rng.random(C) < multi_frac, 2, 1).astype(np.int32)
    obase = np.zeros(C + 1, np.int64)
    obase[0] = n_pi
    np.cumsum(n_out, out=obase[1:])
    obase[1:] += n_pi
    # rewire reads: gate g's net -> one of cell g's outputs
    net = base.fanin_net.astype(np.int64)
    g = net - n_pi
    isg = g >= 0
    gg = np.where(isg, g, 0)
    second = isg & (n_out[gg] == 2) & (rng.random(len(net)) < 0.5)
    fanin_net = np.where(isg, obase[gg] + second, net).astype(np.int32)
    nl4 = 4 ** k
    lut_off = np.zeros(C + 1, np.int64)
    np.cumsum(n_out * nl4, out=lut_off[1:])
    delay_off = np.zeros(C + 1, np.int64)
    np.cumsum(k * n_out * 4, out=delay_off[1:])
    luts = np.zeros(int(lut_off[-1]), np.uint8)
    delays = np.zeros(int(delay_off[-1]), np.int32)
    for kk in (1, 2, 3):
        cells = np.nonzero(k == kk)[0]
        if len(cells) == 0:
            continue
        n4 = 4 ** kk
        idx = np.arange(n4)
        digits = np.stack([(idx >> (2 * p)) & 3 for p in range(kk)])          # [kk, n4]
        all01 = np.all(digits <= 1, axis=0)
        for o in (0, 1):
            cs = cells[n_out[cells] > o]
            if len(cs) == 0:
                continue
            if library > 0:
                T, D = _library_tables(rng, library, cs, kk, n4, idx, all01, x_frac, noarc_frac, edge_frac,
                                       d_min, d_max)
            else:
                T = rng.integers(0, 2, (len(cs), n4)).astype(np.uint8)
                xs = (rng.random((len(cs), n4)) < x_frac) & ~all01
                T[xs] = 2
                D = rng.integers(d_min, d_max + 1, (len(cs), kk, 2, 2)).astype(np.int32)
                same = rng.random(len(cs)) >= edge_frac
                D[same, :, 1, :] = D[same, :, 0, :]
            if kk > 1 and library == 0:
                noarc = rng.random((len(cs), kk)) < noarc_frac
                noarc[noarc.all(axis=1), 0] = False          # keep at least one arc
                for p in range(kk):
                    rows = np.nonzero(noarc[:, p])[0]
                    if len(rows) == 0:
                        continue
                    src = idx & ~(3 << (2 * p))                  # the same entry with pin p at 0
                    T[rows] = T[rows][:, src]
                    D[rows, p] = -1
            base_l = lut_off[cs] + o * n4
            luts[(base_l[:, None] + idx[None, :]).reshape(-1)] = T.reshape(-1)
            # delays[delay_off + ((p * n_out + o) * 2 + e) * 2 + v]
            for p in range(kk):
                for e in (0, 1):
                    for v in (0, 1):
                        at = delay_off[cs] + ((p * n_out[cs] + o) * 2 + e) * 2 + v
                        delays[at] = D[:, p, e, v]
    return CellNetlist(n_pi, n_out, base.fanin_off.astype(np.int32), fanin_net, luts, lut_off, delays, delay_off)


def _library_tables(rng, library, cs, kk, n4, idx, all01, x_frac, noarc_frac, edge_frac, d_min, d_max):
    """Tables of `library` prototypes (pins without an arc made irrelevant to
    the table), one drawn per cell, and per-instance delays with -1 for the
    prototype's pins without an arc."""
    T = rng.integers(0, 2, (library, n4)).astype(np.uint8)
    T[(rng.random((library, n4)) < x_frac) & ~all01] = 2
    noarc = np.zeros((library, kk), bool)
    if kk > 1:
        noarc = rng.random((library, kk)) < noarc_frac
        noarc[noarc.all(axis=1), 0] = False
        for p in range(kk):
            rows = np.nonzero(noarc[:, p])[0]
            if len(rows):
                T[rows] = T[rows][:, idx & ~(3 << (2 * p))]
    pick = rng.integers(0, library, len(cs))
    D = rng.integers(d_min, d_max + 1, (len(cs), kk, 2, 2)).astype(np.int32)
    same = rng.random(len(cs)) >= edge_frac
    D[same, :, 1, :] = D[same, :, 0, :]
    D[noarc[pick]] = -1
    return T[pick], D


@dataclass
class Workload:
    name: str
    netlist: Netlist
    stimulus: Stimulus
    recipe: dict = field(default_factory=dict)


# Workload recipes.  Each stands in for a class of the paper's benchmarks
# (Table 2) with the sizes of the target configurations.
RECIPES = {
    "tiny200": dict(net=dict(n_pi=16, n_gates=200, depth=12, fanout="geometric", d_min=5, d_max=50),
                    stim=dict(mean=100, window=100_000, probs=(0.45, 0.45, 0.07, 0.03))),
    "ind1m": dict(net=dict(n_pi=20_000, n_gates=1_000_000, depth=60, fanout="pareto", pareto_alpha=2.0,
                           fanout_cap=256, d_min=5, d_max=200),
                  stim=dict(mean=2000, window=10_000_000, probs=(0.48, 0.48, 0.03, 0.01))),
    "skew10m": dict(net=dict(n_pi=100_000, n_gates=10_000_000, depth=120, fanout="pareto", pareto_alpha=2.0,
                             fanout_cap=256, d_min=5, d_max=200),
                    stim=dict(mean=200, window=25_000_000, probs=(0.49, 0.49, 0.015, 0.005),
                              n_clock=1000, clock_period=1000, clock_trans=50_000)),
}


def make_workload(name: str, seed: int = 1, **overrides) -> Workload:
    """Build a named recipe; keyword overrides go to the netlist ('net_*') or
    the stimulus ('stim_*') part, e.g. stim_window=10**5 for a shorter run."""
    r = RECIPES[name]
    net = dict(r["net"])
    stim = dict(r["stim"])
    for k, v in overrides.items():
        if k.startswith("net_"):
            net[k[4:]] = v
        elif k.startswith("stim_"):
            stim[k[5:]] = v
        else:
            raise KeyError(k)
    nl = make_netlist(seed=seed, **net)
    st = make_stimulus(net["n_pi"], seed=seed + 1000003, **stim)
    return Workload(name, nl, st, dict(net=net, stim=stim, seed=seed))
