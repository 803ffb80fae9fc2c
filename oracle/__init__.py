"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow reference implementation of timing-aware 4-value gate-level
re-simulation (arXiv 2304.13398, Sec. 2, Eq. 1, Algorithm 2), written in C
(``oracle.c``) and loaded here through ctypes.  Only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this package.  It shares no code with the CUDA library and imports nothing
from it; inputs come from the separate ``synth`` generators or from hand
fixtures.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  cell_eval / cell_lut   Table 1 (AND/OR/XOR) golden fixture; brute-force
                         completion semantics of every cell written in the
                         test; read-once composition of Table 1 gates.
  gate_candidates        Fig. 5 worked example (minimum delay); hand traces.
  cancel_stack           Fig. 6 worked example; brute-force enumeration of
                         Eq. 1 over all short candidate sequences.
  cancel_scan            equal to cancel_stack on every short sequence.
  sim_levelized          equals sim_event (independent code) on seeded
                         random netlists; settle values equal static_eval;
                         BUF/INV chain closed forms; waveform invariants and
                         the Eq. 2 bound; translation of the stimulus by more
                         than 2^32 ps translates every waveform (times are
                         64-bit throughout).
  sim_event              same pins as sim_levelized.
  static_eval            hand-computed settle values of small circuits.
  edge_class             the Verilog posedge/negedge classes, listed by hand
                         (tests/golden/edge_classes.txt).
  cell_candidates /      with edge-independent delays and built-in tables,
  sim_cells              equal to gate_candidates / sim_event (pinned above)
                         on random netlists; several outputs equal separate
                         single-output cells; hand-worked edge-dependent XOR
                         example (tests/golden/edge_delay_xor.txt); a no-arc
                         entry never wins the minimum.
The strength of these pins is itself tested: single mistakes planted in
copies of oracle.c each fail at least one of them
(tests/test_oracle_mutants.py).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

X, Z = 2, 3
INV, BUF, AND2, OR2, NAND2, NOR2, XOR2, XNOR2, MUX2, AOI21, OAI21 = range(11)
ARITY = [1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3]


def build(force: bool = False) -> str:
    """Compile liboracle.so in place with gcc (OpenMP for the level-parallel
    evaluator and the per-gate checker)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", _LIB + ".tmp", _SRC])
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None
P = ctypes.c_void_p


def _bind(lib):
    """Declare the C signatures on a loaded liboracle."""
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    lib.oracle_arity.restype = ctypes.c_int
    lib.oracle_arity.argtypes = [ctypes.c_int]
    lib.oracle_cell_bool.restype = ctypes.c_int
    lib.oracle_cell_bool.argtypes = [ctypes.c_int] * 4
    lib.oracle_cell_eval.restype = ctypes.c_int
    lib.oracle_cell_eval.argtypes = [ctypes.c_int, P]
    lib.oracle_cell_lut.restype = None
    lib.oracle_cell_lut.argtypes = [ctypes.c_int, P]
    lib.oracle_delay.restype = i64
    lib.oracle_delay.argtypes = [i64, i64, ctypes.c_int]
    lib.oracle_gate_candidates.restype = i64
    lib.oracle_gate_candidates.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, P]
    lib.oracle_cancel_stack.restype = i64
    lib.oracle_cancel_stack.argtypes = [i64, P, P, P, P, P]
    lib.oracle_cancel_scan.restype = i64
    lib.oracle_cancel_scan.argtypes = [i64, P, P, P, P]
    lib.oracle_eval_gate.restype = i64
    lib.oracle_eval_gate.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, P, P, P]
    lib.oracle_result_nevents.restype = i64
    lib.oracle_result_nevents.argtypes = [P]
    lib.oracle_result_nnets.restype = i64
    lib.oracle_result_nnets.argtypes = [P]
    lib.oracle_result_copy.restype = None
    lib.oracle_result_copy.argtypes = [P, P, P, P]
    lib.oracle_result_free.restype = None
    lib.oracle_result_free.argtypes = [P]
    net_args = [i32, i32, P, P, P, P, P]
    lib.oracle_sim_levelized.restype = ctypes.c_int
    lib.oracle_sim_levelized.argtypes = net_args + [P, P, P, ctypes.c_int, ctypes.POINTER(P)]
    lib.oracle_sim_event.restype = ctypes.c_int
    lib.oracle_sim_event.argtypes = net_args + [P, P, P, ctypes.POINTER(P)]
    lib.oracle_static_eval.restype = ctypes.c_int
    lib.oracle_static_eval.argtypes = [i32, i32, P, P, P, P, P]
    lib.oracle_check_gates.restype = i64
    lib.oracle_check_gates.argtypes = net_args + [P, P, P, i32, i32, ctypes.c_int, ctypes.POINTER(i64)]
    lib.oracle_edge_class.restype = ctypes.c_int
    lib.oracle_edge_class.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.oracle_arc_delay4.restype = i64
    lib.oracle_arc_delay4.argtypes = [P, ctypes.c_int, ctypes.c_int]
    lib.oracle_cell_candidates.restype = i64
    lib.oracle_cell_candidates.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, P]
    lib.oracle_sim_cells.restype = ctypes.c_int
    lib.oracle_sim_cells.argtypes = [i32, i32, P, P, P, P, P, P, P, P, P, P, ctypes.POINTER(P)]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def library(path: str):
    """Run the oracle's functions on another build of oracle.c (a copy with a
    planted mistake, in the tests that check the pins catch it) for the
    duration of the block."""
    global _lib
    prev = _lib
    _lib = _bind(ctypes.CDLL(os.path.abspath(path)))
    try:
        yield
    finally:
        _lib = prev


def _p(a: np.ndarray):
    return a.ctypes.data_as(P)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


@dataclass
class Result:
    """Waveforms of every net as a CSR: net n owns [off[n], off[n+1])."""
    off: np.ndarray  # int64[N+1]
    t: np.ndarray    # int64[E]
    v: np.ndarray    # uint8[E]

    def net(self, n: int):
        a, b = int(self.off[n]), int(self.off[n + 1])
        return self.t[a:b], self.v[a:b]

    @property
    def n_events(self) -> int:
        return int(self.t.shape[0])


def cell_eval(cell: int, inputs) -> int:
    a = _c(list(inputs) + [X] * (3 - len(inputs)), np.uint8)
    return _load().oracle_cell_eval(cell, _p(a))


def cell_bool(cell: int, a: int, b: int = 0, c: int = 0) -> int:
    return _load().oracle_cell_bool(cell, a, b, c)


def cell_lut(cell: int) -> np.ndarray:
    """4^k table, index sum(in[p] * 4**p)."""
    out = np.zeros(4 ** ARITY[cell], np.uint8)
    _load().oracle_cell_lut(cell, _p(out))
    return out


def delay(rise: int, fall: int, v: int) -> int:
    return _load().oracle_delay(rise, fall, v)


def _pin_arrays(ins):
    ts = [_c(t, np.int64) for t, _ in ins]
    vs = [_c(v, np.uint8) for _, v in ins]
    while len(ts) < 3:
        ts.append(np.zeros(0, np.int64))
        vs.append(np.zeros(0, np.uint8))
    tp = (P * 3)(*[_p(t) for t in ts])
    vp = (P * 3)(*[_p(v) for v in vs])
    n = _c([len(t) for t in ts], np.int64)
    return ts, vs, tp, vp, n


def gate_candidates(cell: int, ins, rise, fall):
    """Algorithm 2 candidates: ins = [(t, v), ...] per pin.  Returns (t_d, t_r, v)."""
    ts, vs, tp, vp, n = _pin_arrays(ins)
    r = _c(list(rise) + [1] * (3 - len(rise)), np.int64)
    f = _c(list(fall) + [1] * (3 - len(fall)), np.int64)
    cap = int(n.sum()) + 1
    td, tr, cv = np.zeros(cap, np.int64), np.zeros(cap, np.int64), np.zeros(cap, np.uint8)
    m = _load().oracle_gate_candidates(cell, ctypes.cast(tp, P), ctypes.cast(vp, P), _p(n), _p(r), _p(f),
                                       _p(td), _p(tr), _p(cv))
    return td[:m], tr[:m], cv[:m]


def cancel_stack(td, tr, v):
    td, tr, v = _c(td, np.int64), _c(tr, np.int64), _c(v, np.uint8)
    ot, ov = np.zeros(len(tr) + 1, np.int64), np.zeros(len(tr) + 1, np.uint8)
    m = _load().oracle_cancel_stack(len(tr), _p(td), _p(tr), _p(v), _p(ot), _p(ov))
    return ot[:m], ov[:m]


def cancel_scan(tr, v):
    tr, v = _c(tr, np.int64), _c(v, np.uint8)
    ot, ov = np.zeros(len(tr) + 1, np.int64), np.zeros(len(tr) + 1, np.uint8)
    m = _load().oracle_cancel_scan(len(tr), _p(tr), _p(v), _p(ot), _p(ov))
    return ot[:m], ov[:m]


def eval_gate(cell: int, ins, rise, fall):
    """One gate's output waveform (Algorithm 2 + Eq. 1)."""
    td, tr, cv = gate_candidates(cell, ins, rise, fall)
    return cancel_stack(td, tr, cv)


def _net(nl):
    return (int(nl.n_pi), int(len(nl.type)), _c(nl.type, np.uint8), _c(nl.fanin_off, np.int32),
            _c(nl.fanin_net, np.int32), _c(nl.d_rise, np.int32), _c(nl.d_fall, np.int32))


def _result(h) -> Result:
    lib = _load()
    N, E = lib.oracle_result_nnets(h), lib.oracle_result_nevents(h)
    off, t, v = np.zeros(N + 1, np.int64), np.zeros(E, np.int64), np.zeros(E, np.uint8)
    lib.oracle_result_copy(h, _p(off), _p(t), _p(v))
    lib.oracle_result_free(h)
    return Result(off, t, v)


class OracleError(RuntimeError):
    pass


# ---- cells with the full delay matrix, several outputs, user tables ----
EDGE_RISE, EDGE_FALL, EDGE_NONE = 0, 1, 2
INF = np.iinfo(np.int64).max


def edge_class(old: int, new: int) -> int:
    """0 rising, 1 falling, 2 neither (X<->Z), -1 no change."""
    return _load().oracle_edge_class(old, new)


def arc_delay4(D4, edge: int, v: int) -> int:
    """Delay of one pin's transition of class `edge` toward output value v;
    D4[edge * 2 + value], -1 = no arc; INF when no arc applies."""
    d = _c(D4, np.int64)
    return _load().oracle_arc_delay4(_p(d), edge, v)


def cell_candidates(lut, D, ins):
    """Algorithm 2 candidates of one cell output: lut = 4^n_in table, D =
    [n_in][edge][value] delays (-1 = no arc), ins = [(t, v), ...]."""
    n_in = len(ins)
    ts, vs, tp, vp, n = _pin_arrays(ins)
    lut = _c(lut, np.uint8)
    D = _c(np.asarray(D).reshape(-1), np.int64)
    cap = int(n.sum()) + 1
    td, tr, cv = np.zeros(cap, np.int64), np.zeros(cap, np.int64), np.zeros(cap, np.uint8)
    m = _load().oracle_cell_candidates(n_in, _p(lut), _p(D), ctypes.cast(tp, P), ctypes.cast(vp, P), _p(n),
                                       _p(td), _p(tr), _p(cv))
    if m < 0:
        raise OracleError("an output without any arc")
    return td[:m], tr[:m], cv[:m]


def eval_cell_output(lut, D, ins):
    """One output waveform of a general cell (Algorithm 2 + Eq. 1)."""
    td, tr, cv = cell_candidates(lut, D, ins)
    return cancel_stack(td, tr, cv)


def sim_cells(cn, st) -> Result:
    """Whole netlist of general cells (synth.CellNetlist): nets are the PIs
    then every cell's outputs in cell order."""
    so, stt, sv = _c(st.off, np.int64), _c(st.t, np.int64), _c(st.v, np.uint8)
    h = P()
    rc = _load().oracle_sim_cells(int(cn.n_pi), len(cn.n_out), _p(_c(cn.n_out, np.int32)), _p(_c(cn.luts, np.uint8)),
                                  _p(_c(cn.lut_off, np.int64)), _p(_c(cn.fanin_off, np.int32)),
                                  _p(_c(cn.fanin_net, np.int32)), _p(_c(cn.delays, np.int64)),
                                  _p(_c(cn.delay_off, np.int64)), _p(so), _p(stt), _p(sv), ctypes.byref(h))
    if rc:
        raise OracleError(f"oracle_sim_cells: {rc}")
    return _result(h)


def sim_levelized(nl, st, nthreads: int = 1) -> Result:
    n_pi, G, typ, fo, fn, dr, df = _net(nl)
    so, stt, sv = _c(st.off, np.int64), _c(st.t, np.int64), _c(st.v, np.uint8)
    h = P()
    rc = _load().oracle_sim_levelized(n_pi, G, _p(typ), _p(fo), _p(fn), _p(dr), _p(df),
                                      _p(so), _p(stt), _p(sv), nthreads, ctypes.byref(h))
    if rc:
        raise OracleError(f"oracle_sim_levelized: {rc}")
    return _result(h)


def sim_event(nl, st) -> Result:
    n_pi, G, typ, fo, fn, dr, df = _net(nl)
    so, stt, sv = _c(st.off, np.int64), _c(st.t, np.int64), _c(st.v, np.uint8)
    h = P()
    rc = _load().oracle_sim_event(n_pi, G, _p(typ), _p(fo), _p(fn), _p(dr), _p(df),
                                  _p(so), _p(stt), _p(sv), ctypes.byref(h))
    if rc:
        raise OracleError(f"oracle_sim_event: {rc}")
    return _result(h)


def static_eval(nl, pi_vals) -> np.ndarray:
    n_pi, G, typ, fo, fn, _, _ = _net(nl)
    pv = _c(pi_vals, np.uint8)
    out = np.zeros(n_pi + G, np.uint8)
    rc = _load().oracle_static_eval(n_pi, G, _p(typ), _p(fo), _p(fn), _p(pv), _p(out))
    if rc:
        raise OracleError(f"oracle_static_eval: {rc}")
    return out


def check_gates(nl, off, t, v, g0: int = 0, g1: int | None = None, nthreads: int = 0):
    """Count gates in [g0, g1) whose waveform in (off, t, v) differs from the
    oracle's evaluation of their fanin waveforms taken from the same arrays."""
    n_pi, G, typ, fo, fn, dr, df = _net(nl)
    g1 = G if g1 is None else g1
    off, t, v = _c(off, np.int64), _c(t, np.int64), _c(v, np.uint8)
    first = ctypes.c_int64(-1)
    bad = _load().oracle_check_gates(n_pi, G, _p(typ), _p(fo), _p(fn), _p(dr), _p(df),
                                     _p(off), _p(t), _p(v), g0, g1, nthreads, ctypes.byref(first))
    return int(bad), int(first.value)
