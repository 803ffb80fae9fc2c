"""ctypes binding of libgls.so (declared in include/gls.h).

The module-level ``gls_*`` names are the C entry points themselves with their
argument types declared; ``Context`` wraps them with numpy marshalling and
raises ``GlsError`` on a negative status.  All computation happens in the
library's CUDA kernels: there is no Python or CPU fallback, and loading fails
loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgls.so")

GLS_OK, GLS_EINVAL, GLS_ECYCLE, GLS_ESTIM, GLS_ERANGE, GLS_ENOMEM, GLS_EOVERFLOW, GLS_ETIMEOUT, GLS_ECUDA, \
    GLS_EAGAIN = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
STATUS_NAMES = {0: "GLS_OK", -1: "GLS_EINVAL", -2: "GLS_ECYCLE", -3: "GLS_ESTIM", -4: "GLS_ERANGE",
                -5: "GLS_ENOMEM", -6: "GLS_EOVERFLOW", -7: "GLS_ETIMEOUT", -8: "GLS_ECUDA", -9: "GLS_EAGAIN"}
CELLS = ["INV", "BUF", "AND2", "OR2", "NAND2", "NOR2", "XOR2", "XNOR2", "MUX2", "AOI21", "OAI21"]
GLS_MAX_DELAY_SPREAD = 255
GLS_NOALLOC_MAX_LEVELS = 4000

P = ctypes.c_void_p
i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64

# (name, restype, argtypes) of every entry point in include/gls.h
SIGNATURES = [
    ("gls_version", ctypes.c_int, []),
    ("gls_cell_arity", ctypes.c_int, [ctypes.c_int]),
    ("gls_check_netlist", ctypes.c_int, [i32, i32, P, P, P, P, P, P, P]),
    ("gls_check_stimulus", ctypes.c_int, [i32, P, P, P]),
    ("gls_create", ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, u64]),
    ("gls_destroy", None, [P]),
    ("gls_last_error", ctypes.c_char_p, [P]),
    ("gls_load_netlist", ctypes.c_int, [P, i32, i32, P, P, P, P, P, ctypes.POINTER(i32)]),
    ("gls_load_stimulus", ctypes.c_int, [P, i32, P, P, P, ctypes.POINTER(i32)]),
    ("gls_update_stimulus", ctypes.c_int, [P, i32, P, P, P]),
    ("gls_simulate", ctypes.c_int, [P, i32, i32, i64, P, ctypes.POINTER(i32)]),
    ("gls_simulate_batch", ctypes.c_int, [P, i32, P, P, P, i64, P, ctypes.POINTER(i32)]),
    ("gls_rerun", ctypes.c_int, [P, i32, P]),
    ("gls_run_query", ctypes.c_int, [P, i32]),
    ("gls_run_info", ctypes.c_int, [P, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
    ("gls_plan_order", ctypes.c_int, [P, i32, i32, i32]),
    ("gls_read_host", ctypes.c_int, [P, i32, i32, ctypes.POINTER(P), P, P]),
    ("gls_cell_table", ctypes.c_int, [i32, P]),
    ("gls_define_cell", ctypes.c_int, [P, i32, i32, P, ctypes.POINTER(i32)]),
    ("gls_load_netlist_cells", ctypes.c_int, [P, i32, i32, P, P, P, P, ctypes.POINTER(i32)]),
    ("gls_load_stimulus64", ctypes.c_int, [P, i32, P, P, P, ctypes.POINTER(i32)]),
    ("gls_simulate_sliced", ctypes.c_int, [P, i32, i32, i64, i64, P, ctypes.POINTER(i32)]),
    ("gls_run_slices", ctypes.c_int, [P, i32, ctypes.POINTER(i32)]),
    ("gls_read_all64", ctypes.c_int, [P, i32, P, P, P, i64]),
    ("gls_read_waveform64", ctypes.c_int, [P, i32, i32, P, P, i64, ctypes.POINTER(i64)]),
    ("gls_run_stats", ctypes.c_int, [P, i32, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)]),
    ("gls_read_waveform", ctypes.c_int, [P, i32, i32, P, P, i64, ctypes.POINTER(i64)]),
    ("gls_read_all", ctypes.c_int, [P, i32, P, P, i64]),
    ("gls_read_item", ctypes.c_int, [P, i32, i32, P, P, i64]),
    ("gls_set_option", ctypes.c_int, [P, ctypes.c_int, i64]),
    ("gls_simulate_noalloc", ctypes.c_int, [P, i32, i32, P, P, P, i64, P, P]),
    ("gls_release", ctypes.c_int, [P, i32]),
]
GLS_OPT_SCHEDULE, GLS_OPT_WARPS_PER_CTA, GLS_OPT_WAIT_LIMIT_MS, GLS_OPT_TEST_WITHHOLD_GATE, GLS_OPT_KERNEL, GLS_OPT_SEGMENT, \
    GLS_OPT_POOL_BYTES, GLS_OPT_HOST_MIRROR, GLS_OPT_HOST_POOL_BYTES, GLS_OPT_SLICE_GROUP = 1, 2, 3, 4, 5, 6, 7, 8, 9, 10
GLS_KERNEL_SEGMENTED, GLS_KERNEL_WINDOWED, GLS_KERNEL_WINDOWED_WIDE = 0, 1, 2
KERNELS = {"segmented": GLS_KERNEL_SEGMENTED, "windowed": GLS_KERNEL_WINDOWED, "wide": GLS_KERNEL_WINDOWED_WIDE}
GLS_SCHEDULE_LEVELS, GLS_SCHEDULE_DEPENDENCY = 0, 1
SCHEDULES = {"levels": GLS_SCHEDULE_LEVELS, "dependency": GLS_SCHEDULE_DEPENDENCY}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libgls.so and declare every signature.  Raises if it is missing:
    the simulator has no fallback path."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2304_13398_gb300.build.build() "
                               "(the simulator has no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
            globals()[name] = f
        _lib = lib
    return _lib


def __getattr__(name):
    if name.startswith("gls_"):
        load_library()
        if name in globals():
            return globals()[name]
    raise AttributeError(name)


class GlsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(P)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)    # torch.cuda.Stream


def check_netlist(n_pi, type, fanin_off, fanin_net, d_rise, d_fall):
    """Host-only validation and levelization; returns (depth, level[G])."""
    lib = load_library()
    typ, fo, fn = _c(type, np.uint8), _c(fanin_off, np.int32), _c(fanin_net, np.int32)
    dr, df = _c(d_rise, np.int32), _c(d_fall, np.int32)
    depth = ctypes.c_int32(0)
    level = np.zeros(len(typ), np.int32)
    rc = lib.gls_check_netlist(n_pi, len(typ), _p(typ), _p(fo), _p(fn), _p(dr), _p(df),
                               ctypes.cast(ctypes.pointer(depth), P), _p(level))
    if rc:
        raise GlsError(rc, lib.gls_last_error(None).decode())
    return depth.value, level


def check_stimulus(n_pi, off, t, v):
    lib = load_library()
    rc = lib.gls_check_stimulus(n_pi, _p(_c(off, np.int64)), _p(_c(t, np.int32)), _p(_c(v, np.uint8)))
    if rc:
        raise GlsError(rc, lib.gls_last_error(None).decode())


@dataclass
class RunStats:
    total_events: int
    kernel_ms: float


class Context:
    """One simulator context on one CUDA device (owns all its device memory)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.lib = load_library()
        h = P()
        rc = self.lib.gls_create(ctypes.byref(h), device, hbm_budget_bytes)
        if rc:
            raise GlsError(rc, self.lib.gls_last_error(None).decode())
        self.h = h
        self.n_nets = {}
        self.n_pis = {}          # netlist id -> primary inputs
        self.run_nets = {}       # run id -> netlist id of each item

    def _ck(self, rc):
        if rc:
            raise GlsError(rc, self.lib.gls_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.gls_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_option(self, option: int, value: int):
        self._ck(self.lib.gls_set_option(self.h, option, value))

    def set_schedule(self, name: str):
        """'levels' (one launch per DAG level) or 'dependency' (one persistent
        launch, gates start when their fanins are done)."""
        self.set_option(GLS_OPT_SCHEDULE, SCHEDULES[name])

    def set_kernel(self, name: str):
        """'windowed' (warp per 128-transition window), 'wide' (256) or
        'segmented' (lane per time segment)."""
        self.set_option(GLS_OPT_KERNEL, KERNELS[name])

    def load_netlist(self, nl) -> int:
        typ, fo, fn = _c(nl.type, np.uint8), _c(nl.fanin_off, np.int32), _c(nl.fanin_net, np.int32)
        dr, df = _c(nl.d_rise, np.int32), _c(nl.d_fall, np.int32)
        nid = ctypes.c_int32(0)
        self._ck(self.lib.gls_load_netlist(self.h, int(nl.n_pi), len(typ), _p(typ), _p(fo), _p(fn),
                                           _p(dr), _p(df), ctypes.byref(nid)))
        self.n_nets[nid.value] = int(nl.n_pi) + len(typ)
        self.n_pis[nid.value] = int(nl.n_pi)
        return nid.value

    def load_stimulus(self, st, n_pi: int | None = None) -> int:
        off, t, v = _c(st.off, np.int64), _c(st.t, np.int32), _c(st.v, np.uint8)
        sid = ctypes.c_int32(0)
        n_pi = len(off) - 1 if n_pi is None else n_pi
        self._ck(self.lib.gls_load_stimulus(self.h, n_pi, _p(off), _p(t), _p(v), ctypes.byref(sid)))
        return sid.value

    def define_cell(self, n_inputs: int, tables) -> int:
        """A user cell (UDP / multi-output cell): tables = n_outputs x 4^n_inputs
        values in {0, 1, 2 = X}.  Returns its cell type id."""
        t = _c(tables, np.uint8)
        n4 = 4 ** n_inputs
        if t.size % n4:
            raise ValueError("tables must hold n_outputs * 4^n_inputs values")
        ct = ctypes.c_int32(0)
        self._ck(self.lib.gls_define_cell(self.h, n_inputs, t.size // n4, _p(t), ctypes.byref(ct)))
        self.__dict__.setdefault("_outs", {})[ct.value] = t.size // n4
        return ct.value

    def load_netlist_cells(self, n_pi: int, cell_type, fanin_off, fanin_net, delays) -> int:
        """A netlist of general cells (see include/gls.h)."""
        ct, fo, fn, d = (_c(cell_type, np.int32), _c(fanin_off, np.int32), _c(fanin_net, np.int32),
                         _c(delays, np.int32))
        nid = ctypes.c_int32(0)
        self._ck(self.lib.gls_load_netlist_cells(self.h, n_pi, len(ct), _p(ct), _p(fo), _p(fn), _p(d),
                                                 ctypes.byref(nid)))
        self.n_nets[nid.value] = n_pi + self._cell_outputs(ct)
        self.n_pis[nid.value] = int(n_pi)
        return nid.value

    def _cell_outputs(self, ct) -> int:
        outs = getattr(self, "_outs", {})
        return int(sum(outs.get(int(x), 1) for x in ct))

    def load_cell_netlist(self, cn) -> int:
        """Load a CellNetlist whose cells each carry their own tables: one
        user cell per instance."""
        types = np.zeros(cn.n_cells, np.int32)
        for c in range(cn.n_cells):
            types[c] = self.define_cell(cn.n_in(c), cn.luts[cn.lut_off[c]:cn.lut_off[c + 1]])
        return self.load_netlist_cells(cn.n_pi, types, cn.fanin_off, cn.fanin_net, cn.delays)

    def load_cell_netlist_shared(self, cn) -> int:
        """Load a CellNetlist, defining each distinct cell (input count and
        tables of all its outputs) once and sharing it between instances."""
        lib: dict = {}
        types = np.zeros(cn.n_cells, np.int32)
        for c in range(cn.n_cells):
            tab = cn.luts[cn.lut_off[c]:cn.lut_off[c + 1]]
            key = (cn.n_in(c), tab.tobytes())
            t = lib.get(key)
            if t is None:
                t = lib[key] = self.define_cell(cn.n_in(c), tab)
            types[c] = t
        return self.load_netlist_cells(cn.n_pi, types, cn.fanin_off, cn.fanin_net, cn.delays)

    def load_stimulus64(self, st, n_pi: int | None = None) -> int:
        """A stimulus with 64-bit times (for simulate_sliced)."""
        off, t, v = _c(st.off, np.int64), _c(st.t, np.int64), _c(st.v, np.uint8)
        sid = ctypes.c_int32(0)
        n_pi = len(off) - 1 if n_pi is None else n_pi
        self._ck(self.lib.gls_load_stimulus64(self.h, n_pi, _p(off), _p(t), _p(v), ctypes.byref(sid)))
        return sid.value

    def simulate_sliced(self, netlist_id: int, stim_id: int, slice_ps: int, arena_events: int = 0,
                        stream=None) -> int:
        """Task division over time (synchronous); read with read_all64 / read_waveform64."""
        rid = ctypes.c_int32(0)
        self._ck(self.lib.gls_simulate_sliced(self.h, netlist_id, stim_id, int(slice_ps), arena_events,
                                              _stream_handle(stream), ctypes.byref(rid)))
        self.n_nets[rid.value] = self.n_nets[netlist_id]
        self.run_nets[rid.value] = [netlist_id]
        return rid.value

    def run_slices(self, run_id: int) -> int:
        n = ctypes.c_int32(0)
        self._ck(self.lib.gls_run_slices(self.h, run_id, ctypes.byref(n)))
        return n.value

    def read_all64(self, run_id: int):
        """(off int64[N+1], t int64[E], v uint8[E]) of a sliced run."""
        N = self.n_nets[run_id]
        N = N[0] if isinstance(N, list) else N
        off = np.zeros(N + 1, np.int64)
        rc = self.lib.gls_read_all64(self.h, run_id, _p(off), None, None, 0)
        if rc not in (GLS_OK, GLS_EOVERFLOW):
            self._ck(rc)
        E = int(off[N])
        t = np.zeros(E, np.int64)
        v = np.zeros(E, np.uint8)
        self._ck(self.lib.gls_read_all64(self.h, run_id, _p(off), _p(t), _p(v), E))
        return off, t, v

    def read_waveform64(self, run_id: int, net: int):
        n = ctypes.c_int64(0)
        rc = self.lib.gls_read_waveform64(self.h, run_id, net, None, None, 0, ctypes.byref(n))
        if rc not in (GLS_OK, GLS_EOVERFLOW):
            self._ck(rc)
        t = np.zeros(n.value, np.int64)
        v = np.zeros(n.value, np.uint8)
        self._ck(self.lib.gls_read_waveform64(self.h, run_id, net, _p(t), _p(v), n.value, ctypes.byref(n)))
        return t, v

    def update_stimulus(self, stim_id: int, off, t, v):
        """off/t/v may be numpy arrays or (pinned) torch CPU tensors."""
        self._ck(self.lib.gls_update_stimulus(self.h, stim_id, _ptr(off, np.int64), _ptr(t, np.int32),
                                              _ptr(v, np.uint8)))

    def simulate(self, netlist_id: int, stim_id: int, arena_events: int = 0, stream=None) -> int:
        rid = ctypes.c_int32(0)
        self._ck(self.lib.gls_simulate(self.h, netlist_id, stim_id, arena_events, _stream_handle(stream),
                                       ctypes.byref(rid)))
        self.n_nets[rid.value] = self.n_nets[netlist_id]
        self.run_nets[rid.value] = [netlist_id]
        return rid.value

    def simulate_batch(self, netlist_ids, stim_ids, t_limits=None, arena_events: int = 0, stream=None) -> int:
        """One launch over several (netlist, stimulus[, time limit]) items; read each with read_item."""
        nids = _c(netlist_ids, np.int32)
        sids = _c(stim_ids, np.int32)
        tls = None if t_limits is None else _c(t_limits, np.int32)
        if len(nids) != len(sids) or (tls is not None and len(tls) != len(nids)):
            raise ValueError("item arrays differ in length")
        rid = ctypes.c_int32(0)
        self._ck(self.lib.gls_simulate_batch(self.h, len(nids), _p(nids), _p(sids), _p(tls), arena_events,
                                             _stream_handle(stream), ctypes.byref(rid)))
        self.n_nets[rid.value] = [self.n_nets[int(n)] for n in nids]
        self.run_nets[rid.value] = [int(n) for n in nids]
        return rid.value

    def read_item(self, run_id: int, item: int, off=None, packed=None):
        """Dense CSR of one item of a batch run (see read_all)."""
        nn = self.n_nets[run_id]
        nn = nn if isinstance(nn, list) else [nn]
        N = nn[item] if 0 <= item < len(nn) else 0   # the library rejects a bad item
        if off is None:
            off = np.zeros(N + 1, np.int64)
        if packed is None:
            rc = self.lib.gls_read_item(self.h, run_id, item, _ptr(off, np.int64), None, 0)
            if rc not in (GLS_OK, GLS_EOVERFLOW):
                self._ck(rc)
            packed = np.zeros(int(off[N]), np.uint32)
        cap = int(packed.shape[0]) if hasattr(packed, "shape") else len(packed)
        self._ck(self.lib.gls_read_item(self.h, run_id, item, _ptr(off, np.int64), _ptr(packed, np.uint32), cap))
        return off, packed

    def rerun(self, run_id: int, stream=None):
        self._ck(self.lib.gls_rerun(self.h, run_id, _stream_handle(stream)))

    def run_done(self, run_id: int) -> bool:
        """True once the run's last enqueued evaluation finished (does not block)."""
        rc = self.lib.gls_run_query(self.h, run_id)
        if rc == GLS_EAGAIN:
            return False
        self._ck(rc)
        return True

    def run_info(self, run_id: int):
        """(arena demand, arena capacity) in 32-bit words."""
        d, c = ctypes.c_int64(0), ctypes.c_int64(0)
        self._ck(self.lib.gls_run_info(self.h, run_id, ctypes.byref(d), ctypes.byref(c)))
        return d.value, c.value

    def read_host(self, run_id: int, item: int = 0, gate_off=None, gate_len=None):
        """Waveforms of a run created with GLS_OPT_HOST_MIRROR, already in host
        memory: (arena, gate_off, gate_len) with gate g's packed transitions at
        arena[gate_off[g]:gate_off[g] + gate_len[g]]; arena is a view of the
        run's pinned mirror (valid until the run is re-run or released)."""
        nets = self.run_nets.get(run_id, [])
        G = 0
        if 0 <= item < len(nets):   # the library rejects a bad item
            G = self.n_nets[nets[item]] - self.n_pis[nets[item]]
        if gate_off is None:
            gate_off = np.zeros(max(G, 1), np.int64)
        if gate_len is None:
            gate_len = np.zeros(max(G, 1), np.uint32)
        ptr = P()
        self._ck(self.lib.gls_read_host(self.h, run_id, item, ctypes.byref(ptr), _ptr(gate_off, np.int64),
                                        _ptr(gate_len, np.uint32)))
        _, cap = self.run_info(run_id)
        arena = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_uint32)), shape=(cap,))
        return arena, gate_off[:G], gate_len[:G]

    def plan_order(self, netlist_id: int, run_id: int = -1, item: int = 0):
        """Critical-path-first dependency order for netlist_id from the net
        activity of a finished run (run_id = -1: back to level order)."""
        self._ck(self.lib.gls_plan_order(self.h, netlist_id, run_id, item))

    def run_stats(self, run_id: int) -> RunStats:
        tot, ms = ctypes.c_int64(0), ctypes.c_double(0.0)
        self._ck(self.lib.gls_run_stats(self.h, run_id, ctypes.byref(tot), ctypes.byref(ms)))
        return RunStats(tot.value, ms.value)

    def run_stats_raw(self, run_id: int):
        """(status, total_events, kernel_ms) without raising."""
        tot, ms = ctypes.c_int64(0), ctypes.c_double(0.0)
        rc = self.lib.gls_run_stats(self.h, run_id, ctypes.byref(tot), ctypes.byref(ms))
        return rc, tot.value, ms.value

    def read_waveform(self, run_id: int, net: int):
        n = ctypes.c_int64(0)
        rc = self.lib.gls_read_waveform(self.h, run_id, net, None, None, 0, ctypes.byref(n))
        if rc not in (GLS_OK, GLS_EOVERFLOW):
            self._ck(rc)
        t = np.zeros(n.value, np.int32)
        v = np.zeros(n.value, np.uint8)
        self._ck(self.lib.gls_read_waveform(self.h, run_id, net, _p(t), _p(v), n.value, ctypes.byref(n)))
        return t, v

    def read_all(self, run_id: int, off=None, packed=None):
        """Dense CSR of every net: (off int64[N+1], packed uint32[E]) with
        packed = (t << 2) | v.  Optional preallocated (pinned) outputs."""
        N = self.n_nets[run_id]
        N = N[0] if isinstance(N, list) else N
        if off is None:
            off = np.zeros(N + 1, np.int64)
        if packed is None:
            rc = self.lib.gls_read_all(self.h, run_id, _ptr(off, np.int64), None, 0)
            if rc not in (GLS_OK, GLS_EOVERFLOW):
                self._ck(rc)
            total = int(off[N])
            packed = np.zeros(total, np.uint32)
        cap = int(packed.shape[0]) if hasattr(packed, "shape") else len(packed)
        self._ck(self.lib.gls_read_all(self.h, run_id, _ptr(off, np.int64), _ptr(packed, np.uint32), cap))
        return off, packed

    def release(self, obj_id: int):
        self._ck(self.lib.gls_release(self.h, obj_id))


def _ptr(a, dt):
    """Pointer of a numpy array or a contiguous CPU torch tensor of dtype dt."""
    if isinstance(a, np.ndarray):
        if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"need a contiguous {np.dtype(dt)} array")
        return _p(a)
    if hasattr(a, "data_ptr"):
        return P(a.data_ptr())
    raise TypeError(type(a))


def cell_table(cell: int) -> np.ndarray:
    """The library's 4^k table of a built-in cell."""
    k = int(load_library().gls_cell_arity(cell))
    out = np.zeros(4 ** k, np.uint8)
    rc = load_library().gls_cell_table(cell, out.ctypes.data_as(ctypes.c_void_p))
    if rc != GLS_OK:
        raise GlsError(rc, "gls_cell_table")
    return out


def unpack(packed: np.ndarray):
    """Split packed transitions into (times int32, values uint8)."""
    p = np.asarray(packed, dtype=np.uint32)
    return (p >> 2).astype(np.int32), (p & 3).astype(np.uint8)
