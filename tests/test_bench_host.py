"""Host-side helpers of bench.py, on the CPU: the algorithmic-byte count
behind the roofline line, the clock-sample summary, and the rule that the
recorded ncu traffic is reported only for the configuration and kernel
source it was captured on."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from synth import Netlist  # noqa: E402


def test_algorithmic_bytes_by_hand():
    # PIs 0, 1; gate 0 = AND2(PI0, PI1) (net 2), gate 1 = INV(gate 0) (net 3)
    nl = Netlist(2, np.array([2, 0], np.uint8), np.array([0, 2, 3], np.int32), np.array([0, 1, 2], np.int32),
                 np.ones(3, np.int32), np.ones(3, np.int32))
    off = np.array([0, 3, 5, 9, 10], np.int64)       # waveform lengths 3, 2, 4, 1
    reads = 4 * (3 + 2 + 4)                          # each fanin arc reads its net once
    writes = 4 * (4 + 1)                             # each gate writes its output once
    meta = 48 * 2 + 12 * 3 + 12 * 2                  # gate records, fanin and output descriptors
    assert bench.algorithmic_bytes(nl, off) == reads + writes + meta


def _line(sm, mx, hw="Not Active", therm="Not Active", swth="Not Active", cap="Not Active"):
    return f"{sm}, {mx}, 900.00, 0x0000000000000000, {hw}, {therm}, {swth}, {cap}"


def test_clock_summary_uses_the_timed_region_only():
    c = bench.ClockSampler(0)
    c.lines = [_line(345, 2070)]          # idle sample before the timed region
    c.mark()
    c.lines += [_line(2070, 2070), _line(2055, 2070), _line(2070, 2070, cap="Active")]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines.append(_line(1500, 2070, hw="Active"))
    assert "hw_slowdown" in c.summary()["reasons"]
    empty = bench.ClockSampler(0)
    empty.lines = [_line(2070, 2070)]
    empty.mark()
    assert empty.summary()["reasons"] == ["unsampled"] and empty.summary()["samples"] == 0


def test_recorded_traffic_only_for_its_own_configuration():
    with open(os.path.join(ROOT, "profiles", "gate_kernel_traffic.json")) as f:
        rec = json.load(f)["ind1m"]
    cfg = dict(rec["applies_to"])
    if rec["kernel_source_sha"] == bench.kernel_source_sha():
        assert bench.ncu_traffic("ind1m", cfg) == rec["dram_bytes_per_run"]
    for key, other in (("gates", 300_000), ("schedule", "levels"), ("kernel", "windowed"), ("seed", 2)):
        assert bench.ncu_traffic("ind1m", dict(cfg, **{key: other})) is None
    assert bench.ncu_traffic("skew10m", cfg) is None


def test_cpu_model_names_something():
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()


def test_trace_copies_are_fresh_requests():
    from paper_2304_13398_gb300.serve import Request
    tr = [Request(0, "n0", 5000, 0.1), Request(1, "n1", 7000, 0.2)]
    tr[0].t_done, tr[0].out_transitions = 1.0, 99
    cp = bench.copy_trace(tr)
    assert [(q.rid, q.netlist, q.t_limit, q.arrival) for q in cp] == [(0, "n0", 5000, 0.1), (1, "n1", 7000, 0.2)]
    assert all(q.t_done < 0 and q.out_transitions == 0 for q in cp) and cp[0] is not tr[0]


def test_mem_available_reads_meminfo():
    m = bench.mem_available_bytes()
    assert m > 0 and m % 1024 == 0
