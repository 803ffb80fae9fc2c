"""Readers for the hand-written fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SYM = {"0": 0, "1": 1, "X": 2, "Z": 3}


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln


def truth_tables(name="table1_truth_tables.txt"):
    """{op: 4x4 list} with rows/cols in the order 0 1 X Z."""
    out, cur = {}, None
    for ln in _lines(name):
        if ln.isalpha():
            cur = ln
            out[cur] = []
        else:
            out[cur].append([SYM[s] for s in ln.split()])
    return out


def waveform_cases(name):
    """{case: (pins {pin: [(t, v)]}, expected [(t, v)])}."""
    out, cur = {}, None
    for ln in _lines(name):
        parts = ln.split()
        if parts[0] == "case":
            cur = parts[1]
            out[cur] = ({}, [])
        elif parts[0] == "expect":
            out[cur][1].append((int(parts[1]), SYM[parts[2]]))
        else:
            out[cur][0].setdefault(parts[0], []).append((int(parts[1]), SYM[parts[2]]))
    return out
