"""Pins of the oracle's 4-value cell functions and delay choice.

- Table 1 (Sec. 2.2): the printed AND/OR/XOR tables, from a golden fixture.
- Sec. 2.2 text: "1 AND X" is X, "1 OR X" is 1, Z is read as X.
- Composition: cells that are read-once formulas of AND/OR/XOR/NOT
  (NAND, NOR, XNOR, AOI21, OAI21) equal the composition of the Table 1
  tables (NOT maps X and Z to X, the only reading of "X may be 0 or 1").
- MUX2 (s ? b : a): under Sec. 2.2's reading of X the select is irrelevant
  when a == b in {0, 1}; composition through AND/OR gives X for a == b == 1
  with an unknown select.  The test checks exactly where the two differ.
"""
import itertools

import numpy as np
import pytest

import oracle
from golden_io import truth_tables

X, Z = 2, 3
V4 = [0, 1, X, Z]


def idx(*ins):
    return sum(v * 4 ** p for p, v in enumerate(ins))


def test_table1_and_or_xor():
    tabs = truth_tables()
    for name, cell in (("AND", oracle.AND2), ("OR", oracle.OR2), ("XOR", oracle.XOR2)):
        lut = oracle.cell_lut(cell)
        for i, a in enumerate(V4):
            for j, b in enumerate(V4):
                assert lut[idx(a, b)] == tabs[name][i][j], (name, a, b)


def test_sec22_sentences():
    assert oracle.cell_eval(oracle.AND2, [1, X]) == X
    assert oracle.cell_eval(oracle.OR2, [1, X]) == 1
    for cell in range(11):
        k = oracle.ARITY[cell]
        for ins in itertools.product(V4, repeat=k):
            zx = [X if v == Z else v for v in ins]
            assert oracle.cell_eval(cell, ins) == oracle.cell_eval(cell, zx)
            assert oracle.cell_eval(cell, ins) in (0, 1, X)   # never Z


def _t1():
    tabs = truth_tables()
    AND = lambda a, b: tabs["AND"][V4.index(a)][V4.index(b)]
    OR = lambda a, b: tabs["OR"][V4.index(a)][V4.index(b)]
    XOR = lambda a, b: tabs["XOR"][V4.index(a)][V4.index(b)]
    NOT = lambda a: {0: 1, 1: 0, X: X, Z: X}[a]
    return AND, OR, XOR, NOT


def test_read_once_cells_equal_composition():
    AND, OR, XOR, NOT = _t1()
    comp = {
        oracle.INV: lambda a: NOT(a),
        oracle.BUF: lambda a: NOT(NOT(a)),
        oracle.AND2: AND,
        oracle.OR2: OR,
        oracle.NAND2: lambda a, b: NOT(AND(a, b)),
        oracle.NOR2: lambda a, b: NOT(OR(a, b)),
        oracle.XOR2: XOR,
        oracle.XNOR2: lambda a, b: NOT(XOR(a, b)),
        oracle.AOI21: lambda a, b, c: NOT(OR(AND(a, b), c)),
        oracle.OAI21: lambda a, b, c: NOT(AND(OR(a, b), c)),
    }
    for cell, f in comp.items():
        k = oracle.ARITY[cell]
        for ins in itertools.product(V4, repeat=k):
            assert oracle.cell_eval(cell, ins) == f(*ins), (cell, ins)


def test_mux2_against_composition():
    AND, OR, XOR, NOT = _t1()
    mux_comp = lambda a, b, s: OR(AND(NOT(s), a), AND(s, b))
    diff = []
    for a, b, s in itertools.product(V4, repeat=3):
        got = oracle.cell_eval(oracle.MUX2, [a, b, s])
        want = mux_comp(a, b, s)
        if got != want:
            diff.append((a, b, s, got, want))
    # composition loses only the case of an unknown select with both data
    # inputs 1 (with both 0 the AND terms already give 0)
    assert sorted((a, b, s) for a, b, s, _, _ in diff) == [(1, 1, X), (1, 1, Z)]
    assert all(got == a and want == X for a, b, s, got, want in diff)
    # with a known select the mux passes the selected input, Z read as X
    for a, b in itertools.product(V4, repeat=2):
        assert oracle.cell_eval(oracle.MUX2, [a, b, 0]) == (X if a == Z else a)
        assert oracle.cell_eval(oracle.MUX2, [a, b, 1]) == (X if b == Z else b)


def test_boolean_corner_of_each_cell():
    # on 0/1 inputs the 4-value function is the Boolean one; spot values by cell name
    AND, OR, XOR, NOT = _t1()
    for a, b, c in itertools.product((0, 1), repeat=3):
        assert oracle.cell_eval(oracle.MUX2, [a, b, c]) == (b if c else a)
        assert oracle.cell_eval(oracle.AOI21, [a, b, c]) == 1 - ((a & b) | c)
        assert oracle.cell_eval(oracle.OAI21, [a, b, c]) == 1 - ((a | b) & c)


def test_delay_by_output_value():
    # Sec. 2.3: delay depends on the output transition value
    assert oracle.delay(7, 5, 1) == 7
    assert oracle.delay(7, 5, 0) == 5
    assert oracle.delay(7, 5, X) == 5
    assert oracle.delay(3, 9, X) == 3
