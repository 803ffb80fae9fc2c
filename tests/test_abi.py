"""CPU checks of the C-ABI library: it loads, exports every entry point its
header declares, and its host-only validation and levelization behave.  No
compute call is made here (there is no GPU on this side)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2304_13398_gb300 as gls
from paper_2304_13398_gb300 import build as gls_build
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gls_build.build()
    return gls.load_library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gls_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    bound = {s[0] for s in gls.gls.SIGNATURES}
    assert set(names) == bound, "binding and header disagree"


def declared_constants():
    """Every GLS_* enumerator of the header with its value."""
    src = open(os.path.join(ROOT, "include", "gls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(GLS_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}


def test_binding_constants_equal_header():
    consts = declared_constants()
    assert "GLS_OPT_SLICE_GROUP" in consts and "GLS_ETIMEOUT" in consts
    for name, value in consts.items():
        if hasattr(gls.gls, name):
            assert getattr(gls.gls, name) == value, name
    for name in [n for n in consts if n.startswith(("GLS_OPT_", "GLS_KERNEL_", "GLS_SCHEDULE_"))]:
        assert hasattr(gls.gls, name), f"{name} is not in the binding"


def test_version_and_arity(lib):
    assert lib.gls_version() >= 100
    assert [lib.gls_cell_arity(c) for c in range(11)] == [1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3]
    assert lib.gls_cell_arity(11) == gls.gls.GLS_EINVAL


def _nl(n_pi, cells, fanins, rise=None, fall=None):
    typ = np.array(cells, np.uint8)
    off = np.zeros(len(cells) + 1, np.int32)
    off[1:] = np.cumsum([len(f) for f in fanins])
    net = np.array([x for f in fanins for x in f], np.int32)
    r = np.full(len(net), 5, np.int32) if rise is None else np.array(rise, np.int32)
    f = np.full(len(net), 7, np.int32) if fall is None else np.array(fall, np.int32)
    return n_pi, typ, off, net, r, f


def expect(code, *args):
    with pytest.raises(gls.GlsError) as ei:
        gls.check_netlist(*args)
    assert ei.value.code == code, str(ei.value)


def test_netlist_validation(lib):
    E = gls.gls
    # ok: gate 1 reads gate 0 (net 2)
    depth, level = gls.check_netlist(*_nl(2, [2, 0], [[0, 1], [2]]))
    assert depth == 2 and level.tolist() == [1, 2]
    # gates may be listed in any order
    depth, level = gls.check_netlist(*_nl(2, [0, 2], [[3], [0, 1]]))
    assert depth == 2 and level.tolist() == [2, 1]
    expect(E.GLS_EINVAL, *_nl(2, [2], [[0]]))                    # pin count
    expect(E.GLS_EINVAL, *_nl(2, [2], [[0, 5]]))                 # net out of range
    expect(E.GLS_EINVAL, *_nl(2, [2], [[0, 1]], rise=[0, 1]))    # delay < 1
    expect(E.GLS_ECYCLE, *_nl(1, [2, 1], [[0, 2], [1]]))         # gate0 <- gate1 <- gate0
    expect(E.GLS_ECYCLE, *_nl(1, [1], [[1]]))                    # self loop
    expect(E.GLS_ERANGE, *_nl(2, [2], [[0, 1]], rise=[5, 300], fall=[5, 5]))   # spread 295
    gls.check_netlist(*_nl(2, [2], [[0, 1]], rise=[5, 260], fall=[5, 5]))      # spread 255 is fine
    expect(E.GLS_EINVAL, *_nl(2, [11], [[0, 1]]))                # unknown cell


def test_levels_match_generator(lib):
    for seed in (1, 2, 3):
        nl = synth.make_netlist(8, 300, 9, seed=seed)
        depth, level = gls.check_netlist(nl.n_pi, nl.type, nl.fanin_off, nl.fanin_net, nl.d_rise, nl.d_fall)
        assert depth == 9
        assert np.array_equal(level, nl.level)
        nl = synth.make_netlist(8, 300, 9, seed=seed, shuffle=True)
        depth, level = gls.check_netlist(nl.n_pi, nl.type, nl.fanin_off, nl.fanin_net, nl.d_rise, nl.d_fall)
        assert np.array_equal(level, nl.level)


def test_stimulus_validation(lib):
    ok = (2, [0, 2, 3], [5, 9, 1], [1, 0, 2])
    gls.check_stimulus(*ok)
    bad = [
        (2, [0, 2, 3], [5, 5, 1], [1, 0, 2]),        # time not increasing
        (2, [0, 2, 3], [5, 9, 1], [1, 1, 2]),        # repeated value
        (2, [0, 2, 3], [5, 9, 1], [1, 0, 4]),        # value > 3
        (2, [0, 2, 3], [-1, 9, 1], [1, 0, 2]),       # negative time
        (2, [0, 2, 3], [5, 9, (1 << 30)], [1, 0, 2]),  # time too large
        (2, [0, 3, 2], [5, 9, 1], [1, 0, 2]),        # offsets not monotone
        (2, [1, 2, 3], [5, 9, 1], [1, 0, 2]),        # off[0] != 0
    ]
    for case in bad:
        with pytest.raises(gls.GlsError) as ei:
            gls.check_stimulus(*case)
        assert ei.value.code == gls.gls.GLS_ESTIM, case


def test_context_needs_a_gpu(lib):
    # without a device the library reports an error instead of crashing
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    rc = lib.gls_create(ctypes.byref(h), 0, 0)
    assert rc in (gls.gls.GLS_ECUDA, gls.gls.GLS_EINVAL)
    assert lib.gls_last_error(None)


def test_builtin_cell_tables_equal_oracle():
    """The library's 4-value tables (Kleene evaluation of prime-implicant
    covers) against the oracle's (enumeration of 0/1 completions): two
    independent derivations of the same cell functions, on the host."""
    import oracle
    import paper_2304_13398_gb300 as gls
    for c in range(11):
        np.testing.assert_array_equal(gls.cell_table(c), oracle.cell_lut(c))
