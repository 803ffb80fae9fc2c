"""Planted mistakes in the oracle: each must fail at least one of its pins.

Every mutant below is one plausible slip in oracle/oracle.c -- a dropped
term, a wrong comparison, swapped operands or indices, a wrong start value
-- applied to a copy of the source, compiled on the CPU and run through the
oracle's own pin tests (Table 1 and the Sec. 2.2 composition rules, the
Fig. 5 / Fig. 6 worked examples, time stepping of Algorithm 2, the Eq. 1
brute force, the BUF/INV closed forms, the two independent whole-netlist
simulators, the static settle values and the general-cell fixtures).  A
mutant that passes every pin would mark a gap in the pins.  The unmodified
source, built the same way, must pass them all.
"""
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import oracle
import test_oracle_cells as tc
import test_oracle_cells_general as tg
import test_oracle_gate as tgate
import test_oracle_netlist as tn

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, exact text in oracle.c, replacement)
MUTANTS = [
    # 2-value cell functions
    ("AND computed as OR", "case C_AND2: return a & b;", "case C_AND2: return a | b;"),
    ("XNOR without its inversion", "case C_XNOR2: return !(a ^ b);", "case C_XNOR2: return a ^ b;"),
    ("MUX data pins swapped", "case C_MUX2: return c ? b : a;", "case C_MUX2: return c ? a : b;"),
    ("AOI21 drops pin c", "case C_AOI21: return !((a & b) | c);", "case C_AOI21: return !(a & b);"),
    ("OAI21 inner OR as AND", "case C_OAI21: return !((a | b) & c);", "case C_OAI21: return !((a & b) & c);"),
    ("OAI21 arity 2", "{1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3};", "{1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 2};"),
    # 4-value completion (Sec. 2.2)
    ("Z read as 1", "if (in[p] == 0 || in[p] == 1) x[p] = in[p];", "if (in[p] != VX) x[p] = in[p] & 1;"),
    ("completion keeps the first value", "else if (result != r) return VX;", "else if (result != r) return result;"),
    # delay choice (Sec. 2.3)
    ("X target takes the larger delay", "return rise < fall ? rise : fall;", "return rise > fall ? rise : fall;"),
    ("rise and fall swapped", "if (v == 1) return rise;\n    if (v == 0) return fall;",
     "if (v == 1) return fall;\n    if (v == 0) return rise;"),
    # Algorithm 2 candidates
    ("cell value starts at 0", "int F = VX;                                   /* the cell value before any input event */",
     "int F = 0;                                    /* the cell value before any input event */"),
    ("delay minimum over every pin", "if (!changed[p]) continue;", "(void)changed[p];"),
    ("simultaneous input events applied one by one", "                changed[p] = 1;\n            }",
     "                changed[p] = 1;\n                break;\n            }"),
    # Eq. 1, stack and scan forms
    ("Eq. 1 tie keeps the old transition", "while (m > 0 && out_t[m - 1] >= tr[i]) m--;",
     "while (m > 0 && out_t[m - 1] > tr[i]) m--;"),
    ("stack dedupe against X only", "int last = m > 0 ? out_v[m - 1] : VX;", "int last = VX;"),
    ("scan survival not strict", "surv[i] = tr[i] < sufmin;", "surv[i] = tr[i] <= sufmin;"),
    ("scan dedupe never advances", "        last = v[i];\n    }\n    free(surv);", "    }\n    free(surv);"),
    # levelized evaluator
    ("levelized: rise and fall of an arc swapped",
     "need += src->n;\n                    ri[p] = d_rise[a]; fa[p] = d_fall[a];",
     "need += src->n;\n                    ri[p] = d_fall[a]; fa[p] = d_rise[a];"),
    ("levelized: pins in reverse order", "int32_t a = fanin_off[g] + p; wave_t *src = &w[fanin_net[a]];",
     "int32_t a = fanin_off[g] + (k - 1 - p); wave_t *src = &w[fanin_net[a]];"),
    # event-driven simulator
    ("event: Eq. 1 tie keeps the old transition", "while (q->n > q->head && q->t[q->n - 1] >= tr) q->n--;",
     "while (q->n > q->head && q->t[q->n - 1] > tr) q->n--;"),
    ("event: dedupe ignores the present output", "int last = (q->n > q->head) ? q->v[q->n - 1] : val[(int64_t)n_pi + g];",
     "int last = (q->n > q->head) ? q->v[q->n - 1] : VX;"),
    ("event: delay minimum over every pin", "if (evt[fanin_net[arc]] != t) continue;", "(void)evt;"),
    ("event: denied transitions still mature", "if (q->head >= q->n || q->seq[q->head] != e.id) continue;",
     "if (q->head >= q->n) continue;"),
    # static evaluation
    ("static: every pin reads the first fanin",
     "for (int p = 0; p < oracle_arity(type[g]); p++) in[p] = net_val[fanin_net[fanin_off[g] + p]];",
     "for (int p = 0; p < oracle_arity(type[g]); p++) in[p] = net_val[fanin_net[fanin_off[g]]];"),
    # general cells: edge classes, 5-D delays, tables
    ("X<->Z counted as a rising edge", "return EDGE_NONE;                            /* X <-> Z */",
     "return EDGE_RISE;                            /* X <-> Z */"),
    ("0 -> X not a rising edge", "if (nw == 1 || old == 0) return EDGE_RISE;", "if (nw == 1) return EDGE_RISE;"),
    ("arc delay ignores the input edge", "if (edge != EDGE_NONE && e != edge) continue;", "(void)edge; (void)e;"),
    ("arc delay toward X uses the fall entries only", "if (v != VX && val != v) continue;",
     "if (val != (v & 1)) continue;"),
    ("no-arc fallback takes the slowest arc", "int64_t dp = oracle_arc_delay4(D + 4 * p, EDGE_NONE, nF);\n"
     "                    if (dp < d) d = dp;",
     "int64_t dp = oracle_arc_delay4(D + 4 * p, EDGE_NONE, nF);\n"
     "                    if (d == INF64 || dp > d) d = dp;"),
    ("table index with pin a most significant", "for (int p = n_in - 1; p >= 0; p--) li = li * 4 + cur[p];",
     "for (int p = 0; p < n_in; p++) li = li * 4 + cur[p];"),
    ("cell output starts at 0", "int F = VX;                                   /* the output before any input event */",
     "int F = 0;                                    /* the output before any input event */"),
    ("multi-output delays indexed by output first",
     "D[4 * p + j] = delays[delay_off[c] + ((int64_t)p * n_out[c] + o) * 4 + j];",
     "D[4 * p + j] = delays[delay_off[c] + ((int64_t)o * k + p) * 4 + j];"),
]

# the pins, cheapest first
PINS = [
    tc.test_table1_and_or_xor, tc.test_sec22_sentences, tc.test_read_once_cells_equal_composition,
    tc.test_mux2_against_composition, tc.test_boolean_corner_of_each_cell, tc.test_delay_by_output_value,
    tgate.test_fig5_min_delay, tgate.test_fig6_glitch_eaten, tgate.test_x_start_and_no_event_gate,
    tgate.test_single_pulse_through_buf, tgate.test_candidates_against_time_stepping,
    tn.test_buf_inv_chain_closed_form, tn.test_event_driven_equals_levelized, tn.test_settle_values_equal_static_eval,
    tn.test_invariants_and_eq2_bound, tn.test_same_net_on_both_pins_closed_forms,
    tg.test_edge_classes_golden, tg.test_arc_delay4_cases, tg.test_edge_delay_golden,
    tg.test_cell_candidates_against_time_stepping, tg.test_cell_candidates_equal_gate_candidates, tg.test_outputs_are_independent, tg.test_general_invariants,
    tgate.test_eq1_bruteforce_all_short_sequences,
]


def _build(src_text, path):
    with open(path + ".c", "w") as f:
        f.write(src_text)
    r = subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-o", path, path + ".c"],
                       capture_output=True, text=True)
    return r.returncode, r.stderr


def _first_failing_pin(lib):
    with oracle.library(lib):
        for pin in PINS:
            try:
                pin()
            except Exception:   # an assertion, or an error the oracle reports
                return pin.__name__
    return None


def test_every_planted_mistake_fails_a_pin(tmp_path):
    src = open(SRC).read()
    variants = [("unmodified", src)]
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, f"mutant '{name}': its text is not found exactly once in oracle.c"
        variants.append((name, src.replace(old, new)))
    paths = [str(tmp_path / f"liboracle_m{i}.so") for i in range(len(variants))]
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        built = list(ex.map(lambda a: _build(a[0][1], a[1]), zip(variants, paths)))
    for (name, _), (rc, err) in zip(variants, built):
        assert rc == 0, f"{name}: {err}"
    assert _first_failing_pin(paths[0]) is None, "the unmodified oracle must pass every pin"
    survivors = [name for (name, _), p in zip(variants[1:], paths[1:]) if _first_failing_pin(p) is None]
    assert survivors == [], f"planted mistakes no pin catches: {survivors}"
