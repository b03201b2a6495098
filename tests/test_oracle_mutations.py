"""Planted mistakes: each plausible slip in the oracle (a dropped term, a
wrong strictness, a wrong constant, an off-by-one) must make at least one of
the pins in test_oracle.py fail.  The mistake is planted in a temporary copy
of the oracle source on the CPU; the committed oracle is untouched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "timest_oracle.c")

MUTATIONS = {
    "c1_not_strict": ("if (P->rank[c] > P->rank[s]) { lo = te + 1; hi = te + d; }",
                      "if (P->rank[c] > P->rank[s]) { lo = te; hi = te + d; }"),
    "exclusion_dropped": ("if (cand_nbr(g, &R, x) != R.excl)\n                                    sum +=",
                          "if (1)\n                                    sum +="),
    "window_closed": ("int64_t wlo = wi * P->wd, whi = (wi + 2) * P->wd - 1;",
                      "int64_t wlo = wi * P->wd, whi = (wi + 2) * P->wd;"),
    "nphi_ignores_first_window": ("int N = 1 + ((a >= wd && (b / wd) == (a / wd)) ? 1 : 0);",
                                  "int N = 1 + (((b / wd) == (a / wd)) ? 1 : 0);"),
    "derive_not_strict": ("if (pos > 0 && t <= prev) continue;",
                          "if (pos > 0 && t < prev) continue;"),
    "validate_order_not_strict": ("if (have && S.tau[e] <= prev) return RS_ORDER;",
                                  "if (have && S.tau[e] < prev) return RS_ORDER;"),
    "philox_multiplier": ("0xD2511F53u", "0xD2511F57u"),
    "philox_key_schedule": ("if (r > 0) { k0 += 0x9E3779B9u;", "if (r >= 0) { k0 += 0x9E3779B9u;"),
    "brute_not_injective": ("if (pa < 0) { if (vertex_used(B, u)) return;", "if (pa < 0) { if (0) return;"),
    "brute_delta_off_by_one": ("int64_t hi = (pos == 0) ? g->T : first + P->delta;",
                               "int64_t hi = (pos == 0) ? g->T : first + P->delta - 1;"),
    "child_pick_off_by_one": ("if (run > rc) { pick = x; break; }", "if (run >= rc) { pick = x; break; }"),
    "root_pick_off_by_one": ("if (C->rootcum[p][mid] <= rr) lo = mid + 1;", "if (C->rootcum[p][mid] < rr) lo = mid + 1;"),
    "window_pick_off_by_one": ("if (r < (u128)C->Wi[i]) { wi = i; break; }", "if (r <= (u128)C->Wi[i]) { wi = i; break; }"),
    "estimate_scale": ("res->estimate = (double)C->W * (double)hits / (2.0 * (double)k);",
                       "res->estimate = (double)C->W * (double)hits / ((double)k);"),
    "brute_c2_always_on": ("if (P->c2 && nbr == og) continue;", "if (nbr == og) continue;"),
    "nphi_uses_delta_not_window_unit": ("int64_t wd = P->wd;", "int64_t wd = P->delta;"),
    "root_total_wrong_layer": ("int64_t wi = window_of(g->t[e], p, P->wd);\n            if (wi < 0) { C->rootcum[p][e] = 0; continue; }",
                               "int64_t wi = window_of(g->t[e], 0, P->wd);\n            if (wi < 0) { C->rootcum[p][e] = 0; continue; }"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", str(lib), str(mutant)])
    env = dict(os.environ, TIMEST_ORACLE_LIB=str(lib))
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode != 0, f"planted mistake {name} was not caught by any pin"


# Planted mistakes in the oracle's temporal CSR (oracle.csr_arrays, Python):
# each must make the loop-built CSR (helpers.csr_by_loops) disagree on at
# least one of the pin cases of test_oracle.py.
PY_SRC = os.path.join(ROOT, "oracle", "__init__.py")
PY_MUTATIONS = {
    "csr_out_sorted_by_dst": ('out_gid = np.argsort(src, kind="stable")', 'out_gid = np.argsort(dst, kind="stable")'),
    "csr_multi_time_before_dst": ("multi = np.lexsort((t, dst, src))", "multi = np.lexsort((dst, t, src))"),
    "csr_xrank_counts_ties": ('"out_xrank": np.searchsorted(in_key, out_key, side="left")',
                              '"out_xrank": np.searchsorted(in_key, out_key, side="right")'),
    "csr_in_to_out_wrong_map": ('"in_to_out": out_pos[in_gid]', '"in_to_out": in_pos[in_gid]'),
    "csr_owner_bits_wrong_owner": ('"own_out": bits(starts(src[out_gid]))', '"own_out": bits(starts(dst[out_gid]))'),
}


@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_planted_csr_mistake_is_caught(name, tmp_path, oracle_mod):
    import importlib.util
    from helpers import csr_by_loops, csr_case
    old, new = PY_MUTATIONS[name]
    src = open(PY_SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    path = tmp_path / "mutant_oracle.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("mutant_oracle", str(path))
    mutant = importlib.util.module_from_spec(spec)
    sys.modules["mutant_oracle"] = mutant   # dataclasses look their module up while it runs
    try:
        spec.loader.exec_module(mutant)
    finally:
        del sys.modules["mutant_oracle"]
    caught = False
    for seed, n, m, t_hi in [(1, 12, 300, 40), (2, 7, 90, 3), (3, 30, 500, 1000)]:
        G = csr_case(oracle_mod, seed, n, m, t_hi)
        s, d, t = G.edges()
        got = mutant.csr_arrays(n, s, d, t)
        want = csr_by_loops(n, s.tolist(), d.tolist(), t.tolist())
        if any(got[k].tolist() != want[k] for k in want):
            caught = True
            break
    assert caught, f"planted mistake {name} was not caught by the loop-built CSR"
