"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle.c (a dropped term, a wrong
sign, a swapped operand, an off-by-one rank, ...), builds it into a temporary
library and runs the pin suite against it in a child process: the suite must
fail.  The oracle source itself is never modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "deductible_dropped": ("net_of(conv, L->ded[j], L->lim[j])", "net_of(conv, 0.0, L->lim[j])"),
    "elt_limit_dropped": ("net_of(conv, L->ded[j], L->lim[j])", "net_of(conv, L->ded[j], 1e300)"),
    "share_dropped": ("g += L->share[j] * net_of(", "g += net_of("),
    "fx_dropped": ("const double conv = L->fx[j] * x;", "const double conv = x;"),
    "retention_sign": ("double a = v - r;", "double a = v + r;"),
    "occ_terms_swapped": ("net_of(g, L->occ_r, L->occ_l)", "net_of(g, L->occ_l, L->occ_r)"),
    "occ_step_skipped": ("const double o = net_of(g, L->occ_r, L->occ_l);", "const double o = g;"),
    "cumulative_sum_dropped": ("S += o;", "S = o;"),
    "agg_limit_from_occ": ("net_of(S, L->agg_r, L->agg_l)", "net_of(S, L->agg_r, L->occ_l)"),
    "ylt_before_agg_terms": ("out->ylt = A;", "out->ylt = S;"),
    "decumulate_forward_in_place": ("prev = A;", "prev = m;"),
    "lookup_wrong_slot": ("return t->p[mid].loss;", "return t->p[lo].loss;"),
    "lookup_wrong_elt": ("dict_lookup(&L->elt[j], ev[d])", "dict_lookup(&L->elt[0], ev[d])"),
    "last_elt_skipped": ("for (int32_t j = 0; j < L->n_elts; ++j) {", "for (int32_t j = 0; j + 1 < L->n_elts; ++j) {"),
    "gross_before_fx": ("gross += conv;", "gross += x;"),
    "pml_rank_off_by_one": ("pml[r] = v[m - 1];", "pml[r] = v[m < n ? m : m - 1];"),
    "tvar_divisor": ("tvar[r] = acc / (double)m;", "tvar[r] = acc / (double)(m + 1);"),
    "level_rank_complement": ("int64_t q = 1000000000 - a_nano;", "int64_t q = a_nano;"),
    "rp_rank_floor": ("return (n * 1000000 + rp_micro - 1) / rp_micro;", "return (n * 1000000) / rp_micro;"),
    "sort_ascending": ("return (x < y) - (x > y);", "return (x > y) - (x < y);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutant = tmp_path / "oracle_mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                           "-shared", str(mutant), "-o", str(lib), "-lm"])
    env = dict(os.environ, ARE_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake {name} passed every pin:\n{r.stdout[-2000:]}"
