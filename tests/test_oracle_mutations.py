"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle's C source (a
dropped term, an off-by-one, a wrong comparison or order, a missing step),
compiles it, and runs the oracle pin tests against it in a subprocess; they
must fail.  Nothing here touches the CUDA path.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "burr_oracle.c")

MUTATIONS = {
    "backsub_drops_last_coefficient": ("for (int k = 1; k < 64; k++)", "for (int k = 1; k < 63; k++)"),
    "no_rollback": ("C[slot_of[q]] = 0;", "(void)0;"),
    "level_above_off_by_one": ("if (levels[i] > o) return", "if (levels[i] >= o) return"),
    "forced_level_ignored": ("int after_cut = (cut_idx < ncuts && cuts[cut_idx] == b * B);",
                             "int after_cut = 0;"),
    "ascending_insertion_order": ("if (oa != ob) return oa > ob ? -1 : 1;",
                                  "if (oa != ob) return oa < ob ? -1 : 1;"),
    "coefficient_missing_pivot_bit": ("*coeff = or_mix64(h + sigma) | 1ULL;", "*coeff = or_mix64(h + sigma);"),
    "bumped_emission_off_by_one": ("if ((uint32_t)(rows[k].start % B) < t) {",
                                   "if ((uint32_t)(rows[k].start % B) <= t) {"),
    "query_window_shifted": ("v ^= or_zbit(z, r, s + (uint64_t)k, q) << q;",
                             "v ^= or_zbit(z, r, s + (uint64_t)k + 1, q) << q;"),
    "range_reduction_wrong": ("*start = or_mulhi(h, m - w + 1);", "*start = or_mulhi(h, m - w);"),
    "value_not_xored": ("y ^= Y[p];", "(void)0;"),
    "exact_threshold_off_by_one": ("t = off + 1;                 /* rows at offsets >= t were all kept */",
                                   "t = off;"),
    "exact_threshold_not_stored": ("texact[b] = (uint8_t)t;", "texact[b] = (uint8_t)(t ? 1 : 0);"),
    "exact_forced_threshold_too_small": ("const uint32_t t_forced = mode == OR_THRESH_1PLUS ? w :",
                                         "const uint32_t t_forced = mode == OR_THRESH_1PLUS ? w - 1 :"),
    "cut_search_prev_window_too_wide": ("if (off >= B - (w - 1)) hi[s / B]++;", "if (off >= B - w) hi[s / B]++;"),
    "cut_search_keeps_last_best": ("if (b == b0 || score < best)", "if (b == b0 || score <= best)"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-I",
                           os.path.join(ROOT, "oracle"), "-o", str(lib), str(mut), "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(lib))
    pins = ["tests/test_oracle_hash.py", "tests/test_oracle_bruteforce.py", "tests/test_oracle_invariants.py",
            "tests/test_oracle_cut_search.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake '{name}' was not caught:\n{r.stdout[-2000:]}"
