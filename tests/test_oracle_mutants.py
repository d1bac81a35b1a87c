"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake in a private copy of md_oracle.c (a dropped term, a
wrong bound, an index off by one, a transposed comparison), builds it on the CPU, and
runs the pin suite (tests/test_oracle_pins.py) against that build in a subprocess.  The
suite must fail for every mutant.  The real oracle source is never modified.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "md_oracle.c")

MUTANTS = {
    "colex_reset_off_by_one": ("for (int t = 0; t < i; t++) c[t] = t;", "for (int t = 0; t < i; t++) c[t] = t + (t > 0);"),
    "colex_rank_position": ("r += mdo_binomial(c[i], i + 1);", "r += mdo_binomial(c[i], i);"),
    "unrank_comparison": ("while (mdo_binomial(v, i) > rank) v--;", "while (mdo_binomial(v, i) >= rank && v > 0) v--;"),
    "bound_drops_plus_one": ("int64_t t = (int64_t)g + 1 - (k - kj);", "int64_t t = (int64_t)g - (k - kj);"),
    "bound_sign": ("int64_t t = (int64_t)g + 1 - (k - kj);", "int64_t t = (int64_t)g + 1 + (k - kj);"),
    "stop_check_strict": ("if (L >= U) { stop = 1; break; }", "if (L > U) { stop = 1; break; }"),
    "no_per_matrix_check": ("if (L >= U) { stop = 1; break; }", "(void)0;"),
    "last_rank_not_first": ("if (w < J->minw) { J->minw = w; J->first = rank; }", "if (w <= J->minw) { J->minw = w; J->first = rank; }"),
    "echelon_not_reduced": ("            if (t != r && get_bit(Gam + (size_t)t * nw, col)) xor_row(Gam + (size_t)t * nw, Gam + (size_t)r * nw, nw);",
                            "            if (t > r && get_bit(Gam + (size_t)t * nw, col)) xor_row(Gam + (size_t)t * nw, Gam + (size_t)r * nw, nw);"),
    "words_truncated": ("static int words_for(int n) { return (n + 63) / 64; }", "static int words_for(int n) { return n / 64 + (n < 64); }"),
    "gray_code_bit": ("int b = __builtin_ctzll(i);", "int b = __builtin_ctzll(i) ^ (__builtin_ctzll(i) == 1);"),
    "skip_last_gamma": ("        for (int j = 0; j < m; j++) {\n            int w; uint64_t first;", "        for (int j = 0; j < m - (m > 1); j++) {\n            int w; uint64_t first;"),
    "witness_drops_row": ("for (int i = 0; i < key_g; i++) xor_row(witness", "for (int i = 1; i < key_g; i++) xor_row(witness"),
    "info_set_not_greedy": ("for (int q = 0; q < nrem && r < k; q++) {\n            int col = remaining[q];", "for (int q = 0; q < nrem && r < k; q++) {\n            int col = remaining[nrem - 1 - q];"),
    "per_matrix_bound_too_strong": ("L += set_bound(i <= j ? g : g - 1, k, ranks[i]);", "L += set_bound(g, k, ranks[i]);"),
    "partial_set_rank_off": ("            ranks[m++] = r;\n", "            ranks[m++] = r - (r > 1);\n"),
    "weight_ignores_column0": ("for (int i = 0; i < nw; i++) w += __builtin_popcountll(row[i]);", "for (int i = 0; i < nw; i++) w += __builtin_popcountll(row[i] & (i ? ~0ull : ~1ull));"),
    # the threaded parts: ranges split across threads and the results combined
    "scan_threads_keep_later_tie": ("if (jobs[t].minw < bw) { bw = jobs[t].minw; br = jobs[t].first; }",
                                    "if (jobs[t].minw <= bw) { bw = jobs[t].minw; br = jobs[t].first; }"),
    "scan_ranges_shifted": ("jobs[t].r0 = r0 + span / nthreads * t + ((uint64_t)t < span % nthreads ? (uint64_t)t : span % nthreads);",
                            "jobs[t].r0 = r0 + span / nthreads * t + ((uint64_t)t < span % nthreads ? (uint64_t)t : span % nthreads) - (t > 0);"),
    # the stage loop's bookkeeping and outputs
    "codewords_count": ("evaluated += count;", "evaluated += count - (j > 0);"),
    "stage_bound_lags": ("        for (int j = 0; j < m; j++) L += set_bound(g, k, ranks[j]);",
                         "        for (int j = 0; j < m; j++) L += set_bound(g - 1, k, ranks[j]);"),
    "witness_from_matrix0": ("xor_row(witness, Gam + ((size_t)key_j * k + c[i]) * nw, nw);",
                             "xor_row(witness, Gam + ((size_t)0 * k + c[i]) * nw, nw);"),
    "stop_after_g_late": ("if (stop_after_g > 0 && g >= stop_after_g) break;", "if (stop_after_g > 0 && g > stop_after_g) break;"),
    "key_ties_later": ("if (w < U) { U = w; key_g = g; key_j = j; key_rank = first; }",
                       "if (w <= U) { U = w; key_g = g; key_j = j; key_rank = first; }"),
    "per_matrix_bound_off_by_one_matrix": ("L += set_bound(i <= j ? g : g - 1, k, ranks[i]);",
                                           "L += set_bound(i < j ? g : g - 1, k, ranks[i]);"),
    "level_count_field": ("rec[4] = (int64_t)count;", "rec[4] = (int64_t)count - (g > 1);"),
    "scan_empty_weight": ("J->minw = J->n + 1;", "J->minw = J->n;"),
    "colex_next_limit": ("int limit = (i + 1 < g) ? c[i + 1] : k;", "int limit = (i + 1 < g) ? c[i + 1] : k - 1;"),
    "bruteforce_rank_check": ("if (dist[0] > 1) return 0;", "if (dist[0] > 2) return 0;"),
    # the information sets (Section 2.1 as read here: leftover columns form the last set)
    "rank1_last_set_dropped": ("        if (r > 0) {\n            for (int q = 0; q < nrem; q++)",
                               "        if (r > 1) {\n            for (int q = 0; q < nrem; q++)"),
    "full_set_order_rest_descending": ("            for (int col = 0; col < n; col++) if (!in_set[col]) order[pos++] = col;\n            ranks[m++] = k;",
                                       "            for (int col = n - 1; col >= 0; col--) if (!in_set[col]) order[pos++] = col;\n            ranks[m++] = k;"),
    "partial_set_order_rest_descending": ("            for (int col = 0; col < n; col++) if (!in_set[col]) order[pos++] = col;\n            ranks[m++] = r;",
                                          "            for (int col = n - 1; col >= 0; col--) if (!in_set[col]) order[pos++] = col;\n            ranks[m++] = r;"),
    "gamma_pivot_search_from_row0": ("    for (int p = 0; p < n && r < k; p++) {\n        int col = order[p];\n        int s = -1;\n        for (int t = r; t < k; t++)",
                                     "    for (int p = 0; p < n && r < k; p++) {\n        int col = order[p];\n        int s = -1;\n        for (int t = 0; t < k; t++)"),
    "bz_skips_stage_k": ("for (int g = 1; g <= k && !stop; g++) {", "for (int g = 1; g < k && !stop; g++) {"),
    "unrank_top_low": ("    int top = k - 1;\n    for (int i = g; i >= 1; i--) {\n        int v = top;",
                       "    int top = k - 2;\n    for (int i = g; i >= 1; i--) {\n        int v = top;"),
    "scan_range_not_clamped": ("    if (r1 > total) r1 = total;\n    if (r0 > r1) r0 = r1;\n    if (nthreads < 1) nthreads = 1;\n    if (nthreads > 256) nthreads = 256;\n    uint64_t span",
                               "    if (r0 > r1) r0 = r1;\n    if (nthreads < 1) nthreads = 1;\n    if (nthreads > 256) nthreads = 256;\n    uint64_t span"),
    "info_sets_skip_rank_check": ("    if (mdo_rank(G, n, k) != k) return MDO_ERANK;\n    int used", "    int used"),
    "bz_starts_at_L0": ("    int64_t L = 1;\n", "    int64_t L = 0;\n"),
    "bruteforce_thread_start_not_gray": ("uint64_t x = J->lo ^ (J->lo >> 1);", "uint64_t x = J->lo;"),
    "bruteforce_ranges_shifted": ("jobs[t].lo = total / nthreads * t + (t < (int)(total % nthreads) ? t : total % nthreads);",
                                  "jobs[t].lo = total / nthreads * t + (t < (int)(total % nthreads) ? t : total % nthreads) - (t > 0);"),
    "bruteforce_ranges_overlap": ("jobs[t].hi = jobs[t].lo + total / nthreads + (t < (int)(total % nthreads) ? 1 : 0);",
                                  "jobs[t].hi = jobs[t].lo + total / nthreads + (t < (int)(total % nthreads) ? 1 : 0) + (t + 1 < nthreads);"),
}


def _build_mutant(name, tmpdir):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor for %s must occur exactly once" % name
    path = os.path.join(tmpdir, name + ".c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(tmpdir, name + ".so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", path, "-o", lib], check=True)
    return lib


def _pins_fail(lib):
    env = dict(os.environ, MDO_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    return r.returncode != 0, r.stdout[-2000:]


def test_every_mutant_is_caught(tmp_path):
    libs = {name: _build_mutant(name, str(tmp_path)) for name in MUTANTS}
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = dict(zip(libs, ex.map(_pins_fail, libs.values())))
    survivors = [name for name, (failed, _) in results.items() if not failed]
    assert not survivors, "mutants not caught by the pins: %s" % survivors
