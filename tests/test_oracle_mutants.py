"""Plant plausible mistakes in a copy of the oracle and check that the pins catch each one.

Each mutant is the oracle source with one textual change (a signed word compare, the word
order reversed, a dropped "minus one", a wrong run numbering, ...), compiled on the CPU and
loaded through REINDEX_ORACLE_LIB by a pytest subprocess running the oracle pins, which must
fail.  The real oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "reindex_oracle.cpp")

MUTANTS = {
    "signed_word_compare": ("    if (a[w] < b[w]) return -1;\n    if (a[w] > b[w]) return 1;",
                            "    if ((int32_t)a[w] < (int32_t)b[w]) return -1;\n"
                            "    if ((int32_t)a[w] > (int32_t)b[w]) return 1;"),
    "least_significant_word_first": ("  for (int w = 0; w < K; ++w) {\n    if (a[w]",
                                     "  for (int w = K - 1; w >= 0; --w) {\n    if (a[w]"),
    "first_word_only": ("  for (int w = 0; w < K; ++w) {\n    if (a[w]", "  for (int w = 0; w < 1; ++w) {\n    if (a[w]"),
    "new_index_off_by_one": ("    old_to_new[i] = (int32_t)(D - 1);", "    old_to_new[i] = (int32_t)(D);"),
    "head_compares_wrong_neighbour": ("key_of(words, K, order[p - 1]), K) != 0;",
                                      "key_of(words, K, order[p > 1 ? p - 2 : 0]), K) != 0;"),
    "paper_no_minus_one": ("    ni[i] = (int32_t)(run - 1);", "    ni[i] = (int32_t)(run);"),
    "paper_overwrite_with_vertex0": ("  const int64_t first = idx[0];", "  const int64_t first = 0;"),
    "paper_perm_not_inverted": ("  for (int64_t j = 0; j < N; ++j) pm[orgID[j]] = (int32_t)j;",
                                "  for (int64_t j = 0; j < N; ++j) pm[j] = orgID[j];"),
    "map_rank_by_insertion": ("      rank[kv.second] = r++;", "      rank[kv.second] = kv.second; r++;"),
    "range_check_off_by_one": ("(int64_t)idx[j] >= nVtx) return false;", "(int64_t)idx[j] > nVtx) return false;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutant = tmp_path / "mutant.cpp"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(so), str(mutant)])
    env = dict(os.environ, REINDEX_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    # exit code 1 = some pin failed (a crash would be a negative code and prove nothing)
    assert r.returncode == 1, f"mutant {name}: pytest exit {r.returncode}\n{r.stdout[-2000:]}"
