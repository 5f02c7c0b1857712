"""Each plausible mistake planted in a copy of the oracle must fail a pin.

The copies are built from the committed oracle source with one textual edit
each, compiled on the CPU into a temporary directory; the committed oracle is
never modified.  This shows the pins are sharp enough to catch a dropped
term, a wrong sign or index, or a transposed operand.
"""
import os

import pytest

import oracle
from oracle_pins import ALL_PINS, pin_lower_bound_exhaustive

MUTANTS = {
    # Eq. 1 case 2: wrong sign of the shift
    "case2_sign": ("q = j - i;", "q = j + i;"),
    # Eq. 1 case 3: off by one
    "case3_off_by_one": ("q = j + i - E - 1;", "q = j + i - E;"),
    # Eq. 1 case 4: out-of-range Q index treated as a match
    "case4_match": ("if (q < 1 || q > m)\n        return 1;",
                    "if (q < 1 || q > m)\n        return 0;"),
    # transposed operands of the comparison
    "transposed": ("base_of(Q[q - 1]) == base_of(R[j - 1])",
                   "base_of(R[q - 1]) == base_of(Q[j - 1])"),
    # run length counts the obstacle too
    "run_includes_obstacle": (
        "        if (sso_cell(Q, R, m, E, i, j) != 0)\n            break;\n"
        "        ++len;",
        "        ++len;\n        if (sso_cell(Q, R, m, E, i, j) != 0)\n"
        "            break;"),
    # step (2) keeps only the main diagonal
    "main_diagonal_only": ("if (len > longest)",
                           "if (i == E + 1 && len > longest)"),
    # step (3) skips one column too many
    "checkpoint_skip": ("checkpoint = checkpoint + longest + 1;",
                        "checkpoint = checkpoint + longest + 2;"),
    # an obstacle counted on reaching the destination
    "count_at_end": ("if (checkpoint + longest > m) {\n"
                     "            st.columns += m - checkpoint + 1;\n"
                     "            break;",
                     "if (checkpoint + longest > m) {\n"
                     "            st.columns += m - checkpoint + 1;\n"
                     "            count += 1;\n            break;"),
    # step (4) never stops (uncapped count reported)
    "no_early_stop": ("if (stop_above_E && count > E)",
                      "if (stop_above_E && 0)"),
    # step (4) stops one obstacle early
    "stop_at_E": ("if (stop_above_E && count > E)",
                  "if (stop_above_E && count >= E)"),
    # step (5) strict comparison
    "accept_strict": ("*accept = (uint8_t)(count <= E);",
                      "*accept = (uint8_t)(count < E);"),
    # Levenshtein: free insertions
    "ed_free_insert": ("int64_t ins = cur[y - 1] + 1;",
                       "int64_t ins = cur[y - 1];"),
    # Levenshtein: substitution always costs 1
    "ed_sub_always": (
        "prev[y - 1] + (same_symbol(a[x - 1], b[y - 1]) ? 0 : 1);",
        "prev[y - 1] + 1;"),
    # packed format: planes swapped
    "pack_planes_swapped": (
        "(lo << (j % 16)) | (hi << (16 + j % 16))",
        "(hi << (j % 16)) | (lo << (16 + j % 16))"),
    # sub-maze: one column too wide (sub-mazes overlap)
    "submaze_off_by_one": (
        "const int64_t last = first + t - 1 < m ? first + t - 1 : m;",
        "const int64_t last = first + t < m ? first + t : m;"),
    # sub-maze: the segment cap ignored
    "submaze_no_cap": ("while (checkpoint <= last && segments < y) {",
                       "while (checkpoint <= last) {"),
    # unequal lengths: the leading/trailing case-4 obstacles still counted
    "unequal_no_correction": ("        return mQ == mR ? 1 : 0;",
                              "        return 1;"),
    # unequal lengths: the correction applied to equal lengths too
    "unequal_always": ("        return mQ == mR ? 1 : 0;",
                       "        return 0;"),
    # unequal lengths: only the trailing ones deducted
    "unequal_trailing_only": (
        "    if (q < 1 || q > mQ)\n        return mQ == mR ? 1 : 0;",
        "    if (q < 1)\n        return 1;\n"
        "    if (q > mQ)\n        return mQ == mR ? 1 : 0;"),
    # unequal lengths: only the leading ones deducted
    "unequal_leading_only": (
        "    if (q < 1 || q > mQ)\n        return mQ == mR ? 1 : 0;",
        "    if (q > mQ)\n        return 1;\n"
        "    if (q < 1)\n        return mQ == mR ? 1 : 0;"),
    # unequal lengths: columns over the query instead of the reference
    "unequal_columns_over_query": (
        "            for (int64_t j = checkpoint; j <= mR; ++j) {\n"
        "                if (sso_cell2",
        "            for (int64_t j = checkpoint; j <= mQ; ++j) {\n"
        "                if (sso_cell2"),
    # bit-sliced packer: groups and blocks swapped in the word index
    "sliced_index_swapped": ("out[((j / 4 * G + g) * 2 + b) * 4 + j % 4]",
                             "out[((g * ((m + 3) / 4) + j / 4) * 2 + b) * 4"
                             " + j % 4]"),
    # bit-sliced packer: the two code bits' planes swapped
    "sliced_planes_swapped": ("out[((j / 4 * G + g) * 2 + b) * 4 + j % 4]",
                              "out[((j / 4 * G + g) * 2 + 1 - b) * 4"
                              " + j % 4]"),
    # min-obstacle DP: a segment may hold two obstacles
    "dp_two_obstacles": (
        "                if (sso_cell(Q, R, m, E, i, e) != 0)\n"
        "                    break; /* a segment holds at most one obstacle */",
        "                if (sso_cell(Q, R, m, E, i, e) != 0 && e > c)\n"
        "                    break; /* a segment holds at most one obstacle */"),
}


def _mutant(tmp_path_factory, name):
    old, new = MUTANTS[name]
    with open(oracle.SOURCE) as f:
        src = f.read()
    assert src.count(old) >= 1, f"mutation site of {name} not found"
    src = src.replace(old, new)
    d = tmp_path_factory.mktemp(name)
    path = os.path.join(str(d), "ss_oracle.c")
    with open(path, "w") as f:
        f.write(src)
    lib = oracle.compile_oracle(path, os.path.join(str(d), "libmut.so"),
                                include_dir=os.path.dirname(oracle.SOURCE))
    return oracle.Oracle(lib)


def _caught(O):
    failed = []
    for pin in ALL_PINS:
        try:
            if pin is pin_lower_bound_exhaustive:
                pin(O, mmax=3, Emax=2)
            else:
                pin(O)
        except (AssertionError, ValueError) as e:
            failed.append((pin.__name__, repr(e)[:80]))
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path_factory, name):
    O = _mutant(tmp_path_factory, name)
    failed = _caught(O)
    assert failed, f"planted mistake {name} passed every pin"
