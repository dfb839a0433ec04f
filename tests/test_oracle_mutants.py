"""Planted mistakes in copies of the oracle must each fail at least one pin.

Each case copies oracle.c, makes one plausible mistake in the copy (a wrong
cost, a dropped term, an off-by-one, a missing saturation, a wrong rounding in
Eq. 1 ...), compiles it and runs the pin suite against it.  The real oracle is
never modified.
"""
import os
import shutil

import pytest

import oracle
import pins

MUTANTS = {
    "lev_sub_cost": ("int64_t sub = prev[j - 1] + (a[i - 1] != b[j - 1]);\n            cur[j] = min3",
                     "int64_t sub = prev[j - 1] + (a[i - 1] == b[j - 1]);\n            cur[j] = min3"),
    "lev_no_insertion": ("cur[j] = min3(prev[j] + 1, cur[j - 1] + 1, sub);",
                         "cur[j] = min3(prev[j] + 1, prev[j] + 1, sub);"),
    "lev_first_row": ("    for (int64_t j = 0; j <= m; j++)\n        prev[j] = j;\n",
                      "    for (int64_t j = 0; j <= m; j++)\n        prev[j] = 0;\n"),
    "ham_skips_last": ("    for (int64_t i = 0; i < n; i++)\n        if (a[i] != b[i])\n            d++;",
                       "    for (int64_t i = 0; i + 1 < n; i++)\n        if (a[i] != b[i])\n            d++;"),
    "occh_half_split": ("(i >= half ? 1 : 0)", "(i > half ? 1 : 0)"),
    "occh_interleave": ("fp |= (uint32_t)1 << (2 * q + (i >= half ? 1 : 0));",
                        "fp |= (uint32_t)1 << (q + (i >= half ? 16 : 0));"),
    "count_no_saturation": ("v = cnt[q] < (int64_t)sat ? (uint32_t)cnt[q] : sat;",
                            "v = (uint32_t)cnt[q] & sat;"),
    "count_gray_wrong": ("v = v ^ (v >> 1);", "v = v ^ (v << 1);"),
    "pos_no_saturation": ("v = i < (int64_t)sat ? (uint32_t)i : sat;", "v = (uint32_t)i;"),
    "pos_last_occurrence": ("                v = i < (int64_t)sat ? (uint32_t)i : sat;\n                break;",
                            "                v = i < (int64_t)sat ? (uint32_t)i : sat;"),
    "pos_occ_bit_offset": ("fp |= (uint32_t)1 << (p * n_pos + (q - n_pos));", "fp |= (uint32_t)1 << (p * n_pos + q);"),
    "fd_pos_counts_bits": ("        if ((x >> (p * j)) & fmask)\n            f++;",
                           "        f += weight((x >> (p * j)) & fmask);"),
    "eq1_floor": ("if ((f + 1) / 2 > J->k)", "if (f / 2 > J->k)"),
    "eq1_off_by_one": ("if ((f + 1) / 2 > J->k)", "if ((f + 1) / 2 >= J->k)"),
    "strip_too_narrow": ("int64_t hi = i + k < m ? i + k : m;", "int64_t hi = i + k - 1 < m ? i + k - 1 : m;"),
    "ham_within_early": ("if (a[i] != b[i] && ++e > k)", "if (a[i] != b[i] && ++e >= k)"),
    "symbol_tie_break": ("(cnt[order[j]] == cnt[c] && order[j] > c)", "(cnt[order[j]] == cnt[c] && order[j] < c)"),
    "rare_order": ("(cnt[rorder[j]] > cnt[c] ||", "(cnt[rorder[j]] < cnt[c] ||"),
    "prune_too_much": ("if (J->prune && (m - n > J->k || n - m > J->k))",
                       "if (J->prune && (m - n >= J->k || n - m > J->k))"),
    "l1_signed": ("f += ca > cb ? ca - cb : cb - ca;", "f += ca - cb;"),
    "l1_skips_last_field": ("for (int q = 0; (q + 1) * bits <= width; q++) {",
                            "for (int q = 0; (q + 2) * bits <= width; q++) {"),
    "l1_as_weight": ("        return orc_fd_count_l1(a, b, width, bits);\n    return orc_fd",
                     "        return orc_fd(a, b, ORC_OCC, width, 0, 0);\n    return orc_fd"),
    "qgram_last_position": ("for (int64_t i = 0; i + q <= n; i++)\n        for (int f = 0;",
                            "for (int64_t i = 0; i + q < n; i++)\n        for (int f = 0;"),
    "qgram_tie_break": ("if (cnt[c] > bc) {", "if (cnt[c] >= bc) {"),
    "qgram_filter_bound_2k": ("int div = 2 * J->qmul;", "int div = 2;"),
    "qgram_sweep_bound_2k": ("int div = 2 * q;", "int div = 2;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique / not found"
    mut_src = tmp_path / "oracle.c"
    mut_src.write_text(src.replace(old, new))
    so = oracle.build(force=True, src=str(mut_src), out=str(tmp_path / "liboracle_mut.so"))
    orc = oracle.Oracle(so)
    caught = None
    for check in pins.ALL_CHECKS:
        try:
            if check is pins.check_bound_sweep:
                check(orc, max_len=4, n_random_maps=1)
            else:
                check(orc)
        except AssertionError:
            caught = check.__name__
            break
    assert caught is not None, f"planted mistake {name} passed every pin"
