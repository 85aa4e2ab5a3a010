"""Plant plausible mistakes in copies of the oracle and require the pins to catch each one.

Each mutant is the oracle's C source with one statement replaced (in every
function that contains it), built with gcc into a temporary directory (CPU
only).  A mutant that passes every pin
would mean the pins cannot tell that mistake from the paper's method.
"""
import os

import numpy as np
import pytest

import pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "pp_oracle.c")

MUTANTS = {
    # Kernel 1
    "k1_sorts_by_end_vertex": ("    for (uint64_t i = 0; i < M; ++i) key[i] = ((uint64_t)u[i] << 32) | v[i];\n    qsort(key, M, sizeof(uint64_t), cmp_u64);\n    for (uint64_t i = 0; i < M; ++i) {\n        u_out",
                               "    for (uint64_t i = 0; i < M; ++i) key[i] = ((uint64_t)v[i] << 32) | u[i];\n    qsort(key, M, sizeof(uint64_t), cmp_u64);\n    for (uint64_t i = 0; i < M; ++i) {\n        u_out"),
    # Kernel 2
    "k2_duplicates_not_summed": ("tc[nnz0 - 1] += 1;", "tc[nnz0 - 1] += 0;"),
    "k2_no_leaf_filter": ("if (is_max || d_in[j] == 1) zero_col[j] = 1;", "if (is_max) zero_col[j] = 1;"),
    "k2_no_supernode_filter": ("int is_max = d_in[j] == dmax &&", "int is_max = 0 && d_in[j] == dmax &&"),
    "k2_out_degree_counts_entries": ("if (!zero_col[tv[e]]) d_out[tu[e]] += tc[e];", "if (!zero_col[tv[e]]) d_out[tu[e]] += 1;"),
    "k2_divides_by_in_degree": ("val[nnz] = (double)tc[e] / (double)d_out[tu[e]];", "val[nnz] = (double)tc[e] / (double)d_in[tv[e]];"),
    "k2_leaf_means_out_degree_one": ("if (is_max || d_in[j] == 1) zero_col[j] = 1;", "if (is_max || d_in[j] == 2) zero_col[j] = 1;"),
    # Kernel 3
    "k3_teleport_without_1_over_N": ("double a = (1.0 - c) / (double)N;", "double a = (1.0 - c);"),
    "k3_transposed_matrix": ("y[col[e]] += cr * val[e];", "y[uu] += c * r[col[e]] * val[e];"),
    "k3_r0_not_normalised": ("r[i] = r0[i] / norm1;", "r[i] = r0[i];"),
    "k3_stale_sum": ("double s = sum_compensated(r, N);", "double s = 1.0;"),
    "k3_teleport_sign": ("r[vv] = y[vv] + a * s;", "r[vv] = y[vv] - a * s;"),
    "k3_damping_not_applied": ("double cr = c * r[uu];", "double cr = r[uu];"),
    # Kernel 3 variants (dangling-node term, convergence test)
    "k3ex_dangling_without_damping": ("double spread = c * dmass / (double)N;", "double spread = dmass / (double)N;"),
    "k3ex_dangling_not_over_N": ("double spread = c * dmass / (double)N;", "double spread = c * dmass;"),
    "k3ex_dangling_takes_every_row": ("if (rowptr[uu] == rowptr[uu + 1]) tmp[n++] = r[uu];", "tmp[n++] = r[uu];"),
    "k3ex_stops_one_early": ("done = it + 1;", "done = it;"),
    "k3ex_never_stops": ("            done = it + 1;\n            break;", "            done = it + 1;"),
    # edge files
    "tsv_eleven_digits": ("if (p == end || end - p > 10) return 0;", "if (p == end || end - p > 11) return 0;"),
    "tsv_trailing_text_accepted": ("if (start != len) *bad = 1;", ""),
    "tsv_overflow_accepted": ("if (x > 0xffffffffull) return 0;", ""),
    "tsv_end_vertex_dropped": ("\"%u\\t%u\\n\", (unsigned)u[i], (unsigned)v[i]", "\"%u\\t%u\\n\", (unsigned)u[i], 0u"),
}


def _all_pins(O):
    failures = []
    for name, check in pins.ALL_CHECKS:
        try:
            check(O)
        except (AssertionError, ValueError, MemoryError) as e:
            failures.append(name)
    rng = np.random.default_rng(3)
    u = rng.integers(0, 256, 3000).astype(np.uint32)
    v = rng.integers(0, 256, 3000).astype(np.uint32)
    for name, fn in (("k1_properties", lambda: pins.check_k1_properties(O, u, v)),
                     ("k2_invariants", lambda: pins.check_k2_invariants(O, u, v, 256)),
                     ("k3_mass_balance", lambda: pins.check_k3_mass_balance(O, u, v, 256))):
        try:
            fn()
        except (AssertionError, ValueError, MemoryError):
            failures.append(name)
    return failures


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_mutant_is_caught(mutant, tmp_path):
    import oracle
    from oracle import build

    old, new = MUTANTS[mutant]
    src = open(SRC).read()
    # a statement shared by the plain and the variant Kernel 3 is mutated in both
    assert src.count(old) >= 1, "mutation anchor not found in the oracle source: %s" % mutant
    msrc = tmp_path / "pp_oracle.c"
    msrc.write_text(src.replace(old, new))
    out = str(tmp_path / "liboracle_mutant.so")
    build.SRC_SAVED = build.SRC
    try:
        build.SRC = str(msrc)
        build.build(force=True, out=out)
    finally:
        build.SRC = build.SRC_SAVED
    failures = _all_pins(oracle.Oracle(out))
    assert failures, "no pin caught the planted mistake %s" % mutant


def test_unmutated_oracle_passes_all_pins():
    import oracle

    assert _all_pins(oracle.default()) == []
