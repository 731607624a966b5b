"""The oracle's pins must catch plausible mistakes.

Each case copies the oracle source, plants one mistake in the copy (a dropped
term, a wrong comparison, a wrong index, a wrong tie rule), compiles it on the
CPU and runs the pins of test_oracle_pins.py, test_oracle_weighted_pins.py and
test_oracle_lsh_pins.py against it: at least one pin must fail. The real oracle is restored afterwards.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle
import test_oracle_lsh_pins as lpins
import test_oracle_pins as pins
import test_oracle_weighted_pins as wpins

SRC = os.path.join(os.path.dirname(oracle.__file__), "scan_oracle.cpp")
LSH = os.path.join(os.path.dirname(oracle.__file__), "lsh_oracle.cpp")

MUTANTS = {
    "cosine without the closed +1": ("const int64_t prod = (du + 1) * (dv + 1);",
                                     "const int64_t prod = du * dv;"),
    "jaccard union without -c": ("return (double)c / (double)(du + 1 + dv + 1 - c);",
                                 "return (double)c / (double)(du + 1 + dv + 1);"),
    "count misses v itself": ("int64_t c = mark[v];  // v itself is in N̄(v)",
                              "int64_t c = 0;"),
    "strict eps in the core test": ("ne += sim[i] >= eps;", "ne += sim[i] > eps;"),
    "core order membership off by one": ("[&](int32_t v) { return deg_of(off, v) + 1 < mu; }",
                                         "[&](int32_t v) { return deg_of(off, v) < mu; }"),
    "border takes the least similar core": (
        "if (core[no_id[i]]) { labels[v] = dsu.find(no_id[i]); break; }",
        "if (core[no_id[i]]) { labels[v] = dsu.find(no_id[i]); }"),
    "union hooks to the larger root": ("if (a < b) p[b] = a; else p[a] = b;",
                                       "if (a > b) p[b] = a; else p[a] = b;"),
    "hub with a single neighbouring cluster": ("else if (l != first) { hub = true; break; }",
                                               "else { hub = true; break; }"),
    "weighted norm without the square (the listing's garble)": (
        "for (double y : wa) s2 += y * y;", "for (double y : wa) s2 += y;"),
    "weighted closed list without the vertex itself": (
        "    if (!self_done) {\n      ids.push_back((int32_t)x);\n      ws.push_back(1.0);\n    }",
        "    (void)self_done;"),
    "weighted per-vertex norm without the square": (
        "s2 += w[i] * w[i];", "s2 += w[i];"),
    "weighted per-vertex numerator without the x = u term": (
        "if (in_v[u]) num += 1.0 * wv[u];  // x = u, w(u,u) = 1", "(void)0;"),
    # mistakes in lsh_oracle.cpp
    "weighted SimHash ignores the weights": (
        "lsh", "s[j] += ((bits >> (j % 64)) & 1u) ? wx : -wx;",
        "s[j] += ((bits >> (j % 64)) & 1u) ? 1.0 : -1.0;"),
    "weighted SimHash without the vertex itself": (
        "lsh", "const double wx = i < off[v] ? 1.0 : w[i];", "const double wx = i < off[v] ? 0.0 : w[i];"),
    "weighted SimHash strict sign": ("lsh", "if (s[j] >= 0.0) out", "if (s[j] > 0.0) out"),
    "neighbour order ascending": (
        "return a.first > b.first;\n                     });\n    for (size_t j",
        "return a.first < b.first;\n                     });\n    for (size_t j"),
}

PINS = [
    lambda: pins.test_counts_equal_dense_square(25, 0.2, 2),
    pins.test_triangle_identity,
    pins.test_clique_all_one,
    lambda: pins.test_star(7),
    pins.test_bridged_cliques_hub,
    pins.test_sigma_exactly_eps_counts,
    pins.test_isolated_vertices_are_outliers,
    pins.test_vertex_next_to_one_cluster_is_outlier,
    pins.test_worked_example_sigma,
    pins.test_figure_captions,
    lambda: pins.test_order_invariants(oracle.COSINE),
    pins.test_exhaustive_five_vertices,
    lambda: wpins.test_weighted_equals_matrix_identity(30, 0.2, 1),
    wpins.test_unit_weights_reduce_to_cosine,
    wpins.test_weighted_triangle_closed_form,
    lambda: wpins.test_vertex_routine_equals_matrix_identity_and_all_arcs(1),
    wpins.test_weighted_bipartite_closed_form,
    lpins.test_weighted_simhash_unit_weights_equal_unweighted,
    lpins.test_weighted_simhash_brute_force_definition,
    lpins.test_weighted_simhash_tracks_weighted_cosine,
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    spec = MUTANTS[name]
    which, old, new = spec if len(spec) == 3 else ("scan", *spec)
    target, other = (SRC, LSH) if which == "scan" else (LSH, SRC)
    text = open(target).read()
    assert text.count(old) == 1, name
    (tmp_path / os.path.basename(target)).write_text(text.replace(old, new))
    shutil.copy(other, tmp_path / os.path.basename(other))
    mutated = tmp_path / "scan_oracle.cpp"
    so = tmp_path / "libmutant.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", str(mutated),
                    str(tmp_path / "lsh_oracle.cpp"), "-o", str(so)], check=True)
    saved = oracle._load()
    oracle._lib = oracle.bind(ctypes.CDLL(str(so)))
    caught = []
    try:
        for pin in PINS:
            try:
                pin()
            except (AssertionError, RuntimeError, ValueError, IndexError):
                caught.append(pin)
                break
    finally:
        oracle._lib = saved
    assert caught, f"no pin caught the mutant '{name}'"
