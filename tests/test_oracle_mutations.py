"""The oracle's pins must be sensitive: compile copies of the oracle with one
planted mistake each (CPU only, temporary directory) and check that at least
one pin rejects every copy."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_operator as T

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "qdvm_oracle.c")

MUTATIONS = {
    "loss_index_drops_l": ("flat_shift(c, T[t].k, T[t].l, d, N)];\n            double gain_t",
                           "flat_shift(c, T[t].k, NULL, d, N)];\n            double gain_t"),
    "loss_term_dropped": ("nsum_add(&q, -loss_t);", ""),
    "gain_operand_swapped": ("double gain_t = T[t].w * a * b;", "double gain_t = T[t].w * a * fi;"),
    "weight_without_gcd": ("return pow(h, 2 * d - 1) * sqrt(n2) / (double)g;", "return pow(h, 2 * d - 1) * sqrt(n2);"),
    "l_also_restricted": ("if (dot != 0) continue;",
                          "if (dot != 0) continue; { long gl = gcd_vec(l, d); int el[3] = {0, 0, 0};"
                          " for (int a = 0; a < d; ++a) el[a] = (int)(l[a] / gl); if (linf_vec(el, d) > m) continue; }"),
    "wrap_off_by_one": ("return r < 0 ? r + N : r;", "return r < 0 ? r + N - 1 : r;"),
}

PINS = [
    (T.test_matches_fourier_side_decomposition, [(2, 9, 3, 2, "hp"), (3, 6, 2, 1, "hp"), (2, 9, 3, 3, "unit")]),
    (T.test_two_deltas_thales_circle, [(2, 16, 3, 3, (5, 5), (7, 6)), (3, 10, 2, 1, (1, 2, 3), (3, 2, 3))]),
    (T.test_mass_conserved_for_any_data, [(2, 16, 2, "unit")]),
    (T.test_maxwellian_is_equilibrium_in_the_interior, [()]),
]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path, monkeypatch):
    a, b = MUTATIONS[name]
    src = open(SRC).read()
    assert a in src
    c_path = tmp_path / f"{name}.c"
    so_path = tmp_path / f"{name}.so"
    c_path.write_text(src.replace(a, b))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", str(c_path), "-o", str(so_path), "-lm"],
                   check=True, capture_output=True)
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: str(so_path))
    caught = False
    for fn, cases in PINS:
        for c in cases:
            try:
                fn(*c)
            except AssertionError:
                caught = True
                break
        if caught:
            break
    monkeypatch.setattr(oracle, "_lib", None)
    assert caught, f"no pin rejects the planted mistake {name}"
