"""Mutation check of the oracle pins: plant one plausible mistake at a time
in a copy of the oracle source (a dropped term, a flipped sign, a wrong
index, a transposed operand), build it, and require that at least one pin
in ``test_oracle.py`` fails on it.  The planted copies live in a temporary
directory and are only ever run on the CPU."""
import os
import subprocess

import pytest

import oracle
from oracle import build as obuild
from tests import test_oracle

# (name, old, new, which occurrence (0-based) to replace)
MUTATIONS = [
    ("tri_fwd_drop_a", "(EL(X, i, j) - a[i] * EL(X, i - 1, j))", "(EL(X, i, j))", 0),
    ("tri_bwd_sign", "EL(X, i, j) - chat[i] * EL(X, i + 1, j)", "EL(X, i, j) + chat[i] * EL(X, i + 1, j)", 0),
    ("tri_factor_index", "b[i] - a[i] * chat[i - 1];", "b[i] - a[i - 1] * chat[i - 1];", 0),
    ("tri_first_row", "EL(X, 0, j) = EL(X, 0, j) / b[0];", "EL(X, 0, j) = EL(X, 0, j);", 0),
    ("penta_alpha_drop", "al[i] = c[i] - a[i] * de[i - 2] - be[i] * ga[i - 1];", "al[i] = c[i] - be[i] * ga[i - 1];", 0),
    ("penta_gamma2_drop", "ga[1] = (d[1] - be[1] * de[0]) / al[1];", "ga[1] = d[1] / al[1];", 0),
    ("penta_delta_unscaled", "de[i] = e[i] / al[i];", "de[i] = e[i];", 0),
    ("penta_last_alpha_index", "al[i] = c[i] - a[i] * de[i - 2] - be[i] * ga[i - 1];",
     "al[i] = c[i] - a[i] * de[i - 1] - be[i] * ga[i - 1];", 2),
    ("penta_fwd_drop_eps", " - ep[i] * EL(X, i - 2, j)", "", 0),
    ("penta_bwd_index", "- de[i] * EL(X, i + 2, j)", "- de[i] * EL(X, i + 1, j)", 0),
    ("penta_bwd_skip_row", "EL(X, N - 2, j) = EL(X, N - 2, j) - ga[N - 2] * EL(X, N - 1, j);", "", 0),
    ("transpose_operand", "bands[(int64_t)(width - 1 - k) * N + r]", "bands[(int64_t)k * N + r]", 0),
    ("band_grad_sign", "dbands[(int64_t)k * N + i] = -s;", "dbands[(int64_t)k * N + i] = s;", 0),
    ("band_grad_index", "s += EL(GB, i, j) * EL(X, col, j);", "s += EL(GB, i, j) * EL(X, i, j);", 0),
    ("residual_sign", "EL(R, i, j) = EL(B, i, j) - s;", "EL(R, i, j) = EL(B, i, j) + s;", 0),
    ("periodic_corner", "bands[N + N - 1] = b[N - 1] - c[N - 1] * a[0] / g;", "bands[N + N - 1] = b[N - 1];", 0),
    ("periodic_vz_sign", "const double vz = z[0] + (a[0] / g) * z[N - 1];",
     "const double vz = z[0] - (a[0] / g) * z[N - 1];", 0),
    ("periodic_u_corner", "z[N - 1] = c[N - 1];", "z[N - 1] = a[0];", 0),
    ("periodic_grad_col", "int64_t col = (i + k - 1 + N) % N;", "int64_t col = (i + k + N) % N;", 0),
    ("periodic_grad_sign", "dbands[(int64_t)k * N + i] = -s;\n    }\n}\n\n/* -----", "dbands[(int64_t)k * N + i] = s;\n    }\n}\n\n/* -----", 0),
    ("cn_explicit_op", "F[i * M + j] = 2.0 * EL(X, i, j) - s;", "F[i * M + j] = EL(X, i, j) - s;", 0),
    ("cn_no_wrap", "if (periodic) col = (col + N) % N;", "", 0),
    ("adi_explicit_sign", "out[y * nx + x] = c0 + r * (lo - 2.0 * c0 + hi);",
     "out[y * nx + x] = c0 - r * (lo - 2.0 * c0 + hi);", 0),
    ("adi_lhs_diag", "bands[n_row + i] = 1.0 + 2.0 * r;", "bands[n_row + i] = 1.0 + r;", 0),
    ("adi_bands_no_transpose", "if (transpose)\n    oracle_transpose_bands(width, n_row, bands, s);",
     "if (0)\n    oracle_transpose_bands(width, n_row, bands, s);", 0),
    ("adi_bands_explicit_axis", "out[y * nx + x] = c0 + r * (lo - 2.0 * c0 + hi);",
     "out[y * nx + x] = c0 + r * (lo - 2.0 * c0 - hi);", 1),
]


def _replace_nth(src: str, old: str, new: str, n: int) -> str:
    idx = -1
    for _ in range(n + 1):
        idx = src.find(old, idx + 1)
        assert idx >= 0, f"mutation anchor not found: {old!r} (occurrence {n})"
    return src[:idx] + new + src[idx + len(old):]


def _pins_fail(path: str) -> list:
    failed = []
    with oracle.using_library(path):
        for name, thunk in test_oracle.all_pins():
            try:
                thunk()
            except Exception:  # assertion, OracleError, NaN comparisons ...
                failed.append(name)
    return failed


@pytest.mark.parametrize("name,old,new,occ", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(tmp_path, name, old, new, occ):
    src = open(obuild.SRC).read()
    mutated = _replace_nth(src, old, new, occ)
    c_path = os.path.join(tmp_path, "mut.c")
    so_path = os.path.join(tmp_path, f"libmut_{name}.so")
    with open(c_path, "w") as f:
        f.write(mutated)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    c_path, "-o", so_path, "-lm"], check=True)
    failed = _pins_fail(so_path)
    assert failed, f"no pin caught the planted mistake {name}"


def test_unmutated_source_passes_all_pins():
    assert _pins_fail(obuild.build()) == []
