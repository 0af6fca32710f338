"""Planted mistakes in the oracle (CPU only).

Each mutant below is one plausible slip in ``oracle/spmv_oracle.c`` (a dropped
term, a wrong sign, a wrong or transposed index, an off-by-one, the printed
form of Eq. (2), a loose comparison in the D* rule). The test compiles the
mutated copy in a temporary folder, runs the pin suite
(``test_oracle_pins.py``) against it in a child process, and requires that at
least one pin fails by assertion. A control run of the unmodified source must
pass. The oracle's own file is never changed.
"""

import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
PINS = os.path.join(HERE, "test_oracle_pins.py")

# (name, text in spmv_oracle.c, replacement); each text occurs exactly once
MUTANTS = [
    # Eq. (4)
    ("sigma_sample_deviation", "double sg = sqrt(q / (double)n_rows);",
     "double sg = sqrt(q / (double)(n_rows - 1));"),
    ("mean_over_n_plus_one", "double m = s / (double)n_rows;", "double m = s / (double)(n_rows + 1);"),
    ("dmat_inverted", "*dmat = (m == 0.0) ? 0.0 : sg / m;", "*dmat = (sg == 0.0) ? 0.0 : m / sg;"),
    ("width_from_pointer", "if (len > w) w = len;", "if (len > w) w = irp[i + 1];"),
    # CRS -> COO-Row, Phase II
    ("irow_one_based", "irow[k] = i;", "irow[k] = i + 1;"),
    ("jcol_one_based", "jcol[p] = j;", "jcol[p] = j + 1;"),
    # CRS / CCS -> ELL (Fig. 3 indexing and padding)
    ("ell_slot_transposed", "int64_t slot = (int64_t)k * n_lines + i;",
     "int64_t slot = (int64_t)i * width + k;"),
    ("ell_pad_index_zero", "eidx[slot] = (len > 0) ? idx[ptr[i + 1] - 1] : 0;", "eidx[slot] = 0;"),
    ("ell_pad_negative_zero", "eval[slot] = 0.0;", "eval[slot] = -0.0;"),
    # Phase I
    ("phase1_reverse_row_order", "    for (int32_t i = 0; i < n_rows; ++i) {\n        for (int32_t k = irp[i]; k < irp[i + 1]; ++k) {\n            int32_t j = icol[k];",
     "    for (int32_t i = n_rows - 1; i >= 0; --i) {\n        for (int32_t k = irp[i]; k < irp[i + 1]; ++k) {\n            int32_t j = icol[k];"),
    ("phase1_stores_column", "icol_t[p] = i;", "icol_t[p] = icol[k];"),
    ("phase1_value_by_target", "val_t[p] = val[k];", "val_t[p] = val[p];"),
    ("phase1_cursor_not_advanced", "cnt[j] = p + 1;", "cnt[j] = p;"),
    # SpMV
    ("crs_drops_last_term", "for (int32_t k = irp[i]; k < irp[i + 1]; ++k) s += val[k] * x[icol[k]];",
     "for (int32_t k = irp[i]; k < irp[i + 1] - 1; ++k) s += val[k] * x[icol[k]];"),
    ("crs_first_column_only", "s += val[k] * x[icol[k]];", "s += val[k] * x[icol[irp[i]]];"),
    ("coo_overwrites", "y[row[k]] += val[k] * x[col[k]];", "y[row[k]] = val[k] * x[col[k]];"),
    ("ell_row_base_by_width", "int64_t base = (int64_t)k * n_rows;", "int64_t base = (int64_t)k * width;"),
    ("ell_col_wrong_sign", "y[erow[base + j]] += eval[base + j] * x[j];",
     "y[erow[base + j]] -= eval[base + j] * x[j];"),
    ("ccs_drops_first_entry", "y[icol_t[p]] += val_t[p] * x[j];",
     "y[icol_t[p]] += (p == irp_t[j]) ? 0.0 : val_t[p] * x[j];"),
    # tolerance reference
    ("neumaier_sign", "*c += (*sum - s2) + t;", "*c += (*sum - s2) - t;"),
    ("reference_drops_product_error", "            neumaier_add(&s, &c, e);\n", ""),
    ("abs_sum_signed", "neumaier_add(&a, &ca, fabs(p));", "neumaier_add(&a, &ca, p);"),
    ("reference_drops_compensation", "y_ref[i] = s + c;", "y_ref[i] = s;"),
    # more Phase I / analysis / ELL slips
    ("count_sets_instead_of_adds", "cnt[icol[k]] += 1;", "cnt[icol[k]] = 1;"),
    ("analyze_skips_last_row", "    for (int32_t i = 0; i < n_rows; ++i) {\n        int32_t len = irp[i + 1] - irp[i];",
     "    for (int32_t i = 0; i < n_rows - 1; ++i) {\n        int32_t len = irp[i + 1] - irp[i];"),
    ("ell_row_skips_last_slot", "    for (int32_t k = 0; k < width; ++k) {\n        int64_t base = (int64_t)k * n_rows;",
     "    for (int32_t k = 0; k < width - 1; ++k) {\n        int64_t base = (int64_t)k * n_rows;"),
    # Eqs. (1)-(3) and the D* rule
    ("sp_inverted", "double sp = t_crs / t_ell;", "double sp = t_ell / t_crs;"),
    ("tt_as_printed", "double tt = t_trans / t_crs;", "double tt = t_crs / t_trans;"),
    ("dstar_fail_inclusive", "if (rell[ord[t]] < c) {", "if (rell[ord[t]] <= c) {"),
    ("dstar_last_passing", "d = (t == 0) ? 0.0 : dmat[ord[t]];", "d = (t == 0) ? 0.0 : dmat[ord[t - 1]];"),
    ("dstar_sorted_descending", "while (j > 0 && dmat[ord[j - 1]] > dmat[i]) {",
     "while (j > 0 && dmat[ord[j - 1]] < dmat[i]) {"),
    ("maxpass_strict", "if (rell[i] >= c && (!found || dmat[i] > best)) {",
     "if (rell[i] > c && (!found || dmat[i] > best)) {"),
]


def _build(tmp_path, text):
    src = tmp_path / "spmv_oracle.c"
    src.write_text(text)
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(lib), str(src), "-lm"])
    return str(lib)


def _run_pins(lib):
    env = dict(os.environ, SPMVAT_ORACLE_LIB=lib)
    return subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                          env=env, capture_output=True, text=True, timeout=300, cwd=os.path.dirname(HERE))


def _source():
    with open(oracle._SRC) as f:
        return f.read()


def test_unmodified_oracle_passes_the_pins_through_the_harness(tmp_path):
    r = _run_pins(_build(tmp_path, _source()))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    src = _source()
    assert src.count(old) == 1, name
    r = _run_pins(_build(tmp_path, src.replace(old, new)))
    out = r.stdout + r.stderr
    assert r.returncode == 1 and " failed" in out, f"mutant {name} was not caught:\n{out[-2000:]}"
