"""The oracle's pins catch plausible mistakes.

Each mutant below is ``oracle.c`` with one planted error of the kinds the pins
are chosen against (a transposed operand, a dropped term, a wrong index or
bound, a wrong sign, a skipped step).  It is compiled in a temporary
directory next to a copy of the oracle's Python wrapper, and every pin of
``test_oracle_pins.py`` (the parameter-free ones and every parametrised case)
is run against it: at least one pin must fail.  The unmodified copy, built
the same way, must pass them all, so a failure is the planted error's doing.
Every mutant stays inside its arrays (no mutant reads or writes out of
bounds), so none can crash the test process.
"""

import importlib.util
import inspect
import itertools
import os
import shutil

import pytest

from tests import test_oracle_pins as pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")

# (name, text in oracle.c, its replacement); the first occurrence is replaced
MUTANTS = [
    ("transposed_K_in_csr_assembly",
     "values[slot] = values[slot] + Ke[(int64_t)r * n_loc + c];",
     "values[slot] = values[slot] + Ke[(int64_t)c * n_loc + r];"),
    ("first_element_dropped_in_csr_assembly",
     "for (int64_t t = 0; t < n_e; ++t) {", "for (int64_t t = 1; t < n_e; ++t) {"),
    ("row_candidates_not_deduplicated",
     "if (buf[k] != buf[w - 1]) buf[w++] = buf[k];", "buf[w++] = buf[k];"),
    ("crac_lookup_skips_last_run",
     "k < crac_ptr[row + 1]; k += 2)", "k + 2 < crac_ptr[row + 1]; k += 2)"),
    ("final_pair_column_off_by_one",
     "ca[w++] = (int32_t)n_cols;", "ca[w++] = (int32_t)(n_cols - 1);"),
    ("run_offset_dropped_in_crac_assembly",
     "Ke[(int64_t)r * n_loc + c + s]", "Ke[(int64_t)r * n_loc + c]"),
    ("colouring_not_first_fit",
     "int32_t k = 0;\n        while (k < cap && used[k]) ++k;",
     "int32_t k = 1;\n        while (k < cap && used[k]) ++k;"),
    ("csr_spmv_sign",
     "s = s + values[k] * x[col_idx[k]];", "s = s - values[k] * x[col_idx[k]];"),
    ("crac_spmv_run_length_off_by_one",
     "int64_t len = (int64_t)col_align[p + 3] - pos;", "int64_t len = (int64_t)col_align[p + 3] - pos - 1;"),
]


def _oracle_copy(tmp_path, name, source):
    d = tmp_path / name / "oracle"
    d.mkdir(parents=True)
    shutil.copy(os.path.join(ORACLE_DIR, "__init__.py"), d / "__init__.py")
    (d / "oracle.c").write_text(source)
    spec = importlib.util.spec_from_file_location(f"oracle_copy_{name}", d / "__init__.py",
                                                  submodule_search_locations=[str(d)])
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _pin_cases():
    """Every pin as (id, function, kwargs): parameter-free tests and each
    case of the parametrised ones (the slowest printed-size cases left out:
    the same code paths run in the smaller printed cases)."""
    cases = []
    for fname, fn in inspect.getmembers(pins, inspect.isfunction):
        if not fname.startswith("test_") or fname.endswith("_large"):
            continue
        params = list(inspect.signature(fn).parameters)
        marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        if not params:
            cases.append((fname, fn, {}))
            continue
        grids = []
        for m in marks:
            names = m.args[0]
            names = [x.strip() for x in names.split(",")] if isinstance(names, str) else list(names)
            vals = []
            for v in m.args[1]:
                if type(v).__name__ == "ParameterSet":  # a pytest.param(...) entry
                    v = v.values
                vals.append(dict(zip(names, v if len(names) > 1 else (v,))))
            grids.append(vals)
        if not grids or set(params) - set(k for g in grids for k in g[0]):
            continue  # needs a fixture: not a pure pin
        for combo in itertools.product(*grids):
            kw = {}
            for part in combo:
                kw.update(part)
            cases.append((f"{fname}{sorted(kw.items())}", fn, kw))
    return cases


def _failures(mod):
    """Ids of the pins that fail with the oracle module `mod`."""
    saved = pins.oracle
    pins.oracle = mod
    failed = []
    try:
        for cid, fn, kw in _pin_cases():
            try:
                fn(**kw)
            except Exception:  # an assertion or an oracle error: the pin caught something
                failed.append(cid)
    finally:
        pins.oracle = saved
    return failed


@pytest.fixture(scope="module")
def source():
    with open(os.path.join(ORACLE_DIR, "oracle.c")) as f:
        return f.read()


def test_unmodified_copy_passes_every_pin(tmp_path, source):
    assert len(_pin_cases()) > 40
    assert _failures(_oracle_copy(tmp_path, "unmodified", source)) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, source, name, old, new):
    assert old in source, "mutation site not found"
    mod = _oracle_copy(tmp_path, name, source.replace(old, new, 1))
    failed = _failures(mod)
    assert failed, f"no pin caught the planted mistake {name}"
