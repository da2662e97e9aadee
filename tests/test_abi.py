"""The C-ABI library: it builds, loads without a GPU, exports every symbol the
header declares, and its host-only helper and argument checks behave."""

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import mlp as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hessmlp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1905_05559_gb300 import build, _lib
    build.build()
    return _lib.load()


def header_symbols():
    txt = open(HEADER).read()
    return re.findall(r"HESS_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt)


def test_header_declares_the_boundary():
    syms = set(header_symbols())
    assert {"hess_mlp_create", "per_example_grads", "opg", "exact_hessian", "opg_topk_eig"} <= syms


def test_library_exports_every_declared_symbol(lib):
    from paper_1905_05559_gb300 import _lib
    for name in header_symbols():
        assert hasattr(lib, name), name
    assert set(header_symbols()) == set(_lib.EXPORTS)


def test_param_permutation_matches_oracle(lib):
    from paper_1905_05559_gb300 import param_permutation
    for widths in ([4, 5, 3], [7, 2], [3, 6, 5, 4]):
        assert np.array_equal(param_permutation(widths), O.param_permutation(widths))


def test_create_rejects_bad_descriptions_before_touching_cuda(lib):
    from paper_1905_05559_gb300 import _lib
    h = ctypes.c_void_p()
    omega = np.zeros(43)
    w = (ctypes.c_int * 3)(4, 5, 3)
    bad_act = (ctypes.c_int * 1)(7)
    ok_act = (ctypes.c_int * 1)(0)
    cases = [
        (None, omega),
        (_lib.HessDesc(1, w, ok_act), omega),
        (_lib.HessDesc(3, w, bad_act), omega),
        (_lib.HessDesc(3, (ctypes.c_int * 3)(4, 0, 3), ok_act), omega),
        (_lib.HessDesc(3, (ctypes.c_int * 3)(4, 5, 1), ok_act), omega),
        (_lib.HessDesc(3, w, ok_act), None),
    ]
    for desc, om in cases:
        st = lib.hess_mlp_create(ctypes.byref(desc) if desc is not None else None,
                                 om.ctypes.data if om is not None else None, None, ctypes.byref(h))
        assert st == _lib.HESS_ERR_INVALID_ARG
        assert lib.hess_last_error()


def test_calls_reject_null_handle_and_bad_sizes(lib):
    from paper_1905_05559_gb300 import _lib
    x = np.zeros(8)
    assert lib.per_example_grads(None, x.ctypes.data, x.ctypes.data, 1, 0, x.ctypes.data) == \
        _lib.HESS_ERR_INVALID_ARG
    assert lib.opg(None, x.ctypes.data, x.ctypes.data, 1, 0, x.ctypes.data) == _lib.HESS_ERR_INVALID_ARG
    assert lib.exact_hessian(None, None, None, 1, 0, None) == _lib.HESS_ERR_INVALID_ARG
    assert lib.opg_topk_eig(None, None, None, 1, 1, 0, None, None) == _lib.HESS_ERR_INVALID_ARG
    assert lib.hess_mlp_num_params(None) == -1
    assert lib.hess_mlp_destroy(None) == _lib.HESS_OK
    assert lib.hess_param_permutation(1, None, None) == _lib.HESS_ERR_INVALID_ARG


def test_batch_entry_points_reject_bad_arguments_before_touching_cuda(lib):
    from paper_1905_05559_gb300 import _lib
    b = ctypes.c_void_p()
    assert lib.hess_batch_create(1 << 20, None, ctypes.byref(b)) == _lib.HESS_ERR_INVALID_ARG
    assert "workspace" in _lib.last_error()
    assert lib.hess_batch_create(1 << 30, None, None) == _lib.HESS_ERR_INVALID_ARG
    info = _lib.BatchInfo()
    assert lib.hess_batch_run(None, None, 0, 3, ctypes.byref(info)) == _lib.HESS_ERR_INVALID_ARG
    assert lib.hess_batch_destroy(None) == _lib.HESS_OK
    assert lib.hess_mlp_set_operand_limit(None, 1 << 30) == _lib.HESS_ERR_INVALID_ARG


def test_autotune_table_load_and_save_on_cpu(lib, tmp_path):
    from paper_1905_05559_gb300 import _lib
    good = tmp_path / "table.txt"
    good.write_text("# mode columns kblocks products3 width\n0 12730 16 1 192\n2 186 16 1 96\n")
    n0 = lib.hess_autotune_entries()
    assert lib.hess_autotune_load(str(good).encode()) == _lib.HESS_OK
    assert lib.hess_autotune_entries() == n0 + 2
    out = tmp_path / "saved.txt"
    assert lib.hess_autotune_save(str(out).encode()) == _lib.HESS_OK
    lines = [ln for ln in out.read_text().splitlines() if not ln.startswith("#")]
    assert "0 12730 16 1 192" in lines and "2 186 16 1 96" in lines
    bad = tmp_path / "bad.txt"
    bad.write_text("0 100 4 1 200\nnot a line\n")  # 200 is not a multiple of 16
    assert lib.hess_autotune_load(str(bad).encode()) == _lib.HESS_ERR_INVALID_ARG
    assert lib.hess_autotune_load(str(tmp_path / "missing.txt").encode()) == _lib.HESS_ERR_INVALID_ARG


def test_package_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the shared library absent, the handle classes
    raise instead of computing anything."""
    from paper_1905_05559_gb300 import _lib, api
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libhessmlp.so"))
    with pytest.raises(RuntimeError, match="missing"):
        api.HessMLP([4, 5, 3], ["sigmoid"], np.zeros(43))
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load()


def test_compute_entry_points_cite_the_paper():
    """Every compute entry point of the header carries a doc comment that
    cites the passage defining its operation."""
    txt = open(HEADER).read()
    compute = {"per_example_grads", "opg", "exact_hessian", "opg_topk_eig", "opg_topk_eig_streaming",
               "hess_curvature", "hessian_vector_products", "hessian_topk_eig", "hessian_minibatches",
               "hess_approx_form", "opg_topk_eig_lowmem"}
    prev_end, seen = 0, set()
    for m in re.finditer(r"HESS_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt):
        comments = re.findall(r"/\*.*?\*/", txt[prev_end:m.start()], re.S)
        if m.group(1) in compute:
            assert comments, m.group(1)
            assert re.search(r"Sec\. \d|Eq\. \w|Appendix", comments[-1]), m.group(1)
            seen.add(m.group(1))
        prev_end = txt.index(";", m.end()) + 1
    assert seen == compute
