"""CPU-side checks of the C ABI: the library builds, loads and exports every
function that include/lindblad_ss.h declares; host-side marshalling."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lindblad_ss.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:[A-Za-z_]\w*[\s\*]+)+([A-Za-z_]\w*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return")))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1504_06768_gb300 import _binding
    return _binding.load()


def test_header_parses():
    names = _declared_functions()
    for must in ("assemble_liouvillian", "rcm_permute", "ilu_factor", "steady_state", "add_trace_row",
                 "add_shift", "permute", "krylov_solve", "lgmres_solve", "spmv", "precond_apply", "ss_ctx_create"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_declares_every_header_function():
    from paper_1504_06768_gb300 import _binding
    assert sorted(_binding.exported_names()) == _declared_functions()


def test_nm_shows_c_linkage(lib):
    from paper_1504_06768_gb300 import _binding
    out = subprocess.run(["nm", "-D", "--defined-only", _binding.LIB_PATH], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in _declared_functions():
        assert name in syms, f"{name} not exported with C linkage"


def test_no_gpu_context_fails_cleanly(lib):
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.ss_ctx_create(0, None, ctypes.byref(h)) != 0
    assert h.value is None


def test_options_defaults(lib):
    import ctypes
    from paper_1504_06768_gb300 import _binding as B
    o = B.Options()
    o.lgmres_k, o.inner_rtol, o.warm_start = 77, 9.0, 5   # the last fields: written at the offsets the header gives
    lib.ss_options_default(ctypes.byref(o))
    assert (o.method, o.precond, o.precision, o.maxiter, o.restart, o.use_rcm) == (2, 0, 0, 1000, 30, 1)
    assert o.tol == 1e-10 and o.sigma == 1e-15 and o.drop_tol == 1e-4 and o.fill_factor == 10.0
    assert o.inner_rtol == 1e-5 and o.lgmres_k == 0 and o.warm_start == 0
    assert B.METHODS["auto"] == 4 and B.METHOD_NAMES[B.METHODS["iterative-lgmres"]] == "iterative-lgmres"


def test_csr_marshalling_sorts_and_keeps_arrays():
    import scipy.sparse as sp
    from paper_1504_06768_gb300 import _CsrHost
    m = sp.csr_matrix((np.array([1 + 2j, 3.0, 4j]), np.array([2, 0, 1]), np.array([0, 2, 3])), shape=(2, 3))
    h = _CsrHost(m)
    assert h.view.n_rows == 2 and h.view.n_cols == 3 and h.view.nnz == 3
    assert h.col.tolist() == [0, 2, 1] and h.val.tolist() == [3.0, 1 + 2j, 4j]
    assert h.view.row_ptr == h.rp.ctypes.data and h.view.on_device == 0
