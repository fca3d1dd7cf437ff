"""CPU-side checks of the compiled library: it loads and exports every C entry point."""
import ctypes
import re
import subprocess

import pytest

import paper_2305_06668_gb300 as lb
from tests.util import golden
from paper_2305_06668_gb300 import build as gpu_build


@pytest.fixture(scope="module")
def libpath():
    return gpu_build.build()


def test_library_exports_every_declared_symbol(libpath):
    declared = lb.exported_symbols()
    assert "lobpcg_create" in declared and "lobpcg_solve" in declared and "lobpcg_destroy" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", str(libpath)], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lobpcg_\w+)", out))
    missing = [s for s in declared if s not in exported]
    assert not missing, missing


def test_library_loads_and_reports_errors_without_gpu(libpath):
    L = lb.lib()
    o = lb._Options()
    assert L.lobpcg_options_default(ctypes.byref(o)) == lb.OK
    # the orthogonality threshold the paper uses in all its calculations (Sec. 4)
    assert o.tau_ortho == golden()["tau_ortho"]["value"]
    assert o.maxiter == 1000 and o.precond == lb.PREC_DIAG
    assert o.precision == lb.FP64 and o.ortho_cap == 6 and o.ortho2_cap == 4 and o.extra == 0
    assert o.autotune == 0 and o.mixed_switch == 0.0 and o.profile == 0 and o.ortho_trim == 1
    assert o.df_products == 0 and o.tc_gram == 1 and o.precond_floor == 0.0
    assert ctypes.sizeof(lb._Info) >= 8 * 6 * 2  # the info struct the binding reads
    assert L.lobpcg_options_default(None) == lb.EINVAL
    # NULL arguments are rejected before any device work
    ctx = ctypes.c_void_p()
    assert L.lobpcg_create(ctypes.byref(ctx), None, None, None) == lb.EINVAL
    assert b"NULL" in L.lobpcg_last_error(None)
    assert L.lobpcg_solve(None, 1, ctypes.c_double(1e-8), None, None, None, None, None) == lb.EINVAL
    L.lobpcg_destroy(None)  # NULL-safe
    # building blocks reject bad sizes on the host, before any device work
    assert L.lobpcg_syev2_f64(ctypes.c_int(0), None, ctypes.c_double(0.0), None, None, None) == lb.EINVAL
    assert L.lobpcg_gram_f32(ctypes.c_int64(10), ctypes.c_int(97), None, ctypes.c_int(97), ctypes.c_int(1), None,
                             ctypes.c_int(1), None, None) == lb.EINVAL
    assert L.lobpcg_spmm_csr_f32(ctypes.c_int64(10), None, None, None, ctypes.c_int64(0), ctypes.c_int(1), None,
                                 ctypes.c_int(4), None, ctypes.c_int(4), ctypes.c_int(-1), None, None) == lb.EINVAL
    # update: nseg outside 1..3, then q > 32 with valid-looking (never dereferenced) pointers
    dummy = (ctypes.c_void_p * 3)(16, 16, 16)
    w = (ctypes.c_int * 3)(4, 4, 4)
    upd = lambda nseg, q: L.lobpcg_update_f32(ctypes.c_int64(10), ctypes.c_int(nseg), dummy, None, w, ctypes.c_int(4),
                                              ctypes.c_void_p(16), ctypes.c_int(q), ctypes.c_double(1.0), None,
                                              ctypes.c_int(0), ctypes.c_void_p(16), None, ctypes.c_int(q), None, None,
                                              None)
    assert upd(4, 4) == lb.EINVAL and upd(0, 4) == lb.EINVAL
    assert upd(1, 33) == lb.EINVAL and b"q <= 32" in L.lobpcg_last_error(None)
    # tridiagonal preconditioner: NULL arrays, n < 1, p outside 1..32, ld < p
    v = ctypes.c_void_p(16)  # never dereferenced: the checks come first
    tri = lambda n, dl, p, ldr, ldw: L.lobpcg_precond_tridiag(ctypes.c_int64(n), dl, v, v, ctypes.c_int(p), v, v,
                                                              ctypes.c_int(ldr), v, ctypes.c_int(ldw), None)
    assert tri(10, None, 1, 1, 1) == lb.EINVAL and b"NULL" in L.lobpcg_last_error(None)
    assert tri(0, v, 1, 1, 1) == lb.EINVAL
    assert tri(10, v, 0, 1, 1) == lb.EINVAL and tri(10, v, 33, 33, 33) == lb.EINVAL
    assert tri(10, v, 4, 3, 4) == lb.EINVAL and tri(10, v, 4, 4, 3) == lb.EINVAL
    # switch-rule replay: NULL history with n > 0, n < 0
    out = ctypes.c_int(7)
    assert L.lobpcg_mixed_switch_replay(None, ctypes.c_int(3), ctypes.c_double(0.0), ctypes.byref(out)) == lb.EINVAL
    assert L.lobpcg_mixed_switch_replay(None, ctypes.c_int(-1), ctypes.c_double(0.0), ctypes.byref(out)) == lb.EINVAL
    assert L.lobpcg_mixed_switch_replay(None, ctypes.c_int(0), ctypes.c_double(0.0), None) == lb.EINVAL


def test_no_cpu_fallback_in_product_package():
    import pathlib
    pkg = pathlib.Path(lb.__file__).parent
    for f in list(pkg.glob("*.py")) + list((pkg / "csrc").glob("*")):
        text = f.read_text()
        assert "import oracle" not in text and "from oracle" not in text, f
        assert "lobpcg_oracle" not in text, f
