"""The C-ABI library builds, loads and exports every entry point declared in
include/sgagg.h; argument errors come back as statuses before any GPU work
(so these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_00152_gb300 import build, sgagg
    build.build()
    return sgagg.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sgagg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sgagg_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("sgagg_create", "sgagg_aggregate", "sgagg_temp_bytes", "sgagg_result_rows",
                 "sgagg_stats", "sgagg_aggregate_batched", "sgagg_destroy", "sgagg_last_error",
                 "sgagg_aggregate_host", "sgagg_set_option"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2010_00152_gb300 import sgagg
    out = subprocess.check_output(["nm", "-D", "--defined-only", sgagg.LIB_PATH]).decode()
    exported = set(re.findall(r"\bT (sgagg_\w+)", out))
    for name in declared_symbols():
        assert name in exported, name
        assert hasattr(lib, name)


def test_library_is_native_sm103a():
    from paper_2010_00152_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.flags())


def test_create_rejects_bad_budget(lib):
    from paper_2010_00152_gb300 import sgagg
    h = ctypes.c_void_p()
    assert lib.sgagg_create(0, ctypes.byref(h)) == sgagg.SGAGG_EINVAL
    assert lib.sgagg_create(-5, ctypes.byref(h)) == sgagg.SGAGG_EINVAL
    assert lib.sgagg_create(10, None) == sgagg.SGAGG_EINVAL
    assert lib.sgagg_temp_bytes(None) == -1


def _call(h, key_bytes=(8,), n=10, aggs=((0, 0),), n_pay=1, key_ptrs=None, pay_ptrs=None, cap=10,
          out_null=False):
    from paper_2010_00152_gb300 import sgagg
    kp = key_ptrs if key_ptrs is not None else [0x1000] * len(key_bytes)
    pp = pay_ptrs if pay_ptrs is not None else [0x2000] * n_pay
    ok = [0 if out_null else 0x3000] * len(key_bytes)
    oa = [0x4000] * len(aggs)
    a = sgagg._Args(kp, list(key_bytes), pp, list(aggs), ok, oa)
    return sgagg.lib().sgagg_aggregate(h, ctypes.byref(a.keys), a.pay, len(pp), n, ctypes.byref(a.spec),
                                       a.ok, a.oa, cap, None)


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_2010_00152_gb300 import sgagg
    h = sgagg.sgagg_create(100)
    try:
        E = sgagg.SGAGG_EINVAL
        assert _call(h, key_bytes=(8, 1)) == E                 # 72-bit key
        assert _call(h, key_bytes=(3,)) == E                   # bad width
        assert _call(h, n=-1) == E
        assert _call(h, aggs=((1, 3),)) == E                   # column out of range
        assert _call(h, aggs=((9, 0),)) == E                   # bad op
        assert _call(h, key_ptrs=[0]) == E                     # null key column
        assert _call(h, aggs=((1, 0),), pay_ptrs=[0]) == E     # null payload column
        assert _call(h, out_null=True) == E                    # null output column
        assert _call(h, cap=-1) == E
        assert "key" in sgagg.sgagg_last_error(h) or sgagg.sgagg_last_error(h)
        # options
        with pytest.raises(sgagg.SgaggError):
            sgagg.sgagg_set_option(h, 99, 1)
        with pytest.raises(sgagg.SgaggError):
            sgagg.sgagg_set_option(h, sgagg.SGAGG_OPT_PREFOLD, 5)
        sgagg.sgagg_set_option(h, sgagg.SGAGG_OPT_PREFOLD, 1)
        # result before any call
        r = ctypes.c_int64()
        assert lib.sgagg_result_rows(h, ctypes.byref(r)) == sgagg.SGAGG_ESTATE
    finally:
        sgagg.sgagg_destroy(h)
    lib.sgagg_destroy(None)


def test_product_does_not_import_oracle():
    """The product path never routes through the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2010_00152_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "sgagg_oracle" not in txt, f
