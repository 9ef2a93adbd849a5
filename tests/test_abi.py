"""The C-ABI library builds, loads, and exports every symbol include/dfacto.h
declares; the ctypes structs match the C layouts.  No GPU needed: nothing here
launches a kernel."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dfacto.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1406_4519_gb300 import build_lib, dfacto
    build_lib.build()
    return dfacto.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dfacto_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dfacto_build", "dfacto_mttkrp", "dfacto_als_iter", "dfacto_gd_iter",
                     "dfacto_fit", "dfacto_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1406_4519_gb300 import dfacto
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in dfacto.SIGNATURES, "binding lacks " + name


def test_struct_layouts_match_header(tmp_path, lib):
    from paper_1406_4519_gb300 import dfacto
    prog = tmp_path / "layout.c"
    prog.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "dfacto.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(dfacto_options), offsetof(dfacto_options, lambda_reg),
         offsetof(dfacto_options, seg_nnz), offsetof(dfacto_options, vec),
         offsetof(dfacto_options, walk), offsetof(dfacto_options, line_search));
  printf("%zu %zu %zu %zu\\n", sizeof(dfacto_info), offsetof(dfacto_info, nnz),
         offsetof(dfacto_info, norm_x2), offsetof(dfacto_info, vec));
  printf("%zu %zu\\n", sizeof(dfacto_csr_view), offsetof(dfacto_csr_view, nz_val));
  printf("%zu %zu\\n", sizeof(dfacto_ratings_view), offsetof(dfacto_ratings_view, val));
  printf("%zu %zu\\n", sizeof(dfacto_batch_options), offsetof(dfacto_batch_options, reserved));
  printf("%zu %zu %zu\\n", sizeof(dfacto_batch_class), offsetof(dfacto_batch_class, nnz),
         offsetof(dfacto_batch_class, tuned_ms));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = subprocess.check_output([str(exe)]).decode().split()
    want = [ctypes.sizeof(dfacto.dfacto_options), dfacto.dfacto_options.lambda_reg.offset,
            dfacto.dfacto_options.seg_nnz.offset, dfacto.dfacto_options.vec.offset,
            dfacto.dfacto_options.walk.offset, dfacto.dfacto_options.line_search.offset,
            ctypes.sizeof(dfacto.dfacto_info), dfacto.dfacto_info.nnz.offset,
            dfacto.dfacto_info.norm_x2.offset, dfacto.dfacto_info.vec.offset,
            ctypes.sizeof(dfacto.dfacto_csr_view), dfacto.dfacto_csr_view.nz_val.offset,
            ctypes.sizeof(dfacto.dfacto_ratings_view), dfacto.dfacto_ratings_view.val.offset,
            ctypes.sizeof(dfacto.dfacto_batch_options), dfacto.dfacto_batch_options.reserved.offset,
            ctypes.sizeof(dfacto.dfacto_batch_class), dfacto.dfacto_batch_class.nnz.offset,
            dfacto.dfacto_batch_class.tuned_ms.offset]
    assert [int(x) for x in got] == want


def test_host_side_argument_checks(lib):
    """Invalid arguments are rejected before any device work."""
    from paper_1406_4519_gb300 import dfacto
    out = ctypes.c_void_p()
    dims = (ctypes.c_int32 * 3)(2, 2, 2)
    assert lib.dfacto_build(None, None, 0, dims, None, None, None) == dfacto.EINVAL
    bad = (ctypes.c_int32 * 3)(2, 0, 2)
    assert lib.dfacto_build(None, None, 0, bad, None, None, ctypes.byref(out)) == dfacto.EINVAL
    assert lib.dfacto_build(None, None, -1, dims, None, None, ctypes.byref(out)) == dfacto.EINVAL
    opt = dfacto.dfacto_options_init(0)
    assert lib.dfacto_build(None, None, 0, dims, ctypes.byref(opt), None,
                            ctypes.byref(out)) == dfacto.EINVAL
    opt = dfacto.dfacto_options_init(33)  # > 32 and not a multiple of 4
    assert lib.dfacto_build(None, None, 0, dims, ctypes.byref(opt), None,
                            ctypes.byref(out)) == dfacto.EINVAL
    opt = dfacto.dfacto_options_init(10, vec=4)  # 4 does not divide 10
    assert lib.dfacto_build(None, None, 0, dims, ctypes.byref(opt), None,
                            ctypes.byref(out)) == dfacto.EINVAL
    opt = dfacto.dfacto_options_init(8, lambda_reg=-1.0)
    assert lib.dfacto_build(None, None, 0, dims, ctypes.byref(opt), None,
                            ctypes.byref(out)) == dfacto.EINVAL
    # nonzero positions stay 32-bit in the walks: at most 2^31 - 2^16 nonzeros
    # (refused before the null pointers are looked at)
    assert lib.dfacto_build(None, None, 2 ** 31 - 2 ** 16 + 1, dims, None, None,
                            ctypes.byref(out)) == dfacto.EINVAL
    opt = dfacto.dfacto_options_init(8, seg_nnz=4097)  # segments of at most 4096
    assert lib.dfacto_build(None, None, 0, dims, ctypes.byref(opt), None,
                            ctypes.byref(out)) == dfacto.EINVAL
    for ls in (-1, 2):  # line searches 0 (backtracking) and 1 (exact) exist
        opt = dfacto.dfacto_options_init(8, line_search=ls)
        assert lib.dfacto_build(None, None, 0, dims, ctypes.byref(opt), None,
                                ctypes.byref(out)) == dfacto.EINVAL
    for walk in (-1, 3, 4):  # walks 0 (library's choice), 1 and 2 exist
        opt = dfacto.dfacto_options_init(8, walk=walk)
        assert lib.dfacto_build(None, None, 0, dims, ctypes.byref(opt), None,
                                ctypes.byref(out)) == dfacto.EINVAL
    assert out.value is None
    for fn in ("dfacto_mttkrp", "dfacto_als_iter", "dfacto_fit", "dfacto_sync"):
        args = {"dfacto_mttkrp": (None, 0, None), "dfacto_als_iter": (None, None),
                "dfacto_fit": (None, None), "dfacto_sync": (None,)}[fn]
        assert getattr(lib, fn)(*args) == dfacto.EINVAL
    assert lib.dfacto_status_str(dfacto.EDUP) == b"duplicate coordinate"
    # the joint model's entry points refuse a null handle
    assert lib.dfacto_joint_set_ratings(None, None, None, 0, 1.0) == dfacto.EINVAL
    assert lib.dfacto_joint_als_iter(None, None) == dfacto.EINVAL
    assert lib.dfacto_joint_gd_iter(None, None, None) == dfacto.EINVAL
    assert lib.dfacto_joint_objective(None, None) == dfacto.EINVAL
    assert lib.dfacto_get_ratings_csr(None, 0, None) == dfacto.EINVAL


def test_batch_host_side_argument_checks(lib):
    """Batch entry points reject null and out-of-range arguments on the host."""
    from paper_1406_4519_gb300 import dfacto
    out = ctypes.c_void_p()
    assert lib.dfacto_batch_create(None, 1, None, None, ctypes.byref(out)) == dfacto.EINVAL
    jobs = (ctypes.c_void_p * 1)(None)
    assert lib.dfacto_batch_create(jobs, 1, None, None, ctypes.byref(out)) == dfacto.EINVAL
    assert lib.dfacto_batch_create(jobs, 0, None, None, ctypes.byref(out)) == dfacto.EINVAL
    assert lib.dfacto_batch_create(jobs, 1, None, None, None) == dfacto.EINVAL
    assert out.value is None
    assert lib.dfacto_batch_mttkrp(None, 0, None) == dfacto.EINVAL
    assert lib.dfacto_batch_als_iter(None, None) == dfacto.EINVAL
    assert lib.dfacto_batch_sync(None) == dfacto.EINVAL
    assert lib.dfacto_batch_num_classes(None) == 0
    c = dfacto.dfacto_batch_class()
    assert lib.dfacto_batch_get_class(None, 0, ctypes.byref(c)) == dfacto.EINVAL
    lib.dfacto_batch_destroy(None)
    opt = dfacto.dfacto_batch_options_init()
    assert (opt.use_graph, opt.autotune) == (1, 1)
