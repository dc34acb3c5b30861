"""The C-ABI library builds, loads and exports every entry point include/qlr.h declares.
No compute calls: these run on a machine without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qlr.h")


@pytest.fixture(scope="module")
def libpath():
    from paper_2507_13731_gb300 import build
    return build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qlr_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_paper_entry_points():
    names = declared_functions()
    for want in ("qlr_qsketch", "qlr_qrangefinder", "qlr_qblock_krylov", "qlr_qsvd_lowrank",
                 "qlr_qsvd_lowrank_batched", "qlr_cholqr", "qlr_qtsvd", "qlr_residual_norm"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(libpath):
    from paper_2507_13731_gb300 import qlr
    L = qlr.lib()
    assert L.qlr_strerror(0) == b"success"
    assert b"Cholesky" in L.qlr_strerror(qlr.ENOTPD)
    ws = qlr.workspace_size(4096, 4096, 100, 10, 4)
    assert 0 < ws < (8 << 30)
    # null-pointer arguments are rejected before any device work
    assert L.qlr_qsketch(None, 0, None, None, None, 0) == qlr.EINVAL
    assert L.qlr_create(None, 0, None) == qlr.EINVAL
    assert L.qlr_qcomplete_update(None, None, None, 1, None, None, None, 0, None) == qlr.EINVAL
    assert L.qlr_qcomplete(None, None, None, 1, 1, 0, 2, qlr.ALG2, 1, None, None, None, None, None, None) == qlr.EINVAL
    kid_count = int(re.search(r"#define QLR_KID_COUNT (\d+)", open(HEADER).read()).group(1))
    assert len(qlr.KID_NAMES) == kid_count


def test_descriptor_layouts_on_cpu_tensors():
    import torch
    from paper_2507_13731_gb300 import qlr
    A = torch.zeros(4, 5, 7)
    d = qlr.qmat(A)
    assert (d.rows, d.cols, d.ld, d.layout, d.dtype) == (5, 7, 7, qlr.ROW_MAJOR, qlr.F32)
    T = qlr.empty_thin(9, 3, torch.float64, "cpu")
    d = qlr.qmat(T)
    assert (d.rows, d.cols, d.ld, d.layout, d.dtype) == (9, 3, 9, qlr.COL_MAJOR, qlr.F64)
    assert d.plane[1] - d.plane[0] == 9 * 3 * 8
    P = torch.zeros(3, 4, 6, dtype=torch.bfloat16)
    d = qlr.qmat(P)
    assert d.plane[0] is None and d.dtype == qlr.BF16


def test_mask_descriptor_on_cpu_tensors():
    import torch
    from paper_2507_13731_gb300 import qlr
    buf = torch.zeros(6, 10, dtype=torch.uint8)
    _, ld = qlr._mask(buf[:, :7], 6, 7)
    assert ld == 10                                   # padded rows keep their stride
    with pytest.raises(ValueError):
        qlr._mask(torch.zeros(6, 7), 6, 7)            # not uint8
    with pytest.raises(ValueError):
        qlr._mask(buf[:, :7], 7, 6)                   # wrong shape
    with pytest.raises(ValueError):
        qlr._mask(buf.t()[:7, :6], 7, 6)              # column-major
