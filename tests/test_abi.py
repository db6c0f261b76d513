"""The C-ABI library builds for sm_103a, loads, and exports every call that
include/mcx.h declares (no compute calls: this runs without a GPU)."""
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "mcx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mcx_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc")
    from paper_1904_12759_gb300 import build as B

    B.build()
    from paper_1904_12759_gb300 import _lib

    return _lib.load()


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("mcx_plan_create", "mcx_estimate", "mcx_trace_paths", "mcx_power_iteration", "mcx_sync",
                 "mcx_plan_destroy", "mcx_status_string"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    from paper_1904_12759_gb300 import _lib

    declared = _declared()
    assert sorted(_lib.EXPORTS) == declared
    for name in declared:
        assert hasattr(lib, name), name


def test_status_strings_and_version(lib):
    assert lib.mcx_version() >= 100
    for code in range(0, -10, -1):
        s = lib.mcx_status_string(code).decode()
        assert s and s != "unknown status"
    assert lib.mcx_status_string(-99).decode() == "unknown status"


def test_missing_library_fails_loudly(tmp_path):
    from paper_1904_12759_gb300 import _lib

    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def test_walker_log_table_matches_the_oracle_table():
    """The CUDA library's FP32 logarithm table (ln_table.cuh, written by its generator
    script) and the oracle's own table (built from libm when the oracle loads) are
    independent statements of one definition: they must hold the same bits."""
    import re

    import numpy as np

    from oracle import walker as OW

    here = os.path.dirname(os.path.abspath(__file__))
    text = open(os.path.join(here, "..", "paper_1904_12759_gb300", "csrc", "ln_table.cuh")).read()
    rows = re.findall(r"\{0x([0-9a-f]{8})u, 0x([0-9a-f]{8})u\}", text)
    assert len(rows) == 65
    inv = np.array([int(a, 16) for a, _ in rows], np.uint32).view(np.float32)
    L = np.array([int(b, 16) for _, b in rows], np.uint32).view(np.float32)
    oinv, oL = OW.ln_table()
    assert np.array_equal(inv.view(np.uint32), oinv.view(np.uint32))
    assert np.array_equal(L.view(np.uint32), oL.view(np.uint32))


def test_exponential_table_matches_its_definition():
    """The FP64 exponential's table (exp_table.cuh, written by its generator script):
    each entry is 2^(j/64) correctly rounded to FP64 (checked against 40-digit decimal
    arithmetic, independently of the script), L1 keeps at most 36 significant bits (so
    N L1 is exact for |N| < 2^17), and L1 + L2 is ln(2)/64 to within an FP64 rounding
    of L2."""
    import re
    import struct
    from decimal import Decimal, getcontext

    here = os.path.dirname(os.path.abspath(__file__))
    text = open(os.path.join(here, "..", "paper_1904_12759_gb300", "csrc", "exp_table.cuh")).read()
    words = [int(w, 16) for w in re.findall(r"0x([0-9a-f]{16})ull", text)]
    assert len(words) == 64
    getcontext().prec = 40
    ln2 = Decimal(2).ln()
    for j, w in enumerate(words):
        x = struct.unpack("<d", struct.pack("<Q", w))[0]
        exact = (Decimal(j) / 64 * ln2).exp()
        ulp = Decimal(x) - Decimal(struct.unpack("<d", struct.pack("<Q", w - 1))[0])
        assert abs(Decimal(x) - exact) <= ulp / 2, j
    l1 = float(re.search(r"EXP_L1 = ([0-9.e+-]+);", text).group(1))
    l2 = float(re.search(r"EXP_L2 = ([0-9.e+-]+);", text).group(1))
    mant = struct.unpack("<Q", struct.pack("<d", l1))[0] & ((1 << 52) - 1)
    assert mant & ((1 << 17) - 1) == 0  # 52 - 17 = 35 stored bits + the implicit one
    assert abs(Decimal(l1) + Decimal(l2) - ln2 / 64) <= Decimal(2) ** -96


def test_cvbatch_rejects_slots_beyond_32_bit_indices(lib):
    """A batch whose pairs' slots (sum of n over pairs) reach 2^31 is rejected with
    MCX_E_INVALID while the description is checked, before any device work (so this
    runs without a GPU): 2100 right-hand sides of a 2^20-state problem."""
    import ctypes as C

    import numpy as np

    from paper_1904_12759_gb300 import _lib

    n, nrhs = 1 << 20, 2100
    rp = np.zeros(n + 1, np.int64)  # no entries
    col = np.zeros(1, np.int32)
    val = np.zeros(1)
    v = np.zeros(8)  # not read: the limit comes first
    t = np.full(nrhs, 0.1)
    pr = _lib.CvProblem(n=n, nnz=0, row_ptr=rp.ctypes.data, col=col.ctypes.data, val=val.ctypes.data,
                        n_rhs=nrhs, v=v.ctypes.data, t=t.ctypes.data, paths=8)
    out = C.c_void_p()
    assert lib.mcx_cvbatch_create(1, C.byref(pr), 0, None, 0, None, None, C.byref(out)) == -1
    assert not out.value
