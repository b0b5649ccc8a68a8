"""The C-ABI library builds, loads and exports every symbol include/mptrac.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mptrac.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mptrac_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2211_12616_gb300 as M
    return M.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/mptrac.h but not exported"


def test_binding_covers_header():
    import paper_2211_12616_gb300 as M
    assert sorted(M.SIGNATURES) == _declared()


def test_no_gpu_calls_fail_cleanly(lib):
    """Without a CUDA device the library reports an error status instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    import paper_2211_12616_gb300 as M
    from workloads import grid_2deg_20lev
    with pytest.raises(M.MptracError) as ei:
        M.Context(grid_2deg_20lev())
    assert ei.value.code in (-3, -2)
    assert lib.mptrac_last_error(None)


def test_invalid_grid_rejected_on_host(lib):
    import numpy as np
    import paper_2211_12616_gb300 as M
    from paper_2211_12616_gb300._native import GridDesc
    plev = np.array([1e5, 5e4, 6e4])   # not decreasing
    gd = GridDesc(10, 5, 3, 0.0, 36.0, -90.0, 45.0, plev.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, 3)
    h = ctypes.c_void_p()
    assert lib.mptrac_init_grid(ctypes.byref(h), ctypes.byref(gd)) == -1
    assert b"decreasing" in lib.mptrac_last_error(None)
    gd = GridDesc(10, 5, 3, 0.0, 30.0, -90.0, 45.0, plev.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, 3)
    assert lib.mptrac_init_grid(ctypes.byref(h), ctypes.byref(gd)) == -1
    many = np.geomspace(1e5, 10.0, M.MAX_NZ + 1)       # one level more than supported
    gd = GridDesc(10, 5, M.MAX_NZ + 1, 0.0, 36.0, -90.0, 45.0,
                  many.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, 3)
    assert lib.mptrac_init_grid(ctypes.byref(h), ctypes.byref(gd)) == -1
    assert lib.mptrac_sort_workspace_bytes(None, 1000) >= 60 * 1000
    assert lib.mptrac_destroy(None) == 0


def test_binding_constants_match_the_header():
    """The constants the Python binding hard-codes equal the #defines of include/mptrac.h."""
    import pathlib
    import re

    import paper_2211_12616_gb300._native as N
    hdr = (pathlib.Path(__file__).resolve().parents[1] / "include" / "mptrac.h").read_text()
    d = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+MPTRAC_(\w+)\s+(-?\d+)", hdr)}
    assert (N.MPTRAC_FP32, N.MPTRAC_BF16, N.MPTRAC_FP16) == (d["FP32"], d["BF16"], d["FP16"])
    assert N.MAX_NZ == d["MAX_NZ"]
    assert (N.SURR_NFEAT, N.SURR_KPAD, N.SURR_HIDDEN, N.SURR_NOUT, N.SURR_NPARAM) == (
        d["SURR_NFEAT"], d["SURR_KPAD"], d["SURR_HIDDEN"], d["SURR_NOUT"], d["SURR_NPARAM"])
    assert (N.SURR_KERNEL_TCGEN05, N.SURR_KERNEL_MMA_SYNC, N.SURR_KERNEL_WAIT_TEST) == (
        d["SURR_KERNEL_TCGEN05"], d["SURR_KERNEL_MMA_SYNC"], d["SURR_KERNEL_WAIT_TEST"])
    for code, name in N.STATUS.items():
        assert d[name] == code, name
    # the surrogate's parameter count follows from its layer sizes
    assert d["SURR_NPARAM"] == d["SURR_KPAD"] * d["SURR_HIDDEN"] + d["SURR_HIDDEN"] + \
        d["SURR_HIDDEN"] ** 2 + d["SURR_HIDDEN"] + d["SURR_HIDDEN"] * d["SURR_NOUT"] + d["SURR_NOUT"]


def test_binding_signatures_match_the_header_prototypes():
    """Every prototype of include/mptrac.h has a binding with the same number of arguments,
    and the binding declares nothing the header does not."""
    import pathlib
    import re

    import paper_2211_12616_gb300._native as N
    hdr = (pathlib.Path(__file__).resolve().parents[1] / "include" / "mptrac.h").read_text()
    code = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(mptrac_\w+)\s*\(([^;{}]*?)\)\s*;", code, flags=re.S):
        args = m.group(2).strip()
        protos[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    assert set(protos) == set(N.SIGNATURES)
    for name, (_, argtypes) in N.SIGNATURES.items():
        assert len(argtypes) == protos[name], name


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libmptrac.so the binding raises; there is no CPU fallback."""
    import paper_2211_12616_gb300._native as N
    monkeypatch.setattr(N, "_lib", None)
    monkeypatch.setattr(N, "LIB_PATH", str(tmp_path / "libmptrac.so"))
    with pytest.raises(ImportError, match="no CPU fallback"):
        N.load()
