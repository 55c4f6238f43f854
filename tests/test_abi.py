"""The C ABI library loads and exports every entry point declared in include/*.h; the
host-only utilities (Philox, primes, L rules) agree with the oracle / numpy.  No GPU needed."""
import ctypes
import glob
import os
import re
import shutil

import numpy as np
import pytest

import oracle as O
from conftest import ROOT


def _lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location("_sfft_build", os.path.join(ROOT, "paper_2006_13053_gb300", "build.py"))
    B = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(B)
    if not B.up_to_date():
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build libsfft.so")
        B.build()
    return ctypes.CDLL(B.LIB)


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(sfft_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    names -= {"sfft_sample_fn"}
    return names


def test_every_declared_symbol_is_exported():
    lib = _lib()
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_philox_matches_numpy():
    lib = _lib()
    f = lib.sfft_philox4x64_word0
    f.restype = ctypes.c_uint64
    f.argtypes = [ctypes.c_uint64] * 5
    rng = np.random.default_rng(3)
    for _ in range(20):
        key = int(rng.integers(0, 2 ** 63))
        ctr = [int(v) for v in rng.integers(1, 2 ** 63, size=4)]
        bg = np.random.Philox(key=np.array([key, 0], dtype=np.uint64),
                              counter=np.array([ctr[0] - 1] + ctr[1:], dtype=np.uint64))
        assert f(key, *ctr) == int(bg.random_raw(1)[0])
        assert f(key, *ctr) == int(O.rand_u64(key, *[np.uint64(c) for c in ctr]))


def test_primes_and_L_rules_match_oracle():
    lib = _lib()
    np_ = lib.sfft_next_prime_above
    np_.restype = ctypes.c_int64
    np_.argtypes = [ctypes.c_double]
    Lr = lib.sfft_L_rule
    Lr.restype = ctypes.c_int
    Lr.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double]
    rng = np.random.default_rng(0)
    for x in list(rng.uniform(1, 2e6, 200)) + [206.6, 10330.0, 11042.77, 103300.0]:
        assert np_(float(x)) == O.next_prime_above(float(x))
    for n in [8, 35937, 2 ** 20, 10 ** 7, 4225, 65000]:
        for delta in (0.1, 0.9, 0.999):
            assert Lr(0, n, delta, 10.33) == O.L_cor26(n, delta)
            assert Lr(1, n, delta, 10.33) == O.L_eq42(n, delta)
        assert Lr(2, n, 0.1, 10.33) == O.L_fallback(n)


def test_invalid_arguments_rejected_on_host():
    lib = _lib()
    Lr = lib.sfft_L_rule
    Lr.restype = ctypes.c_int
    Lr.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double]
    assert Lr(0, 0, 0.1, 10.33) == -1
    assert Lr(0, 100, 1.5, 10.33) == -1
    f = lib.sfft_plan_create
    f.restype = ctypes.c_int
    h = ctypes.c_void_p()
    # NULL candidate pointer -> SFFT_EINVAL before any device work
    assert f(ctypes.byref(h), 3, None, 10, 2, 0, None, None, None, None) == 1
    assert f(None, 3, None, 10, 2, 0, None, None, None, None) == 1


def test_misaligned_candidate_rows_rejected_on_host():
    """int32 rows are read as int4 (d % 4 == 0) or int2 (d % 2 == 0) words: a pointer that is only
    4-byte aligned (a tensor view with an offset) returns SFFT_EINVAL before any device work, from
    the plan and from the allocation-free detection alike (the fake addresses are never touched)."""
    lib = _lib()
    f = lib.sfft_plan_create
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    err = lib.sfft_last_error
    err.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    for d, addr in ((4, 0x10004), (8, 0x10008), (6, 0x10004), (10, 0x1000C)):
        assert f(ctypes.byref(h), d, addr, 100, 2, 0, None, None, None, None) == 1, d
        assert b"aligned" in err()
    det = lib.sfft_detect_noalloc
    det.restype = ctypes.c_int
    det.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64,
                    ctypes.c_void_p, ctypes.c_void_p]
    Ms = np.full(1, 101, dtype=np.int64)
    zz = np.zeros(4, dtype=np.int64)
    taus = np.zeros(1)
    nd = ctypes.c_int64()
    rc = det(4, 0x10004, 100, 1, Ms.ctypes.data, zz.ctypes.data, 0x20000, taus.ctypes.data, 0.5, 0x30000, 100,
             ctypes.byref(nd), None)
    assert rc == 1 and b"aligned" in err()


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's field offsets and sizes."""
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    import importlib.util
    spec = importlib.util.spec_from_file_location("_sfft_native_layout",
                                                  os.path.join(ROOT, "paper_2006_13053_gb300", "_native.py"))
    N = importlib.util.module_from_spec(spec)
    try:
        spec.loader.exec_module(N)
    except Exception:  # the binding module loads the library; read the classes from its source instead
        pytest.skip("binding module not importable without the library")
    pairs = {"sfft_params": N.Params, "sfft_diag": N.Diag, "sfft_dimincr_params": N.DimIncrParams,
             "sfft_fn_sparse_poly_ctx": N.SparsePolyCtx, "sfft_fn_sop_ctx": N.SopCtx,
             "sfft_fn_bspline_ctx": N.BsplineCtx}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sfft.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        c, f, v = line.split()
        got[(c, f)] = int(v)
    for cname, cls in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
