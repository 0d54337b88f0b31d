"""CPU tests of the C-ABI library: it builds, loads, exports every symbol the
header declares, and its host-side setup (1D tables of Algorithm 2's setup,
FD factors) matches the oracle.  No GPU call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1712_08565_gb300 import build as B
from paper_1712_08565_gb300 import inputs, mfwq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def _declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", txt, flags=re.M):
            name = m.group(1)
            if name not in ("if", "for", "while", "sizeof", "return"):
                names.add(name)
    return names


def test_library_exports_every_declared_symbol(libpath):
    names = _declared_functions()
    assert {"mfwq_setup", "mfwq_apply", "mfwq_apply_T", "fd_precond", "mfwq_solve", "mfwq_grad_coeff"} <= names
    L = ctypes.CDLL(libpath)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(libpath):
    L = mfwq.lib()
    for code in range(0, -10, -1):
        assert L.mfwq_status_string(code)
    assert L.mfwq_status_string(-1).decode() == "invalid argument"


@pytest.mark.parametrize("p,nel", [(2, 2), (2, 16), (3, 7), (4, 20), (5, 9), (6, 24), (8, 12), (10, 11)])
def test_host_tables_match_oracle(libpath, p, nel):
    """Points, B-spline tables, the four weight families (double-double in the
    library, 80-digit decimal in the oracle) and the FD factors."""
    knots = inputs.open_uniform_knots(p, nel)
    t = mfwq.tables_1d(p, knots)
    tab = O.tables_1d(knots, p)
    assert t["xq"].shape == tab.xq.shape
    assert np.abs(t["xq"] - tab.xq).max() <= 2e-16
    assert np.abs(t["B0"] - tab.B0).max() <= 1e-14
    assert np.abs(t["B1"] - tab.B1).max() <= 1e-13 * np.abs(tab.B1).max()
    for a in (0, 1):
        for b in (0, 1):
            W = tab.W[(a, b)]
            assert np.abs(t["W"][2 * a + b] - W).max() <= 1e-14 * np.abs(W).max(), (a, b)
    fd = O.fd_setup([tab] * 3)
    # U is unique only up to signs and bases of repeated eigenvalues: compare
    # the eigenvalues and the 1D inverse U diag(1/lam) U^T = K^-1.
    np.testing.assert_allclose(np.sort(t["lam"]), fd.lam[0], rtol=1e-11)
    Ki = t["U"] @ np.diag(1 / t["lam"]) @ t["U"].T
    Ko = fd.U[0] @ np.diag(1 / fd.lam[0]) @ fd.U[0].T
    assert np.abs(Ki - Ko).max() <= 1e-11 * np.abs(Ko).max()
    M = fd.M[0]
    assert np.abs(t["U"].T @ M @ t["U"] - np.eye(tab.n)).max() <= 1e-11


def test_host_tables_nonuniform_knots(libpath):
    p = 4
    knots = inputs.jittered_knots(p, 13, seed=4)
    t = mfwq.tables_1d(p, knots)
    tab = O.tables_1d(knots, p)
    for a in (0, 1):
        for b in (0, 1):
            W = tab.W[(a, b)]
            assert np.abs(t["W"][2 * a + b] - W).max() <= 1e-14 * np.abs(W).max()


@pytest.mark.parametrize("bad", ["degree1", "degree13", "notopen", "repeated", "decreasing", "oneelem"])
def test_host_setup_rejects_bad_knots(libpath, bad):
    p = 3
    k = inputs.open_uniform_knots(p, 6)
    if bad == "degree1":
        p = 1
        k = inputs.open_uniform_knots(1, 6)
    elif bad == "degree13":
        p = 13
        k = inputs.open_uniform_knots(13, 6)
    elif bad == "notopen":
        k = k.copy()
        k[0] = -0.1
    elif bad == "repeated":
        k = k.copy()
        k[p + 2] = k[p + 1]
    elif bad == "decreasing":
        k = k.copy()
        k[p + 2], k[p + 3] = k[p + 3], k[p + 2]
    elif bad == "oneelem":
        k = inputs.open_uniform_knots(p, 1)
    with pytest.raises(mfwq.MfwqError) as e:
        mfwq.tables_1d(p, k)
    assert e.value.status == -1


def test_binding_refuses_without_gpu_tensor(libpath):
    torch = pytest.importorskip("torch")
    with pytest.raises((TypeError, ValueError)):
        mfwq._ptr(torch.zeros(4, dtype=torch.float64), torch.float64)


def _c_driver_build(out):
    """Compile tests/c_driver/solve_ring.c against include/mfwq.h and link it
    with libmfwq.so and the CUDA runtime; returns the command's result."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if cc is None or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("no C compiler or CUDA headers")
    pkg = os.path.join(ROOT, "paper_1712_08565_gb300")
    libdirs = [d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib")) if os.path.isdir(d)]
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c_driver", "solve_ring.c"),
           "-L", pkg, "-lmfwq"] + [f"-L{d}" for d in libdirs] + ["-lcudart", "-o", out]
    return subprocess.run(cmd, capture_output=True, text=True)


def test_c_driver_compiles_and_links(tmp_path):
    """The C ABI is usable from plain C: the driver builds warning-free."""
    r = _c_driver_build(str(tmp_path / "solve_ring"))
    assert r.returncode == 0, r.stderr
