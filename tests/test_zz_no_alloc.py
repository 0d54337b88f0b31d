"""GPU test of mfwq_fd_precond_noalloc, the FD preconditioner for callers that
cannot allocate device memory where they need it (e.g. inside a CUDA-graph
capture in global mode, or with all device memory owned by a framework's
allocator).  It must give what fd_precond gives on a handle, call after call,
although its scratch is one fixed array shared by every call.

This file is collected last on purpose, and passes alone in a fresh process
as well as after the other tests."""
import ctypes

import numpy as np
import pytest

from paper_1712_08565_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-12  # the FP64 FD parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_08565_gb300 import build
    build.build()
    from paper_1712_08565_gb300 import mfwq
    return mfwq


def _factors(mf, ps, knots):
    U, UT, lam = [], [], []
    for l in range(3):
        t = mf.tables_1d(ps[l], knots[l])
        U.append(torch.from_numpy(np.ascontiguousarray(t["U"])).to(DEV))
        UT.append(torch.from_numpy(np.ascontiguousarray(t["U"].T)).to(DEV))
        lam.append(torch.from_numpy(t["lam"]).to(DEV))
    return U, UT, lam


@pytest.mark.parametrize("ps,nel", [((3, 3, 3), (5, 7, 9)), ((4, 4, 4), (40, 36, 30))])
def test_noalloc_matches_fd_precond_twice(mf, ps, nel):
    knots = [inputs.open_uniform_knots(ps[l], nel[l]) for l in range(3)]
    op = mf.Operator(ps, knots, device=DEV)
    U, UT, lam = _factors(mf, ps, knots)
    n = op.n
    for seed in (31, 32):  # two calls in a row through the shared scratch
        r = torch.from_numpy(inputs.uniform_vector(op.shape, seed)).to(DEV)
        ref = op.fd_precond(r)
        z = torch.full_like(r, float("nan"))
        # raw C ABI call
        L = mf.lib()
        nn = (ctypes.c_int * 3)(*n)
        P = lambda ts: (ctypes.c_void_p * 3)(*[t.data_ptr() for t in ts])
        st = L.mfwq_fd_precond_noalloc(nn, P(U), P(UT), P(lam), ctypes.c_void_p(r.data_ptr()),
                                       ctypes.c_void_p(z.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, L.mfwq_last_error()
        torch.cuda.synchronize()
        zr, rr = z.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(zr).all()
        assert np.abs(zr - rr).max() <= TOL * np.abs(rr).max()
    op.close()


def test_noalloc_binding_and_limits(mf):
    ps, nel = (2, 2, 2), (6, 5, 4)
    knots = [inputs.open_uniform_knots(ps[l], nel[l]) for l in range(3)]
    op = mf.Operator(ps, knots, device=DEV)
    U, UT, lam = _factors(mf, ps, knots)
    r = torch.from_numpy(inputs.uniform_vector(op.shape, 33)).to(DEV)
    z = torch.empty_like(r)
    mf.fd_precond_noalloc(op.n, U, UT, lam, r, z)
    ref = op.fd_precond(r)
    torch.cuda.synchronize()
    assert float((z - ref).abs().max()) <= TOL * float(ref.abs().max())
    # sizes beyond the fixed scratch are rejected before any device work
    big = (ctypes.c_int * 3)(256, 256, 128)
    dummy = (ctypes.c_void_p * 3)(r.data_ptr(), r.data_ptr(), r.data_ptr())
    st = mf.lib().mfwq_fd_precond_noalloc(big, dummy, dummy, dummy, ctypes.c_void_p(r.data_ptr()),
                                          ctypes.c_void_p(z.data_ptr()), None)
    assert st == -1 and b"exceeds" in mf.lib().mfwq_last_error()
    st = mf.lib().mfwq_fd_precond_noalloc((ctypes.c_int * 3)(*op.n), dummy, dummy, dummy,
                                          ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(r.data_ptr()), None)
    assert st == -1  # aliased input and output
    # a size triple whose product wraps around 2^64 in size_t is rejected too
    wrap = (ctypes.c_int * 3)(1 << 21, 1 << 21, 1 << 22)
    st = mf.lib().mfwq_fd_precond_noalloc(wrap, dummy, dummy, dummy, ctypes.c_void_p(r.data_ptr()),
                                          ctypes.c_void_p(z.data_ptr()), None)
    assert st == -1 and b"exceeds" in mf.lib().mfwq_last_error()
    # host memory (pageable or pinned) in place of r is rejected before any launch
    n0 = mf.kernel_launches()
    for host in (np.zeros(op.N), torch.zeros(op.N, dtype=torch.float64).pin_memory()):
        hp = host.ctypes.data if isinstance(host, np.ndarray) else host.data_ptr()
        Pd = lambda ts: (ctypes.c_void_p * 3)(*[t.data_ptr() for t in ts])
        st = mf.lib().mfwq_fd_precond_noalloc((ctypes.c_int * 3)(*op.n), Pd(U), Pd(UT), Pd(lam), ctypes.c_void_p(hp),
                                              ctypes.c_void_p(z.data_ptr()), None)
        assert st == -1 and b"not device memory" in mf.lib().mfwq_last_error()
    assert mf.kernel_launches() == n0
    op.close()


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2, reason="needs two CUDA devices")
def test_noalloc_on_second_device(mf):
    """Tensors on cuda:1 while cuda:0 is current: the binding makes r's device
    current, and the raw call with cuda:0 current refuses cuda:1 memory."""
    ps, nel = (3, 3, 3), (6, 5, 7)
    knots = [inputs.open_uniform_knots(ps[l], nel[l]) for l in range(3)]
    dev1 = torch.device("cuda", 1)
    op = mf.Operator(ps, knots, device=dev1)
    U, UT, lam = _factors(mf, ps, knots)
    U, UT, lam = [t.to(dev1) for t in U], [t.to(dev1) for t in UT], [t.to(dev1) for t in lam]
    r = torch.from_numpy(inputs.uniform_vector(op.shape, 34)).to(dev1)
    z = torch.empty_like(r)
    with torch.cuda.device(0):
        mf.fd_precond_noalloc(op.n, U, UT, lam, r, z)
        ref = op.fd_precond(r)
        torch.cuda.synchronize(dev1)
        assert float((z - ref).abs().max()) <= TOL * float(ref.abs().max())
        Pd = lambda ts: (ctypes.c_void_p * 3)(*[t.data_ptr() for t in ts])
        st = mf.lib().mfwq_fd_precond_noalloc((ctypes.c_int * 3)(*op.n), Pd(U), Pd(UT), Pd(lam),
                                              ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), None)
        assert st == -1 and b"current device" in mf.lib().mfwq_last_error()
    op.close()
