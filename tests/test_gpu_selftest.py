"""Failure detection without a GPU fault: the library's bounded device waits
give up, record the timeout and leave the context usable.  The self-test
kernel arms an mbarrier for bytes that no copy delivers (a flag that nothing
sets), so its wait must run out."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1712_08565_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_08565_gb300 import build
    build.build()
    from paper_1712_08565_gb300 import mfwq
    return mfwq


def test_bounded_wait_times_out_and_context_survives(mf):
    L = mf.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.mfwq_selftest_bounded_wait(2_000_000, stream)  # about a millisecond of SM cycles
    assert st == -7, L.mfwq_last_error()  # MFWQ_ETIMEOUT
    assert b"gave up" in L.mfwq_last_error()
    assert L.mfwq_selftest_bounded_wait(0, stream) == -1
    # the context is still usable: an apply matches the oracle
    p, nel = 2, (4, 5, 3)
    knots = [inputs.open_uniform_knots(p, n) for n in nel]
    op = mf.Operator(p, knots, device=DEV)
    op.set_coeff(op.eval_coeff("ring"))
    tabs = [O.tables_1d(knots[l], p) for l in range(3)]
    x = inputs.uniform_vector(op.shape, 71)
    y = op.apply(torch.from_numpy(x).to(DEV)).cpu().numpy()
    ref = O.apply_alg2(tabs, O.full_coeff(O.coefficient_grid(tabs, "ring")), x)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    op.sync()
    op.close()
