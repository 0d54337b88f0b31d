"""The plain C driver (tests/c_driver/solve_ring.c) on the GPU: the same ring
problem solved through the C ABI from C and from the Python binding gives the
same iteration count and relative H1 error."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1712_08565_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_08565_gb300 import build
    build.build()
    from paper_1712_08565_gb300 import mfwq
    return mfwq


def test_c_driver_matches_python(mf, tmp_path):
    from test_capi_host import _c_driver_build
    exe = str(tmp_path / "solve_ring")
    r = _c_driver_build(exe)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.path.join(ROOT, "paper_1712_08565_gb300") + os.pathsep + env.get("LD_LIBRARY_PATH", "")
    p, nel = 3, 16
    out = subprocess.run([exe, str(p), str(nel), "1e-10"], capture_output=True, text=True, env=env, timeout=300)
    assert out.returncode == 0, out.stderr
    m = re.search(r"iterations (\d+) rel_residual (\S+) h1_error (\S+)", out.stdout)
    assert m, out.stdout
    it_c, res_c, err_c = int(m.group(1)), float(m.group(2)), float(m.group(3))
    op = mf.Operator(p, [inputs.open_uniform_knots(p, nel)] * 3, device="cuda:0")
    op.set_coeff(op.eval_coeff("ring"))
    f = op.load_vector("ring", "ring_exact")
    uh, info = op.solve_host(f.cpu().numpy(), rtol=1e-10)
    err_py = op.h1_error(torch.from_numpy(np.ascontiguousarray(uh)).to("cuda:0"), "ring", "ring")
    assert res_c <= 1e-10 and info.iterations == it_c
    assert abs(err_c - err_py) <= 1e-12 * err_py
    assert 0.2 < err_c < 1.2  # Table 1, h = 2^-4: no approximation yet
    op.close()
