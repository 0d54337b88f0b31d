"""GPU tests of the batched solve of independent patches (one CUDA graph
launch per BiCGStab sweep) and of the x-stage autotuner."""
import os

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


def _patch(mf, p, nel, seed, mixed=False):
    knots = [inputs.open_uniform_knots(p, nel[l]) for l in range(3)]
    op = mf.Operator(p, knots, mixed=mixed, device=DEV)
    modes = inputs.fourier_modes(seed)
    op.set_coeff(op.eval_coeff("ring", modes, 0.3))
    return op


def test_batch_equals_separate_solves(mf):
    """Patches of uneven degree and size (the shape of the 64-patch workload,
    scaled down): the batched solve gives bit-for-bit the separate solves
    (same kernels, same deterministic reductions, independent patches)."""
    specs = inputs.batch_patches(count=6, seed=3, nel_range=(3, 12))
    ops = [_patch(mf, p, nel, i) for i, (p, nel) in enumerate(specs)]
    for op in ops:
        op.fd64_path = "pipe"  # the FD kernels with a grouped form
    fs = [op.load_vector("ring", "sines") for op in ops]
    ref = [op.solve(f, rtol=1e-8, force_fp64=True) for op, f in zip(ops, fs)]
    b = mf.Batch(ops)
    b.set_grouped(1)  # one grouped launch per kernel stage over all patches
    us, infos = b.solve(fs, rtol=1e-8, maxit=500)
    assert b.grouped
    for (u0, i0), u, i in zip(ref, us, infos):
        assert i.converged and i0.converged
        assert i.iterations == i0.iterations
        assert torch.equal(u, u0)
    assert max(i.outer_iterations for i in infos) == max(i.iterations for i in infos)
    b.close()
    # and the solutions satisfy each patch's system, checked by the oracle
    for (p, nel), op, f, u in zip(specs, ops, fs, us):
        tabs = [O.tables_1d(inputs.open_uniform_knots(p, nel[l]), p) for l in range(3)]
        C6 = O.coefficient_grid(tabs, "ring", inputs.fourier_modes(ops.index(op)), 0.3)
        K = O.stiffness_wq(tabs, O.full_coeff(C6))
        fn = f.cpu().numpy().ravel()
        res = np.linalg.norm(fn - K @ u.cpu().numpy().ravel()) / np.linalg.norm(fn)
        assert res <= 2e-8
        op.close()


def test_grouped_sweep_equals_per_stream_sweep(mf):
    """The grouped FP64 sweep and the per-patch-stream sweep give the same
    bits (FP64-pipe FD, whose kernels have grouped forms); a patch with a
    reaction term (no grouped form) makes the batch fall back to per-patch
    streams, still matching its separate solve."""
    specs = inputs.batch_patches(count=5, seed=11, nel_range=(3, 10))
    ops = [_patch(mf, p, nel, 40 + i) for i, (p, nel) in enumerate(specs)]
    for op in ops:
        op.fd64_path = "pipe"
    fs = [op.load_vector("ring", "sines") for op in ops]
    b = mf.Batch(ops)
    us, i_s = b.solve(fs, rtol=1e-9)  # per-patch streams (the default)
    assert not b.grouped
    for groups in (1, 2, 3):
        b.set_grouped(groups)
        ug, ig = b.solve(fs, rtol=1e-9)
        assert b.grouped
        for u1, u2, a, c in zip(ug, us, ig, i_s):
            assert a.converged and c.converged and a.iterations == c.iterations
            assert torch.equal(u1, u2)
    ops[2].set_mass_coeff(ops[2].eval_mass_coeff("ring", 3.0), fd_shift=3.0)
    ur, ir = b.solve(fs, rtol=1e-9)
    assert not b.grouped
    u_sep, i_sep = ops[2].solve(fs[2], rtol=1e-9, force_fp64=True)
    assert ir[2].iterations == i_sep.iterations and torch.equal(ur[2], u_sep)
    b.close()
    for op in ops:
        op.close()


def test_batch_mixed_equals_separate_mixed_solves(mf):
    """Mixed form of the batch: FP64 refinement steps in lockstep, inner FP32
    solves of all active patches one graph launch per sweep; each patch ends
    where its own mixed solve ends, at an FP64 residual below 1e-8."""
    specs = [(3, (6, 9, 7)), (5, (5, 4, 8)), (2, (12, 6, 5)), (4, (4, 7, 6))]
    ops = [_patch(mf, p, nel, 10 + i, mixed=True) for i, (p, nel) in enumerate(specs)]
    fs = [op.load_vector("ring", "sines") for op in ops]
    ref = [op.solve(f, rtol=1e-8, inner_rtol=1e-4) for op, f in zip(ops, fs)]
    b = mf.Batch(ops)
    us, infos = b.solve(fs, rtol=1e-8, inner_rtol=1e-4)
    for (u0, i0), u, i in zip(ref, us, infos):
        assert i.converged and i0.converged and i.rel_residual <= 1e-8
        assert i.outer_iterations == i0.outer_iterations and i.iterations == i0.iterations
        assert torch.equal(u, u0)
    u64, i64 = b.solve(fs, rtol=1e-8, force_fp64=True)
    for u, u2, i in zip(us, u64, i64):
        assert i.converged
        assert float(torch.linalg.vector_norm(u - u2) / torch.linalg.vector_norm(u2)) <= 1e-6
    b.close()
    for op in ops:
        op.close()


def test_batch_with_converged_patch_and_maxit(mf):
    ops = [_patch(mf, 3, (5, 6, 7), 0), _patch(mf, 2, (8, 4, 6), 1)]
    fs = [torch.zeros(ops[0].shape, dtype=torch.float64, device=DEV), ops[1].load_vector("ring", "sines")]
    b = mf.Batch(ops)
    us, infos = b.solve(fs, rtol=1e-10)
    assert infos[0].converged and infos[0].iterations == 0 and float(us[0].abs().max()) == 0.0
    assert infos[1].converged and infos[1].iterations > 0
    us, infos = b.solve(fs, rtol=1e-14, maxit=1)
    assert infos[1].status == -6 and infos[1].iterations == 1
    b.close()
    for op in ops:
        op.close()


@pytest.mark.parametrize("mode,lines,rows,carve", [(m, L, 1, 0) for m in (0, 1, 2, 3) for L in (2, 4, 8)]
                         + [(4, 8, 1, 0), (5, 8, 1, 0), (0, 4, 2, 0), (2, 2, 4, 0), (3, 8, 4, 0), (4, 8, 4, 0),
                            (1, 4, 1, 1), (5, 8, 2, 1)])
def test_every_xstage_variant_keeps_parity(mf, tmp_path, mode, lines, rows, carve):
    """Each launch shape the autotuner may pick gives the oracle's apply: x
    stage (mapping, lines, carveout copy) and slow-stage rows per thread; 345
    lines and 10 or 23 rows per slow stage, so every shape leaves a partial
    last block."""
    p, nel = 3, (7, 5, 9)
    op = _patch(mf, p, nel, 4)
    cache = str(tmp_path / "forced.jsonl")
    key = "xstage p=%d n1=%d nq1=%d nq2=%d nq3=%d fp64" % (p, op.n[0], op.nq[0], op.nq[1], op.nq[2])
    code = 1000 * carve + 100 * rows + 10 * mode + lines
    with open(cache, "w") as fh:
        fh.write('{"key": "%s", "xstage": %d}\n' % (key, code))
    assert op.autotune(cache) == code
    tabs = [O.tables_1d(inputs.open_uniform_knots(p, nel[l]), p) for l in range(3)]
    C6 = O.coefficient_grid(tabs, "ring", inputs.fourier_modes(4), 0.3)
    x = inputs.uniform_vector(op.shape, 8)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    y = op.apply(torch.from_numpy(x).to(DEV)).cpu().numpy()
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    if rows > 1:  # the transposed apply runs its slow stages with the same rows
        yT = op.apply_T(torch.from_numpy(x).to(DEV)).cpu().numpy()
        refT = O.apply_T_alg2(tabs, O.full_coeff(C6), x)
        assert np.abs(yT - refT).max() <= 1e-12 * np.abs(refT).max()
    op.close()


@pytest.mark.parametrize("mode,lines", [(m, L) for m in (0, 1, 2, 3) for L in (2, 4, 8)] + [(4, 8), (5, 8)])
def test_every_fp32_xstage_variant(mf, tmp_path, mode, lines):
    """The same for the FP32 operator of a mixed handle (FP32 prefetch needs 4
    or 8 lines; a forced 2-line prefetch runs the plain mapping).  n1 = 11 and
    nq1 = 25 are odd, so the two-row tiles end with a half tile, and 399 lines
    leave a partial last block of the tiled mappings."""
    p, nel = 4, (9, 6, 7)
    knots = [inputs.open_uniform_knots(p, nel[l]) for l in range(3)]
    op = mf.Operator(p, knots, mixed=True, device=DEV)
    tabs = [O.tables_1d(knots[l], p) for l in range(3)]
    C6 = O.coefficient_grid(tabs, "ring", inputs.fourier_modes(5), 0.3)
    op.set_coeff(torch.from_numpy(np.ascontiguousarray(C6)).to(DEV))
    cache = str(tmp_path / "forced32.jsonl")
    base = "xstage p=%d n1=%d nq1=%d nq2=%d nq3=%d" % (p, op.n[0], op.nq[0], op.nq[1], op.nq[2])
    with open(cache, "w") as fh:
        fh.write('{"key": "%s fp64", "xstage": 4}\n' % base)
        fh.write('{"key": "%s fp32", "xstage": %d}\n' % (base, 400 + 10 * mode + lines))
    op.autotune(cache)
    x = inputs.uniform_vector(op.shape, 10)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    y = op.apply_f32(torch.from_numpy(x).float().to(DEV)).double().cpu().numpy()
    assert np.abs(y - ref).max() <= 1e-5 * np.abs(ref).max()
    op.close()


@pytest.mark.parametrize("p,nel", [(2, (21, 6, 5)), (3, (18, 5, 6)), (4, (17, 6, 4)), (5, (20, 4, 5)),
                                   (6, (19, 4, 4)), (7, (22, 3, 4)), (8, (24, 3, 3))])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_stencil_xstage(mf, tmp_path, p, nel, prec):
    """The stencil mapping (code 68: mode 6) on uniform knots, p = 2..8: interior
    filters from the translation-invariant rows, boundary rows from the band
    tables, 16 lines per block with a partial last block."""
    knots = [inputs.open_uniform_knots(p, nel[l]) for l in range(3)]
    op = mf.Operator(p, knots, mixed=(prec == "fp32"), device=DEV)
    tabs = [O.tables_1d(knots[l], p) for l in range(3)]
    C6 = O.coefficient_grid(tabs, "ring", inputs.fourier_modes(6), 0.3)
    op.set_coeff(torch.from_numpy(np.ascontiguousarray(C6)).to(DEV))
    cache = str(tmp_path / "stencil.jsonl")
    base = "xstage p=%d n1=%d nq1=%d nq2=%d nq3=%d" % (p, op.n[0], op.nq[0], op.nq[1], op.nq[2])
    with open(cache, "w") as fh:
        fh.write('{"key": "%s fp64", "xstage": 68}\n{"key": "%s fp32", "xstage": 68}\n' % (base, base))
    op.autotune(cache)
    x = inputs.uniform_vector(op.shape, 11 + p)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    if prec == "fp64":
        y = op.apply(torch.from_numpy(x).to(DEV)).cpu().numpy()
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    else:
        y = op.apply_f32(torch.from_numpy(x).float().to(DEV)).double().cpu().numpy()
        assert np.abs(y - ref).max() <= 1e-5 * np.abs(ref).max()
    op.close()


def test_stencil_xstage_falls_back_on_graded_knots(mf, tmp_path):
    """Jittered knots have no translation-invariant interior: a forced stencil
    code runs the plain mapping and the apply still matches the oracle."""
    p = 3
    knots = [inputs.jittered_knots(p, 9, seed=4), inputs.open_uniform_knots(p, 4), inputs.open_uniform_knots(p, 5)]
    op = mf.Operator(p, knots, mixed=True, device=DEV)
    tabs = [O.tables_1d(knots[l], p) for l in range(3)]
    C6 = O.coefficient_grid(tabs, "ring")
    op.set_coeff(torch.from_numpy(np.ascontiguousarray(C6)).to(DEV))
    cache = str(tmp_path / "stencil_fallback.jsonl")
    base = "xstage p=%d n1=%d nq1=%d nq2=%d nq3=%d" % (p, op.n[0], op.nq[0], op.nq[1], op.nq[2])
    with open(cache, "w") as fh:
        fh.write('{"key": "%s fp64", "xstage": 68}\n{"key": "%s fp32", "xstage": 68}\n' % (base, base))
    op.autotune(cache)
    x = inputs.uniform_vector(op.shape, 12)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    y = op.apply(torch.from_numpy(x).to(DEV)).cpu().numpy()
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    y32 = op.apply_f32(torch.from_numpy(x).float().to(DEV)).double().cpu().numpy()
    assert np.abs(y32 - ref).max() <= 1e-5 * np.abs(ref).max()
    op.close()


def test_autotune_keeps_parity(mf, tmp_path):
    p, nel = 4, (9, 8, 10)
    op = _patch(mf, p, nel, 2)
    cache = str(tmp_path / "tune.jsonl")
    L = op.autotune(cache)
    assert L % 10 in (2, 4, 8) and (L // 10) % 10 in (0, 1, 2, 3, 4, 5, 6) and (L // 100) % 10 in (1, 2, 4)
    assert L // 1000 in (0, 1)
    assert os.path.exists(cache) and '"xstage": %d' % L in open(cache).read()
    assert op.autotune(cache) == L  # cache hit
    tabs = [O.tables_1d(inputs.open_uniform_knots(p, nel[l]), p) for l in range(3)]
    C6 = O.coefficient_grid(tabs, "ring", inputs.fourier_modes(2), 0.3)
    x = inputs.uniform_vector(op.shape, 9)
    ref = O.apply_alg2(tabs, O.full_coeff(C6), x)
    y = op.apply(torch.from_numpy(x).to(DEV)).cpu().numpy()
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    op.close()
