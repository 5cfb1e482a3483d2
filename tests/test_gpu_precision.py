"""Error of 16-bit storage of A's values (BF16 / FP16, FP32 accumulation)
against the FP64 oracle on the ORIGINAL values, beside the kernel gate
against the oracle on the rounded values.

The gate is the parity bound of the path: the GPU run matches the oracle
run on the rounded values within 1e-5 (one sweep) or 1e-3 (a superiorized
run).  The error against the original values is then the oracle's own
rounded-vs-original distance plus at most that gate (triangle inequality);
the test checks that bound and prints both numbers.  Configurations: CT 64x64,
the full 100-iteration superiorized run from box(0); CT 512x512, one sweep
from a seeded point and three superiorized iterations from box(0).
"""
import numpy as np
import pytest

import oracle as O
import paper_2606_27086_gb300 as pk
import synth
from tests.helpers import rel, rel_l2, rounded_values

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DT = {"bf16": pk.SUPPY_BF16, "f16": pk.SUPPY_F16}
# Alg. 1 settings of the CT runs (TV, beta_k = 0.5 * 0.99^k, as in the configurations)
SUP = dict(gamma=0.5, alpha=0.99, n_red=1)
CT512 = dict(N=512, nang=360, nbin=725, I0=5e3, delta=0.02, seed_phantom=201, seed_noise=202)


def _runs(prob, K, dtype):
    ob = O.Objective(O.OBJ_TV_ISO, prob.shape)
    P = O.Params(max_sweeps=K, **SUP)
    S, l, u, lo, hi = O.from_problem(prob)
    r64 = O.run(S, O.CIMMINO, l, u, lo, hi, ob, P)
    Sr, lr, ur, lor, hir = O.from_problem(prob, values=rounded_values(prob.A.val, dtype))
    rr = O.run(Sr, O.CIMMINO, lr, ur, lor, hir, ob, P)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, dtype=DT[dtype])
    st = ctx.suppy_run(pk.suppy_params_default(max_sweeps=K, **SUP))[0]
    ph, fh = ctx.suppy_history()
    return ctx, st, ctx.suppy_get_x(), ph, fh, r64, rr


def _check_run(xg, ph, fh, r64, rr, dtype):
    gate = rel_l2(xg, rr.x)
    assert gate <= 1e-3
    assert rel(ph[-1], rr.prox_hist[-1]) <= 1e-3 and rel(fh[-1], rr.obj_hist[-1]) <= 1e-3
    rounding = rel_l2(rr.x, r64.x)
    err = rel_l2(xg, r64.x)
    assert err <= rounding + gate + 1e-12
    return err, rounding


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_ct64_full_run_error_vs_fp64_oracle(dtype):
    prob = synth.ct_problem()
    ctx, st, xg, ph, fh, r64, rr = _runs(prob, 100, dtype)
    # accepted steps: the same up to a borderline trial or two
    assert st["sweeps"] == 100 and abs(st["accepted"] - sum(rr.accepted)) <= 2
    err, rounding = _check_run(xg, ph, fh, r64, rr, dtype)
    print(f"ct64 100 iterations {dtype}: x rel-L2 vs FP64 oracle {err:.3e} "
          f"(rounding alone {rounding:.3e})")
    ctx.close()


@pytest.mark.slow
@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_ct512_error_vs_fp64_oracle(dtype):
    prob = synth.ct_problem(**CT512)
    # one sweep from a seeded point
    S, l, u, lo, hi = O.from_problem(prob)
    Sr, lr, ur, lor, hir = O.from_problem(prob, values=rounded_values(prob.A.val, dtype))
    x0 = np.random.default_rng(7).uniform(0, 1, prob.A.n).astype(np.float32)
    s64, _ = O.sweep(S, O.CIMMINO, l, u, 1.0, lo, hi, x0.astype(np.float64))
    sr, _ = O.sweep(Sr, O.CIMMINO, lr, ur, 1.0, lor, hir, x0.astype(np.float64))
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, dtype=DT[dtype])
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(pk.suppy_params_default(), 1)
    x1 = ctx.suppy_get_x()
    gate1 = rel_l2(x1, sr)
    assert gate1 <= 1e-5
    assert rel_l2(x1, s64) <= rel_l2(sr, s64) + gate1 + 1e-12
    ctx.close()
    # three superiorized iterations from box(0)
    ctx, st, xg, ph, fh, r64, rr = _runs(prob, 3, dtype)
    err, rounding = _check_run(xg, ph, fh, r64, rr, dtype)
    print(f"ct512 one sweep {dtype}: {rel_l2(x1, s64):.3e}; 3 iterations: {err:.3e} "
          f"(rounding alone {rounding:.3e})")
    ctx.close()


def _scaled(prob, s):
    import copy
    q = copy.deepcopy(prob)
    q.A.val = (prob.A.val.astype(np.float64) * s).astype(np.float32)
    q.l = (prob.l.astype(np.float64) * s).astype(np.float32)
    q.u = (prob.u.astype(np.float64) * s).astype(np.float32)
    return q


@pytest.mark.parametrize("scale,want", [(1.0, "f16"), (1e7, "bf16"), (1e-6, "bf16")])
def test_half_auto_takes_the_format_with_the_smaller_error(scale, want):
    """SUPPY_HALF_AUTO: FP16 for the CT values (in FP16's range: unit
    roundoff 2^-11 against BF16's 2^-8); BF16 when values exceed 65504, or
    when they sit so far below FP16's normal range that its absolute error
    (2^-25) exceeds BF16's relative one.  The sweep then matches the oracle
    on the values rounded to the chosen format (scaling A and the slabs by
    the same factor leaves the projections unchanged)."""
    prob = _scaled(synth.ct_problem(), scale)
    ctx = pk.from_problem(prob, dtype=pk.SUPPY_HALF_AUTO)
    got = ctx.suppy_info_get()["a_dtype"]
    assert got == {"f16": pk.SUPPY_F16, "bf16": pk.SUPPY_BF16}[want]
    x0 = np.random.default_rng(4).uniform(0, 1, prob.A.n).astype(np.float32)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(pk.suppy_params_default(), 1)
    S, l, u, lo, hi = O.from_problem(prob, values=rounded_values(prob.A.val, want))
    xo, _ = O.sweep(S, O.CIMMINO, l, u, 1.0, lo, hi, x0.astype(np.float64))
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
    ctx.close()


def test_half_auto_batched_context():
    """SUPPY_HALF_AUTO in a batched context (three right-hand sides sharing A):
    each right-hand side's sweep matches the oracle on the FP16 values."""
    prob = synth.ct_problem(nrhs=3)
    ctx = pk.from_problem(prob, dtype=pk.SUPPY_HALF_AUTO)
    assert ctx.suppy_info_get()["a_dtype"] == pk.SUPPY_F16
    x0 = np.random.default_rng(5).uniform(0, 1, (prob.A.n, 3)).astype(np.float32)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(pk.suppy_params_default(), 1)
    xg = ctx.suppy_get_x()
    S, l, u, lo, hi = O.from_problem(prob, values=rounded_values(prob.A.val, "f16"))
    for b in range(3):
        xo, _ = O.sweep(S, O.CIMMINO, O.rhs(l, b), O.rhs(u, b), 1.0, lo, hi,
                        x0[:, b].astype(np.float64))
        assert rel_l2(xg[:, b], xo) <= 1e-5
    ctx.close()


def test_half_auto_with_device_resident_values():
    prob = synth.ct_problem()
    ctx = pk.from_problem(prob, dtype=pk.SUPPY_HALF_AUTO, device=True)
    assert ctx.suppy_info_get()["a_dtype"] == pk.SUPPY_F16
    ctx.close()
