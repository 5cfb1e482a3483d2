"""The allocation-free sweep entry point (suppy_sweep_static).

Callers that cannot allocate device memory where they need a sweep (an
allocator that forbids cudaMalloc after start-up, a memory pool they own, or a
loop that must not take cudaMalloc's implicit synchronization) use this entry
point; its scratch is a static device array.  The tests check it through the
C ABI against the context-based suppy_sweep and against the FP64 oracle on
two calls in a row (the second call reuses the scratch the first one left
behind), on rows whose squared norms underflow FP32 (the norms are FP64),
invalid bounds (found on the device: x unchanged, proximity NaN), and the size
limit.  This file sorts last so that a run stopping at the first failure has
run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_2606_27086_gb300 as pk
import synth
from tests.helpers import random_x, rel, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("box", ["scalar", "vector"])
def test_static_sweep_matches_context_sweep_twice(box):
    prob = synth.random_problem(900, 5000, seed=61, feasible=False, mean_len=40,
                                empty_frac=0.05)
    n = prob.A.n
    if box == "vector":
        rng = np.random.default_rng(62)
        prob.box_lo = rng.uniform(-0.1, 0.2, size=n).astype(np.float32)
        prob.box_hi = (prob.box_lo + rng.uniform(0.5, 1.0, size=n)).astype(np.float32)
    x0 = np.clip(random_x(n, 1, seed=63), prob.box_lo, prob.box_hi).astype(np.float32)
    lam = 1.3

    ctx = pk.from_problem(prob)
    ctx.suppy_set_x(x0)
    P = pk.suppy_params_default(lam=lam)
    ref_x, ref_p = [], []
    for _ in range(2):
        ctx.suppy_sweep(P, 1)
        ref_x.append(ctx.suppy_get_x().copy())
    ref_p = list(ctx.suppy_history()[0])

    kept = int(np.count_nonzero(np.diff(prob.A.row_ptr)))
    A = prob.A
    rp, col, val = _dev(A.row_ptr), _dev(A.col), _dev(A.val)
    l, u = _dev(prob.l), _dev(prob.u)
    lo, hi = _dev(prob.box_lo), _dev(prob.box_hi)
    x = _dev(x0)
    prox = torch.zeros(1, dtype=torch.float64, device="cuda")
    S, lo_, uo_, blo, bhi = O.from_problem(prob)
    xo = x0.astype(np.float64)
    for k in range(2):
        pk.suppy_sweep_static(rp, col, val, A.m, n, l, u, 1.0 / kept, lam, lo, hi, x, prox)
        torch.cuda.synchronize()
        xo, po = O.sweep(S, O.CIMMINO, lo_, uo_, lam, blo, bhi, xo)
        assert rel_l2(x.cpu().numpy(), ref_x[k]) <= 1e-5
        assert rel(float(prox.item()), ref_p[k]) <= 1e-5
        assert rel_l2(x.cpu().numpy(), xo) <= 1e-5
        assert rel(float(prox.item()), po) <= 1e-5


def test_static_sweep_tiny_rows_use_fp64_norms():
    """Rows scaled by 1e-23 (squares below the smallest FP32 subnormal) and by
    1e17 stay constraints: two calls in a row against the FP64 oracle."""
    prob = synth.random_problem(600, 3000, seed=64, feasible=False, mean_len=30, empty_frac=0.0)
    A = prob.A
    rng = np.random.default_rng(65)
    scale = np.ones(A.m, np.float64)
    scale[rng.choice(A.m, 120, replace=False)] = 1e-23
    scale[rng.choice(A.m, 60, replace=False)] = 1e17
    rows = np.repeat(np.arange(A.m), np.diff(A.row_ptr))
    A.val = (A.val.astype(np.float64) * scale[rows]).astype(np.float32)
    prob.l = (prob.l.astype(np.float64) * scale).astype(np.float32)
    prob.u = (prob.u.astype(np.float64) * scale).astype(np.float32)
    n = A.n
    x0 = random_x(n, 1, seed=66)
    S, lo_, uo_, blo, bhi = O.from_problem(prob)
    kept = int(np.count_nonzero(np.diff(A.row_ptr)))
    rp, col, val = _dev(A.row_ptr), _dev(A.col), _dev(A.val)
    l, u = _dev(prob.l), _dev(prob.u)
    lo, hi = _dev(prob.box_lo), _dev(prob.box_hi)
    x = _dev(x0)
    prox = torch.zeros(1, dtype=torch.float64, device="cuda")
    xo = x0.astype(np.float64)
    for _ in range(2):
        pk.suppy_sweep_static(rp, col, val, A.m, n, l, u, 1.0 / kept, 1.0, lo, hi, x, prox)
        torch.cuda.synchronize()
        xo, po = O.sweep(S, O.CIMMINO, lo_, uo_, 1.0, blo, bhi, xo)
        assert rel_l2(x.cpu().numpy(), xo) <= 1e-5
        assert rel(float(prox.item()), po) <= 1e-5


def test_static_sweep_invalid_bounds_leave_x_alone():
    prob = synth.random_problem(300, 2000, seed=67, feasible=False, mean_len=20)
    A = prob.A
    x0 = random_x(A.n, 1, seed=68)
    rp, col, val = _dev(A.row_ptr), _dev(A.col), _dev(A.val)
    lo, hi = _dev(prob.box_lo), _dev(prob.box_hi)
    prox = torch.zeros(1, dtype=torch.float64, device="cuda")
    for bad in ("nan", "flip"):
        lb, ub = prob.l.copy(), prob.u.copy()
        if bad == "nan":
            lb[7] = np.nan
        else:
            lb[11], ub[11] = ub[11] + 1.0, lb[11]
        x = _dev(x0)
        pk.suppy_sweep_static(rp, col, val, A.m, A.n, _dev(lb), _dev(ub), 1.0 / A.m, 1.0, lo, hi,
                              x, prox)
        torch.cuda.synchronize()
        assert np.array_equal(x.cpu().numpy(), x0)
        assert np.isnan(float(prox.item()))


def test_static_sweep_rejects_oversized_problems():
    lib = pk.load_library()
    big = torch.zeros(4, dtype=torch.int32, device="cuda")
    fz = torch.zeros(4, dtype=torch.float32, device="cuda")
    A = pk.suppy_csr(1, (1 << 20) + 1, 1, ctypes.c_void_p(big.data_ptr()),
                     ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(fz.data_ptr()), 1)
    p = ctypes.c_void_p(fz.data_ptr())
    st = lib.suppy_sweep_static(ctypes.byref(A), p, p, 1.0, 1.0, p, p, 1, p, None, None)
    assert st == pk.SUPPY_EINVAL
    assert b"exceeds the static scratch" in lib.suppy_last_error(None)
