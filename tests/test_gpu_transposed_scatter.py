"""Rows running down the image handled in the column-major pixel numbering
(opts.scatter_transpose), against the FP64 oracle: in the one-pass sweep
they scatter into a column-major accumulator, in the two-pass sweep their
indices are column-major and they gather from a column-major copy of x.

The sweep computes the same Eq. (3) step either way (Sec. 2.1.1): only the
order of the FP32 additions changes, so the per-sweep bound stays 1e-5
relative L2.  Sizes keep n * 4 bytes above 64 KB, where the one-pass sweep
scatters by L2 reductions (the transposed accumulator serves only that
form).  Covered: square and non-square grids (the index map divides by the
width), Cimmino, BIP with angle blocks (a box step per block), DROP (the
column scaling applies to the sum of both accumulators), a superiorized run
with graphs, and the rejections.  The one-pass cases run in both numberings
of the accumulators: row- and column-major (scatter_transpose 1) and the
patch numbering (2), whose grid is padded to multiples of 8 (the non-square
grids have widths and heights that are not).
"""
import numpy as np
import pytest

import oracle as O
import paper_2606_27086_gb300 as pk
import synth
from tests.helpers import oracle_objective, random_x, rel, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _one_sweep(prob, mode=O.CIMMINO, lam=1.0, **kw):
    ctx = pk.from_problem(prob, mode=mode, strategy=pk.STRATEGY_ONE_PASS, **kw)
    info = ctx.suppy_info_get()
    x0 = random_x(prob.A.n, 1, seed=91)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(pk.suppy_params_default(lam=lam), 1)
    xg = ctx.suppy_get_x()
    ph, _ = ctx.suppy_history()
    S, l, u, lo, hi = O.from_problem(prob, mode)
    xo, po = O.sweep(S, mode, l, u, lam, lo, hi, x0.astype(np.float64))
    ctx.close()
    return info, xg, ph, xo, po


@pytest.mark.parametrize("mode", [O.CIMMINO, O.BIP])
@pytest.mark.parametrize("tr", [1, 2, -1])
def test_ct_one_sweep(mode, tr):
    prob = synth.ct_problem(160, 120, 227)
    if mode == O.BIP:
        prob.blocks = synth.angle_blocks(120, 227, 12)
    info, xg, ph, xo, po = _one_sweep(prob, mode, scatter_transpose=tr)
    assert info["strategy"] == pk.STRATEGY_ONE_PASS and info["scatter"] == 1
    if tr >= 1:
        # about half of the rays are steeper than 45 degrees
        assert 0.3 * prob.A.m < info["transposed_rows"] < 0.7 * prob.A.m
    else:
        assert info["transposed_rows"] == 0
    assert info["scatter_patch"] == (1 if tr == 2 else 0)
    assert rel_l2(xg, xo) <= 1e-5
    assert rel(ph[0], po) <= 1e-5


@pytest.mark.parametrize("tr", [1, 2])
@pytest.mark.parametrize("shape", [(96, 211), (211, 96), (131, 157)])
def test_non_square_grid(shape, tr):
    H, W = shape
    prob = synth.line_problem(H, W, 1500, seed=H)
    info, xg, ph, xo, po = _one_sweep(prob, lam=1.3, scatter_transpose=tr)
    # segments in uniform directions: about half run down the image
    assert 0.3 * prob.A.m < info["transposed_rows"] < 0.7 * prob.A.m
    assert info["scatter_patch"] == (1 if tr == 2 else 0)
    assert rel_l2(xg, xo) <= 1e-5
    assert rel(ph[0], po) <= 1e-5


@pytest.mark.parametrize("mode", [O.CIMMINO, O.BIP])
def test_two_pass_reads_those_rows_column_major(mode):
    """Two passes: the rows running down the image keep column-major indices
    and gather x from its column-major copy (made before each block's row
    pass)."""
    prob = synth.ct_problem(160, 120, 227)
    if mode == O.BIP:
        prob.blocks = synth.angle_blocks(120, 227, 12)
    ctx = pk.from_problem(prob, mode=mode, strategy=pk.STRATEGY_TWO_PASS, scatter_transpose=1)
    info = ctx.suppy_info_get()
    assert info["strategy"] == pk.STRATEGY_TWO_PASS and info["tma"] == 1
    assert 0.3 * prob.A.m < info["transposed_rows"] < 0.7 * prob.A.m
    x0 = random_x(prob.A.n, 1, seed=92)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(pk.suppy_params_default(lam=1.1), 2)
    S, l, u, lo, hi = O.from_problem(prob, mode)
    x = x0.astype(np.float64)
    for _ in range(2):
        x, po = O.sweep(S, mode, l, u, 1.1, lo, hi, x)
    assert rel_l2(ctx.suppy_get_x(), x) <= 1e-5
    ph, _ = ctx.suppy_history()
    assert rel(ph[-1], po) <= 1e-5
    ctx.close()


def test_two_pass_non_square_grid_and_proximity():
    prob = synth.line_problem(211, 96, 1500, seed=7)
    ctx = pk.from_problem(prob, strategy=pk.STRATEGY_TWO_PASS, scatter_transpose=1)
    assert ctx.suppy_info_get()["transposed_rows"] > 0
    x0 = random_x(prob.A.n, 1, seed=93)
    ctx.suppy_set_x(x0)
    S, l, u, lo, hi = O.from_problem(prob)
    # the standalone proximity keeps reading the row-major indices
    assert rel(float(ctx.suppy_proximity()[0]), O.proximity(S, l, u, x0.astype(np.float64))) <= 1e-5
    ctx.suppy_sweep(pk.suppy_params_default(), 1)
    xo, _ = O.sweep(S, O.CIMMINO, l, u, 1.0, lo, hi, x0.astype(np.float64))
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("tr", [1, 2])
def test_drop_scales_both_accumulators(tr):
    prob = synth.ct_problem(160, 120, 227)
    info, xg, ph, xo, po = _one_sweep(prob, O.DROP, scatter_transpose=tr)
    assert info["transposed_rows"] > 0
    assert rel_l2(xg, xo) <= 1e-5


@pytest.mark.parametrize("tr", [1, 2])
def test_superiorized_run_with_graphs(tr):
    prob = synth.ct_problem(160, 120, 227)
    K = 30
    sup = dict(gamma=0.5, alpha=0.99, n_red=1)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, strategy=pk.STRATEGY_ONE_PASS,
                          scatter_transpose=tr)
    assert ctx.suppy_info_get()["transposed_rows"] > 0
    st = ctx.suppy_run(pk.suppy_params_default(max_sweeps=K, use_graphs=1, **sup))[0]
    S, l, u, lo, hi = O.from_problem(prob)
    r = O.run(S, O.CIMMINO, l, u, lo, hi, oracle_objective(prob, O.OBJ_TV_ISO),
              O.Params(max_sweeps=K, **sup))
    assert st["sweeps"] == K and abs(st["accepted"] - sum(r.accepted)) <= 2
    assert rel_l2(ctx.suppy_get_x(), r.x) <= 1e-3
    ph, fh = ctx.suppy_history()
    assert np.max(np.abs(np.asarray(ph) - r.prox_hist) / np.abs(r.prox_hist)) <= 1e-3
    assert rel(fh[-1], r.obj_hist[-1]) <= 1e-3
    ctx.close()


@pytest.mark.parametrize("start", ["box0", "constant"])
def test_patch_copies_from_the_whole_gpu_phase(start):
    """Superiorized iterations with the whole-GPU perturbation phase before
    each patch-numbered sweep: the phase leaves x in the patch layouts
    (written with each accepted step, or copied when no step is taken) and
    the sweep reads those copies.  Three reduction steps per phase; from a
    constant image the TV subgradient is zero, so the phases take no step
    until the sweeps make the image uneven."""
    prob = synth.ct_problem(160, 120, 227)
    K = 12
    sup = dict(gamma=0.5, alpha=0.99, n_red=3)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, strategy=pk.STRATEGY_ONE_PASS,
                          scatter_transpose=2, perturb_path=2)
    assert ctx.suppy_info_get()["scatter_patch"] == 1
    x0 = np.zeros(prob.A.n, np.float32) if start == "box0" else np.full(prob.A.n, 0.3, np.float32)
    ctx.suppy_set_x(x0)
    st = ctx.suppy_run(pk.suppy_params_default(max_sweeps=K, use_graphs=1, use_stopping=0, **sup))[0]
    S, l, u, lo, hi = O.from_problem(prob)
    r = O.run(S, O.CIMMINO, l, u, lo, hi, oracle_objective(prob, O.OBJ_TV_ISO),
              O.Params(max_sweeps=K, **sup), x0=x0.astype(np.float64))
    assert st["sweeps"] == K and abs(st["accepted"] - sum(r.accepted)) <= 2
    assert rel_l2(ctx.suppy_get_x(), r.x) <= 1e-3
    ph, _ = ctx.suppy_history()
    assert np.max(np.abs(np.asarray(ph[:K]) - r.prox_hist[:K]) / np.abs(r.prox_hist[:K])) <= 1e-3
    ctx.close()


def test_rejections():
    prob = synth.random_problem(300, 30000, seed=3, mean_len=40)   # no image grid
    with pytest.raises(pk.SuppyError):
        pk.from_problem(prob, scatter_transpose=1)
    with pytest.raises(pk.SuppyError):
        pk.from_problem(synth.ct_problem(160, 120, 227), scatter_transpose=3)
    two = synth.ct_problem(160, 120, 227, nrhs=2)
    for tr in (1, 2):
        with pytest.raises(pk.SuppyError):
            pk.from_problem(two, scatter_transpose=tr)


@pytest.mark.parametrize("case", ["ct_cimmino", "ct_bip", "lines"])
def test_patch_numbering_vector_box_and_infinite_bounds(case):
    """The patch numbering's box step with a box per pixel and infinite slab
    bounds: on the CT grid (widths a multiple of 4: the box step's 16-byte
    path; BIP writes the next block's patch copies of x), and on a 131 x 157
    grid (the element-wise path and a padded patch grid)."""
    if case == "lines":
        prob = synth.line_problem(131, 157, 2500, seed=31)
    else:
        prob = synth.ct_problem(160, 120, 227)
    mode = O.BIP if case == "ct_bip" else O.CIMMINO
    if mode == O.BIP:
        prob.blocks = synth.angle_blocks(120, 227, 12)
    n = prob.A.n
    rng = np.random.default_rng(32)
    prob.box_lo = rng.uniform(-0.2, 0.3, size=n).astype(np.float32)
    prob.box_hi = (prob.box_lo + rng.uniform(0.1, 1.0, size=n)).astype(np.float32)
    prob.l = prob.l.copy()
    prob.u = prob.u.copy()
    prob.l[::3] = -np.inf
    prob.u[1::3] = np.inf
    ctx = pk.from_problem(prob, mode=mode, strategy=pk.STRATEGY_ONE_PASS, scatter_transpose=2)
    assert ctx.suppy_info_get()["scatter_patch"] == 1
    x0 = random_x(n, 1, seed=33)
    ctx.suppy_set_x(x0)   # projected onto the box
    ctx.suppy_sweep(pk.suppy_params_default(lam=1.2), 1)
    xg = ctx.suppy_get_x()
    ph, _ = ctx.suppy_history()
    ctx.close()
    S, l, u, lo, hi = O.from_problem(prob, mode)
    x0c = np.clip(x0.astype(np.float64), lo, hi)
    xo, po = O.sweep(S, mode, l, u, 1.2, lo, hi, x0c)
    assert rel_l2(xg, xo) <= 1e-5
    assert np.all(xg >= prob.box_lo) and np.all(xg <= prob.box_hi)
    assert rel(ph[0], po) <= 1e-5


@pytest.mark.parametrize("mode", [O.CIMMINO, O.BIP])
def test_patch_numbering_on_scattered_rows(mode):
    """Rows that are not rays (random columns, 32-88 entries) on a 150 x 170
    grid: any index pattern goes through the stored patch positions, the
    copies and the accumulators, and the box step's element-wise path (170
    is not a multiple of 4)."""
    prob = synth.random_problem(6000, 150 * 170, seed=41, feasible=False, mean_len=60)
    prob.shape = (150, 170)
    if mode == O.BIP:
        prob.blocks = np.arange(prob.A.m) % 5
    info, xg, ph, xo, po = _one_sweep(prob, mode, lam=0.9, scatter_transpose=2)
    assert info["scatter_patch"] == 1
    assert rel_l2(xg, xo) <= 1e-5
    assert rel(ph[0], po) <= 1e-5


def test_device_resident_inputs():
    """A, l, u and the box given as device tensors: the row orientation is
    taken from a host copy of the column indices, the sweep is the same."""
    prob = synth.ct_problem(160, 120, 227)
    info, xg, ph, xo, po = _one_sweep(prob, scatter_transpose=1, device=True)
    assert info["transposed_rows"] > 0
    assert rel_l2(xg, xo) <= 1e-5
