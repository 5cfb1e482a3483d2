"""Parity of the tiled one-pass sweep (strategy 3) with the FP64 oracle.

The tiled sweep cuts the unknowns into one tile per SM, streams each tile's
segments of A (runs of a row's entries in the tile) through a shared-memory
ring, and combines the partial dot products of a row across tiles chunk by
chunk.  These cases force many chunks and a small ring (so slices and chunks
wrap around the ring end, and long rows are split into several segments of
one tile), image tiles and column-range tiles, warp splits from one to 24
dot-product warps, Cimmino, BIP (box after each block) and DROP, FP32 and
16-bit values, infinite bounds and per-unknown boxes, several sweeps in one
call (the alternating accumulators), and superiorized runs with CUDA graphs.

Tolerance: one sweep from the same point <= 1e-5 relative L2 against the
oracle (FP32 arithmetic; the order of the FP32 additions is not fixed), a
superiorized run <= 1e-3 (the run's bound: TV subgradient directions at
near-ties amplify FP32 rounding over the iterations).
"""
import numpy as np
import pytest

import oracle as O
import paper_2606_27086_gb300 as pk
import synth
from tests.helpers import oracle_objective, random_x, rel, rel_l2, rounded_values, small_ct

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DT = {"f32": pk.SUPPY_F32, "bf16": pk.SUPPY_BF16, "f16": pk.SUPPY_F16}
# a small ring (8 pieces of 1 KB) and small chunks: every tile's stream wraps
# around the ring many times and spans dozens of chunks
SMALL = dict(tile_ring_bytes=8 * 1024, tile_chunk_bytes=256)


def _params(**kw):
    return pk.suppy_params_default(**kw)


def _oracle_sweeps(prob, x, mode=O.CIMMINO, dtype="f32", lam=1.0, k=1):
    vals = rounded_values(prob.A.val, dtype)
    S, l, u, lo, hi = O.from_problem(prob, mode, values=vals)
    x = np.asarray(x, np.float64)
    ps = []
    for _ in range(k):
        x, p = O.sweep(S, mode, l, u, lam, lo, hi, x)
        ps.append(p)
    return x, ps


def _tiled(prob, **kw):
    ctx = pk.from_problem(prob, strategy=pk.STRATEGY_TILED, **kw)
    info = ctx.suppy_info_get()
    assert info["strategy"] == 3 and info["tiles"] > 1 and info["chunks"] >= 1
    return ctx, info


@pytest.mark.parametrize("warps1", [1, 4, 12, 24])
def test_tiled_one_sweep_ct_small_ring(warps1):
    prob = small_ct()
    ctx, info = _tiled(prob, tile_warps1=warps1, **SMALL)
    assert info["tile_warps1"] == warps1
    assert info["tile_warps2"] == 26 - warps1 and info["tile_coef_warps"] == 4
    assert info["chunks"] > 20 and info["tile_ring"] == 8192
    # every tile's stream is longer than the ring
    assert info["tile_stream_bytes"] > 3 * info["tiles"] * info["tile_ring"]
    x0 = random_x(prob.A.n, 1, seed=11)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(), 1)
    xo, po = _oracle_sweeps(prob, x0)
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
    ph, _ = ctx.suppy_history()
    assert len(ph) == 1 and rel(ph[0], po[0]) <= 1e-5
    ctx.close()


def test_tiled_default_shape_and_several_sweeps():
    """Five sweeps in one call: the row accumulators alternate between two
    buffers (one cleared while the other accumulates) and the chunk counters
    are reset by the last CTA of every launch."""
    prob = synth.ct_problem(96, 120, 137)
    ctx, info = _tiled(prob)
    x0 = random_x(prob.A.n, 1, seed=12)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(), 5)
    xo, po = _oracle_sweeps(prob, x0, k=5)
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
    ph, _ = ctx.suppy_history()
    assert len(ph) == 5
    for a, b in zip(ph, po):
        assert rel(a, b) <= 1e-5
    # the standalone proximity (another kernel) at the result
    S, l, u, lo, hi = O.from_problem(prob)
    assert rel(float(ctx.suppy_proximity()[0]), O.proximity(S, l, u, xo)) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("n", [3001, 20011, 120000])
@pytest.mark.parametrize("mean_len,long_len", [(3, 0), (30, 0), (300, 0), (40, 2100), (250, 5000)])
def test_tiled_row_length_mix(mean_len, long_len, n):
    """Column-range tiles (no image grid), ragged rows, empty rows, rows far
    longer than a segment (split into several segments of one tile), lambda
    1 and 1.7."""
    prob = synth.random_problem(700, n, seed=mean_len + long_len + n, feasible=False,
                                mean_len=mean_len, empty_frac=0.05,
                                long_rows=7 if long_len else 0, long_len=long_len)
    ctx, info = _tiled(prob, **SMALL)
    x0 = random_x(n, 1, seed=13)
    for lam in (1.0, 1.7):
        ctx.suppy_set_x(x0)
        ctx.suppy_sweep(_params(lam=lam), 1)
        xo, po = _oracle_sweeps(prob, x0, lam=lam)
        assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
        ph, _ = ctx.suppy_history()
        assert rel(ph[0], po[0]) <= 1e-5
    ctx.close()


def test_tiled_vector_box_and_infinite_bounds():
    n = 5000
    prob = synth.random_problem(3000, n, seed=15, feasible=False, mean_len=25)
    rng = np.random.default_rng(15)
    prob.box_lo = rng.uniform(-0.2, 0.3, size=n).astype(np.float32)
    prob.box_hi = (prob.box_lo + rng.uniform(0.1, 1.0, size=n)).astype(np.float32)
    prob.l[::3] = -np.inf
    prob.u[1::3] = np.inf
    ctx, _ = _tiled(prob)
    x0 = random_x(n, 1, seed=16, lo=-1, hi=2)
    ctx.suppy_set_x(x0)
    x0c = np.clip(x0, prob.box_lo, prob.box_hi)
    ctx.suppy_sweep(_params(), 2)
    xo, _ = _oracle_sweeps(prob, x0c, k=2)
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("small", [False, True])
def test_tiled_block_iterative(small):
    """BIP with 10 interleaved angle blocks: the box step after every block,
    the next block's dot products from the updated tile."""
    prob = small_ct()
    prob.blocks = synth.angle_blocks(90, 91, 10)
    kw = SMALL if small else {}
    ctx, info = _tiled(prob, mode=pk.SUPPY_BIP, **kw)
    assert info["chunks"] >= 10
    x0 = random_x(prob.A.n, 1, seed=17)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(), 2)
    xo, po = _oracle_sweeps(prob, x0, mode=O.BIP, k=2)
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
    ph, _ = ctx.suppy_history()
    assert rel(ph[0], po[0]) <= 1e-5 and rel(ph[1], po[1]) <= 1e-5
    ctx.close()


def test_tiled_drop():
    prob = small_ct()
    ctx, _ = _tiled(prob, mode=pk.SUPPY_DROP, **SMALL)
    x0 = random_x(prob.A.n, 1, seed=18)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(), 2)
    xo, po = _oracle_sweeps(prob, x0, mode=O.DROP, k=2)
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
    ph, _ = ctx.suppy_history()
    assert rel(ph[1], po[1]) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_tiled_low_precision_values(dtype):
    """16-bit values: parity against the oracle on the rounded values."""
    prob = small_ct()
    ctx, _ = _tiled(prob, dtype=DT[dtype], **SMALL)
    x0 = random_x(prob.A.n, 1, seed=19)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(), 1)
    xo, _ = _oracle_sweeps(prob, x0, dtype=dtype)
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("mode", [O.CIMMINO, O.BIP])
def test_tiled_superiorized_run_with_graphs(mode):
    """Algorithm 1 with TV perturbations over 25 iterations (one captured
    iteration replayed) against the oracle: same accepted steps and exponent,
    iterate and histories within 1e-3."""
    prob = synth.ct_problem(96, 120, 137)
    if mode == O.BIP:
        prob.blocks = synth.angle_blocks(120, 137, 12)
    ctx, _ = _tiled(prob, mode=mode, obj=pk.SUPPY_OBJ_TV_ISO)
    P = dict(gamma=0.5, alpha=0.99, n_red=1, max_sweeps=25)
    x0 = random_x(prob.A.n, 1, seed=20)
    ctx.suppy_set_x(x0)
    st = ctx.suppy_run(pk.suppy_params_default(use_graphs=1, **P))[0]
    S, l, u, lo, hi = O.from_problem(prob, mode)
    r = O.run(S, mode, l, u, lo, hi, oracle_objective(prob, O.OBJ_TV_ISO), O.Params(**P),
              x0=x0.astype(np.float64))
    assert st["sweeps"] == 25
    assert st["accepted"] == sum(r.accepted) and st["ell"] == r.ell
    assert rel_l2(ctx.suppy_get_x(), r.x) <= 1e-3
    ph, _ = ctx.suppy_history()
    po = np.asarray(r.prox_hist)
    assert np.max(np.abs(np.asarray(ph) - po) / np.abs(po)) <= 1e-3
    ctx.close()


def test_tiled_is_rejected_where_it_does_not_apply():
    prob = small_ct()
    with pytest.raises(pk.SuppyError) as e:
        pk.from_problem(prob, mode=pk.SUPPY_EMR, strategy=pk.STRATEGY_TILED)
    assert e.value.status == pk.SUPPY_EINVAL
    prob2 = synth.ct_problem(32, 40, 45, nrhs=3)
    with pytest.raises(pk.SuppyError) as e:
        pk.from_problem(prob2, strategy=pk.STRATEGY_TILED)
    assert e.value.status == pk.SUPPY_EINVAL
    with pytest.raises(pk.SuppyError):
        pk.from_problem(prob, strategy=pk.STRATEGY_TILED, tile_warps1=26)
    with pytest.raises(pk.SuppyError):
        pk.from_problem(prob, strategy=pk.STRATEGY_TILED, tile_ring_bytes=1000)
