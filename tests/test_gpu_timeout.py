"""Bounded device waits that run out (Sec. 2.1.1's sweep and Algorithm 1's
perturbation phase, in the kernels that wait on other CTAs or on bulk
copies): with a budget of a few SM cycles a wait gives up, the kernel stops,
the next synchronizing call returns SUPPY_ETIMEOUT, and after the default
budget is restored the same context computes what the oracle computes.  No
GPU fault is involved: the waits return, their CTAs reach the end of the
launch, and the host resets the synchronisation words."""
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

SHORT = 1   # SM cycles: any wait that is not over at its first look gives up


def _oracle_sweep(prob, x, mode=O.CIMMINO):
    S, l, u, lo, hi = O.from_problem(prob, mode)
    return O.sweep(S, mode, l, u, 1.0, lo, hi, np.asarray(x, np.float64))


def _timeout_then_parity(prob, ctx, mode=O.CIMMINO):
    x0 = random_x(prob.A.n, 1, seed=31)
    ctx.suppy_set_x(x0)
    ctx.suppy_set_wait_limit(SHORT)
    with pytest.raises(pk.SuppyError) as e:
        ctx.suppy_sweep(pk.suppy_params_default(use_graphs=0), 1)
        ctx.suppy_get_x()   # a synchronizing call reports it at the latest
    assert e.value.status == pk.SUPPY_ETIMEOUT
    ctx.suppy_set_wait_limit(0)
    for seed in (32, 33):
        x1 = random_x(prob.A.n, 1, seed=seed)
        ctx.suppy_set_x(x1)
        ctx.suppy_sweep(pk.suppy_params_default(use_graphs=0), 1)
        xo, _ = _oracle_sweep(prob, x1, mode)
        assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5


def test_tiled_sweep_wait_runs_out_and_context_recovers():
    prob = synth.ct_problem(96, 120, 137)
    ctx = pk.from_problem(prob, strategy=pk.STRATEGY_TILED)
    _timeout_then_parity(prob, ctx)
    ctx.close()


def test_tiled_block_iterative_wait_runs_out_and_context_recovers():
    prob = synth.ct_problem(96, 120, 137)
    prob.blocks = synth.angle_blocks(120, 137, 12)
    ctx = pk.from_problem(prob, mode=pk.SUPPY_BIP, strategy=pk.STRATEGY_TILED)
    _timeout_then_parity(prob, ctx, O.BIP)
    ctx.close()


def test_streamed_pass_wait_runs_out_and_context_recovers():
    prob = synth.ct_problem(160, 60, 227)
    ctx = pk.from_problem(prob, strategy=pk.STRATEGY_TWO_PASS)
    assert ctx.suppy_info_get()["tma"] == 1
    _timeout_then_parity(prob, ctx)
    ctx.close()


def test_whole_gpu_perturbation_barrier_runs_out_and_context_recovers():
    """The cooperative perturbation phase's grid barrier gives up; afterwards
    the phase (and a whole superiorized run) matches the oracle again, so the
    barrier's arrival count was reset."""
    prob = synth.ct_problem(256, 90, 363)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, perturb_path=2)
    x0 = random_x(prob.A.n, 1, seed=34)
    ctx.suppy_set_x(x0)
    ctx.suppy_set_wait_limit(SHORT)
    P = dict(gamma=0.5, alpha=0.99, n_red=3, max_sweeps=4)
    with pytest.raises(pk.SuppyError) as e:
        ctx.suppy_run(pk.suppy_params_default(use_graphs=0, **P))
    assert e.value.status == pk.SUPPY_ETIMEOUT
    ctx.suppy_set_wait_limit(0)
    ctx.suppy_set_x(x0)
    st = ctx.suppy_run(pk.suppy_params_default(use_graphs=1, **P))[0]
    S, l, u, lo, hi = O.from_problem(prob)
    r = O.run(S, O.CIMMINO, l, u, lo, hi, oracle_objective(prob, O.OBJ_TV_ISO), O.Params(**P),
              x0=x0.astype(np.float64))
    assert st["accepted"] == sum(r.accepted)
    assert rel_l2(ctx.suppy_get_x(), r.x) <= 1e-4
    ctx.close()
