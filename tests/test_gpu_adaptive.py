"""GPU parity of the adaptive perturbation step (Nikazad et al., Sec. 2.1.2)
against the FP64 oracle, on every perturbation path: the cluster kernel with
the image in shared memory or in global memory, and the whole-GPU phase
kernel (one cooperative launch)."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import oracle_objective, random_x, rel_l2

pk = pytest.importorskip("paper_2606_27086_gb300")

pytestmark = pytest.mark.gpu


def _params(**kw):
    return pk.suppy_params_default(**kw)


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("n_red", [1, 3])
@pytest.mark.parametrize("kind", ["tv", "atv", "l1"])
def test_fixed_reference_phase_matches_oracle(kind, n_red, path):
    """adaptive = 2: beta = (f(y) - f_ref)/||g||, one trial per reduction
    step; the accepted steps and the point match the oracle's phase."""
    prob = synth.ct_problem(128, 60, 181)
    obj = {"tv": pk.SUPPY_OBJ_TV_ISO, "atv": pk.SUPPY_OBJ_TV_ANISO, "l1": pk.SUPPY_OBJ_L1}[kind]
    okind = {"tv": O.OBJ_TV_ISO, "atv": O.OBJ_TV_ANISO, "l1": O.OBJ_L1}[kind]
    x0 = random_x(prob.A.n, 1, seed=81)
    ob = oracle_objective(prob, okind)
    f0 = ob.f(x0.astype(np.float64))
    f_ref = 0.97 * f0
    y, a, t = O.perturbation_phase(ob, x0.astype(np.float64), O.PertState(),
                                   O.Params(adaptive=2, f_ref=f_ref, n_red=n_red))
    assert a >= 1
    ctx = pk.from_problem(prob, obj=obj, perturb_path=path)
    ctx.suppy_set_x(x0)
    acc = ctx.suppy_perturb(_params(adaptive=2, f_ref=f_ref, n_red=n_red))
    st = ctx.suppy_run(_params(max_sweeps=0))[0]
    assert acc[0] == a and st["trials"] == t
    assert st["ell"] == 0                      # the power-law exponent is not used
    assert rel_l2(ctx.suppy_get_x(), y) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("path", [1, 2])
def test_automatic_reference_run_matches_oracle_radiotherapy(path):
    """adaptive = 1 on the mean dose: the reference is the lowest phase-start
    objective so far, so the first phases take no step and later ones pull
    the mean dose back to it; ten superiorized BIP iterations."""
    rt = synth.rt_problem(nx=30, ny=20, nz=12, ns=9, nzb=7)
    S, l, u, lo, hi = O.from_problem(rt, O.BIP)
    ob = oracle_objective(rt, O.OBJ_LINEAR)
    x0 = np.ones(rt.A.n, np.float32)
    K = 10
    r = O.run(S, O.BIP, l, u, lo, hi, ob, O.Params(adaptive=1, max_sweeps=K),
              x0=x0.astype(np.float64))
    assert r.accepted[0] == 0 and sum(r.accepted) >= 2
    ctx = pk.from_problem(rt, mode=pk.SUPPY_BIP, obj=pk.SUPPY_OBJ_LINEAR, perturb_path=path)
    ctx.suppy_set_x(x0)
    st = ctx.suppy_run(_params(adaptive=1, max_sweeps=K, use_stopping=0))[0]
    _, oh = ctx.suppy_history(0)
    assert st["sweeps"] == K
    assert st["accepted"] == sum(r.accepted)
    assert np.allclose(oh[:K], r.obj_hist, rtol=1e-5)
    assert rel_l2(ctx.suppy_get_x(), r.x) <= 1e-4
    ctx.close()


def test_automatic_reference_tv_run_and_batched_references():
    """adaptive = 1 on TV with four right-hand sides (each keeps its own
    reference), graphs on: iterates and objective histories match the
    oracle run of each right-hand side."""
    prob = synth.ct_problem(nrhs=4)
    x0 = random_x(prob.A.n, 4, seed=83)
    K = 8
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO)
    ctx.suppy_set_x(x0)
    ctx.suppy_run(_params(adaptive=1, max_sweeps=K, use_stopping=0))
    xg = ctx.suppy_get_x()
    ob = oracle_objective(prob, O.OBJ_TV_ISO)
    for b in range(4):
        S, l, u, lo, hi = O.from_problem(prob)
        l, u = O.rhs(prob.l, b), O.rhs(prob.u, b)
        S = O.setup(S.A, l, u)
        r = O.run(S, O.CIMMINO, l, u, lo, hi, ob, O.Params(adaptive=1, max_sweeps=K),
                  x0=x0[:, b].astype(np.float64))
        _, oh = ctx.suppy_history(b)
        assert np.allclose(oh[:K], r.obj_hist, rtol=1e-5)
        assert rel_l2(xg[:, b], r.x) <= 1e-4
    ctx.close()


def test_adaptive_parameters_are_validated():
    prob = synth.ct_problem()
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO)
    for kw in (dict(adaptive=3), dict(adaptive=2, f_ref=float("inf")), dict(adaptive=-1)):
        with pytest.raises(pk.SuppyError) as e:
            ctx.suppy_perturb(_params(**kw))
        assert e.value.status == pk.SUPPY_EINVAL
    ctx.close()


def test_checkpoint_keeps_the_adaptive_reference():
    """The automatic reference value travels in the checkpoint: a restored
    context continues the adaptive run exactly as the uninterrupted one (the
    two-pass sweep and the fixed-order perturbation are bitwise
    reproducible)."""
    rt = synth.rt_problem(nx=30, ny=20, nz=12, ns=9, nzb=7)
    P = _params(adaptive=1, max_sweeps=5, use_stopping=0)
    ctx = pk.from_problem(rt, mode=pk.SUPPY_BIP, obj=pk.SUPPY_OBJ_LINEAR,
                          strategy=pk.STRATEGY_TWO_PASS)
    ctx.suppy_set_x(np.ones(rt.A.n, np.float32))
    ctx.suppy_run(P)
    blob = ctx.suppy_get_state()
    ctx.suppy_run(P)
    x_a = ctx.suppy_get_x().copy()
    st_a = ctx.suppy_run(_params(adaptive=1, max_sweeps=0))[0]
    ctx.suppy_set_state(blob)
    ctx.suppy_run(P)
    st_b = ctx.suppy_run(_params(adaptive=1, max_sweeps=0))[0]
    assert np.array_equal(ctx.suppy_get_x(), x_a)
    assert st_b["accepted"] == st_a["accepted"] and st_a["accepted"] >= 2
    ctx.close()
