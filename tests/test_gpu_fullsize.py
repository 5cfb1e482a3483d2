"""GPU parity at the benchmark's full sizes, in the launch configuration the
benchmark times, against the FP64 oracle.

CT 512x512 (m = 261000, n = 262144, 1.2e8 nonzeros): the one-pass sweep with
the strategy form and TMA shapes tuned at create, as the headline runs it (the
patch numbering), and the two-pass sweep tuned the same way.  The oracle computes a
whole sweep at this size in about a second (scipy sparse products), so every
output is compared, not a sample.  Seismic (16 right-hand sides, 4e7
nonzeros): right-hand sides 0, 7 and 15 of one batched sweep.  The
radiotherapy split problem: one CQ step at full size, the oracle deciding on
the device's doses."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import oracle_objective, random_x, rel, rel_l2

pk = pytest.importorskip("paper_2606_27086_gb300")

pytestmark = pytest.mark.gpu

CT512 = dict(N=512, nang=360, nbin=725, I0=5e3, delta=0.02, seed_phantom=201, seed_noise=202)
SUP = dict(gamma=0.5, alpha=0.99, n_red=1)


@pytest.fixture(scope="module")
def ct512():
    prob = synth.ct_problem(**CT512)
    S, l, u, lo, hi = O.from_problem(prob)
    return prob, (S, l, u, lo, hi)


@pytest.fixture(scope="module", params=[pk.STRATEGY_ONE_PASS, pk.STRATEGY_TWO_PASS])
def ct512_ctx(ct512, request):
    prob, _ = ct512
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, tune=1, strategy=request.param)
    yield ctx
    ctx.close()


def test_ct512_headline_sweep_every_output(ct512, ct512_ctx):
    prob, (S, l, u, lo, hi) = ct512
    ctx = ct512_ctx
    info = ctx.suppy_info_get()
    assert info["tma"] == 1
    if info["strategy"] == 1:
        # the tuner times the row-/column-major and patch numberings; the
        # patch numbering is the fastest form here by about a quarter
        assert info["scatter"] == 1 and info["scatter_patch"] == 1
    else:
        assert info["strategy"] == 2
    assert prob.A.nnz == 120309216
    x0 = random_x(prob.A.n, 1, seed=501)
    ctx.suppy_set_x(x0)
    p0 = float(ctx.suppy_proximity()[0])
    ctx.suppy_sweep(pk.suppy_params_default(use_graphs=0), 1)
    x1 = ctx.suppy_get_x()
    p1 = float(ctx.suppy_proximity()[0])
    xo, po_in = O.sweep(S, O.CIMMINO, l, u, 1.0, lo, hi, x0.astype(np.float64))
    ph, _ = ctx.suppy_history(0)
    assert rel(p0, O.proximity(S, l, u, x0.astype(np.float64))) < 1e-5
    assert rel(ph[0], po_in) < 1e-5
    assert rel(p1, O.proximity(S, l, u, xo)) < 1e-4
    assert rel_l2(x1, xo) < 1e-5
    assert np.max(np.abs(x1 - xo)) < 1e-5


def test_ct512_superiorized_iterations_with_graphs(ct512, ct512_ctx):
    """Three headline iterations (TV perturbation, one- or two-pass sweep,
    graphs) from the benchmark's start point box(0) and from a seeded point."""
    prob, (S, l, u, lo, hi) = ct512
    ctx = ct512_ctx
    ob = oracle_objective(prob, O.OBJ_TV_ISO)
    K = 3
    for x0 in (np.zeros(prob.A.n, np.float32), random_x(prob.A.n, 1, seed=502)):
        ctx.suppy_set_x(x0)
        st = ctx.suppy_run(pk.suppy_params_default(max_sweeps=K, use_stopping=0, **SUP))[0]
        xg = ctx.suppy_get_x()
        ph, oh = ctx.suppy_history(0)
        r = O.run(S, O.CIMMINO, l, u, lo, hi, ob, O.Params(max_sweeps=K, **SUP),
                  x0=x0.astype(np.float64))
        assert st["sweeps"] == K and st["accepted"] == sum(r.accepted)
        assert st["ell"] == r.ell
        assert np.allclose(ph[:K], r.prox_hist, rtol=1e-4)
        assert np.allclose(oh[:K], r.obj_hist, rtol=1e-5, atol=1e-9)
        assert rel_l2(xg, r.x) < 1e-5


def test_seismic_batched_sweep_sampled_right_hand_sides():
    prob = synth.seismic_problem(nrhs=16)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ANISO)
    x0 = random_x(prob.A.n, 16, seed=503, lo=1 / 6, hi=1 / 1.5)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(pk.suppy_params_default(use_graphs=0), 1)
    xg = ctx.suppy_get_x()
    ctx.close()
    S, _, _, lo, hi = O.from_problem(prob)
    for b in (0, 7, 15):
        l, u = O.rhs(prob.l, b), O.rhs(prob.u, b)
        Sb = O.setup(S.A, l, u)
        xo, _ = O.sweep(Sb, O.CIMMINO, l, u, 1.0, lo, hi, x0[:, b].astype(np.float64))
        assert rel_l2(xg[:, b], xo) < 1e-5


def test_radiotherapy_split_cq_step_full_size():
    prob = synth.rt_split_problem()
    sp = prob.meta["split"]
    Aq = sp["Aq"]
    n = prob.A.n
    l = np.full(Aq.m, -np.inf, np.float32)
    ctx = pk.Context(Aq.row_ptr, Aq.col, Aq.val, Aq.m, n, l, -l, np.full(1, -np.inf, np.float32),
                     np.full(1, np.inf, np.float32))
    ctx.suppy_set_dvc(Aq.row_ptr, Aq.col, Aq.val, Aq.m, sp["sptr"], sp["dvcs"], 1.0)
    x0 = np.ones(n, np.float32)
    ctx.suppy_set_x(x0)
    d = ctx.suppy_dvc_dose().astype(np.float64)
    pq = ctx.suppy_dvc_proximity()
    ctx.suppy_sweep(pk.suppy_params_default(use_graphs=0), 1)
    xg = ctx.suppy_get_x()
    ctx.close()
    SS = O.split_setup(Aq.to_scipy(), sp["sptr"], [O.DVC(*q) for q in sp["dvcs"]], 1.0)
    assert rel_l2(d, SS.Aq @ x0.astype(np.float64)) < 1e-6
    c, po = O.dvc_corrections(SS, d)
    assert po > 0 and rel(pq, po) < 1e-11
    xo = x0.astype(np.float64) + SS.gamma * (SS.Aq.T @ c)
    assert rel_l2(xg, xo) < 1e-5
