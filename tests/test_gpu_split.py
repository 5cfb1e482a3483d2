"""GPU parity of the split-feasibility path (dose-volume constraints, the CQ
step of Sec. 2.1.1) against the FP64 oracle.

Selections of the projection (which voxels keep their dose) are decided on
float doses; the tests hand the oracle the device's own doses where the
doses are not exact, so that both sides decide on the same numbers, and use
integer-valued matrices and iterates (exact doses in FP32) to compare the
whole step, ties included."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import oracle_objective, rel, rel_l2

pk = pytest.importorskip("paper_2606_27086_gb300")

pytestmark = pytest.mark.gpu

F32 = np.float32
# The device sums the squared corrections in float-float arithmetic (about 44
# significant bits) over short per-thread runs and a fixed-order tree: the
# proximity carries a relative error of a few 2^-44 at most.
PROX_TOL = 1e-11


def _identity_ctx(Aq, n, obj=None):
    """A context whose slabs (l = -inf, u = +inf) and box never move x, so one
    sweep is exactly the CQ step."""
    l = np.full(Aq.m, -np.inf, F32)
    u = np.full(Aq.m, np.inf, F32)
    return pk.Context(Aq.row_ptr, Aq.col, Aq.val, Aq.m, n, l, u, np.full(1, -np.inf, F32),
                      np.full(1, np.inf, F32))


def _oracle_split(Aq, sptr, dvcs, relax):
    return O.split_setup(Aq.to_scipy(), sptr, [O.DVC(*q) for q in dvcs], relax)


def _integer_case(seed, sizes, n=300, mean_len=24):
    """Integer values in {1,2,3} and an integer iterate: every dose is an exact
    integer in FP32 whatever the summation order, and many doses tie."""
    rng = np.random.default_rng(seed)
    m = int(sum(sizes))
    A = synth.random_csr(m, n, seed, mean_len=mean_len)
    A.val[:] = rng.integers(1, 4, size=A.nnz).astype(F32)
    sptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    x = rng.integers(0, 4, size=n).astype(F32)
    return A, sptr, x


def _step_compare(A, sptr, dvcs, x, relax, tol=2e-6):
    ctx = _identity_ctx(A, A.n)
    ctx.suppy_set_dvc(A.row_ptr, A.col, A.val, A.m, sptr, dvcs, relax)
    ctx.suppy_set_x(x)
    d = ctx.suppy_dvc_dose()
    SS = _oracle_split(A, sptr, dvcs, relax)
    d_ref = A.to_scipy() @ x.astype(np.float64)
    p_gpu = ctx.suppy_dvc_proximity()
    p = pk.suppy_params_default(use_graphs=0)
    ctx.suppy_sweep(p, 1)
    xg = ctx.suppy_get_x()
    ctx.close()
    return d, d_ref, p_gpu, xg, SS


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cq_step_is_exact_on_integer_doses_with_ties(seed):
    """Structures of 3000 and 2500 rows (several 1024-row tiles) and one of
    40; three DVCs on the first structure (the lowest rows win ties), one
    each on the others; every decision and the proximity match exactly, the
    step to FP32 rounding."""
    A, sptr, x = _integer_case(seed, [3000, 2500, 40])
    d0 = A.to_scipy() @ x.astype(np.float64)
    q = lambda s, f: float(np.quantile(d0[sptr[s]:sptr[s + 1]], f))
    dvcs = [(1, 0, 0.9, q(0, 0.5) + 0.5), (0, 0, 0.1, q(0, 0.6)), (0, 0, 0.3, q(0, 0.2) - 0.25),
            (0, 1, 0.05, q(1, 0.5)), (1, 2, 0.8, q(2, 0.9))]
    d, d_exact, p_gpu, xg, SS = _step_compare(A, sptr, dvcs, x, 1.3)
    assert np.array_equal(d.astype(np.float64), d_exact)
    assert len(np.unique(d)) < len(d) // 4            # ties are common
    xo, po = O.cq_step(SS, x.astype(np.float64))
    assert po > 0
    assert rel(p_gpu, po) < PROX_TOL
    assert rel_l2(xg, xo) < 2e-6


def test_cq_step_on_a_structure_too_large_for_shared_memory():
    """A structure of 60000 rows (its keys do not fit in shared memory: every
    pass re-reads the doses) next to a small one; exact decisions as above."""
    A, sptr, x = _integer_case(21, [60000, 40], mean_len=8)
    d0 = A.to_scipy() @ x.astype(np.float64)
    dvcs = [(0, 0, 0.15, float(np.quantile(d0[:60000], 0.5))),
            (1, 0, 0.7, float(np.quantile(d0[:60000], 0.4)) + 0.5),
            (0, 1, 0.1, float(np.quantile(d0[60000:], 0.3)))]
    d, d_exact, p_gpu, xg, SS = _step_compare(A, sptr, dvcs, x, 1.0)
    assert np.array_equal(d.astype(np.float64), d_exact)
    xo, po = O.cq_step(SS, x.astype(np.float64))
    assert po > 0
    assert rel(p_gpu, po) < PROX_TOL
    assert rel_l2(xg, xo) < 2e-6


@pytest.mark.parametrize("seed", [3, 4])
def test_cq_step_on_float_doses_decides_like_the_oracle(seed):
    """Continuous values: the oracle takes the device's doses, so both sides
    make the same selections; proximity to FP64 summation order, the step to
    FP32 rounding."""
    rng = np.random.default_rng(seed)
    A = synth.random_csr(5000, 700, seed, mean_len=40)
    A.val[:] = rng.uniform(0.1, 1.0, size=A.nnz).astype(F32)
    sptr = np.array([0, 1800, 1800, 5000], np.int32)          # an empty structure too
    x = rng.uniform(0, 1, size=700).astype(F32)
    d0 = A.to_scipy() @ x.astype(np.float64)
    dvcs = [(1, 0, 0.95, float(np.quantile(d0[:1800], 0.3))),
            (0, 0, 0.05, float(np.quantile(d0[:1800], 0.8))),
            (0, 2, 0.2, float(np.quantile(d0[1800:], 0.5))),
            (0, 1, 0.0, 0.0)]
    d, d_exact, p_gpu, xg, SS = _step_compare(A, sptr, dvcs, x, 1.0)
    assert rel_l2(d, d_exact) < 1e-6
    c, po = O.dvc_corrections(SS, d.astype(np.float64))
    assert rel(p_gpu, po) < PROX_TOL
    xo = x.astype(np.float64) + SS.gamma * (SS.Aq.T @ c)
    assert rel_l2(xg, xo) < 2e-6


def test_extreme_volumes_and_satisfied_constraints():
    """V = 0 (upper) clamps every dose above d_ref, V = 1 (lower) raises every
    dose below it; a satisfied DVC leaves the iterate and adds no proximity."""
    A, sptr, x = _integer_case(7, [1500, 1200])
    d0 = A.to_scipy() @ x.astype(np.float64)
    for dvcs in ([(0, 0, 0.0, float(np.median(d0[:1500])))],
                 [(1, 1, 1.0, float(np.median(d0[1500:])))],
                 [(0, 0, 0.5, float(d0.max()) + 1.0), (1, 1, 0.5, float(d0.min()) - 1.0)]):
        d, d_exact, p_gpu, xg, SS = _step_compare(A, sptr, dvcs, x, 1.0)
        xo, po = O.cq_step(SS, x.astype(np.float64))
        assert rel(p_gpu, po) < PROX_TOL if po > 0 else p_gpu == 0.0
        if po == 0:
            assert np.array_equal(xg, x)
        else:
            assert rel_l2(xg, xo) < 2e-6


def _split_ctx(prob, mode, obj, strategy=0):
    ctx = pk.from_problem(prob, mode=mode, obj=obj, strategy=strategy)
    sp = prob.meta["split"]
    Aq = sp["Aq"]
    ctx.suppy_set_dvc(Aq.row_ptr, Aq.col, Aq.val, Aq.m, sp["sptr"], sp["dvcs"], 1.0)
    return ctx


@pytest.mark.parametrize("mode,omode", [(pk.SUPPY_CIMMINO, O.CIMMINO), (pk.SUPPY_EMR, O.EMR)])
def test_superiorized_split_run_matches_the_oracle(mode, omode):
    """The horseshoe split problem (small grid), mean-dose perturbations with
    gamma = 1, alpha = 0.7 as in the paper's horseshoe plan: 12 iterations of
    [perturbation, CQ step, slab sweep, box]; the monitored proximity is the
    target-space one."""
    prob = synth.rt_split_problem(nx=24, ny=20, nz=12, ns=8, nzb=6)
    sp = prob.meta["split"]
    K = 12
    ctx = _split_ctx(prob, mode, pk.SUPPY_OBJ_LINEAR)
    x0 = np.full(prob.A.n, 1.0, F32)
    ctx.suppy_set_x(x0)
    p = pk.suppy_params_default(gamma=1.0, alpha=0.7, n_red=1, max_sweeps=K, use_stopping=0)
    st = ctx.suppy_run(p)
    xg = ctx.suppy_get_x()
    ph, oh = ctx.suppy_history(0)
    ctx.close()
    S, l, u, lo, hi = O.from_problem(prob, omode)
    SS = _oracle_split(sp["Aq"], sp["sptr"], sp["dvcs"], 1.0)
    obj = oracle_objective(prob, O.OBJ_LINEAR)
    P = O.Params(gamma=1.0, alpha=0.7, n_red=1, max_sweeps=K)
    r = O.run(S, omode, l, u, lo, hi, obj, P, x0=x0.astype(np.float64), split=SS)
    assert st[0]["sweeps"] == K
    assert rel_l2(xg, r.x) < 1e-4
    assert np.allclose(ph[:K], r.prox_hist, rtol=1e-4, atol=0)
    assert r.prox_hist[0] > r.prox_hist[-1] > 0


def test_graphs_and_plain_launches_agree_bitwise():
    """The CQ kernels, the two-pass sweep and the perturbation all sum in a
    fixed order, so captured and plain launches give the same bits."""
    prob = synth.rt_split_problem(nx=24, ny=20, nz=12, ns=8, nzb=6)
    xs = []
    for graphs in (0, 1):
        ctx = _split_ctx(prob, pk.SUPPY_CIMMINO, pk.SUPPY_OBJ_LINEAR, pk.STRATEGY_TWO_PASS)
        ctx.suppy_set_x(np.full(prob.A.n, 1.0, F32))
        ctx.suppy_run(pk.suppy_params_default(gamma=1.0, alpha=0.7, max_sweeps=8, use_graphs=graphs))
        xs.append(ctx.suppy_get_x())
        ctx.close()
    assert np.array_equal(xs[0], xs[1])


def test_stopping_uses_the_target_space_proximity():
    """Sec. 2.2.1: for split problems the stopping rule looks at the target
    space.  With P* between the slab proximity and the DVC proximity of the
    start point, the run must not stop after the first sweep; with P* above
    the DVC proximity it stops there and records that value."""
    prob = synth.rt_split_problem(nx=24, ny=20, nz=12, ns=8, nzb=6)
    x0 = np.full(prob.A.n, 1.0, F32)
    ctx = _split_ctx(prob, pk.SUPPY_CIMMINO, pk.SUPPY_OBJ_NONE)
    ctx.suppy_set_x(x0)
    pq = ctx.suppy_dvc_proximity()
    pc = float(ctx.suppy_proximity()[0])
    assert pc < pq
    p = pk.suppy_params_default(max_sweeps=5, use_stopping=1, prox_abs=(pc + pq) / 2,
                                prox_rel=0.0, check_every=1)
    st = ctx.suppy_run(p)
    assert st[0]["sweeps"] > 1
    ctx.suppy_set_x(x0)
    p.prox_abs = 2 * pq
    st = ctx.suppy_run(p)
    ph, _ = ctx.suppy_history(0)
    assert st[0]["sweeps"] == 1
    assert ph[0] == pq
    ctx.close()


def test_split_validation_and_removal():
    A, sptr, x = _integer_case(9, [200, 100])
    ctx = _identity_ctx(A, A.n)
    with pytest.raises(pk.SuppyError) as e:
        ctx.suppy_dvc_dose()
    assert e.value.status == pk.SUPPY_ESTATE
    bad = [((A.row_ptr, A.col, A.val, A.m, [0, 200, 299], [(0, 0, 0.1, 1.0)], 1.0), "end"),
           ((A.row_ptr, A.col, A.val, A.m, sptr, [(0, 0, 1.5, 1.0)], 1.0), "volume"),
           ((A.row_ptr, A.col, A.val, A.m, sptr, [(2, 0, 0.5, 1.0)], 1.0), "kind"),
           ((A.row_ptr, A.col, A.val, A.m, sptr, [(0, 2, 0.5, 1.0)], 1.0), "structure"),
           ((A.row_ptr, A.col, A.val, A.m, sptr, [(0, 0, 0.5, np.inf)], 1.0), "d_ref"),
           ((A.row_ptr, A.col, A.val, A.m, sptr, [(0, 0, 0.5, 1.0)], 2.0), "relax")]
    for args, what in bad:
        with pytest.raises(pk.SuppyError) as e:
            ctx.suppy_set_dvc(*args)
        assert e.value.status == pk.SUPPY_EINVAL, what
    col = A.col.copy()
    col[5] = A.n
    with pytest.raises(pk.SuppyError):
        ctx.suppy_set_dvc(A.row_ptr, col, A.val, A.m, sptr, [(0, 0, 0.5, 1.0)], 1.0)
    # set, then remove: sweeps are plain slab sweeps again and the device
    # memory the sets held is given back
    held = ctx.suppy_info_get()["device_bytes"]
    ctx.suppy_set_dvc(A.row_ptr, A.col, A.val, A.m, sptr, [(0, 0, 0.0, 0.5)], 1.0)
    assert ctx.suppy_info_get()["device_bytes"] > held
    ctx.suppy_set_dvc(None, None, None, 0, [0], [], 1.0)
    assert ctx.suppy_info_get()["device_bytes"] == held
    ctx.suppy_set_x(x)
    ctx.suppy_sweep(pk.suppy_params_default(), 1)
    assert np.array_equal(ctx.suppy_get_x(), x)
    ctx.close()
    # several right-hand sides: accepted, the same checks apply
    l = np.full((A.m, 2), -np.inf, F32)
    ctx2 = pk.Context(A.row_ptr, A.col, A.val, A.m, A.n, l, -l, np.zeros(1, F32),
                      np.ones(1, F32), nrhs=2)
    with pytest.raises(pk.SuppyError) as e:
        ctx2.suppy_set_dvc(A.row_ptr, A.col, A.val, A.m, sptr, [(0, 0, 1.5, 1.0)], 1.0)
    assert e.value.status == pk.SUPPY_EINVAL
    ctx2.suppy_set_dvc(A.row_ptr, A.col, A.val, A.m, sptr, [(0, 0, 0.5, 1.0)], 1.0)
    assert ctx2.suppy_dvc_dose().shape == (A.m, 2) and ctx2.suppy_dvc_proximity().shape == (2,)
    ctx2.close()


def test_batched_cq_step_equals_the_single_right_hand_side_steps():
    """Three right-hand sides sharing A_q and the sets, each with its own
    integer iterate: every column's doses, target-space proximity and CQ
    step equal (bitwise) those of a one-right-hand-side context on that
    column, and the step matches the oracle's."""
    A, sptr, _ = _integer_case(3, [3000, 2500, 40])
    rng = np.random.default_rng(33)
    X = rng.integers(0, 4, size=(A.n, 3)).astype(F32)
    d0 = A.to_scipy() @ X[:, 0].astype(np.float64)
    q = lambda s, f: float(np.quantile(d0[sptr[s]:sptr[s + 1]], f))
    dvcs = [(1, 0, 0.9, q(0, 0.5) + 0.5), (0, 0, 0.1, q(0, 0.6)), (0, 1, 0.05, q(1, 0.5)),
            (1, 2, 0.8, q(2, 0.9))]
    l = np.full((A.m, 3), -np.inf, F32)
    ctx = pk.Context(A.row_ptr, A.col, A.val, A.m, A.n, l, -l, np.full(1, -np.inf, F32),
                     np.full(1, np.inf, F32), nrhs=3)
    ctx.suppy_set_dvc(A.row_ptr, A.col, A.val, A.m, sptr, dvcs, 1.3)
    ctx.suppy_set_x(X)
    D = ctx.suppy_dvc_dose()
    Pq = ctx.suppy_dvc_proximity()
    ctx.suppy_sweep(pk.suppy_params_default(use_graphs=0), 1)
    XG = ctx.suppy_get_x()
    ctx.close()
    SS = _oracle_split(A, sptr, dvcs, 1.3)
    for b in range(3):
        d, d_ref, p_gpu, xg, _ = _step_compare(A, sptr, dvcs, X[:, b].copy(), 1.3)
        assert np.array_equal(D[:, b], d)
        assert Pq[b] == p_gpu
        assert np.array_equal(XG[:, b], xg)
        xo, _ = O.cq_step(SS, X[:, b].astype(np.float64))
        assert rel_l2(xg, xo) <= 2e-6


def test_batched_superiorized_split_run_matches_the_oracle():
    """Two plans of the horseshoe split problem in one context (OAR2 caps 30
    and 24 Gy), 12 iterations of [perturbation, CQ step, slab sweep, box]:
    each right-hand side against its own oracle run."""
    prob = synth.rt_split_problem(nx=24, ny=20, nz=12, ns=8, nzb=6)
    sp = prob.meta["split"]
    u2 = prob.u.copy()
    u2[prob.blocks == 1] = 24.0
    prob.l = np.stack([prob.l, prob.l], axis=1)
    prob.u = np.stack([prob.u, u2], axis=1)
    K = 12
    ctx = _split_ctx(prob, pk.SUPPY_CIMMINO, pk.SUPPY_OBJ_LINEAR)
    ctx.suppy_set_x(np.full((prob.A.n, 2), 1.0, F32))
    st = ctx.suppy_run(pk.suppy_params_default(gamma=1.0, alpha=0.7, n_red=1, max_sweeps=K,
                                               use_stopping=0))
    XG = ctx.suppy_get_x()
    SS = _oracle_split(sp["Aq"], sp["sptr"], sp["dvcs"], 1.0)
    obj = oracle_objective(prob, O.OBJ_LINEAR)
    P = O.Params(gamma=1.0, alpha=0.7, n_red=1, max_sweeps=K)
    S, l, u, lo, hi = O.from_problem(prob, O.CIMMINO)
    for b in range(2):
        ph, _ = ctx.suppy_history(b)
        r = O.run(S, O.CIMMINO, O.rhs(l, b), O.rhs(u, b), lo, hi, obj, P,
                  x0=np.full(prob.A.n, 1.0), split=SS)
        assert st[b]["sweeps"] == K
        assert rel_l2(XG[:, b], r.x) < 1e-4
        assert np.allclose(ph[:K], r.prox_hist, rtol=1e-4, atol=0)
    ctx.close()


def test_device_inputs_give_the_same_step():
    torch = pytest.importorskip("torch")
    A, sptr, x = _integer_case(13, [900, 700])
    d0 = A.to_scipy() @ x.astype(np.float64)
    dvcs = [(0, 0, 0.1, float(np.median(d0[:900]))), (1, 1, 0.9, float(np.median(d0[900:])))]
    out = []
    for dev in (False, True):
        ctx = _identity_ctx(A, A.n)
        arrs = [A.row_ptr, A.col, A.val]
        if dev:
            arrs = [torch.from_numpy(a).cuda() for a in arrs]
        ctx.suppy_set_dvc(*arrs, A.m, sptr, dvcs, 1.0)
        ctx.suppy_set_x(x)
        ctx.suppy_sweep(pk.suppy_params_default(), 1)
        out.append(ctx.suppy_get_x())
        ctx.close()
    assert np.array_equal(out[0], out[1])
