"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: one sweep from the same point <= 1e-5 relative L2 (FP32 A);
a full superiorized run <= 1e-3; proximity and objective values <= 1e-3
relative (much tighter in practice for single evaluations).
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


def _params(**kw):
    return pk.suppy_params_default(**kw)


def _oracle_sweep(prob, x, mode=O.CIMMINO, dtype="f32", lam=1.0, b=0):
    vals = rounded_values(prob.A.val, dtype)
    S, l, u, lo, hi = O.from_problem(prob, mode, values=vals)
    return O.sweep(S, mode, O.rhs(l, b), O.rhs(u, b), lam, lo, hi, np.asarray(x, np.float64))


# ------------------------------------------------------------ one sweep ----

STRATS = [pk.STRATEGY_ONE_PASS, pk.STRATEGY_TWO_PASS]


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("mode", [O.CIMMINO, O.BIP])
def test_one_sweep_tiny_ct(mode, strategy):
    prob = small_ct()
    if mode == O.BIP:
        prob.blocks = synth.angle_blocks(90, 91, 10)
    ctx = pk.from_problem(prob, mode=mode, strategy=strategy)
    x0 = random_x(prob.A.n, 1, seed=1)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(), 1)
    xg = ctx.suppy_get_x()
    xo, po = _oracle_sweep(prob, x0, mode)
    assert rel_l2(xg, xo) <= 1e-5
    ph, _ = ctx.suppy_history()
    assert len(ph) == 1 and rel(ph[0], po) <= 1e-5


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_one_sweep_low_precision_values(dtype, strategy):
    """BF16/FP16 storage: parity against the oracle run on the rounded values
    (the kernel gate); the error against the FP64 oracle on the original
    values is checked and stated in test_gpu_precision.py."""
    prob = small_ct()
    ctx = pk.from_problem(prob, dtype=DT[dtype], strategy=strategy)
    x0 = random_x(prob.A.n, 1, seed=2)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(), 1)
    xo, _ = _oracle_sweep(prob, x0, dtype=dtype)
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("n", [3001, 20011])
@pytest.mark.parametrize("mean_len,long_len", [(3, 0), (30, 0), (100, 0), (300, 0), (40, 2100),
                                               (250, 1500)])
def test_one_sweep_row_length_mix(mean_len, long_len, n, strategy):
    """Ragged rows covering every launch shape (4..32 lanes per row), empty
    rows, rows longer than the register-held elements, n not a multiple of 4;
    n = 3001 stages the one-pass scatter in shared memory, n = 20011 uses L2
    reductions."""
    prob = synth.random_problem(700, n, seed=mean_len + long_len, feasible=False,
                                mean_len=mean_len, empty_frac=0.05,
                                long_rows=7 if long_len else 0, long_len=long_len)
    ctx = pk.from_problem(prob, strategy=strategy)
    info = ctx.suppy_info_get()
    assert info["strategy"] == strategy
    if strategy == pk.STRATEGY_ONE_PASS:
        assert info["scatter"] == (2 if n * 4 <= 65536 else 1)
    x0 = random_x(n, 1, seed=3)
    for lam in (1.0, 1.7):
        ctx.suppy_set_x(x0)
        ctx.suppy_sweep(_params(lam=lam), 1)
        xo, po = _oracle_sweep(prob, x0, lam=lam)
        assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
        ph, _ = ctx.suppy_history()
        assert rel(ph[0], po) <= 1e-5


def test_vector_box_and_infinite_bounds():
    n = 500
    prob = synth.random_problem(300, n, seed=5, feasible=False, mean_len=25)
    rng = np.random.default_rng(5)
    prob.box_lo = rng.uniform(-0.2, 0.3, size=n).astype(np.float32)
    prob.box_hi = (prob.box_lo + rng.uniform(0.1, 1.0, size=n)).astype(np.float32)
    prob.l[::3] = -np.inf
    prob.u[1::3] = np.inf
    ctx = pk.from_problem(prob)
    x0 = random_x(n, 1, seed=6, lo=-1, hi=2)
    ctx.suppy_set_x(x0)
    x0c = np.clip(x0, prob.box_lo, prob.box_hi)
    np.testing.assert_array_equal(ctx.suppy_get_x(), x0c)
    ctx.suppy_sweep(_params(), 1)
    xo, _ = _oracle_sweep(prob, x0c)
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5


# ------------------------------------------------- proximity / objective ----

def test_proximity_matches_and_is_deterministic():
    prob = small_ct()
    ctx = pk.from_problem(prob)
    x0 = random_x(prob.A.n, 1, seed=7)
    ctx.suppy_set_x(x0)
    p1 = ctx.suppy_proximity()[0]
    p2 = ctx.suppy_proximity()[0]
    assert p1 == p2
    S, l, u, lo, hi = O.from_problem(prob)
    assert rel(p1, O.proximity(S, l, u, x0.astype(np.float64))) <= 1e-5


@pytest.mark.parametrize("kind", ["tv", "atv"])
def test_objective_matches(kind):
    prob = small_ct()
    obj = {"tv": pk.SUPPY_OBJ_TV_ISO, "atv": pk.SUPPY_OBJ_TV_ANISO}[kind]
    ctx = pk.from_problem(prob, obj=obj)
    x0 = random_x(prob.A.n, 1, seed=8)
    ctx.suppy_set_x(x0)
    f = ctx.suppy_objective()[0]
    ob = oracle_objective(prob, {"tv": O.OBJ_TV_ISO, "atv": O.OBJ_TV_ANISO}[kind])
    assert rel(f, ob.f(x0.astype(np.float64))) <= 1e-6


# ----------------------------------------------------------- perturbation ----

@pytest.mark.parametrize("kind", ["tv", "atv"])
def test_perturbation_phase_matches(kind):
    prob = small_ct()
    obj = {"tv": pk.SUPPY_OBJ_TV_ISO, "atv": pk.SUPPY_OBJ_TV_ANISO}[kind]
    okind = {"tv": O.OBJ_TV_ISO, "atv": O.OBJ_TV_ANISO}[kind]
    ctx = pk.from_problem(prob, obj=obj)
    x0 = random_x(prob.A.n, 1, seed=9)
    ctx.suppy_set_x(x0)
    P = dict(gamma=2.0, alpha=0.9, n_red=4, max_trials=50)
    acc = ctx.suppy_perturb(_params(**P))
    ob = oracle_objective(prob, okind)
    st = O.PertState()
    y, a, t = O.perturbation_phase(ob, x0.astype(np.float64), st, O.Params(**P))
    assert acc[0] == a
    blob = ctx.suppy_get_state()
    assert rel_l2(ctx.suppy_get_x(), y) <= 1e-5
    del blob


# --------------------------------------------------------------- full runs ----

def test_full_superiorized_run_tiny_ct():
    """Configuration of the tiny CT workload: 100 superiorized Cimmino sweeps,
    TV, beta = 0.5 * 0.99^l, lambda = 1."""
    prob = small_ct()
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO)
    P = dict(gamma=0.5, alpha=0.99, n_red=1, max_sweeps=100)
    st = ctx.suppy_run(_params(**P))
    S, l, u, lo, hi = O.from_problem(prob)
    r = O.run(S, O.CIMMINO, l, u, lo, hi, oracle_objective(prob, O.OBJ_TV_ISO), O.Params(**P))
    xg = ctx.suppy_get_x()
    assert st[0]["sweeps"] == 100
    assert rel_l2(xg, r.x) <= 1e-3
    ph, oh = ctx.suppy_history()
    assert rel(ph[-1], r.prox_hist[-1]) <= 1e-3
    assert rel(oh[-1], r.obj_hist[-1]) <= 1e-3
    assert st[0]["ell"] == r.ell


def test_full_bip_run_linear_objective_rt_small():
    """Radiotherapy shape (reduced): block-iterative sweeps over target / OAR
    blocks, mean body dose objective computed from the body rows."""
    prob = synth.rt_problem(nx=30, ny=20, nz=12, ns=9, nzb=7)
    ctx = pk.from_problem(prob, mode=pk.SUPPY_BIP, obj=pk.SUPPY_OBJ_LINEAR)
    P = dict(gamma=1.0, alpha=0.99, n_red=1, max_sweeps=40, lam=1.0)
    ctx.suppy_run(_params(**P))
    S, l, u, lo, hi = O.from_problem(prob, O.BIP)
    ob = oracle_objective(prob, O.OBJ_LINEAR)
    r = O.run(S, O.BIP, l, u, lo, hi, ob, O.Params(gamma=1.0, alpha=0.99, n_red=1,
                                                      max_sweeps=40))
    assert rel_l2(ctx.suppy_get_x(), r.x) <= 1e-3
    f = ctx.suppy_objective()[0]
    assert rel(f, ob.f(r.x)) <= 1e-3


def test_stopping_rule_stops_at_the_oracles_sweep():
    prob = synth.random_problem(400, 300, seed=11, feasible=True, mean_len=30)
    ctx = pk.from_problem(prob)
    P = dict(max_sweeps=300, prox_rel=1e-3, patience=3, use_stopping=1, check_every=7,
             obj_rel=0.0)
    st = ctx.suppy_run(_params(**P))
    S, l, u, lo, hi = O.from_problem(prob)
    r = O.run(S, O.CIMMINO, l, u, lo, hi, O.Objective(O.OBJ_NONE),
              O.Params(max_sweeps=300, prox_rel=1e-3, patience=3, use_stopping=True, obj_rel=0.0))
    assert st[0]["stopped"] == 1
    assert st[0]["sweeps"] == r.sweeps
    assert rel_l2(ctx.suppy_get_x(), r.x) <= 1e-4


def test_checkpoint_resume_is_exact_on_state():
    prob = small_ct()
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO)
    P = _params(gamma=0.5, alpha=0.99, max_sweeps=10)
    ctx.suppy_run(P)
    blob = ctx.suppy_get_state()
    x_mid = ctx.suppy_get_x().copy()
    ctx.suppy_run(P)
    x_a = ctx.suppy_get_x().copy()
    ctx.suppy_set_state(blob)
    np.testing.assert_array_equal(ctx.suppy_get_x(), x_mid)
    st = ctx.suppy_run(P)
    assert st[0]["sweeps"] == 20
    assert rel_l2(ctx.suppy_get_x(), x_a) <= 1e-5


# ------------------------------------------------------------------ batched ----

@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("nrhs", [3, 4, 16, 32])
def test_batched_sweep_matches_per_rhs_oracle(nrhs, strategy):
    prob = synth.ct_problem(32, 30, 45, nrhs=nrhs)
    ctx = pk.from_problem(prob, strategy=strategy)
    x0 = random_x(prob.A.n, nrhs, seed=12)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(), 2)
    xg = ctx.suppy_get_x()
    for b in range(nrhs):
        S, l, u, lo, hi = O.from_problem(prob)
        x = x0[:, b].astype(np.float64)
        for _ in range(2):
            x, _ = O.sweep(S, O.CIMMINO, O.rhs(prob.l, b), O.rhs(prob.u, b), 1.0, lo, hi, x)
        assert rel_l2(xg[:, b], x) <= 1e-5


def test_batched_run_equals_single_runs():
    """A right-hand side gives the same result alone and inside a batch."""
    prob = synth.ct_problem(32, 30, 45, nrhs=4)
    P = _params(gamma=0.5, alpha=0.99, max_sweeps=25)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO)
    ctx.suppy_run(P)
    xb = ctx.suppy_get_x()
    for b in range(4):
        p1 = synth.ct_problem(32, 30, 45, nrhs=4)
        p1.l, p1.u = p1.l[:, b].copy(), p1.u[:, b].copy()
        c1 = pk.from_problem(p1, obj=pk.SUPPY_OBJ_TV_ISO)
        c1.suppy_run(P)
        assert rel_l2(xb[:, b], c1.suppy_get_x()) <= 1e-3


# --------------------------------------------------------------- validation ----

def test_invalid_inputs_are_rejected():
    prob = synth.random_problem(50, 40, seed=13, mean_len=5)
    bad = synth.random_problem(50, 40, seed=13, mean_len=5)
    bad.A.col = bad.A.col.copy()
    bad.A.col[3] = 40
    with pytest.raises(pk.SuppyError) as e:
        pk.from_problem(bad)
    assert e.value.status == pk.SUPPY_EINVAL
    bad = synth.random_problem(50, 40, seed=13, mean_len=5)
    bad.l = bad.l.copy()
    bad.l[0] = bad.u[0] + 1
    with pytest.raises(pk.SuppyError):
        pk.from_problem(bad)
    bad = synth.random_problem(50, 40, seed=13, mean_len=5)
    bad.A.val = bad.A.val.copy()
    bad.A.val[0] = np.nan
    with pytest.raises(pk.SuppyError):
        pk.from_problem(bad)
    # a zero row whose slab excludes 0
    bad = synth.random_problem(50, 40, seed=13, mean_len=5, empty_frac=0.3)
    z = np.flatnonzero(np.diff(bad.A.row_ptr) == 0)[0]
    bad.l = bad.l.copy()
    bad.l[z], bad.u[z] = 1.0, 2.0
    with pytest.raises(pk.SuppyError):
        pk.from_problem(bad)
    ctx = pk.from_problem(prob)
    with pytest.raises(pk.SuppyError):
        ctx.suppy_perturb(_params())          # no objective: ESTATE


@pytest.mark.parametrize("strategy", STRATS)
def test_device_inputs_equal_host_inputs(strategy):
    prob = small_ct()
    c_h = pk.from_problem(prob, strategy=strategy)
    c_d = pk.from_problem(prob, device=True, strategy=strategy)
    x0 = random_x(prob.A.n, 1, seed=14)
    for c in (c_h, c_d):
        c.suppy_set_x(x0)
        c.suppy_sweep(_params(), 1)
    assert rel_l2(c_h.suppy_get_x(), c_d.suppy_get_x()) <= 1e-6


def test_two_pass_sweep_is_bitwise_reproducible():
    """The two-pass sweep has no atomics: repeated runs give identical bits."""
    prob = small_ct()
    xs = []
    for _ in range(2):
        ctx = pk.from_problem(prob, strategy=pk.STRATEGY_TWO_PASS, obj=pk.SUPPY_OBJ_TV_ISO)
        ctx.suppy_run(_params(max_sweeps=20))
        xs.append(ctx.suppy_get_x().copy())
    np.testing.assert_array_equal(xs[0], xs[1])


def test_autotuner_picks_a_measured_strategy():
    prob = synth.ct_problem(128, 90, 181)
    ctx = pk.from_problem(prob, tune=1)
    info = ctx.suppy_info_get()
    assert info["strategy"] in (1, 2)
    x0 = random_x(prob.A.n, 1, seed=21)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(), 1)
    xo, _ = _oracle_sweep(prob, x0)
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5


def test_kernel_timing_counts_launches():
    prob = small_ct()
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO)
    ctx.suppy_timing_enable(True)
    ctx.suppy_run(_params(max_sweeps=5))
    for kind, expect in ((0, 5), (1, 5), (2, 5)):
        ms, nl = ctx.suppy_kernel_time(kind)
        assert nl == expect and ms > 0


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("mode", [O.CIMMINO, O.BIP])
def test_graph_replay_equals_direct_launches(strategy, mode):
    """suppy_run through a captured CUDA graph gives the iterates of direct
    launches (bitwise for the atomic-free two-pass sweep)."""
    prob = small_ct()
    if mode == O.BIP:
        prob.blocks = synth.angle_blocks(90, 91, 10)
    xs = []
    for graphs in (0, 1):
        ctx = pk.from_problem(prob, mode=mode, strategy=strategy, obj=pk.SUPPY_OBJ_TV_ISO)
        st = ctx.suppy_run(_params(max_sweeps=15, use_graphs=graphs))
        assert st[0]["sweeps"] == 15
        xs.append(ctx.suppy_get_x().copy())
    if strategy == pk.STRATEGY_TWO_PASS:
        np.testing.assert_array_equal(xs[0], xs[1])
    else:
        # the one-pass scatter adds in a varying order: FP32 rounding
        # differences over 15 superiorized sweeps (1e-5 a sweep)
        assert rel_l2(xs[1], xs[0]) <= 1e-4


def test_perturbation_resident_kernel_on_large_image():
    """Images split across a 16-CTA cluster with halo rows read from the
    neighbouring CTA's shared memory (CT 256x256)."""
    prob = synth.ct_problem(256, 30, 363)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO)
    assert ctx.suppy_info_get()["perturb_cluster"] > 1
    x0 = random_x(prob.A.n, 1, seed=31)
    ctx.suppy_set_x(x0)
    P = dict(gamma=2.0, alpha=0.9, n_red=3, max_trials=40)
    acc = ctx.suppy_perturb(_params(**P))
    ob = oracle_objective(prob, O.OBJ_TV_ISO)
    y, a, _ = O.perturbation_phase(ob, x0.astype(np.float64), O.PertState(), O.Params(**P))
    assert acc[0] == a
    assert rel_l2(ctx.suppy_get_x(), y) <= 1e-5


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_tma_streaming_matches_oracle_and_plain_kernels(strategy, dtype):
    """The bulk-copy (TMA) fed passes give the oracle's sweep and, up to the
    FP32 summation order, the iterates of the register-fed kernels."""
    prob = synth.ct_problem(160, 60, 227)          # n = 25600: L2-reduction scatter
    x0 = random_x(prob.A.n, 1, seed=41)
    out = []
    for tma in (0, -1):
        ctx = pk.from_problem(prob, strategy=strategy, dtype=DT[dtype], tma=tma)
        assert ctx.suppy_info_get()["tma"] == (1 if tma == 0 else 0)
        ctx.suppy_set_x(x0)
        ctx.suppy_sweep(_params(), 3)
        out.append(ctx.suppy_get_x().copy())
        ph, _ = ctx.suppy_history()
    vals = rounded_values(prob.A.val, dtype)
    S, l, u, lo, hi = O.from_problem(prob, values=vals)
    x = x0.astype(np.float64)
    for _ in range(3):
        x, p_last = O.sweep(S, O.CIMMINO, l, u, 1.0, lo, hi, x)
    assert rel_l2(out[0], x) <= 1e-5
    assert rel(ph[-1], p_last) <= 1e-5
    assert rel_l2(out[0], out[1]) <= 1e-5


def test_tma_block_iterative_and_long_rows():
    """Block-iterative sweep through the streaming passes (one launch pair per
    block), and rows longer than the ring window falling back to the
    register-fed kernels."""
    prob = synth.ct_problem(160, 60, 227)
    prob.blocks = synth.angle_blocks(60, 227, 6)
    for strategy in STRATS:
        ctx = pk.from_problem(prob, mode=pk.SUPPY_BIP, strategy=strategy)
        assert ctx.suppy_info_get()["tma"] == 1
        x0 = random_x(prob.A.n, 1, seed=42)
        ctx.suppy_set_x(x0)
        ctx.suppy_sweep(_params(), 1)
        xo, _ = _oracle_sweep(prob, x0, O.BIP)
        assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
    longp = synth.random_problem(300, 30000, seed=43, mean_len=60, long_rows=3, long_len=25000)
    ctx = pk.from_problem(longp, strategy=pk.STRATEGY_TWO_PASS)
    assert ctx.suppy_info_get()["tma"] == 0
    x0 = random_x(30000, 1, seed=44)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(), 1)
    xo, _ = _oracle_sweep(longp, x0)
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5


@pytest.mark.parametrize("stream_map", [1, 2])
@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("shape", [(256, 8, 4), (512, 32, 8), (1024, 4, 16), (2048, 12, 32),
                                   (4096, 2, 32)])
def test_tma_stream_shapes_match_oracle(shape, strategy, stream_map):
    """Every ring shape the tuner may pick (tile length, stages, lanes per
    item, lane map) gives the oracle's sweep on ragged items: row and column
    lengths that are not multiples of four, empty rows, several tiles per CTA
    (items wrap around the ring's end)."""
    prob = synth.random_problem(4000, 30011, seed=45, feasible=False, mean_len=37,
                                empty_frac=0.05, long_rows=5, long_len=190)
    ctx = pk.from_problem(prob, strategy=strategy, stream_shape=shape, stream_map=stream_map)
    info = ctx.suppy_info_get()
    assert info["tma"] == 1 and info["map"] == stream_map
    assert (info["tile"], info["stages"], info["lanes_per_row"]) == shape
    if strategy == pk.STRATEGY_TWO_PASS:
        assert (info["col_tile"], info["col_stages"], info["col_lanes"]) == shape
        assert info["col_map"] == stream_map
    x0 = random_x(prob.A.n, 1, seed=46)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(lam=1.3), 2)
    vals = rounded_values(prob.A.val, "f32")
    S, l, u, lo, hi = O.from_problem(prob, values=vals)
    x = x0.astype(np.float64)
    for _ in range(2):
        x, p_last = O.sweep(S, O.CIMMINO, l, u, 1.3, lo, hi, x)
    assert rel_l2(ctx.suppy_get_x(), x) <= 1e-5
    ph, _ = ctx.suppy_history()
    assert rel(ph[-1], p_last) <= 1e-5


def test_tuned_stream_shapes_match_oracle():
    """tune = 1 times the ring and group shapes of both streaming passes on
    the matrix and keeps a valid one."""
    prob = synth.ct_problem(128, 90, 181)
    ctx = pk.from_problem(prob, tune=1, strategy=pk.STRATEGY_TWO_PASS)
    info = ctx.suppy_info_get()
    assert info["tma"] == 1
    assert info["tile"] in (1024, 2048, 4096) and info["col_tile"] in (1024, 2048, 4096)
    assert 3 <= info["stages"] <= 32 and 3 <= info["col_stages"] <= 32
    assert info["lanes_per_row"] in (4, 8, 16, 32) and info["col_lanes"] in (4, 8, 16, 32)
    assert info["map"] in (1, 2) and info["col_map"] in (1, 2)
    x0 = random_x(prob.A.n, 1, seed=47)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(), 1)
    xo, _ = _oracle_sweep(prob, x0)
    assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5


def test_tuned_configuration_rebuilt_without_timing():
    """A tuned configuration (strategy, ring shape, lane maps per pass, as
    suppy_info reports it) passed back as fixed options gives the same launch
    configuration and the same sweep."""
    prob = synth.ct_problem(128, 90, 181)
    x0 = random_x(prob.A.n, 1, seed=48)
    tuned = pk.from_problem(prob, tune=1, strategy=pk.STRATEGY_TWO_PASS)
    ti = tuned.suppy_info_get()
    for col_map in (1, 2):
        ctx = pk.from_problem(prob, strategy=pk.STRATEGY_TWO_PASS,
                              stream_shape=(ti["tile"], ti["stages"], ti["lanes_per_row"]),
                              stream_map=ti["map"], stream_col_map=col_map)
        info = ctx.suppy_info_get()
        assert (info["tile"], info["stages"], info["lanes_per_row"], info["map"]) == \
            (ti["tile"], ti["stages"], ti["lanes_per_row"], ti["map"])
        assert info["col_map"] == col_map
        ctx.suppy_set_x(x0)
        ctx.suppy_sweep(_params(), 1)
        xo, _ = _oracle_sweep(prob, x0)
        assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
        ctx.close()
    with pytest.raises(pk.SuppyError):
        pk.from_problem(prob, stream_col_map=3)
    tuned.close()


@pytest.mark.parametrize("shape", [(300, 0, 0), (8192, 0, 0), (0, 1, 0), (0, 40, 0), (0, 0, 5)])
def test_invalid_stream_shapes_are_rejected(shape):
    prob = small_ct()
    with pytest.raises(pk.SuppyError):
        pk.from_problem(prob, stream_shape=shape)


@pytest.mark.parametrize("stream_map", [-1, 3])
def test_invalid_stream_maps_are_rejected(stream_map):
    with pytest.raises(pk.SuppyError) as e:
        pk.from_problem(small_ct(), stream_map=stream_map)
    assert e.value.status == pk.SUPPY_EINVAL


@pytest.mark.parametrize("tma", [0, -1])
@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("mode", [O.CIMMINO, O.BIP])
def test_interleaved_row_order_matches_oracle(mode, strategy, tma):
    """Blocks of at least 16384 rows are stored in a chunk-interleaved device
    order; sweeps, the monitored proximity and set_bounds still follow the
    source row order's problem exactly (up to FP32 summation order)."""
    prob = synth.random_problem(40000, 20011, seed=48, feasible=False, mean_len=18,
                                empty_frac=0.03, long_rows=4, long_len=300)
    if mode == O.BIP:
        prob.blocks = (np.arange(prob.A.m) * 2 // prob.A.m).astype(np.int32)
    ctx = pk.from_problem(prob, mode=mode, strategy=strategy, tma=tma)
    x0 = random_x(prob.A.n, 1, seed=49)
    for rnd in range(2):
        if rnd == 1:
            # new bounds through set_bounds (device-order permutation of l, u)
            l2, u2 = prob.l * np.float32(0.9), prob.u * np.float32(1.1)
            prob.l, prob.u = np.minimum(l2, u2), np.maximum(l2, u2)
            ctx.suppy_set_bounds(prob.l, prob.u)
        ctx.suppy_set_x(x0)
        ctx.suppy_sweep(_params(lam=1.5), 1)
        xo, po = _oracle_sweep(prob, x0, mode, lam=1.5)
        assert rel_l2(ctx.suppy_get_x(), xo) <= 1e-5
        ph, _ = ctx.suppy_history()
        assert rel(ph[0], po) <= 1e-5
        S, l, u, _, _ = O.from_problem(prob, mode)
        assert rel(ctx.suppy_proximity()[0], O.proximity(S, l, u, xo)) <= 1e-3


# ------------------------------------------ whole-GPU perturbation phase ----

PERT_CASES = [
    # (gamma, alpha, n_red, max_trials): first trial accepted; later trials only
    # (the first eight rejected: further trial passes); several reduction
    # steps (grid barrier before each next subgradient); fewer trials than one
    # pass evaluates
    (0.05, 0.99, 1, 100),
    (40.0, 0.7, 1, 100),
    (2.0, 0.9, 3, 50),
    (40.0, 0.7, 1, 3),
]


@pytest.mark.parametrize("case", PERT_CASES)
@pytest.mark.parametrize("kind", ["tv", "atv"])
def test_whole_gpu_perturbation_matches_oracle_and_cluster_path(kind, case):
    """The whole-GPU phase (one cooperative launch; two trials in a step's
    first pass, eight in later ones, first acceptance kept; grid barriers
    between passes) gives the oracle's
    phase and the cluster kernel's: the same accepted steps, trial count and
    exponent, and the same point -- also when a step needs more than one
    pass of trials (max_trials 100) or the trials run out (max_trials 3)."""
    gamma, alpha, n_red, max_trials = case
    prob = synth.ct_problem(128, 60, 181)
    obj = {"tv": pk.SUPPY_OBJ_TV_ISO, "atv": pk.SUPPY_OBJ_TV_ANISO}[kind]
    okind = {"tv": O.OBJ_TV_ISO, "atv": O.OBJ_TV_ANISO}[kind]
    x0 = random_x(prob.A.n, 1, seed=51)
    P = dict(gamma=gamma, alpha=alpha, n_red=n_red, max_trials=max_trials)
    ob = oracle_objective(prob, okind)
    ost = O.PertState()
    y, a, t = O.perturbation_phase(ob, x0.astype(np.float64), ost, O.Params(**P))
    xs = []
    for path in (2, 1):
        ctx = pk.from_problem(prob, obj=obj, perturb_path=path)
        ctx.suppy_set_x(x0)
        acc = ctx.suppy_perturb(_params(**P))
        st = ctx.suppy_run(_params(max_sweeps=0))[0]
        assert acc[0] == a
        assert st["trials"] == t and st["ell"] == ost.ell
        xs.append(ctx.suppy_get_x().copy())
        assert rel_l2(xs[-1], y) <= 1e-5
    assert rel_l2(xs[0], xs[1]) <= 1e-6


def test_whole_gpu_perturbation_batched_and_linear():
    """Several right-hand sides in one whole-GPU launch (their phases one
    after the other, each its own exponent and decisions; the padding
    right-hand sides skipped), and the linear mean-dose objective."""
    prob = synth.ct_problem(96, 40, 137, nrhs=5)
    x0 = random_x(prob.A.n, 5, seed=52)
    P = dict(gamma=3.0, alpha=0.8, n_red=2, max_trials=40)
    ob = oracle_objective(prob, O.OBJ_TV_ISO)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, perturb_path=2)
    ctx.suppy_set_x(x0)
    acc = ctx.suppy_perturb(_params(**P))
    xg = ctx.suppy_get_x()
    for b in range(5):
        y, a, _ = O.perturbation_phase(ob, x0[:, b].astype(np.float64), O.PertState(),
                                       O.Params(**P))
        assert acc[b] == a
        assert rel_l2(xg[:, b], y) <= 1e-5
    rt = synth.rt_problem(nx=30, ny=20, nz=12, ns=9, nzb=7)
    obl = oracle_objective(rt, O.OBJ_LINEAR)
    xr = random_x(rt.A.n, 1, seed=53)
    ctx = pk.from_problem(rt, mode=pk.SUPPY_BIP, obj=pk.SUPPY_OBJ_LINEAR, perturb_path=2)
    ctx.suppy_set_x(xr)
    P = dict(gamma=1.0, alpha=0.99, n_red=2, max_trials=10)
    acc = ctx.suppy_perturb(_params(**P))
    y, a, _ = O.perturbation_phase(obl, xr.astype(np.float64), O.PertState(), O.Params(**P))
    assert acc[0] == a
    assert rel_l2(ctx.suppy_get_x(), y) <= 1e-5


# ------------------------------------------------------------------ DROP ----

@pytest.mark.parametrize("tma", [0, -1])
@pytest.mark.parametrize("strategy", STRATS)
def test_drop_sweep_matches_oracle(strategy, tma):
    """DROP (unit row weights, column scaling 1/s_j) through every sweep
    kernel family: one and two passes, streamed and register-fed; ragged
    rows, empty rows and empty columns."""
    prob = synth.random_problem(3000, 20011, seed=55, feasible=False, mean_len=24,
                                empty_frac=0.04, long_rows=3, long_len=400)
    ctx = pk.from_problem(prob, mode=pk.SUPPY_DROP, strategy=strategy, tma=tma)
    x0 = random_x(prob.A.n, 1, seed=56)
    ctx.suppy_set_x(x0)
    ctx.suppy_sweep(_params(lam=1.2), 2)
    S, l, u, lo, hi = O.from_problem(prob, O.DROP)
    x = x0.astype(np.float64)
    for _ in range(2):
        x, p_last = O.sweep(S, O.DROP, l, u, 1.2, lo, hi, x)
    assert rel_l2(ctx.suppy_get_x(), x) <= 1e-5
    ph, _ = ctx.suppy_history()
    assert rel(ph[-1], p_last) <= 1e-5


def test_drop_batched_and_superiorized_seismic_run():
    """The paper's seismic setting: DROP feasibility-seeking with anisotropic
    TV perturbation, several noise realisations at once, against the oracle
    per right-hand side."""
    prob = synth.seismic_problem(32, 64, 16, 64, nrhs=3)
    ctx = pk.from_problem(prob, mode=pk.SUPPY_DROP, obj=pk.SUPPY_OBJ_TV_ANISO)
    P = dict(gamma=0.5, alpha=0.99, n_red=1, max_sweeps=30)
    st = ctx.suppy_run(_params(**P))
    xg = ctx.suppy_get_x()
    S, l, u, lo, hi = O.from_problem(prob, O.DROP)
    ob = oracle_objective(prob, O.OBJ_TV_ANISO)
    for b in range(3):
        r = O.run(S, O.DROP, O.rhs(l, b), O.rhs(u, b), lo, hi, ob, O.Params(**P))
        assert st[b]["ell"] == r.ell
        assert rel_l2(xg[:, b], r.x) <= 1e-3


# ------------------------------------------------------- L1 / L2 perturbations ----

@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("kind", ["l1", "l2"])
def test_norm_perturbations_match_oracle(kind, path):
    """The L1 / L2 perturbations of the seismic study through the cluster
    kernel and the whole-GPU step: one phase (several reduction steps), the
    objective value, and a short superiorized DROP run."""
    prob = synth.seismic_problem(32, 64, 16, 64, nrhs=1)
    obj = {"l1": pk.SUPPY_OBJ_L1, "l2": pk.SUPPY_OBJ_L2}[kind]
    okind = {"l1": O.OBJ_L1, "l2": O.OBJ_L2}[kind]
    ob = oracle_objective(prob, okind)
    x0 = random_x(prob.A.n, 1, seed=57, lo=-0.2, hi=0.5)
    ctx = pk.from_problem(prob, obj=obj, mode=pk.SUPPY_DROP, perturb_path=path)
    ctx.suppy_set_x(x0)
    xb = np.clip(x0.astype(np.float64), prob.box_lo[0], prob.box_hi[0])
    assert rel(ctx.suppy_objective()[0], ob.f(xb)) <= 1e-6
    P = dict(gamma=0.2, alpha=0.9, n_red=3, max_trials=30)
    acc = ctx.suppy_perturb(_params(**P))
    y, a, _ = O.perturbation_phase(ob, xb, O.PertState(), O.Params(**P))
    assert acc[0] == a
    assert rel_l2(ctx.suppy_get_x(), y) <= 1e-5
    ctx = pk.from_problem(prob, obj=obj, mode=pk.SUPPY_DROP, perturb_path=path)
    R = dict(gamma=0.5, alpha=0.99, n_red=1, max_sweeps=25)
    ctx.suppy_run(_params(**R))
    S, l, u, lo, hi = O.from_problem(prob, O.DROP)
    r = O.run(S, O.DROP, l, u, lo, hi, ob, O.Params(**R))
    assert rel_l2(ctx.suppy_get_x(), r.x) <= 1e-3


# ------------------------------------------------ variance stopping rule ----

@pytest.mark.parametrize("graphs", [0, 1])
def test_variance_stopping_rule_stops_with_the_oracle(graphs):
    """The variance rule of the CT study (threshold 0.01) on the tiny CT
    workload with TV: the run stops at the oracle's iteration (within one,
    for FP32 norms near the threshold) for every right-hand side."""
    prob = small_ct(nrhs=2)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO)
    P = dict(gamma=0.5, alpha=0.99, n_red=1, max_sweeps=400)
    st = ctx.suppy_run(_params(variance_tol=1e-2, check_every=7, use_graphs=graphs, **P))
    S, l, u, lo, hi = O.from_problem(prob)
    ob = oracle_objective(prob, O.OBJ_TV_ISO)
    xg = ctx.suppy_get_x()
    for b in range(2):
        r = O.run(S, O.CIMMINO, O.rhs(l, b), O.rhs(u, b), lo, hi, ob,
                  O.Params(variance_tol=1e-2, **P))
        assert r.sweeps < 400
        assert st[b]["stopped"] == 1
        assert abs(st[b]["sweeps"] - r.sweeps) <= 1
        if st[b]["sweeps"] == r.sweeps:
            assert rel_l2(xg[:, b], r.x) <= 1e-3


@pytest.mark.parametrize("mode,omode", [(pk.SUPPY_CIMMINO, O.CIMMINO), (pk.SUPPY_DROP, O.DROP),
                                        (pk.SUPPY_EL, O.EL), (pk.SUPPY_EMR, O.EMR)])
@pytest.mark.parametrize("strategy,tma", [(pk.STRATEGY_ONE_PASS, -1), (pk.STRATEGY_TWO_PASS, -1),
                                          (pk.STRATEGY_TWO_PASS, 0)])
def test_box_step_covers_empty_columns_after_perturbation(mode, omode, strategy, tma):
    """Columns without entries still take the box step: the L1 perturbation
    lowers every positive entry by beta/sqrt(n), so entries starting on the
    lower bound leave the box, and only the sweep's box brings those of empty
    columns back (as in the oracle) -- in the one-pass box kernel, the
    register-fed and streamed column passes, and the extrapolated update."""
    prob = synth.random_problem(400, 3000, seed=61, mean_len=6, box=(0.2, 0.8))
    A = prob.A
    empty = np.setdiff1d(np.arange(A.n), A.col)
    assert len(empty) > 1000
    rng = np.random.default_rng(62)
    x0 = rng.uniform(0.2, 0.8, A.n).astype(np.float32)
    x0[empty[::2]] = 0.2
    K = 3
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_L1, mode=mode, strategy=strategy, tma=tma)
    if mode not in (pk.SUPPY_EL, pk.SUPPY_EMR):   # EL / EMR always take two passes
        assert ctx.suppy_info_get()["strategy"] == strategy
    ctx.suppy_set_x(x0)
    ctx.suppy_run(_params(max_sweeps=K, use_stopping=0))
    xg = ctx.suppy_get_x()
    ctx.close()
    S, l, u, lo, hi = O.from_problem(prob, omode)
    r = O.run(S, omode, l, u, lo, hi, O.Objective(O.OBJ_L1), O.Params(max_sweeps=K),
              x0=x0.astype(np.float64))
    assert sum(r.accepted) == K
    assert xg.min() >= 0.2 and xg.max() <= 0.8
    assert np.array_equal(xg[empty[::2]], np.full(len(empty[::2]), 0.2, np.float32))
    assert rel_l2(xg, r.x) <= 1e-5


def test_enqueued_bounds_updates_and_their_rejection():
    """suppy_update_bounds_async gives the iterations suppy_update_bounds
    gives; a rejected set (NaN) keeps the old bounds and is reported once, by
    the next synchronizing call, also when a valid set follows it."""
    prob = small_ct()
    x0 = random_x(prob.A.n, 1, seed=93)
    l2 = (prob.l - 0.01 * np.abs(prob.l)).astype(np.float32)   # wider slabs
    u2 = (prob.u + 0.01 * np.abs(prob.u)).astype(np.float32)
    out = []
    for use_async in (False, True):
        ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, strategy=pk.STRATEGY_TWO_PASS)
        ctx.suppy_set_x(x0)
        for _ in range(3):
            if use_async:
                ctx.suppy_update_bounds_async(l2, u2)
            else:
                ctx.suppy_update_bounds(l2, u2)
            ctx.suppy_run(_params(max_sweeps=1), want_stats=False)
        out.append(ctx.suppy_get_x())
        ctx.close()
    assert np.array_equal(out[0], out[1])
    bad = l2.copy()
    bad[5] = np.nan
    ref = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, strategy=pk.STRATEGY_TWO_PASS)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, strategy=pk.STRATEGY_TWO_PASS)
    for c in (ref, ctx):
        c.suppy_set_x(x0)
    ctx.suppy_update_bounds_async(bad, u2)          # rejected: the create-time bounds stay
    ctx.suppy_update_bounds_async(prob.l, prob.u)   # valid, the same bounds
    ctx.suppy_run(_params(max_sweeps=2), want_stats=False)
    ref.suppy_run(_params(max_sweeps=2), want_stats=False)
    with pytest.raises(pk.SuppyError) as e:
        ctx.suppy_get_x()
    assert e.value.status == pk.SUPPY_EINVAL
    assert np.array_equal(ctx.suppy_get_x(), ref.suppy_get_x())   # reported once
    ctx.close()
    ref.close()


def test_run_without_statistics_enqueues_the_same_iterations():
    """suppy_run with out = NULL (and no stopping rule) returns after
    enqueuing; the next synchronizing call sees exactly the iterations a
    synchronizing run leaves (two-pass sweep: the iterate bitwise)."""
    prob = small_ct()
    x0 = random_x(prob.A.n, 1, seed=91)
    xs, hs = [], []
    for want in (True, False):
        ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, strategy=pk.STRATEGY_TWO_PASS)
        ctx.suppy_set_x(x0)
        for _ in range(3):
            r = ctx.suppy_run(_params(max_sweeps=2), want_stats=want)
            assert (r is None) == (not want)
        xs.append(ctx.suppy_get_x())
        hs.append(ctx.suppy_history(0)[0])
        ctx.close()
    assert np.array_equal(xs[0], xs[1])
    # the streamed row pass hands items out dynamically: each thread's
    # compensated FP32 proximity sum takes its terms in a varying order (x is
    # bitwise equal, the history to the FP32 compensation error)
    assert len(hs[1]) == 6 and np.allclose(hs[0], hs[1], rtol=1e-6, atol=0)


def test_update_bounds_keeps_the_iteration_state():
    """suppy_update_bounds swaps the slabs and Algorithm 1 continues (same
    exponent l, counters and history) -- the oracle's loop with the bounds
    replaced between iterations; suppy_set_bounds resets the state."""
    prob = small_ct(nrhs=2)
    l0, u0 = O.rhs(prob.l, 0), O.rhs(prob.u, 0)
    l1, u1 = O.rhs(prob.l, 1), O.rhs(prob.u, 1)
    single = synth.ct_problem()
    ctx = pk.from_problem(single, obj=pk.SUPPY_OBJ_TV_ISO)
    ctx.suppy_set_bounds(l0.astype(np.float32), u0.astype(np.float32))
    P = dict(gamma=0.5, alpha=0.99, n_red=1)
    ctx.suppy_run(_params(max_sweeps=12, **P))
    ctx.suppy_update_bounds(l1.astype(np.float32), u1.astype(np.float32))
    st = ctx.suppy_run(_params(max_sweeps=8, **P))[0]
    assert st["sweeps"] == 20
    S, _, _, lo, hi = O.from_problem(single)
    ob = oracle_objective(single, O.OBJ_TV_ISO)
    op = O.Params(**P)
    ps = O.PertState()
    x = np.zeros(single.A.n)
    for k in range(20):
        l, u = (l0, u0) if k < 12 else (l1, u1)
        x, _, _ = O.perturbation_phase(ob, x, ps, op)
        x, p = O.sweep(S, O.CIMMINO, l, u, 1.0, lo, hi, x)
    assert st["ell"] == ps.ell
    assert rel_l2(ctx.suppy_get_x(), x) <= 1e-3
    ph, _ = ctx.suppy_history()
    assert len(ph) == 20 and rel(ph[-1], p) <= 1e-3
    ctx.suppy_set_bounds(l1.astype(np.float32), u1.astype(np.float32))
    st = ctx.suppy_run(_params(max_sweeps=0, **P))[0]
    assert st["sweeps"] == 0 and st["ell"] == 0


# ------------------------------------------------------------- EL / EMR ----

@pytest.mark.parametrize("tma", [0, -1])
@pytest.mark.parametrize("mode", [pk.SUPPY_EL, pk.SUPPY_EMR])
def test_extrapolated_sweeps_match_oracle(mode, tma):
    """EL and EMR (the column pass accumulates, the step size comes from
    grid-wide FP64 reductions, EMR adds a pass over q = A delta), streamed
    and register-fed, with lambda 1 and 0.8, over three sweeps."""
    prob = synth.random_problem(3000, 20011, seed=58, feasible=False, mean_len=24,
                                empty_frac=0.04, long_rows=3, long_len=400)
    om = {pk.SUPPY_EL: O.EL, pk.SUPPY_EMR: O.EMR}[mode]
    for lam in (1.0, 0.8):
        ctx = pk.from_problem(prob, mode=mode, tma=tma)
        assert ctx.suppy_info_get()["strategy"] == 2
        x0 = random_x(prob.A.n, 1, seed=59)
        ctx.suppy_set_x(x0)
        ctx.suppy_sweep(_params(lam=lam), 3)
        S, l, u, lo, hi = O.from_problem(prob)
        x = x0.astype(np.float64)
        for _ in range(3):
            x, p_last = O.sweep(S, om, l, u, lam, lo, hi, x)
        assert rel_l2(ctx.suppy_get_x(), x) <= 1e-5
        ph, _ = ctx.suppy_history()
        assert rel(ph[-1], p_last) <= 1e-5


@pytest.mark.parametrize("mode", [pk.SUPPY_EL, pk.SUPPY_EMR])
def test_superiorized_extrapolated_runs_batched(mode):
    """The CT study's setting: EMR / EL feasibility-seeking with TV
    perturbations, several sinograms at once, against the oracle per
    right-hand side.  EL's extrapolated steps (t up to ~m on this
    inconsistent system) amplify the FP32 / FP64 difference -- the paper
    reports EL fluctuating on inconsistent CT data -- so its run is shorter."""
    prob = small_ct(nrhs=3)
    om = {pk.SUPPY_EL: O.EL, pk.SUPPY_EMR: O.EMR}[mode]
    ctx = pk.from_problem(prob, mode=mode, obj=pk.SUPPY_OBJ_TV_ISO)
    P = dict(gamma=0.5, alpha=0.99, n_red=1, max_sweeps=12 if mode == pk.SUPPY_EL else 30)
    st = ctx.suppy_run(_params(**P))
    xg = ctx.suppy_get_x()
    S, l, u, lo, hi = O.from_problem(prob)
    ob = oracle_objective(prob, O.OBJ_TV_ISO)
    for b in range(3):
        r = O.run(S, om, O.rhs(l, b), O.rhs(u, b), lo, hi, ob, O.Params(**P))
        assert st[b]["ell"] == r.ell
        assert rel_l2(xg[:, b], r.x) <= 1e-3
