"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks a property
that a plausible mistake (dropped term, wrong sign, wrong weight, transposed
index) would break -- closed forms, brute-force minimisers, library
optimisers, invariants of the method, or values the paper prints.
"""
import json
import os

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _dist_to_slab_bruteforce_2d(a, l, u, x, half=3.0, n=1201):
    """Nearest point of the slab to x by dense grid search in 2-D."""
    g = np.linspace(-half, half, n)
    Y = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2) + x
    r = Y @ a
    ins = (r >= l) & (r <= u)
    d = np.linalg.norm(Y[ins] - x, axis=1)
    k = np.argmin(d)
    return Y[ins][k], d[k]


# ------------------------------------------------------ single projection --

@pytest.mark.parametrize("seed", range(6))
def test_hyperslab_projection_is_nearest_point(seed):
    """Eq. (2), two-sided (Q1): P x lies in the slab, P x - x is parallel to a,
    P is idempotent, and P x is the slab's nearest point (SLSQP)."""
    rng = np.random.default_rng(seed)
    n = 5
    a = rng.standard_normal(n)
    l, u = sorted(rng.uniform(-2, 2, size=2))
    for x in [rng.standard_normal(n) * 3 for _ in range(4)]:
        p = O.hyperslab_project(a, l, u, x)
        r = a @ p
        assert l - 1e-12 <= r <= u + 1e-12
        d = p - x
        # parallel to a: the component orthogonal to a vanishes
        perp = d - (d @ a) / (a @ a) * a
        assert np.linalg.norm(perp) <= 1e-12 * (1 + np.linalg.norm(d))
        np.testing.assert_allclose(O.hyperslab_project(a, l, u, p), p, atol=1e-12)
        cons = [{"type": "ineq", "fun": lambda y: a @ y - l},
                {"type": "ineq", "fun": lambda y: u - a @ y}]
        res = so.minimize(lambda y: np.sum((y - x) ** 2), x, constraints=cons,
                          method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
        np.testing.assert_allclose(p, res.x, atol=1e-6)


def test_hyperslab_projection_bruteforce_2d():
    """In 2-D the distance to the slab found by dense grid search matches."""
    rng = np.random.default_rng(11)
    for _ in range(5):
        a = rng.standard_normal(2)
        l, u = sorted(rng.uniform(-1, 1, size=2))
        x = rng.standard_normal(2) * 2
        p = O.hyperslab_project(a, l, u, x)
        _, dbf = _dist_to_slab_bruteforce_2d(a, l, u, x)
        assert abs(np.linalg.norm(p - x) - dbf) < 2 * 6.0 / 1200


def test_halfspace_case_matches_eq2():
    """With l = -inf the slab projection is the halfspace projection of Eq. (2):
    moved by (<a,x> - b)/||a||^2 along -a when <a,x> > b, unchanged otherwise."""
    rng = np.random.default_rng(3)
    a = rng.standard_normal(4)
    b = 0.3
    x_out = rng.standard_normal(4)
    x_out += (b + 1.0 - a @ x_out) / (a @ a) * a          # <a,x> = b + 1 > b
    x_in = x_out - 2.0 / (a @ a) * a                       # <a,x> = b - 1 < b
    p = O.hyperslab_project(a, -np.inf, b, x_out)
    np.testing.assert_allclose(p, x_out - 1.0 / (a @ a) * a, atol=1e-13)
    np.testing.assert_array_equal(O.hyperslab_project(a, -np.inf, b, x_in), x_in)


def test_relaxation_endpoints():
    """Eq. (3): lambda = 0 keeps x, lambda = 1 is the projection, lambda = 2 the
    reflection through the slab face."""
    a = np.array([1.0, 2.0])
    x = np.array([3.0, 3.0])
    p = O.hyperslab_project(a, -1.0, 1.0, x)
    np.testing.assert_allclose(O.relaxed(x, p, 0.0), x)
    np.testing.assert_allclose(O.relaxed(x, p, 1.0), p)
    refl = O.relaxed(x, p, 2.0)
    assert abs((a @ refl) - (2 * 1.0 - a @ x)) < 1e-12


# -------------------------------------------------------------- proximity --

def test_single_constraint_proximity_is_half_squared_distance():
    """Eq. (WeightedProximity) with one constraint (w = 1) is 1/2 dist^2; the
    distance comes from a brute-force grid search, so a dropped 1/2 or a
    missing ||a||^2 fails here."""
    a = np.array([0.6, -1.7])
    l, u = -0.4, 0.5
    x = np.array([1.3, -0.9])
    A = sp.csr_matrix(a[None, :])
    S = O.setup(A, np.array([l]), np.array([u]))
    _, dbf = _dist_to_slab_bruteforce_2d(a, l, u, x, n=2401)
    assert abs(O.proximity(S, np.array([l]), np.array([u]), x) - 0.5 * dbf ** 2) < 5e-3 * dbf


def test_proximity_zero_at_feasible_point():
    rng = np.random.default_rng(5)
    A = sp.random(30, 12, density=0.4, random_state=5, format="csr")
    x = rng.uniform(size=12)
    b = A @ x
    S = O.setup(A, b - 0.1, b + 0.1)
    assert O.proximity(S, b - 0.1, b + 0.1, x) == 0.0


def test_zero_rows_dropped_or_rejected():
    """Q11: an empty row whose slab contains 0 is dropped (weights use m'),
    one whose slab excludes 0 is rejected."""
    A = sp.csr_matrix(np.array([[1.0, 0.0], [0.0, 0.0], [0.0, 2.0]]))
    S = O.setup(A, np.array([0.0, -1.0, 0.0]), np.array([1.0, 1.0, 1.0]))
    np.testing.assert_allclose(S.w_sweep, [0.5, 0.0, 0.5])
    with pytest.raises(ValueError):
        O.setup(A, np.array([0.0, 0.5, 0.0]), np.array([1.0, 1.0, 1.0]))


# ----------------------------------------------------------------- sweeps --

def test_single_row_sweep_lands_on_slab():
    """m = 1, lambda = 1, w = 1: one simultaneous step is the exact projection,
    so the point lands on the violated face."""
    rng = np.random.default_rng(2)
    a = rng.uniform(0.1, 1.0, size=6)
    A = sp.csr_matrix(a[None, :])
    x = rng.uniform(size=6) * 10
    l, u = np.array([1.0]), np.array([2.0])
    S = O.setup(A, l, u)
    x1, _ = O.sweep(S, O.CIMMINO, l, u, 1.0, -np.inf, np.inf, x)
    assert abs(a @ x1 - 2.0) < 1e-14 * 10


def _tiny(seed, m=12, n=6, consistent=True):
    rng = np.random.default_rng(seed)
    A = sp.csr_matrix(rng.uniform(0, 1, size=(m, n)) * (rng.uniform(size=(m, n)) < 0.7))
    A = A[np.asarray(A.multiply(A).sum(1)).ravel() > 0]
    xt = rng.uniform(0, 1, size=n)
    b = A @ xt
    if not consistent:
        b = b * (1 + 0.5 * rng.standard_normal(b.shape))
    l, u = np.minimum(b * 0.97, b * 1.03), np.maximum(b * 0.97, b * 1.03)
    return A, l, u


@pytest.mark.parametrize("lam", [0.5, 1.0, 1.5, 1.9])
@pytest.mark.parametrize("consistent", [True, False])
def test_cimmino_proximity_nonincreasing(lam, consistent):
    """The box-projected simultaneous step is a projected gradient step on
    F = 1/2 sum w_i d_i^2 with Lipschitz constant sum w_i = 1, so F never
    increases for lambda in (0, 2) -- on consistent and inconsistent systems."""
    A, l, u = _tiny(7 + int(consistent), consistent=consistent)
    S = O.setup(A, l, u)
    x = np.full(A.shape[1], 0.9)
    prev = O.proximity(S, l, u, x)
    for _ in range(200):
        x, p_in = O.sweep(S, O.CIMMINO, l, u, lam, 0.0, 1.0, x)
        assert abs(p_in - prev) <= 1e-15 + 1e-12 * prev    # monitor = F at the input
        cur = O.proximity(S, l, u, x)
        assert cur <= prev * (1 + 1e-12) + 1e-300
        prev = cur


def test_cimmino_consistent_converges_to_feasible():
    A, l, u = _tiny(21, consistent=True)
    S = O.setup(A, l, u)
    x = np.zeros(A.shape[1])
    for _ in range(5000):
        x, _ = O.sweep(S, O.CIMMINO, l, u, 1.0, 0.0, 1.0, x)
    assert O.proximity(S, l, u, x) < 1e-10


def test_cimmino_limit_is_bruteforce_least_violation_point_3x3():
    """3 inconsistent slabs in 3 unknowns with a box: the simultaneous method's
    limit minimises the equal-weight proximity over the box.  The minimiser is
    found independently by a dense grid and refined by L-BFGS-B; wrong weights
    or a wrong step would converge elsewhere."""
    A = np.array([[1.0, 0.5, 0.0], [0.2, 1.0, 0.7], [0.9, 0.0, 1.2]])
    l = np.array([1.4, 0.1, 1.9])
    u = np.array([1.6, 0.3, 2.0])
    # a 4th slab conflicting with the first makes the system inconsistent
    A = np.vstack([A, [1.0, 0.5, 0.0]])
    l = np.append(l, 0.2)
    u = np.append(u, 0.3)
    S = O.setup(sp.csr_matrix(A), l, u)
    x = np.full(3, 0.5)
    for _ in range(20000):
        x, _ = O.sweep(S, O.CIMMINO, l, u, 1.0, 0.0, 1.0, x)

    def F(y):   # 1/2 mean of squared distances, written from the geometry
        r = A @ y
        viol = np.maximum(l - r, 0) + np.maximum(r - u, 0)
        return 0.5 * np.mean(viol ** 2 / np.sum(A * A, axis=1))

    g = np.linspace(0, 1, 61)
    G = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    R = G @ A.T
    V = np.maximum(l - R, 0) + np.maximum(R - u, 0)
    Fg = 0.5 * np.mean(V ** 2 / np.sum(A * A, axis=1), axis=1)
    y0 = G[np.argmin(Fg)]
    res = so.minimize(F, y0, method="L-BFGS-B", bounds=[(0, 1)] * 3,
                      options={"ftol": 1e-16, "gtol": 1e-12, "maxiter": 10000})
    assert F(x) <= Fg.min() + 1e-12
    assert abs(F(x) - res.fun) < 1e-10
    np.testing.assert_allclose(x, res.x, atol=2e-4)


def test_bip_single_block_is_cimmino_bitwise():
    A, l, u = _tiny(31, m=20, n=8, consistent=False)
    S1 = O.setup(A, l, u)
    S2 = O.setup(A, l, u, O.BIP, np.zeros(A.shape[0], dtype=np.int32))
    x1 = x2 = np.full(A.shape[1], 0.3)
    for _ in range(20):
        x1, p1 = O.sweep(S1, O.CIMMINO, l, u, 1.0, 0.0, 1.0, x1)
        x2, p2 = O.sweep(S2, O.BIP, l, u, 1.0, 0.0, 1.0, x2)
        np.testing.assert_array_equal(x1, x2)
        assert p1 == p2


def test_bip_block_step_does_not_increase_block_proximity():
    A, l, u = _tiny(41, m=24, n=8, consistent=False)
    blocks = np.arange(A.shape[0]) % 3
    S = O.setup(A, l, u, O.BIP, blocks.astype(np.int32))
    x = np.full(A.shape[1], 0.7)
    for _ in range(30):
        for rows, At in zip(S.blocks, S.sub):
            St = O.setup(At, l[rows], u[rows])
            before = O.proximity(St, l[rows], u[rows], x)
            x, _ = O.simultaneous_step(At, S.rho[rows], S.keep[rows], S.w_sweep[rows],
                                       S.w_prox[rows], l[rows], u[rows], 1.0, 0.0, 1.0, x)
            assert O.proximity(St, l[rows], u[rows], x) <= before * (1 + 1e-12) + 1e-300


def test_bip_weights_are_per_block():
    A = sp.csr_matrix(np.eye(5))
    S = O.setup(A, np.zeros(5), np.ones(5), O.BIP, np.array([0, 0, 1, 1, 1], np.int32))
    np.testing.assert_allclose(S.w_sweep, [0.5, 0.5, 1 / 3, 1 / 3, 1 / 3])
    np.testing.assert_allclose(S.w_prox, np.full(5, 0.2))


# ------------------------------------------------------------- objectives --

def test_tv_constant_image_is_zero():
    assert O.tv_iso(np.full(12, 0.37), 3, 4) == 0.0
    assert O.tv_aniso(np.full(12, 0.37), 3, 4) == 0.0
    assert not np.any(O.tv_iso_subgrad(np.full(12, 0.37), 3, 4))


@pytest.mark.parametrize("H,W,c", [(5, 7, 3), (8, 4, 2)])
def test_tv_vertical_step_edge(H, W, c):
    """A vertical edge of height h between columns c-1 and c crosses H-1 terms
    of Eq. (TV) with value h each (non-square H x W catches a transposition)."""
    h = 0.8
    X = np.zeros((H, W))
    X[:, c:] = h
    assert abs(O.tv_iso(X.ravel(), H, W) - (H - 1) * h) < 1e-14
    assert abs(O.tv_aniso(X.ravel(), H, W) - H * h) < 1e-14
    Xt = np.zeros((H, W))
    Xt[c:, :] = h     # horizontal edge: W-1 terms
    assert abs(O.tv_iso(Xt.ravel(), H, W) - (W - 1) * h) < 1e-14


def test_tv_checkerboard_closed_forms():
    H, W, h = 6, 9, 0.5
    X = h * ((np.arange(H)[:, None] + np.arange(W)[None, :]) % 2).astype(float)
    assert abs(O.tv_iso(X.ravel(), H, W) - (H - 1) * (W - 1) * h * np.sqrt(2)) < 1e-12
    assert abs(O.tv_aniso(X.ravel(), H, W) - h * ((H - 1) * W + H * (W - 1))) < 1e-12


@pytest.mark.parametrize("kind", [O.OBJ_TV_ISO, O.OBJ_TV_ANISO])
def test_tv_subgradient_matches_central_differences(kind):
    """Away from kinks TV is differentiable and its subgradient is the
    gradient: compare with central finite differences."""
    H, W = 7, 5
    rng = np.random.default_rng(9)
    x = rng.uniform(size=H * W)    # distinct values: no kink
    ob = O.Objective(kind, (H, W))
    g = ob.g(x)
    eps = 1e-6
    fd = np.array([(ob.f(x + eps * e) - ob.f(x - eps * e)) / (2 * eps) for e in np.eye(H * W)])
    np.testing.assert_allclose(g, fd, atol=1e-6)


def test_tv_subgradient_inequality_at_kinks():
    """At a kink (flat regions) the returned vector is a subgradient:
    f(y) >= f(x) + g.(y - x) for all y (checked on random y)."""
    H, W = 6, 6
    x = np.zeros(H * W)
    x[7] = 1.0
    x[20:24] = 0.5
    rng = np.random.default_rng(4)
    for kind in (O.OBJ_TV_ISO, O.OBJ_TV_ANISO):
        ob = O.Objective(kind, (H, W))
        g, fx = ob.g(x), ob.f(x)
        for _ in range(200):
            y = x + rng.standard_normal(H * W) * rng.uniform(0.001, 1.0)
            assert ob.f(y) >= fx + g @ (y - x) - 1e-12


def test_mean_dose_vector_hand_example():
    """f_Mean over a 2-voxel structure with doses d = A x: c = A^T 1 / N."""
    body = sp.csr_matrix(np.array([[1.0, 2.0], [3.0, 4.0]]))
    np.testing.assert_allclose(O.mean_dose_vector(body), [2.0, 3.0])


# ---------------------------------------------------------- perturbations --

def test_linear_objective_step_decreases_by_beta_norm():
    """For f = c.x and v = -c/||c||: f(z) = f(y) - beta ||c|| (Sec. 2.1.2, Q3)."""
    c = np.array([0.2, 1.5, 0.7])
    ob = O.Objective(O.OBJ_LINEAR, c=c)
    st = O.PertState()
    P = O.Params(gamma=0.8, alpha=0.9, n_red=1)
    y = np.array([1.0, 2.0, 3.0])
    z, acc, tr = O.perturbation_phase(ob, y.copy(), st, P)
    assert acc == 1 and tr == 1 and st.ell == 1
    assert abs(ob.f(z) - (ob.f(y) - 0.8 * np.linalg.norm(c))) < 1e-14


def test_perturbation_is_nonascending_and_counts_trials():
    """Accepted steps never increase f (Algorithm 1); the exponent advances at
    every trial (Q4) and the step sizes stay below gamma / (1 - alpha)."""
    H, W = 16, 16
    rng = np.random.default_rng(8)
    x = rng.uniform(size=H * W)
    ob = O.Objective(O.OBJ_TV_ISO, (H, W))
    P = O.Params(gamma=2.0, alpha=0.7, n_red=4, max_trials=50)
    st = O.PertState()
    total_beta = 0.0
    f0 = ob.f(x)
    for k in range(30):
        ell0 = st.ell
        x, acc, tr = O.perturbation_phase(ob, x, st, P)
        assert st.ell - ell0 == tr
        total_beta += sum(P.gamma * P.alpha ** e for e in range(ell0, st.ell))
        f1 = ob.f(x)
        assert f1 <= f0 + 1e-12
        f0 = f1
    assert total_beta <= P.gamma / (1 - P.alpha) + 1e-12


def test_unperturbed_run_equals_plain_sweeps():
    """obj = NONE (or gamma = 0) gives exactly the feasibility-seeking iterates."""
    A, l, u = _tiny(51, m=30, n=16, consistent=False)
    S = O.setup(A, l, u)
    P = O.Params(gamma=0.0, max_sweeps=15)
    ob = O.Objective(O.OBJ_TV_ISO, (4, 4))
    r0 = O.run(S, O.CIMMINO, l, u, 0.0, 1.0, O.Objective(O.OBJ_NONE), P)
    r1 = O.run(S, O.CIMMINO, l, u, 0.0, 1.0, ob, P, x0=np.zeros(16))
    x = np.zeros(16)
    for _ in range(15):
        x, _ = O.sweep(S, O.CIMMINO, l, u, 1.0, 0.0, 1.0, x)
    np.testing.assert_array_equal(r0.x, x)
    np.testing.assert_array_equal(r1.x, x)


def test_restart_resets_exponent():
    """Sec. 2.1.2: after the r-th restart the exponent becomes r (Q7)."""
    P = O.Params(restart_every=10)
    st = O.PertState(ell=37)
    O.maybe_restart(st, 9, P)
    assert st.ell == 37
    O.maybe_restart(st, 10, P)
    assert st.ell == 1 and st.restarts == 1
    O.maybe_restart(st, 10, P)      # idempotent within one iteration
    assert st.ell == 1
    st.ell = 50
    O.maybe_restart(st, 20, P)
    assert st.ell == 2


def test_zero_subgradient_skips_phase():
    """x0 = 0 has TV subgradient 0: the phase accepts nothing and leaves l (Q6, Q18)."""
    ob = O.Objective(O.OBJ_TV_ISO, (4, 4))
    st = O.PertState()
    y, acc, tr = O.perturbation_phase(ob, np.zeros(16), st, O.Params())
    assert acc == 0 and tr == 0 and st.ell == 0 and not y.any()


# --------------------------------------------------------------- stopping --

def test_stopping_defaults_are_the_papers():
    with open(os.path.join(GOLD, "paper_defaults.json")) as fh:
        gold = json.load(fh)["stopping"]
    P = O.Params()
    assert P.prox_abs == gold["prox_abs"] and P.prox_rel == gold["prox_rel"]
    assert P.patience == gold["patience"] and P.max_sweeps == gold["max_sweeps"]
    assert P.obj_rel == gold["obj_rel"]


def test_stopping_rule_sequences():
    P = O.Params(prox_abs=1e-6, prox_rel=1e-3, patience=3, obj_rel=0.0)
    ss = O.StopState()
    seq = [1.0, 0.5, 0.4999, 0.49985, 0.4998, 0.49979, 0.3]
    hits = [O.stop_check(ss, p, None, P) for p in seq]
    assert hits == [False, False, False, False, True, True, False]
    ss = O.StopState()
    assert O.stop_check(ss, 1e-7, None, P)          # below P*
    # objective criterion must also hold when enabled
    P2 = O.Params(prox_abs=1e-6, obj_rel=1e-6)
    ss = O.StopState()
    assert not O.stop_check(ss, 1e-7, 10.0, P2)
    assert O.stop_check(ss, 1e-7, 10.0 + 1e-7, P2)
    assert not O.stop_check(ss, 1e-7, 11.0, P2)


# ---------------------------------------------------------------- DROP ----

def test_drop_column_scaling_for_disjoint_rows_is_exact_projection():
    """Rows with disjoint supports: every column has one nonzero, Z = I, and a
    DROP step with lambda = 1 projects onto every slab at once -- the exact
    projection onto their intersection (each slab constrains its own
    coordinates), landing on the feasible set in one step."""
    rng = np.random.default_rng(41)
    blocks = [np.arange(0, 3), np.arange(3, 7), np.arange(7, 9)]
    A = np.zeros((3, 9))
    for i, cols in enumerate(blocks):
        A[i, cols] = rng.uniform(0.5, 2.0, size=len(cols))
    l = np.array([1.0, -0.5, 2.0])
    u = np.array([1.5, 0.5, 2.2])
    S = O.setup(sp.csr_matrix(A), l, u, O.DROP)
    np.testing.assert_array_equal(S.z, np.ones(9))
    x = rng.uniform(-2, 2, size=9)
    y, _ = O.sweep(S, O.DROP, l, u, 1.0, -np.inf, np.inf, x)
    r = A @ y
    assert np.all(r >= l - 1e-12) and np.all(r <= u + 1e-12)
    # and it is the nearest feasible point: each block moved along its row
    for i, cols in enumerate(blocks):
        ri = A[i] @ x
        want = x[cols] + (np.clip(ri, l[i], u[i]) - ri) / (A[i] @ A[i]) * A[i, cols]
        np.testing.assert_allclose(y[cols], want, atol=1e-12)


def test_drop_with_constant_column_counts_is_the_scaled_simultaneous_step():
    """Every column with exactly two nonzeros: Z = I/2, so DROP equals the
    simultaneous step with unit weights halved (w_i = 1/2, not 1/m')."""
    rng = np.random.default_rng(43)
    n = 8
    A = np.zeros((n, n))
    for j in range(n):          # column j lives in rows j and j+1 (cyclic)
        A[j, j] = rng.uniform(0.5, 1.5)
        A[(j + 1) % n, j] = rng.uniform(0.5, 1.5)
    b = A @ rng.uniform(0, 1, n)
    l, u = b * 0.9, b * 1.1
    S = O.setup(sp.csr_matrix(A), l, u, O.DROP)
    np.testing.assert_allclose(S.z, np.full(n, 0.5))
    x = rng.uniform(-1, 2, n)
    y, _ = O.sweep(S, O.DROP, l, u, 1.3, 0.0, 1.0, x)
    # the same step written out row by row
    acc = np.zeros(n)
    for i in range(n):
        r = A[i] @ x
        acc += (np.clip(r, l[i], u[i]) - r) / (A[i] @ A[i]) * A[i]
    np.testing.assert_allclose(y, np.clip(x + 1.3 * 0.5 * acc, 0.0, 1.0), atol=1e-13)


@pytest.mark.parametrize("lam", [0.5, 1.0, 1.9])
def test_drop_unit_weight_proximity_nonincreasing(lam):
    """With unit weights and Z = diag(1/s_j), sum_i a_i a_i^T/||a_i||^2 has norm
    at most 1 in the Z^{-1} metric, so the box-projected DROP step does not
    increase F = 1/2 sum_i d_i^2/||a_i||^2 for lambda in (0, 2)."""
    A, l, u = _tiny(45, consistent=False)
    S = O.setup(A, l, u, O.DROP)
    Ad = A.toarray()

    def F(y):
        r = Ad @ y
        d = np.clip(r, l, u) - r
        return 0.5 * np.sum(d ** 2 / np.sum(Ad * Ad, axis=1))

    x = np.full(A.shape[1], 0.9)
    prev = F(x)
    for _ in range(200):
        x, _ = O.sweep(S, O.DROP, l, u, lam, 0.0, 1.0, x)
        cur = F(x)
        assert cur <= prev * (1 + 1e-12) + 1e-300
        prev = cur


def test_drop_limit_is_the_least_violation_point_3x3():
    """The fixed points of box(x + lambda Z g) are those of box(x + lambda g)
    for a positive diagonal Z, so DROP converges to the same brute-force
    least-violation point as the simultaneous method (unit weights)."""
    A = np.array([[1.0, 0.5, 0.0], [0.2, 1.0, 0.7], [0.9, 0.0, 1.2], [1.0, 0.5, 0.0]])
    l = np.array([1.4, 0.1, 1.9, 0.2])
    u = np.array([1.6, 0.3, 2.0, 0.3])
    S = O.setup(sp.csr_matrix(A), l, u, O.DROP)
    np.testing.assert_allclose(S.z, [1 / 4, 1 / 3, 1 / 2])   # column nonzeros 4, 3, 2
    x = np.full(3, 0.5)
    for _ in range(40000):
        x, _ = O.sweep(S, O.DROP, l, u, 1.0, 0.0, 1.0, x)

    def F(y):
        r = A @ y
        viol = np.maximum(l - r, 0) + np.maximum(r - u, 0)
        return 0.5 * np.sum(viol ** 2 / np.sum(A * A, axis=1))

    g = np.linspace(0, 1, 61)
    G = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    R = G @ A.T
    V = np.maximum(l - R, 0) + np.maximum(R - u, 0)
    Fg = 0.5 * np.sum(V ** 2 / np.sum(A * A, axis=1), axis=1)
    res = so.minimize(F, G[np.argmin(Fg)], method="L-BFGS-B", bounds=[(0, 1)] * 3,
                      options={"ftol": 1e-16, "gtol": 1e-12, "maxiter": 10000})
    assert abs(F(x) - res.fun) < 1e-10
    np.testing.assert_allclose(x, res.x, atol=2e-4)


# ------------------------------------------------------ L1 / L2 objectives ----

def test_l1_objective_value_and_subgradient_inequality():
    """f = ||x||_1: the value is the sum of magnitudes and sign(x) (0 at 0) is
    a subgradient: f(y) >= f(x) + g.(y - x) for every y."""
    rng = np.random.default_rng(61)
    x = rng.normal(size=50)
    x[[3, 17]] = 0.0
    ob = O.Objective(O.OBJ_L1)
    assert ob.f(x) == pytest.approx(sum(abs(v) for v in x), rel=1e-15)
    g = ob.g(x)
    assert g[3] == 0.0 and g[17] == 0.0
    for _ in range(200):
        y = rng.normal(size=50)
        assert ob.f(y) >= ob.f(x) + g @ (y - x) - 1e-12


def test_l2_objective_gradient_by_central_differences():
    rng = np.random.default_rng(62)
    x = rng.normal(size=20)
    ob = O.Objective(O.OBJ_L2)
    assert ob.f(x) == pytest.approx(float(np.dot(x, x)), rel=1e-15)
    h = 1e-6
    fd = np.array([(ob.f(x + h * e) - ob.f(x - h * e)) / (2 * h) for e in np.eye(20)])
    np.testing.assert_allclose(ob.g(x), fd, atol=1e-6)


def test_l2_perturbation_step_shrinks_towards_the_origin():
    """With f = ||x||^2 the normalised direction is -x/||x||, so an accepted
    step of size beta < ||x|| scales x by (1 - beta/||x||) exactly."""
    x = np.array([3.0, -4.0, 0.0, 12.0])          # ||x|| = 13
    P = O.Params(gamma=2.6, alpha=0.5, n_red=1, max_trials=5)
    st = O.PertState()
    y, a, t = O.perturbation_phase(O.Objective(O.OBJ_L2), x, st, P)
    assert (a, t, st.ell) == (1, 1, 1)
    np.testing.assert_allclose(y, x * (1 - 2.6 / 13.0), atol=1e-14)


# ------------------------------------------------- variance stopping rule ----

def test_variance_of_changes_is_the_sample_variance():
    w = [1.0, 0.2, 0.1, 0.05]
    m = sum(w) / 4
    assert O.variance_of_changes(w) == pytest.approx(sum((v - m) ** 2 for v in w) / 3,
                                                     rel=1e-15)


def test_variance_rule_stops_at_the_first_iterate_below_the_threshold():
    """Replaying the run by hand: the rule stops after the first iteration k
    >= 2 whose variance of relative changes falls below the threshold."""
    A, l, u = _tiny(71, m=30, n=10, consistent=False)
    S = O.setup(A, l, u)
    P = O.Params(max_sweeps=400, variance_tol=1e-2)     # the paper's threshold
    r = O.run(S, O.CIMMINO, l, u, 0.0, 1.0, O.Objective(O.OBJ_NONE), P)
    x = np.zeros(A.shape[1])
    omega = []
    for k in range(1, 401):
        y, _ = O.sweep(S, O.CIMMINO, l, u, 1.0, 0.0, 1.0, x)
        omega.append(np.linalg.norm(y - x) / np.linalg.norm(y))
        x = y
        if k >= 2 and np.var(omega, ddof=1) < 1e-2:
            break
    assert r.sweeps == k < 400
    np.testing.assert_array_equal(r.x, x)


# ------------------------------------------------------------ EL / EMR ----

def _orthogonal_rows(seed, m=4, n=9, norm=1.7):
    """Rows with disjoint supports scaled to one norm: pairwise orthogonal."""
    rng = np.random.default_rng(seed)
    A = np.zeros((m, n))
    cols = np.array_split(rng.permutation(n), m)
    for i, c in enumerate(cols):
        v = rng.uniform(0.5, 2.0, size=len(c))
        A[i, c] = norm * v / np.linalg.norm(v)
    return A


@pytest.mark.parametrize("mode", [O.EL, O.EMR])
def test_extrapolated_steps_project_exactly_on_orthogonal_equal_norm_rows(mode):
    """Orthogonal rows of equal norm: the simultaneous direction is the sum of
    the single projections scaled by w, and both EL's t (1/w) and EMR's exact
    line search undo that scaling -- one step lands on the intersection of
    the slabs, the nearest feasible point (the Cimmino step moves 1/m of the
    way)."""
    A = _orthogonal_rows(81)
    rng = np.random.default_rng(82)
    x = rng.uniform(-1, 1, size=A.shape[1])
    l = A @ x + rng.uniform(0.3, 1.0, size=4) * rng.choice([-1, 1], size=4)
    u = l + 0.2
    S = O.setup(sp.csr_matrix(A), l, u)
    y, _ = O.sweep(S, mode, l, u, 1.0, -np.inf, np.inf, x)
    want = x.copy()
    for i in range(4):
        r = A[i] @ x
        want += (np.clip(r, l[i], u[i]) - r) / (A[i] @ A[i]) * A[i]
    np.testing.assert_allclose(y, want, atol=1e-12)
    c, _ = O.sweep(S, O.CIMMINO, l, u, 1.0, -np.inf, np.inf, x)
    np.testing.assert_allclose(c, x + (want - x) / 4, atol=1e-12)


def test_emr_step_is_the_exact_line_search_of_the_weighted_residual():
    """EMR's t minimises phi(t) = sum_i w_i (r_i + t q_i)^2 along the step for an
    equality system (l = u): checked against a dense scan of t."""
    rng = np.random.default_rng(83)
    A = rng.uniform(0, 1, size=(15, 6)) * (rng.uniform(size=(15, 6)) < 0.8)
    A = A[np.sum(A * A, axis=1) > 0]
    b = A @ rng.uniform(0, 1, 6) + 0.1 * rng.standard_normal(A.shape[0])
    S = O.setup(sp.csr_matrix(A), b, b)
    x = rng.uniform(0, 1, 6)
    y, _ = O.sweep(S, O.EMR, b, b, 1.0, -np.inf, np.inf, x)
    w = 1.0 / A.shape[0]
    g = A.T @ (w * (A @ x - b))
    phi = lambda t: np.sum(w * (A @ (x - t * g) - b) ** 2)
    ts = np.linspace(0, 50, 200001)
    vals = np.array([phi(t) for t in ts[::100]])
    t_best = ts[::100][np.argmin(vals)]
    t_emr = np.linalg.norm(x - y) / np.linalg.norm(g)
    assert abs(t_emr - t_best) <= 0.03 * t_best
    assert phi(t_emr) <= vals.min() + 1e-12


def _consistent_slabs(seed, m=14, n=8):
    rng = np.random.default_rng(seed)
    A = rng.uniform(0, 1, size=(m, n)) * (rng.uniform(size=(m, n)) < 0.7)
    A = A[np.sum(A * A, axis=1) > 0]
    xt = rng.uniform(0, 1, size=n)
    b = A @ xt
    return sp.csr_matrix(A), b * 0.97, b * 1.03, xt


def test_el_is_fejer_monotone_for_consistent_slabs():
    """EL extrapolates a firmly nonexpansive simultaneous step (t >= 1 is the
    extrapolation of Cegielski's method), so on a consistent system every
    feasible point z gets no farther away: ||x^(k+1) - z|| <= ||x^k - z||."""
    A, l, u, xt = _consistent_slabs(85)
    S = O.setup(A, l, u)
    x = np.full(A.shape[1], 2.0)
    prev = np.linalg.norm(x - xt)
    for _ in range(300):
        x, _ = O.sweep(S, O.EL, l, u, 1.0, -np.inf, np.inf, x)
        cur = np.linalg.norm(x - xt)
        assert cur <= prev * (1 + 1e-12) + 1e-15
        prev = cur
    assert O.proximity(S, l, u, x) < 1e-8


def test_emr_weighted_residual_never_increases_on_consistent_slabs():
    """EMR's t is the exact minimiser of the weighted residual along its
    direction, so sum_i w_i d_i^2 never increases (up to rounding) and the
    iterates become feasible."""
    A, l, u, _ = _consistent_slabs(86)
    S = O.setup(A, l, u)
    Ad = A.toarray()

    def F(y):
        r = Ad @ y
        d = np.clip(r, l, u) - r
        return np.sum(d ** 2)

    x = np.full(A.shape[1], 2.0)
    prev = F(x)
    for _ in range(300):
        x, _ = O.sweep(S, O.EMR, l, u, 1.0, -np.inf, np.inf, x)
        cur = F(x)
        assert cur <= prev * (1 + 1e-9) + 1e-24
        prev = cur
    assert O.proximity(S, l, u, x) < 1e-8


# ------------------------------------------------- split feasibility (DVC) --

def _dvc_bruteforce(d, kind, K, d_ref):
    """Nearest point of the dose-volume set by enumerating its convex pieces:
    every voxel subset S of size K (upper: S may exceed d_ref; lower: S must
    reach it).  Returns the smallest distance."""
    from itertools import combinations
    best = np.inf
    for S in combinations(range(len(d)), K):
        S = list(S)
        p = d.copy()
        mask = np.zeros(len(d), bool)
        mask[S] = True
        if kind == O.DVC_UPPER:
            p[~mask] = np.minimum(d[~mask], d_ref)
        else:
            p[mask] = np.maximum(d[mask], d_ref)
        best = min(best, float(np.linalg.norm(p - d)))
    return best


@pytest.mark.parametrize("seed", range(8))
def test_dvc_projection_is_the_nearest_point_of_the_union(seed):
    """Q26: the projection onto {at most / at least K voxels beyond d_ref} is
    the nearest point over all K-subsets (brute force), and it lies in the set
    as the paper words it: not more than V N voxels above d_ref (upper), at
    least V N voxels at or above d_ref (lower)."""
    rng = np.random.default_rng(900 + seed)
    for N in range(1, 8):
        for trial in range(6):
            d = rng.standard_normal(N) * 2 + 3
            if trial % 2:
                d = np.round(d)             # ties
            d_ref = float(np.median(d) + rng.uniform(-1, 1))
            for V in (0.0, 0.1, 0.3, 0.5, 0.75, 1.0):
                for kind in (O.DVC_UPPER, O.DVC_LOWER):
                    p = O.dvc_project(d, kind, V, d_ref)
                    K = O.dvc_count(kind, V, N)
                    ref = _dvc_bruteforce(d, kind, K, d_ref)
                    assert abs(np.linalg.norm(p - d) - ref) <= 1e-12
                    if kind == O.DVC_UPPER:
                        assert np.count_nonzero(p > d_ref) <= V * N
                    else:
                        assert np.count_nonzero(p >= d_ref) >= V * N - 1e-12
                    # only voxels on the wrong side move, and only to d_ref
                    moved = p != d
                    assert np.all(p[moved] == d_ref)


def test_dvc_counts_round_towards_the_constraint():
    """'Not more than V%' allows floor(V N) voxels, 'at least V%' demands
    ceil(V N): 5% of 30 voxels is 1.5."""
    assert O.dvc_count(O.DVC_UPPER, 0.05, 30) == 1
    assert O.dvc_count(O.DVC_LOWER, 0.05, 30) == 2
    assert O.dvc_count(O.DVC_UPPER, 0.95, 20) == 19
    assert O.dvc_count(O.DVC_LOWER, 0.95, 20) == 19
    assert O.dvc_count(O.DVC_LOWER, 1.0, 7) == 7
    assert O.dvc_count(O.DVC_UPPER, 0.0, 7) == 0


def test_dvc_equal_doses_rank_lower_index_first():
    p = O.dvc_project(np.array([5.0, 5.0, 5.0, 1.0]), O.DVC_UPPER, 0.25, 2.0)
    assert p.tolist() == [5.0, 2.0, 2.0, 1.0]
    p = O.dvc_project(np.array([1.0, 1.0, 1.0, 9.0]), O.DVC_LOWER, 0.75, 4.0)
    assert p.tolist() == [4.0, 4.0, 1.0, 9.0]


def test_dvc_extreme_volumes_are_the_plain_clamps():
    """V = 0 upper is {d <= d_ref} voxel-wise, V = 1 lower is {d >= d_ref}."""
    rng = np.random.default_rng(77)
    d = rng.standard_normal(50)
    assert np.array_equal(O.dvc_project(d, O.DVC_UPPER, 0.0, 0.1), np.minimum(d, 0.1))
    assert np.array_equal(O.dvc_project(d, O.DVC_LOWER, 1.0, -0.2), np.maximum(d, -0.2))
    assert np.array_equal(O.dvc_project(d, O.DVC_UPPER, 1.0, 0.1), d)
    assert np.array_equal(O.dvc_project(d, O.DVC_LOWER, 0.0, 0.1), d)


def _equal_norm_rows(m, n, seed, norm=1.3):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * (rng.uniform(size=(m, n)) < 0.6)
    A[:, 0] += 0.5                      # no zero rows
    A *= norm / np.linalg.norm(A, axis=1, keepdims=True)
    return A


@pytest.mark.parametrize("relax", [0.8, 1.6])
def test_cq_step_with_halfspace_dvcs_is_the_cimmino_step(relax):
    """With V = 0 every upper DVC is the halfspace family a_i x <= d_ref; on
    rows of equal norm rho the CQ step x + gamma sum_j w_j A_j^T (P - d),
    gamma = relax / sum_j w_j ||A_j||_F^2, is the simultaneous projection step
    x + lambda sum_i (1/m) (clamp(r_i) - r_i)/rho a_i with lambda = relax."""
    m1, m2, n = 7, 5, 6
    A = _equal_norm_rows(m1 + m2, n, 31)
    rng = np.random.default_rng(32)
    x = rng.standard_normal(n)
    u = np.concatenate([np.full(m1, 0.2), np.full(m2, -0.1)])
    dv = [O.DVC(O.DVC_UPPER, 0, 0.0, 0.2), O.DVC(O.DVC_UPPER, 1, 0.0, -0.1)]
    SS = O.split_setup(sp.csr_matrix(A), [0, m1, m1 + m2], dv, relax)
    xq, pq = O.cq_step(SS, x)
    S = O.setup(sp.csr_matrix(A), np.full(m1 + m2, -np.inf), u)
    xc, pc = O.simultaneous_step(S.A, S.rho, S.keep, S.w_sweep, S.w_prox, np.full(m1 + m2, -np.inf),
                                 u, relax, -np.inf, np.inf, x)
    assert np.allclose(xq, xc, rtol=1e-13, atol=1e-14)
    # proximities: target space weights 1/2 per DVC vs 1/m per row with 1/rho
    r = A @ x
    e = np.minimum(r, u) - r
    assert np.isclose(pq, 0.5 * (0.5 * e[:m1] @ e[:m1] + 0.5 * e[m1:] @ e[m1:]), rtol=1e-13)
    assert np.isclose(pc, 0.5 * np.sum(e ** 2) / (m1 + m2) / 1.3 ** 2, rtol=1e-13)


def _split_case(seed):
    rng = np.random.default_rng(seed)
    m1, m2, n = 12, 9, 8
    A = np.abs(rng.standard_normal((m1 + m2, n))) * (rng.uniform(size=(m1 + m2, n)) < 0.7)
    dv = [O.DVC(O.DVC_LOWER, 0, 0.75, 3.0), O.DVC(O.DVC_UPPER, 0, 0.25, 4.0),
          O.DVC(O.DVC_UPPER, 1, 0.2, 1.5)]
    return A, [0, m1, m1 + m2], dv, rng


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_cq_direction_is_minus_the_gradient_of_the_target_proximity(seed):
    """Away from ties and from d_ref the selected voxels stay fixed nearby, so
    p(x) = 1/2 sum_j w_j ||P_Qj(A_j x) - A_j x||^2 is smooth there and the CQ
    step is x - gamma grad p (central differences)."""
    A, sptr, dv, rng = _split_case(seed)
    SS = O.split_setup(sp.csr_matrix(A), sptr, dv, 1.0)
    x = np.abs(rng.standard_normal(A.shape[1])) * 0.7
    d = A @ x
    for q in dv:       # margins: no dose near d_ref, no near-equal doses
        dj = d[sptr[q.structure]:sptr[q.structure + 1]]
        assert np.min(np.abs(dj - q.d_ref)) > 1e-4
        assert np.min(np.diff(np.sort(dj))) > 1e-4
    xn, p0 = O.cq_step(SS, x)
    assert p0 > 0
    h = 1e-6
    grad = np.array([(O.dvc_proximity(SS, x + h * e) - O.dvc_proximity(SS, x - h * e)) / (2 * h)
                     for e in np.eye(len(x))])
    assert np.allclose((xn - x) / SS.gamma, -grad, rtol=1e-6, atol=1e-8)
    # gamma is relax / sum_j w_j ||A_j||_F^2
    F = [np.sum(A[sptr[s]:sptr[s + 1]] ** 2) for s in range(2)]
    assert np.isclose(SS.gamma, 1.0 / ((F[0] + F[0] + F[1]) / 3.0), rtol=1e-14)


@pytest.mark.parametrize("relax", [1.0, 1.9])
def test_cq_iteration_never_increases_the_target_proximity(relax):
    """gamma < 2/L makes the CQ step a descent step of the quadratic built on
    the current projections, and re-projecting can only shorten the distances:
    the target-space proximity never increases, even for these nonconvex sets."""
    A, sptr, dv, rng = _split_case(11)
    SS = O.split_setup(sp.csr_matrix(A), sptr, dv, relax)
    x = np.abs(rng.standard_normal(A.shape[1])) * 2.0
    prev = np.inf
    for _ in range(60):
        x, p = O.cq_step(SS, x)
        assert p <= prev * (1 + 1e-12) + 1e-15
        prev = p


def test_cq_step_is_the_identity_when_every_dvc_holds():
    A, sptr, _, rng = _split_case(12)
    x = np.abs(rng.standard_normal(A.shape[1]))
    d = A @ x
    dv = [O.DVC(O.DVC_UPPER, 0, 0.1, float(d.max()) + 1.0),
          O.DVC(O.DVC_LOWER, 1, 0.9, float(d.min()) - 1.0)]
    SS = O.split_setup(sp.csr_matrix(A), sptr, dv, 1.0)
    xn, p = O.cq_step(SS, x)
    assert p == 0.0 and np.array_equal(xn, x)


# ------------------------------------------------ adaptive step (Nikazad) --

def test_adaptive_step_lands_on_the_reference_level_of_a_linear_objective():
    """For f = c.x the linearisation is exact: one adaptive step
    beta = (f(y) - f_ref)/||g|| along -g/||g|| reaches f(z) = f_ref."""
    rng = np.random.default_rng(41)
    c = rng.uniform(0.1, 1.0, 30)
    obj = O.Objective(O.OBJ_LINEAR, c=c)
    y = rng.uniform(0, 2, 30)
    f_ref = 0.6 * float(c @ y)
    P = O.Params(adaptive=2, f_ref=f_ref, n_red=1)
    z, acc, tri = O.perturbation_phase(obj, y, O.PertState(), P)
    assert acc == 1 and tri == 1
    assert np.isclose(c @ z, f_ref, rtol=1e-13)
    # below the reference level nothing moves
    z2, acc2, tri2 = O.perturbation_phase(obj, y, O.PertState(), O.Params(adaptive=2, f_ref=2 * c @ y))
    assert acc2 == 0 and tri2 == 0 and np.array_equal(z2, y)


@pytest.mark.parametrize("seed", range(4))
def test_adaptive_step_is_the_projection_onto_the_linearised_level_set(seed):
    """The step is the Euclidean projection of y onto {u : f(y) + g.(u - y) <=
    f_ref} (SLSQP on the constrained least-distance problem), here for the
    L1 norm with its subgradient sign(y)."""
    rng = np.random.default_rng(60 + seed)
    y = rng.standard_normal(6)
    obj = O.Objective(O.OBJ_L1)
    f_ref = 0.5 * float(np.abs(y).sum())
    z, acc, _ = O.perturbation_phase(obj, y, O.PertState(), O.Params(adaptive=2, f_ref=f_ref))
    g = np.sign(y)
    fy = float(np.abs(y).sum())
    res = so.minimize(lambda u: np.sum((u - y) ** 2), y.copy(), method="SLSQP",
                      constraints=[{"type": "ineq", "fun": lambda u: f_ref - fy - g @ (u - y)}],
                      options={"ftol": 1e-14, "maxiter": 500})
    assert acc == 1
    assert np.allclose(z, res.x, atol=1e-6)


def test_adaptive_steps_never_move_away_from_the_level_set():
    """Subgradient projections are Fejer monotone with respect to the level
    set: for the convex L1 norm and f_ref >= 0 every point u with
    ||u||_1 <= f_ref (here u = 0) gets no farther away, step after step."""
    rng = np.random.default_rng(71)
    y = rng.standard_normal(40) * 3
    f0 = np.abs(y).sum()
    obj = O.Objective(O.OBJ_L1)
    P = O.Params(adaptive=2, f_ref=1.0, n_red=1)
    prev = np.linalg.norm(y)
    for _ in range(50):
        y, acc, _ = O.perturbation_phase(obj, y, O.PertState(), P)
        cur = np.linalg.norm(y)
        assert cur <= prev * (1 + 1e-12)
        prev = cur
    assert np.abs(y).sum() < 0.1 * f0


def test_adaptive_reference_is_the_lowest_phase_start_objective():
    """Q29: with the automatic reference the first phase takes no step
    (f(x^0) is the reference), and later phases pull f back towards the
    lowest value seen at a phase start."""
    c = np.array([1.0, 2.0, 3.0])
    obj = O.Objective(O.OBJ_LINEAR, c=c)
    st = O.PertState()
    P = O.Params(adaptive=1, n_red=1)
    y0 = np.array([1.0, 1.0, 1.0])
    z, acc, tri = O.perturbation_phase(obj, y0, st, P)
    assert acc == 0 and np.array_equal(z, y0) and st.f_best == 6.0
    y1 = np.array([2.0, 2.0, 2.0])            # f = 12 after a feasibility step
    z, acc, _ = O.perturbation_phase(obj, y1, st, P)
    assert acc == 1 and np.isclose(c @ z, 6.0, rtol=1e-14) and st.f_best == 6.0
    y2 = np.array([0.5, 0.5, 0.5])            # f = 3: a new lowest value, no step
    z, acc, _ = O.perturbation_phase(obj, y2, st, P)
    assert acc == 0 and st.f_best == 3.0
