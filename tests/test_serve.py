"""The serving runtime (suppy_server_*): continuous batching of requests for
several registered matrices through batched contexts.

Each request's result must not depend on the mix it was served in: a
request served alone (its own server) and in a mix (other requests of the
same and other matrices arriving while it runs, slots reused) gives the same
iterate; both agree with the FP64 oracle run for the same number of sweeps,
within the full-run tolerance.
"""
import numpy as np
import pytest

import oracle as O
import paper_2606_27086_gb300 as pk
import synth
from tests.helpers import oracle_objective, rel, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

PARAMS = dict(gamma=0.5, alpha=0.99, n_red=1, max_sweeps=25, use_stopping=1, prox_rel=2e-3,
              patience=3, obj_rel=0.0, prox_abs=1e-9)


def _params(**kw):
    d = dict(PARAMS)
    d.update(use_stopping=0)
    d.update(kw)
    return pk.suppy_params_default(**d)


def _single(prob, l, u):
    import copy
    q = copy.copy(prob)
    q.l, q.u = np.ascontiguousarray(l), np.ascontiguousarray(u)
    return q


def _problems():
    ct = synth.ct_problem(32, 30, 45, nrhs=6)
    ct2 = synth.ct_problem(48, 36, 67, nrhs=3, seed_noise=700)
    return ct, ct2


def _run_all(srv, sched, n_of):
    """sched: list of (step index, matrix id, l, u); returns request ids in order."""
    ids = [None] * len(sched)
    done = set()
    step = 0
    while len(done) < len(sched):
        for k, (t, mid, l, u) in enumerate(sched):
            if ids[k] is None and t <= step:
                ids[k] = srv.suppy_server_submit(mid, l, u)
        srv.suppy_server_step()
        for k, rid in enumerate(ids):
            if rid is not None and k not in done:
                info, _ = srv.suppy_server_query(rid)
                if info["state"] == 2:
                    done.add(k)
        step += 1
        assert step < 200000
    out = []
    for k, rid in enumerate(ids):
        info, x = srv.suppy_server_query(rid, n_of[sched[k][1]])
        out.append((info, x))
    return out


def test_served_results_equal_alone_and_in_the_mix_and_match_the_oracle():
    ct, ct2 = _problems()
    P = pk.suppy_params_default(**PARAMS)
    mix = pk.Server(slots=4, check_every=3)
    m0 = mix.suppy_server_add_matrix(ct, P, obj=pk.SUPPY_OBJ_TV_ISO)
    m1 = mix.suppy_server_add_matrix(ct2, P, obj=pk.SUPPY_OBJ_TV_ISO)
    n_of = {m0: ct.A.n, m1: ct2.A.n}
    # nine requests, arriving over time: more than one context's slots for
    # matrix 0, so slots are reused and a second context may open
    sched = []
    for b in range(6):
        sched.append((3 * b, m0, ct.l[:, b], ct.u[:, b]))
    for b in range(3):
        sched.append((2 + 4 * b, m1, ct2.l[:, b], ct2.u[:, b]))
    res = _run_all(mix, sched, n_of)
    mix.close()
    for k, (t, mid, l, u) in enumerate(sched):
        info, x = res[k]
        assert info["state"] == 2 and x is not None
        assert info["t_done"] >= info["t_start"] >= info["t_submit"]
        alone = pk.Server(slots=4, check_every=3)
        a0 = alone.suppy_server_add_matrix(ct if mid == m0 else ct2, P, obj=pk.SUPPY_OBJ_TV_ISO)
        (ia, xa), = _run_all(alone, [(0, a0, l, u)], {a0: n_of[mid]})
        alone.close()
        assert ia["sweeps"] == info["sweeps"]
        assert rel_l2(x, xa) <= 1e-6
        # the context API with one right-hand side, same sweeps
        prob = ct if mid == m0 else ct2
        ctx = pk.from_problem(_single(prob, l, u), obj=pk.SUPPY_OBJ_TV_ISO)
        ctx.suppy_run(_params(max_sweeps=info["sweeps"]))
        assert rel_l2(x, ctx.suppy_get_x()) <= 1e-3
        # the oracle for the same number of sweeps
        S, _, _, lo, hi = O.from_problem(prob)
        op = O.Params(gamma=0.5, alpha=0.99, n_red=1, max_sweeps=info["sweeps"])
        r = O.run(S, O.CIMMINO, np.asarray(l, np.float64), np.asarray(u, np.float64), lo, hi,
                  oracle_objective(prob, O.OBJ_TV_ISO), op)
        assert rel_l2(x, r.x) <= 1e-3
        assert rel(info["proximity"], r.prox_hist[-1]) <= 1e-3


def test_admission_waits_for_the_memory_budget():
    """A budget that holds one context: requests for a second matrix wait
    until the first matrix's requests finish and its idle context is
    released; every request completes and the budget is never exceeded."""
    ct, ct2 = _problems()
    P = pk.suppy_params_default(**PARAMS)
    probe = pk.Server(slots=2, check_every=4)
    p0 = probe.suppy_server_add_matrix(ct2, P, obj=pk.SUPPY_OBJ_TV_ISO)
    _run_all(probe, [(0, p0, ct2.l[:, 0], ct2.u[:, 0])], {p0: ct2.A.n})
    one = probe.suppy_server_device_bytes()
    probe.close()
    srv = pk.Server(hbm_budget=int(one * 1.5), slots=2, check_every=4)
    m0 = srv.suppy_server_add_matrix(ct, P, obj=pk.SUPPY_OBJ_TV_ISO)
    m1 = srv.suppy_server_add_matrix(ct2, P, obj=pk.SUPPY_OBJ_TV_ISO)
    sched = [(0, m0, ct.l[:, b], ct.u[:, b]) for b in range(3)]
    sched += [(0, m1, ct2.l[:, b], ct2.u[:, b]) for b in range(2)]
    ids = [srv.suppy_server_submit(mid, l, u) for _, mid, l, u in sched]
    peak = 0
    for _ in range(200000):
        r, w = srv.suppy_server_step()
        peak = max(peak, srv.suppy_server_device_bytes())
        if r == 0 and w == 0:
            break
    assert peak <= int(one * 1.5)
    starts = {}
    for k, rid in enumerate(ids):
        info, _ = srv.suppy_server_query(rid)
        assert info["state"] == 2
        starts[k] = (info["t_start"], info["t_done"])
    # the second matrix waited for memory: it started only after requests of
    # the first matrix had finished and released their context
    first_done = min(starts[k][1] for k in range(3))
    assert min(starts[k][0] for k in range(3, 5)) >= first_done
    srv.close()


def test_server_rejects_bad_requests():
    ct, _ = _problems()
    P = pk.suppy_params_default(**PARAMS)
    srv = pk.Server(slots=2)
    m0 = srv.suppy_server_add_matrix(ct, P, obj=pk.SUPPY_OBJ_TV_ISO)
    l, u = ct.l[:, 0].copy(), ct.u[:, 0].copy()
    with pytest.raises(pk.SuppyError):
        srv.suppy_server_submit(m0 + 5, l, u)
    bad = l.copy()
    bad[3] = np.nan
    with pytest.raises(pk.SuppyError):
        srv.suppy_server_submit(m0, bad, u)
    with pytest.raises(pk.SuppyError):
        srv.suppy_server_submit(m0, u + 1.0, u)
    with pytest.raises(pk.SuppyError):
        srv.suppy_server_query(12345)
    srv.close()


def test_served_16_bit_storage_matches_the_oracle_on_rounded_values():
    """A server storing A by SUPPY_HALF_AUTO (FP16 for these CT values)
    serves each request as the oracle runs it on the FP16-rounded values."""
    from tests.helpers import rounded_values
    ct, _ = _problems()
    P = pk.suppy_params_default(**PARAMS)
    srv = pk.Server(slots=4, check_every=3)
    m0 = srv.suppy_server_add_matrix(ct, P, dtype=pk.SUPPY_HALF_AUTO, obj=pk.SUPPY_OBJ_TV_ISO)
    sched = [(2 * b, m0, ct.l[:, b], ct.u[:, b]) for b in range(3)]
    res = _run_all(srv, sched, {m0: ct.A.n})
    srv.close()
    S, _, _, lo, hi = O.from_problem(ct, values=rounded_values(ct.A.val, "f16"))
    for (t, mid, l, u), (info, x) in zip(sched, res):
        assert info["state"] == 2
        op = O.Params(gamma=0.5, alpha=0.99, n_red=1, max_sweeps=info["sweeps"])
        r = O.run(S, O.CIMMINO, np.asarray(l, np.float64), np.asarray(u, np.float64), lo, hi,
                  oracle_objective(ct, O.OBJ_TV_ISO), op)
        assert rel_l2(x, r.x) <= 1e-3
        assert rel(info["proximity"], r.prox_hist[-1]) <= 1e-3
