"""Restarts of the power-law step (Sec. 2.1.2): after the r-th restart the
exponent l is set back to r (reading Q7).  The paper's CT strategies 1 and 3
(gamma = 5, alpha = 0.99 / 0.9, n_red = 4, a restart every 50 iterations;
tests/golden/paper_defaults.json) over 120 superiorized iterations, against
the FP64 oracle: the same accepted steps, the iterate and the proximity
history within the full-run tolerance (1e-3).  Rejected trials whose test
f(z) <= f(y) is a near tie (the two sides equal up to FP32 rounding of z)
can be decided differently in FP32 and FP64: the trial totals agree within
1%, and the final exponent agrees within 2% or the trial difference
(without the restarts it would be about three times larger, the number of
all trials)."""
import json
import os

import numpy as np
import pytest

import oracle as O
import paper_2606_27086_gb300 as pk
import synth
from tests.helpers import oracle_objective, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_defaults.json")))


@pytest.mark.parametrize("strategy_id", ["1", "3"])
@pytest.mark.parametrize("path,sweep", [(1, pk.STRATEGY_TWO_PASS), (2, pk.STRATEGY_TILED),
                                        (1, pk.STRATEGY_ONE_PASS)])
def test_restarts_match_the_oracle(strategy_id, path, sweep):
    s = GOLD["ct_strategies"][strategy_id]
    assert s["restart_every"] == 50
    prob = synth.ct_problem(96, 120, 137)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, perturb_path=path, strategy=sweep)
    P = dict(gamma=float(s["gamma"]), alpha=s["alpha"], n_red=s["n_red"],
             restart_every=s["restart_every"], max_sweeps=120)
    st = ctx.suppy_run(pk.suppy_params_default(use_graphs=1, **P))[0]
    S, l, u, lo, hi = O.from_problem(prob)
    r = O.run(S, O.CIMMINO, l, u, lo, hi, oracle_objective(prob, O.OBJ_TV_ISO), O.Params(**P))
    assert st["sweeps"] == 120 and r.sweeps == 120
    # two restarts happened (after iterations 50 and 100): l was set back to 2
    # and has counted the trials since
    assert r.ell == 2 + sum(r.trials[100:])
    assert st["accepted"] == sum(r.accepted)
    d_trials = st["trials"] - sum(r.trials)
    assert abs(d_trials) <= 0.01 * sum(r.trials)
    assert abs(st["ell"] - r.ell) <= max(abs(d_trials), 0.02 * r.ell)
    assert st["ell"] < st["trials"] // 2
    assert rel_l2(ctx.suppy_get_x(), r.x) <= 1e-3
    ph, _ = ctx.suppy_history()
    po = np.asarray(r.prox_hist)
    assert np.max(np.abs(np.asarray(ph) - po) / np.abs(po)) <= 1e-3
    ctx.close()
