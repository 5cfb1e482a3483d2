"""Full-length superiorized runs (Algorithm 1 from box(0)) at the
configurations' full sizes, in the launch configurations the benchmark
uses, against the FP64 oracle.

The oracle's runs take minutes (about a second per CT 512x512 iteration), so
their results are stored by tests/golden/make_fullruns.py, which calls only
the oracle and the input generators: the totals of accepted steps and trials,
the final exponent, the monitored proximity and objective after every
iteration, and the final iterate at 2048 seeded coordinates with its norm.
The inputs are rebuilt here by the same seeded generators; their fingerprint
(sizes, sums of the values and indices) is checked first.

Gate (the full-run bound): relative L2 <= 1e-3 on the sampled iterate and on
its norm, and <= 1e-3 on the final proximity and objective; the proximity
after every iteration within 1e-3 too.  Configurations: CT 512x512 Cimmino
and BIP with 36 angle blocks, FP32 (200 iterations); CT 512x512 Cimmino with
BF16 values against the oracle on the BF16-rounded values (200); the seismic
problem with 16 right-hand sides in one batched context, right-hand sides 0,
7 and 15 (300); the radiotherapy problem, BIP over its three structures, with
OAR caps 20 / 30 Gy and the infeasible variant with both caps at 5 Gy (500).
"""
import json
import os

import numpy as np
import pytest

import paper_2606_27086_gb300 as pk
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

GOLD = os.path.join(os.path.dirname(__file__), "golden")
CT512 = dict(N=512, nang=360, nbin=725, I0=5e3, delta=0.02, seed_phantom=201, seed_noise=202)


def _gold(name):
    return json.load(open(os.path.join(GOLD, f"fullrun_{name}.json")))


def _bf16(v):
    t = torch.from_numpy(np.ascontiguousarray(v, np.float32))
    return t.to(torch.bfloat16).to(torch.float32).numpy()


def _check_input(prob, fp, values=None):
    A = prob.A
    val = A.val if values is None else values
    assert (A.m, A.n, A.nnz) == (fp["m"], fp["n"], fp["nnz"])
    assert int(np.sum(A.col, dtype=np.int64)) == fp["col_sum"]
    vs = float(np.sum(val, dtype=np.float64))
    assert abs(vs - fp["val_sum"]) <= 1e-9 * abs(fp["val_sum"]), "generator drift"


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _compare(x, stats, prox, obj, run):
    assert stats["sweeps"] == run["sweeps"]
    idx = np.asarray(run["x_idx"])
    xo = np.asarray(run["x_val"])
    xs = np.asarray(x, np.float64)[idx]
    assert np.linalg.norm(xs - xo) <= 1e-3 * np.linalg.norm(xo)
    assert _rel(float(np.linalg.norm(np.asarray(x, np.float64))), run["x_norm2"]) <= 1e-3
    po = np.asarray(run["prox_hist"])
    assert len(prox) == len(po)
    assert _rel(prox[-1], po[-1]) <= 1e-3
    assert np.max(np.abs(np.asarray(prox) - po) / np.abs(po)) <= 1e-3
    if run["obj_hist"]:
        fo = np.asarray(run["obj_hist"])
        assert _rel(obj[-1], fo[-1]) <= 1e-3
    return stats["accepted"] - run["accepted"]


def _run(ctx, sup, sweeps):
    st = ctx.suppy_run(pk.suppy_params_default(max_sweeps=sweeps, use_graphs=1, **sup))
    return st


@pytest.mark.parametrize("name,mode,dtype", [
    ("ct512_cimmino_tv_f32", pk.SUPPY_CIMMINO, pk.SUPPY_F32),
    ("ct512_bip36_tv_f32", pk.SUPPY_BIP, pk.SUPPY_F32),
    ("ct512_cimmino_tv_bf16", pk.SUPPY_CIMMINO, pk.SUPPY_BF16)])
def test_ct512_full_run(name, mode, dtype):
    g = _gold(name)
    prob = synth.ct_problem(**CT512)
    if mode == pk.SUPPY_BIP:
        prob.blocks = synth.angle_blocks(360, 725, 36)
    _check_input(prob, g["input"], _bf16(prob.A.val) if dtype == pk.SUPPY_BF16 else None)
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ISO, mode=mode, dtype=dtype, tune=1)
    run = g["runs"][0]
    st = _run(ctx, g["sup"], run["sweeps"])[0]
    prox, obj = ctx.suppy_history()
    d_acc = _compare(ctx.suppy_get_x(), st, prox, obj, run)
    assert abs(d_acc) <= 2, d_acc
    ctx.close()


def test_seismic_batched_full_run():
    g = _gold("seismic_b16_atv_f32")
    prob = synth.seismic_problem(nrhs=16)
    _check_input(prob, g["input"])
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_TV_ANISO)
    sweeps = g["runs"][0]["sweeps"]
    st = _run(ctx, g["sup"], sweeps)
    x = ctx.suppy_get_x()
    for run in g["runs"]:
        b = run["rhs"]
        prox, obj = ctx.suppy_history(b)
        d_acc = _compare(x[:, b], st[b], prox, obj, run)
        assert abs(d_acc) <= 2, (b, d_acc)
    ctx.close()


@pytest.mark.parametrize("name,caps", [("rt_bip3_meandose_f32", (20.0, 30.0)),
                                       ("rt_bip3_meandose_infeasible_f32", (5.0, 5.0))])
def test_radiotherapy_full_run(name, caps):
    g = _gold(name)
    prob = synth.rt_problem(oar_caps=caps)
    _check_input(prob, g["input"])
    ctx = pk.from_problem(prob, obj=pk.SUPPY_OBJ_LINEAR, mode=pk.SUPPY_BIP)
    run = g["runs"][0]
    st = _run(ctx, g["sup"], run["sweeps"])[0]
    prox, obj = ctx.suppy_history()
    d_acc = _compare(ctx.suppy_get_x(), st, prox, obj, run)
    assert abs(d_acc) <= 2, d_acc
    ctx.close()
