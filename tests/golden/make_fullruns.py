"""Writes the expected values of the full-length superiorized runs
(tests/golden/fullrun_*.json) with the FP64 oracle.

Each workload is the seeded synthetic stand-in of one configuration (the
generators of ``synth`` build the inputs; nothing here computes any part of
the method except through ``oracle``): Algorithm 1 from x0 = box(0) for the
configuration's number of iterations, the power-law perturbation with the
stated gamma, alpha and n_red.  Stored per run: a fingerprint of the input
(sizes, sums of the values and column indices), the totals of accepted steps
and trials, the final exponent, the monitored proximity and objective after
every iteration, and the final iterate at 2048 seeded coordinates together
with its norm and sum, so that a GPU test can compare a run it makes in
seconds against an oracle run that takes minutes.

Usage: python tests/golden/make_fullruns.py [name ...]   (all runs by default;
about 20 minutes on one CPU core).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synth  # noqa: E402

CT512 = dict(N=512, nang=360, nbin=725, I0=5e3, delta=0.02, seed_phantom=201, seed_noise=202)
SUP_CT = dict(gamma=0.5, alpha=0.99, n_red=1)
SUP_RT = dict(gamma=1.0, alpha=0.99, n_red=1)


def bf16_round(v: np.ndarray) -> np.ndarray:
    """FP32 values rounded to the nearest BF16 (ties to even), as FP32: the
    values a BF16-storing solver holds (an input transformation)."""
    u = np.ascontiguousarray(v, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def fingerprint(prob, values=None) -> dict:
    A = prob.A
    val = A.val if values is None else values
    return {"m": int(A.m), "n": int(A.n), "nnz": int(A.nnz),
            "val_sum": float(np.sum(val, dtype=np.float64)),
            "col_sum": int(np.sum(A.col, dtype=np.int64))}


def objective_of(prob, kind: int) -> O.Objective:
    if kind == O.OBJ_LINEAR:
        return O.Objective(kind, c=O.mean_dose_vector(prob.body.to_scipy()))
    return O.Objective(kind, prob.shape)


def one_run(prob, mode, kind, sup, sweeps, b=0, values=None) -> dict:
    S, l, u, lo, hi = O.from_problem(prob, mode, values=values)
    l, u = O.rhs(prob.l, b), O.rhs(prob.u, b)
    P = O.Params(max_sweeps=sweeps, **sup)
    t0 = time.perf_counter()
    r = O.run(S, mode, l, u, lo, hi, objective_of(prob, kind), P)
    el = time.perf_counter() - t0
    rng = np.random.default_rng(2606)
    idx = np.sort(rng.choice(prob.A.n, size=min(2048, prob.A.n), replace=False))
    return {"rhs": b, "sweeps": r.sweeps, "accepted": int(sum(r.accepted)),
            "trials": int(sum(r.trials)), "ell": int(r.ell),
            "prox_hist": [float(v) for v in r.prox_hist],
            "obj_hist": [float(v) for v in r.obj_hist],
            "x_idx": [int(i) for i in idx], "x_val": [float(v) for v in r.x[idx]],
            "x_norm2": float(np.linalg.norm(r.x)), "x_sum": float(np.sum(r.x)),
            "oracle_seconds": el}


def ct512_cimmino_tv_f32():
    prob = synth.ct_problem(**CT512)
    return {"workload": "CT 512x512, Cimmino, isotropic TV, FP32 values", "sup": SUP_CT,
            "input": fingerprint(prob),
            "runs": [one_run(prob, O.CIMMINO, O.OBJ_TV_ISO, SUP_CT, 200)]}


def ct512_bip36_tv_f32():
    prob = synth.ct_problem(**CT512)
    prob.blocks = synth.angle_blocks(360, 725, 36)
    return {"workload": "CT 512x512, BIP with 36 interleaved angle blocks, isotropic TV, FP32",
            "sup": SUP_CT, "input": fingerprint(prob),
            "runs": [one_run(prob, O.BIP, O.OBJ_TV_ISO, SUP_CT, 200)]}


def ct512_cimmino_tv_bf16():
    prob = synth.ct_problem(**CT512)
    vals = bf16_round(prob.A.val)
    return {"workload": "CT 512x512, Cimmino, isotropic TV, BF16-rounded values",
            "sup": SUP_CT, "input": fingerprint(prob, vals),
            "runs": [one_run(prob, O.CIMMINO, O.OBJ_TV_ISO, SUP_CT, 200, values=vals)]}


def seismic_b16_atv_f32():
    prob = synth.seismic_problem(nrhs=16)
    return {"workload": "seismic 256x512, 16 noise realisations, anisotropic TV, FP32",
            "sup": SUP_CT, "input": fingerprint(prob),
            "runs": [one_run(prob, O.CIMMINO, O.OBJ_TV_ANISO, SUP_CT, 300, b=b) for b in (0, 7, 15)]}


def rt_bip3_meandose_f32():
    prob = synth.rt_problem()
    return {"workload": "radiotherapy 300000 voxels x 6003 beamlets, BIP (target, OAR1, OAR2), "
                        "mean body dose, OAR caps 20 / 30 Gy", "sup": SUP_RT,
            "input": fingerprint(prob),
            "runs": [one_run(prob, O.BIP, O.OBJ_LINEAR, SUP_RT, 500)]}


def rt_bip3_meandose_infeasible_f32():
    prob = synth.rt_problem(oar_caps=(5.0, 5.0))
    return {"workload": "radiotherapy, infeasible variant: both OAR caps 5 Gy", "sup": SUP_RT,
            "input": fingerprint(prob),
            "runs": [one_run(prob, O.BIP, O.OBJ_LINEAR, SUP_RT, 500)]}


RUNS = {f.__name__: f for f in (ct512_cimmino_tv_f32, ct512_bip36_tv_f32, ct512_cimmino_tv_bf16,
                                seismic_b16_atv_f32, rt_bip3_meandose_f32,
                                rt_bip3_meandose_infeasible_f32)}


def main(names):
    synth.build()
    for name in names or list(RUNS):
        t0 = time.perf_counter()
        out = RUNS[name]()
        out["_source"] = ("FP64 oracle (oracle/__init__.py), Algorithm 1 from box(0); written by "
                          "tests/golden/make_fullruns.py")
        with open(os.path.join(HERE, f"fullrun_{name}.json"), "w") as f:
            json.dump(out, f, separators=(",", ":"))
        print(f"{name}: {time.perf_counter() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
