"""Shared helpers of the GPU parity tests: build a CUDA context and the FP64
oracle setup from the same seeded ``synth`` problem, and compare results."""
from __future__ import annotations

import numpy as np

import oracle as O
import synth

OBJ_OF = {"none": O.OBJ_NONE, "tv": O.OBJ_TV_ISO, "atv": O.OBJ_TV_ANISO, "lin": O.OBJ_LINEAR,
          "l1": O.OBJ_L1, "l2": O.OBJ_L2}


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def rel(a: float, b: float) -> float:
    return abs(a - b) / max(abs(b), 1e-300)


def rounded_values(val: np.ndarray, dtype: str) -> np.ndarray:
    """FP32 values rounded to nearest even in BF16 / FP16 (what the device stores)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(val, np.float32))
    if dtype == "bf16":
        return t.to(torch.bfloat16).to(torch.float32).numpy()
    if dtype == "f16":
        return t.to(torch.float16).to(torch.float32).numpy()
    return np.asarray(val, np.float32)


def oracle_objective(prob, kind: int) -> O.Objective:
    if kind == O.OBJ_LINEAR:
        c = O.mean_dose_vector(prob.body.to_scipy()) if prob.body is not None else prob.c_lin
        return O.Objective(kind, c=c)
    if kind in (O.OBJ_L1, O.OBJ_L2):
        return O.Objective(kind)
    return O.Objective(kind, prob.shape)


def random_x(n: int, nrhs: int, seed: int, lo=0.0, hi=1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    shape = (n,) if nrhs == 1 else (n, nrhs)
    return rng.uniform(lo, hi, size=shape).astype(np.float32)


def small_ct(N=64, nang=90, nbin=91, **kw):
    return synth.ct_problem(N, nang, nbin, **kw)
