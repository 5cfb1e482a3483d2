"""Seeded synthetic inputs for the superiorized hyperslab-projection path.

This module builds problem INSTANCES (matrices, bounds, boxes, ground truths)
and nothing else: it holds none of the projection or superiorization
arithmetic.  Both the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2606_27086_gb300``) take its arrays as input, and neither side is
imported here.

Matrices are CSR with int32 ``row_ptr``/``col`` and FP32 ``val``; rows are
constraints and columns unknowns.  Ray tracing (Siddon's method) and the
pencil-beam model live in ``synth.c`` for speed; phantoms, noise and bounds are
numpy with ``numpy.random.default_rng(seed)`` (PCG64), which gives the same
stream on every platform.

The workload families stand in for the paper's datasets, which are not
available here: LoDoPaB-CT (CT), AIR Tools II ``seismicwavetomo`` (seismic)
and CORT/matRad (radiotherapy).  Only shapes, sizes and parameters are taken
from the workload descriptions; no dataset item is reproduced.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_synth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``_synth.so`` next to it (gcc, OpenMP)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
        c_int, c_i64, c_d = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.synth_ct_count.argtypes = [c_int, c_int, c_int, i32p]
        lib.synth_ct_count.restype = c_i64
        lib.synth_ct_fill.argtypes = [c_int, c_int, c_int, i64p, i32p, f32p]
        lib.synth_ct_chord.argtypes = [c_int, c_int, c_int, c_int]
        lib.synth_ct_chord.restype = c_d
        lib.synth_segments_count.argtypes = [c_int, c_int, c_d, c_i64, f64p, i32p]
        lib.synth_segments_count.restype = c_i64
        lib.synth_segments_fill.argtypes = [c_int, c_int, c_d, c_i64, f64p, i64p, i32p, f32p]
        rt = [c_int, c_int, c_int, c_d, c_int, f64p, c_int, c_int, c_d, c_d, c_d, c_d, c_d,
              c_i64, i32p]
        lib.synth_rt_count.argtypes = rt + [i32p]
        lib.synth_rt_count.restype = c_i64
        lib.synth_rt_fill.argtypes = rt + [i64p, i32p, f32p]
        lib.synth_num_threads.restype = c_int
        _lib = lib
    return _lib


@dataclass
class CSR:
    """CSR matrix: int32 row_ptr[m+1], int32 col[nnz], float32 val[nnz]."""
    m: int
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self, dtype=np.float64):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val.astype(dtype), self.col, self.row_ptr),
                             shape=(self.m, self.n))

    def rows(self, idx: np.ndarray) -> "CSR":
        """Sub-matrix of the given rows, in the given order."""
        idx = np.asarray(idx, dtype=np.int64)
        lens = (self.row_ptr[idx + 1] - self.row_ptr[idx]).astype(np.int64)
        rp = np.zeros(len(idx) + 1, dtype=np.int64)
        np.cumsum(lens, out=rp[1:])
        sel = np.concatenate([np.arange(self.row_ptr[i], self.row_ptr[i + 1]) for i in idx]) \
            if len(idx) else np.zeros(0, dtype=np.int64)
        return CSR(len(idx), self.n, rp.astype(np.int32), self.col[sel].copy(),
                   self.val[sel].copy())


@dataclass
class Problem:
    """One instance of ``l <= A x <= u`` with box ``lo <= x <= hi``.

    ``l``/``u`` have shape (m,) or (m, B) for B right-hand sides sharing A.
    ``box_lo``/``box_hi`` have length 1 (scalar box) or n.  Image problems give
    ``shape = (H, W)`` with row-major pixel order x[i*W + j].
    """
    name: str
    A: CSR
    l: np.ndarray
    u: np.ndarray
    box_lo: np.ndarray
    box_hi: np.ndarray
    shape: tuple | None = None
    x_true: np.ndarray | None = None
    blocks: np.ndarray | None = None          # block id per row (block-iterative mode)
    c_lin: np.ndarray | None = None           # linear objective vector (radiotherapy)
    body: CSR | None = None                   # objective rows (radiotherapy body)
    meta: dict = field(default_factory=dict)


def _csr_from_counts(m: int, n: int, lens: np.ndarray, fill) -> CSR:
    rp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    nnz = int(rp[-1])
    if nnz >= 2**31:
        raise ValueError("nnz exceeds the int32 CSR range")
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float32)
    fill(rp, col, val)
    return CSR(m, n, rp.astype(np.int32), col, val)


# --------------------------------------------------------------------- CT --

def ct_matrix(N: int, nang: int, nbin: int) -> CSR:
    """Siddon intersection lengths of a parallel-beam geometry on [-1,1]^2."""
    lib = _load()
    m = nang * nbin
    lens = np.empty(m, dtype=np.int32)
    lib.synth_ct_count(N, nang, nbin, lens)
    return _csr_from_counts(m, N * N, lens,
                            lambda rp, c, v: lib.synth_ct_fill(N, nang, nbin, rp, c, v))


def ct_chord(N: int, nang: int, nbin: int, r: int) -> float:
    return float(_load().synth_ct_chord(N, nang, nbin, r))


def ellipse_phantom(N: int, seed: int, n_ell: int = 10) -> np.ndarray:
    """Random-ellipse phantom on the N x N grid over [-1,1]^2, clipped to [0,1].

    Centres uniform in the unit disc, semi-axes U[0.05,0.5], rotation U[0,pi),
    additive value U[-0.3,0.6]; evaluated at pixel centres, row i <-> y.
    """
    rng = np.random.default_rng(seed)
    h = 2.0 / N
    c = -1.0 + (np.arange(N) + 0.5) * h
    Y, X = np.meshgrid(c, c, indexing="ij")
    img = np.zeros((N, N))
    for _ in range(n_ell):
        r = np.sqrt(rng.uniform()) * 0.8
        phi = rng.uniform(0, 2 * np.pi)
        cx, cy = r * np.cos(phi), r * np.sin(phi)
        a, b = rng.uniform(0.05, 0.5, size=2)
        th = rng.uniform(0, np.pi)
        val = rng.uniform(-0.3, 0.6)
        xr = (X - cx) * np.cos(th) + (Y - cy) * np.sin(th)
        yr = -(X - cx) * np.sin(th) + (Y - cy) * np.cos(th)
        img[(xr / a) ** 2 + (yr / b) ** 2 <= 1.0] += val
    return np.clip(img, 0.0, 1.0)


def slab_bounds(b: np.ndarray, delta: float) -> tuple[np.ndarray, np.ndarray]:
    """Hyperslab bounds b(1 -/+ delta), ordered so that l <= u for either sign of b."""
    lo = b * (1.0 - delta)
    hi = b * (1.0 + delta)
    return np.minimum(lo, hi).astype(np.float32), np.maximum(lo, hi).astype(np.float32)


def ct_problem(N: int = 64, nang: int = 90, nbin: int = 91, I0: float = 1e4,
               delta: float = 0.03, seed_phantom: int = 101, seed_noise: int = 102,
               nrhs: int = 1) -> Problem:
    """Low-dose parallel-beam CT with Poisson noise and slabs b(1 -/+ delta).

    Counts ~ Poisson(I0 exp(-A x_T)), clamped to >= 1, and b = -ln(counts/I0).
    A ray that misses the image (empty row) is air-calibrated to b = 0, so its
    slab [0, 0] contains 0.  With nrhs > 1, seeds seed_noise + k give k
    independent sinograms of the same phantom (CT slices sharing a geometry).
    """
    A = ct_matrix(N, nang, nbin)
    xt = ellipse_phantom(N, seed_phantom).ravel()
    S = A.to_scipy()
    bt = S @ xt
    empty = np.diff(A.row_ptr) == 0
    ls, us = [], []
    for k in range(nrhs):
        rng = np.random.default_rng(seed_noise + k)
        counts = np.maximum(rng.poisson(I0 * np.exp(-bt)), 1)
        b = -np.log(counts / I0)
        b[empty] = 0.0
        l, u = slab_bounds(b, delta)
        ls.append(l)
        us.append(u)
    l = ls[0] if nrhs == 1 else np.stack(ls, axis=1)
    u = us[0] if nrhs == 1 else np.stack(us, axis=1)
    m = A.m
    # interleaved angle blocks for the block-iterative mode: block t = angles t, t+T, ...
    return Problem(f"ct{N}", A, l, u, np.zeros(1, np.float32), np.ones(1, np.float32),
                   shape=(N, N), x_true=xt.astype(np.float32),
                   meta=dict(nang=nang, nbin=nbin, I0=I0, delta=delta, m=m))


def angle_blocks(nang: int, nbin: int, nblocks: int) -> np.ndarray:
    """Block id per CT row: angle a belongs to block a mod nblocks."""
    a = np.arange(nang * nbin) // nbin
    return (a % nblocks).astype(np.int32)


# ---------------------------------------------------------------- seismic --

def seismic_geometry(H: int = 256, W: int = 512, h: float = 0.01, nsrc: int = 128,
                     nrec: int = 512) -> np.ndarray:
    """Source/receiver segments (km): sources evenly on the top edge, receivers
    evenly along the left, bottom and right edges (a transmission geometry)."""
    Wk, Hk = W * h, H * h
    sx = (np.arange(nsrc) + 0.5) * Wk / nsrc
    src = np.stack([sx, np.zeros(nsrc)], axis=1)
    L = 2 * Hk + Wk
    s = (np.arange(nrec) + 0.5) * L / nrec
    rec = np.empty((nrec, 2))
    left = s < Hk
    bottom = (s >= Hk) & (s < Hk + Wk)
    right = s >= Hk + Wk
    rec[left] = np.stack([np.zeros(left.sum()), s[left]], axis=1)
    rec[bottom] = np.stack([s[bottom] - Hk, np.full(bottom.sum(), Hk)], axis=1)
    rec[right] = np.stack([np.full(right.sum(), Wk), Hk - (s[right] - Hk - Wk)], axis=1)
    seg = np.empty((nsrc * nrec, 4))
    seg[:, 0:2] = np.repeat(src, nrec, axis=0)
    seg[:, 2:4] = np.tile(rec, (nsrc, 1))
    return seg


def seismic_matrix(H: int, W: int, h: float, seg: np.ndarray) -> CSR:
    lib = _load()
    seg = np.ascontiguousarray(seg, dtype=np.float64)
    m = seg.shape[0]
    lens = np.empty(m, dtype=np.int32)
    lib.synth_segments_count(W, H, h, m, seg.ravel(), lens)
    return _csr_from_counts(m, H * W, lens,
                            lambda rp, c, v: lib.synth_segments_fill(W, H, h, m, seg.ravel(),
                                                                     rp, c, v))


def slowness_model(H: int, W: int, seed: int, vmin: float = 1.5, vmax: float = 6.0,
                   n_if: int = 5, n_anom: int = 8) -> np.ndarray:
    """Slowness (s/km) on an H (depth) x W grid: smooth layers with velocity
    increasing with depth plus Gaussian anomalies of +/-15%, clipped to
    [1/vmax, 1/vmin]."""
    rng = np.random.default_rng(seed)
    z = (np.arange(H) + 0.5) / H
    xw = (np.arange(W) + 0.5) / W
    # n_if smooth interfaces: depth_k(x) = base_k + sum of a few sinusoids
    base = np.sort(rng.uniform(0.1, 0.9, size=n_if))
    iface = np.empty((n_if, W))
    for k in range(n_if):
        amp = rng.uniform(0.01, 0.06, size=3)
        fr = rng.uniform(0.5, 3.0, size=3)
        ph = rng.uniform(0, 2 * np.pi, size=3)
        iface[k] = base[k] + (amp[:, None] * np.sin(2 * np.pi * fr[:, None] * xw[None, :]
                                                    + ph[:, None])).sum(0)
    vel_layers = np.sort(rng.uniform(vmin, vmax, size=n_if + 1))
    Z = np.broadcast_to(z[:, None], (H, W))
    idx = np.zeros((H, W), dtype=np.int64)
    for k in range(n_if):
        idx += (Z > iface[k][None, :]).astype(np.int64)
    vel = vel_layers[idx]
    X = np.broadcast_to(xw[None, :], (H, W))
    for _ in range(n_anom):
        cx, cz = rng.uniform(0.1, 0.9), rng.uniform(0.1, 0.9)
        sx, sz = rng.uniform(0.03, 0.12, size=2)
        sgn = rng.choice([-1.0, 1.0])
        vel = vel * (1.0 + 0.15 * sgn * np.exp(-((X - cx) / sx) ** 2 / 2 - ((Z - cz) / sz) ** 2 / 2))
    return np.clip(1.0 / vel, 1.0 / vmax, 1.0 / vmin)


def seismic_problem(H: int = 256, W: int = 512, nsrc: int = 128, nrec: int = 512,
                    nrhs: int = 16, noise: float = 0.01, delta: float = 0.015,
                    seed_model: int = 300, seed_noise: int = 301) -> Problem:
    """Straight-ray traveltime tomography in km and s/km.

    Cells are 10 m (0.01 km); slowness is in s/km, so the box [1/6000,1/1500]
    s/m is [1/6, 1/1.5] s/km -- the same physical values in units where the
    unknowns are O(1).  Traveltimes t = A s carry 1% Gaussian noise, one
    realisation per right-hand side (seeds seed_noise + k), with slabs
    t(1 -/+ delta).
    """
    h = 0.01
    seg = seismic_geometry(H, W, h, nsrc, nrec)
    A = seismic_matrix(H, W, h, seg)
    s = slowness_model(H, W, seed_model).ravel()
    t = A.to_scipy() @ s
    ls, us = [], []
    for k in range(nrhs):
        rng = np.random.default_rng(seed_noise + k)
        tn = t * (1.0 + noise * rng.standard_normal(t.shape))
        l, u = slab_bounds(tn, delta)
        ls.append(l)
        us.append(u)
    l = ls[0] if nrhs == 1 else np.stack(ls, axis=1)
    u = us[0] if nrhs == 1 else np.stack(us, axis=1)
    return Problem(f"seismic{H}x{W}", A, l, u, np.full(1, 1 / 6.0, np.float32),
                   np.full(1, 1 / 1.5, np.float32), shape=(H, W),
                   x_true=s.astype(np.float32), meta=dict(nsrc=nsrc, nrec=nrec, nrhs=nrhs))


# ----------------------------------------------------------- radiotherapy --

def rt_structures(nx: int, ny: int, nz: int) -> dict:
    """Voxel index lists of a horseshoe target wrapped around a core organ at
    risk (OAR1) and a posterior organ at risk (OAR2) on an nx x ny x nz grid
    (voxel index (iz*ny + iy)*nx + ix).  Sizes are about 8%, 10% and 10%."""
    X = (np.arange(nx)[None, None, :] + 0.5 - nx / 2).astype(np.float64)
    Y = (np.arange(ny)[None, :, None] + 0.5 - ny / 2).astype(np.float64)
    Z = (np.arange(nz)[:, None, None] + 0.5 - nz / 2).astype(np.float64)
    X, Y, Z = np.broadcast_arrays(X, Y, Z)   # shape (nz, ny, nx)
    R = np.sqrt(X ** 2 + Y ** 2)
    ang = np.arctan2(Y, X)
    zin = np.abs(Z) < 0.4 * nz
    core = (R < 0.26 * ny) & zin
    horseshoe = (R >= 0.29 * ny) & (R < 0.39 * ny) & zin & ~(np.abs(ang - np.pi / 2) < 0.6)
    post = (Y < -0.36 * ny) & (np.abs(X) < 0.38 * nx) & ~horseshoe & ~core
    flat = lambda msk: np.flatnonzero(msk.ravel()).astype(np.int32)
    return dict(target=flat(horseshoe), oar1=flat(core), oar2=flat(post))


def rt_matrix(nx, ny, nz, vs, beams_deg, ns, nzb, ds, dz, mu, sigma, cutoff,
              voxels: np.ndarray, nbl: int) -> CSR:
    lib = _load()
    vox = np.ascontiguousarray(voxels, dtype=np.int32)
    bd = np.ascontiguousarray(beams_deg, dtype=np.float64)
    args = (nx, ny, nz, vs, len(bd), bd, ns, nzb, ds, dz, mu, sigma, cutoff, len(vox), vox)
    lens = np.empty(len(vox), dtype=np.int32)
    lib.synth_rt_count(*args, lens)
    return _csr_from_counts(len(vox), nbl, lens,
                            lambda rp, c, v: lib.synth_rt_fill(*args, rp, c, v))


def rt_problem(nx: int = 100, ny: int = 60, nz: int = 50, nbeam: int = 9, ns: int = 29,
               nzb: int = 23, oar_caps=(20.0, 30.0), target=(57.0, 64.2),
               presc: float = 60.0, sigma_vox: float = 1.85, cutoff_sigma: float = 2.35,
               mu: float = 0.004) -> Problem:
    """Pencil-beam dose-influence problem.

    Rows of ``A`` are the constrained voxels in block order (target, OAR1,
    OAR2); ``body`` holds every voxel (the mean-body-dose objective rows).  A is
    scaled so that a unit intensity vector gives a mean target dose of
    ``presc``.  Bounds: target in [57, 64.2] (0.95*60, 1.07*60), OARs below
    their caps (lower bound -inf); box x >= 0.
    """
    vs = 3.0   # mm
    st = rt_structures(nx, ny, nz)
    beams = np.arange(nbeam) * (360.0 / nbeam)
    # BEV grid covering the target with a margin
    ds = 0.9 * ny * vs / ns
    dz = 0.80 * nz * vs / nzb
    sigma = sigma_vox * vs
    cutoff = cutoff_sigma * sigma
    nbl = nbeam * ns * nzb
    geo = (nx, ny, nz, vs, beams, ns, nzb, ds, dz, mu / vs * 3.0, sigma, cutoff)
    body = rt_matrix(*geo, voxels=np.arange(nx * ny * nz, dtype=np.int32), nbl=nbl)
    rows = np.concatenate([st["target"], st["oar1"], st["oar2"]])
    A = body.rows(rows)
    nt = len(st["target"])
    dt = A.rows(np.arange(nt)).to_scipy() @ np.ones(nbl)
    scale = presc / float(dt.mean())
    body.val *= np.float32(scale)
    A.val *= np.float32(scale)
    m = A.m
    l = np.full(m, -np.inf, np.float32)
    u = np.empty(m, np.float32)
    n1, n2 = len(st["oar1"]), len(st["oar2"])
    l[:nt] = target[0]
    u[:nt] = target[1]
    u[nt:nt + n1] = oar_caps[0]
    u[nt + n1:] = oar_caps[1]
    blocks = np.concatenate([np.zeros(nt), np.ones(n1), np.full(n2, 2)]).astype(np.int32)
    return Problem("rt", A, l, u, np.zeros(1, np.float32), np.full(1, np.inf, np.float32),
                   blocks=blocks, body=body,
                   meta=dict(n_target=nt, n_oar1=n1, n_oar2=n2, n_body=body.m,
                             voxels=(nx, ny, nz), beamlets=nbl))


def rt_split_problem(presc: float = 60.0, oar2_cap: float = 30.0, **geo) -> Problem:
    """The horseshoe plan as a split-feasibility problem: the constraint table
    of the horseshoe case in the paper's radiotherapy section, with doses
    scaled from its 2 Gy prescription to ``presc``.

    Hyperslab rows (input-space sets): target voxels in [0.965, 1.135] presc
    and OAR2 voxels below ``oar2_cap``.  Dose-volume sets (target space) on the
    rows of ``meta["split"]["Aq"]``, structure 0 = target, 1 = core (OAR1):
    target D95 >= presc and D5 <= 1.085 presc, core D5 <= 0.165 presc, given as
    (kind, structure, volume, d_ref) with kind 0 = at most (upper), 1 = at
    least (lower).  ``geo`` is passed to ``rt_problem``.
    """
    base = rt_problem(presc=presc, **geo)
    nt, n1, n2 = base.meta["n_target"], base.meta["n_oar1"], base.meta["n_oar2"]
    A = base.A
    rows = np.concatenate([np.arange(nt), np.arange(nt + n1, nt + n1 + n2)])
    Ac = A.rows(rows)
    l = np.concatenate([np.full(nt, 0.965 * presc), np.full(n2, -np.inf)]).astype(np.float32)
    u = np.concatenate([np.full(nt, 1.135 * presc), np.full(n2, oar2_cap)]).astype(np.float32)
    blocks = np.concatenate([np.zeros(nt), np.ones(n2)]).astype(np.int32)
    Aq = A.rows(np.arange(nt + n1))
    dvcs = [(1, 0, 0.95, presc), (0, 0, 0.05, 1.085 * presc), (0, 1, 0.05, 0.165 * presc)]
    meta = dict(base.meta)
    meta["split"] = dict(Aq=Aq, sptr=np.array([0, nt, nt + n1], np.int32), dvcs=dvcs)
    return Problem("rt_split", Ac, l, u, base.box_lo, base.box_hi, blocks=blocks,
                   body=base.body, meta=meta)


# ------------------------------------------------------ small test shapes --

def random_csr(m: int, n: int, seed: int, mean_len: float = 20.0, max_len: int | None = None,
               empty_frac: float = 0.0, long_rows: int = 0, long_len: int = 0,
               nonneg: bool = True) -> CSR:
    """Random sparse matrix with a ragged row-length mix: geometric-ish lengths
    around ``mean_len``, a fraction of empty rows and ``long_rows`` rows of
    ``long_len`` nonzeros.  Column indices are sorted and distinct."""
    rng = np.random.default_rng(seed)
    lens = rng.poisson(mean_len, size=m).astype(np.int64)
    lens = np.maximum(lens, 1)
    if max_len is not None:
        lens = np.minimum(lens, max_len)
    if empty_frac > 0:
        lens[rng.uniform(size=m) < empty_frac] = 0
    if long_rows:
        sel = rng.choice(m, size=min(long_rows, m), replace=False)
        lens[sel] = long_len
    lens = np.minimum(lens, n)
    rp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    col = np.empty(rp[-1], dtype=np.int32)
    for i in range(m):
        col[rp[i]:rp[i + 1]] = np.sort(rng.choice(n, size=lens[i], replace=False))
    if nonneg:
        val = rng.uniform(0.05, 1.0, size=rp[-1]).astype(np.float32)
    else:
        val = rng.standard_normal(rp[-1]).astype(np.float32)
    return CSR(m, n, rp.astype(np.int32), col, val)


def random_problem(m: int, n: int, seed: int, feasible: bool = True, delta: float = 0.05,
                   nrhs: int = 1, box=(0.0, 1.0), **kw) -> Problem:
    """Random slab system: b = A x_T for x_T ~ U(box); slabs b(1 -/+ delta)
    (consistent) or with b perturbed by 20% noise first (typically inconsistent)."""
    A = random_csr(m, n, seed, **kw)
    rng = np.random.default_rng(seed + 7919)
    xt = rng.uniform(box[0], box[1], size=n)
    b = A.to_scipy() @ xt
    ls, us = [], []
    for k in range(nrhs):
        bb = b if feasible else b * (1.0 + 0.2 * rng.standard_normal(m))
        l, u = slab_bounds(bb, delta)
        ls.append(l)
        us.append(u)
    l = ls[0] if nrhs == 1 else np.stack(ls, axis=1)
    u = us[0] if nrhs == 1 else np.stack(us, axis=1)
    return Problem(f"rand{m}x{n}", A, l, u, np.full(1, box[0], np.float32),
                   np.full(1, box[1], np.float32), x_true=xt.astype(np.float32))


def line_problem(H: int, W: int, m: int, seed: int, delta: float = 0.03) -> Problem:
    """Rows along random straight segments of an H x W pixel grid (uniform
    direction, 20-80 unit steps from a random start, the pixels visited,
    weights U(0.2, 1)): ray-like rows on a grid that need not be square.
    Slabs b(1 -/+ delta) around b = A x_T perturbed by 20% noise."""
    rng = np.random.default_rng(seed)
    cols, lens = [], []
    for _ in range(m):
        th = rng.uniform(0.0, np.pi)
        r0, c0 = rng.uniform(0, H), rng.uniform(0, W)
        t = np.arange(int(rng.integers(20, 81)))
        rr = np.floor(r0 + t * np.sin(th)).astype(np.int64)
        cc = np.floor(c0 + t * np.cos(th)).astype(np.int64)
        ok = (rr >= 0) & (rr < H) & (cc >= 0) & (cc < W)
        j = np.unique(rr[ok] * W + cc[ok])
        cols.append(j)
        lens.append(len(j))
    rp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    col = np.concatenate(cols).astype(np.int32) if m else np.zeros(0, np.int32)
    val = rng.uniform(0.2, 1.0, size=len(col)).astype(np.float32)
    A = CSR(m, H * W, rp.astype(np.int32), col, val)
    xt = rng.uniform(0.0, 1.0, size=H * W)
    b = A.to_scipy() @ xt
    b = b * (1.0 + 0.2 * rng.standard_normal(m))
    l, u = slab_bounds(b, delta)
    return Problem(f"lines{H}x{W}", A, l, u, np.zeros(1, np.float32), np.ones(1, np.float32),
                   shape=(H, W), x_true=xt.astype(np.float32))


def num_threads() -> int:
    return int(_load().synth_num_threads())
