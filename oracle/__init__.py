"""FP64 CPU oracle of the superiorized hyperslab-projection method.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or
links this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) use
it.  It shares no code, header, table or helper with the CUDA library; both
take their inputs from the seeded generators in ``synth/``.

Everything here is plain numpy / scipy.sparse in float64, written to be read
against the paper (arXiv 2606.27086, "GPU-accelerated superiorization on
constrained physical problems with SupPy"):

* hyperslab projection -- Sec. 2.1.1, Eq. (2) (the halfspace projection), taken
  two-sided: P_i x = x + ((clamp(<a_i,x>, l_i, u_i) - <a_i,x>) / ||a_i||^2) a_i;
  with l_i = -inf it is Eq. (2) with b_i = u_i;
* relaxation -- Eq. (3), x + lambda (P x - x);
* simultaneous (Cimmino-type) projection -- Sec. 2.1.1, the relaxed weighted
  average x + lambda sum_i w_i (P_i x - x) with w_i > 0, sum w_i = 1;
* extrapolated Landweber (EL) and Landweber with error-minimising relaxation
  (EMR) -- appendix Table of used methods, in slab form (Q25);
* DROP (diagonally relaxed orthogonal projections) -- appendix Table of used
  methods, x <- x - Z A^T M (A x - b) with Z = diag(1/nnz(A_{:,j})), taken in
  slab form with the step of Censor et al. (Q22): x <- box(x + lambda Z sum_i
  (P_i x - x)), unit row weights;
* block-iterative projection (BIP) -- Sec. 2.1.1: the simultaneous step inside
  one block, blocks visited in order;
* box projection after each step -- Sec. 2.3.3 (BoxProjection onto x >= 0);
* weighted proximity -- Eq. (WeightedProximity), 1/2 sum_i w_i ||P_i x - x||^2;
* split feasibility -- Eq. (Split) and the CQ iteration printed after it,
  for the dose-volume constraints of Sec. 2.3.3 (and its table of the
  horseshoe plan's constraints), x <- x + gamma sum_j w_j A_j^T (P_Qj(A_j x) -
  A_j x);
* superiorization -- Algorithm 1 with the power-law step beta = gamma alpha^l
  and the normalised subgradient direction of Sec. 2.1.2, or the adaptive
  step beta = (f(x) - f_ref)/||g|| of Nikazad et al. (Sec. 2.1.2, Q29);
* stopping -- Sec. 2.2.1 (P <= P*, relative proximity change below dP* for N
  consecutive iterations, N_max) and Sec. 2.2.3 (relative objective change);
* objectives -- isotropic TV, Eq. (TV) with the subgradient of the Combettes /
  Penfold method (Sec. 2.3.1), anisotropic TV, the mean dose of Sec. 2.3.3
  (f_Mean, appendix Table of dose objectives), and the L1 / L2 perturbations
  of the seismic study (Sec. 2.3.1): ||x||_1 with subgradient sign(x), and
  ||x||_2^2 with gradient 2x (Q23).

Readings where the paper is silent or garbled (each with its number Q1..Q29):
Q1 two-sided slab; Q2 w_i = 1/m' (Cimmino) and 1/|B_t| (BIP); Q3 descent
direction v = -g/||g||; Q4 the exponent l is one counter advanced at every
trial; Q5 g recomputed after each accepted step; Q6 at most J trials per
reduction step, phase ends when none is accepted or ||g|| = 0; Q7 l <- r after
the r-th restart; Q8 proximity with the 1/2 of Eq. (WeightedProximity);
Q10 box after each sweep (Cimmino) or each block (BIP); Q11 zero rows dropped
(w_i = 0) when 0 lies in their slab; Q13/Q14 TV layout and subgradient; Q16
stopping; Q23 L2 perturbation objective f = ||x||_2^2 (the acceptance test and
the normalised direction are the same for ||x||_2); Q22 DROP in slab form: the appendix prints M = diag(w_i) with
sum w_i = 1 and no 1/||a_i||^2, which would scale the step by 1/m'; the step
taken is the one of the cited DROP method (unit weights, each row's residual
divided by ||a_i||^2, Z = diag(1/s_j) with s_j the nonzeros of column j over
the kept rows), whose fixed points are those of the Cimmino step; Q25 EL / EMR
in slab form: the residual A x - b becomes A x - clamp(A x, l, u), weights
w_i = 1/m' (D = diag(w_i/||a_i||^2), M = diag(w_i)), the step is followed by
the box and scaled by the relaxation lambda; a zero correction leaves x.
Q26 dose-volume sets: an upper DVC lets at most floor(V N) of the structure's N
voxels exceed d_ref, a lower DVC demands at least ceil(V N) at or above d_ref;
the projection keeps (upper) or raises (lower) the K highest doses, equal doses
ranked by voxel index.  Q27 split iteration: the CQ step with weights
w_j = 1/t over the t DVCs and gamma = relax / sum_j w_j ||A_j||_F^2, then the
feasibility sweep over the slabs (P_C), then the box.  Q28 with a split problem
the stopping rule and the recorded proximity use the target-space proximity
1/2 sum_j w_j ||P_Qj(A_j x) - A_j x||^2 (Sec. 2.2.1).  Q29 adaptive step
(Nikazad et al., Sec. 2.1.2): f_ref, "automatically updated", is taken as the
lowest objective value at the start of a perturbation phase so far (or a
value the caller fixes); one step per reduction, kept when f(z) <= f(y).

Parity of the whole superiorized run against printed values is unpinned: the
paper prints no iterates for this path.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

OBJ_NONE, OBJ_TV_ISO, OBJ_TV_ANISO, OBJ_LINEAR, OBJ_L1, OBJ_L2 = 0, 1, 2, 3, 4, 5
CIMMINO, BIP, DROP, EL, EMR = 0, 1, 2, 3, 4


# ------------------------------------------------------------ projections --

def hyperslab_project(a: np.ndarray, l: float, u: float, x: np.ndarray) -> np.ndarray:
    """Projection of x onto {y : l <= <a,y> <= u} (Sec. 2.1.1, Eq. (2), two-sided).

    Eq. (2) moves x along a_i by (<a,x> - b)/||a||^2 when the halfspace is
    violated; the slab is the intersection of <a,y> <= u and <-a,y> <= -l, and
    since the two halfspaces are parallel the projection moves to the nearer
    face: clamp(<a,x>, l, u) - <a,x> along a / ||a||^2.
    """
    r = float(a @ x)
    rho = float(a @ a)
    if rho == 0.0:
        return x.copy()
    return x + ((min(max(r, l), u) - r) / rho) * a


def relaxed(x: np.ndarray, px: np.ndarray, lam: float) -> np.ndarray:
    """Relaxed projection, Eq. (3): x + lambda (P x - x)."""
    return x + lam * (px - x)


def box_project(x: np.ndarray, lo, hi) -> np.ndarray:
    """Projection onto the box lo <= x <= hi (Sec. 2.3.3, BoxProjection)."""
    return np.minimum(np.maximum(x, lo), hi)


# ------------------------------------------------------------------ setup --

@dataclass
class Setup:
    """Per-matrix quantities of the simultaneous method.

    rho[i] = ||a_i||^2 (the denominator of Eq. (2)); rows with rho = 0 are
    dropped (Q11); ``w_sweep`` are the step weights of the chosen mode (Q2) and
    ``w_prox`` = 1/m' the weights of the reported proximity.
    """
    A: sp.csr_matrix
    rho: np.ndarray
    keep: np.ndarray
    w_sweep: np.ndarray
    w_prox: np.ndarray
    blocks: list = field(default_factory=list)     # list of row-index arrays (BIP)
    sub: list = field(default_factory=list)        # A restricted to each block
    z: np.ndarray | None = None                    # DROP: 1 / nonzeros per column


def setup(A: sp.csr_matrix, l: np.ndarray, u: np.ndarray, mode: int = CIMMINO,
          block_of_row: np.ndarray | None = None) -> Setup:
    A = sp.csr_matrix(A, dtype=np.float64)
    rho = np.asarray(A.multiply(A).sum(axis=1)).ravel()
    keep = rho > 0.0
    l2 = l if l.ndim == 1 else l[:, 0]
    u2 = u if u.ndim == 1 else u[:, 0]
    bad = (~keep) & ~((l2 <= 0.0) & (u2 >= 0.0))
    if np.any(bad):
        raise ValueError("a zero row whose slab excludes 0 makes the system inconsistent")
    mk = int(keep.sum())
    w_prox = np.where(keep, 1.0 / max(mk, 1), 0.0)
    S = Setup(A, rho, keep, w_prox.copy(), w_prox)
    if mode == DROP:
        # Q22: unit row weights, column scaling 1/s_j over the kept rows
        S.w_sweep = keep.astype(np.float64)
        s = np.asarray((A[keep] != 0).sum(axis=0)).ravel().astype(np.float64)
        S.z = np.where(s > 0, 1.0 / np.maximum(s, 1.0), 0.0)
    if mode == BIP:
        if block_of_row is None:
            raise ValueError("block-iterative mode needs a block id per row")
        nb = int(block_of_row.max()) + 1
        w = np.zeros(A.shape[0])
        for t in range(nb):
            rows = np.flatnonzero(block_of_row == t)
            kt = int(keep[rows].sum())
            w[rows] = np.where(keep[rows], 1.0 / max(kt, 1), 0.0)
            S.blocks.append(rows)
            S.sub.append(A[rows])
        S.w_sweep = w
    return S


# -------------------------------------------------------------- proximity --

def proximity(S: Setup, l: np.ndarray, u: np.ndarray, x: np.ndarray,
              w: np.ndarray | None = None) -> float:
    """Eq. (WeightedProximity): 1/2 sum_i w_i ||P_i x - x||^2.

    ||P_i x - x|| = |clamp(r_i, l_i, u_i) - r_i| / ||a_i|| with r = A x.
    """
    w = S.w_prox if w is None else w
    r = S.A @ x
    d = np.clip(r, l, u) - r
    ok = S.keep
    return 0.5 * float(np.sum(w[ok] * d[ok] ** 2 / S.rho[ok]))


# ------------------------------------------------------------------ sweeps --

def simultaneous_step(A: sp.csr_matrix, rho: np.ndarray, keep: np.ndarray, w: np.ndarray,
                      wp: np.ndarray, l: np.ndarray, u: np.ndarray, lam: float, lo, hi,
                      x: np.ndarray) -> tuple[np.ndarray, float]:
    """One relaxed simultaneous projection step followed by the box (Eq. (3),
    Sec. 2.1.1, Sec. 2.3.3):  x <- box(x + lambda sum_i w_i (P_i x - x)).

    Returns the new point and 1/2 sum_i wp_i d_i^2 / rho_i evaluated at the
    step's input point (its proximity contribution with weights wp)."""
    r = A @ x
    d = np.clip(r, l, u) - r
    coef = np.zeros_like(r)
    coef[keep] = lam * w[keep] * d[keep] / rho[keep]
    p_in = 0.5 * float(np.sum(wp[keep] * d[keep] ** 2 / rho[keep]))
    return box_project(x + A.T @ coef, lo, hi), p_in


def drop_step(S: Setup, l: np.ndarray, u: np.ndarray, lam: float, lo, hi,
              x: np.ndarray) -> tuple[np.ndarray, float]:
    """One DROP step in slab form (appendix Table of used methods; Q22):
    x <- box(x + lambda Z sum_i (P_i x - x)), Z = diag(1/s_j).  Returns the new
    point and the proximity (weights 1/m') of the step's input point."""
    r = S.A @ x
    d = np.clip(r, l, u) - r
    k = S.keep
    coef = np.zeros_like(r)
    coef[k] = d[k] / S.rho[k]
    p_in = 0.5 * float(np.sum(S.w_prox[k] * d[k] ** 2 / S.rho[k]))
    return box_project(x + lam * S.z * (S.A.T @ coef), lo, hi), p_in


def el_step(S: Setup, l: np.ndarray, u: np.ndarray, lam: float, lo, hi,
            x: np.ndarray) -> tuple[np.ndarray, float]:
    """Extrapolated Landweber (appendix Table of used methods; Q25):
    x <- box(x - lambda t A^T D r), r = A x - clamp(A x, l, u),
    D = diag(w_i/||a_i||^2), t = r^T D r / ||A^T D r||^2."""
    r = S.A @ x
    res = r - np.clip(r, l, u)
    k = S.keep
    Dr = np.zeros_like(r)
    Dr[k] = S.w_prox[k] * res[k] / S.rho[k]
    g = S.A.T @ Dr
    p_in = 0.5 * float(np.sum(S.w_prox[k] * res[k] ** 2 / S.rho[k]))
    gg = float(g @ g)
    if gg == 0.0:
        return box_project(x, lo, hi), p_in
    t = float(res @ Dr) / gg
    return box_project(x - lam * t * g, lo, hi), p_in


def emr_step(S: Setup, l: np.ndarray, u: np.ndarray, lam: float, lo, hi,
             x: np.ndarray) -> tuple[np.ndarray, float]:
    """Landweber with error-minimising relaxation (appendix Table of used
    methods; Q25): x <- box(x - lambda t A^T M r), M = diag(w_i),
    t = ||A^T M r||^2 / ||M^(1/2) A A^T M r||^2."""
    r = S.A @ x
    res = r - np.clip(r, l, u)
    k = S.keep
    Mr = np.zeros_like(r)
    Mr[k] = S.w_prox[k] * res[k]
    g = S.A.T @ Mr
    p_in = 0.5 * float(np.sum(S.w_prox[k] * res[k] ** 2 / S.rho[k]))
    q = S.A @ g
    den = float(np.sum(S.w_prox[k] * q[k] ** 2))
    if den == 0.0:
        return box_project(x, lo, hi), p_in
    t = float(g @ g) / den
    return box_project(x - lam * t * g, lo, hi), p_in


def sweep(S: Setup, mode: int, l: np.ndarray, u: np.ndarray, lam: float, lo, hi,
          x: np.ndarray) -> tuple[np.ndarray, float]:
    """One application of the feasibility-seeking operator T.

    Cimmino: one simultaneous step over all rows (w_i = 1/m').
    BIP: one simultaneous step per block in block order, w_i = 1/|B_t|, box
    after each block (Q10).  The returned monitor value is the sum over blocks
    of each block's proximity terms (weights 1/m') at that block's input point;
    for Cimmino it is the proximity of the sweep's input point.
    """
    if mode == CIMMINO:
        return simultaneous_step(S.A, S.rho, S.keep, S.w_sweep, S.w_prox, l, u, lam, lo, hi, x)
    if mode == DROP:
        return drop_step(S, l, u, lam, lo, hi, x)
    if mode == EL:
        return el_step(S, l, u, lam, lo, hi, x)
    if mode == EMR:
        return emr_step(S, l, u, lam, lo, hi, x)
    p_tot = 0.0
    for rows, At in zip(S.blocks, S.sub):
        x, p = simultaneous_step(At, S.rho[rows], S.keep[rows], S.w_sweep[rows],
                                 S.w_prox[rows], l[rows], u[rows], lam, lo, hi, x)
        p_tot += p
    return x, p_tot


# ------------------------------------------------- split feasibility (DVC) --

DVC_UPPER, DVC_LOWER = 0, 1


@dataclass
class DVC:
    """One dose-volume constraint on a structure (Sec. 2.3.3, radiotherapy):
    DVC_UPPER is D_V <= d_ref (not more than the fraction V of the structure's
    voxels above d_ref), DVC_LOWER is D_V >= d_ref (at least the fraction V at
    or above d_ref).  ``structure`` indexes the row ranges of the split
    matrix."""
    kind: int
    structure: int
    volume: float
    d_ref: float


def dvc_count(kind: int, volume: float, N: int) -> int:
    """Q26: the voxel count a DVC allows (upper: floor(V N) voxels may exceed
    d_ref) or demands (lower: ceil(V N) voxels must reach d_ref); V N is one
    double multiplication."""
    v = float(volume) * float(N)
    return int(np.floor(v)) if kind == DVC_UPPER else int(np.ceil(v))


def dvc_project(d: np.ndarray, kind: int, volume: float, d_ref: float) -> np.ndarray:
    """Euclidean projection of one structure's dose vector onto its DVC set
    (Q26).

    Upper: the set is the union, over voxel subsets S with |S| = K, of
    {p : p_i <= d_ref for i not in S}; the nearest point leaves the K highest
    doses as they are and lowers every other dose above d_ref to d_ref.
    Lower: the union over |S| = K of {p : p_i >= d_ref for i in S}; the nearest
    point raises those of the K highest doses that are below d_ref to d_ref.
    Equal doses are ranked by the lower voxel index first.
    """
    d = np.asarray(d, np.float64)
    N = len(d)
    K = min(max(dvc_count(kind, volume, N), 0), N)
    order = np.lexsort((np.arange(N), -d))      # descending dose, then index
    top = np.zeros(N, dtype=bool)
    top[order[:K]] = True
    p = d.copy()
    if kind == DVC_UPPER:
        sel = (~top) & (d > d_ref)
    else:
        sel = top & (d < d_ref)
    p[sel] = d_ref
    return p


@dataclass
class SplitSetup:
    """The target-space part of a split-feasibility problem (Eq. (Split)):
    rows of ``Aq`` (dose rows of the DVC structures) grouped by structure,
    ``sptr[s]:sptr[s+1]`` the rows of structure s; weights w_j = 1/t over the t
    DVCs and the CQ step gamma = relax / L*, L* = sum_j w_j ||A_j||_F^2 (Q27)."""
    Aq: sp.csr_matrix
    sptr: np.ndarray
    dvcs: list
    w: np.ndarray
    gamma: float


def split_setup(Aq: sp.csr_matrix, sptr, dvcs: list, relax: float = 1.0) -> SplitSetup:
    Aq = sp.csr_matrix(Aq, dtype=np.float64)
    sptr = np.asarray(sptr, np.int64)
    t = len(dvcs)
    w = np.full(t, 1.0 / t) if t else np.zeros(0)
    rows2 = np.asarray(Aq.multiply(Aq).sum(axis=1)).ravel()
    L = 0.0
    for j, q in enumerate(dvcs):
        L += w[j] * float(np.sum(rows2[sptr[q.structure]:sptr[q.structure + 1]]))
    return SplitSetup(Aq, sptr, list(dvcs), w, relax / L if L > 0 else 0.0)


def dvc_corrections(SS: SplitSetup, d: np.ndarray) -> tuple[np.ndarray, float]:
    """Given the doses d = Aq x: c = sum_j w_j (P_Qj(d_j) - d_j) (placed on the
    rows of each DVC's structure) and the target-space proximity
    1/2 sum_j w_j ||P_Qj(d_j) - d_j||^2 (Eq. (WeightedProximity) over the Q_j;
    Q28)."""
    d = np.asarray(d, np.float64)
    c = np.zeros_like(d)
    prox = 0.0
    for j, q in enumerate(SS.dvcs):
        r0, r1 = int(SS.sptr[q.structure]), int(SS.sptr[q.structure + 1])
        dj = d[r0:r1]
        e = dvc_project(dj, q.kind, q.volume, q.d_ref) - dj
        c[r0:r1] += SS.w[j] * e
        prox += 0.5 * SS.w[j] * float(e @ e)
    return c, prox


def dvc_proximity(SS: SplitSetup, x: np.ndarray) -> float:
    return dvc_corrections(SS, SS.Aq @ x)[1]


def cq_step(SS: SplitSetup, x: np.ndarray) -> tuple[np.ndarray, float]:
    """The CQ step of Sec. 2.1.1 (after Eq. (Split)) for the several sets Q_j:
    x <- x + gamma sum_j w_j A_j^T (P_Qj(A_j x) - A_j x).  P_C is applied by
    the feasibility sweep that follows (Q27).  Returns the new point and the
    target-space proximity of the input point."""
    c, prox = dvc_corrections(SS, SS.Aq @ x)
    return x + SS.gamma * (SS.Aq.T @ c), prox


# -------------------------------------------------------------- objectives --

def tv_iso(x: np.ndarray, H: int, W: int) -> float:
    """Eq. (TV): sum_{i<H-1, j<W-1} sqrt((X[i+1,j]-X[i,j])^2 + (X[i,j+1]-X[i,j])^2),
    row-major X[i,j] = x[i*W + j] (Q13)."""
    X = x.reshape(H, W)
    dx = X[1:, :-1] - X[:-1, :-1]
    dy = X[:-1, 1:] - X[:-1, :-1]
    return float(np.sum(np.sqrt(dx * dx + dy * dy)))


def tv_iso_subgrad(x: np.ndarray, H: int, W: int) -> np.ndarray:
    """A subgradient of Eq. (TV) (Combettes / Penfold, Sec. 2.3.1; Q13).

    Term phi_ij = sqrt(dx^2 + dy^2) with dx = X[i+1,j]-X[i,j], dy = X[i,j+1]-X[i,j]
    has partial derivatives -(dx+dy)/phi at (i,j), dx/phi at (i+1,j) and dy/phi
    at (i,j+1); a term with phi = 0 contributes the zero subgradient element.
    """
    X = x.reshape(H, W)
    dx = X[1:, :-1] - X[:-1, :-1]
    dy = X[:-1, 1:] - X[:-1, :-1]
    phi = np.sqrt(dx * dx + dy * dy)
    nz = phi > 0.0
    inv = np.zeros_like(phi)
    inv[nz] = 1.0 / phi[nz]
    G = np.zeros((H, W))
    G[:-1, :-1] -= (dx + dy) * inv
    G[1:, :-1] += dx * inv
    G[:-1, 1:] += dy * inv
    return G.ravel()


def tv_aniso(x: np.ndarray, H: int, W: int) -> float:
    """Anisotropic TV (Q14): sum |X[i+1,j]-X[i,j]| + sum |X[i,j+1]-X[i,j]| over all
    valid index pairs."""
    X = x.reshape(H, W)
    return float(np.sum(np.abs(X[1:, :] - X[:-1, :])) + np.sum(np.abs(X[:, 1:] - X[:, :-1])))


def tv_aniso_subgrad(x: np.ndarray, H: int, W: int) -> np.ndarray:
    """Subgradient of the anisotropic TV with sign(0) = 0 (Q14)."""
    X = x.reshape(H, W)
    sv = np.sign(X[1:, :] - X[:-1, :])
    sh = np.sign(X[:, 1:] - X[:, :-1])
    G = np.zeros((H, W))
    G[1:, :] += sv
    G[:-1, :] -= sv
    G[:, 1:] += sh
    G[:, :-1] -= sh
    return G.ravel()


def mean_dose_vector(body: sp.csr_matrix) -> np.ndarray:
    """f_Mean(d) = (1/N_S) sum_{i in S} d_i with d = A_S x (Sec. 2.3.3) is linear
    in x: f = c.x with c = A_S^T 1 / N_S."""
    body = sp.csr_matrix(body, dtype=np.float64)
    return np.asarray(body.sum(axis=0)).ravel() / body.shape[0]


class Objective:
    """f and a subgradient g_f for the objectives of the three applications."""

    def __init__(self, kind: int, shape=None, c: np.ndarray | None = None):
        self.kind = kind
        self.shape = shape
        self.c = None if c is None else np.asarray(c, dtype=np.float64)

    def f(self, x: np.ndarray) -> float:
        if self.kind == OBJ_TV_ISO:
            return tv_iso(x, *self.shape)
        if self.kind == OBJ_TV_ANISO:
            return tv_aniso(x, *self.shape)
        if self.kind == OBJ_LINEAR:
            return float(self.c @ x)
        if self.kind == OBJ_L1:
            return float(np.sum(np.abs(x)))
        if self.kind == OBJ_L2:
            return float(x @ x)
        return 0.0

    def g(self, x: np.ndarray) -> np.ndarray:
        if self.kind == OBJ_TV_ISO:
            return tv_iso_subgrad(x, *self.shape)
        if self.kind == OBJ_TV_ANISO:
            return tv_aniso_subgrad(x, *self.shape)
        if self.kind == OBJ_LINEAR:
            return self.c.copy()
        if self.kind == OBJ_L1:
            return np.sign(x)
        if self.kind == OBJ_L2:
            return 2.0 * x
        return np.zeros_like(x)


# --------------------------------------------------------- superiorization --

@dataclass
class Params:
    """Parameters of Algorithm 1 and of the stopping rule (Sec. 2.2.1, 2.2.3).

    Defaults of the stopping thresholds are the paper's: P* = 1e-6,
    dP* = 1e-8, N = 5, N_max = 500, df* = 1e-6.
    """
    lam: float = 1.0
    gamma: float = 0.5
    alpha: float = 0.99
    n_red: int = 1
    max_trials: int = 100
    restart_every: int = 0
    max_sweeps: int = 500
    prox_abs: float = 1e-6
    prox_rel: float = 1e-8
    patience: int = 5
    obj_rel: float = 1e-6
    use_stopping: bool = False      # False: run exactly max_sweeps sweeps
    variance_tol: float = 0.0       # > 0: the variance stopping rule (Sec. 2.3.2, CT study)
    adaptive: int = 0               # 1: adaptive step, f_ref automatic (Q29); 2: f_ref fixed
    f_ref: float = 0.0              # the reference value when adaptive == 2


@dataclass
class PertState:
    ell: int = 0
    restarts: int = 0
    last_restart_k: int = 0
    f_best: float | None = None     # adaptive step: lowest objective at a phase start


def adaptive_phase(obj: Objective, y: np.ndarray, st: PertState, P: Params) -> tuple:
    """The perturbation phase with the adaptive step of Nikazad et al.
    (Sec. 2.1.2): beta = (f(y) - f_ref)/||g|| when f(y) > f_ref, else no step,
    i.e. the subgradient projection of y onto the level set {f <= f_ref} of
    the linearisation of f at y.  Reading Q29: f_ref is the lowest objective
    value seen at the start of a perturbation phase so far, this phase's
    included (adaptive = 1), or a fixed value (adaptive = 2); each of the n_red
    reduction steps takes this one step and keeps it when f(z) <= f(y)
    (Algorithm 1's test), else the phase ends; l is not used."""
    f0 = obj.f(y)
    if P.adaptive == 2:
        f_ref = P.f_ref
    else:
        st.f_best = f0 if st.f_best is None else min(st.f_best, f0)
        f_ref = st.f_best
    n = trials = 0
    while n < P.n_red:
        g = obj.g(y)
        gn = float(np.sqrt(g @ g))
        fy = obj.f(y)
        if gn == 0.0 or fy <= f_ref:
            break
        beta = (fy - f_ref) / gn
        z = y - beta * g / gn
        trials += 1
        if obj.f(z) <= fy:
            y = z
            n += 1
        else:
            break
    return y, n, trials


def perturbation_phase(obj: Objective, y: np.ndarray, st: PertState, P: Params) -> tuple:
    """The perturbation phase of Algorithm 1 (nonascending power-law steps).

    While fewer than n_red steps are accepted: g = g_f(y); stop if ||g|| = 0;
    v = -g/||g|| (Q3); trial j: beta = gamma alpha^l, l += 1 (Q4),
    z = y + beta v, accept when f(z) <= f(y) (Algorithm 1); after max_trials
    rejected trials the phase ends (Q6).  Returns (y, accepted, trials).
    """
    if P.adaptive:
        return adaptive_phase(obj, y, st, P)
    n = 0
    trials = 0
    while n < P.n_red:
        g = obj.g(y)
        gn = float(np.sqrt(g @ g))
        if gn == 0.0:
            break
        v = -g / gn
        fy = obj.f(y)
        ok = False
        for _ in range(P.max_trials):
            beta = P.gamma * P.alpha ** st.ell
            st.ell += 1
            trials += 1
            z = y + beta * v
            if obj.f(z) <= fy:
                y = z
                n += 1
                ok = True
                break
        if not ok:
            break
    return y, n, trials


def maybe_restart(st: PertState, k: int, P: Params) -> None:
    """Restarts (Sec. 2.1.2): at the start of iteration k, when k is a positive
    multiple of restart_every, l <- r after the r-th restart (Q7)."""
    if P.restart_every > 0 and k > 0 and k % P.restart_every == 0 and st.last_restart_k != k:
        st.restarts += 1
        st.ell = st.restarts
        st.last_restart_k = k


@dataclass
class StopState:
    p_prev: float | None = None
    f_prev: float | None = None
    calm: int = 0


def stop_check(ss: StopState, p: float, f: float | None, P: Params) -> bool:
    """Stopping rule of Sec. 2.2.1 / 2.2.3 evaluated after a sweep.

    Feasibility part: p <= P*, or |p - p_prev| / max(1, p_prev) < dP* for N
    consecutive sweeps.  Objective part (when an objective is present and
    obj_rel > 0): |f - f_prev| / max(1, |f_prev|) < df*.  Both parts must hold.
    """
    if ss.p_prev is not None and abs(p - ss.p_prev) / max(1.0, ss.p_prev) < P.prox_rel:
        ss.calm += 1
    else:
        ss.calm = 0
    feas = (p <= P.prox_abs) or (ss.calm >= P.patience)
    objok = True
    if f is not None and P.obj_rel > 0:
        objok = ss.f_prev is not None and abs(f - ss.f_prev) / max(1.0, abs(ss.f_prev)) < P.obj_rel
    ss.p_prev = p
    if f is not None:
        ss.f_prev = f
    return feas and objok


@dataclass
class RunResult:
    x: np.ndarray
    sweeps: int
    prox_hist: list
    obj_hist: list
    accepted: list
    trials: list
    ell: int


def variance_of_changes(omega: list) -> float:
    """Variance stopping measure of the CT study (Sec. 2.3.2): the sample
    variance 1/(k-1) sum_i (omega_i - mean)^2 of the relative changes
    omega_i = ||x^i - x^(i-1)|| / ||x^i|| of all iterates so far."""
    w = np.asarray(omega, np.float64)
    return float(np.sum((w - w.mean()) ** 2) / (len(w) - 1))


def run(S: Setup, mode: int, l, u, lo, hi, obj: Objective, P: Params,
        x0: np.ndarray | None = None, n_sweeps: int | None = None,
        split: SplitSetup | None = None) -> RunResult:
    """Algorithm 1: perturbation phase, then one application of T, repeated.

    With ``split`` (a split-feasibility problem, Eq. (Split)) each iteration
    runs the CQ step over the dose-volume sets before T (Q27), and the monitored
    proximity is the target-space one at the CQ step's input point (Q28).

    x0 defaults to box(0) (Q18).  With ``use_stopping`` False the run is exactly
    ``max_sweeps`` sweeps; otherwise it ends at the first sweep after which
    ``stop_check`` holds.  The objective value recorded for iteration k is
    f(x^k) at the start of its perturbation phase.
    """
    n = S.A.shape[1]
    x = box_project(np.zeros(n) if x0 is None else np.asarray(x0, np.float64), lo, hi)
    st = PertState()
    ss = StopState()
    ph, oh, acc, tri = [], [], [], []
    omega = []
    K = P.max_sweeps if n_sweeps is None else n_sweeps
    k = 0
    while k < K:
        x_prev = x
        f_k = None
        if obj.kind != OBJ_NONE:
            maybe_restart(st, k, P)
            f_k = obj.f(x)
            x, a, t = perturbation_phase(obj, x, st, P)
            acc.append(a)
            tri.append(t)
            oh.append(f_k)
        if split is not None:
            x, p_target = cq_step(split, x)
        x, p = sweep(S, mode, l, u, P.lam, lo, hi, x)
        if split is not None:
            p = p_target
        ph.append(p)
        k += 1
        if P.use_stopping and stop_check(ss, p, f_k, P):
            break
        if P.variance_tol > 0:
            nx = float(np.linalg.norm(x))
            omega.append(float(np.linalg.norm(x - x_prev)) / nx if nx > 0 else 0.0)
            if len(omega) >= 2 and variance_of_changes(omega) < P.variance_tol:
                break
    return RunResult(x, k, ph, oh, acc, tri, st.ell)


# -------------------------------------------------------- convenience glue --

def from_problem(prob, mode: int = CIMMINO, values: np.ndarray | None = None):
    """Build (Setup, l, u, lo, hi) from a ``synth.Problem`` for right-hand side 0,
    optionally replacing the matrix values (e.g. by their BF16-rounded copy)."""
    A = prob.A
    val = A.val if values is None else values
    M = sp.csr_matrix((np.asarray(val, np.float64), A.col, A.row_ptr), shape=(A.m, A.n))
    l = np.asarray(prob.l, np.float64)
    u = np.asarray(prob.u, np.float64)
    S = setup(M, l, u, mode, prob.blocks)
    lo = np.asarray(prob.box_lo, np.float64)
    hi = np.asarray(prob.box_hi, np.float64)
    lo = lo[0] if lo.size == 1 else lo
    hi = hi[0] if hi.size == 1 else hi
    return S, l, u, lo, hi


def rhs(a: np.ndarray, b: int) -> np.ndarray:
    return np.asarray(a if a.ndim == 1 else a[:, b], np.float64)
