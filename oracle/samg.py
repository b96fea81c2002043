"""FP64 CPU oracle of the self-learning AMG method for extremal singular
triplets and eigenpairs (H. De Sterck, arXiv:1102.0919).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this module.  It shares no code
with the GPU library and never imports it.

The oracle is a plain restatement of the paper: every step runs in the
paper's order with scipy/numpy primitives (sparse and dense products, dense
QR/SVD/eigh) and the sequential loops of ``oracle.c``.  Where the paper is
silent the readings below are used (numbers as in the design notes):

* R1/R2  minimal relaxation: block Gauss-Seidel, first Kaczmarz over the rows
  of A for v (Eq. genSVDresid1), then over the rows of A^t for u
  (Eq. genSVDresid2); SPD kind: one Kaczmarz sweep over the rows of A-lam*B.
* R3  sweeps in natural row order of the stored matrix.  params["relax_order"]
  = "coloured" selects a variant (not the paper's) for the solve phase's
  relaxations only: rows greedily coloured in natural order (rows of one
  colour share no column) and swept colour by colour, natural order inside a
  colour; the setup phase keeps the natural order.
* R4  V(mu_b, mu_b) cycles in the additive phase.
* R5  random test vectors from SplitMix64 (see oracle.c).
* R6  coarsest level: max(m_l, n_l) <= coarsest_max, or the coarsening keeps
  more than 90% of the points, or min(m_c, n_c) < 2 n_b, or max_levels.
* R7  coarsest additive solve: SVD pseudo-inverse of X - sigma_j Y with the
  single smallest singular value left out (params["coarse_drop"] > 1 leaves
  out more: a variant, not the paper's).  params["coarse_pinv"] = "geneig"
  selects a variant (not the paper's): with the generalized eigenpairs
  X w_k = lam_k Y w_k, W^t Y W = I, z = sum over k != k* of
  w_k (w_k^t r) / (lam_k - sigma_j), k* the lam_k nearest sigma_j (lowest
  k on ties); it equals the paper's form when Y = I.
* R8  strength sums run over all columns including the diagonal.
* R9  Ruge-Stueben ties go to the lowest index.
* R10 coarse points are numbered in increasing fine index.
* R11 residual rho_j = sqrt(|A v - s u|^2 + |A^t u - s v|^2) / s for unit
  u, v; SPD kind |A x - lam x| / |lam|.
* R13 LS weights |RQ| (dominant) or 1/|RQ| (minimal) multiply the squared
  residuals; |RQ| is floored at 1e-300.
* R14 minimal kind: the F-point values are first replaced by one weighted
  Jacobi step on N x = 0 (N = A A^t, A^t A, or A) with weight
  omega_J * 2 / g, g the Gershgorin bound of D^-1 N (g = 2, weight omega_J,
  for 5-point operators).
* R15 C^i is capped to the n_f - 1 strongest members (ties: lowest index).
* R16 minimal kind: test vectors are scaled to unit B (C) norm after each
  block of mu_t relaxations.
* R21 minimal SVD kind with m >= n: the paper's A A^t-based coarsening of the
  row variables cannot represent the minimal left singular vectors of the
  gradient operator (F edges lack same-orientation C neighbours), and
  Kaczmarz on A^t u = 0 drives row test vectors into null(A^t), the |m-n|
  spurious zero modes of Thm genSVD.  The rows are therefore coarsened
  "directly from A" (the option Sec. 3.7 leaves open): P_0 = A Q_0, whose
  range A range(Q_0) holds u = A v / s for v in range(Q_0); below the
  finest level A_l = B_l is symmetric, so Sec. 5.2's specialization applies
  (coarsening on A_l, P_l = Q_l).  Row test vectors are A v_t (finest) or
  v_t (coarser); the coarse boot u is v_b[C] / s (finest) or u_b[C].  The
  Ritz step takes the left basis A V_b (Rayleigh-Ritz for A^t A on span V_b):
  components of u in null(A^t) -- left there by rounding -- are invisible to
  every relaxation and correction and to the two-sided projection, and would
  otherwise stall the residual at the rounding level of the cycle.
* R23 square SVD kind (Sec. 5.1): params["square_form"] = "from_A" takes the
  C/F splitting and the sparsity patterns of both P and Q from the strength
  graph of A itself (Eq. strength on N = A), as in the paper's square
  nonsymmetric example (Sec. 6.1), so every level stays square; P is fitted
  to the u vectors and Q to the v vectors.  "shared" fits one operator to
  both sets (weights repeated) and takes Q = P, so that B_c = C_c.  The
  Ritz step is two-sided.  The default "normal" keeps Sec. 3.7 (or R21).
* R22 redo-P (Sec. 6.3): a triplet counts as converged once rho_j <=
  redo_tol; each time that count grows (some still above), one downward
  sweep of the multiplicative phase runs on copies of the boot triplets with
  the LS weights of the test vectors and of the converged boot vectors
  divided by 1000, replacing P, Q and the coarse operators.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import build as _build

_LIB = None

DEFAULTS = dict(n_t=8, theta=0.06, mu_t=8, mu_b=4, mu_tJ=1, mu_bJ=1, omega_J=0.7,
                n_mult=10, coarsest_max=100, max_levels=30, seed=20110204, coarse_drop=1,
                coarse_pinv="svd", row_form="induced", relax_order="natural",
                square_form="normal")


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.oracle_random_block.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, P]
        L.oracle_random_block.restype = None
        L.oracle_kaczmarz_sweep.argtypes = [ctypes.c_int64, ctypes.c_int32, P, P, P, P, P, P,
                                            P, P, P]
        L.oracle_kaczmarz_sweep.restype = None
        L.oracle_rs_coarsen.argtypes = [ctypes.c_int32, P, P, P]
        L.oracle_rs_coarsen.restype = ctypes.c_int
        L.oracle_ls_fit.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, P]
        L.oracle_ls_fit.restype = ctypes.c_int64
        L.oracle_row_colours.argtypes = [ctypes.c_int64, ctypes.c_int32, P, P, P]
        L.oracle_row_colours.restype = ctypes.c_int32
        _LIB = L
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _csr(a) -> sp.csr_matrix:
    """Canonical CSR: sorted column indices, int64 pointers, int32 columns."""
    a = sp.csr_matrix(a)
    a.sort_indices()
    return sp.csr_matrix((np.ascontiguousarray(a.data, dtype=np.float64),
                          np.ascontiguousarray(a.indices, dtype=np.int32),
                          np.ascontiguousarray(a.indptr, dtype=np.int64)), shape=a.shape)


def _arrs(a: sp.csr_matrix):
    return (np.ascontiguousarray(a.indptr, dtype=np.int64),
            np.ascontiguousarray(a.indices, dtype=np.int32),
            np.ascontiguousarray(a.data, dtype=np.float64))


# --------------------------------------------------------------------------
# primitives
# --------------------------------------------------------------------------

def random_block(seed: int, nrows: int, nvec: int) -> np.ndarray:
    """Random test vectors in [-1, 1) (R5, SplitMix64 counter generator)."""
    out = np.empty((nrows, nvec), dtype=np.float64)
    _lib().oracle_random_block(ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), nrows, nvec, _ptr(out))
    return out


def kaczmarz_sweep(R: sp.csr_matrix, X: np.ndarray, rhs: np.ndarray,
                   B: sp.csr_matrix | None = None, shift: np.ndarray | None = None) -> None:
    """One Kaczmarz sweep in natural row order over the rows of R - shift_j B
    (Sec. 5.3), in place on X (ncols x nb); rhs is nrows x nb."""
    assert X.flags.c_contiguous and X.dtype == np.float64
    nb = X.shape[1]
    rp, rc, rv = _arrs(R)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    if B is not None:
        bp, bc, bv = _arrs(B)
        sh = np.ascontiguousarray(shift, dtype=np.float64)
    else:
        bp = bc = bv = sh = None
    _lib().oracle_kaczmarz_sweep(R.shape[0], nb, _ptr(rp), _ptr(rc), _ptr(rv), _ptr(bp),
                                 _ptr(bc), _ptr(bv), _ptr(sh), _ptr(rhs), _ptr(X))


def row_colours(R: sp.csr_matrix) -> np.ndarray:
    """Greedy colouring of the rows of R in natural order (oracle.c): rows of
    one colour share no column.  Used by the coloured-order variant only."""
    R = _csr(R)
    rp, rc, _ = _arrs(R)
    col = np.zeros(R.shape[0], dtype=np.int32)
    k = _lib().oracle_row_colours(R.shape[0], R.shape[1], _ptr(rp), _ptr(rc), _ptr(col))
    if k < 0:
        raise ValueError("row colouring needs more than 128 colours")
    return col


def colour_order(R: sp.csr_matrix) -> np.ndarray:
    """The coloured sweep order (a variant of R3, not the paper's): rows by
    colour, natural order inside a colour."""
    return np.argsort(row_colours(R), kind="stable")


def kaczmarz_sweep_coloured(R: sp.csr_matrix, X: np.ndarray, rhs: np.ndarray,
                            B: sp.csr_matrix | None = None, shift: np.ndarray | None = None,
                            order: np.ndarray | None = None) -> None:
    """One Kaczmarz sweep over the rows of R - shift_j B in the coloured order
    (the colouring of R's pattern, merged with B's for the shifted form):
    the natural-order sweep of the rows permuted into that order."""
    R = _csr(R)
    if order is None:
        order = colour_order(R if B is None else _csr(abs(R) + abs(B)))
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)[order]
    kaczmarz_sweep(R[order], X, rhs, None if B is None else _csr(B)[order], shift)


def strength(N: sp.csr_matrix, theta: float) -> sp.csr_matrix:
    """Strong influences (Eq. strength): i is strongly influenced by j != i
    iff |n_ij| >= theta * sum_k |n_ik| (k over all columns, R8).  Returns S
    with S[i, j] = |n_ij| for the strong pairs."""
    N = _csr(N)
    absN = abs(N)
    rowsum = np.asarray(absN.sum(axis=1)).ravel()
    coo = absN.tocoo()
    keep = (coo.row != coo.col) & (coo.data >= theta * rowsum[coo.row]) & (coo.data > 0)
    S = sp.csr_matrix((coo.data[keep], (coo.row[keep], coo.col[keep])), shape=N.shape)
    return _csr(S)


def rs_coarsen(S: sp.csr_matrix) -> np.ndarray:
    """One-pass Ruge-Stueben coarsening (Algorithm "coarsening"); cf[i]=1 for C."""
    S = _csr(S)
    sp_, sc, _ = _arrs(S)
    cf = np.zeros(S.shape[0], dtype=np.int32)
    rc = _lib().oracle_rs_coarsen(S.shape[0], _ptr(sp_), _ptr(sc), _ptr(cf))
    if rc != 0:
        raise MemoryError("rs_coarsen")
    return cf


def interp_sets(S: sp.csr_matrix, cf: np.ndarray, cap: int):
    """Coarse interpolatory sets C^i = strong C-point influences of F point i
    (Sec. 3.7), strongest first, capped to `cap` members (R15)."""
    S = _csr(S)
    n = S.shape[0]
    ptr = [0]
    cols = []
    for i in range(n):
        if cf[i]:
            ptr.append(len(cols))
            continue
        lo, hi = S.indptr[i], S.indptr[i + 1]
        js = S.indices[lo:hi]
        ws = S.data[lo:hi]
        sel = cf[js] == 1
        js, ws = js[sel], ws[sel]
        order = np.lexsort((js, -ws))[:cap]
        cols.extend(int(j) for j in js[order])
        ptr.append(len(cols))
    return np.asarray(ptr, dtype=np.int64), np.asarray(cols, dtype=np.int32)


def fit_interp(S: sp.csr_matrix, cf: np.ndarray, Yf: np.ndarray, Yc: np.ndarray,
               w: np.ndarray) -> sp.csr_matrix:
    """Interpolation operator (Secs. 3.7-3.8): C rows carry a single 1 at the
    coarse index alpha(i); F rows carry the weighted LS weights of Eq. LS on
    C^i.  Yf = values used on F points, Yc = values used on C points."""
    n, nf = Yc.shape
    ci_ptr, ci_col = interp_sets(S, cf, max(nf - 1, 1))
    pval = np.zeros(ci_col.size, dtype=np.float64)
    _lib().oracle_ls_fit(n, nf, _ptr(ci_ptr), _ptr(ci_col),
                         _ptr(np.ascontiguousarray(Yf, dtype=np.float64)),
                         _ptr(np.ascontiguousarray(Yc, dtype=np.float64)),
                         _ptr(np.ascontiguousarray(w, dtype=np.float64)), _ptr(pval))
    alpha = np.cumsum(cf) - 1          # R10: increasing fine index
    rows = np.repeat(np.arange(n), np.diff(ci_ptr))
    crow = np.flatnonzero(cf)
    r = np.concatenate([crow, rows])
    c = np.concatenate([alpha[crow], alpha[ci_col]])
    v = np.concatenate([np.ones(crow.size), pval])
    return _csr(sp.csr_matrix((v, (r, c)), shape=(n, int(cf.sum()))))


# --------------------------------------------------------------------------
# hierarchy
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Level:
    """Operators of one level: A (m x n), B (m x m), C (n x n), and the
    interpolation P (m x m_c), Q (n x n_c) to the next coarser level.  The
    SPD kind uses A, B, P only (Sec. 5.2)."""

    A: sp.csr_matrix
    B: sp.csr_matrix
    C: sp.csr_matrix | None = None
    P: sp.csr_matrix | None = None
    Q: sp.csr_matrix | None = None

    def __post_init__(self):
        self.A = _csr(self.A)
        self.B = _csr(self.B)
        self.At = _csr(self.A.T)
        if self.C is not None:
            self.C = _csr(self.C)


@dataclasses.dataclass
class Hierarchy:
    kind: str        # "svd" | "spd"
    target: str      # "minimal" | "dominant"
    levels: list
    params: dict
    Ut: np.ndarray | None = None   # fine test vectors after the setup's last cycle
    Vt: np.ndarray | None = None
    redos: list = dataclasses.field(default_factory=list)  # outer iterations of redo sweeps

    @property
    def spd(self):
        return self.kind == "spd"


def hierarchy_from_interp(A, Ps, Qs, kind: str, target: str, params: dict | None = None):
    """A hierarchy with given interpolation operators (P_l, Q_l for l = 0 ..
    L-1; Qs ignored for the SPD kind): the finest level has B = I, C = I and
    every coarser level the Galerkin operators of Eq. coarseOp."""
    p = dict(DEFAULTS)
    p.update(params or {})
    spd = kind == "spd"
    A = _csr(A)
    m, n = A.shape
    levels = [Level(A, sp.identity(m, format="csr"), None if spd else sp.identity(n, format="csr"))]
    for l, P in enumerate(Ps):
        L = levels[-1]
        L.P = _csr(P)
        if not spd:
            L.Q = _csr(Qs[l])
        levels.append(galerkin(L, spd))
    return Hierarchy(kind, target, levels, p)


def galerkin(L: Level, spd: bool) -> Level:
    """Coarse operators of Eq. coarseOp: A_c = P^t A Q, B_c = P^t B P,
    C_c = Q^t C Q (SPD kind: P^t A P, P^t B P)."""
    P = L.P
    if spd:
        return Level(P.T @ L.A @ P, P.T @ L.B @ P)
    Q = L.Q
    return Level(P.T @ L.A @ Q, P.T @ L.B @ P, Q.T @ L.C @ Q)


# --------------------------------------------------------------------------
# relaxation (Secs. 3.4, 3.5, 5.3)
# --------------------------------------------------------------------------

def _cols_norm(M: sp.csr_matrix, X: np.ndarray) -> np.ndarray:
    return np.sqrt(np.einsum("ij,ij->j", X, M @ X))


def relax_boot(L: Level, spd: bool, target: str, sigma, U, V, K, T, omega: float,
               relax_order: str = "natural") -> None:
    """One block Gauss-Seidel relaxation of the boot vectors on
    A v - s B u = kappa, A^t u - s C v = tau (Eqs. genSVDresid1-2, add) with
    sigma fixed, in place.  Dominant: one weighted-Jacobi step for u, then
    for v (Sec. 3.5).  Minimal: Kaczmarz blocks, v from the rows of A, then u
    from the rows of A^t (Sec. 5.3, R1/R2); SPD: rows of A - lam B."""
    sigma = np.asarray(sigma, dtype=np.float64)
    if target == "minimal":
        sweep = kaczmarz_sweep if relax_order == "natural" else kaczmarz_sweep_coloured
        if spd:
            sweep(L.A, U, K, B=L.B, shift=sigma)
            return
        sweep(L.A, V, sigma * (L.B @ U) + K)
        sweep(L.At, U, sigma * (L.C @ V) + T)
        return
    dB = L.B.diagonal()[:, None]
    if spd:
        U -= omega * (L.B @ U - (L.A @ U - K) / sigma) / dB
        return
    dC = L.C.diagonal()[:, None]
    U -= omega * (L.B @ U - (L.A @ V - K) / sigma) / dB
    V -= omega * (L.C @ V - (L.At @ U - T) / sigma) / dC


def relax_test(L: Level, spd: bool, target: str, Ut, Vt, mu_t: int, omega: float) -> None:
    """mu_t relaxations of the test vectors (Sec. 3.4 power method with one
    omega-Jacobi inner step, v then u; Sec. 5.3 Kaczmarz on A v = 0 then
    A^t u = 0 for the minimal kind), in place."""
    m, n = L.A.shape
    for _ in range(mu_t):
        if target == "minimal":
            if spd:
                kaczmarz_sweep(L.A, Ut, np.zeros_like(Ut))
            else:
                kaczmarz_sweep(L.A, Vt, np.zeros((m, Vt.shape[1])))
                kaczmarz_sweep(L.At, Ut, np.zeros((n, Ut.shape[1])))
            continue
        dB = L.B.diagonal()[:, None]
        if spd:
            xb = Ut - omega * (L.B @ Ut - L.A @ Ut) / dB
            Ut[:] = xb / _cols_norm(L.B, xb)
            continue
        dC = L.C.diagonal()[:, None]
        vb = Vt - omega * (L.C @ Vt - L.At @ Ut) / dC
        Vt[:] = vb / _cols_norm(L.C, vb)
        ub = Ut - omega * (L.B @ Ut - L.A @ Vt) / dB
        Ut[:] = ub / _cols_norm(L.B, ub)
    if target == "minimal":        # R16
        Ut /= _cols_norm(L.B, Ut)
        if not spd:
            Vt /= _cols_norm(L.C, Vt)


def relax_test_v_only(L: Level, Vt, mu_t: int) -> None:
    """Minimal SVD kind under R21: mu_t Kaczmarz sweeps on A v = 0 for the
    column test vectors (Sec. 5.3), then unit C norm (R16); the row test
    vectors are derived from them."""
    for _ in range(mu_t):
        kaczmarz_sweep(L.A, Vt, np.zeros((L.A.shape[0], Vt.shape[1])))
    Vt /= _cols_norm(L.C, Vt)


def rayleigh(L: Level, spd: bool, U, V) -> np.ndarray:
    """Rayleigh quotient (Eq. Rayleigh): u^t A v / (|u|_B |v|_C); SPD:
    x^t A x / x^t B x."""
    if spd:
        return np.einsum("ij,ij->j", U, L.A @ U) / np.einsum("ij,ij->j", U, L.B @ U)
    return np.einsum("ij,ij->j", U, L.A @ V) / (_cols_norm(L.B, U) * _cols_norm(L.C, V))


def relax_boot_rq(L, spd, target, sigma, U, V, mu_b, omega):
    """Multiplicative-phase boot relaxation: mu_b block-GS steps with
    kappa = tau = 0, the sigmas updated by the Rayleigh quotient after each
    (Sec. 3.5); minimal SVD kind flips v_j when its quotient is negative
    (Sec. 5.3)."""
    for _ in range(mu_b):
        Z = np.zeros_like(U)
        relax_boot(L, spd, target, sigma, U, V, Z, None if spd else np.zeros_like(V), omega)
        rq = rayleigh(L, spd, U, V)
        if target == "minimal" and not spd:
            neg = rq < 0
            V[:, neg] *= -1.0
            rq = np.abs(rq)
        sigma = rq
    return sigma


# --------------------------------------------------------------------------
# coarsest level (Sec. 3.6, Thm genSVD) and pseudo-inverse solve (Sec. 4.2)
# --------------------------------------------------------------------------

def dense_XY(L: Level, spd: bool):
    """X = [[0, A], [A^t, 0]], Y = diag(B, C) of Eq. X (SPD kind: A, B)."""
    size = L.A.shape[0] if spd else L.A.shape[0] + L.A.shape[1]
    if size > 20000:
        raise ValueError("coarsest level of %d unknowns is too large for a dense solve "
                         "(the coarsening stopped early: check theta)" % size)
    if spd:
        return L.A.toarray(), L.B.toarray()
    m, n = L.A.shape
    A = L.A.toarray()
    X = np.zeros((m + n, m + n))
    X[:m, m:] = A
    X[m:, :m] = A.T
    Y = np.zeros((m + n, m + n))
    Y[:m, :m] = L.B.toarray()
    Y[m:, m:] = L.C.toarray()
    return X, Y


def coarsest_triplets(L: Level, spd: bool, target: str, nb: int):
    """n_b extremal generalized singular triplets of the coarsest level by the
    symmetric-definite eigenproblem (X - s Y) z = 0 (Thm genSVD): its l =
    min(m, n) largest eigenvalues are the s_j >= 0 with z = [u; v] / sqrt(2)
    for u^t B u = v^t C v = 1.  SPD kind: eigh(A, B)."""
    X, Y = dense_XY(L, spd)
    w, Z = sla.eigh(X, Y)
    if spd:
        sel = np.arange(nb) if target == "minimal" else np.arange(len(w) - 1, len(w) - 1 - nb, -1)
        return w[sel].copy(), np.ascontiguousarray(Z[:, sel]), None
    m, n = L.A.shape
    l = min(m, n)
    desc = np.argsort(-w, kind="stable")
    if target == "dominant":
        sel = desc[:nb]
    else:
        sel = desc[l - nb:l][::-1]          # ascending sigma
    s = np.sqrt(2.0)
    return (w[sel].copy(), np.ascontiguousarray(Z[:m, sel] * s),
            np.ascontiguousarray(Z[m:, sel] * s))


def coarse_geneig(XY):
    """Generalized eigenpairs of the coarsest pencil: X W = Y W diag(lam),
    W^t Y W = I, lam ascending (dense LAPACK, called once per hierarchy by
    the "geneig" variant of the coarsest solve)."""
    X, Y = XY[0], XY[1]
    return sla.eigh(X, Y)


def coarsest_pinv_apply(XY, sigma, K, T, spd: bool, drop: int = 1, form: str = "svd"):
    """[u; v] = (X - s_j Y)^+ [kappa; tau] per column j, with the SVD
    pseudo-inverse leaving out the single smallest singular value (Sec. 4.2,
    R7).  drop > 1 leaves out that many (a variant, not the paper's).

    form = "geneig" (a variant, not the paper's): with X w_k = lam_k Y w_k,
    W^t Y W = I, the inverse of X - s_j Y is W (Lam - s_j)^-1 W^t; the
    `drop` generalized eigenpairs nearest s_j (lowest k on ties) are left
    out.  XY may carry coarse_geneig(XY) as a third item."""
    X, Y = XY[0], XY[1]
    rhs = K if spd else np.vstack([K, T])
    out = np.zeros_like(rhs)
    if form == "geneig":
        lam, Wm = XY[2] if len(XY) > 2 else coarse_geneig(XY)
        for j in range(rhs.shape[1]):
            d = lam - sigma[j]
            near = np.lexsort((np.arange(len(d)), np.abs(d)))[:drop]
            inv = np.zeros_like(d)
            keep = np.ones(len(d), dtype=bool)
            keep[near] = False
            inv[keep] = 1.0 / d[keep]
            out[:, j] = Wm @ (inv * (Wm.T @ rhs[:, j]))
    else:
        for j in range(rhs.shape[1]):
            Uu, s, Vt = np.linalg.svd(X - sigma[j] * Y)
            k = len(s) - drop                 # s is descending: drop the last
            out[:, j] = Vt[:k].T @ ((Uu[:, :k].T @ rhs[:, j]) / s[:k])
    if spd:
        return out, None
    m = K.shape[0]
    return out[:m], out[m:]


# --------------------------------------------------------------------------
# Ritz step (Sec. 4.3) and residuals (R11)
# --------------------------------------------------------------------------

def ritz(A: sp.csr_matrix, spd: bool, target: str, U, V, row_form: str = "induced"):
    """Ritz projection on the finest level (B = I, C = I): orthonormalise the
    boot blocks by Householder QR, form M = U^t A V and take its SVD, which is
    the 2n_b generalized eigenproblem of Eq. genSVDRitz by Thm genSVD.  SPD:
    eigh(X^t A X).  sigma sorted descending (dominant) / ascending (minimal).
    row_form = "paper" keeps the two-sided projection on span(U_b) x span(V_b)
    for every kind; "induced" (R21) takes the left basis A V_b for the minimal
    SVD kind with m >= n."""
    if spd:
        Xh, _ = np.linalg.qr(U)
        M = Xh.T @ (A @ Xh)
        w, Yv = np.linalg.eigh(M)
        order = np.arange(len(w)) if target == "minimal" else np.arange(len(w))[::-1]
        return w[order].copy(), np.ascontiguousarray(Xh @ Yv[:, order]), None
    if row_form == "induced" and target == "minimal" and A.shape[0] >= A.shape[1]:
        # R21: the left basis is A V_b, which excludes the null(A^t) modes
        # (the spurious zero modes of Thm genSVD) from the projection
        U = np.ascontiguousarray(A @ V)
    Uh, _ = np.linalg.qr(U)
    Vh, _ = np.linalg.qr(V)
    M = Uh.T @ (A @ Vh)
    Yl, s, Zt = np.linalg.svd(M)
    order = np.arange(len(s)) if target == "dominant" else np.arange(len(s))[::-1]
    return (s[order].copy(), np.ascontiguousarray(Uh @ Yl[:, order]),
            np.ascontiguousarray(Vh @ Zt.T[:, order]))


def residual_norms(A: sp.csr_matrix, spd: bool, sigma, U, V) -> np.ndarray:
    """rho_j of R11 for unit vectors."""
    U = U / np.linalg.norm(U, axis=0)
    if spd:
        return np.linalg.norm(A @ U - U * sigma, axis=0) / np.abs(sigma)
    V = V / np.linalg.norm(V, axis=0)
    ru = np.linalg.norm(A @ V - U * sigma, axis=0)
    rv = np.linalg.norm(A.T @ U - V * sigma, axis=0)
    return np.sqrt(ru ** 2 + rv ** 2) / np.abs(sigma)


# --------------------------------------------------------------------------
# additive V-cycle (Secs. 4.1-4.2)
# --------------------------------------------------------------------------

def level_residual(L: Level, spd, sigma, U, V, K, T):
    """r = kappa - (A v - s B u), s = tau - (A^t u - s C v) (Eq. add)."""
    if spd:
        return K - (L.A @ U - sigma * (L.B @ U)), None
    r = K - (L.A @ V - sigma * (L.B @ U))
    s = T - (L.At @ U - sigma * (L.C @ V))
    return r, s


def vcycle(H: Hierarchy, l: int, sigma, U, V, K, T, coarse_XY=None) -> None:
    """One additive V-cycle for all columns at once, sigma_j fixed per
    column (Sec. 4.2), in place on U, V."""
    spd = H.spd
    p = H.params
    L = H.levels[l]
    if l == len(H.levels) - 1:
        XY = coarse_XY if coarse_XY is not None else dense_XY(L, spd)
        u, v = coarsest_pinv_apply(XY, sigma, K, T, spd, p.get("coarse_drop", 1),
                                   p.get("coarse_pinv", "svd"))
        U[:] = u
        if not spd:
            V[:] = v
        return
    order = p.get("relax_order", "natural")
    for _ in range(p["mu_b"]):
        relax_boot(L, spd, H.target, sigma, U, V, K, T, p["omega_J"], order)
    r, s = level_residual(L, spd, sigma, U, V, K, T)
    Kc = L.P.T @ r
    Tc = None if spd else L.Q.T @ s
    Uc = np.zeros((L.P.shape[1], U.shape[1]))
    Vc = None if spd else np.zeros((L.Q.shape[1], V.shape[1]))
    vcycle(H, l + 1, sigma, Uc, Vc, Kc, Tc, coarse_XY)
    U += L.P @ Uc
    if not spd:
        V += L.Q @ Vc
    for _ in range(p["mu_b"]):
        relax_boot(L, spd, H.target, sigma, U, V, K, T, p["omega_J"], order)


# --------------------------------------------------------------------------
# multiplicative phase (Sec. 3.3) and the whole method
# --------------------------------------------------------------------------

def _fit_weights(rq: np.ndarray, target: str) -> np.ndarray:
    a = np.maximum(np.abs(rq), 1e-300)
    return a if target == "dominant" else 1.0 / a


def _jacobi_on_N(L: Level, spd: bool, side: str, Y: np.ndarray, omega: float) -> np.ndarray:
    """One weighted Jacobi step on N x = 0 (R14), N = A A^t (u side), A^t A
    (v side) or A (SPD kind).  The weight is omega * 2 / g with g the
    Gershgorin bound max_i sum_k |n_ik| / n_ii of D^-1 N, so that the step
    damps every mode; g = 2 for the 5-point operators (weight omega)."""
    if spd:
        N = L.A
    elif side == "u":
        N = _csr(L.A @ L.At)
    else:
        N = _csr(L.At @ L.A)
    d = N.diagonal()
    g = float(np.max(np.asarray(abs(N).sum(axis=1)).ravel() / d))
    return Y - (omega * 2.0 / g) * (N @ Y) / d[:, None]


def _square(p: dict, spd: bool, shape) -> str | None:
    """The square form (R23) in use, or None."""
    f = p.get("square_form", "normal")
    return f if (f != "normal" and not spd and shape[0] == shape[1]) else None


def _ritz_form(p: dict, spd: bool, shape) -> str:
    """R21's one-sided Ritz step, or the two-sided one (the paper's row form
    and the square forms)."""
    return "paper" if _square(p, spd, shape) else p.get("row_form", "induced")


def _induced(spd: bool, target: str, shape, row_form: str = "induced") -> bool:
    """R21: the minimal SVD kind with m >= n takes its row (u) interpolation
    from the column interpolation, P_0 = A Q_0 on the finest level and
    P_l = Q_l below it (where A_l = B_l by construction).  row_form =
    "paper" keeps Sec. 3.7's form: the rows coarsened on A A^t with their own
    LS-fitted P."""
    return (row_form == "induced" and (not spd) and target == "minimal"
            and shape[0] >= shape[1])


def _down_sweep(A, spd: bool, target: str, nb: int, p: dict, Ut, Vt, sigma, ub, vb,
                wscale=None):
    """Downward sweep of one multiplicative cycle (Sec. 3.3): on each level
    coarsen, relax the test vectors (and the boot vectors, when there are
    any, with Rayleigh-quotient updates), fit P and Q by weighted LS on
    [test, boot], form the Galerkin operators and inject the vectors.  The
    fine test vectors Ut, Vt and the fine boot vectors ub, vb are relaxed in
    place.  wscale (optional, one factor per fitted vector) multiplies the LS
    weights.  Returns (levels, sigma, ub, vb), the last three on the
    coarsest level."""
    m, n = A.shape
    om = p["omega_J"]
    square = _square(p, spd, A.shape)
    induced = (not square) and _induced(spd, target, A.shape, p.get("row_form", "induced"))
    boot = ub is not None
    fine = Level(A, sp.identity(m, format="csr"),
                 None if spd else sp.identity(n, format="csr"))
    levels = [fine]
    ut, vt = Ut, Vt                    # fine test vectors are relaxed in place
    while True:
        L = levels[-1]
        lvl = len(levels) - 1
        ml, nl = L.A.shape
        if max(ml, nl) <= p["coarsest_max"] or len(levels) >= p["max_levels"]:
            break
        # coarsening (Sec. 3.7) depends on A_l only
        if spd or square:
            Su = strength(L.A, p["theta"])
            cfu = rs_coarsen(Su)
            mc = nc = int(cfu.sum())
            total_f, total_c = (ml, mc) if spd else (ml + nl, 2 * mc)
            if square:
                Sv, cfv = Su, cfu
        elif induced:
            Sv = strength(L.At @ L.A if lvl == 0 else L.A, p["theta"])
            cfv = rs_coarsen(Sv)
            mc = nc = int(cfv.sum())
            total_f, total_c = ml + nl, 2 * nc
        else:
            Su = strength(L.A @ L.At, p["theta"])
            Sv = strength(L.At @ L.A, p["theta"])
            cfu, cfv = rs_coarsen(Su), rs_coarsen(Sv)
            mc, nc = int(cfu.sum()), int(cfv.sum())
            total_f, total_c = ml + nl, mc + nc
        if total_c > 0.9 * total_f or min(mc, nc) < 2 * nb:
            break
        # relaxation of the test (and, after the first cycle, boot) vectors
        if induced:
            relax_test_v_only(L, vt, p["mu_t"])
            ut = np.ascontiguousarray(L.A @ vt if lvl == 0 else vt)
        else:
            relax_test(L, spd, target, ut, vt, p["mu_t"], om)
        if boot:
            sigma = relax_boot_rq(L, spd, target, sigma, ub, vb, p["mu_b"], om)
        # LS interpolation (Sec. 3.8) on [U_t, U_b]
        Uf = ut if not boot else np.hstack([ut, ub])
        Vf = None if spd else (vt if not boot else np.hstack([vt, vb]))
        rq = rayleigh(L, spd, Uf, Vf if not spd else None)
        w = _fit_weights(rq, target)
        if wscale is not None:
            w = w * wscale
        if induced:
            Yv = _jacobi_on_N(L, lvl > 0, "v", Vf, om)
            L.Q = fit_interp(Sv, cfv, Yv, Vf, w)
            L.P = _csr(L.A @ L.Q) if lvl == 0 else L.Q
        else:
            if target == "minimal":
                Yu = _jacobi_on_N(L, spd, "u", Uf, om)
                Yv = None if spd else _jacobi_on_N(L, spd, "v", Vf, om)
            else:
                Yu, Yv = Uf, Vf
            if square == "shared":
                # one operator for both sides: the u and v vectors fitted together
                L.P = fit_interp(Su, cfu, np.hstack([Yu, Yv]), np.hstack([Uf, Vf]),
                                 np.concatenate([w, w]))
                L.Q = L.P
            else:
                L.P = fit_interp(Su, cfu, Yu, Uf, w)
                if not spd:
                    L.Q = fit_interp(Sv, cfv, Yv, Vf, w)
        levels.append(galerkin(L, spd))
        # injection to the coarse level
        if induced:
            cv = np.flatnonzero(cfv)
            vt = np.ascontiguousarray(vt[cv])
            if boot:
                # P_0 = A Q_0: u_b = A v_b / s is interpolated by v_b[C] / s
                ub = np.ascontiguousarray(vb[cv] / sigma if lvl == 0 else ub[cv])
                vb = np.ascontiguousarray(vb[cv])
            continue
        cu = np.flatnonzero(cfu)
        ut = np.ascontiguousarray(ut[cu])
        if boot:
            ub = np.ascontiguousarray(ub[cu])
        if not spd:
            cv = np.flatnonzero(cfv)
            vt = np.ascontiguousarray(vt[cv])
            if boot:
                vb = np.ascontiguousarray(vb[cv])
    return levels, sigma, ub, vb


def setup(A, nb: int, target: str, kind: str, params: dict | None = None):
    """Multiplicative (setup) phase: n_mult bootstrap V-cycles (Sec. 3.3).
    Returns (Hierarchy of the last cycle, sigma_b, U_b, V_b) after the final
    Ritz step.  The hierarchy keeps the fine test vectors for later
    downward sweeps (redo_interpolation)."""
    p = dict(DEFAULTS)
    p.update(params or {})
    spd = kind == "spd"
    A = _csr(A)
    m, n = A.shape
    om = p["omega_J"]
    induced = (not _square(p, spd, A.shape)) and _induced(spd, target, A.shape,
                                                            p.get("row_form", "induced"))
    Ut = random_block(p["seed"], m, p["n_t"])
    Vt = None if spd else random_block(p["seed"] ^ (1 << 63), n, p["n_t"])
    if induced:
        Ut = np.ascontiguousarray(A @ Vt)
    sigma = Ub = Vb = None
    levels = []
    for cyc in range(p["n_mult"]):
        levels, sigma, ub, vb = _down_sweep(A, spd, target, nb, p, Ut, Vt, sigma, Ub, Vb)
        # coarsest level: new boot triplets by direct solve (Sec. 3.6)
        sigma, ub, vb = coarsest_triplets(levels[-1], spd, target, nb)
        # upward: interpolate (Eq. ranges), relax with RQ updates
        for l in range(len(levels) - 2, -1, -1):
            L = levels[l]
            ub = np.ascontiguousarray(L.P @ ub)
            if not spd:
                vb = np.ascontiguousarray(L.Q @ vb)
            sigma = relax_boot_rq(L, spd, target, sigma, ub, vb, p["mu_b"], om)
        sigma, Ub, Vb = ritz(A, spd, target, ub, vb, _ritz_form(p, spd, A.shape))
    H = Hierarchy(kind, target, levels, p, Ut, Vt)
    return H, sigma, Ub, Vb


def redo_interpolation(H: Hierarchy, sigma, U, V, converged, factor: float = 1e-3) -> None:
    """Sec. 6.3 remedy for lagging triplets: redetermine the interpolation
    operators by one downward sweep of the multiplicative phase, with the LS
    weights of the test vectors and of the converged boot vectors divided by
    1/factor (1000 in the paper), so that P and Q preferentially fit the
    unconverged triplets.  The sweep relaxes the hierarchy's fine test
    vectors in place and works on copies of the current boot triplets: the
    additive iterate (sigma, U, V) is not changed.  H.levels is replaced."""
    if H.Ut is None:
        raise ValueError("hierarchy without test vectors (not from setup)")
    spd = H.spd
    p = H.params
    A = H.levels[0].A
    nt = H.Ut.shape[1]
    converged = np.asarray(converged, dtype=bool)
    wscale = np.concatenate([np.full(nt, factor), np.where(converged, factor, 1.0)])
    ub = np.array(U, dtype=np.float64, order="C")
    vb = None if spd else np.array(V, dtype=np.float64, order="C")
    levels, _, _, _ = _down_sweep(A, spd, H.target, len(sigma), p, H.Ut, H.Vt,
                                  np.array(sigma, dtype=np.float64), ub, vb, wscale)
    H.levels = levels


def _solve_XY(H: Hierarchy):
    """The coarsest pencil (X, Y), with its generalized eigenpairs for the
    "geneig" form of the coarsest solve."""
    XY = dense_XY(H.levels[-1], H.spd)
    if H.params.get("coarse_pinv", "svd") == "geneig":
        XY = (XY[0], XY[1], coarse_geneig(XY))
    return XY


def solve(H: Hierarchy, sigma, U, V, tol: float = 1e-8, max_outer: int = 100,
          redo_tol: float | None = None, n_conv: int | None = None):
    """Additive phase (Sec. 4): V-cycle per triplet with sigma_j fixed, then a
    Ritz step, until max_j rho_j <= tol.  Returns (sigma, U, V, history)
    where history[i] = rho after i outer iterations.

    n_conv (optional, not in the paper): only the first n_conv triplets must
    meet tol; the rest are guards that keep the block complete past a small
    gap.

    redo_tol (optional; the Sec. 6.3 remedy): each time the number of
    triplets with rho_j <= redo_tol grows while some are still above it, the
    interpolation is redetermined (redo_interpolation, H.levels replaced)
    with those triplets counted as converged, and the cycles go on with the
    new hierarchy.  H.redos lists the outer iterations where that happened."""
    spd = H.spd
    A = H.levels[0].A
    U = np.array(U, dtype=np.float64, order="C")
    V = None if spd else np.array(V, dtype=np.float64, order="C")
    sigma = np.array(sigma, dtype=np.float64)
    XY = _solve_XY(H)
    hist = [residual_norms(A, spd, sigma, U, V)]
    H.redos.clear()
    nconv = 0
    kc = len(sigma) if n_conv is None else int(n_conv)
    for it in range(max_outer):
        if hist[-1][:kc].max() <= tol:
            break
        Z = np.zeros_like(U)
        vcycle(H, 0, sigma, U, V, Z, None if spd else np.zeros_like(V), XY)
        sigma, U, V = ritz(A, spd, H.target, U, V, _ritz_form(H.params, spd, A.shape))
        hist.append(residual_norms(A, spd, sigma, U, V))
        if redo_tol is not None:
            conv = hist[-1] <= redo_tol
            k = int(conv.sum())
            if nconv < k < len(conv):
                redo_interpolation(H, sigma, U, V, conv)
                XY = _solve_XY(H)
                H.redos.append(it + 1)
            nconv = max(nconv, k)
    return sigma, U, V, hist
