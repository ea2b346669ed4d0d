"""Plain FP64 CPU oracle of BiCG and recycling BiCG (RBiCG).

ORACLE / TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import this module.  It shares no code with the CUDA
library: it uses numpy / scipy (SpMV by scipy.sparse, Grams by explicit dense products,
the pencil by scipy.linalg.eig with left and right vectors, SVD by numpy) and follows the
paper's algorithms step by step, in the paper's order and notation.

Paper: Ahuja, de Sturler, Gugercin, Chang, "Recycling BiCG with an application to model
reduction" (arXiv:1010.0762).

  * bicg            -- Algorithm 1 (Section 2).
  * rbicg_pair      -- Algorithm 2 (Section 3) with eq. (CcheckChat) and eq. (minusXR),
                       plus the recycle-space refresh of Section 4.1 (harmonic Ritz pencil,
                       eq. (finalGenEigValue)), Section 4.2 (first system / first cycle) and
                       Section 4.3 (bi-orthogonal C_j, eqs. (equationSVD), (equationForUC)).
  * biorth_recycle  -- Section 4.3, last paragraph (C, Ct at the start of a new system).
  * rbicg_sequence  -- a sequence of dual pairs, carrying the recycle space (Section 4,
                       "the final U_j will be U for the next linear system"; Section 6.2:
                       keep the previous space if a pair converges in fewer than s steps).
  * cg              -- textbook conjugate gradients (Hestenes-Stiefel), used only to pin
                       BiCG (with A Hermitian, bt = b and equal starts, BiCG's primal
                       iterates are CG's).

Readings of the paper taken here where it is silent or ambiguous (each is listed in the
repository's design notes):
  R1 (a, b) = a^H b, so alpha = rt^H r / (pt^H q), beta = rt_i^H r_i / rt_{i-1}^H r_{i-1}.
  R2 stopping test is relative: ||r_i|| <= tol ||b|| and ||rt_i|| <= tol ||bt||; the dual
     test is skipped when bt = 0.  The true residual is recomputed at exit and reported.
  R3 Lanczos scaling of Section 4.1: v_m = r_{m-1}/||r_{m-1}||,
     vt_m = rt_{m-1} / (v_m, rt_{m-1}); then Tt = T^H, so Gamma_t is built from T^H.
  R4 dual recycle space: the left eigenvectors of the same pencil (L, R) for the same
     selected eigenvalues (the dual harmonic-Ritz pencil is (L^H, R^H) in exact
     arithmetic); on the first cycle of the first system this is the paper's "left and
     right eigenvectors of T_1".
  R5 "k eigenvalues closest to the origin": sort by |lambda| (ties by index), drop
     infinite / NaN values.  On a real problem, complex-conjugate pairs are kept together
     as the real and imaginary parts of one eigenvector; if the cut would split a pair,
     k-1 vectors are taken.
  R6 SVD truncation (Section 4.3): columns of C and Ct are first scaled to unit 2-norm
     (U, Ut scaled to match), then singular values >= svd_tol are kept.
  R7 cycles: the refresh for cycle j runs after iteration j*s; a partial final cycle is
     discarded; if no cycle completed the previous recycle space is kept.
  R8 random restart (Algorithm 2 step 3): xt_{-1} <- Philox vector in [-1, 1) from `seed`
     when |(r_0, rt_0)| <= 1e-14 ||r_0|| ||rt_0||.
  R9 breakdowns are not treated by the paper; they are reported as a status when
     |rho| <= 1e-14 ||rt|| ||r|| or |(pt, q)| <= 1e-14 ||pt|| ||q||.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .philox import philox_vector

STATUS_OK = 0
STATUS_NOT_CONVERGED = 1
STATUS_BREAKDOWN_RHO = 2
STATUS_BREAKDOWN_PQ = 3
STATUS_RECYCLE_EMPTY = 4

BREAKDOWN_EPS = 1e-14


def ip(a, b):
    """Standard inner product (a, b) = a^H b (reading R1)."""
    return np.vdot(a, b)


def as_scipy(A):
    """Accept a scipy sparse matrix, a dense array or an object with to_scipy()."""
    if hasattr(A, "to_scipy"):
        return A.to_scipy()
    if sp.issparse(A):
        return A.tocsr()
    return sp.csr_matrix(np.asarray(A))


def adjoint(A):
    """A^H as a CSR matrix."""
    return A.conj().T.tocsr()


@dataclasses.dataclass
class PairResult:
    x: np.ndarray
    xt: np.ndarray
    iters: int
    status: int
    relres: float
    relres_dual: float
    true_relres: float
    true_relres_dual: float
    cycles: int = 0
    recycle_dim: int = 0
    U_next: np.ndarray | None = None
    Ut_next: np.ndarray | None = None
    hist: dict = dataclasses.field(default_factory=dict)


# ----------------------------------------------------------------------------------------
# Algorithm 1: BiCG
# ----------------------------------------------------------------------------------------

def bicg(A, b, bt, x0, xt0, tol, max_itn, seed=0, record=False):
    """BiCG, Algorithm 1, with readings R1, R2, R8, R9."""
    A = as_scipy(A)
    AH = adjoint(A)
    dt = np.result_type(A.dtype, b.dtype, bt.dtype, x0.dtype, xt0.dtype)
    b = b.astype(dt); bt = bt.astype(dt)
    x = x0.astype(dt).copy(); xt = xt0.astype(dt).copy()
    # step 1
    r = b - A @ x
    rt = bt - AH @ xt
    # step 2
    if abs(ip(rt, r)) <= BREAKDOWN_EPS * np.linalg.norm(r) * np.linalg.norm(rt):
        xt = philox_vector(len(b), seed, np.iscomplexobj(xt)).astype(dt)
        rt = bt - AH @ xt
    # step 3
    p = np.zeros_like(r); pt = np.zeros_like(rt); beta = 0.0
    nb, nbt = np.linalg.norm(b), np.linalg.norm(bt)
    rho_old = ip(rt, r)
    hist = {"alpha": [], "beta": [], "rnorm": [np.linalg.norm(r)], "rtnorm": [np.linalg.norm(rt)]}
    if record:
        hist["x"] = [x.copy()]; hist["r"] = [r.copy()]
    status = STATUS_NOT_CONVERGED
    i = 0
    for i in range(1, max_itn + 1):
        p = r + beta * p
        pt = rt + np.conj(beta) * pt
        q = A @ p
        qt = AH @ pt
        pq = ip(pt, q)
        if abs(pq) <= BREAKDOWN_EPS * np.linalg.norm(pt) * np.linalg.norm(q):
            status = STATUS_BREAKDOWN_PQ
            break
        alpha = rho_old / pq
        x = x + alpha * p
        xt = xt + np.conj(alpha) * pt
        r = r - alpha * q
        rt = rt - np.conj(alpha) * qt
        hist["alpha"].append(alpha)
        hist["rnorm"].append(np.linalg.norm(r)); hist["rtnorm"].append(np.linalg.norm(rt))
        if record:
            hist["x"].append(x.copy()); hist["r"].append(r.copy())
        if _converged(r, rt, nb, nbt, tol):
            status = STATUS_OK
            break
        rho = ip(rt, r)
        if abs(rho) <= BREAKDOWN_EPS * np.linalg.norm(r) * np.linalg.norm(rt):
            status = STATUS_BREAKDOWN_RHO
            break
        beta = rho / rho_old
        hist["beta"].append(beta)
        rho_old = rho
    return PairResult(x=x, xt=xt, iters=i, status=status,
                      relres=np.linalg.norm(r) / _nz(nb), relres_dual=np.linalg.norm(rt) / _nz(nbt),
                      true_relres=np.linalg.norm(b - A @ x) / _nz(nb),
                      true_relres_dual=np.linalg.norm(bt - AH @ xt) / _nz(nbt), hist=hist)


def _nz(v):
    return v if v > 0 else 1.0


def _converged(r, rt, nb, nbt, tol):
    ok = np.linalg.norm(r) <= tol * nb
    if nbt > 0:
        ok = ok and np.linalg.norm(rt) <= tol * nbt
    return ok


def cg(A, b, x0, tol, max_itn):
    """Textbook conjugate gradients; returns the per-iteration alpha, beta and residuals."""
    A = as_scipy(A)
    x = x0.astype(np.result_type(A.dtype, b.dtype)).copy()
    r = b - A @ x
    p = r.copy()
    rr = ip(r, r)
    hist = {"alpha": [], "beta": [], "r": [r.copy()], "x": [x.copy()]}
    for _ in range(max_itn):
        q = A @ p
        alpha = rr / ip(p, q)
        x = x + alpha * p
        r = r - alpha * q
        hist["alpha"].append(alpha); hist["r"].append(r.copy()); hist["x"].append(x.copy())
        if np.linalg.norm(r) <= tol * np.linalg.norm(b):
            break
        rr_new = ip(r, r)
        beta = rr_new / rr
        hist["beta"].append(beta)
        p = r + beta * p
        rr = rr_new
    return x, hist


# ----------------------------------------------------------------------------------------
# Section 4.3: bi-orthogonal C, Ct
# ----------------------------------------------------------------------------------------

def biorth_recycle(A, U, Ut, svd_tol, C=None, Ct=None):
    """Make C = A U and Ct = A^H Ut bi-orthogonal with Ct^H C real, positive, diagonal.

    Section 4.3 / eqs. (equationSVD)-(equationForUC): SVD Ct^H C = M Sigma N^H, keep the p
    singular values >= svd_tol (after the column scaling of reading R6), and set
    U <- U N_p, Ut <- Ut M_p, C <- A U, Ct <- A^H Ut.  Returns (U, Ut, C, Ct, Dc) with Dc
    the p diagonal entries of Ct^H C (= Sigma_p in exact arithmetic).
    """
    A = as_scipy(A)
    AH = adjoint(A)
    if C is None:
        C = A @ U
    if Ct is None:
        Ct = AH @ Ut
    nc = np.linalg.norm(C, axis=0)
    nct = np.linalg.norm(Ct, axis=0)
    keep = (nc > 0) & (nct > 0)
    U, C, Ut, Ct = U[:, keep] / nc[keep], C[:, keep] / nc[keep], Ut[:, keep] / nct[keep], Ct[:, keep] / nct[keep]
    Mm, sig, NH = np.linalg.svd(Ct.conj().T @ C)
    N = NH.conj().T
    p = int(np.sum(sig >= svd_tol))
    U = U @ N[:, :p]
    Ut = Ut @ Mm[:, :p]
    C = A @ U
    Ct = AH @ Ut
    Dc = np.real(np.einsum("ij,ij->j", Ct.conj(), C))
    return U, Ut, C, Ct, Dc


# ----------------------------------------------------------------------------------------
# Section 4.1: T from the iteration scalars; cycle blocks
# ----------------------------------------------------------------------------------------

def T_entry(g_row, g_col, alpha, beta, rnorm):
    """Entry (g_row, g_col) (1-based Lanczos indices) of the tridiagonal T of Section 4.1.

    alpha[m], beta[m], rnorm[m] = ||r_m|| indexed by iteration m (alpha[0] unused,
    beta[0] = 0).  T(m,m) = 1/alpha_m + beta_{m-1}/alpha_{m-1};
    T(m+1,m) = -(||r_m||/||r_{m-1}||)/alpha_m; T(m,m+1) = -(||r_{m-1}||/||r_m||) beta_m/alpha_m.
    """
    m = g_col
    if g_row == m:
        val = 1.0 / alpha[m]
        if m >= 2:
            val = val + beta[m - 1] / alpha[m - 1]
        return val
    if g_row == m + 1:
        return -(rnorm[m] / rnorm[m - 1]) / alpha[m]
    if g_row == m - 1:
        mm = m - 1
        return -(rnorm[mm - 1] / rnorm[mm]) * beta[mm] / alpha[mm]
    return 0.0


def T_block(rows, cols, alpha, beta, rnorm, dtype):
    """Block of T with the given 1-based row and column Lanczos indices."""
    out = np.zeros((len(rows), len(cols)), dtype=dtype)
    for a, g_r in enumerate(rows):
        for c, g_c in enumerate(cols):
            if abs(g_r - g_c) <= 1 and g_r >= 1:
                out[a, c] = T_entry(g_r, g_c, alpha, beta, rnorm)
    return out


def Tt_block(rows, cols, alpha, beta, rnorm, dtype):
    """Same block of Tt = T^H (reading R3): Tt(g_r, g_c) = conj(T(g_c, g_r))."""
    out = np.zeros((len(rows), len(cols)), dtype=dtype)
    for a, g_r in enumerate(rows):
        for c, g_c in enumerate(cols):
            if abs(g_r - g_c) <= 1 and g_r >= 1:
                out[a, c] = np.conj(T_entry(g_c, g_r, alpha, beta, rnorm))
    return out


def select_eigs(lam, k, real_path):
    """Indices (and pair flags) of the k eigenvalues closest to the origin (reading R5).

    Returns a list of (index, is_pair) units; is_pair means the unit stands for lam[index]
    and its conjugate and contributes two real vectors.
    """
    finite = np.isfinite(lam)
    order = sorted(np.nonzero(finite)[0], key=lambda i: (abs(lam[i]), i))
    units, used, count = [], set(), 0
    for i in order:
        if i in used:
            continue
        if not real_path or lam[i].imag == 0.0:
            if count + 1 > k:
                break
            units.append((i, False)); used.add(i); count += 1
            continue
        # real problem, complex eigenvalue: find its conjugate partner
        cands = [j for j in order if j not in used and j != i and lam[j] == np.conj(lam[i])]
        if not cands:
            cands = [j for j in order if j not in used and j != i]
            cands = [min(cands, key=lambda j: abs(lam[j] - np.conj(lam[i])))] if cands else []
        if count + 2 > k:
            break
        units.append((i, True)); used.add(i); used.update(cands[:1]); count += 2
    return units


def eig_select(L, R, k, real_path):
    """Solve L w = lambda R w (eq. (finalGenEigValue)); return (W, Wt, lambdas).

    W: right eigenvectors of the selected eigenvalues; Wt: the matching left eigenvectors
    (reading R4).  On a real problem a conjugate pair contributes its real and imaginary
    parts (reading R5).
    """
    lam, VL, VR = sla.eig(L, R, left=True, right=True)
    units = select_eigs(lam, k, real_path)
    return _vectors_from_units(units, lam, VL, VR, real_path)


def _vectors_from_units(units, lam, VL, VR, real_path):
    Wc, Wtc, lams = [], [], []
    for i, pair in units:
        if real_path:
            if pair:
                Wc += [VR[:, i].real, VR[:, i].imag]
                Wtc += [VL[:, i].real, VL[:, i].imag]
                lams += [lam[i], np.conj(lam[i])]
            else:
                Wc.append(VR[:, i].real); Wtc.append(VL[:, i].real); lams.append(lam[i])
        else:
            Wc.append(VR[:, i]); Wtc.append(VL[:, i]); lams.append(lam[i])
    n = VR.shape[0]
    dt = np.float64 if real_path else np.complex128
    if not Wc:
        return np.zeros((n, 0), dt), np.zeros((n, 0), dt), np.array(lams)
    return np.array(Wc, dtype=dt).T, np.array(Wtc, dtype=dt).T, np.array(lams)


def eig_tridiag_select(T, k, real_path):
    """First cycle of the first system (Section 4.2): right and left eigenvectors of T_1."""
    lam, VL, VR = sla.eig(T, left=True, right=True)
    units = select_eigs(lam, k, real_path)
    return _vectors_from_units(units, lam, VL, VR, real_path)


# ----------------------------------------------------------------------------------------
# Algorithm 2: RBiCG for one dual pair, with the Section 4 recycle-space refresh
# ----------------------------------------------------------------------------------------

class _Ring:
    """The last `size` residual vectors, keyed by iteration index."""

    def __init__(self, size):
        self.size = size
        self.d = {}

    def put(self, i, v):
        self.d[i] = v.copy()
        for key in [key for key in self.d if key <= i - self.size]:
            del self.d[key]

    def __getitem__(self, i):
        return self.d[i]


def rbicg_pair(A, b, bt, x_1, xt_1, recycle=None, k=10, s=40, tol=1e-8, max_itn=20000,
               svd_tol=1e-6, seed=0, record=False, refresh=True):
    """Solve the dual pair A x = b, A^H xt = bt with Algorithm 2.

    recycle: None (first system, or no recycle space) or (U, Ut, C, Ct, Dc) as returned by
    biorth_recycle for this A.  Returns a PairResult whose U_next / Ut_next are the
    recycle space for the next system (reading R7).
    """
    A = as_scipy(A)
    AH = adjoint(A)
    real_path = not (np.iscomplexobj(A.data) or np.iscomplexobj(b) or np.iscomplexobj(bt)
                     or np.iscomplexobj(x_1) or np.iscomplexobj(xt_1)
                     or (recycle is not None and np.iscomplexobj(recycle[0])))
    dt = np.float64 if real_path else np.complex128
    n = A.shape[0]
    b = b.astype(dt); bt = bt.astype(dt)
    # step 1: U, Ut, C, Ct, Chat = Ct Dc^{-1}, Ccheck = C Dc^{-1} (eq. (CcheckChat))
    if recycle is not None and recycle[0].shape[1] > 0:
        U, Ut, C, Ct, Dc = recycle
        first_system = False
    else:
        U = Ut = C = Ct = np.zeros((n, 0), dt)
        Dc = np.zeros(0)
        first_system = True
    kc = C.shape[1]
    Chat = Ct / Dc if kc else Ct
    Ccheck = C / Dc if kc else C
    # step 2: eq. (minusXR)
    x = x_1.astype(dt).copy()
    xt = xt_1.astype(dt).copy()
    r_1 = b - A @ x
    x = x + U @ (Chat.conj().T @ r_1)
    r = r_1 - C @ (Chat.conj().T @ r_1)

    def dual_start(xt_m1):
        rt_m1 = bt - AH @ xt_m1
        return xt_m1 + Ut @ (Ccheck.conj().T @ rt_m1), rt_m1 - Ct @ (Ccheck.conj().T @ rt_m1)

    xt, rt = dual_start(xt)
    # step 3
    if abs(ip(rt, r)) <= BREAKDOWN_EPS * np.linalg.norm(r) * np.linalg.norm(rt):
        xt, rt = dual_start(philox_vector(n, seed, not real_path).astype(dt))
    # step 4
    p = np.zeros(n, dt); pt = np.zeros(n, dt); beta = 0.0
    zeta_c = np.zeros(kc, dt); zetat_c = np.zeros(kc, dt)
    nb, nbt = np.linalg.norm(b), np.linalg.norm(bt)

    # histories indexed by iteration m (index 0 = start)
    alpha_h = [None]
    beta_h = [0.0]
    rnorm_h = [np.linalg.norm(r)]
    rho_h = [ip(rt, r)]
    zeta_h = [np.zeros(kc, dt)]
    zetat_h = [np.zeros(kc, dt)]
    ring, ringt = _Ring(s + 2), _Ring(s + 2)
    ring.put(0, r); ringt.put(0, rt)
    hist = {"rnorm": [rnorm_h[0]], "rtnorm": [np.linalg.norm(rt)], "rho0": rho_h[0]}
    if record:
        hist.update(r=[r.copy()], rt=[rt.copy()], p=[], pt=[], x=[x.copy()], xt=[xt.copy()],
                    zeta_c=[zeta_c.copy()], zetat_c=[zetat_c.copy()])

    cyc = {"U": None, "Ut": None, "C": None, "Ct": None, "j": 0}
    status = STATUS_NOT_CONVERGED
    rho_old = rho_h[0]
    i = 0
    for i in range(1, max_itn + 1):
        # step 5, one iteration
        p = r + beta * p
        pt = rt + np.conj(beta) * pt
        z = A @ p
        zt = AH @ pt
        zeta = Chat.conj().T @ z
        zetat = Ccheck.conj().T @ zt
        q = z - C @ zeta
        qt = zt - Ct @ zetat
        pq = ip(pt, q)
        if abs(pq) <= BREAKDOWN_EPS * np.linalg.norm(pt) * np.linalg.norm(q):
            status = STATUS_BREAKDOWN_PQ
            break
        alpha = rho_old / pq
        zeta_c = zeta_c + alpha * zeta
        zetat_c = zetat_c + np.conj(alpha) * zetat
        x = x + alpha * p
        xt = xt + np.conj(alpha) * pt
        r = r - alpha * q
        rt = rt - np.conj(alpha) * qt
        rho = ip(rt, r)
        alpha_h.append(alpha); rnorm_h.append(np.linalg.norm(r)); rho_h.append(rho)
        zeta_h.append(zeta); zetat_h.append(zetat)
        ring.put(i, r); ringt.put(i, rt)
        hist["rnorm"].append(rnorm_h[-1]); hist["rtnorm"].append(np.linalg.norm(rt))
        if record:
            hist["r"].append(r.copy()); hist["rt"].append(rt.copy()); hist["p"].append(p.copy())
            hist["pt"].append(pt.copy()); hist["x"].append(x.copy()); hist["xt"].append(xt.copy())
            hist["zeta_c"].append(zeta_c.copy()); hist["zetat_c"].append(zetat_c.copy())
        done = _converged(r, rt, nb, nbt, tol)
        if refresh and i % s == 0:
            cyc["j"] += 1
            _refresh(cyc, A, AH, U, Ut, C, Ct, Dc, Chat, Ccheck, first_system, k, s, svd_tol,
                     alpha_h, beta_h, rnorm_h, rho_h, zeta_h, zetat_h, ring, ringt, real_path,
                     hist if record else None)
        if done:
            status = STATUS_OK
            break
        if abs(rho) <= BREAKDOWN_EPS * rnorm_h[-1] * np.linalg.norm(rt):
            status = STATUS_BREAKDOWN_RHO
            break
        beta = rho / rho_old
        beta_h.append(beta)
        rho_old = rho
    # step 7
    x = x - U @ zeta_c
    xt = xt - Ut @ zetat_c
    if cyc["j"] > 0 and cyc["U"] is not None:
        U_next, Ut_next = cyc["U"], cyc["Ut"]
    elif not first_system:
        U_next, Ut_next = U, Ut
    else:
        U_next = Ut_next = None
    hist["alpha"] = alpha_h[1:]; hist["beta"] = beta_h[1:]
    return PairResult(
        x=x, xt=xt, iters=i, status=status,
        relres=rnorm_h[-1] / _nz(nb), relres_dual=np.linalg.norm(rt) / _nz(nbt),
        true_relres=np.linalg.norm(b - A @ x) / _nz(nb),
        true_relres_dual=np.linalg.norm(bt - AH @ xt) / _nz(nbt),
        cycles=cyc["j"], recycle_dim=kc, U_next=U_next, Ut_next=Ut_next, hist=hist)


def _lanczos_vectors(ring, ringt, rnorm_h, idx):
    """v_m and vt_m (Section 4.1 scaling, reading R3) for 1-based Lanczos indices idx."""
    V, Vt = [], []
    for m in idx:
        r = ring[m - 1]
        v = r / rnorm_h[m - 1]
        rt = ringt[m - 1]
        vt = rt / ip(v, rt)
        V.append(v); Vt.append(vt)
    return np.array(V).T, np.array(Vt).T


def _refresh(cyc, A, AH, U, Ut, C, Ct, Dc, Chat, Ccheck, first_system, k, s, svd_tol,
             alpha_h, beta_h, rnorm_h, rho_h, zeta_h, zetat_h, ring, ringt, real_path, rec):
    """Recycle-space refresh after iteration j*s (Sections 4.1-4.3)."""
    j = cyc["j"]
    dt = np.float64 if real_path else np.complex128
    cols = list(range((j - 1) * s + 1, j * s + 1))              # V_j
    V, Vt = _lanczos_vectors(ring, ringt, rnorm_h, cols)
    # beta_{js} = rho_{js} / rho_{js-1} is needed by the bottom row of Gamma_t_j
    # (Tt(js+1, js) = conj(T(js, js+1))); rho_{js} is known at this point.
    i = j * s
    alpha, beta, rnorm = alpha_h, beta_h[:i] + [rho_h[i] / rho_h[i - 1]], rnorm_h
    if first_system and j == 1:
        # Section 4.2: eigenvectors of T_1
        T1 = T_block(cols, cols, alpha, beta, rnorm, dt)
        W, Wt, lam = eig_tridiag_select(T1, k, real_path)
        Phi, Phit = V, Vt
        blocks = None
    else:
        if j == 1:
            rows = list(range(1, s + 2))                        # V_1 underlined = [V_1 v_{s+1}]
        else:
            rows = list(range((j - 1) * s, j * s + 2))          # Upsilon_j
        Ups, Upst = _lanczos_vectors(ring, ringt, rnorm_h, rows)
        Gam = T_block(rows, cols, alpha, beta, rnorm, dt)
        Gamt = Tt_block(rows, cols, alpha, beta, rnorm, dt)
        kc = C.shape[1]
        if kc:
            AV = A @ V
            AVt = AH @ Vt
            B = Chat.conj().T @ AV                                # B_j = Chat^H A V_j
            Bt = Ccheck.conj().T @ AVt                            # Bt_j = Ccheck^H A^H Vt_j
        if first_system:
            # Section 4.2, cycles j >= 2 of the first system
            Up, Upt, Cp, Cpt = cyc["U"], cyc["Ut"], cyc["C"], cyc["Ct"]
            kp = Up.shape[1]
            Phi = np.hstack([Up, V]); Phit = np.hstack([Upt, Vt])
            Psi = np.hstack([Cp, Ups]); Psit = np.hstack([Cpt, Upst])
            H = _blockmat([[np.eye(kp), np.zeros((kp, s))], [np.zeros((len(rows), kp)), Gam]], dt)
            Ht = _blockmat([[np.eye(kp), np.zeros((kp, s))], [np.zeros((len(rows), kp)), Gamt]], dt)
        elif j == 1:
            # Section 4.2, first cycle of a later system
            Phi = np.hstack([U, V]); Phit = np.hstack([Ut, Vt])
            Psi = np.hstack([C, Ups]); Psit = np.hstack([Ct, Upst])
            H = _blockmat([[np.eye(kc), B], [np.zeros((len(rows), kc)), Gam]], dt)
            Ht = _blockmat([[np.eye(kc), Bt], [np.zeros((len(rows), kc)), Gamt]], dt)
        else:
            # Section 4.1, general cycle
            Up, Upt, Cp, Cpt = cyc["U"], cyc["Ut"], cyc["C"], cyc["Ct"]
            kp = Up.shape[1]
            Phi = np.hstack([Up, V]); Phit = np.hstack([Upt, Vt])
            Psi = np.hstack([C, Cp, Ups]); Psit = np.hstack([Ct, Cpt, Upst])
            H = _blockmat([[np.zeros((kc, kp)), B], [np.eye(kp), np.zeros((kp, s))],
                           [np.zeros((len(rows), kp)), Gam]], dt)
            Ht = _blockmat([[np.zeros((kc, kp)), Bt], [np.eye(kp), np.zeros((kp, s))],
                            [np.zeros((len(rows), kp)), Gamt]], dt)
        # eq. (finalGenEigValue): Ht^H Psit^H Psi H w = lambda Ht^H Psit^H Phi w
        L = Ht.conj().T @ (Psit.conj().T @ Psi) @ H
        R = Ht.conj().T @ (Psit.conj().T @ Phi)
        W, Wt, lam = eig_select(L, R, k, real_path)
        blocks = dict(Phi=Phi, Phit=Phit, Psi=Psi, Psit=Psit, H=H, Ht=Ht, L=L, R=R)
    # Section 4.3: U_j = Phi W, Ut_j = Phit Wt, then bi-orthogonalise
    Uj, Ujt = Phi @ W, Phit @ Wt
    Uj, Ujt, Cj, Cjt, _ = biorth_recycle(A, Uj, Ujt, svd_tol)
    cyc.update(U=Uj, Ut=Ujt, C=Cj, Ct=Cjt)
    if rec is not None:
        rec.setdefault("cycles", []).append(dict(j=j, V=V, Vt=Vt, lam=lam, W=W, Wt=Wt, U=Uj, Ut=Ujt,
                                                 C=Cj, Ct=Cjt, blocks=blocks))


def _blockmat(rows, dt):
    return np.block([[np.asarray(b, dtype=dt) for b in row] for row in rows])


# ----------------------------------------------------------------------------------------
# Sequences of dual pairs
# ----------------------------------------------------------------------------------------

def rbicg_sequence(problems, k=10, s=40, tol=1e-8, max_itn=20000, svd_tol=1e-6, seed=0,
                   x_1=None, xt_1=None, recycle=True, on_pair=None, guard=0.0, restarts=0, refresh_every=1):
    """Solve a sequence of dual pairs [{A, b, bt}, ...], carrying the recycle space.

    recycle=False gives plain BiCG on every pair (RBiCG with an empty recycle space).
    guard > 0 reproduces the CUDA library's stagnation guard, which is NOT part of the paper:
    a pair solved with a recycle space that has not converged after guard x (iterations of
    the last pair solved from its start without one, all legs counted) iterations, rounded
    up to whole cycles of s, applies
    step 7 to its iterate and continues from it as plain BiCG (Algorithm 2 with an empty
    recycle space).
    restarts > 0 reproduces the library's restart after a breakdown (also not in the paper): a
    pair that ends in a BiCG breakdown (rho or (pt, q) below the relative threshold) continues
    from its iterate as plain BiCG, at most `restarts` times.
    refresh_every > 1 (Section 6.2: the recycle space may be recomputed only for some systems of
    a sequence): pair j computes a new recycle space only when j % refresh_every == 0; the other
    pairs use the space they were given and hand it on unchanged.
    Returns a list of PairResult (iters counts every leg; hist["fallback"] is True after a
    guard fallback or a restart).
    """
    out = []
    Uc = Utc = None
    last_plain = 0
    for j, pr in enumerate(problems):
        A = as_scipy(pr["A"])
        b, bt = pr["b"], pr["bt"]
        n = A.shape[0]
        x0 = np.zeros(n, dtype=b.dtype) if x_1 is None else x_1[j]
        xt0 = np.zeros(n, dtype=bt.dtype) if xt_1 is None else xt_1[j]
        rec = None
        ref_j = recycle and j % refresh_every == 0
        if recycle and Uc is not None and Uc.shape[1] > 0:
            rec = biorth_recycle(A, Uc, Utc, svd_tol)
        limit = max_itn
        if guard > 0 and rec is not None and rec[0].shape[1] > 0 and last_plain > 0:
            # the library tests the guard when a cycle of s iterations ends, so the recycled leg
            # runs to the first multiple of s at or above guard x last_plain
            limit = min(max_itn, -(-int(guard * last_plain) // s) * s)
        res = rbicg_pair(A, b, bt, x0, xt0, recycle=rec, k=k, s=s, tol=tol, max_itn=limit,
                         svd_tol=svd_tol, seed=seed + j, refresh=ref_j)
        res.hist["fallback"] = False
        res.hist["guard_limit"] = limit if limit < max_itn else None
        if limit < max_itn and res.status != STATUS_OK:
            first = res
            res = rbicg_pair(A, b, bt, first.x, first.xt, recycle=None, k=k, s=s, tol=tol,
                             max_itn=max_itn - first.iters, svd_tol=svd_tol, seed=seed + j,
                             refresh=ref_j)
            res.iters += first.iters
            res.hist["fallback"] = True
            res.hist["guard_limit"] = limit
            res.recycle_dim = 0
        used = 0
        while used < restarts and res.status in (STATUS_BREAKDOWN_RHO, STATUS_BREAKDOWN_PQ) and res.iters < max_itn:
            used += 1
            prev = res
            res = rbicg_pair(A, b, bt, prev.x, prev.xt, recycle=None, k=k, s=s, tol=tol,
                             max_itn=max_itn - prev.iters, svd_tol=svd_tol, seed=seed + j, refresh=ref_j)
            res.iters += prev.iters
            res.hist["fallback"] = True
            res.recycle_dim = 0
        # the guard's baseline is the full iteration count of the last pair solved from its
        # start without a recycle space; a leg that continued a stalled or broken solve starts
        # from a nearly converged iterate and would shrink it
        if rec is None or rec[0].shape[1] == 0:
            last_plain = res.iters
        if rec is not None and rec[0].shape[1] == 0 and res.status == STATUS_OK:
            res.status = STATUS_RECYCLE_EMPTY
        out.append(res)
        if on_pair is not None:
            on_pair(j, res)
        if recycle:
            Uc, Utc = res.U_next, res.Ut_next
    return out
