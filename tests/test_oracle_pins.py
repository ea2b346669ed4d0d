"""Pins of the CPU oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: dense LU, textbook CG,
the explicit projected operator A_1 of eq. (augBiLanNew), exact-arithmetic invariants of
Algorithm 2, the block relation A Phi_j = Psi_j H_j (eq. (firstKW)), closed-form
eigenpairs of the 1-D finite-difference operator, published generator answers, and the
qualitative result of Section 6.1 (fewer iterations when the same pair is solved again).
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import rbicg_oracle as O
from oracle.philox import philox4x32_10, philox_vector
from paper_1010_0762_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_complex_matrix(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return sp.csr_matrix(M + 3.0 * np.sqrt(n) * np.eye(n))


# ---------------------------------------------------------------- generator pins
def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        assert philox4x32_10(w[0:4], w[4:6]) == tuple(w[6:10])


def test_philox_vector_matches_block_function():
    seed = 0x1234_5678_9ABC
    v = philox_vector(5, seed, complex_=True)
    for e in range(5):
        c = philox4x32_10((e, 0, 0, 0), (seed & 0xFFFFFFFF, seed >> 32))
        re = (((c[1] << 32) | c[0]) >> 11) / 2.0 ** 53
        im = (((c[3] << 32) | c[2]) >> 11) / 2.0 ** 53
        assert v[e] == complex(2 * re - 1, 2 * im - 1)


def test_convdiff_transpose_is_negated_convection():
    for N, c in [(7, [3.0]), (6, [2.0, -5.0]), (4, [1.0, 2.0, 3.0])]:
        A = I.convdiff(N, c).to_scipy()
        B = I.convdiff(N, [-v for v in c]).to_scipy()
        assert abs(A.T - B).max() == 0.0
        assert A.nnz == I.convdiff_nnz(N, len(c))


# ---------------------------------------------------------------- BiCG (Algorithm 1)
@pytest.mark.parametrize("case", ["1d", "2d", "complex"])
def test_bicg_matches_dense_lu(case):
    if case == "1d":
        A = I.convdiff(40, [5.0]).to_scipy()
    elif case == "2d":
        A = I.convdiff(8, [10.0, 10.0]).to_scipy()
    else:
        A = _rand_complex_matrix(48, 3)
    n = A.shape[0]
    b = I.normal_vector(n, 11, complex_=(case == "complex"))
    bt = I.normal_vector(n, 12, complex_=(case == "complex"))
    res = O.bicg(A, b, bt, np.zeros(n), np.zeros(n), 1e-13, 10 * n)
    Ad = A.toarray()
    x = np.linalg.solve(Ad, b)
    xt = np.linalg.solve(Ad.conj().T, bt)
    kappa = np.linalg.cond(Ad)
    assert res.status == O.STATUS_OK
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) <= 10 * kappa * 1e-13
    assert np.linalg.norm(res.xt - xt) / np.linalg.norm(xt) <= 10 * kappa * 1e-13


def test_bicg_equals_cg_on_hermitian_with_equal_dual():
    # c = 0: symmetric positive definite Laplacian; bt = b, xt0 = x0 => BiCG's primal
    # recurrences are CG's (Hestenes-Stiefel).
    A = I.convdiff(12, [0.0, 0.0]).to_scipy()
    n = A.shape[0]
    b = I.normal_vector(n, 5)
    res = O.bicg(A, b, b.copy(), np.zeros(n), np.zeros(n), 1e-14, 30, record=True)
    _, h = O.cg(A, b, np.zeros(n), 1e-14, 30)
    m = min(len(res.hist["alpha"]), len(h["alpha"]), 30)
    assert m >= 25
    np.testing.assert_allclose(res.hist["alpha"][:m], h["alpha"][:m], rtol=1e-10)
    np.testing.assert_allclose(res.hist["beta"][:m - 1], h["beta"][:m - 1], rtol=1e-9)
    for i in range(m):
        np.testing.assert_allclose(res.hist["r"][i], h["r"][i], rtol=0,
                                   atol=1e-10 * np.linalg.norm(b))


def test_bicg_random_restart_when_dual_start_orthogonal():
    # bt = 0 and xt_{-1} = 0 give rt_0 = 0 -> (r_0, rt_0) = 0 -> Algorithm 1 step 2 draws
    # xt_0 at random; the primal system must still be solved.
    A = I.convdiff(10, [4.0, 1.0]).to_scipy()
    n = A.shape[0]
    b = I.normal_vector(n, 2)
    res = O.bicg(A, b, np.zeros(n), np.zeros(n), np.zeros(n), 1e-10, 2000, seed=99)
    assert res.status == O.STATUS_OK
    assert res.true_relres < 1e-9


def test_bicg_not_converged_status():
    A = I.convdiff(16, [10.0, 10.0]).to_scipy()
    n = A.shape[0]
    res = O.bicg(A, I.normal_vector(n, 1), I.normal_vector(n, 2), np.zeros(n), np.zeros(n), 1e-12, 5)
    assert res.status == O.STATUS_NOT_CONVERGED and res.iters == 5


# ---------------------------------------------------------------- RBiCG (Algorithm 2)
def _eig_recycle(A, k, svd_tol=1e-8, pert=1e-3):
    """Approximate (perturbed) left/right eigenvector spaces of the k smallest eigenvalues.

    Equivalences that hold in exact arithmetic are compared over many iterations only with
    a well-conditioned oblique projector (||I - C Dc^{-1} Ct^H|| ~ 1): an ill-conditioned
    one amplifies rounding differences between two equivalent formulations.
    """
    w, VL, VR = sla.eig(A.toarray(), left=True, right=True)
    idx = np.argsort(abs(w))[:k]
    cplx = np.iscomplexobj(A.data)
    U, Ut = (VR[:, idx].copy(), VL[:, idx].copy()) if cplx else (VR[:, idx].real.copy(), VL[:, idx].real.copy())
    rng = np.random.default_rng(0)
    U = U + pert * rng.standard_normal(U.shape)        # approximate, not exact, spaces
    Ut = Ut + pert * rng.standard_normal(Ut.shape)
    return O.biorth_recycle(A, U, Ut, svd_tol)


def test_biorth_recycle_makes_dc_diagonal_positive():
    A = I.convdiff(12, [10.0, 5.0]).to_scipy()
    U, Ut, C, Ct, Dc = _eig_recycle(A, 6)
    G = Ct.conj().T @ C
    assert np.all(Dc > 0)
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() <= 1e-12 * Dc.max()
    assert np.abs(A @ U - C).max() == 0.0
    assert np.abs(A.conj().T @ Ut - Ct).max() == 0.0


def test_rbicg_without_recycle_space_is_bicg():
    A = I.convdiff(10, [10.0, 3.0]).to_scipy()
    n = A.shape[0]
    b, bt = I.normal_vector(n, 1), I.normal_vector(n, 2)
    r1 = O.rbicg_pair(A, b, bt, np.zeros(n), np.zeros(n), None, k=5, s=1000, tol=1e-10)
    r2 = O.bicg(A, b, bt, np.zeros(n), np.zeros(n), 1e-10, 20000)
    assert r1.iters == r2.iters
    np.testing.assert_allclose(r1.hist["alpha"], r2.hist["alpha"], rtol=1e-12)
    np.testing.assert_allclose(r1.x, r2.x, rtol=0, atol=1e-12 * np.linalg.norm(r2.x))


def test_rbicg_equals_bicg_on_explicit_projected_operator():
    # eq. (augBiLanNew): RBiCG is BiCG applied to A_1 = (I - C Dc^{-1} Ct^H) A (I - ...)
    # from r_0, rt_0 of eq. (minusXR).  Compare the first 20 alphas and residual norms.
    A = I.convdiff(16, [3.0, 1.0]).to_scipy()
    n = A.shape[0]
    rec = _eig_recycle(A, 6)
    U, Ut, C, Ct, Dc = rec
    P = np.eye(n) - C @ np.diag(1.0 / Dc) @ Ct.conj().T
    assert np.linalg.norm(P, 2) < 10.0
    b, bt = I.normal_vector(n, 3), I.normal_vector(n, 4)
    r = O.rbicg_pair(A, b, bt, np.zeros(n), np.zeros(n), rec, k=6, s=1000, tol=1e-14,
                     max_itn=20, record=True)
    A1 = P @ A.toarray() @ P
    # BiCG on A_1 from the projected starts: solve A_1 e = r_0 with zero initial guess
    r0, rt0 = r.hist["r"][0], r.hist["rt"][0]
    rb = O.bicg(sp.csr_matrix(A1), r0, rt0, np.zeros(n), np.zeros(n), 1e-14, 20, record=True)
    np.testing.assert_allclose(r.hist["alpha"][:20], rb.hist["alpha"][:20], rtol=1e-8)
    np.testing.assert_allclose(r.hist["rnorm"][:21], rb.hist["rnorm"][:21], rtol=1e-8)


def test_rbicg_invariants_and_true_residual():
    A = I.convdiff(12, [10.0, 5.0]).to_scipy()
    n = A.shape[0]
    rec = _eig_recycle(A, 6)
    U, Ut, C, Ct, Dc = rec
    b, bt = I.normal_vector(n, 5), I.normal_vector(n, 6)
    r = O.rbicg_pair(A, b, bt, np.zeros(n), np.zeros(n), rec, k=6, s=1000, tol=1e-14,
                     max_itn=25, record=True)
    for i in range(1, 26):
        ri, rti, pi = r.hist["r"][i], r.hist["rt"][i], r.hist["p"][i - 1]
        # Petrov-Galerkin condition (eq. (orth)): r_i _|_ Ct, rt_i _|_ C; and Ct^H p_i = 0
        assert np.abs(Ct.conj().T @ ri).max() <= 1e-9 * np.linalg.norm(Ct) * np.linalg.norm(ri)
        assert np.abs(C.conj().T @ rti).max() <= 1e-9 * np.linalg.norm(C) * np.linalg.norm(rti)
        assert np.abs(Ct.conj().T @ pi).max() <= 1e-9 * np.linalg.norm(Ct) * np.linalg.norm(pi)
        # r_i is the residual of x_i - U zeta_c (step 7 applied at step i), since A U = C
        xi = r.hist["x"][i] - U @ r.hist["zeta_c"][i]
        xti = r.hist["xt"][i] - Ut @ r.hist["zetat_c"][i]
        assert np.linalg.norm(b - A @ xi - ri) <= 1e-10 * np.linalg.norm(b)
        assert np.linalg.norm(bt - A.conj().T @ xti - rti) <= 1e-10 * np.linalg.norm(bt)


def test_rbicg_solution_matches_dense_lu_with_recycling():
    for A, cplx in [(I.convdiff(8, [10.0, 10.0]).to_scipy(), False),
                    (_rand_complex_matrix(48, 4), True)]:
        n = A.shape[0]
        b = I.normal_vector(n, 21, complex_=cplx)
        bt = I.normal_vector(n, 22, complex_=cplx)
        rec = _eig_recycle(A, 4)
        res = O.rbicg_pair(A, b, bt, np.zeros(n), np.zeros(n), rec, k=4, s=16, tol=1e-13,
                           max_itn=20 * n)
        Ad = A.toarray()
        kappa = np.linalg.cond(Ad)
        x, xt = np.linalg.solve(Ad, b), np.linalg.solve(Ad.conj().T, bt)
        assert res.status == O.STATUS_OK
        assert np.linalg.norm(res.x - x) / np.linalg.norm(x) <= 10 * kappa * 1e-13
        assert np.linalg.norm(res.xt - xt) / np.linalg.norm(xt) <= 10 * kappa * 1e-13


def test_manufactured_solution_larger_grid():
    A = I.convdiff(40, [10.0, 10.0]).to_scipy()
    n = A.shape[0]
    xs = I.normal_vector(n, 31)
    b = A @ xs
    bt = A.conj().T @ I.normal_vector(n, 32)
    for rec in (None, _eig_recycle(A, 8, pert=1e-6)):
        r = O.rbicg_pair(A, b, bt, np.zeros(n), np.zeros(n), rec, k=8, s=40, tol=1e-11)
        assert r.status == O.STATUS_OK
        # ||x - x*|| / ||x*|| <= kappa * relres; kappa of this operator is below 1e3
        assert np.linalg.norm(r.x - xs) / np.linalg.norm(xs) < 1e-8


def test_lanczos_biorthogonality_first_cycle():
    A = I.convdiff(16, [10.0, 10.0]).to_scipy()
    n = A.shape[0]
    rec = _eig_recycle(A, 5)
    U, Ut, C, Ct, Dc = rec
    r = O.rbicg_pair(A, I.normal_vector(n, 7), I.normal_vector(n, 8), np.zeros(n), np.zeros(n),
                     rec, k=5, s=12, tol=1e-14, max_itn=12, record=True)
    cyc = r.hist["cycles"][0]
    V, Vt = cyc["V"], cyc["Vt"]
    assert np.abs(Vt.conj().T @ V - np.eye(V.shape[1])).max() < 1e-6       # eq. (scalingfactor)
    assert np.abs(Ct.conj().T @ V).max() < 1e-8 * np.linalg.norm(Ct)       # eq. (biorth)
    assert np.abs(C.conj().T @ Vt).max() < 1e-8 * np.linalg.norm(C) * np.abs(Vt).max()


@pytest.mark.parametrize("case", ["first_j2", "later_j1", "later_j2"])
def test_block_relation_A_Phi_equals_Psi_H(case):
    # eq. (firstKW) for the general cycle and the two special cases of Section 4.2.  The
    # Gamma blocks are built from the iteration scalars with the T formula of Section 4.1,
    # so this pins those formulas (primal and, via Tt = T^H, dual).
    A = I.convdiff(14, [10.0, 6.0]).to_scipy()
    n = A.shape[0]
    b, bt = I.normal_vector(n, 9), I.normal_vector(n, 10)
    s = 10
    rec = None if case == "first_j2" else _eig_recycle(A, 5)
    r = O.rbicg_pair(A, b, bt, np.zeros(n), np.zeros(n), rec, k=5, s=s, tol=1e-14,
                     max_itn=2 * s, record=True)
    j = 1 if case == "later_j1" else 2
    blk = r.hist["cycles"][j - 1]["blocks"]
    AH = A.conj().T
    for Phi, Psi, H, AA in [(blk["Phi"], blk["Psi"], blk["H"], A), (blk["Phit"], blk["Psit"], blk["Ht"], AH)]:
        lhs = AA @ Phi
        assert np.linalg.norm(lhs - Psi @ H) <= 1e-10 * np.linalg.norm(lhs)


def test_first_cycle_T_is_petrov_galerkin_projection():
    # Section 4.1 scaling: Vt^H V = I, so T_1 = Vt_1^H A V_1 (no recycle space).
    A = I.convdiff(12, [10.0, 4.0]).to_scipy()
    n = A.shape[0]
    s = 10
    r = O.rbicg_pair(A, I.normal_vector(n, 1), I.normal_vector(n, 2), np.zeros(n), np.zeros(n),
                     None, k=4, s=s, tol=1e-14, max_itn=s, record=True)
    cyc = r.hist["cycles"][0]
    V, Vt = cyc["V"], cyc["Vt"]
    h = r.hist
    alpha = [None] + list(h["alpha"])
    beta = [0.0] + list(h["beta"])
    rnorm = h["rnorm"]
    T = O.T_block(range(1, s + 1), range(1, s + 1), alpha, beta, rnorm, np.float64)
    np.testing.assert_allclose(Vt.conj().T @ (A @ V), T, rtol=0, atol=1e-8 * np.abs(T).max())


# ---------------------------------------------------------------- eigen-extraction pins
def _fd1d_closed_form(N, c):
    h = 1.0 / (N + 1)
    m = np.arange(1, N + 1)
    lam = (2.0 / h ** 2) * (1.0 - np.sqrt(1.0 - (c * h / 2.0) ** 2) * np.cos(m * np.pi * h))
    a = -1.0 / h ** 2 - c / (2 * h)          # sub-diagonal
    bb = -1.0 / h ** 2 + c / (2 * h)         # super-diagonal
    j = np.arange(1, N + 1)[:, None]
    right = (np.sqrt(a / bb)) ** j * np.sin(j * m[None, :] * np.pi * h)
    left = (np.sqrt(bb / a)) ** j * np.sin(j * m[None, :] * np.pi * h)
    return lam, right, left


def test_closed_form_1d_eigenpairs():
    N, c = 30, 12.0
    A = I.convdiff(N, [c]).to_scipy().toarray()
    lam, right, left = _fd1d_closed_form(N, c)
    assert np.abs(A @ right - right * lam).max() <= 1e-9 * np.abs(A).max() * np.abs(right).max()
    assert np.abs(A.T @ left - left * lam).max() <= 1e-9 * np.abs(A).max() * np.abs(left).max()


def test_harmonic_ritz_from_invariant_subspace_is_exact():
    # eq. (harmonic1) / (finalGenEigValue): if range(Phi) contains an invariant subspace
    # of A (and range(Phit) the matching left one), the harmonic Ritz values include the
    # corresponding eigenvalues exactly and the selected vectors span that subspace.
    N, c, k = 40, 8.0, 4
    As = I.convdiff(N, [c]).to_scipy()
    lam, right, left = _fd1d_closed_form(N, c)
    rng = np.random.default_rng(1)
    Phi = np.hstack([right[:, :k] @ rng.standard_normal((k, k)), rng.standard_normal((N, 3))])
    Phit = np.hstack([left[:, :k] @ rng.standard_normal((k, k)), rng.standard_normal((N, 3))])
    L = (As.T @ Phit).T @ (As @ Phi)
    R = (As.T @ Phit).T @ Phi
    W, Wt, lams = O.eig_select(L, R, k, real_path=True)
    np.testing.assert_allclose(np.sort(lams.real), lam[:k], rtol=1e-8)
    cos = sla.svdvals(np.linalg.qr(Phi @ W)[0].T @ np.linalg.qr(right[:, :k])[0])
    assert cos.min() > 1 - 1e-8
    cos = sla.svdvals(np.linalg.qr(Phit @ Wt)[0].T @ np.linalg.qr(left[:, :k])[0])
    assert cos.min() > 1 - 1e-8


def test_first_cycle_ritz_uses_left_and_right_eigvecs_of_T1():
    # Section 4.2: T_1 w = lambda w and Tt_1 = T_1^H; left vectors of T_1 give the dual.
    rng = np.random.default_rng(2)
    T = np.diag(rng.uniform(1, 10, 8)) + np.diag(rng.standard_normal(7), 1) + np.diag(rng.standard_normal(7), -1)
    W, Wt, lams = O.eig_tridiag_select(T, 3, real_path=False)
    for i in range(W.shape[1]):
        np.testing.assert_allclose(T @ W[:, i], lams[i] * W[:, i], atol=1e-10)
        np.testing.assert_allclose(T.conj().T @ Wt[:, i], np.conj(lams[i]) * Wt[:, i], atol=1e-10)
    assert np.all(np.diff(np.abs(lams)) >= 0)


def test_select_eigs_keeps_conjugate_pairs_together():
    lam = np.array([5.0, 1 + 1j, 1 - 1j, 3.0, 0.5, 2 + 2j, 2 - 2j])
    units = O.select_eigs(lam, 4, real_path=True)
    assert units == [(4, False), (1, True)] or units == [(4, False), (2, True)]
    # a pair straddling the cut gives k-1 vectors
    units = O.select_eigs(lam, 2, real_path=True)
    assert units == [(4, False)]
    units = O.select_eigs(np.array([np.inf, 2.0, 1.0]), 2, real_path=True)
    assert units == [(2, False), (1, False)]


# ---------------------------------------------------------------- qualitative pins
def test_recycling_same_system_again_saves_iterations():
    # Section 6.1 protocol (the same dual pair solved repeatedly): the paper reports about
    # 35% fewer iterations on the second run (on a preconditioned operator).  The
    # constant-coefficient stand-in behaves the same way qualitatively.
    A = I.convdiff(32, [10.0, 10.0])
    n = A.n
    seq = [{"A": A, "b": I.normal_vector(n, 5), "bt": I.normal_vector(n, 6)}] * 3
    rs = O.rbicg_sequence(seq, k=10, s=40, tol=1e-8)
    assert all(r.status == O.STATUS_OK for r in rs)
    assert rs[1].iters <= 0.8 * rs[0].iters
    assert rs[2].iters <= 0.8 * rs[0].iters


def test_conjugate_shift_symmetry():
    # real A, real b and bt: x(conj(sigma)) = conj(x(sigma)) for (sigma I - A) x = b
    A = I.convdiff(8, [10.0, 10.0]).to_scipy()
    n = A.shape[0]
    b, bt = I.normal_vector(n, 1), I.normal_vector(n, 2)
    sig = -30.0 + 400.0j
    out = []
    for s_ in (sig, np.conj(sig)):
        M = (s_ * sp.identity(n, format="csr") - A).tocsr()
        r = O.rbicg_pair(M, b.astype(complex), bt.astype(complex), np.zeros(n, complex),
                         np.zeros(n, complex), None, k=4, s=10, tol=1e-12)
        out.append(r)
    np.testing.assert_allclose(out[1].x, np.conj(out[0].x), rtol=0, atol=1e-9 * np.linalg.norm(out[0].x))
    np.testing.assert_allclose(out[1].xt, np.conj(out[0].xt), rtol=0, atol=1e-9 * np.linalg.norm(out[0].xt))


def test_exact_invariant_subspace_deflates():
    # Section 3: with U spanning an exact invariant subspace of A (and Ut one of A^H), the
    # augmented bi-Lanczos iteration works on the deflated operator, so Algorithm 2 needs fewer
    # iterations than BiCG, and more deflated eigenvalues save more (k = 5, 10 at 48^2)
    import scipy.sparse.linalg as ssla

    pr = I.convdiff_sequence(48, [10.0, 10.0], 2, 0.01, 7, bt_kind="normal")[1]
    A = O.as_scipy(pr["A"]).tocsc()
    n = A.shape[0]
    z = np.zeros(n)
    base = O.bicg(A, pr["b"], pr["bt"], z, z, 1e-8, 5000)
    its = []
    for k in (5, 10):
        _, V = ssla.eigs(A, k=k, sigma=0.0, which="LM", v0=np.ones(n))
        _, W = ssla.eigs(A.T.conj().tocsc(), k=k, sigma=0.0, which="LM", v0=np.ones(n))
        rec = O.biorth_recycle(A, np.real(V), np.real(W), 1e-6)
        assert rec[0].shape[1] == k
        r = O.rbicg_pair(A, pr["b"], pr["bt"], z, z, recycle=rec, k=k, s=40, tol=1e-8, max_itn=5000,
                         refresh=False)
        assert r.status == O.STATUS_OK
        its.append(r.iters)
    assert its[0] < 0.95 * base.iters and its[1] < its[0], (base.iters, its)


# ---------------------------------------------------------------- refresh on iteration data
def _pairs_of(lam):
    """(first column, width) of each eigenvalue unit of eig_select's output: a complex value
    followed by its conjugate is one real-arithmetic unit of two columns (reading R5)."""
    out, i = [], 0
    while i < len(lam):
        if np.imag(lam[i]) != 0 and i + 1 < len(lam) and lam[i + 1] == np.conj(lam[i]):
            out.append((i, 2)); i += 2
        else:
            out.append((i, 1)); i += 1
    return out


def _harmonic_residuals(As, Phi, Phit, W, Wt, lam):
    """Largest relative residual of the harmonic-Ritz conditions, computed with explicit
    sparse products instead of the H_j / Gamma_j / B_j recurrences:
    primal (eq. (harmonic1)): (A u - lambda u) orthogonal to range(A^H Phit), u = Phi w;
    dual (the same definition for A^H with test space A Phi): (A^H ut - conj(lambda) ut)
    orthogonal to range(A Phi), ut = Phit wt.  A conjugate pair of a real problem is checked
    as the 2 x 2 real block it stands for."""
    AH = As.conj().T.tocsr()
    AP, AtPt = As @ Phi, AH @ Phit
    worst_p = worst_d = 0.0
    for i, w in _pairs_of(lam):
        l = lam[i]
        if w == 1:
            Lb, Lbd = np.array([[l]]), np.array([[np.conj(l)]])
        else:
            a, b = l.real, l.imag
            Lb, Lbd = np.array([[a, b], [-b, a]]), np.array([[a, -b], [b, a]])
        u, ut = Phi @ W[:, i:i + w], Phit @ Wt[:, i:i + w]
        rp = AtPt.conj().T @ (As @ u - u @ Lb)
        rd = AP.conj().T @ (AH @ ut - ut @ Lbd)
        worst_p = max(worst_p, np.linalg.norm(rp) / (np.linalg.norm(AtPt) * np.linalg.norm(As @ u)))
        worst_d = max(worst_d, np.linalg.norm(rd) / (np.linalg.norm(AP) * np.linalg.norm(AH @ ut)))
    return worst_p, worst_d


@pytest.mark.parametrize("N,c,seed", [(20, [10.0, 6.0], 1), (16, [3.0, 1.0], 2)])
def test_refresh_satisfies_harmonic_ritz_definition_on_iteration_data(N, c, seed):
    # Every refresh of a first system (Section 4.2, cycles j >= 2) and of a recycled system
    # (first cycle with C, Section 4.2; general cycle, Section 4.1), on a nonsymmetric operator
    # with an unrelated dual right-hand side, returns vectors that satisfy the harmonic-Ritz
    # conditions written with A itself.  This pins the pencil's blocks built from the iteration
    # scalars (T, Gamma, B and their duals) and the dual reading R4 (left eigenvectors of the
    # pencil).  The wrong reading Wt = W fails the dual check by more than 1e-5 on these cases.
    A = I.convdiff(N, c)
    As = A.to_scipy()
    n = A.n
    b, bt = I.normal_vector(n, seed), I.normal_vector(n, seed + 50)
    z = np.zeros(n)
    rec, checked = None, 0
    for _ in range(2):
        r = O.rbicg_pair(A, b, bt, z, z, recycle=rec, k=6, s=20, tol=1e-10, record=True, max_itn=200)
        assert r.status == O.STATUS_OK
        for cy in r.hist["cycles"]:
            blk = cy["blocks"]
            if blk is None:
                continue
            wp, wd = _harmonic_residuals(As, blk["Phi"], blk["Phit"], cy["W"], cy["Wt"], cy["lam"])
            assert wp < 1e-9 and wd < 1e-9, (cy["j"], wp, wd)
            _, wrong = _harmonic_residuals(As, blk["Phi"], blk["Phit"], cy["W"], cy["W"], cy["lam"])
            assert wrong > 1e-5
            checked += 1
        rec = O.biorth_recycle(A, r.U_next, r.Ut_next, 1e-6)
    assert checked >= 4


@pytest.mark.parametrize("dim,N", [(1, 200), (2, 24)])
def test_symmetric_case_both_sides_coincide(dim, N):
    # A symmetric (c = 0), bt = b and xt_{-1} = x_{-1}: the dual iteration repeats the primal
    # one, so Phit = Phi, Ht = H and the pencil of eq. (finalGenEigValue) is symmetric, with
    # R = Phi^T A Phi positive definite: it is the harmonic-Ritz problem of RMINRES that
    # Section 4.1 starts from.  Then at every harmonic refresh the eigenvalues are real, the
    # left eigenvectors span the right ones (Wt = W), and C_j = A Phi W, Ct_j = A Phit Wt are
    # bi-orthogonal already before the SVD of Section 4.3 (eigenvectors of a symmetric-definite
    # pencil are L-orthogonal), so the truncation keeps all k columns (p = k).  Recycling the
    # space on the same pair saves iterations (Section 6.1 protocol).
    A = I.convdiff(N, [0.0] * dim)
    As = A.to_scipy()
    n = A.n
    b = I.normal_vector(n, 3)
    z = np.zeros(n)
    k, rec, its, checked = 8, None, [], 0
    for _ in range(3):
        r = O.rbicg_pair(A, b, b.copy(), z, z, recycle=rec, k=k, s=30, tol=1e-10, record=True)
        assert r.status == O.STATUS_OK
        its.append(r.iters)
        for cy in r.hist["cycles"]:
            W, Wt, lam = cy["W"], cy["Wt"], cy["lam"]
            assert np.abs(np.imag(lam)).max() <= 1e-10 * np.abs(lam).max()
            cos = sla.svdvals(np.linalg.qr(W)[0].T @ np.linalg.qr(Wt)[0])
            assert cos.min() > 1 - 1e-10
            assert cy["U"].shape[1] == k
            blk = cy["blocks"]
            if blk is None:
                continue   # first cycle: Ritz (not harmonic) vectors of T_1
            Cj = As @ (blk["Phi"] @ W)
            Cjt = As.T @ (blk["Phit"] @ Wt)
            G = (Cjt / np.linalg.norm(Cjt, axis=0)).T @ (Cj / np.linalg.norm(Cj, axis=0))
            assert np.abs(G - np.diag(np.diag(G))).max() < (1e-4 if dim == 1 else 1e-8)
            assert np.abs(np.diag(G)).min() > 1 - 1e-8
            checked += 1
        rec = O.biorth_recycle(A, r.U_next, r.Ut_next, 1e-6)
        assert rec[0].shape[1] == k
    assert checked >= 3
    assert its[1] < 0.9 * its[0] and its[2] <= its[1], its


def test_guard_baseline_does_not_shrink_after_a_fallback():
    # The stagnation guard (not in the paper) measures recycled pairs against the full count of
    # the last pair solved from its start without a recycle space.  On this sequence pair 3
    # falls back; pair 4 keeps the same limit (a baseline taken from the continued leg alone
    # would have dropped it to 40).
    seq = I.convdiff_sequence(24, [20.0, 20.0], 5, 0.01, 4, bt_kind="normal")
    rs = O.rbicg_sequence(seq, k=6, s=20, tol=1e-8, guard=1.5)
    assert all(r.status == O.STATUS_OK for r in rs)
    limit = -(-int(1.5 * rs[0].iters) // 20) * 20
    fell = [j for j, r in enumerate(rs) if r.hist["fallback"]]
    assert fell and fell[0] < len(rs) - 1, fell
    for r in rs[1:]:
        assert r.hist["guard_limit"] == limit
        if r.hist["fallback"]:
            assert r.iters > limit


def test_refresh_every_carries_the_space_unchanged():
    # Section 6.2: a recycle space may be recomputed only for some systems of a sequence.  With
    # refresh_every = 2 the odd pairs compute no cycle refresh and hand on the space they were
    # given (the same range after the Section 4.3 rotation of their system start)
    seq = I.convdiff_sequence(24, [1.0, 1.0], 4, 0.01, 17, bt_kind="normal")
    rs = O.rbicg_sequence(seq, k=8, s=30, tol=1e-10, refresh_every=2)
    assert all(r.status == O.STATUS_OK for r in rs)
    assert rs[0].cycles > 0 and rs[2].cycles > 0 and rs[1].cycles == 0 and rs[3].cycles == 0
    for j in (1, 3):
        rec = O.biorth_recycle(seq[j]["A"], rs[j - 1].U_next, rs[j - 1].Ut_next, 1e-6)
        cos = sla.svdvals(np.linalg.qr(rs[j].U_next)[0].T @ np.linalg.qr(rec[0])[0])
        assert rs[j].U_next.shape[1] == rec[0].shape[1] and cos.min() > 1 - 1e-12


def test_breakdown_restart_continues_as_bicg_from_the_iterate():
    # The restart after a breakdown (rbicg_sequence restarts > 0; a library policy, not in the
    # paper) must be plain BiCG (Algorithm 1, the oracle's separate bicg routine) started from the
    # iterate at which the first leg broke down.  On this strongly convective operator BiCG's
    # (pt, q) falls below 1e-14 of the norms after 69 iterations; the restarted leg converges.
    A = I.convdiff(32, [30.0, 30.0])
    rng = np.random.default_rng(7)
    b, bt = rng.standard_normal(A.n), rng.standard_normal(A.n)
    z = np.zeros(A.n)
    first = O.bicg(A, b, bt, z, z, 1e-8, 5000)
    assert first.status in (O.STATUS_BREAKDOWN_RHO, O.STATUS_BREAKDOWN_PQ)
    second = O.bicg(A, b, bt, first.x, first.xt, 1e-8, 5000)
    assert second.status == O.STATUS_OK
    pr = [{"A": A, "b": b, "bt": bt}]
    no = O.rbicg_sequence(pr, k=6, s=20, tol=1e-8, max_itn=5000, restarts=0)[0]
    assert no.status == first.status and abs(no.iters - first.iters) <= 2
    got = O.rbicg_sequence(pr, k=6, s=20, tol=1e-8, max_itn=5000, restarts=1)[0]
    assert got.status == O.STATUS_OK and got.hist["fallback"]
    assert abs(got.iters - (first.iters + second.iters)) <= 3, (got.iters, first.iters, second.iters)
    assert np.linalg.norm(got.x - second.x) <= 1e-6 * np.linalg.norm(second.x)
    assert got.true_relres <= 1e-8 and got.true_relres_dual <= 1e-8


@pytest.mark.parametrize("c", [0.0, 1.0])
def test_rerun_protocol_saves_iterations_at_128(c):
    # Section 6.1 at a size nearer the workloads (128^2, k = 10, s = 40): with the dual right-hand
    # side equal to the primal one (a one-sided extraction), solving the same pair again with the
    # recycle space of the previous solve takes at least 15 % fewer iterations, and all k columns
    # survive the Section 4.3 truncation (c = 0: 375 -> 292 -> 277; c = 1: 372 -> 305 -> 294)
    A = I.convdiff(128, [c, c])
    b = I.normal_vector(A.n, 5)
    rs = O.rbicg_sequence([{"A": A, "b": b, "bt": b}] * 3, k=10, s=40, tol=1e-8, max_itn=4000)
    assert all(r.status == O.STATUS_OK for r in rs)
    assert rs[1].recycle_dim == 10 and rs[2].recycle_dim == 10
    assert rs[1].iters <= 0.85 * rs[0].iters and rs[2].iters <= 0.85 * rs[0].iters, [r.iters for r in rs]
