"""Component parity on the GPU: each step of the hot path, called through the C ABI, against
plain NumPy / SciPy CPU arithmetic on the same seeded inputs."""
import numpy as np
import pytest
import scipy.linalg as sla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1010_0762_gb300 import inputs as I  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_0762_gb300 import rbicg
    return rbicg


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _matrices():
    yield "convdiff2d", I.convdiff(23, [10.0, 7.0]), None
    yield "convdiff3d", I.convdiff(9, [10.0, 10.0, 10.0]), None
    yield "ragged", I.random_csr(777, 5, 3, empty_rows=(0, 5, 776), long_row=100), None
    yield "complex", I.random_csr(513, 4, 4, complex_=True, empty_rows=(7,)), None
    yield "shifted", I.convdiff(17, [10.0, 10.0]), -30.0 + 400.0j


@pytest.mark.parametrize("case", ["convdiff2d", "convdiff3d", "ragged", "complex", "shifted"])
@pytest.mark.parametrize("k", [0, 5, 20])
def test_dual_spmv_project(R, case, k):
    name, A, shift = [m for m in _matrices() if m[0] == case][0]
    n = A.n
    As = A.to_scipy()
    cx = np.iscomplexobj(A.val) or shift is not None
    if shift is not None:
        Op = (shift * __import__("scipy.sparse", fromlist=["x"]).identity(n, format="csr") - As).tocsr()
    else:
        Op = As
    rng = np.random.default_rng(7)
    def vec():
        v = rng.standard_normal(n)
        return v + 1j * rng.standard_normal(n) if cx else v
    r, rt, po, pto = vec(), vec(), vec(), vec()
    beta = (0.3 - 0.2j) if cx else 0.7
    Cm = np.array([vec() for _ in range(k)]).T if k else None
    Ctm = np.array([vec() for _ in range(k)]).T if k else None
    Dc = rng.uniform(0.5, 2.0, k) if k else None
    op = R.Operator.from_csr(A, shift=shift)
    p, pt, z, zt, ze, zet = R.op_dual_spmv_project(op, _dev(r), _dev(rt), _dev(po), _dev(pto), beta,
                                                   _dev(Cm) if k else None, _dev(Ctm) if k else None, Dc)
    p_ref = r + beta * po
    pt_ref = rt + np.conj(beta) * pto
    z_ref = Op @ p_ref
    zt_ref = Op.conj().T @ pt_ref
    tol = 1e-13
    np.testing.assert_allclose(p.cpu().numpy(), p_ref, rtol=0, atol=tol * np.abs(p_ref).max())
    np.testing.assert_allclose(pt.cpu().numpy(), pt_ref, rtol=0, atol=tol * np.abs(pt_ref).max())
    np.testing.assert_allclose(z.cpu().numpy(), z_ref, rtol=0, atol=tol * abs(Op).max() * np.abs(p_ref).max() * 8)
    np.testing.assert_allclose(zt.cpu().numpy(), zt_ref, rtol=0, atol=tol * abs(Op).max() * np.abs(pt_ref).max() * 8)
    if k:
        ze_ref = (Ctm.conj().T @ z_ref) / Dc
        zet_ref = (Cm.conj().T @ zt_ref) / Dc
        np.testing.assert_allclose(ze, ze_ref, rtol=1e-11, atol=1e-11 * np.abs(ze_ref).max())
        np.testing.assert_allclose(zet, zet_ref, rtol=1e-11, atol=1e-11 * np.abs(zet_ref).max())


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("shape", [(1000, 7, 9), (70001, 82, 102), (513, 176, 40)])
def test_gram(R, cx, fp32, shape):
    n, mx, my = shape
    rng = np.random.default_rng(1)
    X = rng.standard_normal((n, mx)) + (1j * rng.standard_normal((n, mx)) if cx else 0)
    Y = rng.standard_normal((n, my)) + (1j * rng.standard_normal((n, my)) if cx else 0)
    G = R.op_gram(_dev(X), _dev(Y), fp32=fp32)
    ref = X.conj().T @ Y
    scale = np.sqrt(np.outer((abs(X) ** 2).sum(0), (abs(Y) ** 2).sum(0)))
    err = (abs(G - ref) / scale).max()
    assert err < (2e-6 if fp32 else 1e-13), err


def _pencil(m, seed, cx):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((m, m)) + (1j * rng.standard_normal((m, m)) if cx else 0)
    Rm = rng.standard_normal((m, m)) + (1j * rng.standard_normal((m, m)) if cx else 0) + 4 * np.eye(m)
    return L, Rm


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("m,k", [(12, 4), (60, 20), (80, 32)])
def test_eig_select_pencil(R, cx, m, k):
    L, Rm = _pencil(m, 10 + m, cx)
    W, Wt, lam = R.op_eig_select(L, Rm, k)
    ref = sla.eigvals(L, Rm)
    ref = ref[np.isfinite(ref)]
    order = np.sort(abs(ref))
    q = W.shape[1]
    assert q in (k, k - 1)
    # the selected eigenvalues are the q closest to the origin
    np.testing.assert_allclose(np.sort(abs(lam)), order[:q], rtol=1e-9)
    # right / left eigen-relations of each selected (complex) eigenpair
    if cx:
        for i in range(q):
            w, wt = W[:, i], Wt[:, i]
            assert np.linalg.norm(L @ w - lam[i] * (Rm @ w)) < 1e-9 * np.linalg.norm(L) * np.linalg.norm(w)
            assert np.linalg.norm(wt.conj() @ L - lam[i] * (wt.conj() @ Rm)) < 1e-9 * np.linalg.norm(L) * np.linalg.norm(wt)
    else:
        # real path: the columns span the real invariant subspace of the selected eigenvalues
        assert np.isrealobj(W) and np.isrealobj(Wt)
        M = np.linalg.solve(Rm, L)
        Q = np.linalg.qr(W)[0]
        assert np.linalg.norm(M @ Q - Q @ (Q.T @ M @ Q)) < 1e-8 * np.linalg.norm(M)
        Ml = np.linalg.solve(Rm.T, L.T)      # left vectors of (L, R): W~^T L = Lam W~^T R
        Qt = np.linalg.qr(Wt)[0]
        assert np.linalg.norm(Ml @ Qt - Qt @ (Qt.T @ Ml @ Qt)) < 1e-8 * np.linalg.norm(Ml)


def test_eig_select_tridiagonal_standard(R):
    # Section 4.2: T_1 w = lambda w, left vectors from T_1^H; compare to scipy
    rng = np.random.default_rng(5)
    s = 40
    T = np.diag(rng.uniform(1, 50, s)) + np.diag(rng.standard_normal(s - 1), 1) + np.diag(rng.standard_normal(s - 1), -1)
    W, Wt, lam = R.op_eig_select(T, None, 10)
    ref = np.sort(abs(sla.eigvals(T)))
    np.testing.assert_allclose(np.sort(abs(lam)), ref[:W.shape[1]], rtol=1e-10)
    Q = np.linalg.qr(W)[0]
    assert np.linalg.norm(T @ Q - Q @ (Q.T @ T @ Q)) < 1e-9 * np.linalg.norm(T)


def test_eig_select_closed_form_1d(R):
    # closed-form eigenvalues of the 1-D convection-diffusion matrix (order 60)
    N, c = 60, 20.0
    A = I.convdiff(N, [c]).to_scipy().toarray()
    h = 1.0 / (N + 1)
    lam_ref = (2 / h ** 2) * (1 - np.sqrt(1 - (c * h / 2) ** 2) * np.cos(np.arange(1, N + 1) * np.pi * h))
    W, Wt, lam = R.op_eig_select(A, None, 8)
    np.testing.assert_allclose(np.sort(lam.real), lam_ref[:8], rtol=1e-9)


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("k", [1, 7, 20, 32])
def test_svd(R, cx, k):
    rng = np.random.default_rng(k)
    S = rng.standard_normal((k, k)) + (1j * rng.standard_normal((k, k)) if cx else 0)
    M, sig, N = R.op_svd(S)
    ref = np.linalg.svd(S, compute_uv=False)
    np.testing.assert_allclose(sig, ref, rtol=1e-12, atol=1e-13 * ref[0])
    np.testing.assert_allclose(M @ np.diag(sig) @ N.conj().T, S, atol=1e-12 * ref[0])
    np.testing.assert_allclose(M.conj().T @ M, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(N.conj().T @ N, np.eye(k), atol=1e-12)
