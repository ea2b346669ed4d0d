"""GPU tests at the workloads' full sizes (properties that hold at any size, plus what the
oracle can still compute) and edge cases of the method: degenerate right-hand sides, the
largest recycle dimension and cycle, tiny and ragged systems."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import rbicg_oracle as O  # noqa: E402
from paper_1010_0762_gb300 import inputs as I  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)
    from paper_1010_0762_gb300 import rbicg
    return rbicg


def _dev(a):
    return torch.as_tensor(np.asarray(a), device="cuda")


def _relres(A, x, b):
    return np.linalg.norm(b - A @ x) / np.linalg.norm(b)


def test_config1_sequence_matches_oracle(R):
    # 32 x 32, c0 = (10, 10), 1 % drift, 5 pairs, b ~ N(0, 1), bt = ones, k = 10, tol 1e-8.
    # Pair 0 (no recycle space) is plain BiCG and compared with the oracle; on later pairs the
    # recycled recurrence is rounding-chaotic here (a 1e-13 relative change of b moves the
    # oracle's pair-1 count from 178 to 142 and flips its guard), so they are checked by what
    # any correct solve must satisfy: convergence and the direct solution.
    import scipy.sparse.linalg as spla
    seq = I.convdiff_sequence(32, [10.0, 10.0], 5, 0.01, 1000, bt_kind="ones")
    ref0 = O.rbicg_sequence(seq[:1], k=10, s=40, tol=1e-8, guard=1.5)[0]
    n = seq[0]["A"].n
    S = R.Solver(n, k=10, s=40, tol=1e-8)
    for j, pr in enumerate(seq):
        op = R.Operator.from_csr(pr["A"])
        x = _dev(np.zeros(n)); xt = _dev(np.zeros(n))
        res = S.solve_pair(op, _dev(pr["b"]), _dev(pr["bt"]), x, xt)
        assert res["status"] in (R.OK, R.RECYCLE_EMPTY), (j, res)
        Ad = pr["A"].to_scipy()
        xh, xth = x.cpu().numpy(), xt.cpu().numpy()
        assert _relres(Ad, xh, pr["b"]) < 2e-8
        assert _relres(Ad.T.tocsr(), xth, pr["bt"]) < 2e-8
        assert np.linalg.norm(xh - spla.spsolve(Ad.tocsc(), pr["b"])) / np.linalg.norm(xh) < 1e-5
        if j == 0:
            assert abs(res["iters"] - ref0.iters) <= 3, (res["iters"], ref0.iters)
            assert np.linalg.norm(xh - ref0.x) / np.linalg.norm(ref0.x) < 1e-6


def test_config2_full_size_pairs(R):
    # 512 x 512 (n = 262144, nnz = 1308672), k = 20, s = 40, the bench's seeds: the first pair
    # is plain BiCG (no recycle space yet), so its iteration count is the oracle's BiCG count;
    # both pairs reach the tolerance in the FP64 true residual
    seq = I.convdiff_sequence(512, [10.0, 10.0], 2, 0.01, 2000, bt_kind="normal")
    n = seq[0]["A"].n
    assert n == 262144 and seq[0]["A"].nnz == 1308672
    ref0 = O.bicg(seq[0]["A"], seq[0]["b"], seq[0]["bt"], np.zeros(n), np.zeros(n), 1e-8, 5000)
    S = R.Solver(n, k=20, s=40, tol=1e-8)
    for j, pr in enumerate(seq):
        x = _dev(np.zeros(n)); xt = _dev(np.zeros(n))
        res = S.solve_pair(R.Operator.from_csr(pr["A"]), _dev(pr["b"]), _dev(pr["bt"]), x, xt)
        assert res["status"] in (R.OK, R.RECYCLE_EMPTY), (j, res)
        Ad = pr["A"].to_scipy()
        assert _relres(Ad, x.cpu().numpy(), pr["b"]) < 1.1e-8
        assert _relres(Ad.T.tocsr(), xt.cpu().numpy(), pr["bt"]) < 1.1e-8
        if j == 0:
            assert abs(res["iters"] - ref0.iters) <= max(5, 0.01 * ref0.iters), (res["iters"], ref0.iters)


def test_config3_shape_batch_residuals(R):
    # 64^3 (n = 262144, nnz = 1810432) real A shared by 8 complex shifts in conjugate pairs,
    # one batched solve; every pair meets the tolerance in its FP64 true residual
    import scipy.sparse as sp
    A = I.convdiff(64, [10.0, 10.0, 10.0], dim=3)
    n = A.n
    assert A.nnz == 1810432
    rng = np.random.default_rng(3001)
    shifts = []
    for _ in range(4):
        re, im = -(10.0 ** rng.uniform(0, 3)), rng.uniform(0, 1e3)
        shifts += [complex(re, im), complex(re, -im)]
    rp, ci, va = _dev(A.row_ptr), _dev(A.col_idx), _dev(A.val)
    hs = [R.Solver(n, dtype=R.C128, k=16, s=40, tol=1e-8) for _ in shifts]
    ops = [R.Operator(rp, ci, va, shift=sg) for sg in shifts]
    bs = [_dev(rng.standard_normal(n) + 0j) for _ in shifts]
    cs = [_dev(rng.standard_normal(n) + 0j) for _ in shifts]
    xs = [torch.zeros(n, dtype=torch.complex128, device="cuda") for _ in shifts]
    xts = [torch.zeros_like(xs[0]) for _ in shifts]
    out = R.solve_batch(hs, ops, bs, cs, xs, xts)
    Ad = A.to_scipy()
    for i, sg in enumerate(shifts):
        assert out[i]["status"] == R.OK, (i, out[i])
        M = (sg * sp.identity(n) - Ad).tocsr()
        b, c = bs[i].cpu().numpy(), cs[i].cpu().numpy()
        assert _relres(M, xs[i].cpu().numpy(), b) < 1.1e-8
        assert _relres(M.conj().T.tocsr(), xts[i].cpu().numpy(), c) < 1.1e-8


def test_config4_full_size_fp32_refined(R):
    # 1024 x 1024 (n = 1048576, nnz = 5238784), FP32-refined to 1e-10: the FP32 BiCG
    # recurrence does not converge on this operator, the handle finishes in FP64 (fallback 2),
    # and the answer meets 1e-10 in the FP64 true residual
    seq = I.convdiff_sequence(1024, [10.0, 10.0], 1, 0.005, 4000, bt_kind="normal")
    A = seq[0]["A"]
    n = A.n
    assert n == 1048576 and A.nnz == 5238784
    S = R.Solver(n, k=20, s=40, tol=1e-10, precision="fp32_refined", inner_tol=1e-5)
    x = _dev(np.zeros(n)); xt = _dev(np.zeros(n))
    res = S.solve_pair(R.Operator.from_csr(A), _dev(seq[0]["b"]), _dev(seq[0]["bt"]), x, xt)
    assert res["status"] in (R.OK, R.RECYCLE_EMPTY), res
    Ad = A.to_scipy()
    assert _relres(Ad, x.cpu().numpy(), seq[0]["b"]) < 1.1e-10
    assert _relres(Ad.T.tocsr(), xt.cpu().numpy(), seq[0]["bt"]) < 1.1e-10


def test_zero_rhs_converges_at_iteration_zero(R):
    A = I.convdiff(12, [3.0, 1.0])
    n = A.n
    S = R.Solver(n, k=4, s=10, tol=1e-8)
    x = _dev(np.zeros(n)); xt = _dev(np.zeros(n))
    res = S.solve_pair(R.Operator.from_csr(A), _dev(np.zeros(n)), _dev(np.zeros(n)), x, xt)
    assert res["status"] == R.OK and res["iters"] == 0
    assert np.all(x.cpu().numpy() == 0) and np.all(xt.cpu().numpy() == 0)


def test_one_by_one_and_ragged_tiny_systems(R):
    # n = 1 (a single equation), and grids whose n is not a multiple of 32 or 256
    for N in (1, 3, 7, 17):
        A = I.convdiff(N, [2.0, 1.0])
        n = A.n
        b, bt = I.normal_vector(n, 3), I.normal_vector(n, 4)
        S = R.Solver(n, k=2, s=4, tol=1e-12)
        x = _dev(np.zeros(n)); xt = _dev(np.zeros(n))
        res = S.solve_pair(R.Operator.from_csr(A), _dev(b), _dev(bt), x, xt)
        assert res["status"] in (R.OK, R.RECYCLE_EMPTY), (N, res)
        Ad = A.to_scipy().toarray()
        assert np.allclose(Ad @ x.cpu().numpy(), b, atol=1e-9 * np.linalg.norm(b))


def test_largest_recycle_space_and_cycle(R):
    # k = 32 (the largest recycle dimension) with s = 48 (k + s = 80, the largest pencil) over a
    # short sequence: the refreshes run at their largest sizes and every pair converges
    seq = I.convdiff_sequence(40, [1.0, 1.0], 3, 0.01, 9100, bt_kind="normal")
    n = seq[0]["A"].n
    S = R.Solver(n, k=32, s=48, tol=1e-9, setup_fp32=0)
    for j, pr in enumerate(seq):
        x = _dev(np.zeros(n)); xt = _dev(np.zeros(n))
        res = S.solve_pair(R.Operator.from_csr(pr["A"]), _dev(pr["b"]), _dev(pr["bt"]), x, xt)
        assert res["status"] in (R.OK, R.RECYCLE_EMPTY), (j, res)
        assert _relres(pr["A"].to_scipy(), x.cpu().numpy(), pr["b"]) < 2e-9
        if j > 0:
            assert res["cycles"] >= 0
    U, Ut = S.export_recycle()
    assert U.shape[1] <= 32


def _import_and_solve(R, S, A, b, bt, U, Ut, n):
    op = R.Operator.from_csr(A)
    S.update_recycle(op)
    S.import_recycle(_dev(np.ascontiguousarray(U)), _dev(np.ascontiguousarray(Ut)))
    x = _dev(np.zeros(n)); xt = _dev(np.zeros(n))
    res = S.solve_pair(op, _dev(b), _dev(bt), x, xt)
    return res, x.cpu().numpy(), xt.cpu().numpy()


def _onset(h1, h2, rtol=1e-8):
    """First index where two residual histories differ by more than rtol (len if never)."""
    d = np.abs(np.asarray(h1) - np.asarray(h2)) > rtol * np.abs(np.asarray(h2))
    return int(np.argmax(d)) if d.any() else len(d)


def test_config2_recycled_pair_two_cycles_match_oracle(R):
    # 512 x 512, k = 20, s = 40, all-FP64 refresh: pair 1 solved with the oracle's recycle space
    # (from two cycles of pair 0) on both sides, so that the recycled iteration itself is compared
    # at full size.  The system start keeps the same columns (Section 4.3) and the recurrence
    # residual norms agree element by element to 1e-8 for as long as the recurrence itself is
    # reproducible: on this unpreconditioned operator the residual grows to 1e4 ||r_0|| within a
    # few dozen iterations and BiCG then amplifies rounding.  The reference for "reproducible" is
    # the oracle run on b perturbed by 1e-13 relative, the size of the differences between two
    # correct FP64 implementations here (n-long sums in another order differ by about sqrt(n)
    # eps = 6e-14 relative; the system start's SVD and rotation add their own rounding): it departs
    # from the unperturbed oracle at some iteration m*, and the library may not depart earlier
    # than m* - 2; up to there the norms agree to 1e-8.
    seq = I.convdiff_sequence(512, [10.0, 10.0], 2, 0.01, 2000, bt_kind="normal")
    n = seq[0]["A"].n
    z = np.zeros(n)
    r0 = O.rbicg_pair(seq[0]["A"], seq[0]["b"], seq[0]["bt"], z, z, None, k=20, s=40, tol=1e-8, max_itn=80)
    rec = O.biorth_recycle(seq[1]["A"], r0.U_next, r0.Ut_next, 1e-6)
    b1 = seq[1]["b"]
    ref = O.rbicg_pair(seq[1]["A"], b1, seq[1]["bt"], z, z, rec, k=20, s=40, tol=1e-8, max_itn=80)
    m_star = 80
    for q in range(2):   # the earlier departure of two perturbations
        bp = b1 * (1.0 + 1e-13 * np.random.default_rng(9 + q).uniform(-1, 1, n))
        refp = O.rbicg_pair(seq[1]["A"], bp, seq[1]["bt"], z, z, rec, k=20, s=40, tol=1e-8, max_itn=80)
        m_star = min(m_star, _onset(refp.hist["rnorm"], ref.hist["rnorm"]))
    assert m_star >= 20, m_star
    S = R.Solver(n, k=20, s=40, tol=1e-8, max_itn=80, setup_fp32=0, guard=0.0)
    res, x, xt = _import_and_solve(R, S, seq[1]["A"], b1, seq[1]["bt"], r0.U_next, r0.Ut_next, n)
    assert res["recycle_dim"] == rec[0].shape[1] == ref.recycle_dim
    assert res["iters"] == ref.iters == 80
    hist = S.residual_history()
    rh = np.array(ref.hist["rnorm"])
    assert len(hist) == len(rh) == 81
    m_gpu = _onset(hist, rh)
    assert m_gpu >= m_star - 2, (m_gpu, m_star)
    np.testing.assert_allclose(hist[:m_star - 2], rh[:m_star - 2], rtol=1e-8, atol=0)


def test_config1_recycled_pairs_match_oracle(R):
    # 32 x 32, c0 = (10, 10), 1 % drift, bt = ones, k = 10, all-FP64 refresh.  For pairs 1..4
    # the oracle's incoming recycle space is imported, so each recycled pair is compared on its
    # own (the full sequence is rounding-chaotic, see above): columns kept by the system start and
    # the first two cycles' residual norms element by element up to the oracle's own
    # reproducibility bound.  The recycled recurrences of this sequence do not reach 1e-12 (the
    # oracle stalls or breaks down at that tolerance), so the full solves run at the benchmark's
    # tolerance 1e-8 with the stagnation guard, like the oracle's sequence, and are compared with
    # the direct solution (kappa(A) is about 440).
    import scipy.sparse.linalg as spla
    seq = I.convdiff_sequence(32, [10.0, 10.0], 5, 0.01, 1000, bt_kind="ones")
    n = seq[0]["A"].n
    z = np.zeros(n)
    refs = O.rbicg_sequence(seq, k=10, s=40, tol=1e-8, guard=1.5)
    compared = 0
    for j in range(1, 5):
        U, Ut = refs[j - 1].U_next, refs[j - 1].Ut_next
        if U is None or U.shape[1] == 0:
            continue   # the previous pair handed on no space (a guard fallback leg without a cycle)
        compared += 1
        pr = seq[j]
        rec = O.biorth_recycle(pr["A"], U, Ut, 1e-6)
        two = O.rbicg_pair(pr["A"], pr["b"], pr["bt"], z, z, rec, k=10, s=40, tol=1e-12, max_itn=80)
        S = R.Solver(n, k=10, s=40, tol=1e-12, max_itn=80, setup_fp32=0, guard=0.0)
        res, _, _ = _import_and_solve(R, S, pr["A"], pr["b"], pr["bt"], U, Ut, n)
        assert res["recycle_dim"] == rec[0].shape[1], (j, res)
        h, rh = S.residual_history(), np.array(two.hist["rnorm"])
        assert len(h) == len(rh), (j, len(h), len(rh))
        # the same reproducibility bound as at 512^2 (see above)
        # where the departure starts depends on where the perturbation lands: the earliest of four
        # (at this size the library's own system start, an SVD and rotation of the imported space,
        # differs from the oracle's by more than the b perturbation: the library is required to
        # reproduce three quarters of the oracle's reproducible window)
        m_star = 80
        for q in range(4):
            bp = pr["b"] * (1.0 + 1e-13 * np.random.default_rng(100 * q + j).uniform(-1, 1, n))
            twop = O.rbicg_pair(pr["A"], bp, pr["bt"], z, z, rec, k=10, s=40, tol=1e-12, max_itn=80)
            m_star = min(m_star, _onset(twop.hist["rnorm"], rh))
        assert m_star >= 10 and _onset(h, rh) >= 0.75 * m_star, (j, _onset(h, rh), m_star)
        S2 = R.Solver(n, k=10, s=40, tol=1e-8, setup_fp32=0, guard=1.5)
        # pair 0 first, so that the guard has the oracle's baseline (pair 0's plain count)
        _import_and_solve(R, S2, seq[0]["A"], seq[0]["b"], seq[0]["bt"], U[:, :0], Ut[:, :0], n)
        res2, x, xt = _import_and_solve(R, S2, pr["A"], pr["b"], pr["bt"], U, Ut, n)
        assert refs[j].status == O.STATUS_OK and res2["status"] in (R.OK, R.RECYCLE_EMPTY), (j, res2)
        Ad = pr["A"].to_scipy().tocsc()
        for a, b_, M in ((x, pr["b"], Ad), (xt, pr["bt"], Ad.T.tocsc())):
            xs = spla.spsolve(M, b_)
            assert np.abs(a - xs).max() <= 1e-5 * np.abs(xs).max(), j
    assert compared >= 2


def test_fp32_refined_fallback_reaches_tol_in_the_true_residual(R):
    # 512 x 512 at tol 1e-10: the FP32 inner recurrence cannot reduce this residual (BiCG's
    # residual peaks), so the handle falls back to FP64 correction solves inside the refinement
    # loop.  The refined iterate must meet tol in the true residual, primal and dual, checked here
    # with SciPy's own products, whatever the FP64 form's recurrence-stopped solve reaches.
    seq = I.convdiff_sequence(512, [10.0, 10.0], 1, 0.01, 2000, bt_kind="normal")
    A, b, bt = seq[0]["A"], seq[0]["b"], seq[0]["bt"]
    n = A.n
    As = A.to_scipy()
    S = R.Solver(n, k=20, s=40, tol=1e-10, precision="fp32_refined", setup_fp32=0)
    x, xt = _dev(np.zeros(n)), _dev(np.zeros(n))
    res = S.solve_pair(R.Operator.from_csr(A), _dev(b), _dev(bt), x, xt)
    assert res["fallback"] == 2 and res["status"] == R.OK, res
    xr, xtr = x.cpu().numpy(), xt.cpu().numpy()
    assert _relres(As, xr, b) <= 1.01e-10
    assert _relres(As.T.tocsr(), xtr, bt) <= 1.01e-10
    assert abs(res["true_relres"] - _relres(As, xr, b)) <= 1e-12
