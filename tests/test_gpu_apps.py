"""GPU parity of what the paper builds on solved dual pairs, through the C ABI: bilinear forms
u^H A^{-1} w (Section 1) and IRKA (Algorithm 3, Section 5) with the recycling strategies of
Section 5.3, against the CPU oracle (oracle/irka_oracle.py)."""
import numpy as np
import pytest
import torch

from oracle import irka_oracle as IR
from oracle import rbicg_oracle as O
from paper_1010_0762_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_0762_gb300 import rbicg
    return rbicg


def _dev(a, cx=False):
    a = np.asarray(a)
    if cx:
        a = a.astype(np.complex128)
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("case", ["real", "shifted_complex"])
def test_bilinear_form_matches_oracle(R, case):
    # a dual pair solved by the library, then u^H Op^{-1} w three ways (primal, dual, corrected);
    # the library's sums equal the oracle's on the same x, xt, and the corrected estimate is exact
    # to the product of the two residuals
    A = I.convdiff(40, [10.0, 4.0])
    n = A.n
    cx = case != "real"
    shift = -50.0 + 300.0j if cx else None
    u, w = I.normal_vector(n, 21, complex_=cx), I.normal_vector(n, 22, complex_=cx)
    S = R.Solver(n, dtype=R.C128 if cx else R.R64, k=8, s=20, tol=1e-8)
    op = R.Operator.from_csr(A, shift=shift)
    x, xt = _dev(np.zeros(n), cx), _dev(np.zeros(n), cx)
    res = S.solve_pair(op, _dev(w, cx), _dev(u, cx), x, xt)
    assert res["status"] == R.OK
    got = R.bilinear_form(op, _dev(u, cx), _dev(w, cx), x, xt)
    M = A.to_scipy()
    if cx:
        import scipy.sparse as sp
        M = (shift * sp.identity(n, format="csr") - M).tocsr()
    ref = IR.bilinear_forms(M, u, w, x.cpu().numpy(), xt.cpu().numpy())
    for g, r in zip(got, ref):
        assert abs(g - r) <= 1e-12 * abs(r), (g, r)
    Md = M.toarray()
    exact = np.vdot(u, np.linalg.solve(Md, w))
    bound = np.linalg.norm(u - Md.conj().T @ xt.cpu().numpy()) * np.linalg.norm(w - Md @ x.cpu().numpy()) \
        / np.linalg.svd(Md, compute_uv=False)[-1]
    assert abs(got[2] - exact) <= 1.01 * bound + 1e-14 * abs(exact)
    assert abs(got[0] - exact) <= 1e-6 * abs(exact)


def _irka_problem(N=12, c=10.0, r=4):
    A = I.convdiff(N, [c, c])
    rng = np.random.default_rng(3000)
    b, cvec = rng.standard_normal(A.n), rng.standard_normal(A.n)
    return A, b, cvec, I.irka_shifts(r, 3001)


@pytest.mark.parametrize("strategy,batched", [(1, 1), (1, 0), (0, 1), (2, 0), (3, 0), (4, 1)])
def test_irka_matches_oracle(R, strategy, batched):
    # Algorithm 3 with the library's RBiCG solves (tol 1e-12) against the oracle's Algorithm 3
    # with direct solves: the shifts after every step and the last reduced model agree
    A, b, c, sh = _irka_problem()
    op = R.Operator.from_csr(A)
    for steps in (1, 3):
        ref = IR.irka(A, b, c, sh, IR.direct_solver(A, b, c), max_steps=steps, shift_tol=1e-14)
        got = R.irka(op, _dev(b), _dev(c), sh, max_steps=steps, shift_tol=1e-14, strategy=strategy,
                     batched=batched, solver_k=8, solver_s=20, solver_tol=1e-12, solver_setup_fp32=0)
        assert got["steps"] == steps and got["failed_solves"] == 0
        assert np.max(np.abs(got["shifts"] - ref["shifts"]) / np.abs(ref["shifts"])) < 1e-8
        m = ref["model"]
        np.testing.assert_allclose(got["model_shifts"], m["shifts"], rtol=1e-8)
        for key in ("Ar", "Er", "br", "cr"):
            np.testing.assert_allclose(got[key], m[key], rtol=0, atol=1e-7 * np.abs(m[key]).max())


def test_irka_recycling_counts_match_oracle_and_save_iterations(R):
    # strategies 1 and 4 (Section 5.3; 4: one space shared by the shifts) through the batched
    # launch: per-solve iteration counts follow the oracle's Algorithm 2 with the same strategy, and
    # recycling needs fewer iterations than BiCG
    A, b, c, sh = _irka_problem(r=8)
    op = R.Operator.from_csr(A)
    tot = {}
    for strategy in (0, 1, 4):
        got = R.irka(op, _dev(b), _dev(c), sh, max_steps=5, shift_tol=1e-14, strategy=strategy, conj_pairs=0,
                     solver_k=8, solver_s=20, solver_tol=1e-10, solver_setup_fp32=0)
        ref = IR.irka(A, b, c, sh, IR.rbicg_solver(A, b, c, k=8, s=20, tol=1e-10, strategy=strategy),
                      max_steps=5, shift_tol=1e-14)
        its, rits = np.array(got["iters"]), np.array(ref["iters"])
        assert its.shape == rits.shape
        assert np.all(np.abs(its - rits) <= np.maximum(3, 0.05 * rits)), (its, rits)
        tot[strategy] = its[1:].sum()
    assert tot[1] < 0.9 * tot[0] and tot[4] < 0.9 * tot[0], tot


def test_irka_refresh_every_keeps_spaces_between_refreshes(R):
    # Section 6.2: recycle spaces recomputed only every second step; the shifts are unchanged
    # (solves are to tolerance either way)
    A, b, c, sh = _irka_problem()
    op = R.Operator.from_csr(A)
    a1 = R.irka(op, _dev(b), _dev(c), sh, max_steps=4, shift_tol=1e-14, refresh_every=1, solver_k=8,
                solver_s=20, solver_tol=1e-12, solver_setup_fp32=0)
    a2 = R.irka(op, _dev(b), _dev(c), sh, max_steps=4, shift_tol=1e-14, refresh_every=2, solver_k=8,
                solver_s=20, solver_tol=1e-12, solver_setup_fp32=0)
    np.testing.assert_allclose(a2["shifts"], a1["shifts"], rtol=1e-8)
    assert a2["failed_solves"] == 0


def test_irka_conjugate_pairs_solved_once(R):
    # real A, b, c: (conj(sigma) I - A)^{-1} b = conj((sigma I - A)^{-1} b) and the same for the dual,
    # so solving one shift of each conjugate pair gives the shifts and reduced model of the oracle's
    # direct solves with fewer iterations (r = 4: two pairs at the start, one pair and two real shifts
    # after the first step, so 2 + 3 + 3 of 12 solves).  A larger r on this n = 144 problem leaves
    # E_r near singular (cond ~ 3e10 at r = 8), where solves at 1e-12 already move the shifts.
    A, b, c, sh = _irka_problem(r=4)
    op = R.Operator.from_csr(A)
    ref = IR.irka(A, b, c, sh, IR.direct_solver(A, b, c), max_steps=3, shift_tol=1e-14)
    kw = dict(max_steps=3, shift_tol=1e-14, strategy=1, solver_k=8, solver_s=20, solver_tol=1e-12,
              solver_setup_fp32=0)
    full = R.irka(op, _dev(b), _dev(c), sh, conj_pairs=0, **kw)
    half = R.irka(op, _dev(b), _dev(c), sh, conj_pairs=1, **kw)
    m = ref["model"]
    for got in (full, half):
        assert np.max(np.abs(got["shifts"] - ref["shifts"]) / np.abs(ref["shifts"])) < 1e-8
        for key in ("Ar", "Er", "br", "cr"):
            np.testing.assert_allclose(got[key], m[key], rtol=0, atol=1e-7 * np.abs(m[key]).max())
    assert half["total_iters"] <= 0.75 * full["total_iters"], (half["total_iters"], full["total_iters"])
