"""Pins of the IRKA (Algorithm 3) and bilinear-form oracle (CPU only).

Each test checks the oracle against what the mathematics fixes: the exact value u^H A^{-1} w of a
bilinear form and the quadratic error identity of the corrected estimate (Section 1); the
Hermite interpolation theorem of Section 5.1 (the reduced model of eq. (red_projection) matches
G and G' at every shift); the fixed point of IRKA (at convergence the shifts are the mirror
images of the reduced poles, the first-order H2 conditions of Section 5.1); and that the shifted
solves of Algorithm 2 with each recycling strategy of Section 5.3 reproduce the direct solves.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import irka_oracle as IR
from oracle import rbicg_oracle as O
from paper_1010_0762_gb300 import inputs as I


def _problem(N, c, dim=2, seed=3000):
    A = I.convdiff(N, [c] * dim, dim=dim)
    rng = np.random.default_rng(seed)
    return A, rng.standard_normal(A.n), rng.standard_normal(A.n)


# ---------------------------------------------------------------- bilinear forms (Section 1)
def test_bilinear_forms_equal_the_exact_value_for_exact_solutions():
    rng = np.random.default_rng(4)
    n = 48
    Ad = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.sqrt(n) * np.eye(n)
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    exact = np.vdot(u, np.linalg.solve(Ad, w))
    x = np.linalg.solve(Ad, w)
    xt = np.linalg.solve(Ad.conj().T, u)
    for est in IR.bilinear_forms(Ad, u, w, x, xt):
        assert abs(est - exact) <= 1e-12 * abs(exact)


def test_bilinear_corrected_error_is_quadratic_in_the_residuals():
    # u^H A^{-1} w - (u^H x + xt^H (w - A x)) = (u - A^H xt)^H A^{-1} (w - A x) for any x, xt
    A = I.convdiff(10, [10.0, 3.0]).to_scipy().toarray()
    n = A.shape[0]
    rng = np.random.default_rng(5)
    u, w = rng.standard_normal(n), rng.standard_normal(n)
    xs, xts = np.linalg.solve(A, w), np.linalg.solve(A.T, u)
    exact = u @ xs
    errs = []
    for eps in (1e-3, 1e-5):
        x = xs + eps * rng.standard_normal(n) * np.abs(xs).max()
        xt = xts + eps * rng.standard_normal(n) * np.abs(xts).max()
        p, d, corr = IR.bilinear_forms(A, u, w, x, xt)
        r, rt = w - A @ x, u - A.T @ xt
        assert abs((exact - corr) - rt @ np.linalg.solve(A, r)) <= 1e-9 * abs(exact)
        errs.append((abs(exact - p), abs(exact - corr)))
    # primal error linear in eps, corrected error quadratic
    assert errs[1][0] < 3e-2 * errs[0][0] and errs[1][1] < 3e-4 * errs[0][1]


# ---------------------------------------------------------------- reduced model and IRKA
def test_shift_order_and_conjugate_closure():
    s = np.array([3 + 4j, 1.0, 3 - 4j, -2 + 0j])
    assert [s[i] for i in IR.order_shifts(s)] == [1.0, -2 + 0j, 3 + 4j, 3 - 4j]
    lam = np.array([5 + 1e-9j, 2 + 3j, 2 - 3.0000001j, 7 - 1e-8j])
    out = IR.conjugate_close(lam)
    assert out[0] == 5.0 and out[3] == 7.0
    assert out[1] == np.conj(out[2]) and abs(out[1] - (2 + 3.00000005j)) < 1e-12


def test_reduced_model_interpolates_at_every_shift():
    # Theorem of Section 5.1 (Hermite interpolation by projection): G_r(sigma_i) = G(sigma_i) and
    # G_r'(sigma_i) = G'(sigma_i) for V, W of eq. (eqn:VrWr) and the model of eq. (red_projection)
    A, b, c = _problem(9, 10.0)
    sh = I.irka_shifts(6, 3001)
    V, W, _ = IR.direct_solver(A, b, c)(list(sh), 0)
    Ar, Er, br, cr = IR.reduced_model(A, V, W, b, c)
    for sg in sh:
        g, gp = IR.transfer(A, b, c, sg)
        gr, grp = IR.transfer_reduced(Ar, Er, br, cr, sg)
        assert abs(g - gr) <= 1e-8 * abs(g) and abs(gp - grp) <= 1e-7 * abs(gp)
    # a wrong reading of the listing's E_r (W^H A V) breaks it
    gr_bad, _ = IR.transfer_reduced(Ar, Ar, br, cr, sh[0])
    assert abs(IR.transfer(A, b, c, sh[0])[0] - gr_bad) > 1e-3 * abs(gr_bad)


def test_irka_converges_to_its_fixed_point():
    # Algorithm 3 on a symmetric operator with real initial shifts: at convergence the shifts are
    # the mirror images of the reduced model's poles, and the model interpolates G there (the
    # first-order H2-optimality conditions of Section 5.1)
    A, b, c = _problem(10, 0.0)
    sh = -np.array([30.0, 300.0, 3000.0, 30000.0])
    res = IR.irka(A, b, c, sh, IR.direct_solver(A, b, c), max_steps=60, shift_tol=1e-10)
    assert res["converged"], res["change"]
    m = res["model"]
    poles = sla.eig(m["Ar"], m["Er"], right=False)
    mirror = np.sort(-poles.real)
    np.testing.assert_allclose(np.sort(res["shifts"].real), mirror, rtol=1e-8)
    for sg in res["shifts"]:
        g, gp = IR.transfer(A, b, c, sg)
        gr, grp = IR.transfer_reduced(m["Ar"], m["Er"], m["br"], m["cr"], sg)
        assert abs(g - gr) <= 1e-7 * abs(g) and abs(gp - grp) <= 1e-6 * abs(gp)


@pytest.mark.parametrize("strategy", [0, 1, 2, 3, 4])
def test_rbicg_solves_reproduce_direct_irka(strategy):
    # the shifted dual solves of Algorithm 3 by Algorithm 2 (with each recycling strategy of
    # Section 5.3) give the shifts of direct solves at every step
    A, b, c = _problem(12, 10.0)
    sh = I.irka_shifts(4, 3001)
    ref = IR.irka(A, b, c, sh, IR.direct_solver(A, b, c), max_steps=4, shift_tol=1e-14)
    res = IR.irka(A, b, c, sh, IR.rbicg_solver(A, b, c, k=8, s=20, tol=1e-12, strategy=strategy),
                  max_steps=4, shift_tol=1e-14)
    for h1, h2 in zip(res["history"], ref["history"]):
        assert np.max(np.abs(h1 - h2) / np.abs(h2)) < 1e-8


def test_irka_recycling_saves_iterations():
    # Section 5.3, strategy 1 (the paper's choice): recycling each shift index's space into the
    # next IRKA step needs fewer iterations than BiCG once the shifts settle
    A, b, c = _problem(12, 10.0)
    sh = I.irka_shifts(8, 3001)
    its = {}
    for strategy in (0, 1, 4):
        res = IR.irka(A, b, c, sh, IR.rbicg_solver(A, b, c, k=8, s=20, tol=1e-10, strategy=strategy),
                      max_steps=6, shift_tol=1e-14)
        its[strategy] = sum(sum(x) for x in res["iters"][1:])
    # strategy 4: one space shared by the shifts (E = I), computed by one solve per step, saves
    # about as much
    assert its[1] < 0.9 * its[0] and its[4] < 0.9 * its[0], its
