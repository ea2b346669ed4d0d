"""Plain CPU oracle of IRKA (Algorithm 3) and of bilinear forms u^H A^{-1} w.

ORACLE / TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import this module.  It shares no code with the CUDA library.

Paper: Ahuja, de Sturler, Gugercin, Chang, "Recycling BiCG with an application to model
reduction" (arXiv:1010.0762).

  * bilinear_forms -- Section 1: u^H A^{-1} w from a solved dual pair A x = w, A^H xt = u; the
                      corrected estimate u^H x + xt^H (w - A x) has the error
                      (u - A^H xt)^H A^{-1} (w - A x), quadratic in the two residuals.
  * reduced_model  -- eq. (red_projection): E_r = W^H E V, A_r = W^H A V, b_r = W^H b,
                      c_r = V^H c, here with E = I.
  * irka           -- Algorithm 3 for G(s) = c^H (s I - A)^{-1} b: V_r and W_r from the dual
                      shifted solves (sigma_i I - A) v_i = b, (sigma_i I - A)^H w_i = c, then
                      sigma_i <- -lambda_i(A_r, E_r) until the shifts stop moving.
  * direct_solver / rbicg_solver -- the solves of Algorithm 3 steps 2-4: dense or sparse direct
                      (scipy), or Algorithm 2 with the recycling strategies of Section 5.3.

Readings where the paper is silent or garbled (listed in the design notes):
  R12 Algorithm 3 writes E_r = W_r^* A V_r and c_r = V_r^* c_r; by eq. (red_projection) they
      read E_r = W_r^* E V_r and c_r = V_r^* c.
  R14 "appropriately ordered" shifts (Section 5.3): ascending modulus, and of two shifts of
      equal modulus the one with the larger imaginary part first (a conjugate pair is then
      adjacent, + before -).
  R15 for real A, b, c a shift set closed under conjugation stays closed in exact arithmetic;
      rounding in lambda(A_r, E_r) is removed: an eigenvalue whose nearest other eigenvalue to
      its conjugate lies closer to that conjugate than the eigenvalue lies to the real axis is
      paired with it (both replaced by the mean of one and the conjugate of the other); an
      eigenvalue without such a partner is replaced by its real part.
  R16 convergence: max_i |sigma_i(new) - sigma_i| / |sigma_i| < shift_tol (Section 6.2 uses
      1e-6), both sets in the order of R14.
  R17 strategy 3 of Section 5.3: for shift i of step m+1 the pool is the spaces of the systems
      solved for sigma^(m)_1..r and sigma^(m+1)_1..i-1; the space of the pool shift with the
      smallest relative change |sigma - sigma'| / |sigma| is used when that change is below
      pool_tol, else the system is solved without one.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import rbicg_oracle as O


def bilinear_forms(A, u, w, x, xt):
    """(u^H x, xt^H w, u^H x + xt^H (w - A x)) for a solved pair A x = w, A^H xt = u."""
    A = O.as_scipy(A)
    r = w - A @ x
    return np.vdot(u, x), np.vdot(xt, w), np.vdot(u, x) + np.vdot(xt, r)


def order_shifts(sig):
    """Indices that put the shifts in the order of reading R14."""
    sig = np.asarray(sig, dtype=complex)
    return sorted(range(len(sig)), key=lambda i: (abs(sig[i]), -sig[i].imag, sig[i].real))


def conjugate_close(lam):
    """Reading R15: make a set of eigenvalues of a real-coefficient pencil closed under
    conjugation (removing rounding)."""
    lam = np.asarray(lam, dtype=complex).copy()
    out = np.empty_like(lam)
    done = np.zeros(len(lam), bool)
    for i in range(len(lam)):
        if done[i]:
            continue
        cand = [j for j in range(len(lam)) if not done[j] and j != i
                and abs(lam[j] - np.conj(lam[i])) < abs(lam[i].imag)]
        if not cand:
            out[i] = lam[i].real
            done[i] = True
            continue
        j = min(cand, key=lambda q: abs(lam[q] - np.conj(lam[i])))
        m = 0.5 * (lam[i] + np.conj(lam[j]))
        out[i], out[j] = m, np.conj(m)
        done[i] = done[j] = True
    return out


def reduced_model(A, V, W, b, c):
    """eq. (red_projection) with E = I (reading R12)."""
    A = O.as_scipy(A)
    WH = W.conj().T
    return WH @ (A @ V), WH @ V, WH @ b, V.conj().T @ c


def transfer(A, b, c, s):
    """G(s) = c^H (s I - A)^{-1} b and G'(s) = -c^H (s I - A)^{-2} b (dense, small n)."""
    A = np.asarray(O.as_scipy(A).todense()) if sp.issparse(O.as_scipy(A)) else np.asarray(A)
    M = s * np.eye(A.shape[0]) - A
    y = np.linalg.solve(M, b.astype(complex))
    return np.vdot(c, y), -np.vdot(c, np.linalg.solve(M, y))


def transfer_reduced(Ar, Er, br, cr, s):
    """G_r(s) = c_r^H (s E_r - A_r)^{-1} b_r and its derivative."""
    M = s * Er - Ar
    y = np.linalg.solve(M, br)
    return np.vdot(cr, y), -np.vdot(cr, np.linalg.solve(M, Er @ y))


def direct_solver(A, b, c):
    """Solves of Algorithm 3 by scipy's sparse direct solver: solve(shifts, step) -> (V, W, iters)."""
    A = O.as_scipy(A).tocsc()
    n = A.shape[0]
    I = sp.identity(n, format="csc")

    def solve(shifts, step):
        V = np.zeros((n, len(shifts)), complex)
        W = np.zeros((n, len(shifts)), complex)
        for i, sg in enumerate(shifts):
            M = (sg * I - A).tocsc()
            V[:, i] = spla.spsolve(M, b.astype(complex))
            W[:, i] = spla.spsolve(M.conj().T.tocsc(), c.astype(complex))
        return V, W, [0] * len(shifts)
    return solve


def rbicg_solver(A, b, c, k=10, s=40, tol=1e-10, max_itn=20000, svd_tol=1e-6, strategy=1, recycle_count=0,
                 refresh_every=1, pool_tol=0.5):
    """Solves of Algorithm 3 by Algorithm 2 with the recycling strategies of Section 5.3.

    strategy 0: no recycling (BiCG); 1: the space of shift index i carries to index i of the next
    step; 2: within a step each solve passes its space to the next shift index (and the last to
    the first index of the next step); 3: pooled (reading R17); 4: one space shared by all shifts
    (E = I, Section 5.3: sigma_i I - A share A's eigenvectors, so approximate invariant subspaces of
    one shifted operator serve every shift): the solve of shift index 0 (smallest modulus) computes
    the space, every shift of the next step uses it, the others compute none.  Only the recycle_count shift
    indices of smallest modulus recycle (0: all).  New spaces are computed only on steps m with
    m % refresh_every == 0 (Section 6.2); on other steps a space is used and carried unchanged.
    Each solve starts from the previous step's solution for the same index (Section 6.2)."""
    A = O.as_scipy(A)
    n = A.shape[0]
    Id = sp.identity(n, format="csr")
    state = {"spaces": {}, "prev_x": {}, "prev_xt": {}, "pool": [], "chain": None}

    def one(i, sg, step, rec_in, refresh_ok=True):
        M = (sg * Id - A).tocsr()
        x0 = state["prev_x"].get(i, np.zeros(n, complex))
        xt0 = state["prev_xt"].get(i, np.zeros(n, complex))
        use = strategy > 0 and (recycle_count == 0 or i < recycle_count)
        rec = None
        if use and rec_in is not None and rec_in[0].shape[1] > 0:
            rec = O.biorth_recycle(M, rec_in[0], rec_in[1], svd_tol)
            if rec[0].shape[1] == 0:
                rec = None
        refresh = use and refresh_ok and step % refresh_every == 0
        res = O.rbicg_pair(M, b.astype(complex), c.astype(complex), x0, xt0, recycle=rec, k=k, s=s, tol=tol,
                           max_itn=max_itn, svd_tol=svd_tol, seed=1000 * step + i, refresh=refresh)
        state["prev_x"][i], state["prev_xt"][i] = res.x, res.xt
        out_space = (res.U_next, res.Ut_next) if use and res.U_next is not None else None
        return res, out_space

    def solve(shifts, step):
        r = len(shifts)
        V = np.zeros((n, r), complex)
        W = np.zeros((n, r), complex)
        its = []
        new_pool = []
        for i, sg in enumerate(shifts):
            if strategy == 1:
                rec_in = state["spaces"].get(i)
            elif strategy == 2:
                rec_in = state["chain"]
            elif strategy == 4:
                rec_in = state["spaces"].get("shared")
            elif strategy == 3:
                cands = [(abs(sg - s2) / abs(sg), sp_) for (s2, sp_) in state["pool"] + new_pool if sp_ is not None]
                rec_in = None
                if cands:
                    best = min(range(len(cands)), key=lambda q: cands[q][0])
                    if cands[best][0] < pool_tol:
                        rec_in = cands[best][1]
            else:
                rec_in = None
            res, sp_out = one(i, sg, step, rec_in, refresh_ok=(strategy != 4 or i == 0))
            V[:, i], W[:, i] = res.x, res.xt
            its.append(res.iters)
            if strategy == 1:
                state["spaces"][i] = sp_out
            elif strategy == 4 and i == 0:
                new_shared = sp_out
            elif strategy == 2:
                if sp_out is not None:
                    state["chain"] = sp_out
            elif strategy == 3:
                new_pool.append((sg, sp_out))
        if strategy == 3:
            state["pool"] = new_pool
        if strategy == 4 and r > 0:
            state["spaces"]["shared"] = new_shared
        return V, W, its
    return solve


def irka(A, b, c, shifts0, solve, max_steps=10, shift_tol=1e-6):
    """Algorithm 3 with E = I.  Returns a dict with the shift history (one ordered set per step,
    reading R14), the reduced model of the last step, the per-step iteration counts and whether
    the shifts converged (reading R16)."""
    A = O.as_scipy(A)
    sig = np.asarray(shifts0, dtype=complex)
    sig = sig[order_shifts(sig)]
    hist, its_hist = [sig.copy()], []
    converged, change = False, np.inf
    model = None
    for step in range(max_steps):
        V, W, its = solve(list(sig), step)                    # steps 2-3 / the loop's solves
        its_hist.append(its)
        Ar, Er, br, cr = reduced_model(A, V, W, b, c)          # step 4, first line
        model = dict(Ar=Ar, Er=Er, br=br, cr=cr, V=V, W=W, shifts=sig.copy())
        lam = sla.eig(Ar, Er, right=False)                     # step 4, second line
        new = conjugate_close(-lam)
        new = new[order_shifts(new)]
        change = float(np.max(np.abs(new - sig) / np.abs(sig)))
        sig = new
        hist.append(sig.copy())
        if change < shift_tol:
            converged = True
            break
    return dict(shifts=sig, history=hist, model=model, iters=its_hist, converged=converged, change=change,
                steps=len(its_hist))
