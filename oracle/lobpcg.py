"""LOBPCG, Algorithm 1 of the paper, in FP64 (oracle; test infrastructure only).

Algorithm 1 is printed for the standard problem; here it is generalized to
L x = lambda B x with B diagonal (B = I, or B = D for the generalized
Laplacian problem), with B-inner products throughout.  The steps, in the
paper's order:

* start:         initial guess X~, Rayleigh-Ritz on span(X~), X0 = X~ Y;
* first residual: R = L X0 - B X0 Theta0 (a fresh product with L);
* precondition:  H_I = M R_I for the unconverged columns I;
* Rayleigh-Ritz: S = [X, H_I, P_I], (Y, Theta) = RR(S, nev);
* update:        X <- S Y;
* residual:      R <- L X - B X Theta (a fresh product with L);
* lock:          I <- unconverged columns, Y_I the matching columns of Y;
* direction:     P_I <- [0, H_I, P_I] Y_I (and L P by the same combination).

Converged columns stay in X and in every Rayleigh-Ritz step but get no new
H or P columns (soft locking: the lock and direction steps).

Rayleigh-Ritz RR(S, nev) (Sec. 3.3): with G_A = S^T L S and G_B = S^T B S
(both symmetrised), scale to unit diagonal, B-orthonormalise the basis in the
small space by a Cholesky factor of the scaled G_B (the Cholesky-QR step) or,
when a pivot falls below tau, by its eigendecomposition with directions below
tau * max dropped (SVQB); then solve the projected standard eigenproblem and
keep the nev smallest pairs.  tau = 10 m u_work for m basis columns.  Each
eigenvector of the projected problem is given the sign that makes its entry
of largest magnitude positive (first such entry on ties).

Convergence (the paper names the tolerance but not the test): column i has
converged when ||r_i||_{B^-1} <= tol |theta_i| (conv="rel_theta", the default;
conv="abs" asks ||r_i||_{B^-1} <= tol instead), or when |theta_i| <= 10 u_work
rho and ||r_i||_{B^-1} <= 10 u_work rho t, with rho = 2 for L_N and the
generalized problem and 2 max deg for L_C (a Gershgorin bound) and t the most
terms in a row of L (max degree + 1); x_i is B-normalised by RR.  The theta
bound only admits the eigenvalue-zero vector, whose relative test can never
be met; the residual bound is the rounding error of one product L x, which
grows with the terms a row adds up (a hub row of 10^5 entries leaves about
3e-15 in FP64, above 10 u rho).

Pins (tests/test_oracle_lobpcg.py): closed-form path, cycle and grid spectra,
dense ``eigh`` on small graphs (eigenvalues and subspace angles), the
Bauer-Fike bound |theta - lambda| <= ||r||, B-orthonormality of the result.
"""

from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

U_FP64 = 2.0 ** -53
U_FP32 = 2.0 ** -24


@dataclasses.dataclass
class LobpcgResult:
    x: np.ndarray            # n x b Ritz vectors (B-orthonormal)
    theta: np.ndarray        # b Ritz values, ascending
    resnorm: np.ndarray      # b residual norms ||r||_{B^-1}
    converged: np.ndarray    # b booleans
    iterations: int
    svqb_steps: int
    status: str              # "ok" or "noconv"


def _sym(a: np.ndarray) -> np.ndarray:
    return 0.5 * (a + a.T)


def _sign_fix(w: np.ndarray) -> np.ndarray:
    """Make the entry of largest magnitude of every column positive."""
    idx = np.argmax(np.abs(w), axis=0)
    s = np.sign(w[idx, np.arange(w.shape[1])])
    s[s == 0] = 1.0
    return w * s


def rayleigh_ritz(ga: np.ndarray, gb: np.ndarray, nev: int, u_work: float = U_FP64):
    """Projected eigenproblem on span(S): returns (theta[nev], Y (m x nev), used_svqb)."""
    ga = _sym(np.asarray(ga, dtype=np.float64))
    gb = _sym(np.asarray(gb, dtype=np.float64))
    m_all = gb.shape[0]
    diag = np.diag(gb)
    keep = np.nonzero(np.isfinite(diag) & (diag > 0.0))[0]
    m = keep.size
    dsc = 1.0 / np.sqrt(diag[keep])
    gbh = dsc[:, None] * gb[np.ix_(keep, keep)] * dsc[None, :]
    tau = 10.0 * m * u_work
    used_svqb = False
    c = None
    try:
        lc = np.linalg.cholesky(gbh)
        if np.min(np.diag(lc)) ** 2 >= tau:
            # S_hat = S D R^{-1} with R = lc^T
            c = dsc[:, None] * sla.solve_triangular(lc.T, np.eye(m), lower=False)
    except np.linalg.LinAlgError:
        c = None
    if c is None:
        used_svqb = True
        lam, u = np.linalg.eigh(gbh)
        sel = lam > tau * lam.max()
        c = dsc[:, None] * (u[:, sel] / np.sqrt(lam[sel])[None, :])
    ap = _sym(c.T @ ga[np.ix_(keep, keep)] @ c)
    th, w = np.linalg.eigh(ap)
    w = _sign_fix(w)
    y = np.zeros((m_all, nev))
    y[keep, :] = c @ w[:, :nev]
    return th[:nev], y, used_svqb


def residual_norms(r: np.ndarray, bdiag) -> np.ndarray:
    """||r_i||_{B^-1} per column (the plain 2-norm when B = I)."""
    if bdiag is None:
        return np.sqrt(np.sum(r * r, axis=0))
    return np.sqrt(np.sum(r * r / bdiag[:, None], axis=0))


def lobpcg(apply_l, bdiag, apply_m, x0: np.ndarray, tol: float, maxit: int,
           rho: float, u_work: float = U_FP64, row_terms: int = 1, conv: str = "rel_theta",
           on_iteration=None) -> LobpcgResult:
    """Algorithm 1 for the nev = x0.shape[1] smallest eigenpairs of L x = lambda B x.

    apply_l(V): L V;  bdiag: diagonal of B or None;  apply_m(R): preconditioner
    (None for no preconditioning);  rho: the Gershgorin bound used by the
    noise floor;  row_terms: the most terms in a row of L (max degree + 1);
    conv: "rel_theta" or "abs" (see the module notes);  on_iteration(it): an
    optional callback before the first iteration (it = 0) and after every
    iteration it (timing only, no effect on the arithmetic)."""
    if conv not in ("rel_theta", "abs"):
        raise ValueError(conv)
    abs_test = conv == "abs"
    n, nev = x0.shape

    def bmul(v):
        return v if bdiag is None else bdiag[:, None] * v

    floor_th = 10.0 * u_work * rho
    floor_res = floor_th * row_terms

    def test(r, th):
        res = residual_norms(r, bdiag)
        bound = tol if abs_test else tol * np.abs(th)
        return res, (res <= bound) | ((np.abs(th) <= floor_th) & (res <= floor_res))

    # start and first residual
    lx0 = apply_l(x0)
    th, y, svqb = rayleigh_ritz(x0.T @ lx0, x0.T @ bmul(x0), nev, u_work)
    svqb_steps = int(svqb)
    x = x0 @ y
    lx = apply_l(x)
    r = lx - bmul(x) * th[None, :]
    res, conv = test(r, th)
    p = np.zeros((n, 0))
    lp = np.zeros((n, 0))
    it = 0
    if on_iteration is not None:
        on_iteration(0)
    while not conv.all() and it < maxit:
        idx = np.nonzero(~conv)[0]
        ri = r[:, idx]
        h = ri.copy() if apply_m is None else apply_m(ri)          # precondition
        lh = apply_l(h)
        s = np.concatenate([x, h, p], axis=1)                      # Rayleigh-Ritz
        ls = np.concatenate([lx, lh, lp], axis=1)
        th, y, svqb = rayleigh_ritz(s.T @ ls, s.T @ bmul(s), nev, u_work)
        svqb_steps += int(svqb)
        xn = s @ y                                                 # update
        lxn = apply_l(xn)                                          # residual
        r = lxn - bmul(xn) * th[None, :]
        res, conv = test(r, th)
        idx2 = np.nonzero(~conv)[0]                                # lock
        yp = y[:, idx2].copy()
        yp[:nev, :] = 0.0                                          # direction
        p = s @ yp
        lp = ls @ yp
        x, lx = xn, lxn
        it += 1
        if on_iteration is not None:
            on_iteration(it)
    return LobpcgResult(x=x, theta=th, resnorm=res, converged=conv, iterations=it,
                        svqb_steps=svqb_steps, status="ok" if conv.all() else "noconv")
