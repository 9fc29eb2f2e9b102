"""Algorithm 1 (Lanczos sampler), Theorem 1 bounds, Proposition 1, Section 6 log det.

FP64 throughout.  The steps follow the paper's order and notation:

Algorithm 1: v_1 = z / ||z||; for j = 1..m: q = Q v_j; q -= beta_{j-1} v_{j-1}
(j > 1); alpha_j = v_j^T q; q -= alpha_j v_j; beta_j = ||q||; v_{j+1} = q / beta_j.
Then x_m = ||z|| V_m T_m^{-1/2} e_1, T_m tridiagonal with diagonal alpha and
off-diagonal beta.  T_m^{-1/2} e_1 is taken from the eigen-decomposition of
T_m (the plain definition; the paper's caption mentions a rational
approximation as an alternative).

Theorem 1: ||x - x_m|| <= lambda_min^{-1/2} ||r_m|| with r_m the m-th conjugate
gradient residual for Q y = z (a posteriori), and the a-priori bound
2 lambda_min^{-1/2} sqrt(kappa) ((sqrt(kappa)-1)/(sqrt(kappa)+1))^m ||z||.

Stopping rule (the reading used here; the paper gives only the bound, and says it
is the practical convergence check): after step m compute
est_m = theta_min(T_m)^{-1/2} ||r_m|| / ||x_m||, with theta_min the smallest
Ritz value standing in for the unknown lambda_min, ||r_m|| = ||z|| beta_m
|e_m^T T_m^{-1} e_1| and ||x_m|| = ||z|| sqrt(e_1^T T_m^{-1} e_1); stop at the
first checked m with est_m <= tol (checks every ``check_every`` steps), or on
breakdown beta_m <= ``breakdown`` * ||T_m||.

Section 6: log det Q ~ N^{-1} sum_i v_i^T log(Q) v_i with Rademacher v_i; each
term is evaluated by Lanczos (Gauss) quadrature ||v||^2 e_1^T log(T_m) e_1
(the method of Bai, Fahey and Golub that the paper cites).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import exact, precond, stencil


# ----------------------------------------------------------------- Algorithm 1
def lanczos_steps(apply_A, z, reorth=False, breakdown=1e-13):
    """Generator over Algorithm 1's iterations.

    Yields after every step j a dict with the current ``alpha`` (list),
    ``beta`` (list), ``V`` (list of basis vectors v_1..v_j), ``znorm`` and
    ``breakdown`` (True once beta_j is negligible: the Krylov space is
    invariant and x_j is exact).
    """
    z = np.asarray(z, dtype=np.float64).reshape(-1)
    znorm = float(np.linalg.norm(z))
    v = z / znorm
    V = [v]
    alpha, beta = [], []
    v_prev = None
    while True:
        q = np.asarray(apply_A(v), dtype=np.float64)
        if v_prev is not None:
            q = q - beta[-1] * v_prev
        a = float(v @ q)
        q = q - a * v
        if reorth:
            W = np.array(V)
            for _ in range(2):
                q = q - W.T @ (W @ q)
        b = float(np.linalg.norm(q))
        alpha.append(a)
        beta.append(b)
        tnorm = max(abs(x) for x in alpha) + max(beta)
        stop = b <= breakdown * tnorm
        yield {"alpha": alpha, "beta": beta, "V": V, "znorm": znorm, "breakdown": stop}
        if stop:
            return
        v_prev, v = v, q / b
        V.append(v)


def lanczos(apply_A, z, m, reorth=False, breakdown=1e-13):
    """Run m steps of Algorithm 1 (fewer on breakdown)."""
    st = None
    for j, st in enumerate(lanczos_steps(apply_A, z, reorth, breakdown), start=1):
        if j >= m or st["breakdown"]:
            break
    k = len(st["alpha"])
    return {"alpha": np.array(st["alpha"]), "beta": np.array(st["beta"]),
            "V": np.array(st["V"][:k]), "znorm": st["znorm"], "m": k,
            "breakdown": st["breakdown"]}


def tridiagonal(alpha, beta):
    """Dense T_m from alpha (m) and beta (>= m-1 values; beta_m is not in T_m)."""
    alpha = np.asarray(alpha, dtype=np.float64)
    m = len(alpha)
    off = np.asarray(beta, dtype=np.float64)[: m - 1]
    return np.diag(alpha) + np.diag(off, 1) + np.diag(off, -1)


def tm_eigh(alpha, beta):
    """Ritz values theta and eigenvectors S of T_m."""
    alpha = np.asarray(alpha, dtype=np.float64)
    m = len(alpha)
    if m == 1:
        return alpha.copy(), np.ones((1, 1))
    return sla.eigh_tridiagonal(alpha, np.asarray(beta, dtype=np.float64)[: m - 1])


def tm_function_e1(alpha, beta, f):
    """f(T_m) e_1 = S f(Theta) S^T e_1."""
    th, S = tm_eigh(alpha, beta)
    return S @ (f(th) * S[0, :])


def tm_inv_sqrt_e1(alpha, beta):
    """T_m^{-1/2} e_1 (Algorithm 1, last step)."""
    th, _ = tm_eigh(alpha, beta)
    if th[0] <= 0:
        raise ValueError("T_m is not positive definite")
    return tm_function_e1(alpha, beta, lambda t: 1.0 / np.sqrt(t))


def tm_log_e1e1(alpha, beta) -> float:
    """e_1^T log(T_m) e_1 = sum_k s_{1k}^2 log theta_k (Gauss quadrature)."""
    th, S = tm_eigh(alpha, beta)
    if th[0] <= 0:
        raise ValueError("T_m is not positive definite")
    return float(np.sum(S[0, :] ** 2 * np.log(th)))


def sample_from_lanczos(run, m=None):
    """x_m = ||z|| V_m T_m^{-1/2} e_1 from a ``lanczos`` result (first m steps)."""
    m = run["m"] if m is None else m
    y = tm_inv_sqrt_e1(run["alpha"][:m], run["beta"][:m])
    return run["znorm"] * (run["V"][:m].T @ y)


def krylov_sample(apply_A, z, m, reorth=False):
    """Algorithm 1 end to end with a fixed subspace size m."""
    return sample_from_lanczos(lanczos(apply_A, z, m, reorth))


# ------------------------------------------------------------------- Theorem 1
def cg_residual_norm(alpha, beta, znorm) -> float:
    """||r_m|| = ||z|| beta_m |e_m^T T_m^{-1} e_1| (Lanczos form of the CG residual)."""
    m = len(alpha)
    T = tridiagonal(alpha, beta)
    w = np.linalg.solve(T, np.eye(m)[0])
    return float(znorm * beta[m - 1] * abs(w[m - 1]))


def cg_residual_direct(apply_A, z, run, m=None) -> float:
    """||z - Q y_m|| with y_m = ||z|| V_m T_m^{-1} e_1, the CG iterate (definition)."""
    m = run["m"] if m is None else m
    T = tridiagonal(run["alpha"][:m], run["beta"][:m])
    y = run["znorm"] * (run["V"][:m].T @ np.linalg.solve(T, np.eye(m)[0]))
    return float(np.linalg.norm(np.asarray(z).reshape(-1) - apply_A(y)))


def cg_solve(apply_A, b, tol, m_max):
    """Conjugate gradients (Hestenes and Stiefel) for A x = b from x_0 = 0:
    r_0 = p_0 = b; a_k = r_k^T r_k / p_k^T A p_k; x_{k+1} = x_k + a_k p_k;
    r_{k+1} = r_k - a_k A p_k; p_{k+1} = r_{k+1} + (r_{k+1}^T r_{k+1} / r_k^T r_k) p_k.
    Stops at the first k with ||r_k|| <= tol ||b|| (k <= m_max).  Its iterates
    are the Lanczos ones, x_k = ||b|| V_k T_k^{-1} e_1 (the link Theorem 1's
    residual r_m rests on).  Returns (x, k, status in {'ok', 'not_converged'})."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros_like(b)
    r = b.copy()
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return x, 0, "ok"
    p = r.copy()
    rr = float(r @ r)
    for k in range(1, m_max + 1):
        Ap = apply_A(p)
        a = rr / float(p @ Ap)
        x = x + a * p
        r = r - a * Ap
        rr_new = float(r @ r)
        if np.sqrt(rr_new) <= tol * bn:
            return x, k, "ok"
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, m_max, "not_converged"


def posterior_bound(lam_min, res_norm) -> float:
    """Theorem 1, eq. (krylov_bound): lambda_min^{-1/2} ||r_m||."""
    return float(res_norm / np.sqrt(lam_min))


def apriori_bound(lam_min, lam_max, m, znorm) -> float:
    """Theorem 1, eq. (apriori)."""
    k = lam_max / lam_min
    rk = np.sqrt(k)
    return float(2.0 / np.sqrt(lam_min) * rk * ((rk - 1) / (rk + 1)) ** m * znorm)


def stopping_estimate(alpha, beta, znorm=1.0) -> float:
    """est_m = theta_min^{-1/2} ||r_m|| / ||x_m|| (relative; see module docstring)."""
    m = len(alpha)
    T = tridiagonal(alpha, beta)
    w = np.linalg.solve(T, np.eye(m)[0])
    th = tm_eigh(alpha, beta)[0]
    if th[0] <= 0 or w[0] <= 0:
        return np.inf
    res = znorm * beta[m - 1] * abs(w[m - 1])
    xnorm = znorm * np.sqrt(w[0])
    return float(res / np.sqrt(th[0]) / xnorm)


def adaptive_run(apply_A, z, tol, m_max, check_every=1, reorth=False, breakdown=1e-13):
    """Algorithm 1 with m chosen by the stopping rule; returns the run, the
    estimate at the chosen m and a status ('ok', 'breakdown', 'not_converged')."""
    status, est = "not_converged", np.inf
    st = None
    for j, st in enumerate(lanczos_steps(apply_A, z, reorth, breakdown), start=1):
        if st["breakdown"]:
            status, est = "breakdown", 0.0
            break
        if j % check_every == 0 or j >= m_max:
            est = stopping_estimate(st["alpha"], st["beta"])
            if est <= tol:
                status = "ok"
                break
        if j >= m_max:
            break
    k = len(st["alpha"])
    run = {"alpha": np.array(st["alpha"]), "beta": np.array(st["beta"]),
           "V": np.array(st["V"][:k]), "znorm": st["znorm"], "m": k,
           "breakdown": st["breakdown"]}
    return run, est, status


def adaptive_sample(apply_A, z, tol, m_max, check_every=1, reorth=False):
    """x_m with the adaptive m; returns (x, m, est, status)."""
    run, est, status = adaptive_run(apply_A, z, tol, m_max, check_every, reorth)
    return sample_from_lanczos(run), run["m"], est, status


# ------------------------------------------------------ operators for the oracle
def operator(shape, bc, op, kappa2, tau=1.0):
    """v -> Q v with Q assembled as a sparse matrix (``stencil``)."""
    Q = stencil.precision_matrix(shape, bc, op, kappa2, tau)
    return (lambda v: Q @ v), Q


def preconditioned_operator(Q, shape, kind, op, kbar2, tau):
    """v -> A v, A = M^{-1/2} Q M^{-1/2} (Proposition 1 with F = M^{1/2})."""
    def apply_A(v):
        w = precond.apply_power(shape, kind, op, kbar2, tau, v, -0.5)
        return precond.apply_power(shape, kind, op, kbar2, tau, Q @ w, -0.5)
    return apply_A


def precond_sample(Q, shape, kind, op, kbar2, tau, z, tol, m_max, check_every=1, reorth=False):
    """Proposition 1: Lanczos on A gives u_m, then x = M^{-1/2} u_m."""
    A = preconditioned_operator(Q, shape, kind, op, kbar2, tau)
    u, m, est, status = adaptive_sample(A, z, tol, m_max, check_every, reorth)
    return precond.apply_power(shape, kind, op, kbar2, tau, u, -0.5), m, est, status


# ----------------------------------------------------------------- Section 6
def quadrature_term(apply_A, v, tol, m_max, check_every=1, reorth=False):
    """||v||^2 e_1^T log(T_m) e_1 for one probe v (Gauss quadrature); m by the
    same Theorem 1 stopping rule as the sampler.  Returns (q, m, status)."""
    run, est, status = adaptive_run(apply_A, v, tol, m_max, check_every, reorth)
    q = run["znorm"] ** 2 * tm_log_e1e1(run["alpha"], run["beta"])
    return q, run["m"], status


def hutchinson_logdet(apply_A, probes, tol, m_max, check_every=1, reorth=False, shift=0.0):
    """(estimate, std_error, q_i) with estimate = mean_i q_i + shift.

    ``shift`` is log det M for the preconditioned estimator (Section 6.2, plus
    sign) and 0 otherwise."""
    qs = np.array([quadrature_term(apply_A, v, tol, m_max, check_every, reorth)[0]
                   for v in np.atleast_2d(probes)])
    est = float(np.mean(qs)) + shift
    se = float(np.std(qs, ddof=1) / np.sqrt(len(qs))) if len(qs) > 1 else float("nan")
    return est, se, qs


def coloured_probe_masks(shape, p):
    """Distance-p colouring of the lattice graph for the coloured Hutchinson
    estimator (Section 6.1): colour(cell) = tuple(coord mod (p + 1)); two cells
    of one colour differ by a multiple of p+1 along every axis where they
    differ, so their lattice distance exceeds p.  Returns a boolean array
    [ncolours][n]."""
    shape = tuple(int(s) for s in shape)
    grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    colour = np.zeros(shape, dtype=np.int64)
    for g in grids:
        colour = colour * (p + 1) + (g % (p + 1))
    ncol = (p + 1) ** len(shape)
    return np.array([(colour == c).reshape(-1) for c in range(ncol)])


def coloured_hutchinson_logdet(apply_A, shape, p, draws, tol, m_max, check_every=1, reorth=False, shift=0.0):
    """Coloured Hutchinson estimator (Section 6.1): each Rademacher draw v is
    split over the colour classes c of the distance-p colouring, v_c = v on c
    and 0 elsewhere, and one draw contributes sum_c v_c^T log(A) v_c (each term
    by Lanczos quadrature).  Returns (estimate, std_error, q [N][ncolours]) with
    estimate = mean over draws of the per-draw sums + shift."""
    masks = coloured_probe_masks(shape, p)
    draws = np.atleast_2d(draws)
    q = np.array([[quadrature_term(apply_A, np.where(mk, v, 0.0), tol, m_max, check_every, reorth)[0]
                   for mk in masks] for v in draws])
    per = q.sum(axis=1)
    est = float(per.mean()) + shift
    se = float(per.std(ddof=1) / np.sqrt(len(per))) if len(per) > 1 else float("nan")
    return est, se, q
