"""Lanczos recurrence, Krylov propagator and eigenvalue mode (oracle; test infrastructure only).

Sec. 2 (Fig. 1 with the modified Gram-Schmidt alpha of Eq. 4), Sec. 4
(Eq. 17: psi(t+dt) ~ ||psi|| Q exp(-i T) e_1 for A = dt * H, and the error
estimate Eq. 18), Sec. 6 (cumulative error bound), Sec. 2/5 (Ritz values,
the bound Eq. 9, full reorthogonalisation applied twice).

Readings where the paper leaves a choice:

* A is the Hermitian matrix of the integral of H over the step (Sec. 4); with
  the first Magnus term and H affine in the field, that is dt * H(A_mean).
  An optional constant energy shift s runs the recurrence on dt * (H - s); the
  step then multiplies by exp(-i s dt), exact in exact arithmetic.
* The recurrence stops early at iteration i < m when (a) the breakdown test
  beta_i <= 1e-12 * scale_i holds, scale_i being the largest |alpha_j + dt s|
  or beta_j (j < i) seen so far -- the invariant-subspace case, or (b) tol > 0
  and the Eq. 18 estimate at i is <= tol * ||psi||.  Otherwise it runs m
  iterations; beta_m is still computed (one extra norm) for Eq. 18.
* The small exponential exp(-i T) e_1 uses the eigendecomposition of the real
  symmetric tridiagonal T (Sec. 4), here LAPACK through SciPy.
* The eigenvalue mode orthogonalises each new vector against all previous
  Lanczos vectors by classical Gram-Schmidt, twice (Sec. 2).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg

from . import hamiltonian as ham
from . import fields

BREAKDOWN_REL = 1e-12


def tridiag_expm_e1(alpha, beta) -> np.ndarray:
    """exp(-i T) e_1 for the symmetric tridiagonal T = tridiag(beta, alpha, beta).

    Sec. 4: diagonalise T = S diag(lambda) S^T, then exp(-iT) e_1 =
    S diag(exp(-i lambda)) S^T e_1.
    """
    alpha = np.asarray(alpha, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    k = alpha.size
    if k == 1:
        return np.array([np.exp(-1j * alpha[0])])
    lam, S = scipy.linalg.eigh_tridiagonal(alpha, beta[: k - 1])
    return S @ (np.exp(-1j * lam) * S[0, :])


@dataclasses.dataclass
class LanczosResult:
    q: list            # orthonormal Lanczos vectors q_1..q_k
    alpha: np.ndarray  # alpha_1..alpha_k
    beta: np.ndarray   # beta_1..beta_k (beta_k is the residual norm after q_k)
    breakdown: bool


def lanczos(apply_a, b: np.ndarray, k: int, stop=None) -> LanczosResult:
    """Fig. 1 (MGS form, Eq. 4), computing alpha_i and beta_i for i = 1..k.

    ``stop(alpha, beta)`` may end the recurrence after any iteration (adaptive
    Krylov dimension, Sec. 4); it returns "breakdown", "tol" or None.
    """
    q = [b / ham.norm(b)]
    z = apply_a(q[0])
    alpha, beta = [], []
    broke = False
    while True:
        i = len(alpha)                      # 0-based: working on q_{i+1}
        a = ham.inner(q[i], z).real         # alpha_i = q_i . (A q_i - beta_{i-1} q_{i-1})
        z = z - a * q[i]
        bt = ham.norm(z)                    # beta_i = ||z||
        alpha.append(a)
        beta.append(bt)
        reason = stop(alpha, beta) if stop is not None else None
        if reason == "breakdown":
            broke = True
        if len(alpha) == k or reason is not None:
            break
        q.append(z / bt)                    # q_{i+1} = z / beta_i
        z = apply_a(q[i + 1]) - bt * q[i]   # z = A q_{i+1} - beta_i q_i
    return LanczosResult(q, np.array(alpha), np.array(beta), broke)


@dataclasses.dataclass
class StepInfo:
    k_used: int
    err_est: float      # Eq. 18 estimate of ||Delta psi||
    norm: float         # ||psi|| before the step
    energy: float       # alpha_1 / dt + shift = <psi|H|psi>/<psi|psi>
    breakdown: bool
    alpha: np.ndarray   # T of the matrix dt*(H - shift)
    beta: np.ndarray


def krylov_step(op: ham.Operator, psi: np.ndarray, dt: float, m: int, tol: float = 0.0):
    """One time step psi -> exp(-i H dt) psi by Eq. 17, with the Eq. 18 estimate."""
    shift = op.shift

    def apply_a(v):
        return dt * ham.apply(op, v)        # A = dt (H - shift)

    psi_norm = ham.norm(psi)

    def stop(alpha, beta):
        i = len(alpha)
        scale = max(max(abs(a + dt * shift) for a in alpha),
                    max(beta[: i - 1]) if i > 1 else 0.0)
        if beta[-1] <= BREAKDOWN_REL * scale:
            return "breakdown"
        if tol > 0.0:
            v = tridiag_expm_e1(alpha, beta)
            if beta[-1] * abs(v[-1]) <= tol:  # Eq. 18 divided by ||psi||
                return "tol"
        return None

    res = lanczos(apply_a, psi, m, stop)
    k = res.alpha.size
    v = tridiag_expm_e1(res.alpha, res.beta)
    out = np.zeros_like(psi)
    for j in range(k):
        out += v[j] * res.q[j]
    out *= psi_norm * np.exp(-1j * shift * dt)
    err = res.beta[k - 1] * psi_norm * abs(v[k - 1])
    info = StepInfo(k, float(err), psi_norm, res.alpha[0] / dt + shift, res.breakdown,
                    res.alpha, res.beta)
    return out, info


def propagate(op: ham.Operator, psi: np.ndarray, dt: float, m: int, steps: int,
              pulse=None, t0: float = 0.0, tol: float = 0.0):
    """``steps`` Krylov steps; with a pulse, A_x of each step is its Magnus-1 mean.

    Returns (psi, list of StepInfo); the cumulative error bound of Sec. 6 is
    the sum of the ``err_est`` values.
    """
    infos = []
    for n in range(steps):
        if pulse is not None:
            op.A = (fields.step_mean(pulse, t0 + n * dt, dt), op.A[1])
        psi, info = krylov_step(op, psi, dt, m, tol)
        infos.append(info)
    return psi, infos


@dataclasses.dataclass
class EigResult:
    values: np.ndarray      # selected Ritz values (energies of H - shift), ascending
    bounds: np.ndarray      # their error bounds (Eq. 9; folded mode: see lanczos_eigs)
    iterations: int
    all_ritz: np.ndarray    # every Ritz value of the recurrence's operator at the end
    all_bounds: np.ndarray
    breakdown: bool = False
    vectors: list = None    # Ritz vectors Q t_i (Eq. 8) of the selected values, if asked


def lanczos_eigs(op: ham.Operator, start: np.ndarray, n_want: int, max_iter: int,
                 tol: float, window: tuple, reorth: bool = True, check_every: int = 10,
                 fold=None, vectors: bool = False):
    """Eigenvalue mode (Sec. 2, Sec. 5): Ritz values with Eq. 9 bounds.

    The recurrence runs on A = H - shift (``fold`` None) or, shift-folded, on
    A = (H - shift - fold)^2, whose smallest eigenvalues belong to the
    eigenvalues of H - shift nearest ``fold``.  Each iteration:
    z = A q_i - beta_{i-1} q_{i-1}; alpha_i = q_i . z; z -= alpha_i q_i; with
    ``reorth``, z is orthogonalised against all previous Lanczos vectors by
    classical Gram-Schmidt, twice, and the coefficients along q_i are added to
    alpha_i; beta_i = ||z||.  The recurrence ends at the breakdown test of the
    propagator (beta_i <= 1e-12 * scale, T's spectrum is then exact).

    Every ``check_every`` iterations (and at the end) T is diagonalised.  A Ritz
    value theta counts as converged when its bound |beta_k t_i^k| (Eq. 9) is
    <= tol * max(1, |theta|).
      direct: stop when ``n_want`` converged Ritz values lie in ``window`` (open
        interval, energies of H - shift); all of them are returned.
      folded: stop when the ``n_want`` smallest Ritz values of A are converged;
        each gives lambda = fold + sign sqrt(theta), the sign being that of the
        Rayleigh quotient of its Ritz vector with H - shift - fold, and the
        bound min(sqrt(r), r / sqrt(theta)) on |lambda - lambda_exact| from the
        Eq. 9 bound r on theta.  ``window`` is not used.
    With ``vectors`` the Ritz vectors Q t_i (Eq. 8, unit norm) of the returned
    values are returned too.
    """
    if fold is None:
        def apply_a(v):
            return ham.apply(op, v)
        ashift = op.shift             # scale of the breakdown test as in the propagator
    else:
        def apply_f(v):
            return ham.apply(op, v) - fold * v
        def apply_a(v):
            return apply_f(apply_f(v))
        ashift = 0.0
    q = [start / ham.norm(start)]
    alpha, beta = [], []
    z = apply_a(q[0])
    while True:
        i = len(alpha)
        a = ham.inner(q[i], z).real
        z = z - a * q[i]
        if reorth:
            Q = np.stack([v.reshape(-1) for v in q], axis=1)
            for _ in range(2):
                h = Q.conj().T @ z.reshape(-1)
                z = z - (Q @ h).reshape(z.shape)
                a += h[i].real
        bt = ham.norm(z)
        alpha.append(a)
        beta.append(bt)
        it = i + 1
        scale = max(max(abs(x + ashift) for x in alpha), max(beta[:-1]) if it > 1 else 0.0)
        broke = bt <= BREAKDOWN_REL * scale
        done = it >= max_iter or broke
        if it % check_every == 0 or done:
            theta, S = scipy.linalg.eigh_tridiagonal(np.array(alpha), np.array(beta[:-1])) \
                if it > 1 else (np.array(alpha), np.ones((1, 1)))
            bnd = np.abs(bt * S[-1, :])
            conv = bnd <= tol * np.maximum(1.0, np.abs(theta))
            if fold is None:
                conv &= (theta > window[0]) & (theta < window[1])
                finished = conv.sum() >= n_want
            else:
                finished = theta.size >= n_want and bool(conv[:n_want].all())
            if finished or done:
                sel = np.nonzero(conv)[0] if fold is None else \
                    np.nonzero(conv[:n_want])[0]
                vecs = None
                if vectors or fold is not None:
                    Q = np.stack([v.reshape(-1) for v in q], axis=1)
                    vecs = [(Q @ S[:, j]).reshape(start.shape) for j in sel]
                vals, bnds = theta[sel], bnd[sel]
                if fold is not None:
                    lam, lb = [], []
                    for j, y in zip(sel, vecs):
                        rq = ham.inner(y, apply_f(y)).real
                        th = max(theta[j], 0.0)
                        lam.append(fold + np.copysign(np.sqrt(th), rq))
                        lb.append(min(np.sqrt(bnd[j]), bnd[j] / np.sqrt(th)) if th > 0
                                  else np.sqrt(bnd[j]))
                    order = np.argsort(lam, kind="stable")
                    vals, bnds = np.asarray(lam)[order], np.asarray(lb)[order]
                    vecs = [vecs[o] for o in order]
                return EigResult(vals, bnds, it, theta, bnd, bool(broke),
                                 vecs if vectors else None)
        q.append(z / bt)
        z = apply_a(q[i + 1]) - bt * q[i]


def energy(op: ham.Operator, psi: np.ndarray) -> float:
    """<psi|H|psi> / <psi|psi> (without the shift)."""
    return ham.inner(psi, ham.apply(op, psi)).real / ham.inner(psi, psi).real + op.shift


def rel_l2(a: np.ndarray, ref: np.ndarray) -> float:
    return ham.norm(a - ref) / ham.norm(ref)


def site_sample(psi: np.ndarray, flat_sites) -> np.ndarray:
    """The spinors at the given flattened site indices (for sampled comparisons)."""
    return psi.reshape(-1, 2)[np.asarray(flat_sites)]


__all__ = ["tridiag_expm_e1", "lanczos", "krylov_step", "propagate", "lanczos_eigs",
           "energy", "rel_l2", "site_sample", "StepInfo", "LanczosResult", "EigResult"]
