"""Oracle: flexible GMRES with a (possibly nonlinear) preconditioner (test infrastructure only).

Follows Alg. 1 and the generalised Arnoldi relation A Z_k = V_{k+1} Hbar_k
(eq. 4): per cycle r0 = b - A x0, beta = ||r0||, v1 = r0 / beta; for
j = 1..m: z_j = M(v_j), w = A z_j, orthogonalise w against v_1..v_j giving
h_{1..j, j}, h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}; then
y = argmin ||Hbar y - beta e1|| and x = x0 + Z y.  Restarted cycles repeat
this from the current x (Sec. 4: l cycles of m iterations).

Readings where the paper is silent:
  * h_ij = v_i^H w (the w update removes the component along v_i);
  * orthogonalisation "mgs" is the paper's inner loop; "cgs2" is classical
    Gram-Schmidt applied twice, h = h1 + h2; "dcgs2" delays the second pass by
    one step (the preconditioner then sees the once-orthogonalised vector);
  * the least-squares problem is solved by complex Givens rotations
    (c real = |a| / sqrt(|a|^2 + |b|^2), s = (a / |a|) conj(b) / sqrt(...),
    c = 0, s = 1 when a = 0) applied as the columns arrive; |g_{j+1}| is the
    residual-norm estimate;
  * a cycle stops early when |g_{j+1}| <= target, or on breakdown
    (h_{j+1,j} <= 1e-14 ||w before orthogonalisation||);
  * success is declared on the true backward error ||b - A x|| / ||b|| (eq. 10).

`refine` is the FP64 iterative-refinement driver of the mixed path: outer
r = b - A x in FP64, an inner solve of A d = r / ||r|| to a relative
reduction `inner_tol` (inner arithmetic optionally cast through complex64
and a BF16-emulated network), x += ||r|| d, until the true eta_b <= tol.

Pins (tests/test_oracle_fgmres.py): identity preconditioner == textbook
GMRES == scipy.sparse.linalg.gmres residual history (MGS, CGS2 and DCGS2);
DCGS2 == CGS2 under a fixed linear preconditioner and at a lagged stop; exact inverse
preconditioner converges in one iteration; a fixed linear preconditioner
equals right-preconditioned GMRES; ||A Z - V Hbar|| and ||V^H V - I|| at
rounding level; y equals numpy.linalg.lstsq on Hbar; the converged x is
within the bound of the sparse direct solution.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CycleResult:
    x: np.ndarray
    iters: int
    est: float                 # |g_{j+1}| at exit
    V: np.ndarray              # [k+1, n]
    Z: np.ndarray              # [k, n]
    Hbar: np.ndarray           # [k+1, k]
    y: np.ndarray
    breakdown: bool
    history: list              # |g_{j+1}| after each iteration


@dataclass
class SolveInfo:
    iters: int = 0
    cycles: int = 0
    outer: int = 0
    relres_true: float = np.inf
    converged: bool = False
    history: list = field(default_factory=list)   # residual estimate / ||b|| per iteration


def givens(a, b):
    """Rotation (c, s) with [c s; -conj(s) c] [a; b] = [r; 0], c real."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, 1.0 + 0.0j
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s


def _rotate_column(col, j, cs, sn):
    """Apply the rotations 0..j-1 to Hessenberg column j (length j + 2), then form rotation j."""
    col = col.copy()
    for i in range(j):
        a, b_ = col[i], col[i + 1]
        col[i] = cs[i] * a + sn[i] * b_
        col[i + 1] = -np.conj(sn[i]) * a + cs[i] * b_
    cs[j], sn[j] = givens(col[j], col[j + 1])
    col[j] = cs[j] * col[j] + sn[j] * col[j + 1]
    col[j + 1] = 0.0
    return col


def _back_substitute(R, g, k):
    y = np.zeros(k, np.complex128)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - R[i, i + 1:k] @ y[i + 1:k]) / R[i, i]
    return y


def _cycle_dcgs2(apply_A, precond, r0, m, target, dtype):
    """One FGMRES(m) cycle with classical Gram-Schmidt whose second pass is delayed by one step.

    The vector u_j entering step j has been orthogonalised once.  Step j preconditions it,
    z_j = M(u_j / ||u_j||), forms w_j = A z_j and, from one pass over V_j = (v_0..v_{j-1}),
    a = V_j^H u_j and b = V_j^H w_j.  The second pass of u_j then finishes column j-1 of Hbar:
    h_{:j, j-1} += a, h_{j, j-1} = rho = sqrt(||u_j||^2 - ||a||^2), v_j = (u_j - V_j a) / rho; and the
    first pass of w_j gives column j: h_{:j, j} = b, h_{j, j} = d = (u_j^H w_j - a^H b) / rho and
    u_{j+1} = w_j - V_j b - v_j d.  Column j-1 is rotated (and the stopping test made) at step j;
    after the last step a final pass finishes column m-1.  v_0 = r0 / ||r0|| needs no second pass.
    Any z_j is admissible in flexible GMRES: A Z = V Hbar holds with the V and Hbar formed here.
    """
    n = r0.size
    beta = np.linalg.norm(r0)
    V = np.zeros((m + 1, n), dtype)
    Z = np.zeros((m, n), dtype)
    H = np.zeros((m + 1, m), np.complex128)
    R = np.zeros((m + 1, m), np.complex128)
    cs = np.zeros(m)
    sn = np.zeros(m, np.complex128)
    g = np.zeros(m + 1, np.complex128)
    g[0] = beta
    V[0] = (r0 / beta).astype(dtype)
    u = V[0].copy()
    wnorm = np.zeros(m)
    history = []
    k, est, breakdown = 0, beta, False

    def finish(j, u):
        """Second pass of u = u_{j+1}: completes column j, sets V[j + 1]; returns (rho, a)."""
        Vp = V[:j + 1]
        a = Vp.conj() @ u
        rho = np.sqrt(max(np.vdot(u, u).real - np.vdot(a, a).real, 0.0))
        H[:j + 1, j] += a
        H[j + 1, j] = rho
        if rho > 0:
            V[j + 1] = ((u - Vp.T @ a.astype(dtype)) / rho).astype(dtype)
        return rho, a

    def rotate(j):
        R[:j + 2, j] = _rotate_column(H[:j + 2, j], j, cs, sn)
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        return abs(g[j + 1])

    stopped = False
    for j in range(m):
        nu = np.linalg.norm(u)
        Z[j] = np.asarray(precond((u / nu).astype(dtype)), dtype)  # the preconditioner sees unit norm
        w = np.asarray(apply_A(Z[j]), np.complex128).astype(dtype)
        wnorm[j] = np.linalg.norm(w)
        rho, a = 1.0, np.zeros(j, np.complex128)  # v_0 needs no second pass
        u_j = u
        if j > 0:
            rho, a = finish(j - 1, u)        # v_j and column j-1
            k = j
            est = rotate(j - 1)
            history.append(est)
            if rho <= 1e-14 * max(wnorm[j - 1], np.finfo(float).tiny):
                breakdown, stopped = True, True
                break
            if est <= target:
                stopped = True
                break
        Vp = V[:j + 1]
        b = Vp[:j].conj() @ w
        H[:j, j] = b
        H[j, j] = (np.vdot(u_j, w) - np.vdot(a, b)) / rho  # = v_j^H w_j
        u = (w - Vp.T @ H[:j + 1, j].astype(dtype)).astype(dtype)
    if not stopped:
        rho, _ = finish(m - 1, u)
        k = m
        est = rotate(m - 1)
        history.append(est)
        breakdown = rho <= 1e-14 * max(wnorm[m - 1], np.finfo(float).tiny)
    y = _back_substitute(R, g, k)
    d = Z[:k].T.astype(np.complex128) @ y
    return CycleResult(d, k, est, V[:k + 1], Z[:k], H[:k + 1, :k], y, breakdown, history)


def cycle(apply_A, precond, r0, m, target, orth="cgs2", dtype=np.complex128):
    """One FGMRES(m) cycle on A d = r0 from d0 = 0.  Returns the correction d in CycleResult.x.
    orth: "mgs" (Alg. 1's loop), "cgs2" (classical Gram-Schmidt twice) or "dcgs2" (second pass
    delayed by one step, see _cycle_dcgs2)."""
    if orth == "dcgs2":
        return _cycle_dcgs2(apply_A, precond, r0, m, target, dtype)
    n = r0.size
    beta = np.linalg.norm(r0)
    V = np.zeros((m + 1, n), dtype)
    Z = np.zeros((m, n), dtype)
    H = np.zeros((m + 1, m), np.complex128)
    R = np.zeros((m + 1, m), np.complex128)
    cs = np.zeros(m)
    sn = np.zeros(m, np.complex128)
    g = np.zeros(m + 1, np.complex128)
    g[0] = beta
    V[0] = (r0 / beta).astype(dtype)
    k = 0
    breakdown = False
    est = beta
    history = []
    for j in range(m):
        Z[j] = np.asarray(precond(V[j]), dtype)
        w = np.asarray(apply_A(Z[j]), np.complex128).astype(dtype)
        w0 = np.linalg.norm(w)
        if orth == "mgs":
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = (w - H[i, j] * V[i]).astype(dtype)
        elif orth == "cgs2":
            Vj = V[:j + 1]
            h1 = Vj.conj() @ w
            w = (w - Vj.T @ h1.astype(dtype)).astype(dtype)
            h2 = Vj.conj() @ w
            w = (w - Vj.T @ h2.astype(dtype)).astype(dtype)
            H[:j + 1, j] = h1 + h2
        else:
            raise ValueError(orth)
        H[j + 1, j] = np.linalg.norm(w)
        k = j + 1
        # apply previous rotations to column j, then a new rotation
        col = H[:j + 2, j].copy()
        for i in range(j):
            a, b_ = col[i], col[i + 1]
            col[i] = cs[i] * a + sn[i] * b_
            col[i + 1] = -np.conj(sn[i]) * a + cs[i] * b_
        cs[j], sn[j] = givens(col[j], col[j + 1])
        col[j] = cs[j] * col[j] + sn[j] * col[j + 1]
        col[j + 1] = 0.0
        R[:j + 2, j] = col
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        est = abs(g[j + 1])
        history.append(est)
        if H[j + 1, j] <= 1e-14 * max(w0, np.finfo(float).tiny):
            breakdown = True
            break
        V[j + 1] = (w / H[j + 1, j]).astype(dtype)
        if est <= target:
            break
    # back substitution R[:k,:k] y = g[:k]
    y = np.zeros(k, np.complex128)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - R[i, i + 1:k] @ y[i + 1:k]) / R[i, i]
    d = Z[:k].T.astype(np.complex128) @ y
    return CycleResult(d, k, est, V[:k + 1], Z[:k], H[:k + 1, :k], y, breakdown, history)


def fgmres(apply_A, precond, b, x0=None, m=30, tol=1e-6, max_cycles=100, orth="cgs2"):
    """Restarted FGMRES(m) in FP64 (Alg. 1 with restarts, Sec. 4); stop on the true eta_b <= tol."""
    b = np.asarray(b, np.complex128)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, np.complex128).copy()
    nb = np.linalg.norm(b)
    info = SolveInfo()
    for _ in range(max_cycles):
        r = b - apply_A(x)
        info.relres_true = np.linalg.norm(r) / nb
        if info.relres_true <= tol:
            info.converged = True
            break
        res = cycle(apply_A, precond, r, m, tol * nb, orth)
        x = x + res.x
        info.iters += res.iters
        info.cycles += 1
        info.history += [e / nb for e in res.history]
        if res.breakdown and res.iters == 0:
            break
    else:
        r = b - apply_A(x)
        info.relres_true = np.linalg.norm(r) / nb
        info.converged = info.relres_true <= tol
    return x, info


def refine(apply_A, precond_lo, b, m=30, tol=1e-6, inner_tol=1e-4, max_outer=20,
           max_cycles_inner=1, orth="cgs2", inner_dtype=np.complex64):
    """FP64 iterative refinement around a low-precision FGMRES(m) inner solve.

    Outer (FP64): r = b - A x, stop when ||r|| / ||b|| <= tol.  Inner: FGMRES on
    A d = r / ||r|| with vectors stored in `inner_dtype`, until the estimate
    drops below max(inner_tol, tol ||b|| / ||r||) relative to ||r / ||r|||| = 1 (the
    inner solve need not go further than the outer target) or m iterations; then
    x += ||r|| d.
    """
    b = np.asarray(b, np.complex128)
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    info = SolveInfo()

    def A_lo(u):
        return np.asarray(apply_A(np.asarray(u, np.complex128)), np.complex128).astype(inner_dtype)

    for _ in range(max_outer):
        r = b - apply_A(x)
        nr = np.linalg.norm(r)
        info.relres_true = nr / nb
        if info.relres_true <= tol:
            info.converged = True
            break
        info.outer += 1
        rhat = (r / nr).astype(inner_dtype)
        d = np.zeros(b.size, np.complex128)
        rr = rhat.astype(np.complex128)
        target = max(inner_tol, tol * nb / nr)
        for _ in range(max_cycles_inner):
            res = cycle(A_lo, precond_lo, rr.astype(inner_dtype), m, target, orth, dtype=inner_dtype)
            d = d + res.x
            info.iters += res.iters
            info.cycles += 1
            rr = rhat.astype(np.complex128) - apply_A(d)
            if np.linalg.norm(rr) <= target:
                break
        x = x + nr * d
    else:
        r = b - apply_A(x)
        info.relres_true = np.linalg.norm(r) / nb
        info.converged = info.relres_true <= tol
    return x, info
