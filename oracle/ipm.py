"""Primal-dual predictor-corrector interior-point method (oracle; test-only).

Sec. IV-A and Algorithm 2 of the paper, with these readings of passages the
paper leaves open or prints garbled (each is stated where it is used):

* R-A6  mu: the paper's "mu = tr(ZX)/3" is read as mu = sigma*tr(ZX)/n_X with
        centring parameter sigma = 1/3 and n_X = (L+M) n, the order of X.
* R-A7  predictor: Delta X_hat = -X + Z^{-1} (G - B^T(Delta y_hat)) X, the form
        for which the printed Delta y_hat equation gives B(X + Delta X_hat) = a.
* R-A8  Delta X_hat and Delta X_bar are symmetrised, (D + D^T)/2.
* R-A9  line search: t = min(1, tau * t_max), tau = 0.95, t_max the exact
        largest step keeping the block PSD (from the smallest eigenvalue of
        L^{-1} Delta L^{-T}, X = L L^T); separate t_p for X and t_d for (y, Z).
* R-A10 Z and y are updated with t_d (Eqs. y, Z).
* R-A11 stop when the relative gap |a^T y - tr(CX)| / (1 + |a^T y| + |tr(CX)|),
        the relative primal residual ||B(X) - a|| / (1 + ||a||) and the relative
        dual residual ||C - B^T(y) + Z||_F / (1 + ||C||_F) are all <= eps.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .sdp import Problem

OK, MAXITER, CHOL_BLOCK, CHOL_SCHUR, STEP, UNBOUNDED, NAN = (
    "OK", "MAXITER", "CHOL_BLOCK", "CHOL_SCHUR", "STEP", "UNBOUNDED", "NAN")


@dataclass
class Options:
    sigma: float = 1.0 / 3.0
    tau: float = 0.95
    eps: float = 1e-7
    max_iter: int = 100
    schur: str = "structured"     # or "literal"
    unbounded_tr: float = 1e8     # R-A11 primal-ray test: tr(X) above this ...
    unbounded_eps: float = 1e-8   # ... and ||B(X)||/tr(X), tr(CX)/tr(X) tests


@dataclass
class State:
    X: np.ndarray
    Z: np.ndarray
    y: np.ndarray
    it: int = 0
    history: list = field(default_factory=list)


def start_point(prob: Problem) -> State:
    """Processors initialisation step of Algorithm 2: X = Z = I, y = 0."""
    return State(prob.identity_blocks(), prob.identity_blocks(), np.zeros(prob.K))


def sym(D: np.ndarray) -> np.ndarray:
    return 0.5 * (D + np.swapaxes(D, -1, -2))


def max_step(X: np.ndarray, D: np.ndarray) -> float:
    """sup{t >= 0 : X + t D >= 0} over all blocks (inf if unbounded)."""
    tmax = np.inf
    for Xb, Db in zip(X, D):
        Lc = np.linalg.cholesky(Xb)
        Li = np.linalg.inv(Lc)
        lam = np.linalg.eigvalsh(sym(Li @ Db @ Li.T)).min()
        if lam < 0:
            tmax = min(tmax, -1.0 / lam)
    return tmax


def scalars(prob: Problem, st: State) -> dict:
    """Processors/Root step 4 of Algorithm 2 plus the residuals of R-A11."""
    phi = float(np.einsum("gij,gji->", prob.C, st.X))          # tr(CX)
    psi = float(prob.a @ st.y)                                  # a^T y
    trZX = float(np.einsum("gij,gji->", st.Z, st.X))
    G = prob.C - prob.BT(st.y) + st.Z
    pres = float(np.linalg.norm(prob.Bop(st.X) - prob.a) / (1.0 + np.linalg.norm(prob.a)))
    dres = float(np.sqrt(np.sum(G * G)) / (1.0 + np.sqrt(np.sum(prob.C * prob.C))))
    relgap = abs(psi - phi) / (1.0 + abs(psi) + abs(phi))
    trX = float(np.einsum("gii->", st.X))
    return dict(phi=phi, psi=psi, trZX=trZX, relgap=relgap, pres=pres, dres=dres,
                gap=abs(psi - phi), trX=trX)


def newton_step(prob: Problem, st: State, opt: Options) -> dict:
    """One predictor-corrector iteration (Processors/Root steps 1-3)."""
    X, Z, y = st.X, st.Z, st.y
    nX = prob.nblk * prob.n
    G = prob.C - prob.BT(y) + Z                                  # Eq. (G)
    try:
        Linv = [np.linalg.inv(np.linalg.cholesky(Zb)) for Zb in Z]
    except np.linalg.LinAlgError:
        return dict(status=CHOL_BLOCK)
    Y = np.stack([Li.T @ Li for Li in Linv])                     # Z^{-1} = L^{-T} L^{-1}
    if opt.schur == "literal":
        Om = prob.schur_literal(Y, X)
    else:
        Om = prob.schur_structured(Y, X)
    try:
        Lom = np.linalg.cholesky(Om)
    except np.linalg.LinAlgError:
        return dict(status=CHOL_SCHUR)

    def solve(rhs):
        return np.linalg.solve(Lom.T, np.linalg.solve(Lom, rhs))

    # predictor (Root step 1, Processors step 2)
    omega = prob.Bop(np.einsum("gab,gbc,gcd->gad", Y, G, X))     # B(Z^{-1} G X)
    dyh = solve(omega - prob.a)
    BTdyh = prob.BT(dyh)
    dZh = -G + BTdyh
    dXh = sym(-X + np.einsum("gab,gbc,gcd->gad", Y, G - BTdyh, X))
    # corrector (Root step 2, Processors step 3)
    mu = opt.sigma * float(np.einsum("gij,gji->", Z, X)) / nX
    YdZdX = np.einsum("gab,gbc,gcd->gad", Y, dZh, dXh)
    dyb = solve(mu * prob.Bop(Y) - prob.Bop(YdZdX))
    dZb = prob.BT(dyb)
    dXb = sym(mu * Y - YdZdX - np.einsum("gab,gbc,gcd->gad", Y, dZb, X))
    dX, dZ, dy = dXh + dXb, dZh + dZb, dyh + dyb
    # step lengths and update (Eqs. X, y, Z)
    try:
        tp = min(1.0, opt.tau * max_step(X, dX))
        td = min(1.0, opt.tau * max_step(Z, dZ))
    except np.linalg.LinAlgError:
        # a block no longer numerically positive definite (the iterate is
        # diverging on an infeasible problem): stop as the library does
        return dict(status=CHOL_BLOCK)
    st.X = X + tp * dX
    st.Z = Z + td * dZ
    st.y = y + td * dy
    st.it += 1
    return dict(status=OK, tp=tp, td=td, mu=mu, Omega=Om, dyh=dyh, dyb=dyb,
                dXh=dXh, dZh=dZh, dXb=dXb, dZb=dZb, G=G, Y=Y)


def solve(prob: Problem, opt: Options | None = None, st: State | None = None) -> tuple[str, State]:
    """Iterate until the R-A11 criteria hold (or a failure / the iteration cap)."""
    opt = opt or Options()
    st = st or start_point(prob)
    for _ in range(opt.max_iter):
        info = newton_step(prob, st, opt)
        if info["status"] != OK:
            return info["status"], st
        sc = scalars(prob, st)
        sc.update(tp=info["tp"], td=info["td"], mu=info["mu"])
        st.history.append(sc)
        if not all(np.isfinite([sc["phi"], sc["psi"], sc["pres"], sc["dres"]])):
            return NAN, st
        if sc["relgap"] <= opt.eps and sc["pres"] <= opt.eps and sc["dres"] <= opt.eps:
            return OK, st
        if sc["trX"] > opt.unbounded_tr:
            bx = np.linalg.norm(prob.Bop(st.X))
            if bx / sc["trX"] < opt.unbounded_eps * 1e2 and sc["phi"] / sc["trX"] > opt.unbounded_eps:
                return UNBOUNDED, st
    return MAXITER, st


# --------------------------------------------------------------- dense mode
def _blockdiag(blocks: np.ndarray) -> np.ndarray:
    nb, n, _ = blocks.shape
    out = np.zeros((nb * n, nb * n))
    for g in range(nb):
        out[g * n:(g + 1) * n, g * n:(g + 1) * n] = blocks[g]
    return out


def dense_solve_steps(prob: Problem, steps: int, opt: Options | None = None):
    """The same iteration with X, Z, C and every B_i as full (L+M)n x (L+M)n
    matrices and no block structure assumed anywhere (the setting of Thm 3).
    Returns the list of (X, Z, y) after each step."""
    opt = opt or Options()
    Bl = prob.literal_B()
    Bf = np.stack([_blockdiag(b) for b in Bl])                   # (K, m, m)
    Cf = _blockdiag(prob.C)
    m = Cf.shape[0]
    X, Z, y = np.eye(m), np.eye(m), np.zeros(prob.K)

    def BT(v):
        return np.einsum("i,iab->ab", v, Bf)

    def Bop(W):
        return np.einsum("iab,ba->i", Bf, W)

    def symm(D):
        return 0.5 * (D + D.T)

    def mstep(Xm, Dm):
        Li = np.linalg.inv(np.linalg.cholesky(Xm))
        lam = np.linalg.eigvalsh(symm(Li @ Dm @ Li.T)).min()
        return np.inf if lam >= 0 else -1.0 / lam

    out = []
    for _ in range(steps):
        G = Cf - BT(y) + Z
        Y = np.linalg.inv(Z)
        Om = np.stack([Bop(Y @ Bf[j] @ X) for j in range(prob.K)], axis=1)
        dyh = np.linalg.solve(Om, Bop(Y @ G @ X) - prob.a)
        dZh = -G + BT(dyh)
        dXh = symm(-X + Y @ (G - BT(dyh)) @ X)
        mu = opt.sigma * np.trace(Z @ X) / m
        dyb = np.linalg.solve(Om, mu * Bop(Y) - Bop(Y @ dZh @ dXh))
        dZb = BT(dyb)
        dXb = symm(mu * Y - Y @ dZh @ dXh - Y @ dZb @ X)
        dX, dZ, dy = dXh + dXb, dZh + dZb, dyh + dyb
        tp = min(1.0, opt.tau * mstep(X, dX))
        td = min(1.0, opt.tau * mstep(Z, dZ))
        X, Z, y = X + tp * dX, Z + td * dZ, y + td * dy
        out.append((X.copy(), Z.copy(), y.copy()))
    return out
