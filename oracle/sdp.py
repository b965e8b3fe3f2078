"""SDP elements of Sec. III-B and the Schur complement (oracle; test-only).

Primal (Eq. primal):  max tr(CX)  s.t.  B(X) = a, X >= 0.
Dual   (Eq. dual):    min a^T y   s.t.  B^T(y) - C = Z >= 0.

All block-diagonal matrices are stored as arrays of shape (L+M, n, n): the L
"P-side" blocks gamma in W_{d_p+d1} first, then the M "Lyapunov" blocks gamma
in W_{d_p+d_a+d2}, both in the paper's lexicographic order.

Basis of S^n (Sec. I).  E_k for k <= n is the diagonal unit matrix e_k e_k^T.
The paper defines E_k = F_k + F_k^T for k > n only on the first superdiagonal
(k <= 2n-1); the oracle extends the printed pattern diagonal by diagonal:
offset 1 pairs (1,2),(2,3),...,(n-1,n), then offset 2 pairs (1,3),..., and so
on, each E = e_r e_s^T + e_s e_r^T with unit entries.  With this basis the dual
variable y_{q + Ntil*(h-1)} equals the (r,s) entry of P_h.

Variables: i <-> (h, q), i = q + Ntil*h (0-based), Eq. (V_h).
"""

from __future__ import annotations

import numpy as np

from . import polya


# ---------------------------------------------------------------- basis / svec
def svec_pairs(n: int) -> list[tuple[int, int]]:
    """0-based (r, s), r <= s, in the basis order: diagonal, then offsets 1, 2, ..."""
    out = [(r, r) for r in range(n)]
    for off in range(1, n):
        out += [(r, r + off) for r in range(n - off)]
    return out


def basis_matrix(n: int, k: int) -> np.ndarray:
    """E_k (0-based k) as a dense n x n matrix."""
    r, s = svec_pairs(n)[k]
    E = np.zeros((n, n))
    E[r, s] = 1.0
    E[s, r] = 1.0
    return E


def smat(v: np.ndarray, n: int) -> np.ndarray:
    """V_h restricted to one coefficient: sum_j E_j v_j."""
    M = np.zeros((n, n))
    for k, (r, s) in enumerate(svec_pairs(n)):
        M[r, s] = v[k]
        M[s, r] = v[k]
    return M


def svec_adjoint(W: np.ndarray) -> np.ndarray:
    """(tr(E_k W))_k for a (not necessarily symmetric) n x n W."""
    n = W.shape[0]
    out = np.empty(n * (n + 1) // 2)
    for k, (r, s) in enumerate(svec_pairs(n)):
        out[k] = W[r, r] if r == s else W[r, s] + W[s, r]
    return out


# -------------------------------------------------------------------- problem
class Problem:
    """The SDP of Eqs. (C), (Cj), (Ai), (Aij), (a) for one system A(alpha).

    A is an array (N_a, n, n) of the coefficients A_lambda, lambda in W_{d_a}
    (for the affine case d_a = 1 these are A_1 ... A_l).
    """

    def __init__(self, A, d_p: int, d1: int, d2: int | None = None, d_a: int = 1,
                 delta: float = 1.0, delta_L: float = 0.0, R=None, d_r: int | None = None, a=None):
        """R, d_r: the constant term of the generalised inequality of Sec. III-C
        (Eq. LMI_general with one term, A~ = A(alpha)^T, B~ = I):
        A(alpha)^T P(alpha) + P(alpha) A(alpha) + R(alpha) < 0 with R(alpha) =
        sum_rho R_rho alpha^rho homogeneous of degree d_r <= d_p + d_a + d2
        (coefficients (card W_{d_r}, n, n), symmetric).  a: the dual objective
        vector (K values), the paper's all-ones vector (Eq. a) by default."""
        A = np.asarray(A, dtype=np.float64)
        self.A = A
        self.n = A.shape[-1]
        self.d_p, self.d1 = d_p, d1
        self.d2 = d1 if d2 is None else d2
        self.d_a = d_a
        self.l = self._infer_l(A.shape[0], d_a)
        self.delta, self.delta_L = delta, delta_L
        sz = polya.sizes(self.n, self.l, d_p, d1, self.d2, d_a)
        self.L0, self.L, self.M, self.Nt, self.K = sz["L0"], sz["L"], sz["M"], sz["Ntil"], sz["K"]
        self.nblk = self.L + self.M
        self.beta = polya.beta_table(self.l, d_p, d1)                   # (L0, L)
        self.c = polya.h_coeff_table(self.l, d_p, d_a, self.d2)         # (L0, M, Na)
        self.H = polya.h_matrices(self.c, A)                            # (L0, M, n, n)
        self.a = np.ones(self.K) if a is None else np.asarray(a, dtype=np.float64)   # Eq. (a)
        if self.a.shape != (self.K,):
            raise ValueError("objective vector a must have K entries")
        self.R, self.d_r = None, None
        if R is not None:
            self.d_r = int(d_r)
            self.R = np.asarray(R, dtype=np.float64)
            if self.d_r > self.d_p + self.d_a + self.d2 or \
                    self.R.shape != (polya.f_card(self.l, self.d_r), self.n, self.n):
                raise ValueError("R must hold card(W_{d_r}) n x n coefficients, d_r <= d_p + d_a + d2")
        self.CR = self._build_CR()                                      # R's part of the Lyapunov C
        self.C = self._build_C()

    @staticmethod
    def _infer_l(Na: int, d_a: int) -> int:
        l = 1
        while polya.f_card(l, d_a) < Na:
            l += 1
        if polya.f_card(l, d_a) != Na:
            raise ValueError("number of A coefficients is not card(W_{d_a}) for any l")
        return l

    def _build_CR(self) -> np.ndarray:
        """Lyapunov-block coefficients of (sum alpha)^e R(alpha), e = d_p + d_a +
        d2 - d_r, the degree of the Lyapunov inequality: on the simplex the
        inequality with R(alpha) and its homogenised form agree, and the dual
        constraint B^T(y)_gamma - C_gamma >= 0 of block gamma then reads
        -(coefficient of A^T P + P A) - R_gamma >= 0."""
        n = self.n
        CR = np.zeros((self.M, n, n))
        if self.R is None:
            return CR
        e = self.d_p + self.d_a + self.d2 - self.d_r
        Wr = polya.monomials(self.l, self.d_r)
        Wpa = polya.monomials(self.l, self.d_p + self.d_a + self.d2)
        for j, g in enumerate(Wpa):
            for k, rho in enumerate(Wr):
                rest = tuple(gi - ri for gi, ri in zip(g, rho))
                if min(rest) >= 0:
                    CR[j] += polya.multinomial(e, rest) * self.R[k]
        return CR

    def _build_C(self) -> np.ndarray:
        """Eq. (Cj): delta*I*sum_h beta_{h,j} d_p!/h! on P-side blocks, 0 (or
        the optional strict margin delta_L*...) on the Lyapunov blocks, plus R's
        coefficients there (generalised form)."""
        n = self.n
        W0 = polya.monomials(self.l, self.d_p)
        w = np.array([polya.multinomial(self.d_p, h) for h in W0], dtype=np.float64)
        C = np.zeros((self.nblk, n, n))
        for j in range(self.L):
            C[j] = self.delta * np.eye(n) * float(self.beta[:, j] @ w)
        if self.delta_L != 0.0:
            Wpa = polya.monomials(self.l, self.d_p + self.d_a + self.d2)
            for j, g in enumerate(Wpa):
                C[self.L + j] = self.delta_L * np.eye(n) * polya.multinomial(sum(g), g)
        C[self.L:] += self.CR
        return C

    # ------------------------------------------------------------ literal B_i
    def literal_B(self) -> np.ndarray:
        """Every B_i (Eq. Aij) materialised: array (K, L+M, n, n)."""
        n, K = self.n, self.K
        B = np.zeros((K, self.nblk, n, n))
        for i in range(K):
            h, q = divmod(i, self.Nt)
            E = basis_matrix(n, q)              # V_h(e_i) for this h, zero for others
            for j in range(self.L):
                B[i, j] = self.beta[h, j] * E
            for j in range(self.M):
                Hh = self.H[h, j]
                B[i, self.L + j] = -(Hh.T @ E + E @ Hh)
        return B

    # ------------------------------------------------- structured B^T and B
    def BT(self, v: np.ndarray) -> np.ndarray:
        """B^T(v) = sum_i v_i B_i (Eq. AT), block by block."""
        n = self.n
        P = np.stack([smat(v[h * self.Nt:(h + 1) * self.Nt], n) for h in range(self.L0)])
        out = np.zeros((self.nblk, n, n))
        for j in range(self.L):
            out[j] = np.einsum("h,hij->ij", self.beta[:, j].astype(np.float64), P)
        for j in range(self.M):
            acc = np.zeros((n, n))
            for h in range(self.L0):
                Hh = self.H[h, j]
                acc += Hh.T @ P[h] + P[h] @ Hh
            out[self.L + j] = -acc
        return out

    def Bop(self, W: np.ndarray) -> np.ndarray:
        """B(W) = (tr(B_i W))_i for block-diagonal W (blocks need not be symmetric)."""
        out = np.zeros(self.K)
        for h in range(self.L0):
            acc = np.zeros(self.Nt)
            for j in range(self.L):
                if self.beta[h, j]:
                    acc += self.beta[h, j] * svec_adjoint(W[j])
            for j in range(self.M):
                Hh = self.H[h, j]
                # tr((H^T E + E H) W) = tr(E (W H^T + H W))
                acc -= svec_adjoint(W[self.L + j] @ Hh.T + Hh @ W[self.L + j])
            out[h * self.Nt:(h + 1) * self.Nt] = acc
        return out

    # ----------------------------------------------------- Schur complement
    def schur_literal(self, Y: np.ndarray, X: np.ndarray, B: np.ndarray | None = None) -> np.ndarray:
        """Omega_ij = tr(B_i Z^{-1} B_j X) straight from the definition (Sec. IV-A),
        Y = Z^{-1} given per block.  Only for small K."""
        if B is None:
            B = self.literal_B()
        Wj = np.einsum("gab,jgbc,gcd->jgad", Y, B, X)          # Y B_j X per block
        return np.einsum("igab,jgba->ij", B, Wj)

    def schur_terms(self, a: int, b: int, Y: np.ndarray, X: np.ndarray):
        """(Psi, Phi) pairs with Omega_{(a,p),(b,q)} = sum tr(E_p Psi E_q Phi).

        P-side block gamma: beta_a beta_b tr(E_p Y E_q X).
        Lyapunov block: (H_a^T E_p + E_p H_a) Y (H_b^T E_q + E_q H_b) X expands,
        by cyclicity of the trace, into the four (Psi, Phi) pairs
        (Y H_b^T, X H_a^T), (Y, H_b X H_a^T), (H_a Y H_b^T, X), (H_a Y, H_b X).
        """
        terms = []
        for j in range(self.L):
            w = float(self.beta[a, j] * self.beta[b, j])
            if w != 0.0:
                terms.append((w * Y[j], X[j]))
        for j in range(self.M):
            g = self.L + j
            Ha, Hb = self.H[a, j], self.H[b, j]
            terms.append((Y[g] @ Hb.T, X[g] @ Ha.T))
            terms.append((Y[g], Hb @ X[g] @ Ha.T))
            terms.append((Ha @ Y[g] @ Hb.T, X[g]))
            terms.append((Ha @ Y[g], Hb @ X[g]))
        return terms

    def schur_structured(self, Y: np.ndarray, X: np.ndarray, blocks=None) -> np.ndarray:
        """Omega from the block formula: for basis pairs p=(r,s), q=(k,m),
        tr(E_p Psi E_q Phi) = sum over ordered (i,v) with {i,v} = {r,s} and
        ordered (j,u) with {j,u} = {k,m} of Psi[i,j] * Phi[u,v].
        blocks: optional list of (a, b) blocks to form (the others stay zero);
        a timing sample of the full computation, same arithmetic."""
        n, Nt = self.n, self.Nt
        pairs = svec_pairs(n)
        r = np.array([p[0] for p in pairs])
        s = np.array([p[1] for p in pairs])
        offdiag = (r != s).astype(np.float64)
        # the two orderings (i, v) of p: (r, s) and, off the diagonal, (s, r)
        orders = [(r, s, np.ones(Nt)), (s, r, offdiag)]
        Om = np.zeros((self.K, self.K))
        for a in range(self.L0):
            for b in range(self.L0):
                if blocks is not None and (a, b) not in blocks:
                    continue
                terms = self.schur_terms(a, b, Y, X)
                Psi = np.stack([t[0].reshape(-1) for t in terms])     # (T, n*n), index i*n+j
                Phi = np.stack([t[1].reshape(-1) for t in terms])     # (T, n*n), index u*n+v
                T = (Psi.T @ Phi).reshape(n, n, n, n)                 # T[i,j,u,v]
                blk = np.zeros((Nt, Nt))
                for (i, v, wp) in orders:
                    for (j, u, wq) in orders:
                        vals = T[i[:, None], j[None, :], u[None, :], v[:, None]]
                        blk += wp[:, None] * wq[None, :] * vals
                Om[a * Nt:(a + 1) * Nt, b * Nt:(b + 1) * Nt] = blk
        return Om

    def schur_matvec(self, Y: np.ndarray, X: np.ndarray, v: np.ndarray) -> np.ndarray:
        """Omega v = B(Z^{-1} B^T(v) X) without forming Omega."""
        S = self.BT(v)
        return self.Bop(np.einsum("gab,gbc,gcd->gad", Y, S, X))

    # ----------------------------------------------------------- utilities
    def identity_blocks(self) -> np.ndarray:
        return np.broadcast_to(np.eye(self.n), (self.nblk, self.n, self.n)).copy()

    def P_from_y(self, y: np.ndarray) -> np.ndarray:
        """Root step 4 of Algorithm 2: P_h = sum_j E_j y_{j + Ntil (h-1)}."""
        return np.stack([smat(y[h * self.Nt:(h + 1) * self.Nt], self.n) for h in range(self.L0)])
