"""Incremental SVD and DMD reduced operators of the oracle (test infrastructure).

App. B (Brand's rank-one update of a thin SVD) and Sec. 3.1 Eq. (dmd-operator):
given R_{m-1} ~ U S V^T and a new column x,
    p = U^T x,  q~ = x - U p,  alpha = ||q~||,  q = q~ / alpha
    [R_{m-1} x] ~ [U q] K [[V^T, 0], [0, 1]],   K = [[S, p], [0, alpha]]     (Eq. (svd_core))
    K = U_c S_c V_c^T,  U <- [U q] U_c,  S <- S_c,  V <- [[V, 0], [0, 1]] V_c.
The DMD operator A_r = U^T B V S^{-1} needs only W = B V, which updates as
    W <- [W b] V_c,
so V itself is never kept.  The reduced solve A_r c = U^T b_tilde is a dense LU
with partial pivoting (Sec. 4), here numpy.linalg.solve.

Readings where the paper leaves a choice:
* q~ is orthogonalised twice (classical Gram-Schmidt, repeated once).
* If alpha <= 1e-12 ||x|| the rank does not grow: the column q is dropped together
  with the last singular triple of K (then exactly zero), Brand's rank-preserving case.
* Singular values are kept in descending order, so s[-1] is the smallest.
* truncate(eps): keep s_k with s_k / sum(s) > eps; then keep at most r_max.
"""
import numpy as np

GROWTH_TOL = 1e-12


class IncrementalSVD:
    def __init__(self, n: int, r_max: int):
        self.n = n
        self.r_max = r_max
        self.U = np.zeros((n, 0))
        self.S = np.zeros(0)
        self.W = np.zeros((n, 0))

    @property
    def rank(self):
        return self.S.size

    def append(self, x, b, trunc_eps=None):
        """Append the snapshot pair (x, b): R <- [R x], B <- [B b] (Eq. (snapshots)).

        Returns True when the rank grew (the new column was not in span U).
        """
        x = np.asarray(x, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        xn = float(np.linalg.norm(x))
        p = self.U.T @ x
        q = x - self.U @ p
        p2 = self.U.T @ q
        q = q - self.U @ p2
        p = p + p2
        alpha = float(np.linalg.norm(q))
        grew = alpha > GROWTH_TOL * xn
        r = self.rank
        K = np.zeros((r + 1, r + 1))
        K[:r, :r] = np.diag(self.S)
        K[:r, r] = p
        K[r, r] = alpha if grew else 0.0
        Uc, Sc, Vct = np.linalg.svd(K)
        Vc = Vct.T
        qcol = (q / alpha) if grew else np.zeros_like(q)
        U_new = np.hstack([self.U, qcol[:, None]]) @ Uc
        W_new = np.hstack([self.W, b[:, None]]) @ Vc
        keep = r + 1 if grew else r
        if trunc_eps is not None and keep > 0:
            tot = float(np.sum(Sc[:keep]))
            keep = int(np.sum(Sc[:keep] / tot > trunc_eps))
        keep = min(keep, self.r_max)
        self.U = U_new[:, :keep]
        self.S = Sc[:keep].copy()
        self.W = W_new[:, :keep]
        return grew

    def stop_ratio(self, grew: bool):
        """s_m / sum_k s_k for the current snapshot count (Eq. (ig_stop), Eq. (pc_stop)).

        A snapshot that did not grow the rank makes s_m = 0."""
        if not grew or self.rank == 0:
            return 0.0
        return float(self.S[-1] / np.sum(self.S))

    def operator(self):
        """A_r = U^T W S^{-1} (Eq. (dmd-operator))."""
        return (self.U.T @ self.W) / self.S[None, :]

    def solve_apply(self, rhs):
        """U c with A_r c = U^T rhs (Eq. (dmd-ig) / Eq. (dmd-sa))."""
        c = np.linalg.solve(self.operator(), self.U.T @ rhs)
        return self.U @ c
