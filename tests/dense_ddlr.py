"""Dense brute-force DDLR (numpy / LAPACK), used only to pin the oracle.

Everything here is formed densely from the paper's definitions, independently
of the oracle's sparse code: classification (Sec. 2.1), the eq. (Bmat)
reordering, E and A0 of eq. (EF)/(split), H = E^T A0^-1 E and its
eigendecomposition, the DDLR-1 preconditioner of eq. (Mprec) with
G_{k,theta}^-1 from eq. (UDU) using the FULL eigenbasis (not prop. gkt), and
DDLR-2 from an eigendecomposition of E^T A0^-2 E (eq. svd, LR, Form2a).
Only for n up to a few thousand.
"""
from __future__ import annotations

import numpy as np

import workloads as W


class DenseDDLR:
    def __init__(self, A, part, p, alpha=1.0, scale_diag=False):
        Ad = W.to_dense(A)
        n = Ad.shape[0]
        part = np.asarray(part)
        if scale_diag:
            d = 1.0 / np.sqrt(np.diag(Ad))
            Ad = Ad * d[:, None] * d[None, :]
            self.dsc = d
        else:
            self.dsc = None
        off = (Ad != 0) & (part[:, None] != part[None, :])
        iface = off.any(axis=1)
        order = []
        for b in range(p):
            order += [i for i in range(n) if part[i] == b and not iface[i]]
        order += [i for i in range(n) if iface[i]]
        self.perm = np.array(order)
        self.n = n
        self.s = int(iface.sum())
        self.m = n - self.s
        P = Ad[np.ix_(self.perm, self.perm)]
        self.Ap = P
        m, s = self.m, self.s
        B = P[:m, :m]
        Eh = P[:m, m:]
        C = P[m:, m:]
        self.alpha = alpha
        self.E = np.vstack([Eh / alpha, -alpha * np.eye(s)])
        self.A0 = np.zeros((n, n))
        self.A0[:m, :m] = B + (Eh @ Eh.T) / alpha ** 2
        self.A0[m:, m:] = C + alpha ** 2 * np.eye(s)
        self.A0inv = np.linalg.inv(self.A0)
        self.H = self.E.T @ self.A0inv @ self.E
        self.H = 0.5 * (self.H + self.H.T)
        lam, U = np.linalg.eigh(self.H)
        idx = np.argsort(-lam, kind="stable")
        self.lam = lam[idx]
        self.Ufull = U[:, idx]

    def minv_ddlr1(self, k, theta_mode=1):
        """M^-1 in eq. Bmat order, G_{k,theta}^-1 from the full eigenbasis."""
        s = self.s
        lt = self.lam.copy()
        theta = self.lam[k] if (theta_mode == 1 and k < s) else 0.0
        lt[k:] = theta
        Ginv = self.Ufull @ np.diag(1.0 / (1.0 - lt)) @ self.Ufull.T
        X = self.A0inv @ self.E
        return self.A0inv + X @ Ginv @ X.T, theta

    def minv_ddlr2(self, k):
        X = self.A0inv @ self.E
        K2 = X.T @ X
        K2 = 0.5 * (K2 + K2.T)
        mu, V = np.linalg.eigh(K2)
        idx = np.argsort(-mu, kind="stable")
        Vk = V[:, idx[:k]]
        Uk = X @ Vk
        Hk = np.linalg.inv(np.eye(k) - Uk.T @ self.E @ Vk)
        Hk = 0.5 * (Hk + Hk.T)
        return self.A0inv + Uk @ Hk @ Uk.T

    def to_original(self, Mp):
        """Matrix in eq. Bmat order -> original order (and undo scaling)."""
        n = self.n
        M = np.zeros((n, n))
        M[np.ix_(self.perm, self.perm)] = Mp
        if self.dsc is not None:
            M = M * self.dsc[:, None] * self.dsc[None, :]
        return M


def oracle_matrix(orc, n):
    """Columns M^-1 e_j from the oracle's apply."""
    M = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        M[:, j] = orc.apply(e)
    return M
