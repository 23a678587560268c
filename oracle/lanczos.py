"""Condition estimate of the preconditioned operator from CG coefficients -- test infrastructure.

The Lanczos tridiagonal T_k hidden in preconditioned CG (Saad, Iterative Methods
for Sparse Linear Systems, Sec. 6.7.3):
    T[j, j]   = 1/alpha_j + beta_{j-1}/alpha_{j-1}   (beta_{-1} = 0)
    T[j, j+1] = sqrt(beta_j) / alpha_j
Its extreme eigenvalues approximate those of M A; kappa(M A) ~ lambda_max / lambda_min.
Used to check the practical bound kappa(M A) <= 2 (beta + 3) (Remark after Lemma
"condition number estimate", Section 5.1).
"""
import numpy as np


def lanczos_tridiagonal(alphas, betas):
    a = np.asarray(alphas, np.float64)
    b = np.asarray(betas, np.float64)
    k = len(a)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / a[j] + (b[j - 1] / a[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(b[j]) / a[j]
    return T


def kappa_estimate(alphas, betas):
    ev = np.linalg.eigvalsh(lanczos_tridiagonal(alphas, betas))
    return ev[-1] / ev[0], ev[0], ev[-1]
