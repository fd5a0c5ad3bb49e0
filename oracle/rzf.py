"""Closed-form RZF in FP64 (the result every iteration converges to).

Paper eq. (precoding): F = beta H (H^H H + xi I)^-1 with the paper's
N_t x K channel.  With the K x N_t system matrix H used here (row k is user
k's channel) the auxiliary vector of eq. (symbols) is
    v = (H H^H + xi I)^-1 s,
and the precoded vector is x = H^H v (Remark 1 gives v as the q-part of the
least-norm solution of B w = s, B = [H, sqrt(xi) I]; Remark 2 stacks K
right-hand sides s = e_k to obtain the precoder matrix).

The Gram matrix A = H H^H + xi I is factored by a plain column-by-column
Cholesky (A = L L^H) written out below, then solved by forward and back
substitution.  H is the complex64 channel promoted to complex128.
"""
import numpy as np


def gram(H: np.ndarray, xi: float) -> np.ndarray:
    H = np.asarray(H, dtype=np.complex128)
    return H @ H.conj().T + xi * np.eye(H.shape[0])


def cholesky(A: np.ndarray) -> np.ndarray:
    """Lower-triangular L with A = L L^H for Hermitian positive definite A."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        diag = A[j, j].real - np.sum(np.abs(L[j, :j]) ** 2)
        if not diag > 0.0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        L[j, j] = np.sqrt(diag)
        if j + 1 < n:
            L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j].conj()) / L[j, j].real
    return L


def forward_subst(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    n = L.shape[0]
    Y = np.zeros_like(B, dtype=np.complex128)
    for i in range(n):
        Y[i] = (B[i] - L[i, :i] @ Y[:i]) / L[i, i]
    return Y


def back_subst_h(L: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Solve L^H X = Y."""
    n = L.shape[0]
    X = np.zeros_like(Y, dtype=np.complex128)
    U = L.conj().T
    for i in range(n - 1, -1, -1):
        X[i] = (Y[i] - U[i, i + 1:] @ X[i + 1:]) / U[i, i]
    return X


def rzf(H: np.ndarray, xi: float, S: np.ndarray):
    """Return (V, X): V = (H H^H + xi I)^-1 S (K x nrhs), X = H^H V (Nt x nrhs)."""
    H = np.asarray(H, dtype=np.complex128)
    S = np.asarray(S, dtype=np.complex128)
    vec = S.ndim == 1
    if vec:
        S = S[:, None]
    L = cholesky(gram(H, xi))
    V = back_subst_h(L, forward_subst(L, S))
    X = H.conj().T @ V
    if vec:
        return V[:, 0], X[:, 0]
    return V, X


def rel_err(x, x_ref, axis=0):
    """Column-wise ||x - x_ref|| / ||x_ref|| (the paper's NMSE form, Sec. VII-B)."""
    x = np.asarray(x, dtype=np.complex128)
    x_ref = np.asarray(x_ref, dtype=np.complex128)
    return np.linalg.norm(x - x_ref, axis=axis) / np.linalg.norm(x_ref, axis=axis)
