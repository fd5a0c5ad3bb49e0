"""Per-user SINR and spectral efficiency of a precoder (eq. (rate)).

With received signal y_k = sqrt(rho) h_k^H F s + n_k and E[s s^H] = I, user
k's SINR is |h_k^H f_k|^2 / (sum_{i != k} |h_k^H f_i|^2 + sigma^2 / rho) and
its rate is log2(1 + SINR_k).  Here row k of the K x Nt matrix H plays the
role of h_k^H, F = beta X with X = H^H V the unnormalised precoder of
eq. (precoding1), and beta = 1 / ||X||_F meets the power budget
||F||_F^2 <= 1 of eq. (power) with equality (the paper does not spell beta
out).  ``snr_lin`` is rho / sigma^2.
"""
import numpy as np


def sinr(H, X, snr_lin):
    H = np.asarray(H, dtype=np.complex128)
    X = np.asarray(X, dtype=np.complex128)
    F = X / np.linalg.norm(X)
    G = H @ F  # G[k, i] = h_k^H f_i
    K = G.shape[0]
    out = np.zeros(K)
    for k in range(K):
        sig = abs(G[k, k]) ** 2
        interf = sum(abs(G[k, i]) ** 2 for i in range(G.shape[1]) if i != k)
        out[k] = sig / (interf + 1.0 / snr_lin)
    return out


def rates(H, X, snr_lin):
    return np.log2(1.0 + sinr(H, X, snr_lin))


def sinr_db(H, X, snr_lin):
    return 10.0 * np.log10(sinr(H, X, snr_lin))
