"""Subarray-wise precoder assembly (Sec. IV-B, eq. (precoding2)) in FP64 (test
infrastructure).

The array is split into S subarrays of consecutive antennas (subarray s holds
antennas [s Nt // S, (s + 1) Nt // S); the paper takes Nt / S integral).
Q_s is the set of users whose VR includes (meets) subarray s, and H_s the
channel between subarray s and the users.  With the K x Nt system matrix H of
this package (row k = user k's channel, so the paper's Nt x K channel is
H^H), the paper's [H_s]_{Q_s} [V]_{Q_s} is

    F_s = H[Q_s, subarray s]^H  V[Q_s, :]

and F stacks the F_s over s.  Rows of H outside Q_s vanish on subarray s, so F
equals the dense H^H V while touching only |Q_s| rows per subarray.  The
power-normalised precoder is beta F with beta = 1 / ||F||_F (eq. (power) met
with equality; the paper leaves beta implicit).
"""
import numpy as np


def subarray_bounds(Nt, S):
    """[(n0, n1)] of the S subarrays."""
    return [(s * Nt // S, (s + 1) * Nt // S) for s in range(S)]


def q_sets(vr_offset, vr_len, Nt, S):
    """Q_s for every subarray: users whose VR [o, o + L) meets the subarray."""
    out = []
    for n0, n1 in subarray_bounds(Nt, S):
        out.append([k for k in range(len(vr_len))
                    if int(vr_offset[k]) < n1 and int(vr_offset[k]) + int(vr_len[k]) > n0])
    return out


def subarray_precoder(H, V, vr_offset, vr_len, S):
    """F (Nt x ncols) by the subarray-wise form, from the dense K x Nt H and V (K x ncols)."""
    H = np.asarray(H, dtype=np.complex128)
    V = np.asarray(V, dtype=np.complex128)
    Nt = H.shape[1]
    F = np.zeros((Nt, V.shape[1]), dtype=np.complex128)
    for (n0, n1), Q in zip(subarray_bounds(Nt, S), q_sets(vr_offset, vr_len, Nt, S)):
        if Q:
            F[n0:n1, :] = H[Q, n0:n1].conj().T @ V[Q, :]
    return F


def normalise(F):
    """(beta F, beta) with beta = 1 / ||F||_F."""
    beta = 1.0 / np.linalg.norm(F)
    return beta * F, beta
