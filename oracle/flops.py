"""Computational complexity of Table I (FLOPs), transcribed as printed (test
infrastructure and reporting).

Every method forms the precoder matrix once (the K-independent setup terms)
and pays a per-iteration cost times its iteration count T.  The set sizes are
the paper's per-user quantities, here means over users: Q (users per
subarray, eq. (precoding2)), M (VR length; the table's |M| in the VR rows is
read as |Gamma|, the number of visible antennas), X (|X_k|), F and V (sizes of
the orthogonal set and its complement).

Pinned by what lies outside the table: with full visibility (|Gamma| = Nt,
|X| = |Q| = K) the VR-OGRK row equals the GK row, and the leading terms that
Sec. V states hold (8 Nt K^2 against 8 Nt K |Q| for the precoder matrix,
8 Nt K against 8 |Gamma| |X| for the residuals of an iteration).  Parity
unpinned for the lower-order terms of the RZF, URK, SWOR-ERK and VR-OAHK
rows: they follow counting conventions the paper does not state.
"""


def table1_flops(scheme, K, Nt, T=0.0, Q=0.0, M=0.0, X=0.0, F=0.0, V=0.0):
    if scheme == "rzf":
        return 8 * K ** 3 + 9 * K ** 2 + 12 * Nt * K ** 2 - 3 * K
    if scheme == "urk":
        return 8 * Nt * K ** 2 + 4 * Nt * K + T * (16 * Nt - 4)
    if scheme == "swor_erk":
        return 8 * Nt * K ** 2 + 4 * Nt * K + K - 1 + T * (16 * Nt + K + 8)
    if scheme == "gk":
        return 8 * Nt * K ** 2 + 4 * Nt * K - K + T * (8 * Nt * (K + 1) + K - 5)
    if scheme == "vr_ogrk":
        return 8 * Nt * K * (Q + 0.5) - K + T * (8 * M * (X + 1) + K - 5)
    if scheme == "vr_oahk":
        return 8 * Nt * K * (Q + 0.5) + T * (8 * M * (2 * V + F + 2) + 24 * V + 14 * Nt + 5)
    raise ValueError(scheme)
