"""Seeded synthetic near-field scenarios shared by the CUDA path and the oracle.

This module only draws inputs: user positions, visibility regions (VRs),
the spherical-wave line-of-sight channel restricted to each VR, the symbol
vectors and the regularisation factor.  It contains none of the precoding
arithmetic, so both sides of every parity test can consume it.

Conventions (paper Sec. II, eqs. (1)-(5) and the simulation set-up of Sec. VII):

* The array is an ``Nt``-element half-wavelength ULA on the x axis centred at
  the origin; antenna ``n`` (0-based) sits at ``x_n = (n - (Nt-1)/2) * lam/2``.
* User ``k`` is at distance ``r_k ~ U[5, 50]`` m and angle ``theta_k ~
  U[-60, 60]`` degrees measured from broadside, so its distance to antenna
  ``n`` is ``sqrt(r^2 + x_n^2 - 2 r x_n sin(theta))`` (law of cosines, eq. (2)
  with the angle taken from broadside).
* The channel gain from antenna ``n`` to user ``k`` is
  ``(lam / (4 pi r_kn)) exp(-j 2 pi r_kn / lam)`` on the user's VR and zero
  elsewhere (eqs. (3)-(4)).  Each VR is one contiguous antenna interval
  ``[vr_offset[k], vr_offset[k] + vr_len[k])``.
* The whole instance is multiplied by one real scalar so that the mean of
  ``|h_kn|^2`` over visible entries is 1, then rounded to complex64.  This
  keeps the relative path loss between users and puts RZF in its usual
  regime (``||h_k||^2 ~ vr_len[k]`` against ``xi = K / SNR``).
* Row ``k`` of the K x Nt system matrix ``H`` is user ``k``'s channel, so the
  received vector is ``y = H x``.  ``H_packed`` stores row ``k``'s VR slice at
  ``sum(vr_len[:k])``.
* Symbols are QPSK ``((1 - 2 b0) + j (1 - 2 b1)) / sqrt(2)``, or the identity
  (one canonical basis vector per right-hand side, the precoder-matrix case of
  Remark 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299_792_458.0
BASE_SEED = 2501_10689


@dataclass
class Instance:
    K: int
    Nt: int
    vr_offset: np.ndarray  # int32 [K]
    vr_len: np.ndarray  # int32 [K]
    H_packed: np.ndarray  # complex64 [sum(vr_len)]
    S: np.ndarray  # complex64 [K, nrhs]
    xi: float
    snr_db: float
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def nrhs(self) -> int:
        return int(self.S.shape[1])

    @property
    def row_ptr(self) -> np.ndarray:
        rp = np.zeros(self.K + 1, dtype=np.int64)
        rp[1:] = np.cumsum(self.vr_len.astype(np.int64))
        return rp

    def dense(self) -> np.ndarray:
        """K x Nt complex64 matrix with zeros outside the VRs."""
        return dense_from_packed(self.H_packed, self.vr_offset, self.vr_len, self.Nt)


def dense_from_packed(H_packed, vr_offset, vr_len, Nt) -> np.ndarray:
    K = len(vr_len)
    out = np.zeros((K, Nt), dtype=H_packed.dtype)
    p = 0
    for k in range(K):
        o, L = int(vr_offset[k]), int(vr_len[k])
        out[k, o:o + L] = H_packed[p:p + L]
        p += L
    return out


def qpsk(rng: np.random.Generator, K: int, nrhs: int) -> np.ndarray:
    b = rng.integers(0, 2, size=(K, nrhs, 2))
    return (((1 - 2 * b[..., 0]) + 1j * (1 - 2 * b[..., 1])) / np.sqrt(2.0)).astype(np.complex64)


def make_instance(seed: int, K: int, Nt: int, *, vr_len_range=None, vr_frac_range=None,
                  fc: float = 28e9, snr_db: float = 10.0, nrhs: int = 1, rhs: str = "qpsk",
                  r_range=(5.0, 50.0), theta_deg_range=(-60.0, 60.0),
                  vr_override=None) -> Instance:
    """Draw one seeded near-field channel instance.

    ``vr_len_range=(lo, hi)`` draws integer VR lengths uniformly in [lo, hi];
    ``vr_frac_range=(a, b)`` draws ``round(U[a, b] * Nt)``.  Offsets are
    uniform integers in ``[0, Nt - L]``.  ``vr_override=(offsets, lengths)``
    fixes the VRs (used for structured edge cases).
    """
    if K < 1 or Nt < 1:
        raise ValueError("K and Nt must be positive")
    rng = np.random.default_rng(seed)
    lam = C_LIGHT / fc
    d = lam / 2.0
    r = rng.uniform(r_range[0], r_range[1], size=K)
    theta = np.deg2rad(rng.uniform(theta_deg_range[0], theta_deg_range[1], size=K))
    if vr_override is not None:
        off = np.asarray(vr_override[0], dtype=np.int64)
        L = np.asarray(vr_override[1], dtype=np.int64)
    else:
        if vr_len_range is not None:
            L = rng.integers(int(vr_len_range[0]), int(vr_len_range[1]) + 1, size=K)
        elif vr_frac_range is not None:
            L = np.rint(rng.uniform(vr_frac_range[0], vr_frac_range[1], size=K) * Nt).astype(np.int64)
        else:
            L = np.full(K, Nt, dtype=np.int64)
        L = np.clip(L, 1, Nt)
        off = np.array([rng.integers(0, Nt - int(Lk) + 1) for Lk in L], dtype=np.int64)
    if np.any(L < 1) or np.any(off < 0) or np.any(off + L > Nt):
        raise ValueError("VR outside the array")
    xs = (np.arange(Nt, dtype=np.float64) - (Nt - 1) / 2.0) * d
    segs = []
    for k in range(K):
        xn = xs[off[k]:off[k] + L[k]]
        rkn = np.sqrt(r[k] ** 2 + xn ** 2 - 2.0 * r[k] * xn * np.sin(theta[k]))
        segs.append((lam / (4.0 * np.pi * rkn)) * np.exp(-2j * np.pi * rkn / lam))
    g = np.concatenate(segs)
    scale = 1.0 / np.sqrt(np.mean(np.abs(g) ** 2))
    Hp = (g * scale).astype(np.complex64)
    if rhs == "qpsk":
        S = qpsk(rng, K, nrhs)
    elif rhs == "identity":
        if nrhs != K:
            raise ValueError("identity right-hand sides need nrhs == K")
        S = np.eye(K, dtype=np.complex64)
    else:
        raise ValueError(f"unknown rhs kind {rhs!r}")
    xi = K * 10.0 ** (-snr_db / 10.0)
    return Instance(K=K, Nt=Nt, vr_offset=off.astype(np.int32), vr_len=L.astype(np.int32),
                    H_packed=Hp, S=S, xi=float(xi), snr_db=float(snr_db), seed=int(seed),
                    meta={"r": r, "theta": theta, "fc": fc, "scale": scale})


# The five workloads.  Seeds: BASE_SEED + 1000 * index (+ instance number).
def config1(seed_offset: int = 0) -> Instance:
    """Single-RHS GRK case: Nt=256, K=16, VR 64-192, SNR 10 dB."""
    return make_instance(BASE_SEED + seed_offset, 16, 256, vr_len_range=(64, 192), snr_db=10.0, nrhs=1)


def config2(snr_db: float = 10.0, nrhs: int = 256, seed_offset: int = 0) -> Instance:
    """Shared-channel multi-RHS case: Nt=1024, K=64, VR 128-512, 256 QPSK vectors."""
    return make_instance(BASE_SEED + 1000 + seed_offset, 64, 1024, vr_len_range=(128, 512),
                         snr_db=snr_db, nrhs=nrhs)


def config3_instance(i: int, nrhs: int = 16, snr_db: float = 10.0) -> Instance:
    """Instance ``i`` of the uneven batch: Nt in {1024, 2048, 4096}, K in U{32..256},
    VR lengths round(U[0.1, 0.4] * Nt), 16 QPSK vectors."""
    seed = BASE_SEED + 2000 + i
    rng = np.random.default_rng(seed ^ 0x5EED)
    Nt = int(rng.choice([1024, 2048, 4096]))
    K = int(rng.integers(32, 257))
    return make_instance(seed, K, Nt, vr_frac_range=(0.10, 0.40), snr_db=snr_db, nrhs=nrhs)


def config3(n: int = 512, nrhs: int = 16, start: int = 0):
    return [config3_instance(start + i, nrhs=nrhs) for i in range(n)]


def config4(nrhs: int = 64, seed_offset: int = 0) -> Instance:
    """Large ELAA case: Nt=16384, K=512, VR 1024-4096, 64 QPSK vectors."""
    return make_instance(BASE_SEED + 3000 + seed_offset, 512, 16384, vr_len_range=(1024, 4096),
                         snr_db=10.0, nrhs=nrhs)


def config5_instance(i: int, rhs: str = "identity", nrhs: int = 128, snr_db: float = 10.0) -> Instance:
    """Channel ``i`` of the gradient batch: Nt=2048, K=128, VR 256-1024."""
    return make_instance(BASE_SEED + 4000 + i, 128, 2048, vr_len_range=(256, 1024), snr_db=snr_db,
                         nrhs=nrhs, rhs=rhs)


def paper_scenario(seed: int, *, Nt: int = 2000, K: int = 30, S: int = 20, p: float = 0.35, L: int = 5,
                   fc: float = 100e9, snr_db: float = 0.0, r_range=(1.0, 50.0),
                   theta_deg_range=(30.0, 150.0)) -> Instance:
    """The paper's simulation scenario (Sec. II eqs. (1)-(5), Sec. VII): an
    Nt-antenna half-wavelength ULA cut into S subarrays of Nt / S antennas,
    K users with L paths each (line of sight from the user, L - 1 from
    scatterers), every subarray visible to a user with probability p.

    Readings of what the paper leaves open: users and scatterers at distance
    U[r_range] and angle U[theta_deg_range] measured from the array axis (the
    paper places a point at (d cos(theta), d sin(theta))); path gains
    beta ~ CN(0, 1); an empty visibility set is replaced by one subarray drawn
    uniformly; every user's channel is scaled to ||h_k|| = 1 (equal per-user
    SNR_k = rho ||h_k||^2 / sigma^2 under power control), so the
    regularisation is the paper's xi = 1 / SNR; identity right-hand sides (the
    precoder matrix).

    The library takes one contiguous interval per user: each VR is stored as
    its hull (first to last visible subarray) with exact zeros on the invisible
    subarrays in between.  meta["M"] lists each user's visible subarrays.
    """
    if Nt % S:
        raise ValueError("Nt / S must be an integer")
    rng = np.random.default_rng(seed)
    lam = C_LIGHT / fc
    d = lam / 2.0
    xs = (np.arange(Nt, dtype=np.float64) - (Nt - 1) / 2.0) * d
    sub = Nt // S
    rows, offs, lens, Ms = [], [], [], []
    for k in range(K):
        dist = rng.uniform(r_range[0], r_range[1], size=L)
        th = np.deg2rad(rng.uniform(theta_deg_range[0], theta_deg_range[1], size=L))
        beta = (rng.normal(size=L) + 1j * rng.normal(size=L)) / np.sqrt(2.0)
        h = np.zeros(Nt, dtype=np.complex128)
        for l in range(L):
            dn = np.sqrt(dist[l] ** 2 + xs ** 2 - 2.0 * xs * dist[l] * np.cos(th[l]))
            h += beta[l] * np.exp(-2j * np.pi * (dn - dist[l]) / lam) / np.sqrt(Nt)
        h *= np.sqrt(Nt / L)
        vis = rng.random(S) < p
        if not vis.any():
            vis[int(rng.integers(0, S))] = True
        M = np.nonzero(vis)[0]
        mask = np.repeat(vis, sub)
        h = h * mask
        h /= np.linalg.norm(h)
        o, e = int(M[0]) * sub, (int(M[-1]) + 1) * sub
        rows.append(h[o:e])
        offs.append(o)
        lens.append(e - o)
        Ms.append([int(s_) for s_ in M])
    Hp = np.concatenate(rows).astype(np.complex64)
    S_ = np.eye(K, dtype=np.complex64)
    xi = 10.0 ** (-snr_db / 10.0)
    return Instance(K=K, Nt=Nt, vr_offset=np.array(offs, dtype=np.int32), vr_len=np.array(lens, dtype=np.int32),
                    H_packed=Hp, S=S_, xi=float(xi), snr_db=float(snr_db), seed=int(seed),
                    meta={"M": Ms, "S": S, "p": p, "L": L, "fc": fc})
