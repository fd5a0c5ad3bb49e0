"""FP64 CPU oracle for the Kaczmarz-type RZF precoders (test infrastructure).

This package is the checker, not the product: only ``tests/``, the smoke
check in ``__graft_entry__`` and the CPU-baseline / reference leg of
``bench.py`` may import it.  It shares no code with the CUDA library and
never imports it; the only thing both sides consume is the seeded input
generator ``kzgen``.

Everything runs in complex128 / float64 with plain NumPy.  Each function
cites the part of the paper it follows:

* ``rzf``        closed-form RZF (eq. (precoding), Theorem 1, Remark 1-2)
                 by a hand-written Cholesky factorisation.
* ``kaczmarz``   literal RK (Alg. 1), GRK (Sec. IV-A), VR-OGRK (Alg. 2),
                 AHK (eqs. (update4), (coefficient)) and VR-OAHK (Alg. 3).
* ``sets``       VR overlap graph, non-orthogonal sets X_k (Sec. IV-B) and the
                 orthogonal set F as a maximum independent set (eq. (max_set)).
* ``rng``        the SplitMix64 counter-based generator used for random row
                 selection (the paper does not name one).
* ``sinr``       per-user SINR and spectral efficiency (eq. (rate)).
* ``precoder``   subarray-wise precoder assembly (eq. (precoding2)) and beta.
* ``flops``      the FLOP counts of Table I (partly pinned: accounting).

Parity unpinned: ``kaczmarz.vr_oahk``'s a-priori rate of Theorem 5 (the
statement is iterate-dependent and garbled; only the Lemma 3 identities,
monotone error decrease and convergence to RZF are pinned) and the
lower-order terms of ``flops``' RZF, URK, SWOR-ERK and VR-OAHK rows (Table
I's accounting conventions, transcribed as printed).
"""
from . import rng, sets, rzf, kaczmarz, sinr, precoder, flops  # noqa: F401
