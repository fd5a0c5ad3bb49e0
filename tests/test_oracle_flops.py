"""Pins of the Table I FLOP counts in oracle/flops.py against what the paper
states outside the table (Sec. V's complexity discussion) and what the
methods' definitions imply, so that a mistyped coefficient or a dropped term
in a row fails here rather than agreeing with a second transcription.

* With every user seeing every antenna (|Gamma| = Nt, |X| = K, |Q| = K) the
  VR-OGRK iteration is the GK one over the whole system: the two rows agree
  exactly, set-up and per-iteration terms.
* Sec. V: forming the precoder matrix costs O(8 Nt K^2) for the schemes
  without VRs and O(8 Nt K |Q|) with the subarray form (eq. (precoding2)):
  the second difference in K of the former is 16 Nt, the slope in |Q| of the
  latter 8 Nt K.
* Sec. V: step 8 (the residuals) costs O(8 Nt K) per iteration for GK and
  O(8 |Gamma| |X|) for VR-OGRK: the mixed differences in (Nt, K) and in
  (|Gamma|, |X|) of the per-iteration terms are 8.

The lower-order terms of the RZF, URK, SWOR-ERK and VR-OAHK rows follow
counting conventions the paper does not state; they stay unpinned.
"""
import itertools

import pytest

from oracle.flops import table1_flops


def per_iter(scheme, K, Nt, **kw):
    return table1_flops(scheme, K, Nt, T=1.0, **kw) - table1_flops(scheme, K, Nt, T=0.0, **kw)


@pytest.mark.parametrize("K,Nt", [(2, 8), (16, 256), (64, 1024), (128, 2048), (512, 16384)])
@pytest.mark.parametrize("T", [0.0, 1.0, 15.0, 123.0])
def test_vr_ogrk_with_full_visibility_is_gk(K, Nt, T):
    assert table1_flops("vr_ogrk", K, Nt, T=T, Q=K, M=Nt, X=K) == table1_flops("gk", K, Nt, T=T)


@pytest.mark.parametrize("scheme", ["urk", "swor_erk", "gk"])
@pytest.mark.parametrize("K,Nt", [(8, 64), (30, 2000), (128, 4096)])
def test_precoder_matrix_term_without_vrs_is_8_Nt_K_squared(scheme, K, Nt):
    f = lambda k: table1_flops(scheme, k, Nt, T=0.0)
    assert f(K + 1) + f(K - 1) - 2 * f(K) == 16 * Nt


@pytest.mark.parametrize("scheme", ["vr_ogrk", "vr_oahk"])
@pytest.mark.parametrize("K,Nt,Q", [(8, 64, 2.0), (30, 2000, 5.5), (128, 4096, 17.0)])
def test_precoder_matrix_term_with_subarrays_is_8_Nt_K_Q(scheme, K, Nt, Q):
    f = lambda q: table1_flops(scheme, K, Nt, T=0.0, Q=q)
    assert f(Q + 1.0) - f(Q) == 8 * Nt * K


@pytest.mark.parametrize("K,Nt", [(8, 64), (30, 2000), (128, 4096)])
def test_gk_residual_term_is_8_Nt_K(K, Nt):
    d = per_iter("gk", K + 1, Nt + 1) - per_iter("gk", K + 1, Nt) - per_iter("gk", K, Nt + 1) + per_iter("gk", K, Nt)
    assert d == 8


@pytest.mark.parametrize("M,X", list(itertools.product([64.0, 300.0], [3.0, 12.5])))
def test_vr_ogrk_residual_term_is_8_Gamma_X(M, X):
    K, Nt = 30, 2000
    g = lambda m, x: per_iter("vr_ogrk", K, Nt, Q=4.0, M=m, X=x)
    assert g(M + 1, X + 1) - g(M + 1, X) - g(M, X + 1) + g(M, X) == 8
    # and the per-iteration cost does not depend on Nt or on the subarray sets
    assert per_iter("vr_ogrk", K, Nt + 100, Q=4.0, M=M, X=X) == g(M, X)
    assert per_iter("vr_ogrk", K, Nt, Q=9.0, M=M, X=X) == g(M, X)


def test_planted_mistakes_are_caught():
    """Each pin fails for a plausible mistyping of the rows it covers."""
    def vr_ogrk_wrong(K, Nt, T=0.0, Q=0.0, M=0.0, X=0.0):  # (X + 1) typed as X
        return 8 * Nt * K * (Q + 0.5) - K + T * (8 * M * X + K - 5)

    def gk_wrong(K, Nt, T=0.0):  # 4 Nt K typed as 8 Nt K
        return 8 * Nt * K ** 2 + 8 * Nt * K - K + T * (8 * Nt * (K + 1) + K - 5)

    K, Nt, T = 16, 256, 15.0
    assert vr_ogrk_wrong(K, Nt, T=T, Q=K, M=Nt, X=K) != table1_flops("gk", K, Nt, T=T)
    assert table1_flops("vr_ogrk", K, Nt, T=T, Q=K, M=Nt, X=K) != gk_wrong(K, Nt, T=T)
