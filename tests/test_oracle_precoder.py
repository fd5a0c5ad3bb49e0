"""Pins for the subarray-wise precoder assembly (eq. (precoding2)).

Against facts fixed outside the function: the dense product H^H V (which the
subarray form must equal, since rows outside Q_s vanish on subarray s), the
RZF precoder of the closed form (eq. (precoding)), Q_s read off the dense
channel's non-zero pattern, and ||beta F||_F = 1.  A planted mistake (a
missing conjugate, a subarray dropped from Q_s) must fail them.
"""
import numpy as np
import pytest

import kzgen
from oracle import precoder as opc
from oracle import rzf as orz


def inst(seed=1, K=12, Nt=200, nrhs=12):
    return kzgen.make_instance(seed, K, Nt, vr_len_range=(20, 90), nrhs=nrhs, rhs="identity" if nrhs == K else "qpsk")


@pytest.mark.parametrize("S", [1, 4, 7, 20, 200])
def test_subarray_form_equals_dense_product(S):
    i = inst()
    H = i.dense().astype(np.complex128)
    V = np.random.default_rng(S).normal(size=(i.K, 5)) + 1j * np.random.default_rng(S + 1).normal(size=(i.K, 5))
    F = opc.subarray_precoder(H, V, i.vr_offset, i.vr_len, S)
    assert np.max(np.abs(F - H.conj().T @ V)) <= 1e-13 * np.max(np.abs(F))


def test_subarray_form_of_the_rzf_auxiliary_matrix_is_the_rzf_precoder():
    i = inst(seed=2)
    V, X = orz.rzf(i.dense(), i.xi, np.eye(i.K))
    F = opc.subarray_precoder(i.dense(), V, i.vr_offset, i.vr_len, 10)
    assert np.max(np.abs(F - X)) <= 1e-13 * np.max(np.abs(X))
    Fn, beta = opc.normalise(F)
    assert abs(np.linalg.norm(Fn) - 1.0) < 1e-14 and beta > 0


def test_q_sets_match_the_channel_support():
    i = inst(seed=3)
    D = i.dense()
    for S in (3, 8, 25):
        Q = opc.q_sets(i.vr_offset, i.vr_len, i.Nt, S)
        for (n0, n1), q in zip(opc.subarray_bounds(i.Nt, S), Q):
            assert q == [k for k in range(i.K) if np.any(D[k, n0:n1] != 0)]


def test_pins_catch_planted_mistakes(monkeypatch):
    i = inst(seed=4)
    H = i.dense().astype(np.complex128)
    V = np.eye(i.K)
    ref = H.conj().T @ V
    bad = np.zeros_like(ref)
    for (n0, n1), Q in zip(opc.subarray_bounds(i.Nt, 8), opc.q_sets(i.vr_offset, i.vr_len, i.Nt, 8)):
        bad[n0:n1] = H[Q, n0:n1].T @ V[Q, :]  # missing conjugate
    assert np.max(np.abs(bad - ref)) > 1e-3
    orig = opc.q_sets
    monkeypatch.setattr(opc, "q_sets", lambda *a: [q[:-1] for q in orig(*a)])  # last user of every Q_s dropped
    F = opc.subarray_precoder(H, V, i.vr_offset, i.vr_len, 8)
    assert np.max(np.abs(F - ref)) > 1e-3
