"""Pins for the oracle's row-selection rules and its sum-rate loss.

Each pin checks the oracle against a fact fixed outside it:

* ``select(rule, r, d, u)`` is an inverse-CDF draw, so sweeping ``u`` over a
  fine grid of [0, 1) reproduces the sampling distribution exactly.  For the
  paper's greedy rule (Sec. IV-A, Alg. 2 step 4) that distribution is
  |r_i|^2 / ||r||^2; for the Bai-Wu rule cited in Sec. IV-A it is the same
  weights restricted to the greedy set U_t, which is enumerated here from its
  unsimplified definition in exact rational arithmetic.
* ``rk`` draws rows with p_i = ||b_i||^2 / ||B||_F^2 (energy) or 1/K (uniform)
  (Sec. III-A); the empirical frequencies of a long run must match.
* ``adjoint.loss_from_VX`` is the negative sum rate of eq. (rate): it must equal
  the loop-by-loop ``sinr.rates`` on the same precoder, the one-user closed form
  log2(1 + snr ||h||^2) and the closed form for users with disjoint VRs.

Each pin is followed by a planted mistake it must catch (the weights divided
by d, energy and uniform swapped, a wrong mean term in the Bai-Wu threshold,
an interference sum taken over the wrong index).
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

import kzgen
import oracle
from oracle import adjoint as oadj
from oracle import kaczmarz as kz
from oracle import rzf as rz

GRID = 20000


def empirical(rule_fn, K):
    """Distribution of an inverse-CDF rule over a uniform grid of u."""
    u = (np.arange(GRID) + 0.5) / GRID
    return np.bincount([rule_fn(x) for x in u], minlength=K) / GRID


def baiwu_exact(r, d):
    """U_t = {i : |r_i|^2 >= eps ||r||^2 d_i} with
    eps = (max_i (|r_i|^2 / d_i) / ||r||^2 + 1 / ||B||_F^2) / 2 and ||B||_F^2 = sum d,
    evaluated in exact rationals on the float inputs; also returns the smallest
    relative margin |lhs - rhs| / rhs over the rows (to skip near-ties)."""
    a2 = [Fraction(float(x.real)) ** 2 + Fraction(float(x.imag)) ** 2 for x in r]
    dd = [Fraction(float(x)) for x in d]
    rn = sum(a2)
    eps = (max(a / di for a, di in zip(a2, dd)) / rn + 1 / sum(dd)) / 2
    U, margin = [], float("inf")
    for a, di in zip(a2, dd):
        rhs = eps * rn * di
        U.append(a >= rhs)
        margin = min(margin, abs(float((a - rhs) / rhs)))
    return np.array(U), margin


def random_rd(rng, K):
    r = rng.normal(size=K) + 1j * rng.normal(size=K)
    r *= rng.uniform(0.05, 1.0, size=K)   # spread the magnitudes so U_t is a proper subset
    d = rng.uniform(0.3, 5.0, size=K)
    return r, d


# ---------------------------------------------------------------- GRK paper rule
def paper_rule_matches(select_fn, r, d):
    want = np.abs(r) ** 2 / np.sum(np.abs(r) ** 2)
    got = empirical(lambda u: select_fn("paper", r, d, u), len(r))
    return np.max(np.abs(got - want)) <= 2.0 / GRID


def test_paper_rule_samples_residual_energy():
    rng = np.random.default_rng(11)
    for _ in range(5):
        r, d = random_rd(rng, 6)
        assert paper_rule_matches(kz.select, r, d)


def test_paper_rule_pin_catches_weights_divided_by_d():
    def planted(rule, r, d, u):
        return kz.pick(np.abs(r) ** 2 / d, u)   # GK-style weights instead of |r_i|^2
    r, d = random_rd(np.random.default_rng(12), 6)
    assert not paper_rule_matches(planted, r, d)


# ---------------------------------------------------------------- Bai-Wu greedy set
def baiwu_rule_matches(set_fn, select_fn, r, d):
    U, margin = baiwu_exact(r, d)
    if margin < 1e-9:
        return None  # a near-tie: membership depends on rounding, skip
    if not np.array_equal(set_fn(r, d), U):
        return False
    w = np.where(U, np.abs(r) ** 2, 0.0)
    got = empirical(lambda u: select_fn("baiwu", r, d, u), len(r))
    return bool(np.max(np.abs(got - w / w.sum())) <= 2.0 / GRID)


def test_baiwu_set_equals_exact_enumeration():
    rng = np.random.default_rng(13)
    checked = proper = 0
    for _ in range(300):
        K = int(rng.integers(1, 7))
        r, d = random_rd(rng, K)
        U, margin = baiwu_exact(r, d)
        if margin < 1e-9:
            continue
        assert np.array_equal(kz.baiwu_set(r, d), U)
        checked += 1
        proper += int(0 < U.sum() < K)
    assert checked > 250 and proper > 50


def test_baiwu_sampling_distribution():
    rng = np.random.default_rng(14)
    done = 0
    while done < 5:
        r, d = random_rd(rng, 6)
        res = baiwu_rule_matches(kz.baiwu_set, kz.select, r, d)
        if res is None:
            continue
        assert res
        done += 1


def test_baiwu_pin_catches_wrong_mean_term():
    def planted_set(r, d):
        a2 = np.abs(r) ** 2
        ratio = a2 / d
        mx = np.max(ratio)
        avg = min(np.sum(a2) / len(r), mx)   # ||r||^2 / K instead of ||r||^2 / ||B||_F^2
        return ratio >= 0.5 * (mx + avg)

    rng = np.random.default_rng(15)
    caught = 0
    for _ in range(200):
        r, d = random_rd(rng, int(rng.integers(2, 7)))
        U, margin = baiwu_exact(r, d)
        if margin < 1e-9:
            continue
        caught += int(not np.array_equal(planted_set(r, d), U))
    assert caught > 10


# ---------------------------------------------------------------- RK weights
def rk_frequencies(inst, energy, steps=24000, rk_fn=None):
    sys = kz.System.from_instance(inst)
    tr = []
    (rk_fn or kz.rk)(sys, inst.S[:, 0], energy=energy, tol=0.0, max_iter=steps, seed=5, trace=tr)
    rows = np.array([t["row"] for t in tr])
    return sys, np.bincount(rows, minlength=sys.K) / len(rows)


def chi2_ok(freq, p, n):
    """Pearson statistic of n draws against p below the 1e-4 tail for K-1 dof (K <= 6)."""
    stat = n * np.sum((freq - p) ** 2 / p)
    return stat < 30.0


@pytest.fixture(scope="module")
def uneven_inst():
    # five users with very different VR lengths, so ||h_k||^2 + xi differ by ~10x
    off = [0, 10, 30, 60, 100]
    L = [6, 14, 24, 36, 60]
    return kzgen.make_instance(3, 5, 160, vr_override=(off, L), snr_db=10.0, nrhs=1)


def test_rk_energy_weights(uneven_inst):
    n = 24000
    sys, f = rk_frequencies(uneven_inst, True, n)
    assert chi2_ok(f, sys.d / sys.d.sum(), n)


def test_rk_uniform_weights(uneven_inst):
    n = 24000
    sys, f = rk_frequencies(uneven_inst, False, n)
    assert chi2_ok(f, np.full(sys.K, 1.0 / sys.K), n)


def test_rk_pin_catches_energy_uniform_swap(uneven_inst):
    def planted_rk(sys, s, *, energy=True, **kw):
        return kz.rk(sys, s, energy=not energy, **kw)
    n = 24000
    sys, f = rk_frequencies(uneven_inst, True, n, rk_fn=planted_rk)
    assert not chi2_ok(f, sys.d / sys.d.sum(), n)


# ---------------------------------------------------------------- sum-rate loss
def loss_np(H, X, snr, loss_fn=oadj.loss_from_VX):
    Ht = torch.tensor(H, dtype=torch.complex128)
    Xt = torch.tensor(X, dtype=torch.complex128)
    return float(loss_fn(Ht, None, Xt, snr).item())


def loss_matches_sinr(loss_fn, inst, snr, X=None):
    """The loss against -sum(sinr.rates) on the RZF precoder, or on a given X.
    (With the RZF precoder H X is Hermitian, so a general X is needed to tell
    the received interference from the caused one.)"""
    H = inst.dense().astype(np.complex128)
    if X is None:
        V, X = rz.rzf(H, inst.xi, np.eye(inst.K))
    return abs(loss_np(H, X, snr, loss_fn) + np.sum(oracle.sinr.rates(H, X, snr))) <= 1e-12 * inst.K


def general_precoder(inst, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(inst.Nt, inst.K)) + 1j * rng.normal(size=(inst.Nt, inst.K))


def test_loss_equals_negative_sum_rate():
    for seed in (1, 2, 3):
        inst = kzgen.make_instance(seed, 7, 64, vr_len_range=(20, 50), nrhs=7, rhs="identity")
        assert loss_matches_sinr(oadj.loss_from_VX, inst, 10.0)
        assert loss_matches_sinr(oadj.loss_from_VX, inst, 10.0, X=general_precoder(inst, seed))


def test_loss_single_user_closed_form():
    inst = kzgen.make_instance(4, 1, 40, vr_len_range=(25, 25), nrhs=1, rhs="identity")
    H = inst.dense().astype(np.complex128)
    V, X = rz.rzf(H, inst.xi, np.eye(1))
    snr = 3.0
    assert loss_np(H, X, snr) == pytest.approx(-np.log2(1 + snr * np.sum(np.abs(H) ** 2)), rel=1e-13)


def test_loss_disjoint_users_closed_form():
    """Disjoint VRs: v_k = e_k / d_k, x_k = h_k^H / d_k, no interference, so
    SINR_k = snr (||h_k||^2 / d_k)^2 / sum_l ||h_l||^2 / d_l^2."""
    off, L = [0, 20, 45], [15, 20, 10]
    inst = kzgen.make_instance(5, 3, 60, vr_override=(off, L), nrhs=3, rhs="identity")
    H = inst.dense().astype(np.complex128)
    V, X = rz.rzf(H, inst.xi, np.eye(3))
    n2 = np.sum(np.abs(H) ** 2, axis=1)
    d = n2 + inst.xi
    snr = 7.0
    sinr = snr * (n2 / d) ** 2 / np.sum(n2 / d ** 2)
    assert loss_np(H, X, snr) == pytest.approx(-np.sum(np.log2(1 + sinr)), rel=1e-12)


def test_sinr_two_user_hand_computed():
    """A 2 x 2 case worked by hand: H = [[1, 1j], [0.5, 2]], X = I.
    F = X / sqrt(2); G = H F = H / sqrt(2).  User 0: signal |1|^2/2, interference
    |1j|^2/2; user 1: signal |2|^2/2, interference |0.5|^2/2; snr = 4 adds 1/4."""
    H = np.array([[1.0, 1j], [0.5, 2.0]])
    X = np.eye(2, dtype=complex)
    want = np.array([0.5 / (0.5 + 0.25), 2.0 / (0.125 + 0.25)])
    assert np.allclose(oracle.sinr.sinr(H, X, 4.0), want, rtol=1e-14)
    assert loss_np(H, X, 4.0) == pytest.approx(-np.sum(np.log2(1 + want)), rel=1e-14)


def test_loss_pin_catches_transposed_interference():
    def planted(H, V, X, snr_lin):
        F = X / torch.linalg.norm(X)
        G = H @ F
        sig = torch.abs(torch.diagonal(G)) ** 2
        tot = torch.sum(torch.abs(G) ** 2, dim=0)   # column sums: interference caused, not received
        return -torch.sum(torch.log2(1.0 + sig / (tot - sig + 1.0 / snr_lin)))
    inst = kzgen.make_instance(1, 7, 64, vr_len_range=(20, 50), nrhs=7, rhs="identity")
    assert not loss_matches_sinr(planted, inst, 10.0, X=general_precoder(inst, 1))


# ---------------------------------------------------------------- SWOR-ERK (Table I's comparison method)
def swor_rows(inst, steps, rk_fn=None, seed=5):
    sys = kz.System.from_instance(inst)
    tr = []
    (rk_fn or kz.rk)(sys, inst.S[:, 0], swor=True, tol=0.0, max_iter=steps, seed=seed, trace=tr)
    return sys, np.array([t["row"] for t in tr])


def test_swor_every_sweep_is_a_permutation(uneven_inst):
    sys, rows = swor_rows(uneven_inst, 5 * 400)
    for c in range(400):
        assert sorted(rows[5 * c:5 * c + 5].tolist()) == list(range(5))


def test_swor_draws_follow_sampling_without_replacement(uneven_inst):
    """First draw of a sweep: d_i / D.  Pair (first, second): d_i/D * d_j/(D - d_i)."""
    n_sweeps = 6000
    sys, rows = swor_rows(uneven_inst, 5 * n_sweeps)
    d = sys.d
    D = d.sum()
    first = rows[0::5]
    second = rows[1::5]
    assert chi2_ok(np.bincount(first, minlength=5) / n_sweeps, d / D, n_sweeps)
    pair = np.zeros((5, 5))
    for a, c in zip(first, second):
        pair[a, c] += 1
    p = np.array([[0.0 if i == j else d[i] / D * d[j] / (D - d[i]) for j in range(5)] for i in range(5)])
    mask = p > 0
    stat = n_sweeps * np.sum((pair[mask] / n_sweeps - p[mask]) ** 2 / p[mask])
    assert stat < 60.0  # 19 dof, far tail


def test_swor_pin_catches_replacement(uneven_inst):
    """Drawing with replacement (plain energy RK) breaks the permutation pin."""
    def planted(sys, s, *, swor=True, **kw):
        return kz.rk(sys, s, energy=True, swor=False, **kw)
    sys, rows = swor_rows(uneven_inst, 5 * 200, rk_fn=planted)
    assert any(sorted(rows[5 * c:5 * c + 5].tolist()) != list(range(5)) for c in range(200))


def test_gk_is_the_argmax_rule():
    inst = kzgen.make_instance(8, 9, 72, vr_len_range=(8, 40), nrhs=2)
    a = kz.solve(inst, inst.S, "gk", tol=1e-10, max_iter=5000)
    b = kz.solve(inst, inst.S, "grk", rule="argmax", tol=1e-10, max_iter=5000)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["iters"], b["iters"])
