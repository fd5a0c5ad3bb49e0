"""Pins for the FP64 oracle: closed forms, invariants, special cases and brute force.

None of these compare the oracle with itself: each checks it against a fact
the paper or the mathematics fixes (Theorem 1's least-squares form solved by
an SVD-based routine, the diagonal closed form for disjoint VRs, Lemma 1-3,
Theorems 2-4, Proposition 1, the repaired Theorem 3 bound, the dual
steepest-descent form of AHK, brute-force maximum independent sets, and the
published SplitMix64 test vectors).
"""
import os

import numpy as np
import pytest

import kzgen
import oracle
from oracle import kaczmarz as kz
from oracle import rzf as rz
from oracle import sets as st

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small(seed=1, K=8, Nt=64, lo=8, hi=40, snr=10.0, nrhs=1, **kw):
    return kzgen.make_instance(seed, K, Nt, vr_len_range=(lo, hi), snr_db=snr, nrhs=nrhs, **kw)


def wstar(inst):
    V, X = rz.rzf(inst.dense(), inst.xi, inst.S)
    return V, X


def werr2(sys, m, q, mstar, qstar):
    """||w - w*||^2 with w = [m; sqrt(xi) q]."""
    return float(np.sum(np.abs(m - mstar) ** 2) + sys.xi * np.sum(np.abs(q - qstar) ** 2))


# ---------------------------------------------------------------- generator
def test_generator_deterministic_and_well_formed():
    a = small(seed=7, nrhs=3)
    b = small(seed=7, nrhs=3)
    assert np.array_equal(a.H_packed, b.H_packed) and np.array_equal(a.S, b.S)
    assert a.H_packed.dtype == np.complex64 and a.S.dtype == np.complex64
    assert np.all(a.vr_offset >= 0) and np.all(a.vr_offset + a.vr_len <= a.Nt)
    assert np.all(a.vr_len >= 8) and np.all(a.vr_len <= 40)
    assert a.H_packed.size == int(a.vr_len.sum())
    # unit mean power over visible entries (before complex64 rounding)
    assert abs(np.mean(np.abs(a.H_packed.astype(np.complex128)) ** 2) - 1.0) < 1e-6
    # QPSK alphabet
    assert np.allclose(np.abs(a.S.real), 1 / np.sqrt(2)) and np.allclose(np.abs(a.S.imag), 1 / np.sqrt(2))
    assert a.xi == pytest.approx(8 / 10.0)


def test_generator_spherical_phase():
    """Entry phases follow exp(-j 2 pi r_kn / lambda) with r_kn from the law of cosines."""
    inst = small(seed=3, K=2, Nt=32, lo=32, hi=32)
    lam = kzgen.C_LIGHT / 28e9
    r, th = inst.meta["r"][0], inst.meta["theta"][0]
    x0 = (0 - 15.5) * lam / 2
    r0 = np.sqrt(r * r + x0 * x0 - 2 * r * x0 * np.sin(th))
    h0 = inst.H_packed[0]
    expect = inst.meta["scale"] * lam / (4 * np.pi * r0) * np.exp(-2j * np.pi * r0 / lam)
    assert abs(h0 - expect) < 1e-5 * abs(expect)


# ---------------------------------------------------------------- RNG
def test_splitmix64_published_vectors():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    assert oracle.rng.splitmix64_sequence(0, len(want)) == want


def test_uniform_draws_are_uniform():
    u = np.array([oracle.rng.uniform(5, 1, 2, t) for t in range(20000)])
    assert np.all((u >= 0) & (u < 1))
    hist = np.histogram(u, bins=20, range=(0, 1))[0]
    chi2 = np.sum((hist - 1000.0) ** 2 / 1000.0)
    assert chi2 < 45.0  # 19 dof, p ~ 1e-3


def test_pick_inverse_cdf():
    w = np.array([0.0, 1.0, 3.0, 0.0, 4.0])
    assert kz.pick(w, 0.0) == 1
    assert kz.pick(w, 0.124) == 1 and kz.pick(w, 0.126) == 2
    assert kz.pick(w, 0.49) == 2 and kz.pick(w, 0.51) == 4
    assert kz.pick(w, 1.0) == 4  # u*total == total falls back to the last positive weight
    grid = (np.arange(4000) + 0.5) / 4000
    counts = np.bincount([kz.pick(w, u) for u in grid], minlength=5) / 4000.0
    assert np.allclose(counts, w / w.sum(), atol=1e-3)


# ---------------------------------------------------------------- RZF closed form
@pytest.mark.parametrize("seed,K,Nt", [(1, 8, 64), (2, 12, 96), (3, 5, 40)])
def test_rzf_matches_theorem1_least_squares(seed, K, Nt):
    """Theorem 1: v = argmin ||G v - g|| with G = [H^H; sqrt(xi) I], g = [0; s/sqrt(xi)]."""
    inst = small(seed=seed, K=K, Nt=Nt, nrhs=3)
    H = inst.dense().astype(np.complex128)
    V, X = rz.rzf(H, inst.xi, inst.S)
    G = np.vstack([H.conj().T, np.sqrt(inst.xi) * np.eye(K)])
    g = np.vstack([np.zeros((Nt, 3)), inst.S.astype(np.complex128) / np.sqrt(inst.xi)])
    Vls = np.linalg.lstsq(G, g, rcond=None)[0]
    assert np.max(np.abs(V - Vls)) < 1e-11 * np.max(np.abs(Vls))
    assert np.allclose(X, H.conj().T @ Vls, rtol=0, atol=1e-11 * np.max(np.abs(X)))


def test_cholesky_factor():
    inst = small(seed=4, K=10, Nt=80)
    A = rz.gram(inst.dense(), inst.xi)
    L = rz.cholesky(A)
    assert np.allclose(np.triu(L, 1), 0)
    assert np.all(np.diag(L).real > 0) and np.allclose(np.diag(L).imag, 0)
    assert np.max(np.abs(L @ L.conj().T - A)) < 1e-12 * np.max(np.abs(A))


def disjoint_instance(K=6, L=10, gap=3, nrhs=2, seed=5):
    off = [k * (L + gap) for k in range(K)]
    Nt = K * (L + gap)
    return kzgen.make_instance(seed, K, Nt, vr_override=(off, [L] * K), nrhs=nrhs)


def test_rzf_disjoint_vrs_closed_form():
    """Lemma 1: disjoint VRs make H H^H diagonal, so v_k = s_k / (||h_k||^2 + xi)."""
    inst = disjoint_instance()
    V, X = rz.rzf(inst.dense(), inst.xi, inst.S)
    Hp = inst.H_packed.astype(np.complex128)
    nrm = np.array([np.sum(np.abs(Hp[k * 10:(k + 1) * 10]) ** 2) for k in range(inst.K)])
    v_closed = inst.S.astype(np.complex128) / (nrm + inst.xi)[:, None]
    assert np.max(np.abs(V - v_closed)) < 1e-14


def test_rzf_single_user_and_mrt_limit():
    inst = small(seed=6, K=1, Nt=32, lo=20, hi=20)
    V, X = rz.rzf(inst.dense(), inst.xi, inst.S)
    nrm = np.sum(np.abs(inst.H_packed.astype(np.complex128)) ** 2)
    assert abs(V[0, 0] - inst.S[0, 0] / (nrm + inst.xi)) < 1e-14
    # xi -> infinity: x -> H^H s / xi (MRT, Sec. II-C); relative gap O(||H||^2 / xi)
    inst = small(seed=7, K=6, Nt=48)
    H = inst.dense().astype(np.complex128)
    xi = 1e7
    V, X = rz.rzf(H, xi, inst.S)
    mrt = H.conj().T @ inst.S.astype(np.complex128) / xi
    assert rz.rel_err(X, mrt)[0] < 1e-4


# ---------------------------------------------------------------- convergence of every method
@pytest.mark.parametrize("algo", kz.ALGOS)
@pytest.mark.parametrize("seed", [11, 12])
def test_every_method_converges_to_rzf(algo, seed):
    inst = small(seed=seed, K=9, Nt=72, nrhs=2)
    V, X = wstar(inst)
    out = kz.solve(inst, inst.S, algo, tol=1e-11, max_iter=200000, seed=3)
    assert out["conv"].all()
    assert np.all(rz.rel_err(out["x"], X) < 1e-9)
    assert np.all(rz.rel_err(out["v"], V) < 1e-9)


@pytest.mark.parametrize("rule", kz.RULES)
def test_greedy_rules_converge(rule):
    inst = small(seed=21, K=10, Nt=80, nrhs=1)
    V, X = wstar(inst)
    for algo in ("grk", "vr_ogrk"):
        out = kz.solve(inst, inst.S, algo, rule=rule, tol=1e-11, max_iter=100000, seed=9)
        assert out["conv"].all() and rz.rel_err(out["x"], X)[0] < 1e-9


# ---------------------------------------------------------------- invariants along trajectories
def traj_grk(inst, rule="paper", steps=60):
    sys = kz.System.from_instance(inst)
    tr = []
    kz.grk(sys, inst.S[:, 0], rule=rule, tol=0.0, max_iter=steps, seed=1, trace=tr)
    return sys, tr


def test_range_invariant_and_selected_row_residual():
    """w stays in range(B^H), i.e. m = H^H q (Remark 1 / eq. (update)); after
    projecting row i its residual is zero (Lemma 2's a_i^H(x^{t+1} - x*) = 0)."""
    inst = small(seed=31, K=8, Nt=64)
    sys, tr = traj_grk(inst)
    s = inst.S[:, 0].astype(np.complex128)
    for st_ in tr:
        m, q, i = st_["m"], st_["q"], st_["row"]
        assert np.linalg.norm(m - sys.HHt(q)) <= 1e-13 * max(np.linalg.norm(m), 1e-300)
        assert abs(sys.residual_row(i, s, m, q)) <= 1e-13 * np.linalg.norm(s)


def test_pythagorean_identity_and_monotone_error():
    """eq. (gougu): ||e^{t+1}||^2 = ||e^t||^2 - ||w^{t+1} - w^t||^2."""
    inst = small(seed=32, K=8, Nt=64)
    V, X = wstar(inst)
    sys, tr = traj_grk(inst)
    m_prev = np.zeros(sys.Nt, complex)
    q_prev = np.zeros(sys.K, complex)
    e_prev = e0 = werr2(sys, m_prev, q_prev, X[:, 0], V[:, 0])
    for st_ in tr:
        e = werr2(sys, st_["m"], st_["q"], X[:, 0], V[:, 0])
        step = werr2(sys, st_["m"], st_["q"], m_prev, q_prev)
        assert abs(e - (e_prev - step)) <= 1e-12 * e0
        assert e <= e_prev + 1e-13 * e0
        m_prev, q_prev, e_prev = st_["m"], st_["q"], e


def test_theorem2_orthogonal_rows_keep_residual_bitwise():
    inst = small(seed=33, K=10, Nt=120, lo=10, hi=30)
    sys, tr = traj_grk(inst, steps=40)
    s = inst.S[:, 0].astype(np.complex128)
    m = np.zeros(sys.Nt, complex)
    q = np.zeros(sys.K, complex)
    checked = 0
    for st_ in tr:
        i = st_["row"]
        before = sys.residual(s, m, q)
        m, q = st_["m"], st_["q"]
        after = sys.residual(s, m, q)
        for j in range(sys.K):
            if not st.overlaps(sys.off[i], sys.len[i], sys.off[j], sys.len[j]) and j != i:
                assert after[j] == before[j]
                checked += 1
    assert checked > 0


def test_lemma1_exact_orthogonality():
    inst = small(seed=34, K=12, Nt=100, lo=5, hi=20)
    H = inst.dense().astype(np.complex128)
    G = H @ H.conj().T
    found = 0
    for i in range(inst.K):
        for j in range(inst.K):
            if i != j and not st.overlaps(inst.vr_offset[i], inst.vr_len[i], inst.vr_offset[j], inst.vr_len[j]):
                assert G[i, j] == 0.0
                found += 1
    assert found > 0


def test_vroahk_theorem4_prop1_lemma3():
    """After the orthogonal half-step r_F = 0 (Thm. 4); the general AHK step on F
    has unit length (Prop. 1); both half-steps satisfy eq. (gougu2)."""
    inst = small(seed=35, K=10, Nt=100, lo=10, hi=45)
    V, X = wstar(inst)
    sys = kz.System.from_instance(inst)
    s = inst.S[:, 0].astype(np.complex128)
    F, Vset = st.split_fv(sys.off, sys.len)
    assert len(F) >= 2 and len(Vset) >= 2
    tr = []
    kz.vr_oahk(sys, s, F=F, V=Vset, tol=0.0, max_iter=8, trace=tr, f_unit=False)
    E0 = werr2(sys, np.zeros(sys.Nt, complex), np.zeros(sys.K, complex), X[:, 0], V[:, 0])
    for st_ in tr:
        assert abs(st_["gF"] - 1.0) < 1e-13  # Prop. 1
        mh, qh = st_["w_half"]
        rF = sys.residual(s, mh, qh, rows=F)[F]
        assert np.max(np.abs(rF)) <= 1e-13 * np.linalg.norm(s)  # Thm. 4
        m0, q0 = st_["w0"]
        e0 = werr2(sys, m0, q0, X[:, 0], V[:, 0])
        eh = werr2(sys, mh, qh, X[:, 0], V[:, 0])
        assert abs(eh - (e0 - werr2(sys, mh, qh, m0, q0))) <= 1e-12 * E0
        if st_["w1"] is not None:
            m1, q1 = st_["w1"]
            e1 = werr2(sys, m1, q1, X[:, 0], V[:, 0])
            assert abs(e1 - (eh - werr2(sys, m1, q1, mh, qh))) <= 1e-12 * E0
            assert e1 <= eh + 1e-13 * E0


def test_theorem3_repaired_bound_exact_expectation():
    """E[||e^{t+1}||^2 | w^t] = sum_i p_i ||e after row i||^2 with p_i = |r_i|^2/||r||^2
    never exceeds (1 - sigma_min^2(B)/||B||_F^2) ||e^t||^2 (Thm. 3, read with
    ||B||_F squared and sigma_min^2(B) = lambda_min(H H^H) + xi)."""
    inst = small(seed=36, K=12, Nt=90, lo=10, hi=50)
    V, X = wstar(inst)
    sys, tr = traj_grk(inst, steps=50)
    s = inst.S[:, 0].astype(np.complex128)
    A = rz.gram(inst.dense(), inst.xi)
    rate = 1.0 - np.linalg.eigvalsh(A)[0] / np.sum(sys.d)
    states = [(np.zeros(sys.Nt, complex), np.zeros(sys.K, complex))] + [(t["m"], t["q"]) for t in tr]
    e0 = werr2(sys, states[0][0], states[0][1], X[:, 0], V[:, 0])
    for m, q in states:
        r = sys.residual(s, m, q)
        p = np.abs(r) ** 2 / np.sum(np.abs(r) ** 2)
        e = werr2(sys, m, q, X[:, 0], V[:, 0])
        exp_next = 0.0
        for i in range(sys.K):
            mi, qi = m.copy(), q.copy()
            sys.project_row(i, r[i] / sys.d[i], mi, qi)
            exp_next += p[i] * werr2(sys, mi, qi, X[:, 0], V[:, 0])
        assert exp_next <= rate * e + 1e-13 * e0


def test_ahk_is_dual_preconditioned_steepest_descent_and_kantorovich():
    """In the dual variable q, AHK is steepest descent on (H H^H + xi I) q = s with
    the Jacobi preconditioner and exact line search; its error contracts at least
    by ((kappa-1)/(kappa+1))^2 per step, kappa = cond(D^-1/2 A D^-1/2)."""
    inst = small(seed=37, K=10, Nt=80, lo=10, hi=50)
    V, X = wstar(inst)
    sys = kz.System.from_instance(inst)
    s = inst.S[:, 0].astype(np.complex128)
    tr = []
    kz.ahk(sys, s, tol=0.0, max_iter=25, trace=tr)
    A = rz.gram(inst.dense(), inst.xi)
    Dinv = 1.0 / np.real(np.diag(A))
    Dh = np.sqrt(Dinv)
    ev = np.linalg.eigvalsh(Dh[:, None] * A * Dh[None, :])
    kappa = ev[-1] / ev[0]
    contraction = ((kappa - 1) / (kappa + 1)) ** 2
    qd = np.zeros(sys.K, complex)
    e_prev = werr2(sys, np.zeros(sys.Nt, complex), qd, X[:, 0], V[:, 0])
    for st_ in tr:
        rd = s - A @ qd
        p = Dinv * rd
        alpha = np.vdot(p, rd).real / np.vdot(p, A @ p).real
        qd = qd + alpha * p
        assert np.linalg.norm(st_["q"] - qd) <= 1e-11 * np.linalg.norm(qd)
        e = werr2(sys, st_["m"], st_["q"], X[:, 0], V[:, 0])
        assert e <= contraction * e_prev * (1 + 1e-9)
        e_prev = e


# ---------------------------------------------------------------- special cases
def test_disjoint_vrs_special_cases():
    inst = disjoint_instance(nrhs=1)
    V, X = wstar(inst)
    out = kz.solve(inst, inst.S, "vr_oahk", tol=1e-13, max_iter=5)
    assert out["iters"][0] == 1 and rz.rel_err(out["x"], X)[0] < 1e-14
    out = kz.solve(inst, inst.S, "grk", rule="argmax", tol=1e-13, max_iter=100)
    assert out["iters"][0] <= inst.K and rz.rel_err(out["x"], X)[0] < 1e-14


def test_single_user_one_step():
    inst = small(seed=41, K=1, Nt=40, lo=30, hi=30)
    V, X = wstar(inst)
    for algo in ("rk_energy", "grk", "vr_ogrk"):
        out = kz.solve(inst, inst.S, algo, tol=1e-13, max_iter=10)
        assert out["iters"][0] == 1 and rz.rel_err(out["x"], X)[0] < 1e-14


# ---------------------------------------------------------------- sets
@pytest.mark.parametrize("seed", range(8))
def test_interval_mis_is_maximum(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(3, 13))
    Nt = 200
    L = rng.integers(5, 60, size=K)
    off = np.array([rng.integers(0, Nt - l + 1) for l in L])
    F = st.mis_interval(off, L)
    assert st.is_independent(F, off, L)
    assert len(F) == st.mis_bruteforce(off, L)


def test_touching_intervals_do_not_overlap_and_x_sets():
    off, L = [0, 10, 20, 5], [10, 10, 10, 10]
    assert not st.overlaps(0, 10, 10, 10)
    X = st.x_sets(off, L)
    assert X[0] == [0, 3] and X[1] == [1, 3] and X[3] == [0, 1, 3]
    assert st.mis_interval(off, L) == [0, 1, 2]


def test_baiwu_set_properties():
    rng = np.random.default_rng(3)
    for _ in range(200):
        K = int(rng.integers(1, 7))
        r = rng.normal(size=K) + 1j * rng.normal(size=K)
        d = rng.uniform(0.5, 3.0, size=K)
        U = kz.baiwu_set(r, d)
        assert U[int(np.argmax(np.abs(r) ** 2 / d))]  # the greedy row is always eligible
    d = np.array([2.0, 2.0, 2.0, 2.0])
    r = np.array([1 + 1j, -1 + 1j, 1 - 1j, -1 - 1j])  # all ratios equal (exactly): U is every row
    assert kz.baiwu_set(r, d).all()


# ---------------------------------------------------------------- SINR
def test_sinr_single_user_and_zf_limit():
    inst = small(seed=51, K=1, Nt=32, lo=32, hi=32)
    H = inst.dense().astype(np.complex128)
    X = H.conj().T  # MRT for one user
    snr = 10.0
    assert oracle.sinr.sinr(H, X, snr)[0] == pytest.approx(snr * np.sum(np.abs(H) ** 2), rel=1e-12)
    inst = small(seed=52, K=6, Nt=64)
    H = inst.dense().astype(np.complex128)
    V, X = rz.rzf(H, 1e-12, np.eye(6))  # xi -> 0: ZF, no inter-user interference
    G = H @ X
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 1e-9 * np.max(np.abs(G))


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes(monkeypatch):
    """A dropped xi q term or a wrong conjugate in the oracle must fail the RZF pin."""
    inst = small(seed=61, K=8, Nt=64)
    V, X = wstar(inst)
    orig_res = kz.System.residual_row
    monkeypatch.setattr(kz.System, "residual_row", lambda self, i, s, m, q: s[i] - self.rows[i] @ m[self.sl(i)])
    out = kz.solve(inst, inst.S, "grk", rule="argmax", tol=1e-10, max_iter=5000)
    assert rz.rel_err(out["x"], X)[0] > 1e-3
    monkeypatch.setattr(kz.System, "residual_row", orig_res)

    def bad_project(self, i, gamma, m, q):
        m[self.sl(i)] += gamma * self.rows[i]  # missing conjugate
        q[i] += gamma
    monkeypatch.setattr(kz.System, "project_row", bad_project)
    out = kz.solve(inst, inst.S, "grk", rule="argmax", tol=1e-10, max_iter=2000)
    assert rz.rel_err(out["x"], X)[0] > 1e-3
