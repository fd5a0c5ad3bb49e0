"""CUDA path vs the FP64 oracle, through the C-ABI (needs a GB300)."""
import numpy as np
import pytest

import kzgen
import oracle
from oracle import kaczmarz as okz
from oracle import rzf as orz
from oracle import sets as osets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_X = 1e-5  # relative error of x against the FP64 RZF after convergence


@pytest.fixture(scope="module")
def kp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_10689_gb300 import kzprecode
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return kzprecode


def run(kp, inst, algo, sel="paper", tol=1e-7, max_iter=20000, J=0, refresh=0, prec="c64", seed=0, S=None):
    plan = kp.plan_from_instance(inst, prec=prec)
    S = inst.S if S is None else S
    out = kp.precode(plan, kp.rhs_tensor(S), inst.xi, algo=algo, sel=sel, tol=tol, max_iter=max_iter, seed=seed,
                     rhs_per_cta=J, refresh=refresh)
    return {"x": out["x"].cpu().numpy().T.astype(np.complex128), "v": out["v"].cpu().numpy().T.astype(np.complex128),
            "iters": out["iters"].cpu().numpy(), "resid": out["resid"].cpu().numpy(), "converged": out["converged"],
            "status": int(out["status"].item())}


def ragged(seed=5, K=13, Nt=333, lo=17, hi=121, nrhs=5, snr=10.0):
    """Odd Nt (ragged last tile), odd offsets and lengths, several tiles."""
    return kzgen.make_instance(seed, K, Nt, vr_len_range=(lo, hi), snr_db=snr, nrhs=nrhs)


ALGOS = ["rk_energy", "rk_uniform", "grk", "ahk", "vr_ogrk", "vr_oahk"]


def test_plan_sets_match_oracle(kp):
    for seed in range(6):
        inst = ragged(seed=seed, K=20, Nt=301)
        plan = kp.plan_from_instance(inst)
        F, xptr, xidx = kp.kz_plan_query(plan)
        assert list(F) == osets.mis_interval(inst.vr_offset, inst.vr_len)
        X = osets.x_sets(inst.vr_offset, inst.vr_len)
        for k in range(inst.K):
            assert list(xidx[xptr[k]:xptr[k + 1]]) == X[k]


@pytest.mark.parametrize("algo", ALGOS)
def test_converges_to_rzf_ragged(kp, algo):
    inst = ragged()
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, algo, tol=1e-7, max_iter=200000)
    assert out["converged"]
    assert np.all(orz.rel_err(out["x"], X) <= TOL_X)
    assert np.all(orz.rel_err(out["v"], V) <= TOL_X)
    assert np.all(out["resid"] <= 1e-7 * (1 + 1e-6))  # stops are confirmed on the true residual


@pytest.mark.parametrize("J", [1, 2, 4, 8])
@pytest.mark.parametrize("algo", ["vr_oahk", "ahk", "grk", "vr_ogrk"])
def test_columns_per_cta(kp, J, algo):
    inst = ragged(seed=9, nrhs=11)  # 11 columns: a ragged last group for J > 1
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, algo, sel="argmax", tol=1e-7, J=J)
    assert out["converged"] and np.all(orz.rel_err(out["x"], X) <= TOL_X)


@pytest.mark.parametrize("rule", ["paper", "baiwu", "argmax"])
def test_greedy_rules(kp, rule):
    inst = kzgen.config1()
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    for algo in ("grk", "vr_ogrk"):
        out = run(kp, inst, algo, sel=rule, tol=1e-6, max_iter=4000)
        assert out["converged"] and orz.rel_err(out["x"], X)[0] <= TOL_X


@pytest.mark.parametrize("algo", ["ahk", "vr_oahk"])
@pytest.mark.parametrize("T", [1, 2, 3, 6])
def test_fixed_iteration_trajectory(kp, algo, T):
    """After exactly T iterations (tol = 0) the iterate equals the oracle's literal one."""
    inst = ragged(seed=3, nrhs=3)
    sys_ = okz.System.from_instance(inst)
    ref = okz.solve(sys_, inst.S, algo, tol=0.0, max_iter=T)
    out = run(kp, inst, algo, tol=0.0, max_iter=T, refresh=1000)
    assert np.all(out["iters"] == T) and not out["converged"]
    assert np.all(orz.rel_err(out["x"], ref["x"]) <= 1e-5)
    assert np.all(orz.rel_err(out["v"], ref["v"]) <= 1e-5)


def test_argmax_grk_first_steps_follow_oracle(kp):
    """Deterministic GRK: the first steps pick the same rows whenever the oracle's
    greedy margin is clear, so the iterates after T steps agree."""
    inst = ragged(seed=4, nrhs=1)
    sys_ = okz.System.from_instance(inst)
    s = inst.S[:, 0].astype(np.complex128)
    tr = []
    okz.grk(sys_, s, rule="argmax", tol=0.0, max_iter=8, trace=tr)
    safe = 0
    for st in tr:
        ratio = np.abs(st["r"]) ** 2 / sys_.d
        top = np.sort(ratio)[-2:]
        if top[1] - top[0] < 1e-3 * top[1]:
            break
        safe += 1
    assert safe >= 3
    out = run(kp, inst, "grk", sel="argmax", tol=0.0, max_iter=safe)
    assert orz.rel_err(out["x"][:, 0], tr[safe - 1]["m"]) <= 1e-5


def test_iteration_counts_close_to_oracle(kp):
    """Same stopping rule; the FP32 true residual carries a ~1e-7 floor (x is
    stored in FP32), worth up to about three iterations at tol = 1e-6."""
    inst = kzgen.config2(10.0, nrhs=4)
    for algo, tol in (("vr_oahk", 1e-6), ("ahk", 1e-6)):
        ref = okz.solve(inst, inst.S, algo, tol=tol, max_iter=1000)
        out = run(kp, inst, algo, tol=tol, max_iter=1000)
        assert np.all(np.abs(out["iters"] - ref["iters"]) <= 3), (algo, out["iters"], ref["iters"])


def test_edge_cases(kp):
    # single user
    inst = kzgen.make_instance(7, 1, 64, vr_len_range=(20, 20), nrhs=2)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    for algo in ALGOS:
        out = run(kp, inst, algo, tol=1e-7)
        assert np.all(orz.rel_err(out["x"], X) <= TOL_X), algo
    # all VRs disjoint: VR-OAHK is exact after one iteration (F = every user)
    off = [1 + 13 * k for k in range(6)]
    inst = kzgen.make_instance(8, 6, 80, vr_override=(off, [11] * 6), nrhs=3)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, "vr_oahk", tol=1e-7)
    assert np.all(out["iters"] == 1) and np.all(orz.rel_err(out["x"], X) <= 1e-6)
    # every VR is the whole array (no spatial non-stationarity: F has one user)
    inst = kzgen.make_instance(9, 8, 32, vr_override=([0] * 8, [32] * 8), nrhs=2, snr_db=10.0)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, "vr_oahk", tol=1e-7, max_iter=5000)
    assert out["converged"] and np.all(orz.rel_err(out["x"], X) <= TOL_X)
    # a zero right-hand side: zero iterations, x = 0
    inst = ragged(seed=10, nrhs=3)
    S = inst.S.copy()
    S[:, 1] = 0
    for algo in ("vr_oahk", "grk"):
        out = run(kp, inst, algo, tol=1e-7, S=S)
        assert out["iters"][1] == 0 and np.all(out["x"][:, 1] == 0) and out["resid"][1] == 0
    # max_iter exhausted: status bit set, outputs still written
    out = run(kp, ragged(seed=11), "grk", sel="argmax", tol=1e-12, max_iter=3)
    assert not out["converged"] and np.all(out["iters"] == 3) and np.all(np.isfinite(out["x"]))


def test_deterministic_rules_bitwise_reproducible(kp):
    inst = ragged(seed=12, nrhs=6)
    for algo, sel in (("vr_oahk", "paper"), ("ahk", "paper"), ("grk", "argmax"), ("vr_ogrk", "paper")):
        a = run(kp, inst, algo, sel=sel, tol=1e-7, seed=5)
        b = run(kp, inst, algo, sel=sel, tol=1e-7, seed=5)
        assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["iters"], b["iters"])


def test_config1_grk(kp):
    inst = kzgen.config1()
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, "grk", sel="paper", tol=1e-6, max_iter=4000)
    assert out["converged"] and orz.rel_err(out["x"], X)[0] <= TOL_X


@pytest.mark.parametrize("algo", ["grk", "vr_ogrk", "vr_oahk", "ahk"])
def test_precoder_matrix_sinr(kp, algo):
    """Identity right-hand sides give the precoder matrix (Remark 2); per-user SINR
    of eq. (rate) within 0.01 dB of the FP64 RZF precoder."""
    inst = kzgen.config1()
    I = np.eye(inst.K, dtype=np.complex64)
    V, X = orz.rzf(inst.dense(), inst.xi, I)
    out = run(kp, inst, algo, sel="paper", tol=1e-6, max_iter=4000, S=I)
    assert out["converged"] and np.all(orz.rel_err(out["x"], X) <= TOL_X)
    snr = 10.0 ** (inst.snr_db / 10.0)
    sinr_gpu = oracle.sinr.sinr_db(inst.dense(), out["x"], snr)
    sinr_ref = oracle.sinr.sinr_db(inst.dense(), X, snr)
    assert np.max(np.abs(sinr_gpu - sinr_ref)) <= 0.01


@pytest.mark.parametrize("snr", [0.0, 10.0, 20.0])
def test_config2_full_vroahk_and_grk(kp, snr):
    inst = kzgen.config2(snr)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    for algo in ("vr_oahk", "grk"):
        out = run(kp, inst, algo, sel="paper", tol=1e-6, max_iter=20000 if algo == "grk" else 2000)
        assert out["converged"]
        err = orz.rel_err(out["x"], X)
        assert np.max(err) <= TOL_X, (algo, snr, np.max(err))
