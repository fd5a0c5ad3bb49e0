"""The small-channel kernel (one CTA per column, K <= 32 users) against the FP64
oracle (GB300, through the C ABI): converged x against the closed-form RZF
(eq. (precoding)) for every method, fixed-iteration iterates against the
oracle's literal iterates (deterministic rules, and RK / SWOR-ERK whose draws
depend only on the row norms), and the edge cases.

The shapes reach each of the kernel's forms: the register-resident one with
16 rows and one antenna per thread (config 1: 16 users, 256 antennas), with
two antennas per thread (12 users, 400 antennas) and with 32 rows (28 users,
200 antennas), and the shared-memory one (20 users, 301 antennas; RK always)."""
import numpy as np
import pytest

import kzgen
from oracle import kaczmarz as okz
from oracle import rzf as orz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL = [("rk_energy", "paper"), ("rk_uniform", "paper"), ("rk_swor", "paper"), ("grk", "paper"), ("grk", "baiwu"),
       ("gk", "paper"), ("vr_ogrk", "argmax"), ("vr_ogrk", "paper"), ("ahk", "paper"), ("vr_oahk", "paper")]


@pytest.fixture(scope="module")
def kp():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_10689_gb300 import kzprecode
    return kzprecode


def run(kp, inst, algo, sel="paper", tol=1e-6, max_iter=100000, cols=0, S=None, seed=0):
    plan = kp.plan_from_instance(inst)
    out = kp.precode(plan, kp.rhs_tensor(inst.S if S is None else S), inst.xi, algo=algo, sel=sel, tol=tol,
                     max_iter=max_iter, kernel="small", rhs_per_cta=cols, seed=seed)
    return {"x": out["x"].cpu().numpy().T, "v": out["v"].cpu().numpy().T, "iters": out["iters"].cpu().numpy(),
            "resid": out["resid"].cpu().numpy(), "converged": out["converged"], "status": int(out["status"].item())}


def ragged(seed=3, nrhs=5, K=20, Nt=301):
    return kzgen.make_instance(seed, K, Nt, vr_len_range=(20, 150), snr_db=10.0, nrhs=nrhs)


SHAPES = {"config1": None, "ragged": (20, 301), "k12_n400": (12, 400), "k28_n200": (28, 200)}


def shaped(case, seed=3, nrhs=5):
    if case == "config1":
        return kzgen.config1()
    K, Nt = SHAPES[case]
    return ragged(seed=seed, nrhs=nrhs, K=K, Nt=Nt)


@pytest.mark.parametrize("algo,sel", ALL)
@pytest.mark.parametrize("case", list(SHAPES))
def test_small_converges_to_rzf(kp, algo, sel, case):
    inst = shaped(case)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, algo, sel, tol=1e-6)
    assert out["converged"], out["status"]
    assert np.all(out["resid"] <= 1e-6 * (1 + 1e-6))
    assert np.max(orz.rel_err(out["x"], X)) <= 1e-5
    assert np.max(orz.rel_err(out["v"], V)) <= 1e-5


@pytest.mark.parametrize("algo,sel,T", [("ahk", "paper", 6), ("vr_oahk", "paper", 4), ("grk", "argmax", 25),
                                        ("vr_ogrk", "argmax", 25), ("rk_energy", "paper", 45),
                                        ("rk_swor", "paper", 45)])
@pytest.mark.parametrize("cols", [0, 1])
@pytest.mark.parametrize("case", ["config1", "ragged", "k12_n400", "k28_n200"])
def test_small_fixed_iterations_follow_the_oracle(kp, algo, sel, T, cols, case):
    inst = shaped(case, seed=4, nrhs=6)
    ref = okz.solve(okz.System.from_instance(inst), inst.S, algo, rule=sel, tol=0.0, max_iter=T, seed=11)
    out = run(kp, inst, algo, sel, tol=0.0, max_iter=T, cols=cols, seed=11)
    assert np.all(out["iters"] == T)
    assert np.max(orz.rel_err(out["x"], ref["x"])) <= 1e-5
    assert np.max(orz.rel_err(out["v"], ref["v"])) <= 1e-5


@pytest.mark.parametrize("case", ["ragged", "k12_n400"])
def test_small_iteration_counts_close_to_oracle(kp, case):
    inst = shaped(case, seed=5, nrhs=4)
    for algo in ("vr_oahk", "ahk"):
        ref = okz.solve(okz.System.from_instance(inst), inst.S, algo, tol=1e-6, max_iter=5000)
        out = run(kp, inst, algo, tol=1e-6)
        assert np.all(np.abs(out["iters"] - ref["iters"]) <= 3), (algo, out["iters"], ref["iters"])


def test_small_edge_cases(kp):
    inst = ragged(seed=6, nrhs=5)
    S = inst.S.copy()
    S[:, 2] = 0
    out = run(kp, inst, "vr_oahk", S=S)
    assert out["converged"] and out["iters"][2] == 0 and np.all(out["x"][:, 2] == 0)
    off = [k * 30 for k in range(8)]
    inst = kzgen.make_instance(7, 8, 240, vr_override=(off, [20] * 8), nrhs=3)
    out = run(kp, inst, "vr_oahk", tol=1e-6)
    assert out["converged"] and np.all(out["iters"] == 1)
    inst = kzgen.make_instance(8, 1, 100, vr_len_range=(40, 40), nrhs=2)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, "grk", "argmax", tol=1e-6)
    assert out["converged"] and np.max(orz.rel_err(out["x"], X)) <= 1e-5
    inst = ragged(seed=9, nrhs=2)
    out = run(kp, inst, "vr_oahk", tol=1e-12, max_iter=3)
    assert not out["converged"] and np.all(out["iters"] == 3)
    S = inst.S.copy()
    S[1, 0] = np.complex64(complex(np.nan, 0))
    plan = kp.plan_from_instance(inst)
    o = kp.precode(plan, kp.rhs_tensor(S), inst.xi, algo="grk", tol=1e-6, max_iter=100, kernel="small", sync=False)
    torch.cuda.synchronize()
    assert int(o["status"].item()) & kp.KZ_STATUS_BIT_NUMERIC


def test_small_rejects_large_channels(kp):
    inst = kzgen.make_instance(10, 40, 300, vr_len_range=(20, 80), nrhs=1)
    plan = kp.plan_from_instance(inst)
    with pytest.raises(kp.KzError):
        kp.precode(plan, kp.rhs_tensor(inst.S), inst.xi, algo="grk", kernel="small")


@pytest.mark.parametrize("seed", range(6))
def test_small_random_shapes(kp, seed):
    """Random channels within the kernel's limits (users 1-32, antennas
    2-511, VRs from 1 antenna to the whole array): every method reaches the
    FP64 RZF at 1e-5."""
    rng = np.random.default_rng(1000 + seed)
    K = int(rng.integers(1, 33))
    Nt = int(rng.integers(K + 1, 512))
    lo = int(rng.integers(1, max(2, Nt // 2)))
    inst = kzgen.make_instance(2000 + seed, K, Nt, vr_len_range=(lo, Nt), snr_db=float(rng.uniform(0, 20)),
                               nrhs=int(rng.integers(1, 5)))
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    for algo, sel in (("grk", "paper"), ("vr_ogrk", "argmax"), ("ahk", "paper"), ("vr_oahk", "paper"),
                      ("rk_energy", "paper")):
        out = run(kp, inst, algo, sel, tol=1e-6, max_iter=400000)
        assert out["converged"], (K, Nt, algo, out["status"])
        assert np.max(orz.rel_err(out["x"], X)) <= 1e-5, (K, Nt, algo)
