"""The group kernel (tcgen05 tensor cores, one channel spread over a group of
CTAs) against the FP64 oracle (GB300, through the C ABI).

* Converged x and v against the closed-form RZF (eq. (precoding), Thm. 1) at
  1e-5, for VR-OAHK (Alg. 3) and AHK (eq. (update4)), FP16 operands (C64
  plans) and BF16 operands (BF16_MIXED plans), on a ragged channel whose last
  column group is partly empty, on config 2 (1024 antennas, 64 users, 256
  columns: one cluster per column group) and config 4 (16384 antennas, 512
  users, 64 columns: every CTA of a cooperative launch).
* Fixed-iteration iterates against the oracle's literal iterates: before any
  refresh the only difference is the 16-bit rounding of the two products, so
  a wrong operand layout, sign or scale would miss by O(1).
* Column chunking over several launches, bitwise reproducibility, and the edge
  cases (zero column, disjoint VRs, one user, max_iter exhausted, NaN input).
"""
import numpy as np
import pytest

import kzgen
from oracle import kaczmarz as okz
from oracle import rzf as orz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_X = 1e-5


@pytest.fixture(scope="module")
def kp():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_10689_gb300 import kzprecode
    return kzprecode


def run(kp, inst, algo, tol=1e-6, max_iter=3000, prec="c64", refresh=0, rhs_per_cta=0, S=None, plan=None):
    plan = plan or kp.plan_from_instance(inst, prec=prec)
    S = kp.rhs_tensor(inst.S if S is None else S)
    out = kp.precode(plan, S, inst.xi, algo=algo, tol=tol, max_iter=max_iter, kernel="group", refresh=refresh,
                     rhs_per_cta=rhs_per_cta)
    return {"x": out["x"].cpu().numpy().T, "v": out["v"].cpu().numpy().T, "iters": out["iters"].cpu().numpy(),
            "resid": out["resid"].cpu().numpy(), "converged": out["converged"], "status": int(out["status"].item())}


def ragged(seed=5, nrhs=37, K=40, Nt=700):
    return kzgen.make_instance(seed, K, Nt, vr_len_range=(50, 300), snr_db=10.0, nrhs=nrhs)


@pytest.mark.parametrize("prec", ["c64", "bf16"])
@pytest.mark.parametrize("algo", ["vr_oahk", "ahk"])
def test_group_ragged_converges_to_rzf(kp, algo, prec):
    inst = ragged()
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, algo, tol=1e-6, prec=prec)
    assert out["converged"], out["status"]
    assert np.all(out["resid"] <= 1e-6 * (1 + 1e-6))
    assert np.max(orz.rel_err(out["x"], X)) <= TOL_X
    assert np.max(orz.rel_err(out["v"], V)) <= TOL_X


@pytest.mark.parametrize("prec,bar", [("c64", 5e-3), ("bf16", 4e-2)])
@pytest.mark.parametrize("T", [1, 2, 4])
@pytest.mark.parametrize("algo", ["vr_oahk", "ahk"])
def test_group_first_iterates_follow_the_oracle(kp, algo, T, prec, bar):
    inst = ragged(seed=3, nrhs=20)
    ref = okz.solve(okz.System.from_instance(inst), inst.S, algo, tol=0.0, max_iter=T)
    out = run(kp, inst, algo, tol=0.0, max_iter=T, prec=prec, refresh=1000)
    assert np.all(out["iters"] == T) and not out["converged"]
    assert np.max(orz.rel_err(out["x"], ref["x"])) <= bar, np.max(orz.rel_err(out["x"], ref["x"]))
    assert np.max(orz.rel_err(out["v"], ref["v"])) <= bar


@pytest.mark.parametrize("snr", [0.0, 10.0, 20.0])
def test_group_config2(kp, snr):
    inst = kzgen.config2(snr)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, "vr_oahk", tol=1e-6)
    assert out["converged"], out["status"]
    assert np.max(orz.rel_err(out["x"], X)) <= TOL_X


@pytest.fixture(scope="module")
def config4():
    inst = kzgen.config4()
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    return inst, V, X


@pytest.mark.parametrize("prec", ["c64", "bf16"])
def test_group_config4(kp, config4, prec):
    """16384 antennas, 512 users, VR 1024-4096, 64 columns: 128 CTAs of one cooperative launch."""
    inst, V, X = config4
    out = run(kp, inst, "vr_oahk", tol=1e-6, prec=prec)
    assert out["converged"], out["status"]
    assert np.max(orz.rel_err(out["x"], X)) <= TOL_X, np.max(orz.rel_err(out["x"], X))


def test_group_column_chunks(kp):
    """4096 antennas (32 blocks: grid barrier), 80 columns at 16 per group: more
    groups than one cooperative launch holds, so two launches."""
    inst = kzgen.make_instance(17, 96, 4096, vr_frac_range=(0.1, 0.4), snr_db=10.0, nrhs=80)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, "vr_oahk", tol=1e-6, rhs_per_cta=16)
    assert out["converged"]
    assert np.max(orz.rel_err(out["x"], X)) <= TOL_X


def test_group_deterministic(kp):
    inst = ragged(seed=8, nrhs=33)
    plan = kp.plan_from_instance(inst)
    a = run(kp, inst, "vr_oahk", plan=plan)
    b = run(kp, inst, "vr_oahk", plan=plan)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["iters"], b["iters"])


def test_group_edge_cases(kp):
    # a zero column among others, and a partial last group
    inst = ragged(seed=9, nrhs=18)
    S = inst.S.copy()
    S[:, 4] = 0
    V, X = orz.rzf(inst.dense(), inst.xi, S)
    out = run(kp, inst, "vr_oahk", S=S)
    assert out["converged"] and out["iters"][4] == 0 and np.all(out["x"][:, 4] == 0)
    keep = [j for j in range(18) if j != 4]
    assert np.max(orz.rel_err(out["x"][:, keep], X[:, keep])) <= TOL_X
    # disjoint VRs: the orthogonal half-step is the whole solution (Lemma 1, Thm. 4)
    off = [k * 40 for k in range(10)]
    inst = kzgen.make_instance(10, 10, 400, vr_override=(off, [30] * 10), nrhs=16)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, "vr_oahk", tol=1e-6)
    assert out["converged"] and np.all(out["iters"] == 1)
    assert np.max(orz.rel_err(out["x"], X)) <= TOL_X
    # one user
    inst = kzgen.make_instance(11, 1, 300, vr_len_range=(100, 100), nrhs=16)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, "ahk", tol=1e-6)
    assert out["converged"] and np.max(orz.rel_err(out["x"], X)) <= TOL_X
    # max_iter exhausted: not converged, outputs written, iters = max_iter
    inst = ragged(seed=12, nrhs=16)
    out = run(kp, inst, "vr_oahk", tol=1e-9, max_iter=3)
    assert not out["converged"] and np.all(out["iters"] == 3) and np.all(np.isfinite(out["x"]))


def test_group_nan_input_sets_numeric_bit(kp):
    inst = ragged(seed=13, nrhs=16)
    S = inst.S.copy()
    S[2, 5] = np.complex64(complex(np.nan, 0.0))
    plan = kp.plan_from_instance(inst)
    Sd = kp.rhs_tensor(S)
    out = kp.precode(plan, Sd, inst.xi, algo="vr_oahk", tol=1e-6, max_iter=100, kernel="group", sync=False)
    torch.cuda.synchronize()
    assert int(out["status"].item()) & kp.KZ_STATUS_BIT_NUMERIC


def test_group_rejects_unsupported(kp):
    inst = ragged(seed=14, nrhs=16)
    plan = kp.plan_from_instance(inst)
    S = kp.rhs_tensor(inst.S)
    with pytest.raises(kp.KzError):
        kp.precode(plan, S, inst.xi, algo="grk", kernel="group")
    with pytest.raises(kp.KzError):
        kp.precode(plan, S, inst.xi, algo="vr_oahk", kernel="group", rhs_per_cta=8)


@pytest.mark.parametrize("seed", range(4))
def test_group_random_shapes(kp, seed):
    """Random channels for the group kernel: antennas not a multiple of the
    128-antenna block, columns not a multiple of the group width, users up to
    a few hundred."""
    rng = np.random.default_rng(3000 + seed)
    Nt = int(rng.integers(300, 3000))
    K = int(rng.integers(8, min(200, Nt // 4)))
    nrhs = int(rng.integers(1, 70))
    inst = kzgen.make_instance(4000 + seed, K, Nt, vr_frac_range=(0.05, 0.5), snr_db=float(rng.uniform(0, 20)),
                               nrhs=nrhs)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    for algo in ("vr_oahk", "ahk"):
        out = run(kp, inst, algo, tol=1e-6, max_iter=3000)
        assert out["converged"], (Nt, K, nrhs, algo, out["status"])
        assert np.max(orz.rel_err(out["x"], X)) <= TOL_X, (Nt, K, nrhs, algo)
