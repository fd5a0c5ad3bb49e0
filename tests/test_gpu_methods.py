"""Table I's comparison methods as first-class algorithms (GB300, through the
C ABI): SWOR-ERK (energy RK drawing without replacement within each sweep)
and GK (the maximal-residual greedy rule), and the FLOP accounting of Table I.

SWOR-ERK's row sequence depends only on the row norms and the counter-based
draws, so after T = 3K + 5 steps the GPU iterate must be the oracle's literal
iterate (a single different draw would move it by O(1))."""
import numpy as np
import pytest

import kzgen
from oracle import flops as oflops
from oracle import kaczmarz as okz
from oracle import precoder as opc
from oracle import rzf as orz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kp():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_10689_gb300 import kzprecode
    return kzprecode


def ragged(seed=2, nrhs=5):
    return kzgen.make_instance(seed, 14, 301, vr_len_range=(25, 140), snr_db=10.0, nrhs=nrhs)


@pytest.mark.parametrize("algo", ["rk_swor", "gk"])
def test_methods_converge_to_rzf(kp, algo):
    inst = ragged()
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    plan = kp.plan_from_instance(inst)
    out = kp.precode(plan, kp.rhs_tensor(inst.S), inst.xi, algo=algo, sel="paper", tol=1e-7, max_iter=400000)
    assert out["converged"]
    assert np.max(orz.rel_err(out["x"].cpu().numpy().T, X)) <= 1e-5


def test_swor_trajectory_follows_the_oracle(kp):
    inst = ragged(seed=4, nrhs=3)
    T = 3 * inst.K + 5
    ref = okz.solve(okz.System.from_instance(inst), inst.S, "rk_swor", tol=0.0, max_iter=T, seed=7)
    plan = kp.plan_from_instance(inst)
    out = kp.precode(plan, kp.rhs_tensor(inst.S), inst.xi, algo="rk_swor", tol=0.0, max_iter=T, seed=7)
    assert np.all(out["iters"].cpu().numpy() == T)
    assert np.max(orz.rel_err(out["x"].cpu().numpy().T, ref["x"])) <= 1e-5


def test_gk_is_grk_with_argmax(kp):
    inst = ragged(seed=5)
    plan = kp.plan_from_instance(inst)
    S = kp.rhs_tensor(inst.S)
    a = kp.precode(plan, S, inst.xi, algo="gk", sel="paper", tol=1e-7, max_iter=100000)
    b = kp.precode(plan, S, inst.xi, algo="grk", sel="argmax", tol=1e-7, max_iter=100000)
    assert torch.equal(a["x"], b["x"]) and torch.equal(a["iters"], b["iters"])


def test_batched_swor_and_gk(kp):
    rng = np.random.default_rng(3)
    insts = [kzgen.make_instance(40 + i, int(rng.integers(3, 20)), int(rng.choice([96, 257])),
                                 vr_frac_range=(0.1, 0.4), nrhs=4) for i in range(6)]
    for algo in ("rk_swor", "gk"):
        items = []
        for inst in insts:
            p = kp.plan_from_instance(inst)
            items.append(dict(plan=p, s=kp.rhs_tensor(inst.S), x=torch.empty((4, inst.Nt), dtype=torch.complex64,
                                                                               device="cuda"),
                              v=None, iters=torch.empty(4, dtype=torch.int32, device="cuda"),
                              resid=torch.empty(4, dtype=torch.float64, device="cuda"), xi=inst.xi))
        b = kp.kz_batch_prepare(items, 4, algo)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        kp.kz_precode_batched(b, "paper", 1e-6, 400000, 1, status=st)  # above the FP32 residual floor
        torch.cuda.synchronize()
        assert st.item() == 0, algo
        for inst, it in zip(insts, items):
            V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
            assert np.max(orz.rel_err(it["x"].cpu().numpy().T, X)) <= 1e-5, algo


def test_plan_flops_is_table1(kp):
    inst = kzgen.config2(10.0, nrhs=4)
    plan = kp.plan_from_instance(inst)
    F, Xsets = kp.kz_plan_query(plan)[0], None
    from oracle import sets as osets
    X = osets.x_sets(inst.vr_offset, inst.vr_len)
    Q = np.mean([len(q) for q in opc.q_sets(inst.vr_offset, inst.vr_len, inst.Nt, 20)])
    stats = dict(Q=Q, M=float(np.mean(inst.vr_len)), X=float(np.mean([len(x) - 1 for x in X])),
                 F=float(len(F)), V=float(inst.K - len(F)))
    for scheme in ("rzf", "urk", "swor_erk", "gk", "vr_ogrk", "vr_oahk"):
        want = oflops.table1_flops(scheme, inst.K, inst.Nt, T=37.0, **stats)
        got = kp.kz_plan_flops(plan, {"swor_erk": "rk_swor"}.get(scheme, scheme), 20, 37.0)
        assert got == pytest.approx(want, rel=1e-12), scheme


def test_auto_routes_small_and_large_channels(kp):
    """KZ_KERNEL_AUTO in kz_precode: a small channel (16 users, 256 antennas,
    few columns) runs on the small-channel kernel and a large one (4096
    antennas, AHK family) on the group kernel: bit-identical to naming them;
    a fixed column count per CTA keeps the resident kernel."""
    small = kzgen.make_instance(31, 16, 256, vr_len_range=(64, 192), snr_db=10.0, nrhs=3)
    large = kzgen.make_instance(32, 128, 4096, vr_len_range=(256, 1024), snr_db=10.0, nrhs=16)
    for inst, algo, named in ((small, "grk", "small"), (small, "vr_oahk", "small"), (large, "vr_oahk", "group")):
        plan = kp.plan_from_instance(inst)
        S = kp.rhs_tensor(inst.S)
        a = kp.precode(plan, S, inst.xi, algo=algo, tol=1e-6, max_iter=20000, kernel="auto")
        b = kp.precode(plan, S, inst.xi, algo=algo, tol=1e-6, max_iter=20000, kernel=named)
        assert torch.equal(a["x"], b["x"]) and torch.equal(a["iters"], b["iters"]), (algo, named)
        V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
        assert np.all(orz.rel_err(a["x"].cpu().numpy().T, X) <= 1e-5)
    plan = kp.plan_from_instance(small)
    S = kp.rhs_tensor(small.S)
    a = kp.precode(plan, S, small.xi, algo="vr_oahk", tol=1e-6, max_iter=20000, kernel="auto", rhs_per_cta=1)
    b = kp.precode(plan, S, small.xi, algo="vr_oahk", tol=1e-6, max_iter=20000, kernel="resident", rhs_per_cta=1)
    assert torch.equal(a["x"], b["x"])
