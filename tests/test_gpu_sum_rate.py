"""Per-user SINR and sum rate of the precoder (eq. (rate)) on the GPU against the FP64 oracle (GB300)."""
import numpy as np
import pytest

import kzgen
from oracle import rzf as orz
from oracle import sinr as osinr

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


def gpu_sum_rate(kp, plan, X_rows, snr):
    sinr = torch.empty(plan.K, dtype=torch.float64, device="cuda")
    rate = torch.empty(1, dtype=torch.float64, device="cuda")
    kp.kz_sum_rate(plan, X_rows, snr, sinr, rate)
    torch.cuda.synchronize()
    return sinr.cpu().numpy(), float(rate.item())


@pytest.mark.parametrize("K,Nt,snr_db", [(12, 160, 10.0), (33, 700, 0.0), (64, 1024, 20.0)])
def test_sum_rate_matches_oracle_on_the_same_precoder(kp, K, Nt, snr_db):
    inst = kzgen.make_instance(300 + K, K, Nt, vr_frac_range=(0.1, 0.4), rhs="identity", nrhs=K, snr_db=snr_db)
    plan = kp.plan_from_instance(inst)
    snr = 10.0 ** (snr_db / 10.0)
    # one-hot right-hand sides: the FP32 residual floor is near 3e-7, so tol 1e-6
    out = kp.precode(plan, kp.rhs_tensor(inst.S), inst.xi, algo="vr_oahk", tol=1e-6, max_iter=3000)
    assert out["converged"]
    sinr, rate = gpu_sum_rate(kp, plan, out["x"], snr)
    X = out["x"].cpu().numpy().T.astype(np.complex128)
    ref = osinr.sinr(inst.dense(), X, snr)
    assert np.max(np.abs(sinr - ref) / ref) <= 1e-5
    assert abs(rate - np.sum(np.log2(1.0 + ref))) <= 1e-5 * abs(rate)
    # against the FP64 RZF precoder: within 0.01 dB per user
    V, Xr = orz.rzf(inst.dense(), inst.xi, inst.S)
    assert np.max(np.abs(10 * np.log10(sinr) - osinr.sinr_db(inst.dense(), Xr, snr))) <= 0.01


def test_sum_rate_single_user_closed_form(kp):
    """K = 1: F = h^H / ||h||, SINR = snr ||h||^2 exactly (the oracle's pin)."""
    inst = kzgen.make_instance(310, 1, 200, vr_len_range=(40, 40), rhs="identity", nrhs=1)
    plan = kp.plan_from_instance(inst)
    X = torch.from_numpy(np.ascontiguousarray(inst.dense().conj().astype(np.complex64))).cuda()
    sinr, rate = gpu_sum_rate(kp, plan, X, 7.0)
    h2 = float(np.sum(np.abs(inst.H_packed.astype(np.complex128)) ** 2))
    assert sinr[0] == pytest.approx(7.0 * h2, rel=1e-6)
    assert rate == pytest.approx(np.log2(1 + 7.0 * h2), rel=1e-6)


def test_sum_rate_orthogonal_users_have_no_interference(kp):
    """Disjoint VRs: H H^H is diagonal, RZF is per-user MRT and nothing leaks."""
    off = [1 + 13 * k for k in range(6)]
    inst = kzgen.make_instance(311, 6, 80, vr_override=(off, [11] * 6), rhs="identity", nrhs=6)
    plan = kp.plan_from_instance(inst)
    out = kp.precode(plan, kp.rhs_tensor(inst.S), inst.xi, algo="vr_oahk", tol=1e-6, max_iter=100)
    sinr, _ = gpu_sum_rate(kp, plan, out["x"], 10.0)
    X = out["x"].cpu().numpy().T.astype(np.complex128)
    G = inst.dense() @ (X / np.linalg.norm(X))
    expect = 10.0 * np.abs(np.diag(G)) ** 2  # no interference term
    assert np.max(np.abs(sinr - expect) / expect) <= 1e-5


def test_sum_rate_batched_matches_single(kp):
    insts = [kzgen.make_instance(320 + i, 24, int(Nt), vr_frac_range=(0.1, 0.4), rhs="identity", nrhs=24)
             for i, Nt in enumerate([300, 640, 1024])]
    items, plans = [], []
    for inst in insts:
        p = kp.plan_from_instance(inst)
        plans.append(p)
        items.append(dict(plan=p, s=kp.rhs_tensor(inst.S),
                          x=torch.empty((24, inst.Nt), dtype=torch.complex64, device="cuda"),
                          v=None, iters=torch.empty(24, dtype=torch.int32, device="cuda"),
                          resid=torch.empty(24, dtype=torch.float64, device="cuda"), xi=inst.xi))
    b = kp.kz_batch_prepare(items, 24, "vr_oahk")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    kp.kz_precode_batched(b, "paper", 1e-6, 3000, 0, status=st)
    sinr = torch.empty((3, 24), dtype=torch.float64, device="cuda")
    rate = torch.empty(3, dtype=torch.float64, device="cuda")
    kp.kz_sum_rate_batched(b, 10.0, sinr, rate)
    torch.cuda.synchronize()
    assert st.item() == 0
    for c in range(3):
        s1, r1 = gpu_sum_rate(kp, plans[c], items[c]["x"], 10.0)
        assert np.array_equal(sinr[c].cpu().numpy(), s1) and rate[c].item() == r1


def test_sum_rate_rejects_bad_input(kp):
    inst = kzgen.make_instance(330, 8, 96, vr_frac_range=(0.1, 0.4), rhs="identity", nrhs=8)
    plan = kp.plan_from_instance(inst)
    X = torch.zeros((8, 96), dtype=torch.complex64, device="cuda")
    with pytest.raises(kp.KzError):
        kp.kz_sum_rate(plan, X, 0.0, rate=torch.empty(1, dtype=torch.float64, device="cuda"))
    items = [dict(plan=plan, s=kp.rhs_tensor(inst.S[:, :4]), x=torch.empty((4, 96), dtype=torch.complex64, device="cuda"),
                  v=None, iters=torch.empty(4, dtype=torch.int32, device="cuda"),
                  resid=torch.empty(4, dtype=torch.float64, device="cuda"), xi=inst.xi)]
    b = kp.kz_batch_prepare(items, 4, "vr_oahk")
    with pytest.raises(kp.KzError):  # 4 columns for 8 users
        kp.kz_sum_rate_batched(b, 10.0, rate=torch.empty(1, dtype=torch.float64, device="cuda"))
