"""Plan update, batch rebinding and the batched adjoint against the FP64 oracle (GB300)."""
import numpy as np
import pytest

import kzgen
from oracle import adjoint as oadj
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


def reshuffled(inst, seed):
    """Same VR layout, another channel: the rows of a second draw cut to inst's VRs."""
    other = kzgen.make_instance(seed, inst.K, inst.Nt, vr_override=(inst.vr_offset, inst.vr_len), nrhs=inst.S.shape[1],
                                snr_db=inst.snr_db)
    assert np.array_equal(other.vr_len, inst.vr_len)
    return other


def test_plan_update_matches_fresh_plan(kp):
    a = kzgen.make_instance(41, 24, 300, vr_len_range=(20, 150), nrhs=12, snr_db=10.0)
    b = reshuffled(a, 42)
    plan = kp.plan_from_instance(a)
    kp.kz_plan_update(plan, torch.from_numpy(b.H_packed).cuda())
    out = kp.precode(plan, kp.rhs_tensor(b.S), b.xi, algo="vr_oahk", tol=1e-7, max_iter=3000)
    V, X = orz.rzf(b.dense(), b.xi, b.S)
    assert out["converged"]
    assert np.all(orz.rel_err(out["x"].cpu().numpy().T.astype(np.complex128), X) <= TOL_X)
    # the Bai-Wu sum of GRK reads the updated norms on the device
    out = kp.precode(plan, kp.rhs_tensor(b.S), b.xi, algo="grk", tol=1e-6, max_iter=40000)
    assert out["converged"]
    assert np.all(orz.rel_err(out["x"].cpu().numpy().T.astype(np.complex128), X) <= TOL_X)


def test_plan_update_rejects_bad_input(kp):
    a = kzgen.make_instance(43, 4, 64, vr_len_range=(8, 20), nrhs=2)
    plan = kp.plan_from_instance(a)
    with pytest.raises(ValueError):
        kp.kz_plan_update(plan, torch.zeros(3, dtype=torch.complex64, device="cuda"))


def _items(kp, insts, nrhs, xi_scale=1.0):
    return [dict(plan=None, s=kp.rhs_tensor(i.S), x=torch.empty((nrhs, i.Nt), dtype=torch.complex64, device="cuda"),
                 v=torch.empty((nrhs, i.K), dtype=torch.complex64, device="cuda"),
                 iters=torch.empty(nrhs, dtype=torch.int32, device="cuda"),
                 resid=torch.empty(nrhs, dtype=torch.float64, device="cuda"), xi=i.xi * xi_scale) for i in insts]


def test_batch_rebind_new_buffers_and_xi(kp):
    insts = [kzgen.make_instance(60 + k, int(K), int(Nt), vr_frac_range=(0.1, 0.4), nrhs=8)
             for k, (K, Nt) in enumerate([(5, 96), (17, 300), (30, 640)])]
    plans = [kp.plan_from_instance(i) for i in insts]
    first = _items(kp, insts, 8)
    for it, p in zip(first, plans):
        it["plan"] = p
    b = kp.kz_batch_prepare(first, 8, "vr_oahk")
    second = _items(kp, insts, 8, xi_scale=3.0)
    for it, p in zip(second, plans):
        it["plan"] = p
    kp.kz_batch_rebind(b, second)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    kp.kz_precode_batched(b, "paper", 1e-7, 3000, 0, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    for inst, it in zip(insts, second):
        V, X = orz.rzf(inst.dense(), 3.0 * inst.xi, inst.S)
        assert np.all(orz.rel_err(it["x"].cpu().numpy().T.astype(np.complex128), X) <= TOL_X)
        assert np.all(orz.rel_err(it["v"].cpu().numpy().T.astype(np.complex128), V) <= TOL_X)
    wrong = list(second)
    wrong[0] = second[1]  # consistent buffers, but not the plan item 0 was prepared with
    with pytest.raises(kp.KzError):
        kp.kz_batch_rebind(b, wrong)


def test_batched_adjoint_matches_per_channel(kp):
    rng = np.random.default_rng(3)
    nrhs = 9
    insts = [kzgen.make_instance(80 + k, int(K), int(Nt), vr_len_range=(lo, hi), nrhs=nrhs, snr_db=10.0)
             for k, (K, Nt, lo, hi) in enumerate([(7, 128, 10, 60), (20, 333, 17, 121), (33, 700, 64, 400)])]
    plans = [kp.plan_from_instance(i) for i in insts]
    fw = []
    for inst, p in zip(insts, plans):
        out = kp.precode(p, kp.rhs_tensor(inst.S), inst.xi, algo="vr_oahk", tol=1e-7, max_iter=3000)
        assert out["converged"]
        gq = torch.from_numpy((rng.standard_normal((nrhs, inst.K)) + 1j * rng.standard_normal((nrhs, inst.K)))
                              .astype(np.complex64)).cuda()
        gx = torch.from_numpy((rng.standard_normal((nrhs, inst.Nt)) + 1j * rng.standard_normal((nrhs, inst.Nt)))
                              .astype(np.complex64)).cuda()
        fw.append((out, gq, gx))
    # per channel
    ref = []
    for inst, p, (out, gq, gx) in zip(insts, plans, fw):
        lam = torch.empty_like(out["v"])
        y = torch.empty_like(out["x"])
        gH = torch.empty(p.sum_len, dtype=torch.complex64, device="cuda")
        gxi = torch.empty(1, dtype=torch.float32, device="cuda")
        it = torch.empty(nrhs, dtype=torch.int32, device="cuda")
        rs = torch.empty(nrhs, dtype=torch.float64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        kp.kz_precode_adjoint(p, nrhs, inst.xi, out["v"], out["x"], gq, gx, 1e-7, 3000, lam, y, gH, gxi, it, rs, st)
        torch.cuda.synchronize()
        assert st.item() == 0
        ref.append((lam.cpu().numpy(), gH.cpu().numpy(), float(gxi.item())))
    # batched, one channel without G_X and one without G_Q
    items = _items(kp, insts, nrhs)
    for it, p in zip(items, plans):
        it["plan"] = p
    b = kp.kz_batch_prepare(items, nrhs, "vr_oahk")
    gHs = [torch.empty(p.sum_len, dtype=torch.complex64, device="cuda") for p in plans]
    gxis = torch.empty(len(insts), dtype=torch.float32, device="cuda")
    adj = [dict(Q=out["v"], X=out["x"], G_Q=gq, G_X=gx, grad_H=gHs[c], grad_xi=gxis[c:c + 1])
           for c, (out, gq, gx) in enumerate(fw)]
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    kp.kz_precode_adjoint_batched(b, adj, 1e-7, 3000, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    for c in range(len(insts)):
        lam_r, gH_r, gxi_r = ref[c]
        lam = items[c]["v"].cpu().numpy()
        assert np.linalg.norm(lam - lam_r) <= 1e-5 * np.linalg.norm(lam_r)
        assert np.linalg.norm(gHs[c].cpu().numpy() - gH_r) <= 1e-5 * np.linalg.norm(gH_r)
        assert abs(float(gxis[c].item()) - gxi_r) <= 1e-4 * abs(gxi_r)


def test_batched_adjoint_one_sided_gradients(kp):
    """G_Q alone and G_X alone, against the dense FP64 adjoint of the oracle's solve."""
    nrhs = 6
    insts = [kzgen.make_instance(90 + k, 12, 200, vr_len_range=(30, 120), nrhs=nrhs, snr_db=5.0) for k in range(2)]
    plans = [kp.plan_from_instance(i) for i in insts]
    rng = np.random.default_rng(11)
    items = _items(kp, insts, nrhs)
    for it, p in zip(items, plans):
        it["plan"] = p
    b = kp.kz_batch_prepare(items, nrhs, "vr_oahk")
    adj, dense = [], []
    gHs = [torch.empty(p.sum_len, dtype=torch.complex64, device="cuda") for p in plans]
    gxis = torch.empty(2, dtype=torch.float32, device="cuda")
    for c, (inst, p) in enumerate(zip(insts, plans)):
        out = kp.precode(p, kp.rhs_tensor(inst.S), inst.xi, algo="vr_oahk", tol=1e-7, max_iter=3000)
        G = (rng.standard_normal((nrhs, inst.K if c == 0 else inst.Nt))
             + 1j * rng.standard_normal((nrhs, inst.K if c == 0 else inst.Nt))).astype(np.complex64)
        Gt = torch.from_numpy(G).cuda()
        adj.append(dict(Q=out["v"], X=out["x"], G_Q=Gt if c == 0 else None, G_X=Gt if c == 1 else None,
                        grad_H=gHs[c], grad_xi=gxis[c:c + 1]))
        dense.append(G)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    kp.kz_precode_adjoint_batched(b, adj, 1e-7, 3000, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    for c, inst in enumerate(insts):
        H = inst.dense()
        A = H @ H.conj().T + inst.xi * np.eye(inst.K)
        Gtil = dense[c].T.astype(np.complex128) if c == 0 else H @ dense[c].T.astype(np.complex128)
        Lam = np.linalg.solve(A, Gtil)
        lam = items[c]["v"].cpu().numpy().T
        assert np.linalg.norm(lam - Lam) <= 1e-5 * np.linalg.norm(Lam)


def test_batched_autograd_vs_fp64(kp):
    """Sum-rate loss over 3 channels through BatchedPrecoder; gradients against FP64 autograd per channel."""
    from paper_2501_10689_gb300 import autograd as kad
    insts = [kzgen.make_instance(70 + k, 12, 160, vr_len_range=(20, 90), nrhs=12, rhs="identity", snr_db=10.0)
             for k in range(3)]
    pre = kad.BatchedPrecoder([(i.vr_offset, i.vr_len, i.Nt) for i in insts], 12, tol=1e-7, max_iter=3000)
    H = torch.from_numpy(np.concatenate([i.H_packed for i in insts])).cuda().requires_grad_(True)
    xi = torch.tensor([i.xi for i in insts], dtype=torch.float32, device="cuda", requires_grad=True)
    S = torch.cat([kp.rhs_tensor(i.S).reshape(-1) for i in insts])
    snr = 10.0
    for rep in range(2):  # second pass reuses the plans and the prepared batches
        if H.grad is not None:
            H.grad = None
            xi.grad = None
        X, V = pre(H, xi, S)
        Xs = torch.stack(pre.split(X, "x"))
        L = kad.sum_rate_loss_batched(pre.dense(H), Xs, snr)
        L.backward()
        gH = H.grad.cpu().numpy().astype(np.complex128)
        for c, inst in enumerate(insts):
            L_ref, gH_ref, gxi_ref = oadj.reference_gradient(inst, snr)
            seg = gH[int(pre.h_off[c]):int(pre.h_off[c + 1])]
            assert np.linalg.norm(seg - gH_ref) <= 1e-4 * np.linalg.norm(gH_ref)
            assert abs(float(xi.grad[c].item()) - gxi_ref) <= 1e-4 * abs(gxi_ref)
        L_tot = sum(oadj.reference_gradient(i, snr)[0] for i in insts)
        assert abs(float(L.item()) - L_tot) <= 1e-5 * abs(L_tot)


def test_batched_autograd_stale_plans_reloaded(kp):
    """Backward of an earlier forward after another forward loaded other channels."""
    from paper_2501_10689_gb300 import autograd as kad
    a = kzgen.make_instance(75, 10, 128, vr_len_range=(20, 80), nrhs=10, rhs="identity", snr_db=10.0)
    b = reshuffled(a, 76)
    pre = kad.BatchedPrecoder([(a.vr_offset, a.vr_len, a.Nt)], 10, tol=1e-7, max_iter=3000)
    xi = torch.tensor([a.xi], dtype=torch.float32, device="cuda")
    S = kp.rhs_tensor(a.S).reshape(-1)
    Ha = torch.from_numpy(a.H_packed).cuda().requires_grad_(True)
    Hb = torch.from_numpy(b.H_packed).cuda().requires_grad_(True)
    Xa, _ = pre(Ha, xi, S)
    Xb, _ = pre(Hb, xi, S)
    La = kad.sum_rate_loss_batched(pre.dense(Ha), Xa.view(1, 10, a.Nt), 10.0)
    La.backward()
    _, gH_ref, _ = oadj.reference_gradient(a, 10.0)
    assert np.linalg.norm(Ha.grad.cpu().numpy() - gH_ref) <= 1e-3 * np.linalg.norm(gH_ref)
