"""Full-size parity of the benchmarked launch, corrupted inputs, dense plans and
full-size gradients (GB300, through the C ABI).

* The 512-channel, 16-column batch the benchmark times, run in the launch the
  benchmark runs (``kz_batch_tune`` on the batch, and the tensor-core J = 8
  launch it picks): every channel's x and v against the FP64 RZF at 1e-5
  (eq. (precoding), Thm. 1).
* NaN in one entry of H, and separately in one entry of s, on the FP32
  resident kernel, the tensor-core kernel and the Kaczmarz row kernel: the call
  returns, and the status word carries KZ_STATUS_BIT_NUMERIC.  (The corruption
  is made on the host; nothing here faults the GPU.)
* A plan built from a dense K x Nt matrix solves bit-identically to the plan
  built from the same VR entries packed (Sec. II, eqs. (3)-(4)).
* The batched gradient on config-5-sized channels against the FP64 dense-RZF
  autograd gradient at 1e-4, and the per-channel backward raising when its
  adjoint solve does not converge or meets a NaN.
"""
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


# ---------------------------------------------------------------- full-size benchmark batch
@pytest.fixture(scope="module")
def config3_batch(kp):
    import bench
    insts = kzgen.config3(bench.N_INST)
    items = []
    for inst in insts:
        p = kp.plan_from_instance(inst)
        items.append(dict(plan=p, s=kp.rhs_tensor(inst.S),
                          x=torch.empty((bench.NRHS, inst.Nt), dtype=torch.complex64, device="cuda"),
                          v=torch.empty((bench.NRHS, inst.K), dtype=torch.complex64, device="cuda"),
                          iters=torch.empty(bench.NRHS, dtype=torch.int32, device="cuda"),
                          resid=torch.empty(bench.NRHS, dtype=torch.float64, device="cuda"), xi=inst.xi))
    ref = [orz.rzf(inst.dense(), inst.xi, inst.S) for inst in insts]
    return insts, items, ref


def _check_all(kp, insts, items, ref, tol):
    worst_x = worst_v = 0.0
    for inst, it, (V, X) in zip(insts, items, ref):
        ex = orz.rel_err(it["x"].cpu().numpy().T, X)
        ev = orz.rel_err(it["v"].cpu().numpy().T, V)
        worst_x, worst_v = max(worst_x, float(ex.max())), max(worst_v, float(ev.max()))
        assert np.all(it["resid"].cpu().numpy() <= tol * (1 + 1e-6))
    assert worst_x <= TOL_X and worst_v <= TOL_X, (worst_x, worst_v)


@pytest.mark.parametrize("launch", ["bench", ("tc", 8, 512)])
def test_benchmark_batch_every_channel(kp, config3_batch, launch):
    """All 512 channels (8192 columns) of the benchmark batch, in the launch the
    benchmark times (autotuned as bench.py does) and in the tensor-core J = 8 launch."""
    import bench
    insts, items, ref = config3_batch
    b = kp.kz_batch_prepare(items, bench.NRHS, "vr_oahk")
    if launch == "bench":
        kp.kz_batch_tune(b, "paper", bench.TOL, bench.MAX_ITER, 0)
    else:
        kp.kz_batch_set_launch(b, *launch)
    for it in items:
        it["x"].zero_()
        it["v"].zero_()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    kp.kz_precode_batched(b, "paper", bench.TOL, bench.MAX_ITER, 0, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    _check_all(kp, insts, items, ref, bench.TOL)


# ---------------------------------------------------------------- corrupted inputs
def _nan_case(kp, where, algo, sel, kernel, K=24, Nt=400):
    inst = kzgen.make_instance(81, K, Nt, vr_len_range=(40, 160), nrhs=8, snr_db=10.0)
    Hp = inst.H_packed.copy()
    S = inst.S.copy()
    if where == "H":
        Hp[int(inst.vr_len[:5].sum()) + 7] = np.complex64(complex(np.nan, 0.0))  # user 5, 8th VR entry
    else:
        S[3, 2] = np.complex64(complex(0.0, np.nan))
    plan = kp.kz_plan_create(inst.K, inst.Nt, inst.vr_offset, inst.vr_len, torch.from_numpy(Hp).cuda())
    out = {}
    x = torch.empty((8, inst.Nt), dtype=torch.complex64, device="cuda")
    v = torch.empty((8, inst.K), dtype=torch.complex64, device="cuda")
    iters = torch.empty(8, dtype=torch.int32, device="cuda")
    resid = torch.empty(8, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    kp.kz_precode_ex(plan, kp.rhs_tensor(S), 8, inst.xi, algo, sel, 1e-6, 200, 0, x, v, iters, resid, status,
                     kernel, 0, 0)
    torch.cuda.synchronize()
    out["status"] = int(status.item())
    out["iters"] = iters.cpu().numpy()
    return out


@pytest.mark.parametrize("where", ["H", "s"])
@pytest.mark.parametrize("algo,sel,kernel", [("vr_oahk", "paper", "resident"), ("vr_oahk", "paper", "tc"),
                                             ("ahk", "paper", "tc"), ("grk", "paper", "auto"),
                                             ("vr_ogrk", "argmax", "auto"), ("rk_energy", "paper", "auto")])
def test_nan_input_sets_numeric_bit(kp, where, algo, sel, kernel):
    out = _nan_case(kp, where, algo, sel, kernel)
    assert out["status"] & kp.KZ_STATUS_BIT_NUMERIC, out


@pytest.mark.parametrize("where", ["H", "s"])
@pytest.mark.parametrize("algo,sel", [("vr_oahk", "paper"), ("ahk", "paper"), ("grk", "paper"),
                                      ("vr_ogrk", "argmax"), ("rk_swor", "paper")])
@pytest.mark.parametrize("shape", [(24, 400), (12, 200)])
def test_nan_input_small_channel_kernel(kp, where, algo, sel, shape):
    """Both forms of the small-channel kernel: shared-memory (24 users, 400
    antennas; RK always) and register-resident (12 users, 200 antennas)."""
    out = _nan_case(kp, where, algo, sel, "small", K=shape[0], Nt=shape[1])
    assert out["status"] & kp.KZ_STATUS_BIT_NUMERIC, out


# ---------------------------------------------------------------- dense plans
@pytest.mark.parametrize("prec", ["c64", "bf16"])
def test_dense_plan_matches_packed_plan_bitwise(kp, prec):
    inst = kzgen.make_instance(91, 30, 513, vr_len_range=(37, 201), nrhs=6, snr_db=10.0)
    D = inst.dense().copy()
    # entries outside the VRs are not part of the channel (eq. (3)): fill them
    # with garbage, which kz_plan_dense must never read
    mask = np.zeros_like(D, dtype=bool)
    for k in range(inst.K):
        mask[k, inst.vr_offset[k]:inst.vr_offset[k] + inst.vr_len[k]] = True
    D[~mask] = np.complex64(1e3 + 1e3j)
    pd = kp.kz_plan_dense(inst.K, inst.Nt, inst.vr_offset, inst.vr_len, torch.from_numpy(D).cuda(), prec=prec)
    pp = kp.plan_from_instance(inst, prec=prec)
    assert kp.kz_plan_query(pd)[0].tolist() == kp.kz_plan_query(pp)[0].tolist()
    S = kp.rhs_tensor(inst.S)
    for algo in (("vr_oahk", "paper"), ("grk", "argmax")):
        if prec == "bf16" and algo[0] == "grk":
            continue
        a = kp.precode(pd, S, inst.xi, algo=algo[0], sel=algo[1], tol=1e-7, max_iter=20000)
        b = kp.precode(pp, S, inst.xi, algo=algo[0], sel=algo[1], tol=1e-7, max_iter=20000)
        assert torch.equal(a["x"], b["x"]) and torch.equal(a["iters"], b["iters"])
        V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
        assert np.all(orz.rel_err(a["x"].cpu().numpy().T, X) <= TOL_X)


# ---------------------------------------------------------------- gradients
def test_batched_gradient_config5_size_vs_fp64(kp):
    """Four channels of the gradient workload (Nt = 2048, K = 128, VR 256-1024,
    identity symbols), batched forward + adjoint in the tuned launch, against
    the FP64 dense-RZF autograd gradient at 1e-4."""
    from paper_2501_10689_gb300 import autograd as kad
    insts = [kzgen.config5_instance(i) for i in range(4)]
    pre = kad.BatchedPrecoder([(i.vr_offset, i.vr_len, i.Nt) for i in insts], nrhs=128, tol=1e-6, max_iter=3000)
    H = torch.tensor(np.concatenate([i.H_packed for i in insts]), device="cuda", requires_grad=True)
    xi = torch.tensor([i.xi for i in insts], dtype=torch.float32, device="cuda", requires_grad=True)
    S = torch.cat([kp.rhs_tensor(i.S).reshape(-1) for i in insts])
    X, V = pre(H, xi, S)
    snr = 10.0 ** (insts[0].snr_db / 10.0)
    L = kad.sum_rate_loss_batched(pre.dense(H), X.view(len(insts), 128, -1), snr)
    L.backward()
    gH = H.grad.cpu().numpy().astype(np.complex128)
    gxi = xi.grad.cpu().numpy()
    off = 0
    for c, inst in enumerate(insts):
        L_ref, gH_ref, gxi_ref = oadj.reference_gradient(inst)
        n = inst.H_packed.size
        assert np.linalg.norm(gH[off:off + n] - gH_ref) <= 1e-4 * np.linalg.norm(gH_ref), c
        assert abs(gxi[c] - gxi_ref) <= 1e-4 * abs(gxi_ref), c
        off += n


def test_backward_raises_when_adjoint_does_not_converge(kp):
    from paper_2501_10689_gb300 import autograd as kad
    inst = kzgen.make_instance(5, 8, 96, vr_len_range=(12, 40), nrhs=8, rhs="identity", snr_db=20.0)
    Hp = torch.tensor(inst.H_packed, device="cuda", requires_grad=True)
    S = kp.rhs_tensor(inst.S)
    X, V = kad.precode(Hp, inst.xi, S, inst.vr_offset, inst.vr_len, inst.Nt, tol=1e-7, adj_max_iter=1)
    L = kad.sum_rate_loss(kad.dense_from_packed(Hp, inst.vr_offset, inst.vr_len, inst.Nt), X, 10.0)
    with pytest.raises(kp.KzError, match="did not converge"):
        L.backward()


def test_backward_raises_on_nan_gradient(kp):
    from paper_2501_10689_gb300 import autograd as kad
    inst = kzgen.make_instance(6, 8, 96, vr_len_range=(12, 40), nrhs=8, rhs="identity", snr_db=10.0)
    Hp = torch.tensor(inst.H_packed, device="cuda", requires_grad=True)
    X, V = kad.precode(Hp, inst.xi, kp.rhs_tensor(inst.S), inst.vr_offset, inst.vr_len, inst.Nt, tol=1e-7)
    g = torch.zeros_like(X)
    g[2, int(inst.vr_offset[0]) + 1] = complex(float("nan"), 0.0)  # an antenna user 0 sees: H G_X carries it
    with pytest.raises(kp.KzError, match="NaN"):
        X.backward(g)


# ---------------------------------------------------------------- batched channel update
def test_batch_update_items_in_ranges_equals_whole_update(kp):
    """kz_batch_update_items over three item ranges, each reading only its
    own channels from a buffer filled range by range, leaves the plans
    exactly as one kz_batch_update does (bit-identical solutions)."""
    rng = np.random.default_rng(6)
    insts = [kzgen.make_instance(800 + i, int(rng.integers(4, 30)), int(rng.choice([97, 256, 640])),
                                 vr_frac_range=(0.1, 0.4), nrhs=4) for i in range(7)]
    new = [kzgen.make_instance(900 + i, inst.K, inst.Nt, vr_override=(inst.vr_offset, inst.vr_len), nrhs=4)
           for i, inst in enumerate(insts)]

    def batch_for():
        items = [dict(plan=kp.plan_from_instance(i), s=kp.rhs_tensor(n.S),
                      x=torch.zeros((4, i.Nt), dtype=torch.complex64, device="cuda"),
                      v=torch.zeros((4, i.K), dtype=torch.complex64, device="cuda"),
                      iters=torch.zeros(4, dtype=torch.int32, device="cuda"),
                      resid=torch.zeros(4, dtype=torch.float64, device="cuda"), xi=n.xi) for i, n in zip(insts, new)]
        return items, kp.kz_batch_prepare(items, 4, "vr_oahk")

    H_new = np.concatenate([i.H_packed for i in new])
    items_a, b_a = batch_for()
    kp.kz_batch_update(b_a, torch.from_numpy(H_new).cuda())
    items_b, b_b = batch_for()
    H_b = torch.full((H_new.size,), complex(float("nan"), 0.0), dtype=torch.complex64, device="cuda")
    off = np.concatenate([[0], np.cumsum([i.vr_len.sum() for i in new])])
    for first, count in ((0, 2), (2, 4), (6, 1)):  # each range's channels arrive just before its update
        a, b = int(off[first]), int(off[first + count])
        H_b[a:b] = torch.from_numpy(H_new[a:b]).cuda()
        kp.kz_batch_update_items(b_b, H_b, first, count)
    for b in (b_a, b_b):
        kp.kz_precode_batched(b, "paper", 1e-7, 3000, 0)
    torch.cuda.synchronize()
    for ia, ib, n in zip(items_a, items_b, new):
        assert torch.equal(ia["x"], ib["x"]) and torch.equal(ia["iters"], ib["iters"])
        V, X = orz.rzf(n.dense(), n.xi, n.S)
        assert np.all(orz.rel_err(ib["x"].cpu().numpy().T, X) <= TOL_X)
    with pytest.raises(kp.KzError):
        kp.kz_batch_update_items(b_b, H_b, 5, 3)
    with pytest.raises(kp.KzError):
        kp.kz_batch_update_items(b_b, H_b, 0, 0)


def test_batch_update_matches_fresh_plans(kp):
    """kz_batch_update with a new channel for every item gives bit-identical
    solutions to a batch prepared from plans built on that channel."""
    rng = np.random.default_rng(5)
    insts = [kzgen.make_instance(600 + i, int(rng.integers(4, 30)), int(rng.choice([97, 256, 640])),
                                 vr_frac_range=(0.1, 0.4), nrhs=6) for i in range(7)]
    new = [kzgen.make_instance(700 + i, inst.K, inst.Nt, vr_override=(inst.vr_offset, inst.vr_len), nrhs=6)
           for i, inst in enumerate(insts)]

    def items_for(src, plans):
        return [dict(plan=p, s=kp.rhs_tensor(i.S), x=torch.zeros((6, i.Nt), dtype=torch.complex64, device="cuda"),
                     v=torch.zeros((6, i.K), dtype=torch.complex64, device="cuda"),
                     iters=torch.zeros(6, dtype=torch.int32, device="cuda"),
                     resid=torch.zeros(6, dtype=torch.float64, device="cuda"), xi=i.xi) for i, p in zip(src, plans)]

    old_items = items_for(insts, [kp.plan_from_instance(i) for i in insts])
    b_old = kp.kz_batch_prepare(old_items, 6, "vr_oahk")
    H_cat = torch.from_numpy(np.concatenate([i.H_packed for i in new])).cuda()
    kp.kz_batch_update(b_old, H_cat)
    for it, i in zip(old_items, new):
        it["s"].copy_(kp.rhs_tensor(i.S))
    kp.kz_batch_rebind(b_old, [dict(it, xi=i.xi) for it, i in zip(old_items, new)])
    kp.kz_precode_batched(b_old, "paper", 1e-7, 3000, 0)
    fresh_items = items_for(new, [kp.plan_from_instance(i) for i in new])
    b_new = kp.kz_batch_prepare(fresh_items, 6, "vr_oahk")
    kp.kz_precode_batched(b_new, "paper", 1e-7, 3000, 0)
    torch.cuda.synchronize()
    for a, c, i in zip(old_items, fresh_items, new):
        assert torch.equal(a["x"], c["x"]) and torch.equal(a["iters"], c["iters"])
        V, X = orz.rzf(i.dense(), i.xi, i.S)
        assert np.all(orz.rel_err(a["x"].cpu().numpy().T, X) <= TOL_X)
