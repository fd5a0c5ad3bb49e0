"""The tensor-core (FP16 products, correction form) AHK / VR-OAHK kernel against the FP64 oracle (GB300)."""
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


def run(kp, inst, algo, tol=1e-7, max_iter=3000, J=0, S=None, kernel="tc", refresh=0):
    plan = kp.plan_from_instance(inst)
    S = inst.S if S is None else S
    out = kp.precode(plan, kp.rhs_tensor(S), inst.xi, algo=algo, tol=tol, max_iter=max_iter, rhs_per_cta=J,
                     kernel=kernel, refresh=refresh)
    return {"x": out["x"].cpu().numpy().T.astype(np.complex128), "v": out["v"].cpu().numpy().T.astype(np.complex128),
            "iters": out["iters"].cpu().numpy(), "resid": out["resid"].cpu().numpy(), "converged": out["converged"]}


def ragged(seed=5, K=13, Nt=333, lo=17, hi=121, nrhs=11):
    return kzgen.make_instance(seed, K, Nt, vr_len_range=(lo, hi), snr_db=10.0, nrhs=nrhs)


@pytest.mark.parametrize("algo", ["ahk", "vr_oahk"])
@pytest.mark.parametrize("J,nrhs", [(4, 11), (8, 11), (8, 3), (4, 1)])
def test_tc_converges_to_rzf(kp, algo, J, nrhs):
    inst = ragged(nrhs=nrhs)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, algo, J=J)
    assert out["converged"]
    assert np.all(orz.rel_err(out["x"], X) <= TOL_X)
    assert np.all(orz.rel_err(out["v"], V) <= TOL_X)
    assert np.all(out["resid"] <= 1e-7 * (1 + 1e-6))


@pytest.mark.parametrize("algo", ["ahk", "vr_oahk"])
@pytest.mark.parametrize("T", [1, 2, 3])
def test_tc_first_iterates_follow_the_oracle(kp, algo, T):
    """Before any refresh the tensor-core iterates are the oracle's up to FP16
    rounding: a wrong fragment layout would miss by O(1)."""
    inst = ragged(seed=3, nrhs=9)
    ref = okz.solve(okz.System.from_instance(inst), inst.S, algo, tol=0.0, max_iter=T)
    for J in (4, 8):
        out = run(kp, inst, algo, tol=0.0, max_iter=T, J=J, refresh=1000)
        assert np.all(out["iters"] == T) and not out["converged"]
        assert np.all(orz.rel_err(out["x"], ref["x"]) <= 5e-3), (J, np.max(orz.rel_err(out["x"], ref["x"])))
        assert np.all(orz.rel_err(out["v"], ref["v"]) <= 5e-3)


def test_tc_matches_resident_kernel(kp):
    inst = kzgen.config2(10.0, nrhs=32)
    a = run(kp, inst, "vr_oahk", tol=1e-6, kernel="tc")
    b = run(kp, inst, "vr_oahk", tol=1e-6, kernel="resident")
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    assert np.max(orz.rel_err(a["x"], X)) <= TOL_X
    assert np.all(orz.rel_err(a["x"], b["x"]) <= 4e-6)
    # refreshes every 16 iterations: the count may move by a few
    assert np.mean(a["iters"]) <= 1.1 * np.mean(b["iters"]) + 2


@pytest.mark.parametrize("snr", [0.0, 20.0])
def test_tc_config2_full(kp, snr):
    inst = kzgen.config2(snr)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, "vr_oahk", tol=1e-6, max_iter=2000)
    assert out["converged"] and np.max(orz.rel_err(out["x"], X)) <= TOL_X


def test_tc_edge_cases(kp):
    inst = kzgen.make_instance(7, 1, 64, vr_len_range=(20, 20), nrhs=8)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    assert np.all(orz.rel_err(run(kp, inst, "vr_oahk")["x"], X) <= TOL_X)
    assert np.all(orz.rel_err(run(kp, inst, "ahk")["x"], X) <= TOL_X)
    off = [1 + 13 * k for k in range(6)]
    inst = kzgen.make_instance(8, 6, 80, vr_override=(off, [11] * 6), nrhs=8)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    out = run(kp, inst, "vr_oahk")
    assert np.all(out["iters"] == 1) and np.all(orz.rel_err(out["x"], X) <= 1e-6)
    inst = ragged(seed=10, nrhs=8)
    S = inst.S.copy()
    S[:, 2] = 0
    out = run(kp, inst, "vr_oahk", S=S)
    assert out["iters"][2] == 0 and np.all(out["x"][:, 2] == 0)
    # VRs that reach the last antenna and start at antenna 0, odd Nt
    off = [0, 300, 150, 0, 200]
    ln = [333, 33, 100, 7, 133]
    inst = kzgen.make_instance(9, 5, 333, vr_override=(off, ln), nrhs=5)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    assert np.all(orz.rel_err(run(kp, inst, "vr_oahk", J=4)["x"], X) <= TOL_X)


def test_tc_batched_and_graph(kp):
    rng = np.random.default_rng(5)
    insts = []
    for i in range(7):
        Nt = int(rng.choice([96, 257, 640]))
        insts.append(kzgen.make_instance(500 + i, int(rng.integers(3, 40)), Nt, vr_frac_range=(0.1, 0.4), nrhs=16))
    items = []
    for inst in insts:
        p = kp.plan_from_instance(inst)
        items.append(dict(plan=p, s=kp.rhs_tensor(inst.S),
                          x=torch.empty((16, inst.Nt), dtype=torch.complex64, device="cuda"),
                          v=None, iters=torch.empty(16, dtype=torch.int32, device="cuda"),
                          resid=torch.empty(16, dtype=torch.float64, device="cuda"), xi=inst.xi))
    b = kp.kz_batch_prepare(items, 16, "vr_oahk")
    for J, threads in ((4, 256), (4, 512), (8, 512)):
        kp.kz_batch_set_launch(b, "tc", J, threads)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            kp.kz_precode_batched(b, "paper", 1e-6, 50000, 0, status=st)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            kp.kz_precode_batched(b, "paper", 1e-6, 50000, 0, status=st)
        for it in items:
            it["x"].zero_()
        g.replay()
        torch.cuda.synchronize()
        assert st.item() == 0
        for inst, it in zip(insts, items):
            V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
            assert np.all(orz.rel_err(it["x"].cpu().numpy().T, X) <= TOL_X), (J, threads)


def test_tc_deterministic(kp):
    inst = ragged(seed=12, K=40, Nt=700, lo=60, hi=300, nrhs=8)
    a = run(kp, inst, "vr_oahk", tol=1e-6)
    b = run(kp, inst, "vr_oahk", tol=1e-6)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["iters"], b["iters"])


def test_tc_rejects_unsupported(kp):
    inst = ragged(nrhs=4)
    plan = kp.plan_from_instance(inst)
    S = kp.rhs_tensor(inst.S)
    with pytest.raises(kp.KzError):
        kp.precode(plan, S, inst.xi, algo="grk", kernel="tc")
    with pytest.raises(kp.KzError):
        kp.precode(plan, S, inst.xi, algo="vr_oahk", kernel="tc", rhs_per_cta=2)
    bplan = kp.plan_from_instance(inst, prec="bf16")
    with pytest.raises(kp.KzError):
        kp.precode(bplan, S, inst.xi, algo="vr_oahk", kernel="tc")


def test_tc_mixed_widths(kp):
    """J = 8 launch over a batch whose widest channel only fits 4 iterate
    columns: that channel's items are 4 columns wide, the others 8."""
    insts = [kzgen.make_instance(700, 200, 6144, vr_frac_range=(0.1, 0.4), nrhs=16),
             kzgen.make_instance(701, 30, 640, vr_frac_range=(0.1, 0.4), nrhs=16),
             kzgen.make_instance(702, 64, 2048, vr_frac_range=(0.1, 0.4), nrhs=16)]
    items = []
    for inst in insts:
        p = kp.plan_from_instance(inst)
        items.append(dict(plan=p, s=kp.rhs_tensor(inst.S),
                          x=torch.empty((16, inst.Nt), dtype=torch.complex64, device="cuda"),
                          v=torch.empty((16, inst.K), dtype=torch.complex64, device="cuda"),
                          iters=torch.empty(16, dtype=torch.int32, device="cuda"),
                          resid=torch.empty(16, dtype=torch.float64, device="cuda"), xi=inst.xi))
    b = kp.kz_batch_prepare(items, 16, "vr_oahk")
    kp.kz_batch_set_launch(b, "tc", 8, 512)
    assert kp.kz_batch_query(b) == {"kernel": "tc", "rhs_per_cta": 8, "threads": 512, "launches": 2}
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    kp.kz_precode_batched(b, "paper", 1e-6, 3000, 0, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    for inst, it in zip(insts, items):
        V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
        assert np.all(orz.rel_err(it["x"].cpu().numpy().T, X) <= TOL_X)
        assert np.all(orz.rel_err(it["v"].cpu().numpy().T, V) <= TOL_X)
        assert np.all(it["resid"].cpu().numpy() <= 1e-6 * (1 + 1e-6))


def test_tc_mixed_widths_graph_replay(kp):
    """The two launches of a mixed-width batch (forked onto an auxiliary
    stream and joined back) are captured into one CUDA graph."""
    insts = [kzgen.make_instance(710 + i, K, Nt, vr_frac_range=(0.1, 0.4), nrhs=16)
             for i, (K, Nt) in enumerate([(150, 6144), (40, 1024), (90, 2048), (60, 4096)])]
    items = []
    for inst in insts:
        p = kp.plan_from_instance(inst)
        items.append(dict(plan=p, s=kp.rhs_tensor(inst.S),
                          x=torch.empty((16, inst.Nt), dtype=torch.complex64, device="cuda"),
                          v=None, iters=torch.empty(16, dtype=torch.int32, device="cuda"),
                          resid=torch.empty(16, dtype=torch.float64, device="cuda"), xi=inst.xi))
    b = kp.kz_batch_prepare(items, 16, "vr_oahk")
    kp.kz_batch_set_launch(b, "tc", 8, 512)
    assert kp.kz_batch_query(b)["launches"] == 2
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        kp.kz_precode_batched(b, "paper", 1e-6, 3000, 0, status=st)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        kp.kz_precode_batched(b, "paper", 1e-6, 3000, 0, status=st)
    for it in items:
        it["x"].zero_()
    g.replay()
    torch.cuda.synchronize()
    assert st.item() == 0
    for inst, it in zip(insts, items):
        V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
        assert np.all(orz.rel_err(it["x"].cpu().numpy().T, X) <= TOL_X)


def _one_item_batch(kp, inst, J, threads, tol):
    p = kp.plan_from_instance(inst)
    n = inst.nrhs
    it = dict(plan=p, s=kp.rhs_tensor(inst.S), x=torch.empty((n, inst.Nt), dtype=torch.complex64, device="cuda"),
              v=torch.empty((n, inst.K), dtype=torch.complex64, device="cuda"),
              iters=torch.empty(n, dtype=torch.int32, device="cuda"),
              resid=torch.empty(n, dtype=torch.float64, device="cuda"), xi=inst.xi)
    b = kp.kz_batch_prepare([it], n, "vr_oahk")
    kp.kz_batch_set_launch(b, "tc", J, threads)
    assert kp.kz_batch_query(b) == {"kernel": "tc", "rhs_per_cta": J, "threads": threads, "launches": 1}
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    kp.kz_precode_batched(b, "paper", tol, 3000, 0, status=st)
    torch.cuda.synchronize()
    return st.item(), it, p


def _check_rzf(inst, it, tol):
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    assert np.all(orz.rel_err(it["x"].cpu().numpy().T, X) <= TOL_X)
    assert np.all(orz.rel_err(it["v"].cpu().numpy().T, V) <= TOL_X)
    assert np.all(it["resid"].cpu().numpy() <= tol * (1 + 1e-6))


@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("J", [4, 8])
def test_tc_long_orthogonal_rows(kp, J, threads):
    """Rows of the orthogonal set longer than two 256-entry steps: the F
    half-step is cut into chunks dealt to every warp (partial dots, then each
    chunk's step from its row's sum)."""
    inst = kzgen.make_instance(720, 48, 8192 if J == 4 else 4096, vr_len_range=(600, 1000), snr_db=10.0, nrhs=16)
    st, it, p = _one_item_batch(kp, inst, J, threads, 1e-7)
    F, _, _ = kp.kz_plan_query(p)
    assert max(int(inst.vr_len[f]) for f in F) > 512
    assert st == 0
    _check_rzf(inst, it, 1e-7)


@pytest.mark.parametrize("threads", [256, 512])
def test_tc_many_orthogonal_rows(kp, threads):
    """17 long rows in the orthogonal set: more than the 16 chunks a 256-thread
    CTA deals (that launch takes the F rows one per warp), fewer than the 32
    of a 512-thread CTA (chunked)."""
    inst = kzgen.make_instance(733, 96, 10240, vr_len_range=(514, 540), snr_db=10.0, nrhs=8)
    st, it, p = _one_item_batch(kp, inst, 4, threads, 1e-7)
    F, _, _ = kp.kz_plan_query(p)
    assert 16 < len(F) <= 32
    assert st == 0
    _check_rzf(inst, it, 1e-7)


@pytest.mark.parametrize("c", [1e-4, 1e4])
def test_tc_scale_range(kp, c):
    """H -> c H with xi -> c^2 xi scales x by 1 / c: the FP16 correction
    (stored divided by a per-column scale taken from the data) converges to
    the RZF solution across eight orders of magnitude of the solution."""
    import dataclasses
    base = kzgen.make_instance(740, 40, 2048, vr_frac_range=(0.1, 0.4), snr_db=10.0, nrhs=16)
    inst = dataclasses.replace(base, H_packed=(base.H_packed * np.float32(c)).astype(np.complex64),
                               xi=float(base.xi * c * c))
    for J in (4, 8):
        st, it, _ = _one_item_batch(kp, inst, J, 512, 1e-6)
        assert st == 0
        _check_rzf(inst, it, 1e-6)


@pytest.mark.parametrize("seed", range(3))
def test_tc_random_batch(kp, seed):
    """A random uneven batch (antennas 64-4600, users 2-256, VR fractions
    5-60%, 1-20 columns, SNR 0-20 dB) under the tensor-core launches and the
    tuner's choice: every column reaches the FP64 RZF at 1e-5."""
    rng = np.random.default_rng(5000 + seed)
    insts = []
    for i in range(10):
        Nt = int(rng.integers(64, 4600))
        K = int(rng.integers(2, min(256, Nt // 2)))
        insts.append(kzgen.make_instance(6000 + 10 * seed + i, K, Nt, vr_frac_range=(0.05, 0.6),
                                         snr_db=float(rng.uniform(0, 20)), nrhs=NR))
    for launch in (("tc", 8, 512), ("tc", 4, 256), None):
        items = []
        for inst in insts:
            p = kp.plan_from_instance(inst)
            items.append(dict(plan=p, s=kp.rhs_tensor(inst.S),
                              x=torch.empty((NR, inst.Nt), dtype=torch.complex64, device="cuda"),
                              v=torch.empty((NR, inst.K), dtype=torch.complex64, device="cuda"),
                              iters=torch.empty(NR, dtype=torch.int32, device="cuda"),
                              resid=torch.empty(NR, dtype=torch.float64, device="cuda"), xi=inst.xi))
        b = kp.kz_batch_prepare(items, NR, "vr_oahk")
        if launch:
            kp.kz_batch_set_launch(b, *launch)
        else:
            kp.kz_batch_tune(b, "paper", 1e-6, 3000, 0)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        kp.kz_precode_batched(b, "paper", 1e-6, 3000, 0, status=st)
        torch.cuda.synchronize()
        assert st.item() == 0, (launch, st.item())
        for inst, it in zip(insts, items):
            V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
            assert np.all(orz.rel_err(it["x"].cpu().numpy().T, X) <= TOL_X), (launch, inst.K, inst.Nt)


NR = 13  # columns per channel in the random batches (not a multiple of the launch widths)


def test_tc_row_scale_spread(kp):
    """Rows scaled by factors from 0.1 to 10 (near and far users, 40 dB of
    power between them): the FP16 copy scales each row by its own power of
    two, so every row keeps FP16's precision; the tensor-core kernel reaches
    the FP64 RZF in about the iterations of the FP32 kernel."""
    import dataclasses
    base = kzgen.make_instance(760, 40, 2048, vr_frac_range=(0.1, 0.4), snr_db=10.0, nrhs=16)
    rng = np.random.default_rng(761)
    c = 10.0 ** rng.uniform(-1.0, 1.0, size=base.K)
    c[0], c[1] = 0.1, 10.0
    rp = np.concatenate([[0], np.cumsum(base.vr_len.astype(np.int64))])
    H = base.H_packed.copy()
    for k in range(base.K):
        H[rp[k]:rp[k + 1]] *= np.float32(c[k])
    inst = dataclasses.replace(base, H_packed=H.astype(np.complex64))
    ref = run(kp, inst, "vr_oahk", tol=1e-6, kernel="resident")
    assert ref["converged"]
    for J in (4, 8):
        st, it, _ = _one_item_batch(kp, inst, J, 512, 1e-6)
        iters = it["iters"].cpu().numpy()
        assert st == 0, (J, st, iters.max(), ref["iters"].max())
        assert iters.max() <= 1.25 * ref["iters"].max() + 16, (J, iters.max(), ref["iters"].max())
        _check_rzf(inst, it, 1e-6)


def test_tc_after_plan_update_matches_fresh_plan(kp):
    """kz_plan_update rewrites the FP16 copy with the complex64 rows: the
    tensor-core kernel on the updated plan equals it on a fresh plan, bit for
    bit (a stale copy would change the inner iteration)."""
    a = kzgen.make_instance(770, 48, 1024, vr_frac_range=(0.1, 0.4), snr_db=10.0, nrhs=8)
    b = kzgen.make_instance(771, a.K, a.Nt, vr_override=(a.vr_offset, a.vr_len), nrhs=8, snr_db=10.0)
    plan = kp.plan_from_instance(a)
    kp.kz_plan_update(plan, torch.from_numpy(b.H_packed).cuda())
    fresh = kp.plan_from_instance(b)
    outs = []
    for p in (plan, fresh):
        o = kp.precode(p, kp.rhs_tensor(b.S), b.xi, algo="vr_oahk", tol=1e-7, max_iter=3000, rhs_per_cta=8,
                       kernel="tc")
        assert o["converged"]
        outs.append(o)
    assert torch.equal(outs[0]["x"], outs[1]["x"]) and torch.equal(outs[0]["iters"], outs[1]["iters"])
    V, X = orz.rzf(b.dense(), b.xi, b.S)
    assert np.all(orz.rel_err(outs[0]["x"].cpu().numpy().T.astype(np.complex128), X) <= TOL_X)


def test_tc_after_batch_update_matches_fresh_plans(kp):
    """kz_batch_update writes every item's FP16 copy with its norms: under the
    tensor-core launch the updated batch equals a batch of fresh plans, bit
    for bit."""
    rng = np.random.default_rng(780)
    insts = [kzgen.make_instance(781 + i, int(rng.integers(8, 80)), int(rng.choice([256, 640, 1500])),
                                 vr_frac_range=(0.1, 0.4), nrhs=8) for i in range(6)]
    new = [kzgen.make_instance(790 + i, inst.K, inst.Nt, vr_override=(inst.vr_offset, inst.vr_len), nrhs=8)
           for i, inst in enumerate(insts)]

    def items_for(src, plans):
        return [dict(plan=p, s=kp.rhs_tensor(i.S), x=torch.zeros((8, i.Nt), dtype=torch.complex64, device="cuda"),
                     v=torch.zeros((8, i.K), dtype=torch.complex64, device="cuda"),
                     iters=torch.zeros(8, dtype=torch.int32, device="cuda"),
                     resid=torch.zeros(8, dtype=torch.float64, device="cuda"), xi=i.xi) for i, p in zip(src, plans)]

    old_items = items_for(insts, [kp.plan_from_instance(i) for i in insts])
    b_old = kp.kz_batch_prepare(old_items, 8, "vr_oahk")
    kp.kz_batch_update(b_old, torch.from_numpy(np.concatenate([i.H_packed for i in new])).cuda())
    for it, i in zip(old_items, new):
        it["s"].copy_(kp.rhs_tensor(i.S))
    kp.kz_batch_rebind(b_old, [dict(it, xi=i.xi) for it, i in zip(old_items, new)])
    kp.kz_batch_set_launch(b_old, "tc", 8, 512)
    fresh_items = items_for(new, [kp.plan_from_instance(i) for i in new])
    b_new = kp.kz_batch_prepare(fresh_items, 8, "vr_oahk")
    kp.kz_batch_set_launch(b_new, "tc", 8, 512)
    for b in (b_old, b_new):
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        kp.kz_precode_batched(b, "paper", 1e-7, 3000, 0, status=st)
        torch.cuda.synchronize()
        assert st.item() == 0
    for a, c, i in zip(old_items, fresh_items, new):
        assert torch.equal(a["x"], c["x"]) and torch.equal(a["iters"], c["iters"])
        V, X = orz.rzf(i.dense(), i.xi, i.S)
        assert np.all(orz.rel_err(a["x"].cpu().numpy().T, X) <= TOL_X)
