"""Fixed-iteration row-action precoders with the selected-row history, and
their unrolled adjoint (GB300, through the C ABI).

* The recorded history of argmax GRK / VR-OGRK (deterministic rules) is the
  oracle's literal trace, and the fixed-T iterate is the oracle's.
* The unrolled adjoint's gradient of the sum-rate loss (eq. (rate)) of the
  T = 15 precoder equals torch autograd through the FP64 unrolled reference
  fed the same rows, at 1e-4, for a random selection rule too.
"""
import numpy as np
import pytest

import kzgen
from oracle import adjoint as oadj
from oracle import kaczmarz as okz
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


def record(kp, inst, algo, sel, T, seed=0):
    plan = kp.plan_from_instance(inst)
    nrhs = inst.nrhs
    x = torch.empty((nrhs, inst.Nt), dtype=torch.complex64, device="cuda")
    v = torch.empty((nrhs, inst.K), dtype=torch.complex64, device="cuda")
    iters = torch.empty(nrhs, dtype=torch.int32, device="cuda")
    resid = torch.empty(nrhs, dtype=torch.float64, device="cuda")
    hr = torch.empty((T, nrhs), dtype=torch.int32, device="cuda")
    hg = torch.empty((T, nrhs), dtype=torch.complex64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    kp.kz_precode_record(plan, kp.rhs_tensor(inst.S), nrhs, inst.xi, algo, sel, T, seed, x, v, iters, resid, hr, hg, st)
    torch.cuda.synchronize()
    return dict(x=x.cpu().numpy().T, v=v.cpu().numpy().T, iters=iters.cpu().numpy(), rows=hr.cpu().numpy(),
                gam=hg.cpu().numpy(), status=int(st.item()))


@pytest.mark.parametrize("algo", ["grk", "vr_ogrk"])
def test_record_is_the_oracle_trace(kp, algo):
    inst = kzgen.make_instance(12, 12, 160, vr_len_range=(20, 80), nrhs=4, snr_db=10.0)
    T = 15
    out = record(kp, inst, algo, "argmax", T)
    assert np.all(out["iters"] == T) and out["status"] & kp.KZ_STATUS_BIT_NOT_CONVERGED
    sysm = okz.System.from_instance(inst)
    for j in range(inst.nrhs):
        tr = []
        fn = okz.grk if algo == "grk" else okz.vr_ogrk
        m, q, t, c = fn(sysm, inst.S[:, j], rule="argmax", tol=0.0, max_iter=T, trace=tr)
        assert out["rows"][:, j].tolist() == [st["row"] for st in tr]
        assert orz.rel_err(out["x"][:, j:j + 1], m[:, None])[0] <= 1e-5


@pytest.mark.parametrize("algo,sel", [("vr_ogrk", "paper"), ("grk", "argmax"), ("rk_swor", "paper")])
def test_unrolled_gradient_vs_fp64_autograd(kp, algo, sel):
    from paper_2501_10689_gb300 import autograd as kad
    inst = kzgen.make_instance(9, 8, 120, vr_len_range=(20, 70), nrhs=8, rhs="identity", snr_db=10.0)
    T = 15
    snr = 10.0 ** (inst.snr_db / 10.0)
    Hp = torch.tensor(inst.H_packed, device="cuda", requires_grad=True)
    xi = torch.tensor(inst.xi, dtype=torch.float32, device="cuda", requires_grad=True)
    X, V = kad.precode_fixed(Hp, xi, kp.rhs_tensor(inst.S), inst.vr_offset, inst.vr_len, inst.Nt, algo=algo,
                             sel=sel, T=T, seed=3)
    L = kad.sum_rate_loss(kad.dense_from_packed(Hp, inst.vr_offset, inst.vr_len, inst.Nt), X, snr)
    L.backward()
    rows = record(kp, inst, algo, sel, T, seed=3)["rows"].tolist()
    Hr = torch.tensor(inst.H_packed.astype(np.complex128), requires_grad=True)
    xr = torch.tensor(float(inst.xi), dtype=torch.float64, requires_grad=True)
    Lr = oadj.unrolled_loss(Hr, xr, torch.tensor(inst.S.astype(np.complex128)), rows, inst.vr_offset, inst.vr_len,
                            inst.Nt, snr)
    Lr.backward()
    assert abs(float(L.detach()) - float(Lr.detach())) <= 1e-5 * abs(float(Lr.detach()))
    gH, gHr = Hp.grad.cpu().numpy(), Hr.grad.numpy()
    assert np.linalg.norm(gH - gHr) <= 1e-4 * np.linalg.norm(gHr), np.linalg.norm(gH - gHr) / np.linalg.norm(gHr)
    assert abs(float(xi.grad) - float(xr.grad)) <= 1e-4 * abs(float(xr.grad))


def test_unrolled_precoder_approaches_rzf_as_T_grows(kp):
    """The fixed-T precoder is not the RZF precoder, but its error decreases with T."""
    inst = kzgen.make_instance(10, 10, 200, vr_len_range=(30, 120), nrhs=10, rhs="identity", snr_db=10.0)
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    errs = [float(np.max(orz.rel_err(record(kp, inst, "vr_ogrk", "argmax", T)["x"], X))) for T in (5, 15, 60)]
    assert errs[0] > errs[1] > errs[2]
