"""Subarray-wise precoder assembly (eq. (precoding2)) on the GPU against the
FP64 oracle's subarray form, and against the solver's own x = H^H v (GB300,
through the C ABI)."""
import numpy as np
import pytest

import kzgen
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


@pytest.mark.parametrize("S", [1, 8, 20, 333])
def test_subarray_precoder_matches_oracle(kp, S):
    inst = kzgen.make_instance(21, 40, 1000, vr_len_range=(60, 300), nrhs=40, rhs="identity")
    V, X = orz.rzf(inst.dense(), inst.xi, np.eye(inst.K))
    ref = opc.subarray_precoder(inst.dense(), V, inst.vr_offset, inst.vr_len, S)
    plan = kp.plan_from_instance(inst)
    Vd = torch.from_numpy(np.ascontiguousarray(V.T.astype(np.complex64))).cuda()
    F = torch.empty((inst.K, inst.Nt), dtype=torch.complex64, device="cuda")
    kp.kz_precoder_matrix(plan, Vd, S, F)
    torch.cuda.synchronize()
    got = F.cpu().numpy().T
    assert np.max(orz.rel_err(got, ref)) <= 1e-5
    beta = torch.empty(1, dtype=torch.float32, device="cuda")
    kp.kz_precoder_matrix(plan, Vd, S, F, normalise=True, beta=beta)
    torch.cuda.synchronize()
    Fn, b = opc.normalise(ref)
    assert abs(beta.item() - b) <= 1e-5 * b
    assert np.linalg.norm(F.cpu().numpy().T - Fn) <= 1e-5


def test_subarray_precoder_equals_solver_x(kp):
    """v of an identity right-hand-side solve, assembled by subarrays, is the solve's x."""
    inst = kzgen.config5_instance(3)
    plan = kp.plan_from_instance(inst)
    out = kp.precode(plan, kp.rhs_tensor(inst.S), inst.xi, algo="vr_oahk", tol=1e-6, max_iter=3000)
    F = torch.empty_like(out["x"])
    kp.kz_precoder_matrix(plan, out["v"], 20, F)
    torch.cuda.synchronize()
    assert np.max(orz.rel_err(F.cpu().numpy().T, out["x"].cpu().numpy().T)) <= 2e-6
    V, X = orz.rzf(inst.dense(), inst.xi, inst.S)
    assert np.max(orz.rel_err(F.cpu().numpy().T, X)) <= 1e-5
