"""The allocation-free adjoint against the allocating one (GB300).

kz_precode_adjoint_noalloc serves callers that cannot allocate device memory
when they differentiate (a real-time loop that must not block in the driver's
allocator, a process whose device memory is reserved up front by another
allocator, or a runtime that forbids allocation after start-up): its scratch
is a fixed device array inside the library.  Both entry points must give the
same lambda, y, grad_H and grad_xi, on two calls in a row (the shared array
keeps the previous call's contents, which must not leak into the next), after
a larger problem, with only G_Q given, and at exactly the array's size.
"""
import numpy as np
import pytest

import kzgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative tolerance of the GPU parity tests


@pytest.fixture(scope="module")
def kp():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_10689_gb300 import kzprecode
    return kzprecode


def _adjoint(kp, fn, plan, nrhs, xi, V, X, gV, gX):
    dev = V.device
    out = dict(lam=torch.empty_like(V), y=torch.empty_like(X),
               gH=torch.empty(plan.sum_len, dtype=torch.complex64, device=dev),
               gxi=torch.empty(1, dtype=torch.float32, device=dev),
               iters=torch.empty(nrhs, dtype=torch.int32, device=dev),
               resid=torch.empty(nrhs, dtype=torch.float64, device=dev),
               status=torch.zeros(1, dtype=torch.int32, device=dev))
    fn(plan, nrhs, xi, V, X, gV, gX, 1e-7, 2000, out["lam"], out["y"], out["gH"], out["gxi"], out["iters"],
       out["resid"], out["status"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _close(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return np.linalg.norm(a - b) <= TOL * max(np.linalg.norm(b), 1e-30)


def test_noalloc_adjoint_matches_allocating_adjoint(kp):
    rng = np.random.default_rng(11)
    for call, seed in enumerate((21, 22)):  # two calls in a row, different data
        inst = kzgen.make_instance(seed, 12, 300, vr_len_range=(40, 140), nrhs=6, snr_db=10.0)
        plan = kp.plan_from_instance(inst)
        S = kp.rhs_tensor(inst.S)
        fwd = kp.precode(plan, S, inst.xi, algo="vr_oahk", tol=1e-7, max_iter=2000)
        V, X = fwd["v"], fwd["x"]
        gV = torch.tensor((rng.normal(size=V.shape) + 1j * rng.normal(size=V.shape)).astype(np.complex64),
                          device="cuda")
        gX = torch.tensor((rng.normal(size=X.shape) + 1j * rng.normal(size=X.shape)).astype(np.complex64),
                          device="cuda")
        ref = _adjoint(kp, kp.kz_precode_adjoint, plan, 6, inst.xi, V, X, gV, gX)
        got = _adjoint(kp, kp.kz_precode_adjoint_noalloc, plan, 6, inst.xi, V, X, gV, gX)
        assert got["status"][0] == 0 and ref["status"][0] == 0
        for k in ("lam", "y", "gH", "gxi"):
            assert _close(got[k], ref[k]), (call, k)
        np.testing.assert_array_equal(got["iters"], ref["iters"])


def test_noalloc_adjoint_rejects_oversized_problem(kp):
    inst = kzgen.make_instance(5, 600, 1200, vr_len_range=(50, 80), nrhs=1)
    plan = kp.plan_from_instance(inst)
    nrhs = 437  # 600 * 437 > 262144
    V = torch.zeros((nrhs, 600), dtype=torch.complex64, device="cuda")
    X = torch.zeros((nrhs, 1200), dtype=torch.complex64, device="cuda")
    with pytest.raises(kp.KzError, match="exceeds the static scratch"):
        _adjoint(kp, kp.kz_precode_adjoint_noalloc, plan, nrhs, inst.xi, V, X, V, X)


def _random_like(rng, t):
    return torch.tensor((rng.normal(size=t.shape) + 1j * rng.normal(size=t.shape)).astype(np.complex64),
                        device="cuda")


def _compare(kp, inst, nrhs, rng, with_gx=True, tol=1e-7):
    plan = kp.plan_from_instance(inst)
    S = kp.rhs_tensor(inst.S)
    fwd = kp.precode(plan, S, inst.xi, algo="vr_oahk", tol=tol, max_iter=4000)
    V, X = fwd["v"], fwd["x"]
    gV = _random_like(rng, V)
    gX = _random_like(rng, X) if with_gx else None
    ref = _adjoint(kp, kp.kz_precode_adjoint, plan, nrhs, inst.xi, V, X, gV, gX)
    got = _adjoint(kp, kp.kz_precode_adjoint_noalloc, plan, nrhs, inst.xi, V, X, gV, gX)
    assert got["status"][0] == 0 and ref["status"][0] == 0
    for k in ("lam", "y", "gH", "gxi"):
        assert _close(got[k], ref[k]), k
    np.testing.assert_array_equal(got["iters"], ref["iters"])


def test_noalloc_adjoint_full_array_then_smaller_gq_only(kp):
    """A call at exactly the array's size (K * nrhs = 256 * 1024 = 262144),
    then calls with far fewer entries, the first with only G_Q (its right-hand
    side is copied into the array, not formed): the full call's entries beyond
    the later calls' K * nrhs must not reach them."""
    rng = np.random.default_rng(13)
    full = kzgen.make_instance(33, 256, 640, vr_len_range=(20, 60), nrhs=1024, snr_db=10.0)
    _compare(kp, full, 1024, rng, tol=1e-6)
    small = kzgen.make_instance(32, 9, 200, vr_len_range=(30, 90), nrhs=5, snr_db=10.0)
    _compare(kp, small, 5, rng, with_gx=False)
    _compare(kp, small, 5, rng, with_gx=True)
