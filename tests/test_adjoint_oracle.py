"""Pins for the FP64 gradient references: autograd of the dense-solve sum-rate
loss against central finite differences, and PyTorch's complex convention."""
import numpy as np
import torch

import kzgen
from oracle import adjoint as oadj


def test_torch_complex_gradient_convention():
    """For real L(z), torch's z.grad g satisfies dL = Re(conj(g) dz): |z|^2 -> 2z."""
    z = torch.tensor(1.0 + 2.0j, dtype=torch.complex128, requires_grad=True)
    (z.abs() ** 2).backward()
    assert torch.allclose(z.grad, torch.tensor(2.0 + 4.0j, dtype=torch.complex128))


def test_reference_gradient_matches_central_differences():
    inst = kzgen.make_instance(3, 6, 48, vr_len_range=(10, 30), nrhs=6, rhs="identity", snr_db=10.0)
    L, gH, gxi = oadj.reference_gradient(inst)
    rng = np.random.default_rng(0)
    picks = rng.choice(inst.H_packed.size, size=6, replace=False)
    coords = [("xi",)] + [("re", int(p)) for p in picks] + [("im", int(p)) for p in picks]
    fd = oadj.central_difference(inst, coords, h=1e-5)
    want = np.array([gxi] + [gH[p].real for p in picks] + [gH[p].imag for p in picks])
    assert np.max(np.abs(fd - want)) <= 1e-6 * max(1.0, np.max(np.abs(want)))



def test_unrolled_steps_equal_the_literal_iteration():
    """The unrolled reference, fed the row sequence of the oracle's literal
    argmax GRK, ends where the literal iteration ends (two independent
    writings of eq. (update))."""
    from oracle import kaczmarz as okz
    inst = kzgen.make_instance(4, 7, 60, vr_len_range=(10, 35), nrhs=3, snr_db=10.0)
    sysm = okz.System.from_instance(inst)
    rows, want = [], []
    for j in range(3):
        tr = []
        m, q, t, c = okz.grk(sysm, inst.S[:, j], rule="argmax", tol=0.0, max_iter=12, trace=tr)
        rows.append([st["row"] for st in tr])
        want.append(m)
    rows_t = [[rows[j][t] for j in range(3)] for t in range(12)]
    X, V = oadj.unrolled(torch.tensor(inst.H_packed.astype(np.complex128)), torch.tensor(inst.xi, dtype=torch.float64),
                         torch.tensor(inst.S.astype(np.complex128)), rows_t, inst.vr_offset, inst.vr_len, inst.Nt)
    assert np.max(np.abs(X.numpy() - np.stack(want, 1))) <= 1e-12 * np.max(np.abs(X.numpy()))


def test_unrolled_gradient_matches_central_differences():
    inst = kzgen.make_instance(5, 5, 40, vr_len_range=(8, 25), nrhs=5, rhs="identity", snr_db=10.0)
    rng = np.random.default_rng(1)
    rows = [[int(rng.integers(0, 5)) for _ in range(5)] for _ in range(9)]
    S = torch.tensor(inst.S.astype(np.complex128))
    Hp = torch.tensor(inst.H_packed.astype(np.complex128), requires_grad=True)
    xi = torch.tensor(float(inst.xi), dtype=torch.float64, requires_grad=True)
    L = oadj.unrolled_loss(Hp, xi, S, rows, inst.vr_offset, inst.vr_len, inst.Nt, 10.0)
    L.backward()

    def f(h, x):
        with torch.no_grad():
            return float(oadj.unrolled_loss(h, torch.tensor(x, dtype=torch.float64), S, rows, inst.vr_offset,
                                             inst.vr_len, inst.Nt, 10.0))
    base = Hp.detach().clone()
    eps = 1e-6
    for p in (0, 7, 30):
        for unit in (1.0, 1j):
            dH = torch.zeros_like(base)
            dH[p] = eps * unit
            fd = (f(base + dH, inst.xi) - f(base - dH, inst.xi)) / (2 * eps)
            want = Hp.grad[p].real if unit == 1.0 else Hp.grad[p].imag
            assert abs(fd - float(want)) <= 1e-6 * max(1.0, abs(fd))
    fd = (f(base, inst.xi + eps) - f(base, inst.xi - eps)) / (2 * eps)
    assert abs(fd - float(xi.grad)) <= 1e-6 * max(1.0, abs(fd))
