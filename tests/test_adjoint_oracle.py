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
