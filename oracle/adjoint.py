"""FP64 references for the sum-rate gradient (test infrastructure).

The paper has no gradient.  The loss is the negative sum rate of eq. (rate)
for the RZF precoder built from the auxiliary matrix V (Remark 2):

    V = (H H^H + xi I)^-1 S,   X = H^H V,   F = X / ||X||_F,
    SINR_k = |(H F)_kk|^2 / (sum_{i != k} |(H F)_ki|^2 + 1/snr),
    L = -sum_k log2(1 + SINR_k).

``loss_dense`` evaluates it in complex128 with plain PyTorch CPU ops (a
dense solve, no Kaczmarz), so torch.autograd gives the FP64 reference
gradient with respect to H (on the VR entries, packed) and xi.
``central_difference`` perturbs one real coordinate at a time.

``unrolled`` is the fixed-iteration precoder instead: T single-row Kaczmarz
steps (eq. (update); Alg. 1 steps 8-11) on a GIVEN row sequence, written
out in complex128 PyTorch ops, so torch.autograd differentiates through the
steps with the selection held fixed (the reference of the unrolled adjoint).
"""
import numpy as np
import torch


def dense_from_packed_t(Hp, vr_offset, vr_len, Nt):
    K = len(vr_len)
    rows = []
    p = 0
    for k in range(K):
        o, L = int(vr_offset[k]), int(vr_len[k])
        row = torch.zeros(Nt, dtype=Hp.dtype)
        row = torch.cat([row[:o], Hp[p:p + L], row[o + L:]])
        rows.append(row)
        p += L
    return torch.stack(rows)


def loss_from_VX(H, V, X, snr_lin):
    F = X / torch.linalg.norm(X)
    G = H @ F
    sig = torch.abs(torch.diagonal(G)) ** 2
    tot = torch.sum(torch.abs(G) ** 2, dim=1)
    sinr = sig / (tot - sig + 1.0 / snr_lin)
    return -torch.sum(torch.log2(1.0 + sinr))


def loss_dense(Hp, xi, vr_offset, vr_len, Nt, S, snr_lin):
    H = dense_from_packed_t(Hp, vr_offset, vr_len, Nt)
    A = H @ H.conj().T + xi * torch.eye(H.shape[0], dtype=H.dtype)
    V = torch.linalg.solve(A, S)
    X = H.conj().T @ V
    return loss_from_VX(H, V, X, snr_lin)


def reference_gradient(inst, snr_lin=None):
    """(loss, dL/dH_packed, dL/dxi) in complex128 / float64, PyTorch convention."""
    snr = 10.0 ** (inst.snr_db / 10.0) if snr_lin is None else snr_lin
    Hp = torch.tensor(inst.H_packed.astype(np.complex128), requires_grad=True)
    xi = torch.tensor(float(inst.xi), dtype=torch.float64, requires_grad=True)
    S = torch.tensor(inst.S.astype(np.complex128))
    L = loss_dense(Hp, xi, inst.vr_offset, inst.vr_len, inst.Nt, S, snr)
    L.backward()
    return float(L.item()), Hp.grad.numpy().copy(), float(xi.grad.item())


def central_difference(inst, coords, h=1e-4, snr_lin=None):
    """dL/d(coordinate) for coordinates ('xi',), ('re', p) or ('im', p) of H_packed."""
    snr = 10.0 ** (inst.snr_db / 10.0) if snr_lin is None else snr_lin
    S = torch.tensor(inst.S.astype(np.complex128))
    base = torch.tensor(inst.H_packed.astype(np.complex128))

    def f(Hp, xi):
        with torch.no_grad():
            return float(loss_dense(Hp, torch.tensor(xi, dtype=torch.float64), inst.vr_offset, inst.vr_len,
                                    inst.Nt, S, snr).item())

    out = []
    for c in coords:
        if c[0] == "xi":
            out.append((f(base, inst.xi + h) - f(base, inst.xi - h)) / (2 * h))
        else:
            d = torch.zeros_like(base)
            d[c[1]] = h if c[0] == "re" else 1j * h
            out.append((f(base + d, inst.xi) - f(base - d, inst.xi)) / (2 * h))
    return np.array(out)


def unrolled(Hp, xi, S, rows, vr_offset, vr_len, Nt):
    """(X, V) after the row steps rows[t][j] (-1: no step) of every column j
    of S (K x nrhs), from m = 0, q = 0: gamma = (s_i - h_i m - xi q_i) /
    (||h_i||^2 + xi), m += gamma conj(h_i), q_i += gamma."""
    H = dense_from_packed_t(Hp, vr_offset, vr_len, Nt)
    K = H.shape[0]
    d = torch.sum(torch.abs(H) ** 2, dim=1) + xi
    Xc, Vc = [], []
    for j in range(S.shape[1]):
        m = torch.zeros(Nt, dtype=H.dtype)
        q = torch.zeros(K, dtype=H.dtype)
        for t in range(len(rows)):
            i = int(rows[t][j])
            if i < 0:
                continue
            g = (S[i, j] - H[i] @ m - xi * q[i]) / d[i]
            m = m + g * H[i].conj()
            q = q + g * torch.nn.functional.one_hot(torch.tensor(i), K).to(H.dtype)
        Xc.append(m)
        Vc.append(q)
    return torch.stack(Xc, dim=1), torch.stack(Vc, dim=1)


def unrolled_loss(Hp, xi, S, rows, vr_offset, vr_len, Nt, snr_lin):
    X, V = unrolled(Hp, xi, S, rows, vr_offset, vr_len, Nt)
    return loss_from_VX(dense_from_packed_t(Hp, vr_offset, vr_len, Nt), V, X, snr_lin)
