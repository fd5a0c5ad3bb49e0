"""Literal FP64 Kaczmarz-type precoders (RK, GRK, VR-OGRK, AHK, VR-OAHK).

All methods solve the consistent system B w = s with B = [H, sqrt(xi) I_K]
(eq. (SLE) with G^H = B), starting from w = 0, and keep w = [m; sqrt(xi) q]
(Remark 1).  Row i of B is [h_i, sqrt(xi) e_i^T] where h_i = H[i, :] is
non-zero only on user i's VR Gamma_i, so

    residual   r_i = s_i - h_i[Gamma_i] . m[Gamma_i] - xi q_i      (Alg. 1 step 8)
    row norm   d_i = ||h_i||^2 + xi                                 (Alg. 1 step 4)
    projection m[Gamma_i] += gamma conj(h_i[Gamma_i]),  q_i += gamma (Alg. 1 steps 9-11)

Each right-hand side is an independent system (Remark 2).  Stopping: the
paper tests an NMSE against the RZF answer; here every method stops on the
relative residual ||s - B w|| / ||s|| <= tol, checked where each method has
the full residual at hand:

* RK (Alg. 1):        full residual every K row steps;
* GRK (Sec. IV-A):    before every selection (all residuals are computed);
* VR-OGRK (Alg. 2):   before every selection, on the maintained residual
                      vector (rows outside X_{i(t-1)} keep their value, Thm. 2);
* AHK (eq. (update4)): before every step;
* VR-OAHK (Alg. 3):   after the orthogonal half-step, where r_F = 0 (Thm. 4)
                      and r_V is computed; the method then returns that
                      half-iterate.

``iters`` counts row projections (RK family) or iterations (AHK family; for
VR-OAHK an iteration stopped after its first half counts as one).

Selection rules for GRK / VR-OGRK: ``paper`` samples p_i = |r_i|^2/||r||^2
(Sec. IV-A and Alg. 2 step 4), ``baiwu`` restricts that sampling to the
greedy set U_t of Bai and Wu (cited in Sec. IV-A), ``argmax`` takes
argmax |r_i|^2 / d_i, lowest index on ties.  A draw picks the smallest i
whose running weight sum exceeds u * total (sums in FP64).
"""
import numpy as np

from . import rng as _rng
from . import sets as _sets

RULES = ("paper", "baiwu", "argmax")


class System:
    """Packed rows of one instance in FP64."""

    def __init__(self, H_packed, vr_offset, vr_len, Nt, xi):
        self.K = len(vr_len)
        self.Nt = int(Nt)
        self.xi = float(xi)
        self.off = [int(o) for o in vr_offset]
        self.len = [int(l) for l in vr_len]
        Hp = np.asarray(H_packed, dtype=np.complex128)
        self.rows = []
        p = 0
        for L in self.len:
            self.rows.append(Hp[p:p + L])
            p += L
        self.nrm = np.array([np.sum(np.abs(h) ** 2) for h in self.rows])
        self.d = self.nrm + self.xi

    @classmethod
    def from_instance(cls, inst, xi=None):
        return cls(inst.H_packed, inst.vr_offset, inst.vr_len, inst.Nt, inst.xi if xi is None else xi)

    def sl(self, i):
        return slice(self.off[i], self.off[i] + self.len[i])

    def residual_row(self, i, s, m, q):
        return s[i] - self.rows[i] @ m[self.sl(i)] - self.xi * q[i]

    def residual(self, s, m, q, rows=None):
        idx = range(self.K) if rows is None else rows
        r = np.zeros(self.K, dtype=np.complex128)
        for i in idx:
            r[i] = self.residual_row(i, s, m, q)
        return r

    def project_row(self, i, gamma, m, q):
        m[self.sl(i)] += gamma * self.rows[i].conj()
        q[i] += gamma

    def HHt(self, phi):
        """u = H^H phi (u_n = sum_i conj(h_in) phi_i)."""
        u = np.zeros(self.Nt, dtype=np.complex128)
        for i in range(self.K):
            if phi[i] != 0:
                u[self.sl(i)] += self.rows[i].conj() * phi[i]
        return u

    def H_times(self, m):
        return np.array([self.rows[i] @ m[self.sl(i)] for i in range(self.K)], dtype=np.complex128)


def pick(weights, u):
    """Smallest i with cumsum(weights)[i] > u * sum(weights)."""
    c = np.cumsum(np.asarray(weights, dtype=np.float64))
    target = u * c[-1]
    i = int(np.searchsorted(c, target, side="right"))
    if i >= len(c):  # u * total rounded up to total: take the last positive weight
        i = int(np.nonzero(np.asarray(weights) > 0)[0][-1])
    return i


def baiwu_set(r, d):
    """Greedy set U_t of Bai & Wu: eps = (max_i |r_i|^2/d_i / ||r||^2 + 1/||B||_F^2) / 2,
    U = {i : |r_i|^2 >= eps ||r||^2 d_i}, with ||B||_F^2 = sum_i d_i.

    Evaluated as ratio_i = |r_i|^2 / d_i >= (max_ratio + min(||r||^2/sum d, max_ratio)) / 2,
    the same set in exact arithmetic (the mean ratio never exceeds the maximum),
    written so that rounding can never drop the maximising row."""
    a2 = np.abs(r) ** 2
    ratio = a2 / d
    mx = np.max(ratio)
    avg = min(np.sum(a2) / np.sum(d), mx)
    return ratio >= 0.5 * (mx + avg)


def select(rule, r, d, u):
    a2 = np.abs(r) ** 2
    if rule == "argmax":
        ratio = a2 / d
        return int(np.argmax(ratio))  # argmax returns the lowest index on ties
    if rule == "paper":
        return pick(a2, u)
    if rule == "baiwu":
        return pick(np.where(baiwu_set(r, d), a2, 0.0), u)
    raise ValueError(rule)


def _trace_state(trace, **kw):
    if trace is not None:
        trace.append({k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in kw.items()})


def rk(sys, s, *, energy=True, swor=False, tol=1e-6, max_iter=10000, seed=0, instance=0, rhs=0, trace=None):
    """Alg. 1: rows drawn with p_i = d_i / sum(d) (energy) or 1/K (uniform).

    ``swor=True`` (the SWOR-ERK comparison method of Table I): energy weights,
    but within each sweep of K consecutive steps (t = cK .. cK + K - 1) a row
    is drawn at most once -- each draw takes p_i proportional to d_i over the
    rows not yet drawn in the sweep (sampling without replacement), so every
    sweep visits every row once."""
    s = np.asarray(s, dtype=np.complex128)
    m = np.zeros(sys.Nt, dtype=np.complex128)
    q = np.zeros(sys.K, dtype=np.complex128)
    w = sys.d if (energy or swor) else np.ones(sys.K)
    drawn = np.zeros(sys.K, dtype=bool)
    sn = np.linalg.norm(s)
    t = 0
    conv = False
    while True:
        if t % sys.K == 0:
            drawn[:] = False
            if np.linalg.norm(sys.residual(s, m, q)) <= tol * sn:
                conv = True
                break
        if t >= max_iter:
            break
        weights = np.where(drawn, 0.0, w) if swor else w
        i = pick(weights, _rng.uniform(seed, instance, rhs, t))
        drawn[i] = True
        r_i = sys.residual_row(i, s, m, q)
        gamma = r_i / sys.d[i]
        sys.project_row(i, gamma, m, q)
        t += 1
        _trace_state(trace, t=t, row=i, m=m, q=q)
    return m, q, t, conv


def grk(sys, s, *, rule="paper", tol=1e-6, max_iter=10000, seed=0, instance=0, rhs=0, trace=None):
    """Sec. IV-A: recompute every residual, draw a row by the greedy rule, project."""
    s = np.asarray(s, dtype=np.complex128)
    m = np.zeros(sys.Nt, dtype=np.complex128)
    q = np.zeros(sys.K, dtype=np.complex128)
    sn = np.linalg.norm(s)
    t = 0
    conv = False
    while True:
        r = sys.residual(s, m, q)
        if np.linalg.norm(r) <= tol * sn:
            conv = True
            break
        if t >= max_iter:
            break
        i = select(rule, r, sys.d, _rng.uniform(seed, instance, rhs, t))
        gamma = r[i] / sys.d[i]
        sys.project_row(i, gamma, m, q)
        t += 1
        _trace_state(trace, t=t, row=i, r=r, m=m, q=q)
    return m, q, t, conv


def vr_ogrk(sys, s, *, rule="paper", tol=1e-6, max_iter=10000, seed=0, instance=0, rhs=0,
            X=None, trace=None):
    """Alg. 2: residuals start at r = s and only rows in X_{i(t-1)} are recomputed."""
    s = np.asarray(s, dtype=np.complex128)
    if X is None:
        X = _sets.x_sets(sys.off, sys.len)
    m = np.zeros(sys.Nt, dtype=np.complex128)
    q = np.zeros(sys.K, dtype=np.complex128)
    r = s.copy()
    sn = np.linalg.norm(s)
    t = 0
    conv = False
    prev = None
    while True:
        if prev is not None:
            for j in X[prev]:
                r[j] = sys.residual_row(j, s, m, q)
        if np.linalg.norm(r) <= tol * sn:
            conv = True
            break
        if t >= max_iter:
            break
        i = select(rule, r, sys.d, _rng.uniform(seed, instance, rhs, t))
        gamma = r[i] / sys.d[i]
        sys.project_row(i, gamma, m, q)
        prev = i
        t += 1
        _trace_state(trace, t=t, row=i, r=r, m=m, q=q)
    return m, q, t, conv


def aggregate_step(sys, rows, r, m, q, unit=False):
    """AHK projection onto the aggregation hyperplane of ``rows`` (eq. (update4)
    with phi_i = r_i / d_i of eq. (coefficient), zero outside ``rows``).
    ``unit=True`` uses the unit step of Prop. 1 (valid for an orthogonal set).
    Returns gamma."""
    phi = np.zeros(sys.K, dtype=np.complex128)
    idx = list(rows)
    phi[idx] = r[idx] / sys.d[idx]
    u = sys.HHt(phi)
    if unit:
        gamma = 1.0
    else:
        num = np.vdot(phi, r).real  # phi^H r = sum |r_i|^2 / d_i
        den = np.vdot(u, u).real + sys.xi * np.vdot(phi, phi).real  # ||B^H phi||^2
        gamma = num / den if num != 0.0 else 0.0
    m += gamma * u
    q += gamma * phi
    return gamma


def ahk(sys, s, *, tol=1e-6, max_iter=1000, trace=None):
    """AHK on all rows: phi = D^-1 r, step length (phi^H r)/||B^H phi||^2."""
    s = np.asarray(s, dtype=np.complex128)
    m = np.zeros(sys.Nt, dtype=np.complex128)
    q = np.zeros(sys.K, dtype=np.complex128)
    sn = np.linalg.norm(s)
    t = 0
    conv = False
    while True:
        r = sys.residual(s, m, q)
        if np.linalg.norm(r) <= tol * sn:
            conv = True
            break
        if t >= max_iter:
            break
        g = aggregate_step(sys, range(sys.K), r, m, q)
        t += 1
        _trace_state(trace, t=t, gamma=g, r=r, m=m, q=q)
    return m, q, t, conv


def vr_oahk(sys, s, *, F=None, V=None, tol=1e-6, max_iter=1000, trace=None, f_unit=True):
    """Alg. 3: per iteration, a unit-step aggregate projection on the orthogonal
    set F (eq. (updateor), Prop. 1), then an AHK projection on V (eq. (updatenor))."""
    s = np.asarray(s, dtype=np.complex128)
    if F is None or V is None:
        F, V = _sets.split_fv(sys.off, sys.len)
    m = np.zeros(sys.Nt, dtype=np.complex128)
    q = np.zeros(sys.K, dtype=np.complex128)
    sn = np.linalg.norm(s)
    t = 0
    conv = False
    while t < max_iter:
        t += 1
        r = sys.residual(s, m, q, rows=F)
        w0 = (m.copy(), q.copy()) if trace is not None else None
        gF = aggregate_step(sys, F, r, m, q, unit=f_unit)
        w_half = (m.copy(), q.copy()) if trace is not None else None
        r = sys.residual(s, m, q, rows=V)
        if np.linalg.norm(r[V]) <= tol * sn:
            conv = True
            _trace_state(trace, t=t, w0=w0, w_half=w_half, w1=None, gF=gF, gV=None)
            break
        gV = aggregate_step(sys, V, r, m, q)
        _trace_state(trace, t=t, w0=w0, w_half=w_half, w1=(m.copy(), q.copy()), gF=gF, gV=gV)
    return m, q, t, conv


ALGOS = ("rk_energy", "rk_uniform", "grk", "ahk", "vr_ogrk", "vr_oahk", "rk_swor", "gk")


def solve(inst_or_sys, S, algo, *, rule="paper", tol=1e-6, max_iter=10000, seed=0, instance=0,
          xi=None):
    """Run ``algo`` on every column of S.  Returns dict(x, v, iters, conv, resid)."""
    sys = inst_or_sys if isinstance(inst_or_sys, System) else System.from_instance(inst_or_sys, xi)
    S = np.asarray(S, dtype=np.complex128)
    if S.ndim == 1:
        S = S[:, None]
    nrhs = S.shape[1]
    X = np.zeros((sys.Nt, nrhs), dtype=np.complex128)
    Vv = np.zeros((sys.K, nrhs), dtype=np.complex128)
    iters = np.zeros(nrhs, dtype=np.int64)
    conv = np.zeros(nrhs, dtype=bool)
    resid = np.zeros(nrhs)
    xsets = _sets.x_sets(sys.off, sys.len) if algo == "vr_ogrk" else None
    F, V = _sets.split_fv(sys.off, sys.len) if algo == "vr_oahk" else (None, None)
    for j in range(nrhs):
        s = S[:, j]
        if algo in ("rk_energy", "rk_uniform", "rk_swor"):
            m, q, t, c = rk(sys, s, energy=(algo != "rk_uniform"), swor=(algo == "rk_swor"), tol=tol,
                            max_iter=max_iter, seed=seed, instance=instance, rhs=j)
        elif algo in ("grk", "gk"):  # GK: the greedy (maximal-residual) rule
            m, q, t, c = grk(sys, s, rule="argmax" if algo == "gk" else rule, tol=tol, max_iter=max_iter,
                             seed=seed, instance=instance, rhs=j)
        elif algo == "vr_ogrk":
            m, q, t, c = vr_ogrk(sys, s, rule=rule, tol=tol, max_iter=max_iter, seed=seed,
                                 instance=instance, rhs=j, X=xsets)
        elif algo == "ahk":
            m, q, t, c = ahk(sys, s, tol=tol, max_iter=max_iter)
        elif algo == "vr_oahk":
            m, q, t, c = vr_oahk(sys, s, F=F, V=V, tol=tol, max_iter=max_iter)
        else:
            raise ValueError(algo)
        X[:, j] = m
        Vv[:, j] = q
        iters[j] = t
        conv[j] = c
        sn = np.linalg.norm(s)
        resid[j] = np.linalg.norm(sys.residual(s, m, q)) / sn if sn > 0 else 0.0
    return {"x": X, "v": Vv, "iters": iters, "conv": conv, "resid": resid}
