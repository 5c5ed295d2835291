"""Momentum/spin block-sparse execution of the FT-CCSD oracle (test
infrastructure only; nothing in the product path imports it).

In the plane-wave electron gas (Sec. IV.B) and the k-space Hubbard ring
(Sec. IV.A) every spin orbital p carries its own conserved charge q_p (crystal
momentum and S_z; no two orbitals share one), and every factor of Eqs. E,
ccS1 and ccS2 conserves it: f_pq and s_i^a vanish unless q_p = q_q, <pq||rs>
and s_ij^ab unless q_p + q_q = q_r + q_s.  So a two-index factor is a vector
(its second index is fixed by its first) and a four-index factor is fixed by
three of its indices: N and N^3 numbers instead of N^2 and N^4.

This module evaluates the SAME term tables as ``ftccsd`` (S1_TERMS,
S2_TERMS, the three sums of Eq. E), the same propagation (``ftccsd.propagate``
applied to the stored elements) and the same fixed point, but each
multi-factor term is contracted pair by pair with the summation restricted
to index tuples whose charges balance.  For one pair contraction
    R[x, y] = sum_c A[x, c] B[c, y]
the charge of the contracted tuple c fixes the charges of x and y, so the sum
splits into independent blocks, one per charge value, each an ordinary matrix
product.  No term is rewritten and no new arithmetic enters; only terms that
are identically zero are skipped.  The result equals the dense oracle up to
rounding order (pinned on 19-, 27- and 33-plane-wave gases and the Hubbard
ring), and it reaches the 114- and 162-spin-orbital gases, where the dense
arrays (N^4 per tau point) do not fit a workstation.

Tensor storage (class ``ST``): letters (one per index), a sign per letter
(+1 for the first two slots of a four-index factor or the first slot of a
two-index one, -1 for the others, so that sum_k sign_k q_{p_k} = 0 on every
non-zero element), the values indexed by the first rank-1 letters (the last
index is determined by charge balance; a slot whose determined charge
belongs to no orbital holds zero) and, for amplitudes and kernels, a
trailing tau axis (the fixed-point arrays keep tau first, as in ``ftccsd``,
and are transposed at the kernel's entry and exit).

The systems must keep every orbital in both the hole-like and the
particle-like set (truncation threshold 0, or one that removes nothing).
"""
import math

import numpy as np
import torch

from . import ftccsd as fc
from . import systems

DT = torch.float64
HOLE = fc.HOLE


# ---------------------------------------------------------------- charges
class Charges:
    """Integer charge vectors q[p] (rows) of the N orbitals; mod[k] > 0 makes
    component k cyclic (crystal momentum of a ring), 0 leaves it in Z."""

    BASE = 1 << 12
    HALF = 1 << 11

    def __init__(self, q, mod):
        self.q = np.asarray(q, dtype=np.int64)
        self.mod = np.asarray(mod, dtype=np.int64)
        self.N, self.d = self.q.shape
        if self.d > 5:
            raise ValueError("at most 5 charge components")
        codes = self.code(self.q)
        if len(np.unique(codes)) != self.N:
            raise ValueError("two orbitals share a charge: the block-sparse oracle needs distinct charges")
        self._order = np.argsort(codes)
        self._sorted = codes[self._order]

    def canon(self, Q):
        Q = np.array(Q, dtype=np.int64, copy=True)
        for k in range(self.d):
            if self.mod[k] > 0:
                Q[..., k] %= self.mod[k]
        return Q

    def code(self, Q):
        Q = self.canon(Q)
        if np.any(np.abs(Q) >= self.HALF):
            raise ValueError("charge out of range")
        c = np.zeros(Q.shape[:-1], dtype=np.int64)
        for k in range(self.d):
            c = c * self.BASE + (Q[..., k] + self.HALF)
        return c

    def find(self, Q):
        """Orbital with charge Q (vectorised), -1 where there is none."""
        c = self.code(Q)
        pos = np.searchsorted(self._sorted, c)
        pos = np.minimum(pos, self.N - 1)
        hit = self._sorted[pos] == c
        return np.where(hit, self._order[pos], -1)

    def total(self, idx, signs):
        """sum_k signs[k] q[idx[:, k]] for index tuples idx (n, k)."""
        Q = np.zeros((idx.shape[0], self.d), dtype=np.int64)
        for k, s in enumerate(signs):
            Q += s * self.q[idx[:, k]]
        return Q


def _all_tuples(N, k):
    if k == 0:
        return np.zeros((1, 0), dtype=np.int64)
    g = np.meshgrid(*([np.arange(N, dtype=np.int64)] * k), indexing="ij")
    return np.stack(g, axis=-1).reshape(-1, k)


def _determined(ch, idx, signs):
    """Index of the last letter fixed by charge balance from the others."""
    Q = ch.total(idx, signs[:-1])
    return ch.find(-signs[-1] * Q)


def _nonzero_tuples(ch, signs):
    """All index tuples of a tensor with these letter signs on which charge balances."""
    r = len(signs)
    head = _all_tuples(ch.N, r - 1)
    last = _determined(ch, head, signs)
    ok = last >= 0
    return np.concatenate([head[ok], last[ok, None]], axis=1)


def _strides(N, r):
    """Element strides of the stored indices (the first r-1 letters)."""
    return [N ** (r - 2 - k) for k in range(r - 1)] + [0] if r > 0 else []


# ---------------------------------------------------------------- tensors
class ST:
    """A charge-conserving tensor (see the module docstring)."""

    def __init__(self, letters, signs, data, tau):
        self.letters = letters
        self.signs = tuple(int(s) for s in signs)
        self.data = data
        self.tau = tau

    @property
    def rank(self):
        return len(self.letters)


_PLANS = {}


def _plan_key(*parts):
    return tuple(parts)


def to_order(ch, T, order):
    """The same tensor stored in another letter order."""
    if T.letters == order:
        return T
    if sorted(T.letters) != sorted(order):
        raise ValueError(f"{T.letters} -> {order}")
    r = T.rank
    pos = [T.letters.index(c) for c in order]
    signs = tuple(T.signs[p] for p in pos)
    key = _plan_key("perm", T.letters, T.signs, order, ch.N)
    if key not in _PLANS:
        N = ch.N
        head = _all_tuples(N, r - 1)
        last = _determined(ch, head, signs)
        ok = last >= 0
        full = np.concatenate([head, np.where(ok, last, 0)[:, None]], axis=1)   # in target order
        src_stride = _strides(N, r)
        off = np.zeros(full.shape[0], dtype=np.int64)
        for k_t, p in enumerate(pos):          # target letter k_t sits at source position p
            off += src_stride[p] * full[:, k_t]
        _PLANS[key] = (torch.from_numpy(off), torch.from_numpy(ok))
    off, ok = _PLANS[key]
    flat = T.data.reshape((-1, T.data.shape[-1]) if T.tau else (-1,))
    out = flat.index_select(0, off)
    out = out * (ok[:, None] if T.tau else ok).to(flat.dtype)
    return ST(order, signs, out.reshape(T.data.shape), T.tau)


def normalise_signs(T):
    """Flip every sign if the first is negative (the same balance condition)."""
    if T.rank and T.signs[0] < 0:
        return ST(T.letters, tuple(-s for s in T.signs), T.data, T.tau)
    return T


def _group(codes):
    order = np.argsort(codes, kind="stable")
    sc = codes[order]
    uniq, start = np.unique(sc, return_index=True)
    end = np.append(start[1:], len(sc))
    return {int(u): order[s:e] for u, s, e in zip(uniq, start, end)}


def contract(ch, A, B):
    """R = sum over the shared letters of A * B, restricted to balanced blocks.

    Letters of R: A's unshared letters then B's, in their own orders.  The
    shared letters must carry the same relative sign in A and B, so that
    A's balance condition and B's combine into one for R.
    """
    Cl = [c for c in A.letters if c in B.letters]
    Xl = [c for c in A.letters if c not in Cl]
    Yl = [c for c in B.letters if c not in Cl]
    if not Cl:
        raise ValueError("outer products are not used")
    rel = {A.signs[A.letters.index(c)] * B.signs[B.letters.index(c)] for c in Cl}
    if len(rel) != 1:
        raise ValueError("shared letters with mixed relative signs")
    eps = -rel.pop()                              # A + eps * B cancels the shared letters
    rsig = tuple(A.signs[A.letters.index(c)] for c in Xl) + tuple(eps * B.signs[B.letters.index(c)] for c in Yl)
    rlet = "".join(Xl + Yl)
    if len(rlet) not in (0, 2, 4):
        raise ValueError(f"intermediate of rank {len(rlet)}")
    N = ch.N
    key = _plan_key("ctr", A.letters, A.signs, B.letters, B.signs, N)
    if key not in _PLANS:
        sA = [A.signs[A.letters.index(c)] for c in Xl]
        sC = [A.signs[A.letters.index(c)] for c in Cl]
        sB = [B.signs[B.letters.index(c)] for c in Yl]
        tx = _all_tuples(N, len(Xl))
        if len(Xl) == 0 and len(Yl) == 0:
            tc = _nonzero_tuples(ch, sC)
        else:
            tc = _all_tuples(N, len(Cl))
        ty = _all_tuples(N, len(Yl))
        gx = _group(ch.code(-ch.total(tx, sA)) if len(Xl) else np.full(1, int(ch.code(np.zeros((1, ch.d)))[0])))
        gc = _group(ch.code(ch.total(tc, sC)))
        gy = _group(ch.code(eps * ch.total(ty, sB)) if len(Yl) else np.full(1, int(ch.code(np.zeros((1, ch.d)))[0])))
        common = sorted(set(gx) & set(gc) & set(gy))

        def lin(tuples, letters, owner_letters, stride):
            off = np.zeros(tuples.shape[0], dtype=np.int64)
            for k, c in enumerate(letters):
                off += stride[owner_letters.index(c)] * tuples[:, k]
            return off

        stA, stB, stR = _strides(N, A.rank), _strides(N, B.rank), _strides(N, len(rlet))
        oAX, oAC = lin(tx, Xl, A.letters, stA), lin(tc, Cl, A.letters, stA)
        oBC, oBY = lin(tc, Cl, B.letters, stB), lin(ty, Yl, B.letters, stB)
        oRX, oRY = lin(tx, Xl, rlet, stR), lin(ty, Yl, rlet, stR)
        blocks, iA, iB, iR = [], [], [], []
        pa = pb = pr = 0
        for g in common:
            xs, cs, ys = gx[g], gc[g], gy[g]
            nx, nc, ny = len(xs), len(cs), len(ys)
            iA.append((oAX[xs][:, None] + oAC[cs][None, :]).ravel())
            iB.append((oBC[cs][:, None] + oBY[ys][None, :]).ravel())
            iR.append((oRX[xs][:, None] + oRY[ys][None, :]).ravel())
            blocks.append((pa, pb, pr, nx, nc, ny))
            pa += nx * nc
            pb += nc * ny
            pr += nx * ny
        cat = (lambda v: torch.from_numpy(np.concatenate(v)) if v else torch.zeros(0, dtype=torch.int64))
        _PLANS[key] = (blocks, cat(iA), cat(iB), cat(iR))
    blocks, iA, iB, iR = _PLANS[key]
    tau = A.tau or B.tau
    nt = A.data.shape[-1] if A.tau else (B.data.shape[-1] if B.tau else None)
    ga = A.data.reshape((-1, nt) if A.tau else (-1,)).index_select(0, iA)
    gb = B.data.reshape((-1, nt) if B.tau else (-1,)).index_select(0, iB)
    tail = (nt,) if tau else ()
    gr = torch.empty((iR.numel(),) + tail, dtype=DT)
    spec = ("xc" + ("t" if A.tau else "") + ",cy" + ("t" if B.tau else "") + "->xy" + ("t" if tau else ""))
    for pa, pb, pr, nx, nc, ny in blocks:
        a = ga[pa:pa + nx * nc].reshape((nx, nc) + ga.shape[1:])
        b = gb[pb:pb + nc * ny].reshape((nc, ny) + gb.shape[1:])
        gr[pr:pr + nx * ny] = torch.einsum(spec, a, b).reshape((nx * ny,) + tail)
    shape = (N,) * (len(rlet) - 1) + tail
    size = N ** (len(rlet) - 1) if len(rlet) else 1
    out = torch.zeros((size,) + tail, dtype=DT)
    if iR.numel():
        out[iR] = gr
    return ST(rlet, rsig, out.reshape(shape), tau)


def _cost(ch, A, B):
    shared = set(A.letters) & set(B.letters)
    if not shared:
        return None
    rank = len(set(A.letters) ^ set(B.letters))
    if rank not in (0, 2, 4):
        return None
    letters = len(set(A.letters) | set(B.letters))
    return (letters - 2, rank)


def einsum(ch, ops, out):
    """Contract a list of ST operands pair by pair down to the letters `out`
    (each letter appears in exactly two places, counting `out`)."""
    cur = list(ops)
    while len(cur) > 1:
        best = None
        for i in range(len(cur)):
            for j in range(i + 1, len(cur)):
                c = _cost(ch, cur[i], cur[j])
                if c is not None and (best is None or c < best[0]):
                    best = (c, i, j)
        if best is None:
            raise ValueError("no admissible pair contraction")
        _, i, j = best
        r = contract(ch, cur[i], cur[j])
        cur = [x for k, x in enumerate(cur) if k not in (i, j)] + [r]
    return normalise_signs(to_order(ch, cur[0], out))


# ---------------------------------------------------------------- systems
def ueg(n_elec, rs, n_pw):
    """Plane-wave gas of ``systems.ueg`` with its integrals stored by charge:
    eri[p, q, r] = <pq||rs> with s the orbital whose momentum and spin
    balance (zero where none), h and eps as vectors.  Same definitions:
    <pq|rs> = 4 pi / (Vc |k_p - k_r|^2) between equal spins, no q = 0 term;
    eps = zero-temperature HF energies of the closed shell."""
    nv = systems.plane_wave_grid(n_pw)
    M = len(nv)
    vol = 4.0 / 3.0 * math.pi * n_elec * rs ** 3
    Lc = vol ** (1.0 / 3.0)
    kin = 0.5 * np.sum((2.0 * math.pi * nv / Lc) ** 2, axis=1)
    spin = np.array([1] * M + [-1] * M)
    q = np.concatenate([np.concatenate([nv, nv]), spin[:, None]], axis=1)
    ch = Charges(q, [0, 0, 0, 0])
    N = 2 * M
    g = np.arange(N) % M

    def coul(p, r):
        d = nv[g[p]] - nv[g[r]]
        q2 = np.sum(d * d, axis=-1).astype(np.float64)
        out = np.zeros_like(q2)
        nz = q2 > 0
        out[nz] = 4.0 * math.pi / (vol * q2[nz] * (2.0 * math.pi / Lc) ** 2)
        return out

    t3 = _all_tuples(N, 3)
    s = _determined(ch, t3, (1, 1, -1, -1))
    ok = s >= 0
    p, qq, r, ss = t3[ok, 0], t3[ok, 1], t3[ok, 2], s[ok]
    direct = np.where(spin[p] == spin[r], coul(p, r), 0.0)      # <pq|rs>
    exch = np.where(spin[p] == spin[ss], coul(p, ss), 0.0)      # <pq|sr>
    eri = np.zeros(N ** 3)
    eri[(p * N + qq) * N + r] = direct - exch
    nocc = n_elec // 2
    eps_sp = kin.copy()
    for a in range(M):
        eps_sp[a] -= sum(coul(np.array([a]), np.array([b]))[0] for b in range(nocc))
    return {"charges": ch, "h": torch.tensor(np.concatenate([kin, kin])), "eps": torch.tensor(
        np.concatenate([eps_sp, eps_sp])), "eri": torch.from_numpy(eri.reshape(N, N, N)), "kind": "ueg"}


def hubbard_1d(L, t, U):
    """k-space Hubbard ring of ``systems.hubbard_1d`` stored by charge
    (crystal momentum m mod L and S_z)."""
    m = np.arange(L)
    hk = -2.0 * t * np.cos(2.0 * np.pi * m / L)
    M, N = L, 2 * L
    spin = np.array([1] * M + [-1] * M)
    q = np.stack([np.concatenate([m, m]), spin], axis=1)
    ch = Charges(q, [L, 0])
    t3 = _all_tuples(N, 3)
    s = _determined(ch, t3, (1, 1, -1, -1))
    ok = s >= 0
    p, qq, r, ss = t3[ok, 0], t3[ok, 1], t3[ok, 2], s[ok]
    direct = np.where(spin[p] == spin[r], U / L, 0.0)
    exch = np.where(spin[p] == spin[ss], U / L, 0.0)
    eri = np.zeros(N ** 3)
    eri[(p * N + qq) * N + r] = direct - exch
    return {"charges": ch, "h": torch.tensor(np.concatenate([hk, hk])),
            "eps": torch.tensor(np.concatenate([hk, hk]) + U / 2.0), "eri": torch.from_numpy(eri.reshape(N, N, N)),
            "kind": "hubbard"}


def expand(sysc):
    """Dense h, <pq||rs>, eps of a charge-stored system (for the pins)."""
    ch = sysc["charges"]
    N = ch.N
    t4 = _nonzero_tuples(ch, (1, 1, -1, -1))
    eri = torch.zeros((N, N, N, N), dtype=DT)
    src = sysc["eri"].reshape(-1)[torch.from_numpy((t4[:, 0] * N + t4[:, 1]) * N + t4[:, 2])]
    eri[t4[:, 0], t4[:, 1], t4[:, 2], t4[:, 3]] = src
    return {"h": torch.diag(sysc["h"]), "eri": eri, "eps": sysc["eps"].clone()}


# ---------------------------------------------------------------- problem
class Problem:
    """Thermal integrals and grid of ``ftccsd.Problem`` for a charge-stored
    system (reference, Fock matrix, Omega0, Omega1, slot factors, Simpson
    tensors, Delta), with every orbital hole-like and particle-like."""

    def __init__(self, sysc, beta, mu, ngrid, thr=0.0):
        self.ch = ch = sysc["charges"]
        N = ch.N
        self.hd = sysc["h"]
        self.eri = sysc["eri"]
        self.eps = sysc["eps"]
        self.beta = torch.as_tensor(beta, dtype=DT)
        self.mu = torch.as_tensor(mu, dtype=DT)
        self.ngrid = ngrid
        self.n, self.nbar = fc.occupations(self.eps, self.beta, self.mu)
        if bool(torch.any(self.n < thr)) or bool(torch.any(self.nbar < thr)):
            raise ValueError("the threshold would truncate an orbital; the block-sparse oracle keeps all")
        ar = np.arange(N)
        # f_pq = h_pq + sum_r n_r <pr||qr> (App. A): diagonal here; <pr||pr> sits at eri[p, r, p]
        self.vdiag = self.eri[torch.from_numpy(ar)[:, None], torch.from_numpy(ar)[None, :],
                              torch.from_numpy(ar)[:, None]]
        self.f = self.hd + self.vdiag @ self.n
        self.omega0 = fc.omega0(self.eps, self.beta, self.mu)
        self.omega1 = torch.sum(self.n * (self.hd - self.eps)) + 0.5 * self.n @ self.vdiag @ self.n
        self.fh = torch.sqrt(self.n)
        self.fp = torch.sqrt(self.nbar)
        self.Fbar = self.f - self.eps                                    # reading R3
        self.tau, self.G, self.g = fc.simpson_G(ngrid, self.beta)
        self.D1 = torch.zeros(N, dtype=DT)                               # Delta_i^a, a = i
        t3 = _all_tuples(N, 3)
        b = _determined(ch, t3, (1, 1, -1, -1))
        ok = torch.from_numpy(b >= 0)
        bb = torch.from_numpy(np.where(b >= 0, b, 0))
        e = self.eps
        d2 = e[torch.from_numpy(t3[:, 2])] + e[bb] - e[torch.from_numpy(t3[:, 0])] - e[torch.from_numpy(t3[:, 1])]
        self.D2 = (d2 * ok).reshape(N, N, N)
        self.mask2 = ok.to(DT).reshape(N, N, N)
        self._vcache = {}

    def _fac(self, letter):
        return self.fh if letter in HOLE else self.fp

    def F(self, letters):
        """Thermal Fock block as a vector over its first index (second = first)."""
        f0, f1 = (self._fac(c) for c in letters)
        return ST(letters, (1, -1), self.Fbar * f0 * f1, False)

    def V(self, letters):
        """Thermal <pq||rs> block with the slot factors of its letters' classes."""
        cls = "".join("o" if c in HOLE else "v" for c in letters)
        if cls not in self._vcache:
            ch, N = self.ch, self.ch.N
            t3 = _all_tuples(N, 3)
            s = _determined(ch, t3, (1, 1, -1, -1))
            s = torch.from_numpy(np.where(s >= 0, s, 0))
            f = [self._fac(c) for c in letters]
            w = (f[0][torch.from_numpy(t3[:, 0])] * f[1][torch.from_numpy(t3[:, 1])]
                 * f[2][torch.from_numpy(t3[:, 2])] * f[3][s])
            self._vcache[cls] = (self.eri.reshape(-1) * w).reshape(N, N, N)
        return ST(letters, (1, 1, -1, -1), self._vcache[cls], False)


def _antisym(ch, R, perm, out):
    """P(pq) X = X - X(p <-> q) on the output letters."""
    pairs = []
    if perm in ("ij", "ijab"):
        pairs.append(("i", "j"))
    if perm in ("ab", "ijab"):
        pairs.append(("a", "b"))
    for p, q in pairs:
        swapped = R.letters.translate(str.maketrans({p: q, q: p}))
        Y = normalise_signs(to_order(ch, ST(swapped, R.signs, R.data, R.tau), out))
        R = ST(out, R.signs, R.data - Y.data, R.tau)
    return R


def _eval_terms(prob, terms, out, t1, t2):
    """Sum of the terms at every tau point; t1 [x, i], t2 [x, i, j, a] in,
    the kernel [x, ...] out (tau moved last inside)."""
    ch = prob.ch
    nx = t1.shape[0]
    t1 = t1.movedim(0, -1).contiguous()
    t2 = t2.movedim(0, -1).contiguous()
    total = None
    for coef, perm, factors in terms:
        ops = []
        for fct in factors:
            kind, letters = fct.split(":")
            if kind == "F":
                ops.append(prob.F(letters))
            elif kind == "V":
                ops.append(prob.V(letters))
            elif kind == "T1":
                ops.append(ST(letters, (1, -1), t1, True))
            else:
                ops.append(ST(letters, (1, 1, -1, -1), t2, True))
        R = einsum(ch, ops, out)
        R = _antisym(ch, R, perm, out)
        d = coef * R.data
        if not R.tau:
            d = d.unsqueeze(-1).expand(tuple(d.shape) + (nx,))
        total = d if total is None else total + d
    return total.movedim(-1, 0).contiguous()


def S1(prob, t1, t2):
    """Singles kernel of Eq. ccS1 at every tau point: [x, i] (a = i)."""
    return _eval_terms(prob, fc.S1_TERMS, "ia", t1, t2)


def S2(prob, t1, t2):
    """Doubles kernel of Eq. ccS2 at every tau point: [x, i, j, a] (b fixed by charge)."""
    return _eval_terms(prob, fc.S2_TERMS, "ijab", t1, t2) * prob.mask2


def energy(prob, t1, t2):
    """E(tau_x) of Eq. E: the same three sums as ``ftccsd.energy``."""
    ch = prob.ch
    t1 = t1.movedim(0, -1).contiguous()
    t2 = t2.movedim(0, -1).contiguous()
    e1 = einsum(ch, [prob.F("ia"), ST("ia", (1, -1), t1, True)], "").data
    e2 = 0.25 * einsum(ch, [prob.V("ijab"), ST("ijab", (1, 1, -1, -1), t2, True)], "").data
    e3 = 0.5 * einsum(ch, [prob.V("ijab"), ST("ia", (1, -1), t1, True), ST("jb", (1, -1), t1, True)], "").data
    return e1 + e2 + e3


def omega_cc(prob, t1, t2):
    return torch.sum(prob.g * energy(prob, t1, t2)) / prob.beta


def fixed_point_map(prob, t1, t2):
    return (fc.propagate(prob, S1(prob, t1, t2), prob.D1),
            fc.propagate(prob, S2(prob, t1, t2), prob.D2))


def solve(prob, tol=1e-12, tol_amp=1e-10, max_iter=400, damping=1.0, verbose=False, t1=None, t2=None):
    """The fixed point of ``ftccsd.solve`` (same start, update and stopping rule)."""
    N, ng = prob.ch.N, prob.ngrid
    if t1 is None:
        t1 = torch.zeros((ng, N), dtype=DT)
        t2 = torch.zeros((ng, N, N, N), dtype=DT)
    occ_old = omega_cc(prob, t1, t2).item()
    converged = False
    it = 0
    history = []
    with torch.no_grad():
        for it in range(1, max_iter + 1):
            n1, n2 = fixed_point_map(prob, t1, t2)
            if damping != 1.0:
                n1 = (1.0 - damping) * t1 + damping * n1
                n2 = (1.0 - damping) * t2 + damping * n2
            dmax = max(torch.max(torch.abs(n1 - t1)).item(), torch.max(torch.abs(n2 - t2)).item())
            smax = max(torch.max(torch.abs(n1)).item(), torch.max(torch.abs(n2)).item())
            dmax = dmax / max(1.0, smax)
            t1, t2 = n1, n2
            occ = omega_cc(prob, t1, t2).item()
            history.append(occ)
            if verbose:
                print(it, repr(occ), occ - occ_old, dmax, flush=True)
            if abs(occ - occ_old) < tol and dmax < tol_amp:
                converged = True
                occ_old = occ
                break
            if not np.isfinite(occ):
                break
            occ_old = occ
    om0 = prob.omega0.item()
    om1 = prob.omega1.item()
    return {"omega": om0 + om1 + occ_old, "omega0": om0, "omega1": om1, "omega_cc": occ_old,
            "t1": t1, "t2": t2, "iterations": it, "converged": converged, "history": history}


def dense_amplitudes(ch, t1, t2):
    """Dense s1 [x, i, a], s2 [x, i, j, a, b] of charge-stored amplitudes."""
    N = ch.N
    nx = t1.shape[0]
    d1 = torch.zeros((nx, N, N), dtype=DT)
    d1[:, torch.arange(N), torch.arange(N)] = t1
    t4 = _nonzero_tuples(ch, (1, 1, -1, -1))
    d2 = torch.zeros((nx, N, N, N, N), dtype=DT)
    src = t2.reshape(nx, -1)[:, torch.from_numpy((t4[:, 0] * N + t4[:, 1]) * N + t4[:, 2])]
    d2[:, t4[:, 0], t4[:, 1], t4[:, 2], t4[:, 3]] = src
    return d1, d2


def random_amplitudes(ch, seed, ngrid, scale=0.1):
    """Random charge-conserving s1 and s2 (s2 antisymmetric in i,j and a,b), stored by charge."""
    N = ch.N
    rng = np.random.default_rng(seed)
    t1 = torch.tensor(scale * rng.standard_normal((ngrid, N)))
    mask = torch.from_numpy(_determined(ch, _all_tuples(N, 3), (1, 1, -1, -1)) >= 0).to(DT).reshape(N, N, N)
    raw = ST("ijab", (1, 1, -1, -1), torch.tensor(scale * rng.standard_normal((N, N, N, ngrid))) * mask[..., None],
             True)
    a = _antisym(ch, raw, "ijab", "ijab")
    return t1, 0.25 * (a.data * mask[..., None]).movedim(-1, 0).contiguous()
