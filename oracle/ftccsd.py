"""Finite-temperature CCSD, plain FP64 CPU oracle (test infrastructure only).

Follows White & Chan, "Finite-temperature coupled cluster: efficient
implementation and application to prototypical systems" (arXiv:2004.01729):

* reference: Fermi-Dirac occupations and the finite-temperature Fock matrix
  (Sec. II.A, App. A), the zeroth- and first-order grand potentials;
* thermal integrals: every hole-like slot carries sqrt(n), every
  particle-like slot sqrt(1-n) (Sec. II.A, App. A);
* quadrature tensors g and G (Sec. II.C, Eqs. g and G);
* kernels E, S1, S2 evaluated term by term as printed (Eqs. E, ccS1, ccS2);
* the integral-form amplitude equations, Eq. smu discretised as in App. A,
  solved as one fixed point over the whole tau grid (Alg. 2 run to
  self-consistency; both reach the same discrete solution);
* Omega_CC = beta^-1 sum_y g_y E(tau_y) (Eq. Ecc, App. A);
* the lambda equations as stationarity of the Lagrangian (Eqs. Lagrangian,
  lmu, ltilde), and property derivatives as partial derivatives of the
  Lagrangian (Sec. II.D, App. B), both by reverse-mode differentiation of the
  functions below.

Readings of passages that are silent or garbled (each also listed in the
design notes of the repository):
  R1  Simpson tensors for an even number of points: G^0 = 0, G^1 = the
      quadratic through tau_0..tau_2 integrated over [0, tau_1]
      (h/12 * (5, 8, -1)), even y composite Simpson 1/3, odd y >= 3 Simpson
      1/3 on [0, tau_{y-3}] plus Simpson 3/8 on [tau_{y-3}, tau_y]; g = G^{ng-1}.
  R3  the diagonal orbital energy is subtracted in all four thermal Fock
      blocks (f_ij, f_ia, f_ai, f_ab), so that the perturbation is H - sum eps.
  R4  Omega0 = -beta^-1 sum_p ln(1 + exp(-beta(eps_p - mu))),
      Omega1 = sum_p n_p (h_pp - eps_p) + 1/2 sum_pq n_p n_q <pq||pq>; the
      derivative of Omega1 with respect to n_q is f_qq - eps_q (App. B).
  R7  truncation keeps an orbital as hole-like if n >= thr, particle-like if
      1 - n >= thr.
  R8  the last term of Eq. ccS1 sums over j, k, b, c.
  R14 the unrelaxed 2-RDM Gamma_N is the Lagrangian's derivative with
      respect to the integrals of the CC equations and energy at a fixed
      reference (the printed blocks of App. B are garbled in places).
"""
import numpy as np
import torch

DT = torch.float64
HOLE = "ijklmn"
PART = "abcdefgh"


# ---------------------------------------------------------------- helpers
def contract(spec, *ops):
    """einsum over float64 tensors; with more than two operands the pairwise
    order comes from numpy's path search (it only changes rounding order)."""
    if len(ops) <= 2:
        return torch.einsum(spec, *ops)
    lhs, out = spec.split("->")
    subs = lhs.split(",")
    dummies = [np.broadcast_to(np.zeros(()), tuple(o.shape)) for o in ops]
    path = np.einsum_path(spec, *dummies, optimize="greedy")[0][1:]
    cur = list(zip(subs, ops))
    for pair in path:
        taken = [cur[p] for p in pair]
        for p in sorted(pair, reverse=True):
            cur.pop(p)
        rest = "".join(s for s, _ in cur) + out
        keep = "".join(c for c in dict.fromkeys("".join(s for s, _ in taken)) if c in rest)
        res = torch.einsum(",".join(s for s, _ in taken) + "->" + keep, *[o for _, o in taken])
        cur.append((keep, res))
    (s, o), = cur
    return torch.einsum(s + "->" + out, o)


def _swap(x, p, q):
    return x.transpose(p, q)


# ---------------------------------------------------------------- reference
def occupations(eps, beta, mu):
    """Fermi-Dirac n_p and 1 - n_p, both in overflow-free form."""
    z = beta * (eps - mu)
    return torch.sigmoid(-z), torch.sigmoid(z)


def omega0(eps, beta, mu):
    """Grand potential of the non-interacting reference (reading R4)."""
    return -torch.sum(torch.logaddexp(torch.zeros_like(eps), -beta * (eps - mu))) / beta


def fock(h, eri, n):
    """f_pq = h_pq + sum_r n_r <pr||qr>: Fock operator of the thermal mean-field density (App. A)."""
    return h + torch.einsum("prqr,r->pq", eri, n)


def omega1(h, eri, eps, n):
    """First-order grand potential (reading R4)."""
    return torch.sum(n * (torch.diagonal(h) - eps)) + 0.5 * torch.einsum(
        "pqpq,p,q->", eri, n, n)


def simpson_G(ngrid, beta):
    """Grid tau_y = y h, h = beta/(ngrid-1), and quadrature tensors (R1).

    Returns tau (ng,), G (ng, ng) with s(tau_y) ~ sum_x G[y, x] I(tau_x), and
    g = G[ng-1] (Sec. II.C, Eqs. g and G).  All entries scale linearly with
    beta, so derivatives with respect to beta flow through.
    """
    ng = ngrid
    if ng < 3:
        raise ValueError("ngrid must be >= 3")
    Gh = np.zeros((ng, ng))
    Gh[1, 0:3] = np.array([5.0, 8.0, -1.0]) / 12.0

    def simpson13(row, lo, hi):       # composite 1/3 on [lo, hi], hi - lo even
        for a in range(lo, hi, 2):
            row[a] += 1.0 / 3.0
            row[a + 1] += 4.0 / 3.0
            row[a + 2] += 1.0 / 3.0

    for y in range(2, ng):
        if y % 2 == 0:
            simpson13(Gh[y], 0, y)
        else:
            simpson13(Gh[y], 0, y - 3)
            Gh[y, y - 3:y + 1] += np.array([3.0, 9.0, 9.0, 3.0]) / 8.0
    hstep = beta / (ng - 1)
    tau = hstep * torch.arange(ng, dtype=DT)
    G = hstep * torch.tensor(Gh, dtype=DT)
    return tau, G, G[ng - 1]


# ---------------------------------------------------------------- the problem
class Problem:
    """Thermal integrals and grid for one (system, beta, mu, ngrid)."""

    def __init__(self, system, beta, mu, ngrid, thr=0.0):
        self.h = system["h"]
        self.eri = system["eri"]
        self.eps = system["eps"]
        self.beta = torch.as_tensor(beta, dtype=DT)
        self.mu = torch.as_tensor(mu, dtype=DT)
        self.ngrid = ngrid
        self.n, self.nbar = occupations(self.eps, self.beta, self.mu)
        self.f = fock(self.h, self.eri, self.n)
        self.omega0 = omega0(self.eps, self.beta, self.mu)
        self.omega1 = omega1(self.h, self.eri, self.eps, self.n)
        nd = self.n.detach()
        nbd = self.nbar.detach()
        self.iO = torch.nonzero(nd >= thr).flatten()
        self.iV = torch.nonzero(nbd >= thr).flatten()
        self.fh = torch.sqrt(self.n[self.iO])
        self.fp = torch.sqrt(self.nbar[self.iV])
        self.Fbar = self.f - torch.diag(self.eps)                 # reading R3
        self.tau, self.G, self.g = simpson_G(ngrid, self.beta)
        eo = self.eps[self.iO]
        ev = self.eps[self.iV]
        self.D1 = ev[None, :] - eo[:, None]                        # Delta_i^a
        self.D2 = (ev[None, None, :, None] + ev[None, None, None, :]
                   - eo[:, None, None, None] - eo[None, :, None, None])
        self._vcache = {}

    # -- index classes ----------------------------------------------------
    def _axis(self, letter, sel):
        if letter in HOLE:
            idx, fac = self.iO, self.fh
        else:
            idx, fac = self.iV, self.fp
        if sel is not None and letter in sel:
            idx, fac = idx[sel[letter]], fac[sel[letter]]
        return idx, fac

    def F(self, letters, sel=None):
        """Thermal Fock block, e.g. F('ai') = sqrt(n_i (1-n_a)) (f_ai - delta eps)."""
        (i0, f0), (i1, f1) = (self._axis(c, sel) for c in letters)
        return self.Fbar[i0][:, i1] * f0[:, None] * f1[None, :]

    def V(self, letters, sel=None):
        """Thermal antisymmetrised block, e.g. V('jabi') = <ja||bi> with slot factors."""
        cls = "".join("o" if c in HOLE else "v" for c in letters)
        ext = tuple(sel is not None and c in sel for c in letters)
        key = (cls, ext)
        if key in self._vcache:
            return self._vcache[key]
        ax = [self._axis(c, sel) for c in letters]
        blk = self.eri[ax[0][0]][:, ax[1][0]][:, :, ax[2][0]][:, :, :, ax[3][0]]
        blk = (blk * ax[0][1][:, None, None, None] * ax[1][1][None, :, None, None]
               * ax[2][1][None, None, :, None] * ax[3][1][None, None, None, :])
        self._vcache[key] = blk
        return blk

    def clear_cache(self):
        self._vcache = {}


def _amp(t1, t2, kind, letters, sel):
    """Amplitude operand s_i^a (T1, stored [x, i, a]) or s_ij^ab (T2, [x, i, j, a, b])."""
    t = t1 if kind == "T1" else t2
    if sel is not None:
        for ax, c in enumerate(letters):
            if c in sel:
                t = t.index_select(ax + 1, sel[c])
    return t


# Term tables.  Each entry is (coefficient, antisymmetriser, factors) with
# factors 'F:pq' (thermal Fock), 'V:pqrs' (thermal <pq||rs>), 'T1:ia' (s_i^a),
# 'T2:ijab' (s_ij^ab); letters i..n are hole-like, a..h particle-like.
# Eq. ccS1, in the order printed (R8 applied to the last term).
S1_TERMS = [
    (1.0, "", ["F:ai"]),
    (1.0, "", ["F:ab", "T1:ib"]),
    (-1.0, "", ["F:ji", "T1:ja"]),
    (1.0, "", ["V:jabi", "T1:jb"]),
    (1.0, "", ["F:jb", "T2:ijab"]),
    (0.5, "", ["V:ajbc", "T2:ijbc"]),
    (-0.5, "", ["V:jkib", "T2:jkab"]),
    (-1.0, "", ["F:jb", "T1:ib", "T1:ja"]),
    (1.0, "", ["V:jabc", "T1:jb", "T1:ic"]),
    (-1.0, "", ["V:jkbi", "T1:jb", "T1:ka"]),
    (-0.5, "", ["V:jkbc", "T1:ib", "T2:jkac"]),
    (-0.5, "", ["V:jkbc", "T1:ja", "T2:ikbc"]),
    (1.0, "", ["V:jkbc", "T1:jb", "T2:kica"]),
    (1.0, "", ["V:jkbc", "T1:ib", "T1:jc", "T1:ka"]),
]

# Eq. ccS2, in the order printed.
S2_TERMS = [
    (1.0, "", ["V:abij"]),
    (1.0, "ij", ["V:abcj", "T1:ic"]),
    (-1.0, "ab", ["V:kbij", "T1:ka"]),
    (1.0, "ab", ["F:bc", "T2:ijac"]),
    (-1.0, "ij", ["F:kj", "T2:ikab"]),
    (0.5, "", ["V:abcd", "T2:ijcd"]),
    (0.5, "", ["V:klij", "T2:klab"]),
    (1.0, "ijab", ["V:kbcj", "T2:ikac"]),
    (0.5, "ij", ["V:abcd", "T1:ic", "T1:jd"]),
    (0.5, "ab", ["V:klij", "T1:ka", "T1:lb"]),
    (-1.0, "ijab", ["V:akcj", "T1:ic", "T1:kb"]),
    (-1.0, "ij", ["F:kc", "T1:ic", "T2:kjab"]),
    (-1.0, "ab", ["F:kc", "T1:ka", "T2:ijcb"]),
    (1.0, "ab", ["V:kacd", "T1:kc", "T2:ijdb"]),
    (-1.0, "ij", ["V:klci", "T1:kc", "T2:ljab"]),
    (1.0, "ijab", ["V:akcd", "T1:ic", "T2:kjdb"]),
    (-1.0, "ijab", ["V:klic", "T1:ka", "T2:ljcb"]),
    (0.5, "ij", ["V:klcj", "T1:ic", "T2:klab"]),
    (-0.5, "ab", ["V:kbcd", "T1:ka", "T2:ijcd"]),
    (0.25, "", ["V:klcd", "T2:ijcd", "T2:klab"]),
    (0.5, "ijab", ["V:klcd", "T2:ikac", "T2:ljdb"]),
    (-0.5, "ab", ["V:klcd", "T2:klca", "T2:ijdb"]),
    (-0.5, "ij", ["V:klcd", "T2:kicd", "T2:ljab"]),
    (-0.5, "ijab", ["V:kbcd", "T1:ic", "T1:ka", "T1:jd"]),
    (0.5, "ijab", ["V:klcj", "T1:ic", "T1:ka", "T1:lb"]),
    (0.25, "ij", ["V:klcd", "T1:ic", "T1:jd", "T2:klab"]),
    (0.25, "ab", ["V:klcd", "T1:ka", "T1:lb", "T2:ijcd"]),
    (-1.0, "ijab", ["V:klcd", "T1:ic", "T1:ka", "T2:ljdb"]),
    (-1.0, "ij", ["V:klcd", "T1:kc", "T1:id", "T2:ljab"]),
    (-1.0, "ab", ["V:klcd", "T1:kc", "T1:la", "T2:ijdb"]),
    (0.25, "ijab", ["V:klcd", "T1:ic", "T1:ka", "T1:lb", "T1:jd"]),
]


def _antisym(res, perm, out):
    """P(pq) X = X - X(p <-> q) on the output axes (axis 0 is tau)."""
    if perm in ("ij", "ijab"):
        a0, a1 = out.index("i") + 1, out.index("j") + 1
        res = res - _swap(res, a0, a1)
    if perm in ("ab", "ijab"):
        a0, a1 = out.index("a") + 1, out.index("b") + 1
        res = res - _swap(res, a0, a1)
    return res


def _eval_terms(prob, terms, out, t1, t2, sel, which=None):
    nx = t1.shape[0]
    if sel is not None:
        prob.clear_cache()
    total = None
    for k, (coef, perm, factors) in enumerate(terms):
        if which is not None and k not in which:
            continue
        ops, subs, has_t = [], [], False
        for fct in factors:
            kind, letters = fct.split(":")
            if kind == "F":
                ops.append(prob.F(letters, sel))
                subs.append(letters)
            elif kind == "V":
                ops.append(prob.V(letters, sel))
                subs.append(letters)
            else:
                ops.append(_amp(t1, t2, kind, letters, sel))
                subs.append("x" + letters)
                has_t = True
        if has_t:
            res = contract(",".join(subs) + "->x" + out, *ops)
        else:
            res = contract(",".join(subs) + "->" + out, *ops)
            res = res.unsqueeze(0).expand((nx,) + tuple(res.shape))
        res = coef * _antisym(res, perm, out)
        total = res if total is None else total + res
    if sel is not None:
        prob.clear_cache()
    return total


def S1(prob, t1, t2, sel=None, which=None):
    """Singles kernel S_i^a(tau_x) for every x (Eq. ccS1); result [x, i, a]."""
    return _eval_terms(prob, S1_TERMS, "ia", t1, t2, sel, which)


def S2(prob, t1, t2, sel=None, which=None):
    """Doubles kernel S_ij^ab(tau_x) for every x (Eq. ccS2); result [x, i, j, a, b]."""
    return _eval_terms(prob, S2_TERMS, "ijab", t1, t2, sel, which)


def energy(prob, t1, t2):
    """E(tau_x) = sum f_ia s_i^a + 1/4 sum <ij||ab> (s_ij^ab + 2 s_i^a s_j^b)  (Eq. E)."""
    fia = prob.F("ia")
    vv = prob.V("ijab")
    e1 = torch.einsum("ia,xia->x", fia, t1)
    e2 = 0.25 * torch.einsum("ijab,xijab->x", vv, t2)
    e3 = 0.5 * torch.einsum("ijab,xia,xjb->x", vv, t1, t1)
    return e1 + e2 + e3


def propagate(prob, S, D):
    """s_mu(tau_y) = -sum_x G[y, x] exp(Delta_mu (tau_x - tau_y)) S_mu(tau_x)  (Eq. smu, App. A).

    On the uniform grid the exponent depends on x - y only; one exponential
    table per offset is formed from tau directly.
    """
    ng = prob.ngrid
    G, tau = prob.G, prob.tau
    out = []
    cache = {}
    for y in range(ng):
        acc = torch.zeros_like(S[0])
        for x in range(ng):
            if G[y, x].item() == 0.0:
                continue
            d = x - y
            if d not in cache:
                cache[d] = torch.exp(D * (tau[x] - tau[y]))
            acc = acc + G[y, x] * cache[d] * S[x]
        out.append(-acc)
    return torch.stack(out)


def omega_cc(prob, t1, t2):
    """Omega_CC = beta^-1 sum_y g_y E(tau_y)  (Eq. Ecc, App. A)."""
    return torch.sum(prob.g * energy(prob, t1, t2)) / prob.beta


def fixed_point_map(prob, t1, t2):
    """One application of the discretised amplitude equations to all tau."""
    return (propagate(prob, S1(prob, t1, t2), prob.D1),
            propagate(prob, S2(prob, t1, t2), prob.D2))


def solve(prob, tol=1e-12, tol_amp=1e-10, max_iter=400, damping=1.0, t1=None, t2=None,
          verbose=False):
    """Converge the amplitudes from s = 0 (Alg. 2 initial value, reading R2/R11).

    Stops when |dOmega_CC| < tol and max|ds| / max(1, max|s|) < tol_amp.
    """
    no, nv, ng = len(prob.iO), len(prob.iV), prob.ngrid
    if t1 is None:
        t1 = torch.zeros((ng, no, nv), dtype=DT)
        t2 = torch.zeros((ng, no, no, nv, nv), dtype=DT)
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
            dmax = max(torch.max(torch.abs(n1 - t1)).item() if n1.numel() else 0.0,
                       torch.max(torch.abs(n2 - t2)).item() if n2.numel() else 0.0)
            smax = max(torch.max(torch.abs(n1)).item() if n1.numel() else 0.0,
                       torch.max(torch.abs(n2)).item() if n2.numel() else 0.0)
            dmax = dmax / max(1.0, smax)
            t1, t2 = n1, n2
            occ = omega_cc(prob, t1, t2).item()
            history.append(occ)
            if verbose:
                print(it, occ, occ - occ_old, dmax)
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


# ---------------------------------------------------------------- adjoint
def lambda_solve(prob, t1, t2, tol=1e-11, max_iter=400):
    """Weighted multipliers m_y = g_y lambda_y / beta at the converged s.

    Stationarity of the discrete Lagrangian
        L = beta^-1 sum_y g_y E(s_y) + beta^-1 sum_y g_y <lambda_y, s_y - Phi(s)_y>,
    Phi the fixed-point map above, gives m = -dE_cc/ds + J_Phi^T m, which is
    Eq. lmu with Eq. ltilde in full-array form (the inner product <., .> runs
    over every element of s1 and s2).  Solved by fixed-point iteration from 0.
    """
    t1 = t1.detach().requires_grad_(True)
    t2 = t2.detach().requires_grad_(True)
    ecc = omega_cc(prob, t1, t2)
    dE1, dE2 = torch.autograd.grad(ecc, (t1, t2))
    p1, p2 = fixed_point_map(prob, t1, t2)
    m1 = torch.zeros_like(t1)
    m2 = torch.zeros_like(t2)
    converged = False
    for it in range(1, max_iter + 1):
        v1, v2 = torch.autograd.grad((p1, p2), (t1, t2), grad_outputs=(m1, m2),
                                     retain_graph=True)
        n1 = -dE1 + v1
        n2 = -dE2 + v2
        d = max(torch.max(torch.abs(n1 - m1)).item(), torch.max(torch.abs(n2 - m2)).item())
        m1, m2 = n1.detach(), n2.detach()
        if d < tol:
            converged = True
            break
    return {"m1": m1, "m2": m2, "iterations": it, "converged": converged}


def lagrangian_total(system, beta, mu, ngrid, t1, t2, m1, m2, thr=0.0):
    """Omega0 + Omega1 + L(s, lambda) as a differentiable function of the
    parameters carried by ``system`` / beta / mu (App. B: partial derivatives
    of the Lagrangian at fixed amplitudes give the response)."""
    prob = Problem(system, beta, mu, ngrid, thr)
    p1, p2 = fixed_point_map(prob, t1, t2)
    ecc = omega_cc(prob, t1, t2)
    res = torch.sum(m1 * (t1 - p1)) + torch.sum(m2 * (t2 - p2))
    return prob.omega0 + prob.omega1 + ecc + res


def response(system, beta, mu, ngrid, thr=0.0, solve_kw=None):
    """Converged Omega with dOmega/dmu, dOmega/dbeta, N, E, S and the
    partially relaxed 1-RDM p^cc (App. B; rdm1[q, p] pairs with X[p, q])."""
    solve_kw = solve_kw or {}
    prob = Problem(system, beta, mu, ngrid, thr)
    sol = solve(prob, **solve_kw)
    lam = lambda_solve(prob, sol["t1"], sol["t2"])
    b = torch.tensor(float(beta), dtype=DT, requires_grad=True)
    m = torch.tensor(float(mu), dtype=DT, requires_grad=True)
    h = system["h"].detach().clone().requires_grad_(True)
    e = system["eps"].detach().clone().requires_grad_(True)
    sysg = dict(system)
    sysg["h"] = h
    sysg["eps"] = e
    lag = lagrangian_total(sysg, b, m, ngrid, sol["t1"].detach(), sol["t2"].detach(),
                           lam["m1"], lam["m2"], thr)
    gb, gm, gh, ge = torch.autograd.grad(lag, (b, m, h, e))
    om = sol["omega"]
    nel = -gm.item()
    dodb = gb.item()
    energy_tot = om + float(beta) * dodb + float(mu) * nel
    rdm1 = gh.detach().T.clone()
    rdm1 += torch.diag(ge.detach())
    return {"omega": om, "lagrangian": lag.item(), "dOmega_dmu": gm.item(),
            "dOmega_dbeta": dodb, "N": nel, "E": energy_tot,
            "S": float(beta) ** 2 * dodb, "rdm1": rdm1, "solve": sol, "lambda": lam}


def rdm2_normal(system, beta, mu, ngrid, thr=0.0, solve_kw=None):
    """Unrelaxed normal-ordered 2-RDM Gamma_N (reading R14).

    The derivative of the CC Lagrangian (Eqs. Lagrangian, E, ccS1, ccS2) with
    respect to the antisymmetrised integrals <pq||rs> that enter the CC
    equations and energy through the thermal blocks, at fixed reference
    (occupations, Fock matrix, orbital energies), projected onto the
    antisymmetric tensors: for any perturbation dV with the symmetries of
    <pq||rs>, dOmega_CC = sum_pqrs Gamma[p, q, r, s] dV[p, q, r, s].
    """
    solve_kw = solve_kw or {}
    prob0 = Problem(system, beta, mu, ngrid, thr)
    sol = solve(prob0, **solve_kw)
    lam = lambda_solve(prob0, sol["t1"], sol["t2"])
    eri = system["eri"].detach().clone().requires_grad_(True)
    prob = Problem(system, beta, mu, ngrid, thr)   # reference from the unperturbed integrals
    prob.eri = eri
    prob.clear_cache()
    t1, t2 = sol["t1"].detach(), sol["t2"].detach()
    p1, p2 = fixed_point_map(prob, t1, t2)
    lag = omega_cc(prob, t1, t2) + torch.sum(lam["m1"] * (t1 - p1)) + torch.sum(lam["m2"] * (t2 - p2))
    (g,) = torch.autograd.grad(lag, eri)
    g = 0.5 * (g - g.permute(1, 0, 2, 3))
    return 0.5 * (g - g.permute(0, 1, 3, 2))


def omega_cc_frozen_reference(system, beta, mu, ngrid, eri_cc, thr=0.0, **kw):
    """Converged Omega_CC with the CC equations and energy built from eri_cc
    and the reference (n, f, eps) from system["eri"] (for finite-difference
    checks of rdm2_normal)."""
    prob = Problem(system, beta, mu, ngrid, thr)
    prob.eri = eri_cc
    prob.clear_cache()
    return solve(prob, **kw)["omega_cc"]


def omega_at(system, beta, mu, ngrid, thr=0.0, **kw):
    """Converged Omega for given parameters (used for finite-difference pins)."""
    return solve(Problem(system, beta, mu, ngrid, thr), **kw)["omega"]
