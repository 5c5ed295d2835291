"""Model Hamiltonians for the oracle (test infrastructure only).

Each builder returns a dict with
  h    (N, N)        one-body matrix in the spin-orbital basis
  eri  (N, N, N, N)  antisymmetrised <pq||rs> = <pq|rs> - <pq|sr>
  eps  (N,)          reference orbital energies
all float64 torch tensors on the CPU.  Spin orbital p = sigma * M + g with
sigma = 0 (up), 1 (down) and g the spatial index.

Sources: 1D Hubbard Hamiltonian (Sec. IV.A), the plane-wave UEG used in
Sec. IV.B / App. D, the k-space restricted reference of the Hubbard model at
half filling (Sec. II.B: orbitals and orbital energies define the
reference), and the Neel-state and zero-temperature UHF references with the
staggered magnetisation of Sec. IV.A (Figs. 4 and 5).
"""
import math

import numpy as np
import torch

DT = torch.float64


def _two_body_from_spatial(v):
    """Spin-orbital antisymmetrised integrals from spatial <pq|rs> (M^4).

    <p s1 q s2 | r s3 t s4> = v[p,q,r,t] delta(s1,s3) delta(s2,s4).
    """
    M = v.shape[0]
    N = 2 * M
    g = torch.zeros((N, N, N, N), dtype=DT)
    for s1 in range(2):
        for s2 in range(2):
            g[s1 * M:(s1 + 1) * M, s2 * M:(s2 + 1) * M,
              s1 * M:(s1 + 1) * M, s2 * M:(s2 + 1) * M] = v
    return g - g.permute(0, 1, 3, 2)


def hubbard_1d(L, t, U, pbc=True):
    """1D Hubbard model in the k-space restricted reference.

    H = -t sum_{i sigma} (a+_{i} a_{i+1} + h.c.) + U sum_i n_i^up n_i^dn.
    Orbitals phi_k(i) = exp(i k i)/sqrt(L), k = 2 pi m / L (PBC), so the
    hopping is diagonal, h_kk = -2 t cos k, and the on-site interaction is
    <k1 k2|k3 k4> = (U/L) delta(k1 + k2 = k3 + k4 mod 2 pi).  Reference
    energies are the restricted Hartree-Fock energies at half filling,
    eps_k = -2 t cos k + U/2.  Only PBC is supported in k space.
    """
    if not pbc:
        raise ValueError("k-space Hubbard reference needs periodic boundaries")
    m = np.arange(L)
    hk = -2.0 * t * np.cos(2.0 * np.pi * m / L)
    v = np.zeros((L, L, L, L))
    for a in range(L):
        for b in range(L):
            for c in range(L):
                d = (a + b - c) % L
                v[a, b, c, d] = U / L
    M = L
    h = torch.zeros((2 * M, 2 * M), dtype=DT)
    h[range(2 * M), range(2 * M)] = torch.tensor(np.concatenate([hk, hk]), dtype=DT)
    eri = _two_body_from_spatial(torch.tensor(v, dtype=DT))
    eps = torch.tensor(np.concatenate([hk, hk]) + U / 2.0, dtype=DT)
    return {"h": h, "eri": eri, "eps": eps, "kind": "hubbard", "L": L, "t": t, "U": U}


def hubbard_1d_sites(L, t, U, pbc=True):
    """Same Hamiltonian in the site basis (used only to pin hubbard_1d)."""
    hs = np.zeros((L, L))
    for i in range(L):
        j = i + 1
        if j == L:
            if not pbc:
                continue
            j = 0
        hs[i, j] += -t
        hs[j, i] += -t
    v = np.zeros((L, L, L, L))
    for i in range(L):
        v[i, i, i, i] = U
    M = L
    h = torch.zeros((2 * M, 2 * M), dtype=DT)
    h[:M, :M] = torch.tensor(hs)
    h[M:, M:] = torch.tensor(hs)
    eri = _two_body_from_spatial(torch.tensor(v, dtype=DT))
    return {"h": h, "eri": eri, "eps": torch.diagonal(h).clone() + U / 2.0}


def hubbard_1d_neel(L, t, U, pbc=True):
    """Site-basis 1D Hubbard model with the Neel-state reference (Sec. IV.A):
    the reference non-interacting system is the diagonal of the
    zero-temperature Fock matrix of the Neel determinant (spin up on even
    sites, spin down on odd sites), eps_{i sigma} = h_ii + U n^Neel_{i, -sigma}."""
    s = hubbard_1d_sites(L, t, U, pbc)
    M = L
    eps = torch.diagonal(s["h"]).clone()
    for i in range(M):
        n_up = 1.0 if i % 2 == 0 else 0.0
        eps[i] += U * (1.0 - n_up)     # spin up on site i meets the Neel down electron
        eps[M + i] += U * n_up         # spin down meets the up electron
    s["eps"] = eps
    s.update(kind="hubbard_neel", L=L, t=t, U=U)
    return s


def uhf_site_hubbard(L, t, U, n_up=None, n_dn=None, pbc=True, max_iter=2000, tol=1e-12, mix=0.5):
    """Zero-temperature unrestricted Hartree-Fock of the site-basis 1D Hubbard
    model, started from the Neel density (Sec. IV.A).

    F_sigma = h + U diag(n_{-sigma}); each spin fills its n_sigma lowest
    orbitals; the densities are mixed linearly until they change by less
    than tol.  Returns the per-spin orbital coefficients C [2, L, L] (columns
    are orbitals in ascending energy), orbital energies e [2, L], densities
    n [2, L] and the UHF energy.
    """
    n_up = L // 2 if n_up is None else n_up
    n_dn = L - n_up if n_dn is None else n_dn
    hs = hubbard_1d_sites(L, t, U, pbc)["h"][:L, :L].numpy()
    dens = np.zeros((2, L))
    for i in range(L):
        dens[0, i] = 1.0 if i % 2 == 0 else 0.0
        dens[1, i] = 1.0 - dens[0, i]
    occ = (n_up, n_dn)
    for _ in range(max_iter):
        C, e, new = [], [], np.zeros((2, L))
        for sg in range(2):
            F = hs + U * np.diag(dens[1 - sg])
            w, v = np.linalg.eigh(F)
            C.append(v)
            e.append(w)
            new[sg] = np.sum(v[:, :occ[sg]] ** 2, axis=1)
        diff = np.max(np.abs(new - dens))
        dens = (1.0 - mix) * dens + mix * new
        if diff < tol:
            dens = new
            break
    C, e = np.array(C), np.array(e)
    P = [C[sg][:, :occ[sg]] @ C[sg][:, :occ[sg]].T for sg in range(2)]
    energy = float(sum(np.sum(hs * P[sg]) for sg in range(2)) + U * np.sum(dens[0] * dens[1]))
    return {"C": C, "e": e, "n": dens, "P": np.array(P), "energy": energy, "h_site": hs}


def hubbard_1d_uhf(L, t, U, pbc=True, **scf):
    """Site-basis 1D Hubbard model in the UHF orbital basis with the UHF
    reference (Sec. IV.A: the reference is the diagonal of the
    zero-temperature Fock matrix, here the UHF orbital energies).  Spin
    orbital sigma * L + k is UHF orbital k of spin sigma."""
    uhf = uhf_site_hubbard(L, t, U, pbc=pbc, **scf)
    s = hubbard_1d_sites(L, t, U, pbc)
    N = 2 * L
    Cso = torch.zeros((N, N), dtype=DT)   # site spin orbital -> UHF spin orbital
    Cso[:L, :L] = torch.tensor(uhf["C"][0])
    Cso[L:, L:] = torch.tensor(uhf["C"][1])
    h = Cso.T @ s["h"] @ Cso
    eri = torch.einsum("pqrs,pa,qb,rc,sd->abcd", s["eri"], Cso, Cso, Cso, Cso)
    eps = torch.tensor(np.concatenate([uhf["e"][0], uhf["e"][1]]), dtype=DT)
    return {"h": h, "eri": eri, "eps": eps, "kind": "hubbard_uhf", "L": L, "t": t, "U": U, "uhf": uhf}


def staggered_magnetisation(rdm1, L):
    """m_s = L^-1 sum_i (-1)^i (<n_i,up> - <n_i,down>) from the diagonal of a
    1-RDM in the site basis (spin orbital sigma * L + i)."""
    d = torch.diagonal(torch.as_tensor(rdm1, dtype=DT))
    sign = torch.tensor([(-1.0) ** i for i in range(L)], dtype=DT)
    return float(torch.sum(sign * (d[:L] - d[L:])) / L)


def plane_wave_grid(n_pw):
    """Integer vectors n with |n|^2 <= c, c the shell closure giving n_pw.

    Ordered by (|n|^2, nx, ny, nz).  Raises if n_pw is not a closed shell.
    """
    r = int(math.isqrt(n_pw)) + 2
    pts = [(x * x + y * y + z * z, x, y, z)
           for x in range(-r, r + 1) for y in range(-r, r + 1) for z in range(-r, r + 1)]
    pts.sort()
    for c in range(0, 3 * r * r + 1):
        cnt = sum(1 for p in pts if p[0] <= c)
        if cnt == n_pw:
            return np.array([p[1:] for p in pts if p[0] <= c], dtype=np.int64)
        if cnt > n_pw:
            break
    raise ValueError(f"{n_pw} plane waves is not a closed shell")


def _ueg_cell(n_elec, rs, n_pw):
    """Plane waves of the cubic cell: integer vectors, volume, edge, k, |k|^2/2
    and the pair interaction 4 pi / (Vc |k_p - k_r|^2) (zero for p = r)."""
    nv = plane_wave_grid(n_pw)
    vol = 4.0 / 3.0 * math.pi * n_elec * rs ** 3
    Lc = vol ** (1.0 / 3.0)
    kv = 2.0 * math.pi * nv / Lc
    kin = 0.5 * np.sum(kv * kv, axis=1)
    diff = nv[:, None, :] - nv[None, :, :]                      # (p, r)
    q2 = np.sum(diff * diff, axis=2).astype(np.float64)
    coul = np.zeros_like(q2)
    nz = q2 > 0
    coul[nz] = 4.0 * math.pi / (vol * q2[nz] * (2.0 * math.pi / Lc) ** 2)
    return nv, vol, Lc, kv, kin, coul


def ueg_hf_energies(n_elec, rs, n_pw):
    """Zero-temperature Hartree-Fock energies of the closed shell of the
    n_elec/2 lowest plane waves per spin (the gas's reference energies):
    eps_p = |k_p|^2/2 - sum_{q occ} 4 pi / (Vc |k_p - k_q|^2), per spatial
    plane wave, with |k|^2/2."""
    nv, vol, Lc, kv, kin, coul = _ueg_cell(n_elec, rs, n_pw)
    nocc = n_elec // 2
    eps_sp = kin.copy()
    for p in range(len(nv)):
        eps_sp[p] -= sum(coul[p, q] for q in range(nocc))
    return eps_sp, kin


def ueg(n_elec, rs, n_pw):
    """Unpolarised uniform electron gas in a cubic cell of plane waves.

    Cell volume Vc = (4 pi / 3) n_elec rs^3; k = 2 pi n / Lc.
    h_pp = |k_p|^2 / 2; <pq|rs> = 4 pi / (Vc |k_p - k_r|^2) when
    k_p + k_q = k_r + k_s and spins match slot-wise, the q = 0 term omitted
    (neutralising background, no Madelung term).  Reference energies are
    zero-temperature Hartree-Fock energies of the closed shell of the n_elec/2
    lowest plane waves per spin: eps_p = |k_p|^2/2 - sum_{q occ} 4 pi/(Vc |k_p-k_q|^2).
    """
    nv, vol, Lc, kv, kin, coul = _ueg_cell(n_elec, rs, n_pw)
    M = len(nv)
    nz = coul > 0
    v = np.zeros((M, M, M, M))
    # v[p,q,r,s] = coul[p,r] if n_p + n_q == n_r + n_s
    key = {tuple(x): i for i, x in enumerate(nv)}
    for p in range(M):
        for r in range(M):
            if not nz[p, r]:
                continue
            dq = nv[p] - nv[r]
            for q in range(M):
                s = key.get(tuple(nv[q] + dq))
                if s is not None:
                    v[p, q, r, s] = coul[p, r]
    eps_sp, _ = ueg_hf_energies(n_elec, rs, n_pw)
    h = torch.zeros((2 * M, 2 * M), dtype=DT)
    h[range(2 * M), range(2 * M)] = torch.tensor(np.concatenate([kin, kin]), dtype=DT)
    eri = _two_body_from_spatial(torch.tensor(v, dtype=DT))
    eps = torch.tensor(np.concatenate([eps_sp, eps_sp]), dtype=DT)
    return {"h": h, "eri": eri, "eps": eps, "kind": "ueg", "vol": vol, "kvec": kv,
            "n_elec": n_elec, "rs": rs}


def ueg_fermi_energy(rs):
    """E_F = k_F^2 / 2 with k_F = (9 pi / 4)^(1/3) / rs (unpolarised 3D gas)."""
    kf = (9.0 * math.pi / 4.0) ** (1.0 / 3.0) / rs
    return 0.5 * kf * kf


def generic(h, eri, eps):
    """Wrap caller-supplied arrays (float64) without modification."""
    return {"h": torch.as_tensor(h, dtype=DT), "eri": torch.as_tensor(eri, dtype=DT),
            "eps": torch.as_tensor(eps, dtype=DT), "kind": "generic"}
