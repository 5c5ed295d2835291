"""Seeded synthetic workloads shared by the tests, the oracle checks and the bench.

This module only names model parameters and draws random numbers; it holds
no finite-temperature coupled-cluster arithmetic and imports neither the CUDA
library nor the oracle.

Workloads (the paper's model systems, Sec. IV; all Hamiltonians are synthetic
by construction):
  HUBBARD_6    1D Hubbard ring, 6 sites, t=1, U=2, mu=U/2, beta=1, 16 tau points
  HUBBARD_10   1D Hubbard ring, 10 sites, t=1, U=4, mu=U/2, beta in {2, 1, 0.5},
               32 tau points
  UEG_57       warm dense electron gas, 14 electrons, rs=1, Theta=0.5,
               57 plane waves (114 spin orbitals), 32 tau points
  UEG_81       same gas at Theta=1, 81 plane waves (162 spin orbitals),
               40 tau points, occupation threshold 1e-8
  HUBBARD_BATCH  64 Hubbard rings of 6..14 sites, U ~ U[1, 8],
               T ~ U[0.25, 4], mu = U/2, 24 tau points (seed 1729)
"""
import math

import numpy as np

HUBBARD_6 = dict(kind="hubbard", L=6, t=1.0, U=2.0, beta=1.0, mu=1.0, ngrid=16)
HUBBARD_10 = [dict(kind="hubbard", L=10, t=1.0, U=4.0, beta=b, mu=2.0, ngrid=32)
              for b in (2.0, 1.0, 0.5)]


def ueg_beta(rs, theta):
    """Inverse temperature of reduced temperature Theta = T / E_F for the
    unpolarised 3D gas, k_F = (9 pi / 4)^(1/3) / rs, E_F = k_F^2 / 2."""
    kf = (9.0 * math.pi / 4.0) ** (1.0 / 3.0) / rs
    return 1.0 / (theta * 0.5 * kf * kf)


UEG_57 = dict(kind="ueg", n_elec=14, rs=1.0, theta=0.5, n_pw=57, ngrid=32, thr=0.0,
              beta=ueg_beta(1.0, 0.5))
UEG_81 = dict(kind="ueg", n_elec=14, rs=1.0, theta=1.0, n_pw=81, ngrid=40, thr=1e-8,
              beta=ueg_beta(1.0, 1.0))


def hubbard_batch(n=64, seed=1729):
    """Parameters of the batched Hubbard instances (even L keeps mu = U/2 at half filling)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        L = int(rng.choice([6, 8, 10, 12, 14]))
        U = float(rng.uniform(1.0, 8.0))
        T = float(rng.uniform(0.25, 4.0))
        out.append(dict(kind="hubbard", L=L, t=1.0, U=U, beta=1.0 / T, mu=U / 2.0, ngrid=24))
    return out


def random_amplitudes(seed, ngrid, no, nv, scale=0.1):
    """Random s1 [x, i, a] and antisymmetric s2 [x, i, j, a, b] (float64)."""
    rng = np.random.default_rng(seed)
    t1 = scale * rng.standard_normal((ngrid, no, nv))
    t2 = scale * rng.standard_normal((ngrid, no, no, nv, nv))
    t2 = t2 - t2.transpose(0, 2, 1, 3, 4)
    t2 = t2 - t2.transpose(0, 1, 2, 4, 3)
    return t1, 0.25 * t2


def random_generic_system(seed, N, h_scale=0.5, v_scale=0.05, eps_noise=0.3):
    """Random real symmetric h, antisymmetrised <pq||rs> with
    <pq||rs> = -<qp||rs> = -<pq||sr> = <rs||pq>, and reference energies near diag(h)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((N, N))
    h = h_scale * 0.5 * (a + a.T) + np.diag(np.linspace(-1.0, 1.0, N))
    b = rng.standard_normal((N, N, N, N))
    b = b + b.transpose(2, 3, 0, 1)
    b = b + b.transpose(1, 0, 3, 2)
    v = b - b.transpose(1, 0, 2, 3) - b.transpose(0, 1, 3, 2) + b.transpose(1, 0, 3, 2)
    eri = v_scale * v
    eps = np.diag(h).copy() + eps_noise * rng.standard_normal(N)
    return h, eri, eps
