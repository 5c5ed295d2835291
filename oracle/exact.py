"""Exact grand potentials used to pin the oracle (test infrastructure only).

* fock_space_omega: Omega = -beta^-1 ln Tr exp(-beta (H - mu N)) by full
  diagonalisation of H = sum h_pq a+_p a_q + 1/4 sum <pq||rs> a+_p a+_q a_s a_r
  in the occupation-number basis (at most ~10 spin orbitals).
* noninteracting_omega: the closed form -beta^-1 sum_k ln(1 + exp(-beta(e_k - mu)))
  over the eigenvalues e_k of a one-body h.
"""
import numpy as np
from scipy.special import logsumexp


def _apply_annihilate(state, q):
    if not (state >> q) & 1:
        return None, 0
    sign = -1 if bin(state & ((1 << q) - 1)).count("1") % 2 else 1
    return state & ~(1 << q), sign


def _apply_create(state, p):
    if (state >> p) & 1:
        return None, 0
    sign = -1 if bin(state & ((1 << p) - 1)).count("1") % 2 else 1
    return state | (1 << p), sign


def fock_space_hamiltonian(h, eri, tol=1e-14):
    """Dense H over all 2^N occupation-number states (bit p = orbital p)."""
    h = np.asarray(h, dtype=np.float64)
    eri = np.asarray(eri, dtype=np.float64)
    N = h.shape[0]
    dim = 1 << N
    H = np.zeros((dim, dim))
    one = [(p, q, h[p, q]) for p in range(N) for q in range(N) if abs(h[p, q]) > tol]
    two = [(p, q, r, s, 0.25 * eri[p, q, r, s])
           for p in range(N) for q in range(N) for r in range(N) for s in range(N)
           if abs(eri[p, q, r, s]) > tol]
    for st in range(dim):
        for p, q, v in one:
            s1, g1 = _apply_annihilate(st, q)
            if s1 is None:
                continue
            s2, g2 = _apply_create(s1, p)
            if s2 is None:
                continue
            H[s2, st] += v * g1 * g2
        for p, q, r, s, v in two:
            s1, g1 = _apply_annihilate(st, r)
            if s1 is None:
                continue
            s2, g2 = _apply_annihilate(s1, s)
            if s2 is None:
                continue
            s3, g3 = _apply_create(s2, q)
            if s3 is None:
                continue
            s4, g4 = _apply_create(s3, p)
            if s4 is None:
                continue
            H[s4, st] += v * g1 * g2 * g3 * g4
    return H


def fock_space_spectrum(h, eri):
    """Eigenvalues and particle numbers of every eigenstate (sector by sector)."""
    H = fock_space_hamiltonian(h, eri)
    N = np.asarray(h).shape[0]
    nel = np.array([bin(s).count("1") for s in range(1 << N)])
    evals, counts = [], []
    for k in range(N + 1):
        idx = np.nonzero(nel == k)[0]
        sub = H[np.ix_(idx, idx)]
        w = np.linalg.eigvalsh(0.5 * (sub + sub.T))
        evals.append(w)
        counts.append(np.full(len(w), k))
    return np.concatenate(evals), np.concatenate(counts)


def fock_space_omega(h, eri, beta, mu, spectrum=None):
    """Exact grand potential of the full Fock space."""
    e, k = spectrum if spectrum is not None else fock_space_spectrum(h, eri)
    return -logsumexp(-beta * (e - mu * k)) / beta


def noninteracting_omega(h, beta, mu):
    """Exact grand potential of a one-body Hamiltonian."""
    e = np.linalg.eigvalsh(np.asarray(h, dtype=np.float64))
    return -np.sum(np.logaddexp(0.0, -beta * (e - mu))) / beta
