// Site-basis references of the 1D Hubbard ring (Sec. IV.A): the Neel
// determinant and the zero-temperature unrestricted Hartree-Fock solution.
// Host code only: the Hamiltonian and the reference energies are built here
// and uploaded like a generic system; everything after build_integrals runs
// on the GPU as for any other system.
//
// Spin orbital p = sigma * L + i (sigma = 0 up, 1 down, i the site).  The
// hopping is -t between neighbouring sites of the ring (both directions;
// on two sites the two bonds add), the interaction U n_i,up n_i,down, i.e.
// <pq|rs> = U when p, q, r, s sit on one site with spin(p) = spin(r) and
// spin(q) = spin(s), and <pq||rs> = <pq|rs> - <pq|sr>.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ftcc_internal.h"

namespace ftcc {
namespace {

// Eigen-decomposition of a symmetric n x n matrix (row-major) by cyclic
// Jacobi rotations; eigenvalues ascending, eigenvectors in the columns of V.
void jacobi_eigh(std::vector<double> A, int n, std::vector<double>& w, std::vector<double>& V) {
  V.assign(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) V[static_cast<size_t>(i) * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[static_cast<size_t>(i) * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += a(i, j) * a(i, j);
        if (i != j) off += a(i, j) * a(i, j);
      }
    if (off <= 1e-30 * std::max(tot, 1e-300)) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        // rotation angle that zeroes a(p, q): tan(2 phi) = 2 a_pq / (a_qq - a_pp)
        const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double tt = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(tt * tt + 1.0), s = tt * c;
        for (int k = 0; k < n; ++k) {   // columns p, q
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double& vkp = V[static_cast<size_t>(k) * n + p];
          double& vkq = V[static_cast<size_t>(k) * n + q];
          const double x = vkp, y = vkq;
          vkp = c * x - s * y;
          vkq = s * x + c * y;
        }
      }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return a(x, x) < a(y, y); });
  w.resize(n);
  std::vector<double> Vs(static_cast<size_t>(n) * n);
  for (int k = 0; k < n; ++k) {
    w[k] = a(ord[k], ord[k]);
    for (int i = 0; i < n; ++i) Vs[static_cast<size_t>(i) * n + k] = V[static_cast<size_t>(i) * n + ord[k]];
  }
  V.swap(Vs);
}

}  // namespace

bool hubbard_site_reference(int L, double t, double U, int reference, std::vector<double>& h,
                            std::vector<double>& eri, std::vector<double>& eps, std::string& err) {
  const int N = 2 * L;
  std::vector<double> hs(static_cast<size_t>(L) * L, 0.0);
  for (int i = 0; i < L; ++i) {
    const int j = (i + 1) % L;
    hs[static_cast<size_t>(i) * L + j] += -t;
    hs[static_cast<size_t>(j) * L + i] += -t;
  }
  h.assign(static_cast<size_t>(N) * N, 0.0);
  for (int sg = 0; sg < 2; ++sg)
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j) h[static_cast<size_t>(sg * L + i) * N + sg * L + j] = hs[static_cast<size_t>(i) * L + j];
  const size_t N4 = static_cast<size_t>(N) * N * N * N;
  eri.assign(N4, 0.0);
  auto at = [&](int p, int q, int r, int s) -> double& {
    return eri[((static_cast<size_t>(p) * N + q) * N + r) * N + s];
  };
  for (int i = 0; i < L; ++i)
    for (int s1 = 0; s1 < 2; ++s1)
      for (int s2 = 0; s2 < 2; ++s2) {
        const int p = s1 * L + i, q = s2 * L + i;
        at(p, q, p, q) += U;   // <pq|rs> with r = p, s = q
        at(p, q, q, p) -= U;   // - <pq|sr>
      }
  eps.assign(N, 0.0);
  if (reference == FTCC_REF_NEEL_SITE) {
    // Neel determinant: spin up on even sites, spin down on odd sites;
    // eps_{i sigma} = h_ii + U n^Neel_{i, -sigma}
    for (int i = 0; i < L; ++i) {
      const double n_up = (i % 2 == 0) ? 1.0 : 0.0;
      eps[i] = hs[static_cast<size_t>(i) * L + i] + U * (1.0 - n_up);
      eps[L + i] = hs[static_cast<size_t>(i) * L + i] + U * n_up;
    }
    return true;
  }
  if (reference != FTCC_REF_UHF_SITE) {
    err = "unknown reference";
    return false;
  }
  // zero-temperature UHF from the Neel density: F_sigma = h + U diag(n_-sigma),
  // each spin fills its lowest orbitals, densities mixed half and half until
  // they change by less than 1e-12
  const int occ[2] = {L / 2, L - L / 2};
  std::vector<double> dens(2 * static_cast<size_t>(L));
  for (int i = 0; i < L; ++i) {
    dens[i] = (i % 2 == 0) ? 1.0 : 0.0;
    dens[L + i] = 1.0 - dens[i];
  }
  std::vector<double> C[2], e[2];
  bool done = false;
  for (int it = 0; it < 2000 && !done; ++it) {
    std::vector<double> nw(2 * static_cast<size_t>(L), 0.0);
    for (int sg = 0; sg < 2; ++sg) {
      std::vector<double> F = hs;
      for (int i = 0; i < L; ++i) F[static_cast<size_t>(i) * L + i] += U * dens[(1 - sg) * L + i];
      jacobi_eigh(F, L, e[sg], C[sg]);
      for (int i = 0; i < L; ++i)
        for (int k = 0; k < occ[sg]; ++k) {
          const double c = C[sg][static_cast<size_t>(i) * L + k];
          nw[sg * L + i] += c * c;
        }
    }
    double diff = 0.0;
    for (size_t k = 0; k < nw.size(); ++k) diff = std::max(diff, std::fabs(nw[k] - dens[k]));
    for (size_t k = 0; k < nw.size(); ++k) dens[k] = 0.5 * dens[k] + 0.5 * nw[k];
    if (diff < 1e-12) {
      dens = nw;
      done = true;
    }
  }
  // spin-orbital coefficients (block diagonal) and the transformation of h
  // and <pq||rs> to the UHF spin orbitals
  std::vector<double> Cs(static_cast<size_t>(N) * N, 0.0);
  for (int sg = 0; sg < 2; ++sg)
    for (int i = 0; i < L; ++i)
      for (int k = 0; k < L; ++k) Cs[static_cast<size_t>(sg * L + i) * N + sg * L + k] = C[sg][static_cast<size_t>(i) * L + k];
  std::vector<double> hu(static_cast<size_t>(N) * N, 0.0);
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      double acc = 0.0;
      for (int p = 0; p < N; ++p)
        for (int q = 0; q < N; ++q)
          acc += Cs[static_cast<size_t>(p) * N + a] * h[static_cast<size_t>(p) * N + q] * Cs[static_cast<size_t>(q) * N + b];
      hu[static_cast<size_t>(a) * N + b] = acc;
    }
  h.swap(hu);
  // four quarter transformations, each contracting the leading index and
  // moving the new one to the back: X[pqrs] -> Y[qrs a] = sum_p X[pqrs] C[p a]
  std::vector<double> tmp(N4);
  for (int pass = 0; pass < 4; ++pass) {
    std::fill(tmp.begin(), tmp.end(), 0.0);
    const size_t N3 = static_cast<size_t>(N) * N * N;
    for (int p = 0; p < N; ++p)
      for (size_t rest = 0; rest < N3; ++rest) {
        const double x = eri[static_cast<size_t>(p) * N3 + rest];
        if (x == 0.0) continue;
        double* y = tmp.data() + rest * N;
        const double* c = Cs.data() + static_cast<size_t>(p) * N;
        for (int a = 0; a < N; ++a) y[a] += x * c[a];
      }
    eri.swap(tmp);
  }
  for (int sg = 0; sg < 2; ++sg)
    for (int k = 0; k < L; ++k) eps[sg * L + k] = e[sg][k];
  if (!done) {
    err = "UHF did not converge in 2000 iterations";
    return false;
  }
  return true;
}

}  // namespace ftcc
