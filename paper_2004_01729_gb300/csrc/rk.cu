// Differential form of the amplitude equations (Eq. smud):
//   ds_mu/dtau = -(Delta_mu s_mu + S_mu[s]),  s(0) = 0,
// marched over the uniform grid by explicit Runge-Kutta steps (Alg. 1; the
// tableaux are read as forward Euler, Heun and the classical four-stage
// method, since the paper names RK1 / RK2 / RK4 without printing them).
// The S kernel is the engine's own (Solver::s_kernel on one tau slice per
// instance); these kernels form the stage inputs, the derivatives and the
// energies the grand potential is integrated from.
#include "ftcc_internal.h"

namespace ftcc {
namespace {

inline int rk_grid(long long n, int threads) {
  const long long b = (n + threads - 1) / threads;
  return static_cast<int>(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

// out[z][mu] = base[z][mu] + h_z sum_j c_j K_j[z][mu] for mu < n, every
// instance z (h_z = hz[z], the step of instance z); out and base carry their
// own instance strides (the marched state keeps every tau point, the stage
// buffers one).
template <class T>
__global__ void rk_combine_kernel(T* __restrict__ out, long long ozs, const T* __restrict__ base, long long bzs,
                                  RkTerms<T> k, const double* __restrict__ hz, long long n, int nz) {
  const long long total = n * nz;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long z = e / n, mu = e - z * n;
    T acc = T(0);
    for (int j = 0; j < k.n; ++j) acc += k.c[j] * k.K[j][z * n + mu];
    out[z * ozs + mu] = base[z * bzs + mu] + static_cast<T>(hz[z]) * acc;
  }
}

// K[z][mu] = -(Delta_mu Y[z][mu] + S[z][mu]); Delta_ia = eps_a - eps_i or
// Delta_ijab = eps_a + eps_b - eps_i - eps_j with the orbital energies of
// instance z (eps [nz][N]; idxO / idxV map the kept hole- / particle-like
// ranges to orbitals).
template <class T>
__global__ void rk_deriv_kernel(T* __restrict__ K, const T* __restrict__ Y, const T* __restrict__ S,
                                const double* __restrict__ eps, const int* __restrict__ idxO,
                                const int* __restrict__ idxV, int N, int no, int nv, int nslot, long long n, int nz) {
  const long long total = n * nz;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long z = e / n;
    long long r = e - z * n;
    const double* ez = eps + z * N;
    double d;
    if (nslot == 2) {   // [i][a]
      const int a = static_cast<int>(r % nv), i = static_cast<int>(r / nv);
      d = ez[idxV[a]] - ez[idxO[i]];
    } else {            // [i][j][a][b]
      const int b = static_cast<int>(r % nv);
      r /= nv;
      const int a = static_cast<int>(r % nv);
      r /= nv;
      const int j = static_cast<int>(r % no), i = static_cast<int>(r / no);
      d = ez[idxV[a]] + ez[idxV[b]] - ez[idxO[i]] - ez[idxO[j]];
    }
    K[e] = -(static_cast<T>(d) * Y[e] + S[e]);
  }
}

// Energy partials of Eq. E for every tau point y and instance z:
//   singles (NS = 2): sum_ia f_ia s_i^a(tau_y)
//   doubles (NS = 4): sum_ijab <ij||ab> (1/4 s_ij^ab + 1/2 s_i^a s_j^b)
// Block b of (y, z) sums elements b, b + nb blockDim, ... in a fixed order
// and writes partials[z][y][b] (the layout the reduction folds with the
// quadrature weights), and zero in the two maxima rows [z][ng], [z][ng+1].
constexpr int kRkThreads = 256;
template <class T, int NS>
__global__ void __launch_bounds__(kRkThreads) rk_energy_kernel(const T* __restrict__ t, const T* __restrict__ t1,
                                                               const double* __restrict__ w, int ng, int no, int nv,
                                                               long long size, int nb, double* partials) {
  const int y = blockIdx.y, z = blockIdx.z;
  const long long n1 = static_cast<long long>(no) * nv;
  const T* ty = t + (static_cast<long long>(z) * ng + y) * size;
  const T* s1 = t1 + (static_cast<long long>(z) * ng + y) * n1;
  const double* wz = w + static_cast<long long>(z) * size;
  double acc = 0.0;
  for (long long mu = blockIdx.x * static_cast<long long>(kRkThreads) + threadIdx.x; mu < size;
       mu += static_cast<long long>(nb) * kRkThreads) {
    double e;
    if (NS == 2) {
      e = static_cast<double>(ty[mu]);
    } else {
      long long r = mu;
      const int b = static_cast<int>(r % nv);
      r /= nv;
      const int a = static_cast<int>(r % nv);
      r /= nv;
      const int j = static_cast<int>(r % no), i = static_cast<int>(r / no);
      e = 0.25 * static_cast<double>(ty[mu]) +
          0.5 * static_cast<double>(s1[i * nv + a]) * static_cast<double>(s1[j * nv + b]);
    }
    acc += wz[mu] * e;
  }
  __shared__ double red[kRkThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kRkThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* p = partials + static_cast<long long>(z) * (ng + 2) * nb;
    p[static_cast<long long>(y) * nb + blockIdx.x] = red[0];
    if (y == 0) {
      p[static_cast<long long>(ng) * nb + blockIdx.x] = 0.0;
      p[static_cast<long long>(ng + 1) * nb + blockIdx.x] = 0.0;
    }
  }
}

}  // namespace

template <class T>
cudaError_t launch_rk_combine(T* out, long long ozs, const T* base, long long bzs, const RkTerms<T>& k,
                              const double* hz, long long n, int nz, cudaStream_t st) {
  if (n <= 0 || nz <= 0) return cudaSuccess;
  if (k.n < 0 || k.n > 4) return cudaErrorInvalidValue;
  rk_combine_kernel<T><<<rk_grid(n * nz, 256), 256, 0, st>>>(out, ozs, base, bzs, k, hz, n, nz);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_rk_deriv(T* K, const T* Y, const T* S, const double* eps, const int* idxO, const int* idxV, int N,
                            int no, int nv, int nslot, int nz, cudaStream_t st) {
  const long long n = nslot == 2 ? static_cast<long long>(no) * nv : static_cast<long long>(no) * no * nv * nv;
  if (n <= 0 || nz <= 0) return cudaSuccess;
  if (nslot != 2 && nslot != 4) return cudaErrorInvalidValue;
  rk_deriv_kernel<T><<<rk_grid(n * nz, 256), 256, 0, st>>>(K, Y, S, eps, idxO, idxV, N, no, nv, nslot, n, nz);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_rk_energy(const T* t1, const T* t2, const double* F64, const double* V64, int ng, int no, int nv,
                             int nz, int nb1, int nb2, double* part1, double* part2, cudaStream_t st) {
  if (ng < 1 || ng > 65535 || nz < 1 || nz > 65535 || nb1 < 1 || nb2 < 1) return cudaErrorInvalidValue;
  const long long n1 = static_cast<long long>(no) * nv, n2 = n1 * no * nv;
  rk_energy_kernel<T, 2><<<dim3(nb1, ng, nz), kRkThreads, 0, st>>>(t1, t1, F64, ng, no, nv, n1, nb1, part1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rk_energy_kernel<T, 4><<<dim3(nb2, ng, nz), kRkThreads, 0, st>>>(t2, t1, V64, ng, no, nv, n2, nb2, part2);
  return cudaGetLastError();
}

template cudaError_t launch_rk_combine<double>(double*, long long, const double*, long long, const RkTerms<double>&,
                                               const double*, long long, int, cudaStream_t);
template cudaError_t launch_rk_deriv<double>(double*, const double*, const double*, const double*, const int*,
                                             const int*, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_rk_energy<double>(const double*, const double*, const double*, const double*, int, int,
                                              int, int, int, int, double*, double*, cudaStream_t);

}  // namespace ftcc
