// Momentum/spin block-sparse execution of the S kernel (Eqs. ccS1/ccS2),
// FP64.
//
// In the plane-wave electron gas (Sec. IV.B) and the k-space Hubbard ring
// (Sec. IV.A) every spin orbital p carries its own conserved charge q_p
// (crystal momentum and S_z): no two orbitals share one.  Every factor of the
// CCSD equations conserves it, so
//   * a two-index factor (f, s1, F_ae, F_mi, F_me, S1) is diagonal: a vector
//     X[p] = X_pp;
//   * a four-index factor with q_0 + q_1 = q_2 + q_3 (in the order it is
//     stored here) is fixed by its first three indices: it is stored as an
//     N^3 array X[p0][p1][p2], the fourth index implied by charge balance.
//     A triple whose implied charge belongs to no orbital (a "hole" of the
//     storage) holds zero.
// The implied index comes from one table imp[a][b][c] = the orbital whose
// charge is q_a + q_b - q_c, or -1 (int16, N^3 entries).
//
// Contractions of two four-index factors over two indices leave one free
// summed index once the output indices are fixed; they run as products of
// small dense blocks ("sectors"): the rows of the left operand are ordered
// index pairs (p, q) grouped by their pair charge (q_p + q_q for the
// ladders, q_p - q_q for the ring), the summed index runs over the K list of
// the sector, and every row of a sector meets every row of the matching
// sector of the right operand (sector_gemm_kernel).  Everything else is
// element by element over the N^3 positions or a reduction to a vector.
//
// Layout of a slice: [x][p0][p1][p2] for four-index tensors, [x][p] for
// vectors; fixed tensors (integrals, Fock diagonals) have no x.
#include <cstdint>

#include "ftcc_internal.h"

namespace ftcc {
namespace {

constexpr int kSpThreads = 256;

inline int sp_grid(long long n, int threads = kSpThreads, int cap = 152 * 16) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return static_cast<int>(b);
}

__device__ __forceinline__ int impl(const int16_t* __restrict__ imp, int n, int a, int b, int c) {
  return imp[(static_cast<long long>(a) * n + b) * n + c];
}

// (p0, p1, p2) of the N^3 position e in 32-bit arithmetic (N^3 < 2^31): a
// 64-bit division or remainder is a long instruction sequence, and three of
// them per element dominated the element-wise kernels
__device__ __forceinline__ void dec3(uint32_t e, uint32_t n, int& p0, int& p1, int& p2) {
  const uint32_t q = e / n;
  p2 = static_cast<int>(e - q * n);
  const uint32_t r = q / n;
  p1 = static_cast<int>(q - r * n);
  p0 = static_cast<int>(r);
}

__device__ __forceinline__ long long pos3(int n, int a, int b, int c) {
  return (static_cast<long long>(a) * n + b) * n + c;
}

// ---- amplitude-derived operands of one S evaluation (one pass over the
// N^3 positions of every slice x):
//   ta[i][j][a]  = tau_ij^ab = s_ij^ab + P(ij) s_i^a s_j^b      (b implied)
//   tp[a][b][m]  = tau_mn^ab                                    (n implied)
//   tr[i][a][m]  = s_im^ae                                      (e implied)
//   xp[j][b][n]  = X_jn^fb = 1/2 s_jn^fb + s_j^f s_n^b          (f implied)
// with s1 diagonal (s_i^a = delta_ia s1[i]).
template <class T>
__global__ void sp_amp_kernel(const T* __restrict__ t1, const T* __restrict__ t2,
                              const int16_t* __restrict__ imp, int n, T* __restrict__ ta,
                              T* __restrict__ tp, T* __restrict__ tr, T* __restrict__ xp, int skip_tau,
                              const int* __restrict__ list, int nlist) {
  // skip_tau with a list: only tr and xp, at the positions (p0, p1, p2) whose
  // (p0, p2, p1) is valid (the only ones the ordered products read)
  const long long n3 = static_cast<long long>(n) * n * n;
  const long long x = blockIdx.y;
  const T* s1 = t1 + x * n;
  const T* s2 = t2 + x * n3;
  const long long nloop = list ? nlist : n3;
  for (long long cc = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; cc < nloop;
       cc += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long e = list ? list[cc] : cc;
    int p0, p1, p2;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), p0, p1, p2);
    const long long o = x * n3 + e;
    if (!skip_tau) {   // ta: (i, j, a) = (p0, p1, p2), b implied
      const int b = impl(imp, n, p0, p1, p2);
      T v = T(0.0);
      if (b >= 0) {
        v = s2[e];
        const T pr = s1[p0] * s1[p1];
        if (p2 == p0) v += pr;
        if (p2 == p1) v -= pr;
      }
      ta[o] = v;
    }
    if (!skip_tau) {   // tp: (a, b, m) = (p0, p1, p2), n = q_a + q_b - q_m
      const int nn = impl(imp, n, p0, p1, p2);
      T v = T(0.0);
      if (nn >= 0) {
        v = s2[pos3(n, p2, nn, p0)];   // s_{m nn}^{a b}
        const T pr = s1[p2] * s1[nn];
        if (p0 == p2) v += pr;
        if (p0 == nn) v -= pr;
      }
      tp[o] = v;
    }
    {   // tr: (i, a, m) = (p0, p1, p2), e = q_i + q_m - q_a
      const int ee = impl(imp, n, p0, p2, p1);
      tr[o] = ee >= 0 ? s2[pos3(n, p0, p2, p1)] : T(0.0);   // s_{i m}^{a e}
    }
    {   // xp: (j, b, n) = (p0, p1, p2), f = q_j + q_n - q_b
      const int f = impl(imp, n, p0, p2, p1);
      T v = T(0.0);
      if (f >= 0) {
        v = T(0.5) * s2[pos3(n, p0, p2, f)];   // 1/2 s_{j n}^{f b}
        if (f == p0) v += s1[p0] * s1[p2];
      }
      xp[o] = v;
    }
  }
}

// ---- F_me = f_me + sum_n s1[n] <mn||mn>   (diagonal, e = m, f = n)
template <class T>
__global__ void sp_fme_kernel(const T* __restrict__ t1, const T* __restrict__ fov,
                              const T* __restrict__ Voovv, int n, int nx, T* __restrict__ Fme) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n * nx) return;
  const int x = warp / n, m = warp % n;
  const T* s1 = t1 + static_cast<long long>(x) * n;
  T acc = T(0.0);
  for (int q = lane; q < n; q += 32) acc += s1[q] * Voovv[pos3(n, m, q, m)];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) Fme[static_cast<long long>(x) * n + m] = fov[m] + acc;
}

// K sums of one block at once: each warp reduces its K values by shuffles,
// one barrier, thread 0 adds the warps' partials in order (the same order per
// value as K separate block_sum calls).  red: K * 32 slots; valid in thread 0.
template <class T, int K>
__device__ __forceinline__ void block_sums(T (&v)[K], T* red) {
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[k * 32 + w] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      T s = T(0.0);
      for (int q = 0; q < (blockDim.x >> 5); ++q) s += red[k * 32 + q];
      v[k] = s;
    }
}

template <class T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T s = T(0.0);
  if (threadIdx.x == 0)
    for (int k = 0; k < (blockDim.x >> 5); ++k) s += red[k];
  return s;   // valid in thread 0
}

// ---- the vector intermediates and S1 of one (x, p):
//   F_ae[p] = f_vv[p] - 1/2 s1[p] F_me[p] + sum_m s1[m] <mp||mp> - 1/2 sum_mn s_mn^pe <mn||pe>
//   F_mi[p] = f_oo[p] + 1/2 s1[p] F_me[p] + sum_n s1[n] <pn||pn> + 1/2 sum_ne s_pn^ef <pn||ef>
//   S1[p]   = f_vo[p] + s1[p] (F_ae[p] - F_mi[p]) + sum_m s_pm^pm F_me[m] - sum_n s1[n] <np||pn>
//             - 1/2 sum_me s_pm^ef <mp||ef> - 1/2 sum_mn s_mn^pe <nm||ep>
//   Ft[p] = F_ae[p] - 1/2 s1[p] F_me[p],  Ft2[p] = F_mi[p] + 1/2 s1[p] F_me[p]
// (the diagonal forms of Eq. ccS1's terms and of the F intermediates; each
// integral block in its own thermal scaling).
template <class T>
struct SpVec {
  const T *t1, *t2, *Fme;
  const T *foo, *fvv, *fvo;
  const T *Voovv, *Vovvv, *Vooov, *Vovov, *Voovo;
  const int16_t* imp;
  const int *l1, *off1, *l2, *off2;   // valid (m, q) = m n + q of (m, q, p) / (p, m, q) per p
  int n;
  T *Fae, *Fmi, *S1, *Ft, *Ft2;
};

template <class T>
__global__ void sp_vec_kernel(SpVec<T> a) {
  __shared__ T red[6 * 32];
  const int n = a.n;
  const long long n3 = static_cast<long long>(n) * n * n;
  const int p = blockIdx.x, x = blockIdx.y;
  const T* s1 = a.t1 + static_cast<long long>(x) * n;
  const T* s2 = a.t2 + x * n3;
  const T* Fme = a.Fme + static_cast<long long>(x) * n;
  T cae = T(0.0), cmi = T(0.0), cs1 = T(0.0);
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    cae += s1[m] * a.Vovvv[pos3(n, m, p, m)];
    cmi += s1[m] * a.Vooov[pos3(n, p, m, p)];
    cs1 += s2[pos3(n, p, m, p)] * Fme[m] - s1[m] * a.Vovov[pos3(n, m, p, p)];
  }
  // only the positions whose implied index exists (the others hold zeros):
  // (m, q, p) from the list l1 of p, (p, m, q) from l2.  The doubles terms
  // carry a factor 1/2, applied once to their sums (hae, hmi, hs1): FP64
  // issues at a few operations per clock per SM on this part, and the scale
  // per term was a third of these loops' FP64 instructions
  T hae = T(0.0), hmi = T(0.0), hs1 = T(0.0);
  for (int k = a.off1[p] + threadIdx.x; k < a.off1[p + 1]; k += blockDim.x) {
    const int mq = a.l1[k];
    const int m = mq / n, q = mq - m * n;
    const long long o1 = pos3(n, m, q, p);
    const T t_mqp = s2[o1];
    hae += t_mqp * a.Voovv[o1];
    const int e = impl(a.imp, n, m, q, p);   // q_e = q_m + q_q - q_p
    hs1 += t_mqp * a.Voovo[pos3(n, q, m, e)];
  }
  for (int k = a.off2[p] + threadIdx.x; k < a.off2[p + 1]; k += blockDim.x) {
    const int mq = a.l2[k];
    const int m = mq / n, q = mq - m * n;
    const long long o2 = pos3(n, p, m, q);
    const T t = s2[o2];
    hmi += t * a.Voovv[o2];
    hs1 += t * a.Vovvv[pos3(n, m, p, q)];
  }
  T sums[6] = {cae, cmi, cs1, hae, hmi, hs1};
  block_sums(sums, red);
  cae = sums[0];
  cmi = sums[1];
  cs1 = sums[2];
  hae = sums[3];
  hmi = sums[4];
  hs1 = sums[5];
  if (threadIdx.x == 0) {
    const long long o = static_cast<long long>(x) * n + p;
    const T s = s1[p], fm = Fme[p];
    const T fae = a.fvv[p] - T(0.5) * s * fm + (cae - T(0.5) * hae);
    const T fmi = a.foo[p] + T(0.5) * s * fm + (cmi + T(0.5) * hmi);
    a.Fae[o] = fae;
    a.Fmi[o] = fmi;
    a.S1[o] = a.fvo[p] + s * (fae - fmi) + (cs1 - T(0.5) * hs1);
    a.Ft[o] = fae - T(0.5) * s * fm;
    a.Ft2[o] = fmi + T(0.5) * s * fm;
  }
}

}  // namespace

namespace {

// ---- bases of the four-index intermediates (one pass over the positions):
//   w1[i][j][m] = W'_mnij without its tau term = <mn||ij> - 2 s1[i] <mn||ji>   (n implied)
//   wab[a][b][e] = W'_abef = <ab||ef> - 2 s1[a] <ab||ef>_ovvv                    (f implied)
//   wr[j][b][m] = W_mbej without its X term
//               = <mb||ej> + s1[j] <mb||ej>_ovvv - s1[b] <mb||ej>_oovo          (e implied)
// (s1 diagonal turns every s1 contraction of these intermediates into a
// scaling; the integral blocks differ only by their thermal factors).
template <class T>
struct SpW {
  const T *t1, *Voooo, *Vooov, *Vvvvv, *Vovvv, *Vovvo, *Voovo;
  const int16_t* imp;
  const int* list;   // anti: the positions (j, b, m) of W_mbej whose e exists
  int nlist;
  int n, anti;
  T *w1, *wab, *wr;
};

template <class T>
__global__ void sp_wbase_kernel(SpW<T> a) {
  const int n = a.n;
  const long long n3 = static_cast<long long>(n) * n * n;
  const long long x = blockIdx.y;
  const T* s1 = a.t1 + x * n;
  const long long nloop = a.list ? a.nlist : n3;
  for (long long cc = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; cc < nloop;
       cc += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long e = a.list ? a.list[cc] : cc;
    int p0, p1, p2;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), p0, p1, p2);
    const long long o = x * n3 + e;
    if (!a.anti) {   // (the antisymmetrised forms come from sp_canon_kernel)
      {   // (i, j, m) = (p0, p1, p2), n = q_i + q_j - q_m
        const int q = impl(a.imp, n, p0, p1, p2);
        a.w1[o] = q >= 0 ? a.Voooo[pos3(n, p2, q, p0)] - T(2.0) * s1[p0] * a.Vooov[pos3(n, p2, q, p1)] : T(0.0);
      }
      // (a, b, e) = (p0, p1, p2): the positions of the blocks coincide
      a.wab[o] = a.Vvvvv[e] - T(2.0) * s1[p0] * a.Vovvv[e];
    }
    {   // (j, b, m) = (p0, p1, p2), e = q_b + q_m - q_j
      const int ee = impl(a.imp, n, p1, p2, p0);
      T v = T(0.0);
      if (ee >= 0) {
        const long long c = pos3(n, p2, p1, ee);   // (m, b, e), j implied
        v = a.Vovvo[c] + s1[p0] * a.Vovvv[c] - s1[p1] * a.Voovo[c];
      }
      a.wr[o] = v;
    }
  }
}

// ---- R (the accumulator that enters S2 through P(ij)P(ab)), the terms
// that need no sector product, for (i, j, a) with b implied:
//   R = 1/2 s_ij^ab Ft[b] + 1/2 Ft2[i] s_ji^ab + 1/2 s1[i] <ab||ij>_vvvo
//     - 1/2 s1[a] <ab||ij>_ovoo + s1[i] s1[b] <ba||ij>_ovvo
// (the last is the s_i^e <mb||ej> s_m^b term of Eq. ccS2).
template <class T>
struct SpR {
  const T *t1, *t2, *Ft, *Ft2, *Vvvvo, *Vovoo, *Vovvo;
  const int16_t* imp;
  const int* list;   // the valid positions (imp >= 0): every warp lane does useful FP64 work
  int nlist;
  int n;
  T* R;
};

template <class T>
__global__ void sp_rinit_kernel(SpR<T> a) {
  const int n = a.n;
  const long long n3 = static_cast<long long>(n) * n * n;
  const long long x = blockIdx.y;
  const T* s1 = a.t1 + x * n;
  const T* s2 = a.t2 + x * n3;
  const T* Ft = a.Ft + x * n;
  const T* Ft2 = a.Ft2 + x * n;
  // positions whose implied index is missing are never read: only the valid
  // list is written (a warp's FP64 instructions cost the pipe for all of its
  // lanes, so a dense loop that skips holes costs as much as one that does not)
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.nlist; c += gridDim.x * blockDim.x) {
    const long long e = a.list[c];
    int i, j, aa;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), i, j, aa);
    const int b = impl(a.imp, n, i, j, aa);
    const long long cb = pos3(n, aa, b, i);  // (a, b, i), j implied
    T h = s2[e] * Ft[b];                       // the four halved terms, scaled once
    h = fma(Ft2[i], s2[pos3(n, j, i, aa)], h);
    h = fma(s1[i], a.Vvvvo[cb], h);
    h = fma(-s1[aa], a.Vovoo[cb], h);
    a.R[x * n3 + e] = fma(T(0.5), h, s1[i] * s1[b] * a.Vovvo[pos3(n, b, aa, i)]);
  }
}

// ---- S2 = P(ij)P(ab) (R + ring) + L + <ab||ij>_vvoo, the ring term held apart
// as Xr[i][a][b] (j implied) when Xr is given, L (antisymmetric, the ladders)
// at the canonical elements when Lc is given
template <class T>
__global__ void sp_s2_kernel(const T* __restrict__ R, const T* __restrict__ Xr, const T* __restrict__ Lc,
                             const T* __restrict__ Vvvoo,
                             const int16_t* __restrict__ imp, const int* __restrict__ canon, int ncanon, int n,
                             T* __restrict__ S2) {
  // one canonical element (i < j, a < b) per thread, written to its four
  // orientations: S2 is exactly antisymmetric (holes of S2 are never read)
  const long long n3 = static_cast<long long>(n) * n * n;
  const long long x = blockIdx.y;
  const T* r = R + x * n3;
  T* s = S2 + x * n3;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncanon; c += gridDim.x * blockDim.x) {
    const int e = canon[c];
    int i, j, aa;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), i, j, aa);
    const int b = imp[e];
    T v = r[e] - r[pos3(n, j, i, aa)] - r[pos3(n, i, j, b)] + r[pos3(n, j, i, b)] + Vvvoo[pos3(n, aa, b, i)];
    if (Xr) {
      const T* xr = Xr + x * n3;
      v += (xr[pos3(n, i, aa, b)] - xr[pos3(n, j, aa, b)]) - (xr[pos3(n, i, b, aa)] - xr[pos3(n, j, b, aa)]);
    }
    if (Lc) v += Lc[x * n3 + e];
    s[e] = v;
    s[pos3(n, j, i, aa)] = -v;
    s[pos3(n, i, j, b)] = -v;
    s[pos3(n, j, i, b)] = v;
  }
}

// The operands the unordered-pair products read, at the canonical positions
// (p0 < p1, p2 < p3 with p3 = imp[p0][p1][p2]) only:
//   ta(i,j,a)  = tau_ij^ab,  tp(a,b,m) = tau_mn^ab,
//   w1(i,j,m)  = (W'_ijmn - W'_jimn)/2 = <mn||ij> - s1[i] <mn||je>_(e=i) + s1[j] <mn||ie>_(e=j),
//   wab(a,b,e) = (W'_abef - W'_baef)/2 = <ab||ef> - s1[a] <ab||ef>_ovvv + s1[b] <ba||ef>_ovvv
template <class T>
struct SpCanon {
  const T *t1, *t2, *Voooo, *Vooov, *Vvvvv, *Vovvv;
  const int16_t* imp;
  const int* canon;
  int ncanon, n;
  T *ta, *tp, *w1, *wab;
};

template <class T>
__global__ void sp_canon_kernel(SpCanon<T> a) {
  const int n = a.n;
  const long long n3 = static_cast<long long>(n) * n * n;
  const long long x = blockIdx.y;
  const T* s1 = a.t1 + x * n;
  const T* s2 = a.t2 + x * n3;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.ncanon; c += gridDim.x * blockDim.x) {
    const int e = a.canon[c];
    int p0, p1, p2;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), p0, p1, p2);
    const int q = a.imp[e];
    const long long o = x * n3 + e;
    {
      T v = s2[e];
      if (p2 == p0) v += s1[p0] * s1[p1];   // (the products only where they enter:
      if (p2 == p1) v -= s1[p0] * s1[p1];   // every FP64 instruction counts here)
      a.ta[o] = v;
    }
    {
      T v = s2[pos3(n, p2, q, p0)];
      if (p0 == p2) v += s1[p2] * s1[q];
      if (p0 == q) v -= s1[p2] * s1[q];
      a.tp[o] = v;
    }
    a.w1[o] = a.Voooo[pos3(n, p2, q, p0)] - s1[p0] * a.Vooov[pos3(n, p2, q, p1)] +
              s1[p1] * a.Vooov[pos3(n, p2, q, p0)];
    a.wab[o] = a.Vvvvv[e] - s1[p0] * a.Vovvv[e] + s1[p1] * a.Vovvv[pos3(n, p1, p0, p2)];
  }
}

// ---- sector products.  For every work item (sector s, row tile, column
// tile) and slice x:
//   C[pos(r, c)] += alpha * sum_{k in K_s} A[rowA(r)][k] * B[rowB(c)][k]
// over the rows r, c of the sector.  Row entries are ordered index pairs
// (p, q); rowA = p n + q, rowB = p n + q, or q n + p with swapB; the output
// position is p_r s0 + q_r s1 + p_c s2 + q_c s3.  A and B are [n^2][n]
// views of N^3 tensors.
// The FP64 pipe bounds these products (a 16-wide padded tile kept it 98 %
// busy with about half of its FMAs on padding), so a CTA takes a tile of
// at most kSecT x kSecT outputs of one sector and assigns only the valid
// ones (flattened, kSecO per thread), and every K chunk runs its exact
// length: no FMA touches padding.
constexpr int kSecT = 48;                      // output tile edge
constexpr int kSecKc = 32;                     // K chunk staged in shared memory
constexpr int kSecThreads = 256;
constexpr int kSecO = (kSecT * kSecT + kSecThreads - 1) / kSecThreads;   // outputs per thread

// TILE x TILE outputs per CTA of THREADS threads: 48 / 256 for the sectors
// of more than 16 pairs, 16 / 64 for the small ones (less staging and
// synchronisation per CTA, more CTAs per SM)
template <class T, int TILE, int THREADS>
__global__ void __launch_bounds__(THREADS) sector_gemm_kernel(SecGemmArgsT<T> g) {
  constexpr int NO = (TILE * TILE + THREADS - 1) / THREADS;
  __shared__ T As[kSecKc][TILE + 1], Bs[kSecKc][TILE + 1];
  const int4 w = g.work[blockIdx.x];
  const int4 sec = g.sec[w.x];   // entry offset, rows, K offset, K count
  const long long x = blockIdx.y;
  const int n = g.n;
  const int nr = min(TILE, sec.y - w.y), nc = min(TILE, sec.y - w.z);
  const int nout = nr * nc;
  T acc[NO];
#pragma unroll
  for (int j = 0; j < NO; ++j) acc[j] = T(0.0);
  for (int prod = 0; prod < (g.A2 ? 2 : 1); ++prod) {
  const T* A = (prod ? g.A2 : g.A) + x * g.ax;
  const T* B = (prod ? g.B2 : g.B) + x * g.bx;
  for (int k0 = 0; k0 < sec.w; k0 += kSecKc) {
    const int kc = min(kSecKc, sec.w - k0);
    // stage A rows [nr][kc] and B rows [nc][kc] (consecutive threads walk a row's K list)
    for (int idx = threadIdx.x; idx < nr * kc; idx += THREADS) {
      const int r = idx / kc, k = idx - r * kc;
      const int2 pr = g.ent[sec.x + w.y + r];
      As[k][r] = A[(static_cast<long long>(pr.x) * n + pr.y) * n + g.kl[sec.z + k0 + k]];
    }
    for (int idx = threadIdx.x; idx < nc * kc; idx += THREADS) {
      const int c = idx / kc, k = idx - c * kc;
      const int2 pr = g.ent[sec.x + w.z + c];
      const long long row = g.swapB ? static_cast<long long>(pr.y) * n + pr.x : static_cast<long long>(pr.x) * n + pr.y;
      Bs[k][c] = B[row * n + g.kl[sec.z + k0 + k]];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      const int o = threadIdx.x + j * THREADS;
      if (o < nout) {
        const int r = o / nc, c = o - r * nc;
        T a = acc[j];
        for (int k = 0; k < kc; ++k) a = As[k][r] * Bs[k][c] + a;
        acc[j] = a;
      }
    }
    __syncthreads();
  }
  }
#pragma unroll
  for (int j = 0; j < NO; ++j) {
    const int o = threadIdx.x + j * THREADS;
    if (o < nout) {
      const int r = o / nc, c = o - r * nc;
      const int2 pr = g.ent[sec.x + w.y + r], pc = g.ent[sec.x + w.z + c];
      const T v = g.alpha * acc[j];
      if (g.anti4) {
        // (i, j) = pr, (a, b) = pc: the four orientations of the antisymmetric result
        T* C = g.C + x * g.cx;
        const long long ni = pr.x, nj = pr.y;
        C[(ni * n + nj) * n + pc.x] += v;
        C[(nj * n + ni) * n + pc.x] -= v;
        C[(ni * n + nj) * n + pc.y] -= v;
        C[(nj * n + ni) * n + pc.y] += v;
      } else {
        const long long q = x * g.cx + static_cast<long long>(pr.x) * g.s0 + static_cast<long long>(pr.y) * g.s1 +
                            static_cast<long long>(pc.x) * g.s2 + static_cast<long long>(pc.y) * g.s3;
        if (g.store) g.C[q] = v;
        else g.C[q] += v;
      }
    }
  }
}

// FP32 form of the same products.  The FP32 pipe issues 64 times the FP64
// rate, so the flattened kernel above is bound there by its staging (index
// arithmetic per element, and global-load latency between two barriers).
// This one
//  * gives each thread a 4 x 4 block of the TILE x TILE tile (rows 4 ty ..
//    4 ty + 3, columns 4 tx .. 4 tx + 3): one float4 of each operand per k
//    feeds 16 FMAs;
//  * keeps the row offsets of the tile in shared memory and gives every
//    staging thread one fixed k of a chunk, so an element costs an address
//    add and an asynchronous copy (cp.async, 4 bytes);
//  * stages chunk c + 1 while chunk c is multiplied (two buffers).
// A warp stages 8 consecutive k of 4 rows at a time: its four row segments
// are contiguous stretches of a row's K list, and its shared stores fall in
// 32 distinct banks (row pitch TILE + 4 words).  Outputs past the sector's
// edge are computed from whatever the unstaged rows hold and never written.
// Every output sums its k terms in the order of the flattened kernel (fma
// into one accumulator, chunk after chunk, the second product after the
// first).
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <int TILE>
__global__ void __launch_bounds__((TILE / 4) * (TILE / 4)) sector_gemm_f32_kernel(SecGemmArgsT<float> g) {
  constexpr int TD = TILE / 4, THREADS = TD * TD, LD = TILE + 4;
  static_assert(THREADS >= 4 * 32 && kSecKc == 32, "four staging warps cover a 32-wide K chunk");
  __shared__ __align__(16) float As[2][kSecKc][LD];
  __shared__ __align__(16) float Bs[2][kSecKc][LD];
  __shared__ int rowA[TILE], rowB[TILE];
  const int4 w = g.work[blockIdx.x];
  const int4 sec = g.sec[w.x];   // entry offset, rows, K offset, K count
  const long long x = blockIdx.y;
  const int n = g.n;
  const int nr = min(TILE, sec.y - w.y), nc = min(TILE, sec.y - w.z);
  for (int r = threadIdx.x; r < nr; r += THREADS) {
    const int2 pr = g.ent[sec.x + w.y + r];
    rowA[r] = (pr.x * n + pr.y) * n;
  }
  for (int c = threadIdx.x; c < nc; c += THREADS) {
    const int2 pr = g.ent[sec.x + w.z + c];
    rowB[c] = (g.swapB ? pr.y * n + pr.x : pr.x * n + pr.y) * n;
  }
  __syncthreads();
  const int nch = (sec.w + kSecKc - 1) / kSecKc;
  const int nchunk = nch * (g.A2 ? 2 : 1);
  const int lane = threadIdx.x & 31;
  const int sk = (lane >> 2) + 8 * (threadIdx.x >> 5), sr = lane & 3;   // staging: k of the chunk, first row
  auto stage = [&](int ci, int buf) {
    if (threadIdx.x >= 128) return;
    const int prod = ci >= nch ? 1 : 0;
    const int k0 = (ci - prod * nch) * kSecKc;
    if (sk >= sec.w - k0) return;
    const float* A = (prod ? g.A2 : g.A) + x * g.ax;
    const float* B = (prod ? g.B2 : g.B) + x * g.bx;
    const int col = g.kl[sec.z + k0 + sk];
    for (int r = sr; r < nr; r += 4) cp_async4(&As[buf][sk][r], A + rowA[r] + col);
    for (int c = sr; c < nc; c += 4) cp_async4(&Bs[buf][sk][c], B + rowB[c] + col);
  };
  const int tx = threadIdx.x % TD, ty = threadIdx.x / TD;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  stage(0, 0);
  cp_async_commit();
  for (int ci = 0; ci < nchunk; ++ci) {
    if (ci + 1 < nchunk) stage(ci + 1, (ci + 1) & 1);
    cp_async_commit();
    cp_async_wait1();   // every group but the newest: chunk ci has landed
    __syncthreads();
    const int prod = ci >= nch ? 1 : 0;
    const int kc = min(kSecKc, sec.w - (ci - prod * nch) * kSecKc);
    const int buf = ci & 1;
    for (int k = 0; k < kc; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&As[buf][k][4 * ty]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][k][4 * tx]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();   // buffer ci & 1 is restaged for chunk ci + 2
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = 4 * ty + i;
    if (r >= nr) continue;
    const int2 pr = g.ent[sec.x + w.y + r];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 4 * tx + j;
      if (c >= nc) continue;
      const int2 pc = g.ent[sec.x + w.z + c];
      const float v = g.alpha * acc[i][j];
      if (g.anti4) {
        float* C = g.C + x * g.cx;
        const long long ni = pr.x, nj = pr.y;
        C[(ni * n + nj) * n + pc.x] += v;
        C[(nj * n + ni) * n + pc.x] -= v;
        C[(ni * n + nj) * n + pc.y] -= v;
        C[(nj * n + ni) * n + pc.y] += v;
      } else {
        const long long q = x * g.cx + static_cast<long long>(pr.x) * g.s0 + static_cast<long long>(pr.y) * g.s1 +
                            static_cast<long long>(pc.x) * g.s2 + static_cast<long long>(pc.y) * g.s3;
        if (g.store) g.C[q] = v;
        else g.C[q] += v;
      }
    }
  }
}

// ---- storage conversions
// Thermal integral block of class (c0 c1 c2 c3) in N^3 storage:
// out[p][q][r] = <pq||rs> f0[p] f1[q] f2[r] f3[s], s implied (0 where none).
template <class T>
__global__ void sp_thermal_eri_kernel(const double* __restrict__ eri, const int16_t* __restrict__ imp, int n,
                                      const double* f0, const double* f1, const double* f2, const double* f3,
                                      T* __restrict__ out) {
  const long long n3 = static_cast<long long>(n) * n * n;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n3;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    int p, q, r;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), p, q, r);
    const int s = imp[e];
    out[e] = static_cast<T>(s >= 0 ? eri[e * n + s] * f0[p] * f1[q] * f2[r] * f3[s] : 0.0);
  }
}

// out[p0][p1][p2] = in[p0][p2][p1] (a hole of one is a hole of the other)
template <class T>
__global__ void sp_swap12_kernel(const T* __restrict__ in, int n, T* __restrict__ out) {
  const long long n3 = static_cast<long long>(n) * n * n;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n3;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    int p0, p1, p2;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), p0, p1, p2);
    out[e] = in[pos3(n, p0, p2, p1)];
  }
}

// diagonal of a thermal Fock block: out[p] = fbar[p][p] f0[p] f1[p]
template <class T>
__global__ void sp_thermal_fock_kernel(const double* __restrict__ fbar, int n, const double* f0, const double* f1,
                                       T* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) out[p] = static_cast<T>(fbar[static_cast<long long>(p) * n + p] * f0[p] * f1[p]);
}

// dense [x][i][j][a][b] / [x][i][a] <-> N^3 [x][i][j][a] / vector [x][i]
__global__ void sp_compress_kernel(const double* __restrict__ d1, const double* __restrict__ d2,
                                   const int16_t* __restrict__ imp, int n, double* __restrict__ s1,
                                   double* __restrict__ s2) {
  const long long n3 = static_cast<long long>(n) * n * n;
  const long long x = blockIdx.y;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n3;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int b = imp[e];
    s2[x * n3 + e] = b >= 0 ? d2[(x * n3 + e) * n + b] : 0.0;
    if (e < n) s1[x * n + e] = d1[(x * n + e) * n + e];
  }
}

__global__ void sp_expand_kernel(const double* __restrict__ s1, const double* __restrict__ s2,
                                 const int16_t* __restrict__ imp, int n, double* __restrict__ d1,
                                 double* __restrict__ d2) {
  const long long n3 = static_cast<long long>(n) * n * n;
  const long long x = blockIdx.y;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n3 * n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long t = e / n;
    const int b = static_cast<int>(e % n);
    d2[x * n3 * n + e] = imp[t] == b ? s2[x * n3 + t] : 0.0;
    if (e < static_cast<long long>(n) * n) {
      const int i = static_cast<int>(e / n), a = static_cast<int>(e % n);
      d1[x * n * n + e] = i == a ? s1[x * n + i] : 0.0;
    }
  }
}

}  // namespace

// ============================================================ transpose (VJP)
// The lambda equations need the transpose of the S kernel: given the
// cotangents S1b, S2b of S1, S2 (per slice), the cotangents of s1, s2 and
// (for the response) of the integral and Fock blocks.  The forward
// intermediates are recomputed first; each forward step is then transposed
// in reverse order.  Vector quantities (the two-index factors) are
// reductions per orbital, element-wise contributions are written in gather
// form (each output element sums what reaches it), so nothing is written by
// two threads and the sums have a fixed order.
namespace {

// Rb = P(ij)P(ab) S2b (the antisymmetriser is its own transpose)
// (over the valid positions only: the holes of Rb are never read)
__global__ void sp_s2_t_kernel(const double* __restrict__ S2b, const int16_t* __restrict__ imp,
                               const int* __restrict__ list, int nlist, int n, double* __restrict__ Rb) {
  const long long n3 = static_cast<long long>(n) * n * n;
  const long long x = blockIdx.y;
  const double* g = S2b + x * n3;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nlist; c += gridDim.x * blockDim.x) {
    const long long e = list[c];
    int i, j, aa;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), i, j, aa);
    const int b = impl(imp, n, i, j, aa);
    Rb[x * n3 + e] = g[e] - g[pos3(n, j, i, aa)] - g[pos3(n, i, j, b)] + g[pos3(n, j, i, b)];
  }
}

// Element-wise transposes, gathered at the s2 position (i, j, a), b implied:
//   from R's terms:   1/2 Rb(ija) Ft[b] + 1/2 Ft2[j] Rb(jia)
//   from S1 and F:    [a = i] S1b[i] Fme[j] - 1/2 S1b[i] <ji||ab>_ovvv(j,i,a) + 1/2 Fmib[i] <ij||ab>_oovv
//                     - 1/2 S1b[a] <ji||bi'>_oovo(j,i,b) - 1/2 Faeb[a] <ij||ab>_oovv
//   from the operands: tab(ija) + tpb(a b i) + trb(i a j) + 1/2 xpb(i b j)
struct SpT2 {
  const double *t1, *Rb, *Ft, *Ft2, *S1b, *Fme, *Fmib, *Faeb, *tab, *tpb, *trb, *xpb;
  const double *Vovvv, *Voovv, *Voovo;
  const int16_t* imp;
  const int* list;   // valid positions (the holes of t2b are zero from the start and stay so)
  int nlist;
  int n;
  double* t2b;
};

__global__ void sp_t2bar_kernel(SpT2 a) {
  const int n = a.n;
  const long long n3 = static_cast<long long>(n) * n * n;
  const long long x = blockIdx.y;
  const double* Rb = a.Rb + x * n3;
  const double* Ft = a.Ft + x * n;
  const double* Ft2 = a.Ft2 + x * n;
  const double* S1b = a.S1b + x * n;
  const double* Fme = a.Fme + x * n;
  const double* Fmib = a.Fmib + x * n;
  const double* Faeb = a.Faeb + x * n;
  const double* tab = a.tab + x * n3;
  const double* tpb = a.tpb + x * n3;
  const double* trb = a.trb + x * n3;
  const double* xpb = a.xpb + x * n3;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.nlist; c += gridDim.x * blockDim.x) {
    const long long e = a.list[c];
    int i, j, aa;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), i, j, aa);
    const int b = impl(a.imp, n, i, j, aa);
    double v = 0.0;
    if (b >= 0) {
      // the halved terms summed first and scaled once (FP64 instructions
      // are the cost here)
      double hsum = Rb[e] * Ft[b];
      hsum = fma(Ft2[j], Rb[pos3(n, j, i, aa)], hsum);
      hsum = fma(-S1b[i], a.Vovvv[pos3(n, j, i, aa)], hsum);
      hsum = fma(Fmib[i] - Faeb[aa], a.Voovv[e], hsum);
      hsum = fma(-S1b[aa], a.Voovo[pos3(n, j, i, b)], hsum);
      hsum += xpb[pos3(n, i, b, j)];
      v = fma(0.5, hsum, tab[e] + tpb[pos3(n, aa, b, i)] + trb[pos3(n, i, aa, j)]);
      if (aa == i) v += S1b[i] * Fme[j];
    }
    a.t2b[x * n3 + e] = v;
  }
}

// Vector cotangents of one (x, p), in two passes.
// Pass 1: Ftb[p], Ft2b[p] (from R's terms), Faeb[p], Fmib[p], Fmeb[p].
//   Ftb[b]  = 1/2 sum_ij Rb(i,j,a) s2(i,j,a),  a = imp(i,j,b)
//   Ft2b[i] = 1/2 sum_ja Rb(i,j,a) s2(j,i,a)
//   Faeb = Ftb + S1b s1,  Fmib = Ft2b - S1b s1
//   Fmeb[m] = s1[m] (-Ftb + Ft2b - Faeb + Fmib)[m] / 2 + sum_p S1b[p] s2(p,m,p)
struct SpVecT {
  const double *t1, *t2, *Rb, *S1b, *Fme, *Fae, *Fmi;
  const double *Vvvvo, *Vovvo, *Vovoo, *Vooov, *Vovvv, *Voovo, *Vovov, *Voovv;
  const double *w1b, *wabb, *wrb, *tab, *tpb, *xpb;
  const int16_t* imp;
  const int *l1, *off1, *l2, *off2;   // valid (m, q) = m n + q of (m, q, p) / (p, m, q) per p
  int n;
  double *Ftb, *Ft2b, *Faeb, *Fmib, *Fmeb, *t1b;
};

__global__ void sp_vec_t1_kernel(SpVecT a) {
  __shared__ double red[3 * 32];
  const int n = a.n;
  const long long n3 = static_cast<long long>(n) * n * n;
  const int p = blockIdx.x, x = blockIdx.y;
  const double* s2 = a.t2 + x * n3;
  const double* Rb = a.Rb + x * n3;
  const double* S1b = a.S1b + static_cast<long long>(x) * n;
  double ftb = 0.0, ft2b = 0.0, fme = 0.0;
  // only the valid positions (the rest of Rb and s2 is zero): (u, w, a) with
  // a = imp(u, w, p) from p's list l1, (p, u, w) from l2
  for (int k = a.off1[p] + threadIdx.x; k < a.off1[p + 1]; k += blockDim.x) {
    const int uw = a.l1[k];
    const int u = uw / n, w = uw - u * n;
    const int aa = impl(a.imp, n, u, w, p);                    // (i, j, a) = (u, w, aa), b = p
    const long long o = pos3(n, u, w, aa);
    ftb += Rb[o] * s2[o];
  }
  for (int k = a.off2[p] + threadIdx.x; k < a.off2[p + 1]; k += blockDim.x) {
    const int uw = a.l2[k];
    const int u = uw / n, w = uw - u * n;
    ft2b += Rb[pos3(n, p, u, w)] * s2[pos3(n, u, p, w)];     // (i, j, a) = (p, u, w)
  }
  for (int q = threadIdx.x; q < n; q += blockDim.x) fme += S1b[q] * s2[pos3(n, q, p, q)];
  double sums[3] = {ftb, ft2b, fme};
  block_sums(sums, red);
  ftb = sums[0];
  ft2b = sums[1];
  fme = sums[2];
  if (threadIdx.x == 0) {
    const long long o = static_cast<long long>(x) * n + p;
    const double s = a.t1[o];
    const double Ftb = 0.5 * ftb, Ft2b = 0.5 * ft2b;
    const double Faeb = Ftb + S1b[p] * s, Fmib = Ft2b - S1b[p] * s;
    a.Ftb[o] = Ftb;
    a.Ft2b[o] = Ft2b;
    a.Faeb[o] = Faeb;
    a.Fmib[o] = Fmib;
    a.Fmeb[o] = 0.5 * s * (-Ftb + Ft2b - Faeb + Fmib) + fme;
  }
}

// Pass 2: the cotangent of s1[p], every contribution:
//   R's terms (p as i, a, b), the W bases (p as i of W_mnij, a of W_abef,
//   j and b of W_mbej), the vector intermediates and S1, and the s1 s1
//   parts of tau, X and the ladder operand.
__global__ void sp_vec_t2_kernel(SpVecT a) {
  __shared__ double red[32];
  const int n = a.n;
  const long long n3 = static_cast<long long>(n) * n * n;
  const int p = blockIdx.x, x = blockIdx.y;
  const double* s1 = a.t1 + static_cast<long long>(x) * n;
  const double* Rb = a.Rb + x * n3;
  const double* w1b = a.w1b + x * n3;
  const double* wabb = a.wabb + x * n3;
  const double* wrb = a.wrb + x * n3;
  const double* tab = a.tab + x * n3;
  const double* tpb = a.tpb + x * n3;
  const double* xpb = a.xpb + x * n3;
  const double* S1b = a.S1b + static_cast<long long>(x) * n;
  const double* Faeb = a.Faeb + static_cast<long long>(x) * n;
  const double* Fmib = a.Fmib + static_cast<long long>(x) * n;
  const double* Fmeb = a.Fmeb + static_cast<long long>(x) * n;
  double acc = 0.0, acch = 0.0, acc2 = 0.0;   // terms of weight 1, 1/2 and -2, scaled once at the end
  // every term below vanishes unless its implied index exists: the terms
  // with a valid (p, u, w) run over p's list l2, those with a valid (u, w, p)
  // over l1, the one with a valid (p, w, u) over l2 with the pair swapped
  for (int k = a.off2[p] + threadIdx.x; k < a.off2[p + 1]; k += blockDim.x) {
    const int uw = a.l2[k];
    const int u = uw / n, w = uw - u * n;
    const long long o = pos3(n, p, u, w);
    const int b = a.imp[o];   // b (R, p as i), n (W'_mnij, p as i), e (W_mbej, p as b)
    const double g = Rb[o];
    // R: p as i, (j, a) = (u, w), b = imp(p, u, w)
    acch = fma(g, a.Vvvvo[pos3(n, w, b, p)], acch);
    acc = fma(g * s1[b], a.Vovvo[pos3(n, b, w, p)], acc);
    // W'_mnij base: p as i, (j, m) = (u, w), n = imp(p, u, w)
    acc2 = fma(w1b[o], a.Vooov[pos3(n, w, b, u)], acc2);
    // W'_abef base: p as a, (b, e) = (u, w)
    acc2 = fma(wabb[o], a.Vovvv[o], acc2);
    // W_mbej base, p as b: (j, m) = (w, u) here, e = imp(p, u, w)
    acc = fma(-wrb[pos3(n, w, p, u)], a.Voovo[pos3(n, u, p, b)], acc);
  }
  for (int k = a.off1[p] + threadIdx.x; k < a.off1[p + 1]; k += blockDim.x) {
    const int uw = a.l1[k];
    const int u = uw / n, w = uw - u * n;
    const int c = impl(a.imp, n, u, w, p);   // b (p as a), a (p as b), e (p as j)
    // R: p as a, (i, j) = (u, w), b = imp(u, w, p)
    acch = fma(-Rb[pos3(n, u, w, p)], a.Vovoo[pos3(n, p, c, u)], acch);
    // R: p as b, (i, j) = (u, w), a = imp(u, w, p)
    acc = fma(Rb[pos3(n, u, w, c)] * s1[u], a.Vovvo[pos3(n, p, c, u)], acc);
    // W_mbej base, p as j: (b, m) = (u, w), e = imp(u, w, p)
    acc = fma(wrb[pos3(n, p, u, w)], a.Vovvv[pos3(n, w, u, c)], acc);
  }
  acc = fma(0.5, acch, fma(-2.0, acc2, acc));
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    // S1 and the F intermediates
    acc += -S1b[q] * a.Vovov[pos3(n, p, q, q)] + Faeb[q] * a.Vovvv[pos3(n, p, q, p)] +
           Fmib[q] * a.Vooov[pos3(n, q, p, q)] + Fmeb[q] * a.Voovv[pos3(n, q, p, q)];
    // s1 s1 parts of tau (ta), of the ladder operand (tp) and of X (xp)
    acc += s1[q] * (tab[pos3(n, p, q, p)] - tab[pos3(n, p, q, q)] + tab[pos3(n, q, p, q)] - tab[pos3(n, q, p, p)] +
                    tpb[pos3(n, p, q, p)] - tpb[pos3(n, p, q, q)] + tpb[pos3(n, q, p, q)] - tpb[pos3(n, q, p, p)] +
                    xpb[pos3(n, p, q, q)] + xpb[pos3(n, q, p, p)]);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) {
    const long long o = static_cast<long long>(x) * n + p;
    const double fm = a.Fme[o], Ftb = a.Ftb[o], Ft2b = a.Ft2b[o];
    acc += 0.5 * fm * (-Ftb + Ft2b - Faeb[p] + Fmib[p]) + S1b[p] * (a.Fae[o] - a.Fmi[o]);
    a.t1b[o] = acc;
  }
}

// Transposed sector products:
//   D[orow(e_o)][k] += alpha sum_{e_s in sector} G[gpos(e_o, e_s)] A[srow(e_s)][k]
// for the pairs e_o of the sector (rows) and k of its K list; orow / srow
// are p n + q or (swapped) q n + p; gpos = p_o g0 + q_o g1 + p_s g2 + q_s g3.
// With dx = 0 the output is fixed (an integral block) and the kernel sums
// the nx slices of G and A itself.
// TILE x TILE outputs per CTA of THREADS threads (48 / 256 for the sectors
// of more than 16 pairs, 16 / 64 for the small ones, as in the forward)
template <int TILE, int THREADS>
__global__ void __launch_bounds__(THREADS) sector_tn_kernel(SecTnArgs g) {
  constexpr int NO = (TILE * TILE + THREADS - 1) / THREADS;
  __shared__ double Gs[kSecKc][TILE + 1], As[kSecKc][TILE + 1];
  const int4 w = g.work[blockIdx.x];
  const int4 sec = g.sec[w.x];
  const int n = g.n;
  const int no_ = min(TILE, sec.y - w.y), nk = min(TILE, sec.w - w.z);   // output rows, k columns
  const int nout = no_ * nk;
  const int xr0 = g.dx ? blockIdx.y : 0, xr1 = g.dx ? blockIdx.y + 1 : g.nx;
  double acc[NO];
#pragma unroll
  for (int j = 0; j < NO; ++j) acc[j] = 0.0;
  for (int x = xr0; x < xr1; ++x) {
    const double* G = g.G + x * g.gx;
    const double* A = g.A + x * g.ax;
    for (int s0 = 0; s0 < sec.y; s0 += kSecKc) {
      const int sc = min(kSecKc, sec.y - s0);
      // Gs[s][o] = G(output row o, summed row s), As[s][k] = A(summed row s, column k)
      for (int idx = threadIdx.x; idx < no_ * sc; idx += THREADS) {
        const int o = idx / sc, ss = idx - o * sc;
        const int2 po = g.ent[sec.x + w.y + o], ps = g.ent[sec.x + s0 + ss];
        Gs[ss][o] = G[static_cast<long long>(po.x) * g.g0 + static_cast<long long>(po.y) * g.g1 +
                      static_cast<long long>(ps.x) * g.g2 + static_cast<long long>(ps.y) * g.g3];
      }
      for (int idx = threadIdx.x; idx < nk * sc; idx += THREADS) {
        const int ss = idx / nk, k = idx - ss * nk;
        const int2 ps = g.ent[sec.x + s0 + ss];
        const long long srow = g.swapA ? static_cast<long long>(ps.y) * n + ps.x : static_cast<long long>(ps.x) * n + ps.y;
        const int col = g.kl[sec.z + w.z + k];
        double v = A[srow * n + col];
        if (g.antiA) {
          const long long srw = g.swapA ? static_cast<long long>(ps.x) * n + ps.y : static_cast<long long>(ps.y) * n + ps.x;
          v = 0.5 * (v - A[srw * n + col]);
        }
        As[ss][k] = v;
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        const int o = threadIdx.x + j * THREADS;
        if (o < nout) {
          const int r = o / nk, k = o - r * nk;
          double a = acc[j];
          for (int ss = 0; ss < sc; ++ss) a = fma(Gs[ss][r], As[ss][k], a);
          acc[j] = a;
        }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int j = 0; j < NO; ++j) {
    const int o = threadIdx.x + j * THREADS;
    if (o < nout) {
      const int r = o / nk, k = o - r * nk;
      const int2 pr = g.ent[sec.x + w.y + r];
      const long long orow = g.swapD ? static_cast<long long>(pr.y) * n + pr.x : static_cast<long long>(pr.x) * n + pr.y;
      const long long base = g.dx ? static_cast<long long>(blockIdx.y) * g.dx : 0;
      const double v = g.alpha * acc[j];
      if (g.anti4) {
        const int2 pk = g.ent[sec.z + w.z + k];   // (k, l)
        const long long r1 = static_cast<long long>(pr.x) * n + pr.y, r2 = static_cast<long long>(pr.y) * n + pr.x;
        g.D[base + r1 * n + pk.x] += v;
        g.D[base + r2 * n + pk.x] -= v;
        g.D[base + r1 * n + pk.y] -= v;
        g.D[base + r2 * n + pk.y] += v;
      } else {
        g.D[base + orow * n + g.kl[sec.z + w.z + k]] += v;
      }
    }
  }
}

}  // namespace

namespace {

// Cotangents of the integral blocks from the element-wise uses (summed over
// the nx slices; blockIdx.y = block: 0 oovv, 1 ovvv, 2 ooov, 3 oooo,
// 4 vvvv, 5 ovvo, 6 oovo, 7 ovov, 8 vvoo, 9 vvvo, 10 ovoo), at the block
// position (p, q, r), s = imp[p][q][r].  With cz (the energy weights g_x /
// beta) the direct use of <ij||ab> in Eq. E is added to oovv.  The products
// of two four-index factors add theirs through sector_tn_kernel.
struct SpFixT {
  const double *t1, *t2, *S2b, *Rb, *w1b, *wabb, *wrb, *S1b, *Faeb, *Fmib, *Fmeb, *cz;
  const int16_t* imp;
  const int* list;   // valid positions of the blocks
  int nlist;
  int n, nx;
  double* Vb[11];
};

__global__ void sp_fixed_bar_kernel(SpFixT a) {
  const int n = a.n;
  const long long n3 = static_cast<long long>(n) * n * n;
  const int blk = blockIdx.y;
  double* out = a.Vb[blk];
  if (!out) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.nlist; c += gridDim.x * blockDim.x) {
    const long long e = a.list[c];
    const int sl = a.imp[e];
    int p, q, r;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), p, q, r);
    double v = 0.0;
    for (int x = 0; x < a.nx; ++x) {
      const double* s1 = a.t1 + static_cast<long long>(x) * n;
      const double* s2 = a.t2 + x * n3;
      const double* S2b = a.S2b + x * n3;
      const double* Rb = a.Rb + x * n3;
      const double* w1b = a.w1b + x * n3;
      const double* wabb = a.wabb + x * n3;
      const double* wrb = a.wrb + x * n3;
      const double* S1b = a.S1b + static_cast<long long>(x) * n;
      const double* Faeb = a.Faeb + static_cast<long long>(x) * n;
      const double* Fmib = a.Fmib + static_cast<long long>(x) * n;
      const double* Fmeb = a.Fmeb + static_cast<long long>(x) * n;
      switch (blk) {
        case 0:   // oovv (m, q, e) [f]
          v += -0.5 * Faeb[r] * s2[e] + 0.5 * Fmib[p] * s2[e];
          if (r == p) v += Fmeb[p] * s1[q];
          if (a.cz) {
            v += a.cz[x] * 0.25 * s2[e];
            if (r == p) v += a.cz[x] * 0.5 * s1[p] * s1[q];
          }
          break;
        case 1:   // ovvv (m, b, e) [f]
          v += -2.0 * s1[p] * wabb[e] + s1[sl] * wrb[pos3(n, sl, q, p)] - 0.5 * S1b[q] * s2[pos3(n, q, p, r)];
          if (r == p) v += Faeb[q] * s1[p];
          break;
        case 2:   // ooov (m, n, j) [i]
          v += -2.0 * s1[sl] * w1b[pos3(n, sl, r, p)];
          if (r == p) v += Fmib[p] * s1[q];
          break;
        case 3:   // oooo (m, n, i) [j]
          v += w1b[pos3(n, r, sl, p)];
          break;
        case 4:   // vvvv
          v += wabb[e];
          break;
        case 5:   // ovvo (b, a, i) [j] from R; (m, b, e) [j] from W_mbej
          v += s1[r] * s1[p] * Rb[pos3(n, r, sl, q)] + wrb[pos3(n, sl, q, p)];
          break;
        case 6:   // oovo (m, b, e) [j] from W_mbej; (q', m', e') [p'] from S1
          v += -s1[q] * wrb[pos3(n, sl, q, p)] - 0.5 * S1b[sl] * s2[pos3(n, q, p, sl)];
          break;
        case 7:   // ovov (m, p', p') [m]
          if (q == r) v += -S1b[q] * s1[p];
          break;
        case 8:   // vvoo (a, b, i) [j]
          v += S2b[pos3(n, r, sl, p)];
          break;
        case 9:   // vvvo (a, b, i) [j]
          v += 0.5 * s1[r] * Rb[pos3(n, r, sl, p)];
          break;
        default:  // ovoo (a, b, i) [j]
          v += -0.5 * s1[p] * Rb[pos3(n, r, sl, p)];
          break;
      }
    }
    out[e] += v;
  }
}

// Fock-diagonal cotangents summed over the slices: fov += Fmeb (+ the
// energy's sum_x cz[x] s1), fvv += Faeb, foo += Fmib, fvo += S1b
__global__ void sp_fock_bar_kernel(const double* __restrict__ t1, const double* __restrict__ Fmeb,
                                   const double* __restrict__ Faeb, const double* __restrict__ Fmib,
                                   const double* __restrict__ S1b, const double* __restrict__ cz, int n, int nx,
                                   double* fov, double* fvv, double* foo, double* fvo) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for (int x = 0; x < nx; ++x) {
    const long long o = static_cast<long long>(x) * n + p;
    a0 += Fmeb[o] + (cz ? cz[x] * t1[o] : 0.0);
    a1 += Faeb[o];
    a2 += Fmib[o];
    a3 += S1b[o];
  }
  if (fov) fov[p] += a0;
  if (fvv) fvv[p] += a1;
  if (foo) foo[p] += a2;
  if (fvo) fvo[p] += a3;
}

// out[p0][p1][p2] += in[p0][p2][p1]
__global__ void sp_swap12_add_kernel(const double* __restrict__ in, int n, double* __restrict__ out) {
  const long long n3 = static_cast<long long>(n) * n * n;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n3;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    int p0, p1, p2;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), p0, p1, p2);
    out[e] += in[pos3(n, p0, p2, p1)];
  }
}

}  // namespace

namespace {

// Direct dependence of Omega_CC = sum_x cz[x] E_x on the energy weights
// (Eq. E): <ij||ab>bar += sum_x cz[x] (1/4 s2 + 1/2 [a = i] s1[i] s1[j]),
// f_ia bar (diagonal) += sum_x cz[x] s1
__global__ void sp_energy_bar_kernel(const double* __restrict__ t1, const double* __restrict__ t2,
                                     const double* __restrict__ cz, const int16_t* __restrict__ imp, int n, int ng,
                                     double* __restrict__ Voovvb, double* __restrict__ fovb) {
  const long long n3 = static_cast<long long>(n) * n * n;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n3;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    if (e < n) {   // the diagonal f_ia (before the hole test: e indexes an orbital here)
      double f = 0.0;
      for (int x = 0; x < ng; ++x) f += cz[x] * t1[static_cast<long long>(x) * n + e];
      fovb[e] += f;
    }
    if (imp[e] < 0) continue;
    int i, j, aa;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), i, j, aa);
    double v = 0.0;
    for (int x = 0; x < ng; ++x) {
      v += cz[x] * 0.25 * t2[x * n3 + e];
      if (aa == i) v += cz[x] * 0.5 * t1[static_cast<long long>(x) * n + i] * t1[static_cast<long long>(x) * n + j];
    }
    Voovvb[e] += v;
  }
}

// Per-orbital sums of I * Ibar over the elements of an N^3 block whose slot
// k (the implied fourth slot included) is orbital q, added to Do[q] for a
// hole-like slot (bit k of cls clear) or Dv[q] (set).  One block per q.
__global__ void sp_slot_sums_kernel(const double* __restrict__ I, const double* __restrict__ Ib,
                                    const int16_t* __restrict__ imp, int n, int cls, double* __restrict__ Do,
                                    double* __restrict__ Dv) {
  __shared__ double red[32];
  const int q = blockIdx.x;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long nn = static_cast<long long>(n) * n;
  for (uint32_t r = threadIdx.x; r < static_cast<uint32_t>(nn); r += blockDim.x) {
    const int u = static_cast<int>(r / static_cast<uint32_t>(n)), w = static_cast<int>(r - static_cast<uint32_t>(u) * n);
    long long e = pos3(n, q, u, w);
    acc[0] += I[e] * Ib[e];
    e = pos3(n, u, q, w);
    acc[1] += I[e] * Ib[e];
    e = pos3(n, u, w, q);
    acc[2] += I[e] * Ib[e];
    const int rr = impl(imp, n, u, w, q);   // (u, w, rr) has q implied
    if (rr >= 0) {
      e = pos3(n, u, w, rr);
      acc[3] += I[e] * Ib[e];
    }
  }
  double so = 0.0, sv = 0.0;
  for (int k = 0; k < 4; ++k) {
    const double t = block_sum(acc[k], red);
    if (threadIdx.x == 0) {
      if (cls & (1 << k)) sv += t;
      else so += t;
    }
  }
  if (threadIdx.x == 0) {
    Do[q] += so;
    Dv[q] += sv;
  }
}

}  // namespace

namespace {

// gamma[p][q][r][s] += bar[p][q][r] f0[p] f1[q] f2[r] f3[s], s implied: the
// cotangent of one thermal block mapped back to <pq||rs> (N^4, dense)
__global__ void sp_eri_adjoint_kernel(const double* __restrict__ bar, const int16_t* __restrict__ imp, int n,
                                      const double* f0, const double* f1, const double* f2, const double* f3,
                                      double* __restrict__ gamma) {
  const long long n3 = static_cast<long long>(n) * n * n;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n3;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int s = imp[e];
    if (s < 0) continue;
    int p, q, r;
    dec3(static_cast<uint32_t>(e), static_cast<uint32_t>(n), p, q, r);
    gamma[e * n + s] += bar[e] * f0[p] * f1[q] * f2[r] * f3[s];
  }
}

}  // namespace

// ------------------------------------------------------------------ launchers
template <class T>
cudaError_t launch_sp_amp(const T* t1, const T* t2, const int16_t* imp, int n, int nx, T* ta, T* tp, T* tr, T* xp,
                          int skip_tau, const int* list, int nlist, cudaStream_t st) {
  const long long n3 = static_cast<long long>(n) * n * n;
  sp_amp_kernel<T><<<dim3(sp_grid(list ? nlist : n3), nx), kSpThreads, 0, st>>>(t1, t2, imp, n, ta, tp, tr, xp,
                                                                                skip_tau, list, nlist);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_sp_canon(const T* t1, const T* t2, const SpBlocksT<T>& V, const int16_t* imp, const int* canon,
                            int ncanon, int n, int nx, T* ta, T* tp, T* w1, T* wab, cudaStream_t st) {
  SpCanon<T> a{t1, t2, V.oooo, V.ooov, V.vvvv, V.ovvv, imp, canon, ncanon, n, ta, tp, w1, wab};
  sp_canon_kernel<T><<<dim3(sp_grid(ncanon), nx), kSpThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_sp_vectors(const SpVecArgsT<T>& v, int nx, cudaStream_t st) {
  const int warps = v.n * nx;
  sp_fme_kernel<T><<<(warps * 32 + 127) / 128, 128, 0, st>>>(v.t1, v.fov, v.Voovv, v.n, nx, v.Fme);
  SpVec<T> a{v.t1, v.t2, v.Fme, v.foo, v.fvv, v.fvo, v.Voovv, v.Vovvv, v.Vooov, v.Vovov, v.Voovo, v.imp,
             v.l1, v.off1, v.l2, v.off2, v.n, v.Fae, v.Fmi, v.S1, v.Ft, v.Ft2};
  sp_vec_kernel<T><<<dim3(v.n, nx), 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_sp_wbase(const T* t1, const SpBlocksT<T>& V, const int16_t* imp, int n, int nx, T* w1, T* wab,
                            T* wr, int anti, const int* list, int nlist, cudaStream_t st) {
  const long long n3 = static_cast<long long>(n) * n * n;
  SpW<T> a{t1, V.oooo, V.ooov, V.vvvv, V.ovvv, V.ovvo, V.oovo, imp, list, nlist, n, anti, w1, wab, wr};
  sp_wbase_kernel<T><<<dim3(sp_grid(list ? nlist : n3), nx), kSpThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_sp_rinit(const T* t1, const T* t2, const T* Ft, const T* Ft2, const SpBlocksT<T>& V,
                            const int16_t* imp, const int* list, int nlist, int n, int nx, T* R, cudaStream_t st) {
  SpR<T> a{t1, t2, Ft, Ft2, V.vvvo, V.ovoo, V.ovvo, imp, list, nlist, n, R};
  sp_rinit_kernel<T><<<dim3(sp_grid(nlist), nx), kSpThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_sp_s2(const T* R, const T* Xr, const T* Lc, const T* Vvvoo, const int16_t* imp, const int* canon,
                         int ncanon, int n, int nx, T* S2, cudaStream_t st) {
  sp_s2_kernel<T><<<dim3(sp_grid(ncanon), nx), kSpThreads, 0, st>>>(R, Xr, Lc, Vvvoo, imp, canon, ncanon, n, S2);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_sector_gemm(const SecGemmArgsT<T>& g, int nwork, int nx, cudaStream_t st) {
  if (nwork <= 0 || nx <= 0) return cudaSuccess;
  if (nx > 65535) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4)
    sector_gemm_f32_kernel<kSecT><<<dim3(nwork, nx), (kSecT / 4) * (kSecT / 4), 0, st>>>(g);
  else
    sector_gemm_kernel<T, kSecT, kSecThreads><<<dim3(nwork, nx), kSecThreads, 0, st>>>(g);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_sector_gemm_small(const SecGemmArgsT<T>& g, int nwork, int nx, cudaStream_t st) {
  if (nwork <= 0 || nx <= 0) return cudaSuccess;
  if (nx > 65535) return cudaErrorInvalidValue;
  sector_gemm_kernel<T, 16, 64><<<dim3(nwork, nx), 64, 0, st>>>(g);
  return cudaGetLastError();
}
int sector_tile() { return kSecT; }

template <class T>
cudaError_t launch_sp_thermal_eri(const double* eri, const int16_t* imp, int n, const double* f0, const double* f1,
                                  const double* f2, const double* f3, T* out, cudaStream_t st) {
  const long long n3 = static_cast<long long>(n) * n * n;
  sp_thermal_eri_kernel<T><<<sp_grid(n3), kSpThreads, 0, st>>>(eri, imp, n, f0, f1, f2, f3, out);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_sp_swap12(const T* in, int n, T* out, cudaStream_t st) {
  const long long n3 = static_cast<long long>(n) * n * n;
  sp_swap12_kernel<T><<<sp_grid(n3), kSpThreads, 0, st>>>(in, n, out);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_sp_thermal_fock(const double* fbar, int n, const double* f0, const double* f1, T* out,
                                   cudaStream_t st) {
  sp_thermal_fock_kernel<T><<<(n + 127) / 128, 128, 0, st>>>(fbar, n, f0, f1, out);
  return cudaGetLastError();
}

#define FTCC_SPARSE_INSTANTIATE(T)                                                                                  \
  template cudaError_t launch_sp_amp<T>(const T*, const T*, const int16_t*, int, int, T*, T*, T*, T*, int,         \
                                        const int*, int, cudaStream_t);                                           \
  template cudaError_t launch_sp_canon<T>(const T*, const T*, const SpBlocksT<T>&, const int16_t*, const int*, int, \
                                          int, int, T*, T*, T*, T*, cudaStream_t);                                \
  template cudaError_t launch_sp_vectors<T>(const SpVecArgsT<T>&, int, cudaStream_t);                              \
  template cudaError_t launch_sp_wbase<T>(const T*, const SpBlocksT<T>&, const int16_t*, int, int, T*, T*, T*, int, \
                                          const int*, int, cudaStream_t);                                         \
  template cudaError_t launch_sp_rinit<T>(const T*, const T*, const T*, const T*, const SpBlocksT<T>&,             \
                                          const int16_t*, const int*, int, int, int, T*, cudaStream_t);            \
  template cudaError_t launch_sp_s2<T>(const T*, const T*, const T*, const T*, const int16_t*, const int*, int, int, \
                                       int, T*, cudaStream_t);                                                    \
  template cudaError_t launch_sector_gemm<T>(const SecGemmArgsT<T>&, int, int, cudaStream_t);                      \
  template cudaError_t launch_sector_gemm_small<T>(const SecGemmArgsT<T>&, int, int, cudaStream_t);                \
  template cudaError_t launch_sp_thermal_eri<T>(const double*, const int16_t*, int, const double*, const double*,  \
                                                const double*, const double*, T*, cudaStream_t);                  \
  template cudaError_t launch_sp_swap12<T>(const T*, int, T*, cudaStream_t);                                       \
  template cudaError_t launch_sp_thermal_fock<T>(const double*, int, const double*, const double*, T*, cudaStream_t);
FTCC_SPARSE_INSTANTIATE(float)
FTCC_SPARSE_INSTANTIATE(double)
#undef FTCC_SPARSE_INSTANTIATE

cudaError_t launch_sp_compress(const double* d1, const double* d2, const int16_t* imp, int n, int nx, double* s1,
                               double* s2, cudaStream_t st) {
  const long long n3 = static_cast<long long>(n) * n * n;
  sp_compress_kernel<<<dim3(sp_grid(n3), nx), kSpThreads, 0, st>>>(d1, d2, imp, n, s1, s2);
  return cudaGetLastError();
}

cudaError_t launch_sp_expand(const double* s1, const double* s2, const int16_t* imp, int n, int nx, double* d1,
                             double* d2, cudaStream_t st) {
  const long long n4 = static_cast<long long>(n) * n * n * n;
  sp_expand_kernel<<<dim3(sp_grid(n4), nx), kSpThreads, 0, st>>>(s1, s2, imp, n, d1, d2);
  return cudaGetLastError();
}

cudaError_t launch_sp_s2_t(const double* S2b, const int16_t* imp, const int* list, int nlist, int n, int nx,
                           double* Rb, cudaStream_t st) {
  sp_s2_t_kernel<<<dim3(sp_grid(nlist), nx), kSpThreads, 0, st>>>(S2b, imp, list, nlist, n, Rb);
  return cudaGetLastError();
}

cudaError_t launch_sector_tn(const SecTnArgs& g, int nwork, cudaStream_t st) {
  if (nwork <= 0 || g.nx <= 0) return cudaSuccess;
  if (g.nx > 65535) return cudaErrorInvalidValue;
  sector_tn_kernel<kSecT, kSecThreads><<<dim3(nwork, g.dx ? g.nx : 1), kSecThreads, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_sector_tn_small(const SecTnArgs& g, int nwork, cudaStream_t st) {
  if (nwork <= 0 || g.nx <= 0) return cudaSuccess;
  if (g.nx > 65535) return cudaErrorInvalidValue;
  sector_tn_kernel<16, 64><<<dim3(nwork, g.dx ? g.nx : 1), 64, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_sp_vjp_vectors(const SpVjpArgs& v, int nx, cudaStream_t st) {
  SpVecT a{v.t1, v.t2, v.Rb, v.S1b, v.Fme, v.Fae, v.Fmi, v.V.vvvo, v.V.ovvo, v.V.ovoo, v.V.ooov, v.V.ovvv,
           v.V.oovo, v.V.ovov, v.V.oovv, v.w1b, v.wabb, v.wrb, v.tab, v.tpb, v.xpb, v.imp,
           v.l1, v.off1, v.l2, v.off2, v.n, v.Ftb, v.Ft2b, v.Faeb, v.Fmib, v.Fmeb, v.t1b};
  sp_vec_t1_kernel<<<dim3(v.n, nx), 256, 0, st>>>(a);
  sp_vec_t2_kernel<<<dim3(v.n, nx), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sp_t2bar(const SpVjpArgs& v, int nx, cudaStream_t st) {
  const long long n3 = static_cast<long long>(v.n) * v.n * v.n;
  SpT2 a{v.t1, v.Rb, v.Ft, v.Ft2, v.S1b, v.Fme, v.Fmib, v.Faeb, v.tab, v.tpb, v.trb, v.xpb, v.V.ovvv, v.V.oovv,
         v.V.oovo, v.imp, v.list, v.nlist, v.n, v.t2b};
  (void)n3;
  sp_t2bar_kernel<<<dim3(sp_grid(v.nlist), nx), kSpThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sp_fixed_bar(const SpVjpArgs& v, const double* S2b, const double* cz, double* const* Vbar,
                                double* const* fbar, int nx, cudaStream_t st) {
  const long long n3 = static_cast<long long>(v.n) * v.n * v.n;
  SpFixT a{};
  a.t1 = v.t1;
  a.t2 = v.t2;
  a.S2b = S2b;
  a.Rb = v.Rb;
  a.w1b = v.w1b;
  a.wabb = v.wabb;
  a.wrb = v.wrb;
  a.S1b = v.S1b;
  a.Faeb = v.Faeb;
  a.Fmib = v.Fmib;
  a.Fmeb = v.Fmeb;
  a.cz = cz;
  a.imp = v.imp;
  a.list = v.list;
  a.nlist = v.nlist;
  a.n = v.n;
  a.nx = nx;
  for (int k = 0; k < 11; ++k) a.Vb[k] = Vbar[k];
  (void)n3;
  sp_fixed_bar_kernel<<<dim3(sp_grid(v.nlist), 11), kSpThreads, 0, st>>>(a);
  sp_fock_bar_kernel<<<(v.n + 127) / 128, 128, 0, st>>>(v.t1, v.Fmeb, v.Faeb, v.Fmib, v.S1b, cz, v.n, nx, fbar[0],
                                                          fbar[1], fbar[2], fbar[3]);
  return cudaGetLastError();
}

cudaError_t launch_sp_energy_bar(const double* t1, const double* t2, const double* cz, const int16_t* imp, int n,
                                 int ng, double* Voovvb, double* fovb, cudaStream_t st) {
  const long long n3 = static_cast<long long>(n) * n * n;
  sp_energy_bar_kernel<<<sp_grid(n3), kSpThreads, 0, st>>>(t1, t2, cz, imp, n, ng, Voovvb, fovb);
  return cudaGetLastError();
}

cudaError_t launch_sp_slot_sums(const double* I, const double* Ib, const int16_t* imp, int n, int cls, double* Do,
                                double* Dv, cudaStream_t st) {
  sp_slot_sums_kernel<<<n, 256, 0, st>>>(I, Ib, imp, n, cls, Do, Dv);
  return cudaGetLastError();
}

cudaError_t launch_sp_fme(const double* t1, const double* fov, const double* Voovv, int n, int nx, double* out,
                          cudaStream_t st) {
  const int warps = n * nx;
  sp_fme_kernel<<<(warps * 32 + 127) / 128, 128, 0, st>>>(t1, fov, Voovv, n, nx, out);
  return cudaGetLastError();
}

cudaError_t launch_sp_eri_adjoint(const double* bar, const int16_t* imp, int n, const double* f0, const double* f1,
                                  const double* f2, const double* f3, double* gamma, cudaStream_t st) {
  const long long n3 = static_cast<long long>(n) * n * n;
  sp_eri_adjoint_kernel<<<sp_grid(n3), kSpThreads, 0, st>>>(bar, imp, n, f0, f1, f2, f3, gamma);
  return cudaGetLastError();
}

cudaError_t launch_sp_swap12_add(const double* in, int n, double* out, cudaStream_t st) {
  const long long n3 = static_cast<long long>(n) * n * n;
  sp_swap12_add_kernel<<<sp_grid(n3), kSpThreads, 0, st>>>(in, n, out);
  return cudaGetLastError();
}

}  // namespace ftcc
