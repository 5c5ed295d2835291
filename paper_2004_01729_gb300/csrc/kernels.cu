// Memory-bound kernels of the FT-CCSD sweep: operand packing, the
// antisymmetrising scatter, tau builds, the model Hamiltonians, the
// reference / Fermi scaling, and the propagator with the fused energy.
#include <atomic>
#include <cuda_bf16.h>
#include <math_constants.h>

#include <algorithm>
#include <climits>

#include "ftcc_internal.h"

namespace ftcc {

namespace {

inline int grid_for(long long n, int threads, int cap = 152 * 16) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return static_cast<int>(b);
}

// ----------------------------------------------------------------- index helpers
__device__ __forceinline__ uint32_t fdiv(const FastDiv& f, uint32_t n) {
  return static_cast<uint32_t>((static_cast<uint64_t>(__umulhi(n, f.m)) + n) >> f.s);
}

// ----------------------------------------------------------------- tiled permute
// dst[k-coords] = beta dst + alpha sum_p sign_p src[sum_k c_k sst_p[k]] over
// the terms p of an antisymmetriser (identity, one swap, two swaps).  One
// block owns one tile: a box over a few "tile letters" (the destination's
// innermost letter and, for every term, the letter at unit source stride),
// every other letter fixed.  Each term is read in its own letter order
// (unit source stride fastest) into shared memory and the tile is written
// in destination order, so both global streams are coalesced whatever the
// permutation.  Used for the GEMM operand packs (one term, beta 0) and the
// antisymmetrising scatters of GEMM outputs.
constexpr int kPermThreads = 256;
constexpr int kPermTile = 4096;   // elements of one tile in shared memory
constexpr int kPermRows = 512;    // rows per pass of the shared row table

constexpr int kPermTerms = 4;     // source terms of one launch (the write is order kPermTerms)

struct DevPerm {
  int nd, nterm, nt;
  FastDiv bcnt[kMaxL];             // blocks along dst letter k
  int bstep[kMaxL];                // coordinate step per block along k (1, or the tile extent)
  int tslot[kMaxL];                // tile-letter slot of dst letter k, -1 if not a tile letter
  const void* src[kPermTerms];     // term p: source tensor
  double coef[kPermTerms];         // term p: coefficient (sign of the antisymmetriser included)
  long long sst[kPermTerms][kMaxL];   // term p: source stride of dst letter k (swaps applied)
  long long dstr[kMaxL];           // destination stride of dst letter k
  // per order o (terms 0..kPermTerms-1, the write = kPermTerms), position l (fastest first):
  FastDiv fd_full[kPermTerms + 1][kMaxL], fd_tail[kPermTerms + 1][kMaxL];   // extent in an inner / last block
  int slot[kPermTerms + 1][kMaxL];        // tile-letter slot at that position
  long long gstr[kPermTerms + 1][kMaxL];  // global stride at that position (source for terms, dst for write)
  int tstr[kPermTerms + 1][kMaxL];        // shared-memory stride at that position
  int tail_blk[kMaxL];             // per tile slot: block coordinate of the last (tail) block
  int ext_full[kMaxL], ext_tail[kMaxL];
  uint32_t block0;
};

template <class T>
struct PermOut {
  T* dst;
  __nv_bfloat16* hi;   // bf16 hi / lo split output (dst unused) when non-null
  __nv_bfloat16* lo;
};

// Rows of one order: every tile element is (row, f) with f the coordinate of
// the order's fastest letter.  A row table (global offset, tile index) is
// built in shared memory; the elements e = row * ext_f + f of up to
// kPermRows rows are then spread over the block's threads (consecutive
// threads on consecutive f), kPermUnroll of them per thread with all loads
// issued before any is used: load(g, t) -> value, then apply(g, t, value).
constexpr int kPermUnroll = 4;

// With VW > 1 each index names VW consecutive elements along the fastest
// letter (unit global stride, extent a multiple of VW, every row offset a
// multiple of VW: checked by the launcher), moved by one vector access on
// the global side and VW accesses tile stride tf apart on the tile side.
template <int O, class V, int VW = 1, class L, class A>
__device__ __forceinline__ void perm_rows(const DevPerm& d, uint32_t tailmask, int n, long long* rowG, int* rowT,
                                          L&& load, A&& apply) {
  const int sl0 = d.slot[O][0];
  const bool tail0 = (tailmask >> sl0) & 1u;
  const FastDiv fe = tail0 ? d.fd_tail[O][0] : d.fd_full[O][0];
  const int ef = static_cast<int>(fe.d);
  const long long gf = d.gstr[O][0];
  const int tf = d.tstr[O][0];
  const int nrows = n / ef;
  for (int r0 = 0; r0 < nrows; r0 += kPermRows) {
    const int nr = min(kPermRows, nrows - r0);
    for (int r = threadIdx.x; r < nr; r += kPermThreads) {
      uint32_t rr = static_cast<uint32_t>(r0 + r);
      long long g = 0;
      int t = 0;
#pragma unroll
      for (int l = 1; l < kMaxL; ++l) {
        if (l < d.nt) {
          const FastDiv f = ((tailmask >> d.slot[O][l]) & 1u) ? d.fd_tail[O][l] : d.fd_full[O][l];
          const uint32_t q = fdiv(f, rr);
          const uint32_t co = rr - q * f.d;
          rr = q;
          g += static_cast<long long>(co) * d.gstr[O][l];
          t += static_cast<int>(co) * d.tstr[O][l];
        }
      }
      rowG[r] = g;
      rowT[r] = t;
    }
    __syncthreads();
    const int ne = nr * ef / VW;
    for (int e0 = threadIdx.x; e0 < ne; e0 += kPermThreads * kPermUnroll) {
      V v[kPermUnroll];
      long long gg[kPermUnroll];
      int tt[kPermUnroll];
#pragma unroll
      for (int u = 0; u < kPermUnroll; ++u) {
        const int e = (e0 + u * kPermThreads) * VW;   // first element of this index
        if (e < ne * VW) {
          const uint32_t q = fdiv(fe, static_cast<uint32_t>(e));
          const int co = e - static_cast<int>(q) * ef;
          gg[u] = rowG[q] + co * gf;
          tt[u] = rowT[q] + co * tf;
          v[u] = load(gg[u], tt[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kPermUnroll; ++u)
        if (e0 + u * kPermThreads < ne) apply(gg[u], tt[u], v[u]);
    }
    __syncthreads();
  }
}

// VW elements of T moved as one 16-byte access
template <class T, int VW>
struct PermVec {
  T x[VW];
};
template <class T, int VW>
__device__ __forceinline__ PermVec<T, VW> vload(const T* p) {
  PermVec<T, VW> r;
  if constexpr (VW == 1) {
    r.x[0] = *p;
  } else if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    r.x[0] = v.x, r.x[1] = v.y, r.x[2] = v.z, r.x[3] = v.w;
  } else {
    const double2 v = *reinterpret_cast<const double2*>(p);
    r.x[0] = v.x, r.x[1] = v.y;
  }
  return r;
}
template <class T, int VW>
__device__ __forceinline__ void vstore(T* p, const PermVec<T, VW>& r) {
  if constexpr (VW == 1) {
    *p = r.x[0];
  } else if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(r.x[0], r.x[1], r.x[2], r.x[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(r.x[0], r.x[1]);
  }
}

// Term P into the tile: term 0 stores, the others add, each scaled by its
// coefficient (the sign of the antisymmetriser included).
template <int P, class T, int VW>
__device__ __forceinline__ void perm_term(const DevPerm& d, const long long* c, uint32_t tailmask, int n,
                                          long long* rowG, int* rowT, T* tile) {
  long long base = 0;
#pragma unroll
  for (int k = 0; k < kMaxL; ++k)
    if (k < d.nd) base += c[k] * d.sst[P][k];
  const T* sp = static_cast<const T*>(d.src[P]) + base;
  const T cf = static_cast<T>(d.coef[P]);
  const int tf = d.tstr[P][0];
  using V = PermVec<T, VW>;
  auto load = [&](long long g, int) { return vload<T, VW>(sp + g); };
  if (P == 0) {
    perm_rows<P, V, VW>(d, tailmask, n, rowG, rowT, load, [&](long long, int t, const V& v) {
#pragma unroll
      for (int w = 0; w < VW; ++w) tile[t + w * tf] = cf * v.x[w];
    });
  } else {
    perm_rows<P, V, VW>(d, tailmask, n, rowG, rowT, load, [&](long long, int t, const V& v) {
#pragma unroll
      for (int w = 0; w < VW; ++w) tile[t + w * tf] += cf * v.x[w];
    });
  }
}

template <class T, bool SPLIT, int VW>
__global__ void __launch_bounds__(kPermThreads, VW == 1 ? 5 : 4) permute_kernel(PermOut<T> out, const __grid_constant__ DevPerm d,
                                                               T alpha, T beta) {
  extern __shared__ __align__(16) unsigned char perm_smem[];
  T* tile = reinterpret_cast<T*>(perm_smem);
  __shared__ long long rowG[kPermRows];
  __shared__ int rowT[kPermRows];
  // block -> coordinates of every dst letter (tile letters: the box start)
  uint32_t r = d.block0 + blockIdx.x;
  long long c[kMaxL];
  uint32_t tailmask = 0;
  int n = 1;
#pragma unroll
  for (int k = kMaxL - 1; k >= 0; --k) {
    c[k] = 0;
    if (k < d.nd) {
      const uint32_t q = fdiv(d.bcnt[k], r);
      const uint32_t bk = r - q * d.bcnt[k].d;
      r = q;
      c[k] = static_cast<long long>(bk) * d.bstep[k];
      const int sl = d.tslot[k];
      if (sl >= 0) {
        const bool tail = bk == static_cast<uint32_t>(d.tail_blk[sl]);
        tailmask |= (tail ? 1u : 0u) << sl;
        n *= tail ? d.ext_tail[sl] : d.ext_full[sl];
      }
    }
  }
  // terms: gather into the tile, each in its own letter order
  perm_term<0, T, VW>(d, c, tailmask, n, rowG, rowT, tile);
  if (d.nterm > 1) perm_term<1, T, VW>(d, c, tailmask, n, rowG, rowT, tile);
  if (d.nterm > 2) perm_term<2, T, VW>(d, c, tailmask, n, rowG, rowT, tile);
  if (d.nterm > 3) perm_term<3, T, VW>(d, c, tailmask, n, rowG, rowT, tile);
  // write in destination order
  long long dbase = 0;
#pragma unroll
  for (int k = 0; k < kMaxL; ++k)
    if (k < d.nd) dbase += c[k] * d.dstr[k];
  if constexpr (SPLIT && VW == 1) {
    __nv_bfloat16* hi = out.hi + dbase;
    __nv_bfloat16* lo = out.lo + dbase;
    perm_rows<kPermTerms, T>(d, tailmask, n, rowG, rowT, [&](long long, int t) { return tile[t]; },
                    [&](long long g, int, T tv) {
                      const float v = static_cast<float>(tv);
                      const __nv_bfloat16 h = __float2bfloat16_rn(v);
                      hi[g] = h;
                      lo[g] = __float2bfloat16_rn(v - __bfloat162float(h));
                    });
  } else if constexpr (SPLIT) {
    // VW = 4 floats of the tile become four bf16 hi and four bf16 lo halves,
    // each stored as one 8-byte access
    static_assert(VW == 4 && sizeof(T) == 4, "vector split of FP32 tiles");
    __nv_bfloat16* hi = out.hi + dbase;
    __nv_bfloat16* lo = out.lo + dbase;
    using V = PermVec<T, VW>;
    const int tf = d.tstr[kPermTerms][0];
    perm_rows<kPermTerms, V, VW>(
        d, tailmask, n, rowG, rowT,
        [&](long long, int t) {
          V v;
#pragma unroll
          for (int w = 0; w < VW; ++w) v.x[w] = tile[t + w * tf];
          return v;
        },
        [&](long long g, int, const V& v) {
          __nv_bfloat162 h2[2], l2[2];
#pragma unroll
          for (int w = 0; w < 2; ++w) {
            const float a = static_cast<float>(v.x[2 * w]), b = static_cast<float>(v.x[2 * w + 1]);
            const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
            h2[w] = __halves2bfloat162(ha, hb);
            l2[w] = __halves2bfloat162(__float2bfloat16_rn(a - __bfloat162float(ha)),
                                       __float2bfloat16_rn(b - __bfloat162float(hb)));
          }
          uint2 uh, ul;
          uh.x = *reinterpret_cast<const uint32_t*>(&h2[0]);
          uh.y = *reinterpret_cast<const uint32_t*>(&h2[1]);
          ul.x = *reinterpret_cast<const uint32_t*>(&l2[0]);
          ul.y = *reinterpret_cast<const uint32_t*>(&l2[1]);
          *reinterpret_cast<uint2*>(hi + g) = uh;
          *reinterpret_cast<uint2*>(lo + g) = ul;
        });
  } else {
    T* dp = out.dst + dbase;
    using V = PermVec<T, VW>;
    const int tf = d.tstr[kPermTerms][0];
    if (beta == T(0)) {
      perm_rows<kPermTerms, V, VW>(
          d, tailmask, n, rowG, rowT,
          [&](long long, int t) {
            V v;
#pragma unroll
            for (int w = 0; w < VW; ++w) v.x[w] = tile[t + w * tf];
            return v;
          },
          [&](long long g, int, const V& v) {
            V o;
#pragma unroll
            for (int w = 0; w < VW; ++w) o.x[w] = alpha * v.x[w];
            vstore<T, VW>(dp + g, o);
          });
    } else {
      // the destination values are the loads; the tile is read at the store
      perm_rows<kPermTerms, V, VW>(
          d, tailmask, n, rowG, rowT, [&](long long g, int) { return vload<T, VW>(dp + g); },
          [&](long long g, int t, const V& old) {
            V o;
#pragma unroll
            for (int w = 0; w < VW; ++w) o.x[w] = beta * old.x[w] + alpha * tile[t + w * tf];
            vstore<T, VW>(dp + g, o);
          });
    }
  }
}

// ----------------------------------------------------------------- doubles antisymmetriser
// dst[zx][i][j][a][b] = sum_s c_s ((X_s(ij,ab) - X_s(ji,ab)) - (X_s(ij,ba) - X_s(ji,ba))) + V(ab,ij)
// evaluated once per unordered pair {i,j} and pair of 32-wide tiles {A,B};
// the other three orientations are written as its exact negatives, so dst
// is exactly antisymmetric and every source element is read once.
constexpr int kAT = 32;   // largest tile edge along a and b

__device__ __forceinline__ void upper_pair(int n, int p, int& i, int& j) {
  // p-th pair (i <= j) of the upper triangle of an n x n grid, rows in order
  // (an FP32 estimate of the row, then exact integer correction)
  const float m = 2.0f * n + 1.0f;
  int r = static_cast<int>((m - sqrtf(fmaxf(m * m - 8.0f * p, 0.0f))) * 0.5f);
  if (r < 0) r = 0;
  if (r > n - 1) r = n - 1;
  auto start = [n](int q) { return q * n - q * (q - 1) / 2; };
  while (r > 0 && start(r) > p) --r;
  while (r + 1 < n && start(r + 1) <= p) ++r;
  i = r;
  j = r + (p - start(r));
}

template <class T, int KP>
__global__ void __launch_bounds__(256, 4) antisym4_kernel(T* __restrict__ dst, Anti4Desc d) {
  extern __shared__ __align__(16) unsigned char as_smem[];
  T* tiles = reinterpret_cast<T*>(as_smem);   // [nsrc][4][TA][TA + 1], then the result [TA][TA + 1]
  const int TA = d.ta, ld = TA + 1, t2 = TA * TA;
  const int nA = (d.nv + TA - 1) / TA;
  const int ntp = nA * (nA + 1) / 2;
  const int npair = d.no * (d.no + 1) / 2;
  // block -> (zx, pair {i,j}, tile pair {A,B}), decoded once by thread 0
  __shared__ int blk[6];
  if (threadIdx.x == 0) {
    unsigned r = blockIdx.x;
    const int tp = static_cast<int>(r % ntp);
    r /= ntp;
    const int pr = static_cast<int>(r % npair);
    blk[0] = static_cast<int>(r / npair);
    upper_pair(d.no, pr, blk[1], blk[2]);
    upper_pair(nA, tp, blk[3], blk[4]);
    blk[5] = blk[0] / d.nx;
  }
  __syncthreads();
  const long long zx = blk[0];
  const int i = blk[1], j = blk[2], tA = blk[3], tB = blk[4];
  const int A0 = tA * TA, B0 = tB * TA;
  // On a diagonal tile (A = B) the (BA) orientations are the (AB) tiles
  // transposed: they are neither loaded nor stored twice.
  const bool diag = tA == tB;
  // thread -> up to KP tile elements e = threadIdx.x + 256 k (KP = the
  // launcher's ceil(TA^2 / 256), so no thread carries idle element slots),
  // row rr = e / TA and column cc = e % TA (the float quotient is exact for
  // e < 1024, TA <= 32); all lanes work when TA < 32, and consecutive
  // threads take consecutive columns, so every global access coalesces
  constexpr int kPer = KP;
  const float inv = 1.0f / static_cast<float>(TA);
  int rr[kPer], cc[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int e = threadIdx.x + 256 * k;
    rr[k] = e < t2 ? static_cast<int>((static_cast<float>(e) + 0.5f) * inv) : TA;   // TA: no element
    cc[k] = e - rr[k] * TA;
  }
  const int nv = d.nv;
  // the four orientations of every source: (ij,AB), (ji,AB), (ij,BA), (ji,BA);
  // each thread issues all of its loads (up to 4 elements x 4 orientations of
  // a source) before it stores any of them
  for (int s = 0; s < d.nsrc; ++s) {
    const AntiSrc& q = d.src[s];
    // offsets inside one zx slice fit in 32 bits (checked by the launcher)
    const int sa = static_cast<int>(q.sa), sb = static_cast<int>(q.sb);
    const T* base = static_cast<const T*>(q.p) + zx * q.sx;
    const T* bij = base + (i * static_cast<int>(q.si) + j * static_cast<int>(q.sj));
    const T* bji = base + (j * static_cast<int>(q.si) + i * static_cast<int>(q.sj));
    T* ts = tiles + s * 4 * TA * ld;
    T v[kPer][4];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int a1 = A0 + rr[k], b1 = B0 + cc[k], a2 = B0 + rr[k], b2 = A0 + cc[k];
      const bool in1 = rr[k] < TA && a1 < nv && b1 < nv;
      const bool in2 = !diag && rr[k] < TA && a2 < nv && b2 < nv;
      const int o1 = a1 * sa + b1 * sb, o2 = a2 * sa + b2 * sb;
      v[k][0] = in1 ? bij[o1] : T(0);
      v[k][1] = in1 ? bji[o1] : T(0);
      v[k][2] = in2 ? bij[o2] : T(0);
      v[k][3] = in2 ? bji[o2] : T(0);
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (rr[k] < TA) {
        const int o = rr[k] * ld + cc[k];
        ts[o] = v[k][0];
        ts[TA * ld + o] = v[k][1];
        if (!diag) {
          ts[2 * TA * ld + o] = v[k][2];
          ts[3 * TA * ld + o] = v[k][3];
        }
      }
    }
  }
  __syncthreads();
  T* res = tiles + d.nsrc * 4 * TA * ld;
  const long long z = blk[5];
  const T* vb = static_cast<const T*>(d.vp) + z * d.vz + i * d.vi + j * d.vj;
  const T c0 = static_cast<T>(d.src[0].coef), c1 = static_cast<T>(d.src[1].coef);
  const int va = static_cast<int>(d.va), vbs = static_cast<int>(d.vb);
  const int off2 = diag ? 0 : 2 * TA, off3 = diag ? TA : 3 * TA;   // where the (BA) tiles live
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int r = rr[k], c = cc[k];
    if (r < TA) {
      const int a = A0 + r, b = B0 + c;
      T v = T(0);
      if (a < nv && b < nv) {
        const T* t0 = tiles;
        v = c0 * ((t0[r * ld + c] - t0[(TA + r) * ld + c]) - (t0[(off2 + c) * ld + r] - t0[(off3 + c) * ld + r]));
        if (d.nsrc > 1) {
          t0 += 4 * TA * ld;
          v += c1 * ((t0[r * ld + c] - t0[(TA + r) * ld + c]) - (t0[(off2 + c) * ld + r] - t0[(off3 + c) * ld + r]));
        }
        if (d.vp) v += vb[a * va + b * vbs];
      }
      res[r * ld + c] = v;
    }
  }
  __syncthreads();
  const long long so = static_cast<long long>(nv) * nv, sj = so, si = static_cast<long long>(d.no) * so;
  T* out = dst + zx * d.no * si;
  T* oij = out + (i * si + j * sj);
  T* oji = out + (j * si + i * sj);
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int r = rr[k], c = cc[k];
    if (r < TA) {
      {
        const int a = A0 + r, b = B0 + c;   // (A, B) orientation
        if (a < nv && b < nv) {
          const T v = res[r * ld + c];
          oij[a * nv + b] = v;
          if (i != j) oji[a * nv + b] = -v;
        }
      }
      if (!diag) {
        const int a = B0 + r, b = A0 + c;   // (B, A) orientation: the transposed tile
        if (a < nv && b < nv) {
          const T v = res[c * ld + r];
          oij[a * nv + b] = -v;
          if (i != j) oji[a * nv + b] = v;
        }
      }
    }
  }
}

// ----------------------------------------------------------------- tau builds
// One tau slice per blockIdx.y; element e = ((i o + j) v + a) v + b.
template <class T>
__global__ void tau_kernel(const T* __restrict__ t1, const T* __restrict__ t2, T* __restrict__ tt,
                           T* __restrict__ ta, T* __restrict__ X, T ctt, T cta, FastDiv fo, FastDiv fv) {
  const uint32_t no = fo.d, nv = fv.d;
  const uint32_t slice = no * no * nv * nv;
  const long long x = blockIdx.y;
  const T* s = t1 + x * no * nv;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < slice; e += gridDim.x * blockDim.x) {
    uint32_t r = e;
    uint32_t q = fdiv(fv, r);
    const uint32_t b = r - q * nv;
    r = q;
    q = fdiv(fv, r);
    const uint32_t a = r - q * nv;
    r = q;
    q = fdiv(fo, r);
    const uint32_t j = r - q * no;
    const uint32_t i = q;
    const T p = s[i * nv + a] * s[j * nv + b] - s[i * nv + b] * s[j * nv + a];
    const long long o = x * slice + e;
    const T v = t2[o];
    if (tt) tt[o] = v + ctt * p;
    if (ta) ta[o] = v + cta * p;
    if (X) X[o] = T(0.5) * v + s[i * nv + a] * s[j * nv + b];   // X_ijab = 1/2 t2 + t1_ia t1_jb
  }
}

template <class Ts, class Td>
__global__ void convert_kernel(const Ts* __restrict__ s, Td* __restrict__ d, long long n) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x)
    d[e] = static_cast<Td>(s[e]);
}

// ----------------------------------------------------------------- Hamiltonians
__global__ void hubbard_kernel(double* h, double* eri, double* eps, int L, double t, double U) {
  const int N = 2 * L;
  const long long total = static_cast<long long>(N) * N * N * N;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    long long r = e;                        // e = ((p N + q) N + p2) N + s
    const int s = r % N; r /= N;
    const int p2 = r % N; r /= N;
    const int q = r % N; r /= N;
    const int p = static_cast<int>(r);
    // <p q | p2 s> - <p q | s p2>; spin = index / L, momentum = index % L
    const int sp = p / L, sq = q / L, sr = p2 / L, ss = s / L;
    const int mp = p % L, mq = q % L, mr = p2 % L, ms = s % L;
    double v = 0.0;
    if (sp == sr && sq == ss && ((mp + mq - mr - ms) % L + L) % L == 0) v += U / L;
    if (sp == ss && sq == sr && ((mp + mq - ms - mr) % L + L) % L == 0) v -= U / L;
    eri[e] = v;
  }
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < N * N) {
    const int p = tid / N, q = tid % N;
    double v = 0.0;
    if (p == q) v = -2.0 * t * cos(2.0 * CUDART_PI * (p % L) / L);
    h[tid] = v;
    if (p == q) eps[p] = v + 0.5 * U;
  }
}

__global__ void ueg_kernel(double* h, double* eri, double* eps, const int* __restrict__ nvec, int M, int nocc,
                           double vol, double kunit) {
  const int N = 2 * M;
  const long long total = static_cast<long long>(N) * N * N * N;
  const double c4 = 4.0 * CUDART_PI / (vol * kunit * kunit);
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    long long r = e;                        // e = ((p N + q) N + p2) N + s
    const int s = r % N; r /= N;
    const int p2 = r % N; r /= N;
    const int q = r % N; r /= N;
    const int p = static_cast<int>(r);
    const int gp = p % M, gq = q % M, gr = p2 % M, gs = s % M;
    const int sp = p / M, sq = q / M, sr = p2 / M, ss = s / M;
    double v = 0.0;
    bool kcons = true;
    int d2d = 0, d2e = 0;
    for (int c = 0; c < 3; ++c) {
      const int a = nvec[3 * gp + c], b = nvec[3 * gq + c], cc = nvec[3 * gr + c], d = nvec[3 * gs + c];
      if (a + b != cc + d) kcons = false;
      d2d += (a - cc) * (a - cc);
      d2e += (a - d) * (a - d);
    }
    if (kcons) {
      if (sp == sr && sq == ss && d2d > 0) v += c4 / d2d;   // direct  <pq|rs>
      if (sp == ss && sq == sr && d2e > 0) v -= c4 / d2e;   // exchange <pq|sr>
    }
    eri[e] = v;
  }
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < N * N) {
    const int p = tid / N, q = tid % N;
    double v = 0.0;
    if (p == q) {
      const int g = p % M;
      double k2 = 0.0;
      for (int c = 0; c < 3; ++c) k2 += static_cast<double>(nvec[3 * g + c]) * nvec[3 * g + c];
      v = 0.5 * k2 * kunit * kunit;
      double ex = 0.0;
      for (int o = 0; o < nocc; ++o) {
        int d2 = 0;
        for (int c = 0; c < 3; ++c) d2 += (nvec[3 * g + c] - nvec[3 * o + c]) * (nvec[3 * g + c] - nvec[3 * o + c]);
        if (d2 > 0) ex += c4 / d2;
      }
      eps[p] = v - ex;
    }
    h[tid] = v;
  }
}

// ----------------------------------------------------------------- reference
__device__ __forceinline__ double fermi(double z) {   // 1 / (1 + e^z)
  if (z > 0.0) {
    const double e = exp(-z);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(z));
}

__global__ void fock_kernel(const double* __restrict__ h, const double* __restrict__ eri,
                            const double* __restrict__ eps, int N, double beta, double mu, double* f, double* fbar) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= N * N) return;
  const int p = tid / N, q = tid % N;
  double acc = 0.0;
  for (int r = 0; r < N; ++r) {
    const double n = fermi(beta * (eps[r] - mu));
    acc += n * eri[((static_cast<long long>(p) * N + r) * N + q) * N + r];
  }
  const double v = h[tid] + acc;
  f[tid] = v;
  fbar[tid] = (p == q) ? v - eps[p] : v;
}

__global__ void reference_scalars_kernel(const double* __restrict__ h, const double* __restrict__ eri,
                                         const double* __restrict__ eps, int N, double beta, double mu, double* n,
                                         double* nbar, double* scal) {
  // scal[0] = Omega0, scal[1] = Omega1, scal[2] = sum n
  __shared__ double red[3][256];
  double o0 = 0.0, o1 = 0.0, ns = 0.0;
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    const double z = beta * (eps[p] - mu);
    const double np = fermi(z);
    n[p] = np;
    nbar[p] = fermi(-z);
    // ln(1 + e^{-z}) without overflow
    o0 += (z > 0.0) ? log1p(exp(-z)) : (-z + log1p(exp(z)));
    o1 += np * (h[static_cast<long long>(p) * N + p] - eps[p]);
    ns += np;
  }
  for (long long pq = threadIdx.x; pq < static_cast<long long>(N) * N; pq += blockDim.x) {
    const int p = pq / N, q = pq % N;
    const double np = fermi(beta * (eps[p] - mu)), nq = fermi(beta * (eps[q] - mu));
    o1 += 0.5 * np * nq * eri[((static_cast<long long>(p) * N + q) * N + p) * N + q];
  }
  red[0][threadIdx.x] = o0;
  red[1][threadIdx.x] = o1;
  red[2][threadIdx.x] = ns;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scal[0] = -red[0][0] / beta;
    scal[1] = red[1][0];
    scal[2] = red[2][0];
  }
}

__global__ void prop_tables_kernel(const double* eps, int N, double h, double* em, double* ep) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) {
    em[p] = exp(-eps[p] * h);
    ep[p] = exp(eps[p] * h);
  }
}

template <class T>
__global__ void thermal_eri_kernel(const double* __restrict__ eri, int N, const int* i0, const double* f0, int n0,
                                   const int* i1, const double* f1, int n1, const int* i2, const double* f2, int n2,
                                   const int* i3, const double* f3, int n3, T* out) {
  const long long total = static_cast<long long>(n0) * n1 * n2 * n3;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    long long r = e;
    const int d = r % n3; r /= n3;
    const int c = r % n2; r /= n2;
    const int b = r % n1; r /= n1;
    const int a = static_cast<int>(r);
    const long long src = ((static_cast<long long>(i0[a]) * N + i1[b]) * N + i2[c]) * N + i3[d];
    out[e] = static_cast<T>(eri[src] * f0[a] * f1[b] * f2[c] * f3[d]);
  }
}

// The transpose of thermal_eri_kernel: the adjoint of one thermal block
// added to the adjoint of the antisymmetrised integrals,
// gamma[i0[a]][i1[b]][i2[c]][i3[d]] += bar[a][b][c][d] f0[a] f1[b] f2[c] f3[d].
// The index maps of one block are injective, so no two elements of a
// launch write the same slot.
__global__ void eri_adjoint_kernel(const double* __restrict__ bar, int N, const int* i0, const double* f0, int n0,
                                   const int* i1, const double* f1, int n1, const int* i2, const double* f2, int n2,
                                   const int* i3, const double* f3, int n3, double* gamma) {
  const long long total = static_cast<long long>(n0) * n1 * n2 * n3;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    long long r = e;
    const int d = r % n3; r /= n3;
    const int c = r % n2; r /= n2;
    const int b = r % n1; r /= n1;
    const int a = static_cast<int>(r);
    const long long dst = ((static_cast<long long>(i0[a]) * N + i1[b]) * N + i2[c]) * N + i3[d];
    gamma[dst] += bar[e] * f0[a] * f1[b] * f2[c] * f3[d];
  }
}

template <class T>
__global__ void thermal_fock_kernel(const double* __restrict__ fbar, int N, const int* i0, const double* f0, int n0,
                                    const int* i1, const double* f1, int n1, T* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n0 * n1) return;
  const int a = e / n1, b = e % n1;
  out[e] = static_cast<T>(fbar[static_cast<long long>(i0[a]) * N + i1[b]] * f0[a] * f1[b]);
}

// ----------------------------------------------------------------- propagation
// Simpson recurrences on the uniform grid (tau_y = y h), r = exp(-Delta h):
//   I_0 = 0
//   I_1 = h/12 (5 r S_0 + 8 S_1 - S_2 / r)
//   I_y = r^2 I_{y-2} + h/3 (r^2 S_{y-2} + 4 r S_{y-1} + S_y)                 (y even)
//   I_y = r^3 I_{y-3} + 3h/8 (r^3 S_{y-3} + 3 r^2 S_{y-2} + 3 r S_{y-1} + S_y)  (y odd >= 3)
// which equals sum_x G[y,x] exp(Delta (tau_x - tau_y)) S_x for the Simpson
// tensors (composite 1/3 for even y, 1/3 then 3/8 for odd y).  s_y = -I_y.
// max(m, |x|) in the type of its arguments (fmaxf / fabsf for float)
__device__ __forceinline__ float max_abs(float m, float x) { return fmaxf(m, fabsf(x)); }
__device__ __forceinline__ double max_abs(double m, double x) { return fmax(m, fabs(x)); }

constexpr int kPropThreads = 128;
constexpr int kPropAhead = 2;   // tau steps of loads in flight per element

template <class T, class A, class EA, int NS>
__global__ void __launch_bounds__(kPropThreads, sizeof(A) == 4 ? 8 : 4) propagate_kernel(const T* __restrict__ S, T* __restrict__ t,
                                                                                     PropArgs a) {
  // T is the storage type of S and s, A the arithmetic type of the
  // recurrence, EA that of the energy terms and their sums.  The element
  // ratios r = exp(-Delta h) are always formed in FP64 from the FP64 tables
  // and rounded once to A.  Per-thread energy slots eacc[y][thread] (each
  // thread sums over its own elements).
  extern __shared__ __align__(16) unsigned char pe_smem[];
  EA* eacc = reinterpret_cast<EA*>(pe_smem);
  const int ng = a.ng;
  const int z = blockIdx.y;                           // instance
  if (a.live && !a.live[z]) return;                   // frozen: amplitudes and partials untouched
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long size = a.size;
  const int y0 = a.y0, y1 = a.y1;                     // tau points of this launch
  S += static_cast<long long>(z) * a.s_ng * size;     // S[(y - y0) * size + mu]
  t += static_cast<long long>(z) * ng * size;
  T* chain = a.chain ? static_cast<T*>(a.chain) + static_cast<long long>(z) * 5 * size : nullptr;
  // per-orbital factors e^{-eps h}, e^{+eps h} (FP64): the element ratios
  // are products of four
  const double* em = a.em + static_cast<long long>(z) * a.N;
  const double* ep = a.ep + static_cast<long long>(z) * a.N;
  const double* wE = a.wE ? a.wE + static_cast<long long>(z) * size : nullptr;
  const bool sparse = a.imp != nullptr;
  const long long n1 = sparse ? a.N : static_cast<long long>(a.no) * a.nv;   // singles per tau point
  const T* t1E = a.t1E ? static_cast<const T*>(a.t1E) + static_cast<long long>(z) * ng * n1 : nullptr;
  double* partials = a.partials + static_cast<long long>(z) * a.nblocks * (ng + 2);
  for (int y = y0; y < y1; ++y) eacc[y * kPropThreads + threadIdx.x] = EA(0);
  T dmax = T(0), smax = T(0);
  const A h = static_cast<A>(a.hz[z]);
  const A c12 = h / A(12), c3 = h / A(3), c38 = A(3) * h / A(8);
  const A damp = static_cast<A>(a.damping);
  const bool damped = a.damping != 1.0;
  const EA cE = static_cast<EA>(a.cE);
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  const bool canon = sparse && NS == 4 && a.canon != nullptr;
  const long long nloop = canon ? a.ncanon : size;
  for (long long cidx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; cidx < nloop;
       cidx += stride) {
    const long long mu = canon ? a.canon[cidx] : cidx;
    int i, j = 0, aa, b = 0;
    if (sparse) {
      // [i][j][a] with b implied (a hole of the storage is skipped), or the
      // diagonal singles [i] (a = i)
      uint32_t r = static_cast<uint32_t>(mu);
      if (NS == 4) {
        uint32_t q = fdiv(a.fv, r);
        aa = r - q * a.nv;
        r = q;
        q = fdiv(a.fv, r);
        j = r - q * a.nv;
        i = q;
        b = a.imp[mu];
        if (b < 0) continue;
      } else {
        i = aa = static_cast<int>(r);
      }
    } else {
      uint32_t r = static_cast<uint32_t>(mu);
      uint32_t q = fdiv(a.fv, r);
      if (NS == 4) {
        b = r - q * a.nv;
        r = q;
        q = fdiv(a.fv, r);
        aa = r - q * a.nv;
        r = q;
        q = fdiv(a.fo, r);
        j = r - q * a.no;
        i = q;
      } else {
        aa = r - q * a.nv;
        i = q;
      }
    }
    const int pi = a.idxO[i], pa = a.idxV[aa];
    double r1d = em[pa] * ep[pi];
    double rinvd = ep[pa] * em[pi];
    if (NS == 4) {
      const int pj = a.idxO[j], pb = a.idxV[b];
      r1d *= em[pb] * ep[pj];
      rinvd *= ep[pb] * em[pj];
    }
    const A r1 = static_cast<A>(r1d), rinv = static_cast<A>(rinvd);
    const EA w = wE ? static_cast<EA>(wE[mu]) : EA(0);
    const A r2 = static_cast<A>(r1d * r1d), r3 = static_cast<A>(r1d * r1d * r1d);
    // S_0..S_2 are needed together at y = 1; a launch that starts at 0
    // covers at least three points
    const bool head = y0 == 0;
    const A s0 = head ? static_cast<A>(S[mu]) : A(0);
    const A s1 = head ? static_cast<A>(S[size + mu]) : A(0);
    const A s2 = head ? static_cast<A>(S[2 * size + mu]) : A(0);
    A sm1 = A(0), sm2 = A(0), sm3 = A(0);   // S_{y-1}, S_{y-2}, S_{y-3}
    A Ilast = A(0), Iprev = A(0);           // I at the last and second-last even y
    if (!head) {                            // the chain state left by the previous launch
      Ilast = static_cast<A>(chain[mu]);
      Iprev = static_cast<A>(chain[size + mu]);
      sm1 = static_cast<A>(chain[2 * size + mu]);
      sm2 = static_cast<A>(chain[3 * size + mu]);
      sm3 = static_cast<A>(chain[4 * size + mu]);
    }
    // S_y and the old s_y are loaded kPropAhead steps ahead (a register
    // window), so that several loads per thread are in flight
    const T* sq = S + mu;
    T* tq = t + y0 * size + mu;
    T sp[kPropAhead], tp[kPropAhead];
#pragma unroll
    for (int k = 0; k < kPropAhead; ++k) {
      const bool in = y0 + k < y1;
      sp[k] = in ? sq[k * size] : T(0);
      tp[k] = in ? tq[k * size] : T(0);
    }
    // singles of this tau point; with diagonal singles only a = i (then b = j)
    // carries the s_i^a s_j^b energy term
    const T* s1y = (t1E && (!sparse || aa == i)) ? t1E + y0 * n1 : nullptr;
    // offsets of the (ji)(ab), (ij)(ba) and (ji)(ba) orientations from mu
    long long mirror[3] = {0, 0, 0};
    if (canon) {
      const long long N = a.N;
      mirror[0] = (static_cast<long long>(j) * N + i) * N + aa - mu;
      mirror[1] = (static_cast<long long>(i) * N + j) * N + b - mu;
      mirror[2] = (static_cast<long long>(j) * N + i) * N + b - mu;
    }
    const int oi = sparse ? i : i * a.nv + aa, oj = sparse ? j : j * a.nv + b;
    EA* ea = eacc + y0 * kPropThreads + threadIdx.x;
    for (int y = y0; y < y1; ++y) {
      const A sy = static_cast<A>(sp[0]);
      const T tp_old = tp[0];
      const A old = static_cast<A>(tp_old);
#pragma unroll
      for (int k = 0; k + 1 < kPropAhead; ++k) {
        sp[k] = sp[k + 1];
        tp[k] = tp[k + 1];
      }
      {
        const bool in = y + kPropAhead < y1;
        sp[kPropAhead - 1] = in ? sq[kPropAhead * size] : T(0);
        tp[kPropAhead - 1] = in ? tq[kPropAhead * size] : T(0);
      }
      A I;
      if (y == 0) {
        I = A(0);
      } else if (y == 1) {
        I = c12 * (A(5) * r1 * s0 + A(8) * s1 - rinv * s2);
      } else if ((y & 1) == 0) {
        I = r2 * Ilast + c3 * (r2 * sm2 + A(4) * r1 * sm1 + sy);
        Iprev = Ilast;
        Ilast = I;
      } else {
        I = r3 * Iprev + c38 * (r3 * sm3 + A(3) * r2 * sm2 + A(3) * r1 * sm1 + sy);
      }
      sm3 = sm2;
      sm2 = sm1;
      sm1 = sy;
      A next = -I;
      if (damped) next = (A(1) - damp) * old + damp * next;
      const T stored = static_cast<T>(next);
      *tq = stored;
      if (canon) {   // the other three orientations of the antisymmetric element
        tq[mirror[0]] = -stored;
        tq[mirror[1]] = -stored;
        tq[mirror[2]] = stored;
      }
      // convergence maxima in the storage type, on what the next iteration reads
      dmax = max_abs(dmax, stored - tp_old);
      smax = max_abs(smax, stored);
      if (wE) {
        // canonical: the four orientations give 4 w s; the s1 s1 term reaches
        // two of them (a = i and its (ji)(ba) image)
        EA e = (canon ? EA(4) : EA(1)) * cE * static_cast<EA>(stored);
        if (NS == 4 && s1y) {
          e += (canon ? EA(1) : EA(0.5)) * static_cast<EA>(s1y[oi]) * static_cast<EA>(s1y[oj]);
          s1y += n1;
        }
        *ea += w * e;
      }
      sq += size;
      tq += size;
      ea += kPropThreads;
    }
    if (chain) {
      chain[mu] = static_cast<T>(Ilast);
      chain[size + mu] = static_cast<T>(Iprev);
      chain[2 * size + mu] = static_cast<T>(sm1);
      chain[3 * size + mu] = static_cast<T>(sm2);
      chain[4 * size + mu] = static_cast<T>(sm3);
    }
  }
  // The block's maxima are exact in any type; the energy sums run in EA and
  // the sum over blocks is FP64.
  __shared__ T dm[kPropThreads], sm[kPropThreads];
  dm[threadIdx.x] = dmax;
  sm[threadIdx.x] = smax;
  __syncthreads();
  // deterministic tree reductions
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      dm[threadIdx.x] = max_abs(dm[threadIdx.x], dm[threadIdx.x + s]);
      sm[threadIdx.x] = max_abs(sm[threadIdx.x], sm[threadIdx.x + s]);
    }
    __syncthreads();
  }
  // partials[q][block] (q = tau point, then the two maxima), so that the
  // reduction over blocks reads contiguous rows; one warp per tau point sums
  // the thread slots in a fixed order
  const long long nbk = a.nblocks;
  double* p = partials + blockIdx.x;
  for (int y = y0 + warp; y < y1; y += kPropThreads / 32) {
    EA acc = EA(0);
    for (int k = lane; k < kPropThreads; k += 32) acc += eacc[y * kPropThreads + k];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) p[y * nbk] = static_cast<double>(acc);
  }
  if (threadIdx.x == 0) {   // maxima over the launches of one iteration
    const double d0 = static_cast<double>(dm[0]), s0 = static_cast<double>(sm[0]);
    p[ng * nbk] = y0 == 0 ? d0 : fmax(p[ng * nbk], d0);
    p[(ng + 1) * nbk] = y0 == 0 ? s0 : fmax(p[(ng + 1) * nbk], s0);
  }
}

// Transposed propagation: u_x = sum_y G[y,x] exp(-Delta (tau_y - tau_x)) m_y,
// the adjoint of the Simpson recurrences above, run from the last tau point
// down with the even-chain adjoint E'_y = m_y + r^2 E'_{y+2} + r^3 m_{y+3}.
// Block-sparse doubles with a canonical list: u = P^T (pi m), pi the
// projection onto tensors antisymmetric in (i, j) and (a, b) (the mean of the
// four signed orientations): each canonical element is propagated once and
// written to its four orientations.  Every consumer of u contracts it with
// antisymmetric tensors (S2, its derivatives, the antisymmetric integrals),
// which see only pi u, and pi P^T m = P^T pi m; the elements with i = j or
// a = b are left alone (zero).
template <class T, int NS>
__global__ void __launch_bounds__(kPropThreads) propagate_t_kernel(const T* __restrict__ m, T* __restrict__ u,
                                                                   PropArgs a) {
  const int ng = a.ng;
  const int z = blockIdx.y;
  const long long size = a.size;
  m += static_cast<long long>(z) * ng * size;
  u += static_cast<long long>(z) * ng * size;
  const double* em = a.em + static_cast<long long>(z) * a.N;
  const double* ep = a.ep + static_cast<long long>(z) * a.N;
  const double h = a.hz[z];
  const bool sparse = a.imp != nullptr;
  const bool canon = sparse && NS == 4 && a.canon != nullptr;
  const long long nloop = canon ? a.ncanon : size;
  for (long long cidx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; cidx < nloop;
       cidx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long mu = canon ? a.canon[cidx] : cidx;
    int i, j = 0, aa, b = 0;
    long long o1 = 0, o2 = 0, o3 = 0;   // canonical: (j, i, a), (i, j, b), (j, i, b)
    if (sparse) {
      // [i][j][a] with b implied (a hole of the storage is skipped), or the
      // diagonal singles [i] (a = i)
      uint32_t r = static_cast<uint32_t>(mu);
      if (NS == 4) {
        uint32_t q = fdiv(a.fv, r);
        aa = r - q * a.nv;
        r = q;
        q = fdiv(a.fv, r);
        j = r - q * a.nv;
        i = q;
        b = a.imp[mu];
        if (b < 0) continue;
        if (canon) {
          const long long nn = a.nv;
          o1 = (static_cast<long long>(j) * nn + i) * nn + aa;
          o2 = (static_cast<long long>(i) * nn + j) * nn + b;
          o3 = (static_cast<long long>(j) * nn + i) * nn + b;
        }
      } else {
        i = aa = static_cast<int>(r);
      }
    } else {
      uint32_t r = static_cast<uint32_t>(mu);
      uint32_t q = fdiv(a.fv, r);
      if (NS == 4) {
        b = r - q * a.nv;
        r = q;
        q = fdiv(a.fv, r);
        aa = r - q * a.nv;
        r = q;
        q = fdiv(a.fo, r);
        j = r - q * a.no;
        i = q;
      } else {
        aa = r - q * a.nv;
        i = q;
      }
    }
    const int pi = a.idxO[i], pa = a.idxV[aa];
    double rr = em[pa] * ep[pi];
    double ri = ep[pa] * em[pi];
    if (NS == 4) {
      const int pj = a.idxO[j], pb = a.idxV[b];
      rr *= em[pb] * ep[pj];
      ri *= ep[pb] * em[pj];
    }
    const double r2 = rr * rr, r3 = r2 * rr;
    auto mval = [&](int x) -> double {
      const T* mr = m + static_cast<long long>(x) * size;
      if (!canon) return static_cast<double>(mr[mu]);
      return 0.25 * ((static_cast<double>(mr[mu]) - static_cast<double>(mr[o1])) -
                     (static_cast<double>(mr[o2]) - static_cast<double>(mr[o3])));
    };
    const double m1 = mval(1);
    double mp1 = 0.0, mp2 = 0.0, mp3 = 0.0;   // m_{x+1}, m_{x+2}, m_{x+3}
    double Ep1 = 0.0, Ep2 = 0.0;              // E'_{x+1}, E'_{x+2}
    for (int x = ng - 1; x >= 0; --x) {
      const double mx = mval(x);
      double Ex = 0.0;
      if ((x & 1) == 0 && x >= 2) Ex = mx + r2 * Ep2 + r3 * mp3;
      double ux = 0.0;
      if ((x & 1) == 0 && x >= 2) ux += h / 3.0 * Ex;
      if (((x + 1) & 1) == 0 && x + 1 >= 2 && x + 1 < ng) ux += 4.0 * h / 3.0 * rr * Ep1;
      if (((x + 2) & 1) == 0 && x + 2 < ng) ux += h / 3.0 * r2 * Ep2;
      if ((x & 1) == 1 && x >= 3) ux += 3.0 * h / 8.0 * mx;
      if (((x + 1) & 1) == 1 && x + 1 >= 3 && x + 1 < ng) ux += 9.0 * h / 8.0 * rr * mp1;
      if (((x + 2) & 1) == 1 && x + 2 >= 3 && x + 2 < ng) ux += 9.0 * h / 8.0 * r2 * mp2;
      if (((x + 3) & 1) == 1 && x + 3 >= 3 && x + 3 < ng) ux += 3.0 * h / 8.0 * r3 * mp3;
      if (x == 0) ux += 5.0 * h / 12.0 * rr * m1;
      if (x == 1) ux += 8.0 * h / 12.0 * m1;
      if (x == 2) ux -= h / 12.0 * ri * m1;
      T* ur = u + static_cast<long long>(x) * size;
      ur[mu] = static_cast<T>(ux);
      if (canon) {
        ur[o1] = static_cast<T>(-ux);
        ur[o2] = static_cast<T>(-ux);
        ur[o3] = static_cast<T>(ux);
      }
      mp3 = mp2;
      mp2 = mp1;
      mp1 = mx;
      Ep2 = Ep1;
      Ep1 = Ex;
    }
  }
}

// m_new = -c_x (f_ov + <ij||ab> s_j^b) - tbar (singles) or -c_x/4 <ij||ab> - tbar
// (doubles), c_x = g_x / beta, and per-block max|m_new - m_old|, max|m_new|.
// E'(s) is the derivative of E (Eq. E) with respect to the amplitudes.
template <class T, class BT>
__global__ void lambda_combine_kernel(const BT* __restrict__ base, const T* __restrict__ tbar,
                                      T* __restrict__ mnew, const T* __restrict__ mold, long long size, int ng,
                                      int nz, const double* __restrict__ cz, double cbase, double* partials,
                                      const int* __restrict__ list, int nlist) {
  __shared__ double dm[256], sm[256];
  double dmax = 0.0, smax = 0.0;
  if (list) {
    // block-sparse doubles: only the valid positions (the holes of base, tbar
    // and m are zero and stay so); slices outer, no index division
    const int stride = gridDim.x * blockDim.x;
    for (int zx = 0; zx < nz * ng; ++zx) {
      const double c = cz[zx];
      const int z = zx / ng;
      const BT* bz = base + static_cast<long long>(z) * size * (cbase != 0.0 ? 1 : ng) +
                     (cbase != 0.0 ? 0 : static_cast<long long>(zx - z * ng) * size);
      for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nlist; k += stride) {
        const long long mu = list[k];
        const long long e = static_cast<long long>(zx) * size + mu;
        const double bval = static_cast<double>(bz[mu]);
        const double v = -c * (cbase != 0.0 ? cbase * bval : bval) - static_cast<double>(tbar[e]);
        const T vs = static_cast<T>(v);
        dmax = fmax(dmax, fabs(static_cast<double>(vs) - static_cast<double>(mold[e])));
        smax = fmax(smax, fabs(static_cast<double>(vs)));
        mnew[e] = vs;
      }
    }
  }
  const long long total = list ? 0 : static_cast<long long>(nz) * ng * size;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long zx = e / size;
    const long long mu = e - zx * size;
    const long long z = zx / ng;
    const int x = static_cast<int>(zx - z * ng);
    const double c = cz[z * ng + x];
    const double bval = static_cast<double>(base[z * size * (cbase != 0.0 ? 1 : ng) + (cbase != 0.0 ? mu : x * size + mu)]);
    const double v = -c * (cbase != 0.0 ? cbase * bval : bval) - static_cast<double>(tbar[e]);
    const T vs = static_cast<T>(v);
    dmax = fmax(dmax, fabs(static_cast<double>(vs) - static_cast<double>(mold[e])));
    smax = fmax(smax, fabs(static_cast<double>(vs)));
    mnew[e] = vs;
  }
  dm[threadIdx.x] = dmax;
  sm[threadIdx.x] = smax;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      dm[threadIdx.x] = fmax(dm[threadIdx.x], dm[threadIdx.x + s]);
      sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = dm[0];
    partials[2 * blockIdx.x + 1] = sm[0];
  }
}

// Response sums of one thermal block (App. B): with I the block and A its
// Lagrangian adjoint, Do[z][q] += sum of A*I over the elements whose hole-like
// slot holds orbital position q, Dv likewise for particle-like slots.  These
// are the derivatives of the Lagrangian with respect to log sqrt(n_q) and
// log sqrt(1 - n_q).
template <class T>
__global__ void slot_sums_kernel(const T* __restrict__ I, const T* __restrict__ A, int nslot, int d0, int d1,
                                 int d2, int d3, int cls, int no, int nv, double* Do, double* Dv) {
  const int z = blockIdx.y;
  const long long per = static_cast<long long>(d0) * d1 * d2 * d3;
  I += z * per;
  A += z * per;
  Do += static_cast<long long>(z) * no;
  Dv += static_cast<long long>(z) * nv;
  const int dims[4] = {d0, d1, d2, d3};
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < per;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const double p = static_cast<double>(I[e]) * static_cast<double>(A[e]);
    if (p == 0.0) continue;
    long long r = e;
    int c[4];
    for (int k = nslot - 1; k >= 0; --k) {
      c[k] = static_cast<int>(r % dims[k]);
      r /= dims[k];
    }
    for (int k = 0; k < nslot; ++k) {
      if ((cls >> k) & 1) atomicAdd(&Dv[c[k]], p);
      else atomicAdd(&Do[c[k]], p);
    }
  }
}

// dL/dFbar[p][q] += A[a][b] fac0[a] fac1[b] for a thermal Fock block.
template <class T>
__global__ void fbar_scatter_kernel(const T* __restrict__ A, int n0, int n1, const int* i0, const double* f0,
                                    long long f0z, const int* i1, const double* f1, long long f1z, int N, double* Fb) {
  const int z = blockIdx.y;
  A += static_cast<long long>(z) * n0 * n1;
  f0 += z * f0z;
  f1 += z * f1z;
  Fb += static_cast<long long>(z) * N * N;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n0 * n1) return;
  const int a = e / n1, b = e % n1;
  atomicAdd(&Fb[static_cast<long long>(i0[a]) * N + i1[b]], static_cast<double>(A[e]) * f0[a] * f1[b]);
}

// Gn[z][r] = sum_pq Fb[z][p][q] <pr||qr>: the occupation dependence of the
// thermal Fock matrix f = h + sum_r n_r <pr||qr>.
__global__ void fock_n_kernel(const double* __restrict__ Fb, const double* __restrict__ eri, int N, double* Gn) {
  const int r = blockIdx.x;
  __shared__ double red[256];
  double acc = 0.0;
  for (long long pq = threadIdx.x; pq < static_cast<long long>(N) * N; pq += blockDim.x) {
    const long long p = pq / N, q = pq % N;
    acc += Fb[pq] * eri[((p * N + r) * N + q) * N + r];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) Gn[r] = red[0];
}

// Propagator dependence of the Lagrangian: per element, with I_y the Simpson
// integral of S (so s = -I) and J_y = sum_x G[y,x] (tau_y - tau_x) e^{-Delta(tau_y - tau_x)} S_x
// (from the r-derivative of the recurrences, J = h r dI/dr):
//   dL/dDelta_mu = -sum_y m_y J_y,   beta dL/dbeta|prop = sum_y m_y (I_y - Delta J_y).
// Accumulated per orbital (dL/deps_q = sum_mu dL/dDelta_mu dDelta_mu/deps_q)
// and per instance (beta part).
template <class T, int NS>
__global__ void __launch_bounds__(kPropThreads) prop_response_kernel(const T* __restrict__ S,
                                                                     const T* __restrict__ m, const double* __restrict__ epsz,
                                                                     PropArgs a, double* Ee, double* Eb) {
  const int ng = a.ng;
  const int z = blockIdx.y;
  const long long size = a.size;
  S += static_cast<long long>(z) * ng * size;
  m += static_cast<long long>(z) * ng * size;
  const double* em = a.em + static_cast<long long>(z) * a.N;
  const double* ep = a.ep + static_cast<long long>(z) * a.N;
  const double* eps = epsz + static_cast<long long>(z) * a.N;
  const double h = a.hz[z];
  __shared__ double bred[kPropThreads];
  double bsum = 0.0;
  const bool sparse = a.imp != nullptr;
  for (long long mu = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; mu < size;
       mu += static_cast<long long>(gridDim.x) * blockDim.x) {
    int i, j = 0, aa, b = 0;
    if (sparse) {
      // [i][j][a] with b implied (a hole of the storage is skipped), or the
      // diagonal singles [i] (a = i)
      uint32_t r = static_cast<uint32_t>(mu);
      if (NS == 4) {
        uint32_t q = fdiv(a.fv, r);
        aa = r - q * a.nv;
        r = q;
        q = fdiv(a.fv, r);
        j = r - q * a.nv;
        i = q;
        b = a.imp[mu];
        if (b < 0) continue;
      } else {
        i = aa = static_cast<int>(r);
      }
    } else {
      uint32_t r = static_cast<uint32_t>(mu);
      uint32_t q = fdiv(a.fv, r);
      if (NS == 4) {
        b = r - q * a.nv;
        r = q;
        q = fdiv(a.fv, r);
        aa = r - q * a.nv;
        r = q;
        q = fdiv(a.fo, r);
        j = r - q * a.no;
        i = q;
      } else {
        aa = r - q * a.nv;
        i = q;
      }
    }
    const int pi = a.idxO[i], pa = a.idxV[aa];
    double rr = em[pa] * ep[pi];
    double ri = ep[pa] * em[pi];
    double delta = eps[pa] - eps[pi];
    int pj = 0, pb = 0;
    if (NS == 4) {
      pj = a.idxO[j];
      pb = a.idxV[b];
      rr *= em[pb] * ep[pj];
      ri *= ep[pb] * em[pj];
      delta += eps[pb] - eps[pj];
    }
    const double r2 = rr * rr, r3 = r2 * rr;
    const double s0 = static_cast<double>(S[mu]), s1 = static_cast<double>(S[size + mu]),
                 s2 = static_cast<double>(S[2 * size + mu]);
    double sm1 = 0.0, sm2 = 0.0, sm3 = 0.0;
    double Il = 0.0, Ip = 0.0, dIl = 0.0, dIp = 0.0;   // last / second-last even I and dI/dr
    double P1 = 0.0, K = 0.0;
    for (int y = 0; y < ng; ++y) {
      const double sy =
          y == 0 ? s0 : (y == 1 ? s1 : (y == 2 ? s2 : static_cast<double>(S[static_cast<long long>(y) * size + mu])));
      double I, dI;
      if (y == 0) {
        I = 0.0;
        dI = 0.0;
      } else if (y == 1) {
        I = h / 12.0 * (5.0 * rr * s0 + 8.0 * s1 - ri * s2);
        dI = h / 12.0 * (5.0 * s0 + ri * ri * s2);
      } else if ((y & 1) == 0) {
        I = r2 * Il + h / 3.0 * (r2 * sm2 + 4.0 * rr * sm1 + sy);
        dI = 2.0 * rr * Il + r2 * dIl + h / 3.0 * (2.0 * rr * sm2 + 4.0 * sm1);
        Ip = Il;
        dIp = dIl;
        Il = I;
        dIl = dI;
      } else {
        I = r3 * Ip + 3.0 * h / 8.0 * (r3 * sm3 + 3.0 * r2 * sm2 + 3.0 * rr * sm1 + sy);
        dI = 3.0 * r2 * Ip + r3 * dIp + 3.0 * h / 8.0 * (3.0 * r2 * sm3 + 6.0 * rr * sm2 + 3.0 * sm1);
      }
      sm3 = sm2;
      sm2 = sm1;
      sm1 = sy;
      const double my = static_cast<double>(m[static_cast<long long>(y) * size + mu]);
      P1 += my * I;
      K += my * h * rr * dI;
    }
    // dL/dDelta = -K; dDelta/deps: +1 for particle slots, -1 for hole slots
    if (K != 0.0) {
      atomicAdd(&Ee[static_cast<long long>(z) * a.N + pa], -K);
      atomicAdd(&Ee[static_cast<long long>(z) * a.N + pi], K);
      if (NS == 4) {
        atomicAdd(&Ee[static_cast<long long>(z) * a.N + pb], -K);
        atomicAdd(&Ee[static_cast<long long>(z) * a.N + pj], K);
      }
    }
    bsum += P1 - delta * K;
  }
  bred[threadIdx.x] = bsum;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) bred[threadIdx.x] += bred[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&Eb[z], bred[0]);
}

__device__ double simpson_weight(int y, int ng) {
  // g = G^{ng-1} in units of h: composite Simpson 1/3, with Simpson 3/8 on the
  // last three intervals when the interval count is odd
  const int last = ng - 1;
  if ((last & 1) == 0) {
    if (y == 0 || y == last) return 1.0 / 3.0;
    return (y & 1) ? 4.0 / 3.0 : 2.0 / 3.0;
  }
  if (last == 1) return y == 0 ? 5.0 / 12.0 : (y == 1 ? 8.0 / 12.0 : -1.0 / 12.0);
  const int m = last - 3;   // Simpson 1/3 on [0, m] then 3/8 on [m, last]
  double w = 0.0;
  if (y <= m && m > 0) {
    if (y == 0 || y == m) w += 1.0 / 3.0;
    else w += (y & 1) ? 4.0 / 3.0 : 2.0 / 3.0;
  }
  if (y >= m) {
    const int k = y - m;
    w += (k == 0 || k == 3) ? 3.0 / 8.0 : 9.0 / 8.0;
  }
  return w;
}

// Block (q, z) reduces quantity q of instance z (E_y for y < ng, then
// max|ds|, max|s|) over the partial rows of both propagation passes: thread
// t takes rows t, t + 256, ... in order, then a fixed shuffle tree and the
// eight warp results in order, so the result is bitwise reproducible.  The
// rows are spread over (ng + 2) x nz blocks because FP64 adds issue at a few
// per clock per SM on this part.  The last block of an instance to finish
// (counter in state[6]) forms Omega_CC from the E_y in a fixed order and
// resets the counter.
constexpr int kReduceThreads = 256;
__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(const double* __restrict__ p1, int nb1,
                                                                const double* __restrict__ p2, int nb2, int ng, int nz,
                                                                const double* __restrict__ hz,
                                                                const int* __restrict__ live, double* state) {
  const int q = blockIdx.x, z = blockIdx.y;
  if (live && !live[z]) return;
  p1 += static_cast<long long>(z) * nb1 * (ng + 2) + static_cast<long long>(q) * nb1;   // partials are [q][block]
  p2 += static_cast<long long>(z) * nb2 * (ng + 2) + static_cast<long long>(q) * nb2;
  state += static_cast<long long>(z) * (8 + 256);
  const bool is_max = q >= ng;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb1; b += kReduceThreads) acc = is_max ? fmax(acc, p1[b]) : acc + p1[b];
  for (int b = threadIdx.x; b < nb2; b += kReduceThreads) acc = is_max ? fmax(acc, p2[b]) : acc + p2[b];
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_down_sync(0xffffffffu, acc, off);
    acc = is_max ? fmax(acc, o) : acc + o;
  }
  __shared__ double wsum[kReduceThreads / 32];
  __shared__ bool last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) wsum[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = wsum[0];
    for (int w = 1; w < kReduceThreads / 32; ++w) v = is_max ? fmax(v, wsum[w]) : v + wsum[w];
    state[q < ng ? 8 + q : 4 + (q - ng)] = v;   // E_y, or state[4] max|ds|, state[5] max|s|
    __threadfence();
    unsigned long long* count = reinterpret_cast<unsigned long long*>(state + 6);
    last = atomicAdd(count, 1ull) == static_cast<unsigned long long>(ng + 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  const volatile double* vs = state;
  const double beta = hz[nz + z];
  const double h = beta / (ng - 1);
  double om = 0.0;
  for (int y = 0; y < ng; ++y) om += simpson_weight(y, ng) * h * vs[8 + y];
  om /= beta;
  const double prev = state[0];
  state[3] = prev;
  state[0] = om;
  state[1] = fabs(om - prev);
  state[2] = vs[4] / fmax(1.0, vs[5]);
  *reinterpret_cast<unsigned long long*>(state + 6) = 0ull;
}

}  // namespace

// ----------------------------------------------------------------- launchers
namespace {
// Host side of the tiled permute: choose the tile letters and their extents,
// the per-term read orders and the block decomposition.
struct PermPlan {
  int nd = 0, nterm = 1;
  long long dim[kMaxL] = {}, sst[kPermTerms][kMaxL] = {}, dstr[kMaxL] = {};
  const void* src[kPermTerms] = {};
  double coef[kPermTerms] = {};
};

template <class T, bool SPLIT>
cudaError_t run_permute(const PermPlan& P0, PermOut<T> out, double alpha, double beta, cudaStream_t st) {
  if (P0.nd < 1 || P0.nd > kMaxL || P0.nterm < 1 || P0.nterm > kPermTerms) return cudaErrorInvalidValue;
  long long total = 1;
  for (int k = 0; k < P0.nd; ++k) total *= P0.dim[k];
  if (total == 0) return cudaSuccess;
  // Drop letters of extent 1 and merge neighbouring destination letters that
  // are neighbours in the same order in every term's source: fewer, longer
  // letters mean longer contiguous runs and less index arithmetic.
  PermPlan P;
  P.nterm = P0.nterm;
  for (int p = 0; p < P0.nterm; ++p) {
    P.src[p] = P0.src[p];
    P.coef[p] = P0.coef[p];
  }
  for (int k = P0.nd - 1; k >= 0; --k) {   // innermost first; P is built reversed
    if (P0.dim[k] == 1) continue;
    bool merge = P.nd > 0;
    if (merge) {
      const int g = P.nd - 1;
      merge = P0.dstr[k] == P.dstr[g] * P.dim[g];
      for (int p = 0; p < P0.nterm && merge; ++p) merge = P0.sst[p][k] == P.sst[p][g] * P.dim[g];
      if (merge && P.dim[g] * P0.dim[k] >= (1LL << 31)) merge = false;
      if (merge) {
        P.dim[g] *= P0.dim[k];
        continue;
      }
    }
    P.dim[P.nd] = P0.dim[k];
    P.dstr[P.nd] = P0.dstr[k];
    for (int p = 0; p < P0.nterm; ++p) P.sst[p][P.nd] = P0.sst[p][k];
    ++P.nd;
  }
  if (P.nd == 0) {   // a single element
    P.nd = 1;
    P.dim[0] = 1;
    P.dstr[0] = 1;
    for (int p = 0; p < P0.nterm; ++p) P.sst[p][0] = 0;
  }
  for (int a = 0, b = P.nd - 1; a < b; ++a, --b) {   // back to outermost first
    std::swap(P.dim[a], P.dim[b]);
    std::swap(P.dstr[a], P.dstr[b]);
    for (int p = 0; p < P.nterm; ++p) std::swap(P.sst[p][a], P.sst[p][b]);
  }
  const int nd = P.nd;
  // tile letters: dst innermost, then each term's unit-stride letter
  auto argmin = [&](const long long* st_) {
    int best = -1;
    for (int k = 0; k < nd; ++k)
      if (P.dim[k] > 1 && st_[k] > 0 && (best < 0 || st_[k] < st_[best])) best = k;
    return best;
  };
  int tl[kMaxL], nt = 0;
  auto add = [&](int k) {
    if (k < 0) return;
    for (int l = 0; l < nt; ++l)
      if (tl[l] == k) return;
    tl[nt++] = k;
  };
  add(argmin(P.dstr));
  for (int p = 0; p < P.nterm; ++p) {
    bool bcast = false;   // a broadcast source is small and read from cache
    for (int k = 0; k < nd; ++k) bcast |= P.dim[k] > 1 && P.sst[p][k] == 0;
    if (!bcast) add(argmin(P.sst[p]));
  }
  if (nt == 0) add(nd - 1);
  long long ext[kMaxL];
  for (int l = 0; l < nt; ++l) ext[l] = P.dim[tl[l]];
  auto prod = [&]() {
    long long v = 1;
    for (int l = 0; l < nt; ++l) v *= ext[l];
    return v;
  };
  // a small tensor gets smaller tiles, so that its blocks cover about two per
  // SM instead of a few SMs running long blocks
  const long long tile_cap = std::max<long long>(256, std::min<long long>(kPermTile, total / (2 * 152)));
  while (prod() > tile_cap) {   // shrink the widest extent
    int w = 0;
    for (int l = 1; l < nt; ++l)
      if (ext[l] > ext[w]) w = l;
    ext[w] = (ext[w] + 1) / 2;
  }
  // grow with destination letters, innermost first: whole letters while they
  // fit, then a part of the next one (long contiguous destination runs and
  // enough work per block to hide the phase latencies)
  {
    int order[kMaxL];
    for (int k = 0; k < nd; ++k) order[k] = k;
    std::sort(order, order + nd, [&](int a, int b) { return P.dstr[a] < P.dstr[b]; });
    for (int i = 0; i < nd; ++i) {
      const int k = order[i];
      bool in = false;
      for (int l = 0; l < nt; ++l) in |= tl[l] == k;
      if (in || P.dim[k] <= 1) continue;
      const long long room = tile_cap / prod();
      if (room < 2) break;
      tl[nt] = k;
      ext[nt] = std::min<long long>(P.dim[k], room);
      ++nt;
      if (ext[nt - 1] < P.dim[k]) break;
    }
  }
  DevPerm d{};
  d.nd = nd;
  d.nterm = P.nterm;
  d.nt = nt;
  for (int p = 0; p < P.nterm; ++p) {
    d.src[p] = P.src[p];
    d.coef[p] = P.coef[p];
  }
  for (int k = 0; k < nd; ++k) {
    d.tslot[k] = -1;
    d.dstr[k] = P.dstr[k];
    for (int p = 0; p < P.nterm; ++p) d.sst[p][k] = P.sst[p][k];
  }
  unsigned long long nblocks = 1;
  for (int k = 0; k < nd; ++k) {
    long long cnt = P.dim[k], step = 1;
    for (int l = 0; l < nt; ++l)
      if (tl[l] == k) {
        d.tslot[k] = l;
        cnt = (P.dim[k] + ext[l] - 1) / ext[l];
        step = ext[l];
        d.tail_blk[l] = static_cast<int>(cnt - 1);
        d.ext_full[l] = static_cast<int>(ext[l]);
        d.ext_tail[l] = static_cast<int>(P.dim[k] - (cnt - 1) * ext[l]);
      }
    if (cnt >= (1LL << 32)) return cudaErrorInvalidValue;
    d.bcnt[k] = make_fastdiv(static_cast<uint32_t>(cnt));
    d.bstep[k] = static_cast<int>(step);
    nblocks *= static_cast<unsigned long long>(cnt);
  }
  if (nblocks >= (1ULL << 32)) return cudaErrorInvalidValue;
  // orders: terms by source stride, the write by destination stride; the
  // shared-memory tile is dense in write order
  int word[kMaxL];
  for (int l = 0; l < nt; ++l) word[l] = l;
  std::sort(word, word + nt, [&](int a, int b) { return P.dstr[tl[a]] < P.dstr[tl[b]]; });
  int tstr[kMaxL];
  long long tile_elems = 1;
  {
    // dense in write order, except that the stride after the fastest letter
    // is made odd so that a transposed pass hits 32 different banks
    long long dense = 1;
    for (int l = 0; l < nt; ++l) dense *= ext[l];
    const bool pad = nt > 1 && (ext[word[0]] & 1) == 0 &&
                     static_cast<size_t>(dense / ext[word[0]] * (ext[word[0]] + 1)) * sizeof(T) <= 40 * 1024;
    long long acc = 1;
    for (int i = 0; i < nt; ++i) {
      tstr[word[i]] = static_cast<int>(acc);
      acc *= ext[word[i]];
      if (i == 0 && pad) acc += 1;
    }
    tile_elems = acc;
  }
  auto fill = [&](int o, const int* ord, const long long* gst) {
    for (int i = 0; i < nt; ++i) {
      const int l = ord[i];
      d.slot[o][i] = l;
      d.fd_full[o][i] = make_fastdiv(static_cast<uint32_t>(d.ext_full[l]));
      d.fd_tail[o][i] = make_fastdiv(static_cast<uint32_t>(d.ext_tail[l]));
      d.gstr[o][i] = gst[tl[l]];
      d.tstr[o][i] = tstr[l];
    }
  };
  for (int p = 0; p < P.nterm; ++p) {
    int ord[kMaxL];
    for (int l = 0; l < nt; ++l) ord[l] = l;
    std::stable_sort(ord, ord + nt, [&](int a, int b) {
      const long long sa = P.sst[p][tl[a]], sb = P.sst[p][tl[b]];
      return (sa == 0 ? LLONG_MAX : sa) < (sb == 0 ? LLONG_MAX : sb);
    });
    fill(p, ord, P.sst[p]);
  }
  fill(kPermTerms, word, P.dstr);
  // 16-byte global accesses when every order's fastest tile letter has unit
  // stride and an extent (full and tail) that is a multiple of the vector
  // width, every other stride and every block's base offset is a multiple
  // of it, and the tensors start on 16-byte boundaries
  constexpr int kVW = 16 / sizeof(T);
  // (a split writes VW bf16 halves: 8-byte aligned hi and lo arrays)
  bool vec = SPLIT ? (sizeof(T) == 4 && reinterpret_cast<uintptr_t>(out.hi) % 8 == 0 &&
                      reinterpret_cast<uintptr_t>(out.lo) % 8 == 0)
                   : reinterpret_cast<uintptr_t>(out.dst) % 16 == 0;
  for (int o = 0; o <= P.nterm && vec; ++o) {
    const int oo = o == P.nterm ? kPermTerms : o;
    const int l0 = d.slot[oo][0];
    vec = d.gstr[oo][0] == 1 && d.ext_full[l0] % kVW == 0 && d.ext_tail[l0] % kVW == 0;
    for (int i = 1; i < nt && vec; ++i) vec = d.gstr[oo][i] % kVW == 0;
    if (o < P.nterm) vec = vec && reinterpret_cast<uintptr_t>(P.src[o]) % 16 == 0;
    for (int k = 0; k < nd && vec; ++k)
      vec = (static_cast<long long>(d.bstep[k]) * (o < P.nterm ? P.sst[o][k] : P.dstr[k])) % kVW == 0;
  }
  const size_t smem = static_cast<size_t>(tile_elems) * sizeof(T);
  for (unsigned long long b0 = 0; b0 < nblocks; b0 += 0x7FFFFFFFull) {
    d.block0 = static_cast<uint32_t>(b0);
    const unsigned int g = static_cast<unsigned int>(std::min<unsigned long long>(nblocks - b0, 0x7FFFFFFFull));
    if (vec)
      permute_kernel<T, SPLIT && sizeof(T) == 4, kVW><<<g, kPermThreads, smem, st>>>(out, d, static_cast<T>(alpha),
                                                                                     static_cast<T>(beta));
    else
      permute_kernel<T, SPLIT, 1><<<g, kPermThreads, smem, st>>>(out, d, static_cast<T>(alpha), static_cast<T>(beta));
  }
  return cudaGetLastError();
}

PermPlan pack_plan(const void* src, const PackDesc& d) {
  PermPlan P;
  P.nd = d.nr + d.nc;
  P.nterm = 1;
  P.src[0] = src;
  P.coef[0] = 1.0;
  long long s = 1;
  for (int k = d.nc - 1; k >= 0; --k) {
    P.dim[d.nr + k] = d.cdim[k];
    P.sst[0][d.nr + k] = d.cst[k];
    P.dstr[d.nr + k] = s;
    s *= d.cdim[k];
  }
  s = d.cpad;
  for (int k = d.nr - 1; k >= 0; --k) {
    P.dim[k] = d.rdim[k];
    P.sst[0][k] = d.rst[k];
    P.dstr[k] = s;
    s *= d.rdim[k];
  }
  return P;
}
}  // namespace

template <class T>
cudaError_t launch_pack(const T* src, T* dst, const PackDesc& d, cudaStream_t st) {
  if (d.rows <= 0 || d.creal <= 0) return cudaSuccess;
  return run_permute<T, false>(pack_plan(src, d), PermOut<T>{dst, nullptr, nullptr}, 1.0, 0.0, st);
}
template cudaError_t launch_pack<float>(const float*, float*, const PackDesc&, cudaStream_t);
template cudaError_t launch_pack<double>(const double*, double*, const PackDesc&, cudaStream_t);

// ---- unordered index pairs (p < q) of antisymmetric tensors
// pair index of (p, q), p < q, among the n(n-1)/2 pairs in row order
__device__ __forceinline__ long long pair_index(int p, int q, int n) {
  return static_cast<long long>(p) * n - static_cast<long long>(p) * (p + 1) / 2 + (q - p - 1);
}

// dst[b][P][Q] = coef * X(l0, l1, l2, l3) over pairs P = (l0 < l1) of n1
// and Q = (l2 < l3) of n2, X read through the strides s0..s3 (sb per batch
// entry); with anti the first pair is antisymmetrised on the way,
// X -> (X(l0, l1, ..) - X(l1, l0, ..)) / 2.  pairs1 / pairs2 hold the
// (p, q) of every pair index.
template <class T>
__global__ void pair_pack_kernel(const T* __restrict__ src, T* __restrict__ dst, long long nb, long long sb,
                                 const int2* __restrict__ pairs1, long long np1, const int2* __restrict__ pairs2,
                                 long long np2, long long s0, long long s1, long long s2, long long s3, int anti,
                                 T coef) {
  // one batch entry per blockIdx.y; 32-bit indices within it (a 64-bit
  // division per element costs a long instruction sequence)
  const uint32_t per = static_cast<uint32_t>(np1 * np2), n2 = static_cast<uint32_t>(np2);
  for (long long b = blockIdx.y; b < nb; b += gridDim.y) {
    const T* xb = src + b * sb;
    T* db = dst + b * static_cast<long long>(per);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < per; e += gridDim.x * blockDim.x) {
      const uint32_t p = e / n2, q = e - p * n2;
      const int2 a = pairs1[p], c = pairs2[q];
      const T* x = xb + c.x * s2 + c.y * s3;
      T v = x[a.x * s0 + a.y * s1];
      if (anti) v = T(0.5) * (v - x[a.y * s0 + a.x * s1]);
      db[e] = coef * v;
    }
  }
}

// R[b][i][j][a][c] += coef * sgn * L[b][pair(i, j)][pair(a, c)] with sgn the
// sign of the two orderings (zero where i = j or a = c): adds the dense
// antisymmetric tensor of a pair-packed one.
template <class T>
__global__ void pair_unpack_add_kernel(T* __restrict__ R, const T* __restrict__ L, long long nb, int no, int nv,
                                       T coef) {
  const long long npo = static_cast<long long>(no) * (no - 1) / 2, npv = static_cast<long long>(nv) * (nv - 1) / 2;
  const uint32_t per = static_cast<uint32_t>(no) * no * nv * nv, uo = no, uv = nv;
  for (long long b = blockIdx.y; b < nb; b += gridDim.y) {
    T* Rb = R + b * static_cast<long long>(per);
    const T* Lb = L + b * npo * npv;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < per; e += gridDim.x * blockDim.x) {
      uint32_t r = e, q = r / uv;
      const int c = static_cast<int>(r - q * uv);
      r = q;
      q = r / uv;
      const int a = static_cast<int>(r - q * uv);
      r = q;
      q = r / uo;
      const int j = static_cast<int>(r - q * uo);
      const int i = static_cast<int>(q);
      if (i == j || a == c) continue;
      const long long P = i < j ? pair_index(i, j, no) : pair_index(j, i, no);
      const long long Q = a < c ? pair_index(a, c, nv) : pair_index(c, a, nv);
      const T v = Lb[P * npv + Q];
      Rb[e] += ((i < j) == (a < c)) ? coef * v : -coef * v;
    }
  }
}

template <class T>
cudaError_t launch_pair_pack(const T* src, T* dst, long long nb, long long sb, const int2* pairs1, long long np1,
                             const int2* pairs2, long long np2, long long s0, long long s1, long long s2, long long s3,
                             int anti, double coef, cudaStream_t st) {
  const long long per = np1 * np2;
  if (nb <= 0 || per <= 0) return cudaSuccess;
  if (per >= (1LL << 31)) return cudaErrorInvalidValue;
  const int by = static_cast<int>(std::min<long long>(nb, 65535));
  const int blocks = static_cast<int>(std::max<long long>(1, std::min<long long>((per + 255) / 256, 152LL * 16 / by + 1)));
  pair_pack_kernel<T><<<dim3(blocks, by), 256, 0, st>>>(src, dst, nb, sb, pairs1, np1, pairs2, np2, s0, s1, s2, s3, anti,
                                              static_cast<T>(coef));
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_pair_unpack_add(T* R, const T* L, long long nb, int no, int nv, double coef, cudaStream_t st) {
  const long long per = static_cast<long long>(no) * no * nv * nv;
  if (nb <= 0 || per <= 0 || no < 2 || nv < 2) return cudaSuccess;
  if (per >= (1LL << 31)) return cudaErrorInvalidValue;
  const int by = static_cast<int>(std::min<long long>(nb, 65535));
  const int blocks = static_cast<int>(std::max<long long>(1, std::min<long long>((per + 255) / 256, 152LL * 16 / by + 1)));
  pair_unpack_add_kernel<T><<<dim3(blocks, by), 256, 0, st>>>(R, L, nb, no, nv, static_cast<T>(coef));
  return cudaGetLastError();
}
template cudaError_t launch_pair_pack<float>(const float*, float*, long long, long long, const int2*, long long,
                                             const int2*, long long, long long, long long, long long, long long, int,
                                             double, cudaStream_t);
template cudaError_t launch_pair_pack<double>(const double*, double*, long long, long long, const int2*, long long,
                                              const int2*, long long, long long, long long, long long, long long, int,
                                              double, cudaStream_t);
template cudaError_t launch_pair_unpack_add<float>(float*, const float*, long long, int, int, double, cudaStream_t);
template cudaError_t launch_pair_unpack_add<double>(double*, const double*, long long, int, int, double, cudaStream_t);

// ---- fast paths of the layout engine for contiguous rows
// hi/lo halves of rows already in GEMM order: src[r][k] (row stride sld) ->
// hi[r][k], lo[r][k] (row stride ld), k < K.  With K, sld and ld multiples of
// four (and aligned bases) a thread moves four floats in one 16-byte load and
// four bf16 halves in one 8-byte store each.
template <bool VEC>
__global__ void split_rows_kernel(const float* __restrict__ src, long long sld, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo, long long ld, long long rows, long long K) {
  const long long per = VEC ? K / 4 : K;
  const long long total = rows * per;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = e / per, c = e - r * per;
    if constexpr (VEC) {
      const float4 v = *reinterpret_cast<const float4*>(src + r * sld + 4 * c);
      const float x[4] = {v.x, v.y, v.z, v.w};
      __nv_bfloat162 h2[2], l2[2];
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        const __nv_bfloat16 ha = __float2bfloat16_rn(x[2 * w]), hb = __float2bfloat16_rn(x[2 * w + 1]);
        h2[w] = __halves2bfloat162(ha, hb);
        l2[w] = __halves2bfloat162(__float2bfloat16_rn(x[2 * w] - __bfloat162float(ha)),
                                   __float2bfloat16_rn(x[2 * w + 1] - __bfloat162float(hb)));
      }
      uint2 uh, ul;
      uh.x = *reinterpret_cast<const uint32_t*>(&h2[0]);
      uh.y = *reinterpret_cast<const uint32_t*>(&h2[1]);
      ul.x = *reinterpret_cast<const uint32_t*>(&l2[0]);
      ul.y = *reinterpret_cast<const uint32_t*>(&l2[1]);
      *reinterpret_cast<uint2*>(hi + r * ld + 4 * c) = uh;
      *reinterpret_cast<uint2*>(lo + r * ld + 4 * c) = ul;
    } else {
      const float v = src[r * sld + c];
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      hi[r * ld + c] = h;
      lo[r * ld + c] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

cudaError_t launch_split_rows(const float* src, long long sld, void* hi, void* lo, long long ld, long long rows,
                              long long K, cudaStream_t st) {
  if (rows <= 0 || K <= 0) return cudaSuccess;
  if (sld < K || ld < K) return cudaErrorInvalidValue;
  const bool vec = K % 4 == 0 && sld % 4 == 0 && ld % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(hi) % 8 == 0 && reinterpret_cast<uintptr_t>(lo) % 8 == 0;
  const long long work = vec ? rows * (K / 4) : rows * K;
  const int blocks = static_cast<int>(std::min<long long>((work + 255) / 256, 152LL * 16));
  if (vec)
    split_rows_kernel<true><<<blocks, 256, 0, st>>>(src, sld, static_cast<__nv_bfloat16*>(hi),
                                                    static_cast<__nv_bfloat16*>(lo), ld, rows, K);
  else
    split_rows_kernel<false><<<blocks, 256, 0, st>>>(src, sld, static_cast<__nv_bfloat16*>(hi),
                                                     static_cast<__nv_bfloat16*>(lo), ld, rows, K);
  return cudaGetLastError();
}

// dst[o][q] = beta * dst[o][q] + alpha * src[soff(o) + q] for a destination
// whose last letters form one contiguous block of B elements that the
// source holds in the same order: o runs over the destination's leading
// letters (blockIdx.y), soff(o) = sum_k c_k(o) * sst_k with sst_k = 0 for a
// letter the source lacks (broadcast).  VW elements per access.
template <class T, int VW>
__global__ void block_copy_kernel(T* __restrict__ dst, const T* __restrict__ src, long long B, BlockCopyDesc d,
                                  T alpha, T beta) {
  long long o = blockIdx.y, soff = 0;
#pragma unroll
  for (int k = kMaxL - 1; k >= 0; --k) {
    if (k < d.nouter) {
      const long long c = o % d.dim[k];
      o /= d.dim[k];
      soff += c * d.sst[k];
    }
  }
  T* dp = dst + static_cast<long long>(blockIdx.y) * B;
  const T* sp = src + soff;
  const long long nv = B / VW;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < nv;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    PermVec<T, VW> v = vload<T, VW>(sp + e * VW);
    if (beta != T(0)) {
      const PermVec<T, VW> old = vload<T, VW>(dp + e * VW);
#pragma unroll
      for (int w = 0; w < VW; ++w) v.x[w] = alpha * v.x[w] + beta * old.x[w];
    } else {
#pragma unroll
      for (int w = 0; w < VW; ++w) v.x[w] = alpha * v.x[w];
    }
    vstore<T, VW>(dp + e * VW, v);
  }
}

template <class T>
cudaError_t launch_block_copy(T* dst, const T* src, long long B, const BlockCopyDesc& d, double alpha, double beta,
                              cudaStream_t st) {
  long long nout = 1;
  for (int k = 0; k < d.nouter; ++k) nout *= d.dim[k];
  if (nout <= 0 || B <= 0) return cudaSuccess;
  if (nout > 65535 || d.nouter > kMaxL) return cudaErrorInvalidValue;
  constexpr int kVW = 16 / sizeof(T);
  bool vec = B % kVW == 0 && reinterpret_cast<uintptr_t>(dst) % 16 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0;
  for (int k = 0; k < d.nouter && vec; ++k) vec = d.sst[k] % kVW == 0;
  const long long per = vec ? B / kVW : B;
  const int bx = static_cast<int>(std::min<long long>((per + 255) / 256, std::max<long long>(1, 152LL * 16 / nout)));
  dim3 grid(bx, static_cast<unsigned>(nout));
  if (vec)
    block_copy_kernel<T, kVW><<<grid, 256, 0, st>>>(dst, src, B, d, static_cast<T>(alpha), static_cast<T>(beta));
  else
    block_copy_kernel<T, 1><<<grid, 256, 0, st>>>(dst, src, B, d, static_cast<T>(alpha), static_cast<T>(beta));
  return cudaGetLastError();
}
template cudaError_t launch_block_copy<float>(float*, const float*, long long, const BlockCopyDesc&, double, double,
                                              cudaStream_t);
template cudaError_t launch_block_copy<double>(double*, const double*, long long, const BlockCopyDesc&, double, double,
                                               cudaStream_t);

cudaError_t launch_pack_bf16x2(const float* src, void* hi, void* lo, const PackDesc& d, cudaStream_t st) {
  if (d.rows <= 0 || d.creal <= 0) return cudaSuccess;
  return run_permute<float, true>(pack_plan(src, d),
                                  PermOut<float>{nullptr, static_cast<__nv_bfloat16*>(hi),
                                                 static_cast<__nv_bfloat16*>(lo)},
                                  1.0, 0.0, st);
}

template <class T>
cudaError_t launch_scatter(const T* src, T* dst, const ScatDesc& d, double alpha, double beta, cudaStream_t st) {
  if (d.total <= 0) return cudaSuccess;
  if (d.nswap < 0 || d.nswap > 2) return cudaErrorInvalidValue;
  PermPlan P;
  P.nd = d.nd;
  P.nterm = 1 << d.nswap;
  long long s = 1;
  for (int k = d.nd - 1; k >= 0; --k) {
    P.dim[k] = d.dim[k];
    P.dstr[k] = s;
    s *= d.dim[k];
  }
  for (int p = 0; p < P.nterm; ++p) {
    int pm[kMaxL];
    for (int k = 0; k < d.nd; ++k) pm[k] = k;
    for (int w = 0; w < 2; ++w)
      if (p & (1 << w)) std::swap(pm[d.sw[w][0]], pm[d.sw[w][1]]);
    for (int k = 0; k < d.nd; ++k) P.sst[p][k] = d.sst[pm[k]];
    P.src[p] = src;
    P.coef[p] = (p == 1 || p == 2) ? -1.0 : 1.0;
  }
  return run_permute<T, false>(P, PermOut<T>{dst, nullptr, nullptr}, alpha, beta, st);
}
template cudaError_t launch_scatter<float>(const float*, float*, const ScatDesc&, double, double, cudaStream_t);
template cudaError_t launch_scatter<double>(const double*, double*, const ScatDesc&, double, double, cudaStream_t);

template <class T>
cudaError_t launch_antisym4(T* dst, const Anti4Desc& d, cudaStream_t st) {
  if (d.nzx <= 0 || d.no <= 0 || d.nv <= 0) return cudaSuccess;
  if (d.nsrc < 1 || d.nsrc > 2 || d.nx < 1) return cudaErrorInvalidValue;
  // element offsets inside one zx slice (and inside one V block) are 32-bit in the kernel
  if (static_cast<long long>(d.no) * d.no * d.nv * d.nv >= (1LL << 31)) return cudaErrorInvalidValue;
  Anti4Desc dd = d;
  dd.ta = std::min(kAT, d.nv);   // a tile spans the whole a/b range when it is short
  const long long nA = (d.nv + dd.ta - 1) / dd.ta;
  const long long blocks = static_cast<long long>(d.nzx) * (static_cast<long long>(d.no) * (d.no + 1) / 2) *
                           (nA * (nA + 1) / 2);
  if (blocks >= (1LL << 31)) return cudaErrorInvalidValue;
  const size_t smem = static_cast<size_t>(d.nsrc * 4 + 1) * dd.ta * (dd.ta + 1) * sizeof(T);
  const int kp = (dd.ta * dd.ta + 255) / 256;   // element slots per thread, 1..4
  static std::atomic<bool> attr[5] = {{false}, {false}, {false}, {false}, {false}};   // per instantiation (this T)
  auto launch = [&](auto kern) -> cudaError_t {
    if (smem > 48 * 1024 && !attr[kp].load()) {   // the largest tile set of this instantiation
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(9 * kAT * (kAT + 1) * sizeof(T)));
      if (e != cudaSuccess) return e;
      attr[kp].store(true);
    }
    kern<<<static_cast<unsigned>(blocks), 256, smem, st>>>(dst, dd);
    return cudaGetLastError();
  };
  switch (kp) {
    case 1: return launch(antisym4_kernel<T, 1>);
    case 2: return launch(antisym4_kernel<T, 2>);
    case 3: return launch(antisym4_kernel<T, 3>);
    default: return launch(antisym4_kernel<T, 4>);
  }
}
template cudaError_t launch_antisym4<float>(float*, const Anti4Desc&, cudaStream_t);
template cudaError_t launch_antisym4<double>(double*, const Anti4Desc&, cudaStream_t);

template <class T>
cudaError_t launch_tau(const T* t1, const T* t2, T* tt, T* ta, T* X, double ctt, double cta, int nx, int no, int nv,
                       cudaStream_t st) {
  const long long slice = static_cast<long long>(no) * no * nv * nv;
  if (slice >= (1LL << 31) || nx > 65535) return cudaErrorInvalidValue;
  dim3 grid(grid_for(slice, 256, 2048), nx);
  tau_kernel<T><<<grid, 256, 0, st>>>(t1, t2, tt, ta, X, static_cast<T>(ctt), static_cast<T>(cta), make_fastdiv(no),
                                      make_fastdiv(nv));
  return cudaGetLastError();
}
template cudaError_t launch_tau<float>(const float*, const float*, float*, float*, float*, double, double, int, int, int,
                                       cudaStream_t);
template cudaError_t launch_tau<double>(const double*, const double*, double*, double*, double*, double, double, int,
                                        int, int,
                                        cudaStream_t);


template <class Ts, class Td>
cudaError_t launch_convert(const Ts* s, Td* d, long long n, cudaStream_t st) {
  convert_kernel<Ts, Td><<<grid_for(n, 256), 256, 0, st>>>(s, d, n);
  return cudaGetLastError();
}
template cudaError_t launch_convert<float, double>(const float*, double*, long long, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double*, float*, long long, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, long long, cudaStream_t);

cudaError_t launch_hubbard(double* h, double* eri, double* eps, int L, double t, double U, cudaStream_t st) {
  const long long N = 2LL * L;
  hubbard_kernel<<<grid_for(N * N * N * N, 256), 256, 0, st>>>(h, eri, eps, L, t, U);
  // the h / eps part needs N*N threads: make sure the grid covers it
  if (grid_for(N * N * N * N, 256) * 256LL < N * N) return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_ueg(double* h, double* eri, double* eps, const int* nvec, int M, int nocc, double vol, double kunit,
                       cudaStream_t st) {
  const long long N = 2LL * M;
  ueg_kernel<<<grid_for(N * N * N * N, 256), 256, 0, st>>>(h, eri, eps, nvec, M, nocc, vol, kunit);
  if (grid_for(N * N * N * N, 256) * 256LL < N * N) return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_reference(const double* h, const double* eri, const double* eps, int N, double beta, double mu,
                             double* n, double* nbar, double* f, double* fbar, double* scal, cudaStream_t st) {
  fock_kernel<<<(N * N + 255) / 256, 256, 0, st>>>(h, eri, eps, N, beta, mu, f, fbar);
  reference_scalars_kernel<<<1, 256, 0, st>>>(h, eri, eps, N, beta, mu, n, nbar, scal);
  return cudaGetLastError();
}

cudaError_t launch_prop_tables(const double* eps, int N, double h, double* em, double* ep, cudaStream_t st) {
  prop_tables_kernel<<<(N + 127) / 128, 128, 0, st>>>(eps, N, h, em, ep);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_thermal_eri(const double* eri, int N, const int* idx0, const double* fac0, int n0, const int* idx1,
                               const double* fac1, int n1, const int* idx2, const double* fac2, int n2,
                               const int* idx3, const double* fac3, int n3, T* out, cudaStream_t st) {
  const long long n = static_cast<long long>(n0) * n1 * n2 * n3;
  thermal_eri_kernel<T><<<grid_for(n, 256), 256, 0, st>>>(eri, N, idx0, fac0, n0, idx1, fac1, n1, idx2, fac2, n2, idx3,
                                                          fac3, n3, out);
  return cudaGetLastError();
}
cudaError_t launch_eri_adjoint(const double* bar, int N, const int* idx0, const double* fac0, int n0, const int* idx1,
                              const double* fac1, int n1, const int* idx2, const double* fac2, int n2,
                              const int* idx3, const double* fac3, int n3, double* gamma, cudaStream_t st) {
  const long long n = static_cast<long long>(n0) * n1 * n2 * n3;
  eri_adjoint_kernel<<<grid_for(n, 256), 256, 0, st>>>(bar, N, idx0, fac0, n0, idx1, fac1, n1, idx2, fac2, n2, idx3,
                                                       fac3, n3, gamma);
  return cudaGetLastError();
}
template cudaError_t launch_thermal_eri<float>(const double*, int, const int*, const double*, int, const int*,
                                               const double*, int, const int*, const double*, int, const int*,
                                               const double*, int, float*, cudaStream_t);
template cudaError_t launch_thermal_eri<double>(const double*, int, const int*, const double*, int, const int*,
                                                const double*, int, const int*, const double*, int, const int*,
                                                const double*, int, double*, cudaStream_t);

template <class T>
cudaError_t launch_thermal_fock(const double* fbar, int N, const int* idx0, const double* fac0, int n0, const int* idx1,
                                const double* fac1, int n1, T* out, cudaStream_t st) {
  const int n = n0 * n1;
  thermal_fock_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(fbar, N, idx0, fac0, n0, idx1, fac1, n1, out);
  return cudaGetLastError();
}
template cudaError_t launch_thermal_fock<float>(const double*, int, const int*, const double*, int, const int*,
                                                const double*, int, float*, cudaStream_t);
template cudaError_t launch_thermal_fock<double>(const double*, int, const int*, const double*, int, const int*,
                                                 const double*, int, double*, cudaStream_t);

// Blocks of the propagators over all instances: 16 per SM, so that enough
// loads are in flight to cover the memory latency.
int prop_blocks() { return 152 * 16; }

template <class T, class A, class EA>
cudaError_t launch_prop_t(const T* S, T* t, const PropArgs& a, dim3 grid, cudaStream_t st) {
  const size_t smem = static_cast<size_t>(a.ng) * kPropThreads * sizeof(EA);   // per-thread energy slots
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (a.nslot == 4) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(propagate_kernel<T, A, EA, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
    propagate_kernel<T, A, EA, 4><<<grid, kPropThreads, smem, st>>>(S, t, a);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(propagate_kernel<T, A, EA, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem));
    propagate_kernel<T, A, EA, 2><<<grid, kPropThreads, smem, st>>>(S, t, a);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_propagate(const T* S, T* t, const PropArgs& a_in, cudaStream_t st) {
  if (a_in.ng < 3 || a_in.size >= (1LL << 31)) return cudaErrorInvalidValue;
  if (a_in.y0 < 0 || a_in.y1 > a_in.ng || a_in.y1 <= a_in.y0 || a_in.s_ng < a_in.y1 - a_in.y0) return cudaErrorInvalidValue;
  if (a_in.y0 == 0 && a_in.y1 < 3) return cudaErrorInvalidValue;                 // S_2 is needed at y = 1
  if (!a_in.chain && (a_in.y0 != 0 || a_in.y1 != a_in.ng)) return cudaErrorInvalidValue;
  PropArgs a = a_in;
  a.fo = make_fastdiv(static_cast<uint32_t>(a.no));
  a.fv = make_fastdiv(static_cast<uint32_t>(a.nv));
  if (a.nz < 1 || a.nz > 65535) return cudaErrorInvalidValue;
  dim3 grid(a.nblocks, a.nz);
  // FP32 storage: arith64 0 = FP32 recurrence and energy sums, 1 = FP32
  // recurrence with FP64 energy sums, 2 = FP64 recurrence and energy sums
  if (sizeof(T) == 4 && a.arith64 == 0) return launch_prop_t<T, float, float>(S, t, a, grid, st);
  if (sizeof(T) == 4 && a.arith64 == 1) return launch_prop_t<T, float, double>(S, t, a, grid, st);
  return launch_prop_t<T, double, double>(S, t, a, grid, st);
}
template cudaError_t launch_propagate<float>(const float*, float*, const PropArgs&, cudaStream_t);
template cudaError_t launch_propagate<double>(const double*, double*, const PropArgs&, cudaStream_t);

cudaError_t launch_reduce(const double* p1, int nb1, const double* p2, int nb2, int ng, int nz, const double* hz,
                          const int* live, double* state, cudaStream_t st) {
  if (ng > 256 || nz < 1) return cudaErrorInvalidValue;
  if (nz > 65535) return cudaErrorInvalidValue;
  reduce_kernel<<<dim3(ng + 2, nz), kReduceThreads, 0, st>>>(p1, nb1, p2, nb2, ng, nz, hz, live, state);
  return cudaGetLastError();
}

double simpson_weight_host(int y, int ng) {
  const int last = ng - 1;
  if ((last & 1) == 0) {
    if (y == 0 || y == last) return 1.0 / 3.0;
    return (y & 1) ? 4.0 / 3.0 : 2.0 / 3.0;
  }
  if (last == 1) return y == 0 ? 5.0 / 12.0 : (y == 1 ? 8.0 / 12.0 : -1.0 / 12.0);
  const int m = last - 3;
  double w = 0.0;
  if (y <= m && m > 0) {
    if (y == 0 || y == m) w += 1.0 / 3.0;
    else w += (y & 1) ? 4.0 / 3.0 : 2.0 / 3.0;
  }
  if (y >= m) {
    const int k = y - m;
    w += (k == 0 || k == 3) ? 3.0 / 8.0 : 9.0 / 8.0;
  }
  return w;
}

template <class T>
cudaError_t launch_propagate_t(const T* m, T* u, const PropArgs& a_in, cudaStream_t st) {
  if (a_in.ng < 3 || a_in.size >= (1LL << 31) || a_in.nz < 1) return cudaErrorInvalidValue;
  PropArgs a = a_in;
  a.fo = make_fastdiv(static_cast<uint32_t>(a.no));
  a.fv = make_fastdiv(static_cast<uint32_t>(a.nv));
  dim3 grid(a.nblocks, a.nz);
  if (a.nslot == 4) propagate_t_kernel<T, 4><<<grid, kPropThreads, 0, st>>>(m, u, a);
  else propagate_t_kernel<T, 2><<<grid, kPropThreads, 0, st>>>(m, u, a);
  return cudaGetLastError();
}

template <class T, class BT>
cudaError_t launch_lambda_combine(const BT* base, const T* tbar, T* mnew, const T* mold, long long size, int ng, int nz,
                                  const double* cz, double cbase, double* partials, int nblocks, cudaStream_t st,
                                  const int* list, int nlist) {
  if (list && static_cast<long long>(nz) * ng * size >= (1LL << 31)) return cudaErrorInvalidValue;
  lambda_combine_kernel<T, BT><<<nblocks, 256, 0, st>>>(base, tbar, mnew, mold, size, ng, nz, cz, cbase, partials,
                                                        list, nlist);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_slot_sums(const T* I, const T* A, int nslot, const int* dims, int cls, int no, int nv,
                             int nz, double* Do, double* Dv, cudaStream_t st) {
  long long per = 1;
  for (int k = 0; k < nslot; ++k) per *= dims[k];
  dim3 grid(grid_for(per, 256, 1024), nz);
  slot_sums_kernel<T><<<grid, 256, 0, st>>>(I, A, nslot, dims[0], dims[1], nslot > 2 ? dims[2] : 1,
                                          nslot > 3 ? dims[3] : 1, cls, no, nv, Do, Dv);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_fbar_scatter(const T* A, int n0, int n1, const int* i0, const double* f0, long long f0z,
                                const int* i1, const double* f1, long long f1z, int N, int nz, double* Fb,
                                cudaStream_t st) {
  dim3 grid((n0 * n1 + 255) / 256, nz);
  fbar_scatter_kernel<T><<<grid, 256, 0, st>>>(A, n0, n1, i0, f0, f0z, i1, f1, f1z, N, Fb);
  return cudaGetLastError();
}

cudaError_t launch_fock_n(const double* Fb, const double* eri, int N, double* Gn, cudaStream_t st) {
  fock_n_kernel<<<N, 256, 0, st>>>(Fb, eri, N, Gn);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_prop_response(const T* S, const T* m, const double* epsz, const PropArgs& a_in, double* Ee,
                                 double* Eb, cudaStream_t st) {
  PropArgs a = a_in;
  a.fo = make_fastdiv(static_cast<uint32_t>(a.no));
  a.fv = make_fastdiv(static_cast<uint32_t>(a.nv));
  dim3 grid(a.nblocks, a.nz);
  if (a.nslot == 4) prop_response_kernel<T, 4><<<grid, kPropThreads, 0, st>>>(S, m, epsz, a, Ee, Eb);
  else prop_response_kernel<T, 2><<<grid, kPropThreads, 0, st>>>(S, m, epsz, a, Ee, Eb);
  return cudaGetLastError();
}

#define FTCC_ADJOINT_INSTANTIATE(T)                                                                                 \
  template cudaError_t launch_propagate_t<T>(const T*, T*, const PropArgs&, cudaStream_t);                         \
  template cudaError_t launch_slot_sums<T>(const T*, const T*, int, const int*, int, int, int, int, double*, double*, \
                                           cudaStream_t);                                                           \
  template cudaError_t launch_fbar_scatter<T>(const T*, int, int, const int*, const double*, long long, const int*,  \
                                              const double*, long long, int, int, double*, cudaStream_t);          \
  template cudaError_t launch_prop_response<T>(const T*, const T*, const double*, const PropArgs&, double*, double*, \
                                               cudaStream_t);                                                       \
  template cudaError_t launch_lambda_combine<T, T>(const T*, const T*, T*, const T*, long long, int, int,           \
                                                   const double*, double, double*, int, cudaStream_t, const int*, int);
FTCC_ADJOINT_INSTANTIATE(float)
FTCC_ADJOINT_INSTANTIATE(double)
#undef FTCC_ADJOINT_INSTANTIATE
template cudaError_t launch_lambda_combine<float, double>(const double*, const float*, float*, const float*, long long,
                                                          int, int, const double*, double, double*, int, cudaStream_t,
                                                          const int*, int);

}  // namespace ftcc
