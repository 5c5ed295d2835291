// SIMT GEMM for the FP64 path (GB300 has no FP64 tensor-core MMA in tcgen05)
// and for FP32 contractions too thin for a 128 x 128 tensor-core tile.
//   C[b][m][n] = alpha * sum_k A[b][m][k] * B[b][n][k] + beta * C[b][m][n]
// (with trans, C[b][n][m]: the output stored transposed)
// 64 x 64 output tile per 256-thread block, 4 x 4 outputs per thread, K
// staged 16 at a time through shared memory (stored k-major so that the
// inner loop reads broadcast rows).
#include <algorithm>

#include "ftcc_internal.h"

namespace ftcc {
namespace {

constexpr int kT = 64;
constexpr int kK = 16;

// fused multiply-add in the type of its arguments (fmaf for float)
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// blockIdx.z = batch * splits + split; with splits > 1 each block sums one
// K range and writes alpha * partial to W[split][batch][M][N] (reduced later).
template <class T>
__global__ void __launch_bounds__(256) gemm_simt_kernel(const T* __restrict__ A, long long lda, long long sa,
                                                        const T* __restrict__ B, long long ldb, long long sb,
                                                        T* __restrict__ C, long long ldc, long long sc, int M,
                                                        int N, int K, T alpha, T beta, int splits, int kchunk,
                                                        T* __restrict__ W, int batch, int trans) {
  __shared__ T As[kK][kT + 1];
  __shared__ T Bs[kK][kT + 1];
  const int bz = blockIdx.z / splits;
  const int sp = blockIdx.z - bz * splits;
  const int kbeg = sp * kchunk;
  const int kend = min(K, kbeg + kchunk);
  A += static_cast<long long>(bz) * sa;
  B += static_cast<long long>(bz) * sb;
  long long csm = ldc, csn = 1;   // element strides of C along m and n
  if (splits > 1) {
    C = W + (static_cast<long long>(sp) * batch + bz) * M * static_cast<long long>(N);
    csm = N;
    beta = T(0);
  } else {
    C += static_cast<long long>(bz) * sc;
    if (trans) {
      csm = 1;
      csn = ldc;
    }
  }
  const int m0 = blockIdx.y * kT;
  const int n0 = blockIdx.x * kT;
  const int tx = threadIdx.x & 15;   // n direction
  const int ty = threadIdx.x >> 4;   // m direction
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = kbeg; k0 < kend; k0 += kK) {
    // 64 rows x 16 k per operand = 1024 elements, 4 per thread, k fastest.
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = threadIdx.x + 256 * r;
      const int row = e >> 4;
      const int kk = e & 15;
      const int gm = m0 + row, gn = n0 + row, gk = k0 + kk;
      As[kk][row] = (gm < M && gk < kend) ? A[static_cast<long long>(gm) * lda + gk] : T(0);
      Bs[kk][row] = (gn < N && gk < kend) ? B[static_cast<long long>(gn) * ldb + gk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma_t(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      T* c = C + static_cast<long long>(gm) * csm + static_cast<long long>(gn) * csn;
      const T v = alpha * acc[i][j];
      *c = (beta == T(0)) ? v : v + beta * *c;
    }
  }
}

template <class T>
__global__ void splitk_reduce_kernel(const T* __restrict__ W, T* __restrict__ C, long long ldc, long long sc, int M,
                                     int N, int batch, int splits, T beta, int trans) {
  const long long mn = static_cast<long long>(M) * N;
  const long long total = mn * batch;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long b = e / mn;
    const long long r = e - b * mn;
    const long long m = r / N, n = r - m * N;
    T acc = T(0);
    for (int s = 0; s < splits; ++s) acc += W[static_cast<long long>(s) * total + e];
    T* c = C + b * sc + (trans ? n * ldc + m : m * ldc + n);
    *c = (beta == T(0)) ? acc : acc + beta * *c;
  }
}

template <class T>
cudaError_t launch(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  const int mt = (g.M + kT - 1) / kT, nt = (g.N + kT - 1) / kT;
  // split K when the output alone gives fewer than ~2 blocks per SM
  int splits = 1;
  const long long tiles = static_cast<long long>(mt) * nt * g.batch;
  const long long outer = static_cast<long long>(g.M) * g.N * g.batch;
  if (g.work && tiles < 304 && g.K >= 4 * kK) {
    splits = static_cast<int>(std::min<long long>((304 + tiles - 1) / tiles, g.K / (2 * kK)));
    splits = std::min(splits, 64);
    while (splits > 1 && static_cast<size_t>(splits) * outer * sizeof(T) > g.work_bytes) --splits;
  }
  int kchunk = (g.K + splits - 1) / splits;
  kchunk = (kchunk + kK - 1) / kK * kK;
  splits = (g.K + kchunk - 1) / kchunk;
  dim3 grid(nt, mt, static_cast<unsigned>(g.batch) * splits);
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidValue;
  gemm_simt_kernel<T><<<grid, 256, 0, st>>>(static_cast<const T*>(g.A), g.lda, g.sa, static_cast<const T*>(g.B),
                                            g.ldb, g.sb, static_cast<T*>(g.C), g.ldc, g.sc, g.M, g.N, g.K,
                                            static_cast<T>(g.alpha), static_cast<T>(g.beta), splits, kchunk,
                                            static_cast<T*>(g.work), g.batch, g.trans);
  if (splits > 1) {
    const long long total = outer;
    int blocks = static_cast<int>(std::min<long long>((total + 255) / 256, 152 * 8));
    splitk_reduce_kernel<T><<<blocks, 256, 0, st>>>(static_cast<const T*>(g.work), static_cast<T*>(g.C), g.ldc, g.sc,
                                                    g.M, g.N, g.batch, splits, static_cast<T>(g.beta), g.trans);
  }
  return cudaGetLastError();
}

// Skinny products (N <= 32 and K <= 32: the t1- and F-sized operands of the
// S kernel).  One thread per row of C: it keeps its row of A in registers,
// B sits in shared memory, and it writes N outputs.  A warp reads 32
// consecutive rows and writes 32 consecutive rows (or, stored transposed,
// 32 consecutive entries of each of N columns), so both streams coalesce
// and the kernel runs at memory speed where a 128-row tensor-core tile
// would be mostly idle.
constexpr int kSkinny = 32;

template <class T>
__global__ void __launch_bounds__(256) gemm_skinny_kernel(const T* __restrict__ A, long long lda, long long sa,
                                                          const T* __restrict__ B, long long ldb, long long sb,
                                                          T* __restrict__ C, long long ldc, long long sc, int M,
                                                          int N, int K, T alpha, T beta, int trans) {
  __shared__ T Bs[kSkinny][kSkinny + 1];
  const int bz = blockIdx.y;
  A += static_cast<long long>(bz) * sa;
  B += static_cast<long long>(bz) * sb;
  C += static_cast<long long>(bz) * sc;
  for (int e = threadIdx.x; e < kSkinny * kSkinny; e += blockDim.x) {   // zero beyond N x K
    const int n = e / kSkinny, k = e - n * kSkinny;
    Bs[n][k] = (n < N && k < K) ? B[static_cast<long long>(n) * ldb + k] : T(0);
  }
  __syncthreads();
  const long long m = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= M) return;
  T a[kSkinny];
#pragma unroll
  for (int k = 0; k < kSkinny; ++k) a[k] = k < K ? A[m * lda + k] : T(0);
  const long long csm = trans ? 1 : ldc, csn = trans ? ldc : 1;
  for (int n = 0; n < N; ++n) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < kSkinny; ++k) acc = fma_t(a[k], Bs[n][k], acc);
    T* c = C + m * csm + n * csn;
    const T v = alpha * acc;
    *c = (beta == T(0)) ? v : v + beta * *c;
  }
}

template <class T>
cudaError_t launch_skinny(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.N > kSkinny || g.K > kSkinny || g.batch > 65535) return cudaErrorInvalidValue;
  dim3 grid(static_cast<unsigned>((g.M + 255) / 256), static_cast<unsigned>(g.batch));
  gemm_skinny_kernel<T><<<grid, 256, 0, st>>>(static_cast<const T*>(g.A), g.lda, g.sa, static_cast<const T*>(g.B),
                                              g.ldb, g.sb, static_cast<T*>(g.C), g.ldc, g.sc, g.M, g.N, g.K,
                                              static_cast<T>(g.alpha), static_cast<T>(g.beta), g.trans);
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_f64(const GemmArgs& g, cudaStream_t st) { return launch<double>(g, st); }
cudaError_t gemm_f32(const GemmArgs& g, cudaStream_t st) { return launch<float>(g, st); }
bool gemm_skinny_fits(const GemmArgs& g) { return g.N <= kSkinny && g.K <= kSkinny && g.batch <= 65535; }
cudaError_t gemm_skinny_f64(const GemmArgs& g, cudaStream_t st) { return launch_skinny<double>(g, st); }
cudaError_t gemm_skinny_f32(const GemmArgs& g, cudaStream_t st) { return launch_skinny<float>(g, st); }

}  // namespace ftcc
