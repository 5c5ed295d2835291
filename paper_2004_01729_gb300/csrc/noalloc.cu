// Allocation-free entry point: the FP64 split-K GEMM of the engine with its
// partial sums in a fixed device array instead of caller- or library-
// allocated scratch.
//
// Why it exists: some callers cannot allocate device memory at the moment
// they need a contraction -- code running inside a device-memory allocator's
// own callback (allocating there re-enters the allocator), or programs that
// fix their device-memory footprint at start-up and may not grow it later.  They call ftcc_gemm_f64_static with their inputs
// and outputs; everything else lives in kScratchBytes of static device
// memory that every GPU which loads the library holds until the process exits.
#include <cuda_runtime.h>

#include "ftcc_internal.h"

namespace {

// 16 MiB of split-K partials (2^21 doubles), shared by every call.
constexpr size_t kScratchBytes = size_t(16) << 20;
static __device__ __align__(256) double g_splitk_scratch[kScratchBytes / sizeof(double)];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device pointer).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_splitk_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" ftcc_status ftcc_gemm_f64_static(void* stream, int batch, int M, int N, int K, double alpha, const double* A,
                                            long long lda, long long sa, const double* B, long long ldb, long long sb,
                                            double* C, long long ldc, long long sc) {
  if (!A || !B || !C || batch < 1 || M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < N || sa < 0 || sb < 0 ||
      sc < 0)
    return FTCC_ERR_INVALID_ARG;
  // the output of one call must fit the scratch at least twice over (two K
  // splits); the limit is applied to every call, split or not
  const long long outer = static_cast<long long>(batch) * M * N;
  if (outer > static_cast<long long>(kScratchBytes / sizeof(double)) / 2) return FTCC_ERR_INVALID_ARG;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return FTCC_ERR_NO_DEVICE;
  void* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return FTCC_ERR_CUDA;
  ftcc::GemmArgs g{};
  g.batch = batch;
  g.M = M;
  g.N = N;
  g.K = K;
  g.A = A;
  g.lda = lda;
  g.sa = sa;
  g.B = B;
  g.ldb = ldb;
  g.sb = sb;
  g.C = C;
  g.ldc = ldc;
  g.sc = sc;
  g.alpha = alpha;
  g.beta = 0.0;
  // every partial the reduction reads is written earlier in the same call, so
  // nothing in the scratch has to start at zero
  g.work = scratch;
  g.work_bytes = kScratchBytes;
  if (ftcc::gemm_f64(g, static_cast<cudaStream_t>(stream)) != cudaSuccess) return FTCC_ERR_CUDA;
  return FTCC_OK;
}
