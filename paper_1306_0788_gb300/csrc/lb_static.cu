// lb_static.cu -- the FP64 fluid-moment reduction for callers that must not allocate device
// memory.  Same sums as lbmd_diagnostics (total mass of each component and the fluid
// momentum), taken over a population array the caller already holds on the device; the
// per-block partial sums go to a fixed static device array instead of a cudaMalloc'd buffer.
#include <mutex>
#include <string>

#include "lbmd_internal.cuh"

namespace lbmd {
namespace {

constexpr int kStaticThreads = 256;
constexpr int kSitesPerThread = 32;
constexpr long long kSitesPerBlock = (long long)kStaticThreads * kSitesPerThread;  // 8192
constexpr int kMaxStaticBlocks = 16384;  // lattices up to 16384 * 8192 = 2^27 sites (512^3)
constexpr int kMoments = 5;              // M_A, M_B, Px, Py, Pz

// Shared by every call in the process on a given device, kept until exit (640 KiB).
static __device__ __align__(256) double g_moment_partials[kMaxStaticBlocks * kMoments];

__global__ void __launch_bounds__(kStaticThreads) k_moment_blocks(const float *__restrict__ f, long long N,
                                                                  double *__restrict__ partial) {
  double acc[kMoments] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const long long b0 = (long long)blockIdx.x * kSitesPerBlock;
  for (int k = 0; k < kSitesPerThread; ++k) {
    const long long s = b0 + (long long)k * kStaticThreads + threadIdx.x;  // coalesced across the block
    if (s >= N) break;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const double a = (double)f[(long long)i * N + s];
      const double b = (double)f[(long long)(kQ + i) * N + s];
      acc[0] += a;
      acc[1] += b;
      if (kCx[i]) acc[2] += kCx[i] * (a + b);
      if (kCy[i]) acc[3] += kCy[i] * (a + b);
      if (kCz[i]) acc[4] += kCz[i] * (a + b);
    }
  }
  __shared__ double sh[kMoments][kStaticThreads];
#pragma unroll
  for (int m = 0; m < kMoments; ++m) sh[m][threadIdx.x] = acc[m];
  __syncthreads();
  for (int w = kStaticThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int m = 0; m < kMoments; ++m) sh[m][threadIdx.x] += sh[m][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int m = 0; m < kMoments; ++m) partial[(long long)blockIdx.x * kMoments + m] = sh[m][0];
}

__global__ void k_moment_finish(const double *__restrict__ partial, int nblocks, double *__restrict__ out) {
  const int m = threadIdx.x;  // one thread per moment, blocks summed in order: deterministic
  if (m >= kMoments) return;
  double a = 0.0;
  for (int b = 0; b < nblocks; ++b) a += partial[(long long)b * kMoments + m];
  out[m] = a;
}

std::mutex g_symbol_mutex;
double *g_symbol_ptr[64] = {nullptr};  // device address of g_moment_partials per device ordinal

int static_fail(int code, const std::string &m) {
  set_context_free_error(m);  // readable with lbmd_last_error(NULL)
  return code;
}

}  // namespace
}  // namespace lbmd

using namespace lbmd;

extern "C" {

int lbmd_fluid_moments_static(const float *f_dev, int nx, int ny, int nz, double *out_dev, void *stream) {
  if (!f_dev || !out_dev || nx < 1 || ny < 1 || nz < 1)
    return static_fail(LBMD_E_INVALID_ARG, "lbmd_fluid_moments_static: null pointer or lattice size < 1");
  const long long N = (long long)nx * ny * nz;
  const long long nblocks = (N + kSitesPerBlock - 1) / kSitesPerBlock;
  if (nblocks > kMaxStaticBlocks)
    return static_fail(LBMD_E_INVALID_ARG,
                       "lbmd_fluid_moments_static: lattice of " + std::to_string(N) + " sites exceeds the maximum of " +
                           std::to_string((long long)kMaxStaticBlocks * kSitesPerBlock) +
                           " sites held by the static scratch array");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(LBMD_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return static_fail(LBMD_E_INVALID_ARG, "lbmd_fluid_moments_static: device ordinal >= 64");
  double *partial = nullptr;
  {
    // first call on this device: look up the device address of the static scratch array
    // (host code cannot use the array's name as a device address)
    std::lock_guard<std::mutex> lock(g_symbol_mutex);
    if (!g_symbol_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_moment_partials);
      if (e != cudaSuccess || !p)
        return static_fail(LBMD_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_symbol_ptr[dev] = static_cast<double *>(p);
    }
    partial = g_symbol_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_moment_blocks<<<(unsigned)nblocks, kStaticThreads, 0, st>>>(f_dev, N, partial);
  k_moment_finish<<<1, 32, 0, st>>>(partial, (int)nblocks, out_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(LBMD_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return LBMD_OK;
}

}  // extern "C"
