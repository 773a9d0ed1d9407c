// lb_static.cu -- the FP64 fluid-moment reduction for callers that must not allocate device
// memory.  Same sums as lbmd_diagnostics (total mass of each component and the fluid
// momentum), taken over a population array the caller already holds on the device; the
// per-block partial sums go to a fixed static device array instead of a cudaMalloc'd buffer.
#include <cuda.h>  // driver types of the entry points below (looked up at run time, not linked)

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

constexpr int kFinishThreads = 256;

// The block partials summed by one block: thread t adds partials t, t + 256, ... in order, then a
// fixed shared-memory tree combines the threads -- the same order on every call (deterministic).
__global__ void __launch_bounds__(kFinishThreads) k_moment_finish(const double *__restrict__ partial, int nblocks,
                                                                  double *__restrict__ out) {
  double acc[kMoments] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += kFinishThreads)
#pragma unroll
    for (int m = 0; m < kMoments; ++m) acc[m] += partial[(long long)b * kMoments + m];
  __shared__ double sh[kMoments][kFinishThreads];
#pragma unroll
  for (int m = 0; m < kMoments; ++m) sh[m][threadIdx.x] = acc[m];
  __syncthreads();
  for (int w = kFinishThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int m = 0; m < kMoments; ++m) sh[m][threadIdx.x] += sh[m][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < kMoments) out[threadIdx.x] = sh[threadIdx.x][0];
}

// Driver calls looked up through the runtime (the library links no libcuda): the identity of
// the current context, and the extent of the allocation holding a device pointer.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
using MemGetAddressRangeFn = CUresult (*)(CUdeviceptr *, size_t *, CUdeviceptr);

struct DriverCalls {
  CtxGetCurrentFn ctx_current = nullptr;
  CtxGetIdFn ctx_id = nullptr;
  MemGetAddressRangeFn range = nullptr;
};

const DriverCalls &driver_calls() {
  static DriverCalls d = [] {
    DriverCalls r;
    cudaDriverEntryPointQueryResult q;
    void *f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      r.ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      r.ctx_id = reinterpret_cast<CtxGetIdFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      r.range = reinterpret_cast<MemGetAddressRangeFn>(f);
    cudaGetLastError();
    return r;
  }();
  return d;
}

// Unique id of the calling thread's current context (0: none, or the driver cannot tell).
unsigned long long current_context_id() {
  const DriverCalls &d = driver_calls();
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!d.ctx_current || !d.ctx_id || d.ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (d.ctx_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// True if [p, p + bytes) is device (or managed) memory inside one allocation of the current
// context.  Where the driver cannot give the allocation's extent, only the memory type is checked.
bool device_range_ok(const void *p, size_t bytes) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return false;
  const DriverCalls &d = driver_calls();
  if (!d.range) return true;
  CUdeviceptr base = 0;
  size_t size = 0;
  if (d.range(&base, &size, (CUdeviceptr)p) != CUDA_SUCCESS) return false;
  const CUdeviceptr q = (CUdeviceptr)p;
  return q >= base && bytes <= size && q - base <= size - bytes;
}

std::mutex g_symbol_mutex;
// device address of g_moment_partials per device ordinal, with the id of the context it was
// looked up in: a context created again on that device (after cudaDeviceReset) looks it up anew
double *g_symbol_ptr[64] = {nullptr};
unsigned long long g_symbol_ctx[64] = {0};

int static_fail(int code, const std::string &m) {
  set_context_free_error(m);  // readable with lbmd_last_error(NULL)
  return code;
}

}  // namespace

bool device_buffer_ok(const void *p, size_t bytes) { return device_range_ok(p, bytes); }

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
    // set-up, once per device and context: the device address of the static scratch array
    // (host code cannot use the array's name as a device address)
    std::lock_guard<std::mutex> lock(g_symbol_mutex);
    const unsigned long long id = current_context_id();
    if (!g_symbol_ptr[dev] || id == 0 || id != g_symbol_ctx[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_moment_partials);
      if (e != cudaSuccess || !p)
        return static_fail(LBMD_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_symbol_ptr[dev] = static_cast<double *>(p);
      g_symbol_ctx[dev] = current_context_id();  // the lookup made the device's context current
    }
    partial = g_symbol_ptr[dev];
  }
  // the buffers must be device memory of the stated length: checked before any launch, so that
  // a host pointer or a short buffer is an error code and not a fault on the device
  if (!device_range_ok(f_dev, sizeof(float) * 2 * kQ * (size_t)N))
    return static_fail(LBMD_E_INVALID_ARG,
                       "lbmd_fluid_moments_static: f_dev is not device memory holding 2 x 19 x nx x ny x nz floats");
  if (!device_range_ok(out_dev, sizeof(double) * kMoments))
    return static_fail(LBMD_E_INVALID_ARG, "lbmd_fluid_moments_static: out_dev is not device memory of 5 doubles");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_moment_blocks<<<(unsigned)nblocks, kStaticThreads, 0, st>>>(f_dev, N, partial);
  k_moment_finish<<<1, kFinishThreads, 0, st>>>(partial, (int)nblocks, out_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(LBMD_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return LBMD_OK;
}

}  // extern "C"
