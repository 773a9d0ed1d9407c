// lb_fluid.cu -- lattice kernels of the coupled Shan-Chen LB / MD step (sm_103a).
//
// Storage: populations of both components in one buffer [19][nz][ny][nx][2] (structure of
// arrays over directions and sites, x fastest, the (A, B) pair of a direction at a node side by
// side, loaded and stored as one word).  The buffer holds the post-collision values f*(r, t-1)
// at their source node; a kernel "pulls" f_i(r, t) = f*_i(r - c_i, t-1), so reads are
// coalesced along x (shifted by at most one node) and writes are fully coalesced.  Element
// type: FP32, or a 16-bit type (FP16, BF16) holding the shifted value f_i - w_i rho0_z with the
// rest populations apart in FP32; all arithmetic is FP32.
#include <type_traits>

#include "lb_site.cuh"

namespace lbmd {

namespace {

constexpr int kBlock = 256;

using namespace site;

template <class T>
__global__ void __launch_bounds__(kBlock) k_init_equilibrium(StepParams P, const float *__restrict__ rhoA,
                                                             const float *__restrict__ rhoB,
                                                             const float *__restrict__ u, T *__restrict__ store,
                                                             float *__restrict__ rest) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const Coord c = site_coord(P, s);
  const float ux = u ? u[3 * s] : 0.f, uy = u ? u[3 * s + 1] : 0.f, uz = u ? u[3 * s + 2] : 0.f;
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  const float rc[2] = {rhoA[s], rhoB[s]};
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    // the post-streaming value at r is pulled from r - c_i: store it there
    const long long dst = site_index(P, wrapi(c.x - kCx[i], P.nx), wrapi(c.y - kCy[i], P.ny), wrapi(c.z - kCz[i], P.nz));
    const float cu = kCx[i] * ux + kCy[i] * uy + kCz[i] * uz;
    const float poly = 1.f + 3.f * cu + 4.5f * cu * cu - usq15;
#pragma unroll
    for (int z = 0; z < 2; ++z) pop_write(P, store, rest, z, i, dst, kW[i] * rc[z] * poly);
  }
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_restream(StepParams P, const float *__restrict__ post, int comp,
                                                     T *__restrict__ store, float *__restrict__ rest) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const Coord c = site_coord(P, s);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const long long dst = site_index(P, wrapi(c.x - kCx[i], P.nx), wrapi(c.y - kCy[i], P.ny), wrapi(c.z - kCz[i], P.nz));
    pop_write(P, store, rest, comp, i, dst, post[(long long)i * P.N + s]);
  }
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_unstream(StepParams P, const T *__restrict__ store,
                                                     const float *__restrict__ rest, int comp,
                                                     float *__restrict__ post) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const Coord c = site_coord(P, s);
  int xs[3], ys[3], zs[3];
  neighbours(P, c, xs, ys, zs);
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    post[(long long)i * P.N + s] = pop_read(P, store, rest, comp, i, pull_source(P, i, xs, ys, zs));
}

// Densities and j' of every site (site::moments).
template <class T>
__global__ void __launch_bounds__(kBlock) k_moments(StepParams P, const T *__restrict__ fin,
                                                    const float *__restrict__ rest, float *__restrict__ rho,
                                                    float *__restrict__ jp) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  moments(P, s, fin, rest, rho, jp);
}

// The lattice update of one step at every site (site::collide; with kMRT the fluctuating MRT
// collision, whose mode transforms spill a few registers at this budget of three blocks per SM
// but run faster than without spills at two; with kBisect the gather over the sub-stepping
// reaction records).
template <class T, bool kParticles, bool kMRT, bool kBisect = false>
__global__ void __launch_bounds__(kBlock, 3) k_collide(StepParams P, const T *__restrict__ fin,
                                                                  T *__restrict__ fout, const float *__restrict__ rho,
                                                                  ParticleArrays pa, ParticleForces pf, CellIndex ci,
                                                                  unsigned *err, const float *__restrict__ rest_in,
                                                                  float *__restrict__ rest_out) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  collide<T, kParticles, kMRT, kBisect>(P, s, P.step, fin, fout, rho, pa, pf, ci, err, rest_in, rest_out);
}

// rho_A, rho_B and u = (j' + g^SC/2)/rho at the current step (for readback).
template <class T>
__global__ void __launch_bounds__(kBlock) k_fields(StepParams P, const T *__restrict__ store,
                                                   const float *__restrict__ rest,
                                                   const float *__restrict__ rho, float *__restrict__ oA,
                                                   float *__restrict__ oB, float *__restrict__ ou) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const Coord c = site_coord(P, s);
  int xs[3], ys[3], zs[3];
  neighbours(P, c, xs, ys, zs);
  float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const long long src = pull_source(P, i, xs, ys, zs);
    const float a = pop_read(P, store, rest, 0, i, src) + pop_read(P, store, rest, 1, i, src);
    jx += kCx[i] * a; jy += kCy[i] * a; jz += kCz[i] * a;
  }
  const float2 *rho2 = reinterpret_cast<const float2 *>(rho);
  const float rA = rho2[s].x, rB = rho2[s].y;
  float SAx = 0.f, SAy = 0.f, SAz = 0.f, SBx = 0.f, SBy = 0.f, SBz = 0.f;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const long long nb = ((long long)zs[1 + kCz[i]] * P.ny + ys[1 + kCy[i]]) * P.nx + xs[1 + kCx[i]];
    const float a = kW[i] * rho2[nb].x, b = kW[i] * rho2[nb].y;
    SAx += kCx[i] * a; SAy += kCy[i] * a; SAz += kCz[i] * a;
    SBx += kCx[i] * b; SBy += kCy[i] * b; SBz += kCz[i] * b;
  }
  const float gx = -P.gAB * rA * SBx - P.gBA * rB * SAx;
  const float gy = -P.gAB * rA * SBy - P.gBA * rB * SAy;
  const float gz = -P.gAB * rA * SBz - P.gBA * rB * SAz;
  const float rinv = 1.f / (rA + rB);
  if (oA) oA[s] = rA;
  if (oB) oB[s] = rB;
  if (ou) {
    ou[3 * s] = (jx + 0.5f * gx) * rinv;
    ou[3 * s + 1] = (jy + 0.5f * gy) * rinv;
    ou[3 * s + 2] = (jz + 0.5f * gz) * rinv;
  }
}

// FP64 block partial sums of [M_A, M_B, Px, Py, Pz] over the stored buffer (streaming
// permutes populations, so sums over stored and post-streaming values agree).
constexpr int kSumBlock = 256;
template <class T>
__global__ void __launch_bounds__(kSumBlock) k_fluid_sums(StepParams P, const T *__restrict__ store,
                                                          const float *__restrict__ rest,
                                                          double *__restrict__ partial) {
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < P.N;
       s += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const double a = (double)pop_read(P, store, rest, 0, i, s);
      const double b = (double)pop_read(P, store, rest, 1, i, s);
      acc[0] += a;
      acc[1] += b;
      if (kCx[i]) acc[2] += kCx[i] * (a + b);
      if (kCy[i]) acc[3] += kCy[i] * (a + b);
      if (kCz[i]) acc[4] += kCz[i] * (a + b);
    }
  }
  __shared__ double sh[5][kSumBlock];
#pragma unroll
  for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kSumBlock / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 5; ++k) partial[(long long)blockIdx.x * 5 + k] = sh[k][0];
}

__global__ void k_finish_sums(const double *__restrict__ partial, int nblocks, int nvals, double *__restrict__ out) {
  // one thread per value, sequential over blocks: deterministic order
  const int k = threadIdx.x;
  if (k >= nvals) return;
  double a = 0.0;
  for (int b = 0; b < nblocks; ++b) a += partial[(long long)b * nvals + k];
  out[k] = a;
}

// The drift check of the conserved totals (appendix: the collision and the forcing term keep
// each component's mass; Sec. 2: the momentum of fluid and particles together).
__global__ void k_drift_check(const double *__restrict__ sums, const double *__restrict__ psum, double *ref,
                              double *last, unsigned *err, long long step, double tol, int set_ref) {
  double t[5];
  for (int k = 0; k < 5; ++k) t[k] = sums[k] + (k >= 2 && psum ? psum[k - 2] : 0.0);
  if (set_ref) {
    for (int k = 0; k < 5; ++k) ref[k] = t[k];
    last[0] = -1.0;
    last[1] = last[2] = last[3] = 0.0;
    last[4] = 0.0;
    return;
  }
  const double dA = fabs(t[0] - ref[0]) / fabs(ref[0]), dB = fabs(t[1] - ref[1]) / fabs(ref[1]);
  const double px = t[2] - ref[2], py = t[3] - ref[3], pz = t[4] - ref[4];
  const double dP = sqrt(px * px + py * py + pz * pz) / (fabs(ref[0]) + fabs(ref[1]));
  last[0] = (double)step;
  last[1] = dA;
  last[2] = dB;
  last[3] = dP;
  last[4] += 1.0;
  // NaN drifts fail the comparison below as well
  if (!(dA <= tol) || !(dB <= tol) || !(dP <= tol)) atomicOr(err, kErrDrift);
}

inline unsigned grid_for(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

}  // namespace

// Run `f` with a typed null pointer of the storage element type of P.
template <class F>
void with_storage(const StepParams &P, F f) {
  switch (P.storage) {
    case LBMD_STORAGE_FP16_SHIFTED: f((__half *)nullptr); break;
    case LBMD_STORAGE_BF16_SHIFTED: f((__nv_bfloat16 *)nullptr); break;
    default: f((float *)nullptr); break;
  }
}

void launch_init_equilibrium(const StepParams &P, const float *rhoA, const float *rhoB, const float *u,
                             void *store, float *rest, cudaStream_t st) {
  with_storage(P, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    k_init_equilibrium<T><<<grid_for(P.N), kBlock, 0, st>>>(P, rhoA, rhoB, u, static_cast<T *>(store), rest);
  });
}
void launch_restream(const StepParams &P, const float *post, int comp, void *store, float *rest, cudaStream_t st) {
  with_storage(P, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    k_restream<T><<<grid_for(P.N), kBlock, 0, st>>>(P, post, comp, static_cast<T *>(store), rest);
  });
}
void launch_unstream(const StepParams &P, const void *store, const float *rest, int comp, float *post,
                     cudaStream_t st) {
  with_storage(P, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    k_unstream<T><<<grid_for(P.N), kBlock, 0, st>>>(P, static_cast<const T *>(store), rest, comp, post);
  });
}
void launch_moments(const StepParams &P, const void *store, const float *rest, float *rho, float *jp,
                    cudaStream_t st) {
  with_storage(P, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    k_moments<T><<<grid_for(P.N), kBlock, 0, st>>>(P, static_cast<const T *>(store), rest, rho, jp);
  });
}
void launch_collide(const StepParams &P, const void *fin, void *fout, float *rest, const float *rho,
                    const ParticleArrays &pa, const ParticleForces &pf, CellIndex ci, unsigned *err,
                    cudaStream_t st) {
  with_storage(P, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    const T *a = static_cast<const T *>(fin);
    T *b = static_cast<T *>(fout);
    const bool mrt = P.collision == LBMD_COLLISION_MRT;
    const bool records = P.np > 0 && P.substeps > 1;
    if (records && mrt)
      k_collide<T, true, true, true><<<grid_for(P.N), kBlock, 0, st>>>(P, a, b, rho, pa, pf, ci, err, rest, rest);
    else if (records)
      k_collide<T, true, false, true><<<grid_for(P.N), kBlock, 0, st>>>(P, a, b, rho, pa, pf, ci, err, rest, rest);
    else if (P.np > 0 && mrt)
      k_collide<T, true, true><<<grid_for(P.N), kBlock, 0, st>>>(P, a, b, rho, pa, pf, ci, err, rest, rest);
    else if (P.np > 0)
      k_collide<T, true, false><<<grid_for(P.N), kBlock, 0, st>>>(P, a, b, rho, pa, pf, ci, err, rest, rest);
    else if (mrt)
      k_collide<T, false, true><<<grid_for(P.N), kBlock, 0, st>>>(P, a, b, rho, pa, pf, ci, err, rest, rest);
    else
      k_collide<T, false, false><<<grid_for(P.N), kBlock, 0, st>>>(P, a, b, rho, pa, pf, ci, err, rest, rest);
  });
}

template <class T>
bool is_noisy_update_of(const void *fn) {
  return fn == reinterpret_cast<const void *>(&k_collide<T, true, true, true>) ||
         fn == reinterpret_cast<const void *>(&k_collide<T, true, true>) ||
         fn == reinterpret_cast<const void *>(&k_collide<T, false, true>);
}

bool is_noisy_update(const void *fn) {
  return is_noisy_update_of<float>(fn) || is_noisy_update_of<__half>(fn) || is_noisy_update_of<__nv_bfloat16>(fn);
}

template <class... A>
constexpr int arity(void (*)(A...)) {
  return (int)sizeof...(A);
}

cudaError_t set_update_step(cudaGraphExec_t exec, cudaGraphNode_t node, unsigned long long step) {
  constexpr int kArgs = arity(&k_collide<float, false, true>);
  cudaKernelNodeParams kp;
  cudaError_t e = cudaGraphKernelNodeGetParams(node, &kp);
  if (e != cudaSuccess) return e;
  if (!is_noisy_update(kp.func) || !kp.kernelParams) return cudaErrorInvalidValue;
  StepParams P;
  std::memcpy(&P, kp.kernelParams[0], sizeof(P));  // the node's own copy of the parameters
  P.step = step;
  void *args[kArgs];
  for (int k = 0; k < kArgs; ++k) args[k] = kp.kernelParams[k];
  args[0] = &P;
  kp.kernelParams = args;
  kp.extra = nullptr;
  return cudaGraphExecKernelNodeSetParams(exec, node, &kp);  // copies the values
}

void launch_fields(const StepParams &P, const void *store, const float *rest, const float *rho, float *rhoA,
                   float *rhoB, float *u, cudaStream_t st) {
  with_storage(P, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    k_fields<T><<<grid_for(P.N), kBlock, 0, st>>>(P, static_cast<const T *>(store), rest, rho, rhoA, rhoB, u);
  });
}
int fluid_sum_blocks(const StepParams &P) {
  long long b = (P.N + kSumBlock - 1) / kSumBlock;
  return (int)(b < 1024 ? b : 1024);
}
void launch_fluid_sums(const StepParams &P, const void *store, const float *rest, double *partial, int nblocks,
                       cudaStream_t st) {
  with_storage(P, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    k_fluid_sums<T><<<nblocks, kSumBlock, 0, st>>>(P, static_cast<const T *>(store), rest, partial);
  });
}
void launch_finish_sums(const double *partial, int nblocks, int nvals, double *out, cudaStream_t st) {
  k_finish_sums<<<1, 32, 0, st>>>(partial, nblocks, nvals, out);
}
void launch_drift_check(const double *sums, const double *psum, double *ref, double *last, unsigned *err,
                        long long step, double tol, int set_ref, cudaStream_t st) {
  k_drift_check<<<1, 1, 0, st>>>(sums, psum, ref, last, err, step, tol, set_ref);
}

// The step base of replayed step graphs (one thread: a write, or an increment at the end of a
// replay, ordered after every launch of the replay that reads it).
__global__ void k_set_step(unsigned long long *base, unsigned long long value) { *base = value; }
__global__ void k_advance_step(unsigned long long *base, unsigned long long n) { *base += n; }

void launch_set_step(unsigned long long *base, unsigned long long value, cudaStream_t st) {
  k_set_step<<<1, 1, 0, st>>>(base, value);
}

void launch_advance_step(unsigned long long *base, unsigned long long n, cudaStream_t st) {
  k_advance_step<<<1, 1, 0, st>>>(base, n);
}

}  // namespace lbmd
