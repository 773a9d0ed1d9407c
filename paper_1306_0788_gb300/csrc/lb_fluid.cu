// lb_fluid.cu -- lattice kernels of the coupled Shan-Chen LB / MD step (sm_103a).
//
// Storage: populations of both components in one buffer [2][19][nz][ny][nx] (structure of
// arrays, x fastest).  The buffer holds the post-collision values f*(r, t-1) at their source
// node; a kernel "pulls" f_i(r, t) = f*_i(r - c_i, t-1), so reads are coalesced along x
// (shifted by at most one element) and writes are fully coalesced.  Element type: FP32, or a
// 16-bit type (FP16, BF16) holding the shifted value f_i - w_i rho0_z; all arithmetic is FP32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "lbmd_internal.cuh"

namespace lbmd {

namespace {

constexpr int kBlock = 256;

// Load / store of one population value; `shift` = w_i rho0_z (ignored for FP32 storage).
// enc / dec convert between the FP32 value and the stored element.
template <class T>
struct Pop;
template <>
struct Pop<float> {
  static __device__ __forceinline__ float enc(float v, float) { return v; }
  static __device__ __forceinline__ float dec(float e, float) { return e; }
  static __device__ __forceinline__ float ld(const float *p, float) { return __ldg(p); }
  static __device__ __forceinline__ float rd(const float *p, float) { return *p; }
  static __device__ __forceinline__ void st(float *p, float v, float) { *p = v; }
};
template <>
struct Pop<__half> {
  static __device__ __forceinline__ __half enc(float v, float sh) { return __float2half_rn(v - sh); }
  static __device__ __forceinline__ float dec(__half e, float sh) { return __half2float(e) + sh; }
  static __device__ __forceinline__ float ld(const __half *p, float sh) { return dec(__ldg(p), sh); }
  static __device__ __forceinline__ float rd(const __half *p, float sh) { return dec(*p, sh); }
  static __device__ __forceinline__ void st(__half *p, float v, float sh) { *p = enc(v, sh); }
};
template <>
struct Pop<__nv_bfloat16> {
  static __device__ __forceinline__ __nv_bfloat16 enc(float v, float sh) { return __float2bfloat16_rn(v - sh); }
  static __device__ __forceinline__ float dec(__nv_bfloat16 e, float sh) { return __bfloat162float(e) + sh; }
  static __device__ __forceinline__ float ld(const __nv_bfloat16 *p, float sh) { return dec(__ldg(p), sh); }
  static __device__ __forceinline__ float rd(const __nv_bfloat16 *p, float sh) { return dec(*p, sh); }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v, float sh) { *p = enc(v, sh); }
};

// With 16-bit storage the rest population f_0 (which does not stream) is kept in an FP32 array
// rest[2][N]; these read / write direction i of component c at site s from the right place.
template <class T>
__device__ __forceinline__ float pop_read(const StepParams &P, const T *buf, const float *rest, int c, int i,
                                          long long s) {
  if (i == 0 && rest) return rest[(long long)c * P.N + s];
  return Pop<T>::rd(buf + ((long long)c * kQ + i) * P.N + s, kW[i] * P.rho0[c]);
}
template <class T>
__device__ __forceinline__ void pop_write(const StepParams &P, T *buf, float *rest, int c, int i, long long s,
                                          float v) {
  if (i == 0 && rest)
    rest[(long long)c * P.N + s] = v;
  else
    Pop<T>::st(buf + ((long long)c * kQ + i) * P.N + s, v, kW[i] * P.rho0[c]);
}

__device__ __forceinline__ float pop_shift(const StepParams &P, int comp, int i) { return kW[i] * P.rho0[comp]; }

struct Coord {
  int x, y, z;
};

__device__ __forceinline__ Coord site_coord(const StepParams &P, long long s) {
  Coord c;
  c.x = (int)(s % P.nx);
  const long long t = s / P.nx;
  c.y = (int)(t % P.ny);
  c.z = (int)(t / P.ny);
  return c;
}

// source coordinate of direction i for a pull at (x, y, z): r - c_i, periodic
__device__ __forceinline__ long long pull_source(const StepParams &P, int i, const int xs[3], const int ys[3],
                                                 const int zs[3]) {
  // xs = {x-1, x, x+1} wrapped; r - c_i selects index 1 - c
  return ((long long)zs[1 - kCz[i]] * P.ny + ys[1 - kCy[i]]) * P.nx + xs[1 - kCx[i]];
}

__device__ __forceinline__ void neighbours(const StepParams &P, const Coord &c, int xs[3], int ys[3], int zs[3]) {
  xs[0] = c.x == 0 ? P.nx - 1 : c.x - 1;
  xs[1] = c.x;
  xs[2] = c.x == P.nx - 1 ? 0 : c.x + 1;
  ys[0] = c.y == 0 ? P.ny - 1 : c.y - 1;
  ys[1] = c.y;
  ys[2] = c.y == P.ny - 1 ? 0 : c.y + 1;
  zs[0] = c.z == 0 ? P.nz - 1 : c.z - 1;
  zs[1] = c.z;
  zs[2] = c.z == P.nz - 1 ? 0 : c.z + 1;
}

// Periodic neighbour offsets of site s: d[a][0] is the offset to coordinate a - 1, d[a][1] to a + 1
// (wrap-aware), so the site r + c is s + d[0][c_x] + d[1][c_y] + d[2][c_z] in 32-bit arithmetic
// (19 N < 2^32 is enforced when a context is created).
struct NOff {
  int m[3], p[3];  // offsets to the -1 and +1 neighbour along x, y, z
};

__device__ __forceinline__ NOff neighbour_offsets(const StepParams &P, const Coord &c) {
  NOff o;
  const int nxny = P.nx * P.ny;
  o.m[0] = c.x == 0 ? P.nx - 1 : -1;
  o.p[0] = c.x == P.nx - 1 ? -(P.nx - 1) : 1;
  o.m[1] = c.y == 0 ? (P.ny - 1) * P.nx : -P.nx;
  o.p[1] = c.y == P.ny - 1 ? -(P.ny - 1) * P.nx : P.nx;
  o.m[2] = c.z == 0 ? (P.nz - 1) * nxny : -nxny;
  o.p[2] = c.z == P.nz - 1 ? -(P.nz - 1) * nxny : nxny;
  return o;
}

// offset of r + (cx, cy, cz) relative to r, each component in {-1, 0, 1}
__device__ __forceinline__ int shift(const NOff &o, int cx, int cy, int cz) {
  return (cx < 0 ? o.m[0] : cx > 0 ? o.p[0] : 0) + (cy < 0 ? o.m[1] : cy > 0 ? o.p[1] : 0) +
         (cz < 0 ? o.m[2] : cz > 0 ? o.p[2] : 0);
}

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

// Densities rho_z = sum_i f_zi (appendix, zeroth mode), stored interleaved (rho_A, rho_B) per
// site, and j' = sum_z sum_i f_zi c_i.
template <class T>
__global__ void __launch_bounds__(kBlock) k_moments(StepParams P, const T *__restrict__ fin,
                                                    const float *__restrict__ rest, float *__restrict__ rho,
                                                    float *__restrict__ jp) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const Coord c = site_coord(P, s);
  const NOff o = neighbour_offsets(P, c);
  const unsigned N32 = (unsigned)P.N, s32 = (unsigned)s;
  const T *finB = fin + (size_t)kQ * N32;
  float rA = 0.f, rB = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const unsigned src = i * N32 + (unsigned)((int)s32 + shift(o, -kCx[i], -kCy[i], -kCz[i]));  // pull r - c_i
    const float a = (i == 0 && rest) ? __ldg(rest + s32) : Pop<T>::ld(fin + src, pop_shift(P, 0, i));
    const float b = (i == 0 && rest) ? __ldg(rest + N32 + s32) : Pop<T>::ld(finB + src, pop_shift(P, 1, i));
    rA += a;
    rB += b;
    jx += kCx[i] * (a + b);
    jy += kCy[i] * (a + b);
    jz += kCz[i] * (a + b);
  }
  reinterpret_cast<float2 *>(rho)[s] = make_float2(rA, rB);
  if (jp) {
    jp[s] = jx;
    jp[P.N + s] = jy;
    jp[2 * P.N + s] = jz;
  }
}

// The lattice update of one step at one node: pull, densities and momentum, Shan-Chen force
// (Eq. SCforce with psi = rho, g_AA = g_BB = 0), fluid-side solvation force and momentum
// return from the particles (Sec. 2), barycentric velocity (Eq. momentum_definition), BGK
// collision with forcing for both components, write.
template <class T, bool kParticles>
__global__ void __launch_bounds__(kBlock, 3) k_collide(StepParams P, const T *__restrict__ fin,
                                                    T *__restrict__ fout, const float *__restrict__ rho,
                                                    ParticleArrays pa, ParticleForces pf, CellIndex ci,
                                                    unsigned *err, const float *__restrict__ rest_in,
                                                    float *__restrict__ rest_out) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const Coord c = site_coord(P, s);
  const NOff o = neighbour_offsets(P, c);
  const unsigned N32 = (unsigned)P.N, s32 = (unsigned)s;
  const T *finB = fin + (size_t)kQ * N32;
  float fA[kQ], fB[kQ];
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const unsigned src = i * N32 + (unsigned)((int)s32 + shift(o, -kCx[i], -kCy[i], -kCz[i]));  // pull r - c_i
    fA[i] = Pop<T>::ld(fin + src, pop_shift(P, 0, i));
    fB[i] = Pop<T>::ld(finB + src, pop_shift(P, 1, i));
  }
  if (rest_in) {  // 16-bit storage: the rest populations are kept in FP32
    fA[0] = __ldg(rest_in + s32);
    fB[0] = __ldg(rest_in + N32 + s32);
  }
  float rA = 0.f, rB = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    rA += fA[i];
    rB += fB[i];
    jx += kCx[i] * (fA[i] + fB[i]);
    jy += kCy[i] * (fA[i] + fB[i]);
    jz += kCz[i] * (fA[i] + fB[i]);
  }
  // S_z = sum_i w_i rho_z(r + c_i) c_i from the density field of this step
  const float2 *rho2 = reinterpret_cast<const float2 *>(rho);
  float SAx = 0.f, SAy = 0.f, SAz = 0.f, SBx = 0.f, SBy = 0.f, SBz = 0.f;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const unsigned nb = (unsigned)((int)s32 + shift(o, kCx[i], kCy[i], kCz[i]));
    const float2 r2 = __ldg(rho2 + nb);
    const float a = kW[i] * r2.x, b = kW[i] * r2.y;
    SAx += kCx[i] * a; SAy += kCy[i] * a; SAz += kCz[i] * a;
    SBx += kCx[i] * b; SBy += kCy[i] * b; SBz += kCz[i] * b;
  }
  float3 gA = make_float3(-P.gAB * rA * SBx, -P.gAB * rA * SBy, -P.gAB * rA * SBz);
  float3 gB = make_float3(-P.gBA * rB * SAx, -P.gBA * rB * SAy, -P.gBA * rB * SAz);
  if (kParticles) gather_coupling(P, c.x, c.y, c.z, rA, rB, pa, pf, ci, true, gA, gB);
  const float r = rA + rB;
  if (!(rA > 0.f) || !(rB > 0.f) || !isfinite(r)) atomicOr(err, isfinite(r) ? kErrNegDensity : kErrNonFinite);
  const float rinv = 1.f / r;
  const float ux = (jx + 0.5f * (gA.x + gB.x)) * rinv;
  const float uy = (jy + 0.5f * (gA.y + gB.y)) * rinv;
  const float uz = (jz + 0.5f * (gA.z + gB.z)) * rinv;
  // BGK + forcing, f* = (1 - 1/tau) f + (1/tau) f^eq + Delta^g, per pair of opposite directions
  // (c_j = -c_i): f^eq and Delta^g split into parts even and odd in c.
  {
    const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float ugA3 = 3.f * (ux * gA.x + uy * gA.y + uz * gA.z);
    const float ugB3 = 3.f * (ux * gB.x + uy * gB.y + uz * gB.z);
    const float om = P.inv_tau, om1 = 1.f - om, fp = P.force_pref;
    const float aA = om * rA, aB = om * rB;
    fA[0] = om1 * fA[0] + aA * kW[0] * (1.f - usq15) - kW[0] * fp * ugA3;
    fB[0] = om1 * fB[0] + aB * kW[0] * (1.f - usq15) - kW[0] * fp * ugB3;
#pragma unroll
    for (int i = 1; i < kQ; i += 2) {
      const int j = i + 1;
      const float cu = kCx[i] * ux + kCy[i] * uy + kCz[i] * uz;
      const float cgA = kCx[i] * gA.x + kCy[i] * gA.y + kCz[i] * gA.z;
      const float cgB = kCx[i] * gB.x + kCy[i] * gB.y + kCz[i] * gB.z;
      const float sym = kW[i] * (1.f + 4.5f * cu * cu - usq15), anti = 3.f * kW[i] * cu;
      const float wf = kW[i] * fp;
      const float symA = wf * (9.f * cu * cgA - ugA3), antiA = 3.f * wf * cgA;
      const float symB = wf * (9.f * cu * cgB - ugB3), antiB = 3.f * wf * cgB;
      const float fAi = fA[i], fAj = fA[j], fBi = fB[i], fBj = fB[j];
      fA[i] = om1 * fAi + aA * (sym + anti) + symA + antiA;
      fA[j] = om1 * fAj + aA * (sym - anti) + symA - antiA;
      fB[i] = om1 * fBi + aB * (sym + anti) + symB + antiB;
      fB[j] = om1 * fBj + aB * (sym - anti) + symB - antiB;
    }
  }
  T *foutB = fout + (size_t)kQ * N32;
  if (rest_out) {
    // 16-bit storage: each moving population is rounded on store; the FP32 rest population takes
    // the rounding error of the node's 18 others, so the node's total (and the total mass of each
    // component) is the one of the collision up to FP32 rounding instead of drifting each step.
    float eA = 0.f, eB = 0.f;
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
      const auto a = Pop<T>::enc(fA[i], pop_shift(P, 0, i));
      const auto b = Pop<T>::enc(fB[i], pop_shift(P, 1, i));
      fout[i * N32 + s32] = a;
      foutB[i * N32 + s32] = b;
      eA += fA[i] - Pop<T>::dec(a, pop_shift(P, 0, i));
      eB += fB[i] - Pop<T>::dec(b, pop_shift(P, 1, i));
    }
    rest_out[s32] = fA[0] + eA;
    rest_out[N32 + s32] = fB[0] + eB;
  } else {
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      Pop<T>::st(fout + (i * N32 + s32), fA[i], pop_shift(P, 0, i));
      Pop<T>::st(foutB + (i * N32 + s32), fB[i], pop_shift(P, 1, i));
    }
  }
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
    if (P.np > 0)
      k_collide<T, true><<<grid_for(P.N), kBlock, 0, st>>>(P, a, b, rho, pa, pf, ci, err, rest, rest);
    else
      k_collide<T, false><<<grid_for(P.N), kBlock, 0, st>>>(P, a, b, rho, pa, pf, ci, err, rest, rest);
  });
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

}  // namespace lbmd
