// lb_fluid.cu -- lattice kernels of the coupled Shan-Chen LB / MD step (sm_103a).
//
// Storage: populations of both components in one FP32 buffer [2][19][nz][ny][nx]
// (structure of arrays, x fastest).  The buffer holds the post-collision values f*(r, t-1)
// at their source node; a kernel "pulls" f_i(r, t) = f*_i(r - c_i, t-1), so reads are
// coalesced along x (shifted by at most one element) and writes are fully coalesced.
#include "lbmd_internal.cuh"

namespace lbmd {

namespace {

constexpr int kBlock = 256;

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

__global__ void __launch_bounds__(kBlock) k_init_equilibrium(StepParams P, const float *__restrict__ rhoA,
                                                             const float *__restrict__ rhoB,
                                                             const float *__restrict__ u, float *__restrict__ store) {
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
    for (int z = 0; z < 2; ++z) store[((long long)z * kQ + i) * P.N + dst] = kW[i] * rc[z] * poly;
  }
}

__global__ void __launch_bounds__(kBlock) k_restream(StepParams P, const float *__restrict__ post, int comp,
                                                     float *__restrict__ store) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const Coord c = site_coord(P, s);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const long long dst = site_index(P, wrapi(c.x - kCx[i], P.nx), wrapi(c.y - kCy[i], P.ny), wrapi(c.z - kCz[i], P.nz));
    store[((long long)comp * kQ + i) * P.N + dst] = post[(long long)i * P.N + s];
  }
}

__global__ void __launch_bounds__(kBlock) k_unstream(StepParams P, const float *__restrict__ store, int comp,
                                                     float *__restrict__ post) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const Coord c = site_coord(P, s);
  int xs[3], ys[3], zs[3];
  neighbours(P, c, xs, ys, zs);
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    post[(long long)i * P.N + s] = store[((long long)comp * kQ + i) * P.N + pull_source(P, i, xs, ys, zs)];
}

// Densities rho_z = sum_i f_zi (appendix, zeroth mode), stored interleaved (rho_A, rho_B) per
// site, and j' = sum_z sum_i f_zi c_i.
__global__ void __launch_bounds__(kBlock) k_moments(StepParams P, const float *__restrict__ fin,
                                                    float *__restrict__ rho, float *__restrict__ jp) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const Coord c = site_coord(P, s);
  const NOff o = neighbour_offsets(P, c);
  const unsigned N32 = (unsigned)P.N, s32 = (unsigned)s;
  const float *finB = fin + (size_t)kQ * N32;
  float rA = 0.f, rB = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const unsigned src = i * N32 + (unsigned)((int)s32 + shift(o, -kCx[i], -kCy[i], -kCz[i]));  // pull r - c_i
    const float a = __ldg(fin + src);
    const float b = __ldg(finB + src);
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
template <bool kParticles>
__global__ void __launch_bounds__(kBlock, 3) k_collide(StepParams P, const float *__restrict__ fin,
                                                    float *__restrict__ fout, const float *__restrict__ rho,
                                                    ParticleArrays pa, ParticleForces pf, CellIndex ci,
                                                    unsigned *err) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const Coord c = site_coord(P, s);
  const NOff o = neighbour_offsets(P, c);
  const unsigned N32 = (unsigned)P.N, s32 = (unsigned)s;
  const float *finB = fin + (size_t)kQ * N32;
  float fA[kQ], fB[kQ];
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const unsigned src = i * N32 + (unsigned)((int)s32 + shift(o, -kCx[i], -kCy[i], -kCz[i]));  // pull r - c_i
    fA[i] = __ldg(fin + src);
    fB[i] = __ldg(finB + src);
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
  float *foutB = fout + (size_t)kQ * N32;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    fout[i * N32 + s32] = fA[i];
    foutB[i * N32 + s32] = fB[i];
  }
}

// rho_A, rho_B and u = (j' + g^SC/2)/rho at the current step (for readback).
__global__ void __launch_bounds__(kBlock) k_fields(StepParams P, const float *__restrict__ store,
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
    const float a = store[(long long)i * P.N + src] + store[(long long)(kQ + i) * P.N + src];
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
__global__ void __launch_bounds__(kSumBlock) k_fluid_sums(StepParams P, const float *__restrict__ store,
                                                          double *__restrict__ partial) {
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < P.N;
       s += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const double a = (double)store[(long long)i * P.N + s];
      const double b = (double)store[(long long)(kQ + i) * P.N + s];
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

void launch_init_equilibrium(const StepParams &P, const float *rhoA, const float *rhoB, const float *u,
                             float *store, cudaStream_t st) {
  k_init_equilibrium<<<grid_for(P.N), kBlock, 0, st>>>(P, rhoA, rhoB, u, store);
}
void launch_restream(const StepParams &P, const float *post, int comp, float *store, cudaStream_t st) {
  k_restream<<<grid_for(P.N), kBlock, 0, st>>>(P, post, comp, store);
}
void launch_unstream(const StepParams &P, const float *store, int comp, float *post, cudaStream_t st) {
  k_unstream<<<grid_for(P.N), kBlock, 0, st>>>(P, store, comp, post);
}
void launch_moments(const StepParams &P, const float *store, float *rho, float *jp, cudaStream_t st) {
  k_moments<<<grid_for(P.N), kBlock, 0, st>>>(P, store, rho, jp);
}
void launch_collide(const StepParams &P, const float *fin, float *fout, const float *rho,
                    const ParticleArrays &pa, const ParticleForces &pf, CellIndex ci, unsigned *err,
                    cudaStream_t st) {
  if (P.np > 0)
    k_collide<true><<<grid_for(P.N), kBlock, 0, st>>>(P, fin, fout, rho, pa, pf, ci, err);
  else
    k_collide<false><<<grid_for(P.N), kBlock, 0, st>>>(P, fin, fout, rho, pa, pf, ci, err);
}
void launch_fields(const StepParams &P, const float *store, const float *rho, float *rhoA, float *rhoB,
                   float *u, cudaStream_t st) {
  k_fields<<<grid_for(P.N), kBlock, 0, st>>>(P, store, rho, rhoA, rhoB, u);
}
int fluid_sum_blocks(const StepParams &P) {
  long long b = (P.N + kSumBlock - 1) / kSumBlock;
  return (int)(b < 1024 ? b : 1024);
}
void launch_fluid_sums(const StepParams &P, const float *store, double *partial, int nblocks, cudaStream_t st) {
  k_fluid_sums<<<nblocks, kSumBlock, 0, st>>>(P, store, partial);
}
void launch_finish_sums(const double *partial, int nblocks, int nvals, double *out, cudaStream_t st) {
  k_finish_sums<<<1, 32, 0, st>>>(partial, nblocks, nvals, out);
}

}  // namespace lbmd
