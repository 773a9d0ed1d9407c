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

// Densities rho_z = sum_i f_zi (appendix, zeroth mode) and j' = sum_z sum_i f_zi c_i.
__global__ void __launch_bounds__(kBlock) k_moments(StepParams P, const float *__restrict__ fin,
                                                    float *__restrict__ rho, float *__restrict__ jp) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const Coord c = site_coord(P, s);
  int xs[3], ys[3], zs[3];
  neighbours(P, c, xs, ys, zs);
  float rA = 0.f, rB = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const long long src = pull_source(P, i, xs, ys, zs);
    const float a = __ldg(fin + (long long)i * P.N + src);
    const float b = __ldg(fin + (long long)(kQ + i) * P.N + src);
    rA += a;
    rB += b;
    jx += kCx[i] * (a + b);
    jy += kCy[i] * (a + b);
    jz += kCz[i] * (a + b);
  }
  rho[s] = rA;
  rho[P.N + s] = rB;
  if (jp) {
    jp[s] = jx;
    jp[P.N + s] = jy;
    jp[2 * P.N + s] = jz;
  }
}

// ---------------------------------------------------------------------------------------
// The lattice update of one step: pull streaming, densities and momentum, Shan-Chen force
// (Eq. SCforce with psi = rho, g_AA = g_BB = 0), fluid-side solvation force and momentum
// return gathered from the particles (Sec. 2), barycentric velocity (Eq.
// momentum_definition), BGK collision with forcing (appendix) for both components.
//
// Each block owns an (x, y) tile of kTX x kTY nodes and marches along a z-range; blocks are
// numbered z-chunk-major so that all tiles of a chunk march in step.  For plane z+1 the
// block pulls the 2 x 19 populations of its tile into shared memory (they are collided one
// plane later without touching DRAM again) and sums them to rho_A, rho_B, j'; it also
// pulls the one-node halo around the tile, keeping only the densities.  A ring of four
// density planes gives the Shan-Chen stencil of plane z.  DRAM traffic per node: the
// populations read once and written once (304 B) plus the halo reads, which hit in L2
// because the neighbouring tile pulls the same lines in the same plane at the same time.
constexpr int kTX = 32, kTY = 8, kFusedThreads = kTX * kTY;
constexpr int kRX = kTX + 2, kRY = kTY + 2;

struct FusedShared {
  float pops[2][2][kQ][kTY][kTX];  // pulled populations of planes z, z+1: [slot][comp][i][y][x]
  float rho[4][2][kRY][kRX];       // densities of planes z-1, z, z+1 (+1 being filled), with halo
  float j[2][3][kTY][kTX];         // j' of the tile, planes z, z+1
};

struct Neigh {
  int xn[3], yn[3], zn[3];  // wrapped coordinates r - 1, r, r + 1 per axis
};

__device__ __forceinline__ Neigh neighbours_of(const StepParams &P, int gx, int gy, int gz) {
  Neigh n;
  n.xn[0] = gx == 0 ? P.nx - 1 : gx - 1; n.xn[1] = gx; n.xn[2] = gx == P.nx - 1 ? 0 : gx + 1;
  n.yn[0] = gy == 0 ? P.ny - 1 : gy - 1; n.yn[1] = gy; n.yn[2] = gy == P.ny - 1 ? 0 : gy + 1;
  n.zn[0] = gz == 0 ? P.nz - 1 : gz - 1; n.zn[1] = gz; n.zn[2] = gz == P.nz - 1 ? 0 : gz + 1;
  return n;
}

__device__ __forceinline__ unsigned pull_src(const StepParams &P, const Neigh &n, int i) {
  // 32-bit: 19 N < 2^32 is enforced when the context is created
  return ((unsigned)n.zn[1 - kCz[i]] * P.ny + n.yn[1 - kCy[i]]) * P.nx + n.xn[1 - kCx[i]];
}

// Pull the 2 x 19 populations of this thread's node of plane p into registers (prefetch).
__device__ __forceinline__ void fused_prefetch(const StepParams &P, const float *__restrict__ fin, int p, int x0,
                                               int y0, float (&fa)[kQ], float (&fb)[kQ]) {
  const unsigned N32 = (unsigned)P.N;
  const float *finB = fin + (size_t)kQ * N32;
  const int lx = threadIdx.x % kTX, ly = threadIdx.x / kTX;
  const Neigh n = neighbours_of(P, wrapi(x0 + lx, P.nx), wrapi(y0 + ly, P.ny), wrapi(p, P.nz));
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const unsigned src = pull_src(P, n, i);
    fa[i] = __ldg(fin + (i * N32 + src));
    fb[i] = __ldg(finB + (i * N32 + src));
  }
}

// Commit plane p: the prefetched populations go to shared memory with their sums rho_A,
// rho_B, j' (tile nodes); the one-node halo around the tile is pulled and summed (rho only).
__device__ __forceinline__ void fused_commit(const StepParams &P, const float *__restrict__ fin, FusedShared &sh,
                                             int p, int zs, int x0, int y0, int w, int h, bool keep_pops,
                                             const float (&fa)[kQ], const float (&fb)[kQ]) {
  const int gz = wrapi(p, P.nz);
  const int slot = (p - zs + 1) & 3;
  const int ps = p & 1;
  const unsigned N32 = (unsigned)P.N;
  const float *finB = fin + (size_t)kQ * N32;
  const int lx = threadIdx.x % kTX, ly = threadIdx.x / kTX;
  if (lx < w && ly < h) {
    float rA = 0.f, rB = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      if (keep_pops) {
        sh.pops[ps][0][i][ly][lx] = fa[i];
        sh.pops[ps][1][i][ly][lx] = fb[i];
      }
      rA += fa[i];
      rB += fb[i];
      jx += kCx[i] * (fa[i] + fb[i]);
      jy += kCy[i] * (fa[i] + fb[i]);
      jz += kCz[i] * (fa[i] + fb[i]);
    }
    sh.rho[slot][0][ly + 1][lx + 1] = rA;
    sh.rho[slot][1][ly + 1][lx + 1] = rB;
    sh.j[ps][0][ly][lx] = jx;
    sh.j[ps][1][ly][lx] = jy;
    sh.j[ps][2][ly][lx] = jz;
  }
  // halo ring of the (w+2) x (h+2) region: rows 0 and h+1, then columns 0 and w+1
  const int nrow = w + 2, nhalo = 2 * nrow + 2 * h;
  for (int k = threadIdx.x; k < nhalo; k += kFusedThreads) {
    int rx, ry;
    if (k < 2 * nrow) {
      ry = k < nrow ? 0 : h + 1;
      rx = k < nrow ? k : k - nrow;
    } else {
      const int c = k - 2 * nrow;
      rx = c < h ? 0 : w + 1;
      ry = 1 + (c < h ? c : c - h);
    }
    const Neigh n = neighbours_of(P, wrapi(x0 + rx - 1, P.nx), wrapi(y0 + ry - 1, P.ny), gz);
    float rA = 0.f, rB = 0.f;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const unsigned src = pull_src(P, n, i);
      rA += __ldg(fin + (i * N32 + src));
      rB += __ldg(finB + (i * N32 + src));
    }
    sh.rho[slot][0][ry][rx] = rA;
    sh.rho[slot][1][ry][rx] = rB;
  }
}

template <bool kParticles>
__global__ void __launch_bounds__(kFusedThreads, 2)
    k_lattice(StepParams P, const float *__restrict__ fin, float *__restrict__ fout, ParticleArrays pa,
              ParticleForces pf, CellIndex ci, unsigned *err, int tiles_x, int ntiles, int zlen) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FusedShared &sh = *reinterpret_cast<FusedShared *>(smem_raw);
  const int lx = threadIdx.x % kTX, ly = threadIdx.x / kTX;
  const int tile = blockIdx.x % ntiles;
  const int zs = (blockIdx.x / ntiles) * zlen;
  const int ze = min(P.nz, zs + zlen);
  const int x0 = (tile % tiles_x) * kTX, y0 = (tile / tiles_x) * kTY;
  const int w = min(kTX, P.nx - x0), h = min(kTY, P.ny - y0);
  const unsigned N32 = (unsigned)P.N;
  float *foutB = fout + (size_t)kQ * N32;
  float fa[kQ], fb[kQ];  // prefetched populations of the next plane to commit
  // prologue: densities of plane zs-1, populations of zs, prefetch of zs+1
  fused_prefetch(P, fin, zs - 1, x0, y0, fa, fb);
  fused_commit(P, fin, sh, zs - 1, zs, x0, y0, w, h, false, fa, fb);
  fused_prefetch(P, fin, zs, x0, y0, fa, fb);
  fused_commit(P, fin, sh, zs, zs, x0, y0, w, h, true, fa, fb);
  fused_prefetch(P, fin, zs + 1, x0, y0, fa, fb);
  for (int z = zs; z < ze; ++z) {
    fused_commit(P, fin, sh, z + 1, zs, x0, y0, w, h, z + 1 < ze, fa, fb);
    // loads of plane z+2 stay in flight while plane z is collided
    if (z + 2 <= ze) fused_prefetch(P, fin, z + 2, x0, y0, fa, fb);
    __syncthreads();
    if (lx < w && ly < h) {
      const int gx = x0 + lx, gy = y0 + ly;
      const int sl[3] = {(z - zs) & 3, (z - zs + 1) & 3, (z - zs + 2) & 3};  // planes z-1, z, z+1
      const int ps = z & 1;
      const float rA = sh.rho[sl[1]][0][ly + 1][lx + 1], rB = sh.rho[sl[1]][1][ly + 1][lx + 1];
      const float jx = sh.j[ps][0][ly][lx], jy = sh.j[ps][1][ly][lx], jz = sh.j[ps][2][ly][lx];
      float SAx = 0.f, SAy = 0.f, SAz = 0.f, SBx = 0.f, SBy = 0.f, SBz = 0.f;
#pragma unroll
      for (int i = 1; i < kQ; ++i) {
        const int s3 = sl[1 + kCz[i]];
        const float a = kW[i] * sh.rho[s3][0][ly + 1 + kCy[i]][lx + 1 + kCx[i]];
        const float b = kW[i] * sh.rho[s3][1][ly + 1 + kCy[i]][lx + 1 + kCx[i]];
        SAx += kCx[i] * a; SAy += kCy[i] * a; SAz += kCz[i] * a;
        SBx += kCx[i] * b; SBy += kCy[i] * b; SBz += kCz[i] * b;
      }
      float3 gA = make_float3(-P.gAB * rA * SBx, -P.gAB * rA * SBy, -P.gAB * rA * SBz);
      float3 gB = make_float3(-P.gBA * rB * SAx, -P.gBA * rB * SAy, -P.gBA * rB * SAz);
      if (kParticles) gather_coupling(P, gx, gy, z, rA, rB, pa, pf, ci, true, gA, gB);
      const float r = rA + rB;
      if (!(rA > 0.f) || !(rB > 0.f) || !isfinite(r)) atomicOr(err, isfinite(r) ? kErrNegDensity : kErrNonFinite);
      const float rinv = 1.f / r;
      const float ux = (jx + 0.5f * (gA.x + gB.x)) * rinv;
      const float uy = (jy + 0.5f * (gA.y + gB.y)) * rinv;
      const float uz = (jz + 0.5f * (gA.z + gB.z)) * rinv;
      const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
      const float ugA3 = 3.f * (ux * gA.x + uy * gA.y + uz * gA.z);
      const float ugB3 = 3.f * (ux * gB.x + uy * gB.y + uz * gB.z);
      const float om = P.inv_tau, fp = P.force_pref;
      const unsigned s = ((unsigned)z * P.ny + gy) * P.nx + gx;
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        const float cu = kCx[i] * ux + kCy[i] * uy + kCz[i] * uz;
        const float poly = kW[i] * (1.f + 3.f * cu + 4.5f * cu * cu - usq15);
        const float cgA = kCx[i] * gA.x + kCy[i] * gA.y + kCz[i] * gA.z;
        const float cgB = kCx[i] * gB.x + kCy[i] * gB.y + kCz[i] * gB.z;
        const float dgA = kW[i] * fp * (3.f * cgA + 9.f * cu * cgA - ugA3);
        const float dgB = kW[i] * fp * (3.f * cgB + 9.f * cu * cgB - ugB3);
        const float fA = sh.pops[ps][0][i][ly][lx], fB = sh.pops[ps][1][i][ly][lx];
        fout[i * N32 + s] = fA - om * (fA - rA * poly) + dgA;
        foutB[i * N32 + s] = fB - om * (fB - rB * poly) + dgB;
      }
    }
    __syncthreads();  // plane z's populations and densities are consumed before they are replaced
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
  const float rA = rho[s], rB = rho[P.N + s];
  float SAx = 0.f, SAy = 0.f, SAz = 0.f, SBx = 0.f, SBy = 0.f, SBz = 0.f;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const long long nb = ((long long)zs[1 + kCz[i]] * P.ny + ys[1 + kCy[i]]) * P.nx + xs[1 + kCx[i]];
    const float a = kW[i] * rho[nb], b = kW[i] * rho[P.N + nb];
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
  (void)rho;
  const int tiles_x = (P.nx + kTX - 1) / kTX, tiles_y = (P.ny + kTY - 1) / kTY;
  const int ntiles = tiles_x * tiles_y;
  const int smem = (int)sizeof(FusedShared);
  static int slots = 0;  // resident blocks of the lattice kernel on this device
  if (slots == 0) {
    cudaFuncSetAttribute(k_lattice<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_lattice<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lattice<true>, kFusedThreads, smem);
    slots = sms * (per_sm > 0 ? per_sm : 1);
  }
  // split z into as many chunks as fit next to one another in one wave
  int chunks = slots / ntiles;
  if (chunks < 1) chunks = 1;
  if (chunks > P.nz) chunks = P.nz;
  const int zlen = (P.nz + chunks - 1) / chunks;
  chunks = (P.nz + zlen - 1) / zlen;
  const unsigned grid = (unsigned)ntiles * (unsigned)chunks;
  if (P.np > 0)
    k_lattice<true><<<grid, kFusedThreads, smem, st>>>(P, fin, fout, pa, pf, ci, err, tiles_x, ntiles, zlen);
  else
    k_lattice<false><<<grid, kFusedThreads, smem, st>>>(P, fin, fout, pa, pf, ci, err, tiles_x, ntiles, zlen);
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
