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

// f^eq (Eq. feq) and the forcing term (appendix, BGK: G = (1 - 1/2tau)(ug + gu)) folded into
// the BGK update f* = f - (f - f^eq)/tau + Delta^g for one component.
__device__ __forceinline__ void collide_component(const StepParams &P, float (&f)[kQ], float rho_c,
                                                  float ux, float uy, float uz, float gx, float gy, float gz) {
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  const float ug3 = 3.f * (ux * gx + uy * gy + uz * gz);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float cu = kCx[i] * ux + kCy[i] * uy + kCz[i] * uz;
    const float cg = kCx[i] * gx + kCy[i] * gy + kCz[i] * gz;
    const float feq = kW[i] * rho_c * (1.f + 3.f * cu + 4.5f * cu * cu - usq15);
    const float dg = kW[i] * P.force_pref * (3.f * cg + 9.f * cu * cg - ug3);
    f[i] = f[i] - P.inv_tau * (f[i] - feq) + dg;
  }
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
// One persistent kernel.  Each block owns an (x, y) tile of kTX x kTY nodes and marches
// along z over a balanced range of tile-planes.  For the plane z+1 it pulls the
// populations of the tile plus a one-node halo and keeps only their sums (rho_A, rho_B,
// and j' for the tile) in a shared-memory ring that holds the planes z-1, z, z+1; then it
// collides plane z one component at a time, pulling that component's 19 populations again
// (they were read one plane earlier and hit in L2).  DRAM traffic per node is the 2 x 19
// populations read once and written once; the Shan-Chen stencil never touches DRAM.
constexpr int kTX = 32, kTY = 8, kFusedThreads = kTX * kTY;
constexpr int kRX = kTX + 2, kRY = kTY + 2;

struct FusedShared {
  float rho[4][2][kRY][kRX];  // ring of densities: planes z-1, z, z+1 (+1 slot being filled)
  float j[3][3][kTY][kTX];    // j' of the tile for planes z, z+1 (+1 slot being filled)
};

__device__ __forceinline__ void fused_fill(const StepParams &P, const float *__restrict__ fin, FusedShared &sh,
                                           int p, int zs, int x0, int y0, int w, int h) {
  const int gz = wrapi(p, P.nz);
  const int slot = (p - zs + 1) & 3;
  const int jslot = (p - zs + 1) % 3;
  int zn[3];
  zn[0] = gz == 0 ? P.nz - 1 : gz - 1;
  zn[1] = gz;
  zn[2] = gz == P.nz - 1 ? 0 : gz + 1;
  const int n = kRX * (h + 2);
  for (int idx = threadIdx.x; idx < n; idx += kFusedThreads) {
    const int ry = idx / kRX, rx = idx - ry * kRX;
    if (rx > w + 1) continue;
    const int gx = wrapi(x0 + rx - 1, P.nx), gy = wrapi(y0 + ry - 1, P.ny);
    int xn[3], yn[3];
    xn[0] = gx == 0 ? P.nx - 1 : gx - 1;
    xn[1] = gx;
    xn[2] = gx == P.nx - 1 ? 0 : gx + 1;
    yn[0] = gy == 0 ? P.ny - 1 : gy - 1;
    yn[1] = gy;
    yn[2] = gy == P.ny - 1 ? 0 : gy + 1;
    float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll 1
    for (int comp = 0; comp < 2; ++comp) {  // one component's 19 loads in flight at a time
      asm volatile("" ::: "memory");
      const float *fc = fin + (long long)comp * kQ * P.N;
      const unsigned N32 = (unsigned)P.N;
      float r = 0.f;
#pragma unroll
      for (int i = 0; i < kQ; ++i) {
        // 32-bit offsets: 19 * N < 2^32 is enforced when the context is created
        const unsigned src = ((unsigned)zn[1 - kCz[i]] * P.ny + yn[1 - kCy[i]]) * P.nx + xn[1 - kCx[i]];
        const float a = __ldg(fc + (i * N32 + src));
        r += a;
        jx += kCx[i] * a;
        jy += kCy[i] * a;
        jz += kCz[i] * a;
      }
      sh.rho[slot][comp][ry][rx] = r;
    }
    if (rx >= 1 && rx <= w && ry >= 1 && ry <= h) {
      sh.j[jslot][0][ry - 1][rx - 1] = jx;
      sh.j[jslot][1][ry - 1][rx - 1] = jy;
      sh.j[jslot][2][ry - 1][rx - 1] = jz;
    }
  }
}

// Collide both components at one node: pull their 2 x 19 populations, BGK + forcing
// (f* = f - (f - f^eq)/tau + Delta^g), write.  Directions [I0, I1) form one batch: its loads
// are issued together, then its updates and stores.
template <int I0, int I1>
__device__ __forceinline__ void fused_collide_batch(const StepParams &P, const float *__restrict__ fin,
                                                    float *__restrict__ fout, unsigned s, const int xn[3],
                                                    const int yn[3], const int zn[3], float rA, float rB,
                                                    float ux, float uy, float uz, float usq15, float3 gA,
                                                    float3 gB, float ugA3, float ugB3) {
  asm volatile("" ::: "memory");  // one batch of loads in registers at a time
  // per-component base pointers; offsets within a component stay below 19 N < 2^32
  const unsigned N32 = (unsigned)P.N;
  const float *finA = fin, *finB = fin + (size_t)kQ * N32;
  float *foutA = fout, *foutB = fout + (size_t)kQ * N32;
  float fA[I1 - I0], fB[I1 - I0];
#pragma unroll
  for (int i = I0; i < I1; ++i) {
    const unsigned src = ((unsigned)zn[1 - kCz[i]] * P.ny + yn[1 - kCy[i]]) * P.nx + xn[1 - kCx[i]];
    fA[i - I0] = __ldg(finA + (i * N32 + src));
    fB[i - I0] = __ldg(finB + (i * N32 + src));
  }
  const float om = P.inv_tau, fp = P.force_pref;
#pragma unroll
  for (int i = I0; i < I1; ++i) {
    const float cu = kCx[i] * ux + kCy[i] * uy + kCz[i] * uz;
    const float poly = kW[i] * (1.f + 3.f * cu + 4.5f * cu * cu - usq15);
    const float cgA = kCx[i] * gA.x + kCy[i] * gA.y + kCz[i] * gA.z;
    const float cgB = kCx[i] * gB.x + kCy[i] * gB.y + kCz[i] * gB.z;
    const float dgA = kW[i] * fp * (3.f * cgA + 9.f * cu * cgA - ugA3);
    const float dgB = kW[i] * fp * (3.f * cgB + 9.f * cu * cgB - ugB3);
    foutA[i * N32 + s] = fA[i - I0] - om * (fA[i - I0] - rA * poly) + dgA;
    foutB[i * N32 + s] = fB[i - I0] - om * (fB[i - I0] - rB * poly) + dgB;
  }
}

__device__ __forceinline__ void fused_collide(const StepParams &P, const float *__restrict__ fin,
                                              float *__restrict__ fout, unsigned s, const int xn[3],
                                              const int yn[3], const int zn[3], float rA, float rB, float ux,
                                              float uy, float uz, float3 gA, float3 gB) {
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  const float ugA3 = 3.f * (ux * gA.x + uy * gA.y + uz * gA.z);
  const float ugB3 = 3.f * (ux * gB.x + uy * gB.y + uz * gB.z);
  fused_collide_batch<0, 10>(P, fin, fout, s, xn, yn, zn, rA, rB, ux, uy, uz, usq15, gA, gB, ugA3, ugB3);
  fused_collide_batch<10, kQ>(P, fin, fout, s, xn, yn, zn, rA, rB, ux, uy, uz, usq15, gA, gB, ugA3, ugB3);
}

template <bool kParticles>
__global__ void __launch_bounds__(kFusedThreads, 4)
    k_lattice(StepParams P, const float *__restrict__ fin, float *__restrict__ fout, ParticleArrays pa,
              ParticleForces pf, CellIndex ci, unsigned *err, int tiles_x, long long work) {
  __shared__ FusedShared sh;
  const int lx = threadIdx.x % kTX, ly = threadIdx.x / kTX;
  const long long G = gridDim.x;
  long long w0 = work * blockIdx.x / G;
  const long long w1 = work * (blockIdx.x + 1) / G;
  while (w0 < w1) {
    const long long tile = w0 / P.nz;
    const int zs = (int)(w0 - tile * P.nz);
    const int ze = (int)(zs + (w1 - w0) < P.nz ? zs + (w1 - w0) : P.nz);
    const int x0 = (int)(tile % tiles_x) * kTX, y0 = (int)(tile / tiles_x) * kTY;
    const int w = min(kTX, P.nx - x0), h = min(kTY, P.ny - y0);
    __syncthreads();  // the previous segment's readers of the rings are done
    fused_fill(P, fin, sh, zs - 1, zs, x0, y0, w, h);
    fused_fill(P, fin, sh, zs, zs, x0, y0, w, h);
    for (int z = zs; z < ze; ++z) {
      fused_fill(P, fin, sh, z + 1, zs, x0, y0, w, h);
      __syncthreads();
      if (lx < w && ly < h) {
        const int gx = x0 + lx, gy = y0 + ly;
        int xn[3], yn[3], zn[3];
        xn[0] = gx == 0 ? P.nx - 1 : gx - 1;
        xn[1] = gx;
        xn[2] = gx == P.nx - 1 ? 0 : gx + 1;
        yn[0] = gy == 0 ? P.ny - 1 : gy - 1;
        yn[1] = gy;
        yn[2] = gy == P.ny - 1 ? 0 : gy + 1;
        zn[0] = z == 0 ? P.nz - 1 : z - 1;
        zn[1] = z;
        zn[2] = z == P.nz - 1 ? 0 : z + 1;
        const int sl[3] = {(z - zs) & 3, (z - zs + 1) & 3, (z - zs + 2) & 3};  // planes z-1, z, z+1
        const int js = (z - zs + 1) % 3;
        const float rA = sh.rho[sl[1]][0][ly + 1][lx + 1], rB = sh.rho[sl[1]][1][ly + 1][lx + 1];
        const float jx = sh.j[js][0][ly][lx], jy = sh.j[js][1][ly][lx], jz = sh.j[js][2][ly][lx];
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
        const unsigned s = ((unsigned)z * P.ny + gy) * P.nx + gx;
        fused_collide(P, fin, fout, s, xn, yn, zn, rA, rB, ux, uy, uz, gA, gB);
      }
    }
    w0 += ze - zs;
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
  const long long work = (long long)tiles_x * tiles_y * P.nz;
  static int grid_cap = 0;  // resident blocks of the persistent kernel (all SMs, full occupancy)
  if (grid_cap == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lattice<true>, kFusedThreads, 0);
    grid_cap = sms * (per_sm > 0 ? per_sm : 1);
  }
  // at least ~4 planes per block so the two prologue planes stay a small overhead
  long long grid = (work + 3) / 4;
  if (grid > grid_cap) grid = grid_cap;
  if (grid < 1) grid = 1;
  if (P.np > 0)
    k_lattice<true><<<(unsigned)grid, kFusedThreads, 0, st>>>(P, fin, fout, pa, pf, ci, err, tiles_x, work);
  else
    k_lattice<false><<<(unsigned)grid, kFusedThreads, 0, st>>>(P, fin, fout, pa, pf, ci, err, tiles_x, work);
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
