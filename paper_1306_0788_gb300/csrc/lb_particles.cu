// lb_particles.cu -- particle kernels of the coupled Shan-Chen LB / MD step (sm_103a):
// deterministic counting sort by lattice row, coupling forces (Eqs. NEWTON,
// solvation_kappa, solvation_lambda with trilinear interpolation), short-range pair and
// bonded forces (owner computes, no atomics), and the particle update.
#include "lbmd_internal.cuh"

namespace lbmd {

namespace {

constexpr int kPBlock = 128;

inline unsigned pgrid(int n) { return (unsigned)((n + kPBlock - 1) / kPBlock); }

// Lattice row (z, y) of each particle and the row histogram.
__global__ void k_bin(StepParams P, ParticleArrays pa, int *__restrict__ row_of, int *__restrict__ row_count,
                      unsigned *err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  int4 c = pa.cell[p];
  if (c.x < 0 || c.x >= P.nx || c.y < 0 || c.y >= P.ny || c.z < 0 || c.z >= P.nz) {
    atomicOr(err, kErrParticle);  // cannot happen for states written by this library
    c.x = wrapi(c.x, P.nx); c.y = wrapi(c.y, P.ny); c.z = wrapi(c.z, P.nz);
    pa.cell[p] = c;
  }
  const int row = c.z * P.ny + c.y;
  row_of[p] = row;
  atomicAdd(row_count + row, 1);
}

// Exclusive scan of the row histogram (rows -> first sorted slot) in three passes: per-block
// sums of 2048 rows, a scan of the block sums, and the in-block scans.  Also primes the
// scatter cursors.
constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 8;
constexpr int kScanRows = kScanThreads * kScanPerThread;

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_tot, int &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;  // inclusive warp-total prefix
  }
  __syncthreads();
  total = warp_tot[kScanThreads / 32 - 1];
  const int before = warp == 0 ? 0 : warp_tot[warp - 1];
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partial(int nrows, const int *__restrict__ count,
                                                               int *__restrict__ bsum) {
  __shared__ int wt[kScanThreads / 32];
  const int base = blockIdx.x * kScanRows + threadIdx.x * kScanPerThread;
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k)
    if (base + k < nrows) sum += count[base + k];
  int total;
  block_exclusive_scan(sum, wt, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int nb, int *__restrict__ bsum) {
  __shared__ int wt[kScanThreads / 32];
  const int per = (nb + kScanThreads - 1) / kScanThreads;
  const int b = threadIdx.x * per;
  int sum = 0;
  for (int k = 0; k < per; ++k)
    if (b + k < nb) sum += bsum[b + k];
  int total;
  int run = block_exclusive_scan(sum, wt, total);
  for (int k = 0; k < per; ++k)
    if (b + k < nb) {
      const int c = bsum[b + k];
      bsum[b + k] = run;
      run += c;
    }
  if (threadIdx.x == 0) bsum[nb] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(int nrows, int nb, const int *__restrict__ count,
                                                             const int *__restrict__ bsum, int *__restrict__ start,
                                                             int *__restrict__ cursor) {
  __shared__ int wt[kScanThreads / 32];
  const int base = blockIdx.x * kScanRows + threadIdx.x * kScanPerThread;
  int c[kScanPerThread];
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    c[k] = base + k < nrows ? count[base + k] : 0;
    sum += c[k];
  }
  int total;
  int run = bsum[blockIdx.x] + block_exclusive_scan(sum, wt, total);
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k)
    if (base + k < nrows) {
      start[base + k] = run;
      cursor[base + k] = run;
      run += c[k];
    }
  if (blockIdx.x == nb - 1 && threadIdx.x == 0) start[nrows] = bsum[nb];
}

__global__ void k_scatter(int np, const int *__restrict__ row_of, int *__restrict__ cursor, int *__restrict__ perm) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  perm[atomicAdd(cursor + row_of[p], 1)] = p;
}

// Order each row by (x cell, particle id) so the sort, and every gather after it, is
// deterministic.  Rows hold few particles: insertion sort, one thread per row.
__global__ void k_row_sort(StepParams P, const int *__restrict__ start, ParticleArrays pa, int *__restrict__ perm) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= P.nrows) return;
  const int b = start[row], e = start[row + 1];
  for (int i = b + 1; i < e; ++i) {
    const int v = perm[i];
    const long long kv = ((long long)pa.cell[v].x << 32) | (unsigned)pa.pid[v];
    int j = i - 1;
    while (j >= b) {
      const int w = perm[j];
      const long long kw = ((long long)pa.cell[w].x << 32) | (unsigned)pa.pid[w];
      if (kw <= kv) break;
      perm[j + 1] = w;
      --j;
    }
    perm[j + 1] = v;
  }
}

__global__ void k_permute(int np, const int *__restrict__ perm, ParticleArrays src, ParticleArrays dst,
                          int *__restrict__ slot_of_id) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  const int p = perm[j];
  dst.cell[j] = src.cell[p];
  dst.frac[j] = src.frac[p];
  dst.vel[j] = src.vel[p];
  const int id = src.pid[p];
  dst.pid[j] = id;
  slot_of_id[id] = j;
}

struct NodeState {
  float rA, rB;
  float3 SA, SB;  // sum_i w_i rho_z(r + c_i) c_i
};

__device__ __forceinline__ NodeState node_state(const StepParams &P, const float *__restrict__ rho, int x, int y,
                                                int z) {
  NodeState n;
  const float2 *rho2 = reinterpret_cast<const float2 *>(rho);  // interleaved (rho_A, rho_B)
  const long long s = site_index(P, x, y, z);
  n.rA = __ldg(rho2 + s).x;
  n.rB = __ldg(rho2 + s).y;
  n.SA = make_float3(0.f, 0.f, 0.f);
  n.SB = make_float3(0.f, 0.f, 0.f);
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const long long nb = site_index(P, wrapi(x + kCx[i], P.nx), wrapi(y + kCy[i], P.ny), wrapi(z + kCz[i], P.nz));
    const float2 r2 = __ldg(rho2 + nb);
    const float a = kW[i] * r2.x, b = kW[i] * r2.y;
    n.SA.x += kCx[i] * a; n.SA.y += kCy[i] * a; n.SA.z += kCz[i] * a;
    n.SB.x += kCx[i] * b; n.SB.y += kCy[i] * b; n.SB.z += kCz[i] * b;
  }
  return n;
}

// Coupling forces on each particle (Sec. 2): the coupling velocity u_cpl = (j' + (g^SC + F^fs)/2)/rho
// and the node gradients S/c_s^2 are interpolated trilinearly from the 8 corners of the
// particle's cell; friction + noise (Eq. NEWTON), solvation (Eq. solvation_kappa) and the
// reaction of the particle's own fluid-side solvation force (Eq. solvation_lambda).
__global__ void __launch_bounds__(kPBlock) k_couple(StepParams P, ParticleArrays pa, CellIndex ci,
                                                    const float *__restrict__ rho, const float *__restrict__ jp,
                                                    ParticleForces pf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  const int4 c = pa.cell[p];
  const float4 fr = pa.frac[p];
  const float4 v = pa.vel[p];
  const TypeParams &T = P.types[c.w];
  float3 up = make_float3(0.f, 0.f, 0.f), gA = up, gB = up, fsr = up;
  for (int k = 0; k < 8; ++k) {
    const int ox = k & 1, oy = (k >> 1) & 1, oz = (k >> 2) & 1;
    const int X = c.x + ox == P.nx ? 0 : c.x + ox;
    const int Y = c.y + oy == P.ny ? 0 : c.y + oy;
    const int Z = c.z + oz == P.nz ? 0 : c.z + oz;
    const NodeState n = node_state(P, rho, X, Y, Z);
    float3 fA = make_float3(-P.gAB * n.rA * n.SB.x, -P.gAB * n.rA * n.SB.y, -P.gAB * n.rA * n.SB.z);
    float3 fB = make_float3(-P.gBA * n.rB * n.SA.x, -P.gBA * n.rB * n.SA.y, -P.gBA * n.rB * n.SA.z);
    gather_coupling(P, X, Y, Z, n.rA, n.rB, pa, pf, ci, false, fA, fB);
    const long long s = site_index(P, X, Y, Z);
    const float rinv = 1.f / (n.rA + n.rB);
    const float w = (ox ? fr.x : 1.f - fr.x) * (oy ? fr.y : 1.f - fr.y) * (oz ? fr.z : 1.f - fr.z);
    up.x += w * (__ldg(jp + s) + 0.5f * (fA.x + fB.x)) * rinv;
    up.y += w * (__ldg(jp + P.N + s) + 0.5f * (fA.y + fB.y)) * rinv;
    up.z += w * (__ldg(jp + 2 * P.N + s) + 0.5f * (fA.z + fB.z)) * rinv;
    gA.x += w * n.SA.x; gA.y += w * n.SA.y; gA.z += w * n.SA.z;
    gB.x += w * n.SB.x; gB.y += w * n.SB.y; gB.z += w * n.SB.z;
    if (T.lam[0] != 0.f || T.lam[1] != 0.f) {
      const float3 geo = fs_geometry(fr.x - ox, fr.y - oy, fr.z - oz);
      const float a = T.lam[0] * n.rA + T.lam[1] * n.rB;
      fsr.x += a * geo.x; fsr.y += a * geo.y; fsr.z += a * geo.z;
    }
  }
  float3 R = make_float3(0.f, 0.f, 0.f);
  if (T.noise_amp > 0.f) {
    const float3 nn = particle_normals(P.seed, P.step, (unsigned)pa.pid[p]);
    R = make_float3(T.noise_amp * nn.x, T.noise_amp * nn.y, T.noise_amp * nn.z);
  }
  pf.fric[p] = make_float4(-T.gamma * (v.x - up.x) + R.x, -T.gamma * (v.y - up.y) + R.y,
                           -T.gamma * (v.z - up.z) + R.z, 0.f);
  const float kA = -T.kappa[0] / kCs2, kB = -T.kappa[1] / kCs2;
  pf.psA[p] = make_float4(kA * gA.x, kA * gA.y, kA * gA.z, 0.f);
  pf.psB[p] = make_float4(kB * gB.x, kB * gB.y, kB * gB.z, 0.f);
  pf.fsr[p] = make_float4(fsr.x, fsr.y, fsr.z, 0.f);
}

__device__ __forceinline__ int min_image_cells(int d, int n) {
  d = wrapi(d, n);
  return 2 * d > n ? d - n : d;
}

// Short-range pair forces (WCA, Sec. 4.1; screened Coulomb, Sec. 4.4) over the rows within
// `reach` cells, and bonded forces from each particle's own bond list.  Each particle
// computes its own force (pairs are visited from both ends): no atomics, fixed order.
__global__ void __launch_bounds__(kPBlock) k_pairs(StepParams P, ParticleArrays pa, CellIndex ci,
                                                   const int *__restrict__ bond_start,
                                                   const int *__restrict__ bond_other,
                                                   const int *__restrict__ slot_of_id, ParticleForces pf,
                                                   unsigned *err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  const int4 c = pa.cell[p];
  const float4 fr = pa.frac[p];
  float3 F = make_float3(0.f, 0.f, 0.f);
  const int m = P.reach;
  const bool allz = 2 * m + 1 >= P.nz, ally = 2 * m + 1 >= P.ny, allx = 2 * m + 1 >= P.nx;
  const int z0 = allz ? 0 : -m, z1 = allz ? P.nz - 1 : m;
  const int y0 = ally ? 0 : -m, y1 = ally ? P.ny - 1 : m;
  const float Lx = (float)P.nx, Ly = (float)P.ny, Lz = (float)P.nz;
  if (m > 0) {
    for (int dz = z0; dz <= z1; ++dz) {
      const int cz = allz ? dz : wrapi(c.z + dz, P.nz);
      for (int dy = y0; dy <= y1; ++dy) {
        const int cy = ally ? dy : wrapi(c.y + dy, P.ny);
        const int row = cz * P.ny + cy;
        const int q0 = ci.row_start[row], q1 = ci.row_start[row + 1];
        for (int q = q0; q < q1; ++q) {
          if (q == p) continue;
          const int4 cq = pa.cell[q];
          const int dcx = min_image_cells(c.x - cq.x, P.nx);
          if (!allx && (dcx > m || dcx < -m)) continue;
          const float4 fq = pa.frac[q];
          float dx = (float)dcx + (fr.x - fq.x);
          float dy_ = (float)min_image_cells(c.y - cq.y, P.ny) + (fr.y - fq.y);
          float dz_ = (float)min_image_cells(c.z - cq.z, P.nz) + (fr.z - fq.z);
          dx -= Lx * rintf(dx / Lx);
          dy_ -= Ly * rintf(dy_ / Ly);
          dz_ -= Lz * rintf(dz_ / Lz);
          const float r2 = dx * dx + dy_ * dy_ + dz_ * dz_;
          float fscal = 0.f;  // -dU/dr / r
          const PairParams &pp = P.pairs[c.w * LBMD_MAX_TYPES + cq.w];
          if (pp.eps > 0.f && r2 < pp.rc2) {
            const float sr2 = pp.sigma2 / r2;
            const float sr6 = sr2 * sr2 * sr2;
            fscal += 24.f * pp.eps * (2.f * sr6 * sr6 - sr6) / r2;
          }
          const float qq = fr.w * fq.w;
          if (P.dh_lB != 0.f && qq != 0.f && r2 < P.dh_rc2) {
            const float r = sqrtf(r2);
            fscal += qq * P.dh_lB * expf(-P.dh_kappa * r) * (1.f / r2 + P.dh_kappa / r) / r;
          }
          F.x += fscal * dx;
          F.y += fscal * dy_;
          F.z += fscal * dz_;
        }
      }
    }
  }
  if (bond_start) {
    const int id = pa.pid[p];
    for (int b = bond_start[id]; b < bond_start[id + 1]; ++b) {
      const int q = slot_of_id[bond_other[b]];
      const int4 cq = pa.cell[q];
      const float4 fq = pa.frac[q];
      float dx = (float)min_image_cells(c.x - cq.x, P.nx) + (fr.x - fq.x);
      float dy_ = (float)min_image_cells(c.y - cq.y, P.ny) + (fr.y - fq.y);
      float dz_ = (float)min_image_cells(c.z - cq.z, P.nz) + (fr.z - fq.z);
      dx -= Lx * rintf(dx / Lx);
      dy_ -= Ly * rintf(dy_ / Ly);
      dz_ -= Lz * rintf(dz_ / Lz);
      const float r2 = dx * dx + dy_ * dy_ + dz_ * dz_;
      float fscal;
      if (P.bond_kind == LBMD_BOND_FENE) {
        const float x2 = r2 / (P.bond_r * P.bond_r);
        if (!(x2 < 1.f)) {
          atomicOr(err, kErrBond);
          continue;
        }
        fscal = -P.bond_k / (1.f - x2);
      } else {
        const float r = sqrtf(r2);
        fscal = r > 0.f ? -P.bond_k * (r - P.bond_r) / r : 0.f;
      }
      F.x += fscal * dx;
      F.y += fscal * dy_;
      F.z += fscal * dz_;
    }
  }
  pf.pair[p] = make_float4(F.x, F.y, F.z, 0.f);
}

// Particle update: v += F dt / m, x += v dt, periodic wrap kept as (cell, fraction).
__global__ void k_integrate(StepParams P, ParticleArrays pa, ParticleForces pf, unsigned *err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.np) return;
  int4 c = pa.cell[p];
  float4 fr = pa.frac[p];
  float4 v = pa.vel[p];
  const TypeParams &T = P.types[c.w];
  const float4 a = pf.fric[p], b = pf.psA[p], d = pf.psB[p], e = pf.fsr[p], g = pf.pair[p];
  const float Fx = a.x + b.x + d.x + e.x + g.x;
  const float Fy = a.y + b.y + d.y + e.y + g.y;
  const float Fz = a.z + b.z + d.z + e.z + g.z;
  pf.total[p] = make_float4(Fx, Fy, Fz, 0.f);
  v.x += Fx * P.dt * T.inv_mass;
  v.y += Fy * P.dt * T.inv_mass;
  v.z += Fz * P.dt * T.inv_mass;
  float nx_ = fr.x + v.x * P.dt, ny_ = fr.y + v.y * P.dt, nz_ = fr.z + v.z * P.dt;
  const float lim = 1.0e6f;
  if (!(fabsf(nx_) < lim && fabsf(ny_) < lim && fabsf(nz_) < lim)) {
    atomicOr(err, kErrParticle | kErrNonFinite);
    pa.vel[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;  // position kept: every index stays inside the lattice
  }
  const float sx = floorf(nx_), sy = floorf(ny_), sz = floorf(nz_);
  nx_ -= sx; ny_ -= sy; nz_ -= sz;
  int ix = (int)sx, iy = (int)sy, iz = (int)sz;
  if (nx_ >= 1.f) { nx_ = 0.f; ++ix; }
  if (ny_ >= 1.f) { ny_ = 0.f; ++iy; }
  if (nz_ >= 1.f) { nz_ = 0.f; ++iz; }
  c.x = wrapi(c.x + ix, P.nx);
  c.y = wrapi(c.y + iy, P.ny);
  c.z = wrapi(c.z + iz, P.nz);
  pa.cell[p] = c;
  pa.frac[p] = make_float4(nx_, ny_, nz_, fr.w);
  pa.vel[p] = v;
}

constexpr int kMomBlock = 256;
__global__ void __launch_bounds__(kMomBlock) k_particle_momentum(StepParams P, ParticleArrays pa,
                                                                 double *__restrict__ partial) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.np; p += gridDim.x * blockDim.x) {
    const float4 v = pa.vel[p];
    const double m = (double)P.types[pa.cell[p].w].mass;
    acc[0] += m * v.x;
    acc[1] += m * v.y;
    acc[2] += m * v.z;
  }
  __shared__ double sh[3][kMomBlock];
  for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kMomBlock / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) partial[(long long)blockIdx.x * 3 + k] = sh[k][0];
}

}  // namespace

void launch_bin(const StepParams &P, const ParticleArrays &pa, int *row_of, int *row_count, unsigned *err,
                cudaStream_t st) {
  k_bin<<<pgrid(P.np), kPBlock, 0, st>>>(P, pa, row_of, row_count, err);
}
int scan_blocks(int nrows) { return (nrows + kScanRows - 1) / kScanRows; }
void launch_scan_rows(int nrows, const int *row_count, int *row_start, int *row_cursor, int *bsum, cudaStream_t st) {
  const int nb = scan_blocks(nrows);
  k_scan_partial<<<nb, kScanThreads, 0, st>>>(nrows, row_count, bsum);
  k_scan_top<<<1, kScanThreads, 0, st>>>(nb, bsum);
  k_scan_final<<<nb, kScanThreads, 0, st>>>(nrows, nb, row_count, bsum, row_start, row_cursor);
}
void launch_scatter(int np, const int *row_of, int *row_cursor, int *perm, cudaStream_t st) {
  k_scatter<<<pgrid(np), kPBlock, 0, st>>>(np, row_of, row_cursor, perm);
}
void launch_row_sort(const StepParams &P, const int *row_start, const ParticleArrays &pa, int *perm,
                     cudaStream_t st) {
  k_row_sort<<<pgrid(P.nrows), kPBlock, 0, st>>>(P, row_start, pa, perm);
}
void launch_permute(int np, const int *perm, const ParticleArrays &src, const ParticleArrays &dst, int *slot_of_id,
                    cudaStream_t st) {
  k_permute<<<pgrid(np), kPBlock, 0, st>>>(np, perm, src, dst, slot_of_id);
}
void launch_couple(const StepParams &P, const ParticleArrays &pa, CellIndex ci, const float *rho, const float *jp,
                   const ParticleForces &pf, cudaStream_t st) {
  k_couple<<<pgrid(P.np), kPBlock, 0, st>>>(P, pa, ci, rho, jp, pf);
}
void launch_pairs(const StepParams &P, const ParticleArrays &pa, CellIndex ci, const int *bond_start,
                  const int *bond_other, const int *slot_of_id, const ParticleForces &pf, unsigned *err,
                  cudaStream_t st) {
  k_pairs<<<pgrid(P.np), kPBlock, 0, st>>>(P, pa, ci, bond_start, bond_other, slot_of_id, pf, err);
}
void launch_integrate(const StepParams &P, const ParticleArrays &pa, const ParticleForces &pf, unsigned *err,
                      cudaStream_t st) {
  k_integrate<<<pgrid(P.np), kPBlock, 0, st>>>(P, pa, pf, err);
}
void launch_particle_momentum(const StepParams &P, const ParticleArrays &pa, double *partial, int nblocks,
                              cudaStream_t st) {
  k_particle_momentum<<<nblocks, kMomBlock, 0, st>>>(P, pa, partial);
}

}  // namespace lbmd
