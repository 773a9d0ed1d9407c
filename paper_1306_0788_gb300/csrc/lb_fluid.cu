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

// ------------------------------------------------------------------ one-pass update
//
// Streaming carries f*_i(r) to r + c_i, so the next density of a node is the sum of the
// post-collision values arriving from its 19 sources: the update can form it from the values it
// has just computed instead of a second pass pulling every population again.  Each warp of a
// block owns one row y of an 8-row column tile and its 32 nodes x0 .. x0 + 31 (one per lane), and
// the block marches along z through one chunk of planes; the blocks of one chunk cover
// neighbouring tiles and are launched together, so that they march in step and the sectors they
// share meet in L2.  Per plane, for each of the 9 (c_y, c_z) groups of directions, a lane adds
// the values arriving at its node from c_x = 0, +1 (lane below) and -1 (lane above); the groups
// with c_y = +-1 go to the neighbouring rows through shared memory (double buffered: one barrier
// per plane), and each row adds what arrives at it into three accumulators, for the planes z - 1,
// z and z + 1.  After plane z the plane z - 1 is complete and is written.  What leaves the tile
// along x -- from lane 0 with c_x = -1, from the last lane with c_x = +1 -- is summed the same way
// into edge partials for the neighbouring tiles' edge nodes, which k_boundary_densities adds.  Every
// sum has a fixed order.  Nodes with sources in another block along y or z -- the first and last
// row of the tile, the first and last plane of the chunk -- get the same treatment: the block
// writes its part (across the tile's bottom and top rows per lane; for the planes below and at
// the chunk's start, and at and above its end, what its accumulators hold), and
// k_boundary_densities adds the parts of the two blocks.  Where a lattice is too thin for the
// partial sums (tiles of fewer than 3 rows or 2 columns; one plane), k_boundary_densities pulls
// those nodes' populations as the density pass does.
constexpr int kOPThreads = kOnePassRows * 32;
// the densities a block's stencils read in one plane: rows y0 - 1 .. y0 + 8, columns x0 - 1 ..
// x0 + 32
constexpr int kRhoRows = kOnePassRows + 2, kRhoCols = kOnePassCols + 2, kRhoSlots = 4;
static_assert(kOnePassCols == 32 && kRhoCols - 32 <= 32, "a warp stages a ring row with one or two copies per lane");
static_assert(kOnePassRows - 1 <= 15, "pair barriers 1 .. kOnePassRows - 1");

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// 8-byte asynchronous copy global -> shared (cp.async), its commit and wait.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Named barrier `id` (1 .. 15; 0 is __syncthreads) for `n` threads of the block, all of whose
// warps take it convergently.
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory"); }

// The staged densities of a block's stencil: a ring of kRhoSlots planes.
struct StagedRho {
  static constexpr bool kStaged = true;
  const float2 (*ring)[kRhoRows][kRhoCols];
  int sm, s0, sp;  // slots of the planes z - 1, z, z + 1
  int k, j;        // this node's row and column in a plane
  __device__ float2 operator()(int cx, int cy, int cz) const {
    return ring[cz < 0 ? sm : (cz > 0 ? sp : s0)][k + cy][j + cx];
  }
};

// The elements of a staged plane: element e of the kRhoRows x kRhoCols rows y0 - 1 + e / kRhoCols,
// columns x0 - 1 + e % kRhoCols (both wrapped periodically) has the offset src[e] = y nx + x within
// a plane.  The same for every plane of a march: computed once per block, kept in shared memory
// (not in registers, which the update needs).
__device__ __forceinline__ void stage_sources(const StepParams &P, int x0, int y0, int *src) {
  for (int e = threadIdx.x; e < kRhoRows * kRhoCols; e += kOPThreads) {
    const int r = e / kRhoCols, j = e - r * kRhoCols;
    const int y = ((y0 - 1 + r) % P.ny + P.ny) % P.ny, x = ((x0 - 1 + j) % P.nx + P.nx) % P.nx;
    src[e] = y * P.nx + x;
  }
}

// The part of plane z's staged densities warp w copies (cp.async) into ring slot `slot_index` % 4:
// ring row w + 1, and the halo rows 0 (warp 0) and kRhoRows - 1 (the last warp).  The stencils
// of warp w read ring rows w .. w + 2, which warps w - 1 .. w + 1 copy.
__device__ __forceinline__ void stage_rows(const StepParams &P, const float *__restrict__ rho,
                                           float2 (*ring)[kRhoRows][kRhoCols], int slot_index, int z,
                                           const int *src, int w, int lane) {
  const float2 *plane = reinterpret_cast<const float2 *>(rho) + (long long)z * P.ny * P.nx;
  float2 *slot = &ring[slot_index & (kRhoSlots - 1)][0][0];
  auto row = [&](int r) {
    const int e = r * kRhoCols + lane;
    cp_async8(slot + e, plane + src[e]);
    if (lane < kRhoCols - 32) cp_async8(slot + e + 32, plane + src[e + 32]);
  };
  row(w + 1);
  if (w == 0) row(0);
  if (w == kOnePassRows - 1) row(kRhoRows - 1);
  cp_async_commit();
}

// Copies (cp.async) the densities of plane z into ring slot `slot_index` % 4 (the elements of
// stage_sources); every thread of the block takes part.  The slot follows the unwrapped plane
// index (z - 1 .. z + 2 of a march take four distinct slots even where the lattice is shorter than
// four planes).
__device__ __forceinline__ void stage_plane(const StepParams &P, const float *__restrict__ rho,
                                            float2 (*ring)[kRhoRows][kRhoCols], int slot_index, int z,
                                            const int *src) {
  const float2 *plane = reinterpret_cast<const float2 *>(rho) + (long long)z * P.ny * P.nx;
  float2 *slot = &ring[slot_index & (kRhoSlots - 1)][0][0];
  for (int e = threadIdx.x; e < kRhoRows * kRhoCols; e += kOPThreads) cp_async8(slot + e, plane + src[e]);
  cp_async_commit();
}

template <class T, bool kParticles>
__global__ void __launch_bounds__(kOPThreads, 3)
    k_collide_onepass(StepParams P, const T *__restrict__ fin, T *__restrict__ fout, const float *__restrict__ rho,
                      float *__restrict__ rho_next, OnePassOut out, ParticleArrays pa, ParticleForces pf,
                      CellIndex ci, unsigned *err, const float *__restrict__ rest_in, float *__restrict__ rest_out,
                      OnePassGeom G) {
  // groups handed to the neighbouring rows: [0..2] c_y = +1 with c_z = -1, 0, +1; [3..5] c_y = -1;
  // row w at index w + 1, indices 0 and kOnePassRows + 1 always 0 (the rows beyond the tile, whose
  // parts arrive as partial sums), so that a row adds its neighbours' without a select
  __shared__ float2 xch[2][6][kOnePassRows + 2][32];
  // the same for what leaves the tile along x: [side][c_y = +1, -1][row] (side 0: from lane 0
  // towards x0 - 1; side 1: from the last lane towards x0 + 32)
  __shared__ float2 xedge[2][2][2][kOnePassRows];
  // each thread's arrivals at its node, and each row's edge partials, in planes p with slot p % 3
  // (in shared memory rather than registers: they live across the whole update of a node)
  __shared__ float2 acc[3][kOPThreads];
  __shared__ float2 accE[3][2][kOnePassRows];
  // what leaves the tile across its bottom (0) and top (1) row, per lane
  __shared__ float2 accY[3][2][32];
  // the stencils' densities, read from global memory once per block and plane
  __shared__ float2 ring[kRhoSlots][kRhoRows][kRhoCols];
  __shared__ int stage_src[kRhoRows * kRhoCols];  // where each staged element comes from (stage_sources)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr unsigned kFull = 0xffffffffu;
  const int ncols = G.ntx * G.nty, chunk = blockIdx.x / ncols, col = blockIdx.x - chunk * ncols;
  const int zs = (int)((long long)chunk * P.nz / G.nchunks), ze = (int)((long long)(chunk + 1) * P.nz / G.nchunks);
  if (ze <= zs) return;  // block-uniform
  const int tx = col % G.ntx, ty = col / G.ntx;
  const int x0 = tx * kOnePassCols, nown = min(kOnePassCols, P.nx - x0);
  const bool own = lane < nown;
  const int x = own ? x0 + lane : x0;
  const int y0 = ty * kOnePassRows, rows = min(kOnePassRows, P.ny - y0);
  const int y = y0 + w;
  const bool inner_row = w >= 1 && w <= rows - 2;  // the sources along y are in the block
  const bool left = lane == 0, right = lane == nown - 1;  // the tile's x edges (both when nown = 1)
  acc[0][threadIdx.x] = acc[1][threadIdx.x] = acc[2][threadIdx.x] = make_float2(0.f, 0.f);
  for (int e = threadIdx.x; e < 2 * 6 * 2 * 32; e += kOPThreads) {
    const int r = (e >> 5) & 1, pg = e >> 6;
    xch[pg / 6][pg % 6][r ? kOnePassRows + 1 : 0][e & 31] = make_float2(0.f, 0.f);
  }
  if (threadIdx.x < 3 * 2 * kOnePassRows) (&accE[0][0][0])[threadIdx.x] = make_float2(0.f, 0.f);
  if (threadIdx.x < 3 * 2 * 32) (&accY[0][0][0])[threadIdx.x] = make_float2(0.f, 0.f);
  // rows whose partial sums the block forms: the inner ones, and with y partials the edge rows too
  // (lacking what arrives from the neighbouring tile's row, which that tile sends)
  const bool summed_row = w < rows && (G.ypart || inner_row);
  const bool lo = w > 0, hi = w < rows - 1;  // the rows below / above are in the block
  stage_sources(P, x0, y0, stage_src);
  __syncthreads();
  for (int dz = -1; dz <= 1; ++dz)
    stage_plane(P, rho, ring, zs + dz + kRhoSlots, (zs + dz + P.nz) % P.nz, stage_src);
  cp_async_wait_all();
  __syncthreads();
  int parity = 0;
  for (int z = zs; z < ze; ++z, parity ^= 1) {
    const int z2 = z + 2 < P.nz ? z + 2 : (z + 2) % P.nz;
    stage_rows(P, rho, ring, z + 2, z2, stage_src, w, lane);  // for the next plane; its slot is free
    float fA[kQ], fB[kQ];
    if (own && w < rows) {
      const long long s = ((long long)z * P.ny + y) * P.nx + x;
      float rA, rB;
      const StagedRho st{ring, (z + kRhoSlots - 1) & (kRhoSlots - 1), z & (kRhoSlots - 1),
                         (z + 1) & (kRhoSlots - 1), w + 1, lane + 1};
      collide_core_at<T, kParticles, false, false, StagedRho>(P, Coord{x, y, z}, s, P.step, fin, rho, pa, pf, ci,
                                                              err, rest_in, fA, fB, rA, rB, st);
      store_node<T, false, true, true>(P, (unsigned)s, fout, rest_out, fA, fB, rA, rB);
    } else {
#pragma unroll
      for (int i = 0; i < kQ; ++i) fA[i] = fB[i] = 0.f;
    }
    // arrivals of one (c_y, c_z) group at this lane's node: c_x = 0, +1 (from the lane below, none
    // for lane 0), -1 (from the lane above, none for the last lane)
    auto group = [&](int i0, int ip, int im) {
      float pA = __shfl_up_sync(kFull, fA[ip], 1), pB = __shfl_up_sync(kFull, fB[ip], 1);
      float mA = __shfl_down_sync(kFull, fA[im], 1), mB = __shfl_down_sync(kFull, fB[im], 1);
      if (lane == 0) pA = pB = 0.f;
      if (lane + 1 >= nown) mA = mB = 0.f;
      return add2(add2(make_float2(fA[i0], fB[i0]), make_float2(pA, pB)), make_float2(mA, mB));
    };
    float2(*X)[kOnePassRows + 2][32] = xch[parity];
    X[0][w + 1][lane] = make_float2(fA[17], fB[17]);  // (c_y, c_z) = (+1, -1)
    X[1][w + 1][lane] = group(3, 7, 10);              // (+1, 0)
    X[2][w + 1][lane] = make_float2(fA[15], fB[15]);  // (+1, +1)
    X[3][w + 1][lane] = make_float2(fA[16], fB[16]);  // (-1, -1)
    X[4][w + 1][lane] = group(4, 9, 8);               // (-1, 0)
    X[5][w + 1][lane] = make_float2(fA[18], fB[18]);  // (-1, +1)
    if (left) {  // leaving towards x0 - 1 with c_y = +1, -1
      xedge[parity][0][0][w] = make_float2(fA[10], fB[10]);
      xedge[parity][0][1][w] = make_float2(fA[8], fB[8]);
    }
    if (right) {  // leaving towards x0 + 32 with c_y = +1, -1
      xedge[parity][1][0][w] = make_float2(fA[7], fB[7]);
      xedge[parity][1][1][w] = make_float2(fA[9], fB[9]);
    }
    const float2 g0m = group(6, 13, 12), g00 = group(0, 1, 2), g0p = group(5, 11, 14);
    cp_async_wait_all();  // this warp's rows of the next plane's densities (issued above) have landed
    // The exchange with the rows below and above, and the staged rows they read: a barrier with
    // each neighbouring warp only (pair (w - 1, w) is barrier w), taken in that order.  A warp
    // passes plane z's barriers after its neighbours have written plane z's exchange and staged
    // rows, and writes the same buffers again (plane z + 2) only after they have passed plane
    // z + 1's, i.e. after they have read plane z's.
    if (w > 0) bar_sync(w, 64);
    if (w < kOnePassRows - 1) bar_sync(w + 1, 64);
    const int km = (z + 2) % 3, k0 = z % 3, kp = (z + 1) % 3;
    // plane z - 1 has all its sources (z - 2 .. z) in the chunk, or (with z partial sums) it is the
    // first plane of the chunk or the one below it, and this is the upper chunk's part
    const bool write = G.zpart || z >= zs + 2;
    const int zm = z == 0 ? P.nz - 1 : z - 1;
    const float2 zero = make_float2(0.f, 0.f);
    if (own && summed_row) {
      // from the row below (c_y = +1), this row (c_y = 0), the row above (c_y = -1), into the
      // planes z - 1, z, z + 1 (rows beyond the block and the rows of a ragged tile's absent
      // warps hold 0)
      const float2 am = add2(add2(add2(acc[km][threadIdx.x], X[0][w][lane]), g0m), X[3][w + 2][lane]);
      acc[k0][threadIdx.x] = add2(add2(add2(acc[k0][threadIdx.x], X[1][w][lane]), g00), X[4][w + 2][lane]);
      acc[kp][threadIdx.x] = add2(add2(add2(acc[kp][threadIdx.x], X[2][w][lane]), g0p), X[5][w + 2][lane]);
      if (write)
        reinterpret_cast<float2 *>(rho_next)[((long long)zm * P.ny + y) * P.nx + x] =
            add2(am, make_float2(shift_sum(P, 0), shift_sum(P, 1)));
      acc[km][threadIdx.x] = zero;  // becomes plane z + 2
    }
    if (summed_row && (left || right)) {
      // what leaves the tile along x, for the neighbouring tiles' edge nodes in this row: the
      // side-0 sums from lane 0 (c_x = -1: directions 2, 10, 8, 14, 12), the side-1 sums from the
      // last lane (c_x = +1: 1, 7, 9, 11, 13)
      float2 *edge2 = reinterpret_cast<float2 *>(out.edge);
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        if (side == 0 ? !left : !right) continue;
        const int i00 = side ? 1 : 2, i0p = side ? 11 : 14, i0m = side ? 13 : 12;
        const float2 em = add2(accE[km][side][w], make_float2(fA[i0m], fB[i0m]));
        accE[k0][side][w] = add2(add2(add2(accE[k0][side][w], lo ? xedge[parity][side][0][w - 1] : zero),
                                      make_float2(fA[i00], fB[i00])),
                                 hi ? xedge[parity][side][1][w + 1] : zero);
        accE[kp][side][w] = add2(accE[kp][side][w], make_float2(fA[i0p], fB[i0p]));
        if (write) edge2[(((long long)zm * P.ny + y) * G.ntx + tx) * 2 + side] = em;
        accE[km][side][w] = zero;
      }
    }
    if (G.ypart && own && (w == 0 || w == rows - 1)) {
      // what leaves the tile across its bottom row (the c_y = -1 groups of row 0) or its top row
      // (the c_y = +1 groups of the last row), for the neighbouring tile's edge row
      const int sy = w == 0 ? 0 : 1, g = sy ? 0 : 3;
      const float2 ym = add2(accY[km][sy][lane], X[g][w + 1][lane]);
      accY[k0][sy][lane] = add2(accY[k0][sy][lane], X[g + 1][w + 1][lane]);
      accY[kp][sy][lane] = add2(accY[kp][sy][lane], X[g + 2][w + 1][lane]);
      if (write)
        reinterpret_cast<float2 *>(out.yedge)[(((long long)sy * P.nz + zm) * G.nty + ty) * (G.ntx * kOnePassCols) +
                                              x0 + lane] = ym;
      accY[km][sy][lane] = zero;
      // the value leaving each corner diagonally (c_z = 0: it arrives in this plane)
      if ((left || right) && (G.zpart || (z >= zs + 1 && z <= ze - 2))) {
        const int k = (sy << 1) | (right ? 1 : 0);  // 0: bottom-left ... 3: top-right
        // directions 8, 9, 10, 7 (constant indices: the arrays stay in registers)
        const float2 d = sy ? (right ? make_float2(fA[7], fB[7]) : make_float2(fA[10], fB[10]))
                            : (right ? make_float2(fA[9], fB[9]) : make_float2(fA[8], fB[8]));
        reinterpret_cast<float2 *>(out.diag)[(((long long)z * G.nty + ty) * G.ntx + tx) * 4 + k] = d;
      }
    }
  }
  if (G.zpart) {
    // this chunk's part of the planes ze - 1 and ze, the first two planes of the boundary with the
    // next chunk (slots 2 b, 2 b + 1): what the last iteration left in the accumulators
    const int b = chunk + 1 == G.nchunks ? 0 : chunk + 1;
    const int k0 = (ze - 1) % 3, kp = ze % 3;
    if (own && summed_row) {
      float2 *zo = reinterpret_cast<float2 *>(out.zown);
      zo[((long long)(2 * b) * P.ny + y) * P.nx + x] = acc[k0][threadIdx.x];
      zo[((long long)(2 * b + 1) * P.ny + y) * P.nx + x] = acc[kp][threadIdx.x];
    }
    if (summed_row && (left || right)) {
      float2 *ze2 = reinterpret_cast<float2 *>(out.zedge);
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        if (side == 0 ? !left : !right) continue;
        ze2[(((long long)(2 * b) * P.ny + y) * G.ntx + tx) * 2 + side] = accE[k0][side][w];
        ze2[(((long long)(2 * b + 1) * P.ny + y) * G.ntx + tx) * 2 + side] = accE[kp][side][w];
      }
    }
    if (G.ypart && own && (w == 0 || w == rows - 1)) {
      const int sy = w == 0 ? 0 : 1;
      float2 *zy = reinterpret_cast<float2 *>(out.zyedge);
      const long long stride = (long long)G.nty * G.ntx * kOnePassCols;
      zy[((long long)sy * 2 * G.nchunks + 2 * b) * stride + (long long)ty * G.ntx * kOnePassCols + x0 + lane] =
          accY[k0][sy][lane];
      zy[((long long)sy * 2 * G.nchunks + 2 * b + 1) * stride + (long long)ty * G.ntx * kOnePassCols + x0 + lane] =
          accY[kp][sy][lane];
    }
  }
  cp_async_wait_all();  // no copy outlives the block
}

// The nodes the one-pass update leaves unfinished, in one launch of five block ranges (range 5
// first):
//  1. the boundary runs, a warp per run: their densities from the new populations, as the density
//     pass computes them (without y partials the first and last row of each tile; without z
//     partials the first and last plane of each chunk);
//  2. the x-edge nodes of the inner rows: own partial (in rho_next) plus what arrives from the
//     neighbouring tile -- from the left one's side-1 sums at x0, from the right one's side-0 sums
//     at x0 + nown - 1 (both, in that order, when a tile has one column);
//  3. with y partials, the edge rows: own partial plus what the tile below (for the bottom row) or
//     above (for the top row) sends across, and at the two corners also the x-neighbour's edge-row
//     sums and the value the diagonal neighbour sends, in that order;
//  4. with z partials, the other nodes of the chunk-edge planes: own partial plus the lower
//     chunk's;
//  5. with particles, j' of the new populations at the 8 corners of each particle's cell, for the
//     next step's coupling (jc, by particle id; pn: the particles as the next step starts).
// In ranges 2 and 3 a chunk-edge plane's node adds the lower chunk's part after each term.  The
// sets of nodes are disjoint, and every node's sum has a fixed order.
template <class T>
__global__ void __launch_bounds__(kBlock) k_boundary_densities(StepParams P, OnePassGeom G, const T *__restrict__ store,
                                                               const float *__restrict__ rest,
                                                               float *__restrict__ rho_next,
                                                               const BoundaryRun *__restrict__ runs, int nruns,
                                                               int corner_blocks, int run_blocks, int edge_blocks,
                                                               int row_blocks, OnePassOut out,
                                                               const int *__restrict__ zslot, ParticleArrays pn,
                                                               int np, float4 *__restrict__ jc) {
  // the latency-bound corner j' blocks first, so that they run beside the others
  if ((int)blockIdx.x < corner_blocks) {
    // 5: corner j' (a thread per particle and corner)
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8LL * np) return;
    const int p = (int)(t >> 3), k = (int)(t & 7);
    const Coord cc = cell_corner(P, __ldg(pn.cell + p), k);
    const float3 j = jprime_at<T>(P, store, cc.x, cc.y, cc.z);
    jc[(long long)__ldg(pn.pid + p) * 8 + k] = make_float4(j.x, j.y, j.z, 0.f);
    return;
  }
  const int bid = (int)blockIdx.x - corner_blocks;
  if (bid < run_blocks) {
    const int r = bid * (kBlock / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= nruns) return;
    const BoundaryRun b = runs[r];
    if (lane >= b.n) return;
    moments(P, (long long)b.row * P.nx + b.x0 + lane, store, rest, rho_next, nullptr);
    return;
  }
  const float2 *e2 = reinterpret_cast<const float2 *>(out.edge);
  const float2 *zo = reinterpret_cast<const float2 *>(out.zown);
  const float2 *ze2 = reinterpret_cast<const float2 *>(out.zedge);
  float2 *rho2 = reinterpret_cast<float2 *>(rho_next);
  const long long plane = (long long)P.ny * P.nx;
  if (bid < run_blocks + edge_blocks) {
    // 32-bit index arithmetic: nz ny ntx < N < 2^32 / 19
    const unsigned t = (unsigned)(bid - run_blocks) * blockDim.x + threadIdx.x;
    const unsigned n = (unsigned)P.nz * P.ny * G.ntx;
    if (t >= n) return;
    const unsigned r = t / G.ntx;  // z * ny + y
    const int tx = (int)(t - r * G.ntx);
    const int z = (int)(r / P.ny), y = (int)(r - (unsigned)z * P.ny);
    const int w = y % kOnePassRows, y0 = y - w, rows = min(kOnePassRows, P.ny - y0);
    if (w < 1 || w > rows - 2) return;  // tile edge rows: runs, or range 3
    const int q = zslot[z];             // chunk-edge plane: its slot in the z arrays
    if (q >= 0 && !G.zpart) return;     // runs
    const int x0 = tx * kOnePassCols, nown = min(kOnePassCols, P.nx - x0);
    const int txl = tx == 0 ? G.ntx - 1 : tx - 1, txr = tx == G.ntx - 1 ? 0 : tx + 1;
    const long long base = (long long)r * P.nx;
    const long long zb = ((long long)q * P.ny + y) * P.nx;  // this row in the z arrays (q >= 0)
    const long long zr = (long long)q * P.ny + y;
    float2 v = rho2[base + x0];
    if (q >= 0) v = add2(v, zo[zb + x0]);
    v = add2(v, e2[((long long)r * G.ntx + txl) * 2 + 1]);  // from the left tile's last lane
    if (q >= 0) v = add2(v, ze2[(zr * G.ntx + txl) * 2 + 1]);
    if (nown == 1) {  // and from the right tile's lane 0
      v = add2(v, e2[((long long)r * G.ntx + txr) * 2 + 0]);
      if (q >= 0) v = add2(v, ze2[(zr * G.ntx + txr) * 2 + 0]);
      rho2[base + x0] = v;
      return;
    }
    rho2[base + x0] = v;
    const int xr = x0 + nown - 1;
    v = rho2[base + xr];
    if (q >= 0) v = add2(v, zo[zb + xr]);
    v = add2(v, e2[((long long)r * G.ntx + txr) * 2 + 0]);
    if (q >= 0) v = add2(v, ze2[(zr * G.ntx + txr) * 2 + 0]);
    rho2[base + xr] = v;
    return;
  }
  if (bid < run_blocks + edge_blocks + row_blocks) {
    // 3: edge rows (y partials): thread per (z, tile row, bottom / top, x)
    const unsigned t = (unsigned)(bid - run_blocks - edge_blocks) * blockDim.x + threadIdx.x;
    const unsigned n = (unsigned)P.nz * G.nty * 2 * P.nx;
    if (t >= n) return;
    const unsigned qq = t / P.nx;
    const int x = (int)(t - qq * P.nx);
    const int sy = (int)(qq & 1u);
    const unsigned zt = qq >> 1;
    const int z = (int)(zt / G.nty), ty = (int)(zt - (unsigned)z * G.nty);
    const int q = zslot[z];
    if (q >= 0 && !G.zpart) return;  // runs
    const int y0 = ty * kOnePassRows, rows = min(kOnePassRows, P.ny - y0), y = sy ? y0 + rows - 1 : y0;
    const int tx = x / kOnePassCols, x0 = tx * kOnePassCols, nown = min(kOnePassCols, P.nx - x0);
    const int txl = tx == 0 ? G.ntx - 1 : tx - 1, txr = tx == G.ntx - 1 ? 0 : tx + 1;
    const int tyn = sy ? (ty == G.nty - 1 ? 0 : ty + 1) : (ty == 0 ? G.nty - 1 : ty - 1);  // the tile sending across
    const float2 *y2 = reinterpret_cast<const float2 *>(out.yedge);
    const float2 *zy = reinterpret_cast<const float2 *>(out.zyedge);
    const float2 *d2 = reinterpret_cast<const float2 *>(out.diag);
    const long long node = ((long long)z * P.ny + y) * P.nx + x;
    const long long ystride = (long long)G.ntx * kOnePassCols;
    float2 v = rho2[node];
    if (q >= 0) v = add2(v, zo[(long long)q * plane + (long long)y * P.nx + x]);
    // the bottom row gets what the tile below sends up (its side 1), the top row what the tile
    // above sends down (its side 0)
    v = add2(v, y2[(((long long)(1 - sy) * P.nz + z) * G.nty + tyn) * ystride + x]);
    if (q >= 0) v = add2(v, zy[(((long long)(1 - sy) * 2 * G.nchunks + q) * G.nty + tyn) * ystride + x]);
    const long long er = (long long)z * P.ny + y, zr = (long long)q * P.ny + y;
    if (x == x0) {  // corner: the left tile's side-1 sums of this row, the diagonal value
      v = add2(v, e2[(er * G.ntx + txl) * 2 + 1]);
      if (q >= 0) v = add2(v, ze2[(zr * G.ntx + txl) * 2 + 1]);
      v = add2(v, d2[(((long long)z * G.nty + tyn) * G.ntx + txl) * 4 + (sy ? 1 : 3)]);
    }
    if (x == x0 + nown - 1) {  // corner: the right tile's side-0 sums of this row, the diagonal value
      v = add2(v, e2[(er * G.ntx + txr) * 2 + 0]);
      if (q >= 0) v = add2(v, ze2[(zr * G.ntx + txr) * 2 + 0]);
      v = add2(v, d2[(((long long)z * G.nty + tyn) * G.ntx + txr) * 4 + (sy ? 0 : 2)]);
    }
    rho2[node] = v;
    return;
  }
  // 4: the other nodes of the chunk-edge planes (z partials): thread per (slot, y, x)
  const unsigned t = (unsigned)(bid - run_blocks - edge_blocks - row_blocks) * blockDim.x + threadIdx.x;
  const unsigned n = (unsigned)(2 * G.nchunks) * P.ny * P.nx;
  if (t >= n) return;
  const unsigned qy = t / P.nx;
  const int x = (int)(t - qy * P.nx);
  const int q = (int)(qy / P.ny), y = (int)(qy - (unsigned)q * P.ny);
  const int w = y % kOnePassRows, rows = min(kOnePassRows, P.ny - (y - w));
  if (w < 1 || w > rows - 2) return;  // tile edge rows: runs, or range 3
  const int xt = x % kOnePassCols, nown = min(kOnePassCols, P.nx - (x - xt));
  if (xt == 0 || xt == nown - 1) return;  // x edges: range 2
  // the plane of slot q: zs - 1 (q even) or zs (q odd) of chunk q / 2
  const int zs = (int)((long long)(q >> 1) * P.nz / G.nchunks);
  const int z = (q & 1) ? zs : (zs == 0 ? P.nz - 1 : zs - 1);
  const long long node = (long long)z * plane + (long long)y * P.nx + x;
  rho2[node] = add2(rho2[node], zo[(long long)q * plane + (long long)y * P.nx + x]);
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
// permutes populations, so sums over stored and post-streaming values agree), each node's sums
// formed as FloatPair (lb_site.cuh): five FP64 additions per node instead of about ninety.
constexpr int kSumBlock = 256;
template <class T>
__global__ void __launch_bounds__(kSumBlock) k_fluid_sums(StepParams P, const T *__restrict__ store,
                                                          const float *__restrict__ rest,
                                                          double *__restrict__ partial) {
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < P.N;
       s += (long long)gridDim.x * blockDim.x) {
    FloatPair m[5];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const float a = pop_read(P, store, rest, 0, i, s);
      const float b = pop_read(P, store, rest, 1, i, s);
      m[0].add(a);
      m[1].add(b);
      if (kCx[i]) { m[2].add(kCx[i] > 0 ? a : -a); m[2].add(kCx[i] > 0 ? b : -b); }
      if (kCy[i]) { m[3].add(kCy[i] > 0 ? a : -a); m[3].add(kCy[i] > 0 ? b : -b); }
      if (kCz[i]) { m[4].add(kCz[i] > 0 ? a : -a); m[4].add(kCz[i] > 0 ? b : -b); }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += m[k].value();
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
  // one warp per value: lane l adds the blocks l, l + 32, ... in order, then a fixed shuffle tree
  // (deterministic; 32 chains instead of one long chain of dependent FP64 additions)
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= nvals) return;  // warp-uniform
  double a = 0.0;
  for (int b = lane; b < nblocks; b += 32) a += partial[(long long)b * nvals + k];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
  if (lane == 0) out[k] = a;
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

void launch_collide_onepass(const StepParams &P, const void *fin, void *fout, float *rest, const float *rho,
                            float *rho_next, OnePassOut out, const ParticleArrays &pa, const ParticleForces &pf,
                            CellIndex ci, unsigned *err, OnePassGeom G, int grid, cudaStream_t st) {
  with_storage(P, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    const T *a = static_cast<const T *>(fin);
    T *b = static_cast<T *>(fout);
    if (P.np > 0)
      k_collide_onepass<T, true><<<grid, kOPThreads, 0, st>>>(P, a, b, rho, rho_next, out, pa, pf, ci, err, rest,
                                                              rest, G);
    else
      k_collide_onepass<T, false><<<grid, kOPThreads, 0, st>>>(P, a, b, rho, rho_next, out, pa, pf, ci, err, rest,
                                                               rest, G);
  });
}

void launch_boundary_densities(const StepParams &P, OnePassGeom G, const void *store, const float *rest,
                               float *rho_next, const BoundaryRun *runs, int nruns, OnePassOut out,
                               const int *zslot, const ParticleArrays &pn, int np, float4 *jc, cudaStream_t st) {
  const long long run_blocks = (nruns + kBlock / 32 - 1) / (kBlock / 32);
  const long long edge_blocks = ((long long)P.nz * P.ny * G.ntx + kBlock - 1) / kBlock;
  const long long row_blocks = G.ypart ? ((long long)P.nz * G.nty * 2 * P.nx + kBlock - 1) / kBlock : 0;
  const long long zplane_blocks = G.zpart ? ((long long)2 * G.nchunks * P.ny * P.nx + kBlock - 1) / kBlock : 0;
  if (!jc) np = 0;
  const long long corner_blocks = (8LL * np + kBlock - 1) / kBlock;
  const long long blocks = run_blocks + edge_blocks + row_blocks + zplane_blocks + corner_blocks;
  if (blocks <= 0) return;
  with_storage(P, [&](auto t) {
    using T = std::remove_pointer_t<decltype(t)>;
    k_boundary_densities<T><<<(unsigned)blocks, kBlock, 0, st>>>(
        P, G, static_cast<const T *>(store), rest, rho_next, runs, nruns, (int)corner_blocks, (int)run_blocks,
        (int)edge_blocks, (int)row_blocks, out, zslot, pn, np, jc);
  });
}

int onepass_blocks_per_sm() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_collide_onepass<float, true>, kOPThreads, 0) !=
          cudaSuccess ||
      b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return b;
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
  k_finish_sums<<<1, 32 * nvals, 0, st>>>(partial, nblocks, nvals, out);
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
