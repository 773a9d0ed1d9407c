// lb_site.cuh -- the arithmetic of one lattice site and of one particle in a coupled step,
// shared by the kernels of a single lattice (lb_fluid.cu, lb_particles.cu) and the batched
// kernels that advance many independent lattices in one launch (lb_batch.cu).  A kernel
// decides which site or particle a thread owns and which lattice's parameters apply; the
// bodies below do the rest, so a lattice gives the same bits whichever kernel ran it.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>
#include <type_traits>

#include "lb_modes.h"
#include "lbmd_internal.cuh"

namespace lbmd {
namespace site {

// Read / write of one population value by the element-wise kernels (initialisation, exchange
// with the host, fields, sums); `shift` = w_i rho0_z (ignored for FP32 storage).  enc / dec
// convert between the FP32 value and the stored element.  The update and the density pass load
// and store whole (A, B) words instead (Pair16 below for 16-bit storage).
template <class T>
struct Pop;
// 16-bit storage keeps the rest populations apart, in FP32; FP32 storage has none
template <class T>
constexpr bool kSplitRest = !std::is_same<T, float>::value;
template <>
struct Pop<float> {
  static __device__ __forceinline__ float enc(float v, float) { return v; }
  static __device__ __forceinline__ float dec(float e, float) { return e; }
  static __device__ __forceinline__ float rd(const float *p, float) { return *p; }
  static __device__ __forceinline__ void st(float *p, float v, float) { *p = v; }
};
template <>
struct Pop<__half> {
  static __device__ __forceinline__ __half enc(float v, float sh) { return __float2half_rn(v - sh); }
  static __device__ __forceinline__ float dec(__half e, float sh) { return __half2float(e) + sh; }
  static __device__ __forceinline__ float rd(const __half *p, float sh) { return dec(*p, sh); }
  static __device__ __forceinline__ void st(__half *p, float v, float sh) { *p = enc(v, sh); }
};
template <>
struct Pop<__nv_bfloat16> {
  static __device__ __forceinline__ __nv_bfloat16 enc(float v, float sh) { return __float2bfloat16_rn(v - sh); }
  static __device__ __forceinline__ float dec(__nv_bfloat16 e, float sh) { return __bfloat162float(e) + sh; }
  static __device__ __forceinline__ float rd(const __nv_bfloat16 *p, float sh) { return dec(*p, sh); }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v, float sh) { *p = enc(v, sh); }
};

// 16-bit storage holds both components' values of a direction at a node in one 32-bit word,
// A in the low half: dec gives (A, B) as floats, enc rounds an (A, B) pair into a word.
template <class T>
struct Pair16;
template <>
struct Pair16<__half> {
  static __device__ __forceinline__ float2 dec(unsigned w) {
    __half2 h;
    memcpy(&h, &w, 4);
    return __half22float2(h);
  }
  static __device__ __forceinline__ unsigned enc(float2 v) {
    const __half2 h = __floats2half2_rn(v.x, v.y);
    unsigned w;
    memcpy(&w, &h, 4);
    return w;
  }
  // acc += dec(w), each lane one mixed-precision addition (the 16-bit operand converts exactly)
  static __device__ __forceinline__ void add_to(unsigned w, float2 &acc) {
    const unsigned short lo = (unsigned short)(w & 0xffffu), hi = (unsigned short)(w >> 16);
    asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(acc.x) : "h"(lo));
    asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(acc.y) : "h"(hi));
  }
};
template <>
struct Pair16<__nv_bfloat16> {
  static __device__ __forceinline__ float2 dec(unsigned w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
  }
  static __device__ __forceinline__ unsigned enc(float2 v) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    unsigned w;
    memcpy(&w, &h, 4);
    return w;
  }
  static __device__ __forceinline__ void add_to(unsigned w, float2 &acc) {
    const unsigned short lo = (unsigned short)(w & 0xffffu), hi = (unsigned short)(w >> 16);
    asm("add.rn.f32.bf16 %0, %1, %0;" : "+f"(acc.x) : "h"(lo));
    asm("add.rn.f32.bf16 %0, %1, %0;" : "+f"(acc.y) : "h"(hi));
  }
};

__device__ __forceinline__ float pop_shift(const StepParams &P, int comp, int i) { return kW[i] * P.rho0[comp]; }

// A sum of FP32 values without rounding error: kept as an unevaluated pair (hi, lo) of FP32
// numbers, each addition split by Knuth's error-free two-sum (s + e == hi + x exactly; plain FP32
// additions, nothing the compiler may contract).  FP64 arithmetic is slow on this GPU, so the FP64
// reductions form each node's sums this way and add only the node totals, hi + lo, in FP64.  The
// pair holds about 48 significant bits: a node total of a few dozen values carries a relative error
// of ~2^-47 at most.
struct FloatPair {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Element index of direction i of component c at site s: [19][N][2], the (A, B) pair of a
// direction at a node side by side (one 8-byte word in FP32, one 4-byte word in 16 bits).
template <class T>
__device__ __forceinline__ long long pop_elem(const StepParams &P, int c, int i, long long s) {
  return ((long long)i * P.N + s) * 2 + c;
}

// Sum of the shifts of the 18 moving populations of component comp, (1 - w_0) rho0: the density
// of a 16-bit node is f_0 + (its 18 stored values) + this.  The update and the mass closure use
// this same FP32 value, so that rounding it moves no mass from step to step.
__device__ __forceinline__ float shift_sum(const StepParams &P, int comp) { return (1.f - kW[0]) * P.rho0[comp]; }

// With 16-bit storage the rest population f_0 (which does not stream) is kept in an FP32 array
// rest[2][N]; these read / write direction i of component c at site s from the right place.
template <class T>
__device__ __forceinline__ float pop_read(const StepParams &P, const T *buf, const float *rest, int c, int i,
                                          long long s) {
  if (i == 0 && rest) return rest[(long long)c * P.N + s];
  return Pop<T>::rd(buf + pop_elem<T>(P, c, i, s), kW[i] * P.rho0[c]);
}
template <class T>
__device__ __forceinline__ void pop_write(const StepParams &P, T *buf, float *rest, int c, int i, long long s,
                                          float v) {
  if (i == 0 && rest)
    rest[(long long)c * P.N + s] = v;
  else
    Pop<T>::st(buf + pop_elem<T>(P, c, i, s), v, kW[i] * P.rho0[c]);
}

struct Coord {
  int x, y, z;
};

// (x, y, z) of site s = (z ny + y) nx + x; s < 2^32 (19 N < 2^32 is enforced)
__device__ __forceinline__ Coord site_coord(const StepParams &P, long long s) {
  const uint32_t s32 = (uint32_t)s;
  const uint32_t t = fast_div(s32, P.divx);  // z ny + y
  const uint32_t z = fast_div(t, P.divy);
  Coord c;
  c.x = (int)(s32 - t * (uint32_t)P.nx);
  c.y = (int)(t - z * (uint32_t)P.ny);
  c.z = (int)z;
  return c;
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

// source coordinate of direction i for a pull at (x, y, z): r - c_i, periodic
__device__ __forceinline__ long long pull_source(const StepParams &P, int i, const int xs[3], const int ys[3],
                                                 const int zs[3]) {
  // xs = {x-1, x, x+1} wrapped; r - c_i selects index 1 - c
  return ((long long)zs[1 - kCz[i]] * P.ny + ys[1 - kCy[i]]) * P.nx + xs[1 - kCx[i]];
}

// Periodic neighbour offsets of site s: m[a] is the offset to coordinate a - 1, p[a] to a + 1
// (wrap-aware), so the site r + c is s + shift(o, c) in 32-bit arithmetic (19 N < 2^32 is
// enforced when a lattice is created).
struct NOff {
  int m[3], p[3];
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

// Densities rho_z = sum_i f_zi (appendix, zeroth mode) of site s, stored interleaved
// (rho_A, rho_B), and j' = sum_z sum_i f_zi c_i (written when jp is not NULL).
template <class T>
__device__ __forceinline__ void moments(const StepParams &P, long long s, const T *__restrict__ fin,
                                        const float *__restrict__ rest, float *__restrict__ rho,
                                        float *__restrict__ jp) {
  const Coord c = site_coord(P, s);
  const NOff o = neighbour_offsets(P, c);
  const unsigned N32 = (unsigned)P.N, s32 = (unsigned)s;
  // 16-bit storage: the moving populations are summed as stored (shifted) and the shifts added
  // once; the shifts cancel in j' (sum_i w_i c_i = 0)
  constexpr bool kShifted = kSplitRest<T>;
  float rA = 0.f, rB = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
  if constexpr (kShifted) {
    // one 32-bit word per direction holds the (A, B) pair; all 18 loads are issued before any is
    // used, so that enough bytes are in flight per thread
    const unsigned *win = reinterpret_cast<const unsigned *>(fin);
    unsigned w[kQ];
#pragma unroll
    for (int i = 1; i < kQ; ++i)
      w[i] = __ldg(win + i * N32 + (unsigned)((int)s32 + shift(o, -kCx[i], -kCy[i], -kCz[i])));  // r - c_i
    rA = __ldg(rest + s32);
    rB = __ldg(rest + N32 + s32);
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
      const float2 v = Pair16<T>::dec(w[i]);
      rA += v.x;
      rB += v.y;
      jx += kCx[i] * (v.x + v.y);
      jy += kCy[i] * (v.x + v.y);
      jz += kCz[i] * (v.x + v.y);
    }
  } else {
    const float2 *fin2 = reinterpret_cast<const float2 *>(fin);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const float2 v = __ldg(fin2 + i * N32 + (unsigned)((int)s32 + shift(o, -kCx[i], -kCy[i], -kCz[i])));  // r - c_i
      rA += v.x;
      rB += v.y;
      jx += kCx[i] * (v.x + v.y);
      jy += kCy[i] * (v.x + v.y);
      jz += kCz[i] * (v.x + v.y);
    }
  }
  if (kShifted) {
    rA += shift_sum(P, 0);
    rB += shift_sum(P, 1);
  }
  reinterpret_cast<float2 *>(rho)[s] = make_float2(rA, rB);
  if (jp) {
    jp[s] = jx;
    jp[P.N + s] = jy;
    jp[2 * P.N + s] = jz;
  }
}

// Fluid-side solvation force (Eq. solvation_lambda) and momentum return (Sec. 2) gathered at
// node (x, y, z) from the particles of the 8 unit cells having that node as a corner.
// ci.row_start is indexed by this lattice's row (z * ny + y); pa, pf by the sorted slot.  The
// cell's w holds the particle type in its low byte and, for the reaction records of MD
// sub-stepping, the substep index above it.  A row is sorted by x cell; with kBisect the
// node's two cells are found in it by bisection (the K records per particle of sub-stepping
// make rows of hundreds of entries), otherwise the row is scanned once (short rows: the
// plain scan keeps the update's register budget).
template <bool kBisect = false>
__device__ __forceinline__ void gather_coupling(const StepParams &P, int x, int y, int z, float rA, float rB,
                                                const ParticleArrays &pa, const ParticleForces &pf,
                                                CellIndex ci, bool with_momentum, float3 &gA, float3 &gB) {
  const float rinv = 1.f / (rA + rB);
  const float sA = rA * rinv, sB = rB * rinv;
  // one particle (or reaction record) q in the cell whose corner offset from it is (ox, oy, oz)
  auto add = [&](int q, int ox, int oy, int oz, int w) {
    const float4 fr = __ldg(pa.frac + q);
    const TypeParams &T = P.types[w & 0xff];
    const float dx = fr.x - ox, dy = fr.y - oy, dz = fr.z - oz;
    // entries of later particle substeps (w >> 8 > 0) carry momentum only: the fluid-side
    // solvation force comes from the positions at the start of the step
    if ((w >> 8) == 0 && (T.lam[0] != 0.f || T.lam[1] != 0.f)) {
      const float3 geo = fs_geometry(dx, dy, dz);
      const float a = -T.lam[0] * rA, b = -T.lam[1] * rB;
      gA.x += a * geo.x; gA.y += a * geo.y; gA.z += a * geo.z;
      gB.x += b * geo.x; gB.y += b * geo.y; gB.z += b * geo.z;
    }
    if (with_momentum) {
      const float wt = (ox ? fr.x : 1.f - fr.x) * (oy ? fr.y : 1.f - fr.y) * (oz ? fr.z : 1.f - fr.z);
      const float4 ff = __ldg(pf.fric + q), pA = __ldg(pf.psA + q), pB = __ldg(pf.psB + q);
      gA.x += wt * (-sA * ff.x - pA.x); gA.y += wt * (-sA * ff.y - pA.y); gA.z += wt * (-sA * ff.z - pA.z);
      gB.x += wt * (-sB * ff.x - pB.x); gB.y += wt * (-sB * ff.y - pB.y); gB.z += wt * (-sB * ff.z - pB.z);
    }
  };
#pragma unroll
  for (int oz = 0; oz < 2; ++oz) {
    const int cz = oz ? (z == 0 ? P.nz - 1 : z - 1) : z;
#pragma unroll
    for (int oy = 0; oy < 2; ++oy) {
      const int cy = oy ? (y == 0 ? P.ny - 1 : y - 1) : y;
      const int row = cz * P.ny + cy;
      const int q0 = __ldg(ci.row_start + row), q1 = __ldg(ci.row_start + row + 1);
      if (kBisect) {
        if (q0 == q1) continue;
        for (int ox = 0; ox < 2; ++ox) {
          const int cx = ox ? (x == 0 ? P.nx - 1 : x - 1) : x;
          int lo = q0, hi = q1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(&pa.cell[mid].x) < cx)
              lo = mid + 1;
            else
              hi = mid;
          }
          for (int q = lo; q < q1; ++q) {
            const int4 c = __ldg(pa.cell + q);
            if (c.x != cx) break;
            add(q, ox, oy, oz, c.w);
          }
        }
      } else {
        for (int q = q0; q < q1; ++q) {
          const int4 c = __ldg(pa.cell + q);
#pragma unroll
          for (int ox = 0; ox < 2; ++ox) {
            const int cx = ox ? (x == 0 ? P.nx - 1 : x - 1) : x;
            if (c.x == cx) add(q, ox, oy, oz, c.w);
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------ fluctuating MRT

// Unit normals 4k .. 4k+3 of the fluid noise at one site and step: Philox4x32-10 (Salmon et
// al., SC'11) with counter (site, step low, step high, 0x464c0000 + k) and key = seed (its round
// keys formed once, StepParams::noise_keys), uniforms from the top 24 bits, Box-Muller on both
// uniform pairs.  The logarithm and the sine / cosine
// are the hardware approximations (absolute error ~1e-6 on a normal, far below what the
// populations can resolve), and so is the radius: x rsqrt(x), a few ulp from sqrt(x); the
// generator's integer stream is exact.  A uniform (v + 1/2) 2^-24 is one FFMA: the scaling by a
// power of two is exact, so one rounding of v 2^-24 + 2^-25 gives the same float.
__device__ __forceinline__ float4 fluid_normals4(const uint2 *__restrict__ keys, unsigned long long step,
                                                 unsigned site, unsigned k) {
  const uint4 r = philox4x32_10_keyed(make_uint4(site, (unsigned)step, (unsigned)(step >> 32), 0x464c0000u + k),
                                      keys);
  // the two Box-Muller pairs side by side: (u0, u2) give the radii, (u1, u3) the angles
  const float2 sc = make_float2(1.f / 16777216.f, 1.f / 16777216.f);
  const float2 h = make_float2(0.5f / 16777216.f, 0.5f / 16777216.f);
  const float2 ur = __ffma2_rn(make_float2((float)(r.x >> 8), (float)(r.z >> 8)), sc, h);
  const float2 ua = __ffma2_rn(make_float2((float)(r.y >> 8), (float)(r.w >> 8)), sc, h);
  // u0 = 1 (v = 2^24 - 1 rounds up) gives x = 0: the floor keeps 0 * rsqrt from being NaN
  const float2 x = __fmul2_rn(make_float2(-2.f, -2.f), make_float2(__logf(ur.x), __logf(ur.y)));
  const float2 rad = __fmul2_rn(x, make_float2(rsqrtf(fmaxf(x.x, 1e-30f)), rsqrtf(fmaxf(x.y, 1e-30f))));
  const float two_pi = 6.28318530717958647692f;
  const float2 ang = __fmul2_rn(make_float2(two_pi, two_pi), ua);
  float s1, c1, s3, c3;
  __sincosf(ang.x, &s1, &c1);
  __sincosf(ang.y, &s3, &c3);
  const float2 n01 = __fmul2_rn(make_float2(rad.x, rad.x), make_float2(c1, s1));
  const float2 n23 = __fmul2_rn(make_float2(rad.y, rad.y), make_float2(c3, s3));
  return make_float4(n01.x, n01.y, n23.x, n23.y);
}

// Eq. MODES, per component: modes m_k = sum_i e_k(c_i) f_i (lb_modes.h), each relaxed toward its
// equilibrium value with factor 1 + lambda_k, plus the moment of the forcing term and the noise;
// back to populations f_i = w_i sum_k e_k(c_i) m_k / b_k.  The equilibrium moments of
// f^eq(rho_z, u) are rho_z u (momentum), rho_z u u (stress), 0 (kinetic); those of the forcing
// term are (2 + lambda_M)/2 g, and G for the stress (appendix), 0 for the kinetic modes.
// Directions come in opposite pairs (2p + 1, 2p + 2) and every e_k is even or odd in c, so both
// transforms work on the pair sums and differences: half the arithmetic of the plain sums.
__device__ __host__ constexpr bool mode_even(int k) { return k == 0 || (k >= 4 && k <= 9) || k >= 16; }

// The collision of both components with the fluctuating MRT operator (Eq. MODES), the two
// components' arithmetic run together on (A, B) pairs with the packed two-lane FP32
// instructions.  With noise: the three momentum normals are shared by A (+) and B (-), amplitude
// over sqrt(rho_A rho_B / rho); the stress and kinetic modes take normals 3-17 (A) and 18-32 (B)
// of the site's 36.  Each normal is added to its relaxed mode as it is drawn, so that no
// component's noise is held whole.
__device__ __forceinline__ void mrt_update(const StepParams &P, unsigned long long step, unsigned site,
                                           float fA[kQ], float fB[kQ], float rA, float rB, float ux, float uy,
                                           float uz, float3 gA, float3 gB) {
  constexpr int kPairs = (kQ - 1) / 2;
  // modes m_k = sum_i e_k(c_i) f_i of both components, from the pair sums and differences
  float2 m[kQ];
  {
    float2 sp[kPairs], dp[kPairs];
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
      const float2 u = make_float2(fA[2 * p + 1], fB[2 * p + 1]), v = make_float2(fA[2 * p + 2], fB[2 * p + 2]);
      sp[p] = __fadd2_rn(u, v);
      dp[p] = __fadd2_rn(u, make_float2(-v.x, -v.y));
    }
    const float2 f0 = make_float2(fA[0], fB[0]);
#pragma unroll
    for (int k = 0; k < kQ; ++k) {
      const float e0 = (float)mode_poly(k, 0, 0, 0);
      float2 a = mode_even(k) ? make_float2(e0 * f0.x, e0 * f0.y) : make_float2(0.f, 0.f);
#pragma unroll
      for (int p = 0; p < kPairs; ++p) {
        const int i = 2 * p + 1;
        const int e = mode_poly(k, kCx[i], kCy[i], kCz[i]);
        const float2 v = mode_even(k) ? sp[p] : dp[p];
        if (e == 1)
          a = __fadd2_rn(a, v);
        else if (e == -1)
          a = __fadd2_rn(a, make_float2(-v.x, -v.y));
        else if (e != 0)
          a = __ffma2_rn(make_float2((float)e, (float)e), v, a);
      }
      m[k] = a;
    }
  }
  // equilibrium moments rho_z (u, u u) and the forcing term's moments of each component; relaxed
  const float uu = ux * ux + uy * uy + uz * uz;
  const float2 rz = make_float2(rA, rB);
  const float2 gx = make_float2(gA.x, gB.x), gy = make_float2(gA.y, gB.y), gz = make_float2(gA.z, gB.z);
  const float2 ug = make_float2(ux * gA.x + uy * gA.y + uz * gA.z, ux * gB.x + uy * gB.y + uz * gB.z);
  // scaling, sum and difference of (A, B) pairs (packed: the compiler does not pair scalar ones)
  auto sc = [](float a, float2 v) { return __fmul2_rn(make_float2(a, a), v); };
  auto ad = [](float2 a, float2 b) { return __fadd2_rn(a, b); };
  auto sb = [](float2 a, float2 b) { return __ffma2_rn(make_float2(-1.f, -1.f), b, a); };
  const float2 meq[10] = {rz,
                          sc(ux, rz),
                          sc(uy, rz),
                          sc(uz, rz),
                          sc(uu, rz),
                          sc(3.f * ux * ux - uu, rz),
                          sc(uy * uy - uz * uz, rz),
                          sc(ux * uy, rz),
                          sc(uy * uz, rz),
                          sc(uz * ux, rz)};
  const float2 mg[10] = {make_float2(0.f, 0.f),
                         sc(P.force[1], gx),
                         sc(P.force[2], gy),
                         sc(P.force[3], gz),
                         sc(P.force[4], ug),
                         sc(P.force[5], sb(sc(3.f * ux, gx), ug)),
                         sc(P.force[6], sb(sc(uy, gy), sc(uz, gz))),
                         sc(P.force[7], ad(sc(ux, gy), sc(uy, gx))),
                         sc(P.force[8], ad(sc(uy, gz), sc(uz, gy))),
                         sc(P.force[9], ad(sc(uz, gx), sc(ux, gz)))};
#pragma unroll
  for (int k = 1; k < kQ; ++k) {
    if (k < 10)
      m[k] = ad(__ffma2_rn(make_float2(P.relax[k], P.relax[k]), sb(m[k], meq[k]), meq[k]), mg[k]);
    else
      m[k] = sc(P.relax[k], m[k]);
  }
  if (P.fluct) {
    // sqrt(rho_A), sqrt(rho_B) and sqrt(rho_A rho_B / rho) from reciprocal square roots, as the
    // Box-Muller radius (a density of 0 gives 0)
    const float sA = rA * rsqrtf(fmaxf(rA, 1e-30f)), sB = rB * rsqrtf(fmaxf(rB, 1e-30f));
    const float am = P.noise[1] * sA * sB * rsqrtf(rA + rB);
    // A: normals 0-3 (momentum, shared; then mode 4), 4-15 (modes 5-16), 16, 17 (modes 17, 18)
    float4 q = fluid_normals4(P.noise_keys, step, site, 0);
    const float2 amAB = make_float2(am, -am);
    m[1] = __ffma2_rn(amAB, make_float2(q.x, q.x), m[1]);
    m[2] = __ffma2_rn(amAB, make_float2(q.y, q.y), m[2]);
    m[3] = __ffma2_rn(amAB, make_float2(q.z, q.z), m[3]);
    m[4].x += P.noise[4] * sA * q.w;
#pragma unroll
    for (int c = 1; c <= 3; ++c) {
      q = fluid_normals4(P.noise_keys, step, site, c);
      const int k = 4 * c + 1;
      m[k].x += P.noise[k] * sA * q.x;
      m[k + 1].x += P.noise[k + 1] * sA * q.y;
      m[k + 2].x += P.noise[k + 2] * sA * q.z;
      m[k + 3].x += P.noise[k + 3] * sA * q.w;
    }
    q = fluid_normals4(P.noise_keys, step, site, 4);
    m[17].x += P.noise[17] * sA * q.x;
    m[18].x += P.noise[18] * sA * q.y;
    // B: modes 4, 5 from the last two of that draw, then 6-18
    m[4].y += P.noise[4] * sB * q.z;
    m[5].y += P.noise[5] * sB * q.w;
#pragma unroll
    for (int c = 5; c <= 7; ++c) {
      q = fluid_normals4(P.noise_keys, step, site, c);
      const int k = 4 * c - 14;
      m[k].y += P.noise[k] * sB * q.x;
      m[k + 1].y += P.noise[k + 1] * sB * q.y;
      m[k + 2].y += P.noise[k + 2] * sB * q.z;
      m[k + 3].y += P.noise[k + 3] * sB * q.w;
    }
    q = fluid_normals4(P.noise_keys, step, site, 8);
    m[18].y += P.noise[18] * sB * q.x;
  }
  // scaled by 1 / b_k for the way back
#pragma unroll
  for (int k = 0; k < kQ; ++k) m[k] = sc(9.f / (float)mode_norm9(k), m[k]);
  // moving populations from the modes; the rest population takes what the node's density
  // (unchanged by the collision) leaves, so that the FP32 weights, whose sum is not exactly 1,
  // do not bias the mass every step
  float2 moving = make_float2(0.f, 0.f);
#pragma unroll
  for (int p = 0; p < kPairs; ++p) {
    const int i = 2 * p + 1;
    float2 even = make_float2(0.f, 0.f), odd = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kQ; ++k) {
      const int e = mode_poly(k, kCx[i], kCy[i], kCz[i]);
      if (e == 0) continue;
      if (mode_even(k))
        even = __ffma2_rn(make_float2((float)e, (float)e), m[k], even);
      else
        odd = __ffma2_rn(make_float2((float)e, (float)e), m[k], odd);
    }
    const float2 fi = sc(kW[i], ad(even, odd)), fj = sc(kW[i], sb(even, odd));
    fA[i] = fi.x;
    fB[i] = fi.y;
    fA[i + 1] = fj.x;
    fB[i + 1] = fj.y;
    moving = ad(moving, ad(fi, fj));
  }
  fA[0] = rA - moving.x;
  fB[0] = rB - moving.y;
}

// Where the update reads the densities of its Shan-Chen stencil: from the density field in global
// memory (GlobalRho, the default), or from a copy a block staged in shared memory (a type with
// kStaged = true whose call operator gives the (rho_A, rho_B) pair at offset (cx, cy, cz)).
struct GlobalRho {
  static constexpr bool kStaged = false;
  __device__ float2 operator()(int, int, int) const { return make_float2(0.f, 0.f); }
};

// The lattice update of one step at site s, up to the store: pull, densities and momentum,
// Shan-Chen force (Eq. SCforce with psi = rho, g_AA = g_BB = 0), fluid-side solvation force and
// momentum return from the particles (Sec. 2), barycentric velocity (Eq. momentum_definition),
// collision with forcing for both components (BGK, or with kMRT the fluctuating MRT of Eq.
// MODES, `step` being the noise counter).  On return fA, fB hold the post-collision values
// (16-bit storage with BGK: the moving ones shifted by w_i rho0, as stored) and rA, rB the node's
// densities before the collision.
template <class T, bool kParticles, bool kMRT = false, bool kBisect = false, class Rho = GlobalRho>
__device__ __forceinline__ void collide_core_at(const StepParams &P, const Coord c, long long s,
                                                unsigned long long step, const T *__restrict__ fin,
                                                const float *__restrict__ rho, const ParticleArrays &pa,
                                                const ParticleForces &pf, CellIndex ci, unsigned *err,
                                                const float *__restrict__ rest_in, float (&fA)[kQ],
                                                float (&fB)[kQ], float &rA_out, float &rB_out,
                                                const Rho &staged = Rho{}) {
  const NOff o = neighbour_offsets(P, c);
  const unsigned N32 = (unsigned)P.N, s32 = (unsigned)s;
  // 16-bit storage with the BGK update: the moving populations stay shifted (f - w_i rho0, as
  // stored) through the update, the shifts folded into its constants, and the FP32 rest
  // population closes the node's mass
  constexpr bool kShifted = kSplitRest<T> && !kMRT;
  if constexpr (kSplitRest<T>) {
    // 16-bit storage: one 32-bit word per direction holds the (A, B) pair; the rest populations
    // are kept in FP32
    const unsigned *win = reinterpret_cast<const unsigned *>(fin);
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
      const unsigned src = i * N32 + (unsigned)((int)s32 + shift(o, -kCx[i], -kCy[i], -kCz[i]));  // pull r - c_i
      const float2 v = Pair16<T>::dec(__ldg(win + src));
      fA[i] = kShifted ? v.x : v.x + pop_shift(P, 0, i);
      fB[i] = kShifted ? v.y : v.y + pop_shift(P, 1, i);
    }
    fA[0] = __ldg(rest_in + s32);
    fB[0] = __ldg(rest_in + N32 + s32);
  } else {
    // FP32 storage: one 8-byte word per direction holds the (A, B) pair
    const float2 *fin2 = reinterpret_cast<const float2 *>(fin);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const float2 v = __ldg(fin2 + i * N32 + (unsigned)((int)s32 + shift(o, -kCx[i], -kCy[i], -kCz[i])));  // pull r - c_i
      fA[i] = v.x;
      fB[i] = v.y;
    }
  }
  // The two components go through the same arithmetic: it runs on (A, B) pairs with the
  // packed two-lane FP32 instructions.  Directions come in opposite pairs (2p + 1, 2p + 2): the
  // densities sum the pair sums, the momenta the pair differences (c_{2p+2} = -c_{2p+1}).
  float2 r2s = make_float2(fA[0], fB[0]);
  float2 jx2 = make_float2(0.f, 0.f), jy2 = jx2, jz2 = jx2;
#pragma unroll
  for (int i = 1; i < kQ; i += 2) {
    const float2 a = make_float2(fA[i], fB[i]), b = make_float2(fA[i + 1], fB[i + 1]);
    r2s = __fadd2_rn(r2s, __fadd2_rn(a, b));
    const float2 d = __fadd2_rn(a, make_float2(-b.x, -b.y));
    if (kCx[i] > 0) jx2 = __fadd2_rn(jx2, d);
    if (kCx[i] < 0) jx2 = __fadd2_rn(jx2, make_float2(-d.x, -d.y));
    if (kCy[i] > 0) jy2 = __fadd2_rn(jy2, d);
    if (kCy[i] < 0) jy2 = __fadd2_rn(jy2, make_float2(-d.x, -d.y));
    if (kCz[i] > 0) jz2 = __fadd2_rn(jz2, d);
    if (kCz[i] < 0) jz2 = __fadd2_rn(jz2, make_float2(-d.x, -d.y));
  }
  const float jx = jx2.x + jx2.y, jy = jy2.x + jy2.y, jz = jz2.x + jz2.y;
  if (kShifted) r2s = __fadd2_rn(r2s, make_float2(shift_sum(P, 0), shift_sum(P, 1)));
  const float rA = r2s.x, rB = r2s.y;
  // S_z = sum_i w_i rho_z(r + c_i) c_i from the density field of this step, as (S_A, S_B) pairs,
  // summed over opposite directions as w_i c_i (rho(r + c_i) - rho(r - c_i)): a profile uniform
  // along an axis gives exactly no force along it
  const float2 *rho2 = reinterpret_cast<const float2 *>(rho);
  float2 Sx = make_float2(0.f, 0.f), Sy = Sx, Sz = Sx;
#pragma unroll
  for (int i = 1; i < kQ; i += 2) {
    float2 rp, rm;
    if constexpr (Rho::kStaged) {
      rp = staged(kCx[i], kCy[i], kCz[i]);
      rm = staged(-kCx[i], -kCy[i], -kCz[i]);
    } else {
      rp = __ldg(rho2 + (unsigned)((int)s32 + shift(o, kCx[i], kCy[i], kCz[i])));
      rm = __ldg(rho2 + (unsigned)((int)s32 + shift(o, -kCx[i], -kCy[i], -kCz[i])));
    }
    const float2 d = __ffma2_rn(make_float2(-1.f, -1.f), rm, rp);
    if (kCx[i]) Sx = __ffma2_rn(make_float2(kW[i] * kCx[i], kW[i] * kCx[i]), d, Sx);
    if (kCy[i]) Sy = __ffma2_rn(make_float2(kW[i] * kCy[i], kW[i] * kCy[i]), d, Sy);
    if (kCz[i]) Sz = __ffma2_rn(make_float2(kW[i] * kCz[i], kW[i] * kCz[i]), d, Sz);
  }
  // g^SC_A = -g_AB rho_A S_B, g^SC_B = -g_BA rho_B S_A
  const float2 gpre = make_float2(-P.gAB * rA, -P.gBA * rB);
  const float2 gx = __fmul2_rn(gpre, make_float2(Sx.y, Sx.x));
  const float2 gy = __fmul2_rn(gpre, make_float2(Sy.y, Sy.x));
  const float2 gz = __fmul2_rn(gpre, make_float2(Sz.y, Sz.x));
  float3 gA = make_float3(gx.x, gy.x, gz.x);
  float3 gB = make_float3(gx.y, gy.y, gz.y);
  if (kParticles) gather_coupling<kBisect>(P, c.x, c.y, c.z, rA, rB, pa, pf, ci, true, gA, gB);
  const float r = rA + rB;
  if (!(rA > 0.f) || !(rB > 0.f) || !isfinite(r)) atomicOr(err, isfinite(r) ? kErrNegDensity : kErrNonFinite);
  const float rinv = 1.f / r;
  const float ux = (jx + 0.5f * (gA.x + gB.x)) * rinv;
  const float uy = (jy + 0.5f * (gA.y + gB.y)) * rinv;
  const float uz = (jz + 0.5f * (gA.z + gB.z)) * rinv;
  if (kMRT) {
    mrt_update(P, step, s32, fA, fB, rA, rB, ux, uy, uz, gA, gB);
  } else {
    // BGK + forcing, f* = (1 - 1/tau) f + (1/tau) f^eq + Delta^g, per pair of opposite directions
    // (c_j = -c_i), with f^eq and Delta^g split into parts even and odd in c.  Per component, with
    // cu = c_i.u and cg = c_i.g_z:
    //   f*_i = om1 f_i + even + odd,   f*_j = om1 f_j + even - odd,
    //   even = w_i E + 4.5 w_i om rho cu^2 + 9 w_i fp cu cg,   odd = 3 w_i om rho cu + 3 w_i fp cg,
    //   E = om rho (1 - 1.5 u^2) - 3 fp u.g_z   (less om rho0 with shifted storage),
    // and the rest population f*_0 = om1 f_0 + w_0 E.  The node-wide factors w E, 4.5 w om rho and
    // 3 w om rho are formed once for each weight of the moving directions (1/18 axis, 1/36
    // diagonal).
    const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float om = P.inv_tau, om1 = 1.f - om, fp = P.force_pref;
    const float2 gx = make_float2(gA.x, gB.x), gy = make_float2(gA.y, gB.y), gz = make_float2(gA.z, gB.z);
    // 3 u.g_z and om rho_z as (A, B) pairs
    const float2 ug3 = __fmul2_rn(make_float2(3.f, 3.f),
                                  __ffma2_rn(make_float2(uz, uz), gz,
                                             __ffma2_rn(make_float2(uy, uy), gy, __fmul2_rn(make_float2(ux, ux), gx))));
    const float2 a2 = __fmul2_rn(make_float2(om, om), make_float2(rA, rB));
    const float2 om1_2 = make_float2(om1, om1);
    float2 E = __ffma2_rn(a2, make_float2(1.f - usq15, 1.f - usq15), __fmul2_rn(make_float2(-fp, -fp), ug3));
    if (!kShifted) {  // (with 16-bit storage the rest population is set by the mass closure)
      const float2 f0 = __ffma2_rn(om1_2, make_float2(fA[0], fB[0]), __fmul2_rn(make_float2(kW[0], kW[0]), E));
      fA[0] = f0.x;
      fB[0] = f0.y;
    } else {
      // shifted storage: f~* = (1 - om) f~ + om (f^eq - w_i rho0) + Delta^g
      E = __ffma2_rn(make_float2(-om, -om), make_float2(P.rho0[0], P.rho0[1]), E);
    }
    constexpr float wa = kW[1], wd = kW[7];  // axis, diagonal
    const float2 Ea = __fmul2_rn(make_float2(wa, wa), E), Ed = __fmul2_rn(make_float2(wd, wd), E);
    const float2 Qa = __fmul2_rn(make_float2(4.5f * wa, 4.5f * wa), a2), Qd = __fmul2_rn(make_float2(4.5f * wd, 4.5f * wd), a2);
    const float2 Ra = __fmul2_rn(make_float2(3.f * wa, 3.f * wa), a2), Rd = __fmul2_rn(make_float2(3.f * wd, 3.f * wd), a2);
    const float fp9a = (9.f * wa) * fp, fp9d = (9.f * wd) * fp, fp3a = (3.f * wa) * fp, fp3d = (3.f * wd) * fp;
#pragma unroll
    for (int i = 1; i < kQ; i += 2) {
      const int j = i + 1;
      const bool axis = i < 7;  // directions 1-6 move along an axis
      const float2 Ew = axis ? Ea : Ed, Qw = axis ? Qa : Qd, Rw = axis ? Ra : Rd;
      const float fp9 = axis ? fp9a : fp9d, fp3 = axis ? fp3a : fp3d;
      const float cu = kCx[i] * ux + kCy[i] * uy + kCz[i] * uz;
      // c_i . g_z for both components (each c component is -1, 0 or 1)
      float2 cg = make_float2(0.f, 0.f);
      if (kCx[i]) cg = __ffma2_rn(make_float2((float)kCx[i], (float)kCx[i]), gx, cg);
      if (kCy[i]) cg = __ffma2_rn(make_float2((float)kCy[i], (float)kCy[i]), gy, cg);
      if (kCz[i]) cg = __ffma2_rn(make_float2((float)kCz[i], (float)kCz[i]), gz, cg);
      const float c9 = fp9 * cu;
      const float2 even = __ffma2_rn(make_float2(c9, c9), cg, __ffma2_rn(make_float2(cu * cu, cu * cu), Qw, Ew));
      const float2 odd = __ffma2_rn(Rw, make_float2(cu, cu), __fmul2_rn(make_float2(fp3, fp3), cg));
      const float2 fi = __ffma2_rn(om1_2, make_float2(fA[i], fB[i]), __fadd2_rn(even, odd));
      const float2 fj = __ffma2_rn(om1_2, make_float2(fA[j], fB[j]), __ffma2_rn(make_float2(-1.f, -1.f), odd, even));
      fA[i] = fi.x;
      fB[i] = fi.y;
      fA[j] = fj.x;
      fB[j] = fj.y;
    }
  }
  rA_out = rA;
  rB_out = rB;
}

// collide_core at site s, its coordinates computed from the index.
template <class T, bool kParticles, bool kMRT = false, bool kBisect = false>
__device__ __forceinline__ void collide_core(const StepParams &P, long long s, unsigned long long step,
                                             const T *__restrict__ fin, const float *__restrict__ rho,
                                             const ParticleArrays &pa, const ParticleForces &pf, CellIndex ci,
                                             unsigned *err, const float *__restrict__ rest_in, float (&fA)[kQ],
                                             float (&fB)[kQ], float &rA_out, float &rB_out) {
  collide_core_at<T, kParticles, kMRT, kBisect>(P, site_coord(P, s), s, step, fin, rho, pa, pf, ci, err, rest_in,
                                                fA, fB, rA_out, rB_out);
}

// The store of the update at site s32 (values from collide_core).  With 16-bit storage rest_out
// is the FP32 rest array (NULL, in the autotuner's trial launches: no rest population is
// written).  kWrite = false computes what would be stored without writing it.  With kKeep, fA and
// fB are left holding the stored values -- the moving ones as stored (16-bit: decoded, still
// shifted) and the rest population at [0] -- whose sum (plus the shifts, 16-bit) is the node's
// share of the next step's densities.
template <class T, bool kMRT = false, bool kWrite = true, bool kKeep = false>
__device__ __forceinline__ void store_node(const StepParams &P, unsigned s32, T *__restrict__ fout,
                                           float *__restrict__ rest_out, float (&fA)[kQ], float (&fB)[kQ],
                                           float rA, float rB, bool write = true) {
  static_assert(!(kMRT && kKeep), "the stored values are kept for the BGK update only");
  const unsigned N32 = (unsigned)P.N;
  constexpr bool kShifted = kSplitRest<T> && !kMRT;
  if constexpr (kSplitRest<T>) {
    unsigned *wout = reinterpret_cast<unsigned *>(fout) + s32;  // direction i at wout[i N]
    if (kShifted) {
      // store the 18 shifted (A, B) pairs; the rest population takes what keeps the node's mass
      // at its value before the update (the BGK update and the forcing term conserve it exactly)
      float2 m = make_float2(rA - shift_sum(P, 0), rB - shift_sum(P, 1));
      if constexpr (kKeep) {
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
          const unsigned w = Pair16<T>::enc(make_float2(fA[i], fB[i]));
          if (kWrite && write) wout[(size_t)i * N32] = w;
          const float2 d = Pair16<T>::dec(w);
          m = __ffma2_rn(make_float2(-1.f, -1.f), d, m);
          fA[i] = d.x;
          fB[i] = d.y;
        }
      } else {
        // the closure negated, -m + d per stored value with mixed-precision additions: round to
        // nearest is symmetric, so each partial is exactly minus the m - d of the form above
        float2 nm = make_float2(-m.x, -m.y);
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
          const unsigned w = Pair16<T>::enc(make_float2(fA[i], fB[i]));
          if (kWrite && write) wout[(size_t)i * N32] = w;
          Pair16<T>::add_to(w, nm);
        }
        m = make_float2(-nm.x, -nm.y);
      }
      if (kWrite && write && rest_out) {
        rest_out[s32] = m.x;
        rest_out[N32 + s32] = m.y;
      }
      if (kKeep) {
        fA[0] = m.x;
        fB[0] = m.y;
      }
    } else {
      // MRT: each moving population is rounded on store as f - w_i rho0; the FP32 rest population
      // takes the rounding error of the node's 18 others, so the node's total (and each
      // component's mass) is the one of the collision up to FP32 rounding
      float2 e = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 1; i < kQ; ++i) {
        const float2 v = make_float2(fA[i] - pop_shift(P, 0, i), fB[i] - pop_shift(P, 1, i));
        const unsigned w = Pair16<T>::enc(v);
        if (kWrite) wout[(size_t)i * N32] = w;
        e = __fadd2_rn(e, __ffma2_rn(make_float2(-1.f, -1.f), Pair16<T>::dec(w), v));
      }
      if (kWrite && rest_out) {
        rest_out[s32] = fA[0] + e.x;
        rest_out[N32 + s32] = fB[0] + e.y;
      }
    }
  } else if (kWrite) {
    float2 *fout2 = reinterpret_cast<float2 *>(fout) + s32;  // direction i at fout2[i N]
    if (write)
#pragma unroll
      for (int i = 0; i < kQ; ++i) fout2[(size_t)i * N32] = make_float2(fA[i], fB[i]);
  }
}

// The whole lattice update of one step at site s: collide_core, then the store.
template <class T, bool kParticles, bool kMRT = false, bool kBisect = false>
__device__ __forceinline__ void collide(const StepParams &P, long long s, unsigned long long step,
                                        const T *__restrict__ fin,
                                        T *__restrict__ fout, const float *__restrict__ rho,
                                        const ParticleArrays &pa, const ParticleForces &pf, CellIndex ci,
                                        unsigned *err, const float *__restrict__ rest_in,
                                        float *__restrict__ rest_out) {
  float fA[kQ], fB[kQ], rA, rB;
  collide_core<T, kParticles, kMRT, kBisect>(P, s, step, fin, rho, pa, pf, ci, err, rest_in, fA, fB, rA, rB);
  store_node<T, kMRT>(P, (unsigned)s, fout, rest_out, fA, fB, rA, rB);
}

// ------------------------------------------------------------------ particles

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

// Coupling forces on a particle (Sec. 2): the coupling velocity u_cpl = (j' + (g^SC + F^fs)/2)/rho
// and the node gradients S/c_s^2 are interpolated trilinearly from the 8 corners of the
// particle's cell; friction + noise (Eq. NEWTON), solvation (Eq. solvation_kappa) and the
// reaction of the particle's own fluid-side solvation force (Eq. solvation_lambda).  `step`
// is this lattice's step counter (the noise counter).
//
// The interpolated sums of one particle: coupling velocity, node gradients S_A, S_B and the
// reaction of its own fluid-side solvation force.
struct CoupleSums {
  float3 up, gA, gB, fsr;
};

// j' = sum_z sum_i f_zi c_i at node (x, y, z), pulled from the populations (the densities'
// pass of the one-pass update stores no j').  16-bit storage: the stored values are shifted by
// w_i rho0, and sum_i w_i c_i = 0, so the shifts drop out.
template <class T>
__device__ __forceinline__ float3 jprime_at(const StepParams &P, const T *__restrict__ fin, int x, int y, int z) {
  const NOff o = neighbour_offsets(P, Coord{x, y, z});
  const unsigned N32 = (unsigned)P.N, s32 = (unsigned)site_index(P, x, y, z);
  float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 1; i < kQ; ++i) {
    const unsigned src = i * N32 + (unsigned)((int)s32 + shift(o, -kCx[i], -kCy[i], -kCz[i]));  // pull r - c_i
    float2 v;
    if constexpr (kSplitRest<T>)
      v = Pair16<T>::dec(__ldg(reinterpret_cast<const unsigned *>(fin) + src));
    else
      v = __ldg(reinterpret_cast<const float2 *>(fin) + src);
    jx += kCx[i] * (v.x + v.y);
    jy += kCy[i] * (v.x + v.y);
    jz += kCz[i] * (v.x + v.y);
  }
  return make_float3(jx, jy, jz);
}

// Node of corner k (offset (k & 1, k >> 1 & 1, k >> 2 & 1)) of the cell c, wrapped.
__device__ __forceinline__ Coord cell_corner(const StepParams &P, int4 c, int k) {
  const int ox = k & 1, oy = (k >> 1) & 1, oz = (k >> 2) & 1;
  return Coord{c.x + ox == P.nx ? 0 : c.x + ox, c.y + oy == P.ny ? 0 : c.y + oy, c.z + oz == P.nz ? 0 : c.z + oz};
}

// Contribution of corner k of the particle's cell.  j' comes from jc (this particle's 8 corner
// values, formed beforehand) when not NULL, else from the field jp.
__device__ __forceinline__ void couple_corner(const StepParams &P, int k, int4 c, float4 fr, const TypeParams &T,
                                              const ParticleArrays &list, CellIndex ci,
                                              const float *__restrict__ rho, const float *__restrict__ jp,
                                              const ParticleForces &pf, bool with_fsr, CoupleSums &S,
                                              const float4 *__restrict__ jc = nullptr) {
  const int ox = k & 1, oy = (k >> 1) & 1, oz = (k >> 2) & 1;
  const Coord cc = cell_corner(P, c, k);
  const int X = cc.x, Y = cc.y, Z = cc.z;
  const long long s = site_index(P, X, Y, Z);
  float3 j;
  if (jc) {
    const float4 v = __ldg(jc + k);
    j = make_float3(v.x, v.y, v.z);
  } else {
    j = make_float3(__ldg(jp + s), __ldg(jp + P.N + s), __ldg(jp + 2 * P.N + s));
  }
  const NodeState n = node_state(P, rho, X, Y, Z);
  float3 fA = make_float3(-P.gAB * n.rA * n.SB.x, -P.gAB * n.rA * n.SB.y, -P.gAB * n.rA * n.SB.z);
  float3 fB = make_float3(-P.gBA * n.rB * n.SA.x, -P.gBA * n.rB * n.SA.y, -P.gBA * n.rB * n.SA.z);
  gather_coupling(P, X, Y, Z, n.rA, n.rB, list, pf, ci, false, fA, fB);
  const float rinv = 1.f / (n.rA + n.rB);
  const float w = (ox ? fr.x : 1.f - fr.x) * (oy ? fr.y : 1.f - fr.y) * (oz ? fr.z : 1.f - fr.z);
  S.up.x += w * (j.x + 0.5f * (fA.x + fB.x)) * rinv;
  S.up.y += w * (j.y + 0.5f * (fA.y + fB.y)) * rinv;
  S.up.z += w * (j.z + 0.5f * (fA.z + fB.z)) * rinv;
  S.gA.x += w * n.SA.x; S.gA.y += w * n.SA.y; S.gA.z += w * n.SA.z;
  S.gB.x += w * n.SB.x; S.gB.y += w * n.SB.y; S.gB.z += w * n.SB.z;
  if (with_fsr && (T.lam[0] != 0.f || T.lam[1] != 0.f)) {
    const float3 geo = fs_geometry(fr.x - ox, fr.y - oy, fr.z - oz);
    const float a = T.lam[0] * n.rA + T.lam[1] * n.rB;
    S.fsr.x += a * geo.x; S.fsr.y += a * geo.y; S.fsr.z += a * geo.z;
  }
}

// Forces from the sums: friction + noise (Eq. NEWTON), solvation (Eq. solvation_kappa), the
// reaction of the fluid-side solvation force.
__device__ __forceinline__ void couple_finish(const StepParams &P, unsigned long long step, int p,
                                              const ParticleArrays &self, const ParticleForces &pf, bool with_fsr,
                                              const TypeParams &T, float4 v, const CoupleSums &S) {
  float3 R = make_float3(0.f, 0.f, 0.f);
  if (T.noise_amp > 0.f) {
    const float3 nn = particle_normals(P.seed, step, (unsigned)self.pid[p]);
    const float amp = T.noise_amp * P.noise_scale;
    R = make_float3(amp * nn.x, amp * nn.y, amp * nn.z);
  }
  pf.fric[p] = make_float4(-T.gamma * (v.x - S.up.x) + R.x, -T.gamma * (v.y - S.up.y) + R.y,
                           -T.gamma * (v.z - S.up.z) + R.z, 0.f);
  const float kA = -T.kappa[0] / kCs2, kB = -T.kappa[1] / kCs2;
  pf.psA[p] = make_float4(kA * S.gA.x, kA * S.gA.y, kA * S.gA.z, 0.f);
  pf.psB[p] = make_float4(kB * S.gB.x, kB * S.gB.y, kB * S.gB.z, 0.f);
  if (with_fsr) pf.fsr[p] = make_float4(S.fsr.x, S.fsr.y, S.fsr.z, 0.f);
}

// Coupling forces on particle p with 8 lanes per particle: lane k of a group of 8 consecutive
// lanes takes corner k, the sums are added over the group by shuffles (mask: the group's
// lanes), and lane 0 writes the forces.  Every lane of the group must call it with the same p.
// `self` holds the particle's own state; `list` and ci the sorted particles whose fluid-side
// solvation force enters the coupling velocity (the same arrays, except in the later particle
// substeps, which keep the list of the step's start).  with_fsr: compute the reaction of the
// particle's own fluid-side solvation force (else keep the value in pf.fsr).
__device__ __forceinline__ void couple8(const StepParams &P, unsigned long long step, int p, int k, unsigned mask,
                                        const ParticleArrays &self, const ParticleArrays &list, CellIndex ci,
                                        const float *__restrict__ rho, const float *__restrict__ jp,
                                        const ParticleForces &pf, bool with_fsr = true,
                                        const float4 *__restrict__ jc = nullptr) {
  const int4 c = self.cell[p];
  const float4 fr = self.frac[p];
  const TypeParams &Ty = P.types[c.w];
  CoupleSums S{};
  couple_corner(P, k, c, fr, Ty, list, ci, rho, jp, pf, with_fsr, S, jc ? jc + (long long)self.pid[p] * 8 : nullptr);
  float *x = &S.up.x;  // the 12 sums, contiguous
#pragma unroll
  for (int off = 4; off > 0; off >>= 1)
#pragma unroll
    for (int q = 0; q < 12; ++q) x[q] += __shfl_xor_sync(mask, x[q], off);
  if (k == 0) couple_finish(P, step, p, self, pf, with_fsr, Ty, self.vel[p], S);
}
__device__ __forceinline__ int min_image_cells(int d, int n) {
  d = wrapi(d, n);
  return 2 * d > n ? d - n : d;
}

// Short-range pair forces (WCA, Sec. 4.1; screened Coulomb, Sec. 4.4) over the rows within
// `reach` cells of a particle, and bonded forces from its own bond list (bond_start indexed by
// the particle id, bond_other holding ids, slot_of_id mapping ids to sorted slots; NULL
// bond_start = no bonds).  Each particle computes its own force (pairs are visited from both
// ends): no atomics, fixed order.
//
// Pair forces on particle p from the particles of one lattice row of the cell index (-dU/dr),
// accumulated into F.
__device__ __forceinline__ void pair_row(const StepParams &P, int p, int4 c, float4 fr, int row, bool allx,
                                         const ParticleArrays &pa, CellIndex ci, float3 &F) {
  const int m = P.reach;
  const float Lx = (float)P.nx, Ly = (float)P.ny, Lz = (float)P.nz;
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

// Bond forces on particle p (FENE or harmonic), accumulated into F; a FENE bond stretched to
// its maximum sets kErrBond.
__device__ __forceinline__ void bond_forces(const StepParams &P, int p, int4 c, float4 fr, const ParticleArrays &pa,
                                            const int *__restrict__ bond_start, const int *__restrict__ bond_other,
                                            const int *__restrict__ slot_of_id, unsigned *err, float3 &F) {
  const float Lx = (float)P.nx, Ly = (float)P.ny, Lz = (float)P.nz;
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

// Pair and bonded forces of particle p with 8 lanes per particle: lane k of a group of 8
// consecutive lanes scans the rows k, k + 8, ... of the (2 reach + 1)^2 rows around the
// particle (the whole axis where the lattice is narrower), the forces are added over the group
// by shuffles (mask: the group's lanes), lane 0 adds the bonds and writes.  Every lane of the
// group must call it with the same p.
__device__ __forceinline__ void pairs8(const StepParams &P, int p, int k, unsigned mask, const ParticleArrays &pa,
                                       CellIndex ci, const int *__restrict__ bond_start,
                                       const int *__restrict__ bond_other, const int *__restrict__ slot_of_id,
                                       const ParticleForces &pf, unsigned *err) {
  const int4 c = pa.cell[p];
  const float4 fr = pa.frac[p];
  float3 F = make_float3(0.f, 0.f, 0.f);
  const int m = P.reach;
  if (m > 0) {
    const bool allz = 2 * m + 1 >= P.nz, ally = 2 * m + 1 >= P.ny, allx = 2 * m + 1 >= P.nx;
    const int z0 = allz ? 0 : -m, nzw = allz ? P.nz : 2 * m + 1;
    const int y0 = ally ? 0 : -m, nyw = ally ? P.ny : 2 * m + 1;
    for (int w = k; w < nzw * nyw; w += 8) {
      const int dz = z0 + w / nyw, dy = y0 + w % nyw;
      const int cz = allz ? dz : wrapi(c.z + dz, P.nz);
      const int cy = ally ? dy : wrapi(c.y + dy, P.ny);
      pair_row(P, p, c, fr, cz * P.ny + cy, allx, pa, ci, F);
    }
  }
#pragma unroll
  for (int off = 4; off > 0; off >>= 1) {
    F.x += __shfl_xor_sync(mask, F.x, off);
    F.y += __shfl_xor_sync(mask, F.y, off);
    F.z += __shfl_xor_sync(mask, F.z, off);
  }
  if (k == 0) {
    if (bond_start) bond_forces(P, p, c, fr, pa, bond_start, bond_other, slot_of_id, err, F);
    pf.pair[p] = make_float4(F.x, F.y, F.z, 0.f);
  }
}

// Particle update of slot p: v += F dt / m, x += v dt, periodic wrap kept as (cell,
// fraction).  Reads src, writes dst (the same arrays for an update in place).
__device__ __forceinline__ void integrate(const StepParams &P, int p, const ParticleArrays &src,
                                          const ParticleArrays &dst, const ParticleForces &pf, unsigned *err) {
  int4 c = src.cell[p];
  float4 fr = src.frac[p];
  float4 v = src.vel[p];
  if (dst.pid != src.pid) dst.pid[p] = src.pid[p];
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
    dst.cell[p] = c;  // position kept: every index stays inside the lattice
    dst.frac[p] = fr;
    dst.vel[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
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
  dst.cell[p] = c;
  dst.frac[p] = make_float4(nx_, ny_, nz_, fr.w);
  dst.vel[p] = v;
}

// ------------------------------------------------------------------ row scan

// Exclusive scan of one value per thread over a block of kScanThreads threads (warp shuffles,
// then a scan of the warp totals); `total` receives the block's sum.  Every thread of the block
// must call it.
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

}  // namespace site
}  // namespace lbmd
