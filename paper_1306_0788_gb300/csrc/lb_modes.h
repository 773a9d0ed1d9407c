// lb_modes.h -- the mode space of the fluctuating MRT collision (Eq. MODES): the orthogonal
// D3Q19 polynomials in the lattice velocity c of Duenweg, Schiller and Ladd, the basis the
// paper cites for its mode space.  Mode k of a population vector f is m_k = sum_i e_k(c_i) f_i;
// the basis is orthogonal in the weighted inner product, sum_i w_i e_k(c_i) e_l(c_i) = b_k
// delta_kl, so f_i = w_i sum_k e_k(c_i) m_k / b_k.
//   k = 0          density
//   k = 1, 2, 3    momentum x, y, z
//   k = 4          bulk stress        c^2 - 1
//   k = 5 .. 9     shear stresses     3c_x^2 - c^2, c_y^2 - c_z^2, c_x c_y, c_y c_z, c_z c_x
//   k = 10 .. 18   kinetic modes      (3c^2 - 5) c_a; (c_y^2 - c_z^2) c_x, (c_z^2 - c_x^2) c_y,
//                                     (c_x^2 - c_y^2) c_z; 3c^4 - 6c^2 + 1;
//                                     (2c^2 - 3)(3c_x^2 - c^2); (2c^2 - 3)(c_y^2 - c_z^2)
#pragma once

#if defined(__CUDACC__)
#define LBMD_MODE_HD __host__ __device__
#else
#define LBMD_MODE_HD
#endif

namespace lbmd {

constexpr int kModes = 19;

LBMD_MODE_HD constexpr int mode_poly(int k, int x, int y, int z) {
  const int c2 = x * x + y * y + z * z;
  return k == 0    ? 1
         : k == 1  ? x
         : k == 2  ? y
         : k == 3  ? z
         : k == 4  ? c2 - 1
         : k == 5  ? 3 * x * x - c2
         : k == 6  ? y * y - z * z
         : k == 7  ? x * y
         : k == 8  ? y * z
         : k == 9  ? z * x
         : k == 10 ? (3 * c2 - 5) * x
         : k == 11 ? (3 * c2 - 5) * y
         : k == 12 ? (3 * c2 - 5) * z
         : k == 13 ? (y * y - z * z) * x
         : k == 14 ? (z * z - x * x) * y
         : k == 15 ? (x * x - y * y) * z
         : k == 16 ? 3 * c2 * c2 - 6 * c2 + 1
         : k == 17 ? (2 * c2 - 3) * (3 * x * x - c2)
                   : (2 * c2 - 3) * (y * y - z * z);
}

// 9 b_k: the norms of the modes in ninths
LBMD_MODE_HD constexpr int mode_norm9(int k) {
  return k == 0 ? 9 : k <= 3 ? 3 : k == 4 ? 6 : k == 5 ? 12 : k == 6 ? 4 : k <= 9 ? 1 : k <= 12 ? 6 : k <= 15 ? 2
         : k == 16 ? 18 : k == 17 ? 12 : 4;
}

}  // namespace lbmd
