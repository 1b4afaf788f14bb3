// Lattice direction table shared by the family build (pd_build.cu) and the lattice step kernels
// (pd_step.cu), and the FP32 break decision of those kernels with its rounding band (host and
// device, so that a host test replays the same code).
//
// On a body whose particles sit on a regular lattice of spacing h, every bond vector is xi = h n with
// n an integer vector, and the family (Section 2.1: the closed ball |xi| <= delta) is the set of
// lattice directions with |n|^2 <= (delta / h)^2.  The table lists the non-zero integer vectors with
// |n|^2 <= kLatQmax[dim] in groups: |n|^2 <= 9, then each ring m^2 < |n|^2 <= (m + 1)^2.  Inside a
// group, each direction n whose first non-zero component from z down to x is positive, ordered by
// (n_z, n_y, n_x), is immediately followed by its opposite -n.  So
//   * every ball |n|^2 <= m^2 with m >= 3 (horizons from 3 h up to just below sqrt(10) h, 4 h, ...)
//     is a prefix of the table (one family = the first S directions); a ball that ends inside a
//     group is not, and such a body keeps the general layout;
//   * entry k and entry k ^ 1 are the two directions of one bond (xi_ji = -xi_ij);
//   * consecutive slots share their row (n_y, n_z): a slice is 32 particles along x (the brick
//     order), so the neighbours of successive slots are the same rows shifted by one along x and
//     the displacement gathers of a slot mostly hit the cache lines of the previous ones.
// In the lattice layout, slot k of every slice holds the neighbour in direction k of the table for
// every lane, so the bond vector of a slot is one value for the whole warp.
#pragma once

#include <math.h>

#include <algorithm>
#include <vector>

#if defined(__CUDACC__)
#define PD_LHD __host__ __device__ __forceinline__
#else
#define PD_LHD inline
#endif

namespace pd {

constexpr int kLatQmax3 = 25;  // 3D: |n|^2 <= 25 (horizons up to 5 h): 514 directions
constexpr int kLatQmax2 = 64;  // 2D: |n|^2 <= 64 (horizons up to 8 h): 196 directions
constexpr int kLatDirs3 = 514;
constexpr int kLatDirs2 = 196;
constexpr int kLatR3 = 5;      // component bound of the 3D table
constexpr int kLatR2 = 8;      // component bound of the 2D table

struct LatDir {
  int n[3];
  int q;  // |n|^2
};

// Group of a direction in the table order: 3 for |n|^2 <= 9, else the m with (m - 1)^2 < |n|^2 <= m^2.
constexpr int lattice_group(int q) {
  int m = 3;
  while (m * m < q) ++m;
  return m;
}

template <int DIM>
struct LatTable {
  static constexpr int kCount = DIM == 3 ? kLatDirs3 : kLatDirs2;
  LatDir d[kCount];
};

// The table as a compile-time constant.  Insertion sort of the positive representatives by
// (group, z, y, x), then each followed by its opposite.
template <int DIM>
constexpr LatTable<DIM> lattice_table() {
  constexpr int qmax = DIM == 3 ? kLatQmax3 : kLatQmax2;
  constexpr int R = DIM == 3 ? kLatR3 : kLatR2;
  LatTable<DIM> t{};
  LatDir pos[LatTable<DIM>::kCount / 2] = {};
  int np = 0;
  for (int z = (DIM == 3 ? -R : 0); z <= (DIM == 3 ? R : 0); ++z)
    for (int y = -R; y <= R; ++y)
      for (int x = -R; x <= R; ++x) {
        const int q = x * x + y * y + z * z;
        if (q == 0 || q > qmax) continue;
        const bool positive = z > 0 || (z == 0 && (y > 0 || (y == 0 && x > 0)));
        if (!positive) continue;
        LatDir e{{x, y, z}, q};
        int k = np++;
        while (k > 0) {
          const LatDir& p = pos[k - 1];
          const int gp = lattice_group(p.q), ge = lattice_group(e.q);
          const bool after = gp != ge ? gp > ge
                                      : (p.n[2] != e.n[2] ? p.n[2] > e.n[2]
                                                          : (p.n[1] != e.n[1] ? p.n[1] > e.n[1] : p.n[0] > e.n[0]));
          if (!after) break;
          pos[k] = pos[k - 1];
          --k;
        }
        pos[k] = e;
      }
  for (int k = 0; k < np; ++k) {
    t.d[2 * k] = pos[k];
    t.d[2 * k + 1] = LatDir{{-pos[k].n[0], -pos[k].n[1], -pos[k].n[2]}, pos[k].q};
  }
  return t;
}

// Number of directions with |n|^2 <= q (a family) when they are the first entries of the table,
// else -1 (the ball is not a prefix: |n|^2 <= q ends inside a group), at compile time.
template <int DIM>
constexpr int lattice_prefix_c(int q) {
  const LatTable<DIM> t = lattice_table<DIM>();
  int k = 0, in = 0;
  for (int e = 0; e < LatTable<DIM>::kCount; ++e) in += t.d[e].q <= q ? 1 : 0;
  while (k < LatTable<DIM>::kCount && t.d[k].q <= q) ++k;
  return k == in ? k : -1;
}

inline std::vector<LatDir> lattice_directions(int dim) {
  std::vector<LatDir> out;
  if (dim == 3) {
    constexpr LatTable<3> t = lattice_table<3>();
    out.assign(t.d, t.d + LatTable<3>::kCount);
  } else {
    constexpr LatTable<2> t = lattice_table<2>();
    out.assign(t.d, t.d + LatTable<2>::kCount);
  }
  return out;
}

// Index into the lookup cube of side 2R + 1 (z ignored in 2D).
inline int lattice_cube_index(int dim, int x, int y, int z) {
  const int R = dim == 3 ? kLatR3 : kLatR2, s = 2 * R + 1;
  return dim == 3 ? ((z + R) * s + (y + R)) * s + (x + R) : (y + R) * s + (x + R);
}

// Cube of side 2R + 1 mapping a direction to its table index (-1 outside the table).
inline std::vector<short> lattice_lookup(int dim) {
  const int R = dim == 3 ? kLatR3 : kLatR2, s = 2 * R + 1;
  std::vector<short> cube((size_t)(dim == 3 ? s * s * s : s * s), (short)-1);
  const std::vector<LatDir> t = lattice_directions(dim);
  for (size_t k = 0; k < t.size(); ++k)
    cube[lattice_cube_index(dim, t[k].n[0], t[k].n[1], t[k].n[2])] = (short)k;
  return cube;
}

// Number of table directions with |n|^2 <= q (the family of a ball of radius sqrt(q) h) when they
// are the first entries of the table, else -1.
inline int lattice_prefix(int dim, int q) {
  const std::vector<LatDir> t = lattice_directions(dim);
  int k = 0, in = 0;
  for (const LatDir& e : t) in += e.q <= q ? 1 : 0;
  while (k < (int)t.size() && t[k].q <= q) ++k;
  return k == in ? k : -1;
}

// ------------------------------------------------------------- FP32 break decision and its band
// In lattice units (u' = u / h in FP32, xi = h n) the failure criterion of Eq 1.30 in its sqrt-free
// form xi.(u_j - u_i) >= s0 |xi|^2 reads d' >= s0 |n|^2 with d' = n.(u'_j - u'_i).  The kernels
// evaluate g = d' - s0 |n|^2 in FP32 (the operations of lat_dprime and lat_g) and bound its
// distance from the FP64 evaluation of the same criterion from the master state and the FP64
// positions (eps = 2^-24; U_i, U_j = |u'|_inf of the two ends, N1 = the largest |n|_1 of the
// family, c = the safety factor pd_params.band_safety):
//   * the FP32 copies of u at both ends: eps |n|_1 (U_i + U_j) (relative rounding of each component);
//   * the differences u'_j - u'_i: eps |n|_1 (U_i + U_j);
//   * the product and the two FMAs of the dot product: 3 eps |n|_1 (U_i + U_j);
//   * the FP64 side: bond vectors within 2^-30 h of h n (checked when the layout is built) and the
//     FP64 rounding of its own dot product and threshold: 0.06 eps (U_i + U_j) + 0.034 eps s0 N1;
//   * s0 rounded to FP32: eps s0 |n|^2; the final FMA: eps |g|;
// so |g - g_FP64| <= B = c (1 + 8 eps) eps [(5.0003 N1 + 0.06)(U_i + U_j) + s0 (|n|^2 + 0.034 N1) + |g|]
// (the 8 eps covers the FP32 evaluation of B itself, for c >= 1).  With the two-word shadow
// (u' = hi + lo, both FP32, lo the rounding remainder of hi) each difference is (hi_j - hi_i) +
// (lo_j - lo_i): the copies then differ from u' by at most eps |lo| <= eps^2 U, and the two roundings
// of the difference stay within the 2 eps |n|_1 (U_i + U_j) of the first two terms above, so the same
// B bounds that evaluation (lat_delta_lo).  Outside +-B the FP32 sign is the
// FP64 decision; inside, the bond is re-decided in FP64.  The screen g < -(Kfast (U_i + U_j) +
// Kcfast), with |g| = -g folded in (division by 1 - c eps) and |n|^2 bounded by the family's
// largest, implies g < -B: it settles the bonds far from their threshold in a few instructions
// (with U_j replaced by the body's bound, below: one FMA and one max per slot).
struct LatBand {
  float Kf, sq, eps_c, s0n1, Kfast, Kcfast;
};

inline LatBand lattice_band(double band_safety, double s0, int n1, int qmax) {
  const double bc = band_safety > 0 ? band_safety : 4.0;
  const double eps = 5.9604644775390625e-8, infl = 1.0 + 8.0 * eps;
  const double k1 = 5.0003 * n1 + 0.06;
  LatBand b;
  b.Kf = (float)(bc * eps * k1 * infl);
  b.sq = (float)(bc * eps * (1.0 + 1.5e-8) * infl);
  b.eps_c = (float)(bc * eps * infl);
  b.s0n1 = (float)(bc * eps * s0 * 0.034 * n1 * infl);
  const double fast = infl / (1.0 - bc * eps);
  b.Kfast = (float)(bc * eps * k1 * fast);
  b.Kcfast = (float)(bc * eps * s0 * (qmax * (1.0 + 1.5e-8) + 0.034 * n1) * fast);
  return b;
}

// d' = n.(u'_j - u'_i) from the differences: one product and two FMAs (one in 2D).
template <int DIM>
PD_LHD float lat_dprime_d(float nx, float ny, float nz, float dx, float dy, float dz) {
  float d = nx * dx;
  d = fmaf(ny, dy, d);
  if (DIM == 3) d = fmaf(nz, dz, d);
  return d;
}

// d' = n.(u'_j - u'_i) from one-word shadows.
template <int DIM>
PD_LHD float lat_dprime(float nx, float ny, float nz, float ujx, float ujy, float ujz, float uix, float uiy,
                        float uiz) {
  return lat_dprime_d<DIM>(nx, ny, nz, ujx - uix, ujy - uiy, ujz - uiz);
}

// One component of u'_j - u'_i from two-word shadows (hi + lo).
PD_LHD float lat_delta_lo(float hj, float lj, float hi, float li) { return (hj - hi) + (lj - li); }

// g = d' - s0 |n|^2 in one FMA.
PD_LHD float lat_g(float d, float s0f, float q) { return fmaf(-s0f, q, d); }

// The screen: true settles the bond as intact.  scr_i = fmaf(Kfast, U_i, Kcfast), once per particle.
PD_LHD bool lat_screen_intact(float g, float Kfast, float Uj, float scr_i) { return fmaf(Kfast, Uj, g) < -scr_i; }

// The same screen as a value: lat_screen_value < 0 exactly when lat_screen_intact (a < -b and the
// rounded a + b < 0 agree: a sum of two floats rounds to zero only when it is exactly zero), NaN when
// an operand is NaN.  scr_i = -inf settles every bond with a finite value (a body without failure).
PD_LHD float lat_screen_value(float g, float Kfast, float Uj, float scr_i) { return fmaf(Kfast, Uj, g) + scr_i; }

// The per-body screen of the kernels: the neighbour's |u'_j|_inf replaced by an upper bound U_max of
// |u'|_inf over the particle's body (the largest the shadow holds), so that the screen's per-particle
// part scr_c = fmaf(Kfast, U_i + U_max', Kcfast) is formed once and a batch of slots is settled as
// intact when (max over its slots of g) + scr_c < 0.  U_max' = U_max (1 + 2^-20): with U_i <= U_max
// it keeps the rounded U_i + U_max' above U_i + U_j for every neighbour j, with a margin far above
// the roundings of the sum and of the FMA, so the screen stays at least as wide as the
// per-neighbour one.  The max propagates NaN (a batch with a NaN extension is not settled).
PD_LHD float lat_umax_bound(float umax) { return umax * (1.0f + 0x1p-20f); }
PD_LHD float lat_screen_part(float Kfast, float Ui, float umax_b, float Kcfast) { return fmaf(Kfast, Ui + umax_b, Kcfast); }
PD_LHD float lat_max_nan(float a, float b) {
#if defined(__CUDA_ARCH__)
  float r;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
#else
  return (a != a || b != b) ? NAN : (a > b ? a : b);
#endif
}

// Full band: 0 intact, 1 broken (FP32 decision), 2 inside the band (decide in FP64).  A NaN g is
// inside (both comparisons false).
PD_LHD int lat_code(float g, float Ui, float Uj, float s0f, float q, float Kf, float sq, float eps_c,
                    float s0n1) {
  const float B = fmaf(Kf, Ui + Uj, fmaf(sq, s0f * q, fmaf(eps_c, fabsf(g), s0n1)));
  return g > B ? 1 : (g < -B ? 0 : 2);
}

// ------------------------------------------------ nonlinear bonds: FP32 break decision and its band
// With the nonlinear extension (Eq 1.10) the failure criterion of Eq 1.30, e / |xi| >= s0, reads
// |Y|^2 - |xi|^2 >= c |xi|^2 with c = s0 (2 + s0), and in lattice units (eta' = u'_j - u'_i, Y' = n +
// eta') g = eta'.(2 n + eta') - c |n|^2 >= 0 (no cancellation between |Y'|^2 and |n|^2).  The kernels
// evaluate it in FP32 as lat_g_nl does: eta'_c one rounding, a_c = 2 n_c + eta'_c one FMA, the dot
// product eta'.a one product and two FMAs, g = fmaf(-c32, |n|^2, p).  With eps = 2^-24, S = U_i + U_j
// (|u'|_inf of the two ends), D = |eta'|_1 (FP32), N1 / Ninf = the family's largest |n|_1 / |n_c|:
//   * the FP32 copies of u move each eta'_c by at most eps S, and p by at most 2 eps S sum |Y'_c| <=
//     2 eps S (N1 + D) (dp / d eta'_c = 2 Y'_c);
//   * the rounding of eta'_c moves p by 2 |Y'_c| eps |eta'_c|, that of a_c by eps |eta'_c a_c|, the dot
//     product's three roundings by 3 eps sum |eta'_c a_c|: together at most eps (10 Ninf D + 6 D^2);
//   * c rounded to FP32: eps c |n|^2; the final FMA: eps |g|;
//   * the FP64 side: bond vectors within 2^-30 h of h n (checked when the layout is built) move its
//     value by 2^-29 (D + c N1) = eps (D + c N1) / 32, and its own roundings stay far below eps;
// so |g - g_FP64| <= k (1 + 8 eps) eps [2 S N1 + c (qmax + N1 / 32) + D (10 Ninf + 2 S + 1/32) +
// 6 D^2 + |g|] (the 8 eps covers the FP32 evaluation of B; k = pd_params.band_safety).  With the
// two-word shadow (u' = hi + lo) eta'_c = (hi_j - hi_i) + (lo_j - lo_i): the copies then differ from
// u' by at most eps |lo| <= eps^2 U (far below the 2 eps S (N1 + D) allotted to them) and eta'_c takes
// two roundings instead of one, 2 eps |eta'_c| (1 + O(eps)), which adds at most eps (2 Ninf D + 2 D^2)
// to the arithmetic term; the band B below carries 12 Ninf and 8 instead of 10 and 6, so one B
// bounds both forms.  The screen replaces U_j by the body's bound U_max (as for linearized bonds) and
// folds |g| = -g in.
struct LatBandNL {
  float A0, A0s, A1, A1s, A2, Ag;  // B = A0 + A0s S + D (A1 + A1s S) + A2 D^2 + Ag |g|
  float F0, F0s, F1, F1s, F2;      // the screen's B for g < 0, |g| folded in (divided by 1 - Ag)
};

inline LatBandNL lattice_band_nl(double band_safety, double s0, int n1, int ninf, int qmax) {
  const double k = band_safety > 0 ? band_safety : 4.0;
  const double eps = 5.9604644775390625e-8, infl = 1.0 + 8.0 * eps;
  const double c = s0 * (2.0 + s0);
  const double m = k * eps * infl;
  LatBandNL b;
  b.A0 = (float)(m * c * (qmax + n1 / 32.0));
  b.A0s = (float)(m * 2.0 * n1);
  b.A1 = (float)(m * (12.0 * ninf + 1.0 / 32.0));
  b.A1s = (float)(m * 2.0);
  b.A2 = (float)(m * 8.0);
  b.Ag = (float)(m);
  const double fast = infl / (1.0 - m);
  b.F0 = (float)(m * c * (qmax + n1 / 32.0) * fast);
  b.F0s = (float)(m * 2.0 * n1 * fast);
  b.F1 = (float)(m * (12.0 * ninf + 1.0 / 32.0) * fast);
  b.F1s = (float)(m * 2.0 * fast);
  b.F2 = (float)(m * 8.0 * fast);
  return b;
}

// The FP32 criterion of a nonlinear bond from eta' = u'_j - u'_i (formed by the caller, one rounding
// per component): p = eta'.(2 n + eta') and g = p - c32 |n|^2; D = |eta'|_1.
template <int DIM>
PD_LHD float lat_p_nl(float nx, float ny, float nz, float ex, float ey, float ez) {
  float p = ex * fmaf(2.0f, nx, ex);
  p = fmaf(ey, fmaf(2.0f, ny, ey), p);
  if (DIM == 3) p = fmaf(ez, fmaf(2.0f, nz, ez), p);
  return p;
}
PD_LHD float lat_g_nl(float p, float c32, float q) { return fmaf(-c32, q, p); }

// The screen's half-width for a slot: S = U_i + U_max' (the lane's part of it precomputed as the
// polynomial's coefficients f0 = F0 + F0s S, f1 = F1 + F1s S); the bond is settled as intact when
// g + lat_screen_nl(...) < 0.
PD_LHD float lat_screen_nl(float D, float f0, float f1, float F2) { return fmaf(D, fmaf(F2, D, f1), f0); }

// Full band: 0 intact, 1 broken (FP32 decision), 2 inside the band (decide in FP64); NaN is inside.
PD_LHD int lat_code_nl(float g, float D, float S, const LatBandNL& b) {
  const float B = fmaf(b.Ag, fabsf(g), fmaf(D, fmaf(b.A2, D, fmaf(b.A1s, S, b.A1)), fmaf(b.A0s, S, b.A0)));
  return g > B ? 1 : (g < -B ? 0 : 2);
}

}  // namespace pd
