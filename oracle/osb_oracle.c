/*
 * Plain double-precision CPU oracle for linearized ordinary state-based peridynamics
 * (T. Ni, M. Zaccariotto, Q. Zhu, U. Galvanetto, "Matrix-based implementation and GPU acceleration
 * of linearized ordinary state-based peridynamic models in MATLAB", arXiv 2309.11273).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check of the package entry
 * module and the CPU-baseline leg of the benchmark may load this library.  It shares no code, header,
 * table or helper with the CUDA library; it is written directly from the paper's definitions, one
 * function per equation, in user particle order, with every neighbour sum taken over the family in
 * ascending neighbour index.  Each particle's sums are computed by one thread in that fixed order, so
 * results do not depend on the number of OpenMP threads.
 *
 * Conventions (the paper's notation):
 *   xi_ij  = x_j - x_i                     reference bond vector           (Eq 1.3)
 *   x_ij   = |xi_ij|                       reference bond length           (Eq 1.5)
 *   M_ij   = xi_ij / x_ij                  linearized unit state           (Eq 1.13, small-deformation form)
 *   e_ij   = M_ij . (u_j - u_i)            linearized extension            (Eqs 1.10, 2.4, 2.7)
 *   (with kin = ORC_NONLINEAR: Y_ij = xi_ij + u_j - u_i, e_ij = |Y_ij| - x_ij, M_ij = Y_ij / |Y_ij|,
 *    Eqs 1.10 and 1.13 without the small-deformation approximation)
 *   w      = 1                             influence function              (Section 2.3, text after Eq 1.26)
 *   rho_ij = 1 intact, 0 broken            bond status                     (Eq 1.30)
 *
 * Parity unpinned: none -- every function here is pinned by the tests (closed forms, invariants,
 * brute force, values printed in the paper).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_3D = 0, ORC_PLANE_STRESS = 1, ORC_PLANE_STRAIN = 2 };
enum { ORC_FREE = 0, ORC_FIXED = 1, ORC_PRESCRIBED = 2 };
enum { ORC_LINEARIZED = 0, ORC_NONLINEAR = 1 };  /* bond kinematics, see bond_kinematics() */

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------------------
 * Material constants.
 *   kappa = E / (3 (1 - 2 nu)), mu = E / (2 (1 + nu))   (classical bulk and shear moduli)
 *   A : Eq 1.8;  K : Eq 1.15;  G : Eq 1.16.
 * ---------------------------------------------------------------------------------------------- */
void orc_constants(int model, double E, double nu, double* A, double* K, double* G, double* kappa,
                   double* mu) {
  double k = E / (3.0 * (1.0 - 2.0 * nu));
  double m = E / (2.0 * (1.0 + nu));
  *kappa = k;
  *mu = m;
  if (model == ORC_3D) {
    *A = 3.0;
    *K = 3.0 * k;
    *G = 15.0 * m;
  } else if (model == ORC_PLANE_STRESS) {
    *A = 2.0 * (1.0 - 2.0 * nu) / (1.0 - nu);
    *K = 2.0 * k * (1.0 - 2.0 * nu) / (1.0 - nu) -
         (2.0 / 3.0) * m * (1.0 + nu) * (1.0 - 3.0 * nu) / ((1.0 - nu) * (1.0 - 2.0 * nu));
    *G = 8.0 * m;
  } else {
    *A = 2.0;
    *K = 2.0 * k - (2.0 / 3.0) * m;
    *G = 8.0 * m;
  }
}

/* ------------------------------------------------------------------------------------------------
 * Critical stretch from the critical energy release rate G_c (w = 1).
 *   3D: Eq 1.26 with beta = 125 delta / 1848 and beta' = 5 delta / 24.
 *       Reading: Eq 1.27 prints beta' = 5 delta / (24 pi); integrating Eq 1.25 for the unit-weight
 *       sphere gives 5 delta / 24 (the tests integrate Eq 1.25 numerically), so the pi is dropped.
 *   2D: Eq 1.28 with Eq 1.29, as printed; kappa' per model.
 * ---------------------------------------------------------------------------------------------- */
double orc_critical_stretch(int model, double E, double nu, double Gc, double delta) {
  double A, K, G, kappa, mu;
  orc_constants(model, E, nu, &A, &K, &G, &kappa, &mu);
  if (model == ORC_3D) {
    double beta = 125.0 * delta / 1848.0;
    double betap = 5.0 * delta / 24.0;
    return sqrt(Gc / ((9.0 * kappa - 15.0 * mu) * beta + 15.0 * mu * betap));
  }
  double pi = 3.14159265358979323846;
  double kp;
  if (model == ORC_PLANE_STRESS) {
    double r = (1.0 + nu) / (1.0 - 2.0 * nu);
    kp = kappa + mu / 9.0 * r * r;
  } else {
    kp = kappa + mu / 9.0;
  }
  double beta = 1087.0 * delta / (1250.0 * pi * pi);
  double betap = 4.0 * delta / (5.0 * pi);
  return sqrt(Gc / (A * A * (kp - 8.0 * mu / 9.0) * beta + 8.0 * mu * betap));
}

/* ------------------------------------------------------------------------------------------------
 * Pre-crack / notch filter (the bonds crossing the crack surface are never created; Section 4.2 and
 * Section 4.4 describe pre-cracked and notched specimens).  A crack is stored as 9 doubles p0,p1,p2.
 *   2D: segment p0-p1 (p2 unused).   3D: parallelogram p0 + a (p1 - p0) + b (p2 - p0), a, b in [0,1].
 * Bond a-b is cut iff a and b lie strictly on opposite sides of the crack line / plane and the point
 * where the bond crosses that line / plane lies on the closed segment / parallelogram.
 * ---------------------------------------------------------------------------------------------- */
static int bond_cut_2d(const double a[3], const double b[3], const double* c) {
  double dx = c[3] - c[0], dy = c[4] - c[1];
  double sa = dx * (a[1] - c[1]) - dy * (a[0] - c[0]);
  double sb = dx * (b[1] - c[1]) - dy * (b[0] - c[0]);
  if (!((sa > 0.0 && sb < 0.0) || (sa < 0.0 && sb > 0.0))) return 0;
  double t = sa / (sa - sb);
  double px = a[0] + t * (b[0] - a[0]);
  double py = a[1] + t * (b[1] - a[1]);
  double lam = ((px - c[0]) * dx + (py - c[1]) * dy) / (dx * dx + dy * dy);
  return lam >= 0.0 && lam <= 1.0;
}

static int bond_cut_3d(const double a[3], const double b[3], const double* c) {
  double e1[3] = {c[3] - c[0], c[4] - c[1], c[5] - c[2]};
  double e2[3] = {c[6] - c[0], c[7] - c[1], c[8] - c[2]};
  double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                 e1[0] * e2[1] - e1[1] * e2[0]};
  double sa = n[0] * (a[0] - c[0]) + n[1] * (a[1] - c[1]) + n[2] * (a[2] - c[2]);
  double sb = n[0] * (b[0] - c[0]) + n[1] * (b[1] - c[1]) + n[2] * (b[2] - c[2]);
  if (!((sa > 0.0 && sb < 0.0) || (sa < 0.0 && sb > 0.0))) return 0;
  double t = sa / (sa - sb);
  double r[3];
  for (int k = 0; k < 3; ++k) r[k] = a[k] + t * (b[k] - a[k]) - c[k];
  /* Solve [e1.e1 e1.e2; e1.e2 e2.e2] [al; be] = [e1.r; e2.r] by Cramer's rule. */
  double g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
  double g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
  double g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
  double r1 = e1[0] * r[0] + e1[1] * r[1] + e1[2] * r[2];
  double r2 = e2[0] * r[0] + e2[1] * r[1] + e2[2] * r[2];
  double det = g11 * g22 - g12 * g12;
  double al = (r1 * g22 - r2 * g12) / det;
  double be = (g11 * r2 - g12 * r1) / det;
  return al >= 0.0 && al <= 1.0 && be >= 0.0 && be <= 1.0;
}

static int bond_cut(int dim, const double a[3], const double b[3], int ncracks, const double* cracks) {
  for (int c = 0; c < ncracks; ++c) {
    const double* cr = cracks + 9 * c;
    if (dim == 2 ? bond_cut_2d(a, b, cr) : bond_cut_3d(a, b, cr)) return 1;
  }
  return 0;
}

static void load_point(int dim, const double* x, const double* y, const double* z, int64_t i,
                       double p[3]) {
  p[0] = x[i];
  p[1] = y[i];
  p[2] = (dim == 3) ? z[i] : 0.0;
}

/* Horizon membership (Section 2.1: H_x = {|xi| <= delta}, a closed ball), tested as xi.xi <= delta^2. */
static int in_horizon(int dim, const double pi_[3], const double pj[3], double delta) {
  double dx = pj[0] - pi_[0], dy = pj[1] - pi_[1], dz = pj[2] - pi_[2];
  double q = dx * dx + dy * dy;
  if (dim == 3) q += dz * dz;
  return q <= delta * delta;
}

/* ------------------------------------------------------------------------------------------------
 * Family of every particle by brute force over all pairs (O(N^2)).  Two-call protocol:
 *   col == NULL : writes counts[i] = |H_i| (cracked bonds excluded) and returns the total;
 *   col != NULL : fills col[row_ptr[i] .. row_ptr[i+1]) with the neighbours in ascending order.
 * ---------------------------------------------------------------------------------------------- */
int64_t orc_family_bruteforce(int64_t n, int dim, const double* x, const double* y, const double* z,
                              double delta, int ncracks, const double* cracks, int64_t* counts,
                              const int64_t* row_ptr, int32_t* col) {
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
  for (int64_t i = 0; i < n; ++i) {
    double pi_[3], pj[3];
    load_point(dim, x, y, z, i, pi_);
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      load_point(dim, x, y, z, j, pj);
      if (!in_horizon(dim, pi_, pj, delta)) continue;
      if (bond_cut(dim, pi_, pj, ncracks, cracks)) continue;
      if (col) col[row_ptr[i] + c] = (int32_t)j;
      ++c;
    }
    if (!col) counts[i] = c;
    total += c;
  }
  return total;
}

/* ------------------------------------------------------------------------------------------------
 * Same family through uniform bins of edge >= delta: only the 3^dim bins around a particle's bin can
 * hold neighbours.  Candidates are collected, sorted ascending, and given the same two tests as the
 * brute-force search, so the output is identical (checked by the tests).
 * ---------------------------------------------------------------------------------------------- */
static int cmp_i64(const void* a, const void* b) {
  int64_t u = *(const int64_t*)a, v = *(const int64_t*)b;
  return (u > v) - (u < v);
}

int64_t orc_family_binned(int64_t n, int dim, const double* x, const double* y, const double* z,
                          double delta, int ncracks, const double* cracks, int64_t* counts,
                          const int64_t* row_ptr, int32_t* col) {
  if (n <= 0) return 0;
  double lo[3] = {x[0], y[0], dim == 3 ? z[0] : 0.0}, hi[3] = {x[0], y[0], dim == 3 ? z[0] : 0.0};
  for (int64_t i = 0; i < n; ++i) {
    double p[3];
    load_point(dim, x, y, z, i, p);
    for (int k = 0; k < 3; ++k) {
      if (p[k] < lo[k]) lo[k] = p[k];
      if (p[k] > hi[k]) hi[k] = p[k];
    }
  }
  double h = delta > 0.0 ? delta : 1.0;
  int64_t nb[3];
  for (int k = 0; k < 3; ++k) nb[k] = (int64_t)floor((hi[k] - lo[k]) / h) + 1;
  if (dim == 2) nb[2] = 1;
  int64_t nbins = nb[0] * nb[1] * nb[2];
  int64_t* bin_of = (int64_t*)malloc(sizeof(int64_t) * n);
  int64_t* bin_start = (int64_t*)calloc(nbins + 1, sizeof(int64_t));
  int64_t* bin_items = (int64_t*)malloc(sizeof(int64_t) * n);
  int64_t* fill = (int64_t*)calloc(nbins, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    double p[3];
    load_point(dim, x, y, z, i, p);
    int64_t b[3];
    for (int k = 0; k < 3; ++k) {
      b[k] = (int64_t)floor((p[k] - lo[k]) / h);
      if (b[k] >= nb[k]) b[k] = nb[k] - 1;
      if (b[k] < 0) b[k] = 0;
    }
    bin_of[i] = (b[2] * nb[1] + b[1]) * nb[0] + b[0];
    bin_start[bin_of[i] + 1]++;
  }
  for (int64_t b = 0; b < nbins; ++b) bin_start[b + 1] += bin_start[b];
  for (int64_t i = 0; i < n; ++i) bin_items[bin_start[bin_of[i]] + fill[bin_of[i]]++] = i;

  int64_t total = 0;
#pragma omp parallel reduction(+ : total)
  {
    int64_t cap = 1024;
    int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * cap);
#pragma omp for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
      double pi_[3], pj[3];
      load_point(dim, x, y, z, i, pi_);
      int64_t bi = bin_of[i];
      int64_t b0 = bi % nb[0], b1 = (bi / nb[0]) % nb[1], b2 = bi / (nb[0] * nb[1]);
      int64_t nc = 0;
      for (int64_t d2 = -1; d2 <= 1; ++d2)
        for (int64_t d1 = -1; d1 <= 1; ++d1)
          for (int64_t d0 = -1; d0 <= 1; ++d0) {
            int64_t c0 = b0 + d0, c1 = b1 + d1, c2 = b2 + d2;
            if (c0 < 0 || c1 < 0 || c2 < 0 || c0 >= nb[0] || c1 >= nb[1] || c2 >= nb[2]) continue;
            int64_t cb = (c2 * nb[1] + c1) * nb[0] + c0;
            for (int64_t t = bin_start[cb]; t < bin_start[cb + 1]; ++t) {
              if (nc == cap) {
                cap *= 2;
                cand = (int64_t*)realloc(cand, sizeof(int64_t) * cap);
              }
              cand[nc++] = bin_items[t];
            }
          }
      qsort(cand, (size_t)nc, sizeof(int64_t), cmp_i64);
      int64_t c = 0;
      for (int64_t t = 0; t < nc; ++t) {
        int64_t j = cand[t];
        if (j == i) continue;
        load_point(dim, x, y, z, j, pj);
        if (!in_horizon(dim, pi_, pj, delta)) continue;
        if (bond_cut(dim, pi_, pj, ncracks, cracks)) continue;
        if (col) col[row_ptr[i] + c] = (int32_t)j;
        ++c;
      }
      if (!col) counts[i] = c;
      total += c;
    }
    free(cand);
  }
  free(bin_of);
  free(bin_start);
  free(bin_items);
  free(fill);
  return total;
}

/* ------------------------------------------------------------------------------------------------
 * Bond geometry helper: xi = x_j - x_i (Eq 1.3) and x = |xi| (Eq 1.5).
 * ---------------------------------------------------------------------------------------------- */
static double bond_vector(int dim, const double* x, const double* y, const double* z, int64_t i,
                          int64_t j, double xi[3]) {
  xi[0] = x[j] - x[i];
  xi[1] = y[j] - y[i];
  xi[2] = (dim == 3) ? z[j] - z[i] : 0.0;
  double q = xi[0] * xi[0] + xi[1] * xi[1];
  if (dim == 3) q += xi[2] * xi[2];
  return sqrt(q);
}

/* Extension scalar e_ij and unit direction M_ij of a bond with reference vector xi (length xlen).
 *   kin = ORC_LINEARIZED (the paper's method, Eqs 2.4, 2.7): M = xi / |xi| (the small-deformation
 *     approximation stated under Eq 1.13) and e = M . (u_j - u_i).
 *   kin = ORC_NONLINEAR (Eqs 1.10 and 1.13 as written): Y = xi + eta with eta = u_j - u_i,
 *     e = |Y| - |xi| and M = Y / |Y|.  The difference of the two lengths is evaluated as
 *     (|Y|^2 - |xi|^2) / (|Y| + |xi|) with |Y|^2 - |xi|^2 = 2 xi.eta + eta.eta, the same number
 *     without the cancellation of two nearly equal lengths. */
static double bond_kinematics(int kin, int dim, const double xi[3], double xlen, const double* ux,
                              const double* uy, const double* uz, int64_t i, int64_t j, double M[3]) {
  double eta[3] = {ux[j] - ux[i], uy[j] - uy[i], dim == 3 ? uz[j] - uz[i] : 0.0};
  if (kin == ORC_LINEARIZED) {
    double e = 0.0;
    for (int k = 0; k < dim; ++k) {
      M[k] = xi[k] / xlen;
      e += M[k] * eta[k];
    }
    if (dim == 2) M[2] = 0.0;
    return e;
  }
  double Y[3], yy = 0.0, p = 0.0;
  for (int k = 0; k < dim; ++k) {
    Y[k] = xi[k] + eta[k];
    yy += Y[k] * Y[k];
    p += 2.0 * xi[k] * eta[k] + eta[k] * eta[k];
  }
  double ylen = sqrt(yy);
  for (int k = 0; k < dim; ++k) M[k] = Y[k] / ylen;
  if (dim == 2) M[2] = 0.0;
  return p / (ylen + xlen);
}

/* Influence function w(|xi|) of Eqs 1.6, 1.9, 1.14 and 1.31.  The paper uses w = 1 (Section 2.3, where
 * the critical stretch is derived) and refers at Eq 1.9 to the published catalogue of other forms;
 * ORC_W_INV is the form w = delta / |xi| from that catalogue. */
enum { ORC_W_ONE = 0, ORC_W_INV = 1 };
static double influence(int infl, double delta, double xlen) {
  return infl == ORC_W_INV ? delta / xlen : 1.0;
}

/* Weighted volume m_i = sum_j w x_ij^2 V_j over the built family (Eq 1.9, discretized). */
void orc_weighted_volume(int64_t n, int dim, const double* x, const double* y, const double* z,
                         const double* vol, const int64_t* row_ptr, const int32_t* col, int infl,
                         double delta, double* m) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
      double xi[3];
      double xl = bond_vector(dim, x, y, z, i, col[b], xi);
      s += influence(infl, delta, xl) * xl * xl * vol[col[b]];
    }
    m[i] = s;
  }
}

/* Denominator of Eq 1.31: D_i = sum_j w V_j over the built family. */
void orc_damage_denominator(int64_t n, int dim, const double* x, const double* y, const double* z,
                            const double* vol, const int64_t* row_ptr, const int32_t* col, int infl,
                            double delta, double* D) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
      double xi[3];
      double xl = bond_vector(dim, x, y, z, i, col[b], xi);
      s += influence(infl, delta, xl) * vol[col[b]];
    }
    D[i] = s;
  }
}

/* Dilatation theta_i = (A / m_i) sum_j w x_ij e_ij V_j rho_ij (Eq 1.6 discretized; the sum over all
 * bonds of the per-bond contributions of Eq 2.3).  A particle with m_i = 0 has no bonds: theta_i = 0. */
void orc_dilatation(int kin, int64_t n, int dim, const double* x, const double* y, const double* z,
                    const double* vol, const int64_t* row_ptr, const int32_t* col,
                    const uint8_t* status, const double* m, double A, int infl, double delta,
                    const double* ux, const double* uy, const double* uz, double* theta) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
      if (!status[b]) continue;
      int64_t j = col[b];
      double xi[3];
      double M[3];
      double xl = bond_vector(dim, x, y, z, i, j, xi);
      double e = bond_kinematics(kin, dim, xi, xl, ux, uy, uz, i, j, M);
      s += influence(infl, delta, xl) * xl * e * vol[j];
    }
    theta[i] = (m[i] > 0.0) ? A * s / m[i] : 0.0;
  }
}

/* Internal force on every particle: F_i = sum_j F_i^{xi_ij} with (Eq 2.2)
 *   F_i^{xi_ij} = [ (K - G/3) theta~_ij x_ij + G e~_ij ] w M_ij V_i V_j rho_ij,
 *   theta~_ij = theta_i / m_i + theta_j / m_j,   e~_ij = e_ij / m_i + e_ij / m_j.
 * F points from i towards j for a stretched bond (Appendix B adds it to the external force). */
void orc_force(int kin, int64_t n, int dim, const double* x, const double* y, const double* z,
               const double* vol, const int64_t* row_ptr, const int32_t* col,
               const uint8_t* status, const double* m, const double* theta, double K, double G,
               int infl, double delta, const double* ux, const double* uy, const double* uz,
               double* fx, double* fy, double* fz) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double f[3] = {0.0, 0.0, 0.0};
    for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
      if (!status[b]) continue;
      int64_t j = col[b];
      double xi[3];
      double M[3];
      double xl = bond_vector(dim, x, y, z, i, j, xi);
      double e = bond_kinematics(kin, dim, xi, xl, ux, uy, uz, i, j, M);
      double th = theta[i] / m[i] + theta[j] / m[j];
      double et = e / m[i] + e / m[j];
      double mag = ((K - G / 3.0) * th * xl + G * et) * influence(infl, delta, xl) * vol[i] * vol[j];
      for (int k = 0; k < dim; ++k) f[k] += mag * M[k];
    }
    fx[i] = f[0];
    fy[i] = f[1];
    if (dim == 3) fz[i] = f[2];
  }
}

/* Failure criterion (Eqs 1.17, 1.30): stretch s_ij = e_ij / x_ij; an intact bond breaks for good when
 * s_ij >= s0.  Returns the number of bonds broken by this call; *min_margin receives
 * min |s_ij - s0| / s0 over the bonds that are still intact afterwards (1e300 if there are none). */
int64_t orc_failure(int kin, int64_t n, int dim, const double* x, const double* y, const double* z,
                    const int64_t* row_ptr, const int32_t* col, uint8_t* status, double s0,
                    const double* ux, const double* uy, const double* uz, double* min_margin) {
  int64_t broken = 0;
  double mm = 1e300;
#pragma omp parallel for schedule(static) reduction(+ : broken) reduction(min : mm)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
      if (!status[b]) continue;
      int64_t j = col[b];
      double xi[3];
      double M[3];
      double xl = bond_vector(dim, x, y, z, i, j, xi);
      double s = bond_kinematics(kin, dim, xi, xl, ux, uy, uz, i, j, M) / xl;
      if (s >= s0) {
        status[b] = 0;
        ++broken;
      } else {
        double r = fabs(s - s0) / s0;
        if (r < mm) mm = r;
      }
    }
  }
  *min_margin = mm;
  return broken;
}

/* Damage phi_i = 1 - sum_j w rho_ij V_j / sum_j w V_j over the built family (Eq 1.31); 0 without bonds. */
void orc_damage(int64_t n, int dim, const double* x, const double* y, const double* z,
                const double* vol, const int64_t* row_ptr, const int32_t* col,
                const uint8_t* status, int infl, double delta, double* phi) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double num = 0.0, den = 0.0;
    for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
      double xi[3];
      double xl = bond_vector(dim, x, y, z, i, col[b], xi);
      double wv = influence(infl, delta, xl) * vol[col[b]];
      den += wv;
      if (status[b]) num += wv;
    }
    phi[i] = (den > 0.0) ? 1.0 - num / den : 0.0;
  }
}

/* Boundary conditions (Appendix B applies them at the top of each iteration and moves only the free
 * degrees of freedom).  flag: 0 free, 1 fixed (u = v = 0), 2 prescribed rigid rotation about the axis
 * through c with unit direction a at angle phi(t) = rate * t, linearized: u = phi(t) a x (p - c),
 * v = rate a x (p - c). */
static void bc_value(int dim, const double* x, const double* y, const double* z, int64_t i,
                     uint8_t flag, const double c[3], const double a[3], double rate, double t,
                     double u[3], double v[3]) {
  u[0] = u[1] = u[2] = v[0] = v[1] = v[2] = 0.0;
  if (flag != ORC_PRESCRIBED) return;
  double r[3] = {x[i] - c[0], y[i] - c[1], (dim == 3 ? z[i] : 0.0) - c[2]};
  double g[3] = {a[1] * r[2] - a[2] * r[1], a[2] * r[0] - a[0] * r[2], a[0] * r[1] - a[1] * r[0]};
  for (int k = 0; k < 3; ++k) {
    v[k] = rate * g[k];
    u[k] = rate * t * g[k];
  }
}

/* vp (may be NULL): a prescribed velocity per particle (3 arrays) that replaces the rotation:
 * u = t vp_i, v = vp_i (a constant velocity applied to the impacted nodes, as in Section 4.3). */
static void apply_bc(int64_t n, int dim, const double* x, const double* y, const double* z,
                     const uint8_t* flag, const double c[3], const double a[3], double rate, double t,
                     double* ux, double* uy, double* uz, double* vx, double* vy, double* vz,
                     const double* const* vp) {
  if (!flag) return;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    if (flag[i] == ORC_FREE) continue;
    double u[3], v[3];
    bc_value(dim, x, y, z, i, flag[i], c, a, rate, t, u, v);
    if (vp && flag[i] == ORC_PRESCRIBED)
      for (int k = 0; k < 3; ++k) {
        v[k] = vp[k] ? vp[k][i] : 0.0;
        u[k] = t * v[k];
      }
    ux[i] = u[0];
    uy[i] = u[1];
    vx[i] = v[0];
    vy[i] = v[1];
    if (dim == 3) {
      uz[i] = u[2];
      vz[i] = v[2];
    }
  }
}

/* ------------------------------------------------------------------------------------------------
 * Explicit dynamics (Section 3.2, Eq 2.11, and the solver loop of Appendix B), one call = nsteps
 * iterations starting at step index step0 (time t_n = n dt).  Each iteration n:
 *   1. boundary conditions at t_n on the constrained particles;
 *   2. theta from u^n and the current bond status (Eq 1.6);
 *   3. internal forces from u^n and theta (Eq 2.2);
 *   4. v^{n+1} = v^n + dt (F_i + b_i V_i) / (rho V_i),  u^{n+1} = u^n + dt v^{n+1} for the free particles
 *      (Eqs 2.1, 2.11, 2.12 with the diagonal mass rho V_i); constrained particles take their
 *      boundary value at t_{n+1}, so the failure check below sees a single time level;
 *   5. failure criterion on u^{n+1} (Eq 1.30), when s0 > 0.
 * margins[k] (may be NULL) receives the minimum relative stretch margin after iteration k, and
 * broken[k] (may be NULL) the number of bonds broken in it.  theta holds the last iteration's
 * dilatation on return; fx/fy/fz its internal force.  b* may be NULL (no body force).
 * ---------------------------------------------------------------------------------------------- */
void orc_run(int kin, int infl, double delta, int64_t n, int dim, const double* x, const double* y,
             const double* z, const double* vol, const int64_t* row_ptr, const int32_t* col, uint8_t* status,
             const double* m, double A, double K, double G, double rho, double dt, double s0,
             const uint8_t* flag, const double* bx, const double* by, const double* bz,
             const double* axis_point, const double* axis_dir, double rate, const double* vpx,
             const double* vpy, const double* vpz, int64_t step0, int64_t nsteps, double* ux,
             double* uy, double* uz, double* vx, double* vy, double* vz, double* theta, double* fx,
             double* fy, double* fz, double* margins, int64_t* broken) {
  const double* vpa[3] = {vpx, vpy, vpz};
  const double* const* vp = vpx ? vpa : NULL;
  double c[3] = {0, 0, 0}, a[3] = {0, 0, 0};
  if (axis_point)
    for (int k = 0; k < 3; ++k) c[k] = axis_point[k];
  if (axis_dir)
    for (int k = 0; k < 3; ++k) a[k] = axis_dir[k];
  for (int64_t s = 0; s < nsteps; ++s) {
    int64_t step = step0 + s;
    double tn = (double)step * dt, tn1 = (double)(step + 1) * dt;
    apply_bc(n, dim, x, y, z, flag, c, a, rate, tn, ux, uy, uz, vx, vy, vz, vp);
    orc_dilatation(kin, n, dim, x, y, z, vol, row_ptr, col, status, m, A, infl, delta, ux, uy, uz, theta);
    orc_force(kin, n, dim, x, y, z, vol, row_ptr, col, status, m, theta, K, G, infl, delta, ux, uy, uz, fx, fy,
              fz);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      if (flag && flag[i] != ORC_FREE) continue;
      double f[3] = {fx[i], fy[i], dim == 3 ? fz[i] : 0.0};
      double b[3] = {bx ? bx[i] : 0.0, by ? by[i] : 0.0, (dim == 3 && bz) ? bz[i] : 0.0};
      double* v[3] = {vx, vy, vz};
      double* u[3] = {ux, uy, uz};
      for (int k = 0; k < dim; ++k) {
        double acc = (f[k] + b[k] * vol[i]) / (rho * vol[i]);
        v[k][i] = v[k][i] + dt * acc;
        u[k][i] = u[k][i] + dt * v[k][i];
      }
    }
    apply_bc(n, dim, x, y, z, flag, c, a, rate, tn1, ux, uy, uz, vx, vy, vz, vp);
    double mm = 1e300;
    int64_t nb = 0;
    if (s0 > 0.0) nb = orc_failure(kin, n, dim, x, y, z, row_ptr, col, status, s0, ux, uy, uz, &mm);
    if (margins) margins[s] = mm;
    if (broken) broken[s] = nb;
  }
}

/* ------------------------------------------------------------------------------------------------
 * Adaptive dynamic relaxation (the quasi-static solver of Section 4.4, which cites Underwood 1983 and
 * Kilic & Madenci 2010 for it).  The static problem f(u) + b = 0 (f = F_i / V_i, the internal force
 * density) is solved as the damped fictitious dynamics  L u'' + c L u' = f(u) + b  with a diagonal
 * fictitious density L = diag(lambda_i), fictitious time step 1, and the damping c re-estimated every
 * iteration from a Rayleigh quotient of the local (diagonal) stiffness.
 * ---------------------------------------------------------------------------------------------- */

/* Fictitious density lambda_i = (1/4) R_i (time step 1), where R_i bounds the absolute row sums of
 * the stiffness of the force density, |d f_ia / d u_kb| summed over k, b, for every component a
 * (Gerschgorin: then every eigenvalue of L^-1 K is at most 4 and the unit step is stable).  For the
 * linearized force of Eq 2.2, with |M_ij|_1 = |xi_ij|_1 / |xi_ij| and
 *   alpha_i = (A / m_i) sum_l |xi_il| V_l |M_il|_1        (bound of sum |d theta_i / d u|, halved),
 *   R_i = 2 G sum_j (1/m_i + 1/m_j) V_j |M_ij|_1 + 2 |K - G/3| sum_j |xi_ij| V_j (alpha_i/m_i + alpha_j/m_j),
 * the first term from the extension part and the second from the dilatation part; sums over the
 * built family.  K, G, A per particle (a body's constants). */
void orc_adr_lambda(int64_t n, int dim, const double* x, const double* y, const double* z,
                    const double* vol, const int64_t* row_ptr, const int32_t* col, const double* m,
                    const double* A, const double* K, const double* G, double* lambda) {
  double* alpha = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
      double xi[3];
      double xl = bond_vector(dim, x, y, z, i, col[b], xi);
      double m1 = (fabs(xi[0]) + fabs(xi[1]) + fabs(xi[2])) / xl;
      s += xl * vol[col[b]] * m1;
    }
    alpha[i] = (m[i] > 0.0) ? A[i] * s / m[i] : 0.0;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double rg = 0.0, rt = 0.0;
    for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
      int64_t j = col[b];
      double xi[3];
      double xl = bond_vector(dim, x, y, z, i, j, xi);
      double m1 = (fabs(xi[0]) + fabs(xi[1]) + fabs(xi[2])) / xl;
      rg += (1.0 / m[i] + 1.0 / m[j]) * vol[j] * m1;
      rt += xl * vol[j] * (alpha[i] / m[i] + alpha[j] / m[j]);
    }
    double R = 2.0 * G[i] * rg + 2.0 * fabs(K[i] - G[i] / 3.0) * rt;
    lambda[i] = 0.25 * R;
  }
  free(alpha);
}

/* ADR iterations.  Iteration n (fictitious time step 1; boundary values at t_n = n dt as in orc_run):
 *   1. boundary conditions at t_n;
 *   2. g^n = f(u^n) + b (force density: internal force / V_i plus the body-force density);
 *   3. damping: c^n = 2 sqrt( sum u.(k u) / sum u.u ) over the free particles' components, with the
 *      local stiffness k_ia = -(g_ia^n - g_ia^{n-1}) / (lambda_i v_ia^{n-1/2}) (0 where v_ia = 0);
 *      c^n = 0 when the quotient is not positive or sum u.u = 0;
 *   4. free particles: v^{n+1/2} = ((2 - c^n) v^{n-1/2} + 2 g^n / lambda_i) / (2 + c^n), except on the
 *      first iteration of a run (first != 0), which starts from rest: v^{1/2} = g^0 / (2 lambda_i);
 *      a particle without bonds (lambda_i = 0, no stiffness) is held in place (v = 0);
 *      u^{n+1} = u^n + v^{n+1/2};  constrained particles take their boundary value at t_{n+1};
 *   5. failure check on u^{n+1} (Eq 1.30), when s0 > 0.
 * v holds v^{n-1/2} on entry and g_prev (3 arrays) the previous g; both are updated.  damping[k]
 * (may be NULL) receives c of iteration k. */
void orc_adr_run(int kin, int64_t n, int dim, const double* x, const double* y, const double* z,
                 const double* vol, const int64_t* row_ptr, const int32_t* col, uint8_t* status,
                 const double* m, const double* A, const double* K, const double* G,
                 const double* lambda, double s0, const uint8_t* flag, const double* bx,
                 const double* by, const double* bz, const double* axis_point, const double* axis_dir,
                 double rate, double dt, int64_t step0, int64_t nsteps, int first, double* ux,
                 double* uy, double* uz, double* vx, double* vy, double* vz, double* gx, double* gy,
                 double* gz, double* theta, double* fx, double* fy, double* fz, double* damping,
                 double* margins, int64_t* broken) {
  double c[3] = {0, 0, 0}, a[3] = {0, 0, 0};
  if (axis_point)
    for (int k = 0; k < 3; ++k) c[k] = axis_point[k];
  if (axis_dir)
    for (int k = 0; k < 3; ++k) a[k] = axis_dir[k];
  double* u[3] = {ux, uy, uz};
  double* v[3] = {vx, vy, vz};
  double* gp[3] = {gx, gy, gz};
  double* f[3] = {fx, fy, fz};
  const double* bb[3] = {bx, by, bz};
  for (int64_t s = 0; s < nsteps; ++s) {
    int64_t step = step0 + s;
    double tn = (double)step * dt, tn1 = (double)(step + 1) * dt;
    apply_bc(n, dim, x, y, z, flag, c, a, rate, tn, ux, uy, uz, vx, vy, vz, NULL);
    /* theta and internal forces with per-particle constants: one call per distinct (A, K, G) would
     * do, but bodies are independent, so the per-particle form below is the same sum. */
    for (int64_t i = 0; i < n; ++i) theta[i] = 0.0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double sum = 0.0;
      for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
        if (!status[b]) continue;
        int64_t j = col[b];
        double xi[3], M[3];
        double xl = bond_vector(dim, x, y, z, i, j, xi);
        sum += xl * bond_kinematics(kin, dim, xi, xl, ux, uy, uz, i, j, M) * vol[j];
      }
      theta[i] = (m[i] > 0.0) ? A[i] * sum / m[i] : 0.0;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double fi[3] = {0.0, 0.0, 0.0};
      for (int64_t b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
        if (!status[b]) continue;
        int64_t j = col[b];
        double xi[3], M[3];
        double xl = bond_vector(dim, x, y, z, i, j, xi);
        double e = bond_kinematics(kin, dim, xi, xl, ux, uy, uz, i, j, M);
        double th = theta[i] / m[i] + theta[j] / m[j];
        double et = e / m[i] + e / m[j];
        double mag = ((K[i] - G[i] / 3.0) * th * xl + G[i] * et) * vol[j];  /* per unit V_i */
        for (int k = 0; k < dim; ++k) fi[k] += mag * M[k];
      }
      for (int k = 0; k < dim; ++k) f[k][i] = fi[k] + (bb[k] ? bb[k][i] : 0.0);
    }
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if ((flag && flag[i] != ORC_FREE) || !(lambda[i] > 0.0)) continue;
      for (int k = 0; k < dim; ++k) {
        double kk = 0.0;
        if (v[k][i] != 0.0) kk = -(f[k][i] - gp[k][i]) / (lambda[i] * v[k][i]);
        num += u[k][i] * kk * u[k][i];
        den += u[k][i] * u[k][i];
      }
    }
    double cn = (den > 0.0 && num > 0.0) ? 2.0 * sqrt(num / den) : 0.0;
    int start = first && s == 0;
    if (damping) damping[s] = start ? 0.0 : cn;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      if (flag && flag[i] != ORC_FREE) continue;
      if (!(lambda[i] > 0.0)) {  /* no bonds, no stiffness: held in place */
        for (int k = 0; k < dim; ++k) v[k][i] = 0.0;
        continue;
      }
      for (int k = 0; k < dim; ++k) {
        if (start)
          v[k][i] = f[k][i] / (2.0 * lambda[i]);
        else
          v[k][i] = ((2.0 - cn) * v[k][i] + 2.0 * f[k][i] / lambda[i]) / (2.0 + cn);
        u[k][i] = u[k][i] + v[k][i];
      }
    }
    for (int k = 0; k < dim; ++k)
      for (int64_t i = 0; i < n; ++i) gp[k][i] = f[k][i];
    apply_bc(n, dim, x, y, z, flag, c, a, rate, tn1, ux, uy, uz, vx, vy, vz, NULL);
    double mm = 1e300;
    int64_t nb = 0;
    if (s0 > 0.0) nb = orc_failure(kin, n, dim, x, y, z, row_ptr, col, status, s0, ux, uy, uz, &mm);
    if (margins) margins[s] = mm;
    if (broken) broken[s] = nb;
  }
}

/* ------------------------------------------------------------------------------------------------
 * pdref_*: the oracle behind the same call sequence as the GPU library's C ABI (create, build the
 * family, boundary conditions, state, step, read back), so one harness can drive both.  The
 * parameter and crack blocks have the GPU library's field layout, declared here on their own.
 * Single body, explicit solver; every computation is one of the functions above.  Status codes:
 * 0 ok, -1 bad argument, -2 call out of order.
 * ---------------------------------------------------------------------------------------------- */
typedef struct {
  int32_t model, precision;
  double E, nu, rho, horizon, s0, dt, band_safety;
  int32_t device, ordering;
  void* stream;
  int32_t kinematics, reserved;
} pdref_params;

typedef struct {
  double p0[3], p1[3], p2[3];
  int32_t body, reserved;
} pdref_crack;

typedef struct pdref_ctx {
  int64_t n;
  int dim, model, kin, built;
  double rho, delta, s0, dt, A, K, G, kappa, mu;
  double *x, *y, *z, *vol;
  int64_t* row_ptr;
  int32_t* col;
  uint8_t* status;
  double *m, *u[3], *v[3], *theta, *f[3], *b[3];
  uint8_t* flag;
  double axis_point[3], axis_dir[3], rate;
  int64_t steps;
} pdref_ctx;

static double* pdref_copy(const double* a, int64_t n) {
  double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (a) memcpy(p, a, sizeof(double) * (size_t)n);
  else memset(p, 0, sizeof(double) * (size_t)(n > 0 ? n : 1));
  return p;
}

void pdref_destroy(pdref_ctx* c) {
  if (!c) return;
  free(c->x); free(c->y); free(c->z); free(c->vol);
  free(c->row_ptr); free(c->col); free(c->status); free(c->m); free(c->theta); free(c->flag);
  for (int k = 0; k < 3; ++k) {
    free(c->u[k]); free(c->v[k]); free(c->f[k]); free(c->b[k]);
  }
  free(c);
}

int pdref_create_particles(pdref_ctx** out, const pdref_params* p, int64_t n, const double* x,
                           const double* y, const double* z, const double* vol) {
  if (!out || !p || !x || !y || !vol || n < 1) return -1;
  if (p->model < 0 || p->model > 2 || (p->model == ORC_3D) != (z != NULL)) return -1;
  pdref_ctx* c = (pdref_ctx*)calloc(1, sizeof(pdref_ctx));
  c->n = n;
  c->dim = z ? 3 : 2;
  c->model = p->model;
  c->kin = p->kinematics;
  c->rho = p->rho;
  c->delta = p->horizon;
  c->s0 = p->s0;
  c->dt = p->dt;
  orc_constants(p->model, p->E, p->nu, &c->A, &c->K, &c->G, &c->kappa, &c->mu);
  c->x = pdref_copy(x, n);
  c->y = pdref_copy(y, n);
  c->z = z ? pdref_copy(z, n) : NULL;
  c->vol = pdref_copy(vol, n);
  for (int k = 0; k < 3; ++k) {
    c->u[k] = pdref_copy(NULL, n);
    c->v[k] = pdref_copy(NULL, n);
    c->f[k] = pdref_copy(NULL, n);
  }
  c->theta = pdref_copy(NULL, n);
  *out = c;
  return 0;
}

int pdref_build_neighbors(pdref_ctx* c, const pdref_crack* cracks, int32_t ncracks) {
  if (!c || ncracks < 0 || (ncracks > 0 && !cracks)) return -1;
  double* cr = (double*)malloc(sizeof(double) * 9 * (size_t)(ncracks > 0 ? ncracks : 1));
  for (int32_t k = 0; k < ncracks; ++k)
    for (int t = 0; t < 3; ++t) {
      cr[9 * k + t] = cracks[k].p0[t];
      cr[9 * k + 3 + t] = cracks[k].p1[t];
      cr[9 * k + 6 + t] = cracks[k].p2[t];
    }
  int64_t* counts = (int64_t*)calloc((size_t)c->n, sizeof(int64_t));
  orc_family_binned(c->n, c->dim, c->x, c->y, c->z ? c->z : c->x, c->delta, ncracks, cr, counts, NULL, NULL);
  free(c->row_ptr); free(c->col); free(c->status); free(c->m);
  c->row_ptr = (int64_t*)calloc((size_t)c->n + 1, sizeof(int64_t));
  for (int64_t i = 0; i < c->n; ++i) c->row_ptr[i + 1] = c->row_ptr[i] + counts[i];
  int64_t nb = c->row_ptr[c->n];
  c->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nb > 0 ? nb : 1));
  orc_family_binned(c->n, c->dim, c->x, c->y, c->z ? c->z : c->x, c->delta, ncracks, cr, counts, c->row_ptr,
                    c->col);
  c->status = (uint8_t*)malloc((size_t)(nb > 0 ? nb : 1));
  memset(c->status, 1, (size_t)(nb > 0 ? nb : 1));
  c->m = pdref_copy(NULL, c->n);
  orc_weighted_volume(c->n, c->dim, c->x, c->y, c->z ? c->z : c->x, c->vol, c->row_ptr, c->col, ORC_W_ONE, 0.0,
                      c->m);
  free(counts);
  free(cr);
  c->built = 1;
  return 0;
}

int pdref_set_bc(pdref_ctx* c, const uint8_t* flag, const double* b, const double* axis_point,
                 const double* axis_dir, double rate) {
  if (!c) return -1;
  if (!c->built) return -2;
  free(c->flag);
  c->flag = NULL;
  if (flag) {
    c->flag = (uint8_t*)malloc((size_t)c->n);
    memcpy(c->flag, flag, (size_t)c->n);
  }
  for (int k = 0; k < 3; ++k) {
    free(c->b[k]);
    c->b[k] = (b && k < c->dim) ? pdref_copy(b + (int64_t)k * c->n, c->n) : NULL;
    c->axis_point[k] = axis_point ? axis_point[k] : 0.0;
    c->axis_dir[k] = axis_dir ? axis_dir[k] : 0.0;
  }
  c->rate = rate;
  return 0;
}

int pdref_set_state(pdref_ctx* c, const double* u, const double* v) {
  if (!c || !u) return -1;
  if (!c->built) return -2;
  for (int k = 0; k < c->dim; ++k) {
    memcpy(c->u[k], u + (int64_t)k * c->n, sizeof(double) * (size_t)c->n);
    if (v) memcpy(c->v[k], v + (int64_t)k * c->n, sizeof(double) * (size_t)c->n);
    else memset(c->v[k], 0, sizeof(double) * (size_t)c->n);
  }
  return 0;
}

int pdref_step(pdref_ctx* c, int64_t nsteps) {
  if (!c || nsteps < 0) return -1;
  if (!c->built) return -2;
  const double* zz = c->z ? c->z : c->x;
  orc_run(c->kin, ORC_W_ONE, 0.0, c->n, c->dim, c->x, c->y, zz, c->vol, c->row_ptr, c->col, c->status, c->m, c->A, c->K,
          c->G, c->rho, c->dt, c->s0, c->flag, c->b[0], c->b[1], c->b[2], c->axis_point, c->axis_dir,
          c->rate, NULL, NULL, NULL, c->steps, nsteps, c->u[0], c->u[1], c->u[2], c->v[0], c->v[1], c->v[2], c->theta,
          c->f[0], c->f[1], c->f[2], NULL, NULL);
  c->steps += nsteps;
  return 0;
}

int pdref_get_state(pdref_ctx* c, double* u, double* v, double* theta) {
  if (!c) return -1;
  if (!c->built) return -2;
  for (int k = 0; k < c->dim; ++k) {
    if (u) memcpy(u + (int64_t)k * c->n, c->u[k], sizeof(double) * (size_t)c->n);
    if (v) memcpy(v + (int64_t)k * c->n, c->v[k], sizeof(double) * (size_t)c->n);
  }
  if (theta) memcpy(theta, c->theta, sizeof(double) * (size_t)c->n);
  return 0;
}

int pdref_get_damage(pdref_ctx* c, double* phi) {
  if (!c || !phi) return -1;
  if (!c->built) return -2;
  orc_damage(c->n, c->dim, c->x, c->y, c->z ? c->z : c->x, c->vol, c->row_ptr, c->col, c->status, ORC_W_ONE, 0.0,
             phi);
  return 0;
}

int pdref_num_bonds(pdref_ctx* c, int64_t* nbonds) {
  if (!c || !nbonds) return -1;
  if (!c->built) return -2;
  *nbonds = c->row_ptr[c->n];
  return 0;
}

int pdref_get_neighbors(pdref_ctx* c, int64_t* row_ptr, int32_t* col, uint8_t* intact) {
  if (!c || !row_ptr || !col) return -1;
  if (!c->built) return -2;
  int64_t nb = c->row_ptr[c->n];
  memcpy(row_ptr, c->row_ptr, sizeof(int64_t) * (size_t)(c->n + 1));
  memcpy(col, c->col, sizeof(int32_t) * (size_t)nb);
  if (intact) memcpy(intact, c->status, (size_t)nb);
  return 0;
}
