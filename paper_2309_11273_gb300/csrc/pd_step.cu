// Per-time-step kernels of linearized OSB-PD and their launch sequence.
//
// One time step = two kernels over the sliced neighbour layout built in pd_build.cu:
//   pass 1: failure criterion on u^n (Eqs 1.17, 1.30: the paper's failure block after the previous
//           update), then the dilatation theta_i = (A/m_i) sum_j V_j rho_ij xi.(u_j - u_i)
//           (Eq 1.6 with x e = xi.(u_j - u_i) for the linearized extension of Eqs 2.4, 2.7);
//   pass 2: the bond forces of Eq 2.2 summed over the family,
//           F_i / V_i = sum_j rho_ij V_j [ (K - G/3)(theta_i/m_i + theta_j/m_j)
//                                         + G (1/m_i + 1/m_j) xi.(u_j - u_i) / |xi|^2 ] xi,
//           followed by the explicit update of Eq 2.11 and the boundary conditions (Appendix B).
// Both passes gather: every directed bond is visited from its own particle and every sum runs in a
// fixed order, with no floating-point atomics.  A warp owns one 32-particle slice (one particle
// per lane); with SPLIT > 1 several warps share a slice, each taking every SPLIT-th slot, and
// their partial sums are combined in shared memory in a fixed order.  The tabled FP64 kernels run
// pass 1 in a pair form by default: its first kernel forms each bond's extension once, at the entry
// that owns the bond, and writes it to both entries (the other entry's status bit is cleared with
// an atomic AND); its second kernel forms the dilatation sums.
//
// The break test is evaluated without square roots: s = e/|xi| >= s0  <=>  xi.du >= s0 |xi|^2.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "pd_internal.h"
#include "pd_order.h"
#include "pd_lattice.h"

namespace pd {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct SliceIdx {
  int64_t i;
  int64_t base;
  int W;
  int lane;
  int sub;
  bool active;
};

template <int SPLIT>
__device__ __forceinline__ SliceIdx slice_index(int64_t n_pad, const int64_t* __restrict__ slice_ptr) {
  SliceIdx r;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  r.lane = threadIdx.x & 31;
  r.sub = (int)(gwarp % SPLIT);
  const int64_t s = gwarp / SPLIT;
  r.i = s * 32 + r.lane;
  r.active = r.i < n_pad;  // n_pad is a multiple of 32: uniform over the warp
  r.base = 0;
  r.W = 0;
  if (r.active) {
    r.base = slice_ptr[s];
    r.W = (int)((slice_ptr[s + 1] - r.base) >> 5);
  }
  return r;
}

// Partial sums of the SPLIT warps sharing a slice, combined by the first warp (fixed order).
template <int SPLIT, int NC, class T>
__device__ __forceinline__ void split_reduce(T (&v)[NC]) {
  if (SPLIT == 1) return;
  extern __shared__ unsigned char smem_raw[];
  T* red = reinterpret_cast<T*>(smem_raw);
#pragma unroll
  for (int c = 0; c < NC; ++c) red[c * blockDim.x + threadIdx.x] = v[c];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w % SPLIT == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T s = red[c * blockDim.x + w * 32 + lane];
#pragma unroll
      for (int q = 1; q < SPLIT; ++q) s += red[c * blockDim.x + (w + q) * 32 + lane];
      v[c] = s;
    }
  }
}

// xi = x_j - x_i, du = u_j - u_i, d = xi . du, q = xi . xi in FP64.  Shared by the FP64 path and by
// the FP64 re-decision of the mixed path, so both decide a bond with identical arithmetic.
template <int DIM>
__device__ __forceinline__ void bond_f64(const double4& pi, const double4& pj, const double4& ui,
                                         const double4& uj, double& ex, double& ey, double& ez,
                                         double& d, double& q) {
  ex = pj.x - pi.x;
  ey = pj.y - pi.y;
  const double dx = uj.x - ui.x, dy = uj.y - ui.y;
  d = ex * dx + ey * dy;
  q = ex * ex + ey * ey;
  if (DIM == 3) {
    ez = pj.z - pi.z;
    const double dz = uj.z - ui.z;
    d = fma(ez, dz, d);
    q = fma(ez, ez, q);
  } else {
    ez = 0.0;
  }
}

// FP64 decision of one bond.  Out of line for the general mixed kernels, which call it only for the
// few bonds inside their rounding band; inlined into the lattice kernel's slow path (fewer registers
// held across a call in its hot loop).
template <int DIM>
__device__ __forceinline__ bool fp64_breaks_inl(const StepArgs& a, int64_t i, int32_t j,
                                                const double4* __restrict__ disp, double s0) {
  double ex, ey, ez, d, q;
  bond_f64<DIM>(a.pos[i], a.pos[j], disp[i], disp[j], ex, ey, ez, d, q);
  return d >= s0 * q;
}
template <int DIM>
__device__ __noinline__ bool fp64_breaks(const StepArgs& a, int64_t i, int32_t j,
                                         const double4* __restrict__ disp, double s0) {
  return fp64_breaks_inl<DIM>(a, i, j, disp, s0);
}

// Nonlinear FP64 re-decision for the mixed path: |Y|^2 - |xi|^2 >= s0 (2 + s0) |xi|^2 with the
// arithmetic of the FP64 nonlinear kernels (defined with them below).
template <int DIM>
__device__ __noinline__ bool fp64_breaks_nl(const StepArgs& a, int64_t i, int32_t j,
                                            const double4* __restrict__ disp);

// Explicit update (Eq 2.11) with the diagonal mass rho V_i (Eqs 2.1, 2.12) and the boundary
// conditions at t_{n+1}; f = F_i / V_i.
__device__ __forceinline__ void update(const StepArgs& a, int64_t i, int b, const double f[3],
                                       const double4* __restrict__ disp, double4* __restrict__ disp_out,
                                       double4& u) {
  const BodyDev& bp = a.bp[b];
  if (a.adr) {  // adaptive dynamic relaxation: k_adr_update moves the particles after the reduction
    const double4 bb = a.bacc ? a.bacc[i] : make_double4(0.0, 0.0, 0.0, 0.0);
    a.gnew[i] = make_double4(f[0] + bb.x, f[1] + bb.y, f[2] + bb.z, 0.0);
    u = disp[i];
    return;
  }
  const uint8_t fl = a.flag ? a.flag[i] : (uint8_t)0;
  u = disp[i];
  double4 v = a.vel[i];
  if (fl == 0) {
    const double4 bb = a.bacc ? a.bacc[i] : make_double4(0.0, 0.0, 0.0, 0.0);
    v.x = v.x + bp.dt * ((f[0] + bb.x) * bp.inv_rho);
    v.y = v.y + bp.dt * ((f[1] + bb.y) * bp.inv_rho);
    v.z = v.z + bp.dt * ((f[2] + bb.z) * bp.inv_rho);
    u.x = u.x + bp.dt * v.x;
    u.y = u.y + bp.dt * v.y;
    u.z = u.z + bp.dt * v.z;
  } else if (fl == 1) {
    u = make_double4(0.0, 0.0, 0.0, u.w);
    v = make_double4(0.0, 0.0, 0.0, 0.0);
  } else {
    const double t1 = (double)(*a.d_step + 1) * bp.dt;
    const double4 g = a.gvec[i];
    const double rt = bp.rate * t1;
    u = make_double4(rt * g.x, rt * g.y, rt * g.z, u.w);
    v = make_double4(bp.rate * g.x, bp.rate * g.y, bp.rate * g.z, 0.0);
  }
  disp_out[i] = u;  // .w carries V_i unchanged
  a.vel[i] = v;
}

// Slot batches: each thread handles U slots per iteration; the neighbour indices and status words
// of the next batch are loaded while the current batch's gathers are in flight, so that several
// dependent index -> gather chains overlap.
template <int U, int SPLIT>
__device__ __forceinline__ void load_slots(const SliceIdx& t, const int32_t* __restrict__ cl,
                                           const uint32_t* __restrict__ bw, int k0, int32_t (&j)[U],
                                           uint32_t (&wd)[U]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int k = k0 + u * SPLIT;
    const bool ok = k < t.W;
    j[u] = ok ? cl[(int64_t)k << 5] : (int32_t)t.i;  // past the row: the particle itself, status 0
    wd[u] = ok ? bw[k] : 0u;
  }
}

// ------------------------------------------------------------------------------------ FP64 path
constexpr int kU64 = 2;
constexpr int kU32 = 4;

// Plain FP64 kernels: the reference geometry of each bond is recomputed from the coordinates.
template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass1_f64(StepArgs a, const double4* __restrict__ disp,
                                                    int write_theta) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  if (write_theta && blockIdx.x == 0 && threadIdx.x == 0) *a.d_step += 1;
  double acc[1] = {0.0};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const double s0 = a.bp[b].s0;
    const bool can_break = a.bp[b].breaks != 0;
    const double4 pi = a.pos[t.i], ui = disp[t.i];
    uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    constexpr int U = kU64;
    int32_t jn[U];
    uint32_t wn[U];
    load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      uint32_t wd[U];
      double4 pj[U], uj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        wd[u] = wn[u];
        pj[u] = a.pos[jn[u]];
        uj[u] = disp[jn[u]];
      }
      load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        double ex, ey, ez, d, q;
        bond_f64<DIM>(pi, pj[u], ui, uj[u], ex, ey, ez, d, q);
        bool intact = (wd[u] >> t.lane) & 1u;
        if (a.check) {
          const bool brk = intact && can_break && d >= s0 * q;
          const unsigned m = __ballot_sync(kFull, brk);
          if (m) {
            intact = intact && !brk;
            if (t.lane == 0) bw[k0 + u * SPLIT] = wd[u] & ~m;
          }
        }
        acc[0] = fma(intact ? pj[u].w : 0.0, d, acc[0]);
      }
    }
  }
  split_reduce<SPLIT, 1>(acc);
  if (t.active && t.sub == 0 && write_theta) {
    const double th = a.aA[t.i] * acc[0];
    const double mu = a.mu[t.i];
    a.theta[t.i] = th;
    // gathered by pass 2: (K - G/3) theta_i / m_i and G / m_i
    a.thm[t.i] = make_double2(a.bp[b].Kp * (th * mu), a.bp[b].G * mu);
  }
}

template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass2_f64(StepArgs a, const double4* __restrict__ disp,
                                                    double4* __restrict__ disp_out) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  double f[3] = {0.0, 0.0, 0.0};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const double4 pi = a.pos[t.i], ui = disp[t.i];
    const double2 ti = a.thm[t.i];
    const uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    constexpr int U = kU64;
    int32_t jn[U];
    uint32_t wn[U];
    load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      uint32_t wd[U];
      double4 pj[U], uj[U];
      double2 tj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        wd[u] = wn[u];
        pj[u] = a.pos[jn[u]];
        uj[u] = disp[jn[u]];
        tj[u] = a.thm[jn[u]];
      }
      load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        double ex, ey, ez, d, q;
        bond_f64<DIM>(pi, pj[u], ui, uj[u], ex, ey, ez, d, q);
        // Eq 2.2: [(K - G/3)(theta_i/m_i + theta_j/m_j) + G (1/m_i + 1/m_j) xi.du / |xi|^2] V_j xi
        double c = fma(ti.y + tj[u].y, d / q, ti.x + tj[u].x);
        c = ((wd[u] >> t.lane) & 1u) ? c * pj[u].w : 0.0;
        f[0] = fma(c, ex, f[0]);
        f[1] = fma(c, ey, f[1]);
        if (DIM == 3) f[2] = fma(c, ez, f[2]);
      }
    }
  }
  split_reduce<SPLIT, 3>(f);
  if (t.active && t.sub == 0) {
    double4 u;
    update(a, t.i, b, f, disp, disp_out, u);
  }
}

// Geometrically nonlinear FP64 kernels (PD_NONLINEAR): Y = xi + eta, e = |Y| - |xi| (Eq 1.10) and the
// pair force along M = Y / |Y| (Eq 1.13) with the force state of Eq 1.14.  |Y|^2 - |xi|^2 is formed
// as eta . (xi + Y) = 2 xi.eta + eta.eta, so e = (|Y|^2 - |xi|^2) / (|Y| + |xi|) carries no
// cancellation, and the break test e / |xi| >= s0 (Eq 1.30) is taken without square roots as
// |Y|^2 - |xi|^2 >= s0 (2 + s0) |xi|^2.
template <int DIM>
struct BondNL {
  double yx, yy, yz;  // Y
  double p;           // |Y|^2 - |xi|^2
  double q;           // |xi|^2
};

template <int DIM>
__device__ __forceinline__ BondNL<DIM> bond_nl(const double4& pi, const double4& pj, const double4& ui,
                                              const double4& uj) {
  BondNL<DIM> r;
  const double ex = pj.x - pi.x, ey = pj.y - pi.y, ez = DIM == 3 ? pj.z - pi.z : 0.0;
  const double hx = uj.x - ui.x, hy = uj.y - ui.y, hz = DIM == 3 ? uj.z - ui.z : 0.0;
  r.yx = ex + hx;
  r.yy = ey + hy;
  r.yz = ez + hz;
  r.p = hx * (ex + r.yx) + hy * (ey + r.yy);
  r.q = ex * ex + ey * ey;
  if (DIM == 3) {
    r.p = fma(hz, ez + r.yz, r.p);
    r.q = fma(ez, ez, r.q);
  }
  return r;
}

template <int DIM>
__device__ __noinline__ bool fp64_breaks_nl(const StepArgs& a, int64_t i, int32_t j,
                                            const double4* __restrict__ disp) {
  const int b = a.body ? a.body[i] : 0;
  const BondNL<DIM> r = bond_nl<DIM>(a.pos[i], a.pos[j], disp[i], disp[j]);
  return r.p >= a.bp[b].s0nl * r.q;
}

template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass1_nl(StepArgs a, const double4* __restrict__ disp,
                                                   int write_theta) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  if (write_theta && blockIdx.x == 0 && threadIdx.x == 0) *a.d_step += 1;
  double acc[1] = {0.0};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const double s0nl = a.bp[b].s0nl;
    const bool can_break = a.bp[b].breaks != 0;
    const double4 pi = a.pos[t.i], ui = disp[t.i];
    uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    constexpr int U = kU64;
    int32_t jn[U];
    uint32_t wn[U];
    load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      uint32_t wd[U];
      double4 pj[U], uj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        wd[u] = wn[u];
        pj[u] = a.pos[jn[u]];
        uj[u] = disp[jn[u]];
      }
      load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const BondNL<DIM> r = bond_nl<DIM>(pi, pj[u], ui, uj[u]);
        bool intact = (wd[u] >> t.lane) & 1u;
        if (a.check) {
          const bool brk = intact && can_break && r.p >= s0nl * r.q;
          const unsigned m = __ballot_sync(kFull, brk);
          if (m) {
            intact = intact && !brk;
            if (t.lane == 0) bw[k0 + u * SPLIT] = wd[u] & ~m;
          }
        }
        if (intact) {
          double yl2 = r.yx * r.yx + r.yy * r.yy;
          if (DIM == 3) yl2 = fma(r.yz, r.yz, yl2);
          const double xl = sqrt(r.q);
          const double e = r.p / (sqrt(yl2) + xl);
          acc[0] = fma(pj[u].w * xl, e, acc[0]);  // Eq 1.6: w x e V_j
        }
      }
    }
  }
  split_reduce<SPLIT, 1>(acc);
  if (t.active && t.sub == 0 && write_theta) {
    const double th = a.aA[t.i] * acc[0];
    const double mu = a.mu[t.i];
    a.theta[t.i] = th;
    a.thm[t.i] = make_double2(a.bp[b].Kp * (th * mu), a.bp[b].G * mu);
  }
}

template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass2_nl(StepArgs a, const double4* __restrict__ disp,
                                                   double4* __restrict__ disp_out) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  double f[3] = {0.0, 0.0, 0.0};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const double4 pi = a.pos[t.i], ui = disp[t.i];
    const double2 ti = a.thm[t.i];
    const uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    constexpr int U = kU64;
    int32_t jn[U];
    uint32_t wn[U];
    load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      uint32_t wd[U];
      double4 pj[U], uj[U];
      double2 tj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        wd[u] = wn[u];
        pj[u] = a.pos[jn[u]];
        uj[u] = disp[jn[u]];
        tj[u] = a.thm[jn[u]];
      }
      load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!((wd[u] >> t.lane) & 1u)) continue;
        const BondNL<DIM> r = bond_nl<DIM>(pi, pj[u], ui, uj[u]);
        double yl2 = r.yx * r.yx + r.yy * r.yy;
        if (DIM == 3) yl2 = fma(r.yz, r.yz, yl2);
        const double yl = sqrt(yl2), xl = sqrt(r.q);
        const double e = r.p / (yl + xl);
        // Eq 1.14 for both ends: [(K - G/3)(theta_i/m_i + theta_j/m_j) |xi| + G (1/m_i + 1/m_j) e] V_j,
        // along M = Y / |Y| (Eq 1.13)
        const double c = fma(ti.x + tj[u].x, xl, (ti.y + tj[u].y) * e) * pj[u].w / yl;
        f[0] = fma(c, r.yx, f[0]);
        f[1] = fma(c, r.yy, f[1]);
        if (DIM == 3) f[2] = fma(c, r.yz, f[2]);
      }
    }
  }
  split_reduce<SPLIT, 3>(f);
  if (t.active && t.sub == 0) {
    double4 u;
    update(a, t.i, b, f, disp, disp_out, u);
  }
}

// Tabled nonlinear FP64 kernels (PD_OPT_BOND_CACHE on): per slot the reference vector and length
// (xi, |xi|) are read from a table built once per family, and pass 1 leaves (e, 1/|Y|) of every slot
// in a second table, so pass 2 forms only Y = xi + eta and the force along Y / |Y| (no root, no divide).
template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass1_nlt(StepArgs a, const double4* __restrict__ disp,
                                                    int write_theta) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  if (write_theta && blockIdx.x == 0 && threadIdx.x == 0) *a.d_step += 1;
  double acc[1] = {0.0};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const double s0nl = a.bp[b].s0nl;
    const bool can_break = a.bp[b].breaks != 0;
    const double4 ui = disp[t.i];
    uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    const double4* __restrict__ ta = a.bA + t.base + t.lane;
    double2* __restrict__ te = a.bE + t.base + t.lane;
    constexpr int U = kU64;
    int32_t jn[U];
    uint32_t wn[U];
    load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      uint32_t wd[U];
      double4 g[U], uj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = min(k0 + u * SPLIT, t.W - 1);
        wd[u] = wn[u];
        g[u] = ta[(int64_t)k << 5];
        uj[u] = disp[jn[u]];
      }
      load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const double hx = uj[u].x - ui.x, hy = uj[u].y - ui.y, hz = DIM == 3 ? uj[u].z - ui.z : 0.0;
        const double yx = g[u].x + hx, yy = g[u].y + hy, yz = g[u].z + hz;
        double p = hx * (g[u].x + yx) + hy * (g[u].y + yy);
        if (DIM == 3) p = fma(hz, g[u].z + yz, p);
        const int k = k0 + u * SPLIT;
        bool intact = (wd[u] >> t.lane) & 1u;
        if (a.check) {
          const bool brk = intact && can_break && p >= s0nl * (g[u].w * g[u].w);
          const unsigned m = __ballot_sync(kFull, brk);
          if (m) {
            intact = intact && !brk;
            if (t.lane == 0) bw[k] = wd[u] & ~m;
          }
        }
        if (intact) {
          double yl2 = yx * yx + yy * yy;
          if (DIM == 3) yl2 = fma(yz, yz, yl2);
          const double ry = rsqrt(yl2);
          const double e = p / fma(yl2, ry, g[u].w);
          te[(int64_t)k << 5] = make_double2(e, ry);
          acc[0] = fma(uj[u].w * g[u].w, e, acc[0]);  // Eq 1.6: w x e V_j
        }
      }
    }
  }
  split_reduce<SPLIT, 1>(acc);
  if (t.active && t.sub == 0 && write_theta) {
    const double th = a.aA[t.i] * acc[0];
    const double mu = a.mu[t.i];
    a.theta[t.i] = th;
    a.thm[t.i] = make_double2(a.bp[b].Kp * (th * mu), a.bp[b].G * mu);
  }
}

template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass2_nlt(StepArgs a, const double4* __restrict__ disp,
                                                    double4* __restrict__ disp_out) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  double f[3] = {0.0, 0.0, 0.0};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const double4 ui = disp[t.i];
    const double2 ti = a.thm[t.i];
    const uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    const double4* __restrict__ ta = a.bA + t.base + t.lane;
    const double2* __restrict__ te = a.bE + t.base + t.lane;
    constexpr int U = kU64;
    int32_t jn[U];
    uint32_t wn[U];
    load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      uint32_t wd[U];
      double4 g[U], uj[U];
      double2 tj[U], ev[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = min(k0 + u * SPLIT, t.W - 1);
        wd[u] = wn[u];
        const bool on = (wd[u] >> t.lane) & 1u;
        g[u] = ta[(int64_t)k << 5];
        ev[u] = on ? te[(int64_t)k << 5] : make_double2(0.0, 0.0);
        uj[u] = disp[jn[u]];
        tj[u] = a.thm[jn[u]];
      }
      load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const double yx = g[u].x + (uj[u].x - ui.x), yy = g[u].y + (uj[u].y - ui.y);
        const double yz = DIM == 3 ? g[u].z + (uj[u].z - ui.z) : 0.0;
        // Eq 1.14 for both ends along M = Y / |Y| (Eq 1.13); 0 for broken and unused slots (ev = 0)
        const double c = fma(ti.x + tj[u].x, g[u].w, (ti.y + tj[u].y) * ev[u].x) * (uj[u].w * ev[u].y);
        f[0] = fma(c, yx, f[0]);
        f[1] = fma(c, yy, f[1]);
        if (DIM == 3) f[2] = fma(c, yz, f[2]);
      }
    }
  }
  split_reduce<SPLIT, 3>(f);
  if (t.active && t.sub == 0) {
    double4 u;
    update(a, t.i, b, f, disp, disp_out, u);
  }
}

// -x exactly, by the sign bit (on the integer pipe rather than the FP64 one).
__device__ __forceinline__ double flip_sign(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// Pair form of the tabled nonlinear pass 1.  Y and u_j - u_i change sign between the two entries of a
// bond and |Y|^2 - |xi|^2 does not, so the failure test, e and 1/|Y| are the same numbers at both
// ends: pass 1a forms them once, at the owned entry, clears both bits of a broken bond, and writes
// (M = Y/|Y|, e) and the theta terms V_j |xi| e and V_i |xi| e of both entries (M changes sign);
// pass 1b sums theta, and pass 2 takes the bond's direction and extension from the table instead of
// recomputing Y from the displacements.  The root and the divide, most of the FP64 work of the
// single pass, run once per bond.
// UV: every body has one particle volume, so both entries' dilatation terms (V_j |xi| e and V_i |xi| e)
// are the same product, formed once (bitwise the same values).
template <int DIM, int SPLIT, bool UV>
__global__ void __launch_bounds__(512) k_pass1a_nlp(StepArgs a, const double4* __restrict__ disp) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  if (!t.active) return;  // whole warps; no block-wide barrier below
  const int b = a.body ? a.body[t.i] : 0;
  const double s0nl = a.bp[b].s0nl;
  const bool can_break = a.bp[b].breaks != 0;
  const int own = a.own0[t.i], cnt = a.cnt[t.i];
  const int k_lo = __reduce_min_sync(kFull, (unsigned)own);
  const int k_hi = __reduce_max_sync(kFull, (unsigned)cnt);
  const double4 ui = disp[t.i];
  uint32_t* bw = a.bits + (t.base >> 5);
  const int32_t* __restrict__ cl = a.col + t.base + t.lane;
  const int32_t* __restrict__ tw = a.twin + t.base + t.lane;
  const double4* __restrict__ ta = a.bA + t.base + t.lane;
  for (int k = k_lo + t.sub; k < k_hi; k += SPLIT) {
    const bool mine = k >= own && k < cnt;
    const int64_t e = t.base + t.lane + ((int64_t)k << 5);
    double p = 0.0, yl2 = 0.0, xl = 0.0, vj = 0.0, yx = 0.0, yy = 0.0, yz = 0.0;
    int32_t te = 0;
    if (mine) {
      const int32_t j = cl[(int64_t)k << 5];
      const double4 g = ta[(int64_t)k << 5];
      const double4 uj = disp[j];
      te = tw[(int64_t)k << 5];
      const double hx = uj.x - ui.x, hy = uj.y - ui.y, hz = DIM == 3 ? uj.z - ui.z : 0.0;
      yx = g.x + hx;
      yy = g.y + hy;
      yz = g.z + hz;
      p = hx * (g.x + yx) + hy * (g.y + yy);
      if (DIM == 3) p = fma(hz, g.z + yz, p);
      yl2 = yx * yx + yy * yy;
      if (DIM == 3) yl2 = fma(yz, yz, yl2);
      xl = g.w;
      vj = uj.w;
    }
    bool intact = mine && ((bw[k] >> t.lane) & 1u);  // this warp's owned bits change only here
    if (a.check) {
      const bool brk = intact && can_break && p >= s0nl * (xl * xl);
      const unsigned m = __ballot_sync(kFull, brk);
      if (m) {
        if (t.lane == 0) atomicAnd(&bw[k], ~m);
        if (brk) atomicAnd(a.bits + (te >> 5), ~(1u << (te & 31)));
        intact = intact && !brk;
      }
    }
    if (intact) {
      const double ry = rsqrt(yl2);
      const double ev = p / fma(yl2, ry, xl);
      const double mx = ry * yx, my = ry * yy, mz = ry * yz;  // M = Y / |Y| (Eq 1.13), -M at j
      a.bY[e] = make_double4(mx, my, mz, ev);
      a.bY[te] = make_double4(flip_sign(mx), flip_sign(my), flip_sign(mz), ev);
      const double tij = (vj * xl) * ev;  // Eq 1.6 term of entry (i, j): w |xi| e V_j
      a.bt[e] = tij;
      a.bt[te] = UV ? tij : (ui.w * xl) * ev;  // and of entry (j, i): w |xi| e V_i
    }
  }
}

template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass1b_nlp(StepArgs a, int write_theta) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  if (write_theta && blockIdx.x == 0 && threadIdx.x == 0) *a.d_step += 1;
  double acc[1] = {0.0};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const double* __restrict__ tt = a.bt + t.base + t.lane;
    for (int k = t.sub; k < t.W; k += SPLIT)
      if ((bw[k] >> t.lane) & 1u) acc[0] += tt[(int64_t)k << 5];
  }
  split_reduce<SPLIT, 1>(acc);
  if (t.active && t.sub == 0 && write_theta) {
    const double th = a.aA[t.i] * acc[0];
    const double mu = a.mu[t.i];
    a.theta[t.i] = th;
    a.thm[t.i] = make_double2(a.bp[b].Kp * (th * mu), a.bp[b].G * mu);
  }
}

// Pass 2 of the nonlinear pair form: Eq 1.14 for both ends along M (Eq 1.13),
// f_i = sum_j [(K - G/3)(theta_i/m_i + theta_j/m_j) |xi| V_j + G (1/m_i + 1/m_j) e V_j] M, with
// (M, e) from pass 1a and (|xi| V_j, V_j) from a per-slot table built once.
template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass2_nlp(StepArgs a, const double4* __restrict__ disp,
                                                    double4* __restrict__ disp_out) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  double f[3] = {0.0, 0.0, 0.0};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const double2 ti = a.thm[t.i];
    const uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    const double4* __restrict__ ty = a.bY + t.base + t.lane;
    const double2* __restrict__ tx = a.bX + t.base + t.lane;
    constexpr int U = 4;
    int32_t jn[U];
    uint32_t wn[U];
    load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      uint32_t wd[U];
      double4 y[U];
      double2 x[U], tj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = min(k0 + u * SPLIT, t.W - 1);
        wd[u] = wn[u];
        y[u] = ty[(int64_t)k << 5];
        x[u] = tx[(int64_t)k << 5];
        tj[u] = a.thm[jn[u]];
      }
      load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        double c = fma(ti.x + tj[u].x, x[u].x, (ti.y + tj[u].y) * (y[u].w * x[u].y));
        c = ((wd[u] >> t.lane) & 1u) ? c : 0.0;  // broken and unused slots
        f[0] = fma(c, y[u].x, f[0]);
        f[1] = fma(c, y[u].y, f[1]);
        if (DIM == 3) f[2] = fma(c, y[u].z, f[2]);
      }
    }
  }
  split_reduce<SPLIT, 3>(f);
  if (t.active && t.sub == 0) {
    double4 u;
    update(a, t.i, b, f, disp, disp_out, u);
  }
}

// (|xi| V_j, V_j) per slot for k_pass2_nlp, |xi| as in k_bond_tables_nl.
template <int DIM>
__global__ void k_bond_tables_nlp(StepArgs a, double2* __restrict__ bX) {
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (!t.active) return;
  const double4 pi = a.pos[t.i];
  const double4 zero = make_double4(0.0, 0.0, 0.0, 0.0);
  for (int k = 0; k < t.W; ++k) {
    const int64_t e = t.base + t.lane + ((int64_t)k << 5);
    const double4 pj = a.pos[a.col[e]];
    double ex, ey, ez, d, q;
    bond_f64<DIM>(pi, pj, zero, zero, ex, ey, ez, d, q);
    bX[e] = make_double2(sqrt(q) * pj.w, pj.w);
  }
}

template <int DIM>
__global__ void k_bond_tables_nl(StepArgs a, double4* __restrict__ bA) {
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (!t.active) return;
  const double4 pi = a.pos[t.i];
  const double4 zero = make_double4(0.0, 0.0, 0.0, 0.0);
  for (int k = 0; k < t.W; ++k) {
    const int64_t e = t.base + t.lane + ((int64_t)k << 5);
    const double4 pj = a.pos[a.col[e]];
    double ex, ey, ez, d, q;
    bond_f64<DIM>(pi, pj, zero, zero, ex, ey, ez, d, q);
    bA[e] = make_double4(ex, ey, ez, sqrt(q));
  }
}

// Tabled FP64 kernels.  GB300 issues FP64 at 1/64 of the FP32 rate, so everything that does not
// depend on the displacement is computed once per family into per-slot tables:
//   bA = (xi, s0 |xi|^2)                       read by pass 1 (the break test xi.du >= s0 |xi|^2, Eq 1.30);
//   bB = (V_j xi, G (1/m_i + 1/m_j) / |xi|^2)  read by pass 2 (m is fixed once the family is built);
// pass 1 stores each slot's xi.du (the per-bond extension times |xi|, the paper's E array of
// Appendix B) in bd for pass 2, which then needs neither u_j nor a divide.  The i-end dilatation term
// of Eq 2.2 is the same for every bond of particle i, so pass 2 multiplies it once by
//   bS_i = sum of V_j xi over the intact slots of i
// instead of adding it to every bond's coefficient; bS changes only when a bond breaks, and the pass
// that breaks it recomputes bS for that slice.  Per bond pass 1 issues 7 FP64 instructions (the
// difference, the dot product and the theta sum) and pass 2 4 (the bond coefficient and the force),
// against 15 and 14 when everything is recomputed.  The break test compares the two doubles' bit
// patterns as signed integers: for a positive threshold s0 |xi|^2 that order equals the FP64 order of
// xi.du (negative values and -0 sort below every positive double), and it runs on the integer pipe
// instead of the FP64 one.

// bS_i from the status bits and bB, in slot order (so bS is a function of the bits alone).  The
// words are read through L2: other warps of the block may have just written them.
__device__ __forceinline__ void bond_sum_row(const StepArgs& a, const SliceIdx& t) {
  const uint32_t* bw = a.bits + (t.base >> 5);
  const double4* tb = a.bB + t.base + t.lane;
  double sx = 0.0, sy = 0.0, sz = 0.0;
  for (int k = 0; k < t.W; ++k) {
    if ((__ldcg(bw + k) >> t.lane) & 1u) {
      const double4 g = tb[(int64_t)k << 5];
      sx += g.x;
      sy += g.y;
      sz += g.z;
    }
  }
  a.bS[t.i] = make_double4(sx, sy, sz, 0.0);
}

__global__ void k_bond_sums(StepArgs a) {
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (t.active) bond_sum_row(a, t);
}

// THETA = false: the failure check alone (applied to the current state before it is read), with no
// theta sum and no xi.du store: 6 FP64 instructions per bond.
template <int DIM, int SPLIT, bool THETA>
__global__ void __launch_bounds__(512) k_pass1_f64t(StepArgs a, const double4* __restrict__ disp,
                                                     int write_theta) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  if (write_theta && blockIdx.x == 0 && threadIdx.x == 0) *a.d_step += 1;
  double acc[2] = {0.0, 0.0};  // theta sum, and 1 if a bond of this warp's slots broke (warp-uniform)
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const bool can_break = a.bp[b].breaks != 0;
    const double4 ui = disp[t.i];
    uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    const double4* __restrict__ ta = a.bA + t.base + t.lane;
    double* __restrict__ td = a.bd + t.base + t.lane;
    constexpr int U = kU64;
    int32_t jn[U];
    uint32_t wn[U];
    load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      uint32_t wd[U];
      double4 g[U], uj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = min(k0 + u * SPLIT, t.W - 1);
        wd[u] = wn[u];
        g[u] = ta[(int64_t)k << 5];
        uj[u] = disp[jn[u]];
      }
      load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        double d = g[u].x * (uj[u].x - ui.x) + g[u].y * (uj[u].y - ui.y);
        if (DIM == 3) d = fma(g[u].z, uj[u].z - ui.z, d);
        const int k = k0 + u * SPLIT;
        if (THETA && k < t.W) td[(int64_t)k << 5] = d;
        bool intact = (wd[u] >> t.lane) & 1u;
        if (a.check) {
          const bool ge = pd_ge_threshold(d, g[u].w);  // d >= s0 |xi|^2
          const bool brk = intact && can_break && ge;
          const unsigned m = __ballot_sync(kFull, brk);
          if (m) {
            intact = intact && !brk;
            if (t.lane == 0) bw[k] = wd[u] & ~m;
            acc[1] = 1.0;
          }
        }
        if (THETA) acc[0] = fma(intact ? uj[u].w : 0.0, d, acc[0]);
      }
    }
  }
  if (SPLIT == 1) __syncwarp();  // lane 0's status words, for the bS recomputation below
  split_reduce<SPLIT, 2>(acc);   // (SPLIT > 1: its block barrier orders the other warps' words)
  if (t.active && t.sub == 0) {
    if (THETA && write_theta) {
      const double th = a.aA[t.i] * acc[0];
      const double mu = a.mu[t.i];
      a.theta[t.i] = th;
      a.thm[t.i] = make_double2(a.bp[b].Kp * (th * mu), a.bp[b].G * mu);
    }
    if (acc[1] != 0.0) bond_sum_row(a, t);
  }
}

// Pair form of the tabled FP64 pass 1, used when the build paired the two entries of every bond.
// ξ·(u_j − u_i) is the same number at both ends (ξ and u_j − u_i both change sign, exactly), so
// pass 1a forms it once, at the owned entry, applies the failure check to the pair (clearing both
// entries' bits) and stores it in both entries' bd slots; pass 1b then sums theta from bd over the
// intact entries in slot order.  Per directed bond that is 3 FP64 instructions in 1a and 1 in 1b
// against 7 in the single pass, with the same values: d, the decisions, bd and theta are bitwise
// those of k_pass1_f64t.  A slice in which a bond broke (at either end) is marked for pass 1b,
// which recomputes its bS.
template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass1a_f64p(StepArgs a, const double4* __restrict__ disp) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  if (!t.active) return;  // whole warps; no block-wide barrier below
  const int b = a.body ? a.body[t.i] : 0;
  const bool can_break = a.bp[b].breaks != 0;
  const int own = a.own0[t.i], cnt = a.cnt[t.i];
  const int k_lo = __reduce_min_sync(kFull, (unsigned)own);
  const int k_hi = __reduce_max_sync(kFull, (unsigned)cnt);
  const double4 ui = disp[t.i];
  uint32_t* bw = a.bits + (t.base >> 5);
  const int32_t* __restrict__ cl = a.col + t.base + t.lane;
  const int32_t* __restrict__ tw = a.twin + t.base + t.lane;
  const double4* __restrict__ ta = a.bA + t.base + t.lane;
  double* td = a.bd;
  // the owned-slot streams (index, table row, twin entry) of the next slot are loaded while the
  // current slot's displacement gather and arithmetic run
  int k = k_lo + t.sub;
  bool mn = k < k_hi && k >= own && k < cnt;
  int32_t jn = (int32_t)t.i, ten = 0;
  double4 gn = make_double4(0.0, 0.0, 0.0, 0.0);
  if (mn) {
    jn = cl[(int64_t)k << 5];
    gn = ta[(int64_t)k << 5];
    ten = tw[(int64_t)k << 5];
  }
  for (; k < k_hi; k += SPLIT) {
    const bool mine = mn;
    const int32_t j = jn, te = ten;
    const double4 g = gn;
    const double4 uj = disp[j];
    const int kn = k + SPLIT;
    mn = kn < k_hi && kn >= own && kn < cnt;
    if (mn) {
      jn = cl[(int64_t)kn << 5];
      gn = ta[(int64_t)kn << 5];
      ten = tw[(int64_t)kn << 5];
    }
    const int64_t e = t.base + t.lane + ((int64_t)k << 5);
    double d = g.x * (uj.x - ui.x) + g.y * (uj.y - ui.y);
    if (DIM == 3) d = fma(g.z, uj.z - ui.z, d);
    if (mine) {
      td[e] = d;
      td[te] = d;
    }
    if (a.check) {
      const uint32_t wd = bw[k];  // this warp's owned bits change only here
      const bool brk = mine && can_break && ((wd >> t.lane) & 1u) &&
                       pd_ge_threshold(d, g.w);  // d >= s0 |xi|^2
      const unsigned m = __ballot_sync(kFull, brk);
      if (m) {
        if (t.lane == 0) {
          atomicAnd(&bw[k], ~m);
          a.dirty[t.i >> 5] = 1;
        }
        if (brk) {
          atomicAnd(a.bits + (te >> 5), ~(1u << (te & 31)));
          a.dirty[j >> 5] = 1;
        }
      }
    }
  }
}

// UV: every body has one particle volume, so V_j = V_i for every bond (same body) and the sum takes
// the lane's own V_i: the same FMAs on the same values, without the neighbour index stream and the
// gather of V_j.
template <int DIM, int SPLIT, bool UV>
__global__ void __launch_bounds__(512) k_pass1b_f64p(StepArgs a, const double4* __restrict__ disp, int write_theta) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  if (write_theta && blockIdx.x == 0 && threadIdx.x == 0) *a.d_step += 1;
  double acc[1] = {0.0};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    const double* __restrict__ td = a.bd + t.base + t.lane;
    const double vi = UV ? disp[t.i].w : 0.0;
    constexpr int U = 4;
    int32_t jn[U];
    uint32_t wn[U];
    if (UV) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = t.sub + u * SPLIT;
        wn[u] = k < t.W ? bw[k] : 0u;
      }
    } else {
      load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    }
    double dn[U];
#pragma unroll
    for (int u = 0; u < U; ++u) dn[u] = td[(int64_t)min(t.sub + u * SPLIT, t.W - 1) << 5];
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      uint32_t wd[U];
      double d[U], v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        wd[u] = wn[u];
        d[u] = dn[u];
        v[u] = UV ? vi : disp[jn[u]].w;
      }
      if (UV) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int k = k0 + (U + u) * SPLIT;
          wn[u] = k < t.W ? bw[k] : 0u;
        }
      } else {
        load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) dn[u] = td[(int64_t)min(k0 + (U + u) * SPLIT, t.W - 1) << 5];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if ((wd[u] >> t.lane) & 1u) acc[0] = fma(v[u], d[u], acc[0]);
    }
  }
  split_reduce<SPLIT, 1>(acc);
  if (t.active && t.sub == 0) {
    if (write_theta) {
      const double th = a.aA[t.i] * acc[0];
      const double mu = a.mu[t.i];
      a.theta[t.i] = th;
      a.thm[t.i] = make_double2(a.bp[b].Kp * (th * mu), a.bp[b].G * mu);
    }
    if (a.dirty[t.i >> 5]) {  // uniform over the warp
      bond_sum_row(a, t);
      __syncwarp();
      if (t.lane == 0) a.dirty[t.i >> 5] = 0;
    }
  }
}

// The failure check alone in the nonlinear pair form, applied to the current state before its bond
// status is read between steps: |Y|^2 - |xi|^2 >= s0 (2 + s0) |xi|^2 (Eq 1.30 with the extension of
// Eq 1.10) once per intact bond at its owned entry, with pass 1a's arithmetic so that each decision
// is the one pass 1a takes, but without its reciprocal square root, division and table stores: the
// next step's pass 1a (which does not check again) forms M, e and the dilatation terms of the bonds
// still intact.
template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_check_nlp(StepArgs a, const double4* __restrict__ disp) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  if (!t.active) return;  // whole warps; no block-wide barrier below
  const int b = a.body ? a.body[t.i] : 0;
  const double s0nl = a.bp[b].s0nl;
  const bool can_break = a.bp[b].breaks != 0;
  if (!__any_sync(kFull, can_break)) return;
  const int own = a.own0[t.i], cnt = a.cnt[t.i];
  const int k_lo = __reduce_min_sync(kFull, (unsigned)own);
  const int k_hi = __reduce_max_sync(kFull, (unsigned)cnt);
  const double4 ui = disp[t.i];
  uint32_t* bw = a.bits + (t.base >> 5);
  const int32_t* __restrict__ cl = a.col + t.base + t.lane;
  const double4* __restrict__ ta = a.bA + t.base + t.lane;
  // the next slot's index and table row are loaded while the current slot's gather runs
  int k = k_lo + t.sub;
  bool mn = k < k_hi && k >= own && k < cnt && can_break;
  int32_t jn = (int32_t)t.i;
  double4 gn = make_double4(0.0, 0.0, 0.0, 0.0);
  if (mn) {
    jn = cl[(int64_t)k << 5];
    gn = ta[(int64_t)k << 5];
  }
  for (; k < k_hi; k += SPLIT) {
    const uint32_t wd = bw[k];  // this warp's owned bits change only here
    const bool mine = mn && ((wd >> t.lane) & 1u);
    const int32_t j = jn;
    const double4 g = gn;
    const int kn = k + SPLIT;
    mn = kn < k_hi && kn >= own && kn < cnt && can_break;
    if (mn) {
      jn = cl[(int64_t)kn << 5];
      gn = ta[(int64_t)kn << 5];
    }
    bool brk = false;
    if (mine) {
      const double4 uj = disp[j];
      const double hx = uj.x - ui.x, hy = uj.y - ui.y, hz = DIM == 3 ? uj.z - ui.z : 0.0;
      const double yx = g.x + hx, yy = g.y + hy, yz = g.z + hz;
      double p = hx * (g.x + yx) + hy * (g.y + yy);
      if (DIM == 3) p = fma(hz, g.z + yz, p);
      const double xl = g.w;
      brk = p >= s0nl * (xl * xl);
    }
    const unsigned m = __ballot_sync(kFull, brk);
    if (m) {
      if (t.lane == 0) atomicAnd(&bw[k], ~m);
      if (brk) {
        const int32_t te = a.twin[t.base + t.lane + ((int64_t)k << 5)];
        atomicAnd(a.bits + (te >> 5), ~(1u << (te & 31)));
      }
    }
  }
}

// The failure check alone in the pair form, applied to the current state before its bond status is
// read between steps: ξ·(u_j − u_i) once per intact bond at its owned entry, as in pass 1a, but
// with no bd store (the next step's pass 1a stores it) and the twin entry's index loaded only
// for a bond that breaks.  Slices with broken bonds are marked for the next pass 1b.
//
// SCREEN: each bond is first evaluated in FP32, from FP32 copies of u (cu) and of the slot's ξ with
// its threshold rounded down (cA).  With M = Σ_c |ξ_c| (|u_jc| + |u_ic|), the FP32 value differs
// from the FP64 one by at most 6.01 u₃₂ M (u₃₂ = 2⁻²⁴: the roundings of ξ, of both u and of their
// difference, and three for the products and sums; the FP64 rounding is below 2⁻⁵⁰ M), and the
// FP32-evaluated M by a few u₃₂ M.  A bond whose FP32 value plus 2⁻¹⁹ (M + |value|) (five times
// that bound, so the final FP32 addition cannot close the gap) is still below the rounded-down
// threshold is below the FP64 threshold in FP64 too, and stays intact; the small absolute terms
// cover gradual underflow.  Every other bond, and every non-finite value (its comparisons are
// false), is evaluated in FP64 exactly as pass 1a does, so each decision is pass 1a's.
template <int DIM, int SPLIT, bool SCREEN>
__global__ void __launch_bounds__(512) k_check_f64p(StepArgs a, const double4* __restrict__ disp,
                                                     const float4* __restrict__ cu,
                                                     const float4* __restrict__ cA) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  if (!t.active) return;  // whole warps; no block-wide barrier below
  const int b = a.body ? a.body[t.i] : 0;
  const bool can_break = a.bp[b].breaks != 0;
  if (!__any_sync(kFull, can_break)) return;
  const int own = a.own0[t.i], cnt = a.cnt[t.i];
  const int k_lo = __reduce_min_sync(kFull, (unsigned)own);
  const int k_hi = __reduce_max_sync(kFull, (unsigned)cnt);
  const double4 ui = disp[t.i];
  const float4 ui32 = SCREEN ? cu[t.i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  uint32_t* bw = a.bits + (t.base >> 5);
  const int32_t* __restrict__ cl = a.col + t.base + t.lane;
  const double4* __restrict__ ta = a.bA + t.base + t.lane;
  const float4* __restrict__ ts = SCREEN ? cA + t.base + t.lane : nullptr;
  // the next slot's index and table row are loaded while the current slot's gather runs
  int k = k_lo + t.sub;
  bool mn = k < k_hi && k >= own && k < cnt && can_break;
  int32_t jn = (int32_t)t.i;
  double4 gn = make_double4(0.0, 0.0, 0.0, 0.0);
  float4 sn = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (mn) {
    jn = cl[(int64_t)k << 5];
    if (SCREEN)
      sn = ts[(int64_t)k << 5];
    else
      gn = ta[(int64_t)k << 5];
  }
  for (; k < k_hi; k += SPLIT) {
    const uint32_t wd = bw[k];  // this warp's owned bits change only here
    const bool mine = mn && ((wd >> t.lane) & 1u);
    const int32_t j = jn;
    const double4 g0 = gn;
    const float4 sc = sn;
    const int kn = k + SPLIT;
    mn = kn < k_hi && kn >= own && kn < cnt && can_break;
    if (mn) {
      jn = cl[(int64_t)kn << 5];
      if (SCREEN)
        sn = ts[(int64_t)kn << 5];
      else
        gn = ta[(int64_t)kn << 5];
    }
    bool brk = false;
    if (mine) {
      bool exact = true;
      if (SCREEN) {
        const float4 uj = cu[j];
        const float dx = uj.x - ui32.x, dy = uj.y - ui32.y;
        float d = fmaf(sc.x, dx, sc.y * dy);
        float m = fmaf(fabsf(sc.x), fabsf(uj.x) + fabsf(ui32.x), fabsf(sc.y) * (fabsf(uj.y) + fabsf(ui32.y)));
        float l1 = fabsf(sc.x) + fabsf(sc.y);
        if (DIM == 3) {
          d = fmaf(sc.z, uj.z - ui32.z, d);
          m = fmaf(fabsf(sc.z), fabsf(uj.z) + fabsf(ui32.z), m);
          l1 += fabsf(sc.z);
        }
        const float bound = fmaf(0x1p-19f, m + fabsf(d), fmaf(0x1p-120f, l1, 0x1p-140f));
        exact = !(d + bound < sc.w);
      }
      if (exact) {
        const double4 g = SCREEN ? ta[(int64_t)k << 5] : g0;
        const double4 uj = disp[j];
        double d = g.x * (uj.x - ui.x) + g.y * (uj.y - ui.y);
        if (DIM == 3) d = fma(g.z, uj.z - ui.z, d);
        brk = pd_ge_threshold(d, g.w);  // d >= s0 |xi|^2
      }
    }
    const unsigned m = __ballot_sync(kFull, brk);
    if (m) {
      if (t.lane == 0) {
        atomicAnd(&bw[k], ~m);
        a.dirty[t.i >> 5] = 1;
      }
      if (brk) {
        const int32_t te = a.twin[t.base + t.lane + ((int64_t)k << 5)];
        atomicAnd(a.bits + (te >> 5), ~(1u << (te & 31)));
        a.dirty[j >> 5] = 1;
      }
    }
  }
}

// FP32 tables of the screened check: per slot ξ rounded to nearest and s0|ξ|² rounded down.
__global__ void k_check_tables(int64_t nentries, const double4* __restrict__ bA, float4* __restrict__ cA) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nentries;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double4 g = bA[e];
    cA[e] = make_float4(__double2float_rn(g.x), __double2float_rn(g.y), __double2float_rn(g.z),
                        __double2float_rd(g.w));
  }
}

// u rounded to FP32 for the screened check.
__global__ void k_check_u32(int64_t n_pad, const double4* __restrict__ disp, float4* __restrict__ cu) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  const double4 u = disp[i];
  cu[i] = make_float4(__double2float_rn(u.x), __double2float_rn(u.y), __double2float_rn(u.z), 0.0f);
}

template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass2_f64t(StepArgs a, const double4* __restrict__ disp,
                                                     double4* __restrict__ disp_out) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  double f[3] = {0.0, 0.0, 0.0};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    const double4* __restrict__ tb = a.bB + t.base + t.lane;
    const double* __restrict__ td = a.bd + t.base + t.lane;
    constexpr int U = 4;
    int32_t jn[U];
    uint32_t wn[U];
    load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      uint32_t wd[U];
      double4 g[U];
      double d[U], tj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = min(k0 + u * SPLIT, t.W - 1);
        wd[u] = wn[u];
        g[u] = tb[(int64_t)k << 5];
        d[u] = td[(int64_t)k << 5];
        tj[u] = a.thm[jn[u]].x;
      }
      load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        // Eq 2.2 with V_j folded into the tabled xi, G (1/m_i + 1/m_j) / |xi|^2 tabled and the
        // i-end term (K - G/3) theta_i / m_i applied to bS_i below:
        // [(K - G/3) theta_j / m_j + G (1/m_i + 1/m_j) e / |xi|] (V_j xi)
        double c = fma(g[u].w, d[u], tj[u]);
        c = ((wd[u] >> t.lane) & 1u) ? c : 0.0;
        f[0] = fma(c, g[u].x, f[0]);
        f[1] = fma(c, g[u].y, f[1]);
        if (DIM == 3) f[2] = fma(c, g[u].z, f[2]);
      }
    }
  }
  split_reduce<SPLIT, 3>(f);
  if (t.active && t.sub == 0) {
    const double ti = a.thm[t.i].x;
    const double4 S = a.bS[t.i];
    f[0] = fma(ti, S.x, f[0]);
    f[1] = fma(ti, S.y, f[1]);
    f[2] = fma(ti, S.z, f[2]);
    double4 u;
    update(a, t.i, b, f, disp, disp_out, u);
  }
}

// Per-slot tables of the tabled FP64 path, with xi and |xi|^2 evaluated exactly as bond_f64 does
// (so both FP64 variants decide a bond identically).
template <int DIM>
__global__ void k_bond_tables(StepArgs a, double4* __restrict__ bA, double4* __restrict__ bB) {
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (!t.active) return;
  const int b = a.body ? a.body[t.i] : 0;
  const double s0 = a.bp[b].s0, G = a.bp[b].G, wd = a.bp[b].wdelta;
  const double4 pi = a.pos[t.i];
  const double mi = a.mu[t.i];
  const double4 zero = make_double4(0.0, 0.0, 0.0, 0.0);
  for (int k = 0; k < t.W; ++k) {
    const int64_t e = t.base + t.lane + ((int64_t)k << 5);
    const int32_t j = a.col[e];
    const double4 pj = a.pos[j];
    double ex, ey, ez, d, q;
    bond_f64<DIM>(pi, pj, zero, zero, ex, ey, ez, d, q);
    // With an influence function w (Eqs 1.6, 1.9, 1.14) the tables hold w xi and w s0 |xi|^2 (so that
    // the stored extension is w xi.du, the theta sum sum w V_j xi.du and the failure test, w > 0,
    // unchanged), w V_j xi and G (1/m_i + 1/m_j) / (w |xi|^2): the step kernels are the same.
    const double w = (wd > 0.0 && q > 0.0) ? wd / sqrt(q) : 1.0;
    bA[e] = make_double4(w * ex, w * ey, w * ez, w * (s0 * q));
    bB[e] = make_double4(w * pj.w * ex, w * pj.w * ey, w * pj.w * ez, q > 0.0 ? G * (mi + a.mu[j]) / (w * q) : 0.0);
  }
}

// ----------------------------------------------------------------------------------- mixed path
// The hardware approximations of 1 / sqrt(x) and 1 / x with a subnormal x read as zero (PTX
// rsqrt.approx.ftz.f32, rcp.approx.ftz.f32), for the FP32 nonlinear kernels: without .ftz each call
// carries a test and rescaling for subnormal inputs.  Their arguments are squared bond lengths and
// sums of bond lengths: |Y|^2 and |Y| + |xi| in units of the coordinate quantum (|xi| >= 1), and
// |Y'|^2 = |n|^2 + p and |Y'| + |n| >= 1 in lattice units, normal numbers for every bond not
// compressed to within 2^-63 of its length, where the results equal those of rsqrtf and __fdividef
// bit for bit.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp_ftz(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// FP32 bond arithmetic on fixed-point coordinates (xi exact as an integer multiple of the quantum Q,
// then rounded once to FP32) and an FP32 shadow copy of u.  The band half-width B bounds
// |g32 - g| for g = xi.du - s0 |xi|^2 (in Q units) from the FP32 representation of u, the rounding
// of xi, du, the dot products and the final FMA; outside the band the FP32 sign equals the FP64
// decision, inside it the bond is re-decided in FP64 from the FP64 master state.
template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass1_mixed(StepArgs a, const float4* __restrict__ u32,
                                                      const double4* __restrict__ disp, int write_theta) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  if (write_theta && blockIdx.x == 0 && threadIdx.x == 0) *a.d_step += 1;
  float acc[1] = {0.0f};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const double s0 = a.bp[b].s0;
    const float sig = a.bp[b].sigma32;
    const bool can_break = a.bp[b].breaks != 0;
    const int4 Pi = a.pos32[t.i];
    const float4 Ui = u32[t.i];
    const float ui1 = fabsf(Ui.x) + fabsf(Ui.y) + (DIM == 3 ? fabsf(Ui.z) : 0.0f);
    // Band half-width B (see the comment above k_pass1_mixed) with |xi|_1 and |xi|^2 replaced by
    // their per-body maxima: B <= du1 k1 + k2 + k3 |g|, two FMAs per bond.
    const float xim = a.bp[b].xi1max, qm = a.bp[b].qmax;
    const float band_k1 = a.band_c * fmaf(6.0f * 5.9604645e-8f, xim, 1.01f);
    const float band_k2 = a.band_c * fmaf(sig, fmaf(2.01f, xim, 3.02f),
                                          5.9604645e-8f * fmaf(2.0f * xim, ui1, 6.0f * sig * qm));
    const float band_k3 = a.band_c * 5.9604645e-8f;
    uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    constexpr int U = kU32;
    int32_t jn[U];
    uint32_t wn[U];
    load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      int32_t j[U];
      uint32_t wd[U];
      int4 Pj[U];
      float4 Uj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        j[u] = jn[u];
        wd[u] = wn[u];
        Pj[u] = a.pos32[j[u]];
        Uj[u] = u32[j[u]];
      }
      load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
      // FP32 decisions of the batch; bonds inside the rounding band are flagged (code 2) and re-decided
      // in FP64 below, in a warp-uniform block outside the unrolled arithmetic.
      float dv[U], vj[U];
      int code[U];
      bool intact[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float ex = (float)(Pj[u].x - Pi.x), ey = (float)(Pj[u].y - Pi.y);
        const float ez = DIM == 3 ? (float)(Pj[u].z - Pi.z) : 0.0f;
        const float dx = Uj[u].x - Ui.x, dy = Uj[u].y - Ui.y, dz = DIM == 3 ? Uj[u].z - Ui.z : 0.0f;
        float d = ex * dx + ey * dy;
        if (DIM == 3) d = fmaf(ez, dz, d);
        dv[u] = d;
        vj[u] = __int_as_float(Pj[u].w);
        intact[u] = (wd[u] >> t.lane) & 1u;
        code[u] = 0;
        if (a.check && can_break && intact[u]) {
          float q = ex * ex + ey * ey;
          if (DIM == 3) q = fmaf(ez, ez, q);
          const float g = fmaf(-sig, q, d);
          const float du1 = fabsf(dx) + fabsf(dy) + fabsf(dz);
          const float B = fmaf(du1, band_k1, fmaf(band_k3, fabsf(g), band_k2));
          code[u] = fabsf(g) > B ? (g >= 0.0f ? 1 : 0) : 2;
        }
      }
      if (a.check) {
        bool band = false;
#pragma unroll
        for (int u = 0; u < U; ++u) band = band || code[u] == 2;
        if (__any_sync(kFull, band)) {
          for (int u = 0; u < U; ++u)
            if (code[u] == 2) {
              code[u] = fp64_breaks<DIM>(a, t.i, j[u], disp, s0) ? 1 : 0;
              atomicAdd(&a.counters[0], 1ull);
            }
        }
        if (a.validate) {
          for (int u = 0; u < U; ++u)
            if (can_break && intact[u] && (code[u] == 1) != fp64_breaks<DIM>(a, t.i, j[u], disp, s0))
              atomicAdd(&a.counters[1], 1ull);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned m = __ballot_sync(kFull, code[u] == 1);
          if (m) {
            intact[u] = intact[u] && code[u] != 1;
            if (t.lane == 0) bw[k0 + u * SPLIT] = wd[u] & ~m;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) acc[0] += intact[u] ? vj[u] * dv[u] : 0.0f;
    }
  }
  split_reduce<SPLIT, 1>(acc);
  if (t.active && t.sub == 0 && write_theta) {
    const float th = a.aA32[t.i] * acc[0];
    const float mu = a.mu32[t.i];
    a.theta32[t.i] = th;
    // gathered by pass 2: (K - G/3) Q theta_i / m_i and G / m_i (Q folded into the first)
    a.thm32[t.i] = make_float2(a.bp[b].Kp32 * (th * mu), a.bp[b].G32 * mu);
  }
}

template <int DIM, int SPLIT>
__global__ void __launch_bounds__(512) k_pass2_mixed(StepArgs a, const float4* __restrict__ u32,
                                                      float4* __restrict__ u32_out,
                                                      const double4* __restrict__ disp,
                                                      double4* __restrict__ disp_out) {
  const SliceIdx t = slice_index<SPLIT>(a.n_pad, a.slice_ptr);
  float f[3] = {0.0f, 0.0f, 0.0f};
  int b = 0;
  if (t.active) {
    b = a.body ? a.body[t.i] : 0;
    const int4 Pi = a.pos32[t.i];
    const float4 Ui = u32[t.i];
    const float2 ti = a.thm32[t.i];
    const uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
    const int32_t* __restrict__ cl = a.col + t.base + t.lane;
    constexpr int U = kU32;
    int32_t jn[U];
    uint32_t wn[U];
    load_slots<U, SPLIT>(t, cl, bw, t.sub, jn, wn);
    for (int k0 = t.sub; k0 < t.W; k0 += U * SPLIT) {
      uint32_t wd[U];
      int4 Pj[U];
      float4 Uj[U];
      float2 tj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        wd[u] = wn[u];
        Pj[u] = a.pos32[jn[u]];
        Uj[u] = u32[jn[u]];
        tj[u] = a.thm32[jn[u]];
      }
      load_slots<U, SPLIT>(t, cl, bw, k0 + U * SPLIT, jn, wn);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float ex = (float)(Pj[u].x - Pi.x), ey = (float)(Pj[u].y - Pi.y);
        const float ez = DIM == 3 ? (float)(Pj[u].z - Pi.z) : 0.0f;
        float d = ex * (Uj[u].x - Ui.x) + ey * (Uj[u].y - Ui.y);
        float q = ex * ex + ey * ey;
        if (DIM == 3) {
          d = fmaf(ez, Uj[u].z - Ui.z, d);
          q = fmaf(ez, ez, q);
        }
        float c = fmaf(ti.y + tj[u].y, d * __frcp_rn(q), ti.x + tj[u].x);
        c = ((wd[u] >> t.lane) & 1u) ? c * __int_as_float(Pj[u].w) : 0.0f;
        f[0] = fmaf(c, ex, f[0]);
        f[1] = fmaf(c, ey, f[1]);
        if (DIM == 3) f[2] = fmaf(c, ez, f[2]);
      }
    }
  }
  split_reduce<SPLIT, 3>(f);
  if (t.active && t.sub == 0) {
    const double fd[3] = {(double)f[0], (double)f[1], (double)f[2]};
    double4 u;
    update(a, t.i, b, fd, disp, disp_out, u);
    const double sc = a.uscale;
    u32_out[t.i] = make_float4((float)(u.x * sc), (float)(u.y * sc), (float)(u.z * sc), 0.0f);
  }
}

// ------------------------------------------------------------ mixed path, TMA-staged index stream
// The neighbour indices and status words of a warp's slice are one contiguous stream.  Lane 0 keeps
// kStageBuf chunks of kStageCh slots in flight with 1D bulk copies (cp.async.bulk, completion on an
// mbarrier) into the warp's shared-memory ring, so the DRAM stream runs far ahead of the gathers,
// which read their indices from shared memory.  Every wait is bounded: on expiry the kernel records
// an error word, drains (again bounded) the copies it issued and skips its outputs.
constexpr int kStageCh = 16;   // slots per chunk: 2 KB of indices + 64 B of status words
constexpr int kStageBuf = 3;   // chunks in flight per warp
constexpr int kStageWarpBytes = kStageBuf * (kStageCh * 128 + kStageCh * 4) + 64;  // the general kernels' ring
constexpr unsigned kWaitLimit = 1u << 24;              // polls (a second bound besides the clock)
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s: no staged copy legitimately takes this long

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after kWaitNs of the global timer (or kWaitLimit polls, whichever first).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0; it < kWaitLimit; it += 64) {
    for (int k = 0; k < 64; ++k)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// Stage<NB, CH>: NB chunks of CH slots each (CH a multiple of 4, so every chunk's status words start
// on a 16-byte boundary); the general mixed kernels use kStageBuf x kStageCh, the lattice kernels a
// ring chosen by the autotuner (PD_OPT_LAT_STAGE), smaller rings leaving more of the SM's combined
// L1 / shared memory to the displacement gathers.
template <int NB, int CH>
struct StageGeom {
  static constexpr int kWarpBytes = NB * (CH * 128 + CH * 4) + 64;  // 64: the NB <= 8 barriers
};

template <int NB = kStageBuf, int CH = kStageCh>
struct Stage {
  uint64_t* bar;    // NB barriers
  int32_t* col;     // NB x CH x 32 indices
  uint32_t* words;  // NB x CH status words
  const int32_t* gcol;
  const uint32_t* gwords;
  int W, nchunks, issued;
};

template <int NB = kStageBuf, int CH = kStageCh>
__device__ __forceinline__ Stage<NB, CH> stage_init(unsigned char* smem, const SliceIdx& t, const StepArgs& a) {
  Stage<NB, CH> st;
  unsigned char* base = smem + (threadIdx.x >> 5) * StageGeom<NB, CH>::kWarpBytes;
  st.bar = reinterpret_cast<uint64_t*>(base);
  st.col = reinterpret_cast<int32_t*>(base + 64);
  st.words = reinterpret_cast<uint32_t*>(base + 64 + NB * CH * 128);
  st.gcol = a.col + t.base;
  st.gwords = a.bits + (t.base >> 5);
  st.W = t.W;
  st.nchunks = (t.W + CH - 1) / CH;
  st.issued = 0;
  if ((threadIdx.x & 31) == 0)
    for (int b = 0; b < NB; ++b) mbar_init(&st.bar[b], 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();
  return st;
}

// Lane 0: start the copy of chunk c into buffer c % NB.
template <int NB, int CH>
__device__ __forceinline__ void stage_issue(Stage<NB, CH>& st, int c) {
  const int b = c % NB;
  const int k0 = c * CH;
  const int n = min(CH, st.W - k0);  // a multiple of 4 (slot counts are)
  const unsigned cb = (unsigned)n * 128u, wb = (unsigned)n * 4u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(&st.bar[b], cb + wb);
  bulk_to_smem(st.col + b * CH * 32, st.gcol + (int64_t)k0 * 32, cb, &st.bar[b]);
  bulk_to_smem(st.words + b * CH, st.gwords + k0, wb, &st.bar[b]);
}

// After a failed wait: wait (bounded) for every chunk still in flight, so that no copy lands in
// shared memory after the block has moved on.
template <int NB, int CH>
__device__ __forceinline__ void stage_drain(Stage<NB, CH>& st, int from) {
  for (int c = from; c < st.issued; ++c) mbar_wait(&st.bar[c % NB], (unsigned)((c / NB) & 1));
}

template <int DIM, int KIN>
__global__ void __launch_bounds__(512) k_pass1_mixed_staged(StepArgs a, const float4* __restrict__ u32,
                                                             const double4* __restrict__ disp, int write_theta) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (write_theta && blockIdx.x == 0 && threadIdx.x == 0) *a.d_step += 1;
  if (!t.active) return;  // whole warps: the staging below is per warp
  auto st = stage_init<>(smem, t, a);
  const int lane = t.lane;
  const int b = a.body ? a.body[t.i] : 0;
  const double s0 = a.bp[b].s0;
  const float sig = a.bp[b].sigma32;
  const bool can_break = a.bp[b].breaks != 0;
  const int4 Pi = a.pos32[t.i];
  const float4 Ui = u32[t.i];
  const float ui1 = fabsf(Ui.x) + fabsf(Ui.y) + (DIM == 3 ? fabsf(Ui.z) : 0.0f);
  // Band half-width B (see the comment above k_pass1_mixed) with |xi|_1 and |xi|^2 replaced by
  // their per-body maxima: B <= du1 k1 + k2 + k3 |g|, two FMAs per bond.
  const float xim = a.bp[b].xi1max, qm = a.bp[b].qmax;
  const float band_k1 = a.band_c * fmaf(6.0f * 5.9604645e-8f, xim, 1.01f);
  const float band_k2 = a.band_c * fmaf(sig, fmaf(2.01f, xim, 3.02f),
                                        5.9604645e-8f * fmaf(2.0f * xim, ui1, 6.0f * sig * qm));
  const float band_k3 = a.band_c * 5.9604645e-8f;
  // Nonlinear bonds (KIN 1, u32 holds u / Q): g = eta.(2 xi + eta) - c |xi|^2, c = s0 (2 + s0), with
  // |g32 - g| <= K0 + h1 (K1 + K2 h1) + eps |g32|, h1 = |eta|_1 (see the comment above
  // fp64_breaks_nl): fixed-point coordinates (1 quantum per axis), the FP32 shadow of u and the
  // rounding of xi, the products, the sums and the final FMA.
  const float eps = 5.9604645e-8f, c32 = a.bp[b].s0nl32;
  const float nl_k0 = a.band_c * (c32 * fmaf(2.0f, xim, 3.0f) + eps * (4.0f * ui1 * xim + 7.0f * c32 * qm));
  const float nl_k1 = a.band_c * (2.0f + eps * (16.0f * xim + 4.0f * ui1));
  const float nl_k2 = a.band_c * 10.0f * eps;
  uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
  if (lane == 0)
    for (; st.issued < min(kStageBuf, st.nchunks); ++st.issued)
      if (!(a.expire && st.issued == 0)) stage_issue(st, st.issued);  // testing: chunk 0 never arrives
  float acc = 0.0f;
  bool ok = true;
  for (int c = 0; c < st.nchunks; ++c) {
    const int buf = c % kStageBuf;
    if (!mbar_wait(&st.bar[buf], (unsigned)((c / kStageBuf) & 1))) {
      ok = false;
      if (lane == 0) atomicExch(&a.counters[4], 1ull);
      stage_drain(st, c + 1);
      break;
    }
    const int32_t* cs = st.col + buf * kStageCh * 32 + lane;
    const uint32_t* ws = st.words + buf * kStageCh;
    const int k0 = c * kStageCh;
    const int n = min(kStageCh, st.W - k0);
    constexpr int U = kU32;
    for (int kk = 0; kk < n; kk += U) {
      int4 Pj[U];
      float4 Uj[U];
      int32_t j[U];
      uint32_t wd[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {  // n is a multiple of 4 = U
        j[u] = cs[(kk + u) * 32];
        wd[u] = ws[kk + u];
        Pj[u] = a.pos32[j[u]];
        Uj[u] = u32[j[u]];
      }
      // FP32 decisions of the batch; bonds inside the rounding band are flagged (code 2) and re-decided
      // in FP64 below, in a warp-uniform block outside the unrolled arithmetic.
      float dv[U], vj[U];
      int code[U];
      bool intact[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float ex = (float)(Pj[u].x - Pi.x), ey = (float)(Pj[u].y - Pi.y);
        const float ez = DIM == 3 ? (float)(Pj[u].z - Pi.z) : 0.0f;
        const float dx = Uj[u].x - Ui.x, dy = Uj[u].y - Ui.y, dz = DIM == 3 ? Uj[u].z - Ui.z : 0.0f;
        float d;
        if (KIN == 0) {
          d = ex * dx + ey * dy;
          if (DIM == 3) d = fmaf(ez, dz, d);
        } else {  // p = eta.(2 xi + eta) = |Y|^2 - |xi|^2 in quanta^2
          d = dx * fmaf(2.0f, ex, dx) + dy * fmaf(2.0f, ey, dy);
          if (DIM == 3) d = fmaf(dz, fmaf(2.0f, ez, dz), d);
        }
        dv[u] = d;
        vj[u] = __int_as_float(Pj[u].w);
        intact[u] = (wd[u] >> lane) & 1u;
        code[u] = 0;
        if (a.check && can_break && intact[u]) {
          float q = ex * ex + ey * ey;
          if (DIM == 3) q = fmaf(ez, ez, q);
          const float du1 = fabsf(dx) + fabsf(dy) + fabsf(dz);
          float g, B;
          if (KIN == 0) {
            g = fmaf(-sig, q, d);
            B = fmaf(du1, band_k1, fmaf(band_k3, fabsf(g), band_k2));
          } else {
            g = fmaf(-c32, q, d);
            B = fmaf(du1, fmaf(nl_k2, du1, nl_k1), fmaf(band_k3, fabsf(g), nl_k0));
          }
          code[u] = fabsf(g) > B ? (g >= 0.0f ? 1 : 0) : 2;
        }
        if (KIN == 1) {  // theta term |xi| e with e = p / (|Y| + |xi|) (Eqs 1.6, 1.10)
          const float yx = ex + dx, yy = ey + dy, yz = ez + dz;
          float q = ex * ex + ey * ey, y2 = yx * yx + yy * yy;
          if (DIM == 3) {
            q = fmaf(ez, ez, q);
            y2 = fmaf(yz, yz, y2);
          }
          const float xl = q * rsqrt_ftz(q);
          dv[u] = xl * (d * rcp_ftz(fmaf(y2, rsqrt_ftz(y2), xl)));
        }
      }
      if (a.check) {
        bool band = false;
#pragma unroll
        for (int u = 0; u < U; ++u) band = band || code[u] == 2;
        if (__any_sync(kFull, band)) {
          for (int u = 0; u < U; ++u)
            if (code[u] == 2) {
              code[u] = (KIN == 0 ? fp64_breaks<DIM>(a, t.i, j[u], disp, s0)
                                  : fp64_breaks_nl<DIM>(a, t.i, j[u], disp)) ? 1 : 0;
              atomicAdd(&a.counters[0], 1ull);
            }
        }
        if (a.validate) {
          for (int u = 0; u < U; ++u)
            if (can_break && intact[u] &&
                (code[u] == 1) != (KIN == 0 ? fp64_breaks<DIM>(a, t.i, j[u], disp, s0)
                                            : fp64_breaks_nl<DIM>(a, t.i, j[u], disp)))
              atomicAdd(&a.counters[1], 1ull);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const unsigned m = __ballot_sync(kFull, code[u] == 1);
          if (m) {
            intact[u] = intact[u] && code[u] != 1;
            if (lane == 0) bw[k0 + kk + u] = wd[u] & ~m;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) acc += intact[u] ? vj[u] * dv[u] : 0.0f;
    }
    __syncwarp();  // every lane is done with this buffer before it is refilled
    if (lane == 0 && st.issued < st.nchunks) stage_issue(st, st.issued++);
  }
  if (ok && write_theta) {
    const float th = a.aA32[t.i] * acc;
    const float mu = a.mu32[t.i];
    a.theta32[t.i] = th;
    a.thm32[t.i] = make_float2(a.bp[b].Kp32 * (th * mu), (KIN == 0 ? a.bp[b].G32 : a.bp[b].G32q) * mu);
  }
}

template <int DIM, int KIN>
__global__ void __launch_bounds__(512) k_pass2_mixed_staged(StepArgs a, const float4* __restrict__ u32,
                                                             float4* __restrict__ u32_out,
                                                             const double4* __restrict__ disp,
                                                             double4* __restrict__ disp_out) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (!t.active) return;
  auto st = stage_init<>(smem, t, a);
  const int lane = t.lane;
  const int b = a.body ? a.body[t.i] : 0;
  const int4 Pi = a.pos32[t.i];
  const float4 Ui = u32[t.i];
  const float2 ti = a.thm32[t.i];
  if (lane == 0)
    for (; st.issued < min(kStageBuf, st.nchunks); ++st.issued)
      if (!(a.expire && st.issued == 0)) stage_issue(st, st.issued);  // testing: chunk 0 never arrives
  float f[3] = {0.0f, 0.0f, 0.0f};
  bool ok = true;
  for (int c = 0; c < st.nchunks; ++c) {
    const int buf = c % kStageBuf;
    if (!mbar_wait(&st.bar[buf], (unsigned)((c / kStageBuf) & 1))) {
      ok = false;
      if (lane == 0) atomicExch(&a.counters[4], 1ull);
      stage_drain(st, c + 1);
      break;
    }
    const int32_t* cs = st.col + buf * kStageCh * 32 + lane;
    const uint32_t* ws = st.words + buf * kStageCh;
    const int n = min(kStageCh, st.W - c * kStageCh);
    constexpr int U = kU32;
    for (int kk = 0; kk < n; kk += U) {
      int4 Pj[U];
      float4 Uj[U];
      float2 tj[U];
      uint32_t wd[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t j = cs[(kk + u) * 32];
        wd[u] = ws[kk + u];
        Pj[u] = a.pos32[j];
        Uj[u] = u32[j];
        tj[u] = a.thm32[j];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float ex = (float)(Pj[u].x - Pi.x), ey = (float)(Pj[u].y - Pi.y);
        const float ez = DIM == 3 ? (float)(Pj[u].z - Pi.z) : 0.0f;
        if (KIN == 0) {
          float d = ex * (Uj[u].x - Ui.x) + ey * (Uj[u].y - Ui.y);
          float q = ex * ex + ey * ey;
          if (DIM == 3) {
            d = fmaf(ez, Uj[u].z - Ui.z, d);
            q = fmaf(ez, ez, q);
          }
          float cf = fmaf(ti.y + tj[u].y, d * __frcp_rn(q), ti.x + tj[u].x);
          cf = ((wd[u] >> lane) & 1u) ? cf * __int_as_float(Pj[u].w) : 0.0f;
          f[0] = fmaf(cf, ex, f[0]);
          f[1] = fmaf(cf, ey, f[1]);
          if (DIM == 3) f[2] = fmaf(cf, ez, f[2]);
        } else {  // Eq 1.14 for both ends along M = Y / |Y| (Eq 1.13), in quanta (Q folded into thm32)
          const float hx = Uj[u].x - Ui.x, hy = Uj[u].y - Ui.y, hz = DIM == 3 ? Uj[u].z - Ui.z : 0.0f;
          const float yx = ex + hx, yy = ey + hy, yz = ez + hz;
          float pp = hx * (ex + yx) + hy * (ey + yy);
          float q = ex * ex + ey * ey, y2 = yx * yx + yy * yy;
          if (DIM == 3) {
            pp = fmaf(hz, ez + yz, pp);
            q = fmaf(ez, ez, q);
            y2 = fmaf(yz, yz, y2);
          }
          // rsqrtf here: with rsqrt_ftz ptxas gives the 2D instance 40 registers and spills
          const float xl = q * rsqrtf(q), ry = rsqrtf(y2);
          const float e = pp * rcp_ftz(fmaf(y2, ry, xl));
          float cf = fmaf(ti.x + tj[u].x, xl, (ti.y + tj[u].y) * e) * ry;
          cf = ((wd[u] >> lane) & 1u) ? cf * __int_as_float(Pj[u].w) : 0.0f;
          f[0] = fmaf(cf, yx, f[0]);
          f[1] = fmaf(cf, yy, f[1]);
          if (DIM == 3) f[2] = fmaf(cf, yz, f[2]);
        }
      }
    }
    __syncwarp();
    if (lane == 0 && st.issued < st.nchunks) stage_issue(st, st.issued++);
  }
  if (ok) {
    const double fd[3] = {(double)f[0], (double)f[1], (double)f[2]};
    double4 u;
    update(a, t.i, b, fd, disp, disp_out, u);
    const double sc = a.uscale;
    u32_out[t.i] = make_float4((float)(u.x * sc), (float)(u.y * sc), (float)(u.z * sc), 0.0f);
  }
}


// ------------------------------------------------------------------- lattice layout, mixed form
// On a lattice body (pd_build.cu: every bond vector is h n with an integer n; slot k of every slice
// holds direction k of the table for every lane) the bond vector of a slot is one value for the
// whole warp, read from constant memory, and the FP32 arithmetic runs in lattice units:
//   u' = u / h (the FP32 shadow, written by the FP64 update, with |u'|_inf in its 4th word),
//   d'_ij = n.(u'_j - u'_i) = xi.(u_j - u_i) / h^2 (Eqs 2.4, 2.7: x e),
//   pass 1: sigma_i = sum_j rho_ij d'_ij, theta_i = A sigma_i / N_i (Eq 1.6 with m_i = V h^2 N_i),
//   pass 2: F_i / V_i = G / (h N_ref) sum_j rho_ij n [P_i + P_j + (N_ref/N_i + N_ref/N_j) d'_ij / |n|^2]
//           (Eq 2.2), P_i = (K - G/3) / G theta_i N_ref / N_i,
// so that no coordinate is gathered and the per-bond work is the displacement gather, the dot
// product and the force FMAs.  The constants that multiply every bond (1 / |n|^2 per direction,
// (K - G/3) A / (G N_ref) per body) are carried as FP32 hi + lo pairs, and the interior factors
// N_ref / N_i are exactly 1, so no rounding of a constant is shared by all bonds of a direction or
// of the body (such a shared rounding would shift every vibration frequency by the same amount and
// grow as a phase error).  The failure check (Eq 1.30, d' >= s0 |n|^2) is decided in FP32 where its
// rounding band (see BodyDev) cannot reach the threshold, and in FP64 from the master state
// otherwise: a screen against the band with |n|^2 bounded per body, |u'_i| per particle and |u'_j| by
// the body's largest |u'| (raised by every kernel that writes the shadow) settles nearly every bond
// with one FMA and one max per slot; a warp with any bond the screen does not settle evaluates the
// full band and re-decides the bonds inside it with the FP64 path's arithmetic.
// Sized to a multiple of 4: slice widths are rounded up to 4 slots, and the slots past the table
// (unused, status 0) still index it.
constexpr int kLatPad3 = (kLatDirs3 + 3) & ~3, kLatPad2 = (kLatDirs2 + 3) & ~3;
__constant__ float4 c_lat3[kLatPad3];   // (n_x, n_y, n_z, |n|^2)
__constant__ float2 c_latr3[kLatPad3];  // 1 / |n|^2 as hi + lo
__constant__ float4 c_lat2[kLatPad2];
__constant__ float2 c_latr2[kLatPad2];
// w' = 1 / |n| as hi + lo: the per-direction factor of the influence function w = delta / |xi|
// (w = (delta / h) w', and delta / h cancels between w and m_i)
__constant__ float2 c_latw3[kLatPad3];
__constant__ float2 c_latw2[kLatPad2];
// |n| rounded to FP32 (nonlinear bonds: e' = (|Y'|^2 - |n|^2) / (|Y'| + |n|) and the dilatation term |n| e')
__constant__ float c_latn3[kLatPad3];
__constant__ float c_latn2[kLatPad2];

template <int DIM>
__device__ __forceinline__ float4 lat_dir(int k) {
  return DIM == 3 ? c_lat3[k] : c_lat2[k];
}
template <int DIM>
__device__ __forceinline__ float2 lat_rcp(int k) {
  return DIM == 3 ? c_latr3[k] : c_latr2[k];
}
template <int DIM>
__device__ __forceinline__ float2 lat_wgt(int k) {
  return DIM == 3 ? c_latw3[k] : c_latw2[k];
}
template <int DIM>
__device__ __forceinline__ float lat_len(int k) {
  return DIM == 3 ? c_latn3[k] : c_latn2[k];
}
// Entry k ^ 1 of the table is -entry k exactly (integer components), with the same |n|^2, 1 / |n|^2
// and w', and a batch starts at a multiple of 4 slots: its four directions are two loaded entries
// and their negations, the sign folded into the arithmetic that uses them (bitwise the same values
// as loading all four).
__device__ __forceinline__ float4 lat_twin(const float4& d, bool odd) {
  return odd ? make_float4(-d.x, -d.y, -d.z, d.w) : d;
}

// The update of the lattice kernels (Eq 2.11 as update() computes it) with F_i / V_i = lat_C x the
// FP32 force sum f and the constants folded: v += lat_K f (+ lat_Kb b), u += dt v, so that a free
// particle costs two FP64 FMAs per component; the z components stay zero in 2D.  Particles under a
// boundary condition and the relaxation solver take update().
template <int DIM>
__device__ __forceinline__ void update_lat(const StepArgs& a, int64_t i, int b, const float f[3],
                                           const double4* __restrict__ disp, double4* __restrict__ disp_out,
                                           double4& u) {
  const BodyDev& bp = a.bp[b];
  const uint8_t fl = a.flag ? a.flag[i] : (uint8_t)0;
  if (a.adr || fl != 0) {
    const double C = bp.lat_C;
    const double fd[3] = {C * (double)f[0], C * (double)f[1], C * (double)f[2]};
    update(a, i, b, fd, disp, disp_out, u);
    return;
  }
  u = disp[i];
  double4 v = a.vel[i];
  const double K = bp.lat_K;
  v.x = fma(K, (double)f[0], v.x);
  v.y = fma(K, (double)f[1], v.y);
  if (DIM == 3) v.z = fma(K, (double)f[2], v.z);
  if (a.bacc) {
    const double4 bb = a.bacc[i];
    const double kb = bp.lat_Kb;
    v.x = fma(kb, bb.x, v.x);
    v.y = fma(kb, bb.y, v.y);
    if (DIM == 3) v.z = fma(kb, bb.z, v.z);
  }
  const double dt = bp.dt;
  u.x = fma(dt, v.x, u.x);
  u.y = fma(dt, v.y, u.y);
  if (DIM == 3) u.z = fma(dt, v.z, u.z);
  disp_out[i] = u;  // .w carries V_i unchanged
  a.vel[i] = v;
}

// The FP32 shadow of a displacement in lattice units, (u / h, |u / h|_inf).
template <int DIM>
__device__ __forceinline__ float4 shadow_lat(double inv_h, const double4& u) {
  const float x = (float)(u.x * inv_h), y = (float)(u.y * inv_h), z = DIM == 3 ? (float)(u.z * inv_h) : 0.0f;
  return make_float4(x, y, z, fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z))));
}

// lat_dprime with the x and y differences as one packed FP32 pair addition (the same roundings).
template <int DIM>
__device__ __forceinline__ float lat_dprime_pair(const float4& dn, const float4& uj, const float4& nui) {
  const float2 dxy = __fadd2_rn(make_float2(uj.x, uj.y), make_float2(nui.x, nui.y));
  return lat_dprime_d<DIM>(dn.x, dn.y, dn.z, dxy.x, dxy.y, uj.z + nui.z);
}

// The two-word shadow: hi as shadow_lat, lo = u / h - hi rounded to FP32 (the subtraction is exact in
// FP64), so that hi + lo carries u / h to about 2^-48 of its size.
template <int DIM>
__device__ __forceinline__ void shadow_lat_lo(double inv_h, const double4& u, float4& hi, float4& lo) {
  const double x = u.x * inv_h, y = u.y * inv_h, z = DIM == 3 ? u.z * inv_h : 0.0;
  const float hx = (float)x, hy = (float)y, hz = (float)z;
  hi = make_float4(hx, hy, hz, fmaxf(fabsf(hx), fmaxf(fabsf(hy), fabsf(hz))));
  lo = make_float4((float)(x - (double)hx), (float)(y - (double)hy), (float)(z - (double)hz), 0.0f);
}

// The FP32 shadow of a displacement in the context's format.
__device__ __forceinline__ float4 shadow_of(const StepArgs& a, int b, const double4& u) {
  if (a.lattice) {
    const double s = a.bp[b].lat_inv_h;
    const float x = (float)(u.x * s), y = (float)(u.y * s), z = (float)(u.z * s);
    return make_float4(x, y, z, fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z))));
  }
  const double sc = a.uscale;
  return make_float4((float)(u.x * sc), (float)(u.y * sc), (float)(u.z * sc), 0.0f);
}

// Raises the body's bound umax[b] to at least U (|u'|_inf of a shadow just written; non-negative
// floats order as their bits): one atomic per warp when its particles share a body, else one per
// lane.  All 32 lanes call it.  A NaN U raises the bound to NaN, which settles nothing.
__device__ __forceinline__ void lat_raise_umax(unsigned* umax, int b, float U) {
  const unsigned bits = __float_as_uint(U);
  const int b0 = __shfl_sync(kFull, b, 0);
  if (__all_sync(kFull, b == b0)) {
    const unsigned m = __reduce_max_sync(kFull, bits);
    if ((threadIdx.x & 31) == 0) atomicMax(umax + b0, m);
  } else {
    atomicMax(umax + b, bits);
  }
}

// WI: influence function w = delta / |xi| (its per-direction factor w' = 1 / |n| multiplies each
// bond's term in both sums); WI = false: w = 1.
// The row loop of the lattice kernels, called twice in each kernel: with UNI, bounded by the
// context's common slice width (a kernel argument, so the slot index and everything indexed by it
// is warp-uniform by construction and the direction table is read through the uniform datapath);
// otherwise by the slice's own width.  The staged-copy wait goes through a warp vote, so the loop's
// exit is warp-uniform as well.
template <int NB, int CH, class Body>
__device__ __forceinline__ bool lat_rows(const StepArgs& a, Stage<NB, CH>& st, int W, int lane, Body body) {
  const int nchunks = (W + CH - 1) / CH;
  if (lane == 0)
    for (; st.issued < min(NB, nchunks); ++st.issued)
      if (!(a.expire && st.issued == 0)) stage_issue(st, st.issued);  // testing: chunk 0 never arrives
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c % NB;
    if (!__all_sync(kFull, mbar_wait(&st.bar[buf], (unsigned)((c / NB) & 1)))) {
      if (lane == 0) atomicExch(&a.counters[4], 1ull);
      stage_drain(st, c + 1);
      return false;
    }
    const int32_t* cs = st.col + buf * CH * 32 + lane;
    const uint32_t* ws = st.words + buf * CH;
    const int k0 = c * CH;
    const int n = min(CH, W - k0);
    for (int kk = 0; kk < n; kk += kU32) {  // n is a multiple of 4 = kU32
      const uint4 w4 = *reinterpret_cast<const uint4*>(ws + kk);  // 16-byte aligned: CH and kk multiples of 4
      if ((w4.x | w4.y | w4.z | w4.w) == 0u) continue;  // no intact bond in the batch (the same words in every lane)
      body(cs + kk * 32, ws + kk, w4, k0 + kk);
    }
    __syncwarp();  // every lane is done with this buffer before it is refilled
    if (lane == 0 && st.issued < nchunks) stage_issue(st, st.issued++);
  }
  return true;
}

// LO: two-word shadow (u' = hi + lo, PD_OPT_SHADOW_LO): each end's lo words come from lo32 and the
// differences are formed as (hi_j - hi_i) + (lo_j - lo_i).
template <int DIM, bool WI, bool LO, int NB, int CH>
__global__ void __launch_bounds__(512) k_pass1_lat(StepArgs a, const float4* __restrict__ u32,
                                                    const float4* __restrict__ lo32,
                                                    const double4* __restrict__ disp, int write_theta) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (write_theta && blockIdx.x == 0 && threadIdx.x == 0) *a.d_step += 1;
  if (blockIdx.x == 0)  // the bound of the shadow that pass 2 writes next starts from zero
    for (int k = threadIdx.x; k < a.nbody; k += blockDim.x) a.lat_umax_next[k] = 0u;
  if (!t.active) return;  // whole warps: the staging below is per warp
  auto st = stage_init<NB, CH>(smem, t, a);
  const int lane = t.lane;
  const int b = a.body ? a.body[t.i] : 0;
  const BodyDev& bp = a.bp[b];
  const double s0 = bp.s0;
  const float s0f = bp.lat_s0;
  const bool can_break = bp.breaks != 0;
  const float4 Ui = u32[t.i];
  const float4 Li = LO ? lo32[t.i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const float4 nUi = make_float4(-Ui.x, -Ui.y, -Ui.z, 0.0f);  // u'_j - u'_i as u'_j + (-u'_i), exactly
  const float Kfast = bp.lat_Kfast;
  const bool checking = a.check != 0;  // warp-uniform (can_break is per body: per lane in a batch)
  // the screen's per-particle part with the body's bound of |u'_j| (pd_lattice.h); -inf settles
  // every bond with a finite extension, for a body without failure and in a pass that checks
  // nothing, so that the per-batch test needs no flag (a NaN still reaches the slow path, which
  // decides nothing unless checking)
  const float umax_b = lat_umax_bound(__uint_as_float(a.lat_umax[b]));
  const float scr_i = (can_break && checking) ? lat_screen_part(Kfast, Ui.w, umax_b, bp.lat_Kcfast) : -INFINITY;
  const bool every = checking && a.validate != 0;  // validation: every batch takes the slow path
  uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
  float acc = 0.0f;
  const uint32_t lmask = 1u << lane;
  // one batch of U = 4 slots starting at slot k: the extensions of the intact bonds (0 for the
  // others) and the screen first, the failure decisions next (the rare slow path zeroes the terms
  // of the bonds it breaks), then the dilatation terms in slot order, so that the sum does not
  // depend on whether a bond broke here or in an earlier check (a state read between steps)
  auto batch = [&](const int32_t* cs, const uint32_t* ws, uint4 w4, int k) {
    constexpr int U = kU32;
    const uint32_t wd[U] = {w4.x, w4.y, w4.z, w4.w};
    float4 Uj[U], Lj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t j = cs[u * 32];
      Uj[u] = u32[j];
      if (LO) Lj[u] = lo32[j];
    }
    float dm[U];
    float gmax = -INFINITY;  // the largest g = d' - s0 |n|^2 of the batch's intact bonds (0 - s0 |n|^2 for the others)
    const float4 dA = lat_dir<DIM>(k), dB = lat_dir<DIM>(k + 2);  // k is a multiple of 4
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float4 dn = lat_twin(u < 2 ? dA : dB, u & 1);
      const float d =
          LO ? lat_dprime_d<DIM>(dn.x, dn.y, dn.z, lat_delta_lo(Uj[u].x, Lj[u].x, Ui.x, Li.x),
                                 lat_delta_lo(Uj[u].y, Lj[u].y, Ui.y, Li.y), lat_delta_lo(Uj[u].z, Lj[u].z, Ui.z, Li.z))
             : lat_dprime_pair<DIM>(dn, Uj[u], nUi);
      dm[u] = (wd[u] & lmask) ? d : 0.0f;
      gmax = lat_max_nan(gmax, lat_g(dm[u], s0f, dn.w));
    }
    const bool near = !(gmax + scr_i < 0.0f);
    if (__any_sync(kFull, near) | every) {
      // full band for the bonds the screen did not settle, FP64 inside it; the neighbour index and
      // its |u'| are reloaded (staged chunk, L1) so that little stays live across this block
      unsigned brk = 0u;
#pragma unroll 1
      for (int u = 0; u < U; ++u) {
        int code = 0;
        if (checking && can_break && (ws[u] & lmask) != 0u) {
          const int32_t jj = cs[u * 32];
          const float Ujw = u32[jj].w;
          const float q = lat_dir<DIM>(k + u).w;
          const float du = u == 0 ? dm[0] : (u == 1 ? dm[1] : (u == 2 ? dm[2] : dm[3]));  // no indexed array
          code = lat_code(lat_g(du, s0f, q), Ui.w, Ujw, s0f, q, bp.lat_Kf, bp.lat_sq, bp.lat_eps_c, bp.lat_s0n1);
          if (code == 2) {
            code = fp64_breaks_inl<DIM>(a, t.i, jj, disp, s0) ? 1 : 0;
            atomicAdd(&a.counters[0], 1ull);
          }
          if (a.validate && (code == 1) != fp64_breaks_inl<DIM>(a, t.i, jj, disp, s0))
            atomicAdd(&a.counters[1], 1ull);
        }
        const unsigned m = __ballot_sync(kFull, code == 1);
        if (m) {
          if (lane == 0) bw[k + u] = ws[u] & ~m;
          if (code == 1) brk |= 1u << u;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) dm[u] = ((brk >> u) & 1u) ? 0.0f : dm[u];
    }
    float2 wA = make_float2(1.0f, 0.0f), wB = wA;
    if (WI) {
      wA = lat_wgt<DIM>(k);
      wB = lat_wgt<DIM>(k + 2);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (WI) {  // acc += w' d' with w' as hi + lo
        const float2 wk = u < 2 ? wA : wB;
        acc = fmaf(wk.x, dm[u], fmaf(wk.y, dm[u], acc));
      } else {
        acc += dm[u];
      }
    }
  };
  const bool ok = a.lat_wuni > 0 ? lat_rows<NB, CH>(a, st, a.lat_wuni, lane, batch)
                                 : lat_rows<NB, CH>(a, st, st.W, lane, batch);
  if (ok && write_theta) {
    const float2 f = a.lat_f[t.i];  // (N_ref / N_i, A / N_i)
    a.theta32[t.i] = f.y * acc;
    const float x = acc * (f.x * f.x);
    // the record pass 2 gathers: (u'_i, P_i)
    a.lat_up[t.i] = make_float4(Ui.x, Ui.y, Ui.z, fmaf(bp.lat_lam_hi, x, bp.lat_lam_lo * x));
  }
}

template <int DIM, bool WI, bool LO, int NB, int CH>
__global__ void __maxnreg__(56) k_pass2_lat(StepArgs a, const float4* __restrict__ u32,
                                                    float4* __restrict__ u32_out,
                                                    const float4* __restrict__ lo32, float4* __restrict__ lo32_out,
                                                    const double4* __restrict__ disp,
                                                    double4* __restrict__ disp_out) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (!t.active) return;
  auto st = stage_init<NB, CH>(smem, t, a);
  const int lane = t.lane;
  const int b = a.body ? a.body[t.i] : 0;
  const float4 Ui = a.lat_up[t.i];  // (u'_i, P_i)
  const float4 Li = LO ? lo32[t.i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const float4 nUi = make_float4(-Ui.x, -Ui.y, -Ui.z, 0.0f);  // u'_j - u'_i as u'_j + (-u'_i), exactly
  const float rho_i = a.lat_f[t.i].x;
  // every particle around this slice (lanes and neighbours) has N_j = N_ref: N_ref/N_i + N_ref/N_j
  // = 2 exactly, so the per-neighbour factor is not gathered (the result is bitwise the same); the
  // vote makes the per-slice flag warp-uniform for the compiler
  const bool interior = __all_sync(kFull, a.lat_int[t.i >> 5] != 0);
  const uint32_t lmask = 1u << lane;
  float f[3] = {0.0f, 0.0f, 0.0f};
  auto batch_t = [&](auto intr, auto full, const int32_t* cs, uint4 w4, int k) {
    constexpr bool INTR = decltype(intr)::value;
    constexpr bool FULL = decltype(full)::value;  // every bond of the batch intact for every lane
    constexpr int U = kU32;
    const uint32_t wd[U] = {w4.x, w4.y, w4.z, w4.w};
    float4 Uj[U], Lj[U];
    float rr[U], cfm[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t j = cs[u * 32];
      Uj[u] = a.lat_up[j];
      if (LO) Lj[u] = lo32[j];
      rr[u] = INTR ? 2.0f : rho_i + a.lat_rho[j];
    }
    const float4 dA = lat_dir<DIM>(k), dB = lat_dir<DIM>(k + 2);  // k is a multiple of 4
    const float2 rA = lat_rcp<DIM>(k), rB = lat_rcp<DIM>(k + 2);
    float2 wA = make_float2(1.0f, 0.0f), wB = wA;
    if (WI) {
      wA = lat_wgt<DIM>(k);
      wB = lat_wgt<DIM>(k + 2);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float4 dn = lat_twin(u < 2 ? dA : dB, u & 1);
      const float2 r = u < 2 ? rA : rB;
      const float d =
          LO ? lat_dprime_d<DIM>(dn.x, dn.y, dn.z, lat_delta_lo(Uj[u].x, Lj[u].x, Ui.x, Li.x),
                                 lat_delta_lo(Uj[u].y, Lj[u].y, Ui.y, Li.y), lat_delta_lo(Uj[u].z, Lj[u].z, Ui.z, Li.z))
             : lat_dprime<DIM>(dn.x, dn.y, dn.z, Uj[u].x, Uj[u].y, Uj[u].z, Ui.x, Ui.y, Ui.z);
      const float dr = fmaf(d, r.x, d * r.y);  // d / |n|^2 with 1 / |n|^2 carried as hi + lo
      float cf = fmaf(rr[u], dr, Ui.w + Uj[u].w);
      if (WI) {  // cf w' with w' as hi + lo
        const float2 wk = u < 2 ? wA : wB;
        cf = fmaf(cf, wk.x, cf * wk.y);
      }
      cfm[u] = FULL ? cf : ((wd[u] & lmask) ? cf : 0.0f);
    }
#pragma unroll
    for (int p = 0; p < U / 2; ++p) {  // twin slots 2p, 2p + 1: cf_a n + cf_b (-n) = (cf_a - cf_b) n
      const float dd = cfm[2 * p] - cfm[2 * p + 1];
      const float4& dn = p == 0 ? dA : dB;
      f[0] = fmaf(dd, dn.x, f[0]);
      f[1] = fmaf(dd, dn.y, f[1]);
      if (DIM == 3) f[2] = fmaf(dd, dn.z, f[2]);
    }
  };
  auto batch = [&](const int32_t* cs, const uint32_t*, uint4 w4, int k) {
    if (interior) {
      if ((w4.x & w4.y & w4.z & w4.w) == 0xffffffffu) batch_t(std::true_type{}, std::true_type{}, cs, w4, k);
      else batch_t(std::true_type{}, std::false_type{}, cs, w4, k);
    } else {
      batch_t(std::false_type{}, std::false_type{}, cs, w4, k);
    }
  };
  const bool ok = a.lat_wuni > 0 ? lat_rows<NB, CH>(a, st, a.lat_wuni, lane, batch)
                                 : lat_rows<NB, CH>(a, st, st.W, lane, batch);
  if (ok) {  // warp-uniform
    double4 u;
    update_lat<DIM>(a, t.i, b, f, disp, disp_out, u);
    float4 hi;
    if (LO) {
      float4 lo;
      shadow_lat_lo<DIM>(a.bp[b].lat_inv_h, u, hi, lo);
      lo32_out[t.i] = lo;
    } else {
      hi = shadow_lat<DIM>(a.bp[b].lat_inv_h, u);
    }
    u32_out[t.i] = hi;
    lat_raise_umax(a.lat_umax_next, b, hi.w);
  }
}

// ------------------------------------------------- lattice layout, mixed form, nonlinear bonds
// Geometrically nonlinear bonds (Eqs 1.10, 1.13, 1.14) on the lattice layout, in lattice units:
// eta' = u'_j - u'_i, Y' = n + eta', p = |Y'|^2 - |n|^2 = eta'.(2 n + eta') (no cancellation),
// e' = e / h = p / (|Y'| + |n|), M = Y' / |Y'|;
//   pass 1: theta_i = (A / N_i) sum_j |n| e'_ij (Eq 1.6 with m_i = V h^2 N_i, w = 1);
//   pass 2: F_i / V_i = G / (h N_ref) sum_j M [(P_i + P_j) |n| + (N_ref/N_i + N_ref/N_j) e'_ij] with
//           P_i = (K - G/3) / G theta_i N_ref / N_i (Eq 1.14 with the nonlinear e and M),
// which for small eta' is the linearized kernels' sum term by term.  The failure check (Eq 1.30 as
// p >= s0 (2 + s0) |n|^2) is decided in FP32 outside the band of pd_lattice.h (LatBandNL) and in FP64
// from the master state otherwise (fp64_breaks_nl, the FP64 nonlinear kernels' arithmetic); the
// screen uses the body's bound of |u'_j| as the linearized kernels do.  LO: the two-word shadow (eta'
// formed as (hi_j - hi_i) + (lo_j - lo_i); the band of pd_lattice.h covers both forms).
template <int DIM, bool LO, int NB, int CH>
__global__ void __maxnreg__(72) k_pass1_latnl(StepArgs a, const float4* __restrict__ u32,
                                               const float4* __restrict__ lo32,
                                                      const double4* __restrict__ disp, int write_theta) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (write_theta && blockIdx.x == 0 && threadIdx.x == 0) *a.d_step += 1;
  if (blockIdx.x == 0)  // the bound of the shadow that pass 2 writes next starts from zero
    for (int k = threadIdx.x; k < a.nbody; k += blockDim.x) a.lat_umax_next[k] = 0u;
  if (!t.active) return;  // whole warps: the staging below is per warp
  auto st = stage_init<NB, CH>(smem, t, a);
  const int lane = t.lane;
  const int b = a.body ? a.body[t.i] : 0;
  const BodyDev& bp = a.bp[b];
  const bool can_break = bp.breaks != 0;
  const bool checking = a.check != 0;
  const bool screening = can_break && checking;
  const bool every = checking && a.validate != 0;
  const float4 Ui = u32[t.i];
  const float4 Li = LO ? lo32[t.i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const float4 nUi = make_float4(-Ui.x, -Ui.y, -Ui.z, 0.0f);
  const float c32 = bp.s0nl32;
  // the screen's per-lane coefficients with S = U_i + the body's bound of |u'_j|
  const float Smax = Ui.w + lat_umax_bound(__uint_as_float(a.lat_umax[b]));
  const float f0 = fmaf(bp.nl_F0s, Smax, bp.nl_F0), f1 = fmaf(bp.nl_F1s, Smax, bp.nl_F1), F2 = bp.nl_F2;
  uint32_t* __restrict__ bw = a.bits + (t.base >> 5);
  float acc = 0.0f;
  const uint32_t lmask = 1u << lane;
  // per batch of 4 slots: p and |Y'|^2 of each bond, the screen, the decisions (the rare slow path
  // marks the bonds it breaks), then the dilatation terms in slot order (as the linearized kernel)
  auto batch = [&](const int32_t* cs, const uint32_t* ws, uint4 w4, int k) {
    constexpr int U = kU32;
    const uint32_t wd[U] = {w4.x, w4.y, w4.z, w4.w};
    float4 Uj[U], Lj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t j = cs[u * 32];
      Uj[u] = u32[j];
      if (LO) Lj[u] = lo32[j];
    }
    float ev[U];  // e' of the intact bonds (0 for the others)
    float smax = -INFINITY;
    const float4 dA = lat_dir<DIM>(k), dB = lat_dir<DIM>(k + 2);  // k is a multiple of 4
    const float lA = lat_len<DIM>(k), lB = lat_len<DIM>(k + 2);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float4 dn = lat_twin(u < 2 ? dA : dB, u & 1);
      const float nl = u < 2 ? lA : lB;
      const float2 exy = LO ? make_float2(lat_delta_lo(Uj[u].x, Lj[u].x, Ui.x, Li.x), lat_delta_lo(Uj[u].y, Lj[u].y, Ui.y, Li.y))
                            : __fadd2_rn(make_float2(Uj[u].x, Uj[u].y), make_float2(nUi.x, nUi.y));
      const float ez = DIM == 3 ? (LO ? lat_delta_lo(Uj[u].z, Lj[u].z, Ui.z, Li.z) : Uj[u].z + nUi.z) : 0.0f;
      const bool in = (wd[u] & lmask) != 0u;
      const float p = lat_p_nl<DIM>(dn.x, dn.y, dn.z, exy.x, exy.y, ez);
      const float q2 = dn.w + p;  // |Y'|^2 = |n|^2 + p
      const float pm = in ? p : 0.0f;
      ev[u] = in ? p * rcp_ftz(fmaf(q2, rsqrt_ftz(q2), nl)) : 0.0f;
      if (screening) {
        const float D = in ? fabsf(exy.x) + fabsf(exy.y) + fabsf(ez) : 0.0f;
        smax = lat_max_nan(smax, lat_g_nl(pm, c32, dn.w) + lat_screen_nl(D, f0, f1, F2));
      }
    }
    const bool near = screening && !(smax < 0.0f);
    unsigned brk = 0u;
    if (__any_sync(kFull, near) | every) {
      // full band for every intact bond of the batch, FP64 inside it (neighbour index and record
      // reloaded from the staged chunk and L1)
#pragma unroll 1
      for (int u = 0; u < U; ++u) {
        int code = 0;
        if (checking && can_break && (ws[u] & lmask) != 0u) {
          const int32_t jj = cs[u * 32];
          const float4 uj = u32[jj];
          const float4 lj = LO ? lo32[jj] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          const float4 dn = lat_dir<DIM>(k + u);
          const float ex = LO ? lat_delta_lo(uj.x, lj.x, Ui.x, Li.x) : uj.x - Ui.x;
          const float ey = LO ? lat_delta_lo(uj.y, lj.y, Ui.y, Li.y) : uj.y - Ui.y;
          const float ez = DIM == 3 ? (LO ? lat_delta_lo(uj.z, lj.z, Ui.z, Li.z) : uj.z - Ui.z) : 0.0f;
          const float g = lat_g_nl(lat_p_nl<DIM>(dn.x, dn.y, dn.z, ex, ey, ez), c32, dn.w);
          LatBandNL band;
          band.A0 = bp.nl_A0;
          band.A0s = bp.nl_A0s;
          band.A1 = bp.nl_A1;
          band.A1s = bp.nl_A1s;
          band.A2 = bp.nl_A2;
          band.Ag = bp.nl_Ag;
          code = lat_code_nl(g, fabsf(ex) + fabsf(ey) + fabsf(ez), Ui.w + uj.w, band);
          if (code == 2) {
            code = fp64_breaks_nl<DIM>(a, t.i, jj, disp) ? 1 : 0;
            atomicAdd(&a.counters[0], 1ull);
          }
          if (a.validate && (code == 1) != fp64_breaks_nl<DIM>(a, t.i, jj, disp)) atomicAdd(&a.counters[1], 1ull);
        }
        const unsigned m = __ballot_sync(kFull, code == 1);
        if (m) {
          if (lane == 0) bw[k + u] = ws[u] & ~m;
          if (code == 1) brk |= 1u << u;
        }
      }
    }
    // dilatation terms |n| e' of the bonds intact after the decisions, in slot order
#pragma unroll
    for (int u = 0; u < U; ++u) acc = fmaf(u < 2 ? lA : lB, ((brk >> u) & 1u) ? 0.0f : ev[u], acc);
  };
  const bool ok = a.lat_wuni > 0 ? lat_rows<NB, CH>(a, st, a.lat_wuni, lane, batch)
                                 : lat_rows<NB, CH>(a, st, st.W, lane, batch);
  if (ok && write_theta) {
    const float2 f = a.lat_f[t.i];  // (N_ref / N_i, A / N_i)
    a.theta32[t.i] = f.y * acc;
    const float x = acc * (f.x * f.x);
    a.lat_up[t.i] = make_float4(Ui.x, Ui.y, Ui.z, fmaf(bp.lat_lam_hi, x, bp.lat_lam_lo * x));
  }
}

template <int DIM, bool LO, int NB, int CH>
__global__ void __maxnreg__(64) k_pass2_latnl(StepArgs a, const float4* __restrict__ u32, float4* __restrict__ u32_out,
                                               const float4* __restrict__ lo32, float4* __restrict__ lo32_out,
                                               const double4* __restrict__ disp, double4* __restrict__ disp_out) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (!t.active) return;
  auto st = stage_init<NB, CH>(smem, t, a);
  const int lane = t.lane;
  const int b = a.body ? a.body[t.i] : 0;
  const float4 Ui = a.lat_up[t.i];  // (u'_i, P_i)
  const float4 Li = LO ? lo32[t.i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const float4 nUi = make_float4(-Ui.x, -Ui.y, -Ui.z, 0.0f);
  const float rho_i = a.lat_f[t.i].x;
  const bool interior = __all_sync(kFull, a.lat_int[t.i >> 5] != 0);
  const uint32_t lmask = 1u << lane;
  float f[3] = {0.0f, 0.0f, 0.0f};
  auto batch_t = [&](auto intr, const int32_t* cs, uint4 w4, int k) {
    constexpr bool INTR = decltype(intr)::value;
    constexpr int U = kU32;
    const uint32_t wd[U] = {w4.x, w4.y, w4.z, w4.w};
    float4 Uj[U], Lj[U];
    float rr[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t j = cs[u * 32];
      Uj[u] = a.lat_up[j];
      if (LO) Lj[u] = lo32[j];
      rr[u] = INTR ? 2.0f : rho_i + a.lat_rho[j];
    }
    const float4 dA = lat_dir<DIM>(k), dB = lat_dir<DIM>(k + 2);  // k is a multiple of 4
    const float lA = lat_len<DIM>(k), lB = lat_len<DIM>(k + 2);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float4 dn = lat_twin(u < 2 ? dA : dB, u & 1);
      const float nl = u < 2 ? lA : lB;
      const float2 exy = LO ? make_float2(lat_delta_lo(Uj[u].x, Lj[u].x, Ui.x, Li.x), lat_delta_lo(Uj[u].y, Lj[u].y, Ui.y, Li.y))
                            : __fadd2_rn(make_float2(Uj[u].x, Uj[u].y), make_float2(nUi.x, nUi.y));
      const float ez = DIM == 3 ? (LO ? lat_delta_lo(Uj[u].z, Lj[u].z, Ui.z, Li.z) : Uj[u].z + nUi.z) : 0.0f;
      const float p = lat_p_nl<DIM>(dn.x, dn.y, dn.z, exy.x, exy.y, ez);
      const float yx = dn.x + exy.x, yy = dn.y + exy.y, yz = dn.z + ez;
      const float q2 = dn.w + p;  // |Y'|^2 = |n|^2 + p
      const float ry = rsqrt_ftz(q2);
      const float e = p * rcp_ftz(fmaf(q2, ry, nl));
      // coefficient along M = Y' / |Y'|: (P_i + P_j) |n| + (rho_i + rho_j) e'
      float cf = fmaf(rr[u], e, (Ui.w + Uj[u].w) * nl) * ry;
      cf = (wd[u] & lmask) ? cf : 0.0f;
      f[0] = fmaf(cf, yx, f[0]);
      f[1] = fmaf(cf, yy, f[1]);
      if (DIM == 3) f[2] = fmaf(cf, yz, f[2]);
    }
  };
  auto batch = [&](const int32_t* cs, const uint32_t*, uint4 w4, int k) {
    if (interior) batch_t(std::true_type{}, cs, w4, k);
    else batch_t(std::false_type{}, cs, w4, k);
  };
  const bool ok = a.lat_wuni > 0 ? lat_rows<NB, CH>(a, st, a.lat_wuni, lane, batch)
                                 : lat_rows<NB, CH>(a, st, st.W, lane, batch);
  if (ok) {  // warp-uniform
    double4 u;
    update_lat<DIM>(a, t.i, b, f, disp, disp_out, u);
    float4 hi;
    if (LO) {
      float4 lo;
      shadow_lat_lo<DIM>(a.bp[b].lat_inv_h, u, hi, lo);
      lo32_out[t.i] = lo;
    } else {
      hi = shadow_lat<DIM>(a.bp[b].lat_inv_h, u);
    }
    u32_out[t.i] = hi;
    lat_raise_umax(a.lat_umax_next, b, hi.w);
  }
}

// ---------------------------------------------------------------- adaptive dynamic relaxation
// The quasi-static solver of Section 4.4 (cited there from the literature): fictitious dynamics
// L u'' + c L u' = g(u), g = f + b, unit fictitious step.  Pass 1 and pass 2 run as in the explicit
// step (pass 2 stores g instead of moving the particles); three small kernels then form the damping
// c from a Rayleigh quotient of the local stiffness (a deterministic two-level reduction) and move
// the particles.

// alpha_i = (A / m_i) sum_j |xi_ij| V_j |M_ij|_1 over the built family (unused slots have xi = 0).
template <int DIM>
__global__ void k_adr_alpha(StepArgs a, double* __restrict__ alpha) {
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (!t.active) return;
  const double4 pi = a.pos[t.i];
  const double4 zero = make_double4(0.0, 0.0, 0.0, 0.0);
  double s = 0.0;
  for (int k = 0; k < t.W; ++k) {
    const double4 pj = a.pos[a.col[t.base + t.lane + ((int64_t)k << 5)]];
    double ex, ey, ez, d, q;
    bond_f64<DIM>(pi, pj, zero, zero, ex, ey, ez, d, q);
    if (q > 0.0) {
      const double xl = sqrt(q);
      s += xl * pj.w * ((fabs(ex) + fabs(ey) + fabs(ez)) / xl);
    }
  }
  alpha[t.i] = a.aA[t.i] * s;
}

// lambda_i = R_i / 4 with R_i = 2 G sum_j (1/m_i + 1/m_j) V_j |M_ij|_1
//                              + 2 |K - G/3| sum_j |xi_ij| V_j (alpha_i / m_i + alpha_j / m_j),
// an upper bound of the absolute row sums of the force-density stiffness (Gerschgorin); stored with
// its reciprocal, which the update multiplies by (an FP64 division costs many times an FMA on the
// FP64 pipe, and lambda is fixed for the run).
template <int DIM>
__global__ void k_adr_lambda(StepArgs a, const double* __restrict__ alpha, double2* __restrict__ lam) {
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (!t.active) return;
  const int b = a.body ? a.body[t.i] : 0;
  const double4 pi = a.pos[t.i];
  const double4 zero = make_double4(0.0, 0.0, 0.0, 0.0);
  const double mui = a.mu[t.i], ai = alpha[t.i];
  double rg = 0.0, rt = 0.0;
  for (int k = 0; k < t.W; ++k) {
    const int32_t j = a.col[t.base + t.lane + ((int64_t)k << 5)];
    const double4 pj = a.pos[j];
    double ex, ey, ez, d, q;
    bond_f64<DIM>(pi, pj, zero, zero, ex, ey, ez, d, q);
    if (q > 0.0) {
      const double xl = sqrt(q);
      const double m1 = (fabs(ex) + fabs(ey) + fabs(ez)) / xl;
      rg += (mui + a.mu[j]) * pj.w * m1;
      rt += xl * pj.w * (ai * mui + alpha[j] * a.mu[j]);
    }
  }
  const double R = 2.0 * a.bp[b].G * rg + 2.0 * fabs(a.bp[b].Kp) * rt;
  const double l = 0.25 * R;
  lam[t.i] = make_double2(l, l > 0.0 ? 1.0 / l : 0.0);
}

constexpr int kAdrBlock = 256;

// Per block: sum over its free particles' components of u (k u) and u u, k = -(g - g_prev) / (lambda v).
__global__ void __launch_bounds__(kAdrBlock) k_adr_sums(StepArgs a, const double4* __restrict__ disp,
                                                         const double4* __restrict__ gold,
                                                         const double2* __restrict__ lam,
                                                         double2* __restrict__ part) {
  __shared__ double sn[kAdrBlock], sd[kAdrBlock];
  const int64_t i = blockIdx.x * (int64_t)kAdrBlock + threadIdx.x;
  double num = 0.0, den = 0.0;
  if (i < a.n_pad && (!a.flag || a.flag[i] == 0) && lam[i].x > 0.0) {
    const double4 u = disp[i], v = a.vel[i], g = a.gnew[i], go = gold[i];
    const double li = lam[i].x;
    const double uu[3] = {u.x, u.y, u.z}, vv[3] = {v.x, v.y, v.z}, gg[3] = {g.x, g.y, g.z},
                 gp[3] = {go.x, go.y, go.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double kk = vv[k] != 0.0 ? -(gg[k] - gp[k]) / (li * vv[k]) : 0.0;
      num += uu[k] * kk * uu[k];
      den += uu[k] * uu[k];
    }
  }
  sn[threadIdx.x] = num;
  sd[threadIdx.x] = den;
  __syncthreads();
  for (int w = kAdrBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sn[threadIdx.x] += sn[threadIdx.x + w];
      sd[threadIdx.x] += sd[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sn[0], sd[0]);
}

// One block: c = 2 sqrt(num / den) (0 unless both are positive), the start flag of this iteration and
// 1 / (2 + c).
__global__ void __launch_bounds__(1024) k_adr_coef(const double2* __restrict__ part, int nblk, int* first,
                                                   double4* st) {
  __shared__ double sn[1024], sd[1024];
  double num = 0.0, den = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 1024) {
    num += part[b].x;
    den += part[b].y;
  }
  sn[threadIdx.x] = num;
  sd[threadIdx.x] = den;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sn[threadIdx.x] += sn[threadIdx.x + w];
      sd[threadIdx.x] += sd[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double c = (sd[0] > 0.0 && sn[0] > 0.0) ? 2.0 * sqrt(sn[0] / sd[0]) : 0.0;
    *st = make_double4(c, (double)*first, 1.0 / (2.0 + c), 0.0);
    *first = 0;
  }
}

// v^{n+1/2} = ((2 - c) v^{n-1/2} + 2 g / lambda) / (2 + c) (from rest on a start: g / (2 lambda)),
// u^{n+1} = u^n + v^{n+1/2}; constrained particles take their boundary value at t_{n+1}.  The two
// divisions are multiplications by the stored reciprocals 1 / lambda and 1 / (2 + c).
__global__ void __launch_bounds__(kAdrBlock) k_adr_update(StepArgs a, const double4* __restrict__ disp,
                                                           double4* __restrict__ disp_out,
                                                           double4* __restrict__ gold,
                                                           const double2* __restrict__ lam,
                                                           const double4* __restrict__ st,
                                                           float4* __restrict__ u32_out, unsigned* umax) {
  const int64_t i = blockIdx.x * (int64_t)kAdrBlock + threadIdx.x;
  if (i >= a.n_pad) return;
  const int b = a.body ? a.body[i] : 0;
  const BodyDev& bp = a.bp[b];
  const uint8_t fl = a.flag ? a.flag[i] : (uint8_t)0;
  double4 u = disp[i], v = a.vel[i];
  const double4 g = a.gnew[i];
  if (fl == 0) {
    const double2 li = lam[i];  // (lambda, 1 / lambda)
    if (li.x > 0.0) {
      const double4 s = *st;
      if (s.y != 0.0) {
        const double h = 0.5 * li.y;
        v = make_double4(g.x * h, g.y * h, g.z * h, 0.0);
      } else {
        const double cm = 2.0 - s.x, r2 = 2.0 * li.y;
        v.x = (cm * v.x + g.x * r2) * s.z;
        v.y = (cm * v.y + g.y * r2) * s.z;
        v.z = (cm * v.z + g.z * r2) * s.z;
      }
      u.x = u.x + v.x;
      u.y = u.y + v.y;
      u.z = u.z + v.z;
    } else {
      v = make_double4(0.0, 0.0, 0.0, 0.0);
    }
  } else if (fl == 1) {
    u = make_double4(0.0, 0.0, 0.0, u.w);
    v = make_double4(0.0, 0.0, 0.0, 0.0);
  } else {
    const double t1 = (double)(*a.d_step + 1) * bp.dt;
    const double4 gv = a.gvec[i];
    const double rt = bp.rate * t1;
    u = make_double4(rt * gv.x, rt * gv.y, rt * gv.z, u.w);
    v = make_double4(bp.rate * gv.x, bp.rate * gv.y, bp.rate * gv.z, 0.0);
  }
  disp_out[i] = u;
  a.vel[i] = v;
  gold[i] = g;
  if (u32_out) {  // mixed form: the FP32 shadow of the new state (and, lattice layout, its bound)
    const float4 sh = shadow_of(a, b, u);
    u32_out[i] = sh;
    if (umax) lat_raise_umax(umax, b, sh.w);  // whole warps: n_pad is a multiple of 32
  }
}


// ------------------------------------------------------------------------- state diagnostics
// pd_get_stats: theta, the strain energy sum_i V_i [(K - G/3)/(2A) theta_i^2 + G/(2 m_i) sum_j e^2 V_j]
// and the smallest relative stretch margin |s - s0| / s0 over the intact breakable bonds (pass A),
// then the force at the same state and 1/2 rho V v^n . v^{n+1} (pass B), all in FP64 from the master
// state and the current bond status; per-block sums in a fixed order.
constexpr int kDiagBlock = 256;

template <int DIM, int KIN>
__device__ __forceinline__ void diag_bond(const double4& pi, const double4& pj, const double4& ui, const double4& uj,
                                          double& xl, double& e, double& s, double dir[3]) {
  if (KIN == 0) {
    double ex, ey, ez, d, q;
    bond_f64<DIM>(pi, pj, ui, uj, ex, ey, ez, d, q);
    xl = sqrt(q);
    e = d / xl;
    s = d / q;
    dir[0] = ex / xl;
    dir[1] = ey / xl;
    dir[2] = ez / xl;
  } else {
    const BondNL<DIM> r = bond_nl<DIM>(pi, pj, ui, uj);
    double y2 = r.yx * r.yx + r.yy * r.yy;
    if (DIM == 3) y2 = fma(r.yz, r.yz, y2);
    const double yl = sqrt(y2);
    xl = sqrt(r.q);
    e = r.p / (yl + xl);
    s = e / xl;
    dir[0] = r.yx / yl;
    dir[1] = r.yy / yl;
    dir[2] = r.yz / yl;
  }
}

template <int DIM, int KIN>
__global__ void __launch_bounds__(kDiagBlock) k_diag_a(StepArgs a, const double4* __restrict__ disp,
                                                        double* __restrict__ theta, double4* __restrict__ part) {
  __shared__ double se[kDiagBlock], sm[kDiagBlock];
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  double energy = 0.0, margin = 1e300;
  if (t.active) {
    const int b = a.body ? a.body[t.i] : 0;
    const BodyDev& bp = a.bp[b];
    const double4 pi = a.pos[t.i], ui = disp[t.i];
    double th = 0.0, ee = 0.0;
    for (int k = 0; k < t.W; ++k) {
      if (!((a.bits[(t.base >> 5) + k] >> t.lane) & 1u)) continue;
      const int32_t j = a.col[t.base + t.lane + ((int64_t)k << 5)];
      const double4 pj = a.pos[j];
      double xl, e, sv, dir[3];
      diag_bond<DIM, KIN>(pi, pj, ui, disp[j], xl, e, sv, dir);
      const double w = bp.wdelta > 0.0 ? bp.wdelta / xl : 1.0;
      th += w * xl * e * pj.w;
      ee += w * e * e * pj.w;
      if (bp.breaks) margin = fmin(margin, fabs(sv - bp.s0) / bp.s0);
    }
    const double theta_i = a.aA[t.i] * th;
    theta[t.i] = theta_i;
    energy = pi.w * (bp.Kp / (2.0 * bp.A) * theta_i * theta_i + 0.5 * bp.G * a.mu[t.i] * ee);
  }
  se[threadIdx.x] = energy;
  sm[threadIdx.x] = margin;
  __syncthreads();
  for (int w = kDiagBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      se[threadIdx.x] += se[threadIdx.x + w];
      sm[threadIdx.x] = fmin(sm[threadIdx.x], sm[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = make_double4(se[0], sm[0], 0.0, 0.0);
}

template <int DIM, int KIN>
__global__ void __launch_bounds__(kDiagBlock) k_diag_b(StepArgs a, const double4* __restrict__ disp,
                                                        const double* __restrict__ theta, double4* __restrict__ part) {
  __shared__ double sk[kDiagBlock];
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  double kin = 0.0;
  if (t.active) {
    const int b = a.body ? a.body[t.i] : 0;
    const BodyDev& bp = a.bp[b];
    const double4 pi = a.pos[t.i], ui = disp[t.i];
    const double txi = bp.Kp * theta[t.i] * a.mu[t.i], tyi = bp.G * a.mu[t.i];
    double f[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < t.W; ++k) {
      if (!((a.bits[(t.base >> 5) + k] >> t.lane) & 1u)) continue;
      const int32_t j = a.col[t.base + t.lane + ((int64_t)k << 5)];
      const double4 pj = a.pos[j];
      double xl, e, sv, dir[3];
      diag_bond<DIM, KIN>(pi, pj, ui, disp[j], xl, e, sv, dir);
      // Eq 1.14 for both ends (Eq 2.2 in the linearized model), force density on i
      const double w = bp.wdelta > 0.0 ? bp.wdelta / xl : 1.0;
      const double cf = ((txi + bp.Kp * theta[j] * a.mu[j]) * xl + (tyi + bp.G * a.mu[j]) * e) * w * pj.w;
      f[0] = fma(cf, dir[0], f[0]);
      f[1] = fma(cf, dir[1], f[1]);
      f[2] = fma(cf, dir[2], f[2]);
    }
    const double4 v = a.vel[t.i];
    const uint8_t fl = a.flag ? a.flag[t.i] : (uint8_t)0;
    double vn[3] = {v.x, v.y, v.z};
    if (fl == 0) {
      const double4 bb = a.bacc ? a.bacc[t.i] : make_double4(0.0, 0.0, 0.0, 0.0);
      vn[0] += bp.dt * ((f[0] + bb.x) * bp.inv_rho);
      vn[1] += bp.dt * ((f[1] + bb.y) * bp.inv_rho);
      vn[2] += bp.dt * ((f[2] + bb.z) * bp.inv_rho);
    }
    kin = 0.5 * (pi.w / bp.inv_rho) * (v.x * vn[0] + v.y * vn[1] + v.z * vn[2]);
  }
  sk[threadIdx.x] = kin;
  __syncthreads();
  for (int w = kDiagBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sk[threadIdx.x] += sk[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x].z = sk[0];
}

// ----------------------------------------------------------------------------- auxiliary kernels
__global__ void k_set_step(int64_t* d_step, int64_t v) { *d_step = v; }

// phi_i of Eq 1.31 (with the body's influence function w), written in caller order.
__global__ void k_damage(StepArgs a, int64_t n, const double* __restrict__ dden,
                         const int64_t* __restrict__ perm, double* __restrict__ out) {
  const SliceIdx t = slice_index<1>(a.n_pad, a.slice_ptr);
  if (!t.active) return;
  double num = 0.0;
  const double wd = a.bp[a.body ? a.body[t.i] : 0].wdelta;
  const double4 pi = a.pos[t.i];
  for (int k = 0; k < t.W; ++k) {
    const uint32_t word = a.bits[(t.base >> 5) + k];
    if (!((word >> t.lane) & 1u)) continue;
    const double4 pj = a.pos[a.col[t.base + t.lane + ((int64_t)k << 5)]];
    double w = 1.0;
    if (wd > 0.0) {  // |xi|^2 rounded term by term, as the build's denominator D_i (no contraction)
      const double ex = pj.x - pi.x, ey = pj.y - pi.y, ez = pj.z - pi.z;
      w = wd / sqrt(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
    }
    num = __dadd_rn(num, __dmul_rn(w, pj.w));
  }
  if (t.i < n) out[perm[t.i]] = dden[t.i] > 0.0 ? 1.0 - num / dden[t.i] : 0.0;
}

// Caller-order SoA -> internal double4; .w taken from wsrc[k].w (the particle volume) when given.
__global__ void k_gather_soa(int64_t n, int64_t n_pad, int comps, const double* __restrict__ src,
                             const int64_t* __restrict__ perm, const double4* __restrict__ wsrc,
                             double4* __restrict__ dst) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n_pad) return;
  const double w = wsrc ? wsrc[k].w : 0.0;
  if (k >= n) {
    dst[k] = make_double4(0.0, 0.0, 0.0, w);
    return;
  }
  const int64_t u = perm[k];
  dst[k] = make_double4(src[u], src[n + u], comps == 3 ? src[2 * n + u] : 0.0, w);
}

// Any non-finite value among n doubles (grid-stride) -> *flag = 1.
__global__ void k_nonfinite(int64_t n, const double* __restrict__ a, unsigned long long* flag) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bad = bad || !isfinite(a[i]);
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1ull);
}

// disp[.].w = V (set once after allocation; every writer of disp keeps it).
__global__ void k_set_w(int64_t n_pad, const double4* __restrict__ pos, double4* __restrict__ d0,
                        double4* __restrict__ d1) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n_pad) return;
  d0[k].w = pos[k].w;
  d1[k].w = pos[k].w;
}

__global__ void k_scatter_soa(int64_t n, int comps, const double4* __restrict__ src,
                              const int64_t* __restrict__ perm, double* __restrict__ dst) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t u = perm[k];
  const double4 v = src[k];
  dst[u] = v.x;
  dst[n + u] = v.y;
  if (comps == 3) dst[2 * n + u] = v.z;
}

__global__ void k_scatter_scalar(int64_t n, const double* __restrict__ src, const float* __restrict__ src32,
                                 const int64_t* __restrict__ perm, double* __restrict__ dst) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  dst[perm[k]] = src ? src[k] : (double)src32[k];
}

// Boundary values at the current time for the constrained particles (fixed / prescribed).
__global__ void k_apply_bc(StepArgs a, double4* __restrict__ disp, int64_t step) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n_pad || !a.flag) return;
  const uint8_t fl = a.flag[i];
  if (fl == 0) return;
  const double w = disp[i].w;
  if (fl == 1) {
    disp[i] = make_double4(0.0, 0.0, 0.0, w);
    a.vel[i] = make_double4(0.0, 0.0, 0.0, 0.0);
    return;
  }
  const BodyDev& bp = a.bp[a.body ? a.body[i] : 0];
  const double tn = (double)step * bp.dt;
  const double4 g = a.gvec[i];
  const double rt = bp.rate * tn;
  disp[i] = make_double4(rt * g.x, rt * g.y, rt * g.z, w);
  a.vel[i] = make_double4(bp.rate * g.x, bp.rate * g.y, bp.rate * g.z, 0.0);
}

__global__ void k_shadow(StepArgs a, const double4* __restrict__ disp, float4* __restrict__ u32,
                         float4* __restrict__ lo32, unsigned* __restrict__ umax) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n_pad) return;  // whole warps: n_pad is a multiple of 32
  const int b = a.body ? a.body[i] : 0;
  const float4 sh = shadow_of(a, b, disp[i]);
  u32[i] = sh;
  if (umax) lat_raise_umax(umax, b, sh.w);  // lattice layout: the bound of this shadow (zeroed before)
  if (lo32) {  // two-word shadow of the lattice layout (3D formula: z is zero in 2D)
    float4 hi, lo;
    shadow_lat_lo<3>(a.bp[b].lat_inv_h, disp[i], hi, lo);
    lo32[i] = lo;
  }
}

// max |u_k| over all particles and components (order-independent: max of non-negative doubles as
// integers), plus a count of non-finite components.
// Sets *flag when any displacement component is not finite (checked after each pd_step).
__global__ void k_flag_nonfinite(int64_t n, const double4* __restrict__ disp, unsigned long long* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double4 u = disp[i];
  if (!isfinite(u.x) || !isfinite(u.y) || !isfinite(u.z)) atomicExch(flag, 1ull);
}

__global__ void k_max_abs(int64_t n, const double4* __restrict__ disp, unsigned long long* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double m = 0.0;
  unsigned bad = 0;
  if (i < n) {
    const double4 u = disp[i];
    const double c[3] = {u.x, u.y, u.z};
    for (int k = 0; k < 3; ++k) {
      if (!isfinite(c[k])) bad = 1;
      else m = fmax(m, fabs(c[k]));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_down_sync(kFull, m, o));
    bad |= __shfl_down_sync(kFull, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], (unsigned long long)__double_as_longlong(m));
    if (bad) atomicAdd(&out[1], 1ull);
  }
}

// ------------------------------------------------------------------------------ host dispatch
StepArgs make_args(pd_ctx* c) {
  StepArgs a{};
  a.n_pad = c->n_pad;
  a.slice_ptr = c->slice_ptr;
  a.col = c->col;
  a.bits = c->bits;
  a.pos = c->pos;
  a.body = c->nbodies > 1 ? c->body : nullptr;
  a.bp = c->bp;
  a.aA = c->aA;
  a.mu = c->mu;
  a.theta = c->theta;
  a.thm = c->thm;
  a.vel = c->vel;
  a.flag = c->has_flag ? c->flag : nullptr;
  a.bacc = c->has_b ? c->bacc : nullptr;
  a.gvec = c->gvec;
  a.d_step = c->d_step;
  a.pos32 = c->pos32;
  a.thm32 = c->thm32;
  a.mu32 = c->mu32;
  a.aA32 = c->aA32;
  a.theta32 = c->theta32;
  a.counters = c->counters;
  double bc = 4.0;
  if (c->prm[0].band_safety > 0) bc = c->prm[0].band_safety;
  a.band_c = (float)bc;
  a.validate = c->validate;
  a.check = 1;
  a.bA = c->bond_cache ? c->bA : nullptr;
  a.bB = c->bond_cache ? c->bB : nullptr;
  a.bd = c->bond_cache ? c->bd : nullptr;
  a.bS = c->bond_cache ? c->bS : nullptr;
  a.cnt = c->cnt;
  const bool pairs_ready = c->kin == PD_NONLINEAR ? c->bX != nullptr : c->dirty != nullptr;
  a.own0 = (c->bond_cache && c->pairs && c->pairs_ok && pairs_ready) ? c->own0 : nullptr;
  a.bt = c->bt;
  a.bY = c->bY;
  a.bX = c->bX;
  a.twin = c->twin;
  a.dirty = c->dirty;
  a.bE = c->bond_cache ? c->bE : nullptr;
  a.expire = c->expire_waits;
  a.uscale = c->kin == PD_NONLINEAR ? 1.0 / c->q : 1.0;
  a.adr = c->solver == PD_SOLVER_ADR ? 1 : 0;
  a.gnew = c->gnew;
  a.lattice = c->lattice ? 1 : 0;
  a.lat_f = c->lat_f;
  a.lat_rho = c->lat_rho;
  a.lat_up = c->lat_up;
  a.lat_int = c->lat_int;
  a.lat_wuni = c->lat_wuni;
  a.lat_umax = c->lat_umax ? c->lat_umax + (size_t)c->cur * c->nbodies : nullptr;
  a.lat_umax_next = c->lat_umax ? c->lat_umax + (size_t)(c->cur ^ 1) * c->nbodies : nullptr;
  a.nbody = c->nbodies;
  return a;
}

cudaEvent_t take_event(pd_ctx* c) {
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

template <int DIM, int SPLIT>
void launch_pass1(pd_ctx* c, const StepArgs& a, int write_theta, unsigned grid, int block, size_t sm) {
  if (c->kin == PD_NONLINEAR && a.bA && a.own0 && !write_theta) {
    if (a.check) k_check_nlp<DIM, SPLIT><<<grid, block, 0, c->stream>>>(a, c->disp[c->cur]);
  } else if (c->kin == PD_NONLINEAR && a.bA && a.own0) {
    if (c->vol_uniform)
      k_pass1a_nlp<DIM, SPLIT, true><<<grid, block, 0, c->stream>>>(a, c->disp[c->cur]);
    else
      k_pass1a_nlp<DIM, SPLIT, false><<<grid, block, 0, c->stream>>>(a, c->disp[c->cur]);
    if (write_theta) {
      if (c->profile) {
        c->times.mid = take_event(c);
        cudaEventRecord(c->times.mid, c->stream);
      }
      k_pass1b_nlp<DIM, SPLIT><<<grid, block, sm, c->stream>>>(a, write_theta);
    }
  } else if (c->kin == PD_NONLINEAR && a.bA)
    k_pass1_nlt<DIM, SPLIT><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], write_theta);
  else if (c->kin == PD_NONLINEAR)
    k_pass1_nl<DIM, SPLIT><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], write_theta);
  else if (c->precision == PD_FP64 && a.bA && a.own0 && !write_theta) {
    if (a.check && c->cA32) {
      const int tb = 256;
      k_check_u32<<<(unsigned)((c->n_pad + tb - 1) / tb), tb, 0, c->stream>>>(c->n_pad, c->disp[c->cur], c->cu32);
      k_check_f64p<DIM, SPLIT, true><<<grid, block, 0, c->stream>>>(a, c->disp[c->cur], c->cu32, c->cA32);
    } else if (a.check) {
      k_check_f64p<DIM, SPLIT, false><<<grid, block, 0, c->stream>>>(a, c->disp[c->cur], nullptr, nullptr);
    }
  } else if (c->precision == PD_FP64 && a.bA && a.own0) {
    k_pass1a_f64p<DIM, SPLIT><<<grid, block, 0, c->stream>>>(a, c->disp[c->cur]);
    if (c->profile) {
      c->times.mid = take_event(c);
      cudaEventRecord(c->times.mid, c->stream);
    }
    if (c->vol_uniform)
      k_pass1b_f64p<DIM, SPLIT, true><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], write_theta);
    else
      k_pass1b_f64p<DIM, SPLIT, false><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], write_theta);
  } else if (c->precision == PD_FP64 && a.bA) {
    if (write_theta)
      k_pass1_f64t<DIM, SPLIT, true><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], write_theta);
    else
      k_pass1_f64t<DIM, SPLIT, false><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], write_theta);
  }
  else if (c->precision == PD_FP64)
    k_pass1_f64<DIM, SPLIT><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], write_theta);
  else
    k_pass1_mixed<DIM, SPLIT><<<grid, block, sm, c->stream>>>(a, c->u32[c->cur], c->disp[c->cur], write_theta);
}

template <int DIM, int SPLIT>
void launch_pass2(pd_ctx* c, const StepArgs& a, unsigned grid, int block, size_t sm) {
  if (c->kin == PD_NONLINEAR && a.bA && a.own0)
    k_pass2_nlp<DIM, SPLIT><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], c->disp[c->cur ^ 1]);
  else if (c->kin == PD_NONLINEAR && a.bA)
    k_pass2_nlt<DIM, SPLIT><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], c->disp[c->cur ^ 1]);
  else if (c->kin == PD_NONLINEAR)
    k_pass2_nl<DIM, SPLIT><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], c->disp[c->cur ^ 1]);
  else if (c->precision == PD_FP64 && a.bA)
    k_pass2_f64t<DIM, SPLIT><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], c->disp[c->cur ^ 1]);
  else if (c->precision == PD_FP64)
    k_pass2_f64<DIM, SPLIT><<<grid, block, sm, c->stream>>>(a, c->disp[c->cur], c->disp[c->cur ^ 1]);
  else
    k_pass2_mixed<DIM, SPLIT>
        <<<grid, block, sm, c->stream>>>(a, c->u32[c->cur], c->u32[c->cur ^ 1], c->disp[c->cur], c->disp[c->cur ^ 1]);
}

// Lattice kernels: the ring of PD_OPT_LAT_STAGE (0: 3 x 16 slots, 1: 2 x 16, 2: 3 x 8, 3: 2 x 8).
template <int DIM, bool WI, bool LO, int NB, int CH>
void optin_lat_ring() {
  const int mx = 16 * StageGeom<NB, CH>::kWarpBytes;
  cudaFuncSetAttribute(k_pass1_lat<DIM, WI, LO, NB, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_pass2_lat<DIM, WI, LO, NB, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}
template <int DIM, bool LO, int NB, int CH>
void optin_latnl_ring() {
  const int mx = 16 * StageGeom<NB, CH>::kWarpBytes;
  cudaFuncSetAttribute(k_pass1_latnl<DIM, LO, NB, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_pass2_latnl<DIM, LO, NB, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}
template <int DIM, bool WI>
void optin_lat() {
  optin_lat_ring<DIM, WI, false, 3, 16>();
  optin_lat_ring<DIM, WI, false, 2, 16>();
  optin_lat_ring<DIM, WI, false, 3, 8>();
  optin_lat_ring<DIM, WI, false, 2, 8>();
  optin_lat_ring<DIM, WI, true, 2, 16>();
  optin_lat_ring<DIM, WI, true, 2, 8>();
}

template <int DIM, bool WI, bool LO, int NB, int CH>
void launch_lat_ring(pd_ctx* c, const StepArgs& a, int pass, int write_theta, int block) {
  const unsigned g1 = (unsigned)((c->nslices * 32 + block - 1) / block);
  const size_t smb = (size_t)(block / 32) * StageGeom<NB, CH>::kWarpBytes;
  const float4* lo = LO ? c->u32lo[c->cur] : nullptr;
  if (pass == 1)
    k_pass1_lat<DIM, WI, LO, NB, CH><<<g1, block, smb, c->stream>>>(a, c->u32[c->cur], lo, c->disp[c->cur],
                                                                    write_theta);
  else
    k_pass2_lat<DIM, WI, LO, NB, CH><<<g1, block, smb, c->stream>>>(
        a, c->u32[c->cur], c->u32[c->cur ^ 1], lo, LO ? c->u32lo[c->cur ^ 1] : nullptr, c->disp[c->cur],
        c->disp[c->cur ^ 1]);
}
// The two-word shadow's kernels exist for the two-chunk rings only (rings 0 and 2 map to 1 and 3).
template <int DIM, bool WI>
void launch_lat(pd_ctx* c, const StepArgs& a, int pass, int write_theta, int block) {
  if (c->shadow_lo) {
    if (c->lat_stage >= 2) launch_lat_ring<DIM, WI, true, 2, 8>(c, a, pass, write_theta, block);
    else launch_lat_ring<DIM, WI, true, 2, 16>(c, a, pass, write_theta, block);
    return;
  }
  switch (c->lat_stage) {
    case 1: launch_lat_ring<DIM, WI, false, 2, 16>(c, a, pass, write_theta, block); break;
    case 2: launch_lat_ring<DIM, WI, false, 3, 8>(c, a, pass, write_theta, block); break;
    case 3: launch_lat_ring<DIM, WI, false, 2, 8>(c, a, pass, write_theta, block); break;
    default: launch_lat_ring<DIM, WI, false, 3, 16>(c, a, pass, write_theta, block); break;
  }
}

// Nonlinear bonds on the lattice layout: rings 0 and 1 run 2 x 16 slots, rings 2 and 3 run 2 x 8.
template <int DIM, bool LO, int NB, int CH>
void launch_latnl_ring(pd_ctx* c, const StepArgs& a, int pass, int write_theta, int block) {
  const unsigned g1 = (unsigned)((c->nslices * 32 + block - 1) / block);
  const size_t smb = (size_t)(block / 32) * StageGeom<NB, CH>::kWarpBytes;
  const float4* lo = LO ? c->u32lo[c->cur] : nullptr;
  if (pass == 1)
    k_pass1_latnl<DIM, LO, NB, CH><<<g1, block, smb, c->stream>>>(a, c->u32[c->cur], lo, c->disp[c->cur], write_theta);
  else
    k_pass2_latnl<DIM, LO, NB, CH><<<g1, block, smb, c->stream>>>(a, c->u32[c->cur], c->u32[c->cur ^ 1], lo,
                                                                   LO ? c->u32lo[c->cur ^ 1] : nullptr,
                                                                   c->disp[c->cur], c->disp[c->cur ^ 1]);
}
template <int DIM>
void launch_latnl(pd_ctx* c, const StepArgs& a, int pass, int write_theta, int block) {
  const bool lo = c->shadow_lo;
  if (c->lat_stage >= 2) {
    if (lo) launch_latnl_ring<DIM, true, 2, 8>(c, a, pass, write_theta, block);
    else launch_latnl_ring<DIM, false, 2, 8>(c, a, pass, write_theta, block);
  } else {
    if (lo) launch_latnl_ring<DIM, true, 2, 16>(c, a, pass, write_theta, block);
    else launch_latnl_ring<DIM, false, 2, 16>(c, a, pass, write_theta, block);
  }
}

template <int DIM>
void optin_staged() {
  const int mx = 16 * kStageWarpBytes;
  optin_lat<DIM, false>();
  optin_lat<DIM, true>();
  optin_latnl_ring<DIM, false, 2, 16>();
  optin_latnl_ring<DIM, false, 2, 8>();
  optin_latnl_ring<DIM, true, 2, 16>();
  optin_latnl_ring<DIM, true, 2, 8>();
  cudaFuncSetAttribute(k_pass1_mixed_staged<DIM, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_pass2_mixed_staged<DIM, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_pass1_mixed_staged<DIM, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_pass2_mixed_staged<DIM, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

}  // namespace

// Shared-memory opt-in of the staged kernels (up to 512 threads per block) on the current device;
// called when a mixed context is built, outside any stream capture.
pd_status prepare_staged_kernels(pd_ctx* c) {
  if (c->dim == 3) optin_staged<3>();
  else optin_staged<2>();
  PD_CUDA(cudaGetLastError());
  if (c->lattice) return upload_lattice_tables(c->device);
  return PD_OK;
}

// The direction tables of the lattice kernels, once per device (every context uses the same
// tables, so later uploads would write the same values).
pd_status upload_lattice_tables(int device) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> lock(mu);
  if (std::find(done.begin(), done.end(), device) != done.end()) return PD_OK;
  for (int dim = 2; dim <= 3; ++dim) {
    const std::vector<LatDir> t = lattice_directions(dim);
    const size_t pad = dim == 3 ? kLatPad3 : kLatPad2;
    std::vector<float4> dn(pad, make_float4(0.0f, 0.0f, 0.0f, 1.0f));
    std::vector<float2> rc(pad, make_float2(0.0f, 0.0f));
    for (size_t k = 0; k < t.size(); ++k) {
      dn[k] = make_float4((float)t[k].n[0], (float)t[k].n[1], (float)t[k].n[2], (float)t[k].q);
      const double r = 1.0 / t[k].q;
      const float hi = (float)r;
      rc[k] = make_float2(hi, (float)(r - (double)hi));
    }
    std::vector<float> ln(pad, 1.0f);
    for (size_t k = 0; k < t.size(); ++k) ln[k] = (float)std::sqrt((double)t[k].q);
    std::vector<float2> wt(pad, make_float2(0.0f, 0.0f));
    for (size_t k = 0; k < t.size(); ++k) {
      const double r = 1.0 / std::sqrt((double)t[k].q);
      const float hi = (float)r;
      wt[k] = make_float2(hi, (float)(r - (double)hi));
    }
    if (dim == 3) {
      PD_CUDA(cudaMemcpyToSymbol(c_lat3, dn.data(), sizeof(float4) * dn.size()));
      PD_CUDA(cudaMemcpyToSymbol(c_latr3, rc.data(), sizeof(float2) * rc.size()));
      PD_CUDA(cudaMemcpyToSymbol(c_latw3, wt.data(), sizeof(float2) * wt.size()));
      PD_CUDA(cudaMemcpyToSymbol(c_latn3, ln.data(), sizeof(float) * ln.size()));
    } else {
      PD_CUDA(cudaMemcpyToSymbol(c_lat2, dn.data(), sizeof(float4) * dn.size()));
      PD_CUDA(cudaMemcpyToSymbol(c_latr2, rc.data(), sizeof(float2) * rc.size()));
      PD_CUDA(cudaMemcpyToSymbol(c_latw2, wt.data(), sizeof(float2) * wt.size()));
      PD_CUDA(cudaMemcpyToSymbol(c_latn2, ln.data(), sizeof(float) * ln.size()));
    }
  }
  done.push_back(device);
  return PD_OK;
}

namespace {

template <int DIM>
void dispatch_pass(pd_ctx* c, const StepArgs& a, int pass, int write_theta) {
  const int block = c->block;
  const int split = c->split;
  const int64_t threads = c->nslices * 32 * (int64_t)split;
  const unsigned grid = (unsigned)((threads + block - 1) / block);
  if (c->precision == PD_MIXED && c->lattice) {
    // lattice layout: one warp per slice, whatever the split and stage options
    if (c->kin == PD_NONLINEAR) launch_latnl<DIM>(c, a, pass, write_theta, block);
    else if (c->prm[0].influence == PD_W_INV) launch_lat<DIM, true>(c, a, pass, write_theta, block);
    else launch_lat<DIM, false>(c, a, pass, write_theta, block);
    return;
  }
  if (c->precision == PD_MIXED && ((split == 1 && c->stage) || c->kin == PD_NONLINEAR)) {
    // nonlinear bonds in the mixed form run the staged kernels only (one warp per slice)
    const unsigned g1 = (unsigned)((c->nslices * 32 + block - 1) / block);
    const size_t smb = (size_t)(block / 32) * kStageWarpBytes;
    if (c->kin == PD_NONLINEAR) {
      if (pass == 1)
        k_pass1_mixed_staged<DIM, 1><<<g1, block, smb, c->stream>>>(a, c->u32[c->cur], c->disp[c->cur], write_theta);
      else
        k_pass2_mixed_staged<DIM, 1><<<g1, block, smb, c->stream>>>(a, c->u32[c->cur], c->u32[c->cur ^ 1],
                                                                    c->disp[c->cur], c->disp[c->cur ^ 1]);
    } else {
      if (pass == 1)
        k_pass1_mixed_staged<DIM, 0><<<g1, block, smb, c->stream>>>(a, c->u32[c->cur], c->disp[c->cur], write_theta);
      else
        k_pass2_mixed_staged<DIM, 0><<<g1, block, smb, c->stream>>>(a, c->u32[c->cur], c->u32[c->cur ^ 1],
                                                                    c->disp[c->cur], c->disp[c->cur ^ 1]);
    }
    return;
  }
  const size_t sm = split > 1 ? (size_t)block * 3 * sizeof(double) : 0;
  if (pass == 1) {
    if (split == 1) launch_pass1<DIM, 1>(c, a, write_theta, grid, block, sm);
    else if (split == 2) launch_pass1<DIM, 2>(c, a, write_theta, grid, block, sm);
    else launch_pass1<DIM, 4>(c, a, write_theta, grid, block, sm);
  } else {
    if (split == 1) launch_pass2<DIM, 1>(c, a, grid, block, sm);
    else if (split == 2) launch_pass2<DIM, 2>(c, a, grid, block, sm);
    else launch_pass2<DIM, 4>(c, a, grid, block, sm);
  }
}

void dispatch(pd_ctx* c, const StepArgs& a, int pass, int write_theta) {
  if (c->dim == 3) dispatch_pass<3>(c, a, pass, write_theta);
  else dispatch_pass<2>(c, a, pass, write_theta);
}


}  // namespace

pd_status init_disp_w(pd_ctx* c) {
  const int tb = 256;
  k_set_w<<<(unsigned)((c->n_pad + tb - 1) / tb), tb, 0, c->stream>>>(c->n_pad, c->pos, c->disp[0], c->disp[1]);
  PD_CUDA(cudaGetLastError());
  return PD_OK;
}

// Allocates and fills the per-slot tables of the tabled FP64 path (once per build), and brings the
// per-particle intact sums up to date with the status bits.
pd_status ensure_bond_cache(pd_ctx* c) {
  if (!c->bond_cache || c->precision != PD_FP64) return PD_OK;
  pd_status st;
  const size_t ne = (size_t)std::max<int64_t>(c->nentries, 32);
  const int tb = 256;
  const unsigned grid = (unsigned)((c->n_pad + tb - 1) / tb);
  if (c->kin == PD_NONLINEAR) {
    if (c->bA) return PD_OK;
    if ((st = alloc(c, &c->bA, ne)) != PD_OK) return st;
    if ((st = alloc(c, &c->bE, ne)) != PD_OK) return st;
    PD_CUDA(cudaMemsetAsync(c->bE, 0, sizeof(double2) * ne, c->stream));
    if (c->pairs_ok) {
      if ((st = alloc(c, &c->bt, ne)) != PD_OK) return st;
      PD_CUDA(cudaMemsetAsync(c->bt, 0, sizeof(double) * ne, c->stream));
      if ((st = alloc(c, &c->bY, ne)) != PD_OK) return st;
      PD_CUDA(cudaMemsetAsync(c->bY, 0, sizeof(double4) * ne, c->stream));
      if ((st = alloc(c, &c->bX, ne)) != PD_OK) return st;
      StepArgs ax = make_args(c);
      if (c->dim == 3)
        k_bond_tables_nlp<3><<<grid, tb, 0, c->stream>>>(ax, c->bX);
      else
        k_bond_tables_nlp<2><<<grid, tb, 0, c->stream>>>(ax, c->bX);
      PD_CUDA(cudaGetLastError());
    }
    StepArgs a = make_args(c);
    if (c->dim == 3)
      k_bond_tables_nl<3><<<grid, tb, 0, c->stream>>>(a, c->bA);
    else
      k_bond_tables_nl<2><<<grid, tb, 0, c->stream>>>(a, c->bA);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
  }
  if (!c->bA) {
    if ((st = alloc(c, &c->bA, ne)) != PD_OK) return st;
    if ((st = alloc(c, &c->bB, ne)) != PD_OK) return st;
    if ((st = alloc(c, &c->bd, ne)) != PD_OK) return st;
    if ((st = alloc(c, &c->bS, (size_t)c->n_pad)) != PD_OK) return st;
    PD_CUDA(cudaMemsetAsync(c->bd, 0, sizeof(double) * ne, c->stream));  // padding slots stay 0
    if (c->pairs_ok) {
      if ((st = alloc(c, &c->dirty, (size_t)c->nslices)) != PD_OK) return st;
      PD_CUDA(cudaMemsetAsync(c->dirty, 0, (size_t)c->nslices, c->stream));
    }
    StepArgs a = make_args(c);
    if (c->dim == 3)
      k_bond_tables<3><<<grid, tb, 0, c->stream>>>(a, c->bA, c->bB);
    else
      k_bond_tables<2><<<grid, tb, 0, c->stream>>>(a, c->bA, c->bB);
    PD_CUDA(cudaGetLastError());
    c->bs_stale = true;
  }
  if (c->bs_stale) {
    k_bond_sums<<<grid, tb, 0, c->stream>>>(make_args(c));
    PD_CUDA(cudaGetLastError());
    c->bs_stale = false;
  }
  return PD_OK;
}

__global__ void k_set_flag(int* p, int v) { *p = v; }

pd_status ensure_adr(pd_ctx* c) {
  if (c->solver != PD_SOLVER_ADR) return PD_OK;
  pd_status st;
  if (!c->lam) {
    const int64_t np = c->n_pad;
    const size_t nblk = (size_t)((np + kAdrBlock - 1) / kAdrBlock);
    if ((st = alloc(c, &c->lam, np)) != PD_OK) return st;
    if ((st = alloc(c, &c->gnew, np)) != PD_OK) return st;
    if ((st = alloc(c, &c->gold, np)) != PD_OK) return st;
    if ((st = alloc(c, &c->adr_part, nblk)) != PD_OK) return st;
    if ((st = alloc(c, &c->adr_st, 1)) != PD_OK) return st;
    if ((st = alloc(c, &c->adr_first, 1)) != PD_OK) return st;
    PD_CUDA(cudaMemsetAsync(c->gnew, 0, sizeof(double4) * np, c->stream));
    PD_CUDA(cudaMemsetAsync(c->gold, 0, sizeof(double4) * np, c->stream));
    double* alpha = nullptr;
    if (cudaMalloc(&alpha, sizeof(double) * np) != cudaSuccess) {
      cudaGetLastError();
      return fail(PD_ERR_OOM, "cudaMalloc of the ADR temporary failed");
    }
    StepArgs a = make_args(c);
    const int tb = 256;
    const unsigned grid = (unsigned)((np + tb - 1) / tb);
    if (c->dim == 3) {
      k_adr_alpha<3><<<grid, tb, 0, c->stream>>>(a, alpha);
      k_adr_lambda<3><<<grid, tb, 0, c->stream>>>(a, alpha, c->lam);
    } else {
      k_adr_alpha<2><<<grid, tb, 0, c->stream>>>(a, alpha);
      k_adr_lambda<2><<<grid, tb, 0, c->stream>>>(a, alpha, c->lam);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(alpha);
    if (e != cudaSuccess) return cuda_fail(e, "ADR density");
  }
  if (c->adr_restart) {
    k_set_flag<<<1, 1, 0, c->stream>>>(c->adr_first, 1);
    PD_CUDA(cudaGetLastError());
    c->adr_restart = false;
  }
  return PD_OK;
}

pd_status diagnostics(pd_ctx* c, double* min_margin, double* strain, double* kinetic) {
  const int64_t np = c->n_pad;
  const unsigned nblk = (unsigned)((np + kDiagBlock - 1) / kDiagBlock);
  pd_status st;
  if (!c->diag_theta && (st = alloc(c, &c->diag_theta, np)) != PD_OK) return st;
  if (!c->diag_part && (st = alloc(c, &c->diag_part, nblk)) != PD_OK) return st;
  StepArgs a = make_args(c);
  const double4* u = c->disp[c->cur];
  if (c->dim == 3 && c->kin == PD_NONLINEAR) {
    k_diag_a<3, 1><<<nblk, kDiagBlock, 0, c->stream>>>(a, u, c->diag_theta, c->diag_part);
    k_diag_b<3, 1><<<nblk, kDiagBlock, 0, c->stream>>>(a, u, c->diag_theta, c->diag_part);
  } else if (c->dim == 3) {
    k_diag_a<3, 0><<<nblk, kDiagBlock, 0, c->stream>>>(a, u, c->diag_theta, c->diag_part);
    k_diag_b<3, 0><<<nblk, kDiagBlock, 0, c->stream>>>(a, u, c->diag_theta, c->diag_part);
  } else if (c->kin == PD_NONLINEAR) {
    k_diag_a<2, 1><<<nblk, kDiagBlock, 0, c->stream>>>(a, u, c->diag_theta, c->diag_part);
    k_diag_b<2, 1><<<nblk, kDiagBlock, 0, c->stream>>>(a, u, c->diag_theta, c->diag_part);
  } else {
    k_diag_a<2, 0><<<nblk, kDiagBlock, 0, c->stream>>>(a, u, c->diag_theta, c->diag_part);
    k_diag_b<2, 0><<<nblk, kDiagBlock, 0, c->stream>>>(a, u, c->diag_theta, c->diag_part);
  }
  PD_CUDA(cudaGetLastError());
  std::vector<double4> h(nblk);
  PD_CUDA(cudaMemcpyAsync(h.data(), c->diag_part, sizeof(double4) * nblk, cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaStreamSynchronize(c->stream));
  double e = 0.0, k = 0.0, m = 1e300;
  for (const double4& p : h) {
    e += p.x;
    m = std::min(m, p.y);
    k += p.z;
  }
  *min_margin = m;
  *strain = e;
  *kinetic = k;
  return PD_OK;
}

pd_status launch_set_step(pd_ctx* c, int64_t value) {
  k_set_step<<<1, 1, 0, c->stream>>>(c->d_step, value);
  PD_CUDA(cudaGetLastError());
  return PD_OK;
}

// One full time step (pass 1 + pass 2); flips the double buffers.
pd_status launch_step(pd_ctx* c, bool check) {
  StepArgs a = make_args(c);
  a.check = check ? 1 : 0;
  const bool prof = c->profile != 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  if (prof) {
    e0 = take_event(c);
    e1 = take_event(c);
    e2 = take_event(c);
    cudaEventRecord(e0, c->stream);
  }
  dispatch(c, a, 1, 1);
  if (prof) cudaEventRecord(e1, c->stream);
  dispatch(c, a, 2, 1);
  if (a.adr) {
    const unsigned nblk = (unsigned)((c->n_pad + kAdrBlock - 1) / kAdrBlock);
    k_adr_sums<<<nblk, kAdrBlock, 0, c->stream>>>(a, c->disp[c->cur], c->gold, c->lam, c->adr_part);
    k_adr_coef<<<1, 1024, 0, c->stream>>>(c->adr_part, (int)nblk, c->adr_first, c->adr_st);
    k_adr_update<<<nblk, kAdrBlock, 0, c->stream>>>(a, c->disp[c->cur], c->disp[c->cur ^ 1], c->gold, c->lam,
                                                    c->adr_st,
                                                    c->precision == PD_MIXED ? c->u32[c->cur ^ 1] : nullptr,
                                                    c->precision == PD_MIXED && c->lattice ? a.lat_umax_next : nullptr);
  }
  if (prof) {
    cudaEventRecord(e2, c->stream);
    if (c->times.mid) {  // pair form: two pass-1 kernels
      c->times.ev.push_back(e0);
      c->times.ev.push_back(c->times.mid);
      c->times.which.push_back(PD_K_PASS1);
      c->times.ev.push_back(c->times.mid);
      c->times.ev.push_back(e1);
      c->times.which.push_back(PD_K_PASS1B);
      c->times.mid = nullptr;
    } else {
      c->times.ev.push_back(e0);
      c->times.ev.push_back(e1);
      c->times.which.push_back(PD_K_PASS1);
    }
    c->times.ev.push_back(e1);
    c->times.ev.push_back(e2);
    c->times.which.push_back(PD_K_PASS2);
  }
  c->cur ^= 1;
  PD_CUDA(cudaGetLastError());
  return PD_OK;
}

pd_status read_profile(pd_ctx* c) {
  if (c->times.which.empty()) return PD_OK;
  PD_CUDA(cudaStreamSynchronize(c->stream));
  for (size_t k = 0; k < c->times.which.size(); ++k) {
    float ms = 0.0f;
    PD_CUDA(cudaEventElapsedTime(&ms, c->times.ev[2 * k], c->times.ev[2 * k + 1]));
    c->times.ms[c->times.which[k]] += ms;
    c->times.launches[c->times.which[k]] += 1;
  }
  // events are shared between consecutive pairs: destroy each distinct handle once
  std::vector<cudaEvent_t> uniq(c->times.ev.begin(), c->times.ev.end());
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  for (cudaEvent_t e : uniq) cudaEventDestroy(e);
  c->times.ev.clear();
  c->times.which.clear();
  return PD_OK;
}

// The failure criterion on the current state, without advancing (used before reading damage,
// status or state, so that they equal the paper's end-of-iteration failure block).
// FP32 tables of the screened check before a read (FP64 pair form), built at the first such check;
// without them (another form, or no device memory left) the check runs in FP64 alone.
static void ensure_check_tables(pd_ctx* c) {
  if (c->cA32 || c->precision != PD_FP64 || c->kin == PD_NONLINEAR || !c->bond_cache || !c->pairs ||
      !c->pairs_ok || !c->bA || c->nentries <= 0)
    return;
  float4* cA = nullptr;
  float4* cu = nullptr;
  if (alloc(c, &cA, (size_t)c->nentries) != PD_OK || alloc(c, &cu, (size_t)c->n_pad) != PD_OK) {
    clear_error();
    return;
  }
  const int tb = 256;
  const unsigned grid = (unsigned)std::min<int64_t>((c->nentries + tb - 1) / tb, 152 * 64);
  k_check_tables<<<grid, tb, 0, c->stream>>>(c->nentries, c->bA, cA);
  if (cudaGetLastError() != cudaSuccess) return;
  c->cA32 = cA;
  c->cu32 = cu;
}

pd_status launch_refresh_check(pd_ctx* c) {
  if (!c->check_pending) return PD_OK;
  ensure_check_tables(c);
  StepArgs a = make_args(c);
  a.check = 1;
  dispatch(c, a, 1, 0);
  PD_CUDA(cudaGetLastError());
  c->check_pending = false;
  c->skip_next_check = true;  // the next step must not apply the same check again
  return PD_OK;
}

pd_status launch_damage(pd_ctx* c, double* phi_caller_dev) {
  StepArgs a = make_args(c);
  const int tb = 256;
  k_damage<<<(unsigned)((c->n_pad + tb - 1) / tb), tb, 0, c->stream>>>(a, c->n, c->dden, c->perm_dev,
                                                                      phi_caller_dev);
  PD_CUDA(cudaGetLastError());
  return PD_OK;
}

pd_status upload_field(pd_ctx* c, const double* host_soa, double4* dst, int comps) {
  PD_CUDA(cudaMemcpyAsync(c->scratch, host_soa, sizeof(double) * comps * c->n, cudaMemcpyHostToDevice, c->stream));
  return gather_field(c, c->scratch, dst, comps);
}

// Caller-order SoA field already on the device -> internal order (double4; disp keeps V in .w).
pd_status gather_field(pd_ctx* c, const double* dev_soa, double4* dst, int comps) {
  const int tb = 256;
  const bool is_disp = dst == c->disp[0] || dst == c->disp[1];
  k_gather_soa<<<(unsigned)((c->n_pad + tb - 1) / tb), tb, 0, c->stream>>>(c->n, c->n_pad, comps, dev_soa,
                                                                          c->perm_dev, is_disp ? c->pos : nullptr, dst);
  PD_CUDA(cudaGetLastError());
  return PD_OK;
}

// Sets *flag (device word) to 1 if any of the n doubles at a is not finite.
pd_status launch_nonfinite(const double* a, int64_t n, unsigned long long* flag, cudaStream_t s) {
  const int tb = 256;
  const unsigned grid = (unsigned)std::min<int64_t>((n + tb - 1) / tb, 4096);
  if (grid == 0) return PD_OK;
  k_nonfinite<<<grid, tb, 0, s>>>(n, a, flag);
  PD_CUDA(cudaGetLastError());
  return PD_OK;
}

pd_status download_field(pd_ctx* c, const double4* src, double* host_soa, int comps, cudaStream_t s) {
  const int64_t n = c->n;
  const int tb = 256;
  k_scatter_soa<<<(unsigned)((n + tb - 1) / tb), tb, 0, s>>>(n, comps, src, c->perm_dev, c->scratch);
  PD_CUDA(cudaGetLastError());
  PD_CUDA(cudaMemcpyAsync(host_soa, c->scratch, sizeof(double) * comps * n, cudaMemcpyDeviceToHost, s));
  return PD_OK;
}

pd_status download_scalar(pd_ctx* c, const double* src, double* host, cudaStream_t s) {
  const int64_t n = c->n;
  const int tb = 256;
  const bool mixed = c->precision == PD_MIXED && src == c->theta;
  k_scatter_scalar<<<(unsigned)((n + tb - 1) / tb), tb, 0, s>>>(
      n, mixed ? nullptr : src, mixed ? c->theta32 : nullptr, c->perm_dev, c->scratch);
  PD_CUDA(cudaGetLastError());
  PD_CUDA(cudaMemcpyAsync(host, c->scratch, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  return PD_OK;
}

pd_status apply_bc_now(pd_ctx* c) {
  if (!c->has_flag) return PD_OK;
  StepArgs a = make_args(c);
  const int tb = 256;
  k_apply_bc<<<(unsigned)((c->n_pad + tb - 1) / tb), tb, 0, c->stream>>>(a, c->disp[c->cur], c->steps);
  PD_CUDA(cudaGetLastError());
  return PD_OK;
}

pd_status ensure_shadow_lo(pd_ctx* c) {
  c->shadow_lo = false;
  if (!c->lattice || !c->shadow_lo_opt) return PD_OK;
  pd_status st;
  for (int k = 0; k < 2; ++k)
    if (!c->u32lo[k]) {
      if ((st = alloc(c, &c->u32lo[k], (size_t)c->n_pad)) != PD_OK) return st;
      PD_CUDA(cudaMemsetAsync(c->u32lo[k], 0, sizeof(float4) * c->n_pad, c->stream));
    }
  c->shadow_lo = true;
  return sync_shadow(c);
}

pd_status sync_shadow(pd_ctx* c) {
  if (c->precision != PD_MIXED) return PD_OK;
  const int tb = 256;
  unsigned* umax = c->lattice ? c->lat_umax + (size_t)c->cur * c->nbodies : nullptr;
  if (umax) PD_CUDA(cudaMemsetAsync(umax, 0, sizeof(unsigned) * c->nbodies, c->stream));
  k_shadow<<<(unsigned)((c->n_pad + tb - 1) / tb), tb, 0, c->stream>>>(make_args(c), c->disp[c->cur], c->u32[c->cur],
                                                                        c->shadow_lo ? c->u32lo[c->cur] : nullptr, umax);
  PD_CUDA(cudaGetLastError());
  return PD_OK;
}

// Error word of the staged kernels (a bounded wait expired); cleared after it is reported.
pd_status check_device_error(pd_ctx* c) {
  unsigned long long flag = 0;
  unsigned long long nonfinite = 0;
  PD_CUDA(cudaMemcpyAsync(&flag, c->counters + 4, sizeof(flag), cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaMemcpyAsync(&nonfinite, c->counters + 5, sizeof(nonfinite), cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaStreamSynchronize(c->stream));
  if (flag) {
    PD_CUDA(cudaMemsetAsync(c->counters + 4, 0, sizeof(flag), c->stream));
    return fail(PD_ERR_TIMEOUT, "a staged neighbour-index copy did not complete within the wait limit; "
                                "the step's results were not written");
  }
  if (nonfinite) {
    PD_CUDA(cudaMemsetAsync(c->counters + 5, 0, sizeof(nonfinite), c->stream));
    return fail(PD_ERR_NUMERIC, "the displacement became non-finite (the run diverged)");
  }
  return PD_OK;
}

pd_status max_abs_u(pd_ctx* c, double* out, int* nonfinite) {
  unsigned long long* acc = c->counters + 2;
  PD_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), c->stream));
  const int tb = 256;
  k_max_abs<<<(unsigned)((c->n + tb - 1) / tb), tb, 0, c->stream>>>(c->n, c->disp[c->cur], acc);
  PD_CUDA(cudaGetLastError());
  unsigned long long h[2];
  PD_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaStreamSynchronize(c->stream));
  double m;
  memcpy(&m, &h[0], sizeof(double));
  *out = m;
  *nonfinite = (int)h[1];
  return PD_OK;
}

// nsteps time steps: the first step after a state change skips the failure check at its head (the
// paper checks after each update, never before the first force evaluation); then CUDA-graph
// chunks of graph_chunk steps, then single steps.
pd_status run_steps(pd_ctx* c, int64_t nsteps) {
  if (nsteps <= 0) return PD_OK;
  if (c->prm[0].influence == PD_W_INV) {
    // w = delta / |xi| lives in the FP64 per-slot tables and in the lattice kernels' direction table
    if (c->solver == PD_SOLVER_ADR)
      return fail(PD_ERR_ARG, "the influence function delta / |xi| is not supported by the relaxation solver");
    if (c->precision == PD_FP64 && !c->bond_cache)
      return fail(PD_ERR_ARG, "the influence function delta / |xi| needs the FP64 bond cache (PD_OPT_BOND_CACHE)");
    if (c->precision == PD_MIXED && !c->lattice)
      return fail(PD_ERR_ARG, "the influence function delta / |xi| in PD_MIXED needs the lattice layout "
                              "(a lattice body, PD_OPT_LATTICE)");
  }
  pd_status st = ensure_bond_cache(c);
  if (st != PD_OK) return st;
  if (c->precision == PD_FP64 && !c->bond_cache) c->bs_stale = true;  // untabled kernels break bonds
  if ((st = ensure_adr(c)) != PD_OK) return st;
  st = launch_set_step(c, c->steps - 1);
  if (st != PD_OK) return st;
  int64_t left = nsteps;
  if (c->skip_next_check) {
    st = launch_step(c, false);
    if (st != PD_OK) return st;
    c->skip_next_check = false;
    --left;
    c->steps += 1;
  }
  const int chunk = c->graph_chunk;
  while (left > 0) {
    if (chunk > 0 && !c->profile && left >= chunk) {
      cudaGraphExec_t& ge = c->graph[c->cur];
      const int cur0 = c->cur;
      if (!ge) {
        cudaGraph_t g = nullptr;
        PD_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        for (int s = 0; s < chunk; ++s) {
          st = launch_step(c, true);
          if (st != PD_OK) {
            cudaStreamEndCapture(c->stream, &g);
            if (g) cudaGraphDestroy(g);
            c->cur = cur0;
            return st;
          }
        }
        PD_CUDA(cudaStreamEndCapture(c->stream, &g));
        cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          ge = nullptr;
          c->cur = cur0;
          return cuda_fail(e, "cudaGraphInstantiate");
        }
        c->cur = cur0;
      }
      PD_CUDA(cudaGraphLaunch(ge, c->stream));
      if (chunk & 1) c->cur ^= 1;
      left -= chunk;
      c->steps += chunk;
    } else {
      st = launch_step(c, true);
      if (st != PD_OK) return st;
      --left;
      c->steps += 1;
    }
  }
  c->check_pending = true;
  // divergence check, reported by the next pd_sync / pd_get_* (PD_ERR_NUMERIC)
  const int tb = 256;
  k_flag_nonfinite<<<(unsigned)((c->n + tb - 1) / tb), tb, 0, c->stream>>>(c->n, c->disp[c->cur], c->counters + 5);
  PD_CUDA(cudaGetLastError());
  return PD_OK;
}

}  // namespace pd
