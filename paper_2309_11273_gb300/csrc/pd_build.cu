// Context creation and family (neighbour-list) construction.
//
// Compiled with --fmad=false: the horizon test |xi|^2 <= delta^2 (Section 2.1, closed ball) and the
// crack-crossing test round every product and sum separately, as plain IEEE expressions, so their
// decisions do not depend on FMA contraction.
//
// Layout produced here (all in the internal Morton order of the particles):
//   slices of 32 consecutive particles (one warp); slice s owns W_s = max family size in the slice
//   "slots"; the neighbour of particle (s, lane) in slot k is col[slice_ptr[s] + 32 k + lane]
//   (sliced ELLPACK: a warp reading slot k reads 128 contiguous bytes).  Each row is sorted by the
//   reference bond vector xi (lexicographic z, y, x), so on a lattice slot k holds the same lattice
//   direction for every interior lane.  Unused slots hold the particle itself.
//   bits[slice_ptr[s] / 32 + k] bit lane = status of that entry (1 intact, 0 broken or unused).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "pd_internal.h"
#include "pd_lattice.h"

namespace pd {
namespace {

struct BuildArgs {
  int64_t n, n_pad;
  const double4* pos;
  const int4* cellc;         // cell coordinates (x, y, z) and body in .w
  const BodyGrid* grids;
  const int64_t* cell_start;
  const int32_t* cell_items;
  const CrackDev* cracks;
  int32_t ncracks;
  int32_t* cnt;
  const int64_t* slice_ptr;
  int32_t* col;
  unsigned long long* keys;
  uint32_t* bits;
  const double* body_A;
  const double* body_w;      // per body: 0 (w = 1) or delta (w = delta / |xi|)
  double* m;
  double* mu;
  double* aA;
  double* dden;
  int32_t* own0;             // pair tables (FP64 linearized contexts), else nullptr
  int32_t* twin;
  unsigned long long* missing;
};

// A bond a-b is cut by a crack iff a and b lie strictly on opposite sides of the crack line (2D) or
// plane (3D) and the crossing point lies on the closed segment / parallelogram.
template <int DIM>
__device__ bool crack_cuts(const double4& a, const double4& b, const CrackDev& c) {
  if (DIM == 2) {
    double dx = c.p[3] - c.p[0], dy = c.p[4] - c.p[1];
    double sa = dx * (a.y - c.p[1]) - dy * (a.x - c.p[0]);
    double sb = dx * (b.y - c.p[1]) - dy * (b.x - c.p[0]);
    if (!((sa > 0.0 && sb < 0.0) || (sa < 0.0 && sb > 0.0))) return false;
    double t = sa / (sa - sb);
    double px = a.x + t * (b.x - a.x);
    double py = a.y + t * (b.y - a.y);
    double lam = ((px - c.p[0]) * dx + (py - c.p[1]) * dy) / (dx * dx + dy * dy);
    return lam >= 0.0 && lam <= 1.0;
  } else {
    double e1x = c.p[3] - c.p[0], e1y = c.p[4] - c.p[1], e1z = c.p[5] - c.p[2];
    double e2x = c.p[6] - c.p[0], e2y = c.p[7] - c.p[1], e2z = c.p[8] - c.p[2];
    double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    double sa = nx * (a.x - c.p[0]) + ny * (a.y - c.p[1]) + nz * (a.z - c.p[2]);
    double sb = nx * (b.x - c.p[0]) + ny * (b.y - c.p[1]) + nz * (b.z - c.p[2]);
    if (!((sa > 0.0 && sb < 0.0) || (sa < 0.0 && sb > 0.0))) return false;
    double t = sa / (sa - sb);
    double rx = a.x + t * (b.x - a.x) - c.p[0];
    double ry = a.y + t * (b.y - a.y) - c.p[1];
    double rz = a.z + t * (b.z - a.z) - c.p[2];
    double g11 = e1x * e1x + e1y * e1y + e1z * e1z;
    double g12 = e1x * e2x + e1y * e2y + e1z * e2z;
    double g22 = e2x * e2x + e2y * e2y + e2z * e2z;
    double r1 = e1x * rx + e1y * ry + e1z * rz;
    double r2 = e2x * rx + e2y * ry + e2z * rz;
    double det = g11 * g22 - g12 * g12;
    double al = (r1 * g22 - r2 * g12) / det;
    double be = (g11 * r2 - g12 * r1) / det;
    return al >= 0.0 && al <= 1.0 && be >= 0.0 && be <= 1.0;
  }
}

// Sort key of an entry: xi quantized to delta / 2^19 per component, z major.
__device__ unsigned long long xi_key(double ex, double ey, double ez, double inv_delta) {
  const double s = 524288.0 * inv_delta;
  long long kx = llrint(ex * s) + 524288, ky = llrint(ey * s) + 524288, kz = llrint(ez * s) + 524288;
  kx = kx < 0 ? 0 : (kx > 2097151 ? 2097151 : kx);
  ky = ky < 0 ? 0 : (ky > 2097151 ? 2097151 : ky);
  kz = kz < 0 ? 0 : (kz > 2097151 ? 2097151 : kz);
  return ((unsigned long long)kz << 42) | ((unsigned long long)ky << 21) | (unsigned long long)kx;
}

// Family search over the 3^DIM cells around the particle.  EMIT = false counts; EMIT = true writes
// the entries (in cell order), sorts the row by xi and pads the unused slots.
template <int DIM, bool EMIT>
__global__ void k_family(BuildArgs A) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= A.n_pad) return;
  const int lane = (int)(i & 31);
  int64_t base = 0;
  int W = 0;
  if (EMIT) {
    const int64_t s = i >> 5;
    base = A.slice_ptr[s] + lane;
    W = (int)((A.slice_ptr[s + 1] - A.slice_ptr[s]) >> 5);
  }
  int cnt = 0;
  if (i < A.n) {
    const int4 cc = A.cellc[i];
    const BodyGrid g = A.grids[cc.w];
    const double4 pi = A.pos[i];
    const double inv_delta = 1.0 / sqrt(g.delta2);
    const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
      const int cz = cc.z + dz;
      if (cz < 0 || cz >= g.nc[2]) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int cy = cc.y + dy;
        if (cy < 0 || cy >= g.nc[1]) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int cx = cc.x + dx;
          if (cx < 0 || cx >= g.nc[0]) continue;
          const int64_t cid = g.cell_off + ((int64_t)cz * g.nc[1] + cy) * g.nc[0] + cx;
          for (int64_t t = A.cell_start[cid]; t < A.cell_start[cid + 1]; ++t) {
            const int32_t j = A.cell_items[t];
            if (j == i) continue;
            const double4 pj = A.pos[j];
            const double ex = pj.x - pi.x, ey = pj.y - pi.y, ez = pj.z - pi.z;
            double q = ex * ex + ey * ey;
            if (DIM == 3) q = q + ez * ez;
            if (!(q <= g.delta2)) continue;
            bool cut = false;
            for (int c = 0; c < A.ncracks && !cut; ++c) {
              const CrackDev& cr = A.cracks[c];
              if (cr.body >= 0 && cr.body != cc.w) continue;
              cut = crack_cuts<DIM>(pi, pj, cr);
            }
            if (cut) continue;
            if (EMIT) {
              if (cnt < W) {
                A.col[base + (int64_t)cnt * 32] = j;
                A.keys[base + (int64_t)cnt * 32] = xi_key(ex, ey, DIM == 3 ? ez : 0.0, inv_delta);
              }
            }
            ++cnt;
          }
        }
      }
    }
  }
  if (!EMIT) {
    A.cnt[i] = cnt;
    return;
  }
  if (cnt > W) cnt = W;  // cannot happen: W is the slice maximum of the same count
  // insertion sort of the row by (key, neighbour)
  for (int a = 1; a < cnt; ++a) {
    const unsigned long long ka = A.keys[base + (int64_t)a * 32];
    const int32_t ja = A.col[base + (int64_t)a * 32];
    int b = a - 1;
    while (b >= 0) {
      const unsigned long long kb = A.keys[base + (int64_t)b * 32];
      const int32_t jb = A.col[base + (int64_t)b * 32];
      if (kb < ka || (kb == ka && jb < ja)) break;
      A.keys[base + (int64_t)(b + 1) * 32] = kb;
      A.col[base + (int64_t)(b + 1) * 32] = jb;
      --b;
    }
    A.keys[base + (int64_t)(b + 1) * 32] = ka;
    A.col[base + (int64_t)(b + 1) * 32] = ja;
  }
  for (int a = cnt; a < W; ++a) A.col[base + (int64_t)a * 32] = (int32_t)i;
}

__global__ void k_slice_width(int64_t nslices, const int32_t* cnt, int32_t* width) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  int w = 0;
  for (int l = 0; l < 32; ++l) w = max(w, cnt[s * 32 + l]);
  width[s] = w;
}

// Initial status words (every built bond intact) and the per-particle sums m_i (Eq 1.9) and
// D_i = sum_j V_j (Eq 1.31 denominator), both in FP64 over the built family.  A slot holds a bond
// when its neighbour is not the particle itself (unused slots point at the particle), in both the
// sorted and the lattice layout.
template <int DIM>
__global__ void k_init_bonds(BuildArgs A) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= A.n_pad) return;  // n_pad is a multiple of 32: whole warps leave together
  const int lane = (int)(i & 31);
  const int64_t s = i >> 5;
  const int64_t base = A.slice_ptr[s];
  const int W = (int)((A.slice_ptr[s + 1] - base) >> 5);
  const double4 pi = A.pos[i];
  const double wd = A.body_w[A.cellc[i].w];
  double m = 0.0, d = 0.0;
  for (int k = 0; k < W; ++k) {
    const int32_t jk = A.col[base + (int64_t)k * 32 + lane];
    const bool built = jk != (int32_t)i;
    const unsigned word = __ballot_sync(0xffffffffu, built);
    if (lane == 0) A.bits[(base >> 5) + k] = word;
    if (built) {
      const int32_t j = jk;
      const double4 pj = A.pos[j];
      const double ex = pj.x - pi.x, ey = pj.y - pi.y, ez = pj.z - pi.z;
      double q = ex * ex + ey * ey;
      if (DIM == 3) q = q + ez * ez;
      const double w = wd > 0.0 ? wd / sqrt(q) : 1.0;  // influence function
      m += w * q * pj.w;
      d += w * pj.w;
    }
  }
  A.m[i] = m;
  A.dden[i] = d;
  const double mu = m > 0.0 ? 1.0 / m : 0.0;
  A.mu[i] = mu;
  A.aA[i] = (i < A.n) ? A.body_A[A.cellc[i].w] * mu : 0.0;
}

// Pair tables of the FP64 path.  Each undirected bond is evaluated once, by the end that owns it:
// entry (i, k) with neighbour j is owned when its key is above the key of xi = 0, or equal to it with
// j > i (so of the two entries of a pair exactly one is owned, the key of -xi being the mirror image
// of the key of xi component by component).  Rows are sorted by (key, neighbour), so a particle's
// owned entries are the tail of its row from own0[i]; twin[e] of an owned entry is the index of the
// entry (j, k') whose neighbour is i, found by binary search of row j for (mirror key, i).  A pair
// whose second entry is missing (a family that is not exactly symmetric) is counted in *missing.
__device__ __forceinline__ unsigned long long mirror_key(unsigned long long k) {
  const unsigned long long c = 1048576ull, m = 2097151ull;
  return ((c - ((k >> 42) & m)) << 42) | ((c - ((k >> 21) & m)) << 21) | (c - (k & m));
}

__global__ void k_twins(BuildArgs A) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= A.n_pad) return;
  const int lane = (int)(i & 31);
  const int64_t base = A.slice_ptr[i >> 5] + lane;
  const int cnt = A.cnt[i];
  const unsigned long long key0 = (524288ull << 42) | (524288ull << 21) | 524288ull;
  int own = cnt;
  for (int k = 0; k < cnt; ++k) {
    const unsigned long long key = A.keys[base + (int64_t)k * 32];
    if (key > key0 || (key == key0 && A.col[base + (int64_t)k * 32] > i)) {
      own = k;
      break;
    }
  }
  A.own0[i] = own;
  for (int k = own; k < cnt; ++k) {
    const int64_t e = base + (int64_t)k * 32;
    const int32_t j = A.col[e];
    const unsigned long long mk = mirror_key(A.keys[e]);
    const int64_t bj = A.slice_ptr[j >> 5] + (j & 31);
    int lo = 0, hi = A.cnt[j];  // first entry of row j not below (mk, i)
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      const unsigned long long km = A.keys[bj + (int64_t)mid * 32];
      const int32_t jm = A.col[bj + (int64_t)mid * 32];
      if (km < mk || (km == mk && jm < (int32_t)i)) lo = mid + 1;
      else hi = mid;
    }
    const int64_t t = bj + (int64_t)lo * 32;
    if (lo < A.cnt[j] && A.col[t] == (int32_t)i && A.keys[t] == mk) {
      A.twin[e] = (int32_t)t;
    } else {
      A.twin[e] = -1;
      atomicAdd(A.missing, 1ull);
    }
  }
}

// ----------------------------------------------------------------------------- lattice layout
// A body whose particles sit on a regular lattice of spacing h has every bond vector equal to h n,
// n an integer vector, and its family (the closed ball of Section 2.1) is the set of lattice
// directions with |n|^2 <= (delta / h)^2, a prefix of the direction table of pd_lattice.h.  The three
// kernels below find each body's shortest bond (its spacing), check every bond vector of the sorted
// layout against h n, and move each bond to the slot of its direction in the lattice layout, where
// slot k of every slice holds direction k for every lane (unused slots point at the particle).
struct LatArgs {
  int64_t n_pad;
  const double4* pos;
  const int32_t* body;        // per particle, internal order
  const int64_t* slice_ptr;   // sorted layout
  const int32_t* col;
  const int32_t* cnt;
  const double* inv_h;        // per body: 1 / h
  unsigned long long* minq;   // per body: shortest |xi|^2 (bits of a positive double)
  int* stats;                 // per body: [0] not a lattice, [1] largest |n|^2, [2] largest |n|_1
  int* emit_fail;             // a bond without a free slot of its direction (duplicate direction)
  const short* lookup;        // direction index of n (lattice_lookup)
  int R;                      // component bound of the table
  const int64_t* slice_ptr2;  // lattice layout
  int32_t* col2;
  double* nsum;               // per particle: sum of w' |n|^2 over its bonds (m_i = V h^2 nsum_i (w / w'))
  const double* body_w;       // per body: 0 (w = 1, w' = 1) or delta (w = delta / |xi|, w' = 1 / |n|)
};

template <int DIM>
__global__ void k_lat_minq(LatArgs L) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= L.n_pad) return;
  const int cnt = L.cnt[i];
  if (cnt == 0) return;
  const int64_t base = L.slice_ptr[i >> 5] + (i & 31);
  const double4 pi = L.pos[i];
  double mq = 1e300;
  for (int k = 0; k < cnt; ++k) {
    const double4 pj = L.pos[L.col[base + (int64_t)k * 32]];
    const double ex = pj.x - pi.x, ey = pj.y - pi.y, ez = DIM == 3 ? pj.z - pi.z : 0.0;
    mq = fmin(mq, ex * ex + ey * ey + ez * ez);
  }
  atomicMin(&L.minq[L.body[i]], (unsigned long long)__double_as_longlong(mq));
}

// n of a bond vector in units of h, with its largest deviation from the integers.
template <int DIM>
__device__ __forceinline__ void lat_n(const double4& pi, const double4& pj, double inv_h, int (&n)[3], double& dev) {
  const double f[3] = {(pj.x - pi.x) * inv_h, (pj.y - pi.y) * inv_h, DIM == 3 ? (pj.z - pi.z) * inv_h : 0.0};
  dev = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double r = rint(f[c]);
    dev = fmax(dev, fabs(f[c] - r));
    n[c] = fabs(r) < 1e6 ? (int)r : 1000000;
  }
}

template <int DIM>
__device__ __forceinline__ int lat_dir(const LatArgs& L, const int (&n)[3]) {
  if (abs(n[0]) > L.R || abs(n[1]) > L.R || abs(n[2]) > (DIM == 3 ? L.R : 0)) return -1;
  const int s = 2 * L.R + 1;
  const int idx = DIM == 3 ? ((n[2] + L.R) * s + (n[1] + L.R)) * s + (n[0] + L.R) : (n[1] + L.R) * s + (n[0] + L.R);
  return L.lookup[idx];
}

template <int DIM>
__global__ void k_lat_classify(LatArgs L) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= L.n_pad) return;
  const int cnt = L.cnt[i];
  if (cnt == 0) return;
  const int b = L.body[i];
  const double inv_h = L.inv_h[b];
  const int64_t base = L.slice_ptr[i >> 5] + (i & 31);
  const double4 pi = L.pos[i];
  int q1 = 0, n1m = 0;
  bool bad = false;
  for (int k = 0; k < cnt; ++k) {
    const double4 pj = L.pos[L.col[base + (int64_t)k * 32]];
    int n[3];
    double dev;
    lat_n<DIM>(pi, pj, inv_h, n, dev);
    // bond vectors within 2^-30 h of h n (the positions of a lattice, rounded), inside the table
    if (!(dev <= 9.313225746154785e-10) || lat_dir<DIM>(L, n) < 0) {
      bad = true;
      break;
    }
    q1 = max(q1, n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n1m = max(n1m, abs(n[0]) + abs(n[1]) + abs(n[2]));
  }
  if (bad) {
    atomicOr(&L.stats[3 * b], 1);
    return;
  }
  atomicMax(&L.stats[3 * b + 1], q1);
  atomicMax(&L.stats[3 * b + 2], n1m);
}

template <int DIM>
__global__ void k_lat_emit(LatArgs L) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= L.n_pad) return;
  const int64_t s = i >> 5;
  const int64_t base2 = L.slice_ptr2[s] + (i & 31);
  const int W2 = (int)((L.slice_ptr2[s + 1] - L.slice_ptr2[s]) >> 5);
  for (int k = 0; k < W2; ++k) L.col2[base2 + (int64_t)k * 32] = (int32_t)i;
  const int cnt = L.cnt[i];
  const int64_t base = L.slice_ptr[s] + (i & 31);
  const double4 pi = L.pos[i];
  const double inv_h = L.inv_h[L.body[i]];
  const bool winv = L.body_w[L.body[i]] > 0.0;
  double nsum = 0.0;
  for (int k = 0; k < cnt; ++k) {
    const int32_t j = L.col[base + (int64_t)k * 32];
    int n[3];
    double dev;
    lat_n<DIM>(pi, L.pos[j], inv_h, n, dev);
    const int d = lat_dir<DIM>(L, n);
    if (d < 0 || d >= W2 || L.col2[base2 + (int64_t)d * 32] != (int32_t)i) {
      atomicOr(L.emit_fail, 1);
      continue;
    }
    L.col2[base2 + (int64_t)d * 32] = j;
    const int q = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
    nsum += winv ? sqrt((double)q) : (double)q;  // w' |n|^2 with w' = 1 / |n| or 1
  }
  L.nsum[i] = nsum;
}

// Per slice: 1 when every lane and every neighbour of it has N_j = N_ref (rho = 1), so the force
// pass need not gather the neighbours' N_ref / N_j.
__global__ void k_lat_interior(int64_t n_pad, const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ col,
                               const float2* __restrict__ f, uint8_t* __restrict__ flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_pad) return;  // n_pad is a multiple of 32: whole warps
  const int64_t s = i >> 5;
  const int64_t base = slice_ptr[s] + (i & 31);
  const int W = (int)((slice_ptr[s + 1] - slice_ptr[s]) >> 5);
  bool ok = f[i].x == 1.0f;
  for (int k = 0; k < W && ok; ++k) {
    const int32_t j = col[base + (int64_t)k * 32];
    if (j != (int32_t)i) ok = f[j].x == 1.0f;
  }
  const unsigned all = __ballot_sync(0xffffffffu, ok);
  if ((i & 31) == 0) flag[s] = all == 0xffffffffu ? 1 : 0;
}

// Tries the lattice layout for a mixed-precision context with linearized bonds (called after the
// sorted layout and its status words are built).  Every body must have uniform volumes and bond
// vectors within 2^-30 h of h n with n inside the direction table; otherwise the sorted layout stays
// and *done is false.  On success the context's col, bits and slice_ptr are replaced, m_i and D_i
// are recomputed over the new slots, and the per-particle factors of the lattice kernels are set.
pd_status build_lattice(pd_ctx* c, BuildArgs& A, bool* done) {
  *done = false;
  const int dim = c->dim, nb = c->nbodies;
  const int64_t n = c->n, n_pad = c->n_pad;
  for (int b = 0; b < nb; ++b) {
    const double v0 = c->hvol[c->body_off[b]];
    for (int64_t u = c->body_off[b]; u < c->body_off[b + 1]; ++u)
      if (c->hvol[u] != v0) return PD_OK;  // non-uniform volumes: sorted layout
  }
  cudaStream_t s = c->stream;
  const std::vector<short> cube = lattice_lookup(dim);
  double* d_inv_h = nullptr;
  unsigned long long* d_minq = nullptr;
  int* d_stats = nullptr;
  short* d_lookup = nullptr;
  double* d_nsum = nullptr;
  double* d_bw = nullptr;
  int64_t* sptr2_dev = nullptr;
  int32_t* col2 = nullptr;
  uint32_t* bits2 = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_inv_h);
    cudaFree(d_minq);
    cudaFree(d_stats);
    cudaFree(d_lookup);
    cudaFree(d_nsum);
    cudaFree(d_bw);
  };
  auto tmp = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  if (!tmp((void**)&d_inv_h, sizeof(double) * nb) || !tmp((void**)&d_minq, sizeof(unsigned long long) * nb) ||
      !tmp((void**)&d_stats, sizeof(int) * (3 * nb + 1)) || !tmp((void**)&d_lookup, sizeof(short) * cube.size()) ||
      !tmp((void**)&d_nsum, sizeof(double) * n_pad) || !tmp((void**)&d_bw, sizeof(double) * nb)) {
    cleanup();
    return fail(PD_ERR_OOM, "cudaMalloc of lattice build temporaries failed");
  }
  const unsigned long long big = 0x7fefffffffffffffull;  // bits of the largest finite double
  std::vector<unsigned long long> hminq(nb, big);
  std::vector<int> hstats(3 * nb + 1, 0);
  LatArgs L{};
  L.n_pad = n_pad;
  L.pos = c->pos;
  L.body = c->body;
  L.slice_ptr = c->slice_ptr;
  L.col = c->col;
  L.cnt = c->cnt;
  L.inv_h = d_inv_h;
  L.minq = d_minq;
  L.stats = d_stats;
  L.emit_fail = d_stats + 3 * nb;
  L.lookup = d_lookup;
  L.R = dim == 3 ? kLatR3 : kLatR2;
  L.nsum = d_nsum;
  L.body_w = d_bw;
  std::vector<double> hbw(nb);
  for (int b = 0; b < nb; ++b) hbw[b] = c->prm[b].influence == PD_W_INV ? c->prm[b].horizon : 0.0;
  const int tb = 128;
  const unsigned gb = (unsigned)((n_pad + tb - 1) / tb);
  cudaError_t e = cudaMemcpyAsync(d_minq, hminq.data(), sizeof(unsigned long long) * nb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_stats, hstats.data(), sizeof(int) * hstats.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_lookup, cube.data(), sizeof(short) * cube.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_bw, hbw.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    if (dim == 3) k_lat_minq<3><<<gb, tb, 0, s>>>(L);
    else k_lat_minq<2><<<gb, tb, 0, s>>>(L);
    e = cudaMemcpyAsync(hminq.data(), d_minq, sizeof(unsigned long long) * nb, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "lattice spacing");
  }
  std::vector<double> h(nb), inv_h(nb);
  for (int b = 0; b < nb; ++b) {
    double q;
    std::memcpy(&q, &hminq[b], sizeof(q));
    if (hminq[b] == big || !(q > 0.0)) {  // a body without bonds
      cleanup();
      return PD_OK;
    }
    h[b] = std::sqrt(q);
    inv_h[b] = 1.0 / h[b];
  }
  e = cudaMemcpyAsync(d_inv_h, inv_h.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    if (dim == 3) k_lat_classify<3><<<gb, tb, 0, s>>>(L);
    else k_lat_classify<2><<<gb, tb, 0, s>>>(L);
    e = cudaMemcpyAsync(hstats.data(), d_stats, sizeof(int) * hstats.size(), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "lattice check");
  }
  std::vector<int> S(nb);
  for (int b = 0; b < nb; ++b) {
    if (hstats[3 * b] != 0 || hstats[3 * b + 1] < 1) {
      cleanup();
      return PD_OK;
    }
    S[b] = lattice_prefix(dim, hstats[3 * b + 1]);
    if (S[b] < 0) {  // the family is not a prefix of the table: keep the general layout
      cleanup();
      return PD_OK;
    }
  }
  // slice widths of the lattice layout: the largest family prefix among the slice's bodies, rounded
  // up to a multiple of 4 (16-byte aligned status words for the bulk copies)
  std::vector<int64_t> sptr2(c->nslices + 1, 0);
  for (int64_t t = 0; t < c->nslices; ++t) {
    int w = 0;
    for (int l = 0; l < 32; ++l) {
      const int64_t k = t * 32 + l;
      if (k < n) w = std::max(w, S[c->body_of[k]]);
    }
    sptr2[t + 1] = sptr2[t] + 32 * (((int64_t)w + 3) & ~3LL);
  }
  const int64_t ne2 = sptr2[c->nslices];
  pd_status st = PD_OK;
  if ((st = alloc(c, &sptr2_dev, (size_t)c->nslices + 1)) != PD_OK ||
      (st = alloc(c, &col2, (size_t)std::max<int64_t>(ne2, 32))) != PD_OK ||
      (st = alloc(c, &bits2, (size_t)std::max<int64_t>(ne2 / 32, 1))) != PD_OK) {
    release(c, sptr2_dev);
    release(c, col2);
    release(c, bits2);
    cleanup();
    if (st == PD_ERR_OOM) {  // not enough memory for a second layout: keep the sorted one
      clear_error();
      return PD_OK;
    }
    return st;
  }
  L.slice_ptr2 = sptr2_dev;
  L.col2 = col2;
  int efail = 0;
  e = cudaMemcpyAsync(sptr2_dev, sptr2.data(), sizeof(int64_t) * sptr2.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    if (dim == 3) k_lat_emit<3><<<gb, tb, 0, s>>>(L);
    else k_lat_emit<2><<<gb, tb, 0, s>>>(L);
    e = cudaMemcpyAsync(&efail, d_stats + 3 * nb, sizeof(int), cudaMemcpyDeviceToHost, s);
  }
  std::vector<double> hnsum(n_pad);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hnsum.data(), d_nsum, sizeof(double) * n_pad, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || efail) {
    release(c, sptr2_dev);
    release(c, col2);
    release(c, bits2);
    cleanup();
    return e != cudaSuccess ? cuda_fail(e, "lattice layout") : PD_OK;
  }
  // the lattice layout replaces the sorted one; m_i, D_i and the status words over the new slots
  release(c, c->col);
  release(c, c->bits);
  release(c, c->slice_ptr);
  c->col = col2;
  c->bits = bits2;
  c->slice_ptr = sptr2_dev;
  c->nentries = ne2;
  A.slice_ptr = c->slice_ptr;
  A.col = c->col;
  A.bits = c->bits;
  if (dim == 3) k_init_bonds<3><<<gb, tb, 0, s>>>(A);
  else k_init_bonds<2><<<gb, tb, 0, s>>>(A);
  // per particle (N_ref / N_i, A / N_i), N_ref the largest N_i of the body (its interior value; every
  // interior particle sums the same terms in the same order, so their N_i are equal bit for bit)
  c->lat_h = h;
  c->lat_nref.assign(nb, 0.0);
  c->lat_qmax.assign(nb, 0);
  c->lat_n1.assign(nb, 0);
  for (int64_t k = 0; k < n; ++k) c->lat_nref[c->body_of[k]] = std::max(c->lat_nref[c->body_of[k]], hnsum[k]);
  for (int b = 0; b < nb; ++b) {
    c->lat_qmax[b] = hstats[3 * b + 1];
    c->lat_n1[b] = hstats[3 * b + 2];
  }
  std::vector<float2> hf(n_pad, make_float2(0.0f, 0.0f));
  for (int64_t k = 0; k < n; ++k) {
    const int b = c->body_of[k];
    double A_b, K_b, G_b;
    material_constants(c->prm[b].model, c->prm[b].E, c->prm[b].nu, &A_b, &K_b, &G_b);
    if (hnsum[k] > 0)
      hf[k] = make_float2((float)(c->lat_nref[b] / hnsum[k]), (float)(A_b / hnsum[k]));
  }
  std::vector<float> hr(n_pad);
  for (int64_t k = 0; k < n_pad; ++k) hr[k] = hf[k].x;
  if ((st = alloc(c, &c->lat_f, (size_t)n_pad)) != PD_OK || (st = alloc(c, &c->lat_rho, (size_t)n_pad)) != PD_OK ||
      (st = alloc(c, &c->lat_up, (size_t)n_pad)) != PD_OK ||
      (st = alloc(c, &c->lat_int, (size_t)c->nslices)) != PD_OK ||
      (st = alloc(c, &c->lat_umax, (size_t)2 * nb)) != PD_OK) {
    cleanup();
    return st;
  }
  e = cudaMemcpyAsync(c->lat_f, hf.data(), sizeof(float2) * n_pad, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->lat_rho, hr.data(), sizeof(float) * n_pad, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->lat_up, 0, sizeof(float4) * n_pad, s);
  // 0x7f7f7f7f = 3.4e38: a bound above any shadow until the first shadow write replaces it
  if (e == cudaSuccess) e = cudaMemsetAsync(c->lat_umax, 0x7f, sizeof(unsigned) * 2 * nb, s);
  if (e == cudaSuccess) {
    k_lat_interior<<<gb, tb, 0, s>>>(n_pad, c->slice_ptr, c->col, c->lat_f, c->lat_int);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "lattice factors");
  // the common slice width (one family prefix for the whole context), 0 if the widths differ
  c->lat_wuni = (int)((sptr2[1] - sptr2[0]) >> 5);
  for (int64_t t = 0; t < c->nslices; ++t)
    if ((int)((sptr2[t + 1] - sptr2[t]) >> 5) != c->lat_wuni) c->lat_wuni = 0;
  c->lattice = true;
  *done = true;
  return upload_body_params(c);
}

// Morton key of 21-bit quantized coordinates.
uint64_t spread3(uint64_t v) {
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}
uint64_t spread2(uint64_t v) {
  v &= 0xffffffffULL;
  v = (v | v << 16) & 0x0000ffff0000ffffULL;
  v = (v | v << 8) & 0x00ff00ff00ff00ffULL;
  v = (v | v << 4) & 0x0f0f0f0f0f0f0f0fULL;
  v = (v | v << 2) & 0x3333333333333333ULL;
  v = (v | v << 1) & 0x5555555555555555ULL;
  return v;
}

bool finite_all(const double* a, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

pd_status check_params(const pd_params& p, int dim) {
  if (p.model < 0 || p.model > 2) return fail(PD_ERR_ARG, "unknown model");
  if ((p.model == PD_3D) != (dim == 3)) return fail(PD_ERR_ARG, "z must be given exactly for PD_3D");
  if (p.precision != PD_FP64 && p.precision != PD_MIXED) return fail(PD_ERR_ARG, "unknown precision");
  if (p.influence != PD_W_ONE && p.influence != PD_W_INV) return fail(PD_ERR_ARG, "unknown influence function");
  if (p.influence == PD_W_INV && p.kinematics != PD_LINEARIZED)
    return fail(PD_ERR_ARG, "the influence function delta / |xi| is supported with linearized bonds only");
  if (!(p.E > 0) || !std::isfinite(p.E)) return fail(PD_ERR_ARG, "E must be > 0");
  if (!(p.nu > -1.0 && p.nu < 0.5)) return fail(PD_ERR_ARG, "nu must lie in (-1, 0.5)");
  if (!(p.rho > 0) || !std::isfinite(p.rho)) return fail(PD_ERR_ARG, "rho must be > 0");
  if (!(p.horizon > 0) || !std::isfinite(p.horizon)) return fail(PD_ERR_ARG, "horizon must be > 0");
  if (!(p.dt > 0) || !std::isfinite(p.dt)) return fail(PD_ERR_ARG, "dt must be > 0");
  if (!std::isfinite(p.s0)) return fail(PD_ERR_ARG, "s0 must be finite");
  if (p.ordering != PD_ORDER_BRICKS && p.ordering != PD_ORDER_MORTON) return fail(PD_ERR_ARG, "unknown ordering");
  if (p.kinematics != PD_LINEARIZED && p.kinematics != PD_NONLINEAR) return fail(PD_ERR_ARG, "unknown kinematics");
  return PD_OK;
}

}  // namespace

// Material constants: A (Eq 1.8), K (Eq 1.15), G (Eq 1.16) from E and nu.
void material_constants(int model, double E, double nu, double* A, double* K, double* G) {
  const double kappa = E / (3.0 * (1.0 - 2.0 * nu));
  const double mu = E / (2.0 * (1.0 + nu));
  if (model == PD_3D) {
    *A = 3.0;
    *K = 3.0 * kappa;
    *G = 15.0 * mu;
  } else if (model == PD_PLANE_STRESS) {
    *A = 2.0 * (1.0 - 2.0 * nu) / (1.0 - nu);
    *K = 2.0 * kappa * (1.0 - 2.0 * nu) / (1.0 - nu) -
         2.0 / 3.0 * mu * (1.0 + nu) * (1.0 - 3.0 * nu) / ((1.0 - nu) * (1.0 - 2.0 * nu));
    *G = 8.0 * mu;
  } else {
    *A = 2.0;
    *K = 2.0 * kappa - 2.0 / 3.0 * mu;
    *G = 8.0 * mu;
  }
}

pd_status upload_body_params(pd_ctx* c);

// Creation shared by pd_create_particles and pd_create_batch.
pd_status create(pd_ctx** out, int32_t nbodies, const pd_params* prm, const int64_t* offsets,
                 const double* x, const double* y, const double* z, const double* vol) {
  clear_error();
  if (!out) return fail(PD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!prm || !x || !y || !vol) return fail(PD_ERR_ARG, "prm, x, y and vol are required");
  if (nbodies < 1) return fail(PD_ERR_ARG, "nbodies must be >= 1");
  const int dim = z ? 3 : 2;
  const int64_t n = offsets[nbodies];
  if (n < 1 || n > 2147483647LL - 64) return fail(PD_ERR_ARG, "particle count out of range");
  for (int b = 0; b < nbodies; ++b) {
    if (offsets[b + 1] <= offsets[b]) return fail(PD_ERR_ARG, "every body needs >= 1 particle");
    pd_status st = check_params(prm[b], dim);
    if (st != PD_OK) return st;
    if (prm[b].model != prm[0].model || prm[b].precision != prm[0].precision ||
        prm[b].device != prm[0].device || prm[b].stream != prm[0].stream ||
        prm[b].kinematics != prm[0].kinematics || prm[b].influence != prm[0].influence)
      return fail(PD_ERR_ARG, "bodies must share model, precision, kinematics, influence, device and stream");
  }
  if (!finite_all(x, n) || !finite_all(y, n) || (z && !finite_all(z, n)) || !finite_all(vol, n))
    return fail(PD_ERR_ARG, "non-finite coordinate or volume");
  for (int64_t i = 0; i < n; ++i)
    if (!(vol[i] > 0)) return fail(PD_ERR_ARG, "volumes must be > 0");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(PD_ERR_CUDA, "no CUDA device available");
  }
  if (prm[0].device < 0 || prm[0].device >= ndev) return fail(PD_ERR_ARG, "bad device ordinal");
  PD_CUDA(cudaSetDevice(prm[0].device));

  pd_ctx* c = new pd_ctx();
  c->device = prm[0].device;
  c->dim = dim;
  c->model = prm[0].model;
  c->precision = prm[0].precision;
  c->kin = prm[0].kinematics;
  c->n = n;
  c->nslices = (n + kSlice - 1) / kSlice;
  c->n_pad = c->nslices * kSlice;
  c->nbodies = nbodies;
  c->prm.assign(prm, prm + nbodies);
  c->body_off.assign(offsets, offsets + nbodies + 1);
  c->hx.assign(x, x + n);
  c->hy.assign(y, y + n);
  if (z) c->hz.assign(z, z + n);
  c->hvol.assign(vol, vol + n);
  c->vol_uniform = true;
  for (int b = 0; b < nbodies && c->vol_uniform; ++b)
    for (int64_t u = offsets[b]; u < offsets[b + 1]; ++u)
      if (vol[u] != vol[offsets[b]]) {
        c->vol_uniform = false;
        break;
      }
  if (prm[0].stream) {
    c->stream = (cudaStream_t)prm[0].stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    c->own_stream = true;
  }

  // Internal order inside each body (bodies stay contiguous in their given order):
  //   PD_ORDER_MORTON: Morton curve of the coordinates;
  //   PD_ORDER_BRICKS: bricks of 32 x 4 x 4 (3D) / 32 x 8 (2D) points of the body's typical spacing
  //     h = (mean V)^(1/dim), row-major (x fastest) inside a brick, bricks along a Morton curve.  A
  //     32-particle slice is then one x-row, and the 32 neighbours a warp gathers for one slot (the
  //     same bond direction on a lattice) form a shifted contiguous row.
  std::vector<uint64_t> key(n);
  c->body_of.assign(n, 0);
  const int ordering = prm[0].ordering;
  for (int b = 0; b < nbodies; ++b) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    double vsum = 0.0;
    for (int64_t i = offsets[b]; i < offsets[b + 1]; ++i) {
      const double p[3] = {x[i], y[i], z ? z[i] : 0.0};
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], p[k]);
        hi[k] = std::max(hi[k], p[k]);
      }
      vsum += vol[i];
    }
    double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    if (!(ext > 0)) ext = 1.0;
    const int64_t nb = offsets[b + 1] - offsets[b];
    double h = std::pow(vsum / (double)nb, 1.0 / dim);
    if (!(h > 0) || ext / h > 1e6) h = ext / 1e6;
    for (int64_t i = offsets[b]; i < offsets[b + 1]; ++i) {
      c->body_of[i] = b;
      const double p[3] = {x[i], y[i], z ? z[i] : 0.0};
      if (ordering == PD_ORDER_MORTON) {
        const double bitsmax = dim == 3 ? 2097151.0 : 4294967295.0;
        const double sc = bitsmax / ext;
        uint64_t q[3];
        for (int k = 0; k < 3; ++k) q[k] = (uint64_t)std::min(bitsmax, std::max(0.0, (p[k] - lo[k]) * sc));
        key[i] = dim == 3 ? (spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2))
                          : (spread2(q[0]) | (spread2(q[1]) << 1));
      } else {
        int64_t g[3];
        for (int k = 0; k < 3; ++k) g[k] = std::max<int64_t>(0, std::llrint((p[k] - lo[k]) / h));
        if (dim == 3) {
          const uint64_t loc = (uint64_t)(((g[2] & 3) * 4 + (g[1] & 3)) * 32 + (g[0] & 31));
          key[i] = ((spread3((uint64_t)(g[0] >> 5)) | (spread3((uint64_t)(g[1] >> 2)) << 1) |
                     (spread3((uint64_t)(g[2] >> 2)) << 2)) << 9) | loc;
        } else {
          const uint64_t loc = (uint64_t)((g[1] & 7) * 32 + (g[0] & 31));
          key[i] = ((spread2((uint64_t)(g[0] >> 5)) | (spread2((uint64_t)(g[1] >> 3)) << 1)) << 8) | loc;
        }
      }
    }
  }
  c->perm.resize(n);
  std::iota(c->perm.begin(), c->perm.end(), 0);
  std::stable_sort(c->perm.begin(), c->perm.end(), [&](int64_t a, int64_t b) {
    if (c->body_of[a] != c->body_of[b]) return c->body_of[a] < c->body_of[b];
    return key[a] < key[b];
  });
  std::vector<int32_t> body_int(c->n_pad, 0);
  for (int64_t k = 0; k < n; ++k) body_int[k] = c->body_of[c->perm[k]];
  for (int64_t k = n; k < c->n_pad; ++k) body_int[k] = body_int[n - 1];
  c->body_of.assign(body_int.begin(), body_int.end());

  pd_status st = PD_OK;
  std::vector<double4> hpos(c->n_pad);
  for (int64_t k = 0; k < c->n_pad; ++k) {
    if (k < n) {
      const int64_t u = c->perm[k];
      hpos[k] = make_double4(x[u], y[u], z ? z[u] : 0.0, vol[u]);
    } else {
      // padding particles: far from everything, unit volume, never part of a family
      const int64_t u = c->perm[n - 1];
      hpos[k] = make_double4(x[u], y[u], z ? z[u] : 0.0, 1.0);
    }
  }
  std::vector<int64_t> hperm(c->perm.begin(), c->perm.end());
#define PD_TRY(expr)              \
  do {                            \
    st = (expr);                  \
    if (st != PD_OK) goto failed; \
  } while (0)
  PD_TRY(alloc(c, &c->pos, c->n_pad));
  PD_TRY(alloc(c, &c->body, c->n_pad));
  PD_TRY(alloc(c, &c->bp, nbodies));
  PD_TRY(alloc(c, &c->perm_dev, n));
  PD_TRY(alloc(c, &c->d_step, 1));
  PD_TRY(alloc(c, &c->counters, 8));
  PD_TRY(alloc(c, &c->scratch, (size_t)c->n_pad * 3));
  PD_TRY(alloc(c, &c->scratch2, (size_t)c->n_pad * 3));
  if (cudaMemcpyAsync(c->pos, hpos.data(), sizeof(double4) * c->n_pad, cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->body, body_int.data(), sizeof(int32_t) * c->n_pad, cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->perm_dev, hperm.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * 8, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    st = cuda_fail(cudaGetLastError(), "upload of particles");
    goto failed;
  }
  {
    // Fixed-point quantum of the mixed path: a power of two with every coordinate offset < 2^30 Q.
    // (A quantum that makes lattice bond vectors exact was measured to give larger FP32 errors: the
    // rounding becomes systematic across the symmetric family.)
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < n; ++i) {
      const double p[3] = {x[i], y[i], z ? z[i] : 0.0};
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], p[k]);
        hi[k] = std::max(hi[k], p[k]);
      }
    }
    double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    if (!(ext > 0)) ext = 1.0;
    c->q = std::ldexp(1.0, (int)std::ceil(std::log2(ext / 1073741824.0)));
    for (int k = 0; k < 3; ++k) c->qlo[k] = lo[k];
  }
  c->n_create_allocs = c->allocs.size();
  PD_TRY(upload_body_params(c));
  *out = c;
  return PD_OK;
failed:
  free_all(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return st;
#undef PD_TRY
}

// Per-body constants for the kernels (also refreshed when the rotation rate changes).
pd_status upload_body_params(pd_ctx* c) {
  std::vector<BodyDev> h(c->nbodies);
  for (int b = 0; b < c->nbodies; ++b) {
    const pd_params& p = c->prm[b];
    double A, K, G;
    material_constants(p.model, p.E, p.nu, &A, &K, &G);
    BodyDev& d = h[b];
    d.A = A;
    d.Kp = K - G / 3.0;
    d.G = G;
    d.inv_rho = 1.0 / p.rho;
    d.dt = p.dt;
    d.s0 = p.s0;
    d.s0nl = p.s0 * (2.0 + p.s0);
    d.breaks = p.s0 > 0.0 ? 1 : 0;
    d.rate = 0.0;
    d.wdelta = p.influence == PD_W_INV ? p.horizon : 0.0;
    d.Kp32 = (float)(d.Kp * c->q);
    d.G32 = (float)d.G;
    d.G32q = (float)(d.G * c->q);
    d.s0nl32 = (float)d.s0nl;
    d.inv_rho32 = (float)d.inv_rho;
    d.sigma_q = p.s0 * c->q;
    d.sigma32 = (float)d.sigma_q;
    // |xi| <= delta; each fixed-point component of xi is within one quantum of the exact value
    const double lq = p.horizon / c->q + 2.0;
    d.xi1max = (float)(std::sqrt((double)c->dim) * lq * 1.0001);
    d.qmax = (float)(lq * lq * 1.0001);
    d.lat_h = d.lat_inv_h = d.lat_C = d.lat_K = d.lat_Kb = 0.0;
    d.lat_lam_hi = d.lat_lam_lo = d.lat_s0 = 0.0f;
    d.lat_Kf = d.lat_sq = d.lat_eps_c = d.lat_s0n1 = d.lat_Kfast = d.lat_Kcfast = 0.0f;
    if (c->lattice) {
      // FP32 sums in lattice units (u' = u / h, xi = h n, m_i = V h^2 N_i): F_i / V_i = G / (h N_ref) x
      // sum_j rho_ij n [P_i + P_j + (N_ref/N_i + N_ref/N_j) n.(u'_j - u'_i) / |n|^2] with
      // P_i = lambda sigma_i (N_ref/N_i)^2, sigma_i = sum_j rho_ij n.(u'_j - u'_i), theta_i = A sigma_i / N_i
      const double h = c->lat_h[b];
      const double nref = c->lat_nref[b];
      const int n1 = c->lat_n1[b], qm = c->lat_qmax[b];
      d.lat_h = h;
      d.lat_inv_h = 1.0 / h;
      d.lat_C = G / (h * nref);
      d.lat_K = d.lat_C * p.dt * d.inv_rho;
      d.lat_Kb = p.dt * d.inv_rho;
      const double lam = (K - G / 3.0) * A / (G * nref);
      d.lat_lam_hi = (float)lam;
      d.lat_lam_lo = (float)(lam - (double)d.lat_lam_hi);
      d.lat_s0 = (float)p.s0;
      // rounding band of the FP32 break test (pd_lattice.h)
      const LatBand lb = lattice_band(p.band_safety, p.s0, n1, qm);
      d.lat_Kf = lb.Kf;
      d.lat_sq = lb.sq;
      d.lat_eps_c = lb.eps_c;
      d.lat_s0n1 = lb.s0n1;
      d.lat_Kfast = lb.Kfast;
      d.lat_Kcfast = lb.Kcfast;
      // nonlinear bonds: |n_c| <= sqrt(qmax) for every direction of the family
      const LatBandNL nb = lattice_band_nl(p.band_safety, p.s0, n1, (int)std::floor(std::sqrt((double)qm)), qm);
      d.nl_A0 = nb.A0;
      d.nl_A0s = nb.A0s;
      d.nl_A1 = nb.A1;
      d.nl_A1s = nb.A1s;
      d.nl_A2 = nb.A2;
      d.nl_Ag = nb.Ag;
      d.nl_F0 = nb.F0;
      d.nl_F0s = nb.F0s;
      d.nl_F1 = nb.F1;
      d.nl_F1s = nb.F1s;
      d.nl_F2 = nb.F2;
    }
  }
  for (int b = 0; b < c->nbodies; ++b) h[b].rate = c->rate;
  PD_CUDA(cudaMemcpyAsync(c->bp, h.data(), sizeof(BodyDev) * c->nbodies, cudaMemcpyHostToDevice, c->stream));
  PD_CUDA(cudaStreamSynchronize(c->stream));
  return PD_OK;
}

pd_status build_neighbors(pd_ctx* c, const pd_crack* cracks, int32_t ncracks) {
  clear_error();
  if (!c) return fail(PD_ERR_ARG, "context is NULL");
  if (ncracks < 0 || (ncracks > 0 && !cracks)) return fail(PD_ERR_ARG, "bad crack list");
  PD_CUDA(cudaSetDevice(c->device));
  drop_graphs(c);
  const int64_t n = c->n, n_pad = c->n_pad;
  const int dim = c->dim;
  std::vector<CrackDev> hcr(ncracks);
  for (int k = 0; k < ncracks; ++k) {
    for (int t = 0; t < 3; ++t) {
      hcr[k].p[t] = cracks[k].p0[t];
      hcr[k].p[3 + t] = cracks[k].p1[t];
      hcr[k].p[6 + t] = cracks[k].p2[t];
    }
    for (double v : hcr[k].p)
      if (!std::isfinite(v)) return fail(PD_ERR_ARG, "non-finite crack coordinate");
    hcr[k].body = cracks[k].body;
    if (cracks[k].body >= c->nbodies) return fail(PD_ERR_ARG, "crack body index out of range");
  }

  // Per-body cell grids (edge = delta) and cell coordinates of every particle (internal order).
  std::vector<BodyGrid> grids(c->nbodies);
  std::vector<int4> cellc(n_pad);
  int64_t ncells = 0;
  std::vector<double> bodyA(c->nbodies), bodyW(c->nbodies);
  for (int b = 0; b < c->nbodies; ++b) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t u = c->body_off[b]; u < c->body_off[b + 1]; ++u) {
      const double p[3] = {c->hx[u], c->hy[u], dim == 3 ? c->hz[u] : 0.0};
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], p[k]);
        hi[k] = std::max(hi[k], p[k]);
      }
    }
    BodyGrid& g = grids[b];
    g.h = c->prm[b].horizon;
    g.delta2 = c->prm[b].horizon * c->prm[b].horizon;
    for (int k = 0; k < 3; ++k) {
      g.lo[k] = lo[k];
      double cells = std::floor((hi[k] - lo[k]) / g.h) + 1.0;
      if (k == 2 && dim == 2) cells = 1.0;
      if (cells > 2.0e6) return fail(PD_ERR_ARG, "horizon too small for the body extent");
      g.nc[k] = (int32_t)cells;
    }
    g.cell_off = ncells;
    ncells += (int64_t)g.nc[0] * g.nc[1] * g.nc[2];
    if (ncells > (int64_t)4e9) return fail(PD_ERR_ARG, "too many search cells");
    double A, K, G;
    material_constants(c->prm[b].model, c->prm[b].E, c->prm[b].nu, &A, &K, &G);
    bodyA[b] = A;
    bodyW[b] = c->prm[b].influence == PD_W_INV ? c->prm[b].horizon : 0.0;
  }
  std::vector<int64_t> cell_of(n);
  for (int64_t k = 0; k < n_pad; ++k) {
    if (k >= n) {
      cellc[k] = make_int4(0, 0, 0, c->body_of[k]);
      continue;
    }
    const int64_t u = c->perm[k];
    const int b = c->body_of[k];
    const BodyGrid& g = grids[b];
    const double p[3] = {c->hx[u], c->hy[u], dim == 3 ? c->hz[u] : 0.0};
    int cc[3];
    for (int t = 0; t < 3; ++t) {
      double f = std::floor((p[t] - g.lo[t]) / g.h);
      if (f < 0) f = 0;
      if (f > g.nc[t] - 1) f = g.nc[t] - 1;
      cc[t] = (int)f;
    }
    cellc[k] = make_int4(cc[0], cc[1], cc[2], b);
    cell_of[k] = g.cell_off + ((int64_t)cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
  }
  std::vector<int64_t> cell_start(ncells + 1, 0);
  for (int64_t k = 0; k < n; ++k) cell_start[cell_of[k] + 1]++;
  for (int64_t t = 0; t < ncells; ++t) cell_start[t + 1] += cell_start[t];
  std::vector<int32_t> cell_items(std::max<int64_t>(n, 1));
  {
    std::vector<int64_t> fill(cell_start.begin(), cell_start.end() - 1);
    for (int64_t k = 0; k < n; ++k) cell_items[fill[cell_of[k]]++] = (int32_t)k;
  }

  // Temporaries (released at the end of the build).
  int4* d_cellc = nullptr;
  BodyGrid* d_grids = nullptr;
  int64_t* d_cell_start = nullptr;
  int32_t* d_cell_items = nullptr;
  CrackDev* d_cracks = nullptr;
  double* d_bodyA = nullptr;
  double* d_bodyW = nullptr;
  double* d_m = nullptr;
  int32_t* d_width = nullptr;
  unsigned long long* d_keys = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_cellc);
    cudaFree(d_grids);
    cudaFree(d_cell_start);
    cudaFree(d_cell_items);
    cudaFree(d_cracks);
    cudaFree(d_bodyA);
    cudaFree(d_bodyW);
    cudaFree(d_m);
    cudaFree(d_width);
    cudaFree(d_keys);
  };
  auto tmp_alloc = [&](void** p, size_t bytes) -> pd_status {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      return fail(PD_ERR_OOM, "cudaMalloc of build temporaries failed");
    }
    return PD_OK;
  };
  // Arrays of a previous build are released first.
  free_build(c);
  c->built = false;
  pd_status st = PD_OK;
#define PD_TRY2(expr)    \
  do {                   \
    st = (expr);         \
    if (st != PD_OK) {   \
      cleanup();         \
      return st;         \
    }                    \
  } while (0)
  PD_TRY2(tmp_alloc((void**)&d_cellc, sizeof(int4) * n_pad));
  PD_TRY2(tmp_alloc((void**)&d_grids, sizeof(BodyGrid) * c->nbodies));
  PD_TRY2(tmp_alloc((void**)&d_cell_start, sizeof(int64_t) * (ncells + 1)));
  PD_TRY2(tmp_alloc((void**)&d_cell_items, sizeof(int32_t) * cell_items.size()));
  PD_TRY2(tmp_alloc((void**)&d_cracks, sizeof(CrackDev) * std::max(ncracks, 1)));
  PD_TRY2(tmp_alloc((void**)&d_bodyA, sizeof(double) * c->nbodies));
  PD_TRY2(tmp_alloc((void**)&d_bodyW, sizeof(double) * c->nbodies));
  PD_TRY2(tmp_alloc((void**)&d_m, sizeof(double) * n_pad));
  PD_TRY2(tmp_alloc((void**)&d_width, sizeof(int32_t) * c->nslices));
  PD_TRY2(alloc(c, &c->cnt, n_pad));
  PD_TRY2(alloc(c, &c->slice_ptr, c->nslices + 1));
  PD_TRY2(alloc(c, &c->mu, n_pad));
  PD_TRY2(alloc(c, &c->aA, n_pad));
  PD_TRY2(alloc(c, &c->dden, n_pad));
  {
    cudaStream_t s = c->stream;
    auto up = [&](void* dst, const void* src, size_t bytes) -> pd_status {
      if (bytes == 0) return PD_OK;
      cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
      return e == cudaSuccess ? PD_OK : cuda_fail(e, "cudaMemcpyAsync (build)");
    };
    PD_TRY2(up(d_cellc, cellc.data(), sizeof(int4) * n_pad));
    PD_TRY2(up(d_grids, grids.data(), sizeof(BodyGrid) * c->nbodies));
    PD_TRY2(up(d_cell_start, cell_start.data(), sizeof(int64_t) * (ncells + 1)));
    PD_TRY2(up(d_cell_items, cell_items.data(), sizeof(int32_t) * cell_items.size()));
    PD_TRY2(up(d_cracks, hcr.data(), sizeof(CrackDev) * ncracks));
    PD_TRY2(up(d_bodyA, bodyA.data(), sizeof(double) * c->nbodies));
    PD_TRY2(up(d_bodyW, bodyW.data(), sizeof(double) * c->nbodies));

    BuildArgs A{};
    A.n = n;
    A.n_pad = n_pad;
    A.pos = c->pos;
    A.cellc = d_cellc;
    A.grids = d_grids;
    A.cell_start = d_cell_start;
    A.cell_items = d_cell_items;
    A.cracks = d_cracks;
    A.ncracks = ncracks;
    A.cnt = c->cnt;
    A.body_A = d_bodyA;
    A.body_w = d_bodyW;
    A.m = d_m;
    A.mu = c->mu;
    A.aA = c->aA;
    A.dden = c->dden;
    const int tb = 128;
    const unsigned gb = (unsigned)((n_pad + tb - 1) / tb);
    if (dim == 3)
      k_family<3, false><<<gb, tb, 0, s>>>(A);
    else
      k_family<2, false><<<gb, tb, 0, s>>>(A);
    k_slice_width<<<(unsigned)((c->nslices + 127) / 128), 128, 0, s>>>(c->nslices, c->cnt, d_width);
    std::vector<int32_t> width(c->nslices);
    std::vector<int32_t> hcnt(n_pad);
    PD_CUDA(cudaMemcpyAsync(width.data(), d_width, sizeof(int32_t) * c->nslices, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaMemcpyAsync(hcnt.data(), c->cnt, sizeof(int32_t) * n_pad, cudaMemcpyDeviceToHost, s));
    PD_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> sptr(c->nslices + 1, 0);
    // slot counts rounded up to a multiple of 4: every slice's status words then start on a
    // 16-byte boundary, as the bulk copies of the staged kernels require
    for (int64_t t = 0; t < c->nslices; ++t) sptr[t + 1] = sptr[t] + 32 * (((int64_t)width[t] + 3) & ~3LL);
    c->nentries = sptr[c->nslices];
    c->nbonds = 0;
    for (int64_t k = 0; k < n; ++k) c->nbonds += hcnt[k];
    PD_TRY2(alloc(c, &c->col, (size_t)std::max<int64_t>(c->nentries, 32)));
    PD_TRY2(alloc(c, &c->bits, (size_t)std::max<int64_t>(c->nentries / 32, 1)));
    PD_TRY2(tmp_alloc((void**)&d_keys, sizeof(unsigned long long) * std::max<int64_t>(c->nentries, 32)));
    PD_TRY2(up(c->slice_ptr, sptr.data(), sizeof(int64_t) * (c->nslices + 1)));
    A.slice_ptr = c->slice_ptr;
    A.col = c->col;
    A.keys = d_keys;
    A.bits = c->bits;
    if (dim == 3) {
      k_family<3, true><<<gb, tb, 0, s>>>(A);
      k_init_bonds<3><<<gb, tb, 0, s>>>(A);
    } else {
      k_family<2, true><<<gb, tb, 0, s>>>(A);
      k_init_bonds<2><<<gb, tb, 0, s>>>(A);
    }
    PD_CUDA(cudaGetLastError());
    c->lattice = false;
    c->lat_f = nullptr;
    c->lat_rho = nullptr;
    c->lat_up = nullptr;
    c->lat_int = nullptr;
    c->lat_umax = nullptr;
    c->lat_wuni = 0;
    c->u32lo[0] = c->u32lo[1] = nullptr;
    c->shadow_lo = false;
    if (c->precision == PD_MIXED && c->lattice_opt) {
      PD_CUDA(cudaStreamSynchronize(s));
      bool lat = false;
      PD_TRY2(build_lattice(c, A, &lat));
    }
    c->pairs_ok = false;
    if (c->precision == PD_FP64 && c->nentries < (int64_t)INT32_MAX) {
      // pair tables of the FP64 path (entry indices fit in 32 bits)
      PD_TRY2(alloc(c, &c->own0, (size_t)n_pad));
      PD_TRY2(alloc(c, &c->twin, (size_t)std::max<int64_t>(c->nentries, 32)));
      A.own0 = c->own0;
      A.twin = c->twin;
      A.missing = c->counters + 7;
      PD_CUDA(cudaMemsetAsync(c->counters + 7, 0, sizeof(unsigned long long), s));
      k_twins<<<gb, tb, 0, s>>>(A);
      PD_CUDA(cudaGetLastError());
      unsigned long long missing = 0;
      PD_CUDA(cudaMemcpyAsync(&missing, c->counters + 7, sizeof(missing), cudaMemcpyDeviceToHost, s));
      PD_CUDA(cudaStreamSynchronize(s));
      c->pairs_ok = missing == 0;
    }
    PD_CUDA(cudaStreamSynchronize(s));
  }
  cleanup();
#undef PD_TRY2
  {
    pd_status st2 = alloc_state(c);
    if (st2 != PD_OK) return st2;
  }
  c->built = true;
  return ensure_shadow_lo(c);
}

}  // namespace pd
