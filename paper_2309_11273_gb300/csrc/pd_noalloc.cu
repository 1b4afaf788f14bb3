// pd_step_noalloc: one explicit time step on caller-owned device arrays, without allocating memory.
//
// Some callers cannot allocate device memory at all: code running inside a host framework whose
// allocator owns the whole device (a solver plug-in handed fixed buffers), real-time loops that
// must not enter the driver's allocator, or callers recording work into a stream while allocation
// is forbidden.  This entry point takes every input and output from the caller and keeps its only
// intermediate -- the per-particle pair (theta_i / m_i, 1 / m_i) passed from the dilatation kernel
// to the force kernel -- in a fixed file-scope device array of at most kMaxParticles entries.
//
// That array is one per GPU that loads the library and lives until the process exits.  Every call
// shares it and it keeps the last call's contents; the dilatation kernel overwrites every entry the
// force kernel reads, so nothing has to start at zero.  Calls whose kernels overlap on the GPU (two
// streams, two host threads) race on it: serialize them.
#include <cuda_runtime.h>

#include <mutex>

#include "pd_internal.h"

namespace pd {
namespace {

constexpr int64_t kMaxParticles = 1 << 20;  // 1,048,576 particles -> 16 MiB of scratch per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_step_scratch[kMaxParticles];

std::mutex g_setup_mutex;
double2* g_scratch_addr[kMaxDevices] = {nullptr};

// Host code may not take the address of a __device__ array directly (that is a host-side stand-in);
// the device address comes from the runtime, once per device, with that device current.
pd_status scratch_for_current_device(double2** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(PD_ERR_ARG, "device ordinal beyond the supported range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_step_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_addr[dev] = static_cast<double2*>(p);
  }
  *out = g_scratch_addr[dev];
  return PD_OK;
}

// Device (or managed) memory that the current device can address: a host array, or device memory
// of another GPU, would reach the kernels as an address they cannot use.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Byte ranges [p, p + bytes) of two arrays overlap.
bool overlap(const void* p, size_t pb, const void* q, size_t qb) {
  const uintptr_t a = (uintptr_t)p, b = (uintptr_t)q;
  return a < b + qb && b < a + pb;
}

struct NoAllocArgs {
  int64_t n;
  const double *x, *y, *z, *vol;
  const int64_t* row_ptr;
  const int32_t* col;
  const uint8_t* intact;
  const double *u, *v;
  double *u_out, *v_out, *theta;
  double A, Kp, G, inv_rho, dt;
  double2* scratch;
};

// m_i over the given family (Eq 1.9) and theta_i (Eq 1.6) over its intact bonds.
template <int DIM>
__global__ void k_noalloc_dilatation(NoAllocArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t n = a.n;
  double m = 0.0, s = 0.0;
  for (int64_t b = a.row_ptr[i]; b < a.row_ptr[i + 1]; ++b) {
    const int32_t j = a.col[b];
    const double ex = a.x[j] - a.x[i], ey = a.y[j] - a.y[i], ez = DIM == 3 ? a.z[j] - a.z[i] : 0.0;
    double q = ex * ex + ey * ey, d = ex * (a.u[j] - a.u[i]) + ey * (a.u[n + j] - a.u[n + i]);
    if (DIM == 3) {
      q = fma(ez, ez, q);
      d = fma(ez, a.u[2 * n + j] - a.u[2 * n + i], d);
    }
    m = fma(q, a.vol[j], m);
    if (!a.intact || a.intact[b]) s = fma(d, a.vol[j], s);
  }
  const double mu = m > 0.0 ? 1.0 / m : 0.0;
  const double th = a.A * mu * s;
  if (a.theta) a.theta[i] = th;
  a.scratch[i] = make_double2(a.Kp * (th * mu), a.G * mu);
}

// Eq 2.2 summed over the intact bonds, then Eq 2.11 with the diagonal mass rho V_i.
template <int DIM>
__global__ void k_noalloc_force_update(NoAllocArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t n = a.n;
  const double2 ti = a.scratch[i];
  double f[3] = {0.0, 0.0, 0.0};
  for (int64_t b = a.row_ptr[i]; b < a.row_ptr[i + 1]; ++b) {
    if (a.intact && !a.intact[b]) continue;
    const int32_t j = a.col[b];
    const double ex = a.x[j] - a.x[i], ey = a.y[j] - a.y[i], ez = DIM == 3 ? a.z[j] - a.z[i] : 0.0;
    double q = ex * ex + ey * ey, d = ex * (a.u[j] - a.u[i]) + ey * (a.u[n + j] - a.u[n + i]);
    if (DIM == 3) {
      q = fma(ez, ez, q);
      d = fma(ez, a.u[2 * n + j] - a.u[2 * n + i], d);
    }
    const double2 tj = a.scratch[j];
    // a coincident pair (q = 0) carries no bond direction: no force, as in the context path's tables
    const double c = fma(ti.y + tj.y, q > 0.0 ? d / q : 0.0, ti.x + tj.x) * a.vol[j];
    f[0] = fma(c, ex, f[0]);
    f[1] = fma(c, ey, f[1]);
    f[2] = fma(c, ez, f[2]);
  }
  for (int k = 0; k < DIM; ++k) {
    const double vk = a.v[k * n + i] + a.dt * (f[k] * a.inv_rho);
    a.v_out[k * n + i] = vk;
    a.u_out[k * n + i] = a.u[k * n + i] + a.dt * vk;
  }
}

}  // namespace
}  // namespace pd

extern "C" pd_status pd_step_noalloc(int32_t model, double E, double nu, double rho, double dt, int64_t n,
                                     const double* x_dev, const double* y_dev, const double* z_dev,
                                     const double* vol_dev, const int64_t* row_ptr_dev,
                                     const int32_t* col_dev, const uint8_t* intact_dev,
                                     const double* u_dev, const double* v_dev, double* u_out_dev,
                                     double* v_out_dev, double* theta_dev, void* stream) {
  using namespace pd;
  clear_error();
  if (model < 0 || model > 2) return fail(PD_ERR_ARG, "unknown model");
  if (!(E > 0) || !(nu > -1.0 && nu < 0.5) || !(rho > 0) || !(dt > 0))
    return fail(PD_ERR_ARG, "E, rho, dt must be > 0 and nu in (-1, 0.5)");
  if (n < 1) return fail(PD_ERR_ARG, "n must be >= 1");
  if (n > kMaxParticles)
    return fail(PD_ERR_ARG, "pd_step_noalloc handles at most 1048576 particles (fixed scratch); use the "
                            "context API for larger bodies");
  const int dim = model == PD_3D ? 3 : 2;
  if (!x_dev || !y_dev || (dim == 3) != (z_dev != nullptr) || !vol_dev || !row_ptr_dev || !col_dev || !u_dev ||
      !v_dev || !u_out_dev || !v_out_dev)
    return fail(PD_ERR_ARG, "a required device pointer is NULL (z must be given exactly for PD_3D)");
  int dev = -1;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess) return cuda_fail(e0, "cudaGetDevice");
  // every array the kernels touch must be addressable by the current device
  const size_t nb = (size_t)n * sizeof(double), vb = (size_t)dim * nb;
  const void* ptrs[] = {x_dev, y_dev, z_dev, vol_dev, row_ptr_dev, col_dev, intact_dev,
                        u_dev, v_dev, u_out_dev, v_out_dev, theta_dev};
  for (const void* p : ptrs)
    if (p && !on_device(p, dev))
      return fail(PD_ERR_ARG, "every array must be device (or managed) memory of the current device");
  // The kernels write u_out, v_out and theta while other threads still read u, v (and the rest):
  // no output may share a byte with an input of known length or with another output.  The lengths
  // of col and intact (row_ptr[n] entries) are not read on the host (that would synchronize), so for
  // those two only their first entry is checked against the outputs.
  {
    const size_t rp_b = (size_t)(n + 1) * sizeof(int64_t);
    struct Range {
      const void* p;
      size_t b;
    };
    const Range in[] = {{x_dev, nb}, {y_dev, nb}, {z_dev, z_dev ? nb : 0}, {vol_dev, nb}, {row_ptr_dev, rp_b},
                        {col_dev, sizeof(int32_t)}, {intact_dev, intact_dev ? 1 : 0}, {u_dev, vb}, {v_dev, vb}};
    const Range out[] = {{u_out_dev, vb}, {v_out_dev, vb}, {theta_dev, theta_dev ? nb : 0}};
    for (int o = 0; o < 3; ++o) {
      if (!out[o].p) continue;
      for (const Range& r : in)
        if (r.p && r.b && overlap(out[o].p, out[o].b, r.p, r.b))
          return fail(PD_ERR_ARG, "an output array overlaps an input array");
      for (int o2 = o + 1; o2 < 3; ++o2)
        if (out[o2].p && overlap(out[o].p, out[o].b, out[o2].p, out[o2].b))
          return fail(PD_ERR_ARG, "two output arrays overlap");
    }
  }
  double2* scratch = nullptr;
  pd_status st = scratch_for_current_device(&scratch);
  if (st != PD_OK) return st;
  NoAllocArgs a{};
  a.n = n;
  a.x = x_dev;
  a.y = y_dev;
  a.z = z_dev;
  a.vol = vol_dev;
  a.row_ptr = row_ptr_dev;
  a.col = col_dev;
  a.intact = intact_dev;
  a.u = u_dev;
  a.v = v_dev;
  a.u_out = u_out_dev;
  a.v_out = v_out_dev;
  a.theta = theta_dev;
  double K;
  material_constants(model, E, nu, &a.A, &K, &a.G);
  a.Kp = K - a.G / 3.0;
  a.inv_rho = 1.0 / rho;
  a.dt = dt;
  a.scratch = scratch;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int tb = 256;
  const unsigned grid = (unsigned)((n + tb - 1) / tb);
  if (dim == 3) {
    k_noalloc_dilatation<3><<<grid, tb, 0, s>>>(a);
    k_noalloc_force_update<3><<<grid, tb, 0, s>>>(a);
  } else {
    k_noalloc_dilatation<2><<<grid, tb, 0, s>>>(a);
    k_noalloc_force_update<2><<<grid, tb, 0, s>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pd_step_noalloc launch");
  return PD_OK;
}
