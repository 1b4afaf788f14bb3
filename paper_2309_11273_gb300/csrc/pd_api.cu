// extern "C" entry points of libosbpd (declared and documented in include/osbpd.h).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "pd_internal.h"

namespace pd {

static thread_local std::string g_err;

pd_status fail(pd_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

pd_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return PD_ERR_CUDA;
}

void clear_error() { g_err.clear(); }

void drop_graphs(pd_ctx* c) {
  for (auto& g : c->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

void free_build(pd_ctx* c) {
  drop_graphs(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (size_t k = c->n_create_allocs; k < c->allocs.size(); ++k) {
    cudaFree(c->allocs[k]);
    c->device_bytes -= (int64_t)c->alloc_bytes[k];
  }
  c->allocs.resize(std::min(c->allocs.size(), c->n_create_allocs));
  c->alloc_bytes.resize(c->allocs.size());
  c->cnt = nullptr;
  c->own0 = nullptr;
  c->twin = nullptr;
  c->dirty = nullptr;
  c->cA32 = nullptr;
  c->cu32 = nullptr;
  c->pairs_ok = false;
  c->slice_ptr = nullptr;
  c->col = nullptr;
  c->bits = nullptr;
  c->mu = c->aA = c->dden = c->theta = nullptr;
  c->thm = nullptr;
  c->disp[0] = c->disp[1] = nullptr;
  c->vel = c->bacc = c->gvec = nullptr;
  c->flag = nullptr;
  c->pos32 = nullptr;
  c->bA = nullptr;
  c->bB = nullptr;
  c->bd = nullptr;
  c->bS = nullptr;
  c->bs_stale = true;
  c->bE = nullptr;
  c->bt = nullptr;
  c->bY = nullptr;
  c->bX = nullptr;
  c->lam = nullptr;
  c->gnew = c->gold = nullptr;
  c->adr_part = nullptr;
  c->adr_st = nullptr;
  c->adr_first = nullptr;
  c->adr_restart = true;
  c->diag_theta = nullptr;
  c->diag_part = nullptr;
  c->u32[0] = c->u32[1] = nullptr;
  c->thm32 = nullptr;
  c->mu32 = c->aA32 = c->theta32 = nullptr;
  c->lattice = false;
  c->lat_f = nullptr;
  c->lat_rho = nullptr;
  c->lat_up = nullptr;
  c->lat_int = nullptr;
  c->lat_umax = nullptr;
  c->lat_wuni = 0;
}

void release(pd_ctx* c, void* p) {
  if (!p) return;
  for (size_t k = 0; k < c->allocs.size(); ++k) {
    if (c->allocs[k] != p) continue;
    cudaFree(p);
    c->device_bytes -= (int64_t)c->alloc_bytes[k];
    c->allocs.erase(c->allocs.begin() + k);
    c->alloc_bytes.erase(c->alloc_bytes.begin() + k);
    if (k < c->n_create_allocs) --c->n_create_allocs;
    return;
  }
}

void free_all(pd_ctx* c) {
  drop_graphs(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  c->alloc_bytes.clear();
  c->device_bytes = 0;
}

namespace {

// FP32 per-particle factors of the mixed path: 1/m_i and A/m_i * Q (the quantum folded in).
__global__ void k_init_mixed(int64_t n_pad, const double* __restrict__ mu, const double* __restrict__ aA,
                             double q, float* __restrict__ mu32, float* __restrict__ aA32,
                             float2* __restrict__ thm32, float* __restrict__ theta32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  mu32[i] = (float)mu[i];
  aA32[i] = (float)(aA[i] * q);
  thm32[i] = make_float2(0.0f, (float)mu[i]);
  theta32[i] = 0.0f;
}

__global__ void k_init_thm(int64_t n_pad, const double* __restrict__ mu, double2* __restrict__ thm) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  thm[i] = make_double2(0.0, mu[i]);
}

// The transfer stream of pd_get_state / pd_set_state, on the context's device.
pd_status ensure_xfer(pd_ctx* c) {
  if (c->xfer) return PD_OK;
  PD_CUDA(cudaStreamCreateWithFlags(&c->xfer, cudaStreamNonBlocking));
  cudaError_t e = cudaEventCreateWithFlags(&c->xfer_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaStreamDestroy(c->xfer);
    c->xfer = nullptr;
    c->xfer_ev = nullptr;
    return cuda_fail(e, "cudaEventCreateWithFlags");
  }
  return PD_OK;
}

pd_status check_ctx(pd_ctx* c, bool need_built) {
  clear_error();
  if (!c) return fail(PD_ERR_ARG, "context is NULL");
  if (need_built && !c->built) return fail(PD_ERR_STATE, "pd_build_neighbors has not been called");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return PD_OK;
}

bool all_finite(const double* a, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

}  // namespace

// State arrays (allocated after the family is built; zero state).
pd_status alloc_state(pd_ctx* c) {
  const int64_t np = c->n_pad;
  pd_status st;
  if ((st = alloc(c, &c->disp[0], np)) != PD_OK) return st;
  if ((st = alloc(c, &c->disp[1], np)) != PD_OK) return st;
  if ((st = alloc(c, &c->vel, np)) != PD_OK) return st;
  if ((st = alloc(c, &c->theta, np)) != PD_OK) return st;
  if ((st = alloc(c, &c->thm, np)) != PD_OK) return st;
  if ((st = alloc(c, &c->flag, np)) != PD_OK) return st;
  if ((st = alloc(c, &c->bacc, np)) != PD_OK) return st;
  if ((st = alloc(c, &c->gvec, np)) != PD_OK) return st;
  cudaStream_t s = c->stream;
  PD_CUDA(cudaMemsetAsync(c->disp[0], 0, sizeof(double4) * np, s));
  PD_CUDA(cudaMemsetAsync(c->disp[1], 0, sizeof(double4) * np, s));
  PD_CUDA(cudaMemsetAsync(c->vel, 0, sizeof(double4) * np, s));
  PD_CUDA(cudaMemsetAsync(c->theta, 0, sizeof(double) * np, s));
  PD_CUDA(cudaMemsetAsync(c->flag, 0, np, s));
  PD_CUDA(cudaMemsetAsync(c->bacc, 0, sizeof(double4) * np, s));
  PD_CUDA(cudaMemsetAsync(c->gvec, 0, sizeof(double4) * np, s));
  const int tb = 256;
  const unsigned gb = (unsigned)((np + tb - 1) / tb);
  k_init_thm<<<gb, tb, 0, s>>>(np, c->mu, c->thm);
  if ((st = init_disp_w(c)) != PD_OK) return st;
  if (c->precision == PD_MIXED) {
    if ((st = alloc(c, &c->pos32, np)) != PD_OK) return st;
    if ((st = alloc(c, &c->u32[0], np)) != PD_OK) return st;
    if ((st = alloc(c, &c->u32[1], np)) != PD_OK) return st;
    if ((st = alloc(c, &c->thm32, np)) != PD_OK) return st;
    if ((st = alloc(c, &c->mu32, np)) != PD_OK) return st;
    if ((st = alloc(c, &c->aA32, np)) != PD_OK) return st;
    if ((st = alloc(c, &c->theta32, np)) != PD_OK) return st;
    // fixed-point coordinates X = rint((x - lo) / Q) (Q a power of two), V as float bits
    std::vector<int4> hp(np);
    for (int64_t k = 0; k < np; ++k) {
      const int64_t u = c->perm[std::min<int64_t>(k, c->n - 1)];
      const double p[3] = {c->hx[u], c->hy[u], c->dim == 3 ? c->hz[u] : 0.0};
      int v[3];
      for (int t = 0; t < 3; ++t) v[t] = (int)std::llrint((p[t] - c->qlo[t]) / c->q);
      const float vol = k < c->n ? (float)c->hvol[u] : 1.0f;
      int vb;
      std::memcpy(&vb, &vol, sizeof(vb));
      hp[k] = make_int4(v[0], v[1], v[2], vb);
    }
    PD_CUDA(cudaMemcpyAsync(c->pos32, hp.data(), sizeof(int4) * np, cudaMemcpyHostToDevice, s));
    PD_CUDA(cudaMemsetAsync(c->u32[0], 0, sizeof(float4) * np, s));
    PD_CUDA(cudaMemsetAsync(c->u32[1], 0, sizeof(float4) * np, s));
    // theta = aA32 sum: Q folded in once (linearized: xi in quanta, u in metres) or twice (nonlinear:
    // both in quanta)
    k_init_mixed<<<gb, tb, 0, s>>>(np, c->mu, c->aA, c->kin == PD_NONLINEAR ? c->q * c->q : c->q, c->mu32,
                                   c->aA32, c->thm32, c->theta32);
    if ((st = prepare_staged_kernels(c)) != PD_OK) return st;
  }
  PD_CUDA(cudaGetLastError());
  PD_CUDA(cudaStreamSynchronize(s));
  c->cur = 0;
  c->has_flag = c->has_b = c->has_prescribed = false;
  c->check_pending = false;
  c->skip_next_check = true;
  return PD_OK;
}

}  // namespace pd

using namespace pd;

extern "C" {

const char* pd_last_error(void) { return g_err.c_str(); }

pd_status pd_material_constants(int32_t model, double E, double nu, double* A, double* K, double* G) {
  clear_error();
  if (model < 0 || model > 2 || !(E > 0) || !(nu > -1.0 && nu < 0.5)) return fail(PD_ERR_ARG, "bad model, E or nu");
  if (!A || !K || !G) return fail(PD_ERR_ARG, "A, K and G are required");
  material_constants(model, E, nu, A, K, G);
  return PD_OK;
}

double pd_critical_stretch(int32_t model, double E, double nu, double Gc, double delta) {
  if (model < 0 || model > 2 || !(E > 0) || !(nu > -1.0 && nu < 0.5) || !(Gc > 0) || !(delta > 0))
    return -1.0;
  const double kappa = E / (3.0 * (1.0 - 2.0 * nu));
  const double mu = E / (2.0 * (1.0 + nu));
  if (model == PD_3D) {
    const double beta = 125.0 * delta / 1848.0;  // Eq 1.27
    const double betap = 5.0 * delta / 24.0;     // Eq 1.25 integrated (Eq 1.27 prints an extra 1/pi)
    const double den = (9.0 * kappa - 15.0 * mu) * beta + 15.0 * mu * betap;
    return den > 0 ? std::sqrt(Gc / den) : -1.0;
  }
  const double pi = 3.14159265358979323846;
  double A, K, G;
  material_constants(model, E, nu, &A, &K, &G);
  const double r = (1.0 + nu) / (1.0 - 2.0 * nu);
  const double kp = model == PD_PLANE_STRESS ? kappa + mu / 9.0 * r * r : kappa + mu / 9.0;  // Eq 1.28
  const double beta = 1087.0 * delta / (1250.0 * pi * pi);  // Eq 1.29
  const double betap = 4.0 * delta / (5.0 * pi);
  const double den = A * A * (kp - 8.0 * mu / 9.0) * beta + 8.0 * mu * betap;
  return den > 0 ? std::sqrt(Gc / den) : -1.0;
}

pd_status pd_create_particles(pd_ctx** out, const pd_params* prm, int64_t n, const double* x,
                              const double* y, const double* z, const double* vol) {
  if (n < 1) {
    clear_error();
    return fail(PD_ERR_ARG, "n must be >= 1");
  }
  const int64_t off[2] = {0, n};
  return create(out, 1, prm, off, x, y, z, vol);
}

pd_status pd_create_batch(pd_ctx** out, int32_t nbodies, const pd_params* per_body,
                          const int64_t* body_offsets, const double* x, const double* y,
                          const double* z, const double* vol) {
  if (!body_offsets || body_offsets[0] != 0 || nbodies < 1) {
    clear_error();
    return fail(PD_ERR_ARG, "body_offsets must start at 0 and nbodies must be >= 1");
  }
  return create(out, nbodies, per_body, body_offsets, x, y, z, vol);
}

pd_status pd_build_neighbors(pd_ctx* c, const pd_crack* cracks, int32_t ncracks) {
  pd_status st = check_ctx(c, false);
  if (st != PD_OK) return st;
  st = build_neighbors(c, cracks, ncracks);
  if (st != PD_OK) return st;
  return upload_body_params(c);
}

pd_status pd_set_bc(pd_ctx* c, const uint8_t* flag, const double* b, const double* axis_point,
                    const double* axis_dir, double rate) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  const int64_t n = c->n;
  const int dim = c->dim;
  bool prescribed = false;
  if (flag) {
    for (int64_t i = 0; i < n; ++i) {
      if (flag[i] > 2) return fail(PD_ERR_ARG, "flag values must be 0, 1 or 2");
      prescribed |= flag[i] == 2;
    }
  }
  if (prescribed && (!axis_point || !axis_dir)) return fail(PD_ERR_ARG, "prescribed particles need an axis");
  if (!std::isfinite(rate)) return fail(PD_ERR_ARG, "rate must be finite");
  if (b && !all_finite(b, dim * n)) return fail(PD_ERR_ARG, "non-finite body force");
  drop_graphs(c);
  PD_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<uint8_t> hf(c->n_pad, 1);  // padding particles are fixed
  for (int64_t k = 0; k < n; ++k) hf[k] = flag ? flag[c->perm[k]] : 0;
  PD_CUDA(cudaMemcpyAsync(c->flag, hf.data(), c->n_pad, cudaMemcpyHostToDevice, c->stream));
  PD_CUDA(cudaStreamSynchronize(c->stream));
  c->has_flag = flag != nullptr;
  c->has_b = b != nullptr;
  c->has_prescribed = prescribed;
  if (b) {
    st = upload_field(c, b, c->bacc, dim);
    if (st != PD_OK) return st;
  }
  c->rate = prescribed ? rate : 0.0;
  if (prescribed) {
    for (int t = 0; t < 3; ++t) {
      c->bc_point[t] = axis_point[t];
      c->bc_dir[t] = axis_dir[t];
    }
    // g = a x (p - c) in caller order, then permuted on the device
    std::vector<double> g(3 * n);
    const double* a = axis_dir;
    for (int64_t i = 0; i < n; ++i) {
      const double r[3] = {c->hx[i] - axis_point[0], c->hy[i] - axis_point[1],
                           (dim == 3 ? c->hz[i] : 0.0) - axis_point[2]};
      g[i] = a[1] * r[2] - a[2] * r[1];
      g[n + i] = a[2] * r[0] - a[0] * r[2];
      g[2 * n + i] = a[0] * r[1] - a[1] * r[0];
    }
    st = upload_field(c, g.data(), c->gvec, 3);
    if (st != PD_OK) return st;
    PD_CUDA(cudaStreamSynchronize(c->stream));
  }
  st = upload_body_params(c);
  if (st != PD_OK) return st;
  st = apply_bc_now(c);
  if (st != PD_OK) return st;
  st = sync_shadow(c);
  if (st != PD_OK) return st;
  PD_CUDA(cudaStreamSynchronize(c->stream));
  return PD_OK;
}

pd_status pd_set_prescribed_velocity(pd_ctx* c, const double* vp) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if (!vp || !all_finite(vp, c->dim * c->n)) return fail(PD_ERR_ARG, "vp must be a finite dim * n array");
  if (!c->has_prescribed) return fail(PD_ERR_STATE, "no particle is prescribed (pd_set_bc flag 2)");
  drop_graphs(c);
  // u = rate t g with rate 1 and g = vp (the prescribed particles' rows of gvec)
  std::vector<double> g(3 * c->n, 0.0);
  for (int t = 0; t < c->dim; ++t)
    for (int64_t i = 0; i < c->n; ++i) g[(size_t)t * c->n + i] = vp[(size_t)t * c->n + i];
  if ((st = upload_field(c, g.data(), c->gvec, 3)) != PD_OK) return st;
  c->rate = 1.0;
  if ((st = upload_body_params(c)) != PD_OK) return st;
  if ((st = apply_bc_now(c)) != PD_OK) return st;
  if ((st = sync_shadow(c)) != PD_OK) return st;
  PD_CUDA(cudaStreamSynchronize(c->stream));
  return PD_OK;
}

pd_status pd_set_state(pd_ctx* c, const double* u, const double* v) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if (!u) return fail(PD_ERR_ARG, "u is required");
  if ((st = ensure_xfer(c)) != PD_OK) return st;
  const int dim = c->dim;
  // Both arrays are copied to the device and checked there (a host scan of 6n doubles costs more
  // than the copies); the state changes only once both are known to be finite.  The copies and
  // checks run on the transfer stream: they use only the staging buffers and one flag word, which
  // no main-stream work still in flight uses, so a failure check that pd_get_state left running
  // overlaps them; the state itself changes on the main stream, after that check.
  const int64_t nd = (int64_t)dim * c->n;
  unsigned long long* flag = c->counters + 6;
  cudaStream_t s = c->xfer;
  unsigned long long bad = 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(*flag), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->scratch, u, sizeof(double) * nd, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) st = launch_nonfinite(c->scratch, nd, flag, s);
  if (e == cudaSuccess && st == PD_OK && v) {
    e = cudaMemcpyAsync(c->scratch2, v, sizeof(double) * nd, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) st = launch_nonfinite(c->scratch2, nd, flag, s);
  }
  if (e == cudaSuccess && st == PD_OK) e = cudaMemcpyAsync(&bad, flag, sizeof(bad), cudaMemcpyDeviceToHost, s);
  const cudaError_t es = cudaStreamSynchronize(s);  // also on an error: nothing stays in flight
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return cuda_fail(e, "pd_set_state upload");
  if (st != PD_OK) return st;
  if (bad) return fail(PD_ERR_ARG, "non-finite state");
  if ((st = gather_field(c, c->scratch, c->disp[c->cur], dim)) != PD_OK) return st;
  if (v) {
    st = gather_field(c, c->scratch2, c->vel, dim);
  } else {
    PD_CUDA(cudaMemsetAsync(c->vel, 0, sizeof(double4) * c->n_pad, c->stream));
  }
  if (st != PD_OK) return st;
  st = apply_bc_now(c);
  if (st != PD_OK) return st;
  st = sync_shadow(c);
  if (st != PD_OK) return st;
  c->check_pending = false;
  c->skip_next_check = true;
  c->adr_restart = true;
  PD_CUDA(cudaStreamSynchronize(c->stream));
  return PD_OK;
}

pd_status pd_step(pd_ctx* c, int64_t nsteps) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if (nsteps < 0) return fail(PD_ERR_ARG, "nsteps must be >= 0");
  return run_steps(c, nsteps);
}

pd_status pd_sync(pd_ctx* c) {
  pd_status st = check_ctx(c, false);
  if (st != PD_OK) return st;
  PD_CUDA(cudaStreamSynchronize(c->stream));
  return c->built ? check_device_error(c) : PD_OK;
}

pd_status pd_get_damage(pd_ctx* c, double* phi) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if (!phi) return fail(PD_ERR_ARG, "phi is NULL");
  if ((st = launch_refresh_check(c)) != PD_OK) return st;
  if ((st = check_device_error(c)) != PD_OK) return st;
  if ((st = launch_damage(c, c->scratch)) != PD_OK) return st;
  PD_CUDA(cudaMemcpyAsync(phi, c->scratch, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaStreamSynchronize(c->stream));
  return PD_OK;
}

pd_status pd_get_state(pd_ctx* c, double* u, double* v, double* theta) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if ((st = check_device_error(c)) != PD_OK) return st;
  if ((st = ensure_xfer(c)) != PD_OK) return st;
  // u, v and theta do not depend on the bond status, so their copies run on the transfer stream,
  // after the work enqueued so far, while the pending failure check runs on the main stream (it
  // writes only bond status); the call returns once the copies are done.
  PD_CUDA(cudaEventRecord(c->xfer_ev, c->stream));
  PD_CUDA(cudaStreamWaitEvent(c->xfer, c->xfer_ev, 0));
  if (u) st = download_field(c, c->disp[c->cur], u, c->dim, c->xfer);
  if (st == PD_OK && v) st = download_field(c, c->vel, v, c->dim, c->xfer);
  if (st == PD_OK && theta) st = download_scalar(c, c->theta, theta, c->xfer);
  if (st == PD_OK) st = launch_refresh_check(c);
  const cudaError_t e = cudaStreamSynchronize(c->xfer);  // also on an error: nothing stays in flight
  if (st != PD_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  return PD_OK;
}

pd_status pd_num_bonds(pd_ctx* c, int64_t* nbonds) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if (!nbonds) return fail(PD_ERR_ARG, "nbonds is NULL");
  *nbonds = c->nbonds;
  return PD_OK;
}

pd_status pd_get_neighbors(pd_ctx* c, int64_t* row_ptr, int32_t* col, uint8_t* intact) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if (!row_ptr || !col) return fail(PD_ERR_ARG, "row_ptr and col are required");
  if ((st = launch_refresh_check(c)) != PD_OK) return st;
  std::vector<int64_t> sptr(c->nslices + 1);
  std::vector<int32_t> hcol(c->nentries);
  std::vector<uint32_t> hbits(c->nentries / 32);
  std::vector<int32_t> hcnt(c->n_pad);
  PD_CUDA(cudaMemcpyAsync(sptr.data(), c->slice_ptr, sizeof(int64_t) * sptr.size(), cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaMemcpyAsync(hcol.data(), c->col, sizeof(int32_t) * hcol.size(), cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaMemcpyAsync(hbits.data(), c->bits, sizeof(uint32_t) * hbits.size(), cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaMemcpyAsync(hcnt.data(), c->cnt, sizeof(int32_t) * hcnt.size(), cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaStreamSynchronize(c->stream));
  const int64_t n = c->n;
  std::vector<int64_t> inv(n);
  for (int64_t k = 0; k < n; ++k) inv[c->perm[k]] = k;
  row_ptr[0] = 0;
  for (int64_t u = 0; u < n; ++u) row_ptr[u + 1] = row_ptr[u] + hcnt[inv[u]];
  std::vector<std::pair<int32_t, uint8_t>> row;
  for (int64_t u = 0; u < n; ++u) {
    const int64_t k = inv[u];
    const int64_t s = k >> 5, lane = k & 31;
    row.clear();
    const int W = (int)((sptr[s + 1] - sptr[s]) >> 5);
    for (int t = 0; t < W; ++t) {  // a slot holds a bond unless it points at the particle itself
      const int64_t e = sptr[s] + 32 * (int64_t)t + lane;
      if (hcol[e] == (int32_t)k) continue;
      const uint8_t ok = (hbits[(sptr[s] >> 5) + t] >> lane) & 1u;
      row.emplace_back((int32_t)c->perm[hcol[e]], ok);
    }
    if ((int64_t)row.size() != hcnt[k]) return fail(PD_ERR_STATE, "neighbour layout does not match the family sizes");
    std::sort(row.begin(), row.end());
    for (size_t t = 0; t < row.size(); ++t) {
      col[row_ptr[u] + t] = row[t].first;
      if (intact) intact[row_ptr[u] + t] = row[t].second;
    }
  }
  return PD_OK;
}

pd_status pd_get_stats(pd_ctx* c, pd_stats* s) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if (!s) return fail(PD_ERR_ARG, "stats is NULL");
  if ((st = launch_refresh_check(c)) != PD_OK) return st;
  std::vector<uint32_t> hbits(c->nentries / 32);
  unsigned long long cnt[2];
  PD_CUDA(cudaMemcpyAsync(hbits.data(), c->bits, sizeof(uint32_t) * hbits.size(), cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaMemcpyAsync(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaStreamSynchronize(c->stream));
  int64_t intact = 0;
  for (uint32_t w : hbits) intact += __builtin_popcount(w);
  s->steps = c->steps;
  s->bonds = c->nbonds;
  s->broken_bonds = c->nbonds - intact;
  s->band_rechecks = (int64_t)cnt[0];
  s->validate_mismatches = (int64_t)cnt[1];
  int nonfinite = 0;
  double m = 0.0;
  if ((st = max_abs_u(c, &m, &nonfinite)) != PD_OK) return st;
  s->max_abs_u = nonfinite ? NAN : m;
  double kin = 0.0;
  if ((st = diagnostics(c, &s->min_rel_margin, &s->strain_energy, &kin)) != PD_OK) return st;
  s->shadow_energy = s->strain_energy + kin;
  return PD_OK;
}

pd_status pd_check_state(pd_ctx* c, double max_abs) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if (!(max_abs > 0)) return fail(PD_ERR_ARG, "max_abs_u must be > 0");
  int nonfinite = 0;
  double m = 0.0;
  if ((st = max_abs_u(c, &m, &nonfinite)) != PD_OK) return st;
  if (nonfinite) return fail(PD_ERR_NUMERIC, "non-finite displacement");
  if (m > max_abs) return fail(PD_ERR_NUMERIC, "displacement exceeds the divergence guard");
  return PD_OK;
}

pd_status pd_set_option(pd_ctx* c, int32_t option, int64_t value) {
  pd_status st = check_ctx(c, false);
  if (st != PD_OK) return st;
  switch (option) {
    case PD_OPT_GRAPH_CHUNK:
      if (value < 0 || value > 100000) return fail(PD_ERR_ARG, "graph chunk out of range");
      c->graph_chunk = (int)value;
      break;
    case PD_OPT_PROFILE:
      c->profile = value != 0;
      break;
    case PD_OPT_VALIDATE:
      c->validate = value != 0;
      break;
    case PD_OPT_BLOCK:
      if (value < 32 || value > 512 || value % 32) return fail(PD_ERR_ARG, "block must be a multiple of 32 in [32, 512]");
      if ((value / 32) % c->split) return fail(PD_ERR_ARG, "block warps must be a multiple of split");
      c->block = (int)value;
      break;
    case PD_OPT_SPLIT:
      if (value != 1 && value != 2 && value != 4) return fail(PD_ERR_ARG, "split must be 1, 2 or 4");
      if ((c->block / 32) % value) return fail(PD_ERR_ARG, "block warps must be a multiple of split");
      c->split = (int)value;
      break;
    case PD_OPT_BOND_CACHE:
      c->bond_cache = value != 0;
      break;
    case PD_OPT_STAGE:
      c->stage = value != 0;
      break;
    case PD_OPT_EXPIRE_WAITS:
      c->expire_waits = value != 0;
      break;
    case PD_OPT_LATTICE:
      c->lattice_opt = value != 0;  // read by the next pd_build_neighbors
      break;
    case PD_OPT_LAT_STAGE:
      if (value < 0 || value > 3) return fail(PD_ERR_ARG, "PD_OPT_LAT_STAGE must be 0, 1, 2 or 3");
      if (c->lat_stage != (int)value) drop_graphs(c);
      c->lat_stage = (int)value;
      break;
    case PD_OPT_SHADOW_LO:
      c->shadow_lo_opt = value != 0;
      if (c->built) {
        drop_graphs(c);
        const pd_status st = ensure_shadow_lo(c);
        if (st != PD_OK) return st;
      }
      break;
    case PD_OPT_PAIRS:
      // A failure check of the pair form marks slices whose bS its next pass 1b recomputes; the
      // other form never reads those marks, so a switch recomputes every bS before the next step.
      if ((value != 0) != (c->pairs != 0)) c->bs_stale = true;
      c->pairs = value != 0;
      break;
    case PD_OPT_SOLVER:
      if (value != PD_SOLVER_EXPLICIT && value != PD_SOLVER_ADR) return fail(PD_ERR_ARG, "unknown solver");
      if (value == PD_SOLVER_ADR && c->nbodies > 1)
        return fail(PD_ERR_ARG, "PD_SOLVER_ADR needs a single-body context (its damping is one Rayleigh quotient)");
      c->solver = (int)value;
      c->adr_restart = true;
      break;
    default:
      return fail(PD_ERR_ARG, "unknown option");
  }
  drop_graphs(c);
  return PD_OK;
}

pd_status pd_get_option(pd_ctx* c, int32_t option, int64_t* value) {
  pd_status st = check_ctx(c, false);
  if (st != PD_OK) return st;
  if (!value) return fail(PD_ERR_ARG, "value is NULL");
  switch (option) {
    case PD_OPT_GRAPH_CHUNK: *value = c->graph_chunk; break;
    case PD_OPT_PROFILE: *value = c->profile; break;
    case PD_OPT_VALIDATE: *value = c->validate; break;
    case PD_OPT_BLOCK: *value = c->block; break;
    case PD_OPT_SPLIT: *value = c->split; break;
    case PD_OPT_BOND_CACHE: *value = c->bond_cache; break;
    case PD_OPT_STAGE: *value = c->stage; break;
    case PD_OPT_EXPIRE_WAITS: *value = c->expire_waits; break;
    case PD_OPT_SOLVER: *value = c->solver; break;
    case PD_OPT_PAIRS: *value = (c->pairs && c->pairs_ok && c->precision == PD_FP64) ? 1 : 0; break;
    case PD_OPT_LATTICE: *value = c->built ? (c->lattice ? 1 : 0) : c->lattice_opt; break;
    case PD_OPT_LAT_STAGE: *value = c->lat_stage; break;
    case PD_OPT_SHADOW_LO: *value = c->built ? (c->shadow_lo ? 1 : 0) : c->shadow_lo_opt; break;
    default: return fail(PD_ERR_ARG, "unknown option");
  }
  return PD_OK;
}

pd_status pd_get_profile(pd_ctx* c, int32_t kernel, double* total_ms, int64_t* launches, int32_t reset) {
  pd_status st = check_ctx(c, false);
  if (st != PD_OK) return st;
  if (kernel < 0 || kernel >= PD_K_COUNT) return fail(PD_ERR_ARG, "unknown kernel id");
  if ((st = read_profile(c)) != PD_OK) return st;
  if (total_ms) *total_ms = c->times.ms[kernel];
  if (launches) *launches = c->times.launches[kernel];
  if (reset) {
    for (int k = 0; k < PD_K_COUNT; ++k) {
      c->times.ms[k] = 0;
      c->times.launches[k] = 0;
    }
  }
  return PD_OK;
}

namespace {

// The checkpoint's checksum and problem hash: the 64-bit FNV-1a scheme (Fowler, Noll and Vo) applied
// to 8-byte words (then to the trailing bytes), which hashes the gigabytes of a large family eight
// times faster than byte by byte.
constexpr uint64_t kFnvBasis = 14695981039346656037ull;
uint64_t fnv1a(uint64_t h, const void* p, size_t bytes) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  size_t k = 0;
  for (; k + 8 <= bytes; k += 8) {
    uint64_t w;
    std::memcpy(&w, b + k, 8);
    h ^= w;
    h *= 1099511628211ull;
  }
  for (; k < bytes; ++k) {
    h ^= b[k];
    h *= 1099511628211ull;
  }
  return h;
}

struct CheckpointHeader {
  char magic[8];  // "OSBPDCK1"
  uint32_t version;
  int32_t dim;
  int64_t n, n_pad, nentries, nbonds, steps;
  int32_t precision, kinematics, nbodies, flags;  // flags: 1 check pending, 2 skip next check
  uint64_t problem;  // hash of the parameters, positions and family
};
const char kCkptMagic[8] = {'O', 'S', 'B', 'P', 'D', 'C', 'K', '1'};

// Hash of everything that fixes the meaning of a state: sizes, per-body parameters (not the device
// or stream), and the device copies of the positions and of the built family.
pd_status problem_hash(pd_ctx* c, uint64_t* out) {
  uint64_t h = kFnvBasis;
  const int64_t sizes[4] = {c->n, c->n_pad, c->nentries, c->nbonds};
  h = fnv1a(h, sizes, sizeof(sizes));
  const int32_t kinds[3] = {c->dim, c->precision, c->kin};
  h = fnv1a(h, kinds, sizeof(kinds));
  for (const pd_params& p : c->prm) {
    const double v[8] = {p.E, p.nu, p.rho, p.horizon, p.s0, p.dt, p.band_safety, 0.0};
    const int32_t k[4] = {p.model, p.precision, p.ordering, p.kinematics};
    h = fnv1a(h, v, sizeof(v));
    h = fnv1a(h, k, sizeof(k));
  }
  std::vector<double4> pos(c->n_pad);
  std::vector<int32_t> col(c->nentries);
  PD_CUDA(cudaMemcpyAsync(pos.data(), c->pos, sizeof(double4) * c->n_pad, cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaMemcpyAsync(col.data(), c->col, sizeof(int32_t) * c->nentries, cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaStreamSynchronize(c->stream));
  h = fnv1a(h, pos.data(), sizeof(double4) * pos.size());
  h = fnv1a(h, col.data(), sizeof(int32_t) * col.size());
  *out = h;
  return PD_OK;
}

}  // namespace

pd_status pd_save_state(pd_ctx* c, const char* path) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if (!path) return fail(PD_ERR_ARG, "path is NULL");
  if ((st = check_device_error(c)) != PD_OK) return st;
  CheckpointHeader hd{};
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = 1;
  hd.dim = c->dim;
  hd.n = c->n;
  hd.n_pad = c->n_pad;
  hd.nentries = c->nentries;
  hd.nbonds = c->nbonds;
  hd.steps = c->steps;
  hd.precision = c->precision;
  hd.kinematics = c->kin;
  hd.nbodies = c->nbodies;
  hd.flags = (c->check_pending ? 1 : 0) | (c->skip_next_check ? 2 : 0);
  if ((st = problem_hash(c, &hd.problem)) != PD_OK) return st;
  const size_t nw = (size_t)std::max<int64_t>(c->nentries / 32, 1);
  std::vector<double4> u(c->n_pad), v(c->n_pad);
  std::vector<uint32_t> bits(nw);
  PD_CUDA(cudaMemcpyAsync(u.data(), c->disp[c->cur], sizeof(double4) * c->n_pad, cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaMemcpyAsync(v.data(), c->vel, sizeof(double4) * c->n_pad, cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaMemcpyAsync(bits.data(), c->bits, sizeof(uint32_t) * nw, cudaMemcpyDeviceToHost, c->stream));
  PD_CUDA(cudaStreamSynchronize(c->stream));
  uint64_t sum = kFnvBasis;
  sum = fnv1a(sum, &hd, sizeof(hd));
  sum = fnv1a(sum, u.data(), sizeof(double4) * u.size());
  sum = fnv1a(sum, v.data(), sizeof(double4) * v.size());
  sum = fnv1a(sum, bits.data(), sizeof(uint32_t) * bits.size());
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(PD_ERR_ARG, std::string("cannot open ") + path + " for writing");
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 && std::fwrite(u.data(), sizeof(double4), u.size(), f) == u.size() &&
            std::fwrite(v.data(), sizeof(double4), v.size(), f) == v.size() &&
            std::fwrite(bits.data(), sizeof(uint32_t), bits.size(), f) == bits.size() &&
            std::fwrite(&sum, sizeof(sum), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(PD_ERR_ARG, std::string("write to ") + path + " failed");
  return PD_OK;
}

pd_status pd_load_state(pd_ctx* c, const char* path) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if (!path) return fail(PD_ERR_ARG, "path is NULL");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(PD_ERR_ARG, std::string("cannot open ") + path);
  CheckpointHeader hd{};
  const size_t nw = (size_t)std::max<int64_t>(c->nentries / 32, 1);
  std::vector<double4> u(c->n_pad), v(c->n_pad);
  std::vector<uint32_t> bits(nw);
  uint64_t sum_file = 0;
  bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, kCkptMagic, 8) == 0 && hd.version == 1 &&
            hd.dim == c->dim && hd.n == c->n && hd.n_pad == c->n_pad && hd.nentries == c->nentries &&
            hd.nbonds == c->nbonds && hd.precision == c->precision && hd.kinematics == c->kin &&
            hd.nbodies == c->nbodies;
  if (ok)
    ok = std::fread(u.data(), sizeof(double4), u.size(), f) == u.size() &&
         std::fread(v.data(), sizeof(double4), v.size(), f) == v.size() &&
         std::fread(bits.data(), sizeof(uint32_t), bits.size(), f) == bits.size() &&
         std::fread(&sum_file, sizeof(sum_file), 1, f) == 1;
  std::fclose(f);
  if (!ok) return fail(PD_ERR_ARG, std::string(path) + " is not a checkpoint of this problem");
  uint64_t sum = kFnvBasis;
  sum = fnv1a(sum, &hd, sizeof(hd));
  sum = fnv1a(sum, u.data(), sizeof(double4) * u.size());
  sum = fnv1a(sum, v.data(), sizeof(double4) * v.size());
  sum = fnv1a(sum, bits.data(), sizeof(uint32_t) * bits.size());
  if (sum != sum_file) return fail(PD_ERR_ARG, std::string(path) + ": checksum mismatch");
  uint64_t problem = 0;
  if ((st = problem_hash(c, &problem)) != PD_OK) return st;
  if (problem != hd.problem)
    return fail(PD_ERR_ARG, std::string(path) + " was written for different particles, parameters or family");
  if ((st = check_device_error(c)) != PD_OK) return st;
  PD_CUDA(cudaMemcpyAsync(c->disp[c->cur], u.data(), sizeof(double4) * c->n_pad, cudaMemcpyHostToDevice, c->stream));
  PD_CUDA(cudaMemcpyAsync(c->vel, v.data(), sizeof(double4) * c->n_pad, cudaMemcpyHostToDevice, c->stream));
  PD_CUDA(cudaMemcpyAsync(c->bits, bits.data(), sizeof(uint32_t) * nw, cudaMemcpyHostToDevice, c->stream));
  if ((st = sync_shadow(c)) != PD_OK) return st;
  if (c->dirty) PD_CUDA(cudaMemsetAsync(c->dirty, 0, (size_t)c->nslices, c->stream));
  PD_CUDA(cudaStreamSynchronize(c->stream));
  c->steps = hd.steps;
  c->check_pending = (hd.flags & 1) != 0;
  c->skip_next_check = (hd.flags & 2) != 0;
  c->bs_stale = true;  // the loaded status bits
  c->adr_restart = true;
  drop_graphs(c);
  return PD_OK;
}

}  // extern "C"

namespace pd_probe {
// FP64 fused multiply-add throughput, registers only: 8 independent chains per thread, so that the
// FP64 pipe, not the dependency latency, sets the rate.  Iterates x <- x a + b with |a| < 1 (bounded).
__global__ void __launch_bounds__(256) k_probe_dfma(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (threadIdx.x + 1) * 1e-9 * (k + 1);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == -1.0) out[0] = s;  // never true: keeps the chains live without a store per thread
}
}  // namespace pd_probe

extern "C" {

pd_status pd_probe_fp64(int32_t device, int32_t repeats, double* flops_per_s, double* ms_per_launch) {
  clear_error();
  if (!flops_per_s || repeats < 1) return fail(PD_ERR_ARG, "flops_per_s is required and repeats must be >= 1");
  PD_CUDA(cudaSetDevice(device));
  int sms = 0;
  PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  double* out = nullptr;
  PD_CUDA(cudaMalloc(&out, sizeof(double)));
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int iters = 1 << 14, tb = 256;
  const unsigned grid = (unsigned)sms * 8;  // 2048 resident threads per SM
  float ms = 0.0f;
  if (e == cudaSuccess) {
    pd_probe::k_probe_dfma<<<grid, tb, 0, s>>>(out, 64, 0.999999, 1e-9);  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < repeats; ++r) pd_probe::k_probe_dfma<<<grid, tb, 0, s>>>(out, iters, 0.999999, 1e-9);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "FP64 probe");
  const double flops = 2.0 * 8.0 * iters * (double)grid * tb * repeats;
  *flops_per_s = flops / (ms * 1e-3);
  if (ms_per_launch) *ms_per_launch = ms / repeats;
  return PD_OK;
}

pd_status pd_get_info(pd_ctx* c, int64_t* n, int32_t* dim, int64_t* device_bytes) {
  pd_status st = check_ctx(c, false);
  if (st != PD_OK) return st;
  if (n) *n = c->n;
  if (dim) *dim = c->dim;
  if (device_bytes) *device_bytes = c->device_bytes;
  return PD_OK;
}

pd_status pd_autotune(pd_ctx* c, int32_t trial_steps, int32_t* block_out, int32_t* split_out) {
  pd_status st = check_ctx(c, true);
  if (st != PD_OK) return st;
  if (trial_steps < 1) return fail(PD_ERR_ARG, "trial_steps must be >= 1");
  cudaDeviceProp prop;
  PD_CUDA(cudaGetDeviceProperties(&prop, c->device));
  char key[512];
  std::snprintf(key, sizeof(key), "osbpd n=%lld bonds=%lld entries=%lld dim=%d prec=%d bodies=%d lattice=%d dev=%s",
                (long long)c->n, (long long)c->nbonds, (long long)c->nentries, c->dim, c->precision,
                c->nbodies, c->lattice ? 1 : 0, prop.name);
  for (char* p = key; *p; ++p)
    if (*p == '\n' || *p == '|') *p = ' ';
  const char* cache = std::getenv("PD_AUTOTUNE_CACHE");
  int best_block = -1, best_split = -1, best_pairs = -1, best_lat = -1;
  if (cache) {
    if (FILE* f = std::fopen(cache, "r")) {
      char line[700];
      while (std::fgets(line, sizeof(line), f)) {
        char* bar = std::strchr(line, '|');
        if (!bar) continue;
        *bar = 0;
        int b = 0, s = 0, pr = -1, rg = -1;
        if (std::strcmp(line, key) == 0 && std::sscanf(bar + 1, "%d %d %d %d", &b, &s, &pr, &rg) >= 2) {
          best_block = b;
          best_split = s;
          best_pairs = pr;
          best_lat = rg;
        }
      }
      std::fclose(f);
    }
  }
  if (best_block < 0) {
    // snapshot of everything a step modifies
    const int64_t np = c->n_pad;
    double4 *su = nullptr, *sv = nullptr, *sg = nullptr;
    uint32_t* sb = nullptr;
    float4* s32 = nullptr;
    const size_t nw = (size_t)std::max<int64_t>(c->nentries / 32, 1);
    if (cudaMalloc(&su, sizeof(double4) * np) != cudaSuccess || cudaMalloc(&sv, sizeof(double4) * np) != cudaSuccess ||
        cudaMalloc(&sb, sizeof(uint32_t) * nw) != cudaSuccess ||
        (c->precision == PD_MIXED && cudaMalloc(&s32, sizeof(float4) * np) != cudaSuccess) ||
        (c->gold && cudaMalloc(&sg, sizeof(double4) * np) != cudaSuccess)) {
      cudaGetLastError();
      cudaFree(su);
      cudaFree(sv);
      cudaFree(sb);
      cudaFree(s32);
      cudaFree(sg);
      return fail(PD_ERR_OOM, "autotune snapshot allocation failed");
    }
    double4* const gold0 = c->gold;  // ADR: previous force density (allocated at the first ADR step)
    const bool adr_restart0 = c->adr_restart;
    const int cur0 = c->cur;
    const int64_t steps0 = c->steps;
    const bool skip0 = c->skip_next_check, pend0 = c->check_pending;
    const int prof0 = c->profile, chunk0 = c->graph_chunk, block0 = c->block, split0 = c->split;
    cudaStream_t s = c->stream;
    PD_CUDA(cudaMemcpyAsync(su, c->disp[cur0], sizeof(double4) * np, cudaMemcpyDeviceToDevice, s));
    PD_CUDA(cudaMemcpyAsync(sv, c->vel, sizeof(double4) * np, cudaMemcpyDeviceToDevice, s));
    PD_CUDA(cudaMemcpyAsync(sb, c->bits, sizeof(uint32_t) * nw, cudaMemcpyDeviceToDevice, s));
    if (s32) PD_CUDA(cudaMemcpyAsync(s32, c->u32[cur0], sizeof(float4) * np, cudaMemcpyDeviceToDevice, s));
    if (sg) PD_CUDA(cudaMemcpyAsync(sg, gold0, sizeof(double4) * np, cudaMemcpyDeviceToDevice, s));
    auto restore = [&]() -> pd_status {
      c->cur = cur0;
      PD_CUDA(cudaMemcpyAsync(c->disp[cur0], su, sizeof(double4) * np, cudaMemcpyDeviceToDevice, s));
      PD_CUDA(cudaMemcpyAsync(c->vel, sv, sizeof(double4) * np, cudaMemcpyDeviceToDevice, s));
      PD_CUDA(cudaMemcpyAsync(c->bits, sb, sizeof(uint32_t) * nw, cudaMemcpyDeviceToDevice, s));
      if (s32) PD_CUDA(cudaMemcpyAsync(c->u32[cur0], s32, sizeof(float4) * np, cudaMemcpyDeviceToDevice, s));
      if (sg) PD_CUDA(cudaMemcpyAsync(gold0, sg, sizeof(double4) * np, cudaMemcpyDeviceToDevice, s));
      PD_CUDA(cudaStreamSynchronize(s));
      // an ADR run in progress continues from the restored v and g_prev; one that had not started
      // (or whose arrays were allocated by the trials) starts from rest
      c->adr_restart = adr_restart0 || !gold0;
      c->bs_stale = true;  // the restored status bits
      c->steps = steps0;
      c->skip_next_check = skip0;
      c->check_pending = pend0;
      // the two-word shadow from the restored displacements (the FP32 words are as saved)
      return (c->shadow_lo || c->lattice) ? sync_shadow(c) : PD_OK;  // lattice: the shadow's bound too
    };
    c->profile = 0;
    c->graph_chunk = 0;
    double best_ms = 1e300;
    const int blocks[] = {64, 128, 256, 512};
    const int splits[] = {1, 2, 4};
    // FP64 with the pair tables: the pair form (one more launch per step, fewer FP64 instructions)
    // against the single pass, which wins on small bodies where launches dominate
    const int pairs0 = c->pairs;
    const bool try_pairs = c->precision == PD_FP64 && c->pairs_ok && c->bond_cache;
    const int pair_opts[2] = {1, 0};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int stage0 = c->lat_stage;
    const int nrings = c->lattice ? 4 : 1;
    int best_ring = stage0;
    for (int bl : blocks) {
      for (int sp : splits) {
        if ((bl / 32) % sp) continue;
        if (c->lattice && sp != 1) continue;  // the lattice kernels run one warp per slice
        for (int po = 0; po < (try_pairs ? 2 : 1) * nrings; ++po) {
          c->block = bl;
          c->split = sp;
          c->pairs = try_pairs ? pair_opts[po] : pairs0;
          if (c->lattice) c->lat_stage = po;  // the staging ring of the lattice kernels
          if ((st = restore()) != PD_OK) break;
          run_steps(c, 1);  // warm-up
          cudaEventRecord(e0, s);
          st = run_steps(c, trial_steps);
          cudaEventRecord(e1, s);
          if (st != PD_OK) break;
          if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = cuda_fail(cudaGetLastError(), "autotune trial");
            break;
          }
          float ms = 0.0f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best_ms) {
            best_ms = ms;
            best_block = bl;
            best_split = sp;
            best_pairs = c->pairs;
            best_ring = c->lat_stage;
          }
        }
        if (st != PD_OK) break;
      }
      if (st != PD_OK) break;
    }
    c->pairs = pairs0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pd_status st2 = restore();
    cudaFree(sg);
    cudaFree(su);
    cudaFree(sv);
    cudaFree(sb);
    cudaFree(s32);
    c->profile = prof0;
    c->graph_chunk = chunk0;
    c->block = block0;
    c->split = split0;
    c->lat_stage = stage0;
    if (st != PD_OK) return st;
    if (st2 != PD_OK) return st2;
    best_lat = best_ring;
    if (cache && best_block > 0) {
      if (FILE* f = std::fopen(cache, "a")) {
        std::fprintf(f, "%s|%d %d %d %d\n", key, best_block, best_split, best_pairs, best_ring);
        std::fclose(f);
      }
    }
  }
  c->block = best_block;
  c->split = best_split;
  if (best_lat >= 0) c->lat_stage = best_lat;
  if (best_pairs >= 0) {
    if ((best_pairs != 0) != (c->pairs != 0)) c->bs_stale = true;  // as a PD_OPT_PAIRS switch
    c->pairs = best_pairs;
  }
  drop_graphs(c);
  if (block_out) *block_out = best_block;
  if (split_out) *split_out = best_split;
  return PD_OK;
}

void pd_destroy(pd_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  read_profile(c);
  if (c->xfer) cudaStreamSynchronize(c->xfer);
  free_all(c);
  if (c->xfer_ev) cudaEventDestroy(c->xfer_ev);
  if (c->xfer) cudaStreamDestroy(c->xfer);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
