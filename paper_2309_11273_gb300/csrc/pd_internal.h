// Internal declarations shared by the translation units of libosbpd (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "osbpd.h"

namespace pd {

constexpr int kSlice = 32;  // particles per SELL slice (one warp)

// Per-body constants read by the step kernels (one entry per body; a single body otherwise).
struct BodyDev {
  double A;        // Eq 1.8
  double Kp;       // K - G/3 (Eqs 1.14, 2.2)
  double G;        // Eq 1.16
  double inv_rho;  // 1 / rho
  double dt;       // time step
  double s0;       // critical stretch (<= 0: no breaking)
  double s0nl;     // s0 (2 + s0): nonlinear break test |Y|^2 - |xi|^2 >= s0nl |xi|^2
  double rate;     // prescribed rotation rate
  double wdelta;   // influence function: 0 for w = 1, delta for w = delta / |xi| (Eq 1.9)
  float Kp32, G32, inv_rho32, sigma32;  // FP32 copies for the mixed path (sigma32 = s0 * Q)
  float G32q;      // G * Q (mixed path, nonlinear bonds)
  float s0nl32;    // s0 (2 + s0) in FP32 (mixed path, nonlinear bonds)
  double sigma_q;  // s0 * Q in double (Q = fixed-point quantum of the mixed coordinates)
  int32_t breaks;  // 1 if s0 > 0 (bond breaking on), else 0
  float xi1max;    // upper bound of |xi|_1 in quanta: sqrt(dim) (delta / Q + 2)
  float qmax;      // upper bound of |xi|^2 in quanta^2: (delta / Q + 2)^2
  // Lattice layout (mixed path, linearized bonds): bond vectors xi = h n with integer n, weighted
  // volumes m_i = V h^2 N_i with integer N_i, N_ref = the largest N_i of the body.  The FP32 sums run
  // in lattice units (u' = u / h) and are scaled back in FP64 by lat_C.
  double lat_h;       // lattice spacing h
  double lat_inv_h;   // 1 / h
  double lat_C;       // G / (h N_ref): F_i / V_i = lat_C * (FP32 force sum)
  double lat_K;       // lat_C dt / rho: the velocity update's factor of the FP32 force sum
  double lat_Kb;      // dt / rho: its factor of the body force density b
  float lat_lam_hi;   // lambda = (K - G/3) A / (G N_ref), split hi + lo (P_i = lambda sigma_i rho_i^2)
  float lat_lam_lo;
  float lat_s0;       // s0 in FP32
  // Rounding band of the FP32 break test g = n.(u'_j - u'_i) - s0 |n|^2 (see k_pass1_lat):
  // |g - g_FP64| <= Kf (U_i + U_j) + sq s0 |n|^2 + eps_c |g| + s0n1, U = |u'|_inf of each end.
  float lat_Kf;
  float lat_sq;
  float lat_eps_c;
  float lat_s0n1;
  // ... and the screen that settles most bonds: g < -(Kfast (U_i + U_j) + Kcfast) implies intact.
  float lat_Kfast;
  float lat_Kcfast;
  // lattice layout, nonlinear bonds: the FP32 break decision's band (pd_lattice.h, LatBandNL)
  float nl_A0, nl_A0s, nl_A1, nl_A1s, nl_A2, nl_Ag, nl_F0, nl_F0s, nl_F1, nl_F1s, nl_F2;
};

// Per-body neighbour-search grid (cells of edge >= delta).
struct BodyGrid {
  double lo[3];
  double h;
  double delta2;   // delta * delta
  int32_t nc[3];
  int32_t pad;
  int64_t cell_off;
};

// Crack (Section 4.2 / 4.4 pre-cracks and notches) as used by the build kernels.
struct CrackDev {
  double p[9];
  int32_t body;
  int32_t pad;
};

// Arguments shared by the step kernels.
struct StepArgs {
  int64_t n_pad;
  const int64_t* slice_ptr;
  const int32_t* col;
  uint32_t* bits;
  const double4* pos;      // x, y, z (0 in 2D), V
  const int32_t* body;     // nullptr: single body
  const BodyDev* bp;
  const double* aA;        // A / m_i
  const double* mu;        // 1 / m_i
  double* theta;           // theta_i (Eq 1.6)
  double2* thm;            // (theta_i / m_i, 1 / m_i) gathered by pass 2
  double4* vel;            // v (x, y, z, 0)
  const uint8_t* flag;     // nullptr: all free
  const double4* bacc;     // body force density b (x, y, z, 0) or nullptr
  const double4* gvec;     // a x (p - c) per particle (prescribed rotation) or nullptr
  int64_t* d_step;         // device step counter (index of the step being executed)
  // mixed path
  const int4* pos32;       // fixed-point coordinates (x, y, z) and V as float bits in .w
  float2* thm32;           // (theta_i / m_i, 1 / m_i) in FP32
  float* mu32;             // 1 / m_i in FP32
  float* aA32;             // A / m_i * Q in FP32 (Q folded in)
  float* theta32;          // theta_i in FP32
  unsigned long long* counters;  // [0] band rechecks, [1] validate mismatches, [2..3] max |u|, [4] wait expired,
                                 // [5] non-finite displacement after a pd_step, [6] non-finite pd_set_state input,
                                 // [7] pair entries missing at the build
  float band_c;            // safety factor of the band
  int validate;            // mixed: also decide every bond in FP64 and count mismatches
  int check;               // apply the failure criterion at the head of pass 1
  const double4* bA;       // tabled FP64 path: per slot (xi, s0 |xi|^2), or nullptr
  const double4* bB;       // tabled FP64 path: per slot (V_j xi, G (1/m_i + 1/m_j) / |xi|^2)
  double* bd;              // tabled FP64 path: per slot xi.(u_j - u_i), written by pass 1
  double4* bS;             // tabled FP64 path: per particle sum of V_j xi over the intact slots
  const int32_t* cnt;      // family size of each row
  const int32_t* own0;     // FP64 pair path (or nullptr): first owned slot of each row
  const int32_t* twin;     // FP64 pair path: per owned slot, the entry index of the same bond at j
  uint8_t* dirty;          // FP64 pair path: per slice, bS needs recomputing
  double2* bE;             // tabled nonlinear path: per slot (e, 1 / |Y|), written by pass 1 (bA = (xi, |xi|))
  double* bt;              // tabled nonlinear pair form: per slot V_j |xi| e, written by pass 1a
  double4* bY;             // tabled nonlinear pair form: per slot (Y/|Y|, e), written by pass 1a
  const double2* bX;       // tabled nonlinear pair form: per slot (|xi| V_j, V_j), built once
  int expire;              // testing (PD_OPT_EXPIRE_WAITS): staged kernels skip their first copy
  double uscale;           // mixed path: the FP32 shadow holds u * uscale (1, or 1/Q for nonlinear bonds)
  int adr;                 // PD_SOLVER_ADR: pass 2 stores g = f + b in gnew instead of updating
  double4* gnew;           // ADR: force density g^n of this iteration
  int lattice;             // mixed path: the lattice layout and its FP32 shadow u / h (with |u / h|_inf in .w)
  const float2* lat_f;     // lattice layout: per particle (rho_i = N_ref / N_i, A / N_i)
  const float* lat_rho;    // lattice layout: per particle N_ref / N_i (the pass-2 gather)
  float4* lat_up;          // lattice layout: per particle (u'_i, P_i), written by pass 1 for pass 2
  const uint8_t* lat_int;  // lattice layout: per slice, 1 if N_j = N_ref for its lanes and neighbours
  int lat_wuni;            // lattice layout: the common slice width, or 0 if the widths differ
  // lattice layout: per body, an upper bound of |u'|_inf over the current shadow (float bits; the
  // failure screen's neighbour term), and the same for the shadow the step writes (reset by pass 1,
  // raised by every kernel that writes that shadow)
  const unsigned* lat_umax;
  unsigned* lat_umax_next;
  int nbody;
};

struct KernelTimes {
  std::vector<cudaEvent_t> ev;  // pairs (start, stop) per launch
  std::vector<int> which;       // kernel id per pair
  double ms[PD_K_COUNT] = {};
  int64_t launches[PD_K_COUNT] = {};
  cudaEvent_t mid = nullptr;    // pair form: recorded between the two pass-1 kernels of a step
};

}  // namespace pd

struct pd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // Host transfers of pd_get_state / pd_set_state (created at first use).  Its work touches only
  // the scratch buffers, one flag word and state that the main stream's work in flight does not
  // write, and it is always synchronized before the call that used it returns.
  cudaStream_t xfer = nullptr;
  cudaEvent_t xfer_ev = nullptr;
  int dim = 3;
  int model = 0;
  int precision = 0;
  int kin = 0;                    // pd_kinematics
  int64_t n = 0, n_pad = 0, nslices = 0;
  int32_t nbodies = 1;
  std::vector<pd_params> prm;
  std::vector<int64_t> body_off;  // caller-order offsets of the bodies (nbodies + 1)
  std::vector<double> hx, hy, hz, hvol;   // caller order, host copies
  bool vol_uniform = false;               // every body has one particle volume (V_j = V_i on every bond)
  std::vector<int64_t> perm;              // internal k -> caller index (k < n)
  std::vector<int32_t> body_of;           // internal k -> body
  // device storage
  double4* pos = nullptr;
  int32_t* body = nullptr;
  pd::BodyDev* bp = nullptr;
  int64_t* slice_ptr = nullptr;
  int32_t* col = nullptr;
  uint32_t* bits = nullptr;
  int32_t* cnt = nullptr;
  int32_t* own0 = nullptr;       // FP64 pair path: first owned slot of each row
  int32_t* twin = nullptr;       // FP64 pair path: per owned slot, the entry of the same bond at j
  bool pairs_ok = false;         // the pair tables exist and every pair has both entries
  uint8_t* dirty = nullptr;      // FP64 pair path: per slice, a bond of the slice broke (bS to redo)
  float4* cA32 = nullptr;        // FP64 pair path, check before a read: per slot FP32 (xi, s0 |xi|^2 rounded down)
  float4* cu32 = nullptr;        // ... and its FP32 copy of u
  int64_t nentries = 0, nbonds = 0;
  double* mu = nullptr;
  double* aA = nullptr;
  double* dden = nullptr;
  double* theta = nullptr;
  double2* thm = nullptr;
  double4* disp[2] = {nullptr, nullptr};
  double4* vel = nullptr;
  uint8_t* flag = nullptr;
  double4* bacc = nullptr;
  double4* gvec = nullptr;
  int64_t* d_step = nullptr;
  int64_t* perm_dev = nullptr;   // internal -> caller (n)
  double* scratch = nullptr;     // n_pad * 3 doubles for transfers
  double* scratch2 = nullptr;    // a second n_pad * 3 (pd_set_state checks u and v before either lands)
  // mixed path
  int4* pos32 = nullptr;
  float4* u32[2] = {nullptr, nullptr};
  float4* u32lo[2] = {nullptr, nullptr};  // lattice layout, two-word shadow: the lo words of u32
  unsigned* lat_umax = nullptr;           // lattice layout: [2][nbodies] bounds of |u'|_inf per shadow buffer
  int shadow_lo_opt = 0;                  // PD_OPT_SHADOW_LO as set
  bool shadow_lo = false;                 // the lattice kernels run with the two-word shadow
  float2* thm32 = nullptr;
  float* mu32 = nullptr;
  float* aA32 = nullptr;
  float* theta32 = nullptr;
  unsigned long long* counters = nullptr;
  double4* bA = nullptr;          // FP64 per-slot table (xi, s0 |xi|^2)
  double4* bB = nullptr;          // FP64 per-slot table (V_j xi, G (1/m_i + 1/m_j) / |xi|^2)
  double* bd = nullptr;           // FP64 per-slot xi.du of the current step
  double4* bS = nullptr;          // FP64 per-particle sum of V_j xi over the intact slots
  bool bs_stale = true;           // bS no longer matches the status bits (recomputed before a step)
  double2* bE = nullptr;          // nonlinear FP64: per-slot (e, 1/|Y|) of the current step
  double* bt = nullptr;           // nonlinear FP64 pair form: per-slot theta term V_j |xi| e
  double4* bY = nullptr;          // nonlinear FP64 pair form: per-slot (Y/|Y|, e)
  double2* bX = nullptr;          // nonlinear FP64 pair form: per-slot (|xi| V_j, V_j)
  int bond_cache = 1;             // use the table in the FP64 path
  int pairs = 1;                  // FP64 tabled path: evaluate each bond once per pair (needs pairs_ok)
  int stage = 1;                  // mixed path: TMA-staged index streams (split 1)
  int expire_waits = 0;           // testing: make the staged kernels' first wait expire
  int solver = 0;                 // pd_solver
  bool adr_restart = true;        // next ADR iteration starts from rest
  double2* lam = nullptr;         // ADR fictitious density (lambda_i, 1 / lambda_i)
  double4* gnew = nullptr;        // ADR g^n (force density incl. body force)
  double4* gold = nullptr;        // ADR g^{n-1}
  double2* adr_part = nullptr;    // ADR per-block partial sums (u.k.u, u.u)
  double4* adr_st = nullptr;      // ADR (c^n, start flag, 1 / (2 + c^n)) of the current iteration
  int* adr_first = nullptr;       // ADR: 1 = the next iteration starts from rest
  double* diag_theta = nullptr;   // pd_get_stats: theta at the current state
  double4* diag_part = nullptr;   // pd_get_stats: per-block (strain energy, min margin, kinetic, 0)
  int lattice_opt = 1;            // PD_OPT_LATTICE: build the lattice layout when the bodies qualify
  int lat_stage = 0;              // PD_OPT_LAT_STAGE: staging ring of the lattice kernels (0..3)
  bool lattice = false;           // the built layout is the lattice layout (mixed, linearized bonds)
  float2* lat_f = nullptr;        // lattice layout: per particle (N_ref / N_i, A / N_i)
  float* lat_rho = nullptr;       // lattice layout: per particle N_ref / N_i
  float4* lat_up = nullptr;       // lattice layout: per particle (u'_i, P_i) from pass 1
  uint8_t* lat_int = nullptr;     // lattice layout: per slice, every N_j = N_ref around it
  int lat_wuni = 0;               // lattice layout: the common slice width (0: widths differ)
  std::vector<double> lat_h;      // lattice layout: spacing per body
  std::vector<double> lat_nref;   // lattice layout: N_ref per body
  std::vector<int> lat_n1;        // lattice layout: largest |n|_1 of the body's family
  std::vector<int> lat_qmax;      // lattice layout: largest |n|^2 of the body's family
  double q = 0.0;               // fixed-point quantum of the mixed coordinates [m]
  double qlo[3] = {0, 0, 0};     // origin of the fixed-point coordinates
  // state
  int cur = 0;
  int64_t steps = 0;
  bool built = false;
  bool check_pending = false;   // a step ran since the last failure check
  bool skip_next_check = true;  // first step after set_state / build: no check at its head
  bool has_flag = false, has_b = false, has_prescribed = false;
  double rate = 0.0;                      // prescribed rotation rate
  double bc_point[3] = {0, 0, 0}, bc_dir[3] = {0, 0, 0};
  // options
  int graph_chunk = 100;
  int profile = 0;
  int validate = 0;
  int block = 256;
  int split = 1;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  pd::KernelTimes times;
  int64_t device_bytes = 0;
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;
  size_t n_create_allocs = 0;  // allocations made at creation; later ones belong to the build
};

namespace pd {
// error reporting (thread-local message)
pd_status fail(pd_status st, const std::string& msg);
pd_status cuda_fail(cudaError_t e, const char* what);
void clear_error();
// device memory owned by the context
template <class T>
pd_status alloc(pd_ctx* c, T** p, size_t count);
void free_all(pd_ctx* c);
void release(pd_ctx* c, void* p);  // frees one allocation of the context (nullptr: nothing)
void free_build(pd_ctx* c);
void material_constants(int model, double E, double nu, double* A, double* K, double* G);
pd_status upload_body_params(pd_ctx* c);
pd_status create(pd_ctx** out, int32_t nbodies, const pd_params* prm, const int64_t* offsets,
                 const double* x, const double* y, const double* z, const double* vol);
pd_status build_neighbors(pd_ctx* c, const pd_crack* cracks, int32_t ncracks);
pd_status alloc_state(pd_ctx* c);
void drop_graphs(pd_ctx* c);
// launches (pd_step.cu)
pd_status launch_step(pd_ctx* c, bool check);
pd_status launch_refresh_check(pd_ctx* c);
pd_status launch_damage(pd_ctx* c, double* phi_caller);
pd_status launch_set_step(pd_ctx* c, int64_t value);
pd_status init_disp_w(pd_ctx* c);
pd_status ensure_bond_cache(pd_ctx* c);
pd_status ensure_adr(pd_ctx* c);      // ADR arrays and lambda (once per build)
pd_status diagnostics(pd_ctx* c, double* min_margin, double* strain, double* kinetic);
pd_status prepare_staged_kernels(pd_ctx* c);  // shared-memory opt-in of the staged kernels
pd_status upload_lattice_tables(int device);   // direction tables of the lattice kernels (once per device)
pd_status ensure_shadow_lo(pd_ctx* c);        // two-word shadow arrays and their contents (PD_OPT_SHADOW_LO)
pd_status upload_field(pd_ctx* c, const double* host_soa, double4* dst, int comps);
pd_status gather_field(pd_ctx* c, const double* dev_soa, double4* dst, int comps);
pd_status launch_nonfinite(const double* a, int64_t n, unsigned long long* flag, cudaStream_t s);
pd_status download_field(pd_ctx* c, const double4* src, double* host_soa, int comps, cudaStream_t s);
pd_status download_scalar(pd_ctx* c, const double* src, double* host, cudaStream_t s);
pd_status apply_bc_now(pd_ctx* c);
pd_status sync_shadow(pd_ctx* c);
pd_status max_abs_u(pd_ctx* c, double* out, int* nonfinite);
pd_status check_device_error(pd_ctx* c);
pd_status run_steps(pd_ctx* c, int64_t nsteps);
pd_status read_profile(pd_ctx* c);
}  // namespace pd

#define PD_CUDA(call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return pd::cuda_fail(e_, #call);  \
  } while (0)

template <class T>
pd_status pd::alloc(pd_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return pd::fail(PD_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  c->allocs.push_back(q);
  c->alloc_bytes.push_back(count * sizeof(T));
  c->device_bytes += (int64_t)(count * sizeof(T));
  *p = static_cast<T*>(q);
  return PD_OK;
}
