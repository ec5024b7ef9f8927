// Internal declarations of the GB300 PSE library (not part of the C ABI).
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>
#include <cufft.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pse.h"

namespace pse {

// Physical and numerical parameters of one handle (host copy).
struct Params {
  int64_t N;
  double L, a, eta, kT, xi, tol;
  int rule;
  double rcut, kcut, h, eta_g, m;
  int Ng, P;
  int nkx;                 // Ng/2 + 1
  int nc;                  // real-space cells per side (cell side >= rcut)
  double cs;               // cell side
  int tile[3], ntile[3];   // spreading tile and tiles per side
  int ts;                  // bytes per real (4 mixed, 8 FP64)
  // lattice deformation (Sec. 2.3.3): the cell is spanned by the columns of L A
  int def = 0;             // 1: deformed lattice
  double A[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, Ai[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};  // row-major
  double detA = 1, lam_min = 1, lam_max = 1, cmax = 1;  // of the current A
  double lam_P = 1, lam_cells = 1, cmax_grid = 1;       // what P, the cells and the grid were chosen for
  double V() const { return L * L * L * detA; }
  double sigma() const { return h * h * h * detA; }
};

// Lattice quantities of a deformation A (row-major 3 x 3): inverse, determinant,
// extreme eigenvalues of A^T A and the largest column norm.  Returns 1 (with a
// message) unless det A > 0 and every entry is finite.
int lattice_of(const double A[9], double Ai[9], double &det, double &lam_min, double &lam_max, double &cmax,
               std::string &err);
// Sets p.A and its derived quantities (not the budgets lam_P, lam_cells, cmax_grid).
int set_lattice(Params &p, const double A[9], std::string &err);

// Host-side parameter rules (Sec. 2.3.1 real-space cutoff, Eq. bound support size).
int choose_params(Params &p, const pse_options &opt, std::string &err);
// Spreading tile within caps (fixed[d] > 0 overrides dimension d); sets tile and ntile.
int choose_tile(Params &p, const int caps[3], const int fixed[3], std::string &err);

// Real-space scalar functions tabulated on r = i * dr, i = 0 .. len-1 (dr divides 2a).
// Per node 8 values: fperp, fpar, gS, gR, kS, kX, kR, 0 (see tables.cpp for meaning).
struct RealTable {
  int len = 0;
  int k2 = 0;              // node index of r = 2a
  double dr = 0;
  double self_uf = 0;      // real-space self mobility (UF block, scalar x I)
  double self_es = 0;      // real-space self mobility (ES block, scalar x I_5)
  std::vector<double> v;   // len x 8
};
void build_real_table(const Params &p, int points_per_2a, RealTable &t);
// The same table rounded to FP32 into a caller buffer of len x 8 floats (no allocation).
void fill_real_table_f32(const Params &p, int points_per_2a, int len, float *out, double *self_uf,
                         double *self_es);
// Direct evaluation of the 7 functions at r > 0 (host, FP64); used for the table and tests.
void real_functions(const Params &p, double r, double out[7]);
// The three scalars of the rotation couplings of the 11-moment form at r > 0:
// out[0] = Phi_ab'/(2 eta) (Omega from F: out[0] rh x F; U from L: out[0] rh x L),
// out[1] = -(Phi_bb'' + Phi_bb'/r)/(4 eta), out[2] = (Phi_bb'' - Phi_bb'/r)/(4 eta)
// (Omega from L: out[1] L + out[2] (rh.L) rh; Omega from S: 2 out[2] (S rh) x rh;
// E from L: out[2] symY(rh x L, rh)).
void rot_functions(const Params &p, double r, double out[3]);
// Table of the rotation scalars, 4 reals per node (the three, then 0), len nodes of
// spacing 2a / points_per_2a from r = 0 (where the values are the r -> 0 limits:
// 0, the rotation self mobility U_bb^(5)(0)/(6 eta), 0).
void build_rot_table(const Params &p, int points_per_2a, int len, std::vector<double> &v, double *self_ol);

// Small dense algebra on the host (FP64).
// Symmetric tridiagonal eigen-decomposition (implicit QL, Wilkinson shifts).
// d: diagonal (n), e: off-diagonal (n-1); on return d holds eigenvalues and
// Z (n x n, row-major, Z[i*n+k] = component i of eigenvector k).
bool tridiag_eigen(int n, std::vector<double> &d, std::vector<double> e, std::vector<double> &Z);

}  // namespace pse

namespace pse {
// Per-suspension constants of a handle (device copy in pse_ctx::d_sys).  A
// handle holds nsys >= 1 independent suspensions; their particles, spreading
// tiles, cells, half-spectrum points and vector blocks are concatenated, and
// every kernel finds the suspension of its work item from the prefix tables
// (d_p0, d_tile0, d_k0, d_blk0).
struct SysDev {
  int64_t p0;              // first particle (same range in user and sorted order)
  int64_t nbr0;            // first neighbour slot
  int64_t k0;              // first half-spectrum point of the concatenated spectra
  int64_t grid0, gstride;  // real grid component c at grid0 + c * gstride (reals)
  int64_t cgrid0, cstride; // half spectrum component c at cgrid0 + c * cstride (complex)
  int N, Ng, nkx, nc, slots, tile0, cell0, blk0;
  int T[3], nt[3];
  int cubic;               // 1: mixed precision, P in {5, 6, 8}, 16^3 tiles, >= 2 tiles per side
  double L, h, cs;
  double inv_h, inv_cs;    // 1/h and 1/cs (binning without FP64 divisions)
  float Lf, csf;
  double alpha, pref;      // spreading Gaussian exp(-alpha r^2) and its prefactor
  double kfac, eta_g;      // 2 pi / L, Gaussian width
  double c_apply, c_noise; // sigma^2/(V eta) and sigma/sqrt(eta V)
  // deformed lattice (Sec. 2.3.3); def = 0 for the cube, where only qa is read
  int def;
  double A[9], Ai[9];      // deformation and its inverse, row-major (x = A z)
  double Bt[9];            // (2 pi / L) A^{-T}, row-major: wave vector k = Bt m
  float Af[9], Btf[9];
  double qa[6];            // Gaussian exponent alpha |A d|^2 = qa0 dx^2 + qa1 dy^2 + qa2 dz^2
                           //   + qa3 dx dy + qa4 dx dz + qa5 dy dz (cube: alpha, alpha, alpha, 0, 0, 0)
  // FP32 copies for the mixed-precision kernels, which then run no FP64
  // instruction per grid point or particle (FP64 issues at a small fraction of
  // the FP32 rate on sm_103a)
  float hf, alphaf, preff, kfacf, eta_gf, c_applyf, c_noisef;
  float qaf[6];
};

// Fills the lattice fields of d (def, A, Ai, Bt, qa, c_apply, c_noise and their FP32 copies) from p.
void fill_lattice(const Params &p, SysDev &d);

// Index s with start[s] <= x < start[s + 1] (start has n + 1 entries).
template <typename I>
__host__ __device__ __forceinline__ int find_sys(const I *start, int n, int64_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if ((int64_t)start[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One cuFFT group: the suspensions with the same grid size, whose grids are
// stored as [component][suspension][Ng^3] so that any leading set of
// components of the whole group is one strided batch.
struct FftGroup {
  int Ng = 0, nsys = 0;
  std::vector<int> members;           // suspensions of the group, in slot order
  int64_t grid0 = 0, cgrid0 = 0;
  cufftHandle r2c[12] = {0}, c2r[12] = {0};  // indexed by components per suspension
  bool ok[2][12] = {{false}};
};

constexpr int VEC_CHUNK = 16384;   // vector elements per block of the chunked vector kernels
constexpr int COEF_STRIDE = 512;   // doubles of Krylov coefficients per suspension
constexpr int MAX_ROWS = 128;      // Krylov vectors per dot-product / combination launch
constexpr int CUBE_TILE = 16;      // tile side of the specialised spreading / interpolation kernels
constexpr int SUB_SIDE = 4;        // sub-blocks per tile side in the sort key
constexpr int SUB_BLOCKS = SUB_SIDE * SUB_SIDE * SUB_SIDE;  // sub-blocks of a spreading tile
// Per-suspension coefficient block (COEF_STRIDE doubles): first and second
// Gram-Schmidt projections, |w|^2, a scale factor, the constants +1 and -1, and
// the coefficients of the final Krylov combination.
constexpr int CO_H1 = 0, CO_H2 = 128, CO_NRM = 256, CO_FAC = 257, CO_ONE = 258, CO_MONE = 259, CO_Y = 384;

// Device state of the per-suspension Krylov iterations; the control kernels
// (krylov_dev.cu) take the FP64 scalar steps of Lanczos (tridiagonal square
// root, stopping rule) and GMRES (Givens rotations, back substitution) on the
// device, so that an iteration needs no host round trip.
struct KDev {
  int nsys, lmax, gmax;
  double ltol, gtol;
  double *coef;
  int *active, *nrows, *iter, *flag;   // flag[0]: continue the loop
  double *l_alpha, *l_beta, *l_cprev, *l_c, *l_work, *l_b0, *l_err;
  int *l_it, *l_capped;
  double *g_H, *g_cs, *g_sn, *g_g, *g_beta, *g_rel;
  int *g_it, *g_capped;
};
}  // namespace pse

// ---------------------------------------------------------------------------
// Device-side state of a handle.
struct pse_ctx {
  pse::Params p;           // shared parameters; p.N = total particles (per-suspension values in ps)
  int n_cubic = 0;         // suspensions with SysDev::cubic set
  int lattice = 0;         // 1: created with a lattice deformation (options.deform): general spreading and
                           // interpolation kernels, Cartesian mapping in the neighbour search, lattice wrap
  int prec;                // pse_precision
  size_t ts;               // sizeof real type (4 or 8)
  pse_options opt;
  int lanczos_max, krylov_max;
  double lanczos_tol, krylov_tol;
  std::string err;
  int device = 0, nsm = 0;
  size_t smem_optin = 0;        // largest dynamic shared memory a 1024-thread pair-sum CTA may take
  int real_smem_table = 0;      // pair sum with the table staged in shared memory (autotuned)
  int64_t dev_bytes = 0;
  std::vector<void *> allocs;

  // suspensions
  int nsys = 1;
  std::vector<pse::Params> ps;     // per suspension (N, L, Ng, cells, tiles)
  std::vector<pse::SysDev> hs;     // host copy of d_sys
  pse::SysDev *d_sys = nullptr;
  int64_t *d_p0 = nullptr, *d_k0 = nullptr;  // nsys + 1 prefix tables
  int *d_tile0 = nullptr, *d_blk0 = nullptr; // nsys + 1 prefix tables
  int *d_active = nullptr;                   // per suspension: 1 = take part in the next kernels
  std::vector<int> h_active;
  std::vector<pse::FftGroup> groups;
  int64_t nk_tot = 0, nvblk = 0;             // half-spectrum points, vector blocks
  std::vector<pse_stats> sys_stats;          // per suspension, last call
  int *d_queue = nullptr;                    // work counters of the persistent kernels
  int queue_slot = 0;

  // real-space table (device, real type), self terms
  void *d_table = nullptr;
  // FP32 interval tables for the partial products: per interval q the values at
  // q and q + 1 of f4..f6 (S -> E) or of f0..f3 ([F; S] -> U), 8 floats each
  void *d_table_e = nullptr, *d_table_u = nullptr;
  int table_len = 0, table_k2 = 0;
  double table_dr = 0, self_uf = 0, self_es = 0;

  // configuration state (sorted order = by suspension, then spreading tile)
  double *d_posw = nullptr;     // wrapped positions, user order, N x 3
  int *d_tile_key = nullptr, *d_cell_key = nullptr;
  int *d_perm = nullptr, *d_inv = nullptr;   // sorted -> user, user -> sorted
  int *d_tile_start = nullptr, *d_tile_cur = nullptr;   // ntiles + 1
  int *d_fine_start = nullptr, *d_fine_cur = nullptr;   // ntiles * SUB_BLOCKS + 1 (sort by tile and sub-block)
  int *d_cell_start = nullptr, *d_cell_cur = nullptr;   // ncells + 1
  int *d_cell_list = nullptr;
  void *d_vcell = nullptr;     // the input vector of a real-space product in cell-list order (8N reals)
  void *d_rfd = nullptr;       // RFD step work space (4 x 8N reals, user order), allocated on first use
  // 11-moment product (option torque): rotation table (4 reals per node), 12-slot vectors
  void *d_table_rot = nullptr, *d_v12[2] = {nullptr, nullptr}, *d_vcell12 = nullptr;
  double self_ol = 0;
  void *d_rs_cell = nullptr;   // records of d_rs in cell-list order
  int *d_nbr_start = nullptr;   // neighbour counts (N + 1 ints)
  void *d_nbr_geo = nullptr;    // neighbour slots, particle i of suspension s owning nbr0 + (i - p0) slots ...:
                                // real4 (x_i - x_j, j) per neighbour, written by the list build
  int64_t nbr_cap = 0, npairs = 0, npairs_est = 0;  // last list's pairs; estimate from the densities
  std::vector<int64_t> npairs_sys;
  unsigned long long *d_nbr_tot = nullptr;  // per suspension: total pairs and maximum count
  unsigned long long *h_nbr_tot = nullptr;  // pinned copy
  void *d_sp_i0 = nullptr;      // int4 per particle: wrapped support start
  void *d_sp_d0 = nullptr;      // real4: i0*h - x per dimension
  void *d_rs = nullptr;         // float4 (cell offset + packed cell) or double4_32a positions
  int *d_scan_tmp = nullptr;    // block sums for scans
  int64_t ntiles = 0, ncells = 0;
  int64_t tile_cap = 0, scan_cap = 0;  // allocated tile-array and scan-scratch capacities
  int *d_flag = nullptr;        // device status word
  int *h_pinned_int = nullptr;  // host pinned scratch: 8 words, then active and row-count staging (2 x nsys)

  // grids
  void *d_grid = nullptr;       // real grids of all suspensions (FftGroup layout)
  void *d_cgrid = nullptr;      // half spectra, same layout
  void *d_fft_work = nullptr;
  int64_t grid_elems = 0, cgrid_elems = 0;

  // particle vectors, sorted order, [N][8] real
  void *d_v[6] = {nullptr};
  void *d_B = nullptr;          // Brownian velocities, user order [N][8]
  void *d_basis = nullptr;      // Krylov basis (max+1) x 8N
  double *d_dots = nullptr;     // per-block partial dot products
  double *d_coef = nullptr;     // per suspension COEF_STRIDE doubles: dots and combination coefficients
  double *h_dots = nullptr;     // pinned, nsys x COEF_STRIDE (device-to-host)
  double *h_wbuf = nullptr;     // pinned, nsys x COEF_STRIDE (host-to-device)
  bool h2d_pending = false;     // a host-to-device copy from pinned staging may still be queued

  double *d_pos0 = nullptr, *d_posh = nullptr;  // FP64 positions, user order
  void *d_stage[8] = {nullptr}; // staging for host arrays
  size_t stage_bytes[8] = {0};
  int *d_nrows = nullptr;       // per suspension: vectors in the final Krylov combination
  pse::KDev kd{};               // Krylov control state (device arrays)
  int *h_flag = nullptr;        // pinned copy of kd.flag and kd.active
  void *d_vin = nullptr;        // current Krylov vector, input of the products
  double *d_posout = nullptr;   // FP64 positions after a step (user order)
  bool capturing = false;       // a CUDA graph of the step is being captured
  cudaStream_t cap_stream = nullptr, g_stream = nullptr;  // capture streams of the loop bodies / the step
  cudaGraphExec_t g_exec = nullptr;
  cudaGraph_t g_graph = nullptr;
  double g_dt = 0;
  int g_force = -1, g_version = -1, layout_version = 0;
  uint64_t *d_rng = nullptr, *h_rng = nullptr;  // (seed, counter) read by the noise kernels in a graph
  std::string graph_error;      // why graph capture was given up, if it was

  // profiling
  bool prof_on = false;
  double prof_ms[PSE_NSTAGES] = {0};
  int64_t prof_calls[PSE_NSTAGES] = {0};
  double prof_vms[PSE_NSTAGES][PSE_NVARIANTS] = {{0}};
  int64_t prof_vcalls[PSE_NSTAGES][PSE_NVARIANTS] = {{0}};
  int64_t nlaunch = 0, nfft = 0;
  struct Pending { int stage, variant; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_pool;
};

namespace pse {
cudaEvent_t prof_event(pse_ctx *c);
// Records events around one stage section on stream s while profiling is on.
// Also opens an NVTX range named after the stage for the host-side extent of the
// section (visible to timeline tools; a no-op when none is attached).
// Scoped NVTX range around an entry point.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
inline const char *stage_range_name(int stage) {
  static const char *names[PSE_NSTAGES] = {"pse:setup", "pse:real", "pse:spread", "pse:fft",
                                           "pse:scale", "pse:interp", "pse:noise", "pse:vector"};
  return (stage >= 0 && stage < PSE_NSTAGES) ? names[stage] : "pse";
}
struct StageTimer {
  pse_ctx *c;
  int stage, variant;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageTimer(pse_ctx *c_, int stage_, cudaStream_t s_, int variant_ = 0)
      : c(c_), stage(stage_), variant(variant_), s(s_) {
    nvtxRangePushA(stage_range_name(stage));
    if (c->prof_on) {
      a = prof_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~StageTimer() {
    nvtxRangePop();
    if (c->prof_on && a) {
      cudaEvent_t b = prof_event(c);
      cudaEventRecord(b, s);
      c->pending.push_back({stage, variant, a, b});
      c->prof_calls[stage] += 1;
      c->prof_vcalls[stage][variant] += 1;
    }
  }
};
}  // namespace pse

#define PSE_CUDA_TRY(ctx, call)                                                          \
  do {                                                                                   \
    cudaError_t e__ = (call);                                                            \
    if (e__ != cudaSuccess) {                                                            \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e__);                  \
      return PSE_ERR_CUDA;                                                               \
    }                                                                                    \
  } while (0)

#define PSE_CUFFT_TRY(ctx, call)                                                         \
  do {                                                                                   \
    cufftResult r__ = (call);                                                            \
    if (r__ != CUFFT_SUCCESS) {                                                          \
      (ctx)->err = std::string(#call) + ": cufft error " + std::to_string((int)r__);     \
      return PSE_ERR_CUDA;                                                               \
    }                                                                                    \
  } while (0)

#define PSE_TRY(call)                   \
  do {                                  \
    pse_status s__ = (call);            \
    if (s__ != PSE_OK) return s__;      \
  } while (0)

// Kernel launchers (defined in the .cu files).
namespace pse {
struct Scan;
pse_status setup_config(pse_ctx *c, const double *d_pos, cudaStream_t s);
pse_status real_apply(pse_ctx *c, const void *vin, void *vout, int mode, cudaStream_t s);
// Harmonic overlap force of the current configuration into F (user order, N x 3).
pse_status overlap_force(pse_ctx *c, double kspring, void *F, cudaStream_t s);
pse_status wave_apply(pse_ctx *c, const void *vin, void *vout, int mode, bool add, cudaStream_t s);
// 11-moment product (option torque): 12-slot rows [F, L, S] -> [U, Omega, E], sorted order
pse_status wave_apply11(pse_ctx *c, const void *vin12, void *vout12, bool add, cudaStream_t s);
pse_status real_apply11(pse_ctx *c, const void *vin12, void *vout12, cudaStream_t s);
pse_status wave_noise(pse_ctx *c, const void *w2, uint64_t seed, uint64_t counter, void *vout,
                      cudaStream_t s);
// mode flags for real/wave products
// M_SU: S -> U (the final velocity when there is no external force)
enum { M_FULL = 0, M_SE = 1, M_FSU = 2, M_SU = 3 };
pse_status mobility(pse_ctx *c, const void *vin, void *vout, int mode, int parts, cudaStream_t s);

// vector helpers
pse_status gather_in(pse_ctx *c, const void *F, const void *S, void *vout, cudaStream_t s);
pse_status scatter_out(pse_ctx *c, const void *vin, void *U, void *E, double scale, cudaStream_t s);
pse_status gather_user8(pse_ctx *c, const void *user8, void *vout, cudaStream_t s);
pse_status scatter_user8(pse_ctx *c, const void *vin, void *user8, double scale, cudaStream_t s);
pse_status philox_w1(pse_ctx *c, uint64_t seed, uint64_t counter, void *vout, cudaStream_t s);
// Per-suspension Krylov helpers over [N][8] vectors; coefficients and results
// live at d_coef + s * COEF_STRIDE + off for suspension s, and suspensions
// with d_active[s] == 0 are skipped.
pse_status multidot(pse_ctx *c, const void *rows, int nrows, const void *w, int off, cudaStream_t s);
pse_status combine_sub(pse_ctx *c, void *w, const void *rows, int nrows, int off, cudaStream_t s);
pse_status combine_set(pse_ctx *c, void *y, const void *rows, const int *d_nrows, int maxrows, int off,
                       cudaStream_t s);
// dst = a * src (a uniform) or dst = coef[s][off] * src per suspension when off >= 0.
pse_status vscale(pse_ctx *c, void *dst, const void *src, double a, int off, cudaStream_t s);
pse_status vzero_slots(pse_ctx *c, void *v, int slot0, int nslot, cudaStream_t s);
pse_status midpoint(pse_ctx *c, const double *x0, const void *B_user, double fac, double *xout,
                    cudaStream_t s);
pse_status final_update(pse_ctx *c, const double *x0, const void *B_user, const void *U_sorted,
                        double dt, double *xout, cudaStream_t s);
pse_status check_finite(pse_ctx *c, const void *ptr, int64_t n, bool dbl, int *bad, cudaStream_t s);
pse_status rfd_noise(pse_ctx *c, const void *wt, uint64_t seed, uint64_t counter, void *W8, cudaStream_t s);
pse_status gather12(pse_ctx *c, const void *F, const void *L, const void *S, void *vout, cudaStream_t s);
pse_status scatter12(pse_ctx *c, const void *vin, void *U, void *Om, void *E, cudaStream_t s);
pse_status rfd_final(pse_ctx *c, const double *x0, const void *B, const void *U0, const void *Rp, const void *Rm,
                     double dt, double fac, double *xout, cudaStream_t s);
// Krylov control kernels (krylov_dev.cu); handle = 0 and graph = 0 outside a graph.
void kd_lz_start(pse_ctx *c, cudaStream_t s);
void kd_lz_step(pse_ctx *c, cudaStream_t s);
void kd_gm_start(pse_ctx *c, cudaStream_t s);
void kd_gm_step(pse_ctx *c, cudaStream_t s);
void kd_loop_begin(pse_ctx *c, cudaGraphConditionalHandle h, int graph, cudaStream_t s);
void kd_loop_end(pse_ctx *c, int cap, cudaGraphConditionalHandle h, int graph, cudaStream_t s);
void kd_all_active(pse_ctx *c, cudaStream_t s);
// Rows 0 .. *kd.iter + add - 1 of the basis: dot products into coef[s][off + r] and w -= sum coef rows.
pse_status multidot_rows(pse_ctx *c, const void *rows, int add, const void *w, int off, cudaStream_t s);
pse_status combine_sub_rows(pse_ctx *c, void *w, const void *rows, int add, int off, cudaStream_t s);
// Row *kd.iter + delta of the basis (and vin, if given) = coef[s][off] * src.
pse_status vscale_row(pse_ctx *c, void *basis, int delta, const void *src, void *vin, int off, cudaStream_t s);
// Work counter for the next persistent launch (cleared on stream s).
int *next_queue(pse_ctx *c, cudaStream_t s);
// Resident CTAs of a persistent kernel: SMs x blocks per SM (queried once into
// per_sm, 0 on entry), at most `items`.
template <typename K>
unsigned persistent_grid(pse_ctx *c, K kern, int threads, size_t smem, int64_t items, std::atomic<int> &per_sm) {
  int v = per_sm.load(std::memory_order_relaxed);
  if (v <= 0) {
    int q = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, kern, threads, smem) != cudaSuccess || q < 1) {
      cudaGetLastError();
      q = 1;
    }
    per_sm.store(q, std::memory_order_relaxed);
    v = q;
  }
  int64_t g = (int64_t)v * c->nsm;
  if (g > items) g = items;
  return (unsigned)(g < 1 ? 1 : g);
}
}  // namespace pse
