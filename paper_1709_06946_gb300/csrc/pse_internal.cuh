// Internal declarations of the GB300 PSE library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
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
  double V() const { return L * L * L; }
  double sigma() const { return h * h * h; }
};

// Host-side parameter rules (Sec. 2.3.1 real-space cutoff, Eq. bound support size).
int choose_params(Params &p, const pse_options &opt, std::string &err);

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

// Small dense algebra on the host (FP64).
// Symmetric tridiagonal eigen-decomposition (implicit QL, Wilkinson shifts).
// d: diagonal (n), e: off-diagonal (n-1); on return d holds eigenvalues and
// Z (n x n, row-major, Z[i*n+k] = component i of eigenvector k).
bool tridiag_eigen(int n, std::vector<double> &d, std::vector<double> e, std::vector<double> &Z);

}  // namespace pse

// ---------------------------------------------------------------------------
// Device-side state of a handle.
struct pse_ctx {
  pse::Params p;
  int prec;                // pse_precision
  size_t ts;               // sizeof real type (4 or 8)
  pse_options opt;
  int lanczos_max, krylov_max;
  double lanczos_tol, krylov_tol;
  std::string err;
  int device = 0;
  int64_t dev_bytes = 0;
  std::vector<void *> allocs;

  // real-space table (device, real type), self terms
  void *d_table = nullptr;
  int table_len = 0, table_k2 = 0;
  double table_dr = 0, self_uf = 0, self_es = 0;

  // configuration state (sorted order = by spreading tile)
  double *d_posw = nullptr;     // wrapped positions, user order, N x 3
  int *d_tile_key = nullptr, *d_cell_key = nullptr;
  int *d_perm = nullptr, *d_inv = nullptr;   // sorted -> user, user -> sorted
  int *d_tile_start = nullptr, *d_tile_cur = nullptr;   // ntiles + 1
  int *d_cell_start = nullptr, *d_cell_cur = nullptr;   // ncells + 1
  int *d_cell_list = nullptr;
  int *d_nbr_start = nullptr;   // neighbour counts (N + 1 ints)
  int *d_nbr = nullptr;         // neighbour slots: particle i owns [i*nbr_slots, (i+1)*nbr_slots)
  int nbr_slots = 0;            // slots per particle
  int64_t nbr_cap = 0, npairs = 0;
  unsigned long long *d_nbr_tot = nullptr;  // total pairs and maximum count
  void *d_sp_i0 = nullptr;      // int4 per particle: wrapped support start
  void *d_sp_d0 = nullptr;      // real4: i0*h - x per dimension
  void *d_rs = nullptr;         // float4 (cell offset + packed cell) or double4_32a positions
  int *d_scan_tmp = nullptr;    // block sums for scans
  int64_t ntiles = 0, ncells = 0;
  int *d_flag = nullptr;        // device status word
  int *h_pinned_int = nullptr;  // host pinned scratch

  // grids
  void *d_grid = nullptr;       // 8 x Ng^3 real
  void *d_cgrid = nullptr;      // 8 x Ng^2 (Ng/2+1) complex
  void *d_fft_work = nullptr;
  cufftHandle plan_r2c[9] = {0}, plan_c2r[9] = {0};  // indexed by batch size
  bool plan_ok[9] = {false};

  // particle vectors, sorted order, [N][8] real
  void *d_v[6] = {nullptr};
  void *d_B = nullptr;          // Brownian velocities, user order [N][8]
  void *d_basis = nullptr;      // Krylov basis (max+1) x 8N
  double *d_dots = nullptr;     // partial / final dot products
  double *d_coef = nullptr;     // coefficient vectors for combinations
  double *h_dots = nullptr;     // pinned
  int dots_blocks = 0;

  double *d_pos0 = nullptr, *d_posh = nullptr;  // FP64 positions, user order
  void *d_stage[4] = {nullptr}; // staging for host arrays
  size_t stage_bytes[4] = {0};

  cudaStream_t side = nullptr;  // second stream for the real-space sum
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // profiling
  bool prof_on = false;
  double prof_ms[PSE_NSTAGES] = {0};
  int64_t prof_calls[PSE_NSTAGES] = {0};
  int64_t nlaunch = 0, nfft = 0;
  struct Pending { int stage; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_pool;
};

namespace pse {
cudaEvent_t prof_event(pse_ctx *c);
// Records events around one stage section on stream s while profiling is on.
struct StageTimer {
  pse_ctx *c;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageTimer(pse_ctx *c_, int stage_, cudaStream_t s_) : c(c_), stage(stage_), s(s_) {
    if (c->prof_on) {
      a = prof_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~StageTimer() {
    if (c->prof_on && a) {
      cudaEvent_t b = prof_event(c);
      cudaEventRecord(b, s);
      c->pending.push_back({stage, a, b});
      c->prof_calls[stage] += 1;
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
pse_status wave_apply(pse_ctx *c, const void *vin, void *vout, int mode, bool add, cudaStream_t s);
pse_status wave_noise(pse_ctx *c, const void *w2, uint64_t seed, uint64_t counter, void *vout,
                      cudaStream_t s);
// mode flags for real/wave products
enum { M_FULL = 0, M_SE = 1, M_FSU = 2 };
pse_status mobility(pse_ctx *c, const void *vin, void *vout, int mode, int parts, cudaStream_t s);

// vector helpers
pse_status gather_in(pse_ctx *c, const void *F, const void *S, void *vout, cudaStream_t s);
pse_status scatter_out(pse_ctx *c, const void *vin, void *U, void *E, double scale, cudaStream_t s);
pse_status gather_user8(pse_ctx *c, const void *user8, void *vout, cudaStream_t s);
pse_status scatter_user8(pse_ctx *c, const void *vin, void *user8, double scale, cudaStream_t s);
pse_status philox_w1(pse_ctx *c, uint64_t seed, uint64_t counter, void *vout, cudaStream_t s);
pse_status multidot(pse_ctx *c, const void *rows, int nrows, int64_t n, const void *w,
                    double *d_out, cudaStream_t s);
pse_status combine_sub(pse_ctx *c, void *w, const void *rows, int nrows, int64_t n,
                       const double *d_coef, cudaStream_t s);
pse_status combine_set(pse_ctx *c, void *y, const void *rows, int nrows, int64_t n,
                       const double *d_coef, cudaStream_t s);
pse_status vscale(pse_ctx *c, void *dst, const void *src, double a, int64_t n, cudaStream_t s);
pse_status vzero_slots(pse_ctx *c, void *v, int slot0, int nslot, cudaStream_t s);
pse_status midpoint(pse_ctx *c, const double *x0, const void *B_user, double fac, double *xout,
                    cudaStream_t s);
pse_status final_update(pse_ctx *c, const double *x0, const void *B_user, const void *U_sorted,
                        double dt, double *xout, cudaStream_t s);
pse_status check_finite(pse_ctx *c, const void *ptr, int64_t n, bool dbl, int *bad, cudaStream_t s);
}  // namespace pse
