/*
 * pse.h -- C ABI of the GB300 positively-split Ewald (PSE) library with
 * stresslet constraints (Fiore & Swan, arXiv:1709.06946).
 *
 * The library computes, for N identical spheres of radius a in a cubic
 * periodic box of side L (fluid viscosity eta, thermal energy kT):
 *
 *   [U; E] = M [F; S]            the periodic grand mobility restricted to
 *                                (velocity, rate of strain) x (force, stresslet)
 *                                (Sec. 2.1 Eqs. MUF-MDC, Sec. 2.2.1 rigid-particle
 *                                relation), split as M = M_r + M_w (Sec. 2.2) and
 *                                evaluated with a cell-list real-space sum
 *                                (Sec. 2.3.1) and a Gaussian NUFFT wave-space sum
 *                                (Sec. 2.3.2, Eq. WSops2);
 *   [U^B; E^B]                   Brownian slip velocities with covariance
 *                                (2 kT/dt) M (App. B), sampled as
 *                                M_r^{1/2} dW1 + M_w^{1/2} dW2 (Sec. 3, Eq. split)
 *                                with Lanczos for M_r^{1/2} (Sec. 3.2) and the
 *                                wave-space square root (Sec. 3.3, Eq. FFTsqrt);
 *   one constrained mid-point step (Sec. 3.4, App. B): x_{k+1/2} = x_k + dt/2 U^B,
 *                                M_ES S = -E^B - M_EF F^P at x_{k+1/2} (GMRES),
 *                                x_{k+1} = x_k + dt (U^B + M_UF F^P + M_US S).
 *
 * Conventions (all arrays dense, C order, little endian):
 *   pos   N x 3 float64, any real values (wrapped into [0, L) internally).
 *   F, U  N x 3, S, E  N x 5: the 5 stresslet / strain components in the
 *         orthonormal symmetric traceless basis
 *         Y1=(xx-yy)/sqrt2, Y2=(xx+yy-2zz)/sqrt6, Y3=(xy+yx)/sqrt2,
 *         Y4=(xz+zx)/sqrt2, Y5=(yz+zy)/sqrt2  (s_k = S:Y_k, e_k = E:Y_k),
 *         so every block of M is symmetric.
 *   Element type of F, S, U, E, noise arrays: float32 in PSE_MIXED,
 *         float64 in PSE_FP64 (positions are always float64).
 *   Pointers may be device or host memory (the library checks with
 *         cudaPointerGetAttributes and stages host arrays through its own
 *         device buffers).  The caller owns every array it passes; the library
 *         owns everything reachable from a handle.
 *   All work is issued on the given stream.  pse_mobility_apply returns
 *         without waiting; the sampling and step calls wait on the stream
 *         (the Krylov loops read their scalars on the host).
 *   Errors are returned as pse_status; pse_last_error gives a message.
 *   There is no CPU fallback: without a CUDA device every call that needs
 *         one returns PSE_ERR_CUDA.
 */
#ifndef PSE_H
#define PSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pse_ctx *pse_handle;
typedef void *pse_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  PSE_OK = 0,
  PSE_ERR_INVALID_ARG = 1,   /* bad size, parameter or pointer; nothing was done */
  PSE_ERR_OOM = 2,           /* device allocation failed */
  PSE_ERR_CUDA = 3,          /* CUDA / cuFFT error (message in pse_last_error) */
  PSE_ERR_NOT_CONVERGED = 4, /* Lanczos or GMRES hit its iteration cap; results of
                                the last iterate were still written */
  PSE_ERR_NONFINITE = 5,     /* NaN or Inf in the inputs; nothing was written */
  PSE_ERR_TIMEOUT = 6        /* reserved for bounded device-side waits */
} pse_status;

typedef enum {
  PSE_MIXED = 0, /* FP32 grids, FFTs, pair sums and vectors; FP64 Krylov/Lanczos
                    scalars (inner products, tridiagonal/Hessenberg algebra) */
  PSE_FP64 = 1   /* everything in FP64 (comparison form) */
} pse_precision;

typedef enum {
  PSE_RULE_STRICT = 0, /* r_cut = a + sqrt(ln(10/tol))/xi, support P from Eq. bound at
                          tol/10: measured error vs. the exact Ewald sum stays below tol */
  PSE_RULE_PAPER = 1   /* r_cut = sqrt(ln(1/tol))/xi, P from Eq. bound at tol with C = 1
                          (Table tab:lmax: P = 5 at 1e-3); error is a few x tol */
} pse_rule;

enum { PSE_PART_REAL = 1, PSE_PART_WAVE = 2, PSE_PART_ALL = 3 };

typedef struct pse_options {
  int32_t rule;            /* pse_rule (default PSE_RULE_STRICT) */
  int32_t Ng;              /* FFT grid points per side; 0 = rule (even, 2,3,5,7-smooth) */
  int32_t P;               /* Gaussian support points per side; 0 = rule */
  int32_t table_points;    /* real-space table points per 2a; 0 = default */
  double rcut;             /* real-space cutoff; 0 = rule (must be <= L/2) */
  double lanczos_tol;      /* < 0: use tol; 0: run exactly lanczos_maxiter steps */
  int32_t lanczos_maxiter; /* 0 = 100 */
  double krylov_tol;       /* GMRES |r|/|b| target; < 0: use tol */
  int32_t krylov_maxiter;  /* 0 = 50 */
  int32_t tile[3];         /* spreading/interpolation tile (x, y, z); 0 = auto */
  int32_t real_lanes;      /* lanes sharing one particle in the pair sum (1,4,8,16,32); 0 = auto */
  int32_t grid_ladder;     /* 1 (default): round the rule's grid up to an even 2^i 3^j size (a finer grid
                              only lowers the NUFFT error; cuFFT runs these sizes faster, and a batch then
                              has few distinct grids and few FFT groups); 0: the 2,3,5,7-smooth rule */
  int32_t use_graph;       /* 1: pse_constrained_step runs as one CUDA graph (captured on first use and
                              again when dt, the presence of a force or the layout changes), with the
                              Krylov loops as conditional while nodes; 0 = launches from the host */
  int32_t wave_kernel;     /* kernels for 16^3 tiles (mixed precision), bit mask.  0 (default): spreading
                              with the grid columns of a tile held in registers, interpolation with the
                              whole support region of a z-layer of a tile staged in shared memory (one
                              read-out per particle, no atomics).  Bit 0 set: spreading with the tile
                              in shared memory; bit 1 set: interpolation with the grid columns in
                              registers; bit 4 set: interpolation with the 16^3 tile in shared memory
                              (a support split over the tiles it meets); bit 2 set: in the register-column
                              spreading every warp scans the candidate particles itself (otherwise
                              the CTA scans them once and hands each warp its hit list); bit 3 set:
                              the 5-component spreading keeps a whole 16-point column per thread
                              (default: 8 z points, two z halves) */
  int32_t torque;          /* 1: also set up the 11-moment product pse_mobility_apply11 (forces,
                              torques and stresslets): 11 grids per suspension instead of 8, their
                              transforms, 12-slot work vectors and the rotation table */
  int32_t lambda_support;  /* deformed lattices only: 1 (default) = support size P from Eq. bound with
                              lambda_max of A^T A (Sec. 2.3.3); 0 = with lambda_max = 1, the orthorhombic
                              rule (the comparison of Fig. fig:shear; the NUFFT error then exceeds tol) */
  int32_t reserved[2];
  double deform[9];        /* deformation A of the periodic lattice, row-major (Sec. 2.3.3): the cell is
                              spanned by the columns of L A (simple shear: A = [[1, gamma, 0], [0, 1, 0],
                              [0, 0, 1]]; planar extension: diag(e, 1/e, 1)); det A > 0.  All zero (the
                              default) or the identity: the cubic box.  Every suspension of a handle
                              shares it.  See "Deformed lattices" before pse_create_batch. */
} pse_options;

typedef struct pse_info {
  int64_t N;
  double L, a, eta, kT, xi, tol;
  int32_t precision, rule;
  double rcut, kcut, h, eta_g, m;
  int32_t Ng, P;
  int32_t cells_per_side;
  int32_t tile[3];
  int32_t table_len;
  double table_dr;
  int64_t device_bytes;    /* bytes allocated on the device by this handle */
  int32_t deformed;        /* 1: the lattice is deformed (options.deform or pse_set_deformation) */
  int32_t tile_kernels;    /* 1: spreading and interpolation run the kernels specialised for 16^3 tiles
                              (mixed precision, P = 5, 6, 8 or 10, at least two tiles per side; on a
                              deformed lattice only with z orthogonal to the deformed plane) */
  double deform[9];        /* current deformation A (row-major; the identity for the cube) */
  double lambda_max;       /* largest eigenvalue of A^T A that the support size P was chosen for */
  double lambda_min_cells; /* smallest eigenvalue of A^T A that the cells and r_cut allow */
  double colnorm_max;      /* largest column norm of A that the grid resolves to k_cut */
} pse_info;

typedef struct pse_stats {
  int32_t lanczos_iters;
  int32_t krylov_iters;
  double lanczos_change;   /* last relative change |y_m - y_{m-1}|/|y_m| */
  double krylov_relres;    /* final |r|/|b| of the stresslet solve */
  int64_t neighbor_pairs;  /* ordered pairs in the last real-space list */
  int32_t products;        /* mobility products issued by the call */
  int32_t reserved[5];
} pse_stats;

/* Per-stage device-time profile (CUDA events recorded on the caller's stream
 * around each stage while profiling is enabled).  Stage indices: */
enum {
  PSE_STAGE_SETUP = 0,  /* wrap, sort by spreading tile, cell and neighbour lists */
  PSE_STAGE_REAL = 1,   /* real-space pair sum */
  PSE_STAGE_SPREAD = 2, /* Gaussian spreading */
  PSE_STAGE_FFT = 3,    /* cuFFT transforms (forward and inverse) */
  PSE_STAGE_SCALE = 4,  /* per-k scaling of the wave-space product */
  PSE_STAGE_INTERP = 5, /* Gaussian interpolation */
  PSE_STAGE_NOISE = 6,  /* wave-space noise generation and scaling */
  PSE_STAGE_VECTOR = 7, /* Krylov inner products, combinations, permutations, updates */
  PSE_NSTAGES = 8
};

/* Each stage's time is also split by product variant, so that one kernel
 * instance can be timed on its own: variant 0 = full product [F; S] -> [U; E]
 * (8 components; the wave-space noise interpolation counts here too), 1 = S -> E
 * (5 components), 2 = [F; S] -> U, 3 = S -> U.  The FFT stage uses the variant of
 * the product it transforms for; setup, noise and vector use variant 0. */
#define PSE_NVARIANTS 4

typedef struct pse_profile {
  double ms[PSE_NSTAGES];      /* accumulated device time per stage */
  int64_t calls[PSE_NSTAGES];  /* timed sections per stage */
  int64_t launches;            /* kernels of this library launched (cuFFT's excluded) */
  int64_t fft_execs;           /* cuFFT executions */
  double variant_ms[PSE_NSTAGES][PSE_NVARIANTS];      /* ms split by product variant */
  int64_t variant_calls[PSE_NSTAGES][PSE_NVARIANTS];  /* calls split by product variant */
} pse_profile;

/* Fills *opt with the defaults listed above. */
void pse_default_options(pse_options *opt);

/* Creates a handle for N particles.  Chooses r_cut, P, m = sqrt(pi P), the
 * grid Ng (k_cut from H(k_cut, xi) = tol, Ng >= k_cut L/pi) and the Gaussian
 * width eta_g = (h P xi / m)^2 < 1 (Sec. 2.3.2-2.3.3), builds the real-space
 * tables (inverse Fourier transform of M - M^(w), Sec. 2.2 / App. A), the
 * cuFFT plans and all device work space on the current device.
 * Returns INVALID_ARG for N < 1, L, a, eta, xi <= 0, kT < 0, tol outside
 * (0, 0.1], r_cut > L/2 or eta_g >= 1.  opt may be NULL (defaults). */
pse_status pse_create(pse_handle *out, int64_t N, double L, double a, double eta, double kT,
                      double xi, double tol, pse_precision prec, const pse_options *opt);

/* Deformed lattices (Sec. 2.3.3; Lees-Edwards shear, Kraynik-Reinelt extension).
 * With options.deform = A the periodic cell is spanned by the columns of L A
 * (volume V = L^3 det A).  Positions are Cartesian; internally each particle
 * has the lattice coordinate z = A^{-1} x wrapped into [0, L)^3, the FFT grid
 * nodes sit at h A n (h = L/Ng), a particle's support is the P^3 nodes nearest
 * z, its Gaussian weight is K(A d) for the lattice displacement d, the wave
 * vectors are (2 pi/L) A^{-T} m, and the real-space pairs are the lattice images
 * closer than r_cut.  Parameter rules on top of those of pse_create: P from
 * Eq. bound with lambda_max of A^T A (option lambda_support); Ng >= k_cut L c / pi
 * with c the largest column norm of A (every |k| <= k_cut on the grid); cells of
 * side >= r_cut / (2 sqrt(lambda_min)) in lattice coordinates and
 * r_cut <= L sqrt(lambda_min) / 2 (a pair closer than r_cut has one image).
 * Deformed handles run the general spreading / interpolation kernels (weights
 * evaluated per support point); positions written back by the step calls are
 * wrapped into the cell (A z with z in [0, L)^3). */

/* Creates one handle for nsys independent suspensions (no counterpart in the
 * paper, which treats one suspension: this is the batching layer).  Suspension s
 * has N[s] particles in a cubic box of side L[s]; a, eta, kT, xi and tol are
 * shared (so is the real-space table), and every suspension gets its own r_cut
 * check, grid, cells and tiles by the same rules as pse_create.  Every array
 * argument of the other calls is the concatenation of the suspensions' arrays
 * in suspension order (positions, forces, stresslets, velocities, w1), and w2
 * the concatenation of the suspensions' half-spectrum noise blocks.  Each stage
 * runs as one launch over all suspensions (one cuFFT plan per group of equal
 * grids); the Krylov iterations run in lockstep and a converged suspension drops
 * out.  Results equal those of separate handles up to rounding (the noise
 * indices are global: suspension s's Philox indices follow those of 0..s-1).
 * Errors name the suspension.  1 <= nsys <= 65536. */
pse_status pse_create_batch(pse_handle *out, int32_t nsys, const int64_t *N, const double *L, double a,
                            double eta, double kT, double xi, double tol, pse_precision prec,
                            const pse_options *opt);

/* Device bytes a handle with these arguments would allocate (an estimate that
 * bounds the real figure from above; no device memory is touched).  Same
 * argument checks as pse_create_batch. */
pse_status pse_estimate_bytes(int32_t nsys, const int64_t *N, const double *L, double a, double eta,
                              double kT, double xi, double tol, pse_precision prec,
                              const pse_options *opt, int64_t *bytes);

pse_status pse_destroy(pse_handle h);

/* For a batch handle: N is the total and the grid fields are suspension 0's. */
pse_status pse_get_info(pse_handle h, pse_info *out);

/* Changes the lattice deformation of a handle to A (row-major, det A > 0) for
 * the following calls, without new allocation: a Lees-Edwards run creates the
 * handle at its largest strain and sets the current one before each step.
 * Allowed when the handle's parameters still hold for A: lambda_max(A^T A) no
 * larger than the one P was chosen for, lambda_min(A^T A) no smaller than the
 * one the cells allow, the largest column norm of A no larger than the one the
 * grid resolves (the pse_info fields lambda_max, lambda_min_cells,
 * colnorm_max); else INVALID_ARG and nothing changes.  Only for handles created
 * with a deformation (options.deform not zero).  The device copy of the
 * parameters is updated in stream order on `stream`: work queued before the
 * call uses the old lattice, work queued after it the new one (a captured step
 * graph reads them at its next launch). */
pse_status pse_set_deformation(pse_handle h, const double *A, pse_stream stream);

/* Number of suspensions of a handle (0 for NULL). */
int32_t pse_num_systems(pse_handle h);

/* 1 if use_graph is on and the step graph has been captured (after a first
 * pse_constrained_step), else 0. */
int32_t pse_graph_ready(pse_handle h);

/* Why graph capture was given up for this handle (steps then launch from the
 * host), or "" if it was not. */
const char *pse_graph_error(pse_handle h);

/* Parameters of suspension s. */
pse_status pse_get_system_info(pse_handle h, int32_t s, pse_info *out);

/* Statistics of suspension s in the last sample or step call. */
pse_status pse_get_system_stats(pse_handle h, int32_t s, pse_stats *out);

/* [U; E] = M [F; S] at positions pos (Sec. 2.2 Eq. pairsums, rigid-particle
 * form).  F or S may be NULL (treated as zero); U or E may be NULL (not
 * written).  A NULL output or a NULL F selects a reduced product (E from S
 * alone, U from [F; S], U from S alone) with the same result for the outputs
 * asked for.  Asynchronous on stream. */
pse_status pse_mobility_apply(pse_handle h, const double *pos, const void *F, const void *S,
                              void *U, void *E, pse_stream stream);

/* As pse_mobility_apply, restricted to the real-space (PSE_PART_REAL) or
 * wave-space (PSE_PART_WAVE) part of the split, or both (PSE_PART_ALL). */
pse_status pse_mobility_apply_parts(pse_handle h, const double *pos, const void *F, const void *S,
                                    void *U, void *E, int32_t parts, pse_stream stream);

/* 11-moment product [U; Omega; E] = M [F; L; S] (Sec. 2.1 Eqs. MUF-MDC with the
 * torque of the rigid-particle relation, Sec. 2.2.1): the couplet of a particle
 * is sum_k L_k A_k + sum_k s_k Y_k with A_k = -eps_k../2 (A_k : A_l = delta/2),
 * the angular velocity is Omega_k = A_k : (grad u) = (curl u / 2)_k, so the
 * 11 x 11 blocks are symmetric; restricted to [U; E] x [F; S] it is
 * pse_mobility_apply.  The split and its sums are those of pse_mobility_apply
 * with 11 components: real space uses the tabulated free-space and Ewald-screened
 * rotation functions, wave space 11 grids.  Needs a handle created with
 * option torque = 1 (else PSE_ERR_INVALID_ARG).  F, L (N x 3) and S (N x 5)
 * may each be NULL (zero); U, Omega (N x 3) and E (N x 5) may each be NULL
 * (not written).  parts: PSE_PART_REAL, PSE_PART_WAVE or PSE_PART_ALL.
 * Element type as for pse_mobility_apply.  Single-suspension handles only.
 * Asynchronous on stream. */
pse_status pse_mobility_apply11(pse_handle h, const double *pos, const void *F, const void *L,
                                const void *S, void *U, void *Omega, void *E, int32_t parts,
                                pse_stream stream);

/* Brownian slip velocities [U^B; E^B] = sqrt(2 kT/dt) (M_r^{1/2} w1 + M_w^{1/2} dW2)
 * (Sec. 3 Eq. split, Sec. 3.2-3.3).  Noise is either external or drawn in-kernel:
 *   w1  N x 8 standard normals in the order [F_x F_y F_z s1..s5] per particle;
 *   w2  3 x Ng x Ng x (Ng/2+1) x 2 standard normals (component, z, y, x-half,
 *       re/im) of the R2C half spectrum; dW2 = (re + i im)/sqrt2, and on the
 *       kx = 0 plane the entry (z, y) with z > Ng/2 or (z = 0, y > Ng/2) is the
 *       conjugate of entry (-z, -y) mod Ng; k = 0 and Nyquist modes are unused.
 *   If w1 (w2) is NULL the library draws it with Philox4x32-10 (Salmon et al.
 *   2011): counter (index_lo, index_hi, counter, stream), key (seed_lo, seed_hi),
 *   Box-Muller on words 0 and 1; stream 1 = w1 (index = 8 n + c), stream 2 = w2
 *   (index over the half spectrum in the layout above; z0 = re, z1 = im).
 * UB: N x 3, EB: N x 5.  Waits on the stream (Lanczos scalars are read back). */
pse_status pse_brownian_sample(pse_handle h, const double *pos, double dt, uint64_t seed,
                               uint64_t counter, const void *w1, const void *w2, void *UB, void *EB,
                               pse_stats *stats, pse_stream stream);

/* One constrained mid-point step (Sec. 3.4 / App. B), positions updated in
 * place and wrapped into [0, L).  FP (N x 3, may be NULL) is the conservative
 * force evaluated at x_k; S_out (N x 5, may be NULL) receives the mid-point
 * stresslets; stats may be NULL.  Noise is drawn in-kernel from (seed, step).
 * Returns NOT_CONVERGED (after completing the step) if a Krylov cap was hit. */
pse_status pse_constrained_step(pse_handle h, double *pos, const void *FP, double dt, uint64_t seed,
                                uint64_t step, void *S_out, pse_stats *stats, pse_stream stream);

/* As pse_constrained_step with external noise arrays w1, w2 (layouts as in
 * pse_brownian_sample; both required). */
pse_status pse_constrained_step_noise(pse_handle h, double *pos, const void *FP, double dt,
                                      const void *w1, const void *w2, void *S_out, pse_stats *stats,
                                      pse_stream stream);

/* One Euler-Maruyama step with a random-finite-difference drift: the
 * alternative to the mid-point scheme that Sec. 3.4 discusses (three stresslet
 * solves per step instead of one).  With [U^B; E^B] drawn at x_k as in
 * pse_brownian_sample, the velocity U = U^B + M_UF F^P + M_US S with
 * M_ES S = -E^B - M_EF F^P (one solve at x_k, covariance (2kT/dt) R_FU^{-1} with
 * R_FU^{-1} = M_UF - M_US M_ES^{-1} M_EF, Eq. constrained_vel), and the drift
 * kT div R_FU^{-1} ~ (kT/delta) [R_FU^{-1}(x_k + delta/2 W) - R_FU^{-1}(x_k - delta/2 W)] W
 * with W a standard normal N x 3 vector (two more solves);
 * x_{k+1} = x_k + dt (U + drift), wrapped.  delta is a length (0: 1e-3 a).
 * pos is updated in place; FP (N x 3, may be NULL) is the conservative force at
 * x_k; S_out (N x 5, may be NULL) receives S of the solve at x_k.  Noise from
 * (seed, step): w1 and dW2 as pse_constrained_step, W from Philox stream 3 at
 * index 3 u + d.  stats->krylov_iters is the total over the three solves.
 * Single-suspension handles only (INVALID_ARG otherwise); launched from the
 * host; waits for its result.  Returns NOT_CONVERGED (after completing the
 * step) if a Krylov cap was hit. */
pse_status pse_rfd_step(pse_handle h, double *pos, const void *FP, double dt, double delta, uint64_t seed,
                        uint64_t step, void *S_out, pse_stats *stats, pse_stream stream);

/* As pse_rfd_step with external noise: w1, w2 as pse_brownian_sample and wt
 * (N x 3, user order, dtype of the handle's vectors) the direction W; all three
 * required. */
pse_status pse_rfd_step_noise(pse_handle h, double *pos, const void *FP, double dt, double delta, const void *w1,
                              const void *w2, const void *wt, void *S_out, pse_stats *stats, pse_stream stream);

/* Real-space part M_r [F; S] of the mobility product without any device
 * allocation.  No counterpart in the paper: this is a convenience for callers
 * that cannot allocate device memory -- host codes that must never make the
 * device wait inside their loop (cudaMalloc/cudaFree synchronise the device)
 * and applications whose device memory belongs to their own pool allocator.
 * Mixed precision only (F, S, U, E float32; pos float64), all five arrays must
 * be device memory (nothing is staged), F or S may be NULL (zero), U or E may be
 * NULL (not written).  Same physics as pse_mobility_apply_parts(PSE_PART_REAL)
 * with the default (strict) cutoff r_cut = a + sqrt(ln(10/tol))/xi, which must
 * not exceed L/2.  Limit: N <= 65536 (INVALID_ARG beyond it, or if r_cut/a
 * needs more than 16384 table rows).  Scratch is a fixed 1.3 MB static device
 * array held by every GPU that loads the library until exit; the first call on
 * a device looks up its address (call it once before any stream capture); the
 * call clears what must start at zero; calls that overlap on the GPU race on
 * the shared array.  Asynchronous on stream except when the table parameters
 * change (the new table is uploaded and the call waits for the copy); on a
 * stream that is being captured such a call returns INVALID_ARG without
 * touching the capture, so make one call with the same a, eta, xi and tol
 * before capturing.  Arrays must be device (or managed) memory of the current
 * device; device memory of another GPU is refused with INVALID_ARG. */
pse_status pse_mobility_real_noalloc(int64_t N, double L, double a, double eta, double xi, double tol,
                                     const double *pos, const float *F, const float *S, float *U, float *E,
                                     pse_stream stream);

/* Message for the last error of pse_mobility_real_noalloc on this thread. */
const char *pse_noalloc_last_error(void);

/* ------------------------------------------------------------------------
 * Serving loop (no counterpart in the paper).  A server owns `slots` worker
 * threads, each with its own CUDA stream on the current device.  Requests for
 * suspensions of any size arrive at any time and run concurrently on the
 * device; a request starts when a slot is free and its suspension's state fits
 * the device-memory budget.  State stays resident: a later request with the
 * same parameters (N, L, a, eta, kT, xi, tol, precision and options) reuses the handle
 * (tables, cuFFT plans, grids, neighbour lists); a new handle is created when
 * its estimate (pse_estimate_bytes) fits, after evicting idle resident handles,
 * least recently used first.  Requests that do not fit yet wait in arrival
 * order while later ones that fit go ahead.  A request whose estimate alone
 * exceeds the budget is rejected (OOM) at submission.
 * ------------------------------------------------------------------------ */
typedef struct pse_server pse_server;

enum { PSE_REQ_MOBILITY = 0, PSE_REQ_SAMPLE = 1, PSE_REQ_STEP = 2 };

typedef struct pse_request {
  int32_t kind;              /* PSE_REQ_* */
  int32_t precision;         /* pse_precision */
  int64_t N;
  double L, a, eta, kT, xi, tol;
  const pse_options *options; /* may be NULL (defaults); read at submission and at handle creation */
  double *pos;               /* N x 3 FP64 positions (host or device); updated in place by a step */
  const void *F, *S;         /* mobility: forces / stresslets; step: F = conservative force (may be NULL) */
  void *U, *E;               /* mobility: U, E; sample: U^B, E^B */
  void *S_out;               /* step: mid-point stresslets (may be NULL) */
  double dt;                 /* sample, step */
  uint64_t seed, counter;    /* sample: (seed, counter); step: (seed, step) */
  pse_stats *stats;          /* may be NULL */
} pse_request;

typedef struct pse_server_stats {
  int64_t completed, queued;
  int32_t running, peak_running;     /* requests on the device now / at most at once */
  double p50_ms, p99_ms;             /* latency, submission to completion */
  double wait_p50_ms, wait_p99_ms;   /* submission to start */
  double service_p50_ms;             /* start to completion */
  double requests_per_s;             /* completed / (first submission .. last completion) */
  int64_t resident_bytes, peak_resident_bytes;
  int32_t resident_handles;
  int64_t handles_created, handles_reused, handles_evicted, rejected;
} pse_server_stats;

/* 1 <= slots <= 64, budget_bytes > 0.  CUDA error if no device is present. */
pse_status pse_server_create(pse_server **out, int32_t slots, int64_t budget_bytes);

/* Queues a request (the arrays must stay valid until it completes); returns its ticket. */
pse_status pse_server_submit(pse_server *srv, const pse_request *req, uint64_t *ticket);

/* Waits at most timeout_ms for the request; TIMEOUT if it has not completed (it
 * stays queued or running and can be waited for again), else OK with the
 * request's own status in *result and its latency in *latency_ms. */
pse_status pse_server_wait(pse_server *srv, uint64_t ticket, double timeout_ms, pse_status *result,
                           double *latency_ms);

pse_status pse_server_get_stats(pse_server *srv, pse_server_stats *out);

/* Clears the latency record and counters (not the resident handles). */
pse_status pse_server_reset_stats(pse_server *srv);

/* Stops the workers after their current requests (queued ones are dropped) and
 * frees every resident handle. */
pse_status pse_server_destroy(pse_server *srv);

/* Pairwise hard-sphere repulsion as a harmonic overlap force (the paper's
 * hard-sphere repulsion is not specified; read here as this force):
 * F_i = sum_j k (2a - r_ij) (x_i - x_j)/r_ij over pairs closer than contact,
 * minimum image, into F (N x 3 in the handle's precision, user order).  Uses
 * the handle's cell and neighbour lists (r_cut >= 2a). */
pse_status pse_overlap_force(pse_handle h, const double *pos, double kspring, void *F, pse_stream stream);

/* Autotuner (no counterpart in the paper).  Times, on the configuration pos and
 * the handle's own stream, `reps` calls of each candidate: lanes per particle of
 * the pair sum (1, 4, 8, 16, 32; the S -> E plus the full product), then at the
 * chosen lanes the pair sum with its table staged in shared memory by one
 * 1024-thread CTA per SM (FP32, when the table fits), and spreading
 * tile caps (x, y, z) in {16,16,16}, {16,8,16}, {8,8,16}, {8,16,16}, {16,16,32},
 * {16,8,32}, {32,8,16} (the S -> E wave product; each suspension's tile is the
 * largest shape within the caps that divides its grid and fits shared memory),
 * and keeps the fastest of each.  Waits for the device.  The choice persists for
 * the handle's later calls; out (may be NULL) reports it and every timing. */
typedef struct pse_tuning {
  int32_t real_lanes;
  int32_t real_smem_table;    /* 1: the pair sum reads its table from shared memory (FP32, if it fits) */
  double real_smem_ms;        /* its time, when tried */
  int32_t tile[3];            /* chosen tile of suspension 0 */
  double best_real_ms, best_wave_ms;
  int32_t n_lanes, n_tiles;   /* candidates timed */
  double real_ms[8];          /* per lanes candidate 1, 4, 8, 16, 32 */
  int32_t tiles[8][3];        /* distinct tile candidates (suspension 0) */
  double wave_ms[8];
} pse_tuning;

pse_status pse_autotune(pse_handle h, const double *pos, int32_t reps, pse_tuning *out, pse_stream stream);

/* Enables (1) or disables (0) stage timing and resets the profile and the
 * launch counters.  Timing adds two event records per stage section. */
pse_status pse_set_profiling(pse_handle h, int32_t enable);

/* Waits for the recorded events and returns the accumulated profile. */
pse_status pse_get_profile(pse_handle h, pse_profile *out);

/* Name of a stage index ("setup", "real", ...), or "" when out of range. */
const char *pse_stage_name(int32_t stage);

/* Waits for all work of the handle and reports any pending CUDA error. */
pse_status pse_sync(pse_handle h);

const char *pse_status_string(pse_status s);

/* Message for the last error on this handle (or the last create failure if h is NULL). */
const char *pse_last_error(pse_handle h);

#ifdef __cplusplus
}
#endif
#endif /* PSE_H */
