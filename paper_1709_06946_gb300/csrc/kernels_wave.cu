// Wave-space part of the split mobility (Sec. 2.3.2, Eq. WSops2) and the
// wave-space square root (Sec. 3.3, Eq. FFTsqrt):
//   spread (Q) -> R2C FFT -> per-k scaling (P^+ B P with the Gaussian
//   deconvolution) -> C2R FFT -> interpolate (sigma Q^T).
//
// A handle may hold several suspensions: their half spectra are concatenated
// (one thread per half-spectrum point of any suspension), and the transforms run
// as one batched cuFFT plan per group of suspensions with the same grid size.
//
// Spreading: a CTA owns one output tile of the grid at a time and accumulates it
// in shared memory; it visits the particles of the 2x2x2 bins whose Gaussian
// supports can reach the tile (bins hold particles by the grid index where their
// support starts), so every grid value is written exactly once with coalesced
// stores and no global atomics or zeroing pass.  Interpolation mirrors it: the
// CTA stages its tile in shared memory, each visiting particle sums its
// in-tile support, and the partial sums are added to the particle outputs.
// The Gaussian K(r) = (2 xi^2/(pi eta_g))^{3/2} exp(-2 xi^2 r^2/eta_g) is
// evaluated separably (3P exponentials per particle visit, not P^3).
#include <cmath>

#include "wave_common.cuh"

namespace pse {
namespace {

// Launch-wide arguments of the per-k kernels; per-suspension values come from SysDev.
struct ScaleArgs {
  int nsys;
  int64_t nk_tot;
  double a, q4;
  float af, q4f;       // FP32 copies for the mixed-precision kernels
  const SysDev *sys;
  const int64_t *k0;   // nsys + 1 prefix of half-spectrum points
  const int *active;
};

// Per-suspension constants in the arithmetic type of the kernel: the FP32 form
// reads the FP32 copies, so no FP64 conversion runs per half-spectrum point.
template <typename T>
__device__ __forceinline__ T sa_a(const ScaleArgs &sa) {
  if constexpr (sizeof(T) == 4) return sa.af;
  else return sa.a;
}
template <typename T>
__device__ __forceinline__ T sa_q4(const ScaleArgs &sa) {
  if constexpr (sizeof(T) == 4) return sa.q4f;
  else return sa.q4;
}
template <typename T>
__device__ __forceinline__ T sd_c_apply(const SysDev &s) {
  if constexpr (sizeof(T) == 4) return s.c_applyf;
  else return s.c_apply;
}
template <typename T>
__device__ __forceinline__ T sd_c_noise(const SysDev &s) {
  if constexpr (sizeof(T) == 4) return s.c_noisef;
  else return s.c_noise;
}
template <typename T>
__device__ __forceinline__ T sd_eta_g(const SysDev &s) {
  if constexpr (sizeof(T) == 4) return s.eta_gf;
  else return s.eta_g;
}

template <typename T>
__device__ __forceinline__ void shape(T x, T &s0, T &s1) {
  if (x < (T)0.5) {  // series: cancellation in sin x - x cos x
    T x2 = x * x;
    s0 = (T)1 + x2 * ((T)(-1.0 / 6) + x2 * ((T)(1.0 / 120) + x2 * ((T)(-1.0 / 5040) + x2 * (T)(1.0 / 362880))));
    s1 = (T)(1.0 / 3) + x2 * ((T)(-1.0 / 30) + x2 * ((T)(1.0 / 840) + x2 * ((T)(-1.0 / 45360) +
                                x2 * ((T)(1.0 / 3991680) + x2 * (T)(-1.0 / 518918400)))));
  } else {
    T sn, cs;
    if (sizeof(T) == 4) {
      float a, b;
      sincosf((float)x, &a, &b);
      sn = a;
      cs = b;
    } else {
      double a, b;
      sincos((double)x, &a, &b);
      sn = a;
      cs = b;
    }
    s0 = sn / x;
    s1 = (sn - x * cs) / (x * x * x);
  }
}

// Half-spectrum indices of point idx (32-bit arithmetic: a suspension's half
// spectrum has fewer than 2^31 points, and 64-bit division is slow on the GPU).
__device__ __forceinline__ bool kvector(const SysDev &s, size_t idx, int &ix, int &iy, int &iz) {
  const unsigned u = (unsigned)idx, nkx = (unsigned)s.nkx, ng = (unsigned)s.Ng;
  const unsigned q = u / nkx;
  ix = (int)(u - q * nkx);
  iz = (int)(q / ng);
  iy = (int)(q - (unsigned)iz * ng);
  int h = s.Ng / 2;
  return !(ix == h || iy == h || iz == h || (ix == 0 && iy == 0 && iz == 0));
}

// Wave vector of half-spectrum indices (ix, iy, iz): k = (2 pi/L) m for the cube,
// k = (2 pi/L) A^{-T} m on a deformed lattice (Sec. 2.3.3), m the signed indices.
template <typename T>
__device__ __forceinline__ void kcart(const SysDev &s, int ix, int iy, int iz, T k[3]) {
  const int h = s.Ng / 2;
  const int my = iy <= h ? iy : iy - s.Ng, mz = iz <= h ? iz : iz - s.Ng;
  if (!s.def && sizeof(T) == 4) {  // no FP64 instruction in the FP32 form
    k[0] = (T)((float)ix * s.kfacf);
    k[1] = (T)((float)my * s.kfacf);
    k[2] = (T)((float)mz * s.kfacf);
  } else if (!s.def) {
    k[0] = (T)(ix * s.kfac);
    k[1] = (T)(my * s.kfac);
    k[2] = (T)(mz * s.kfac);
  } else if (sizeof(T) == 4) {
    const float fx = (float)ix, fy = (float)my, fz = (float)mz;
#pragma unroll
    for (int d = 0; d < 3; ++d) k[d] = (T)(s.Btf[3 * d] * fx + s.Btf[3 * d + 1] * fy + s.Btf[3 * d + 2] * fz);
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) k[d] = (T)(s.Bt[3 * d] * ix + s.Bt[3 * d + 1] * my + s.Bt[3 * d + 2] * mz);
  }
}

// P^+ of a velocity mode uh: U = s0 uh, e = (3i s1 / 2) symY(uh, k)   (D = 3i s1 uh k^T)
template <typename T, bool WU, bool WE>
__device__ __forceinline__ void project_out(typename Cx<T>::t *g, size_t idx, size_t cs, int slotU, int slotE,
                                            const T k[3], T s0, T s1, const T ur[3], const T ui[3]) {
  using C2 = typename Cx<T>::t;
  if (WU) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      C2 o;
      o.x = s0 * ur[m];
      o.y = s0 * ui[m];
      g[(slotU + m) * cs + idx] = o;
    }
  }
  if (WE) {
    T er[5], ei[5];
    symY(ur, k, er);
    symY(ui, k, ei);
    T f = (T)1.5 * s1;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      C2 o;
      o.x = -f * ei[m];
      o.y = f * er[m];
      g[(slotE + m) * cs + idx] = o;
    }
  }
}

// P^+ B P with the Gaussian deconvolution at one half-spectrum point (Sec. 2.3.2):
// f = s0 F - 3i s1 S.k,  u = c (I - kk) f,  c = sigma^2/(eta V) (1 + k^2/4xi^2) e^{-(1 - eta_g) k^2/4xi^2} / k^2,
// then U = s0 u and E = Y : sym(3i s1 u k^T).  vin holds F (slots 0..2, when the mode
// has a force) and S (the next five slots); vout receives U (slots 0..2) and / or E
// (slots 0..4 for S -> E, 3..7 for the full product).  Modes k = 0 and on a Nyquist
// plane give zeros.
template <typename T, int MODE>
__device__ __forceinline__ void scale_point(const ScaleArgs &sa, const SysDev &s, size_t idx,
                                            const typename Cx<T>::t (&vin)[8], typename Cx<T>::t (&vout)[8]) {
  constexpr bool HF = MODE == M_FULL || MODE == M_FSU, WU = MODE != M_SE, WE = MODE == M_FULL || MODE == M_SE;
  constexpr int sIn = HF ? 3 : 0, eOut = (MODE == M_SE) ? 0 : 3;
  int ix, iy, iz;
  const bool live = kvector(s, idx, ix, iy, iz);
#pragma unroll
  for (int m = 0; m < 8; ++m) vout[m].x = vout[m].y = (T)0;
  if (!live) return;
  T k[3];
  kcart<T>(s, ix, iy, iz, k);
  T k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  T kk = sqrt(k2), ik = (T)1 / kk;
  T s0, s1;
  shape<T>(kk * sa_a<T>(sa), s0, s1);
  T u = k2 * sa_q4<T>(sa);
  T c = sd_c_apply<T>(s) * ((T)1 + u) * exp(-((T)1 - sd_eta_g<T>(s)) * u) / k2;
  T fr[3] = {0, 0, 0}, fi[3] = {0, 0, 0};
  if (HF) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      fr[m] = s0 * vin[m].x;
      fi[m] = s0 * vin[m].y;
    }
  }
  T sr[5], si[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    sr[m] = vin[sIn + m].x;
    si[m] = vin[sIn + m].y;
  }
  T skr[3], ski[3];
  Smul(sr, k, skr);
  Smul(si, k, ski);
  T t3 = (T)3 * s1;
#pragma unroll
  for (int m = 0; m < 3; ++m) {  // f = s0 F - 3i s1 S.k
    fr[m] += t3 * ski[m];
    fi[m] -= t3 * skr[m];
  }
  T kh[3] = {k[0] * ik, k[1] * ik, k[2] * ik};
  T pr = kh[0] * fr[0] + kh[1] * fr[1] + kh[2] * fr[2], pi = kh[0] * fi[0] + kh[1] * fi[1] + kh[2] * fi[2];
  T ur[3], ui[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    ur[m] = c * (fr[m] - kh[m] * pr);
    ui[m] = c * (fi[m] - kh[m] * pi);
  }
  if (WU) {  // U = s0 u
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      vout[m].x = s0 * ur[m];
      vout[m].y = s0 * ui[m];
    }
  }
  if (WE) {  // e = (3i s1 / 2) symY(u, k)
    T er[5], ei[5];
    symY(ur, k, er);
    symY(ui, k, ei);
    T f = (T)1.5 * s1;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      vout[eOut + m].x = -f * ei[m];
      vout[eOut + m].y = f * er[m];
    }
  }
}

// In-place scaling of the half spectra, NP consecutive points per thread (FP32:
// NP = 2, each component read and written as one 16-byte vector; every
// suspension's point count N_g^2 (N_g/2 + 1) is even, so pairs never straddle two
// suspensions and stay 16-byte aligned).
template <typename T, int MODE, int NP>
__global__ void k_scale(ScaleArgs sa, typename Cx<T>::t *g_all) {
  using C2 = typename Cx<T>::t;
  constexpr int NIN = (MODE == M_FULL || MODE == M_FSU) ? 8 : 5;
  constexpr int NOUT = (MODE == M_FULL) ? 8 : (MODE == M_SE ? 5 : 3);  // outputs occupy slots [0, NOUT)
  static_assert(NP == 1 || (NP == 2 && sizeof(T) == 4), "pairs in FP32 only");
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * NP;
  if (g0 >= sa.nk_tot) return;
  const int sidx = find_sys(sa.k0, sa.nsys, g0);
  if (!sa.active[sidx]) return;
  const SysDev &s = sa.sys[sidx];
  const size_t idx = (size_t)(g0 - s.k0);
  C2 *g = g_all + s.cgrid0;
  const size_t cs = s.cstride;
  C2 vin[NP][8], vout[NP][8];
#pragma unroll
  for (int m = 0; m < NIN; ++m) {
    if constexpr (NP == 2) {
      const float4 q = *(const float4 *)(g + m * cs + idx);
      vin[0][m].x = q.x;
      vin[0][m].y = q.y;
      vin[1][m].x = q.z;
      vin[1][m].y = q.w;
    } else {
      vin[0][m] = g[m * cs + idx];
    }
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) scale_point<T, MODE>(sa, s, idx + p, vin[p], vout[p]);
#pragma unroll
  for (int m = 0; m < NOUT; ++m) {
    if constexpr (NP == 2) {
      *(float4 *)(g + m * cs + idx) = make_float4(vout[0][m].x, vout[0][m].y, vout[1][m].x, vout[1][m].y);
    } else {
      g[m * cs + idx] = vout[0][m];
    }
  }
}

// P^+ B P of the 11-moment product at every half-spectrum point (Sec. 2.3.2, the
// paper's 11 grids): grids 0..2 F, 3..5 L, 6..10 S in, 0..2 U, 3..5 Omega, 6..10 E
// out.  With the torque in the couplet as sum_k L_k A_k (A_k = -eps_k/2),
// f = s0 F - 3i s1 S.k + (3i/2) s1 k x L, u = c (I - kk) f, U = s0 u, and from
// D = 3i s1 u k^T: Omega = A : D = -(3i/2) s1 u x k, e = Y : D = (3i s1/2) symY(u, k).
template <typename T>
__global__ void k_scale11(ScaleArgs sa, typename Cx<T>::t *g_all) {
  using C2 = typename Cx<T>::t;
  const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= sa.nk_tot) return;
  const int sidx = find_sys(sa.k0, sa.nsys, gidx);
  if (!sa.active[sidx]) return;
  const SysDev &s = sa.sys[sidx];
  const size_t idx = (size_t)(gidx - s.k0);
  C2 *g = g_all + s.cgrid0;
  const size_t cs = s.cstride;
  int ix, iy, iz;
  const bool live = kvector(s, idx, ix, iy, iz);
  C2 o[11];
#pragma unroll
  for (int m = 0; m < 11; ++m) o[m].x = o[m].y = (T)0;
  if (live) {
    T k[3];
    kcart<T>(s, ix, iy, iz, k);
    const T k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const T kk = sqrt(k2), ik = (T)1 / kk;
    T s0, s1;
    shape<T>(kk * sa_a<T>(sa), s0, s1);
    const T u = k2 * sa_q4<T>(sa);
    const T c = sd_c_apply<T>(s) * ((T)1 + u) * exp(-((T)1 - sd_eta_g<T>(s)) * u) / k2;
    T fr[3], fi[3], Lr[3], Li[3], sr[5], si[5];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const C2 F = g[m * cs + idx], Lv = g[(3 + m) * cs + idx];
      fr[m] = s0 * F.x;
      fi[m] = s0 * F.y;
      Lr[m] = Lv.x;
      Li[m] = Lv.y;
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      const C2 v = g[(6 + m) * cs + idx];
      sr[m] = v.x;
      si[m] = v.y;
    }
    T skr[3], ski[3];
    Smul(sr, k, skr);
    Smul(si, k, ski);
    const T t3 = (T)3 * s1, t15 = (T)1.5 * s1;
    const T kLr[3] = {k[1] * Lr[2] - k[2] * Lr[1], k[2] * Lr[0] - k[0] * Lr[2], k[0] * Lr[1] - k[1] * Lr[0]};
    const T kLi[3] = {k[1] * Li[2] - k[2] * Li[1], k[2] * Li[0] - k[0] * Li[2], k[0] * Li[1] - k[1] * Li[0]};
#pragma unroll
    for (int m = 0; m < 3; ++m) {  // f = s0 F - 3i s1 S.k + (3i/2) s1 k x L
      fr[m] += t3 * ski[m] - t15 * kLi[m];
      fi[m] += -t3 * skr[m] + t15 * kLr[m];
    }
    const T kh[3] = {k[0] * ik, k[1] * ik, k[2] * ik};
    const T pr = kh[0] * fr[0] + kh[1] * fr[1] + kh[2] * fr[2], pi = kh[0] * fi[0] + kh[1] * fi[1] + kh[2] * fi[2];
    T ur[3], ui[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      ur[m] = c * (fr[m] - kh[m] * pr);
      ui[m] = c * (fi[m] - kh[m] * pi);
    }
    const T ukr[3] = {ur[1] * k[2] - ur[2] * k[1], ur[2] * k[0] - ur[0] * k[2], ur[0] * k[1] - ur[1] * k[0]};
    const T uki[3] = {ui[1] * k[2] - ui[2] * k[1], ui[2] * k[0] - ui[0] * k[2], ui[0] * k[1] - ui[1] * k[0]};
    T er[5], ei[5];
    symY(ur, k, er);
    symY(ui, k, ei);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      o[m].x = s0 * ur[m];
      o[m].y = s0 * ui[m];
      o[3 + m].x = t15 * uki[m];   // Omega = -(3i/2) s1 u x k
      o[3 + m].y = -t15 * ukr[m];
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      o[6 + m].x = -t15 * ei[m];
      o[6 + m].y = t15 * er[m];
    }
  }
#pragma unroll
  for (int m = 0; m < 11; ++m) g[m * cs + idx] = o[m];
}

// Wave-space noise: dW2 on the half spectrum (Hermitian partners on kx = 0),
// u = sigma e^{eta_g k^2/8xi^2} sqrt(H/(eta V k^2)) (I - kk) dW2, then P^+.
template <typename T, bool EXT>
__global__ void k_noise(ScaleArgs sa, const T *__restrict__ w2, uint64_t seed, uint64_t counter,
                        const uint64_t *rng, typename Cx<T>::t *g_all) {
  const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= sa.nk_tot) return;
  if (rng) {  // a captured graph reads (seed, counter) at launch
    seed = rng[0];
    counter = rng[1];
  }
  const int sidx = find_sys(sa.k0, sa.nsys, gidx);
  if (!sa.active[sidx]) return;
  const SysDev &s = sa.sys[sidx];
  const size_t idx = (size_t)(gidx - s.k0), nk = (size_t)s.Ng * s.Ng * s.nkx;
  using C2 = typename Cx<T>::t;
  C2 *g = g_all + s.cgrid0;
  int ix, iy, iz;
  bool live = kvector(s, idx, ix, iy, iz);
  const size_t cs = s.cstride;
  if (!live) {
    C2 z;
    z.x = 0;
    z.y = 0;
    for (int m = 0; m < 8; ++m) g[m * cs + idx] = z;
    return;
  }
  int h = s.Ng / 2, Ng = s.Ng;
  bool partner = ix == 0 && (iz > h || (iz == 0 && iy > h));
  size_t src = idx;
  if (partner) src = ((size_t)((Ng - iz) % Ng) * Ng + (size_t)((Ng - iy) % Ng)) * s.nkx;
  T dr[3], di[3];
  const T isq2 = (T)0.70710678118654752;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    T re, im;
    size_t n = 3 * (size_t)s.k0 + (size_t)m * nk + src;  // normals of suspension s follow those of 0..s-1
    if (EXT) {
      re = w2[2 * n];
      im = w2[2 * n + 1];
    } else {
      normal_pair<T>(seed, counter, 2u, (uint64_t)n, re, im);
    }
    dr[m] = re * isq2;
    di[m] = (partner ? -im : im) * isq2;
  }
  T k[3];
  kcart<T>(s, ix, iy, iz, k);
  T k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  T kk = sqrt(k2), ik = (T)1 / kk;
  T s0, s1;
  shape<T>(kk * sa_a<T>(sa), s0, s1);
  T u = k2 * sa_q4<T>(sa);
  T c = sd_c_noise<T>(s) * sqrt(((T)1 + u) / k2) * exp(-(T)0.5 * ((T)1 - sd_eta_g<T>(s)) * u);
  T kh[3] = {k[0] * ik, k[1] * ik, k[2] * ik};
  T pr = kh[0] * dr[0] + kh[1] * dr[1] + kh[2] * dr[2], pi = kh[0] * di[0] + kh[1] * di[1] + kh[2] * di[2];
  T ur[3], ui[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    ur[m] = c * (dr[m] - kh[m] * pr);
    ui[m] = c * (di[m] - kh[m] * pi);
  }
  project_out<T, true, true>(g, idx, cs, 0, 3, k, s0, s1, ur, ui);
}

ScaleArgs scale_args(const pse_ctx *c) {
  ScaleArgs s;
  s.nsys = c->nsys;
  s.nk_tot = c->nk_tot;
  s.a = c->p.a;
  s.q4 = 1.0 / (4.0 * c->p.xi * c->p.xi);
  s.af = (float)s.a;
  s.q4f = (float)s.q4;
  s.sys = c->d_sys;
  s.k0 = c->d_k0;
  s.active = c->d_active;
  return s;
}

// One batched transform per grid-size group over the leading `comps` components
// of every suspension in the group.
template <typename T>
pse_status fft(pse_ctx *c, bool forward, int comps, cudaStream_t s, int variant = 0) {
  StageTimer timer(c, PSE_STAGE_FFT, s, variant);
  for (FftGroup &g : c->groups) {
    bool any = false;
    for (int q : g.members) any = any || c->h_active[q];
    if (!any) continue;
    c->nfft += 1;
    cufftHandle plan = forward ? g.r2c[comps] : g.c2r[comps];
    PSE_CUFFT_TRY(c, cufftSetStream(plan, s));
    T *rg = (T *)c->d_grid + g.grid0;
    typename Cx<T>::t *cg = (typename Cx<T>::t *)c->d_cgrid + g.cgrid0;
    if (sizeof(T) == 4) {
      if (forward) PSE_CUFFT_TRY(c, cufftExecR2C(plan, (cufftReal *)rg, (cufftComplex *)cg));
      else PSE_CUFFT_TRY(c, cufftExecC2R(plan, (cufftComplex *)cg, (cufftReal *)rg));
    } else {
      if (forward) PSE_CUFFT_TRY(c, cufftExecD2Z(plan, (cufftDoubleReal *)rg, (cufftDoubleComplex *)cg));
      else PSE_CUFFT_TRY(c, cufftExecZ2D(plan, (cufftDoubleComplex *)cg, (cufftDoubleReal *)rg));
    }
  }
  return PSE_OK;
}

template <typename T>
pse_status wave_apply_t(pse_ctx *c, const void *vin, void *vout, int mode, bool add, cudaStream_t s) {
  WaveArgs a = wave_args(c);
  if (!add) PSE_CUDA_TRY(c, cudaMemsetAsync(vout, 0, sizeof(T) * 8 * (size_t)c->p.N, s));
  int cin = (mode == M_SE || mode == M_SU) ? 5 : 8, cout = mode == M_FULL ? 8 : (mode == M_SE ? 5 : 3);
  {
    StageTimer timer(c, PSE_STAGE_SPREAD, s, mode);
    c->nlaunch += 2;  // counter reset + kernel
    spread_launch(c, a, vin, mode, s);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  PSE_TRY(fft<T>(c, true, cin, s, mode));
  ScaleArgs sa = scale_args(c);
  using C2 = typename Cx<T>::t;
  {
    StageTimer timer(c, PSE_STAGE_SCALE, s, mode);
    c->nlaunch += 1;
    constexpr int NP = sizeof(T) == 4 ? 2 : 1;
    const unsigned nb = (unsigned)ceil_div(c->nk_tot, 256 * NP);
    if (mode == M_FULL) k_scale<T, M_FULL, NP><<<nb, 256, 0, s>>>(sa, (C2 *)c->d_cgrid);
    else if (mode == M_SE) k_scale<T, M_SE, NP><<<nb, 256, 0, s>>>(sa, (C2 *)c->d_cgrid);
    else if (mode == M_SU) k_scale<T, M_SU, NP><<<nb, 256, 0, s>>>(sa, (C2 *)c->d_cgrid);
    else k_scale<T, M_FSU, NP><<<nb, 256, 0, s>>>(sa, (C2 *)c->d_cgrid);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  PSE_TRY(fft<T>(c, false, cout, s, mode));
  {
    StageTimer timer(c, PSE_STAGE_INTERP, s, mode);
    c->nlaunch += 2;
    interp_launch(c, a, vout, mode, s);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

template <typename T>
pse_status wave_noise_t(pse_ctx *c, const void *w2, uint64_t seed, uint64_t counter, void *vout, cudaStream_t s) {
  WaveArgs a = wave_args(c);
  ScaleArgs sa = scale_args(c);
  unsigned nb = (unsigned)ceil_div(c->nk_tot, 256);
  using C2 = typename Cx<T>::t;
  {
    StageTimer timer(c, PSE_STAGE_NOISE, s);
    c->nlaunch += 1;
    const uint64_t *rng = c->capturing ? c->d_rng : nullptr;
    if (w2) k_noise<T, true><<<nb, 256, 0, s>>>(sa, (const T *)w2, seed, counter, nullptr, (C2 *)c->d_cgrid);
    else k_noise<T, false><<<nb, 256, 0, s>>>(sa, nullptr, seed, counter, rng, (C2 *)c->d_cgrid);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  PSE_TRY(fft<T>(c, false, 8, s));
  {
    StageTimer timer(c, PSE_STAGE_INTERP, s);
    c->nlaunch += 2;
    interp_launch(c, a, vout, M_FULL, s);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

template <typename T>
pse_status wave_apply11_t(pse_ctx *c, const void *vin12, void *vout12, bool add, cudaStream_t s) {
  if (!add) PSE_CUDA_TRY(c, cudaMemsetAsync(vout12, 0, sizeof(T) * 12 * (size_t)c->p.N, s));
  {
    StageTimer timer(c, PSE_STAGE_SPREAD, s);
    spread11_launch(c, vin12, s);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  PSE_TRY(fft<T>(c, true, 11, s));
  ScaleArgs sa = scale_args(c);
  {
    StageTimer timer(c, PSE_STAGE_SCALE, s);
    c->nlaunch += 1;
    k_scale11<T><<<(unsigned)ceil_div(c->nk_tot, 256), 256, 0, s>>>(sa, (typename Cx<T>::t *)c->d_cgrid);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  PSE_TRY(fft<T>(c, false, 11, s));
  {
    StageTimer timer(c, PSE_STAGE_INTERP, s);
    interp11_launch(c, vout12, s);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

}  // namespace

pse_status wave_apply11(pse_ctx *c, const void *vin12, void *vout12, bool add, cudaStream_t s) {
  return c->prec == PSE_MIXED ? wave_apply11_t<float>(c, vin12, vout12, add, s)
                              : wave_apply11_t<double>(c, vin12, vout12, add, s);
}

WaveArgs wave_args(const pse_ctx *c) {
  WaveArgs a;
  a.P = c->p.P;
  a.want = -1;
  a.nsys = c->nsys;
  a.ntiles = (int)c->ntiles;
  a.sys = c->d_sys;
  a.tile0 = c->d_tile0;
  a.active = c->d_active;
  return a;
}

pse_status wave_apply(pse_ctx *c, const void *vin, void *vout, int mode, bool add, cudaStream_t s) {
  return c->prec == PSE_MIXED ? wave_apply_t<float>(c, vin, vout, mode, add, s)
                              : wave_apply_t<double>(c, vin, vout, mode, add, s);
}

pse_status wave_noise(pse_ctx *c, const void *w2, uint64_t seed, uint64_t counter, void *vout, cudaStream_t s) {
  return c->prec == PSE_MIXED ? wave_noise_t<float>(c, w2, seed, counter, vout, s)
                              : wave_noise_t<double>(c, w2, seed, counter, vout, s);
}

}  // namespace pse
