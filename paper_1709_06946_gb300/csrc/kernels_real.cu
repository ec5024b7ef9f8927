// Real-space part of the split mobility (Sec. 2.3.1): for every particle the sum
// over neighbours closer than r_cut of the 8x8 real-space block (Eqs. MUFr-MDCr)
// applied to [F; S], plus the real-space self term (App. A, Case 3).
//
// G lanes per particle walk its slotted neighbour list.  Outputs are in sorted
// order (by suspension, then spreading tile); each neighbour record holds the
// neighbour's position in the cell list, and the input vector is first copied
// into cell-list order, so the lanes of a particle, walking consecutive entries
// of the list (runs of cells along x), read neighbouring rows of that copy and
// share cache lines.  A persistent grid takes blocks of particles from a work
// counter; particles of suspensions marked inactive are skipped.  The seven scalar functions
// come from a table on r: linear interpolation in FP32 (mixed form), cubic
// Lagrange interpolation in FP64 with one-sided stencils at the r = 2a node
// where the functions have a kink.
#include <algorithm>

#include "device_common.cuh"
#include "pse_internal.cuh"

namespace pse {
namespace {

struct RealArgs {
  int64_t Ntot;
  int nsys, len, k2;
  double inv_dr, self_uf, self_es;
};

// 32 bytes (8 floats) from 32-byte aligned read-only global memory in one
// 256-bit load.
__device__ __forceinline__ void ldg8(const float *p, float4 &lo, float4 &hi) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
      : "l"(p));
}

// f[0..7) at r by linear interpolation.  The full product reads two 8-float
// entries (q and q + 1); the partial products read one 8-float interval record
// holding the values they need at both ends: f4..f6 (S -> E) or f0..f3
// ([F; S] -> U); the other functions are left unset.
template <bool SH = false, int MODE = M_FULL>
__device__ __forceinline__ void lookup(const float *tab, const RealArgs &a, float r, float f[7]) {
  float x = r * (float)a.inv_dr;
  int q = min((int)x, a.len - 2);
  float t = x - (float)q;
  const float4 *t4 = (const float4 *)tab;
  float4 a0, a1, b0, b1;
  if (!SH && MODE == M_SE) {
    ldg8(tab + 8 * q, a0, a1);  // f4 f5 f6 at q, then at q + 1
    f[4] = fmaf(t, a0.w - a0.x, a0.x);
    f[5] = fmaf(t, a1.x - a0.y, a0.y);
    f[6] = fmaf(t, a1.y - a0.z, a0.z);
    return;
  }
  if (!SH && (MODE == M_FSU || MODE == M_SU)) {
    ldg8(tab + 8 * q, a0, a1);  // f0..f3 at q, then at q + 1
    f[0] = fmaf(t, a1.x - a0.x, a0.x);
    f[1] = fmaf(t, a1.y - a0.y, a0.y);
    f[2] = fmaf(t, a1.z - a0.z, a0.z);
    f[3] = fmaf(t, a1.w - a0.w, a0.w);
    return;
  }
  if (SH) {  // table staged in shared memory
    a0 = t4[2 * q];
    a1 = t4[2 * q + 1];
    b0 = t4[2 * q + 2];
    b1 = t4[2 * q + 3];
  } else {  // entries are 8 floats (32 bytes): one 256-bit load each
    ldg8(tab + 8 * q, a0, a1);
    ldg8(tab + 8 * q + 8, b0, b1);
  }
  f[0] = fmaf(t, b0.x - a0.x, a0.x);
  f[1] = fmaf(t, b0.y - a0.y, a0.y);
  f[2] = fmaf(t, b0.z - a0.z, a0.z);
  f[3] = fmaf(t, b0.w - a0.w, a0.w);
  f[4] = fmaf(t, b1.x - a1.x, a1.x);
  f[5] = fmaf(t, b1.y - a1.y, a1.y);
  f[6] = fmaf(t, b1.z - a1.z, a1.z);
}

template <bool SH = false, int MODE = M_FULL>
__device__ __forceinline__ void lookup(const double *tab, const RealArgs &a, double r, double f[7]) {
  double x = r * a.inv_dr;
  int q = min((int)x, a.len - 2);
  int b = q - 1;
  if (q < a.k2) b = min(b, a.k2 - 3);
  else b = max(b, a.k2);
  b = max(0, min(b, a.len - 4));
  double t = x - (double)b;
  double w0 = -(t - 1) * (t - 2) * (t - 3) / 6.0, w1 = t * (t - 2) * (t - 3) / 2.0;
  double w2 = -t * (t - 1) * (t - 3) / 2.0, w3 = t * (t - 1) * (t - 2) / 6.0;
  const double *r0 = tab + 8 * (size_t)b;
#pragma unroll
  for (int k = 0; k < 7; ++k)
    f[k] = w0 * __ldg(r0 + k) + w1 * __ldg(r0 + 8 + k) + w2 * __ldg(r0 + 16 + k) + w3 * __ldg(r0 + 24 + k);
}

// G lanes share one particle: they walk its neighbour list with stride G (so
// the neighbours' records are fetched in parallel) and the partial sums are
// reduced with shuffles; the first lane of the group adds the self term.
// FP32: at most 64 registers so that four 256-thread CTAs fit an SM (the full
// 8 -> 8 product would otherwise take 74 and leave room for three).  With
// SHT (FP32 only) one 1024-thread CTA per SM first copies the table into shared
// memory and the lookups leave L1 to the neighbours' records.
template <typename T, int MODE, int G, bool SHT = false, int NT = SHT ? 1024 : 256>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? (SHT ? 1 : 4) : 1) k_real(RealArgs a,
                                              const SysDev *__restrict__ sys,
                                              const int64_t *__restrict__ p0, const int *__restrict__ active,
                                              int *queue, int nitems,
                                              const int *__restrict__ nstart,
                                              const typename V4<T>::t *__restrict__ geo,
                                              const T *__restrict__ vin, const T *__restrict__ vcell,
                                              T *__restrict__ vout, const T *__restrict__ gtab) {
  extern __shared__ __align__(16) unsigned char tab_raw[];
  const T *tab = gtab;
  if (SHT) {
    float4 *dst = (float4 *)tab_raw;
    const float4 *src = (const float4 *)gtab;
    for (int q = threadIdx.x; q < 2 * a.len; q += blockDim.x) dst[q] = src[q];
    __syncthreads();
    tab = (const T *)tab_raw;
  }
  constexpr bool HAS_F = MODE == M_FULL || MODE == M_FSU, WANT_U = MODE != M_SE;
  constexpr bool WANT_E = MODE == M_FULL || MODE == M_SE;
  using T4 = typename V4<T>::t;
  for_each_item(queue, nitems, [&](int item) {
    const int64_t gid = ((int64_t)item * NT + threadIdx.x) / G;
    const int sub = threadIdx.x % G;
    const int64_t i = gid < a.Ntot ? gid : a.Ntot - 1;
    const int si = find_sys(p0, a.nsys, i);
    const bool live = gid < a.Ntot && active[si];
    const SysDev &sd = sys[si];
    const T4 *v4 = (const T4 *)vin, *vc4 = (const T4 *)vcell;
    T U[3] = {0, 0, 0}, E[5] = {0, 0, 0, 0, 0};
    // particle i's row of slots; an overflowed list is flagged and redone
    const int64_t k0 = sd.nbr0 + (i - sd.p0) * sd.slots;
    const int cnt = live ? min(nstart[i], sd.slots) : 0;
    for (int n = sub; n < cnt; n += G) {
      const int64_t k = k0 + n;
      const T4 gg = geo[k];  // separation x_i - x_j and j, stored by the list build
      const int j = real_as_index<T>(gg.w);
      const T r2 = gg.x * gg.x + gg.y * gg.y + gg.z * gg.z;
      const T ir = sizeof(T) == 4 ? (T)rsqrtf((float)r2) : (T)1 / sqrt(r2), r = r2 * ir;
      T rh[3] = {gg.x * ir, gg.y * ir, gg.z * ir};
      T f[7];
      lookup<SHT, MODE>(tab, a, r, f);
      T4 q0, q1;
      if constexpr (sizeof(T) == 4) ldg8((const float *)vcell + 8 * (size_t)j, q0, q1);  // the 8 slots of row j
      else q0 = vc4[2 * j], q1 = vc4[2 * j + 1];
      T s[5] = {q0.w, q1.x, q1.y, q1.z, q1.w};
      T v[3];
      Smul(s, rh, v);
      const T q = rh[0] * v[0] + rh[1] * v[1] + rh[2] * v[2];
      const T F[3] = {q0.x, q0.y, q0.z};
      const T rf = HAS_F ? rh[0] * F[0] + rh[1] * F[1] + rh[2] * F[2] : (T)0;
      // the terms of each output along the same direction are collected first:
      // U = f2 v + f0 F + (f3 q + (f1 - f0) rf) rh;
      // E = f4 s + Y(f5 v - f2 F / 2, rh) + (f6 q - f3 rf) / 2 Y(rh, rh)
      // (Y(., rh) is linear in its first argument)
      if (WANT_U) {
        T c = f[3] * q;
        if (HAS_F) c += (f[1] - f[0]) * rf;
#pragma unroll
        for (int m = 0; m < 3; ++m) U[m] += f[2] * v[m] + c * rh[m] + (HAS_F ? f[0] * F[m] : (T)0);
      }
      if (WANT_E) {
        T pv[3], sy[5], yr[5];
#pragma unroll
        for (int m = 0; m < 3; ++m) pv[m] = f[5] * v[m] - (HAS_F ? (T)0.5 * f[2] * F[m] : (T)0);
        symY(pv, rh, sy);
        symY(rh, rh, yr);  // = 2 y(rh)
        const T cy = (T)0.5 * (f[6] * q - (HAS_F ? f[3] * rf : (T)0));
#pragma unroll
        for (int m = 0; m < 5; ++m) E[m] += f[4] * s[m] + sy[m] + cy * yr[m];
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
#pragma unroll
      for (int m = 0; m < 3; ++m) U[m] += __shfl_xor_sync(0xffffffffu, U[m], o, G);
#pragma unroll
      for (int m = 0; m < 5; ++m) E[m] += __shfl_xor_sync(0xffffffffu, E[m], o, G);
    }
    if (live && sub == 0) {
      T4 s0 = v4[2 * i], s1 = v4[2 * i + 1];
      if (WANT_U && HAS_F) {
        U[0] += (T)a.self_uf * s0.x;
        U[1] += (T)a.self_uf * s0.y;
        U[2] += (T)a.self_uf * s0.z;
      }
      if (WANT_E) {
        E[0] += (T)a.self_es * s0.w;
        E[1] += (T)a.self_es * s1.x;
        E[2] += (T)a.self_es * s1.y;
        E[3] += (T)a.self_es * s1.z;
        E[4] += (T)a.self_es * s1.w;
      }
      T4 o0, o1;
      o0.x = U[0];
      o0.y = U[1];
      o0.z = U[2];
      o0.w = E[0];
      o1.x = E[1];
      o1.y = E[2];
      o1.z = E[3];
      o1.w = E[4];
      T4 *o4 = (T4 *)vout;
      o4[2 * i] = o0;
      o4[2 * i + 1] = o1;
    }
  });
}

template <typename T, int MODE, int G>
void launch_real_m(pse_ctx *c, const RealArgs &a, const void *vin, void *vout, cudaStream_t s) {
  const size_t tab_bytes = sizeof(T) * 8 * (size_t)a.len;
  if (sizeof(T) == 4 && c->real_smem_table && tab_bytes <= c->smem_optin) {
    auto kern = k_real<T, MODE, G, true>;
    static std::once_flag once;
    std::call_once(once, [&] {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_optin);
      cudaGetLastError();
    });
    static std::atomic<int> per_sm{0};
    const int64_t items = ceil_div(a.Ntot * G, 1024);
    unsigned grid = persistent_grid(c, kern, 1024, tab_bytes, items, per_sm);
    int *q = next_queue(c, s);
    kern<<<grid, 1024, tab_bytes, s>>>(a, c->d_sys, c->d_p0, c->d_active, q, (int)items, c->d_nbr_start,
                                       (const typename V4<T>::t *)c->d_nbr_geo, (const T *)vin,
                                       (const T *)c->d_vcell, (T *)vout, (const T *)c->d_table);
    return;
  }
  auto kern = k_real<T, MODE, G>;
  static std::atomic<int> per_sm{0};
  const int64_t items = ceil_div(a.Ntot * G, 256);
  const void *tab = c->d_table;  // FP32 partial products: their interval table
  if (sizeof(T) == 4 && MODE == M_SE) tab = c->d_table_e;
  if (sizeof(T) == 4 && (MODE == M_FSU || MODE == M_SU)) tab = c->d_table_u;
  unsigned grid = persistent_grid(c, kern, 256, 0, items, per_sm);
  int *q = next_queue(c, s);
  kern<<<grid, 256, 0, s>>>(a, c->d_sys, c->d_p0, c->d_active, q, (int)items, c->d_nbr_start,
                            (const typename V4<T>::t *)c->d_nbr_geo, (const T *)vin, (const T *)c->d_vcell,
                            (T *)vout, (const T *)tab);
}

template <typename T, int G>
void launch_real_g(pse_ctx *c, const RealArgs &a, const void *vin, void *vout, int mode, cudaStream_t s) {
  if (mode == M_FULL) launch_real_m<T, M_FULL, G>(c, a, vin, vout, s);
  else if (mode == M_SE) launch_real_m<T, M_SE, G>(c, a, vin, vout, s);
  else if (mode == M_SU) launch_real_m<T, M_SU, G>(c, a, vin, vout, s);
  else launch_real_m<T, M_FSU, G>(c, a, vin, vout, s);
}

template <typename T>
void launch_real(pse_ctx *c, const RealArgs &a, const void *vin, void *vout, int mode, cudaStream_t s) {
  // lanes per particle from the mean neighbour count of the current lists
  int g = c->opt.real_lanes;
  if (g <= 0) {
    const int64_t pairs = c->npairs > 0 ? c->npairs : c->npairs_est;  // before the first list: the estimate
    double mean = a.Ntot > 0 ? (double)pairs / a.Ntot : 0.0;
    g = mean >= 200.0 ? 8 : (mean >= 24.0 ? 4 : 1);  // 4 lanes measured fastest near 100 neighbours
  }
  switch (g) {
    case 32: launch_real_g<T, 32>(c, a, vin, vout, mode, s); break;
    case 16: launch_real_g<T, 16>(c, a, vin, vout, mode, s); break;
    case 8: launch_real_g<T, 8>(c, a, vin, vout, mode, s); break;
    case 4: launch_real_g<T, 4>(c, a, vin, vout, mode, s); break;
    default: launch_real_g<T, 1>(c, a, vin, vout, mode, s);
  }
}

// The three rotation scalars of the 11-moment form at r (4 reals per node): linear
// interpolation in FP32; in FP64 cubic Lagrange interpolation with the same
// one-sided stencils at the r = 2a node as lookup().
__device__ __forceinline__ void rot_lookup(const float *tab, const RealArgs &a, float r, float g[3]) {
  float x = r * (float)a.inv_dr;
  int q = min((int)x, a.len - 2);
  float t = x - (float)q;
  const float4 u = ((const float4 *)tab)[q], v = ((const float4 *)tab)[q + 1];
  g[0] = fmaf(t, v.x - u.x, u.x);
  g[1] = fmaf(t, v.y - u.y, u.y);
  g[2] = fmaf(t, v.z - u.z, u.z);
}
__device__ __forceinline__ void rot_lookup(const double *tab, const RealArgs &a, double r, double g[3]) {
  double x = r * a.inv_dr;
  int q = min((int)x, a.len - 2);
  int b = q - 1;
  if (q < a.k2) b = min(b, a.k2 - 3);
  else b = max(b, a.k2);
  b = max(0, min(b, a.len - 4));
  double t = x - (double)b;
  double w0 = -(t - 1) * (t - 2) * (t - 3) / 6.0, w1 = t * (t - 2) * (t - 3) / 2.0;
  double w2 = -t * (t - 1) * (t - 3) / 2.0, w3 = t * (t - 1) * (t - 2) / 6.0;
  const double *r0 = tab + 4 * (size_t)b;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    g[k] = w0 * __ldg(r0 + k) + w1 * __ldg(r0 + 4 + k) + w2 * __ldg(r0 + 8 + k) + w3 * __ldg(r0 + 12 + k);
}

// The 11-moment real-space product (Sec. 2.2.1 rigid-particle relation): rows of 12
// slots, [F(3), L(3), s(5), -] in and [U(3), Omega(3), e(5), -] out.  Per pair, the
// 8 x 8 force-stresslet terms of k_real plus the rotation couplings
//   U += gF rh x L,   Omega += gF rh x F + gL1 L + gL2 (rh.L) rh + 2 gL2 (S rh) x rh,
//   e += gL2 symY(rh x L, rh)
// (gF, gL1, gL2 the rotation scalars); self terms self_uf, self_ol, self_es.  G lanes
// per particle walk its neighbour records, neighbours' rows from the cell-ordered copy.
template <typename T, int G>
__global__ void __launch_bounds__(256) k_real11(RealArgs a, const SysDev *__restrict__ sys,
                                                const int64_t *__restrict__ p0, const int *__restrict__ active,
                                                int *queue, int nitems, const int *__restrict__ nstart,
                                                const typename V4<T>::t *__restrict__ geo,
                                                const T *__restrict__ vin, const T *__restrict__ vcell,
                                                T *__restrict__ vout, const T *__restrict__ tab,
                                                const T *__restrict__ rtab, T self_ol) {
  using T4 = typename V4<T>::t;
  for_each_item(queue, nitems, [&](int item) {
    const int64_t gid = ((int64_t)item * 256 + threadIdx.x) / G;
    const int sub = threadIdx.x % G;
    const int64_t i = gid < a.Ntot ? gid : a.Ntot - 1;
    const int si = find_sys(p0, a.nsys, i);
    const bool live = gid < a.Ntot && active[si];
    const SysDev &sd = sys[si];
    T o[11];
#pragma unroll
    for (int m = 0; m < 11; ++m) o[m] = 0;
    const int64_t k0 = sd.nbr0 + (i - sd.p0) * sd.slots;
    const int cnt = live ? min(nstart[i], sd.slots) : 0;
    for (int n = sub; n < cnt; n += G) {
      const T4 gg = geo[k0 + n];
      const int j = real_as_index<T>(gg.w);
      const T r2 = gg.x * gg.x + gg.y * gg.y + gg.z * gg.z;
      const T ir = sizeof(T) == 4 ? (T)rsqrtf((float)r2) : (T)1 / sqrt(r2), r = r2 * ir;
      const T rh[3] = {gg.x * ir, gg.y * ir, gg.z * ir};
      T f[7], gr[3];
      lookup<false, M_FULL>(tab, a, r, f);
      rot_lookup(rtab, a, r, gr);
      const T *row = vcell + 12 * (size_t)j;
      const T F[3] = {row[0], row[1], row[2]}, Lv[3] = {row[3], row[4], row[5]};
      const T s[5] = {row[6], row[7], row[8], row[9], row[10]};
      T v[3];
      Smul(s, rh, v);
      const T q = rh[0] * v[0] + rh[1] * v[1] + rh[2] * v[2];
      const T rf = rh[0] * F[0] + rh[1] * F[1] + rh[2] * F[2];
      const T rl = rh[0] * Lv[0] + rh[1] * Lv[1] + rh[2] * Lv[2];
      const T rxL[3] = {rh[1] * Lv[2] - rh[2] * Lv[1], rh[2] * Lv[0] - rh[0] * Lv[2], rh[0] * Lv[1] - rh[1] * Lv[0]};
      const T rxF[3] = {rh[1] * F[2] - rh[2] * F[1], rh[2] * F[0] - rh[0] * F[2], rh[0] * F[1] - rh[1] * F[0]};
      const T vxr[3] = {v[1] * rh[2] - v[2] * rh[1], v[2] * rh[0] - v[0] * rh[2], v[0] * rh[1] - v[1] * rh[0]};
      const T cu = f[3] * q + (f[1] - f[0]) * rf;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        o[m] += f[2] * v[m] + f[0] * F[m] + cu * rh[m] + gr[0] * rxL[m];
        o[3 + m] += gr[0] * rxF[m] + gr[1] * Lv[m] + gr[2] * rl * rh[m] + (T)2 * gr[2] * vxr[m];
      }
      T pv[3], sy[5], yr[5], yl[5];
#pragma unroll
      for (int m = 0; m < 3; ++m) pv[m] = f[5] * v[m] - (T)0.5 * f[2] * F[m];
      symY(pv, rh, sy);
      symY(rh, rh, yr);
      symY(rxL, rh, yl);
      const T cy = (T)0.5 * (f[6] * q - f[3] * rf);
#pragma unroll
      for (int m = 0; m < 5; ++m) o[6 + m] += f[4] * s[m] + sy[m] + cy * yr[m] + gr[2] * yl[m];
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
      for (int m = 0; m < 11; ++m) o[m] += __shfl_xor_sync(0xffffffffu, o[m], off, G);
    if (live && sub == 0) {
      const T *me = vin + 12 * (size_t)i;
      T *out = vout + 12 * (size_t)i;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        out[m] = o[m] + (T)a.self_uf * me[m];
        out[3 + m] = o[3 + m] + self_ol * me[3 + m];
      }
#pragma unroll
      for (int m = 0; m < 5; ++m) out[6 + m] = o[6 + m] + (T)a.self_es * me[6 + m];
      out[11] = 0;
    }
  });
}

// vcell12[k] = vin12[list[k]] (12-real rows).
template <typename T>
__global__ void k_cell_gather12(int64_t N, const int *__restrict__ list, const T *__restrict__ vin,
                                T *__restrict__ vcell) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 12 * N) return;
  const int64_t k = e / 12;
  vcell[e] = vin[12 * (int64_t)list[k] + (e - 12 * k)];
}

// vcell[k] = vin[list[k]]: the 8-real rows of the input vector in cell-list order.
template <typename T>
__global__ void k_cell_gather(int64_t N, const int *__restrict__ list, const typename V4<T>::t *__restrict__ vin,
                              typename V4<T>::t *__restrict__ vcell) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int64_t j = list[k];
  vcell[2 * k] = vin[2 * j];
  vcell[2 * k + 1] = vin[2 * j + 1];
}

// Harmonic overlap repulsion F_i = sum_j k (2a - r_ij) rh_ij over neighbours
// closer than 2a (from the list's separation records), written in user order.
template <typename T>
__global__ void k_overlap(const SysDev *__restrict__ sys, const int64_t *__restrict__ p0, int nsys, int64_t Ntot,
                          double contact, double kspring, const int *__restrict__ nstart,
                          const typename V4<T>::t *__restrict__ geo, const int *__restrict__ perm, T *F) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Ntot) return;
  const SysDev &sd = sys[find_sys(p0, nsys, i)];
  double f[3] = {0, 0, 0};
  const int64_t k0 = sd.nbr0 + (i - sd.p0) * sd.slots;
  const int cnt = min(nstart[i], sd.slots);
  for (int n = 0; n < cnt; ++n) {
    const typename V4<T>::t g = geo[k0 + n];
    const double d[3] = {(double)g.x, (double)g.y, (double)g.z};
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (r >= contact || r == 0.0) continue;
    double c = kspring * (contact - r) / r;
    for (int m = 0; m < 3; ++m) f[m] += c * d[m];
  }
  const int64_t u = perm[i];
  for (int m = 0; m < 3; ++m) F[3 * u + m] = (T)f[m];
}

}  // namespace

pse_status overlap_force(pse_ctx *c, double kspring, void *F, cudaStream_t s) {
  c->nlaunch += 1;
  const int64_t N = c->p.N;
  const unsigned nb = (unsigned)ceil_div(N, 256);
  if (c->prec == PSE_MIXED)
    k_overlap<float><<<nb, 256, 0, s>>>(c->d_sys, c->d_p0, c->nsys, N, 2.0 * c->p.a, kspring, c->d_nbr_start,
                                        (const float4 *)c->d_nbr_geo, c->d_perm, (float *)F);
  else
    k_overlap<double><<<nb, 256, 0, s>>>(c->d_sys, c->d_p0, c->nsys, N, 2.0 * c->p.a, kspring, c->d_nbr_start,
                                         (const double4_32a *)c->d_nbr_geo, c->d_perm, (double *)F);
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

// vout = M_r vin for the current configuration (sorted order, [N][8]); rows of
// inactive suspensions are left untouched.
pse_status real_apply(pse_ctx *c, const void *vin, void *vout, int mode, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_REAL, s, mode);
  c->nlaunch += 1;
  RealArgs a;
  a.Ntot = c->p.N;
  a.nsys = c->nsys;
  a.len = c->table_len;
  a.k2 = c->table_k2;
  a.inv_dr = 1.0 / c->table_dr;
  a.self_uf = c->self_uf;
  a.self_es = c->self_es;
  c->nlaunch += 1;
  const unsigned nb = (unsigned)ceil_div(c->p.N, 256);
  if (c->prec == PSE_MIXED) {
    k_cell_gather<float><<<nb, 256, 0, s>>>(c->p.N, c->d_cell_list, (const float4 *)vin, (float4 *)c->d_vcell);
    launch_real<float>(c, a, vin, vout, mode, s);
  } else {
    k_cell_gather<double><<<nb, 256, 0, s>>>(c->p.N, c->d_cell_list, (const double4_32a *)vin,
                                             (double4_32a *)c->d_vcell);
    launch_real<double>(c, a, vin, vout, mode, s);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

// vout12 = M_r vin12 for the 11-moment form (12-slot rows, sorted order).
pse_status real_apply11(pse_ctx *c, const void *vin12, void *vout12, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_REAL, s);
  c->nlaunch += 2;
  RealArgs a;
  a.Ntot = c->p.N;
  a.nsys = c->nsys;
  a.len = c->table_len;
  a.k2 = c->table_k2;
  a.inv_dr = 1.0 / c->table_dr;
  a.self_uf = c->self_uf;
  a.self_es = c->self_es;
  constexpr int G = 4;
  const int64_t items = ceil_div(a.Ntot * G, 256);
  const unsigned ng = (unsigned)ceil_div(12 * c->p.N, 256);
  int *q = next_queue(c, s);
  if (c->prec == PSE_MIXED) {
    static std::atomic<int> per_sm{0};
    k_cell_gather12<float><<<ng, 256, 0, s>>>(c->p.N, c->d_cell_list, (const float *)vin12, (float *)c->d_vcell12);
    auto kern = k_real11<float, G>;
    const unsigned grid = persistent_grid(c, kern, 256, 0, items, per_sm);
    kern<<<grid, 256, 0, s>>>(a, c->d_sys, c->d_p0, c->d_active, q, (int)items, c->d_nbr_start,
                              (const float4 *)c->d_nbr_geo, (const float *)vin12, (const float *)c->d_vcell12,
                              (float *)vout12, (const float *)c->d_table, (const float *)c->d_table_rot,
                              (float)c->self_ol);
  } else {
    static std::atomic<int> per_sm{0};
    k_cell_gather12<double><<<ng, 256, 0, s>>>(c->p.N, c->d_cell_list, (const double *)vin12,
                                               (double *)c->d_vcell12);
    auto kern = k_real11<double, G>;
    const unsigned grid = persistent_grid(c, kern, 256, 0, items, per_sm);
    kern<<<grid, 256, 0, s>>>(a, c->d_sys, c->d_p0, c->d_active, q, (int)items, c->d_nbr_start,
                              (const double4_32a *)c->d_nbr_geo, (const double *)vin12,
                              (const double *)c->d_vcell12, (double *)vout12, (const double *)c->d_table,
                              (const double *)c->d_table_rot, c->self_ol);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

}  // namespace pse
