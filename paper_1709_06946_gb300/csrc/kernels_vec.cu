// Vector kernels: user-order <-> sorted-order permutations, in-kernel noise for
// the Lanczos start vector, Krylov inner products and combinations, and the
// position updates of the mid-point scheme (Sec. 3.4).
//
// Inner products in the mixed form: each thread sums its FP32 products over a
// short stretch of the vector, the cross-thread and cross-block sums are FP64.
// Inner products and combinations are per suspension: every block covers one
// chunk of one suspension's vector, results and coefficients live at
// d_coef[s * COEF_STRIDE + ...], and suspensions marked inactive are skipped.
#include <algorithm>

#include "device_common.cuh"
#include "pse_internal.cuh"

namespace pse {
namespace {

constexpr int DOT_NT = 256, DOT_ROWS = 8;

template <typename T>
__global__ void k_gather_in(int64_t N, const int *perm, const T *F, const T *S, T *out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int u = perm[i];
  T *o = out + 8 * (size_t)i;
  for (int m = 0; m < 3; ++m) o[m] = F ? F[3 * (size_t)u + m] : (T)0;
  for (int m = 0; m < 5; ++m) o[3 + m] = S ? S[5 * (size_t)u + m] : (T)0;
}

template <typename T>
__global__ void k_scatter_out(int64_t N, const int *perm, const T *in, T *U, T *E, T scale) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int u = perm[i];
  const T *v = in + 8 * (size_t)i;
  if (U)
    for (int m = 0; m < 3; ++m) U[3 * (size_t)u + m] = scale * v[m];
  if (E)
    for (int m = 0; m < 5; ++m) E[5 * (size_t)u + m] = scale * v[3 + m];
}

// 12-slot sorted rows [F(3), L(3), S(5), 0] from user-order arrays (any may be NULL: zero).
template <typename T>
__global__ void k_gather12(int64_t N, const int *perm, const T *F, const T *L, const T *S, T *out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t u = perm[i];
  T *o = out + 12 * (size_t)i;
  for (int m = 0; m < 3; ++m) o[m] = F ? F[3 * u + m] : (T)0;
  for (int m = 0; m < 3; ++m) o[3 + m] = L ? L[3 * u + m] : (T)0;
  for (int m = 0; m < 5; ++m) o[6 + m] = S ? S[5 * u + m] : (T)0;
  o[11] = (T)0;
}

// user-order U, Omega, E (any may be NULL: not written) from 12-slot sorted rows.
template <typename T>
__global__ void k_scatter12(int64_t N, const int *perm, const T *in, T *U, T *Om, T *E) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t u = perm[i];
  const T *v = in + 12 * (size_t)i;
  if (U)
    for (int m = 0; m < 3; ++m) U[3 * u + m] = v[m];
  if (Om)
    for (int m = 0; m < 3; ++m) Om[3 * u + m] = v[3 + m];
  if (E)
    for (int m = 0; m < 5; ++m) E[5 * u + m] = v[6 + m];
}

template <typename T>
__global__ void k_gather8(int64_t N, const int *perm, const T *in, T *out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8 * N) return;
  int64_t i = e >> 3;
  int c = (int)(e & 7);
  out[e] = in[8 * (size_t)perm[i] + c];
}

template <typename T>
__global__ void k_scatter8(int64_t N, const int *perm, const T *in, T *out, T scale) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8 * N) return;
  int64_t i = e >> 3;
  int c = (int)(e & 7);
  out[8 * (size_t)perm[i] + c] = scale * in[e];
}

// (seed, counter) come from rng[0..2) when rng is given (a captured graph reads them at launch)
template <typename T>
__global__ void k_philox_w1(int64_t N, const int *perm, uint64_t seed, uint64_t counter, const uint64_t *rng, T *out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8 * N) return;
  if (rng) {
    seed = rng[0];
    counter = rng[1];
  }
  int64_t i = e >> 3;
  int c = (int)(e & 7);
  T z0, z1;
  normal_pair<T>(seed, counter, 1u, 8ull * (uint64_t)perm[i] + (uint64_t)c, z0, z1);
  out[e] = z0;
}

// The chunked vector kernels: block b covers VEC_CHUNK elements of the [N][8]
// vectors of one suspension (blocks of suspension s start at blk0[s]).
struct Chunk {
  int s;
  int64_t beg, end;
};
__device__ __forceinline__ Chunk chunk_of(const SysDev *sys, const int *blk0, int nsys) {
  Chunk ch;
  ch.s = find_sys(blk0, nsys, blockIdx.x);
  const SysDev &q = sys[ch.s];
  ch.beg = 8 * q.p0 + (int64_t)(blockIdx.x - q.blk0) * VEC_CHUNK;
  int64_t lim = 8 * (q.p0 + q.N);
  ch.end = ch.beg + VEC_CHUNK < lim ? ch.beg + VEC_CHUNK : lim;
  return ch;
}

struct VecArgs {
  const SysDev *sys;
  const int *blk0, *active;
  int nsys;
};

// 16-byte vectors of the chunked kernels (a chunk holds a multiple of 8 elements
// and starts 32-byte aligned): 4 floats or 2 doubles per access.
template <typename T> struct V16;
template <> struct V16<float> {
  using t = float4;
  static constexpr int n = 4;
  static __device__ __forceinline__ void get(const float4 &v, float a[4]) {
    a[0] = v.x;
    a[1] = v.y;
    a[2] = v.z;
    a[3] = v.w;
  }
  static __device__ __forceinline__ float4 put(const float a[4]) { return make_float4(a[0], a[1], a[2], a[3]); }
};
template <> struct V16<double> {
  using t = double2;
  static constexpr int n = 2;
  static __device__ __forceinline__ void get(const double2 &v, double a[2]) {
    a[0] = v.x;
    a[1] = v.y;
  }
  static __device__ __forceinline__ double2 put(const double a[2]) { return make_double2(a[0], a[1]); }
};

// acc[r] += rows[r0 + r] . w over the block's chunk, r < nr <= DOT_ROWS; each
// thread keeps VEC_UNROLL independent 16-byte loads per row in flight
constexpr int VEC_UNROLL = 4;
template <typename T>
__device__ __forceinline__ void chunk_dots(const Chunk &ch, const T *__restrict__ rows, int64_t stride, int r0, int nr,
                                           const T *__restrict__ w, T acc[DOT_ROWS]) {
  using V = V16<T>;
  using VT = typename V::t;
#pragma unroll
  for (int r = 0; r < DOT_ROWS; ++r) acc[r] = 0;
  const int64_t step = (int64_t)blockDim.x * V::n;
  for (int64_t e0 = ch.beg + (int64_t)threadIdx.x * V::n; e0 < ch.end; e0 += VEC_UNROLL * step) {
    T wv[VEC_UNROLL][V::n];
#pragma unroll
    for (int u = 0; u < VEC_UNROLL; ++u) {
      const int64_t e = e0 + u * step;
      if (e < ch.end) V::get(*(const VT *)(w + e), wv[u]);
      else
#pragma unroll
        for (int i = 0; i < V::n; ++i) wv[u][i] = 0;
    }
#pragma unroll
    for (int r = 0; r < DOT_ROWS; ++r)
      if (r < nr) {
        const T *row = rows + (r0 + r) * stride;
        T x[VEC_UNROLL][V::n];
#pragma unroll
        for (int u = 0; u < VEC_UNROLL; ++u) {
          const int64_t e = e0 + u * step;
          if (e < ch.end) V::get(*(const VT *)(row + e), x[u]);
          else
#pragma unroll
            for (int i = 0; i < V::n; ++i) x[u][i] = 0;
        }
#pragma unroll
        for (int u = 0; u < VEC_UNROLL; ++u)
#pragma unroll
          for (int i = 0; i < V::n; ++i) acc[r] += x[u][i] * wv[u][i];
      }
  }
}

// partial[b * pstride + r0 + r] = block sum of acc[r] (FP64 across threads), r < nr
template <typename T>
__device__ __forceinline__ void block_sums(const T acc[DOT_ROWS], int nr, double *partial, int pstride, int r0,
                                           double red[DOT_ROWS][DOT_NT / 32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < DOT_ROWS; ++r) {
    if (r < nr) {
      double v = (double)acc[r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[r][wid] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < nr) {
    double sum = 0;
    for (int k = 0; k < DOT_NT / 32; ++k) sum += red[threadIdx.x][k];
    partial[(size_t)blockIdx.x * pstride + r0 + threadIdx.x] = sum;
  }
  __syncthreads();
}

// partial[b][r] = sum over block b's chunk of rows[r] . w   (r < nrows <= DOT_ROWS)
template <typename T>
__global__ void k_multidot(VecArgs va, const T *__restrict__ rows, int64_t stride, int nrows,
                           const T *__restrict__ w, double *partial) {
  __shared__ double red[DOT_ROWS][DOT_NT / 32];
  const Chunk ch = chunk_of(va.sys, va.blk0, va.nsys);
  if (!va.active[ch.s]) return;
  T acc[DOT_ROWS];
  chunk_dots(ch, rows, stride, 0, nrows, w, acc);
  block_sums(acc, nrows, partial, DOT_ROWS, 0, red);
}

// out[s * COEF_STRIDE + r] = sum of the partials of suspension s (one block per suspension).
__global__ void k_dot_final(VecArgs va, const double *partial, int nrows, double *out) {
  const int s = blockIdx.x;
  if (!va.active[s]) return;
  int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const int b0 = va.blk0[s], b1 = va.blk0[s + 1];
  double sum = 0;
  for (int b = b0 + lane; b < b1; b += 32) sum += partial[(size_t)b * DOT_ROWS + r];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) out[(size_t)s * COEF_STRIDE + r] = sum;
}

// w[e] = (SET ? 0 : w[e]) + sgn * sum_r coef[s][r] rows[r][e], r < nrows (or nrows_s[s])
template <typename T, bool SET>
__global__ void k_combine(VecArgs va, T *w, const T *__restrict__ rows, int64_t stride, int nrows,
                          const int *__restrict__ nrows_s, const double *__restrict__ coef, T sgn,
                          const int *__restrict__ nrows_dev = nullptr, int add = 0) {
  using V = V16<T>;
  using VT = typename V::t;
  __shared__ T cs[MAX_ROWS];
  const Chunk ch = chunk_of(va.sys, va.blk0, va.nsys);
  if (!va.active[ch.s]) return;
  int nr = nrows_dev ? min(*nrows_dev + add, MAX_ROWS) : nrows;
  if (nrows_s) nr = min(nr, nrows_s[ch.s]);
  const double *cf = coef + (size_t)ch.s * COEF_STRIDE;
  for (int r = threadIdx.x; r < nr; r += blockDim.x) cs[r] = (T)cf[r];
  __syncthreads();
  const int64_t step = (int64_t)blockDim.x * V::n;
  for (int64_t e0 = ch.beg + (int64_t)threadIdx.x * V::n; e0 < ch.end; e0 += VEC_UNROLL * step) {
    T sum[VEC_UNROLL][V::n];
#pragma unroll
    for (int u = 0; u < VEC_UNROLL; ++u)
#pragma unroll
      for (int i = 0; i < V::n; ++i) sum[u][i] = 0;
    for (int r = 0; r < nr; ++r) {
      const T *row = rows + r * stride;
      T x[VEC_UNROLL][V::n];
#pragma unroll
      for (int u = 0; u < VEC_UNROLL; ++u) {
        const int64_t e = e0 + u * step;
        if (e < ch.end) V::get(*(const VT *)(row + e), x[u]);
        else
#pragma unroll
          for (int i = 0; i < V::n; ++i) x[u][i] = 0;
      }
#pragma unroll
      for (int u = 0; u < VEC_UNROLL; ++u)
#pragma unroll
        for (int i = 0; i < V::n; ++i) sum[u][i] += cs[r] * x[u][i];
    }
#pragma unroll
    for (int u = 0; u < VEC_UNROLL; ++u) {
      const int64_t e = e0 + u * step;
      if (e >= ch.end) continue;
      T out[V::n];
      if (SET) {
#pragma unroll
        for (int i = 0; i < V::n; ++i) out[i] = sgn * sum[u][i];
      } else {
        V::get(*(const VT *)(w + e), out);
#pragma unroll
        for (int i = 0; i < V::n; ++i) out[i] += sgn * sum[u][i];
      }
      *(VT *)(w + e) = V::put(out);
    }
  }
}

// partial[b][r] = sum over block b's chunk of rows[r] . w for r < *nrows_dev + add
// (at most MAX_ROWS), eight rows per pass over w.
template <typename T>
__global__ void k_multidot_rows(VecArgs va, const T *__restrict__ rows, int64_t stride, const int *nrows_dev, int add,
                                const T *__restrict__ w, double *partial) {
  __shared__ double red[DOT_ROWS][DOT_NT / 32];
  const Chunk ch = chunk_of(va.sys, va.blk0, va.nsys);
  if (!va.active[ch.s]) return;
  const int nrows = min(*nrows_dev + add, MAX_ROWS);
  for (int r0 = 0; r0 < nrows; r0 += DOT_ROWS) {
    const int nr = min(DOT_ROWS, nrows - r0);
    T acc[DOT_ROWS];
    chunk_dots(ch, rows, stride, r0, nr, w, acc);
    block_sums(acc, nr, partial, MAX_ROWS, r0, red);
  }
}

// out[s * COEF_STRIDE + r] = sum of suspension s's partials, r < *nrows_dev + add (one block per suspension).
__global__ void k_dot_final_rows(VecArgs va, const double *partial, const int *nrows_dev, int add, double *out) {
  const int s = blockIdx.x;
  if (!va.active[s]) return;
  const int nrows = min(*nrows_dev + add, MAX_ROWS);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int b0 = va.blk0[s], b1 = va.blk0[s + 1];
  for (int r = wid; r < nrows; r += nw) {
    double sum = 0;
    for (int b = b0 + lane; b < b1; b += 32) sum += partial[(size_t)b * MAX_ROWS + r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) out[(size_t)s * COEF_STRIDE + r] = sum;
  }
}

// basis row *iter + delta (and vin when given) = coef[s][0] * src
template <typename T>
__global__ void k_vscale_row(VecArgs va, T *basis, int64_t stride, const int *iter, int delta, const T *src, T *vin,
                             const double *__restrict__ coef) {
  using V = V16<T>;
  using VT = typename V::t;
  const Chunk ch = chunk_of(va.sys, va.blk0, va.nsys);
  if (!va.active[ch.s]) return;
  const T f = (T)coef[(size_t)ch.s * COEF_STRIDE];
  T *dst = basis + (int64_t)(*iter + delta) * stride;
  for (int64_t e = ch.beg + (int64_t)threadIdx.x * V::n; e < ch.end; e += (int64_t)blockDim.x * V::n) {
    T x[V::n];
    V::get(*(const VT *)(src + e), x);
#pragma unroll
    for (int i = 0; i < V::n; ++i) x[i] *= f;
    *(VT *)(dst + e) = V::put(x);
    if (vin) *(VT *)(vin + e) = V::put(x);
  }
}

// dst = f * src with f = a, or f = coef[s][0] per suspension when coef is given
template <typename T>
__global__ void k_vscale(VecArgs va, T *dst, const T *src, T a, const double *__restrict__ coef) {
  using V = V16<T>;
  using VT = typename V::t;
  const Chunk ch = chunk_of(va.sys, va.blk0, va.nsys);
  if (!va.active[ch.s]) return;
  const T f = coef ? (T)coef[(size_t)ch.s * COEF_STRIDE] : a;
  for (int64_t e = ch.beg + (int64_t)threadIdx.x * V::n; e < ch.end; e += (int64_t)blockDim.x * V::n) {
    T x[V::n];
    V::get(*(const VT *)(src + e), x);
#pragma unroll
    for (int i = 0; i < V::n; ++i) x[i] *= f;
    *(VT *)(dst + e) = V::put(x);
  }
}

template <typename T>
__global__ void k_zero_slots(T *v, int64_t N, int slot0, int nslot) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * nslot) return;
  int64_t i = e / nslot;
  int c = (int)(e % nslot);
  v[8 * (size_t)i + slot0 + c] = 0;
}

__device__ __forceinline__ double wrapL(double x, double L) {
  if (x >= 0.0 && x < L) return x;  // already inside: fmod would return x itself
  x = fmod(x, L);
  if (x < 0) x += L;
  if (x >= L) x = 0.0;
  return x;
}

template <typename T>
__global__ void k_midpoint(VecArgs va, const int64_t *__restrict__ p0, int64_t N, const double *x0, const T *B,
                           double fac, double *xo) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 * N) return;
  int64_t u = e / 3;
  int d = (int)(e % 3);
  const SysDev &sd = va.sys[find_sys(p0, va.nsys, u)];
  const double x = x0[e] + fac * (double)B[8 * (size_t)u + d];
  xo[e] = sd.def ? x : wrapL(x, sd.L);  // on a deformed lattice the set-up wraps lattice coordinates
}

template <typename T>
__global__ void k_final(VecArgs va, const int64_t *__restrict__ p0, int64_t N, const int *inv, const double *x0,
                        const T *B, const T *Us, double dt, double *xo) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 * N) return;
  int64_t u = e / 3;
  int d = (int)(e % 3);
  const SysDev &sd = va.sys[find_sys(p0, va.nsys, u)];
  double U = (double)B[8 * (size_t)u + d] + (double)Us[8 * (size_t)inv[u] + d];
  const double x = x0[e] + dt * U;
  xo[e] = sd.def ? x : wrapL(x, sd.L);
}

// Positions of a deformed cell (Sec. 2.3.3) wrapped per particle: x = A (A^{-1} x mod L).
__global__ void k_wrap_lattice(VecArgs va, const int64_t *__restrict__ p0, int64_t N, double *x) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= N) return;
  const SysDev &sd = va.sys[find_sys(p0, va.nsys, u)];
  if (!sd.def) return;
  double *xu = x + 3 * u;
  double z[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) z[i] = wrapL(sd.Ai[3 * i] * xu[0] + sd.Ai[3 * i + 1] * xu[1] + sd.Ai[3 * i + 2] * xu[2], sd.L);
#pragma unroll
  for (int i = 0; i < 3; ++i) xu[i] = sd.A[3 * i] * z[0] + sd.A[3 * i + 1] * z[1] + sd.A[3 * i + 2] * z[2];
}

// The direction W of the random finite difference as user-order 8-slot rows
// (slots 0..2, the rest zero): from wt (N x 3) or in-kernel (Philox stream 3,
// index 3 u + d, first normal of the pair).
template <typename T>
__global__ void k_rfd_noise(int64_t N, const T *wt, uint64_t seed, uint64_t counter, T *W8) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8 * N) return;
  const int64_t u = e >> 3;
  const int d = (int)(e & 7);
  T v = (T)0;
  if (d < 3) {
    if (wt) {
      v = wt[3 * u + d];
    } else {
      T z1;
      normal_pair<T>(seed, counter, 3u, 3ull * (uint64_t)u + (uint64_t)d, v, z1);
    }
  }
  W8[e] = v;
}

// x_{k+1} = x_k + dt (U^B + U_0 + fac (R_+ - R_-)), wrapped (all rows user order, slots 0..2).
template <typename T>
__global__ void k_rfd_final(VecArgs va, const int64_t *__restrict__ p0, int64_t N, const double *x0, const T *B,
                            const T *U0, const T *Rp, const T *Rm, double dt, double fac, double *xo) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 * N) return;
  const int64_t u = e / 3;
  const int d = (int)(e % 3);
  const SysDev &sd = va.sys[find_sys(p0, va.nsys, u)];
  const size_t r = 8 * (size_t)u + d;
  const double U = (double)B[r] + (double)U0[r] + fac * ((double)Rp[r] - (double)Rm[r]);
  const double x = x0[e] + dt * U;
  xo[e] = sd.def ? x : wrapL(x, sd.L);
}

template <typename T>
__global__ void k_finite(const T *p, int64_t n, int *bad) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite((double)p[e])) {
      atomicOr(bad, 1);
      return;
    }
}

__global__ void k_clear(int *q) { *q = 0; }

unsigned grid_for(int64_t n, int nt = 256) { return (unsigned)ceil_div(n, nt); }

VecArgs vec_args(const pse_ctx *c) {
  VecArgs v;
  v.sys = c->d_sys;
  v.blk0 = c->d_blk0;
  v.active = c->d_active;
  v.nsys = c->nsys;
  return v;
}

}  // namespace

#define DISPATCH(c, EXPR_F, EXPR_D) \
  do {                              \
    if ((c)->prec == PSE_MIXED) {   \
      EXPR_F;                       \
    } else {                        \
      EXPR_D;                       \
    }                               \
  } while (0)

int *next_queue(pse_ctx *c, cudaStream_t s) {
  int *q = c->d_queue + (c->queue_slot++ & 63);
  k_clear<<<1, 1, 0, s>>>(q);
  return q;
}

pse_status gather_in(pse_ctx *c, const void *F, const void *S, void *vout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  DISPATCH(c, (k_gather_in<float><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const float *)F, (const float *)S, (float *)vout)),
           (k_gather_in<double><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const double *)F, (const double *)S, (double *)vout)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status gather12(pse_ctx *c, const void *F, const void *L, const void *S, void *vout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  DISPATCH(c, (k_gather12<float><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const float *)F, (const float *)L, (const float *)S, (float *)vout)),
           (k_gather12<double><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const double *)F, (const double *)L, (const double *)S, (double *)vout)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status scatter12(pse_ctx *c, const void *vin, void *U, void *Om, void *E, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  DISPATCH(c, (k_scatter12<float><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const float *)vin, (float *)U, (float *)Om, (float *)E)),
           (k_scatter12<double><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const double *)vin, (double *)U, (double *)Om, (double *)E)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status scatter_out(pse_ctx *c, const void *vin, void *U, void *E, double scale, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  DISPATCH(c, (k_scatter_out<float><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const float *)vin, (float *)U, (float *)E, (float)scale)),
           (k_scatter_out<double><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const double *)vin, (double *)U, (double *)E, scale)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status gather_user8(pse_ctx *c, const void *user8, void *vout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  DISPATCH(c, (k_gather8<float><<<grid_for(8 * N), 256, 0, s>>>(N, c->d_perm, (const float *)user8, (float *)vout)),
           (k_gather8<double><<<grid_for(8 * N), 256, 0, s>>>(N, c->d_perm, (const double *)user8, (double *)vout)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status scatter_user8(pse_ctx *c, const void *vin, void *user8, double scale, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  DISPATCH(c, (k_scatter8<float><<<grid_for(8 * N), 256, 0, s>>>(N, c->d_perm, (const float *)vin, (float *)user8, (float)scale)),
           (k_scatter8<double><<<grid_for(8 * N), 256, 0, s>>>(N, c->d_perm, (const double *)vin, (double *)user8, scale)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status philox_w1(pse_ctx *c, uint64_t seed, uint64_t counter, void *vout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  const uint64_t *rng = c->capturing ? c->d_rng : nullptr;
  DISPATCH(c, (k_philox_w1<float><<<grid_for(8 * N), 256, 0, s>>>(N, c->d_perm, seed, counter, rng, (float *)vout)),
           (k_philox_w1<double><<<grid_for(8 * N), 256, 0, s>>>(N, c->d_perm, seed, counter, rng, (double *)vout)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

// coef[s][off + r] = rows[r] . w over suspension s, for r < nrows (rows of length 8N, contiguous).
pse_status multidot(pse_ctx *c, const void *rows, int nrows, const void *w, int off, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  const int64_t n = 8 * c->p.N;
  const unsigned nb = (unsigned)c->nvblk;
  VecArgs va = vec_args(c);
  for (int r0 = 0; r0 < nrows; r0 += DOT_ROWS) {
    int nr = std::min(DOT_ROWS, nrows - r0);
    DISPATCH(c, (k_multidot<float><<<nb, DOT_NT, 0, s>>>(va, (const float *)rows + (size_t)r0 * n, n, nr, (const float *)w, c->d_dots)),
             (k_multidot<double><<<nb, DOT_NT, 0, s>>>(va, (const double *)rows + (size_t)r0 * n, n, nr, (const double *)w, c->d_dots)));
    k_dot_final<<<c->nsys, 32 * DOT_ROWS, 0, s>>>(va, c->d_dots, nr, c->d_coef + off + r0);
    c->nlaunch += 2;
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status multidot_rows(pse_ctx *c, const void *rows, int add, const void *w, int off, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  const int64_t n = 8 * c->p.N;
  VecArgs va = vec_args(c);
  c->nlaunch += 2;
  DISPATCH(c, (k_multidot_rows<float><<<(unsigned)c->nvblk, DOT_NT, 0, s>>>(va, (const float *)rows, n, c->kd.iter, add, (const float *)w, c->d_dots)),
           (k_multidot_rows<double><<<(unsigned)c->nvblk, DOT_NT, 0, s>>>(va, (const double *)rows, n, c->kd.iter, add, (const double *)w, c->d_dots)));
  k_dot_final_rows<<<c->nsys, 256, 0, s>>>(va, c->d_dots, c->kd.iter, add, c->d_coef + off);
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status combine_sub_rows(pse_ctx *c, void *w, const void *rows, int add, int off, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  const int64_t n = 8 * c->p.N;
  VecArgs va = vec_args(c);
  c->nlaunch += 1;
  DISPATCH(c, (k_combine<float, false><<<(unsigned)c->nvblk, 256, 0, s>>>(va, (float *)w, (const float *)rows, n, 0, nullptr, c->d_coef + off, -1.0f, c->kd.iter, add)),
           (k_combine<double, false><<<(unsigned)c->nvblk, 256, 0, s>>>(va, (double *)w, (const double *)rows, n, 0, nullptr, c->d_coef + off, -1.0, c->kd.iter, add)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status vscale_row(pse_ctx *c, void *basis, int delta, const void *src, void *vin, int off, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  const int64_t n = 8 * c->p.N;
  VecArgs va = vec_args(c);
  c->nlaunch += 1;
  DISPATCH(c, (k_vscale_row<float><<<(unsigned)c->nvblk, 256, 0, s>>>(va, (float *)basis, n, c->kd.iter, delta, (const float *)src, (float *)vin, c->d_coef + off)),
           (k_vscale_row<double><<<(unsigned)c->nvblk, 256, 0, s>>>(va, (double *)basis, n, c->kd.iter, delta, (const double *)src, (double *)vin, c->d_coef + off)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

// w -= sum_r coef[s][off + r] rows[r]  (r < nrows)
pse_status combine_sub(pse_ctx *c, void *w, const void *rows, int nrows, int off, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  const int64_t n = 8 * c->p.N;
  const unsigned nb = (unsigned)c->nvblk;
  VecArgs va = vec_args(c);
  for (int r0 = 0; r0 < nrows; r0 += 128) {
    int nr = std::min(128, nrows - r0);
    c->nlaunch += 1;
    DISPATCH(c, (k_combine<float, false><<<nb, 256, 0, s>>>(va, (float *)w, (const float *)rows + (size_t)r0 * n, n, nr, nullptr, c->d_coef + off + r0, -1.0f)),
             (k_combine<double, false><<<nb, 256, 0, s>>>(va, (double *)w, (const double *)rows + (size_t)r0 * n, n, nr, nullptr, c->d_coef + off + r0, -1.0)));
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

// y = sum_r coef[s][off + r] rows[r]  (r < d_nrows[s] <= maxrows <= 128)
pse_status combine_set(pse_ctx *c, void *y, const void *rows, const int *d_nrows, int maxrows, int off,
                       cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  const int64_t n = 8 * c->p.N;
  const unsigned nb = (unsigned)c->nvblk;
  VecArgs va = vec_args(c);
  if (maxrows > MAX_ROWS) {
    c->err = "too many Krylov vectors";
    return PSE_ERR_INVALID_ARG;
  }
  c->nlaunch += 1;
  DISPATCH(c, (k_combine<float, true><<<nb, 256, 0, s>>>(va, (float *)y, (const float *)rows, n, maxrows, d_nrows, c->d_coef + off, 1.0f)),
           (k_combine<double, true><<<nb, 256, 0, s>>>(va, (double *)y, (const double *)rows, n, maxrows, d_nrows, c->d_coef + off, 1.0)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status vscale(pse_ctx *c, void *dst, const void *src, double a, int off, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  const unsigned nb = (unsigned)c->nvblk;
  VecArgs va = vec_args(c);
  const double *cf = off >= 0 ? c->d_coef + off : nullptr;
  DISPATCH(c, (k_vscale<float><<<nb, 256, 0, s>>>(va, (float *)dst, (const float *)src, (float)a, cf)),
           (k_vscale<double><<<nb, 256, 0, s>>>(va, (double *)dst, (const double *)src, a, cf)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status vzero_slots(pse_ctx *c, void *v, int slot0, int nslot, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  DISPATCH(c, (k_zero_slots<float><<<grid_for(N * nslot), 256, 0, s>>>((float *)v, N, slot0, nslot)),
           (k_zero_slots<double><<<grid_for(N * nslot), 256, 0, s>>>((double *)v, N, slot0, nslot)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status midpoint(pse_ctx *c, const double *x0, const void *B_user, double fac, double *xout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  VecArgs va = vec_args(c);
  DISPATCH(c, (k_midpoint<float><<<grid_for(3 * N), 256, 0, s>>>(va, c->d_p0, N, x0, (const float *)B_user, fac, xout)),
           (k_midpoint<double><<<grid_for(3 * N), 256, 0, s>>>(va, c->d_p0, N, x0, (const double *)B_user, fac, xout)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status final_update(pse_ctx *c, const double *x0, const void *B_user, const void *U_sorted, double dt,
                        double *xout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  VecArgs va = vec_args(c);
  DISPATCH(c, (k_final<float><<<grid_for(3 * N), 256, 0, s>>>(va, c->d_p0, N, c->d_inv, x0, (const float *)B_user, (const float *)U_sorted, dt, xout)),
           (k_final<double><<<grid_for(3 * N), 256, 0, s>>>(va, c->d_p0, N, c->d_inv, x0, (const double *)B_user, (const double *)U_sorted, dt, xout)));
  if (c->lattice) {
    c->nlaunch += 1;
    k_wrap_lattice<<<grid_for(N), 256, 0, s>>>(va, c->d_p0, N, xout);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status rfd_noise(pse_ctx *c, const void *wt, uint64_t seed, uint64_t counter, void *W8, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  DISPATCH(c, (k_rfd_noise<float><<<grid_for(8 * N), 256, 0, s>>>(N, (const float *)wt, seed, counter, (float *)W8)),
           (k_rfd_noise<double><<<grid_for(8 * N), 256, 0, s>>>(N, (const double *)wt, seed, counter, (double *)W8)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status rfd_final(pse_ctx *c, const double *x0, const void *B, const void *U0, const void *Rp, const void *Rm,
                     double dt, double fac, double *xout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int64_t N = c->p.N;
  VecArgs va = vec_args(c);
  DISPATCH(c, (k_rfd_final<float><<<grid_for(3 * N), 256, 0, s>>>(va, c->d_p0, N, x0, (const float *)B, (const float *)U0, (const float *)Rp, (const float *)Rm, dt, fac, xout)),
           (k_rfd_final<double><<<grid_for(3 * N), 256, 0, s>>>(va, c->d_p0, N, x0, (const double *)B, (const double *)U0, (const double *)Rp, (const double *)Rm, dt, fac, xout)));
  if (c->lattice) {
    c->nlaunch += 1;
    k_wrap_lattice<<<grid_for(N), 256, 0, s>>>(va, c->d_p0, N, xout);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status check_finite(pse_ctx *c, const void *ptr, int64_t n, bool dbl, int *bad, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  unsigned nb = std::min<unsigned>(grid_for(n), 2048);
  if (dbl) k_finite<double><<<nb, 256, 0, s>>>((const double *)ptr, n, bad);
  else k_finite<float><<<nb, 256, 0, s>>>((const float *)ptr, n, bad);
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

}  // namespace pse
