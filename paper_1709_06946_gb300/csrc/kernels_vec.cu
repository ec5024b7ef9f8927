// Vector kernels: user-order <-> sorted-order permutations, in-kernel noise for
// the Lanczos start vector, Krylov inner products and combinations, and the
// position updates of the mid-point scheme (Sec. 3.4).
//
// Inner products in the mixed form: each thread sums its FP32 products over a
// short stretch of the vector, the cross-thread and cross-block sums are FP64.
#include "device_common.cuh"
#include "pse_internal.cuh"

namespace pse {
namespace {

constexpr int DOT_NT = 256, DOT_ROWS = 8;

template <typename T>
__global__ void k_gather_in(int N, const int *perm, const T *F, const T *S, T *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int u = perm[i];
  T *o = out + 8 * (size_t)i;
  for (int m = 0; m < 3; ++m) o[m] = F ? F[3 * (size_t)u + m] : (T)0;
  for (int m = 0; m < 5; ++m) o[3 + m] = S ? S[5 * (size_t)u + m] : (T)0;
}

template <typename T>
__global__ void k_scatter_out(int N, const int *perm, const T *in, T *U, T *E, T scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int u = perm[i];
  const T *v = in + 8 * (size_t)i;
  if (U)
    for (int m = 0; m < 3; ++m) U[3 * (size_t)u + m] = scale * v[m];
  if (E)
    for (int m = 0; m < 5; ++m) E[5 * (size_t)u + m] = scale * v[3 + m];
}

template <typename T>
__global__ void k_gather8(int N, const int *perm, const T *in, T *out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8 * (int64_t)N) return;
  int i = (int)(e >> 3), c = (int)(e & 7);
  out[e] = in[8 * (size_t)perm[i] + c];
}

template <typename T>
__global__ void k_scatter8(int N, const int *perm, const T *in, T *out, T scale) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8 * (int64_t)N) return;
  int i = (int)(e >> 3), c = (int)(e & 7);
  out[8 * (size_t)perm[i] + c] = scale * in[e];
}

template <typename T>
__global__ void k_philox_w1(int N, const int *perm, uint64_t seed, uint64_t counter, T *out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8 * (int64_t)N) return;
  int i = (int)(e >> 3), c = (int)(e & 7);
  T z0, z1;
  normal_pair<T>(seed, counter, 1u, 8ull * (uint64_t)perm[i] + (uint64_t)c, z0, z1);
  out[e] = z0;
}

// partial[b][r] = sum over this block's share of rows[r] . w   (r < nrows <= DOT_ROWS)
template <typename T>
__global__ void k_multidot(const T *__restrict__ rows, int64_t stride, int nrows, int64_t n, const T *__restrict__ w,
                           double *partial) {
  __shared__ double red[DOT_ROWS][DOT_NT / 32];
  T acc[DOT_ROWS];
#pragma unroll
  for (int r = 0; r < DOT_ROWS; ++r) acc[r] = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    T we = w[e];
#pragma unroll
    for (int r = 0; r < DOT_ROWS; ++r)
      if (r < nrows) acc[r] += rows[r * stride + e] * we;
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < DOT_ROWS; ++r) {
    double v = (double)acc[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[r][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < DOT_ROWS) {
    double s = 0;
    for (int k = 0; k < DOT_NT / 32; ++k) s += red[threadIdx.x][k];
    partial[(size_t)blockIdx.x * DOT_ROWS + threadIdx.x] = s;
  }
}

__global__ void k_dot_final(const double *partial, int nblocks, int nrows, double *out) {
  int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (r >= nrows) return;
  double s = 0;
  for (int b = lane; b < nblocks; b += 32) s += partial[(size_t)b * DOT_ROWS + r];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[r] = s;
}

// w[e] = (SET ? 0 : w[e]) + sgn * sum_r coef[r] rows[r][e]
template <typename T, bool SET>
__global__ void k_combine(T *w, const T *__restrict__ rows, int64_t stride, int nrows, int64_t n,
                          const double *__restrict__ coef, T sgn) {
  __shared__ T cs[128];
  for (int r = threadIdx.x; r < nrows && r < 128; r += blockDim.x) cs[r] = (T)coef[r];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int r = 0; r < nrows; ++r) s += cs[r] * rows[r * stride + e];
    w[e] = SET ? sgn * s : w[e] + sgn * s;
  }
}

template <typename T>
__global__ void k_vscale(T *dst, const T *src, T a, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = a * src[e];
}

template <typename T>
__global__ void k_zero_slots(T *v, int N, int slot0, int nslot) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)N * nslot) return;
  int i = (int)(e / nslot), c = (int)(e % nslot);
  v[8 * (size_t)i + slot0 + c] = 0;
}

__device__ __forceinline__ double wrapL(double x, double L) {
  x = fmod(x, L);
  if (x < 0) x += L;
  if (x >= L) x = 0.0;
  return x;
}

template <typename T>
__global__ void k_midpoint(int N, double L, const double *x0, const T *B, double fac, double *xo) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 * (int64_t)N) return;
  int u = (int)(e / 3), d = (int)(e % 3);
  xo[e] = wrapL(x0[e] + fac * (double)B[8 * (size_t)u + d], L);
}

template <typename T>
__global__ void k_final(int N, double L, const int *inv, const double *x0, const T *B, const T *Us, double dt,
                        double *xo) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 * (int64_t)N) return;
  int u = (int)(e / 3), d = (int)(e % 3);
  double U = (double)B[8 * (size_t)u + d] + (double)Us[8 * (size_t)inv[u] + d];
  xo[e] = wrapL(x0[e] + dt * U, L);
}

template <typename T>
__global__ void k_finite(const T *p, int64_t n, int *bad) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite((double)p[e])) {
      atomicOr(bad, 1);
      return;
    }
}

unsigned grid_for(int64_t n, int nt = 256) { return (unsigned)ceil_div(n, nt); }

}  // namespace

#define DISPATCH(c, EXPR_F, EXPR_D) \
  do {                              \
    if ((c)->prec == PSE_MIXED) {   \
      EXPR_F;                       \
    } else {                        \
      EXPR_D;                       \
    }                               \
  } while (0)

pse_status gather_in(pse_ctx *c, const void *F, const void *S, void *vout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int N = (int)c->p.N;
  DISPATCH(c, (k_gather_in<float><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const float *)F, (const float *)S, (float *)vout)),
           (k_gather_in<double><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const double *)F, (const double *)S, (double *)vout)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status scatter_out(pse_ctx *c, const void *vin, void *U, void *E, double scale, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int N = (int)c->p.N;
  DISPATCH(c, (k_scatter_out<float><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const float *)vin, (float *)U, (float *)E, (float)scale)),
           (k_scatter_out<double><<<grid_for(N), 256, 0, s>>>(N, c->d_perm, (const double *)vin, (double *)U, (double *)E, scale)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status gather_user8(pse_ctx *c, const void *user8, void *vout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int N = (int)c->p.N;
  DISPATCH(c, (k_gather8<float><<<grid_for(8 * (int64_t)N), 256, 0, s>>>(N, c->d_perm, (const float *)user8, (float *)vout)),
           (k_gather8<double><<<grid_for(8 * (int64_t)N), 256, 0, s>>>(N, c->d_perm, (const double *)user8, (double *)vout)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status scatter_user8(pse_ctx *c, const void *vin, void *user8, double scale, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int N = (int)c->p.N;
  DISPATCH(c, (k_scatter8<float><<<grid_for(8 * (int64_t)N), 256, 0, s>>>(N, c->d_perm, (const float *)vin, (float *)user8, (float)scale)),
           (k_scatter8<double><<<grid_for(8 * (int64_t)N), 256, 0, s>>>(N, c->d_perm, (const double *)vin, (double *)user8, scale)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status philox_w1(pse_ctx *c, uint64_t seed, uint64_t counter, void *vout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int N = (int)c->p.N;
  DISPATCH(c, (k_philox_w1<float><<<grid_for(8 * (int64_t)N), 256, 0, s>>>(N, c->d_perm, seed, counter, (float *)vout)),
           (k_philox_w1<double><<<grid_for(8 * (int64_t)N), 256, 0, s>>>(N, c->d_perm, seed, counter, (double *)vout)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

// d_out[r] = rows[r] . w for r < nrows (rows contiguous with stride n).
pse_status multidot(pse_ctx *c, const void *rows, int nrows, int64_t n, const void *w, double *d_out, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  int nb = c->dots_blocks;
  double *partial = c->d_dots;
  for (int r0 = 0; r0 < nrows; r0 += DOT_ROWS) {
    int nr = std::min(DOT_ROWS, nrows - r0);
    DISPATCH(c, (k_multidot<float><<<nb, DOT_NT, 0, s>>>((const float *)rows + (size_t)r0 * n, n, nr, n, (const float *)w, partial)),
             (k_multidot<double><<<nb, DOT_NT, 0, s>>>((const double *)rows + (size_t)r0 * n, n, nr, n, (const double *)w, partial)));
    k_dot_final<<<1, 32 * DOT_ROWS, 0, s>>>(partial, nb, nr, d_out + r0);
    c->nlaunch += 2;
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status combine_sub(pse_ctx *c, void *w, const void *rows, int nrows, int64_t n, const double *d_coef, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  unsigned nb = std::min<unsigned>(grid_for(n), 4096);
  for (int r0 = 0; r0 < nrows; r0 += 128) {
    int nr = std::min(128, nrows - r0);
    c->nlaunch += 1;
    DISPATCH(c, (k_combine<float, false><<<nb, 256, 0, s>>>((float *)w, (const float *)rows + (size_t)r0 * n, n, nr, n, d_coef + r0, -1.0f)),
             (k_combine<double, false><<<nb, 256, 0, s>>>((double *)w, (const double *)rows + (size_t)r0 * n, n, nr, n, d_coef + r0, -1.0)));
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status combine_set(pse_ctx *c, void *y, const void *rows, int nrows, int64_t n, const double *d_coef, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  unsigned nb = std::min<unsigned>(grid_for(n), 4096);
  for (int r0 = 0; r0 < nrows; r0 += 128) {
    int nr = std::min(128, nrows - r0);
    c->nlaunch += 1;
    if (r0 == 0) {
      DISPATCH(c, (k_combine<float, true><<<nb, 256, 0, s>>>((float *)y, (const float *)rows, n, nr, n, d_coef, 1.0f)),
               (k_combine<double, true><<<nb, 256, 0, s>>>((double *)y, (const double *)rows, n, nr, n, d_coef, 1.0)));
    } else {
      DISPATCH(c, (k_combine<float, false><<<nb, 256, 0, s>>>((float *)y, (const float *)rows + (size_t)r0 * n, n, nr, n, d_coef + r0, 1.0f)),
               (k_combine<double, false><<<nb, 256, 0, s>>>((double *)y, (const double *)rows + (size_t)r0 * n, n, nr, n, d_coef + r0, 1.0)));
    }
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status vscale(pse_ctx *c, void *dst, const void *src, double a, int64_t n, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  unsigned nb = std::min<unsigned>(grid_for(n), 4096);
  DISPATCH(c, (k_vscale<float><<<nb, 256, 0, s>>>((float *)dst, (const float *)src, (float)a, n)),
           (k_vscale<double><<<nb, 256, 0, s>>>((double *)dst, (const double *)src, a, n)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status vzero_slots(pse_ctx *c, void *v, int slot0, int nslot, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int N = (int)c->p.N;
  DISPATCH(c, (k_zero_slots<float><<<grid_for((int64_t)N * nslot), 256, 0, s>>>((float *)v, N, slot0, nslot)),
           (k_zero_slots<double><<<grid_for((int64_t)N * nslot), 256, 0, s>>>((double *)v, N, slot0, nslot)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status midpoint(pse_ctx *c, const double *x0, const void *B_user, double fac, double *xout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int N = (int)c->p.N;
  DISPATCH(c, (k_midpoint<float><<<grid_for(3 * (int64_t)N), 256, 0, s>>>(N, c->p.L, x0, (const float *)B_user, fac, xout)),
           (k_midpoint<double><<<grid_for(3 * (int64_t)N), 256, 0, s>>>(N, c->p.L, x0, (const double *)B_user, fac, xout)));
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

pse_status final_update(pse_ctx *c, const double *x0, const void *B_user, const void *U_sorted, double dt,
                        double *xout, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_VECTOR, s);
  c->nlaunch += 1;
  int N = (int)c->p.N;
  DISPATCH(c, (k_final<float><<<grid_for(3 * (int64_t)N), 256, 0, s>>>(N, c->p.L, c->d_inv, x0, (const float *)B_user, (const float *)U_sorted, dt, xout)),
           (k_final<double><<<grid_for(3 * (int64_t)N), 256, 0, s>>>(N, c->p.L, c->d_inv, x0, (const double *)B_user, (const double *)U_sorted, dt, xout)));
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
