// Device-side control of the Krylov iterations: the FP64 scalar steps of the
// Lanczos square root (Sec. 3.2: tridiagonal T_m, c_m = T_m^{1/2} e1, stopping
// rule |c_m - [c_{m-1}; 0]| / |c_m| <= tol) and of unrestarted GMRES for the
// stresslet constraint (Hessenberg column, Givens rotations, |r|/|b| <= tol,
// back substitution), one thread per suspension (one warp for the Lanczos
// square root).  The dot products they read
// and the scale factors and combination coefficients they write live in the
// per-suspension coefficient blocks; loop control sets a flag (and, inside a
// CUDA graph, the while-node condition) so an iteration needs no host round trip.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "krylov_math.cuh"
#include "pse_internal.cuh"

namespace pse {
namespace {

__global__ void k_lz_start(KDev k) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < k.nsys; q += gridDim.x * blockDim.x) {
    double *cf = k.coef + (size_t)q * COEF_STRIDE;
    double b0 = sqrt(fmax(cf[CO_NRM], 0.0));
    k.l_b0[q] = b0;
    k.l_err[q] = HUGE_VAL;
    k.l_it[q] = 0;
    k.l_capped[q] = 0;
    k.nrows[q] = 0;
    k.active[q] = b0 > 0.0;
    cf[CO_FAC] = b0 > 0.0 ? 1.0 / b0 : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *k.iter = 0;
}

// T^{1/2} e1 of the tridiagonal tridiag(be, al, be) of order n <= LZ_SMEM by one
// warp: the implicit QL sweeps of tql_eigen with d, e and the eigenvectors in
// shared memory, the scalar recurrence evaluated by every lane alike (each step
// reads its operands, synchronises, then lane 0 writes) and each Givens
// rotation of the eigenvector columns spread over the lanes (rows).
constexpr int LZ_SMEM = 48;
__device__ bool tridiag_sqrt_e1_warp(int n, const double *al, const double *be, double *d, double *e, double *Z,
                                     double *cv, int lane) {
  for (int i = lane; i < n; i += 32) {
    d[i] = al[i];
    e[i] = i < n - 1 ? be[i] : 0.0;
  }
  for (int q = lane; q < n * n; q += 32) Z[q] = (q / n == q % n) ? 1.0 : 0.0;
  __syncwarp();
  const double eps = 2.220446049250313e-16;
  bool ok = true;
  for (int l = 0; l < n && ok; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;
      for (; m < n - 1; ++m) {
        const double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (iter > 100) {
        ok = false;
        break;
      }
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double rr = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? rr : -rr));
      double sn = 1.0, cs = 1.0, pp = 0.0;
      bool deflated = false;
      for (int i = m - 1; i >= l; --i) {
        const double ei = e[i], di = d[i], di1 = d[i + 1];
        __syncwarp();  // every lane has read before lane 0 writes
        const double f = sn * ei, b = cs * ei;
        const double hf = hypot(f, g);
        if (hf == 0.0) {  // underflow: split the problem
          if (lane == 0) {
            e[i + 1] = 0.0;
            d[i + 1] = di1 - pp;
            e[m] = 0.0;
          }
          __syncwarp();
          deflated = true;
          break;
        }
        sn = f / hf;
        cs = g / hf;
        g = di1 - pp;
        rr = (di - g) * sn + 2.0 * cs * b;
        pp = sn * rr;
        if (lane == 0) {
          e[i + 1] = hf;
          d[i + 1] = g + pp;
        }
        g = cs * rr - b;
        for (int k = lane; k < n; k += 32) {  // rotate columns i, i+1
          const double zf = Z[k * n + i + 1], zi = Z[k * n + i];
          Z[k * n + i + 1] = sn * zi + cs * zf;
          Z[k * n + i] = cs * zi - sn * zf;
        }
        __syncwarp();
      }
      if (deflated) continue;
      if (lane == 0) {
        d[l] -= pp;
        e[l] = g;
        e[m] = 0.0;
      }
      __syncwarp();
    }
  }
  if (!ok) return false;
  for (int i = lane; i < n; i += 32) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += Z[i * n + k] * sqrt(d[k] > 0.0 ? d[k] : 0.0) * Z[k];
    cv[i] = s;
  }
  __syncwarp();
  return true;
}

// One warp per suspension (the launch has one 32-thread block per suspension).
__global__ void __launch_bounds__(32) k_lz_step(KDev k) {
  __shared__ double s_d[LZ_SMEM], s_e[LZ_SMEM], s_z[LZ_SMEM * LZ_SMEM];
  const int j = *k.iter, m = j + 1, L = k.lmax;
  const int q = blockIdx.x, lane = threadIdx.x;
  if (q >= k.nsys || !k.active[q]) return;
  double *cf = k.coef + (size_t)q * COEF_STRIDE;
  double *al = k.l_alpha + (size_t)q * L, *be = k.l_beta + (size_t)q * L;
  double *cp = k.l_cprev + (size_t)q * L, *cv = k.l_c + (size_t)q * L;
  double *wk = k.l_work + (size_t)q * (2 * L + L * L);
  if (lane == 0) al[j] = cf[CO_H1 + j] + cf[CO_H2 + j];
  __syncwarp();
  const double bj = sqrt(fmax(cf[CO_NRM], 0.0));
  bool ok = true;
  if (j == 0) {
    if (lane == 0) cv[0] = sqrt(fmax(al[0], 0.0));
  } else if (m <= LZ_SMEM) {
    ok = tridiag_sqrt_e1_warp(m, al, be, s_d, s_e, s_z, cv, lane);
  } else if (lane == 0) {  // long recurrences: one thread, work arrays in global memory
    ok = tridiag_sqrt_e1(m, al, be, wk, cv);
  }
  __syncwarp();
  if (lane != 0) return;
  bool stop = !ok;
  double err = k.l_err[q];
  if (ok && j > 0) {
    double num = 0, den = 0;
    for (int i = 0; i < m; ++i) {
      double dv = cv[i] - (i < m - 1 ? cp[i] : 0.0);
      num += dv * dv;
      den += cv[i] * cv[i];
    }
    err = sqrt(num / den);
    if (k.ltol > 0 && err <= k.ltol) stop = true;
  }
  if (!stop) {
    for (int i = 0; i < m; ++i) cp[i] = cv[i];
    if (bj == 0.0 || j == L - 1) stop = true;
  }
  k.l_err[q] = err;
  k.l_it[q] = m;
  if (stop) {
    k.active[q] = 0;
    k.nrows[q] = m;
    const double b0 = k.l_b0[q];
    for (int i = 0; i < m; ++i) cf[CO_Y + i] = b0 * cv[i];
    k.l_capped[q] = !ok || (k.ltol > 0 && !(err <= k.ltol) && m == L);
  } else {
    be[j] = bj;
    cf[CO_FAC] = 1.0 / bj;
  }
}

__global__ void k_gm_start(KDev k) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < k.nsys; q += gridDim.x * blockDim.x) {
    double *cf = k.coef + (size_t)q * COEF_STRIDE;
    double beta = sqrt(fmax(cf[CO_NRM], 0.0));
    k.g_beta[q] = beta;
    k.g_rel[q] = beta > 0.0 ? 1.0 : 0.0;
    k.g_g[(size_t)q * (k.gmax + 1)] = beta;
    k.g_it[q] = 0;
    k.g_capped[q] = 0;
    k.nrows[q] = 0;
    k.active[q] = beta > 0.0;
    cf[CO_FAC] = beta > 0.0 ? 1.0 / beta : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *k.iter = 0;
}

__global__ void k_gm_step(KDev k) {
  const int j = *k.iter, M = k.gmax;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < k.nsys; q += gridDim.x * blockDim.x) {
    if (!k.active[q]) continue;
    double *cf = k.coef + (size_t)q * COEF_STRIDE;
    double *H = k.g_H + (size_t)q * (M + 1) * M, *cs = k.g_cs + (size_t)q * M, *sn = k.g_sn + (size_t)q * M;
    double *g = k.g_g + (size_t)q * (M + 1);
    for (int i = 0; i <= j; ++i) H[i * M + j] = cf[CO_H1 + i] + cf[CO_H2 + i];
    const double hn = sqrt(fmax(cf[CO_NRM], 0.0));
    H[(j + 1) * M + j] = hn;
    for (int i = 0; i < j; ++i) {  // previous rotations
      double a = H[i * M + j], b = H[(i + 1) * M + j];
      H[i * M + j] = cs[i] * a + sn[i] * b;
      H[(i + 1) * M + j] = -sn[i] * a + cs[i] * b;
    }
    double a = H[j * M + j], b = H[(j + 1) * M + j];
    double r = hypot(a, b);
    cs[j] = r == 0 ? 1.0 : a / r;
    sn[j] = r == 0 ? 0.0 : b / r;
    H[j * M + j] = r;
    H[(j + 1) * M + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const double rel = fabs(g[j + 1]) / k.g_beta[q];
    k.g_rel[q] = rel;
    k.g_it[q] = j + 1;
    if (rel <= k.gtol || hn == 0.0 || j == M - 1) {
      k.active[q] = 0;
      k.nrows[q] = j + 1;
      k.g_capped[q] = !(rel <= k.gtol) && j + 1 == M;
      for (int i = j; i >= 0; --i) {  // back substitution H y = g into the combination coefficients
        double sum = g[i];
        for (int l = i + 1; l <= j; ++l) sum -= H[i * M + l] * cf[CO_Y + l];
        cf[CO_Y + i] = sum / H[i * M + i];
      }
    } else {
      cf[CO_FAC] = 1.0 / hn;
    }
  }
}

// flag[0] = (any suspension active); inside a graph also the while condition.
__global__ void k_loop_begin(KDev k, cudaGraphConditionalHandle h, int graph) {
  int any = 0;
  for (int q = threadIdx.x; q < k.nsys; q += blockDim.x) any |= k.active[q];
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    k.flag[0] = any;
    if (graph) cudaGraphSetConditional(h, any ? 1u : 0u);
  }
}

// Advances the iteration counter; the loop continues while a suspension is
// active and fewer than `cap` iterations ran (so it always terminates).
__global__ void k_loop_end(KDev k, int cap, cudaGraphConditionalHandle h, int graph) {
  int any = 0;
  for (int q = threadIdx.x; q < k.nsys; q += blockDim.x) any |= k.active[q];
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    const int j = *k.iter + 1;
    *k.iter = j;
    const int cont = any && j < cap;
    k.flag[0] = cont;
    if (graph) cudaGraphSetConditional(h, cont ? 1u : 0u);
  }
}

__global__ void k_all_active(int nsys, int *active) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nsys; q += gridDim.x * blockDim.x) active[q] = 1;
}

unsigned sys_blocks(const pse_ctx *c) { return (unsigned)std::min<int64_t>(ceil_div(c->nsys, 128), 512); }

}  // namespace

void kd_lz_start(pse_ctx *c, cudaStream_t s) {
  c->nlaunch += 1;
  k_lz_start<<<sys_blocks(c), 128, 0, s>>>(c->kd);
}
void kd_lz_step(pse_ctx *c, cudaStream_t s) {
  c->nlaunch += 1;
  k_lz_step<<<(unsigned)c->nsys, 32, 0, s>>>(c->kd);
}
void kd_gm_start(pse_ctx *c, cudaStream_t s) {
  c->nlaunch += 1;
  k_gm_start<<<sys_blocks(c), 128, 0, s>>>(c->kd);
}
void kd_gm_step(pse_ctx *c, cudaStream_t s) {
  c->nlaunch += 1;
  k_gm_step<<<sys_blocks(c), 128, 0, s>>>(c->kd);
}
void kd_loop_begin(pse_ctx *c, cudaGraphConditionalHandle h, int graph, cudaStream_t s) {
  c->nlaunch += 1;
  k_loop_begin<<<1, 256, 0, s>>>(c->kd, h, graph);
}
void kd_loop_end(pse_ctx *c, int cap, cudaGraphConditionalHandle h, int graph, cudaStream_t s) {
  c->nlaunch += 1;
  k_loop_end<<<1, 256, 0, s>>>(c->kd, cap, h, graph);
}
void kd_all_active(pse_ctx *c, cudaStream_t s) {
  c->nlaunch += 1;
  k_all_active<<<sys_blocks(c), 128, 0, s>>>(c->nsys, c->d_active);
}

}  // namespace pse
