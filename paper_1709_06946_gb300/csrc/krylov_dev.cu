// Device-side control of the Krylov iterations: the FP64 scalar steps of the
// Lanczos square root (Sec. 3.2: tridiagonal T_m, c_m = T_m^{1/2} e1, stopping
// rule |c_m - [c_{m-1}; 0]| / |c_m| <= tol) and of unrestarted GMRES for the
// stresslet constraint (Hessenberg column, Givens rotations, |r|/|b| <= tol,
// back substitution), one thread per suspension.  The dot products they read
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

__global__ void k_lz_step(KDev k) {
  const int j = *k.iter, m = j + 1, L = k.lmax;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < k.nsys; q += gridDim.x * blockDim.x) {
    if (!k.active[q]) continue;
    double *cf = k.coef + (size_t)q * COEF_STRIDE;
    double *al = k.l_alpha + (size_t)q * L, *be = k.l_beta + (size_t)q * L;
    double *cp = k.l_cprev + (size_t)q * L, *cv = k.l_c + (size_t)q * L;
    double *wk = k.l_work + (size_t)q * (2 * L + L * L);
    al[j] = cf[CO_H1 + j] + cf[CO_H2 + j];
    const double bj = sqrt(fmax(cf[CO_NRM], 0.0));
    bool ok = true;
    if (j == 0) cv[0] = sqrt(fmax(al[0], 0.0));
    else ok = tridiag_sqrt_e1(m, al, be, wk, cv);
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
  k_lz_step<<<sys_blocks(c), 128, 0, s>>>(c->kd);
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
