// C ABI entry points (include/pse.h): handle set-up, the mobility product,
// split Brownian sampling (Lanczos + wave-space noise) and the constrained
// mid-point step.  Krylov scalars (Lanczos tridiagonal, GMRES Hessenberg and
// Givens rotations) are FP64 on the host; vectors live on the device.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "device_common.cuh"
#include "pse_internal.cuh"

namespace pse {
pse_status exclusive_scan(pse_ctx *c, int *buf, int64_t n1, cudaStream_t s);
int64_t scan_tmp_ints(int64_t n1);
}  // namespace pse

using namespace pse;

namespace {

thread_local std::string g_create_err;

void *dalloc(pse_ctx *c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  c->allocs.push_back(p);
  c->dev_bytes += (int64_t)bytes;
  return p;
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device view of a caller array: the pointer itself if it is device memory,
// otherwise a staging buffer (copied in when `in`).
pse_status stage(pse_ctx *c, int slot, const void *p, size_t bytes, bool in, cudaStream_t s, void **dev) {
  if (!p) {
    *dev = nullptr;
    return PSE_OK;
  }
  if (is_device_ptr(p)) {
    *dev = const_cast<void *>(p);
    return PSE_OK;
  }
  if (c->stage_bytes[slot] < bytes) {
    void *q = dalloc(c, bytes);
    if (!q) {
      c->err = "cannot allocate staging buffer";
      return PSE_ERR_OOM;
    }
    c->d_stage[slot] = q;
    c->stage_bytes[slot] = bytes;
  }
  *dev = c->d_stage[slot];
  if (in) PSE_CUDA_TRY(c, cudaMemcpyAsync(*dev, p, bytes, cudaMemcpyHostToDevice, s));
  return PSE_OK;
}

pse_status unstage(pse_ctx *c, void *host, const void *dev, size_t bytes, cudaStream_t s) {
  if (!host || host == dev) return PSE_OK;
  PSE_CUDA_TRY(c, cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
  return PSE_OK;
}

}  // namespace

namespace pse {

cudaEvent_t prof_event(pse_ctx *c) {
  cudaEvent_t e = nullptr;
  if (!c->ev_pool.empty()) {
    e = c->ev_pool.back();
    c->ev_pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  return e;
}

pse_status mobility(pse_ctx *c, const void *vin, void *vout, int mode, int parts, cudaStream_t s) {
  if (parts & PSE_PART_REAL) PSE_TRY(real_apply(c, vin, vout, mode, s));
  if (parts & PSE_PART_WAVE) PSE_TRY(wave_apply(c, vin, vout, mode, (parts & PSE_PART_REAL) != 0, s));
  if (!(parts & PSE_PART_ALL)) PSE_CUDA_TRY(c, cudaMemsetAsync(vout, 0, c->ts * 8 * (size_t)c->p.N, s));
  return PSE_OK;
}

}  // namespace pse

namespace {

// Reads `count` doubles at d_src into h (waits on the stream).
pse_status read_doubles(pse_ctx *c, const double *d_src, int count, double *h, cudaStream_t s) {
  PSE_CUDA_TRY(c, cudaMemcpyAsync(c->h_dots, d_src, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  std::memcpy(h, c->h_dots, sizeof(double) * count);
  return PSE_OK;
}

pse_status write_doubles(pse_ctx *c, double *d_dst, const double *h, int count, cudaStream_t s) {
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));  // h_dots may still be read by an earlier copy
  std::memcpy(c->h_dots, h, sizeof(double) * count);
  PSE_CUDA_TRY(c, cudaMemcpyAsync(d_dst, c->h_dots, sizeof(double) * count, cudaMemcpyHostToDevice, s));
  return PSE_OK;
}

void *row(pse_ctx *c, int r) { return (char *)c->d_basis + (size_t)r * 8 * c->p.N * c->ts; }

// Orthogonalise w against rows 0..j of the basis twice (classical Gram-Schmidt,
// FP64 coefficients); returns the summed coefficients in h and |w|^2 in nrm2.
pse_status cgs2(pse_ctx *c, void *w, int j, std::vector<double> &h, double &nrm2, cudaStream_t s) {
  int64_t n = 8 * c->p.N;
  double *h1 = c->d_coef, *h2 = c->d_coef + 128, *nr = c->d_coef + 256;
  PSE_TRY(multidot(c, c->d_basis, j + 1, n, w, h1, s));
  PSE_TRY(combine_sub(c, w, c->d_basis, j + 1, n, h1, s));
  PSE_TRY(multidot(c, c->d_basis, j + 1, n, w, h2, s));
  PSE_TRY(combine_sub(c, w, c->d_basis, j + 1, n, h2, s));
  PSE_TRY(multidot(c, w, 1, n, w, nr, s));
  std::vector<double> buf(257);
  PSE_TRY(read_doubles(c, c->d_coef, 257, buf.data(), s));
  h.resize(j + 1);
  for (int i = 0; i <= j; ++i) h[i] = buf[i] + buf[128 + i];
  nrm2 = buf[256];
  return PSE_OK;
}

// y = M_r^{1/2} z by Lanczos with full reorthogonalisation (Sec. 3.2); mirrors the
// stopping rule |c_m - [c_{m-1}; 0]| / |c_m| <= tol (tol = 0: fixed maxiter steps).
pse_status lanczos(pse_ctx *c, const void *z, void *y, void *w, double tol, int maxiter, pse_stats *st,
                   cudaStream_t s) {
  int64_t n = 8 * c->p.N;
  double *nr = c->d_coef + 256;
  PSE_TRY(multidot(c, z, 1, n, z, nr, s));
  double b0;
  PSE_TRY(read_doubles(c, nr, 1, &b0, s));
  b0 = std::sqrt(b0);
  if (b0 == 0.0) {
    PSE_CUDA_TRY(c, cudaMemsetAsync(y, 0, c->ts * n, s));
    return PSE_OK;
  }
  PSE_TRY(vscale(c, row(c, 0), z, 1.0 / b0, n, s));
  std::vector<double> alpha, beta, cvec, cprev;
  double err = INFINITY;
  int it = 0;
  for (int j = 0; j < maxiter; ++j) {
    it = j + 1;
    PSE_TRY(real_apply(c, row(c, j), w, M_FULL, s));
    std::vector<double> h;
    double n2;
    PSE_TRY(cgs2(c, w, j, h, n2, s));
    alpha.push_back(h[j]);
    double bj = std::sqrt(std::max(n2, 0.0));
    int m = j + 1;
    cvec.assign(m, 0.0);
    if (j == 0) {
      cvec[0] = std::sqrt(std::max(alpha[0], 0.0));
    } else {
      std::vector<double> d(alpha), e(beta), Z;
      if (!tridiag_eigen(m, d, e, Z)) {
        c->err = "tridiagonal eigen-solver failed";
        return PSE_ERR_NOT_CONVERGED;
      }
      for (int i = 0; i < m; ++i) {
        double sum = 0;
        for (int k = 0; k < m; ++k) sum += Z[(size_t)i * m + k] * std::sqrt(std::max(d[k], 0.0)) * Z[k];
        cvec[i] = sum;
      }
    }
    bool stop = false;
    if (!cprev.empty()) {
      double num = 0, den = 0;
      for (int i = 0; i < m; ++i) {
        double dv = cvec[i] - (i < m - 1 ? cprev[i] : 0.0);
        num += dv * dv;
        den += cvec[i] * cvec[i];
      }
      err = std::sqrt(num / den);
      if (tol > 0 && err <= tol) stop = true;
    }
    if (stop) break;
    cprev = cvec;
    if (bj == 0.0 || j == maxiter - 1) break;
    beta.push_back(bj);
    PSE_TRY(vscale(c, row(c, j + 1), w, 1.0 / bj, n, s));
  }
  std::vector<double> coef(it);
  for (int i = 0; i < it; ++i) coef[i] = b0 * cvec[i];
  PSE_TRY(write_doubles(c, c->d_coef + 384, coef.data(), it, s));
  PSE_TRY(combine_set(c, y, c->d_basis, it, n, c->d_coef + 384, s));
  if (st) {
    st->lanczos_iters = it;
    st->lanczos_change = std::isfinite(err) ? err : 0.0;
  }
  bool capped = tol > 0 && !(err <= tol) && it == maxiter;
  return capped ? PSE_ERR_NOT_CONVERGED : PSE_OK;
}

// Unrestarted GMRES (x0 = 0) for M_ES x = b at the current configuration;
// stops at |r|/|b| <= tol.  b and x hold the stresslet in slots 3..7.
pse_status gmres(pse_ctx *c, const void *b, void *x, void *w, double tol, int maxiter, pse_stats *st,
                 cudaStream_t s) {
  int64_t n = 8 * c->p.N;
  double *nr = c->d_coef + 256;
  PSE_TRY(multidot(c, b, 1, n, b, nr, s));
  double beta;
  PSE_TRY(read_doubles(c, nr, 1, &beta, s));
  beta = std::sqrt(beta);
  if (beta == 0.0) {
    PSE_CUDA_TRY(c, cudaMemsetAsync(x, 0, c->ts * n, s));
    if (st) {
      st->krylov_iters = 0;
      st->krylov_relres = 0;
    }
    return PSE_OK;
  }
  PSE_TRY(vscale(c, row(c, 0), b, 1.0 / beta, n, s));
  int M = maxiter;
  std::vector<double> H((size_t)(M + 1) * M, 0.0), cs(M), sn(M), g(M + 1, 0.0);
  g[0] = beta;
  double rel = 1.0;
  int it = 0;
  for (int j = 0; j < M; ++j) {
    it = j + 1;
    PSE_TRY(mobility(c, row(c, j), w, M_SE, PSE_PART_ALL, s));
    std::vector<double> h;
    double n2;
    PSE_TRY(cgs2(c, w, j, h, n2, s));
    for (int i = 0; i <= j; ++i) H[(size_t)i * M + j] = h[i];
    double hn = std::sqrt(std::max(n2, 0.0));
    H[(size_t)(j + 1) * M + j] = hn;
    for (int i = 0; i < j; ++i) {  // previous rotations
      double a = H[(size_t)i * M + j], bb = H[(size_t)(i + 1) * M + j];
      H[(size_t)i * M + j] = cs[i] * a + sn[i] * bb;
      H[(size_t)(i + 1) * M + j] = -sn[i] * a + cs[i] * bb;
    }
    double a = H[(size_t)j * M + j], bb = H[(size_t)(j + 1) * M + j];
    double r = std::hypot(a, bb);
    cs[j] = r == 0 ? 1.0 : a / r;
    sn[j] = r == 0 ? 0.0 : bb / r;
    H[(size_t)j * M + j] = r;
    H[(size_t)(j + 1) * M + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    rel = std::fabs(g[j + 1]) / beta;
    if (rel <= tol || hn == 0.0) break;
    PSE_TRY(vscale(c, row(c, j + 1), w, 1.0 / hn, n, s));
  }
  std::vector<double> yv(it);
  for (int i = it - 1; i >= 0; --i) {
    double sum = g[i];
    for (int k = i + 1; k < it; ++k) sum -= H[(size_t)i * M + k] * yv[k];
    yv[i] = sum / H[(size_t)i * M + i];
  }
  PSE_TRY(write_doubles(c, c->d_coef + 384, yv.data(), it, s));
  PSE_TRY(combine_set(c, x, c->d_basis, it, n, c->d_coef + 384, s));
  if (st) {
    st->krylov_iters = it;
    st->krylov_relres = rel;
  }
  return rel <= tol ? PSE_OK : (it == M ? PSE_ERR_NOT_CONVERGED : PSE_OK);
}

// Unscaled Brownian slip [M_r^{1/2} w1 + M_w^{1/2} dW2] in sorted order into out.
pse_status sample_sorted(pse_ctx *c, const void *d_w1, const void *d_w2, uint64_t seed, uint64_t counter, void *out,
                         pse_stats *st, cudaStream_t s) {
  if (d_w1) PSE_TRY(gather_user8(c, d_w1, c->d_v[0], s));
  else PSE_TRY(philox_w1(c, seed, counter, c->d_v[0], s));
  pse_status ls = lanczos(c, c->d_v[0], out, c->d_v[1], c->lanczos_tol, c->lanczos_max, st, s);
  if (ls != PSE_OK && ls != PSE_ERR_NOT_CONVERGED) return ls;
  PSE_TRY(wave_noise(c, d_w2, seed, counter, out, s));
  return ls;
}

pse_status check_inputs(pse_ctx *c, const void *p, int64_t n, bool dbl, cudaStream_t s) {
  if (!p) return PSE_OK;
  PSE_CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
  PSE_TRY(check_finite(c, p, n, dbl, c->d_flag, s));
  PSE_CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned_int + 2, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  if (c->h_pinned_int[2]) {
    c->err = "non-finite input";
    return PSE_ERR_NONFINITE;
  }
  return PSE_OK;
}

pse_status step_impl(pse_ctx *c, double *pos, const void *FP, double dt, const void *w1, const void *w2, uint64_t seed,
                     uint64_t stepno, void *S_out, pse_stats *st, cudaStream_t s) {
  const Params &p = c->p;
  int64_t N = p.N;
  size_t vb = c->ts * 8 * N;
  if (!(dt > 0) || !pos) {
    c->err = "dt must be > 0 and pos non-NULL";
    return PSE_ERR_INVALID_ARG;
  }
  void *dpos, *dFP, *dw1, *dw2;
  PSE_TRY(stage(c, 0, pos, sizeof(double) * 3 * N, true, s, &dpos));
  PSE_TRY(stage(c, 1, FP, c->ts * 3 * N, true, s, &dFP));
  PSE_TRY(stage(c, 2, w1, vb, true, s, &dw1));
  PSE_TRY(stage(c, 3, w2, c->ts * 6 * (size_t)p.Ng * p.Ng * p.nkx, true, s, &dw2));
  PSE_TRY(check_inputs(c, dFP, 3 * N, c->prec == PSE_FP64, s));
  pse_stats local{};
  // 1. Brownian slip at x_k (unconstrained), user order, scaled by sqrt(2kT/dt)
  PSE_CUDA_TRY(c, cudaMemcpyAsync(c->d_pos0, dpos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
  PSE_TRY(setup_config(c, c->d_pos0, s));
  pse_status sst = sample_sorted(c, dw1, dw2, seed, stepno, c->d_v[2], &local, s);
  if (sst != PSE_OK && sst != PSE_ERR_NOT_CONVERGED) return sst;
  PSE_TRY(scatter_user8(c, c->d_v[2], c->d_B, std::sqrt(2.0 * p.kT / dt), s));
  // 2. x_{k+1/2} = x_k + dt/2 U^B
  PSE_TRY(midpoint(c, c->d_pos0, c->d_B, 0.5 * dt, c->d_posh, s));
  PSE_TRY(setup_config(c, c->d_posh, s));
  // 3. M_ES S = -E^B - M_EF F^P at x_{k+1/2}
  PSE_TRY(gather_user8(c, c->d_B, c->d_v[2], s));
  PSE_TRY(vscale(c, c->d_v[2], c->d_v[2], -1.0, 8 * N, s));
  if (dFP) {
    PSE_TRY(gather_in(c, dFP, nullptr, c->d_v[3], s));
    PSE_TRY(mobility(c, c->d_v[3], c->d_v[4], M_FULL, PSE_PART_ALL, s));
    PSE_TRY(combine_sub(c, c->d_v[2], c->d_v[4], 1, 8 * N, c->d_coef + 510, s));  // coef[510] = 1
  }
  PSE_TRY(vzero_slots(c, c->d_v[2], 0, 3, s));
  pse_status gst = gmres(c, c->d_v[2], c->d_v[5], c->d_v[1], c->krylov_tol, c->krylov_max, &local, s);
  if (gst != PSE_OK && gst != PSE_ERR_NOT_CONVERGED) return gst;
  PSE_TRY(vzero_slots(c, c->d_v[5], 0, 3, s));
  // 4. U = U^B + M_UF F^P + M_US S;  x_{k+1} = x_k + dt U
  if (dFP) {
    PSE_TRY(gather_in(c, dFP, nullptr, c->d_v[3], s));
    PSE_TRY(combine_sub(c, c->d_v[3], c->d_v[5], 1, 8 * N, c->d_coef + 511, s));  // coef[511] = -1
  } else {
    PSE_CUDA_TRY(c, cudaMemcpyAsync(c->d_v[3], c->d_v[5], vb, cudaMemcpyDeviceToDevice, s));
  }
  PSE_TRY(mobility(c, c->d_v[3], c->d_v[4], M_FSU, PSE_PART_ALL, s));
  PSE_TRY(final_update(c, c->d_pos0, c->d_B, c->d_v[4], dt, (double *)dpos, s));
  PSE_TRY(unstage(c, pos, dpos, sizeof(double) * 3 * N, s));
  if (S_out) {
    void *dS;
    PSE_TRY(stage(c, 1, S_out, c->ts * 5 * N, false, s, &dS));
    PSE_TRY(scatter_out(c, c->d_v[5], nullptr, dS, 1.0, s));
    PSE_TRY(unstage(c, S_out, dS, c->ts * 5 * N, s));
  }
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  local.neighbor_pairs = c->npairs;
  if (st) *st = local;
  return (sst == PSE_ERR_NOT_CONVERGED || gst == PSE_ERR_NOT_CONVERGED) ? PSE_ERR_NOT_CONVERGED : PSE_OK;
}

pse_status create_impl(pse_ctx *c, const pse_options &o) {
  Params &p = c->p;
  if (choose_params(p, o, c->err)) return PSE_ERR_INVALID_ARG;
  if (p.N > 200000000LL) {
    c->err = "N too large for 32-bit particle indices";
    return PSE_ERR_INVALID_ARG;
  }
  c->lanczos_max = o.lanczos_maxiter > 0 ? o.lanczos_maxiter : 100;
  c->krylov_max = o.krylov_maxiter > 0 ? o.krylov_maxiter : 50;
  c->lanczos_max = std::min(c->lanczos_max, 120);
  c->krylov_max = std::min(c->krylov_max, 120);
  c->lanczos_tol = o.lanczos_tol < 0 ? p.tol : o.lanczos_tol;
  c->krylov_tol = o.krylov_tol < 0 ? p.tol : o.krylov_tol;
  PSE_CUDA_TRY(c, cudaGetDevice(&c->device));
  const size_t ts = c->ts;
  const int64_t N = p.N;
  c->ntiles = (int64_t)p.ntile[0] * p.ntile[1] * p.ntile[2];
  c->ncells = (int64_t)p.nc * p.nc * p.nc;
  // real-space table
  RealTable t;
  int ppa = o.table_points > 0 ? o.table_points : (c->prec == PSE_MIXED ? 1024 : 2048);
  build_real_table(p, ppa, t);
  c->table_len = t.len;
  c->table_k2 = t.k2;
  c->table_dr = t.dr;
  c->self_uf = t.self_uf;
  c->self_es = t.self_es;
  bool fail = false;
  auto A = [&](size_t bytes) {
    void *q = dalloc(c, bytes);
    if (!q) fail = true;
    return q;
  };
  c->d_table = A(ts * 8 * (size_t)t.len);
  c->d_posw = (double *)A(sizeof(double) * 3 * N);
  c->d_tile_key = (int *)A(sizeof(int) * N);
  c->d_cell_key = (int *)A(sizeof(int) * N);
  c->d_perm = (int *)A(sizeof(int) * N);
  c->d_inv = (int *)A(sizeof(int) * N);
  c->d_tile_start = (int *)A(sizeof(int) * (c->ntiles + 1));
  c->d_tile_cur = (int *)A(sizeof(int) * (c->ntiles + 1));
  c->d_cell_start = (int *)A(sizeof(int) * (c->ncells + 1));
  c->d_cell_cur = (int *)A(sizeof(int) * (c->ncells + 1));
  c->d_cell_list = (int *)A(sizeof(int) * N);
  c->d_nbr_start = (int *)A(sizeof(int) * (N + 1));
  double dens = N / p.V();
  double mean_nbr = 4.0 / 3.0 * M_PI * p.rcut * p.rcut * p.rcut * dens;
  c->nbr_slots = (int)std::min<double>(N, (std::ceil((1.4 * mean_nbr + 24) / 8.0) * 8.0));
  c->nbr_slots = std::max(c->nbr_slots, 8);
  c->nbr_cap = (int64_t)c->nbr_slots * N;
  c->d_nbr = (int *)A(sizeof(int) * (size_t)c->nbr_cap);
  c->d_nbr_tot = (unsigned long long *)A(2 * sizeof(unsigned long long));
  c->d_sp_i0 = A(sizeof(int4) * N);
  c->d_sp_d0 = A(4 * ts * N);
  c->d_rs = A(4 * ts * N);
  int64_t big = std::max<int64_t>(std::max<int64_t>(c->ntiles, c->ncells), N) + 1;
  c->d_scan_tmp = (int *)A(sizeof(int) * (size_t)scan_tmp_ints(big));
  c->d_flag = (int *)A(sizeof(int) * 4);
  size_t n3 = (size_t)p.Ng * p.Ng * p.Ng, nk = (size_t)p.Ng * p.Ng * p.nkx;
  if (8 * n3 > (size_t)2147483647) {
    c->err = "FFT grid too large";
    return PSE_ERR_INVALID_ARG;
  }
  c->d_grid = A(ts * 8 * n3);
  c->d_cgrid = A(2 * ts * 8 * nk);
  for (int i = 0; i < 6; ++i) c->d_v[i] = A(ts * 8 * N);
  c->d_B = A(ts * 8 * N);
  c->d_basis = A(ts * 8 * N * (size_t)(std::max(c->lanczos_max, c->krylov_max) + 1));
  c->dots_blocks = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(8 * N, 256), 1), 1024);
  c->d_dots = (double *)A(sizeof(double) * 8 * c->dots_blocks);
  c->d_coef = (double *)A(sizeof(double) * 512);
  c->d_pos0 = (double *)A(sizeof(double) * 3 * N);
  c->d_posh = (double *)A(sizeof(double) * 3 * N);
  if (fail) {
    c->err = "device allocation failed (" + std::to_string(c->dev_bytes) + " bytes so far)";
    return PSE_ERR_OOM;
  }
  PSE_CUDA_TRY(c, cudaMallocHost((void **)&c->h_dots, sizeof(double) * 512));
  PSE_CUDA_TRY(c, cudaMallocHost((void **)&c->h_pinned_int, sizeof(int) * 8));
  // table to device in the working precision
  if (c->prec == PSE_MIXED) {
    std::vector<float> f(t.v.begin(), t.v.end());
    PSE_CUDA_TRY(c, cudaMemcpy(c->d_table, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice));
  } else {
    PSE_CUDA_TRY(c, cudaMemcpy(c->d_table, t.v.data(), sizeof(double) * t.v.size(), cudaMemcpyHostToDevice));
  }
  double consts[2] = {1.0, -1.0};
  PSE_CUDA_TRY(c, cudaMemcpy(c->d_coef + 510, consts, sizeof(consts), cudaMemcpyHostToDevice));
  // cuFFT plans (shared work area)
  int n[3] = {p.Ng, p.Ng, p.Ng};
  size_t work = 0;
  const int batches_r2c[2] = {5, 8}, batches_c2r[3] = {3, 5, 8};
  cufftType tr = c->prec == PSE_MIXED ? CUFFT_R2C : CUFFT_D2Z, tc = c->prec == PSE_MIXED ? CUFFT_C2R : CUFFT_Z2D;
  for (int b : batches_r2c) {
    size_t ws = 0;
    PSE_CUFFT_TRY(c, cufftCreate(&c->plan_r2c[b]));
    PSE_CUFFT_TRY(c, cufftSetAutoAllocation(c->plan_r2c[b], 0));
    PSE_CUFFT_TRY(c, cufftMakePlanMany(c->plan_r2c[b], 3, n, nullptr, 1, (int)n3, nullptr, 1, (int)nk, tr, b, &ws));
    work = std::max(work, ws);
  }
  for (int b : batches_c2r) {
    size_t ws = 0;
    PSE_CUFFT_TRY(c, cufftCreate(&c->plan_c2r[b]));
    PSE_CUFFT_TRY(c, cufftSetAutoAllocation(c->plan_c2r[b], 0));
    PSE_CUFFT_TRY(c, cufftMakePlanMany(c->plan_c2r[b], 3, n, nullptr, 1, (int)nk, nullptr, 1, (int)n3, tc, b, &ws));
    work = std::max(work, ws);
  }
  c->d_fft_work = A(work);
  if (fail) {
    c->err = "cannot allocate cuFFT work area";
    return PSE_ERR_OOM;
  }
  for (int b : batches_r2c) PSE_CUFFT_TRY(c, cufftSetWorkArea(c->plan_r2c[b], c->d_fft_work));
  for (int b : batches_c2r) PSE_CUFFT_TRY(c, cufftSetWorkArea(c->plan_c2r[b], c->d_fft_work));
  for (int b : batches_r2c) c->plan_ok[b] = true;
  for (int b : batches_c2r) c->plan_ok[b] = true;
  PSE_CUDA_TRY(c, cudaDeviceSynchronize());
  return PSE_OK;
}

void resolve_profile(pse_ctx *c) {
  for (auto &q : c->pending) {
    cudaEventSynchronize(q.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) c->prof_ms[q.stage] += ms;
    c->ev_pool.push_back(q.a);
    c->ev_pool.push_back(q.b);
  }
  c->pending.clear();
  cudaGetLastError();
}

void destroy_impl(pse_ctx *c) {
  resolve_profile(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
  for (int b = 0; b < 9; ++b) {
    if (c->plan_r2c[b]) cufftDestroy(c->plan_r2c[b]);
    if (c->plan_c2r[b]) cufftDestroy(c->plan_c2r[b]);
  }
  for (void *q : c->allocs) cudaFree(q);
  if (c->h_dots) cudaFreeHost(c->h_dots);
  if (c->h_pinned_int) cudaFreeHost(c->h_pinned_int);
  c->allocs.clear();
}

}  // namespace

extern "C" {

void pse_default_options(pse_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->rule = PSE_RULE_STRICT;
  o->lanczos_tol = -1.0;
  o->krylov_tol = -1.0;
  o->lanczos_maxiter = 100;
  o->krylov_maxiter = 50;
}

pse_status pse_create(pse_handle *out, int64_t N, double L, double a, double eta, double kT, double xi, double tol,
                      pse_precision prec, const pse_options *opt) {
  if (!out) return PSE_ERR_INVALID_ARG;
  *out = nullptr;
  if (prec != PSE_MIXED && prec != PSE_FP64) {
    g_create_err = "unknown precision";
    return PSE_ERR_INVALID_ARG;
  }
  pse_options o;
  pse_default_options(&o);
  if (opt) o = *opt;
  pse_ctx *c = new (std::nothrow) pse_ctx();
  if (!c) return PSE_ERR_OOM;
  c->prec = prec;
  c->ts = prec == PSE_MIXED ? 4 : 8;
  c->opt = o;
  Params &p = c->p;
  p.ts = (int)c->ts;
  p.N = N;
  p.L = L;
  p.a = a;
  p.eta = eta;
  p.kT = kT;
  p.xi = xi;
  p.tol = tol;
  pse_status st = create_impl(c, o);
  if (st != PSE_OK) {
    g_create_err = c->err;
    destroy_impl(c);
    delete c;
    return st;
  }
  *out = c;
  return PSE_OK;
}

pse_status pse_destroy(pse_handle h) {
  if (!h) return PSE_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  destroy_impl(h);
  delete h;
  return PSE_OK;
}

pse_status pse_get_info(pse_handle h, pse_info *o) {
  if (!h || !o) return PSE_ERR_INVALID_ARG;
  const Params &p = h->p;
  std::memset(o, 0, sizeof(*o));
  o->N = p.N;
  o->L = p.L;
  o->a = p.a;
  o->eta = p.eta;
  o->kT = p.kT;
  o->xi = p.xi;
  o->tol = p.tol;
  o->precision = h->prec;
  o->rule = p.rule;
  o->rcut = p.rcut;
  o->kcut = p.kcut;
  o->h = p.h;
  o->eta_g = p.eta_g;
  o->m = p.m;
  o->Ng = p.Ng;
  o->P = p.P;
  o->cells_per_side = p.nc;
  for (int d = 0; d < 3; ++d) o->tile[d] = p.tile[d];
  o->table_len = h->table_len;
  o->table_dr = h->table_dr;
  o->device_bytes = h->dev_bytes;
  return PSE_OK;
}

pse_status pse_mobility_apply_parts(pse_handle h, const double *pos, const void *F, const void *S, void *U, void *E,
                                    int32_t parts, pse_stream stream) {
  if (!h || !pos) return PSE_ERR_INVALID_ARG;
  if (parts < 1 || parts > 3) {
    h->err = "parts must be PSE_PART_REAL, PSE_PART_WAVE or PSE_PART_ALL";
    return PSE_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  pse_ctx *c = h;
  int64_t N = c->p.N;
  void *dpos, *dF, *dS, *dU, *dE;
  PSE_TRY(stage(c, 0, pos, sizeof(double) * 3 * N, true, s, &dpos));
  PSE_TRY(stage(c, 1, F, c->ts * 3 * N, true, s, &dF));
  PSE_TRY(stage(c, 2, S, c->ts * 5 * N, true, s, &dS));
  PSE_TRY(stage(c, 3, U, c->ts * 3 * N, false, s, &dU));
  PSE_TRY(stage(c, 4, E, c->ts * 5 * N, false, s, &dE));
  PSE_TRY(setup_config(c, (const double *)dpos, s));
  PSE_TRY(gather_in(c, dF, dS, c->d_v[0], s));
  int mode = M_FULL;
  if (!E) mode = M_FSU;
  else if (!dF && !U) mode = M_SE;
  PSE_TRY(mobility(c, c->d_v[0], c->d_v[1], mode, parts, s));
  PSE_TRY(scatter_out(c, c->d_v[1], dU, dE, 1.0, s));
  PSE_TRY(unstage(c, U, dU, c->ts * 3 * N, s));
  PSE_TRY(unstage(c, E, dE, c->ts * 5 * N, s));
  if ((U && U != dU) || (E && E != dE)) PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  return PSE_OK;
}

pse_status pse_mobility_apply(pse_handle h, const double *pos, const void *F, const void *S, void *U, void *E,
                              pse_stream stream) {
  return pse_mobility_apply_parts(h, pos, F, S, U, E, PSE_PART_ALL, stream);
}

pse_status pse_brownian_sample(pse_handle h, const double *pos, double dt, uint64_t seed, uint64_t counter,
                               const void *w1, const void *w2, void *UB, void *EB, pse_stats *stats,
                               pse_stream stream) {
  if (!h || !pos || !(dt > 0)) return PSE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  pse_ctx *c = h;
  const Params &p = c->p;
  int64_t N = p.N;
  void *dpos, *dw1, *dw2, *dU, *dE;
  PSE_TRY(stage(c, 0, pos, sizeof(double) * 3 * N, true, s, &dpos));
  PSE_TRY(stage(c, 1, w1, c->ts * 8 * N, true, s, &dw1));
  PSE_TRY(stage(c, 2, w2, c->ts * 6 * (size_t)p.Ng * p.Ng * p.nkx, true, s, &dw2));
  PSE_TRY(stage(c, 3, UB, c->ts * 3 * N, false, s, &dU));
  PSE_TRY(stage(c, 4, EB, c->ts * 5 * N, false, s, &dE));
  PSE_TRY(check_inputs(c, dw1, 8 * N, c->prec == PSE_FP64, s));
  PSE_TRY(setup_config(c, (const double *)dpos, s));
  pse_stats local{};
  pse_status st = sample_sorted(c, dw1, dw2, seed, counter, c->d_v[2], &local, s);
  if (st != PSE_OK && st != PSE_ERR_NOT_CONVERGED) return st;
  PSE_TRY(scatter_out(c, c->d_v[2], dU, dE, std::sqrt(2.0 * p.kT / dt), s));
  PSE_TRY(unstage(c, UB, dU, c->ts * 3 * N, s));
  PSE_TRY(unstage(c, EB, dE, c->ts * 5 * N, s));
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  local.neighbor_pairs = c->npairs;
  if (stats) *stats = local;
  return st;
}

pse_status pse_constrained_step(pse_handle h, double *pos, const void *FP, double dt, uint64_t seed, uint64_t step,
                                void *S_out, pse_stats *stats, pse_stream stream) {
  if (!h) return PSE_ERR_INVALID_ARG;
  return step_impl(h, pos, FP, dt, nullptr, nullptr, seed, step, S_out, stats, (cudaStream_t)stream);
}

pse_status pse_constrained_step_noise(pse_handle h, double *pos, const void *FP, double dt, const void *w1,
                                      const void *w2, void *S_out, pse_stats *stats, pse_stream stream) {
  if (!h || !w1 || !w2) return PSE_ERR_INVALID_ARG;
  return step_impl(h, pos, FP, dt, w1, w2, 0, 0, S_out, stats, (cudaStream_t)stream);
}

pse_status pse_set_profiling(pse_handle h, int32_t enable) {
  if (!h) return PSE_ERR_INVALID_ARG;
  resolve_profile(h);
  h->prof_on = enable != 0;
  for (int i = 0; i < PSE_NSTAGES; ++i) {
    h->prof_ms[i] = 0;
    h->prof_calls[i] = 0;
  }
  h->nlaunch = 0;
  h->nfft = 0;
  return PSE_OK;
}

pse_status pse_get_profile(pse_handle h, pse_profile *out) {
  if (!h || !out) return PSE_ERR_INVALID_ARG;
  resolve_profile(h);
  std::memset(out, 0, sizeof(*out));
  for (int i = 0; i < PSE_NSTAGES; ++i) {
    out->ms[i] = h->prof_ms[i];
    out->calls[i] = h->prof_calls[i];
  }
  out->launches = h->nlaunch;
  out->fft_execs = h->nfft;
  return PSE_OK;
}

const char *pse_stage_name(int32_t stage) {
  static const char *names[PSE_NSTAGES] = {"setup", "real", "spread", "fft", "scale", "interp", "noise", "vector"};
  return (stage >= 0 && stage < PSE_NSTAGES) ? names[stage] : "";
}

pse_status pse_sync(pse_handle h) {
  if (!h) return PSE_ERR_INVALID_ARG;
  PSE_CUDA_TRY(h, cudaDeviceSynchronize());
  PSE_CUDA_TRY(h, cudaGetLastError());
  return PSE_OK;
}

const char *pse_status_string(pse_status s) {
  switch (s) {
    case PSE_OK: return "ok";
    case PSE_ERR_INVALID_ARG: return "invalid argument";
    case PSE_ERR_OOM: return "out of device memory";
    case PSE_ERR_CUDA: return "CUDA error";
    case PSE_ERR_NOT_CONVERGED: return "Krylov iteration cap reached";
    case PSE_ERR_NONFINITE: return "non-finite input";
    case PSE_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char *pse_last_error(pse_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
