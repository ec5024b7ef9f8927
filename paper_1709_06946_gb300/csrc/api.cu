// C ABI entry points (include/pse.h): handle set-up, the mobility product,
// split Brownian sampling (Lanczos + wave-space noise) and the constrained
// mid-point step.
//
// A handle holds one suspension (pse_create) or a group of independent
// suspensions (pse_create_batch) that every kernel processes in one launch.
// The Krylov iterations of the suspensions run in lockstep, each with its own
// FP64 scalars on the host (Lanczos tridiagonal, GMRES Hessenberg and Givens
// rotations); a suspension that has converged drops out of the launches.
// Vectors live on the device.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>

#include "device_common.cuh"
#include "pse_internal.cuh"

namespace pse {
pse_status exclusive_scan(pse_ctx *c, int *buf, int64_t n1, cudaStream_t s);
int64_t scan_tmp_ints(int64_t n1);
int64_t layout_neighbours(pse_ctx *c);
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

namespace pse {

// Host-to-device copies read pinned staging buffers; a buffer is rewritten only
// after the stream has passed the copies that read it.
pse_status staging_ready(pse_ctx *c, cudaStream_t s) {
  if (c->h2d_pending) {
    PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
    c->h2d_pending = false;
  }
  return PSE_OK;
}


}  // namespace pse

namespace {

pse_status set_all_active(pse_ctx *c, cudaStream_t s) {
  std::fill(c->h_active.begin(), c->h_active.end(), 1);
  kd_all_active(c, s);
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

// Runs `body` (one Krylov iteration, launched on the stream it is given) until
// the control kernels clear the loop flag, at most `cap` times.  Outside a
// capture this is a host loop that reads the flag (and the active set) after
// every iteration; while the step is being captured it becomes a conditional
// while node whose body graph is captured from a second stream, so the whole
// loop runs on the device.
template <typename Body>
pse_status krylov_loop(pse_ctx *c, int cap, cudaStream_t s, Body &&body) {
  if (!c->capturing) {
    for (int j = 0; j < cap; ++j) {
      PSE_TRY(body(s));
      kd_loop_end(c, cap, 0, 0, s);
      PSE_CUDA_TRY(c, cudaMemcpyAsync(c->h_flag, c->kd.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      PSE_CUDA_TRY(c, cudaMemcpyAsync(c->h_flag + 1, c->d_active, sizeof(int) * c->nsys, cudaMemcpyDeviceToHost, s));
      PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
      c->h2d_pending = false;
      std::copy(c->h_flag + 1, c->h_flag + 1 + c->nsys, c->h_active.begin());
      if (!c->h_flag[0]) break;
    }
    return PSE_OK;
  }
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  cudaGraphConditionalHandle h;
  PSE_CUDA_TRY(c, cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive || !g) {  // an earlier capture error invalidated the sequence
    c->err = "stream capture is not active";
    return PSE_ERR_CUDA;
  }
  PSE_CUDA_TRY(c, cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  kd_loop_begin(c, h, 1, s);
  PSE_CUDA_TRY(c, cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive || !g) {
    c->err = "stream capture is not active";
    return PSE_ERR_CUDA;
  }
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  PSE_CUDA_TRY(c, cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
  PSE_CUDA_TRY(c, cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t body_g = np.conditional.phGraph_out[0];
  PSE_CUDA_TRY(c, cudaStreamBeginCaptureToGraph(c->cap_stream, body_g, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeRelaxed));
  pse_status st = body(c->cap_stream);
  kd_loop_end(c, cap, h, 1, c->cap_stream);
  cudaGraph_t out_g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &out_g);
  PSE_TRY(st);
  PSE_CUDA_TRY(c, e);
  return PSE_OK;
}

// Orthogonalise w against basis rows 0..j (j = the device iteration counter)
// twice (classical Gram-Schmidt, FP64 coefficients), then |w|^2.
pse_status cgs2(pse_ctx *c, void *w, cudaStream_t s) {
  PSE_TRY(multidot_rows(c, c->d_basis, 1, w, CO_H1, s));
  PSE_TRY(combine_sub_rows(c, w, c->d_basis, 1, CO_H1, s));
  PSE_TRY(multidot_rows(c, c->d_basis, 1, w, CO_H2, s));
  PSE_TRY(combine_sub_rows(c, w, c->d_basis, 1, CO_H2, s));
  return multidot(c, w, 1, w, CO_NRM, s);
}

// y = M_r^{1/2} z by Lanczos with full reorthogonalisation (Sec. 3.2), per
// suspension, stopping rule and tridiagonal square root on the device.
pse_status lanczos(pse_ctx *c, const void *z, void *y, void *w, cudaStream_t s) {
  const int cap = c->lanczos_max;
  PSE_TRY(set_all_active(c, s));
  PSE_TRY(multidot(c, z, 1, z, CO_NRM, s));
  kd_lz_start(c, s);
  PSE_TRY(vscale_row(c, c->d_basis, 0, z, c->d_vin, CO_FAC, s));
  PSE_TRY(krylov_loop(c, cap, s, [&](cudaStream_t t) {
    PSE_TRY(real_apply(c, c->d_vin, w, M_FULL, t));
    PSE_TRY(cgs2(c, w, t));
    kd_lz_step(c, t);
    return vscale_row(c, c->d_basis, 1, w, c->d_vin, CO_FAC, t);
  }));
  PSE_TRY(set_all_active(c, s));
  return combine_set(c, y, c->d_basis, c->d_nrows, cap, CO_Y, s);
}

// Unrestarted GMRES (x0 = 0) for M_ES x = b at the current configuration, per
// suspension; stops at |r|/|b| <= tol.  b and x hold the stresslet in slots 3..7.
pse_status gmres(pse_ctx *c, const void *b, void *x, void *w, cudaStream_t s) {
  const int cap = c->krylov_max;
  PSE_TRY(set_all_active(c, s));
  PSE_TRY(multidot(c, b, 1, b, CO_NRM, s));
  kd_gm_start(c, s);
  PSE_TRY(vscale_row(c, c->d_basis, 0, b, c->d_vin, CO_FAC, s));
  PSE_TRY(krylov_loop(c, cap, s, [&](cudaStream_t t) {
    PSE_TRY(mobility(c, c->d_vin, w, M_SE, PSE_PART_ALL, t));
    PSE_TRY(cgs2(c, w, t));
    kd_gm_step(c, t);
    return vscale_row(c, c->d_basis, 1, w, c->d_vin, CO_FAC, t);
  }));
  PSE_TRY(set_all_active(c, s));
  return combine_set(c, x, c->d_basis, c->d_nrows, cap, CO_Y, s);
}

// Unscaled Brownian slip [M_r^{1/2} w1 + M_w^{1/2} dW2] in sorted order into out.
pse_status sample_sorted(pse_ctx *c, const void *d_w1, const void *d_w2, uint64_t seed, uint64_t counter, void *out,
                         cudaStream_t s) {
  if (d_w1) PSE_TRY(gather_user8(c, d_w1, c->d_v[0], s));
  else PSE_TRY(philox_w1(c, seed, counter, c->d_v[0], s));
  PSE_TRY(lanczos(c, c->d_v[0], out, c->d_v[1], s));
  return wave_noise(c, d_w2, seed, counter, out, s);
}

pse_status check_inputs(pse_ctx *c, const void *p, int64_t n, bool dbl, cudaStream_t s) {
  if (!p) return PSE_OK;
  PSE_CUDA_TRY(c, cudaMemsetAsync(c->d_flag + 2, 0, sizeof(int), s));
  PSE_TRY(check_finite(c, p, n, dbl, c->d_flag + 2, s));
  PSE_CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned_int + 2, c->d_flag + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  c->h2d_pending = false;
  if (c->h_pinned_int[2]) {
    c->err = "non-finite input";
    return PSE_ERR_NONFINITE;
  }
  return PSE_OK;
}

// Per-suspension iteration counts and residuals of the last Lanczos / GMRES run
// (read from the device after the stream has been synchronised); returns
// NOT_CONVERGED if a cap was reached.
pse_status read_krylov_stats(pse_ctx *c, bool lz, bool gm, cudaStream_t s) {
  const int ns = c->nsys;
  std::vector<int> it(2 * ns);
  std::vector<double> r(2 * ns);
  PSE_CUDA_TRY(c, cudaMemcpyAsync(it.data(), c->kd.l_it, sizeof(int) * 2 * ns, cudaMemcpyDeviceToHost, s));
  PSE_CUDA_TRY(c, cudaMemcpyAsync(r.data(), c->kd.l_err, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
  PSE_CUDA_TRY(c, cudaMemcpyAsync(r.data() + ns, c->kd.g_rel, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
  std::vector<int> gi(2 * ns);
  PSE_CUDA_TRY(c, cudaMemcpyAsync(gi.data(), c->kd.g_it, sizeof(int) * 2 * ns, cudaMemcpyDeviceToHost, s));
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  bool capped = false;
  for (int q = 0; q < ns; ++q) {
    pse_stats &o = c->sys_stats[q];
    if (lz) {
      o.lanczos_iters = it[q];
      o.lanczos_change = std::isfinite(r[q]) ? r[q] : 0.0;
      capped = capped || it[ns + q];
    }
    if (gm) {
      o.krylov_iters = gi[q];
      o.krylov_relres = r[ns + q];
      capped = capped || gi[ns + q];
    }
  }
  return capped ? PSE_ERR_NOT_CONVERGED : PSE_OK;
}

// Aggregate of the per-suspension statistics (largest iteration counts and
// residuals, total neighbour pairs).
void gather_stats(pse_ctx *c, pse_stats *st) {
  for (int q = 0; q < c->nsys; ++q) c->sys_stats[q].neighbor_pairs = c->npairs_sys.empty() ? 0 : c->npairs_sys[q];
  if (!st) return;
  pse_stats o{};
  for (const pse_stats &q : c->sys_stats) {
    o.lanczos_iters = std::max(o.lanczos_iters, q.lanczos_iters);
    o.krylov_iters = std::max(o.krylov_iters, q.krylov_iters);
    o.lanczos_change = std::max(o.lanczos_change, q.lanczos_change);
    o.krylov_relres = std::max(o.krylov_relres, q.krylov_relres);
  }
  o.neighbor_pairs = c->npairs;
  *st = o;
}

void reset_stats(pse_ctx *c) {
  for (pse_stats &q : c->sys_stats) q = pse_stats{};
}

size_t w2_bytes(const pse_ctx *c) { return c->ts * 6 * (size_t)c->nk_tot; }

// The constrained mid-point step (Sec. 3.4, App. B) from x_k in d_pos0 to
// x_{k+1} in d_posout; S in d_v[5].  Same launches eagerly and under capture.
pse_status step_body(pse_ctx *c, const void *dFP, double dt, const void *dw1, const void *dw2, uint64_t seed,
                     uint64_t stepno, cudaStream_t s) {
  const Params &p = c->p;
  const int64_t N = p.N;
  const size_t vb = c->ts * 8 * N;
  // 1. Brownian slip at x_k (unconstrained), user order, scaled by sqrt(2kT/dt)
  PSE_TRY(setup_config(c, c->d_pos0, s));
  PSE_TRY(sample_sorted(c, dw1, dw2, seed, stepno, c->d_v[2], s));
  PSE_TRY(scatter_user8(c, c->d_v[2], c->d_B, std::sqrt(2.0 * p.kT / dt), s));
  // 2. x_{k+1/2} = x_k + dt/2 U^B
  PSE_TRY(midpoint(c, c->d_pos0, c->d_B, 0.5 * dt, c->d_posh, s));
  PSE_TRY(setup_config(c, c->d_posh, s));
  // 3. M_ES S = -E^B - M_EF F^P at x_{k+1/2}
  PSE_TRY(gather_user8(c, c->d_B, c->d_v[2], s));
  PSE_TRY(vscale(c, c->d_v[2], c->d_v[2], -1.0, -1, s));
  if (dFP) {
    PSE_TRY(gather_in(c, dFP, nullptr, c->d_v[3], s));
    PSE_TRY(mobility(c, c->d_v[3], c->d_v[4], M_FULL, PSE_PART_ALL, s));
    PSE_TRY(combine_sub(c, c->d_v[2], c->d_v[4], 1, CO_ONE, s));
  }
  PSE_TRY(vzero_slots(c, c->d_v[2], 0, 3, s));
  PSE_TRY(gmres(c, c->d_v[2], c->d_v[5], c->d_v[1], s));
  PSE_TRY(vzero_slots(c, c->d_v[5], 0, 3, s));
  // 4. U = U^B + M_UF F^P + M_US S;  x_{k+1} = x_k + dt U
  if (dFP) {
    PSE_TRY(gather_in(c, dFP, nullptr, c->d_v[3], s));
    PSE_TRY(combine_sub(c, c->d_v[3], c->d_v[5], 1, CO_MONE, s));
  } else {
    PSE_CUDA_TRY(c, cudaMemcpyAsync(c->d_v[3], c->d_v[5], vb, cudaMemcpyDeviceToDevice, s));
  }
  PSE_TRY(mobility(c, c->d_v[3], c->d_v[4], dFP ? M_FSU : M_SU, PSE_PART_ALL, s));
  return final_update(c, c->d_pos0, c->d_B, c->d_v[4], dt, c->d_posout, s);
}

// Captures step_body (in-kernel noise read from d_rng, force from d_stage[1] when
// given) as a CUDA graph with the Krylov loops as conditional while nodes.
pse_status capture_step(pse_ctx *c, const void *dFP, double dt) {
  // captured on the handle's own stream (the caller's may be the legacy default
  // stream, which cannot be captured); the graph is launched on the caller's stream
  if (!c->g_stream) PSE_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->g_stream, cudaStreamNonBlocking));
  cudaStream_t s = c->g_stream;
  if (c->g_exec) {
    cudaGraphExecDestroy(c->g_exec);
    c->g_exec = nullptr;
  }
  if (c->g_graph) {
    cudaGraphDestroy(c->g_graph);
    c->g_graph = nullptr;
  }
  if (!c->cap_stream) PSE_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  const bool prof = c->prof_on;
  c->prof_on = false;  // stage events cannot live inside conditional bodies
  PSE_CUDA_TRY(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  c->capturing = true;
  std::fill(c->h_active.begin(), c->h_active.end(), 1);
  pse_status st = PSE_OK;
  cudaError_t e = cudaMemsetAsync(c->d_flag, 0, sizeof(int) * 4, s);
  if (e == cudaSuccess && dFP) st = check_finite(c, dFP, 3 * c->p.N, c->prec == PSE_FP64, c->d_flag + 2, s);
  if (e == cudaSuccess && st == PSE_OK) st = step_body(c, dFP, dt, nullptr, nullptr, 0, 0, s);
  c->capturing = false;
  c->prof_on = prof;
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess || st != PSE_OK || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (st == PSE_OK) {
      c->err = std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
      st = PSE_ERR_CUDA;
    }
    return st;
  }
  c->g_graph = g;
  PSE_CUDA_TRY(c, cudaGraphInstantiate(&c->g_exec, g, 0));
  c->g_dt = dt;
  c->g_force = dFP ? 1 : 0;
  c->g_version = c->layout_version;
  return PSE_OK;
}

// After a graph step: non-finite inputs, neighbour-list overflow (the list grows
// and the step is repeated eagerly), per-suspension pair counts.
pse_status graph_checks(pse_ctx *c, bool *redo, cudaStream_t s) {
  const int ns = c->nsys;
  PSE_CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned_int, c->d_flag, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
  PSE_CUDA_TRY(c, cudaMemcpyAsync(c->h_nbr_tot, c->d_nbr_tot, 2 * sizeof(unsigned long long) * ns,
                                  cudaMemcpyDeviceToHost, s));
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  c->h2d_pending = false;
  *redo = false;
  if (c->h_pinned_int[0]) {
    c->err = "non-finite particle position";
    return PSE_ERR_NONFINITE;
  }
  if (c->h_pinned_int[2]) {
    c->err = "non-finite input";
    return PSE_ERR_NONFINITE;
  }
  c->npairs = 0;
  c->npairs_sys.assign(ns, 0);
  for (int q = 0; q < ns; ++q) {
    c->npairs_sys[q] = (int64_t)c->h_nbr_tot[2 * q];
    c->npairs += c->npairs_sys[q];
  }
  *redo = c->h_pinned_int[1] != 0;  // a list overflowed in one of the two builds
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
  reset_stats(c);
  PSE_TRY(set_all_active(c, s));
  void *dpos, *dFP, *dw1, *dw2;
  PSE_TRY(stage(c, 0, pos, sizeof(double) * 3 * N, true, s, &dpos));
  PSE_TRY(stage(c, 2, w1, vb, true, s, &dw1));
  PSE_TRY(stage(c, 3, w2, w2_bytes(c), true, s, &dw2));
  PSE_CUDA_TRY(c, cudaMemcpyAsync(c->d_pos0, dpos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
  const bool graph = c->opt.use_graph != 0 && !w1 && !w2 && !c->prof_on;
  bool done = false;
  if (graph) {
    // the force always comes from the same buffer so that the captured graph can read it
    dFP = nullptr;
    if (FP) {
      if (c->stage_bytes[1] < c->ts * 3 * N) {
        void *q = dalloc(c, c->ts * 3 * N);
        if (!q) {
          c->err = "cannot allocate staging buffer";
          return PSE_ERR_OOM;
        }
        c->d_stage[1] = q;
        c->stage_bytes[1] = c->ts * 3 * N;
      }
      dFP = c->d_stage[1];
      PSE_CUDA_TRY(c, cudaMemcpyAsync(dFP, FP, c->ts * 3 * N, cudaMemcpyDefault, s));
    }
    if (!c->g_exec || c->g_dt != dt || c->g_force != (dFP ? 1 : 0) || c->g_version != c->layout_version) {
      PSE_CUDA_TRY(c, cudaStreamSynchronize(s));  // inputs staged on s are complete before capture
      pse_status cs = capture_step(c, dFP, dt);
      if (cs != PSE_OK) {  // fall back to host-launched steps for this handle
        cudaGetLastError();
        c->graph_error = c->err;
        c->opt.use_graph = 0;
        PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
        return step_impl(c, pos, FP, dt, w1, w2, seed, stepno, S_out, st, s);
      }
    }
    PSE_TRY(staging_ready(c, s));
    c->h_rng[0] = seed;
    c->h_rng[1] = stepno;
    PSE_CUDA_TRY(c, cudaMemcpyAsync(c->d_rng, c->h_rng, 2 * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    c->h2d_pending = true;
    PSE_CUDA_TRY(c, cudaGraphLaunch(c->g_exec, s));
    c->nlaunch += 1;
    bool redo = false;
    PSE_TRY(graph_checks(c, &redo, s));
    if (redo) ++c->layout_version;  // the eager rerun below grows the lists; recapture next time
    done = !redo;
  }
  if (!done) {
    PSE_TRY(stage(c, 1, FP, c->ts * 3 * N, true, s, &dFP));
    PSE_TRY(check_inputs(c, dFP, 3 * N, c->prec == PSE_FP64, s));
    PSE_TRY(step_body(c, dFP, dt, dw1, dw2, seed, stepno, s));
  }
  PSE_CUDA_TRY(c, cudaMemcpyAsync(dpos, c->d_posout, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
  PSE_TRY(unstage(c, pos, dpos, sizeof(double) * 3 * N, s));
  if (S_out) {
    void *dS;
    PSE_TRY(stage(c, 4, S_out, c->ts * 5 * N, false, s, &dS));
    PSE_TRY(scatter_out(c, c->d_v[5], nullptr, dS, 1.0, s));
    PSE_TRY(unstage(c, S_out, dS, c->ts * 5 * N, s));
  }
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  c->h2d_pending = false;
  pse_status ks = read_krylov_stats(c, true, true, s);
  gather_stats(c, st);
  return ks;
}

// Euler-Maruyama step with a random-finite-difference drift (the alternative to
// the mid-point scheme discussed in Sec. 3.4): the Brownian and deterministic
// velocity from one constrained solve at x_k, and the drift kT div R_FU^{-1} from
// (kT/delta) [R_FU^{-1}(x_k + delta/2 W) - R_FU^{-1}(x_k - delta/2 W)] W, two more
// solves.  Host-launched (not captured).  S_out receives the stresslets of the
// solve at x_k.
pse_status rfd_impl(pse_ctx *c, double *pos, const void *FP, double dt, double delta, const void *w1,
                    const void *w2, const void *wt, uint64_t seed, uint64_t stepno, void *S_out, pse_stats *st,
                    cudaStream_t s) {
  const Params &p = c->p;
  const int64_t N = p.N;
  const size_t vb = c->ts * 8 * N;
  if (!(dt > 0) || !pos || !(delta >= 0) || !std::isfinite(delta)) {
    c->err = "dt must be > 0, delta >= 0 and pos non-NULL";
    return PSE_ERR_INVALID_ARG;
  }
  if (delta == 0) delta = 1e-3 * p.a;
  if (!c->d_rfd) {
    c->d_rfd = dalloc(c, 4 * vb);
    if (!c->d_rfd) {
      c->err = "cannot allocate the RFD work space";
      return PSE_ERR_OOM;
    }
  }
  char *rb = (char *)c->d_rfd;
  void *W8 = rb, *U0 = rb + vb, *Rp = rb + 2 * vb, *Rm = rb + 3 * vb;
  reset_stats(c);
  PSE_TRY(set_all_active(c, s));
  void *dpos, *dFP, *dw1, *dw2, *dwt;
  PSE_TRY(stage(c, 0, pos, sizeof(double) * 3 * N, true, s, &dpos));
  PSE_TRY(stage(c, 1, FP, c->ts * 3 * N, true, s, &dFP));
  PSE_TRY(stage(c, 2, w1, vb, true, s, &dw1));
  PSE_TRY(stage(c, 3, w2, w2_bytes(c), true, s, &dw2));
  PSE_TRY(stage(c, 5, wt, c->ts * 3 * N, true, s, &dwt));
  PSE_CUDA_TRY(c, cudaMemcpyAsync(c->d_pos0, dpos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
  PSE_TRY(check_inputs(c, dFP, 3 * N, c->prec == PSE_FP64, s));
  int kit = 0;
  double krel = 0.0;
  bool capped = false;
  auto solve_stats = [&]() -> pse_status {
    pse_status ks = read_krylov_stats(c, false, true, s);
    capped = capped || ks == PSE_ERR_NOT_CONVERGED;
    for (const pse_stats &q : c->sys_stats) {
      kit += q.krylov_iters;
      krel = std::max(krel, q.krylov_relres);
    }
    return (ks == PSE_OK || ks == PSE_ERR_NOT_CONVERGED) ? PSE_OK : ks;
  };
  // 1. at x_k: slip, constrained solve, U = U^B + M_UF F^P + M_US S
  PSE_TRY(setup_config(c, c->d_pos0, s));
  PSE_TRY(sample_sorted(c, dw1, dw2, seed, stepno, c->d_v[2], s));
  PSE_TRY(scatter_user8(c, c->d_v[2], c->d_B, std::sqrt(2.0 * p.kT / dt), s));
  PSE_TRY(read_krylov_stats(c, true, false, s) == PSE_ERR_CUDA ? PSE_ERR_CUDA : PSE_OK);
  const pse_stats lz0 = c->sys_stats.empty() ? pse_stats{} : c->sys_stats[0];
  PSE_TRY(gather_user8(c, c->d_B, c->d_v[2], s));
  PSE_TRY(vscale(c, c->d_v[2], c->d_v[2], -1.0, -1, s));
  if (dFP) {
    PSE_TRY(gather_in(c, dFP, nullptr, c->d_v[3], s));
    PSE_TRY(mobility(c, c->d_v[3], c->d_v[4], M_FULL, PSE_PART_ALL, s));
    PSE_TRY(combine_sub(c, c->d_v[2], c->d_v[4], 1, CO_ONE, s));
  }
  PSE_TRY(vzero_slots(c, c->d_v[2], 0, 3, s));
  PSE_TRY(gmres(c, c->d_v[2], c->d_v[5], c->d_v[1], s));
  PSE_TRY(vzero_slots(c, c->d_v[5], 0, 3, s));
  PSE_TRY(solve_stats());
  if (S_out) {
    void *dS;
    PSE_TRY(stage(c, 4, S_out, c->ts * 5 * N, false, s, &dS));
    PSE_TRY(scatter_out(c, c->d_v[5], nullptr, dS, 1.0, s));
    PSE_TRY(unstage(c, S_out, dS, c->ts * 5 * N, s));
  }
  if (dFP) {
    PSE_TRY(gather_in(c, dFP, nullptr, c->d_v[3], s));
    PSE_TRY(combine_sub(c, c->d_v[3], c->d_v[5], 1, CO_MONE, s));
  } else {
    PSE_CUDA_TRY(c, cudaMemcpyAsync(c->d_v[3], c->d_v[5], vb, cudaMemcpyDeviceToDevice, s));
  }
  PSE_TRY(mobility(c, c->d_v[3], c->d_v[4], dFP ? M_FSU : M_SU, PSE_PART_ALL, s));
  PSE_TRY(scatter_user8(c, c->d_v[4], U0, 1.0, s));
  // 2. R_FU^{-1}(x_k +- delta/2 W) W, one solve each
  PSE_TRY(rfd_noise(c, dwt, seed, stepno, W8, s));
  for (int side = 0; side < 2; ++side) {
    PSE_TRY(midpoint(c, c->d_pos0, W8, side ? -0.5 * delta : 0.5 * delta, c->d_posh, s));
    PSE_TRY(setup_config(c, c->d_posh, s));
    PSE_TRY(gather_user8(c, W8, c->d_v[0], s));
    PSE_TRY(mobility(c, c->d_v[0], c->d_v[3], M_FULL, PSE_PART_ALL, s));  // (M_UF W, M_EF W)
    PSE_TRY(vscale(c, c->d_v[2], c->d_v[3], -1.0, -1, s));
    PSE_TRY(vzero_slots(c, c->d_v[2], 0, 3, s));
    PSE_TRY(gmres(c, c->d_v[2], c->d_v[5], c->d_v[1], s));
    PSE_TRY(vzero_slots(c, c->d_v[5], 0, 3, s));
    PSE_TRY(solve_stats());
    PSE_TRY(mobility(c, c->d_v[5], c->d_v[4], M_SU, PSE_PART_ALL, s));     // M_US S
    PSE_TRY(combine_sub(c, c->d_v[4], c->d_v[3], 1, CO_MONE, s));           // + M_UF W
    PSE_TRY(scatter_user8(c, c->d_v[4], side ? Rm : Rp, 1.0, s));
  }
  // 3. x_{k+1} = x_k + dt (U^B + U + drift)
  PSE_TRY(rfd_final(c, c->d_pos0, c->d_B, U0, Rp, Rm, dt, p.kT / delta, c->d_posout, s));
  PSE_CUDA_TRY(c, cudaMemcpyAsync(dpos, c->d_posout, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
  PSE_TRY(unstage(c, pos, dpos, sizeof(double) * 3 * N, s));
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  c->h2d_pending = false;
  for (pse_stats &q : c->sys_stats) {
    q.lanczos_iters = lz0.lanczos_iters;
    q.lanczos_change = lz0.lanczos_change;
    q.krylov_iters = kit;
    q.krylov_relres = krel;
  }
  gather_stats(c, st);
  return capped ? PSE_ERR_NOT_CONVERGED : PSE_OK;
}

// Device memory of a handle before it is created (the admission estimate of a
// serving loop); mirrors the allocations of create_group.
int64_t estimate_bytes(const pse_ctx *c) {
  const size_t ts = c->ts;
  int64_t Nt = 0, ntile = 0, ncell = 0, n3 = 0, nk = 0, nbr = 0, vblk = 0;
  for (const Params &q : c->ps) {
    Nt += q.N;
    ntile += (int64_t)q.ntile[0] * q.ntile[1] * q.ntile[2];
    ncell += (int64_t)q.nc * q.nc * q.nc;
    n3 += (int64_t)q.Ng * q.Ng * q.Ng;
    nk += (int64_t)q.Ng * q.Ng * q.nkx;
    double mean = 4.0 / 3.0 * M_PI * q.rcut * q.rcut * q.rcut * q.N / q.V();
    nbr += (int64_t)std::max(8.0, std::ceil((1.4 * mean + 24) / 8.0) * 8.0) * q.N;
    vblk += ceil_div(8 * q.N, VEC_CHUNK);
  }
  int rows = std::max(c->lanczos_max, c->krylov_max) + 1;
  int64_t b = 0;
  b += (int64_t)ts * 8 * 2048 * 16;                 // table (upper bound)
  b += Nt * (24 + 4 * 6 + 16 + 12 * (int64_t)ts);  // positions, keys, perm/inv, cells, records (two orders)
  b += nbr * 4 * (int64_t)ts + (Nt + 1) * 4;
  b += (ntile * (8 + 8 * SUB_BLOCKS) + ncell * 8);
  const int64_t ncomp = c->opt.torque ? 11 : 8;
  b += (int64_t)ts * ncomp * n3 + 2 * (int64_t)ts * ncomp * nk;   // grids and half spectra
  b += (int64_t)ts * 8 * n3;                               // cuFFT work area (upper bound)
  b += (int64_t)ts * 8 * Nt * (7 + rows);                 // vectors and Krylov basis
  b += Nt * 48;                                            // FP64 positions (x_k, x_{k+1/2})
  b += vblk * 8 * MAX_ROWS + (int64_t)c->nsys * (COEF_STRIDE * 8 + 256);
  const int64_t L = c->lanczos_max, M = c->krylov_max;
  b += (int64_t)c->nsys * 8 * (6 * L + L * L + (M + 1) * M + 3 * M + 8);  // Krylov control state
  b += (int64_t)ts * 8 * Nt + 24 * Nt;                                    // current Krylov vector, output positions
  b += (int64_t)ts * 8 * Nt;                                              // real-space input in cell order
  if (c->opt.torque) b += (int64_t)ts * (36 * Nt + 4 * 2048 * 16);     // 12-slot vectors, rotation table
  return b;
}

}  // namespace

// Lattice fields of a suspension's device constants (Sec. 2.3.3): the cube has
// def = 0, A = I and qa = alpha (1, 1, 1, 0, 0, 0).
void pse::fill_lattice(const Params &p, SysDev &d) {
  d.def = p.def;
  const double kf = 2.0 * M_PI / p.L;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      d.A[3 * i + j] = p.A[3 * i + j];
      d.Ai[3 * i + j] = p.Ai[3 * i + j];
      d.Bt[3 * i + j] = kf * p.Ai[3 * j + i];  // (2 pi/L) (A^{-1})^T
      d.Af[3 * i + j] = (float)d.A[3 * i + j];
      d.Btf[3 * i + j] = (float)d.Bt[3 * i + j];
    }
  // G = A^T A: alpha |A d|^2 = alpha d.G d
  double G[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G[3 * i + j] = p.A[i] * p.A[j] + p.A[3 + i] * p.A[3 + j] + p.A[6 + i] * p.A[6 + j];
  const double al = 2.0 * p.xi * p.xi / p.eta_g;
  d.qa[0] = al * G[0];
  d.qa[1] = al * G[4];
  d.qa[2] = al * G[8];
  d.qa[3] = 2.0 * al * G[1];
  d.qa[4] = 2.0 * al * G[2];
  d.qa[5] = 2.0 * al * G[5];
  if (!p.def) {  // exact cube values
    d.qa[0] = d.qa[1] = d.qa[2] = al;
    d.qa[3] = d.qa[4] = d.qa[5] = 0.0;
  }
  d.c_apply = p.sigma() * p.sigma() / (p.V() * p.eta);
  d.c_noise = p.sigma() / std::sqrt(p.eta * p.V());
  d.c_applyf = (float)d.c_apply;
  d.c_noisef = (float)d.c_noise;
  for (int k = 0; k < 6; ++k) d.qaf[k] = (float)d.qa[k];
}

namespace {

// Marks a suspension for the spreading / interpolation kernels specialised for
// 16^3 tiles (mixed precision, P = 5, 6 or 8, at least two tiles per side) and
// counts it in c->n_cubic.
// Whether A^T A couples z with x or y (the 16^3-tile kernels on a deformed
// lattice need the z axis orthogonal to the deformed plane, as in shear and
// planar extension).
bool z_coupled(const double A[9]) {
  const double g13 = A[0] * A[2] + A[3] * A[5] + A[6] * A[8], g23 = A[1] * A[2] + A[4] * A[5] + A[7] * A[8];
  return g13 != 0.0 || g23 != 0.0;
}

void set_cubic(pse_ctx *c, SysDev &d, const Params &p) {
  // P = 10 and deformed lattices only with the default kernels (the optional
  // 16^3 variants have neither)
  const bool defaults = c->opt.wave_kernel == 0;
  bool ok = c->prec == PSE_MIXED && (c->p.P == 5 || c->p.P == 6 || c->p.P == 8 || (c->p.P == 10 && defaults));
  if (c->lattice) ok = ok && defaults && !z_coupled(p.A);
  for (int k = 0; k < 3; ++k) ok = ok && d.T[k] == CUBE_TILE && d.nt[k] >= 2;
  d.cubic = ok ? 1 : 0;
  c->n_cubic += d.cubic;
}

pse_status choose_group(pse_ctx *c, int nsys, const int64_t *N, const double *L, const pse_options &o) {
  c->nsys = nsys;
  c->ps.assign(nsys, c->p);
  int64_t Nt = 0;
  for (int q = 0; q < nsys; ++q) {
    Params &p = c->ps[q];
    p.N = N[q];
    p.L = L[q];
    std::string e;
    if (choose_params(p, o, e)) {
      c->err = nsys > 1 ? "suspension " + std::to_string(q) + ": " + e : e;
      return PSE_ERR_INVALID_ARG;
    }
    Nt += p.N;
  }
  if (Nt > 200000000LL) {
    c->err = "N too large for 32-bit particle indices";
    return PSE_ERR_INVALID_ARG;
  }
  Params shared = c->ps[0];
  shared.N = Nt;
  c->p = shared;
  c->lanczos_max = o.lanczos_maxiter > 0 ? o.lanczos_maxiter : 100;
  c->krylov_max = o.krylov_maxiter > 0 ? o.krylov_maxiter : 50;
  c->lanczos_max = std::min(c->lanczos_max, 120);
  c->krylov_max = std::min(c->krylov_max, 120);
  c->lanczos_tol = o.lanczos_tol < 0 ? shared.tol : o.lanczos_tol;
  c->krylov_tol = o.krylov_tol < 0 ? shared.tol : o.krylov_tol;
  return PSE_OK;
}

pse_status create_group(pse_ctx *c, const pse_options &o) {
  const int ns = c->nsys;
  const size_t ts = c->ts;
  const int64_t N = c->p.N;
  PSE_CUDA_TRY(c, cudaGetDevice(&c->device));
  PSE_CUDA_TRY(c, cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device));
  {
    int optin = 0;
    PSE_CUDA_TRY(c, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    c->smem_optin = optin > 4096 ? (size_t)optin - 4096 : 0;  // room for the kernel's static shared memory
  }
  // per-suspension layout: particles, tiles, cells, half spectra, vector blocks
  c->hs.assign(ns, SysDev{});
  c->n_cubic = 0;
  c->lattice = 0;
  for (int i = 0; i < 9; ++i) c->lattice |= o.deform[i] != 0.0 ? 1 : 0;
  std::vector<int64_t> p0(ns + 1, 0), k0(ns + 1, 0);
  std::vector<int> tile0(ns + 1, 0), blk0(ns + 1, 0);
  int64_t cell_tot = 0;
  for (int q = 0; q < ns; ++q) {
    const Params &p = c->ps[q];
    SysDev &d = c->hs[q];
    d.p0 = p0[q];
    d.N = (int)p.N;
    d.Ng = p.Ng;
    d.nkx = p.nkx;
    d.nc = p.nc;
    for (int k = 0; k < 3; ++k) {
      d.T[k] = p.tile[k];
      d.nt[k] = p.ntile[k];
    }
    set_cubic(c, d, p);
    d.L = p.L;
    d.h = p.h;
    d.cs = p.cs;
    d.inv_h = 1.0 / p.h;
    d.inv_cs = 1.0 / p.cs;
    d.Lf = (float)p.L;
    d.csf = (float)p.cs;
    d.alpha = 2.0 * p.xi * p.xi / p.eta_g;
    d.pref = std::pow(2.0 * p.xi * p.xi / (M_PI * p.eta_g), 1.5);
    d.kfac = 2.0 * M_PI / p.L;
    d.eta_g = p.eta_g;
    d.hf = (float)d.h;
    d.alphaf = (float)d.alpha;
    d.preff = (float)d.pref;
    d.kfacf = (float)d.kfac;
    d.eta_gf = (float)d.eta_g;
    fill_lattice(p, d);
    double mean = 4.0 / 3.0 * M_PI * p.rcut * p.rcut * p.rcut * p.N / p.V();
    d.slots = (int)std::min<double>(std::max<int64_t>(p.N, 8), std::ceil((1.4 * mean + 24) / 8.0) * 8.0);
    d.slots = std::max(d.slots, 8);
    c->npairs_est += (int64_t)(mean * p.N);
    d.tile0 = tile0[q];
    d.cell0 = (int)cell_tot;
    d.k0 = k0[q];
    d.blk0 = blk0[q];
    p0[q + 1] = p0[q] + p.N;
    tile0[q + 1] = tile0[q] + p.ntile[0] * p.ntile[1] * p.ntile[2];
    cell_tot += (int64_t)p.nc * p.nc * p.nc;
    k0[q + 1] = k0[q] + (int64_t)p.Ng * p.Ng * p.nkx;
    blk0[q + 1] = blk0[q] + (int)ceil_div(8 * p.N, VEC_CHUNK);
  }
  if (cell_tot > 1500000000LL || (int64_t)tile0[ns] > 1500000000LL) {
    c->err = "too many cells or tiles";
    return PSE_ERR_INVALID_ARG;
  }
  c->ntiles = tile0[ns];
  c->ncells = cell_tot;
  c->nk_tot = k0[ns];
  c->nvblk = blk0[ns];
  // FFT groups: suspensions with equal grids share one strided batch, [component][suspension][Ng^3]
  std::map<int, std::vector<int>> by_ng;
  for (int q = 0; q < ns; ++q) by_ng[c->ps[q].Ng].push_back(q);
  int64_t g0 = 0, cg0 = 0;
  c->groups.clear();
  for (auto &kv : by_ng) {
    FftGroup g;
    g.Ng = kv.first;
    g.nsys = (int)kv.second.size();
    g.members = kv.second;
    g.grid0 = g0;
    g.cgrid0 = cg0;
    const int64_t n3 = (int64_t)g.Ng * g.Ng * g.Ng, nk = (int64_t)g.Ng * g.Ng * (g.Ng / 2 + 1);
    for (int j = 0; j < g.nsys; ++j) {
      SysDev &d = c->hs[kv.second[j]];
      d.grid0 = g0 + j * n3;
      d.gstride = g.nsys * n3;
      d.cgrid0 = cg0 + j * nk;
      d.cstride = g.nsys * nk;
    }
    const int ncomp = o.torque ? 11 : 8;  // grids per suspension
    g0 += ncomp * g.nsys * n3;
    cg0 += ncomp * g.nsys * nk;
    c->groups.push_back(g);
  }
  c->grid_elems = g0;
  c->cgrid_elems = cg0;
  // real-space table (shared: it depends on a, eta, xi and r_cut only)
  RealTable t;
  int ppa = o.table_points > 0 ? o.table_points : (c->prec == PSE_MIXED ? 1024 : 2048);
  build_real_table(c->p, ppa, t);
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
  c->d_sys = (SysDev *)A(sizeof(SysDev) * ns);
  c->d_p0 = (int64_t *)A(sizeof(int64_t) * (ns + 1));
  c->d_k0 = (int64_t *)A(sizeof(int64_t) * (ns + 1));
  c->d_tile0 = (int *)A(sizeof(int) * (ns + 1));
  c->d_blk0 = (int *)A(sizeof(int) * (ns + 1));
  c->d_active = (int *)A(sizeof(int) * ns);
  c->d_nrows = (int *)A(sizeof(int) * ns);
  c->kd.active = c->d_active;
  c->kd.nrows = c->d_nrows;
  c->d_queue = (int *)A(sizeof(int) * 64);
  c->d_table = A(ts * 8 * (size_t)t.len);
  if (c->prec == PSE_MIXED) {
    c->d_table_e = A(sizeof(float) * 8 * (size_t)t.len);
    c->d_table_u = A(sizeof(float) * 8 * (size_t)t.len);
  }
  c->d_posw = (double *)A(sizeof(double) * 3 * N);
  c->d_tile_key = (int *)A(sizeof(int) * N);
  c->d_cell_key = (int *)A(sizeof(int) * N);
  c->d_perm = (int *)A(sizeof(int) * N);
  c->d_inv = (int *)A(sizeof(int) * N);
  c->d_tile_start = (int *)A(sizeof(int) * (c->ntiles + 1));
  c->d_tile_cur = (int *)A(sizeof(int) * (c->ntiles + 1));
  c->d_fine_start = (int *)A(sizeof(int) * (c->ntiles * SUB_BLOCKS + 1));
  c->d_fine_cur = (int *)A(sizeof(int) * (c->ntiles * SUB_BLOCKS + 1));
  c->d_cell_start = (int *)A(sizeof(int) * (c->ncells + 1));
  c->d_cell_cur = (int *)A(sizeof(int) * (c->ncells + 1));
  c->d_cell_list = (int *)A(sizeof(int) * N);
  c->d_vcell = A(8 * ts * (size_t)N);
  if (o.torque) {
    std::vector<double> rot;
    build_rot_table(c->p, ppa, t.len, rot, &c->self_ol);
    c->d_table_rot = A(ts * 4 * (size_t)t.len);
    if (c->d_table_rot) {
      if (c->prec == PSE_MIXED) {
        std::vector<float> rf(rot.begin(), rot.end());
        PSE_CUDA_TRY(c, cudaMemcpy(c->d_table_rot, rf.data(), sizeof(float) * rf.size(), cudaMemcpyHostToDevice));
      } else {
        PSE_CUDA_TRY(c, cudaMemcpy(c->d_table_rot, rot.data(), sizeof(double) * rot.size(), cudaMemcpyHostToDevice));
      }
    }
    for (int i = 0; i < 2; ++i) c->d_v12[i] = A(12 * ts * (size_t)N);
    c->d_vcell12 = A(12 * ts * (size_t)N);
  }
  c->d_nbr_start = (int *)A(sizeof(int) * (N + 1));
  c->nbr_cap = layout_neighbours(c);
  if ((double)c->nbr_cap > 2.0e9) {
    c->err = "neighbour list exceeds 2^31 entries";
    return PSE_ERR_INVALID_ARG;
  }
  c->d_nbr_geo = A(4 * ts * (size_t)c->nbr_cap);
  c->d_nbr_tot = (unsigned long long *)A(2 * sizeof(unsigned long long) * ns);
  c->d_sp_i0 = A(sizeof(int4) * N);
  c->d_sp_d0 = A(4 * ts * N);
  c->d_rs = A(4 * ts * N);
  c->d_rs_cell = A(4 * ts * N);
  int64_t big = std::max<int64_t>(std::max<int64_t>(c->ntiles * SUB_BLOCKS, c->ncells), N) + 1;
  c->scan_cap = scan_tmp_ints(big);
  c->tile_cap = c->ntiles;
  c->d_scan_tmp = (int *)A(sizeof(int) * (size_t)c->scan_cap);
  c->d_flag = (int *)A(sizeof(int) * 4);
  c->d_grid = A(ts * (size_t)c->grid_elems);
  c->d_cgrid = A(2 * ts * (size_t)c->cgrid_elems);
  for (int i = 0; i < 6; ++i) c->d_v[i] = A(ts * 8 * N);
  c->d_B = A(ts * 8 * N);
  c->d_basis = A(ts * 8 * N * (size_t)(std::max(c->lanczos_max, c->krylov_max) + 1));
  c->d_dots = (double *)A(sizeof(double) * MAX_ROWS * (size_t)c->nvblk);
  c->d_vin = A(ts * 8 * N);
  c->d_posout = (double *)A(sizeof(double) * 3 * N);
  c->d_rng = (uint64_t *)A(2 * sizeof(uint64_t));
  {  // Krylov control state
    KDev &k = c->kd;
    const int L = c->lanczos_max, M = c->krylov_max;
    k.nsys = ns;
    k.lmax = L;
    k.gmax = M;
    k.ltol = c->lanczos_tol;
    k.gtol = c->krylov_tol;
    k.iter = (int *)A(sizeof(int) * 4);
    k.flag = k.iter + 2;
    k.l_it = (int *)A(sizeof(int) * 2 * ns);   // l_it then l_capped (read back together)
    k.l_capped = k.l_it + ns;
    k.g_it = (int *)A(sizeof(int) * 2 * ns);   // g_it then g_capped
    k.g_capped = k.g_it + ns;
    k.l_alpha = (double *)A(sizeof(double) * ns * (size_t)L);
    k.l_beta = (double *)A(sizeof(double) * ns * (size_t)L);
    k.l_cprev = (double *)A(sizeof(double) * ns * (size_t)L);
    k.l_c = (double *)A(sizeof(double) * ns * (size_t)L);
    k.l_work = (double *)A(sizeof(double) * ns * (size_t)(2 * L + L * L));
    k.l_b0 = (double *)A(sizeof(double) * ns);
    k.l_err = (double *)A(sizeof(double) * ns);
    k.g_H = (double *)A(sizeof(double) * ns * (size_t)(M + 1) * M);
    k.g_cs = (double *)A(sizeof(double) * ns * (size_t)M);
    k.g_sn = (double *)A(sizeof(double) * ns * (size_t)M);
    k.g_g = (double *)A(sizeof(double) * ns * (size_t)(M + 1));
    k.g_beta = (double *)A(sizeof(double) * ns);
    k.g_rel = (double *)A(sizeof(double) * ns);
  }
  c->d_coef = (double *)A(sizeof(double) * COEF_STRIDE * (size_t)ns);
  c->kd.coef = c->d_coef;
  c->d_pos0 = (double *)A(sizeof(double) * 3 * N);
  c->d_posh = (double *)A(sizeof(double) * 3 * N);
  if (fail) {
    c->err = "device allocation failed (" + std::to_string(c->dev_bytes) + " bytes so far)";
    return PSE_ERR_OOM;
  }
  PSE_CUDA_TRY(c, cudaMallocHost((void **)&c->h_dots, sizeof(double) * COEF_STRIDE * (size_t)ns));
  PSE_CUDA_TRY(c, cudaMallocHost((void **)&c->h_wbuf, sizeof(double) * COEF_STRIDE * (size_t)ns));
  PSE_CUDA_TRY(c, cudaMallocHost((void **)&c->h_pinned_int, sizeof(int) * (8 + 2 * (size_t)ns)));
  PSE_CUDA_TRY(c, cudaMallocHost((void **)&c->h_nbr_tot, 2 * sizeof(unsigned long long) * ns));
  PSE_CUDA_TRY(c, cudaMallocHost((void **)&c->h_flag, sizeof(int) * (1 + (size_t)ns)));
  PSE_CUDA_TRY(c, cudaMallocHost((void **)&c->h_rng, 2 * sizeof(uint64_t)));
  PSE_CUDA_TRY(c, cudaMemset(c->kd.iter, 0, sizeof(int) * 4));
  PSE_CUDA_TRY(c, cudaMemset(c->kd.l_it, 0, sizeof(int) * 2 * ns));
  PSE_CUDA_TRY(c, cudaMemset(c->kd.g_it, 0, sizeof(int) * 2 * ns));
  PSE_CUDA_TRY(c, cudaMemcpy(c->d_sys, c->hs.data(), sizeof(SysDev) * ns, cudaMemcpyHostToDevice));
  PSE_CUDA_TRY(c, cudaMemcpy(c->d_p0, p0.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice));
  PSE_CUDA_TRY(c, cudaMemcpy(c->d_k0, k0.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice));
  PSE_CUDA_TRY(c, cudaMemcpy(c->d_tile0, tile0.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice));
  PSE_CUDA_TRY(c, cudaMemcpy(c->d_blk0, blk0.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice));
  c->h_active.assign(ns, 1);
  std::vector<int> ones(ns, 1);
  PSE_CUDA_TRY(c, cudaMemcpy(c->d_active, ones.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
  PSE_CUDA_TRY(c, cudaMemset(c->d_queue, 0, sizeof(int) * 64));
  c->sys_stats.assign(ns, pse_stats{});
  // table to device in the working precision
  if (c->prec == PSE_MIXED) {
    std::vector<float> f(t.v.begin(), t.v.end());
    PSE_CUDA_TRY(c, cudaMemcpy(c->d_table, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice));
    const size_t len = (size_t)t.len;
    std::vector<float> fe(8 * len, 0.0f), fu(8 * len, 0.0f);
    for (size_t q = 0; q < len; ++q) {
      const size_t q1 = q + 1 < len ? q + 1 : q;
      for (int k = 0; k < 3; ++k) {
        fe[8 * q + k] = f[8 * q + 4 + k];
        fe[8 * q + 3 + k] = f[8 * q1 + 4 + k];
      }
      for (int k = 0; k < 4; ++k) {
        fu[8 * q + k] = f[8 * q + k];
        fu[8 * q + 4 + k] = f[8 * q1 + k];
      }
    }
    PSE_CUDA_TRY(c, cudaMemcpy(c->d_table_e, fe.data(), sizeof(float) * fe.size(), cudaMemcpyHostToDevice));
    PSE_CUDA_TRY(c, cudaMemcpy(c->d_table_u, fu.data(), sizeof(float) * fu.size(), cudaMemcpyHostToDevice));
  } else {
    PSE_CUDA_TRY(c, cudaMemcpy(c->d_table, t.v.data(), sizeof(double) * t.v.size(), cudaMemcpyHostToDevice));
  }
  {
    std::vector<double> consts((size_t)COEF_STRIDE * ns, 0.0);
    for (int q = 0; q < ns; ++q) {
      consts[(size_t)q * COEF_STRIDE + CO_ONE] = 1.0;
      consts[(size_t)q * COEF_STRIDE + CO_MONE] = -1.0;
    }
    PSE_CUDA_TRY(c, cudaMemcpy(c->d_coef, consts.data(), sizeof(double) * consts.size(), cudaMemcpyHostToDevice));
  }
  // cuFFT plans per group (shared work area)
  size_t work = 0;
  std::vector<int> comps_r2c = {5, 8}, comps_c2r = {3, 5, 8};
  if (o.torque) {
    comps_r2c.push_back(11);
    comps_c2r.push_back(11);
  }
  cufftType tr = c->prec == PSE_MIXED ? CUFFT_R2C : CUFFT_D2Z, tc = c->prec == PSE_MIXED ? CUFFT_C2R : CUFFT_Z2D;
  for (FftGroup &g : c->groups) {
    int n[3] = {g.Ng, g.Ng, g.Ng};
    const int n3 = g.Ng * g.Ng * g.Ng, nk = g.Ng * g.Ng * (g.Ng / 2 + 1);
    for (int b : comps_r2c) {
      size_t ws = 0;
      PSE_CUFFT_TRY(c, cufftCreate(&g.r2c[b]));
      g.ok[0][b] = true;
      PSE_CUFFT_TRY(c, cufftSetAutoAllocation(g.r2c[b], 0));
      PSE_CUFFT_TRY(c, cufftMakePlanMany(g.r2c[b], 3, n, nullptr, 1, n3, nullptr, 1, nk, tr, b * g.nsys, &ws));
      work = std::max(work, ws);
    }
    for (int b : comps_c2r) {
      size_t ws = 0;
      PSE_CUFFT_TRY(c, cufftCreate(&g.c2r[b]));
      g.ok[1][b] = true;
      PSE_CUFFT_TRY(c, cufftSetAutoAllocation(g.c2r[b], 0));
      PSE_CUFFT_TRY(c, cufftMakePlanMany(g.c2r[b], 3, n, nullptr, 1, nk, nullptr, 1, n3, tc, b * g.nsys, &ws));
      work = std::max(work, ws);
    }
  }
  c->d_fft_work = A(std::max<size_t>(work, 16));
  if (fail) {
    c->err = "cannot allocate cuFFT work area";
    return PSE_ERR_OOM;
  }
  for (FftGroup &g : c->groups) {
    for (int b : comps_r2c) PSE_CUFFT_TRY(c, cufftSetWorkArea(g.r2c[b], c->d_fft_work));
    for (int b : comps_c2r) PSE_CUFFT_TRY(c, cufftSetWorkArea(g.c2r[b], c->d_fft_work));
  }
  PSE_CUDA_TRY(c, cudaDeviceSynchronize());
  return PSE_OK;
}

void resolve_profile(pse_ctx *c) {
  for (auto &q : c->pending) {
    cudaEventSynchronize(q.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      c->prof_ms[q.stage] += ms;
      c->prof_vms[q.stage][q.variant] += ms;
    }
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
  for (FftGroup &g : c->groups)
    for (int b = 0; b < 12; ++b) {
      if (g.ok[0][b]) cufftDestroy(g.r2c[b]);
      if (g.ok[1][b]) cufftDestroy(g.c2r[b]);
    }
  c->groups.clear();
  if (c->g_exec) cudaGraphExecDestroy(c->g_exec);
  if (c->g_graph) cudaGraphDestroy(c->g_graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->g_stream) cudaStreamDestroy(c->g_stream);
  c->g_stream = nullptr;
  c->g_exec = nullptr;
  c->g_graph = nullptr;
  c->cap_stream = nullptr;
  for (void *q : c->allocs) cudaFree(q);
  if (c->h_dots) cudaFreeHost(c->h_dots);
  if (c->h_wbuf) cudaFreeHost(c->h_wbuf);
  if (c->h_pinned_int) cudaFreeHost(c->h_pinned_int);
  if (c->h_nbr_tot) cudaFreeHost(c->h_nbr_tot);
  if (c->h_flag) cudaFreeHost(c->h_flag);
  if (c->h_rng) cudaFreeHost(c->h_rng);
  c->allocs.clear();
}

// Re-tiles every suspension with the tile caps (x, y, z); the tile arrays grow if needed.
pse_status retile(pse_ctx *c, const int caps[3]) {
  std::vector<Params> ps = c->ps;
  std::vector<int> tile0(c->nsys + 1, 0);
  for (int q = 0; q < c->nsys; ++q) {
    std::string e;
    if (choose_tile(ps[q], caps, c->opt.tile, e)) {
      c->err = e;
      return PSE_ERR_INVALID_ARG;
    }
    tile0[q + 1] = tile0[q] + ps[q].ntile[0] * ps[q].ntile[1] * ps[q].ntile[2];
  }
  const int64_t nt = tile0[c->nsys];
  if (nt > c->tile_cap) {
    void *a = dalloc(c, sizeof(int) * (size_t)(nt + 1)), *b = dalloc(c, sizeof(int) * (size_t)(nt + 1));
    void *fa = dalloc(c, sizeof(int) * (size_t)(nt * SUB_BLOCKS + 1));
    void *fb = dalloc(c, sizeof(int) * (size_t)(nt * SUB_BLOCKS + 1));
    if (!a || !b || !fa || !fb) {
      c->err = "cannot allocate tile arrays";
      return PSE_ERR_OOM;
    }
    c->d_tile_start = (int *)a;
    c->d_tile_cur = (int *)b;
    c->d_fine_start = (int *)fa;
    c->d_fine_cur = (int *)fb;
    c->tile_cap = nt;
  }
  int64_t need = scan_tmp_ints(std::max<int64_t>(std::max<int64_t>(nt * SUB_BLOCKS, c->ncells), c->p.N) + 1);
  if (need > c->scan_cap) {
    void *q = dalloc(c, sizeof(int) * (size_t)need);
    if (!q) {
      c->err = "cannot allocate scan scratch";
      return PSE_ERR_OOM;
    }
    c->d_scan_tmp = (int *)q;
    c->scan_cap = need;
  }
  c->ps = ps;
  c->n_cubic = 0;
  for (int q = 0; q < c->nsys; ++q) {
    for (int d = 0; d < 3; ++d) {
      c->hs[q].T[d] = ps[q].tile[d];
      c->hs[q].nt[d] = ps[q].ntile[d];
    }
    set_cubic(c, c->hs[q], c->ps[q]);
    c->hs[q].tile0 = tile0[q];
  }
  c->ntiles = nt;
  for (int d = 0; d < 3; ++d) {
    c->p.tile[d] = ps[0].tile[d];
    c->p.ntile[d] = ps[0].ntile[d];
  }
  PSE_CUDA_TRY(c, cudaDeviceSynchronize());
  PSE_CUDA_TRY(c, cudaMemcpy(c->d_sys, c->hs.data(), sizeof(SysDev) * c->nsys, cudaMemcpyHostToDevice));
  PSE_CUDA_TRY(c, cudaMemcpy(c->d_tile0, tile0.data(), sizeof(int) * (c->nsys + 1), cudaMemcpyHostToDevice));
  return PSE_OK;
}

// Mean device time (ms) of `reps` calls of f on stream s after one untimed call.
template <typename F>
pse_status time_ms(pse_ctx *c, cudaStream_t s, int reps, F &&f, double *ms) {
  PSE_TRY(f());
  cudaEvent_t a, b;
  PSE_CUDA_TRY(c, cudaEventCreate(&a));
  PSE_CUDA_TRY(c, cudaEventCreate(&b));
  PSE_CUDA_TRY(c, cudaEventRecord(a, s));
  for (int k = 0; k < reps; ++k) PSE_TRY(f());
  PSE_CUDA_TRY(c, cudaEventRecord(b, s));
  PSE_CUDA_TRY(c, cudaEventSynchronize(b));
  float t = 0.f;
  PSE_CUDA_TRY(c, cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / reps;
  return PSE_OK;
}

pse_status autotune_impl(pse_ctx *c, const double *pos, int reps, pse_tuning *out, cudaStream_t s) {
  void *dpos;
  PSE_TRY(set_all_active(c, s));
  PSE_TRY(stage(c, 0, pos, sizeof(double) * 3 * c->p.N, true, s, &dpos));
  PSE_TRY(setup_config(c, (const double *)dpos, s));
  PSE_TRY(philox_w1(c, 1, 1, c->d_v[0], s));  // any dense vector will do
  pse_tuning t{};
  // lanes per particle of the pair sum: the S -> E product of the GMRES loop plus the full product
  const int lanes[5] = {1, 4, 8, 16, 32};
  double best = INFINITY;
  int bestg = c->opt.real_lanes;
  for (int g : lanes) {
    c->opt.real_lanes = g;
    double ms = 0;
    PSE_TRY(time_ms(c, s, reps, [&] {
      pse_status a = real_apply(c, c->d_v[0], c->d_v[1], M_SE, s);
      return a != PSE_OK ? a : real_apply(c, c->d_v[0], c->d_v[2], M_FULL, s);
    }, &ms));
    t.real_ms[t.n_lanes++] = ms;
    if (ms < best) {
      best = ms;
      bestg = g;
    }
  }
  c->opt.real_lanes = bestg;
  t.real_lanes = bestg;
  // the table in shared memory (FP32, when it fits), at the chosen lanes
  t.real_smem_table = 0;
  if (c->prec == PSE_MIXED && sizeof(float) * 8 * (size_t)c->table_len <= c->smem_optin) {
    c->real_smem_table = 1;
    double ms = 0;
    PSE_TRY(time_ms(c, s, reps, [&] {
      pse_status a = real_apply(c, c->d_v[0], c->d_v[1], M_SE, s);
      return a != PSE_OK ? a : real_apply(c, c->d_v[0], c->d_v[2], M_FULL, s);
    }, &ms));
    t.real_smem_ms = ms;
    if (ms < best) {
      best = ms;
      t.real_smem_table = 1;
    } else {
      c->real_smem_table = 0;
    }
  }
  // spreading / interpolation tiles: candidate caps, timed on the S -> E wave product
  const int cand[][3] = {{16, 16, 16}, {16, 8, 16}, {8, 8, 16}, {8, 16, 16}, {16, 16, 32}, {16, 8, 32}, {32, 8, 16}};
  std::vector<std::vector<int>> seen;
  double bw = INFINITY;
  int bi = 0;
  for (int k = 0; k < (int)(sizeof(cand) / sizeof(cand[0])); ++k) {
    PSE_TRY(retile(c, cand[k]));
    std::vector<int> sig;
    for (const Params &q : c->ps) sig.insert(sig.end(), q.tile, q.tile + 3);
    if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
    seen.push_back(sig);
    PSE_TRY(setup_config(c, (const double *)dpos, s));
    double ms = 0;
    PSE_TRY(time_ms(c, s, reps, [&] { return wave_apply(c, c->d_v[0], c->d_v[1], M_SE, false, s); }, &ms));
    if (t.n_tiles < 8) {
      for (int d = 0; d < 3; ++d) t.tiles[t.n_tiles][d] = c->ps[0].tile[d];
      t.wave_ms[t.n_tiles++] = ms;
    }
    if (ms < bw) {
      bw = ms;
      bi = k;
    }
  }
  PSE_TRY(retile(c, cand[bi]));
  PSE_TRY(setup_config(c, (const double *)dpos, s));
  ++c->layout_version;  // a captured step graph holds the old tiles and lanes
  for (int d = 0; d < 3; ++d) t.tile[d] = c->ps[0].tile[d];
  t.best_real_ms = best;
  t.best_wave_ms = bw;
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  if (out) *out = t;
  return PSE_OK;
}

pse_ctx *new_ctx(pse_precision prec, const pse_options &o, double a, double eta, double kT, double xi, double tol) {
  pse_ctx *c = new (std::nothrow) pse_ctx();
  if (!c) return nullptr;
  c->prec = prec;
  c->ts = prec == PSE_MIXED ? 4 : 8;
  c->opt = o;
  Params &p = c->p;
  std::memset(&p, 0, sizeof(p));
  p.ts = (int)c->ts;
  p.a = a;
  p.eta = eta;
  p.kT = kT;
  p.xi = xi;
  p.tol = tol;
  return c;
}

pse_status create_common(pse_handle *out, int32_t nsys, const int64_t *N, const double *L, double a, double eta,
                         double kT, double xi, double tol, pse_precision prec, const pse_options *opt) {
  if (!out) return PSE_ERR_INVALID_ARG;
  *out = nullptr;
  if (prec != PSE_MIXED && prec != PSE_FP64) {
    g_create_err = "unknown precision";
    return PSE_ERR_INVALID_ARG;
  }
  if (nsys < 1 || nsys > 65536 || !N || !L) {
    g_create_err = "need 1 <= nsys <= 65536 and N, L arrays";
    return PSE_ERR_INVALID_ARG;
  }
  pse_options o;
  pse_default_options(&o);
  if (opt) o = *opt;
  pse_ctx *c = new_ctx(prec, o, a, eta, kT, xi, tol);
  if (!c) return PSE_ERR_OOM;
  pse_status st = choose_group(c, nsys, N, L, o);
  if (st == PSE_OK) st = create_group(c, o);
  if (st != PSE_OK) {
    g_create_err = c->err;
    destroy_impl(c);
    delete c;
    return st;
  }
  *out = c;
  return PSE_OK;
}

void fill_info(const pse_ctx *h, const Params &p, int64_t bytes, pse_info *o) {
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
  o->device_bytes = bytes;
  o->deformed = p.def;
  for (int i = 0; i < 9; ++i) o->deform[i] = p.A[i];
  o->lambda_max = p.lam_P;
  o->lambda_min_cells = p.lam_cells;
  o->colnorm_max = p.cmax_grid;
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
  o->grid_ladder = 1;
  o->lambda_support = 1;
}

pse_status pse_create(pse_handle *out, int64_t N, double L, double a, double eta, double kT, double xi, double tol,
                      pse_precision prec, const pse_options *opt) {
  return create_common(out, 1, &N, &L, a, eta, kT, xi, tol, prec, opt);
}

pse_status pse_create_batch(pse_handle *out, int32_t nsys, const int64_t *N, const double *L, double a, double eta,
                            double kT, double xi, double tol, pse_precision prec, const pse_options *opt) {
  return create_common(out, nsys, N, L, a, eta, kT, xi, tol, prec, opt);
}

pse_status pse_estimate_bytes(int32_t nsys, const int64_t *N, const double *L, double a, double eta, double kT,
                              double xi, double tol, pse_precision prec, const pse_options *opt, int64_t *bytes) {
  if (!bytes || nsys < 1 || !N || !L || (prec != PSE_MIXED && prec != PSE_FP64)) return PSE_ERR_INVALID_ARG;
  pse_options o;
  pse_default_options(&o);
  if (opt) o = *opt;
  pse_ctx *c = new_ctx(prec, o, a, eta, kT, xi, tol);
  if (!c) return PSE_ERR_OOM;
  pse_status st = choose_group(c, nsys, N, L, o);
  if (st == PSE_OK) *bytes = estimate_bytes(c);
  else g_create_err = c->err;
  delete c;
  return st;
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
  fill_info(h, h->ps.empty() ? h->p : h->ps[0], h->dev_bytes, o);
  o->N = h->p.N;
  o->tile_kernels = h->hs.empty() ? 0 : h->hs[0].cubic;
  return PSE_OK;
}

pse_status pse_set_deformation(pse_handle h, const double *A, pse_stream stream) {
  if (!h || !A) return PSE_ERR_INVALID_ARG;
  bool created_deformed = false;
  for (int i = 0; i < 9; ++i) created_deformed = created_deformed || h->opt.deform[i] != 0.0;
  if (!created_deformed) {
    h->err = "pse_set_deformation: the handle was created for the cube (options.deform all zero)";
    return PSE_ERR_INVALID_ARG;
  }
  std::vector<Params> ps = h->ps;
  for (Params &p : ps) {
    std::string e;
    if (set_lattice(p, A, e)) {
      h->err = "pse_set_deformation: " + e;
      return PSE_ERR_INVALID_ARG;
    }
    const double tiny = 1e-12;
    if (p.lam_max > p.lam_P * (1 + tiny) && h->opt.lambda_support && h->opt.P <= 0) {
      h->err = "pse_set_deformation: lambda_max " + std::to_string(p.lam_max) + " exceeds the " +
               std::to_string(p.lam_P) + " the support size was chosen for";
      return PSE_ERR_INVALID_ARG;
    }
    if (p.lam_min < p.lam_cells * (1 - tiny)) {
      h->err = "pse_set_deformation: lambda_min " + std::to_string(p.lam_min) + " is below the " +
               std::to_string(p.lam_cells) + " the cells and r_cut were chosen for";
      return PSE_ERR_INVALID_ARG;
    }
    if (h->n_cubic > 0 && z_coupled(p.A)) {
      h->err = "pse_set_deformation: the handle runs the 16^3-tile kernels, which need A^T A to leave z "
               "uncoupled (shear or extension in the x-y plane)";
      return PSE_ERR_INVALID_ARG;
    }
    if (p.cmax > p.cmax_grid * (1 + tiny) && h->opt.Ng <= 0) {
      h->err = "pse_set_deformation: column norm " + std::to_string(p.cmax) + " exceeds the " +
               std::to_string(p.cmax_grid) + " the grid was chosen for";
      return PSE_ERR_INVALID_ARG;
    }
  }
  h->ps = ps;
  for (int q = 0; q < h->nsys; ++q) fill_lattice(h->ps[q], h->hs[q]);
  Params shared = h->ps[0];
  shared.N = h->p.N;
  h->p = shared;
  cudaStream_t s = (cudaStream_t)stream;
  PSE_CUDA_TRY(h, cudaMemcpyAsync(h->d_sys, h->hs.data(), sizeof(SysDev) * h->nsys, cudaMemcpyHostToDevice, s));
  return PSE_OK;
}

int32_t pse_num_systems(pse_handle h) { return h ? h->nsys : 0; }

int32_t pse_graph_ready(pse_handle h) { return h && h->opt.use_graph && h->g_exec ? 1 : 0; }

const char *pse_graph_error(pse_handle h) { return h ? h->graph_error.c_str() : ""; }

pse_status pse_get_system_info(pse_handle h, int32_t s, pse_info *o) {
  if (!h || !o || s < 0 || s >= h->nsys) return PSE_ERR_INVALID_ARG;
  fill_info(h, h->ps[s], h->dev_bytes, o);
  o->tile_kernels = h->hs[s].cubic;
  return PSE_OK;
}

pse_status pse_get_system_stats(pse_handle h, int32_t s, pse_stats *o) {
  if (!h || !o || s < 0 || s >= h->nsys) return PSE_ERR_INVALID_ARG;
  *o = h->sys_stats[s];
  return PSE_OK;
}

pse_status pse_mobility_apply_parts(pse_handle h, const double *pos, const void *F, const void *S, void *U, void *E,
                                    int32_t parts, pse_stream stream) {
  if (!h || !pos) return PSE_ERR_INVALID_ARG;
  NvtxRange range("pse_mobility_apply");
  if (parts < 1 || parts > 3) {
    h->err = "parts must be PSE_PART_REAL, PSE_PART_WAVE or PSE_PART_ALL";
    return PSE_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  pse_ctx *c = h;
  int64_t N = c->p.N;
  PSE_TRY(set_all_active(c, s));
  void *dpos, *dF, *dS, *dU, *dE;
  PSE_TRY(stage(c, 0, pos, sizeof(double) * 3 * N, true, s, &dpos));
  PSE_TRY(stage(c, 1, F, c->ts * 3 * N, true, s, &dF));
  PSE_TRY(stage(c, 2, S, c->ts * 5 * N, true, s, &dS));
  PSE_TRY(stage(c, 3, U, c->ts * 3 * N, false, s, &dU));
  PSE_TRY(stage(c, 4, E, c->ts * 5 * N, false, s, &dE));
  PSE_TRY(setup_config(c, (const double *)dpos, s));
  PSE_TRY(gather_in(c, dF, dS, c->d_v[0], s));
  int mode = M_FULL;
  if (!E) mode = dF ? M_FSU : M_SU;
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
  NvtxRange range("pse_brownian_sample");
  cudaStream_t s = (cudaStream_t)stream;
  pse_ctx *c = h;
  const Params &p = c->p;
  int64_t N = p.N;
  reset_stats(c);
  PSE_TRY(set_all_active(c, s));
  void *dpos, *dw1, *dw2, *dU, *dE;
  PSE_TRY(stage(c, 0, pos, sizeof(double) * 3 * N, true, s, &dpos));
  PSE_TRY(stage(c, 1, w1, c->ts * 8 * N, true, s, &dw1));
  PSE_TRY(stage(c, 2, w2, w2_bytes(c), true, s, &dw2));
  PSE_TRY(stage(c, 3, UB, c->ts * 3 * N, false, s, &dU));
  PSE_TRY(stage(c, 4, EB, c->ts * 5 * N, false, s, &dE));
  PSE_TRY(check_inputs(c, dw1, 8 * N, c->prec == PSE_FP64, s));
  PSE_TRY(setup_config(c, (const double *)dpos, s));
  PSE_TRY(sample_sorted(c, dw1, dw2, seed, counter, c->d_v[2], s));
  PSE_TRY(scatter_out(c, c->d_v[2], dU, dE, std::sqrt(2.0 * p.kT / dt), s));
  PSE_TRY(unstage(c, UB, dU, c->ts * 3 * N, s));
  PSE_TRY(unstage(c, EB, dE, c->ts * 5 * N, s));
  PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  c->h2d_pending = false;
  pse_status st = read_krylov_stats(c, true, false, s);
  gather_stats(c, stats);
  return st;
}

pse_status pse_constrained_step(pse_handle h, double *pos, const void *FP, double dt, uint64_t seed, uint64_t step,
                                void *S_out, pse_stats *stats, pse_stream stream) {
  if (!h) return PSE_ERR_INVALID_ARG;
  NvtxRange range("pse_constrained_step");
  return step_impl(h, pos, FP, dt, nullptr, nullptr, seed, step, S_out, stats, (cudaStream_t)stream);
}

pse_status pse_constrained_step_noise(pse_handle h, double *pos, const void *FP, double dt, const void *w1,
                                      const void *w2, void *S_out, pse_stats *stats, pse_stream stream) {
  if (!h || !w1 || !w2) return PSE_ERR_INVALID_ARG;
  NvtxRange range("pse_constrained_step");
  return step_impl(h, pos, FP, dt, w1, w2, 0, 0, S_out, stats, (cudaStream_t)stream);
}

pse_status pse_mobility_apply11(pse_handle h, const double *pos, const void *F, const void *L, const void *S,
                                void *U, void *Om, void *E, int32_t parts, pse_stream stream) {
  if (!h || !pos) return PSE_ERR_INVALID_ARG;
  NvtxRange range("pse_mobility_apply11");
  pse_ctx *c = h;
  if (!c->opt.torque || !c->d_table_rot) {
    c->err = "the 11-moment product needs a handle created with option torque = 1";
    return PSE_ERR_INVALID_ARG;
  }
  if (c->nsys != 1) {
    c->err = "the 11-moment product takes single-suspension handles";
    return PSE_ERR_INVALID_ARG;
  }
  if (parts < 1 || parts > 3) {
    c->err = "parts must be PSE_PART_REAL, PSE_PART_WAVE or PSE_PART_ALL";
    return PSE_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = c->p.N;
  PSE_TRY(set_all_active(c, s));
  void *dpos, *dF, *dL, *dS, *dU, *dO, *dE;
  PSE_TRY(stage(c, 0, pos, sizeof(double) * 3 * N, true, s, &dpos));
  PSE_TRY(stage(c, 1, F, c->ts * 3 * N, true, s, &dF));
  PSE_TRY(stage(c, 5, L, c->ts * 3 * N, true, s, &dL));
  PSE_TRY(stage(c, 2, S, c->ts * 5 * N, true, s, &dS));
  PSE_TRY(check_inputs(c, dF, 3 * N, c->prec == PSE_FP64, s));
  PSE_TRY(check_inputs(c, dL, 3 * N, c->prec == PSE_FP64, s));
  PSE_TRY(check_inputs(c, dS, 5 * N, c->prec == PSE_FP64, s));
  PSE_TRY(setup_config(c, (const double *)dpos, s));
  PSE_TRY(gather12(c, dF, dL, dS, c->d_v12[0], s));
  if (parts & PSE_PART_REAL) PSE_TRY(real_apply11(c, c->d_v12[0], c->d_v12[1], s));
  if (parts & PSE_PART_WAVE) PSE_TRY(wave_apply11(c, c->d_v12[0], c->d_v12[1], (parts & PSE_PART_REAL) != 0, s));
  PSE_TRY(stage(c, 3, U, c->ts * 3 * N, false, s, &dU));
  PSE_TRY(stage(c, 4, E, c->ts * 5 * N, false, s, &dE));
  PSE_TRY(stage(c, 6, Om, c->ts * 3 * N, false, s, &dO));
  PSE_TRY(scatter12(c, c->d_v12[1], dU, dO, dE, s));
  PSE_TRY(unstage(c, U, dU, c->ts * 3 * N, s));
  PSE_TRY(unstage(c, Om, dO, c->ts * 3 * N, s));
  PSE_TRY(unstage(c, E, dE, c->ts * 5 * N, s));
  return PSE_OK;
}

pse_status pse_rfd_step(pse_handle h, double *pos, const void *FP, double dt, double delta, uint64_t seed,
                        uint64_t step, void *S_out, pse_stats *stats, pse_stream stream) {
  if (!h) return PSE_ERR_INVALID_ARG;
  NvtxRange range("pse_rfd_step");
  if (h->nsys != 1) {
    h->err = "the RFD step takes a single suspension";
    return PSE_ERR_INVALID_ARG;
  }
  return rfd_impl(h, pos, FP, dt, delta, nullptr, nullptr, nullptr, seed, step, S_out, stats, (cudaStream_t)stream);
}

pse_status pse_rfd_step_noise(pse_handle h, double *pos, const void *FP, double dt, double delta, const void *w1,
                              const void *w2, const void *wt, void *S_out, pse_stats *stats, pse_stream stream) {
  if (!h || !w1 || !w2 || !wt) return PSE_ERR_INVALID_ARG;
  NvtxRange range("pse_rfd_step");
  if (h->nsys != 1) {
    h->err = "the RFD step takes a single suspension";
    return PSE_ERR_INVALID_ARG;
  }
  return rfd_impl(h, pos, FP, dt, delta, w1, w2, wt, 0, 0, S_out, stats, (cudaStream_t)stream);
}

pse_status pse_overlap_force(pse_handle h, const double *pos, double kspring, void *F, pse_stream stream) {
  if (!h || !pos || !F || !(kspring >= 0)) return PSE_ERR_INVALID_ARG;
  pse_ctx *c = h;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = c->p.N;
  if (c->p.rcut < 2.0 * c->p.a) {
    c->err = "r_cut below contact: the neighbour lists cannot hold the overlapping pairs";
    return PSE_ERR_INVALID_ARG;
  }
  void *dpos, *dF;
  PSE_TRY(stage(c, 0, pos, sizeof(double) * 3 * N, true, s, &dpos));
  PSE_TRY(stage(c, 4, F, c->ts * 3 * N, false, s, &dF));
  PSE_TRY(setup_config(c, (const double *)dpos, s));
  PSE_TRY(overlap_force(c, kspring, dF, s));
  PSE_TRY(unstage(c, F, dF, c->ts * 3 * N, s));
  if (F != dF) PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
  return PSE_OK;
}

pse_status pse_autotune(pse_handle h, const double *pos, int32_t reps, pse_tuning *out, pse_stream stream) {
  if (!h || !pos || reps < 1 || reps > 100) return PSE_ERR_INVALID_ARG;
  return autotune_impl(h, pos, reps, out, (cudaStream_t)stream);
}

pse_status pse_set_profiling(pse_handle h, int32_t enable) {
  if (!h) return PSE_ERR_INVALID_ARG;
  resolve_profile(h);
  h->prof_on = enable != 0;
  for (int i = 0; i < PSE_NSTAGES; ++i) {
    h->prof_ms[i] = 0;
    h->prof_calls[i] = 0;
    for (int v = 0; v < PSE_NVARIANTS; ++v) {
      h->prof_vms[i][v] = 0;
      h->prof_vcalls[i][v] = 0;
    }
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
    for (int v = 0; v < PSE_NVARIANTS; ++v) {
      out->variant_ms[i][v] = h->prof_vms[i][v];
      out->variant_calls[i][v] = h->prof_vcalls[i][v];
    }
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
