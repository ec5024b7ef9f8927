// Gaussian interpolation sigma Q^T (Sec. 2.3.2, Eq. WSops2).
//
// Persistent CTAs take grid tiles (of any suspension) from a work counter: the
// tile is staged in shared memory (one coalesced pass over the component-major
// grids), then the warps scan the candidate particles 32 at a time (each warp its
// own groups) and interpolate every one whose support overlaps the tile: each
// lane takes whole (x, y) columns of the footprint and then leftover points,
// the partial sums are reduced across the warp (9 shuffles for up to 8
// components) and added to the particle's outputs (a particle whose support
// straddles tiles receives one addition per tile).
#include "wave_common.cuh"

namespace pse {
namespace {

template <typename T>
__device__ __forceinline__ void add_out(T *dst, T v) {
  atomicAdd(dst, v);
}

// NT threads per CTA: 1024 for 8 components (whose tile leaves room for one CTA
// per SM), 512 otherwise.
// ROW: slots per particle row of vout; COMP0: first grid component read
template <typename T, int C, int SLOT0, int PT, int NT, int ROW = 8, int COMP0 = 0>
__global__ void __launch_bounds__(NT) k_interp(WaveArgs wa, int *queue, const int4 *__restrict__ sp_i0,
                                               const typename V4<T>::t *__restrict__ sp_d0,
                                               const int *__restrict__ tile_start, const T *__restrict__ grid_all,
                                               T *__restrict__ vout) {
  // footprint work split: NFULL passes in which each lane takes one whole (x, y)
  // column (P points along z), then the REM leftover columns' REM * P points one
  // per lane over NMINI passes (P = 6: one full pass and one of 24 points)
  constexpr int PP = PT > 0 ? PT * PT : 1;
  constexpr int NFULL = PP / 32, REM = PP % 32;
  constexpr int NMINI = PT > 0 ? (REM * (PT > 0 ? PT : 1) + 31) / 32 : 0;
  constexpr int PZ = PT > 0 ? PT : 1;
  using T4 = typename V4<T>::t;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  for_each_item(queue, wa.ntiles, [&](int item) {
    const int si = find_sys(wa.tile0, wa.nsys, item);
    const SysDev &a = wa.sys[si];
    if (wave_skip(wa, si, a)) return;
    const int P = PT > 0 ? PT : wa.P;
    const int Tx = a.T[0], Ty = a.T[1], Tz = a.T[2];
    const int RX = tile_rx(Tx, P);
    const int npts = Tz * Ty * RX;
    TileL<T, C> tl;
    tl.init(smem_raw, npts);
    int t[3], t0[3], beg[8], cum[9];
    tile_of(a, item - a.tile0, t, t0);
    const int Ng = a.Ng;
    const T *grid = grid_all + a.grid0;
    const int tv = Tx * Ty * Tz;
    for (int q = threadIdx.x; q < tv; q += blockDim.x) {
      int x = q % Tx, y = (q / Tx) % Ty, z = q / (Tx * Ty);
      size_t g = ((size_t)(t0[2] + z) * Ng + (t0[1] + y)) * Ng + (t0[0] + x);
      T v[C];
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = grid[(COMP0 + c) * a.gstride + g];
      tl.store((z * Ty + y) * RX + x, v);
    }
    __syncthreads();
    const int nb = tile_bins(a, t, tile_start, beg, cum);
    const int total = cum[nb];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T alpha = sd_alpha<T>(a), hs = sd_h<T>(a), pref = sd_pref<T>(a);
    const int zstride = Ty * RX;
    // this lane's columns (full passes) and points (leftover passes)
    int fjx[NFULL > 0 ? NFULL : 1], fjy[NFULL > 0 ? NFULL : 1];
    int mjx[NMINI > 0 ? NMINI : 1], mjy[NMINI > 0 ? NMINI : 1], mjz[NMINI > 0 ? NMINI : 1];
    bool mok[NMINI > 0 ? NMINI : 1];
#pragma unroll
    for (int ps = 0; ps < NFULL; ++ps) {
      const int col = ps * 32 + lane;
      fjx[ps] = col % PZ;
      fjy[ps] = col / PZ;
    }
#pragma unroll
    for (int ms = 0; ms < NMINI; ++ms) {
      const int it = ms * 32 + lane;
      mok[ms] = it < REM * PZ;
      const int col = NFULL * 32 + (mok[ms] ? it / PZ : 0);
      mjx[ms] = col % PZ;
      mjy[ms] = col / PZ;
      mjz[ms] = mok[ms] ? it % PZ : 0;
    }
    for (int base = warp * 32; base < total; base += (NT / 32) * 32) {
      const int v = base + lane;
      int k = 0, ox = 0, oy = 0, oz = 0;
      bool hit = false;
      if (v < total) {
        k = candidate(v, nb, beg, cum);
        hit = overlaps(a, P, t0, sp_i0[k], ox, oy, oz);
      }
      // signed offsets fit the packing for any grid (a hit's offset is in (-P, T))
      const int pk = pack_offsets(signed_offset(ox, Ng, P), signed_offset(oy, Ng, P), signed_offset(oz, Ng, P));
      unsigned mask = __ballot_sync(0xffffffffu, hit);
      while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const int ke = __shfl_sync(0xffffffffu, k, src);
        int ex, ey, ez;
        unpack_offsets(__shfl_sync(0xffffffffu, pk, src), ex, ey, ez);
        ex += ex < 0 ? Ng : 0;  // back to offsets in [0, Ng)
        ey += ey < 0 ? Ng : 0;
        ez += ez < 0 ? Ng : 0;
        const T4 d0 = sp_d0[ke];
        T acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = (T)0;
        if (PT > 0) {
          const T wl = lane_weight(lane, PZ, alpha, hs, d0);
          T wz[PZ];
          int lzs[PZ];
#pragma unroll
          for (int jz = 0; jz < PZ; ++jz) {
            wz[jz] = __shfl_sync(0xffffffffu, wl, 2 * PZ + jz);
            int lz = ez + jz;
            if (lz >= Ng) lz -= Ng;
            lzs[jz] = lz < Tz ? lz : -1;
          }
#pragma unroll
          for (int ps = 0; ps < NFULL; ++ps) {
            const T wxy = __shfl_sync(0xffffffffu, wl, fjx[ps]) * __shfl_sync(0xffffffffu, wl, PZ + fjy[ps]);
            int lx = ex + fjx[ps], ly = ey + fjy[ps];
            if (lx >= Ng) lx -= Ng;
            if (ly >= Ng) ly -= Ng;
            if (lx < Tx && ly < Ty) {
              const int col = ly * RX + lx;
#pragma unroll
              for (int jz = 0; jz < PZ; ++jz) {
                if (lzs[jz] >= 0) {
                  const T wt = wxy * wz[jz];
                  T vv[C];
                  tl.load(col + lzs[jz] * zstride, vv);
#pragma unroll
                  for (int c = 0; c < C; ++c) acc[c] += wt * vv[c];
                }
              }
            }
          }
#pragma unroll
          for (int ms = 0; ms < NMINI; ++ms) {
            const T wt = __shfl_sync(0xffffffffu, wl, mjx[ms]) * __shfl_sync(0xffffffffu, wl, PZ + mjy[ms]) *
                         __shfl_sync(0xffffffffu, wl, 2 * PZ + mjz[ms]);
            int lx = ex + mjx[ms], ly = ey + mjy[ms], lz = ez + mjz[ms];
            if (lx >= Ng) lx -= Ng;
            if (ly >= Ng) ly -= Ng;
            if (lz >= Ng) lz -= Ng;
            if (mok[ms] && lx < Tx && ly < Ty && lz < Tz) {
              T vv[C];
              tl.load((ly * RX + lx) + lz * zstride, vv);
#pragma unroll
              for (int c = 0; c < C; ++c) acc[c] += wt * vv[c];
            }
          }
        } else {  // any support size and any lattice: weights on the fly, exp(-alpha |A d|^2)
          for (int b0 = 0; b0 < P * P; b0 += 32) {
            const int it = b0 + lane;
            const int jx = it % P, jy = it / P;
            int lx = ex + jx, ly = ey + jy;
            if (lx >= Ng) lx -= Ng;
            if (ly >= Ng) ly -= Ng;
            if (it < P * P && lx < Tx && ly < Ty) {
              const T dx = d0.x + (T)jx * hs, dy = d0.y + (T)jy * hs;
              const T qxy = sd_qa<T>(a, 0) * dx * dx + sd_qa<T>(a, 1) * dy * dy + sd_qa<T>(a, 3) * dx * dy;
              const T lin = sd_qa<T>(a, 4) * dx + sd_qa<T>(a, 5) * dy, q2 = sd_qa<T>(a, 2);
              const int col = ly * RX + lx;
              for (int jz = 0; jz < P; ++jz) {
                int lz = ez + jz;
                if (lz >= Ng) lz -= Ng;
                if (lz < Tz) {
                  const T dz = d0.z + (T)jz * hs;
                  const T wt = exp(-(qxy + dz * (lin + q2 * dz)));
                  T vv[C];
                  tl.load(col + lz * zstride, vv);
#pragma unroll
                  for (int c = 0; c < C; ++c) acc[c] += wt * vv[c];
                }
              }
            }
          }
        }
        const T tot = warp_reduce8(acc, lane);
        const int comp = reduce8_component(lane);
        if ((lane & 3) == 0 && comp < C) add_out(vout + ROW * (size_t)ke + SLOT0 + comp, pref * tot);
      }
    }
    __syncthreads();  // the staged tile is no longer read when the next item overwrites it
  });
}

template <typename T, int C, int SLOT0, int PT, int ROW = 8, int COMP0 = 0>
void launch_interp(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  static std::once_flag once;
  static OccCache occ;
  constexpr int NT = C == 8 ? 1024 : WAVE_THREADS;
  auto kern = k_interp<T, C, SLOT0, PT, NT, ROW, COMP0>;
  set_smem(kern, once);
  size_t sm = wave_smem_max<T, C>(c, a.want);
  unsigned grid = wave_grid(c, kern, sm, a.ntiles, occ, NT);
  int *q = next_queue(c, s);
  kern<<<grid, NT, sm, s>>>(a, q, (const int4 *)c->d_sp_i0, (const typename V4<T>::t *)c->d_sp_d0,
                            c->d_tile_start, (const T *)c->d_grid, (T *)vout);
}

template <typename T, int C, int SLOT0, int ROW = 8, int COMP0 = 0>
void interp_p(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  if (c->lattice) return launch_interp<T, C, SLOT0, 0, ROW, COMP0>(c, a, vout, s);  // non-separable weights
  switch (a.P) {
    case 5: launch_interp<T, C, SLOT0, 5, ROW, COMP0>(c, a, vout, s); break;
    case 6: launch_interp<T, C, SLOT0, 6, ROW, COMP0>(c, a, vout, s); break;
    case 8: launch_interp<T, C, SLOT0, 8, ROW, COMP0>(c, a, vout, s); break;
    default: launch_interp<T, C, SLOT0, 0, ROW, COMP0>(c, a, vout, s);
  }
}

}  // namespace

// mode selects the interpolated components: M_FULL U,E (8), M_SE E (5), M_FSU U (3)
// Suspensions with 16^3 tiles: the shared-memory tile (default) or grid columns
// in registers (bit 1 of option wave_kernel).
void interp_cubic(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s) {
  if (c->opt.wave_kernel & 2) interp_col_launch(c, a, vout, mode, s);
  else if (c->opt.wave_kernel & 16) interp16_launch(c, a, vout, mode, s);
  else interp_halo_launch(c, a, vout, mode, s);
}

void interp_general_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s) {
  if (c->prec == PSE_MIXED) {
    if (mode == M_FULL) interp_p<float, 8, 0>(c, a, vout, s);
    else if (mode == M_SE) interp_p<float, 5, 3>(c, a, vout, s);
    else interp_p<float, 3, 0>(c, a, vout, s);
  } else {
    if (mode == M_FULL) interp_p<double, 8, 0>(c, a, vout, s);
    else if (mode == M_SE) interp_p<double, 5, 3>(c, a, vout, s);
    else interp_p<double, 3, 0>(c, a, vout, s);
  }
}

void interp_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s) {
  if (c->n_cubic == c->nsys) return interp_cubic(c, a, vout, mode, s);
  WaveArgs ag = a;
  if (c->n_cubic > 0) {  // both kinds of suspensions: one launch each
    WaveArgs ac = a;
    ac.want = 1;
    ag.want = 0;
    interp_cubic(c, ac, vout, mode, s);
    c->nlaunch += 2;
  }
  if (c->prec == PSE_MIXED) {
    if (mode == M_FULL) interp_p<float, 8, 0>(c, ag, vout, s);
    else if (mode == M_SE) interp_p<float, 5, 3>(c, ag, vout, s);
    else interp_p<float, 3, 0>(c, ag, vout, s);
  } else {
    if (mode == M_FULL) interp_p<double, 8, 0>(c, ag, vout, s);
    else if (mode == M_SE) interp_p<double, 5, 3>(c, ag, vout, s);
    else interp_p<double, 3, 0>(c, ag, vout, s);
  }
}

// Grids 0..10 interpolated into the 11 components [U, Omega, E] of 12-slot rows
// (general kernels, two passes: 8 and 3 components; outputs are added).
void interp11_launch(pse_ctx *c, void *vout12, cudaStream_t s) {
  WaveArgs a = wave_args(c);
  if (c->prec == PSE_MIXED) {
    interp_p<float, 8, 0, 12, 0>(c, a, vout12, s);
    interp_p<float, 3, 8, 12, 8>(c, a, vout12, s);
  } else {
    interp_p<double, 8, 0, 12, 0>(c, a, vout12, s);
    interp_p<double, 3, 8, 12, 8>(c, a, vout12, s);
  }
  c->nlaunch += 4;
}

}  // namespace pse
