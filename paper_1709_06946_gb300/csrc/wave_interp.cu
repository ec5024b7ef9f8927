// Gaussian interpolation sigma Q^T (Sec. 2.3.2, Eq. WSops2).
//
// Persistent CTAs take grid tiles (of any suspension) from a work counter: the
// tile is staged in shared memory ([z][y][x][comp],
// one coalesced pass over the component-major grids), then each warp takes a
// particle overlapping the tile; lanes map to (x, y, component-half) items of
// its footprint, loop over z in registers, and the partial sums are reduced
// across the warp and added to the particle's outputs (a particle whose support
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
template <typename T, int C, int SLOT0, int PT, int NT = (C == 8 ? 1024 : WAVE_THREADS)>
__global__ void __launch_bounds__(NT) k_interp(WaveArgs wa, int *queue, const int4 *__restrict__ sp_i0,
                                                         const typename V4<T>::t *__restrict__ sp_d0,
                                                         const int *__restrict__ tile_start,
                                                         const T *__restrict__ grid_all, T *__restrict__ vout) {
  constexpr int CP = CPad<C>::v;
  // footprint work split: NFULL passes in which each lane takes one whole (x, y)
  // column (P points along z), then the REM leftover columns' REM * P points one
  // per lane over NMINI passes (P = 6: one full pass and one of 24 points)
  constexpr int PP = PT > 0 ? PT * PT : 1;
  constexpr int NFULL = PP / 32, REM = PP % 32;
  constexpr int NMINI = PT > 0 ? (REM * (PT > 0 ? PT : 1) + 31) / 32 : 0;
  using T4 = typename V4<T>::t;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  __shared__ int s_count;
  for_each_item(queue, wa.ntiles, [&](int item) {
    const int si = find_sys(wa.tile0, wa.nsys, item);
    if (!wa.active[si]) return;
    const SysDev &a = wa.sys[si];
    const int Tx = a.T[0], Ty = a.T[1], Tz = a.T[2], RX = tile_rx(Tx);
    const int npts = Tz * Ty * RX;
    TileL<T, C> tl;
    tl.init(smem_raw, npts);
    int4 *s_meta = (int4 *)(smem_raw + TileL<T, C>::bytes(npts));
    T4 *s_d0 = (T4 *)(s_meta + LIST_CAP);
    T *s_m = (T *)(s_d0 + LIST_CAP);
    T *s_w = s_m + LIST_CAP * CP;
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
      for (int c = 0; c < C; ++c) v[c] = grid[c * a.gstride + g];
      tl.store((z * Ty + y) * RX + x, v);
    }
    const int nb = tile_bins(a, t, tile_start, beg, cum);
    const int P = PT > 0 ? PT : wa.P, nitem = P * P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T alpha = (T)a.alpha, hs = (T)a.h, pref = (T)a.pref;
    const int zstride = Ty * RX;
    // this lane's columns (full passes) and points (leftover passes)
    int fjx[NFULL > 0 ? NFULL : 1], fjy[NFULL > 0 ? NFULL : 1];
    int mjx[NMINI > 0 ? NMINI : 1], mjy[NMINI > 0 ? NMINI : 1], mjz[NMINI > 0 ? NMINI : 1];
    bool mok[NMINI > 0 ? NMINI : 1];
#pragma unroll
    for (int ps = 0; ps < NFULL; ++ps) {
      const int col = ps * 32 + lane;
      fjx[ps] = col % P;
      fjy[ps] = col / P;
    }
#pragma unroll
    for (int ms = 0; ms < NMINI; ++ms) {
      const int it = ms * 32 + lane;
      mok[ms] = it < REM * P;
      const int col = NFULL * 32 + (mok[ms] ? it / P : 0);
      mjx[ms] = col % P;
      mjy[ms] = col / P;
      mjz[ms] = mok[ms] ? it % P : 0;
    }
    for (int c0 = 0; c0 < cum[nb]; c0 += LIST_CAP) {
      if (threadIdx.x == 0) s_count = 0;
      __syncthreads();  // also orders the tile staging before the first use
      const int n = build_list<T, C, SLOT0>(a, P, t0, nb, beg, cum, c0, sp_i0, sp_d0, (const T *)nullptr, s_meta,
                                            s_d0, s_m, s_w, &s_count);
      for (int e = warp; e < n; e += NT / 32) {
        const int4 m4 = s_meta[e];
        T acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = (T)0;
        if (PT > 0) {
          const T *w = s_w + e * 3 * WMAX;
          T wz[PT > 0 ? PT : 1];
          int lzs[PT > 0 ? PT : 1];
#pragma unroll
          for (int jz = 0; jz < (PT > 0 ? PT : 1); ++jz) {
            int lz = m4.w + jz;
            if (lz >= Ng) lz -= Ng;
            lzs[jz] = lz < Tz ? lz : -1;
            wz[jz] = w[2 * WMAX + jz];
          }
#pragma unroll
          for (int ps = 0; ps < NFULL; ++ps) {
            int lx = m4.y + fjx[ps], ly = m4.z + fjy[ps];
            if (lx >= Ng) lx -= Ng;
            if (ly >= Ng) ly -= Ng;
            if (lx < Tx && ly < Ty) {
              const T wxy = w[fjx[ps]] * w[WMAX + fjy[ps]];
              const int col = ly * RX + lx;
#pragma unroll
              for (int jz = 0; jz < (PT > 0 ? PT : 1); ++jz) {
                if (lzs[jz] >= 0) {
                  const T wt = wxy * wz[jz];
                  T v[C];
                  tl.load(col + lzs[jz] * zstride, v);
#pragma unroll
                  for (int c = 0; c < C; ++c) acc[c] += wt * v[c];
                }
              }
            }
          }
#pragma unroll
          for (int ms = 0; ms < NMINI; ++ms) {
            int lx = m4.y + mjx[ms], ly = m4.z + mjy[ms];
            if (lx >= Ng) lx -= Ng;
            if (ly >= Ng) ly -= Ng;
            int lz = m4.w + mjz[ms];
            if (lz >= Ng) lz -= Ng;
            if (mok[ms] && lx < Tx && ly < Ty && lz < Tz) {
              const T wt = w[mjx[ms]] * w[WMAX + mjy[ms]] * w[2 * WMAX + mjz[ms]];
              T v[C];
              tl.load((ly * RX + lx) + lz * zstride, v);
#pragma unroll
              for (int c = 0; c < C; ++c) acc[c] += wt * v[c];
            }
          }
        } else {  // any support size: weights on the fly
          const T4 d0 = s_d0[e];
          for (int base = 0; base < nitem; base += 32) {
            const int it = base + lane;
            const int jx = it % P, jy = it / P;
            int lx = m4.y + jx, ly = m4.z + jy;
            if (lx >= Ng) lx -= Ng;
            if (ly >= Ng) ly -= Ng;
            if (it < nitem && lx < Tx && ly < Ty) {
              const T dx = d0.x + (T)jx * hs, dy = d0.y + (T)jy * hs;
              const T wxy = exp(-alpha * (dx * dx + dy * dy));
              const int col = ly * RX + lx;
              for (int jz = 0; jz < P; ++jz) {
                int lz = m4.w + jz;
                if (lz >= Ng) lz -= Ng;
                if (lz < Tz) {
                  const T dz = d0.z + (T)jz * hs;
                  const T wt = wxy * exp(-alpha * dz * dz);
                  T v[C];
                  tl.load(col + lz * zstride, v);
#pragma unroll
                  for (int c = 0; c < C; ++c) acc[c] += wt * v[c];
                }
              }
            }
          }
        }
        const T tot = warp_reduce8(acc, lane);
        const int comp = reduce8_component(lane);
        if ((lane & 3) == 0 && comp < C) add_out(vout + 8 * (size_t)m4.x + SLOT0 + comp, pref * tot);
      }
      __syncthreads();
    }
    __syncthreads();  // the staged tile is no longer read when the next item overwrites it
  });
}

template <typename T, int C, int SLOT0, int PT>
void launch_interp(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  static std::once_flag once;
  static OccCache occ;
  constexpr int NT = C == 8 ? 1024 : WAVE_THREADS;
  auto kern = k_interp<T, C, SLOT0, PT, NT>;
  set_smem(kern, once);
  size_t sm = wave_smem_max<T, C>(c);
  unsigned grid = wave_grid(c, kern, sm, a.ntiles, occ, NT);
  int *q = next_queue(c, s);
  kern<<<grid, NT, sm, s>>>(a, q, (const int4 *)c->d_sp_i0, (const typename V4<T>::t *)c->d_sp_d0,
                                      c->d_tile_start, (const T *)c->d_grid, (T *)vout);
}

template <typename T, int C, int SLOT0>
void interp_p(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  switch (a.P) {
    case 5: launch_interp<T, C, SLOT0, 5>(c, a, vout, s); break;
    case 6: launch_interp<T, C, SLOT0, 6>(c, a, vout, s); break;
    case 8: launch_interp<T, C, SLOT0, 8>(c, a, vout, s); break;
    default: launch_interp<T, C, SLOT0, 0>(c, a, vout, s);
  }
}

}  // namespace

// mode selects the interpolated components: M_FULL U,E (8), M_SE E (5), M_FSU U (3)
void interp_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s) {
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

}  // namespace pse
