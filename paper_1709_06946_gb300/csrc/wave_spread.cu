// Gaussian spreading Q (Sec. 2.3.2, Eq. WSops2).
//
// Persistent CTAs take output tiles (of any suspension) from a work counter.
// Warp w owns the tile's z-planes w, w + 16, ...; for
// every particle overlapping the tile it adds the particle's P x P footprint in
// its plane to the shared tile with plain read-modify-writes (each lane owns one
// (x, y) point of the footprint and updates all its components; no other warp
// touches the plane), so there are no atomics and the result is deterministic.  The tile is
// then written once to the component-major grids with coalesced stores; no grid
// zeroing pass is needed because the tiles cover the grid.
#include "wave_common.cuh"

namespace pse {
namespace {

template <typename T, int C, int SLOT0, int PT>
__global__ void __launch_bounds__(WAVE_THREADS) k_spread(WaveArgs wa, int *queue, const int4 *__restrict__ sp_i0,
                                                         const typename V4<T>::t *__restrict__ sp_d0,
                                                         const T *__restrict__ vin, const int *__restrict__ tile_start,
                                                         T *__restrict__ grid_all) {
  constexpr int CP = CPad<C>::v;
  constexpr int NPASS = PT > 0 ? (PT * PT + 31) / 32 : 1;
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
    {
      T zero[C];
#pragma unroll
      for (int c = 0; c < C; ++c) zero[c] = (T)0;
      for (int q = threadIdx.x; q < npts; q += blockDim.x) tl.store(q, zero);
    }
    __syncthreads();  // cleared before any update or (for a tile with no particles) the read-out
    int t[3], t0[3], beg[8], cum[9];
    tile_of(a, item - a.tile0, t, t0);
    const int nb = tile_bins(a, t, tile_start, beg, cum);
    const int P = PT > 0 ? PT : wa.P, Ng = a.Ng, nitem = P * P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T alpha = (T)a.alpha, hs = (T)a.h, pref = (T)a.pref;
    // this lane's (x, y) footprint point in every pass (fixed for the whole tile)
    int pjx[NPASS], pjy[NPASS];
    bool pok[NPASS];
#pragma unroll
    for (int ps = 0; ps < NPASS; ++ps) {
      int it = ps * 32 + lane;
      pok[ps] = it < nitem;
      pjx[ps] = pok[ps] ? it % P : 0;
      pjy[ps] = pok[ps] ? it / P : 0;
    }
    for (int c0 = 0; c0 < cum[nb]; c0 += LIST_CAP) {
      if (threadIdx.x == 0) s_count = 0;
      __syncthreads();
      const int n = build_list<T, C, SLOT0, true>(a, P, t0, nb, beg, cum, c0, sp_i0, sp_d0, vin, s_meta, s_d0, s_m,
                                                  s_w, &s_count);
      for (int lz = warp; lz < Tz; lz += WAVE_WARPS) {
        const int plane = lz * Ty * RX;
        // the warp finds the particles whose support crosses its plane 32 list entries at a
        // time; group g holds entries g, g + ng, g + 2 ng, ... so that particles taken one
        // after the other lie far apart in the (spatially sorted) list and rarely update
        // the same points back to back
        const int ng = (n + 31) >> 5;
        for (int g = 0; g < ng; ++g) {
          const int mine = lane * ng + g;
          int jzl = P;
          if (mine < n) {
            jzl = lz - s_meta[mine].w;
            if (jzl < 0) jzl += Ng;
          }
          unsigned hits = __ballot_sync(0xffffffffu, jzl < P);
          while (hits) {
            const int b = __ffs(hits) - 1;
            hits &= hits - 1;
            const int e = b * ng + g;
            const int jz = __shfl_sync(0xffffffffu, jzl, b);
            const int4 m4 = s_meta[e];
            T mv[C];
#pragma unroll
            for (int c = 0; c < C; ++c) mv[c] = s_m[e * CP + c];
            if (PT > 0) {
              const T *w = s_w + e * 3 * WMAX;
              const T wz = pref * w[2 * WMAX + jz];
#pragma unroll
              for (int ps = 0; ps < NPASS; ++ps) {
                int lx = m4.y + pjx[ps], ly = m4.z + pjy[ps];
                if (lx >= Ng) lx -= Ng;
                if (ly >= Ng) ly -= Ng;
                if (pok[ps] && lx < Tx && ly < Ty) {
                  const T wt = w[pjx[ps]] * w[WMAX + pjy[ps]] * wz;
                  const int i = plane + ly * RX + lx;
                  T v[C];
                  tl.load(i, v);
#pragma unroll
                  for (int c = 0; c < C; ++c) v[c] += wt * mv[c];
                  tl.store(i, v);
                }
              }
            } else {  // any support size: weights on the fly
              const T4 d0 = s_d0[e];
              const T dz = d0.z + (T)jz * hs;
              const T wz = pref * exp(-alpha * dz * dz);
              for (int ib = 0; ib < nitem; ib += 32) {
                const int it = ib + lane;
                const int jx = it % P, jy = it / P;
                int lx = m4.y + jx, ly = m4.z + jy;
                if (lx >= Ng) lx -= Ng;
                if (ly >= Ng) ly -= Ng;
                if (it < nitem && lx < Tx && ly < Ty) {
                  const T dx = d0.x + (T)jx * hs, dy = d0.y + (T)jy * hs;
                  const T wt = exp(-alpha * (dx * dx + dy * dy)) * wz;
                  const int i = plane + ly * RX + lx;
                  T v[C];
                  tl.load(i, v);
#pragma unroll
                  for (int c = 0; c < C; ++c) v[c] += wt * mv[c];
                  tl.store(i, v);
                }
              }
            }
            __syncwarp();  // the next particle may update the same points from other lanes
          }
        }
      }
      __syncthreads();
    }
    T *grid = grid_all + a.grid0;
    const int tv = Tx * Ty * Tz;
    for (int q = threadIdx.x; q < tv; q += blockDim.x) {
      int x = q % Tx, y = (q / Tx) % Ty, z = q / (Tx * Ty);
      size_t g = ((size_t)(t0[2] + z) * Ng + (t0[1] + y)) * Ng + (t0[0] + x);
      T v[C];
      tl.load((z * Ty + y) * RX + x, v);
#pragma unroll
      for (int c = 0; c < C; ++c) grid[c * a.gstride + g] = v[c];
    }
    __syncthreads();  // the tile is read out before the next item clears it
  });
}

template <typename T, int C, int SLOT0, int PT>
void launch_spread(pse_ctx *c, const WaveArgs &a, const void *vin, cudaStream_t s) {
  static std::once_flag once;
  static OccCache occ;
  auto kern = k_spread<T, C, SLOT0, PT>;
  set_smem(kern, once);
  size_t sm = wave_smem_max<T, C>(c);
  unsigned grid = wave_grid(c, kern, sm, a.ntiles, occ);
  int *q = next_queue(c, s);
  kern<<<grid, WAVE_THREADS, sm, s>>>(a, q, (const int4 *)c->d_sp_i0, (const typename V4<T>::t *)c->d_sp_d0,
                                      (const T *)vin, c->d_tile_start, (T *)c->d_grid);
}

template <typename T, int C, int SLOT0>
void spread_p(pse_ctx *c, const WaveArgs &a, const void *vin, cudaStream_t s) {
  switch (a.P) {
    case 5: launch_spread<T, C, SLOT0, 5>(c, a, vin, s); break;
    case 6: launch_spread<T, C, SLOT0, 6>(c, a, vin, s); break;
    case 8: launch_spread<T, C, SLOT0, 8>(c, a, vin, s); break;
    default: launch_spread<T, C, SLOT0, 0>(c, a, vin, s);
  }
}

}  // namespace

void spread_launch(pse_ctx *c, const WaveArgs &a, const void *vin, int mode, cudaStream_t s) {
  if (c->prec == PSE_MIXED) {
    if (mode == M_SE) spread_p<float, 5, 3>(c, a, vin, s);
    else spread_p<float, 8, 0>(c, a, vin, s);
  } else {
    if (mode == M_SE) spread_p<double, 5, 3>(c, a, vin, s);
    else spread_p<double, 8, 0>(c, a, vin, s);
  }
}

}  // namespace pse
