// Gaussian spreading Q (Sec. 2.3.2, Eq. WSops2).
//
// Persistent CTAs take output tiles (of any suspension) from a work counter.
// Warp w owns the tile's z-planes w, w + 16, ...: it scans the candidate
// particles whose support can cross its plane 32 at a time (a ballot picks the
// hits) and adds each hit's P x P footprint in the plane to the shared tile with
// plain read-modify-writes (each lane owns one (x, y) point of the footprint and
// updates all its components; no other warp touches the plane), so there are no
// atomics, the result is deterministic, and the warps never wait for one another
// between the clearing of a tile and its read-out.  The tile is then written
// once to the component-major grids with coalesced stores; no grid zeroing pass
// is needed because the tiles cover the grid.
#include "wave_common.cuh"

namespace pse {
namespace {

// moments [SLOT0, SLOT0 + C) of particle k (a ROW-slot row: 8, or 12 in the
// 11-moment product), read by the whole warp
template <typename T, int C, int SLOT0, int ROW = 8>
__device__ __forceinline__ void load_moments(const T *__restrict__ vin, int k, T mv[C]) {
  const T *row = vin + ROW * (size_t)k;
  if (sizeof(T) == 4 && SLOT0 == 3 && C == 5) {
    mv[0] = row[3];
    const float4 q = *(const float4 *)(row + 4);
    mv[1] = q.x;
    mv[2] = q.y;
    mv[3] = q.z;
    mv[4] = q.w;
  } else if (sizeof(T) == 4 && SLOT0 == 0 && C == 8) {
    const float4 q = *(const float4 *)row, r = *(const float4 *)(row + 4);
    mv[0] = q.x;
    mv[1] = q.y;
    mv[2] = q.z;
    mv[3] = q.w;
    mv[4] = r.x;
    mv[5] = r.y;
    mv[6] = r.z;
    mv[7] = r.w;
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) mv[c] = row[SLOT0 + c];
  }
}

// ROW: slots per particle row of vin; COMP0: first grid component written
template <typename T, int C, int SLOT0, int PT, int ROW = 8, int COMP0 = 0>
__global__ void __launch_bounds__(WAVE_THREADS) k_spread(WaveArgs wa, int *queue, const int4 *__restrict__ sp_i0,
                                                         const typename V4<T>::t *__restrict__ sp_d0,
                                                         const T *__restrict__ vin, const int *__restrict__ fine_start,
                                                         T *__restrict__ grid_all) {
  constexpr int NPASS = PT > 0 ? (PT * PT + 31) / 32 : 1;
  constexpr int PZ = PT > 0 ? PT : 1;
  using T4 = typename V4<T>::t;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  for_each_item(queue, wa.ntiles, [&](int item) {
    const int si = find_sys(wa.tile0, wa.nsys, item);
    const SysDev &a = wa.sys[si];
    if (wave_skip(wa, si, a)) return;
    const int P = PT > 0 ? PT : wa.P, Ng = a.Ng, nitem = P * P;
    const int Tx = a.T[0], Ty = a.T[1], Tz = a.T[2];
    const int RX = tile_rx(Tx, P);
    const int npts = Tz * Ty * RX;
    TileL<T, C> tl;
    tl.init(smem_raw, npts);
    {
      T zero[C];
#pragma unroll
      for (int c = 0; c < C; ++c) zero[c] = (T)0;
      for (int q = threadIdx.x; q < npts; q += blockDim.x) tl.store(q, zero);
    }
    __syncthreads();  // cleared before any update or (for a tile with no particles) the read-out
    int t[3], t0[3], beg[8], cum[9];
    tile_of(a, item - a.tile0, t, t0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T alpha = sd_alpha<T>(a), hs = sd_h<T>(a), pref = sd_pref<T>(a);
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
    for (int lz = warp; lz < Tz; lz += WAVE_WARPS) {
      const int plane = lz * Ty * RX;
      const int nb = plane_bins(a, t, lz, P, fine_start, beg, cum);
      const int total = cum[nb];
      for (int base = 0; base < total; base += 32) {
        const int v = base + lane;
        int k = 0, ox = 0, oy = 0, jz = P;
        if (v < total) {
          k = candidate(v, nb, beg, cum);
          int oz;
          if (overlaps(a, P, t0, sp_i0[k], ox, oy, oz)) {
            jz = lz - oz;
            if (jz < 0) jz += Ng;
          }
        }
        // signed offsets fit the packing for any grid (a hit's offset is in (-P, T))
        const int pk = pack_offsets(signed_offset(ox, Ng, P), signed_offset(oy, Ng, P), jz < P ? jz : 0);
        unsigned hits = __ballot_sync(0xffffffffu, jz < P);
        while (hits) {
          const int src = __ffs(hits) - 1;
          hits &= hits - 1;
          const int ke = __shfl_sync(0xffffffffu, k, src);
          int ex, ey, ez;
          unpack_offsets(__shfl_sync(0xffffffffu, pk, src), ex, ey, ez);
          ex += ex < 0 ? Ng : 0;  // back to offsets in [0, Ng)
          ey += ey < 0 ? Ng : 0;
          const T4 d0 = sp_d0[ke];
          T mv[C];
          load_moments<T, C, SLOT0, ROW>(vin, ke, mv);
          if (PT > 0) {
            const T wl = lane_weight(lane, PZ, alpha, hs, d0);
            const T wz = pref * __shfl_sync(0xffffffffu, wl, 2 * PZ + ez);
#pragma unroll
            for (int ps = 0; ps < NPASS; ++ps) {
              const T wxy = __shfl_sync(0xffffffffu, wl, pjx[ps]) * __shfl_sync(0xffffffffu, wl, PZ + pjy[ps]);
              int lx = ex + pjx[ps], ly = ey + pjy[ps];
              if (lx >= Ng) lx -= Ng;
              if (ly >= Ng) ly -= Ng;
              if (pok[ps] && lx < Tx && ly < Ty) {
                const T wt = wxy * wz;
                const int i = plane + ly * RX + lx;
                T vv[C];
                tl.load(i, vv);
#pragma unroll
                for (int c = 0; c < C; ++c) vv[c] += wt * mv[c];
                tl.store(i, vv);
              }
            }
          } else {  // any support size and any lattice: weights on the fly, exp(-alpha |A d|^2)
            const T dz = d0.z + (T)ez * hs;
            const T qz = sd_qa<T>(a, 2) * dz * dz, q4 = sd_qa<T>(a, 4) * dz, q5 = sd_qa<T>(a, 5) * dz;
            for (int ib = 0; ib < nitem; ib += 32) {
              const int it = ib + lane;
              const int jx = it % P, jy = it / P;
              int lx = ex + jx, ly = ey + jy;
              if (lx >= Ng) lx -= Ng;
              if (ly >= Ng) ly -= Ng;
              if (it < nitem && lx < Tx && ly < Ty) {
                const T dx = d0.x + (T)jx * hs, dy = d0.y + (T)jy * hs;
                const T q = sd_qa<T>(a, 0) * dx * dx + sd_qa<T>(a, 1) * dy * dy + sd_qa<T>(a, 3) * dx * dy + q4 * dx + q5 * dy + qz;
                const T wt = pref * exp(-q);
                const int i = plane + ly * RX + lx;
                T vv[C];
                tl.load(i, vv);
#pragma unroll
                for (int c = 0; c < C; ++c) vv[c] += wt * mv[c];
                tl.store(i, vv);
              }
            }
          }
          __syncwarp();  // the next particle may update the same points from other lanes
        }
      }
    }
    __syncthreads();
    T *grid = grid_all + a.grid0;
    const int tv = Tx * Ty * Tz;
    for (int q = threadIdx.x; q < tv; q += blockDim.x) {
      int x = q % Tx, y = (q / Tx) % Ty, z = q / (Tx * Ty);
      size_t g = ((size_t)(t0[2] + z) * Ng + (t0[1] + y)) * Ng + (t0[0] + x);
      T v[C];
      tl.load((z * Ty + y) * RX + x, v);
#pragma unroll
      for (int c = 0; c < C; ++c) grid[(COMP0 + c) * a.gstride + g] = v[c];
    }
    __syncthreads();  // the tile is read out before the next item clears it
  });
}

template <typename T, int C, int SLOT0, int PT, int ROW = 8, int COMP0 = 0>
void launch_spread(pse_ctx *c, const WaveArgs &a, const void *vin, cudaStream_t s) {
  static std::once_flag once;
  static OccCache occ;
  auto kern = k_spread<T, C, SLOT0, PT, ROW, COMP0>;
  set_smem(kern, once);
  size_t sm = wave_smem_max<T, C>(c, a.want);
  unsigned grid = wave_grid(c, kern, sm, a.ntiles, occ);
  int *q = next_queue(c, s);
  kern<<<grid, WAVE_THREADS, sm, s>>>(a, q, (const int4 *)c->d_sp_i0, (const typename V4<T>::t *)c->d_sp_d0,
                                      (const T *)vin, c->d_fine_start, (T *)c->d_grid);
}

template <typename T, int C, int SLOT0, int ROW = 8, int COMP0 = 0>
void spread_p(pse_ctx *c, const WaveArgs &a, const void *vin, cudaStream_t s) {
  if (c->lattice) return launch_spread<T, C, SLOT0, 0, ROW, COMP0>(c, a, vin, s);  // non-separable weights
  switch (a.P) {
    case 5: launch_spread<T, C, SLOT0, 5, ROW, COMP0>(c, a, vin, s); break;
    case 6: launch_spread<T, C, SLOT0, 6, ROW, COMP0>(c, a, vin, s); break;
    case 8: launch_spread<T, C, SLOT0, 8, ROW, COMP0>(c, a, vin, s); break;
    default: launch_spread<T, C, SLOT0, 0, ROW, COMP0>(c, a, vin, s);
  }
}

}  // namespace

// Suspensions with 16^3 tiles: grid columns in registers (default) or the
// shared-memory tile (bit 0 of option wave_kernel).
void spread_cubic(pse_ctx *c, const WaveArgs &a, const void *vin, int mode, cudaStream_t s) {
  if (c->opt.wave_kernel & 1) spread16_launch(c, a, vin, mode, s);
  else spread_col_launch(c, a, vin, mode, s);
}

void spread_launch(pse_ctx *c, const WaveArgs &a, const void *vin, int mode, cudaStream_t s) {
  if (c->n_cubic == c->nsys) return spread_cubic(c, a, vin, mode, s);
  WaveArgs ag = a;
  if (c->n_cubic > 0) {  // both kinds of suspensions: one launch each
    WaveArgs ac = a;
    ac.want = 1;
    ag.want = 0;
    spread_cubic(c, ac, vin, mode, s);
    c->nlaunch += 2;
  }
  if (c->prec == PSE_MIXED) {
    if (mode == M_SE || mode == M_SU) spread_p<float, 5, 3>(c, ag, vin, s);
    else spread_p<float, 8, 0>(c, ag, vin, s);
  } else {
    if (mode == M_SE || mode == M_SU) spread_p<double, 5, 3>(c, ag, vin, s);
    else spread_p<double, 8, 0>(c, ag, vin, s);
  }
}

// The 11 components [F, L, S] of 12-slot rows onto grids 0..10 of every suspension
// (general kernels for any tile, two passes: 8 and 3 components).
void spread11_launch(pse_ctx *c, const void *vin12, cudaStream_t s) {
  WaveArgs a = wave_args(c);
  if (c->prec == PSE_MIXED) {
    spread_p<float, 8, 0, 12, 0>(c, a, vin12, s);
    spread_p<float, 3, 8, 12, 8>(c, a, vin12, s);
  } else {
    spread_p<double, 8, 0, 12, 0>(c, a, vin12, s);
    spread_p<double, 3, 8, 12, 8>(c, a, vin12, s);
  }
  c->nlaunch += 4;
}

}  // namespace pse
