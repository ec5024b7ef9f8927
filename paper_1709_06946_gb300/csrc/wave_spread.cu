// Gaussian spreading Q (Sec. 2.3.2, Eq. WSops2): one CTA per output tile,
// shared-memory accumulation, coalesced tile write-out (no global atomics).
#include "wave_common.cuh"

namespace pse {
namespace {

template <typename T, int C, int SLOT0, int PT>
__global__ void __launch_bounds__(256) k_spread(WaveArgs a, const int4 *__restrict__ sp_i0,
                                                const typename V4<T>::t *__restrict__ sp_d0,
                                                const T *__restrict__ vin, const int *__restrict__ tile_start,
                                                T *__restrict__ grid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *acc = (T *)smem_raw;
  const int Tx = a.T[0], Ty = a.T[1], Tz = a.T[2], Rx = Tx + 1;
  const int vol = Tz * Ty * Rx;
  for (int q = threadIdx.x; q < C * vol; q += blockDim.x) acc[q] = 0;
  int t0[3], bins[8];
  int nbins = tile_bins(a, blockIdx.x, t0, bins);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int P = PT > 0 ? PT : a.P, Ng = a.Ng, PP = P * P;
  for (int b = 0; b < nbins; ++b) {
    int beg = tile_start[bins[b]], end = tile_start[bins[b] + 1];
    for (int k = beg + warp; k < end; k += nw) {
      int4 i0 = sp_i0[k];
      int ox = wrapi(i0.x - t0[0], Ng), oy = wrapi(i0.y - t0[1], Ng), oz = wrapi(i0.z - t0[2], Ng);
      if (!((ox < Tx || ox + P - 1 >= Ng) && (oy < Ty || oy + P - 1 >= Ng) && (oz < Tz || oz + P - 1 >= Ng)))
        continue;  // warp-uniform: the support misses this tile
      typename V4<T>::t d0 = sp_d0[k];
      T m[C];
#pragma unroll
      for (int c = 0; c < C; ++c) m[c] = vin[8 * (size_t)k + SLOT0 + c];
      T wxl = weight_lane<T>(a, d0.x, lane);
      for (int base = 0; base < PP; base += 32) {
        int pq = base + lane;
        int jy = pq % P, jz = pq / P;
        int ly = oy + jy, lz = oz + jz;
        if (ly >= Ng) ly -= Ng;
        if (lz >= Ng) lz -= Ng;
        bool ok = pq < PP && ly < Ty && lz < Tz;
        T dy = d0.y + (T)jy * (T)a.h, dz = d0.z + (T)jz * (T)a.h;
        T wyz = ok ? (T)a.pref * exp(-(T)a.alpha * (dy * dy + dz * dz)) : (T)0;
        int row = (lz * Ty + ly) * Rx;
#pragma unroll
        for (int jx = 0; jx < P; ++jx) {
          T wx = __shfl_sync(0xffffffffu, wxl, jx);
          int lx = ox + jx;
          if (lx >= Ng) lx -= Ng;
          if (ok && lx < Tx) {
            T w = wyz * wx;
#pragma unroll
            for (int c = 0; c < C; ++c) atomicAdd(&acc[c * vol + row + lx], w * m[c]);
          }
        }
      }
    }
  }
  __syncthreads();
  const size_t n3 = (size_t)Ng * Ng * Ng;
  const int tv = Tx * Ty * Tz;
  for (int q = threadIdx.x; q < C * tv; q += blockDim.x) {
    int x = q % Tx, y = (q / Tx) % Ty, z = (q / (Tx * Ty)) % Tz, c = q / tv;
    grid[c * n3 + ((size_t)(t0[2] + z) * Ng + (t0[1] + y)) * Ng + (t0[0] + x)] = acc[c * vol + (z * Ty + y) * Rx + x];
  }
}

template <typename T, int C, int SLOT0, int PT>
void launch_spread(pse_ctx *c, const WaveArgs &a, const void *vin, cudaStream_t s) {
  static bool init = false;
  auto kern = k_spread<T, C, SLOT0, PT>;
  if (!init) {
    set_smem(kern);
    init = true;
  }
  size_t sm = (size_t)C * a.T[2] * a.T[1] * (a.T[0] + 1) * sizeof(T);
  kern<<<(unsigned)c->ntiles, 256, sm, s>>>(a, (const int4 *)c->d_sp_i0, (const typename V4<T>::t *)c->d_sp_d0,
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
