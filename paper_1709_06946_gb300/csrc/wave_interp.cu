// Gaussian interpolation sigma Q^T (Sec. 2.3.2, Eq. WSops2): one CTA per grid
// tile staged in shared memory; visiting particles add their in-tile partial sums.
#include "wave_common.cuh"

namespace pse {
namespace {

template <typename T, int C, int SLOT0, int PT>
__global__ void __launch_bounds__(256) k_interp(WaveArgs a, const int4 *__restrict__ sp_i0,
                                                const typename V4<T>::t *__restrict__ sp_d0,
                                                const int *__restrict__ tile_start, const T *__restrict__ grid,
                                                T *__restrict__ vout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *tile = (T *)smem_raw;
  const int Tx = a.T[0], Ty = a.T[1], Tz = a.T[2], Rx = Tx + 1;
  const int vol = Tz * Ty * Rx;
  int t0[3], bins[8];
  int nbins = tile_bins(a, blockIdx.x, t0, bins);
  const int Ng = a.Ng, P = PT > 0 ? PT : a.P, PP = P * P;
  const size_t n3 = (size_t)Ng * Ng * Ng;
  const int tv = Tx * Ty * Tz;
  for (int q = threadIdx.x; q < C * tv; q += blockDim.x) {
    int x = q % Tx, y = (q / Tx) % Ty, z = (q / (Tx * Ty)) % Tz, c = q / tv;
    tile[c * vol + (z * Ty + y) * Rx + x] = grid[c * n3 + ((size_t)(t0[2] + z) * Ng + (t0[1] + y)) * Ng + (t0[0] + x)];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = 0; b < nbins; ++b) {
    int beg = tile_start[bins[b]], end = tile_start[bins[b] + 1];
    for (int k = beg + warp; k < end; k += nw) {
      int4 i0 = sp_i0[k];
      int ox = wrapi(i0.x - t0[0], Ng), oy = wrapi(i0.y - t0[1], Ng), oz = wrapi(i0.z - t0[2], Ng);
      if (!((ox < Tx || ox + P - 1 >= Ng) && (oy < Ty || oy + P - 1 >= Ng) && (oz < Tz || oz + P - 1 >= Ng)))
        continue;  // warp-uniform
      typename V4<T>::t d0 = sp_d0[k];
      T wxl = weight_lane<T>(a, d0.x, lane);
      T acc[C];
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = 0;
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
            for (int c = 0; c < C; ++c) acc[c] += w * tile[c * vol + row + lx];
          }
        }
      }
#pragma unroll
      for (int c = 0; c < C; ++c) {
        T v = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[c] = v;
      }
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < C; ++c) atomicAdd(&vout[8 * (size_t)k + SLOT0 + c], acc[c]);
      }
    }
  }
}

template <typename T, int C, int SLOT0, int PT>
void launch_interp(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  static bool init = false;
  auto kern = k_interp<T, C, SLOT0, PT>;
  if (!init) {
    set_smem(kern);
    init = true;
  }
  size_t sm = (size_t)C * a.T[2] * a.T[1] * (a.T[0] + 1) * sizeof(T);
  kern<<<(unsigned)c->ntiles, 256, sm, s>>>(a, (const int4 *)c->d_sp_i0, (const typename V4<T>::t *)c->d_sp_d0,
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
