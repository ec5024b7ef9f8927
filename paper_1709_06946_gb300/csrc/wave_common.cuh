// Spreading / interpolation kernels shared by wave_spread.cu and wave_interp.cu.
#pragma once

#include <cmath>

#include "device_common.cuh"
#include "pse_internal.cuh"

namespace pse {

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

struct WaveArgs {
  int N, Ng, P;
  int T[3], nt[3];
  double h, alpha, pref;
};

// x-direction weight of support point `lane` (lanes 0..P-1), read by the other
// lanes with a shuffle inside a warp-uniform loop.
template <typename T>
__device__ __forceinline__ T weight_lane(const WaveArgs &a, T d0x, int lane) {
  T d = d0x + (T)lane * (T)a.h;
  return lane < a.P ? exp(-(T)a.alpha * d * d) : (T)0;
}

__device__ __forceinline__ int tile_bins(const WaveArgs &a, int tile, int t0[3], int bins[8]) {
  int t[3] = {tile % a.nt[0], (tile / a.nt[0]) % a.nt[1], tile / (a.nt[0] * a.nt[1])};
  for (int d = 0; d < 3; ++d) t0[d] = t[d] * a.T[d];
  int nb = 0;
  int nz = a.nt[2] > 1 ? 2 : 1, ny = a.nt[1] > 1 ? 2 : 1, nx = a.nt[0] > 1 ? 2 : 1;
  for (int bz = 0; bz < nz; ++bz)
    for (int by = 0; by < ny; ++by)
      for (int bx = 0; bx < nx; ++bx) {
        int z = wrapi(t[2] - bz, a.nt[2]), y = wrapi(t[1] - by, a.nt[1]), x = wrapi(t[0] - bx, a.nt[0]);
        bins[nb++] = (z * a.nt[1] + y) * a.nt[0] + x;
      }
  return nb;
}


template <typename K>
inline void set_smem(K kern) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// launchers (wave_spread.cu / wave_interp.cu)
void spread_launch(pse_ctx *c, const WaveArgs &a, const void *vin, int mode, cudaStream_t s);
void interp_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s);

}  // namespace pse
