// Helpers of the spreading / interpolation kernels (wave_spread.cu and
// wave_interp.cu for any tile, wave_cubic.cu for 16^3 tiles).
//
// Both kernels are persistent: each CTA takes grid tiles (Tx x Ty x Tz points)
// of any suspension from a work counter and keeps the tile in shared memory,
// points in [z][y][x] order, components split into a vector array (components
// 0..3, one 16-byte access) and, for 5 or 8 components, a second array
// (component 4 alone, or components 4..7): one lane updates all components of
// one point with two accesses and no padding.
// The particles that can reach a tile are those of the 2x2x2 bins below it
// (bins hold particles by the grid index where their support starts); the warps
// scan these candidates themselves, 32 at a time with a ballot, so there is no
// shared particle list and no CTA barrier between the staging of a tile and its
// read-out.  The Gaussian weights of a particle are computed on the lanes: the 1D
// weights one per lane, broadcast with shuffles, or (16^3 spreading) each lane
// the weight of its own footprint point.
#pragma once

#include <cmath>

#include "device_common.cuh"
#include "pse_internal.cuh"

namespace pse {

// Gaussian constants of a suspension in the arithmetic type of a kernel: the
// FP32 form reads the FP32 copies, so no FP64 conversion runs per particle or
// support point.
template <typename T>
__device__ __forceinline__ T sd_alpha(const SysDev &a) {
  if constexpr (sizeof(T) == 4) return a.alphaf;
  else return a.alpha;
}
template <typename T>
__device__ __forceinline__ T sd_h(const SysDev &a) {
  if constexpr (sizeof(T) == 4) return a.hf;
  else return a.h;
}
template <typename T>
__device__ __forceinline__ T sd_pref(const SysDev &a) {
  if constexpr (sizeof(T) == 4) return a.preff;
  else return a.pref;
}
template <typename T>
__device__ __forceinline__ T sd_qa(const SysDev &a, int k) {
  if constexpr (sizeof(T) == 4) return a.qaf[k];
  else return a.qa[k];
}

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

// Launch-wide arguments; the per-suspension ones come from SysDev.
struct WaveArgs {
  int P, nsys, ntiles;
  int want;            // -1: every suspension; 0 / 1: only those with SysDev::cubic = want
  const SysDev *sys;
  const int *tile0;   // nsys + 1 prefix of tiles
  const int *active;
};

constexpr int WAVE_THREADS = 512;
constexpr int WAVE_WARPS = WAVE_THREADS / 32;

// Padded row length (points) of the shared tile.  Rows of 16 points or more:
// the smallest RX >= Tx with RX = P (mod 8); a warp that takes footprint point
// (j mod P, j / P) in lane j then touches 16-byte slots RX (j / P) + j mod P = j
// (mod 8), so each quarter warp of a 16-byte access hits 8 different bank
// groups.  Shorter rows (where that padding would cost up to 7/8 of the tile):
// 2 points of padding when Tx is a multiple of 4.
__host__ __device__ constexpr int tile_rx(int Tx, int P) {
  return Tx >= 16 ? Tx + (((P - Tx) % 8) + 8) % 8 : Tx + ((Tx & 3) == 0 ? 2 : 0);
}

template <int C> struct CPad { static constexpr int v = C <= 4 ? 4 : 8; };

// Tile storage for C components: a[i] holds components 0..3 of point i, b the
// rest (one real for C = 5, a second vector for C = 8, nothing for C <= 4).
template <typename T, int C>
struct TileL {
  using T4 = typename V4<T>::t;
  static constexpr int EXTRA = C == 5 ? 1 : (C == 8 ? 4 : 0);  // reals per point in b
  // rounded up to 64 bytes so that the particle list after the tile stays aligned
  // (5 components take 20 or 40 bytes per point)
  __host__ __device__ static size_t bytes(size_t npts) {
    size_t b = npts * (sizeof(T4) + (EXTRA == 4 ? sizeof(T4) : EXTRA * sizeof(T)));
    return (b + 63) / 64 * 64;
  }
  T4 *a;
  void *b;
  __device__ void init(void *base, int npts) {
    a = (T4 *)base;
    b = (void *)(a + npts);
  }
  // address of component c of point i
  __device__ __forceinline__ T *comp(int i, int c) const {
    if (c < 4) return &a[i].x + c;
    if (EXTRA == 1) return (T *)b + i;
    return &((T4 *)b)[i].x + (c - 4);
  }
  __device__ __forceinline__ void load(int i, T v[C]) const {
    const T4 x = a[i];
    v[0] = x.x;
    if (C > 1) v[1] = x.y;
    if (C > 2) v[2] = x.z;
    if (C > 3) v[3] = x.w;
    if (EXTRA == 1) v[4] = ((const T *)b)[i];
    if (EXTRA == 4) {
      const T4 y = ((const T4 *)b)[i];
      v[4] = y.x;
      v[5] = y.y;
      v[6] = y.z;
      v[7] = y.w;
    }
  }
  __device__ __forceinline__ void store(int i, const T v[C]) const {
    T4 x;
    x.x = v[0];
    x.y = C > 1 ? v[1] : (T)0;
    x.z = C > 2 ? v[2] : (T)0;
    x.w = C > 3 ? v[3] : (T)0;
    a[i] = x;
    if (EXTRA == 1) ((T *)b)[i] = v[4];
    if (EXTRA == 4) {
      T4 y;
      y.x = v[4];
      y.y = v[5];
      y.z = v[6];
      y.w = v[7];
      ((T4 *)b)[i] = y;
    }
  }
};

// shared memory of a spreading/interpolation CTA (the tile)
template <typename T, int C>
__host__ __device__ inline size_t wave_smem(const int T3[3], int P) {
  return TileL<T, C>::bytes((size_t)T3[2] * T3[1] * tile_rx(T3[0], P));
}

// Sum of v[0..8) over the warp in 9 shuffles: each exchange halves the
// components a lane keeps, so lane l ends with the total of component
// 4 b4 + 2 b3 + b2 (b_k = bit k of l), the same in the four lanes l, l^1, l^2, l^3.
template <typename T>
__device__ __forceinline__ T warp_reduce8(const T v[8], int lane) {
  const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
  T k4[4], k2[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const T keep = b4 ? v[i + 4] : v[i], send = b4 ? v[i] : v[i + 4];
    k4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const T keep = b3 ? k4[i + 2] : k4[i], send = b3 ? k4[i] : k4[i + 2];
    k2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  T k1 = (b2 ? k2[1] : k2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? k2[0] : k2[1], 4);
  k1 += __shfl_xor_sync(0xffffffffu, k1, 2);
  k1 += __shfl_xor_sync(0xffffffffu, k1, 1);
  return k1;
}
__device__ __forceinline__ int reduce8_component(int lane) {
  return 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
}

__device__ __forceinline__ void tile_of(const SysDev &a, int tile, int t[3], int t0[3]) {
  t[0] = tile % a.nt[0];
  t[1] = (tile / a.nt[0]) % a.nt[1];
  t[2] = tile / (a.nt[0] * a.nt[1]);
  for (int d = 0; d < 3; ++d) t0[d] = t[d] * a.T[d];
}

// The (up to) 8 source bins of a tile and the running offsets of their ranges.
__device__ __forceinline__ int tile_bins(const SysDev &a, const int t[3], const int *tile_start, int beg[8],
                                         int cum[9]) {
  int nb = 0;
  int nz = a.nt[2] > 1 ? 2 : 1, ny = a.nt[1] > 1 ? 2 : 1, nx = a.nt[0] > 1 ? 2 : 1;
  cum[0] = 0;
  for (int bz = 0; bz < nz; ++bz)
    for (int by = 0; by < ny; ++by)
      for (int bx = 0; bx < nx; ++bx) {
        int z = wrapi(t[2] - bz, a.nt[2]), y = wrapi(t[1] - by, a.nt[1]), x = wrapi(t[0] - bx, a.nt[0]);
        int b = a.tile0 + (z * a.nt[1] + y) * a.nt[0] + x;
        beg[nb] = tile_start[b];
        cum[nb + 1] = cum[nb] + (tile_start[b + 1] - tile_start[b]);
        ++nb;
      }
  return nb;
}

// Candidates of plane lz of a tile for a spreading warp: per source bin, only
// the sub-block z-layers (particles are sorted by 4 x 4 x 4 sub-blocks of their
// tile, z-layer major) whose support starts can reach the plane, i.e. whose
// start z within its tile lies in [lz - P + 1, lz] (same z layer of tiles) or
// [Tz + lz - P + 1, Tz + lz] (the layer below).  With one tile along z (where
// supports wrap onto the same tile) every bin is taken whole.
__device__ __forceinline__ int plane_bins(const SysDev &a, const int t[3], int lz, int P, const int *fine_start,
                                          int beg[8], int cum[9]) {
  int nb = 0;
  const int nz = a.nt[2] > 1 ? 2 : 1, ny = a.nt[1] > 1 ? 2 : 1, nx = a.nt[0] > 1 ? 2 : 1, Tz = a.T[2];
  cum[0] = 0;
  for (int bz = 0; bz < nz; ++bz) {
    int lo = 0, hi = SUB_SIDE - 1;
    if (nz > 1) {
      const int zlo = max(0, lz - P + 1 + bz * Tz), zhi = min(Tz - 1, lz + bz * Tz);
      if (zlo > zhi) continue;
      lo = zlo * SUB_SIDE / Tz;
      hi = zhi * SUB_SIDE / Tz;
    }
    const int z = wrapi(t[2] - bz, a.nt[2]);
    for (int by = 0; by < ny; ++by)
      for (int bx = 0; bx < nx; ++bx) {
        const int y = wrapi(t[1] - by, a.nt[1]), x = wrapi(t[0] - bx, a.nt[0]);
        const int64_t b = (int64_t)(a.tile0 + (z * a.nt[1] + y) * a.nt[0] + x) * SUB_BLOCKS;
        beg[nb] = fine_start[b + lo * SUB_SIDE * SUB_SIDE];
        cum[nb + 1] = cum[nb] + (fine_start[b + (hi + 1) * SUB_SIDE * SUB_SIDE] - beg[nb]);
        ++nb;
      }
  }
  return nb;
}

// Particle index of candidate v (0 <= v < cum[nb]) of the tile's bins.
__device__ __forceinline__ int candidate(int v, int nb, const int beg[8], const int cum[9]) {
  int b = 0;
  while (b + 1 < nb && v >= cum[b + 1]) ++b;
  return beg[b] + (v - cum[b]);
}

// Offsets (wrapped) of a support start from the tile origin; true if the P^3
// support overlaps the tile.
__device__ __forceinline__ bool overlaps(const SysDev &a, int P, const int t0[3], const int4 &i0, int &ox, int &oy,
                                         int &oz) {
  const int Ng = a.Ng;
  ox = i0.x - t0[0];  // in (-Ng, Ng): support starts and tile origins lie in [0, Ng)
  oy = i0.y - t0[1];
  oz = i0.z - t0[2];
  ox += ox < 0 ? Ng : 0;
  oy += oy < 0 ? Ng : 0;
  oz += oz < 0 ? Ng : 0;
  return (ox < a.T[0] || ox + P - 1 >= Ng) && (oy < a.T[1] || oy + P - 1 >= Ng) &&
         (oz < a.T[2] || oz + P - 1 >= Ng);
}

// Signed offset of a support start from the tile origin (in (-P, T) for a
// support that overlaps the tile when there are at least two tiles per side),
// and the three packed into one int (10 bits each, biased by 512) for a shuffle.
__device__ __forceinline__ int signed_offset(int o, int Ng, int P) { return o > Ng - P ? o - Ng : o; }
__device__ __forceinline__ int pack_offsets(int x, int y, int z) { return (x + 512) | ((y + 512) << 10) | ((z + 512) << 20); }
__device__ __forceinline__ void unpack_offsets(int p, int &x, int &y, int &z) {
  x = (p & 1023) - 512;
  y = ((p >> 10) & 1023) - 512;
  z = ((p >> 20) & 1023) - 512;
}

// One 1D Gaussian weight per lane: lanes [0, P) along x, [P, 2P) along y,
// [2P, 3P) along z (3P <= 32); exp(-alpha (d0 + j h)^2).
template <typename T>
__device__ __forceinline__ T lane_weight(int lane, int P, T alpha, T hs, const typename V4<T>::t &d0) {
  if (lane >= 3 * P) return (T)0;
  const int d = lane / P, j = lane - d * P;
  const T o = (d == 0 ? d0.x : (d == 1 ? d0.y : d0.z)) + (T)j * hs;
  return exp(-alpha * o * o);
}

// launchers (wave_spread.cu / wave_interp.cu)
WaveArgs wave_args(const pse_ctx *c);
void spread_launch(pse_ctx *c, const WaveArgs &a, const void *vin, int mode, cudaStream_t s);
void interp_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s);

// Largest shared memory of a spreading/interpolation CTA over the suspensions
// of a launch (want as in WaveArgs).
template <typename T, int C>
inline size_t wave_smem_max(const pse_ctx *c, int want = -1) {
  size_t m = 0;
  for (const SysDev &q : c->hs) {
    if (want >= 0 && q.cubic != want) continue;
    size_t v = wave_smem<T, C>(q.T, c->p.P);
    if (v > m) m = v;
  }
  return m;
}

// The kernels specialised for 16^3 tiles run the suspensions marked
// SysDev::cubic (mixed precision, P = 5, 6 or 8, at least two tiles per side, so
// that a support crosses the periodic boundary into another tile, never back
// into the same one, and offsets from the tile origin can be kept signed); the
// general kernels run the others.  WaveArgs::want selects the suspensions of a
// launch: -1 all, 0 the unmarked ones, 1 the marked ones.
constexpr int CUBE = CUBE_TILE;
__device__ __forceinline__ bool wave_skip(const WaveArgs &wa, int si, const SysDev &a) {
  return !wa.active[si] || (wa.want >= 0 && a.cubic != wa.want);
}
void spread16_launch(pse_ctx *c, const WaveArgs &a, const void *vin, int mode, cudaStream_t s);
void spread_col_launch(pse_ctx *c, const WaveArgs &a, const void *vin, int mode, cudaStream_t s);
void interp_col_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s);
// General interpolation kernels (any tile) for the suspensions a selects; the
// 16^3-tile kernels fall back to them where their staging does not fit.
void interp_general_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s);
// 11-moment product (12-slot rows [F, L, S] / [U, Omega, E]), general kernels
void spread11_launch(pse_ctx *c, const void *vin12, cudaStream_t s);
void interp11_launch(pse_ctx *c, void *vout12, cudaStream_t s);
void interp16_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s);
void interp_halo_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s);

// Persistent grid of a wave kernel for a given shared-memory size (occupancy
// looked up once per kernel and size; handles on several threads share the cache).
struct OccCache {
  std::mutex mu;
  size_t smem[8] = {0};
  int per_sm[8] = {0};
};

template <typename K>
inline unsigned wave_grid(pse_ctx *c, K kern, size_t smem, int items, OccCache &oc, int threads = WAVE_THREADS) {
  std::atomic<int> v{0};
  {
    std::lock_guard<std::mutex> g(oc.mu);
    for (int k = 0; k < 8; ++k)
      if (oc.per_sm[k] > 0 && oc.smem[k] == smem) v.store(oc.per_sm[k]);
  }
  const bool known = v.load() > 0;
  unsigned grid = persistent_grid(c, kern, threads, smem, items, v);
  if (!known) {
    std::lock_guard<std::mutex> g(oc.mu);
    for (int k = 0; k < 8; ++k)
      if (oc.per_sm[k] <= 0) {
        oc.smem[k] = smem;
        oc.per_sm[k] = v.load();
        break;
      }
  }
  return grid;
}

// Allows the kernel the device's opt-in shared memory per block minus its own
// static shared memory.
template <typename K>
inline void set_smem(K kern, std::once_flag &once) {
  std::call_once(once, [&] {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    cudaGetLastError();
  });
}

}  // namespace pse
