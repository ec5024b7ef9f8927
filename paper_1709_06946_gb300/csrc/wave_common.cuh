// Spreading / interpolation kernels shared by wave_spread.cu and wave_interp.cu.
//
// Both kernels are persistent: each CTA takes grid tiles (Tx x Ty x Tz points)
// of any suspension from a work counter and keeps the tile in shared memory,
// points in [z][y][x] order, components split into a vector array (components
// 0..3, one 16-byte access) and, for 5 or 8 components, a second array
// (component 4 alone, or components 4..7): one lane updates all components of
// one point with two accesses and no padding.
// The CTA walks the particles of the 2x2x2 bins whose Gaussian supports can
// reach the tile (bins hold particles by the grid index where their support
// starts) in chunks: the particles that overlap the tile are compacted into a
// shared-memory list together with their offsets, weights' origins and
// moments, then processed by the warps.
#pragma once

#include <cmath>

#include "device_common.cuh"
#include "pse_internal.cuh"

namespace pse {

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

// Launch-wide arguments; the per-suspension ones come from SysDev.
struct WaveArgs {
  int P, nsys, ntiles;
  const SysDev *sys;
  const int *tile0;   // nsys + 1 prefix of tiles
  const int *active;
};

constexpr int WAVE_THREADS = 512;
constexpr int WAVE_WARPS = WAVE_THREADS / 32;
constexpr int LIST_CAP = 128;
constexpr int WMAX = 8;   // weights kept in the list for supports up to WMAX points per side

// padded row length (points) of the shared tile: keeps vector accesses of
// neighbouring rows in different banks
__host__ __device__ inline int tile_rx(int Tx) { return Tx + ((Tx & 3) == 0 ? 2 : 0); }

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

// shared memory of a spreading/interpolation CTA (tile + particle list)
template <typename T, int C>
__host__ __device__ inline size_t wave_smem(const int T3[3]) {
  constexpr int CP = CPad<C>::v;
  return TileL<T, C>::bytes((size_t)T3[2] * T3[1] * tile_rx(T3[0])) +
         (size_t)LIST_CAP * (sizeof(int4) + 4 * sizeof(T) + CP * sizeof(T) + 3 * WMAX * sizeof(T));
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

// Compacts the candidates [c0, c0 + LIST_CAP) of the tile's bins that overlap
// the tile into the shared list (offsets, weight origins, moments when vin is
// given, and the 3 x P one-dimensional Gaussian weights when P <= WMAX);
// returns the number of entries (after a barrier).
// Candidate order of the chunks: with SPREAD, candidate v of n is taken at
// (v * stride) mod n for a stride coprime to n, so that every chunk samples the
// whole tile (the sorted order is spatially coherent; a chunk of neighbouring
// particles would cross only a few z planes and leave most plane-owning warps idle).
__device__ __forceinline__ int spread_stride(int n) {
  int st = 97;
  for (;;) {  // the first odd stride from 97 that is coprime to n (a few steps at most)
    int x = n, y = st;
    while (y) {
      int r = x % y;
      x = y;
      y = r;
    }
    if (x == 1 || n <= 1) return st;
    st += 2;
  }
}

template <typename T, int C, int SLOT0, bool SPREAD = false>
__device__ __forceinline__ int build_list(const SysDev &a, int P, const int t0[3], int nb, const int beg[8],
                                          const int cum[9],
                                          int c0, const int4 *__restrict__ sp_i0,
                                          const typename V4<T>::t *__restrict__ sp_d0, const T *__restrict__ vin,
                                          int4 *s_meta, typename V4<T>::t *s_d0, T *s_m, T *s_w, int *s_count) {
  constexpr int CP = CPad<C>::v;
  const int Ng = a.Ng;
  const int total = cum[nb];
  const int st = SPREAD ? spread_stride(total) : 1;
  for (int q = threadIdx.x; q < LIST_CAP; q += blockDim.x) {
    int v = c0 + q;
    if (v >= total) break;
    if (SPREAD) v = (int)(((int64_t)v * st) % total);
    int b = 0;
    while (v >= cum[b + 1]) ++b;
    int k = beg[b] + (v - cum[b]);
    int4 i0 = sp_i0[k];
    int ox = wrapi(i0.x - t0[0], Ng), oy = wrapi(i0.y - t0[1], Ng), oz = wrapi(i0.z - t0[2], Ng);
    bool hit = (ox < a.T[0] || ox + P - 1 >= Ng) && (oy < a.T[1] || oy + P - 1 >= Ng) &&
               (oz < a.T[2] || oz + P - 1 >= Ng);
    if (hit) {
      int e = atomicAdd(s_count, 1);
      s_meta[e] = make_int4(k, ox, oy, oz);
      typename V4<T>::t d0 = sp_d0[k];
      s_d0[e] = d0;
      if (vin) {
#pragma unroll
        for (int c = 0; c < CP; ++c) s_m[e * CP + c] = c < C ? vin[8 * (size_t)k + SLOT0 + c] : (T)0;
      }
      if (P <= WMAX) {
        const T al = (T)a.alpha, hs = (T)a.h;
        T *w = s_w + e * 3 * WMAX;
        for (int j = 0; j < P; ++j) {
          T dx = d0.x + (T)j * hs, dy = d0.y + (T)j * hs, dz = d0.z + (T)j * hs;
          w[j] = exp(-al * dx * dx);
          w[WMAX + j] = exp(-al * dy * dy);
          w[2 * WMAX + j] = exp(-al * dz * dz);
        }
      }
    }
  }
  __syncthreads();
  return *s_count;
}

// launchers (wave_spread.cu / wave_interp.cu)
WaveArgs wave_args(const pse_ctx *c);
void spread_launch(pse_ctx *c, const WaveArgs &a, const void *vin, int mode, cudaStream_t s);
void interp_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s);

// Largest shared memory of a spreading/interpolation CTA over the suspensions.
template <typename T, int C>
inline size_t wave_smem_max(const pse_ctx *c) {
  size_t m = 0;
  for (const SysDev &q : c->hs) {
    size_t v = wave_smem<T, C>(q.T);
    if (v > m) m = v;
  }
  return m;
}

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
