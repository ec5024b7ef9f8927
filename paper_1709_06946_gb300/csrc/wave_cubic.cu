// Spreading Q and interpolation sigma Q^T (Sec. 2.3.2, Eq. WSops2) specialised
// for mixed precision and 16^3 grid tiles with at least two tiles per side.
//
// The work split is that of the general kernels (persistent CTAs over tiles,
// a shared-memory tile, warps scanning candidate particles 32 at a time) with
// the per-particle overhead cut down: the tile strides are compile-time
// constants, offsets from the tile origin are signed (no periodic wrap tests:
// a footprint point is in the tile when (x | y) < 16 as unsigned), the three
// offsets travel in one shuffle, each lane's footprint positions are fixed for
// the whole kernel, the candidate ranges of the source bins sit in shared
// memory, and spreading lanes compute the Gaussian weight of their own point
// (no weight shuffles; interpolation keeps one 1D weight per lane, shuffled,
// because it needs the six z weights on every lane).  Interpolation warps take
// candidate groups from a counter in shared memory (the bins below the tile
// hold far fewer hits than the tile's own, so a static split leaves warps idle
// at the tile barrier) and skip the sub-block layers of the bins below the tile
// that cannot reach it.
#include "wave_common.cuh"

namespace pse {
namespace {

constexpr float LOG2E = 1.4426950408889634f;

// Candidate ranges of up to 8 source bins: beg[b], and cum[b] = candidates in bins < b.
struct Ranges {
  int beg[8];
  int cum[9];
};

// Lanes 0..7 hold bin b = lane's (beg, len); the warp forms the running sums
// and lane 0..8 writes the table.  Every lane of the warp must call it.
__device__ __forceinline__ void publish_ranges(Ranges &r, int lane, int beg, int len) {
  int inc = lane < 8 ? len : 0;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane < 8) {
    r.beg[lane] = beg;
    r.cum[lane + 1] = inc;
  }
  if (lane == 0) r.cum[0] = 0;
}

// Sum of v[0..8) over each 16-lane half of the warp in 8 shuffles: each exchange
// halves the components a lane keeps, so lane l of a half ends with the total
// of component 4 b3 + 2 b2 + b1 (b_k = bit k of l), the same in lanes l and l^1.
__device__ __forceinline__ float half_reduce8(const float v[8], int sub) {
  const bool b3 = (sub >> 3) & 1, b2 = (sub >> 2) & 1, b1 = (sub >> 1) & 1;
  float k4[4], k2[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float keep = b3 ? v[i + 4] : v[i], send = b3 ? v[i] : v[i + 4];
    k4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float keep = b2 ? k4[i + 2] : k4[i], send = b2 ? k4[i] : k4[i + 2];
    k2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  float k1 = (b1 ? k2[1] : k2[0]) + __shfl_xor_sync(0xffffffffu, b1 ? k2[0] : k2[1], 2);
  k1 += __shfl_xor_sync(0xffffffffu, k1, 1);
  return k1;
}
__device__ __forceinline__ int half_reduce8_component(int sub) {
  return 4 * ((sub >> 3) & 1) + 2 * ((sub >> 2) & 1) + ((sub >> 1) & 1);
}

// Particle index of candidate v < cum[8] (binary search over the 8 bins).
__device__ __forceinline__ int range_candidate(const Ranges &r, int v) {
  int b = v >= r.cum[4] ? 4 : 0;
  b += v >= r.cum[b + 2] ? 2 : 0;
  b += v >= r.cum[b + 1] ? 1 : 0;
  return r.beg[b] + (v - r.cum[b]);
}

// Global tile index of source bin b (bits: z, y, x step down) of tile t.
__device__ __forceinline__ int64_t source_bin(const SysDev &a, const int t[3], int b) {
  const int bz = b >> 2, by = (b >> 1) & 1, bx = b & 1;
  int z = t[2] - bz, y = t[1] - by, x = t[0] - bx;
  z += z < 0 ? a.nt[2] : 0;
  y += y < 0 ? a.nt[1] : 0;
  x += x < 0 ? a.nt[0] : 0;
  return a.tile0 + (z * a.nt[1] + y) * a.nt[0] + x;
}

// Signed offset of a support start from the tile origin along one axis.
__device__ __forceinline__ int soff(int i0, int t0, int Ng, int P) {
  int o = i0 - t0;
  o += o < 0 ? Ng : 0;
  return o > Ng - P ? o - Ng : o;
}

// moments [SLOT0, SLOT0 + C) of particle k (an 8-slot row), read by the whole warp
template <int C, int SLOT0>
__device__ __forceinline__ void moments(const float *__restrict__ vin, int k, float mv[C]) {
  const float *row = vin + 8 * (size_t)k;
  if (C == 5 && SLOT0 == 3) {
    mv[0] = row[3];
    const float4 q = *(const float4 *)(row + 4);
    mv[1] = q.x;
    mv[2] = q.y;
    mv[3] = q.z;
    mv[4] = q.w;
  } else if (C == 8 && SLOT0 == 0) {
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

// ------------------------------------------------------------------ spreading
template <int C, int SLOT0, int P>
__global__ void __launch_bounds__(WAVE_THREADS) k_spread16(WaveArgs wa, int *queue, const int4 *__restrict__ sp_i0,
                                                           const float4 *__restrict__ sp_d0,
                                                           const float *__restrict__ vin,
                                                           const int *__restrict__ fine_start,
                                                           float *__restrict__ grid_all) {
  constexpr int TS = CUBE, RX = tile_rx(TS, P), ZS = TS * RX, NPT = TS * ZS;
  constexpr int NPASS = (P * P + 31) / 32;
  static_assert(TS == WAVE_WARPS, "one z plane per warp");
  extern __shared__ __align__(32) unsigned char smem_raw[];
  __shared__ Ranges s_rng[WAVE_WARPS];
  TileL<float, C> tl;
  tl.init(smem_raw, NPT);
  const int lane = threadIdx.x & 31, lz = threadIdx.x >> 5;
  Ranges &rg = s_rng[lz];
  // lane roles fixed for the whole kernel: footprint point of each pass (an
  // invalid point gets x = 64, outside every tile)
  int jx[NPASS], jy[NPASS];
#pragma unroll
  for (int ps = 0; ps < NPASS; ++ps) {
    const int it = ps * 32 + lane;
    jx[ps] = it < P * P ? it % P : 64;
    jy[ps] = it < P * P ? it / P : 0;
  }
  for_each_item(queue, wa.ntiles, [&](int item) {
    const int si = find_sys(wa.tile0, wa.nsys, item);
    const SysDev &a = wa.sys[si];
    if (wave_skip(wa, si, a)) return;
    const int Ng = a.Ng;
    {
      float4 *z4 = (float4 *)smem_raw;
      const int n4 = (int)(TileL<float, C>::bytes(NPT) / 16);
      for (int q = threadIdx.x; q < n4; q += blockDim.x) z4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int t[3], t0[3];
    tile_of(a, item - a.tile0, t, t0);
    // candidate ranges of this warp's plane: per source bin, the sub-block z
    // layers whose support starts lie within P - 1 planes below it
    {
      int beg = 0, len = 0;
      if (lane < 8) {
        const int bz = lane >> 2;
        const int zlo = max(0, lz - P + 1 + bz * TS), zhi = min(TS - 1, lz + bz * TS);
        if (zlo <= zhi) {
          const int64_t b = source_bin(a, t, lane) * SUB_BLOCKS;
          beg = fine_start[b + (zlo * SUB_SIDE / TS) * SUB_SIDE * SUB_SIDE];
          len = fine_start[b + (zhi * SUB_SIDE / TS + 1) * SUB_SIDE * SUB_SIDE] - beg;
        }
      }
      publish_ranges(rg, lane, beg, len);
    }
    const float nal = -(float)a.alpha * LOG2E, hs = (float)a.h, pref = (float)a.pref;
    __syncthreads();  // tile cleared, ranges published
    const int total = rg.cum[8];
    for (int base = 0; base < total; base += 32) {
      const int v = base + lane;
      int k = 0, pk = 0;
      bool hit = false;
      if (v < total) {
        k = range_candidate(rg, v);
        const int4 i0 = sp_i0[k];
        const int sx = soff(i0.x, t0[0], Ng, P), sy = soff(i0.y, t0[1], Ng, P);
        const int jz = lz - soff(i0.z, t0[2], Ng, P);
        hit = (unsigned)(sx + P - 1) < (unsigned)(TS + P - 1) && (unsigned)(sy + P - 1) < (unsigned)(TS + P - 1) &&
              (unsigned)jz < (unsigned)P;
        pk = (sx + 512) | ((sy + 512) << 10) | (jz << 20);
      }
      unsigned hits = __ballot_sync(0xffffffffu, hit);
      while (hits) {
        const int src = __ffs(hits) - 1;
        hits &= hits - 1;
        const int ke = __shfl_sync(0xffffffffu, k, src), pe = __shfl_sync(0xffffffffu, pk, src);
        const int ex = (pe & 1023) - 512, ey = ((pe >> 10) & 1023) - 512, ez = pe >> 20;
        const float4 d0 = sp_d0[ke];
        float mv[C];
        moments<C, SLOT0>(vin, ke, mv);
        // weights computed by each lane for its own point (no shuffles: the
        // shared-memory pipe, not issue, limits this kernel)
        const float oz = d0.z + (float)ez * hs;
        const float wz = pref * exp2f(nal * oz * oz);
        const int pb = lz * ZS + ey * RX + ex;
#pragma unroll
        for (int ps = 0; ps < NPASS; ++ps) {
          const float ox = d0.x + (float)jx[ps] * hs, oy = d0.y + (float)jy[ps] * hs;
          const float wt = exp2f(nal * (ox * ox + oy * oy)) * wz;
          if ((unsigned)((ex + jx[ps]) | (ey + jy[ps])) < (unsigned)TS) {
            const int i = pb + jy[ps] * RX + jx[ps];
            float vv[C];
            tl.load(i, vv);
#pragma unroll
            for (int c = 0; c < C; ++c) vv[c] += wt * mv[c];
            tl.store(i, vv);
          }
        }
        __syncwarp();  // the next particle may update the same points from other lanes
      }
    }
    __syncthreads();
    float *grid = grid_all + a.grid0;
    for (int q = threadIdx.x; q < TS * TS * TS; q += blockDim.x) {
      const int x = q % TS, y = (q / TS) % TS, z = q / (TS * TS);
      const size_t g = ((size_t)(t0[2] + z) * Ng + (t0[1] + y)) * Ng + (t0[0] + x);
      float vv[C];
      tl.load(z * ZS + y * RX + x, vv);
#pragma unroll
      for (int c = 0; c < C; ++c) grid[c * a.gstride + g] = vv[c];
    }
    __syncthreads();  // the tile is read out before the next item clears it
  });
}

// -------------------------------------------------------------- interpolation
template <int C, int SLOT0, int P, int NT>
__global__ void __launch_bounds__(NT) k_interp16(WaveArgs wa, int *queue, const int4 *__restrict__ sp_i0,
                                                 const float4 *__restrict__ sp_d0,
                                                 const int *__restrict__ fine_start,
                                                 const float *__restrict__ grid_all, float *__restrict__ vout) {
  constexpr int TS = CUBE, RX = tile_rx(TS, P), ZS = TS * RX, NPT = TS * ZS;
  // footprint split: NFULL passes of whole (x, y) columns (P points along z) per
  // lane, then the REM leftover columns' REM * P points one per lane
  // two particles at a time, one per 16-lane half-warp: NFULL passes of whole
  // (x, y) columns (P points along z) per lane, then the REM leftover columns'
  // REM * P points one per lane over NMINI passes (P = 6: two full passes and
  // two leftover passes of 16 and 8 points)
  constexpr int NFULL = (P * P) / 16, REM = (P * P) % 16, NMINI = (REM * P + 15) / 16;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  __shared__ Ranges s_rng;
  __shared__ int s_next;
  TileL<float, C> tl;
  tl.init(smem_raw, NPT);
  const int lane = threadIdx.x & 31, half = lane >> 4, sub = lane & 15;
  int fx[NFULL > 0 ? NFULL : 1], fy[NFULL > 0 ? NFULL : 1];
  int mx[NMINI > 0 ? NMINI : 1], my[NMINI > 0 ? NMINI : 1], mz[NMINI > 0 ? NMINI : 1];
#pragma unroll
  for (int ps = 0; ps < NFULL; ++ps) {
    fx[ps] = (ps * 16 + sub) % P;
    fy[ps] = (ps * 16 + sub) / P;
  }
#pragma unroll
  for (int ms = 0; ms < NMINI; ++ms) {
    const int it = ms * 16 + sub;
    const int col = NFULL * 16 + (it < REM * P ? it / P : 0);
    mx[ms] = it < REM * P ? col % P : 64;  // invalid: outside every tile
    my[ms] = col / P;
    mz[ms] = it < REM * P ? it % P : 0;
  }
  // 1D Gaussian weights of the half's particle: index i < 3P (axis i / P, point
  // i % P) held by lane i (wa) or lane i - 16 (wb) of the half
  const int ia = sub, ib = 16 + sub;
  const int axa = ia / P, axb = ib < 3 * P ? ib / P : 2;
  const int ja = ia % P, jb = ib < 3 * P ? ib % P : 0;
  for_each_item(queue, wa.ntiles, [&](int item) {
    const int si = find_sys(wa.tile0, wa.nsys, item);
    const SysDev &a = wa.sys[si];
    if (wave_skip(wa, si, a)) return;
    const int Ng = a.Ng;
    int t[3], t0[3];
    tile_of(a, item - a.tile0, t, t0);
    const float *grid = grid_all + a.grid0;
    for (int q = threadIdx.x; q < TS * TS * TS; q += blockDim.x) {
      const int x = q % TS, y = (q / TS) % TS, z = q / (TS * TS);
      const size_t g = ((size_t)(t0[2] + z) * Ng + (t0[1] + y)) * Ng + (t0[0] + x);
      float vv[C];
#pragma unroll
      for (int c = 0; c < C; ++c) vv[c] = grid[c * a.gstride + g];
      tl.store(z * ZS + y * RX + x, vv);
    }
    if (threadIdx.x < 32) {
      // source bins; those one tile below keep only the sub-block z layers
      // whose supports can reach the tile
      int beg = 0, len = 0;
      if (lane < 8) {
        const int lo = (lane >> 2) ? (TS - P + 1) * SUB_SIDE / TS : 0;
        const int64_t b = source_bin(a, t, lane) * SUB_BLOCKS;
        beg = fine_start[b + lo * SUB_SIDE * SUB_SIDE];
        len = fine_start[b + SUB_BLOCKS] - beg;
      }
      publish_ranges(s_rng, lane, beg, len);
      if (lane == 0) s_next = 0;
    }
    const float nal = -(float)a.alpha * LOG2E, hs = (float)a.h, pref = (float)a.pref;
    const float jah = (float)ja * hs, jbh = (float)jb * hs;
    __syncthreads();  // tile staged, ranges published
    const int total = s_rng.cum[8];
    for (;;) {
      int g = 0;
      if (lane == 0) g = atomicAdd(&s_next, 1);
      const int base = __shfl_sync(0xffffffffu, g, 0) * 32;
      if (base >= total) break;
      const int v = base + lane;
      int k = 0, pk = 0;
      bool hit = false;
      if (v < total) {
        k = range_candidate(s_rng, v);
        const int4 i0 = sp_i0[k];
        const int sx = soff(i0.x, t0[0], Ng, P), sy = soff(i0.y, t0[1], Ng, P), sz = soff(i0.z, t0[2], Ng, P);
        hit = (unsigned)(sx + P - 1) < (unsigned)(TS + P - 1) && (unsigned)(sy + P - 1) < (unsigned)(TS + P - 1) &&
              (unsigned)(sz + P - 1) < (unsigned)(TS + P - 1);
        pk = (sx + 512) | ((sy + 512) << 10) | ((sz + 512) << 20);
      }
      unsigned mask = __ballot_sync(0xffffffffu, hit);
      while (mask) {
        // the next two hits: the first for half 0, the second (if any) for half 1
        const int src0 = __ffs(mask) - 1;
        mask &= mask - 1;
        const int src1 = mask ? __ffs(mask) - 1 : -1;
        if (mask) mask &= mask - 1;
        const int src = half ? src1 : src0;
        const bool live = src >= 0;
        const int ke = __shfl_sync(0xffffffffu, k, src & 31), pe = __shfl_sync(0xffffffffu, pk, src & 31);
        const int ex = (pe & 1023) - 512, ey = ((pe >> 10) & 1023) - 512, ez = (pe >> 20) - 512;
        const float4 d0 = sp_d0[ke];
        const float oa = (axa == 0 ? d0.x : (axa == 1 ? d0.y : d0.z)) + jah;
        const float ob = (axb == 0 ? d0.x : (axb == 1 ? d0.y : d0.z)) + jbh;
        const float wa = exp2f(nal * oa * oa), wb = exp2f(nal * ob * ob);
        float wz[P];
#pragma unroll
        for (int jz = 0; jz < P; ++jz)
          wz[jz] = 2 * P + jz < 16 ? __shfl_sync(0xffffffffu, wa, 2 * P + jz, 16)
                                   : __shfl_sync(0xffffffffu, wb, 2 * P + jz - 16, 16);
        const int pb = ez * ZS + ey * RX + ex;
        float acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = 0.f;
#pragma unroll
        for (int ps = 0; ps < NFULL; ++ps) {
          const float wxy = __shfl_sync(0xffffffffu, wa, fx[ps], 16) * __shfl_sync(0xffffffffu, wa, P + fy[ps], 16);
          if (live && (unsigned)((ex + fx[ps]) | (ey + fy[ps])) < (unsigned)TS) {
            const int col = pb + fy[ps] * RX + fx[ps];
#pragma unroll
            for (int jz = 0; jz < P; ++jz) {
              if ((unsigned)(ez + jz) < (unsigned)TS) {
                const float wt = wxy * wz[jz];
                float vv[C];
                tl.load(col + jz * ZS, vv);
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] += wt * vv[c];
              }
            }
          }
        }
#pragma unroll
        for (int ms = 0; ms < NMINI; ++ms) {
          const int iz = 2 * P + mz[ms];  // the z weight's index: lane iz (wa) or iz - 16 (wb)
          const float za = __shfl_sync(0xffffffffu, wa, iz & 15, 16), zb = __shfl_sync(0xffffffffu, wb, iz & 15, 16);
          const float wt = __shfl_sync(0xffffffffu, wa, mx[ms] & 15, 16) * __shfl_sync(0xffffffffu, wa, P + my[ms], 16) *
                           (iz < 16 ? za : zb);
          if (live && (unsigned)((ex + mx[ms]) | (ey + my[ms]) | (ez + mz[ms])) < (unsigned)TS) {
            float vv[C];
            tl.load(pb + mz[ms] * ZS + my[ms] * RX + mx[ms], vv);
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] += wt * vv[c];
          }
        }
        const float tot = half_reduce8(acc, sub);
        const int comp = half_reduce8_component(sub);
        if (live && (sub & 1) == 0 && comp < C) atomicAdd(vout + 8 * (size_t)ke + SLOT0 + comp, pref * tot);
      }
    }
    __syncthreads();  // the staged tile is no longer read when the next item overwrites it
  });
}

template <int C, int SLOT0, int P>
void launch_spread16(pse_ctx *c, const WaveArgs &a, const void *vin, cudaStream_t s) {
  static std::once_flag once;
  static OccCache occ;
  auto kern = k_spread16<C, SLOT0, P>;
  set_smem(kern, once);
  const size_t sm = TileL<float, C>::bytes((size_t)CUBE * CUBE * tile_rx(CUBE, P));
  const unsigned grid = wave_grid(c, kern, sm, a.ntiles, occ);
  int *q = next_queue(c, s);
  kern<<<grid, WAVE_THREADS, sm, s>>>(a, q, (const int4 *)c->d_sp_i0, (const float4 *)c->d_sp_d0, (const float *)vin,
                                      c->d_fine_start, (float *)c->d_grid);
}

template <int C, int SLOT0, int P>
void launch_interp16(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  static std::once_flag once;
  static OccCache occ;
  constexpr int NT = C == 8 ? 1024 : WAVE_THREADS;
  auto kern = k_interp16<C, SLOT0, P, NT>;
  set_smem(kern, once);
  const size_t sm = TileL<float, C>::bytes((size_t)CUBE * CUBE * tile_rx(CUBE, P));
  const unsigned grid = wave_grid(c, kern, sm, a.ntiles, occ, NT);
  int *q = next_queue(c, s);
  kern<<<grid, NT, sm, s>>>(a, q, (const int4 *)c->d_sp_i0, (const float4 *)c->d_sp_d0, c->d_fine_start,
                            (const float *)c->d_grid, (float *)vout);
}

template <int C, int SLOT0>
void spread16_p(pse_ctx *c, const WaveArgs &a, const void *vin, cudaStream_t s) {
  switch (a.P) {
    case 5: launch_spread16<C, SLOT0, 5>(c, a, vin, s); break;
    case 6: launch_spread16<C, SLOT0, 6>(c, a, vin, s); break;
    default: launch_spread16<C, SLOT0, 8>(c, a, vin, s);
  }
}

template <int C, int SLOT0>
void interp16_p(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  switch (a.P) {
    case 5: launch_interp16<C, SLOT0, 5>(c, a, vout, s); break;
    case 6: launch_interp16<C, SLOT0, 6>(c, a, vout, s); break;
    default: launch_interp16<C, SLOT0, 8>(c, a, vout, s);
  }
}

}  // namespace

void spread16_launch(pse_ctx *c, const WaveArgs &a, const void *vin, int mode, cudaStream_t s) {
  if (mode == M_SE || mode == M_SU) spread16_p<5, 3>(c, a, vin, s);
  else spread16_p<8, 0>(c, a, vin, s);
}

void interp16_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s) {
  if (mode == M_FULL) interp16_p<8, 0>(c, a, vout, s);
  else if (mode == M_SE) interp16_p<5, 3>(c, a, vout, s);
  else interp16_p<3, 0>(c, a, vout, s);
}

}  // namespace pse
