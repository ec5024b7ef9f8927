// Gaussian spreading Q (Sec. 2.3.2, Eq. WSops2) onto 16^3 grid tiles with the
// grid held in registers: every thread owns one (x, y) column of a tile, ZT
// consecutive z points of it, all C components, and accumulates into them; no
// shared-memory read-modify-write and no atomics.
//
// Work split: a CTA takes a tile from the work counter.  Its warps own 8 x 4
// column blocks (8 blocks cover the 16 x 16 columns; with ZT = 8 a second set
// of 8 warps takes the upper half of the z range).  Each warp scans, 32 at a
// time, the particles whose support starts lie in the 2 x 2 x 2 source bins of
// the tile (only the sub-block layers of the bins below that can reach it) and
// keeps those whose P^3 support overlaps its block.  For the kept particles the
// lanes write one record each to a per-warp queue in shared memory: the offsets
// of the support start from the tile origin, the x and y offsets of the
// particle from that start, the moments times the Gaussian prefactor, and the P
// z weights.  The warp then takes the records one by one (broadcast reads): each
// lane evaluates the x-y weight of its own column (zero outside the footprint)
// and adds weight x moment into the P z points the support covers.  The z start
// is the same on every lane, so a short tree of uniform branches selects the
// fully unrolled update with compile-time register indices.  At the end each
// thread writes its column once (8 consecutive x per 32-byte sector).
//
// Cost per particle and warp visit: four 16-byte shared reads, one exponential,
// C multiplications and P x C FMAs; a 6 x 6 footprint meets about 3.7 column
// blocks per z range of the tile.
//
// Interpolation sigma Q^T is the transpose on the same split: each thread loads
// its column's ZT x C grid values into registers once per tile; per queued
// particle every lane forms the P-point z sums of its column (P x C FMAs),
// weights them by its x-y weight, the warp sums the C values over its lanes in
// nine shuffles, and C lanes add the totals to the particle's outputs (one
// atomic add per component and warp visit).
#include "wave_common.cuh"

namespace pse {
namespace {

constexpr float COL_LOG2E = 1.4426950408889634f;

// Candidate ranges of the 8 source bins of a tile (see wave_cubic.cu).
struct ColRanges {
  int beg[8];
  int cum[9];
};

__device__ __forceinline__ int col_candidate(const ColRanges &r, int v) {
  int b = v >= r.cum[4] ? 4 : 0;
  b += v >= r.cum[b + 2] ? 2 : 0;
  b += v >= r.cum[b + 1] ? 1 : 0;
  return r.beg[b] + (v - r.cum[b]);
}

__device__ __forceinline__ int col_soff(int i0, int t0, int Ng, int P) {
  int o = i0 - t0;
  o += o < 0 ? Ng : 0;
  return o > Ng - P ? o - Ng : o;
}

// acc[z][c] += wz[j] * m[c] for z = ez + j in [0, ZT); ez (uniform over the
// warp) selects the case by a binary tree of branches, so every register index
// is a compile-time constant.
template <int LO, int HI, int ZT, int P, int C>
struct ZAdd {
  __device__ static __forceinline__ void run(int ez, float (&acc)[ZT][C], const float (&wz)[P], const float (&m)[C]) {
    if constexpr (LO == HI) {
#pragma unroll
      for (int j = 0; j < P; ++j) {
        if (LO + j >= 0 && LO + j < ZT) {
#pragma unroll
          for (int c = 0; c < C; ++c) acc[(LO + j >= 0 && LO + j < ZT) ? LO + j : 0][c] += wz[j] * m[c];
        }
      }
    } else {
      constexpr int MID = LO + (HI - LO) / 2;
      if (ez <= MID) ZAdd<LO, MID, ZT, P, C>::run(ez, acc, wz, m);
      else ZAdd<MID + 1, HI, ZT, P, C>::run(ez, acc, wz, m);
    }
  }
};

// out[c] = sum_j wz[j] g[ez + j][c] over the z = ez + j in [0, ZT) (uniform ez, as ZAdd).
template <int LO, int HI, int ZT, int P, int C>
struct ZDot {
  __device__ static __forceinline__ void run(int ez, const float (&g)[ZT][C], const float (&wz)[P], float (&out)[C]) {
    if constexpr (LO == HI) {
#pragma unroll
      for (int j = 0; j < P; ++j) {
        if (LO + j >= 0 && LO + j < ZT) {
#pragma unroll
          for (int c = 0; c < C; ++c) out[c] += wz[j] * g[(LO + j >= 0 && LO + j < ZT) ? LO + j : 0][c];
        }
      }
    } else {
      constexpr int MID = LO + (HI - LO) / 2;
      if (ez <= MID) ZDot<LO, MID, ZT, P, C>::run(ez, g, wz, out);
      else ZDot<MID + 1, HI, ZT, P, C>::run(ez, g, wz, out);
    }
  }
};

// Candidate ranges of a warp (source bins below the tile keep the sub-block layers that can reach the warp's z range), published to rg by the warp.
__device__ __forceinline__ void col_ranges(const SysDev &a, const int t[3], int wz0, int ZT, int P, int lane,
                                           const int *__restrict__ fine_start, ColRanges &rg) {
  constexpr int TS = CUBE;
  int beg = 0, len = 0;
  if (lane < 8) {
    const int bz = lane >> 2, by = (lane >> 1) & 1, bx = lane & 1;
    const int bzc = t[2] - bz < 0 ? t[2] - bz + a.nt[2] : t[2] - bz;
    const int byc = t[1] - by < 0 ? t[1] - by + a.nt[1] : t[1] - by;
    const int bxc = t[0] - bx < 0 ? t[0] - bx + a.nt[0] : t[0] - bx;
    const int64_t b = (int64_t)(a.tile0 + (bzc * a.nt[1] + byc) * a.nt[0] + bxc) * SUB_BLOCKS;
    const int zlo = max(0, wz0 - P + 1 + bz * TS), zhi = min(TS - 1, wz0 + ZT - 1 + bz * TS);
    if (zlo <= zhi) {
      beg = fine_start[b + (zlo * SUB_SIDE / TS) * SUB_SIDE * SUB_SIDE];
      len = fine_start[b + (zhi * SUB_SIDE / TS + 1) * SUB_SIDE * SUB_SIDE] - beg;
    }
  }
  int inc = lane < 8 ? len : 0;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane < 8) {
    rg.beg[lane] = beg;
    rg.cum[lane + 1] = inc;
  }
  if (lane == 0) rg.cum[0] = 0;
  __syncwarp();
}

// Floats of one queued particle record: [packed offsets, x offset, y offset, -,
// C moments, P z weights], padded to whole 16-byte vectors.
template <int C, int P>
struct ColRec {
  static constexpr int FLOATS = (4 + C + P + 3) / 4 * 4;
};

template <int C, int SLOT0, int P, int ZT>
__global__ void __launch_bounds__(32 * 8 * (16 / ZT), 16 / ZT == 1 ? 2 : 1)
    k_spread_col(WaveArgs wa, int *queue, const int4 *__restrict__ sp_i0, const float4 *__restrict__ sp_d0,
                 const float *__restrict__ vin, const int *__restrict__ fine_start, float *__restrict__ grid_all) {
  constexpr int TS = CUBE, NW = 8 * (TS / ZT), RF = ColRec<C, P>::FLOATS;
  static_assert(TS % ZT == 0, "z split");
  __shared__ __align__(16) float s_rec[NW][32 * RF];
  __shared__ ColRanges s_rng[NW];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int wx0 = (w & 1) * 8, wy0 = ((w >> 1) & 3) * 4, wz0 = (w >> 3) * ZT;
  const int cx = wx0 + (lane & 7), cy = wy0 + (lane >> 3);
  float *rec = s_rec[w];
  ColRanges &rg = s_rng[w];
  for_each_item(queue, wa.ntiles, [&](int item) {
    const int si = find_sys(wa.tile0, wa.nsys, item);
    const SysDev &a = wa.sys[si];
    if (wave_skip(wa, si, a)) return;
    const int Ng = a.Ng;
    int t[3], t0[3];
    tile_of(a, item - a.tile0, t, t0);
    // source bins of the tile; those one tile below in z keep the sub-block
    // layers whose supports can reach this warp's z range
    col_ranges(a, t, wz0, ZT, P, lane, fine_start, rg);
    const float nal = -(float)a.alpha * COL_LOG2E, hs = (float)a.h, pref = (float)a.pref;
    float acc[ZT][C];
#pragma unroll
    for (int z = 0; z < ZT; ++z)
#pragma unroll
      for (int c = 0; c < C; ++c) acc[z][c] = 0.f;
    const int total = rg.cum[8];
    for (int base = 0; base < total; base += 32) {
      const int v = base + lane;
      int k = 0, ex = 0, ey = 0, ez = 0;
      bool hit = false;
      if (v < total) {
        k = col_candidate(rg, v);
        const int4 i0 = sp_i0[k];
        ex = col_soff(i0.x, t0[0], Ng, P);
        ey = col_soff(i0.y, t0[1], Ng, P);
        ez = col_soff(i0.z, t0[2], Ng, P) - wz0;
        hit = ex > wx0 - P && ex < wx0 + 8 && ey > wy0 - P && ey < wy0 + 4 && ez > -P && ez < ZT;
      }
      const unsigned hits = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        // this lane's record: slot = rank of the lane among the hit lanes
        float *r = rec + RF * __popc(hits & ((1u << lane) - 1u));
        const float4 d0 = sp_d0[k];
        const float *row = vin + 8 * (size_t)k + SLOT0;
        float q[RF];
#pragma unroll
        for (int i = 0; i < RF; ++i) q[i] = 0.f;
        q[0] = __int_as_float((ex + 512) | ((ey + 512) << 10) | ((ez + 512) << 20));
        q[1] = d0.x;
        q[2] = d0.y;
#pragma unroll
        for (int c = 0; c < C; ++c) q[4 + c] = pref * row[c];
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const float oz = d0.z + (float)j * hs;
          q[4 + C + j] = exp2f(nal * oz * oz);
        }
#pragma unroll
        for (int i = 0; i < RF; i += 4) *(float4 *)(r + i) = make_float4(q[i], q[i + 1], q[i + 2], q[i + 3]);
      }
      __syncwarp();
      const int nh = __popc(hits);
      for (int h = 0; h < nh; ++h) {
        const float *r = rec + RF * h;
        float q[RF];
#pragma unroll
        for (int i = 0; i < RF; i += 4) {
          const float4 u = *(const float4 *)(r + i);
          q[i] = u.x;
          q[i + 1] = u.y;
          q[i + 2] = u.z;
          q[i + 3] = u.w;
        }
        const int pk = __float_as_int(q[0]);
        const int px = (pk & 1023) - 512, py = ((pk >> 10) & 1023) - 512, pz = (pk >> 20) - 512;
        const int jx = cx - px, jy = cy - py;
        const float ox = q[1] + (float)jx * hs, oy = q[2] + (float)jy * hs;
        float wxy = exp2f(nal * (ox * ox + oy * oy));
        wxy = ((unsigned)jx < (unsigned)P && (unsigned)jy < (unsigned)P) ? wxy : 0.f;
        float m[C], wz[P];
#pragma unroll
        for (int c = 0; c < C; ++c) m[c] = wxy * q[4 + c];
#pragma unroll
        for (int j = 0; j < P; ++j) wz[j] = q[4 + C + j];
        ZAdd<1 - P, ZT - 1, ZT, P, C>::run(pz, acc, wz, m);
      }
      __syncwarp();  // the records are read before the next round overwrites them
    }
    float *grid = grid_all + a.grid0;
    const size_t g0 = ((size_t)(t0[2] + wz0) * Ng + (t0[1] + cy)) * Ng + (t0[0] + cx);
#pragma unroll
    for (int z = 0; z < ZT; ++z)
#pragma unroll
      for (int c = 0; c < C; ++c) grid[c * a.gstride + g0 + (size_t)z * Ng * Ng] = acc[z][c];
  });
}

// Bit w set for each warp w whose column block (and z range, for ZT = 8) the P^3
// support with start offsets (ex, ey, ez) from the tile origin overlaps.
template <int NW, int ZT, int P>
__device__ __forceinline__ unsigned region_mask(int ex, int ey, int ez) {
  constexpr int TS = CUBE;
  if (ex <= -P || ex >= TS || ey <= -P || ey >= TS || ez <= -P || ez >= TS) return 0u;
  const unsigned xm = (ex <= 7 ? 1u : 0u) | (ex + P - 1 >= 8 ? 2u : 0u);
  const int ylo = max(ey, 0) >> 2, yhi = min(ey + P - 1, TS - 1) >> 2;
  unsigned m = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) m |= (b >= ylo && b <= yhi) ? xm << (2 * b) : 0u;
  if (ZT == TS) return m;
  const unsigned zm = (ez <= ZT - 1 ? 1u : 0u) | (ez + P - 1 >= ZT ? 2u : 0u);
  return ((zm & 1u) ? m : 0u) | ((zm & 2u) ? m << 8 : 0u);
}

// Spreading as k_spread_col, with the candidate scan shared by the CTA: in
// chunks of two candidates per thread, every thread tests its candidates
// against all column blocks, writes one record per candidate that reaches the
// tile, and appends its slot to the hit list of each warp whose block it meets;
// after a barrier each warp adds the records of its list into its columns.  One
// scan and one record per candidate instead of one per candidate and warp.
// DEF: deformed lattice (Sec. 2.3.3) with the z axis orthogonal to the sheared
// plane (A^T A couples x and y only): the x-y weight of a column is
// exp(-alpha (G_xx dx^2 + 2 G_xy dx dy + G_yy dy^2)) and the z weights use G_zz,
// from the suspension's coefficients SysDev::qa.
template <int C, int SLOT0, int P, int ZT, bool DEF = false>
__global__ void __launch_bounds__(32 * 8 * (16 / ZT), (16 / ZT == 1 || C <= 5) ? 2 : 1)
    k_spread_colq(WaveArgs wa, int *queue, const int4 *__restrict__ sp_i0, const float4 *__restrict__ sp_d0,
                  const float *__restrict__ vin, const int *__restrict__ fine_start, float *__restrict__ grid_all) {
  constexpr int TS = CUBE, NW = 8 * (TS / ZT), NT = 32 * NW, RF = ColRec<C, P>::FLOATS, CH = 2 * NT;
  static_assert(TS % ZT == 0 && NW <= 32, "z split");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *rec = (float *)smem_raw;                                       // CH records of RF floats
  unsigned short *lists = (unsigned short *)(rec + (size_t)CH * RF);    // NW lists of up to CH slots
  __shared__ int s_cnt[2][NW];
  __shared__ ColRanges s_rng;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int wx0 = (w & 1) * 8, wy0 = ((w >> 1) & 3) * 4, wz0 = (w >> 3) * ZT;
  const int cx = wx0 + (lane & 7), cy = wy0 + (lane >> 3);
  const unsigned below = (1u << lane) - 1u;
  for_each_item(queue, wa.ntiles, [&](int item) {
    const int si = find_sys(wa.tile0, wa.nsys, item);
    const SysDev &a = wa.sys[si];
    if (wave_skip(wa, si, a)) return;
    const int Ng = a.Ng;
    int t[3], t0[3];
    tile_of(a, item - a.tile0, t, t0);
    if (w == 0) col_ranges(a, t, 0, TS, P, lane, fine_start, s_rng);
    if (tid < 2 * NW) (&s_cnt[0][0])[tid] = 0;
    const float nal = -(float)a.alpha * COL_LOG2E, hs = (float)a.h, pref = (float)a.pref;
    // deformed lattice: exponent coefficients (base 2) of the x-y form and of z
    const float kxx = DEF ? -(float)a.qa[0] * COL_LOG2E : nal, kyy = DEF ? -(float)a.qa[1] * COL_LOG2E : nal;
    const float kxy = DEF ? -(float)a.qa[3] * COL_LOG2E : 0.f, kzz = DEF ? -(float)a.qa[2] * COL_LOG2E : nal;
    float acc[ZT][C];
#pragma unroll
    for (int z = 0; z < ZT; ++z)
#pragma unroll
      for (int c = 0; c < C; ++c) acc[z][c] = 0.f;
    __syncthreads();  // ranges and counters
    const int total = s_rng.cum[8];
    int par = 0;
    for (int base = 0; base < total; base += CH, par ^= 1) {
      int kk[2];
      int4 i0[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int v = base + tid + u * NT;
        kk[u] = v < total ? col_candidate(s_rng, v) : -1;
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (kk[u] >= 0) i0[u] = sp_i0[kk[u]];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        unsigned mask = 0;
        int ex = 0, ey = 0, ez = 0;
        if (kk[u] >= 0) {
          ex = col_soff(i0[u].x, t0[0], Ng, P);
          ey = col_soff(i0[u].y, t0[1], Ng, P);
          ez = col_soff(i0[u].z, t0[2], Ng, P);
          mask = region_mask<NW, ZT, P>(ex, ey, ez);
        }
        const int slot = tid + u * NT;
        if (mask) {
          const int k = kk[u];
          const float4 d0 = sp_d0[k];
          const float *row = vin + 8 * (size_t)k + SLOT0;
          float q[RF];
#pragma unroll
          for (int i = 0; i < RF; ++i) q[i] = 0.f;
          q[0] = __int_as_float((ex + 512) | ((ey + 512) << 10) | ((ez + 512) << 20));
          q[1] = d0.x;
          q[2] = d0.y;
#pragma unroll
          for (int c = 0; c < C; ++c) q[4 + c] = pref * row[c];
#pragma unroll
          for (int j = 0; j < P; ++j) {
            const float oz = d0.z + (float)j * hs;
            q[4 + C + j] = exp2f((DEF ? kzz : nal) * oz * oz);
          }
          float *r = rec + (size_t)slot * RF;
#pragma unroll
          for (int i = 0; i < RF; i += 4) *(float4 *)(r + i) = make_float4(q[i], q[i + 1], q[i + 2], q[i + 3]);
        }
        // append the slot to the list of every warp whose block the support meets
#pragma unroll
        for (int q = 0; q < NW; ++q) {
          const bool b = (mask >> q) & 1u;
          const unsigned bal = __ballot_sync(0xffffffffu, b);
          if (bal) {
            const int lead = __ffs(bal) - 1;
            int at = 0;
            if (lane == lead) at = atomicAdd(&s_cnt[par][q], __popc(bal));
            at = __shfl_sync(0xffffffffu, at, lead);
            if (b) lists[q * CH + at + __popc(bal & below)] = (unsigned short)slot;
          }
        }
      }
      __syncthreads();  // records and lists complete
      const int n = s_cnt[par][w];
      if (lane == 0) s_cnt[par ^ 1][w] = 0;  // the next chunk's counter (its appends follow the next barrier)
      for (int h = 0; h < n; ++h) {
        const float *r = rec + (size_t)lists[w * CH + h] * RF;
        float q[RF];
#pragma unroll
        for (int i = 0; i < RF; i += 4) {
          const float4 u4 = *(const float4 *)(r + i);
          q[i] = u4.x;
          q[i + 1] = u4.y;
          q[i + 2] = u4.z;
          q[i + 3] = u4.w;
        }
        const int pk = __float_as_int(q[0]);
        const int px = (pk & 1023) - 512, py = ((pk >> 10) & 1023) - 512, pz = (pk >> 20) - 512 - wz0;
        const int jx = cx - px, jy = cy - py;
        const float ox = q[1] + (float)jx * hs, oy = q[2] + (float)jy * hs;
        float wxy = DEF ? exp2f(kxx * ox * ox + kxy * ox * oy + kyy * oy * oy) : exp2f(nal * (ox * ox + oy * oy));
        wxy = ((unsigned)jx < (unsigned)P && (unsigned)jy < (unsigned)P) ? wxy : 0.f;
        float m[C], wz[P];
#pragma unroll
        for (int c = 0; c < C; ++c) m[c] = wxy * q[4 + c];
#pragma unroll
        for (int j = 0; j < P; ++j) wz[j] = q[4 + C + j];
        ZAdd<1 - P, ZT - 1, ZT, P, C>::run(pz, acc, wz, m);
      }
      __syncthreads();  // the records and lists are read before the next chunk overwrites them
    }
    float *grid = grid_all + a.grid0;
    const size_t g0 = ((size_t)(t0[2] + wz0) * Ng + (t0[1] + cy)) * Ng + (t0[0] + cx);
#pragma unroll
    for (int z = 0; z < ZT; ++z)
#pragma unroll
      for (int c = 0; c < C; ++c) grid[c * a.gstride + g0 + (size_t)z * Ng * Ng] = acc[z][c];
  });
}

// Floats of one queued interpolation record: [packed offsets, x offset, y
// offset, particle index, P z weights], padded to whole 16-byte vectors.
template <int P>
struct ColIRec {
  static constexpr int FLOATS = (4 + P + 3) / 4 * 4;
};

template <int C, int SLOT0, int P, int ZT>
__global__ void __launch_bounds__(32 * 8 * (16 / ZT), 16 / ZT == 1 ? 2 : 1)
    k_interp_col(WaveArgs wa, int *queue, const int4 *__restrict__ sp_i0, const float4 *__restrict__ sp_d0,
                 const int *__restrict__ fine_start, const float *__restrict__ grid_all, float *__restrict__ vout) {
  constexpr int TS = CUBE, NW = 8 * (TS / ZT), RF = ColIRec<P>::FLOATS;
  static_assert(TS % ZT == 0 && C <= 8, "z split, components");
  __shared__ __align__(16) float s_rec[NW][32 * RF];
  __shared__ ColRanges s_rng[NW];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int wx0 = (w & 1) * 8, wy0 = ((w >> 1) & 3) * 4, wz0 = (w >> 3) * ZT;
  const int cx = wx0 + (lane & 7), cy = wy0 + (lane >> 3);
  const int comp = reduce8_component(lane);
  float *rec = s_rec[w];
  ColRanges &rg = s_rng[w];
  for_each_item(queue, wa.ntiles, [&](int item) {
    const int si = find_sys(wa.tile0, wa.nsys, item);
    const SysDev &a = wa.sys[si];
    if (wave_skip(wa, si, a)) return;
    const int Ng = a.Ng;
    int t[3], t0[3];
    tile_of(a, item - a.tile0, t, t0);
    // this thread's column of the tile
    float g[ZT][C];
    {
      const float *grid = grid_all + a.grid0;
      const size_t g0 = ((size_t)(t0[2] + wz0) * Ng + (t0[1] + cy)) * Ng + (t0[0] + cx);
#pragma unroll
      for (int z = 0; z < ZT; ++z)
#pragma unroll
        for (int c = 0; c < C; ++c) g[z][c] = grid[c * a.gstride + g0 + (size_t)z * Ng * Ng];
    }
    col_ranges(a, t, wz0, ZT, P, lane, fine_start, rg);
    const float nal = -(float)a.alpha * COL_LOG2E, hs = (float)a.h, pref = (float)a.pref;
    const int total = rg.cum[8];
    for (int base = 0; base < total; base += 32) {
      const int v = base + lane;
      int k = 0, ex = 0, ey = 0, ez = 0;
      bool hit = false;
      if (v < total) {
        k = col_candidate(rg, v);
        const int4 i0 = sp_i0[k];
        ex = col_soff(i0.x, t0[0], Ng, P);
        ey = col_soff(i0.y, t0[1], Ng, P);
        ez = col_soff(i0.z, t0[2], Ng, P) - wz0;
        hit = ex > wx0 - P && ex < wx0 + 8 && ey > wy0 - P && ey < wy0 + 4 && ez > -P && ez < ZT;
      }
      const unsigned hits = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        float *r = rec + RF * __popc(hits & ((1u << lane) - 1u));
        const float4 d0 = sp_d0[k];
        float q[RF];
#pragma unroll
        for (int i = 0; i < RF; ++i) q[i] = 0.f;
        q[0] = __int_as_float((ex + 512) | ((ey + 512) << 10) | ((ez + 512) << 20));
        q[1] = d0.x;
        q[2] = d0.y;
        q[3] = __int_as_float(k);
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const float oz = d0.z + (float)j * hs;
          q[4 + j] = exp2f(nal * oz * oz);
        }
#pragma unroll
        for (int i = 0; i < RF; i += 4) *(float4 *)(r + i) = make_float4(q[i], q[i + 1], q[i + 2], q[i + 3]);
      }
      __syncwarp();
      const int nh = __popc(hits);
      for (int h = 0; h < nh; ++h) {
        const float *r = rec + RF * h;
        float q[RF];
#pragma unroll
        for (int i = 0; i < RF; i += 4) {
          const float4 u = *(const float4 *)(r + i);
          q[i] = u.x;
          q[i + 1] = u.y;
          q[i + 2] = u.z;
          q[i + 3] = u.w;
        }
        const int pk = __float_as_int(q[0]);
        const int px = (pk & 1023) - 512, py = ((pk >> 10) & 1023) - 512, pz = (pk >> 20) - 512;
        const int jx = cx - px, jy = cy - py;
        const float ox = q[1] + (float)jx * hs, oy = q[2] + (float)jy * hs;
        float wxy = pref * exp2f(nal * (ox * ox + oy * oy));
        wxy = ((unsigned)jx < (unsigned)P && (unsigned)jy < (unsigned)P) ? wxy : 0.f;
        float wz[P], part[C];
#pragma unroll
        for (int j = 0; j < P; ++j) wz[j] = q[4 + j];
#pragma unroll
        for (int c = 0; c < C; ++c) part[c] = 0.f;
        ZDot<1 - P, ZT - 1, ZT, P, C>::run(pz, g, wz, part);
        float v8[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) v8[c] = c < C ? wxy * part[c < C ? c : 0] : 0.f;
        const float tot = warp_reduce8(v8, lane);
        if ((lane & 3) == 0 && comp < C) atomicAdd(vout + 8 * (size_t)__float_as_int(q[3]) + SLOT0 + comp, tot);
      }
      __syncwarp();  // the records are read before the next round overwrites them
    }
  });
}

template <int C, int SLOT0, int P>
void launch_interp_col(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  static OccCache occ;
  constexpr int ZT = C > 5 ? 8 : 16;
  constexpr int NT = 32 * 8 * (CUBE / ZT);
  auto kern = k_interp_col<C, SLOT0, P, ZT>;
  const unsigned grid = wave_grid(c, kern, 0, a.ntiles, occ, NT);
  int *q = next_queue(c, s);
  kern<<<grid, NT, 0, s>>>(a, q, (const int4 *)c->d_sp_i0, (const float4 *)c->d_sp_d0, c->d_fine_start,
                           (const float *)c->d_grid, (float *)vout);
}

template <int C, int SLOT0>
void interp_col_p(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  switch (a.P) {
    case 5: launch_interp_col<C, SLOT0, 5>(c, a, vout, s); break;
    case 6: launch_interp_col<C, SLOT0, 6>(c, a, vout, s); break;
    default: launch_interp_col<C, SLOT0, 8>(c, a, vout, s);
  }
}

template <int C, int SLOT0, int P, int ZT, bool DEF = false>
void launch_spread_col_z(pse_ctx *c, const WaveArgs &a, const void *vin, cudaStream_t s) {
  constexpr int NT = 32 * 8 * (CUBE / ZT);
  int *q = next_queue(c, s);
  if (!DEF && (c->opt.wave_kernel & 4)) {  // every warp scans the candidates itself
    static OccCache occ;
    auto kern = k_spread_col<C, SLOT0, P, ZT>;
    const unsigned grid = wave_grid(c, kern, 0, a.ntiles, occ, NT);
    kern<<<grid, NT, 0, s>>>(a, q, (const int4 *)c->d_sp_i0, (const float4 *)c->d_sp_d0, (const float *)vin,
                             c->d_fine_start, (float *)c->d_grid);
    return;
  }
  static std::once_flag once;
  static OccCache occ;
  auto kern = k_spread_colq<C, SLOT0, P, ZT, DEF>;
  set_smem(kern, once);
  constexpr size_t sm = (size_t)2 * NT * ColRec<C, P>::FLOATS * sizeof(float) +
                        (size_t)(NT / 32) * 2 * NT * sizeof(unsigned short);
  const unsigned grid = wave_grid(c, kern, sm, a.ntiles, occ, NT);
  kern<<<grid, NT, sm, s>>>(a, q, (const int4 *)c->d_sp_i0, (const float4 *)c->d_sp_d0, (const float *)vin,
                            c->d_fine_start, (float *)c->d_grid);
}

// ZT: z points per thread, 8 (two z halves: 40 accumulators for 5 components,
// two 512-thread CTAs per SM; measured 13 % faster than whole columns) by
// default, 16 (one whole column per thread) for up to 5 components with bit 3
// of option wave_kernel.
template <int C, int SLOT0, int P>
void launch_spread_col(pse_ctx *c, const WaveArgs &a, const void *vin, cudaStream_t s) {
  if (c->lattice) launch_spread_col_z<C, SLOT0, P, 8, true>(c, a, vin, s);  // default split only
  else if (C <= 5 && (c->opt.wave_kernel & 8)) launch_spread_col_z<C, SLOT0, P, 16>(c, a, vin, s);
  else launch_spread_col_z<C, SLOT0, P, 8>(c, a, vin, s);
}

// P = 10 (the support Eq. bound gives on a cell sheared by 1/2) only with the
// default kernels (set_cubic admits it only then).
template <int C, int SLOT0>
void spread_col_p(pse_ctx *c, const WaveArgs &a, const void *vin, cudaStream_t s) {
  switch (a.P) {
    case 5: launch_spread_col<C, SLOT0, 5>(c, a, vin, s); break;
    case 6: launch_spread_col<C, SLOT0, 6>(c, a, vin, s); break;
    case 10:
      if (c->lattice) launch_spread_col_z<C, SLOT0, 10, 8, true>(c, a, vin, s);
      else launch_spread_col_z<C, SLOT0, 10, 8>(c, a, vin, s);
      break;
    default: launch_spread_col<C, SLOT0, 8>(c, a, vin, s);
  }
}

}  // namespace

void spread_col_launch(pse_ctx *c, const WaveArgs &a, const void *vin, int mode, cudaStream_t s) {
  if (mode == M_SE || mode == M_SU) spread_col_p<5, 3>(c, a, vin, s);
  else spread_col_p<8, 0>(c, a, vin, s);
}

void interp_col_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s) {
  if (mode == M_FULL) interp_col_p<8, 0>(c, a, vout, s);
  else if (mode == M_SE) interp_col_p<5, 3>(c, a, vout, s);
  else interp_col_p<3, 0>(c, a, vout, s);
}

}  // namespace pse
