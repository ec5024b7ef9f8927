// Interpolation sigma Q^T (Sec. 2.3.2, Eq. WSops2) for 16^3 tiles, mixed precision,
// with the whole support region of a group of particles staged in shared memory.
//
// Work item: one z-layer of a tile, i.e. the particles whose support starts lie in
// the tile and in one of its SUB_SIDE layers of 16/SUB_SIDE planes (one contiguous
// range of the sort by tile and sub-block).  Their supports lie inside the region
// [t0x, t0x + 16 + P - 1) x [t0y, t0y + 16 + P - 1) x [z0, z0 + 16/SUB_SIDE + P - 1),
// which the CTA copies from the grid (periodic wrap) into shared memory in the
// TileL layout.  Each particle is then read out once and complete by one quarter
// warp: its 8 lanes take the P x P columns of the support (column l + 8 s on lane
// l), walk each column along z, and the quarter sums its lanes with three
// shuffles, so every output row is written by one lane with no atomic addition
// (the tile-owned kernel splits a support over up to 8 tiles and adds the parts).
// Two CTAs share an SM (about 83 KB each for 5 components, P = 6), so one CTA's
// staging overlaps the other's read-out.
#include "wave_common.cuh"

namespace pse {
namespace {

constexpr int HALO_THREADS = 512;

// 4 bytes from global to shared memory without a register round trip (cp.async,
// cached in L1); completion is awaited with cp_async_wait_all before a barrier.
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
constexpr float HALO_LOG2E = 1.4426950408889634f;  // log2(e): exp(-x) = exp2(-x log2 e)
constexpr int LAYER = CUBE / SUB_SIDE;  // planes of support starts per work item

template <int P> struct Halo {
  static constexpr int R = CUBE + P - 1;           // region side along x and y
  static constexpr int RZ = LAYER + P - 1;         // region depth along z
  static constexpr int RX = tile_rx(R, P);         // padded row (RX = P mod 8: conflict-free quarter reads)
  static constexpr int ZS = R * RX;                // plane stride (points)
  static constexpr int NPT = RZ * ZS;              // points of the staged region
  static constexpr int NCOL = (P * P + 7) / 8;     // column passes per lane
};

// DEF: deformed lattice with z orthogonal to the sheared plane (as the
// register-column spreading): the x-y weight of each support column is its own
// exponential of the x-y quadratic form; the z weights use G_zz.
// COMP0: first grid component read (grid components COMP0 .. COMP0 + C - 1 go
// to output slots SLOT0 .. SLOT0 + C - 1).
template <int C, int SLOT0, int P, bool DEF = false, int COMP0 = 0>
__global__ void __launch_bounds__(HALO_THREADS, 2)
    k_interp_halo(WaveArgs wa, int *queue, const int4 *__restrict__ sp_i0, const float4 *__restrict__ sp_d0,
                  const int *__restrict__ fine_start, const float *__restrict__ grid_all, float *__restrict__ vout) {
  using H = Halo<P>;
  constexpr int R = H::R, RZ = H::RZ, RX = H::RX, ZS = H::ZS;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  TileL<float, C> tl;
  tl.init(smem_raw, H::NPT);
  const int lane = threadIdx.x & 31, quarter = lane >> 3, sub = lane & 7, warp = threadIdx.x >> 5;
  for_each_item(queue, wa.ntiles * SUB_SIDE, [&](int item) {
    const int tile = item / SUB_SIDE, kz = item % SUB_SIDE;
    const int si = find_sys(wa.tile0, wa.nsys, tile);
    const SysDev &a = wa.sys[si];
    if (wave_skip(wa, si, a)) return;
    const int Ng = a.Ng;
    int t[3], t0[3];
    tile_of(a, tile - a.tile0, t, t0);
    const int z0 = t0[2] + kz * LAYER;
    const float *grid = grid_all + a.grid0;
    // stage the region with asynchronous 4-byte copies straight into the tile layout
    // (no register round trip: every copy of the thread is in flight before the wait)
    constexpr int NREG = RZ * R * R;
    for (int q = threadIdx.x; q < NREG; q += HALO_THREADS) {
      const int x = q % R, y = (q / R) % R, z = q / (R * R);
      int gx = t0[0] + x, gy = t0[1] + y, gz = z0 + z;
      gx -= gx >= Ng ? Ng : 0;
      gy -= gy >= Ng ? Ng : 0;
      gz -= gz >= Ng ? Ng : 0;
      const size_t g = ((size_t)gz * Ng + gy) * Ng + gx;
      const int d = z * ZS + y * RX + x;
#pragma unroll
      for (int c = 0; c < C; ++c) cp_async4(tl.comp(d, c), grid + (COMP0 + c) * a.gstride + g);
    }
    cp_async_wait_all();
    const int64_t fb = (int64_t)tile * SUB_BLOCKS + kz * SUB_SIDE * SUB_SIDE;
    const int beg = fine_start[fb], end = fine_start[fb + SUB_SIDE * SUB_SIDE];
    const float nal = -(float)a.alpha * HALO_LOG2E, hs = (float)a.h, pref = (float)a.pref;
    const float kxx = DEF ? -(float)a.qa[0] * HALO_LOG2E : nal, kyy = DEF ? -(float)a.qa[1] * HALO_LOG2E : nal;
    const float kxy = DEF ? -(float)a.qa[3] * HALO_LOG2E : 0.f, kzz = DEF ? -(float)a.qa[2] * HALO_LOG2E : nal;
    __syncthreads();  // region staged
    // four particles per warp per round, one per quarter (warp-uniform loop: the
    // shuffles below run on all 32 lanes)
    for (int base = beg + 4 * warp; base < end; base += 4 * (HALO_THREADS / 32)) {
      const int k = base + quarter;
      const bool live = k < end;
      const int ke = live ? k : end - 1;
      const int4 i0 = sp_i0[ke];
      const float4 d0 = sp_d0[ke];
      const int ex = i0.x - t0[0], ey = i0.y - t0[1], ez = i0.z - z0;  // in [0, 16) and [0, LAYER)
      // 1D weights: lane sub < P holds the x, y and z weights of point sub (P <= 8,
      // the lanes of a quarter); a larger support has every lane form its own
      float wz[P], wx = 0.f, wy = 0.f;
      if constexpr (P <= 8) {
        const float fs = (float)(sub < P ? sub : 0) * hs;
        const float ox = d0.x + fs, oy = d0.y + fs, oz = d0.z + fs;
        wx = exp2f(nal * ox * ox);
        wy = exp2f(nal * oy * oy);
        const float wzl = exp2f(kzz * oz * oz);
#pragma unroll
        for (int j = 0; j < P; ++j) wz[j] = __shfl_sync(0xffffffffu, wzl, j, 8);
      } else {
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const float oz = d0.z + (float)j * hs;
          wz[j] = exp2f(kzz * oz * oz);
        }
      }
      float acc[C];
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = 0.f;
      const int pb = ez * ZS + ey * RX + ex;
      constexpr int CU = P >= 8 ? 2 : H::NCOL;  // P = 8: partial unroll (register pressure)
#pragma unroll CU
      for (int s = 0; s < H::NCOL; ++s) {
        // this lane's column (px, py) = (c mod P, c / P) of the support, c = sub + 8 s
        const int cc = sub + 8 * s, px = cc % P, py = cc < P * P ? cc / P : 0;
        float wxy;
        if (DEF || P > 8) {  // the column's own x-y weight
          const float cx = d0.x + (float)px * hs, cy = d0.y + (float)py * hs;
          wxy = exp2f(kxx * cx * cx + kxy * cx * cy + kyy * cy * cy);
        } else {
          wxy = __shfl_sync(0xffffffffu, wx, px, 8) * __shfl_sync(0xffffffffu, wy, py, 8);
        }
        if (cc < P * P) {
          const int col = pb + py * RX + px;
#pragma unroll
          for (int jz = 0; jz < P; ++jz) {
            float vv[C];
            tl.load(col + jz * ZS, vv);
            const float w = wxy * wz[jz];
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = fmaf(w, vv[c], acc[c]);
          }
        }
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
      // lane c of the quarter adds component c
      float mine = acc[0];
#pragma unroll
      for (int c = 1; c < C; ++c) mine = sub == c ? acc[c] : mine;
      if (live && sub < C) {
        float *o = vout + 8 * (size_t)k + SLOT0 + sub;
        *o += pref * mine;
      }
    }
    __syncthreads();  // the region is no longer read when the next item overwrites it
  });
}

template <int C, int SLOT0, int P, bool DEF = false, int COMP0 = 0>
void launch_interp_halo(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  static std::once_flag once;
  static OccCache occ;
  const size_t sm = TileL<float, C>::bytes((size_t)Halo<P>::NPT);
  if (sm > c->smem_optin) {
    // the staged region of all components does not fit: components 0-4 and 5-7 in two passes
    // (a region of 5 components is the largest that fits), else the general kernel
    if constexpr (C == 8 && COMP0 == 0) {
      if (TileL<float, 5>::bytes((size_t)Halo<P>::NPT) <= c->smem_optin) {
        launch_interp_halo<5, SLOT0, P, DEF, 0>(c, a, vout, s);
        launch_interp_halo<3, SLOT0 + 5, P, DEF, 5>(c, a, vout, s);
        c->nlaunch += 1;
        return;
      }
    }
    return interp_general_launch(c, a, vout, C == 8 ? M_FULL : (C == 5 ? M_SE : M_FSU), s);
  }
  auto kern = k_interp_halo<C, SLOT0, P, DEF, COMP0>;
  set_smem(kern, once);
  const unsigned grid = wave_grid(c, kern, sm, a.ntiles * SUB_SIDE, occ, HALO_THREADS);
  int *q = next_queue(c, s);
  kern<<<grid, HALO_THREADS, sm, s>>>(a, q, (const int4 *)c->d_sp_i0, (const float4 *)c->d_sp_d0, c->d_fine_start,
                                      (const float *)c->d_grid, (float *)vout);
}

template <int C, int SLOT0, bool DEF>
void interp_halo_pd(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  switch (a.P) {
    case 5: launch_interp_halo<C, SLOT0, 5, DEF>(c, a, vout, s); break;
    case 6: launch_interp_halo<C, SLOT0, 6, DEF>(c, a, vout, s); break;
    case 10: launch_interp_halo<C, SLOT0, 10, DEF>(c, a, vout, s); break;
    default: launch_interp_halo<C, SLOT0, 8, DEF>(c, a, vout, s);
  }
}

template <int C, int SLOT0>
void interp_halo_p(pse_ctx *c, const WaveArgs &a, void *vout, cudaStream_t s) {
  if (c->lattice) interp_halo_pd<C, SLOT0, true>(c, a, vout, s);
  else interp_halo_pd<C, SLOT0, false>(c, a, vout, s);
}

}  // namespace

void interp_halo_launch(pse_ctx *c, const WaveArgs &a, void *vout, int mode, cudaStream_t s) {
  if (mode == M_FULL) interp_halo_p<8, 0>(c, a, vout, s);
  else if (mode == M_SE) interp_halo_p<5, 3>(c, a, vout, s);
  else interp_halo_p<3, 0>(c, a, vout, s);
}

}  // namespace pse
