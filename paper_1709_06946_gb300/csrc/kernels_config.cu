// Configuration set-up: wrapping, binning by spreading tile, counting sort,
// per-particle spreading/real-space records, linked-cell list and neighbour list.
//
// Sorted order = by the spreading tile that holds the first grid index of a
// particle's Gaussian support; the spreading and interpolation kernels visit the
// 2x2x2 neighbouring bins of their tile, and the pair sum walks a neighbour list
// built from cells of side >= r_cut (Sec. 2.3.1, linked-cell lists).
#include <cmath>

#include "device_common.cuh"
#include "pse_internal.cuh"

namespace pse {
namespace {

constexpr int SCAN_NT = 256, SCAN_IPT = 8, SCAN_BLK = SCAN_NT * SCAN_IPT;

// Exclusive scan of in[0..n) into out (in-place allowed) per block of SCAN_BLK items.
__global__ void k_scan_block(const int *in, int *out, int64_t n, int *block_sums) {
  __shared__ int warp_tot[SCAN_NT / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_BLK + (int64_t)threadIdx.x * SCAN_IPT;
  int v[SCAN_IPT], tot = 0;
#pragma unroll
  for (int i = 0; i < SCAN_IPT; ++i) {
    int64_t idx = base + i;
    v[i] = idx < n ? in[idx] : 0;
    tot += v[i];
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int x = lane < SCAN_NT / 32 ? warp_tot[lane] : 0, xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += t;
    }
    if (lane < SCAN_NT / 32) warp_tot[lane] = xi - x;  // exclusive warp offsets
    if (lane == SCAN_NT / 32 - 1 && block_sums) block_sums[blockIdx.x] = xi;
  }
  __syncthreads();
  int run = warp_tot[w] + incl - tot;
#pragma unroll
  for (int i = 0; i < SCAN_IPT; ++i) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = run;
    run += v[i];
  }
}

__global__ void k_scan_add(int *out, int64_t n, const int *offs) {
  int64_t base = (int64_t)blockIdx.x * SCAN_BLK;
  int add = offs[blockIdx.x];
  for (int64_t i = threadIdx.x; i < SCAN_BLK; i += blockDim.x) {
    int64_t idx = base + i;
    if (idx < n) out[idx] += add;
  }
}

__device__ __forceinline__ double wrap_coord(double x, double L) {
  if (x >= 0.0 && x < L) return x;  // already inside: fmod would return x itself
  x = fmod(x, L);
  if (x < 0) x += L;
  if (x >= L) x = 0.0;
  return x;
}

// floor(x / y) and rint(x / y) of the rounded FP64 quotient, for 0 <= x / y < 2^20,
// mostly without the FP64 division (a long instruction sequence at sm_103a's
// FP64 rate): q = x * (1/y) lies within a few units in the last place of the
// rounded quotient, so its floor (rint) is the same unless q lies that close to
// an integer (a half-integer); there the division decides.
__device__ __forceinline__ double quot_floor(double x, double y, double iy) {
  const double q = x * iy, f = floor(q), e = 1e-12 * (q + 1.0);
  return (q - f < e || q - f > 1.0 - e) ? floor(x / y) : f;
}
__device__ __forceinline__ double quot_rint(double x, double y, double iy) {
  const double q = x * iy, e = 1e-12 * (q + 1.0);
  return fabs(q - floor(q) - 0.5) < e ? rint(x / y) : rint(q);
}

// First grid index of the support of a particle at wrapped coordinate x.
__device__ __forceinline__ int support_start(double x, double h, double ih, int P) {
  return (P & 1) ? (int)quot_rint(x, h, ih) - (P - 1) / 2 : (int)quot_floor(x, h, ih) - P / 2 + 1;
}

// Wraps particle u (user order) of its suspension into [0, L) and counts it in
// the spreading tile that holds the first grid index of its support, refined by
// the 4 x 4 x 4 sub-block of the tile (so that the sorted order is spatially
// coherent inside a tile: neighbours' records then lie close together).
__global__ void k_bin(const SysDev *__restrict__ sys, const int64_t *__restrict__ p0, int nsys, int64_t Ntot,
                      int P, const double *pos, double *posw, int *tile_key, int *tile_cnt, int *bad) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= Ntot) return;
  const SysDev &b = sys[find_sys(p0, nsys, u)];
  int iw[3];
  double xin[3];
  for (int d = 0; d < 3; ++d) {
    xin[d] = pos[3 * u + d];
    if (!isfinite(xin[d])) {
      atomicOr(bad, 1);
      xin[d] = 0.0;
    }
  }
  if (b.def) {  // lattice coordinates z = A^{-1} x (Sec. 2.3.3); everything below works on z
    const double z0 = b.Ai[0] * xin[0] + b.Ai[1] * xin[1] + b.Ai[2] * xin[2];
    const double z1 = b.Ai[3] * xin[0] + b.Ai[4] * xin[1] + b.Ai[5] * xin[2];
    const double z2 = b.Ai[6] * xin[0] + b.Ai[7] * xin[1] + b.Ai[8] * xin[2];
    xin[0] = z0;
    xin[1] = z1;
    xin[2] = z2;
  }
  for (int d = 0; d < 3; ++d) {
    const double x = wrap_coord(xin[d], b.L);
    posw[3 * u + d] = x;
    iw[d] = wrapi(support_start(x, b.h, b.inv_h, P), b.Ng);
  }
  int tk = b.tile0 + ((iw[2] / b.T[2]) * b.nt[1] + iw[1] / b.T[1]) * b.nt[0] + iw[0] / b.T[0];
  int sub = (((iw[2] % b.T[2]) * SUB_SIDE / b.T[2]) * SUB_SIDE + (iw[1] % b.T[1]) * SUB_SIDE / b.T[1]) * SUB_SIDE +
            (iw[0] % b.T[0]) * SUB_SIDE / b.T[0];
  tk = tk * SUB_BLOCKS + sub;
  tile_key[u] = tk;
  atomicAdd(&tile_cnt[tk], 1);
}

// tile_start[t] = fine_start[t * SUB_BLOCKS] for t = 0 .. ntiles
__global__ void k_tile_starts(int64_t ntiles, const int *fine_start, int *tile_start) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= ntiles) tile_start[t] = fine_start[t * SUB_BLOCKS];
}

__global__ void k_scatter(int64_t N, const int *key, const int *start, int *cur, int *perm, int *inv) {
  int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= N) return;
  int k = key[u];
  int i = start[k] + atomicAdd(&cur[k], 1);
  perm[i] = (int)u;
  inv[u] = i;
}

template <typename T>
__global__ void k_derive(const SysDev *__restrict__ sys, const int64_t *__restrict__ p0, int nsys, int64_t Ntot,
                         int P, const int *perm, const double *posw, int4 *sp_i0, typename V4<T>::t *sp_d0,
                         void *rs, int *cell_key, int *cell_cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Ntot) return;
  const SysDev &b = sys[find_sys(p0, nsys, i)];
  int u = perm[i];
  double x[3];
  int iw[3], c[3];
  T d0[3];
  for (int d = 0; d < 3; ++d) {
    x[d] = posw[3 * (int64_t)u + d];
    int i0 = support_start(x[d], b.h, b.inv_h, P);
    iw[d] = wrapi(i0, b.Ng);
    d0[d] = (T)(i0 * b.h - x[d]);
    c[d] = min((int)quot_floor(x[d], b.cs, b.inv_cs), b.nc - 1);
  }
  sp_i0[i] = make_int4(iw[0], iw[1], iw[2], 0);
  typename V4<T>::t dd;
  dd.x = d0[0];
  dd.y = d0[1];
  dd.z = d0[2];
  dd.w = 0;
  sp_d0[i] = dd;
  if (sizeof(T) == 4) {
    int packed = c[0] | (c[1] << 10) | (c[2] << 20);
    ((float4 *)rs)[i] = make_float4((float)(x[0] - c[0] * b.cs), (float)(x[1] - c[1] * b.cs),
                                    (float)(x[2] - c[2] * b.cs), __int_as_float(packed));
  } else {
    ((double4_32a *)rs)[i] = make_double4_32a(x[0], x[1], x[2], 0.0);
  }
  int ck = b.cell0 + (c[2] * b.nc + c[1]) * b.nc + c[0];
  cell_key[i] = ck;
  atomicAdd(&cell_cnt[ck], 1);
}

// Cell list: the particles of every cell, and a copy of their records (cell
// offsets or positions) in the same order, so that the neighbour search reads
// contiguous records.
template <typename T>
__global__ void k_cell_scatter(int64_t N, int *cell_key, const int *start, int *cur, int *list,
                               const typename V4<T>::t *rs, typename V4<T>::t *rs_cell) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int ck = cell_key[i];
  const int k = start[ck] + atomicAdd(&cur[ck], 1);
  list[k] = (int)i;
  rs_cell[k] = rs[i];
  cell_key[i] = k;  // from here on: the particle's own position in the cell list
}

__device__ __forceinline__ void unpack_cell(float w, int c[3]) {
  int p = __float_as_int(w);
  c[0] = p & 1023;
  c[1] = (p >> 10) & 1023;
  c[2] = (p >> 20) & 1023;
}

// Separation x_i - x_j (minimum image) from cell-relative FP32 offsets.
__device__ __forceinline__ float3 sep(const float4 &pi, const int ci[3], const float4 &pj, const SysDev &a) {
  int cj[3];
  unpack_cell(pj.w, cj);
  int dc[3];
  for (int d = 0; d < 3; ++d) {
    int t = ci[d] - cj[d];
    if (t > a.nc / 2) t -= a.nc;
    if (t < -(a.nc / 2)) t += a.nc;
    dc[d] = t;
  }
  float3 r = make_float3(dc[0] * a.csf + (pi.x - pj.x), dc[1] * a.csf + (pi.y - pj.y),
                         dc[2] * a.csf + (pi.z - pj.z));
  if (a.nc < 5) {
    r.x -= a.Lf * rintf(r.x / a.Lf);
    r.y -= a.Lf * rintf(r.y / a.Lf);
    r.z -= a.Lf * rintf(r.z / a.Lf);
  }
  return r;
}

// Neighbour list in one pass, one thread per particle i: for each neighbour j
// (r < r_cut, minimum image within its own suspension) the separation x_i - x_j
// and j go into i's own row of slots, and the row's length into cnt[i]; per
// suspension the total and the largest count are accumulated for the host's
// capacity check.  The stencil is 5 x 5 x 5 cells (every cell once when there
// are fewer than 5 per side); each of its 25 x runs of cells is one range of
// the cell-ordered records, or two where it wraps, so a thread streams through
// contiguous records, NB of them loaded before the first is tested.  The
// particle itself is recognised by its own position in the cell list (no read of
// the list per hit).
// DEF: deformed lattice (Sec. 2.3.3): records and cells hold lattice coordinates z,
// and each candidate's separation is mapped to x_i - x_j = A (z_i - z_j) before the
// test, so the stored separations are Cartesian as for the cube.
template <typename T4>
__device__ __forceinline__ void to_cartesian(const SysDev &a, T4 &r) {
  if (sizeof(r.x) == 4) {
    const float x = a.Af[0] * r.x + a.Af[1] * r.y + a.Af[2] * r.z;
    const float y = a.Af[3] * r.x + a.Af[4] * r.y + a.Af[5] * r.z;
    const float z = a.Af[6] * r.x + a.Af[7] * r.y + a.Af[8] * r.z;
    r.x = x;
    r.y = y;
    r.z = z;
  } else {
    const double x = a.A[0] * r.x + a.A[1] * r.y + a.A[2] * r.z;
    const double y = a.A[3] * r.x + a.A[4] * r.y + a.A[5] * r.z;
    const double z = a.A[6] * r.x + a.A[7] * r.y + a.A[8] * r.z;
    r.x = x;
    r.y = y;
    r.z = z;
  }
}

template <typename T, int NB = 4, bool DEF = false>
__global__ void __launch_bounds__(128) k_nbr(const SysDev *__restrict__ sys, const int64_t *__restrict__ p0,
                                             int nsys, int64_t Ntot, float rc2f, double rc2, const void *rs,
                                             const void *rs_cell, const int *__restrict__ cell_start,
                                             const int *__restrict__ cell_pos, int *cnt, typename V4<T>::t *geo,
                                             unsigned long long *tot, int *ovf) {
  using T4 = typename V4<T>::t;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Ntot) return;
  const int kself = cell_pos[i];  // i's own record in the cell-ordered copy (skipped)
  const int si = find_sys(p0, nsys, i);
  const SysDev &a = sys[si];
  const int nc = a.nc, slots = a.slots;
  int ci[3];
  float4 pf;
  double4_32a pd;
  if (sizeof(T) == 4) {
    pf = ((const float4 *)rs)[i];
    unpack_cell(pf.w, ci);
  } else {
    pd = ((const double4_32a *)rs)[i];
    ci[0] = min((int)(pd.x / a.cs), nc - 1);
    ci[1] = min((int)(pd.y / a.cs), nc - 1);
    ci[2] = min((int)(pd.z / a.cs), nc - 1);
  }
  const bool wide = nc >= 5;
  const int span = wide ? 5 : nc;
  const int x0 = wide ? ci[0] - 2 : 0, x1 = wide ? ci[0] + 2 : nc - 1;
  T4 *mgeo = geo + a.nbr0 + (i - a.p0) * slots;
  int n = 0;
  for (int dz = 0; dz < span; ++dz)
    for (int dy = 0; dy < span; ++dy) {
      int cz = dz, cy = dy;
      if (wide) {
        cz += ci[2] - 2;
        cy += ci[1] - 2;
        cz += cz < 0 ? nc : (cz >= nc ? -nc : 0);
        cy += cy < 0 ? nc : (cy >= nc ? -nc : 0);
      }
      const int rowc = a.cell0 + (cz * nc + cy) * nc;
      // FP32 with five or more cells per side: the row's y and z cell offsets
      // (minimum image) are shared by all its candidates; only x varies
      float offy = 0.f, offz = 0.f;
      if (sizeof(T) == 4 && wide) {
        int ty = ci[1] - cy, tz = ci[2] - cz;
        if (ty > nc / 2) ty -= nc;
        if (ty < -(nc / 2)) ty += nc;
        if (tz > nc / 2) tz -= nc;
        if (tz < -(nc / 2)) tz += nc;
        offy = ty * a.csf;
        offz = tz * a.csf;
      }
      int s1, e1, s2 = 0, e2 = 0;
      if (x0 < 0) {  // cells [x0 + nc, nc) and [0, x1]
        s1 = cell_start[rowc + x0 + nc];
        e1 = cell_start[rowc + nc];
        s2 = cell_start[rowc];
        e2 = cell_start[rowc + x1 + 1];
      } else if (x1 >= nc) {  // cells [x0, nc) and [0, x1 - nc]
        s1 = cell_start[rowc + x0];
        e1 = cell_start[rowc + nc];
        s2 = cell_start[rowc];
        e2 = cell_start[rowc + x1 - nc + 1];
      } else {
        s1 = cell_start[rowc + x0];
        e1 = cell_start[rowc + x1 + 1];
      }
      for (int part = 0; part < 2; ++part) {
        const int kb = part ? s2 : s1, ke = part ? e2 : e1;
        // NB candidate records loaded before any is tested: NB reads in flight per thread
        for (int k = kb; k < ke; k += NB) {
          T4 q[NB];
#pragma unroll
          for (int u = 0; u < NB; ++u)
            if (k + u < ke) q[u] = ((const T4 *)rs_cell)[k + u];
#pragma unroll
          for (int u = 0; u < NB; ++u) {
            if (k + u >= ke) break;
            T4 rec;
            bool hit;
            if (sizeof(T) == 4 && wide) {  // as sep(), with the row's y and z offsets
              const float4 pj = *(const float4 *)&q[u];
              int tx = ci[0] - (__float_as_int(pj.w) & 1023);
              if (tx > nc / 2) tx -= nc;
              if (tx < -(nc / 2)) tx += nc;
              rec.x = tx * a.csf + (pf.x - pj.x);
              rec.y = offy + (pf.y - pj.y);
              rec.z = offz + (pf.z - pj.z);
              if (DEF) to_cartesian(a, rec);
              hit = rec.x * rec.x + rec.y * rec.y + rec.z * rec.z < rc2f;
            } else if (sizeof(T) == 4) {
              const float3 d = sep(pf, ci, *(const float4 *)&q[u], a);
              rec.x = d.x;
              rec.y = d.y;
              rec.z = d.z;
              if (DEF) to_cartesian(a, rec);
              hit = rec.x * rec.x + rec.y * rec.y + rec.z * rec.z < rc2f;
            } else {
              const double4_32a qj = *(const double4_32a *)&q[u];
              double rx = pd.x - qj.x, ry = pd.y - qj.y, rz = pd.z - qj.z;
              rx -= a.L * rint(rx / a.L);
              ry -= a.L * rint(ry / a.L);
              rz -= a.L * rint(rz / a.L);
              if (DEF) {
                const double x = a.A[0] * rx + a.A[1] * ry + a.A[2] * rz;
                const double y = a.A[3] * rx + a.A[4] * ry + a.A[5] * rz;
                const double z = a.A[6] * rx + a.A[7] * ry + a.A[8] * rz;
                rx = x;
                ry = y;
                rz = z;
              }
              rec.x = (T)rx;
              rec.y = (T)ry;
              rec.z = (T)rz;
              hit = rx * rx + ry * ry + rz * rz < rc2;
            }
            if (hit && k + u != kself) {
              if (n < slots) {  // separation x_i - x_j and the neighbour's cell-list position in one record
                rec.w = index_as_real<T>(k + u);
                mgeo[n] = rec;
              }
              ++n;
            }
          }
        }
      }
    }
  cnt[i] = n;
  if (n > slots) atomicOr(ovf, 1);
  // per-suspension totals: one atomic per warp when the warp's particles share a suspension
  const unsigned act = __activemask();
  const int leader = __ffs(act) - 1;
  if (__all_sync(act, si == __shfl_sync(act, si, leader))) {
    const unsigned sum = __reduce_add_sync(act, (unsigned)n), big = __reduce_max_sync(act, (unsigned)n);
    if ((int)(threadIdx.x & 31) == leader) {
      atomicAdd(&tot[2 * si], (unsigned long long)sum);
      atomicMax(&tot[2 * si + 1], (unsigned long long)big);
    }
  } else {
    atomicAdd(&tot[2 * si], (unsigned long long)n);
    atomicMax(&tot[2 * si + 1], (unsigned long long)n);
  }
}

void *alloc_dev(pse_ctx *c, size_t bytes) {
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  c->allocs.push_back(p);
  c->dev_bytes += (int64_t)bytes;
  return p;
}

}  // namespace

// Exclusive scan of n+1 ints (in[n] must be 0) so that out[n] is the total.
pse_status exclusive_scan(pse_ctx *c, int *buf, int64_t n1, cudaStream_t s) {
  // level sizes
  int64_t sizes[8];
  int levels = 0;
  int64_t len = n1;
  while (true) {
    sizes[levels++] = len;
    if (len <= SCAN_BLK) break;
    len = ceil_div(len, SCAN_BLK);
    if (levels >= 7) break;
  }
  int *bufs[8];
  bufs[0] = buf;
  int64_t off = 0;
  for (int l = 1; l < levels; ++l) {
    bufs[l] = c->d_scan_tmp + off;
    off += sizes[l];
  }
  c->nlaunch += 2 * levels - 1;
  for (int l = 0; l < levels; ++l) {
    int64_t nb = ceil_div(sizes[l], SCAN_BLK);
    k_scan_block<<<(unsigned)nb, SCAN_NT, 0, s>>>(bufs[l], bufs[l], sizes[l], l + 1 < levels ? bufs[l + 1] : nullptr);
  }
  for (int l = levels - 2; l >= 0; --l) {
    int64_t nb = ceil_div(sizes[l], SCAN_BLK);
    k_scan_add<<<(unsigned)nb, SCAN_NT, 0, s>>>(bufs[l], sizes[l], bufs[l + 1]);
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

int64_t scan_tmp_ints(int64_t n1) {
  int64_t tot = 0, len = n1;
  while (len > SCAN_BLK) {
    len = ceil_div(len, SCAN_BLK);
    tot += len;
  }
  return tot + 16;
}

// Slot layout of the neighbour list: per suspension `slots` entries per particle.
int64_t layout_neighbours(pse_ctx *c) {
  int64_t off = 0;
  for (int q = 0; q < c->nsys; ++q) {
    c->hs[q].nbr0 = off;
    off += (int64_t)c->hs[q].slots * c->hs[q].N;
  }
  return off;
}

// Builds the sorted configuration for positions d_pos (device, user order, FP64).
pse_status setup_config(pse_ctx *c, const double *d_pos, cudaStream_t s) {
  StageTimer timer(c, PSE_STAGE_SETUP, s);
  c->nlaunch += 6;  // bin, scatter, derive, cell scatter, neighbour count and fill (+ scans)
  const Params &p = c->p;
  const int64_t N = p.N;
  const int ns = c->nsys;
  unsigned nb = (unsigned)ceil_div(N, 256);
  const int64_t nfine = c->ntiles * SUB_BLOCKS;
  PSE_CUDA_TRY(c, cudaMemsetAsync(c->d_fine_start, 0, sizeof(int) * (nfine + 1), s));
  PSE_CUDA_TRY(c, cudaMemsetAsync(c->d_fine_cur, 0, sizeof(int) * (nfine + 1), s));
  PSE_CUDA_TRY(c, cudaMemsetAsync(c->d_cell_start, 0, sizeof(int) * (c->ncells + 1), s));
  PSE_CUDA_TRY(c, cudaMemsetAsync(c->d_cell_cur, 0, sizeof(int) * (c->ncells + 1), s));
  if (!c->capturing) PSE_CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));  // a graph clears it once
  k_bin<<<nb, 256, 0, s>>>(c->d_sys, c->d_p0, ns, N, p.P, d_pos, c->d_posw, c->d_tile_key, c->d_fine_start,
                           c->d_flag);
  PSE_TRY(exclusive_scan(c, c->d_fine_start, nfine + 1, s));
  k_scatter<<<nb, 256, 0, s>>>(N, c->d_tile_key, c->d_fine_start, c->d_fine_cur, c->d_perm, c->d_inv);
  k_tile_starts<<<(unsigned)ceil_div(c->ntiles + 1, 256), 256, 0, s>>>(c->ntiles, c->d_fine_start, c->d_tile_start);
  if (c->prec == PSE_MIXED)
    k_derive<float><<<nb, 256, 0, s>>>(c->d_sys, c->d_p0, ns, N, p.P, c->d_perm, c->d_posw, (int4 *)c->d_sp_i0,
                                       (float4 *)c->d_sp_d0, c->d_rs, c->d_cell_key, c->d_cell_start);
  else
    k_derive<double><<<nb, 256, 0, s>>>(c->d_sys, c->d_p0, ns, N, p.P, c->d_perm, c->d_posw, (int4 *)c->d_sp_i0,
                                        (double4_32a *)c->d_sp_d0, c->d_rs, c->d_cell_key, c->d_cell_start);
  PSE_TRY(exclusive_scan(c, c->d_cell_start, c->ncells + 1, s));
  if (c->prec == PSE_MIXED)
    k_cell_scatter<float><<<nb, 256, 0, s>>>(N, c->d_cell_key, c->d_cell_start, c->d_cell_cur, c->d_cell_list,
                                             (const float4 *)c->d_rs, (float4 *)c->d_rs_cell);
  else
    k_cell_scatter<double><<<nb, 256, 0, s>>>(N, c->d_cell_key, c->d_cell_start, c->d_cell_cur, c->d_cell_list,
                                              (const double4_32a *)c->d_rs, (double4_32a *)c->d_rs_cell);
  const double rc2 = p.rcut * p.rcut;
  const unsigned nb128 = (unsigned)ceil_div(N, 128);
  for (int attempt = 0; attempt < 2; ++attempt) {
    PSE_CUDA_TRY(c, cudaMemsetAsync(c->d_nbr_tot, 0, 2 * sizeof(unsigned long long) * ns, s));
    const bool def = c->lattice != 0;
    if (c->prec == PSE_MIXED)
      (def ? k_nbr<float, 4, true> : k_nbr<float, 4, false>)<<<nb128, 128, 0, s>>>(
          c->d_sys, c->d_p0, ns, N, (float)rc2, rc2, c->d_rs, c->d_rs_cell, c->d_cell_start, c->d_cell_key,
          c->d_nbr_start, (float4 *)c->d_nbr_geo, c->d_nbr_tot, c->d_flag + 1);
    else
      (def ? k_nbr<double, 4, true> : k_nbr<double, 4, false>)<<<nb128, 128, 0, s>>>(
          c->d_sys, c->d_p0, ns, N, (float)rc2, rc2, c->d_rs, c->d_rs_cell, c->d_cell_start, c->d_cell_key,
          c->d_nbr_start, (double4_32a *)c->d_nbr_geo, c->d_nbr_tot, c->d_flag + 1);
    if (c->capturing) return PSE_OK;  // the graph's caller checks the flags and the totals afterwards
    PSE_CUDA_TRY(c, cudaMemcpyAsync(c->h_pinned_int + 1, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    PSE_CUDA_TRY(c, cudaMemcpyAsync(c->h_nbr_tot, c->d_nbr_tot, 2 * sizeof(unsigned long long) * ns,
                                    cudaMemcpyDeviceToHost, s));
    PSE_CUDA_TRY(c, cudaGetLastError());
    PSE_CUDA_TRY(c, cudaStreamSynchronize(s));
    if (c->h_pinned_int[1]) {
      c->err = "non-finite particle position";
      return PSE_ERR_NONFINITE;
    }
    bool grow = false;
    c->npairs = 0;
    c->npairs_sys.assign(ns, 0);
    for (int q = 0; q < ns; ++q) {
      c->npairs_sys[q] = (int64_t)c->h_nbr_tot[2 * q];
      c->npairs += c->npairs_sys[q];
      int64_t mx = (int64_t)c->h_nbr_tot[2 * q + 1];
      if (mx > c->hs[q].slots) {
        c->hs[q].slots = (int)((mx + 15) / 8 * 8);  // a particle has more neighbours than slots
        grow = true;
      }
    }
    if (!grow) break;
    // enlarge the list and rebuild once
    int64_t cap = layout_neighbours(c);
    if ((double)cap > 2.0e9) {
      c->err = "neighbour list exceeds 2^31 entries";
      return PSE_ERR_INVALID_ARG;
    }
    void *gq = alloc_dev(c, 4 * c->ts * (size_t)cap);
    if (!gq) {
      c->err = "cannot allocate neighbour list";
      return PSE_ERR_OOM;
    }
    c->d_nbr_geo = gq;  // the old list stays in c->allocs and is freed at destroy
    c->nbr_cap = cap;
    ++c->layout_version;
    PSE_CUDA_TRY(c, cudaMemcpyAsync(c->d_sys, c->hs.data(), sizeof(SysDev) * ns, cudaMemcpyHostToDevice, s));
  }
  PSE_CUDA_TRY(c, cudaGetLastError());
  return PSE_OK;
}

}  // namespace pse
