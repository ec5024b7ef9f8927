// pse_mobility_real_noalloc: the real-space part of the mobility product for
// callers that cannot allocate device memory.
//
// Who needs it: host codes that must never make the device wait in the middle
// of their loop (cudaMalloc and cudaFree synchronise the whole device), and
// applications whose device memory is owned by their own pool allocator and
// cannot hand raw allocations to a third-party library.  The regular entry
// points allocate their grids, lists and Krylov space in pse_create; this one
// allocates nothing on the device.
//
// Its scratch (cell counts, cell list, per-particle cell keys and the FP32
// real-space table) lives in one file-scope __device__ array of fixed size
// (NA_BYTES below, about 1.3 MB), which every GPU that loads the library holds
// until the process exits.  The first call on a device looks up the array's
// device address with cudaGetSymbolAddress (with that device current) and caches
// it; that first call should come before any stream capture.  All calls share
// the array and it keeps the last call's contents: the cell counters are cleared
// at the start of every call, the table is re-uploaded whenever its parameters
// change.  Calls that overlap on the GPU (other streams, other threads) race on
// the array and must be serialised by the caller.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "pse_internal.cuh"

namespace {

constexpr int NA_MAX_N = 65536;        // particles
constexpr int NA_MAX_NC = 32;          // cells per side (cells may be larger than r_cut)
constexpr int NA_MAX_CELLS = NA_MAX_NC * NA_MAX_NC * NA_MAX_NC;
constexpr int NA_MAX_TABLE = 16384;    // table rows (8 floats each)

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_KEY = 0;
constexpr size_t OFF_CNT = align256(OFF_KEY + sizeof(int) * NA_MAX_N);
constexpr size_t OFF_CUR = align256(OFF_CNT + sizeof(int) * (NA_MAX_CELLS + 1));
constexpr size_t OFF_LIST = align256(OFF_CUR + sizeof(int) * (NA_MAX_CELLS + 1));
constexpr size_t OFF_TABLE = align256(OFF_LIST + sizeof(int) * NA_MAX_N);
constexpr size_t NA_BYTES = align256(OFF_TABLE + sizeof(float) * 8 * NA_MAX_TABLE);

static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

std::mutex g_na_mu;
void *g_na_addr[128] = {nullptr};
struct TableKey {
  double a, eta, xi, rcut;
  bool operator==(const TableKey &o) const { return a == o.a && eta == o.eta && xi == o.xi && rcut == o.rcut; }
};
TableKey g_na_uploaded[128];
bool g_na_has_table[128] = {false};
thread_local std::string g_na_err;
// host copy of the last generated table (static: the entry point allocates nothing)
float g_host_table[8 * NA_MAX_TABLE];
double g_host_self[2] = {0, 0};
TableKey g_host_key{0, 0, 0, 0};
double g_dev_self[128][2];

struct NAArgs {
  int N, nc, len;
  double L, cs, rc2;
  float inv_dr, self_uf, self_es;
};

__global__ void k_na_bin(NAArgs a, const double *pos, int *key, int *cnt) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= a.N) return;
  int c[3];
  for (int d = 0; d < 3; ++d) {
    double x = fmod(pos[3 * (size_t)u + d], a.L);
    if (x < 0) x += a.L;
    c[d] = min(max((int)(x / a.cs), 0), a.nc - 1);
  }
  int k = (c[2] * a.nc + c[1]) * a.nc + c[0];
  key[u] = k;
  atomicAdd(&cnt[k], 1);
}

// Exclusive scan of cnt[0..n) in one block of 1024 threads; cnt[n] receives the total.
__global__ void k_na_scan(int *cnt, int n) {
  __shared__ int part[1024];
  int t = threadIdx.x, per = (n + 1023) / 1024, lo = t * per, hi = min(lo + per, n);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += cnt[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;
  for (int i = lo; i < hi; ++i) {
    int v = cnt[i];
    cnt[i] = run;
    run += v;
  }
  if (t == 1023) cnt[n] = part[1023];
}

__global__ void k_na_fill(int N, const int *key, const int *start, int *cur, int *list) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= N) return;
  int k = key[u];
  list[start[k] + atomicAdd(&cur[k], 1)] = u;
}

__global__ void __launch_bounds__(128) k_na_real(NAArgs a, const double *__restrict__ pos, const float *__restrict__ F,
                                                 const float *__restrict__ S, const int *__restrict__ start,
                                                 const int *__restrict__ list, const float *__restrict__ tab,
                                                 float *__restrict__ U, float *__restrict__ E) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  double xi[3];
  int ci[3];
  for (int d = 0; d < 3; ++d) {
    double x = fmod(pos[3 * (size_t)i + d], a.L);
    if (x < 0) x += a.L;
    xi[d] = x;
    ci[d] = min(max((int)(x / a.cs), 0), a.nc - 1);
  }
  float u[3] = {0, 0, 0}, e[5] = {0, 0, 0, 0, 0};
  if (F)
    for (int m = 0; m < 3; ++m) u[m] = a.self_uf * F[3 * (size_t)i + m];
  if (S)
    for (int m = 0; m < 5; ++m) e[m] = a.self_es * S[5 * (size_t)i + m];
  int lo = a.nc >= 3 ? -1 : 0, hi = a.nc >= 2 ? 1 : 0;
  const float4 *t4 = (const float4 *)tab;
  for (int dz = lo; dz <= hi; ++dz)
    for (int dy = lo; dy <= hi; ++dy)
      for (int dx = lo; dx <= hi; ++dx) {
        int c = (pse::wrapi(ci[2] + dz, a.nc) * a.nc + pse::wrapi(ci[1] + dy, a.nc)) * a.nc +
                pse::wrapi(ci[0] + dx, a.nc);
        for (int q = start[c]; q < start[c + 1]; ++q) {
          int j = list[q];
          if (j == i) continue;
          double dd[3];
          for (int d = 0; d < 3; ++d) {
            dd[d] = xi[d] - pos[3 * (size_t)j + d];
            dd[d] -= a.L * rint(dd[d] / a.L);
          }
          double r2d = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
          if (r2d >= a.rc2) continue;
          float r = sqrtf((float)r2d), ir = 1.0f / r;
          float rh[3] = {(float)dd[0] * ir, (float)dd[1] * ir, (float)dd[2] * ir};
          float x = r * a.inv_dr;
          int k = min((int)x, a.len - 2);
          float t = x - (float)k;
          float4 a0 = t4[2 * k], a1 = t4[2 * k + 1], b0 = t4[2 * k + 2], b1 = t4[2 * k + 3];
          float f[7] = {a0.x + t * (b0.x - a0.x), a0.y + t * (b0.y - a0.y), a0.z + t * (b0.z - a0.z),
                        a0.w + t * (b0.w - a0.w), a1.x + t * (b1.x - a1.x), a1.y + t * (b1.y - a1.y),
                        a1.z + t * (b1.z - a1.z)};
          float s[5] = {0, 0, 0, 0, 0}, Fj[3] = {0, 0, 0};
          if (S)
            for (int m = 0; m < 5; ++m) s[m] = S[5 * (size_t)j + m];
          if (F)
            for (int m = 0; m < 3; ++m) Fj[m] = F[3 * (size_t)j + m];
          float v[3];
          pse::Smul(s, rh, v);
          float qv = rh[0] * v[0] + rh[1] * v[1] + rh[2] * v[2];
          float rf = rh[0] * Fj[0] + rh[1] * Fj[1] + rh[2] * Fj[2];
          for (int m = 0; m < 3; ++m)
            u[m] += f[0] * Fj[m] + (f[1] - f[0]) * rf * rh[m] + f[2] * v[m] + f[3] * qv * rh[m];
          float sy[5], yr[5], sf[5];
          pse::symY(v, rh, sy);
          pse::symY(rh, rh, yr);
          pse::symY(Fj, rh, sf);
          for (int m = 0; m < 5; ++m)
            e[m] += f[4] * s[m] + f[5] * sy[m] + 0.5f * f[6] * qv * yr[m] - 0.5f * f[2] * sf[m] -
                    0.5f * f[3] * rf * yr[m];
        }
      }
  if (U)
    for (int m = 0; m < 3; ++m) U[3 * (size_t)i + m] = u[m];
  if (E)
    for (int m = 0; m < 5; ++m) E[5 * (size_t)i + m] = e[m];
}

// True for NULL, for managed memory, and for device memory of device `dev` (the
// current device, whose copy of the scratch array the kernels use).  Device
// memory of another GPU is refused: without peer access the kernels would fault.
bool on_device(const void *p, int dev) {
  if (!p) return true;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" pse_status pse_mobility_real_noalloc(int64_t N, double L, double a, double eta, double xi, double tol,
                                                const double *pos, const float *F, const float *S, float *U,
                                                float *E, pse_stream stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (N < 1 || N > NA_MAX_N) {
    g_na_err = "pse_mobility_real_noalloc: N must be in [1, " + std::to_string(NA_MAX_N) + "]";
    return PSE_ERR_INVALID_ARG;
  }
  if (!(L > 0) || !(a > 0) || !(eta > 0) || !(xi > 0) || !(tol > 0 && tol <= 0.1) || !pos) {
    g_na_err = "pse_mobility_real_noalloc: invalid parameter or NULL positions";
    return PSE_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    cudaGetLastError();
    g_na_err = "pse_mobility_real_noalloc: no current CUDA device";
    return PSE_ERR_CUDA;
  }
  if (!on_device(pos, dev) || !on_device(F, dev) || !on_device(S, dev) || !on_device(U, dev) || !on_device(E, dev)) {
    g_na_err = "pse_mobility_real_noalloc: all arrays must be device memory of the current device "
               "(nothing is staged)";
    return PSE_ERR_INVALID_ARG;
  }
  pse::Params p{};
  p.N = N;
  p.L = L;
  p.a = a;
  p.eta = eta;
  p.xi = xi;
  p.tol = tol;
  p.rcut = a + std::sqrt(std::log(10.0 / tol)) / xi;  // the default (strict) cutoff rule of pse_create
  if (p.rcut > 0.5 * L) {
    g_na_err = "pse_mobility_real_noalloc: r_cut exceeds L/2";
    return PSE_ERR_INVALID_ARG;
  }
  const int ppa = 1024;  // table points per 2a, as in the mixed form of pse_create
  int len = (int)std::ceil(p.rcut / (2.0 * a / ppa)) + 4;
  if (len > NA_MAX_TABLE) {
    g_na_err = "pse_mobility_real_noalloc: r_cut/a too large for the fixed table (max " +
               std::to_string(NA_MAX_TABLE) + " rows)";
    return PSE_ERR_INVALID_ARG;
  }
  int nc = std::max(1, std::min(NA_MAX_NC, (int)std::floor(L / p.rcut)));
  unsigned char *base = nullptr;
  double self_uf = 0, self_es = 0;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&g_na_addr[dev], g_na_scratch);
      if (e != cudaSuccess) {
        g_na_addr[dev] = nullptr;
        g_na_err = std::string("pse_mobility_real_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return PSE_ERR_CUDA;
      }
    }
    base = (unsigned char *)g_na_addr[dev];
    TableKey key{a, eta, xi, p.rcut};
    if (!g_na_has_table[dev] || !(g_na_uploaded[dev] == key)) {
      // the upload waits for its copy, which a stream being captured cannot do
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        g_na_err = "pse_mobility_real_noalloc: cannot query the stream's capture status";
        return PSE_ERR_CUDA;
      }
      if (cs != cudaStreamCaptureStatusNone) {
        g_na_err = "pse_mobility_real_noalloc: a new table (a, eta, xi or tol changed) must be uploaded "
                   "outside stream capture; make one call with these parameters before capturing";
        return PSE_ERR_INVALID_ARG;
      }
      if (!(g_host_key == key)) {
        pse::fill_real_table_f32(p, ppa, len, g_host_table, &g_host_self[0], &g_host_self[1]);
        g_host_key = key;
      }
      cudaError_t e = cudaMemcpyAsync(base + OFF_TABLE, g_host_table, sizeof(float) * 8 * (size_t)len,
                                      cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        g_na_has_table[dev] = false;
        g_na_err = std::string("pse_mobility_real_noalloc: table upload: ") + cudaGetErrorString(e);
        return PSE_ERR_CUDA;
      }
      g_na_uploaded[dev] = key;
      g_na_has_table[dev] = true;
    }
    self_uf = g_dev_self[dev][0] = (g_host_key == key) ? g_host_self[0] : g_dev_self[dev][0];
    self_es = g_dev_self[dev][1] = (g_host_key == key) ? g_host_self[1] : g_dev_self[dev][1];
  }
  NAArgs g;
  g.N = (int)N;
  g.nc = nc;
  g.len = len;
  g.L = L;
  g.cs = L / nc;
  g.rc2 = p.rcut * p.rcut;
  g.inv_dr = (float)(ppa / (2.0 * a));
  g.self_uf = (float)self_uf;
  g.self_es = (float)self_es;
  int ncell = nc * nc * nc;
  int *key = (int *)(base + OFF_KEY), *cnt = (int *)(base + OFF_CNT), *cur = (int *)(base + OFF_CUR);
  int *list = (int *)(base + OFF_LIST);
  const float *tab = (const float *)(base + OFF_TABLE);
  cudaError_t me = cudaMemsetAsync(cnt, 0, sizeof(int) * (ncell + 1), s);
  if (me == cudaSuccess) me = cudaMemsetAsync(cur, 0, sizeof(int) * (ncell + 1), s);
  if (me != cudaSuccess) {
    cudaGetLastError();
    g_na_err = std::string("pse_mobility_real_noalloc: clearing the cell counters: ") + cudaGetErrorString(me);
    return PSE_ERR_CUDA;
  }
  unsigned nb = (unsigned)((N + 255) / 256);
  k_na_bin<<<nb, 256, 0, s>>>(g, pos, key, cnt);
  k_na_scan<<<1, 1024, 0, s>>>(cnt, ncell);
  k_na_fill<<<nb, 256, 0, s>>>((int)N, key, cnt, cur, list);
  k_na_real<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(g, pos, F, S, cnt, list, tab, U, E);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_na_err = std::string("pse_mobility_real_noalloc: ") + cudaGetErrorString(e);
    return PSE_ERR_CUDA;
  }
  return PSE_OK;
}

extern "C" const char *pse_noalloc_last_error(void) { return g_na_err.c_str(); }
