// Device helpers shared by the PSE kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pse {

template <typename T> struct V4;
template <> struct V4<float> { using t = float4; };
template <> struct V4<double> { using t = double4_32a; };

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Persistent work loop: the CTA takes work items from the counter *queue (which
// starts at zero) until `total` have been handed out; every thread of the CTA
// calls f(item) for the same items, so f may use __syncthreads.
template <class F>
__device__ __forceinline__ void for_each_item(int *queue, int total, F &&f) {
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= total) return;
    f(item);
  }
}

// A particle index carried in the fourth component of a separation record (the
// bits of the index in FP32; the value, exactly, in FP64).
template <typename T> __device__ __forceinline__ T index_as_real(int j);
template <> __device__ __forceinline__ float index_as_real<float>(int j) { return __int_as_float(j); }
template <> __device__ __forceinline__ double index_as_real<double>(int j) { return (double)j; }
template <typename T> __device__ __forceinline__ int real_as_index(T x);
template <> __device__ __forceinline__ int real_as_index<float>(float x) { return __float_as_int(x); }
template <> __device__ __forceinline__ int real_as_index<double>(double x) { return (int)x; }

// wrap an integer index into [0, n)
__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Box-Muller pair from Philox words 0 and 1; counter (index_lo, index_hi, step, stream).
template <typename T>
__device__ __forceinline__ void normal_pair(uint64_t seed, uint64_t step, uint32_t stream, uint64_t index,
                                            T &z0, T &z1) {
  uint4 c = make_uint4((uint32_t)index, (uint32_t)(index >> 32), (uint32_t)step, stream);
  uint2 k = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  uint4 w = philox4x32_10(c, k);
  T u1 = ((T)w.x + (T)0.5) * (T)2.3283064365386963e-10;
  T u2 = ((T)w.y + (T)0.5) * (T)2.3283064365386963e-10;
  T rad = sqrt((T)-2 * log(u1));
  T s, co;
  if (sizeof(T) == 4) {
    float sf, cf;
    sincospif(2.0f * (float)u2, &sf, &cf);
    s = (T)sf;
    co = (T)cf;
  } else {
    double sd, cd;
    sincospi(2.0 * (double)u2, &sd, &cd);
    s = (T)sd;
    co = (T)cd;
  }
  z0 = rad * co;
  z1 = rad * s;
}

// Orthonormal symmetric-traceless basis (Y1..Y5) helpers.
// Y components of the symmetric tensor p q^T + q p^T.
template <typename T>
__device__ __forceinline__ void symY(const T p[3], const T q[3], T e[5]) {
  const T r2 = (T)1.4142135623730951, i2 = (T)0.70710678118654752, i6 = (T)0.40824829046386302;
  T xx = 2 * p[0] * q[0], yy = 2 * p[1] * q[1], zz = 2 * p[2] * q[2];
  e[0] = (xx - yy) * i2;  // products with 1/sqrt(2), 1/sqrt(6): no division in the pair loop
  e[1] = (xx + yy - 2 * zz) * i6;
  e[2] = r2 * (p[0] * q[1] + p[1] * q[0]);
  e[3] = r2 * (p[0] * q[2] + p[2] * q[0]);
  e[4] = r2 * (p[1] * q[2] + p[2] * q[1]);
}
// v = S p for S = sum_k s_k Y_k.
template <typename T>
__device__ __forceinline__ void Smul(const T s[5], const T p[3], T v[3]) {
  const T i2 = (T)0.70710678118654752, i6 = (T)0.40824829046386302;
  T sxx = s[0] * i2 + s[1] * i6, syy = -s[0] * i2 + s[1] * i6, szz = -2 * s[1] * i6;
  T sxy = s[2] * i2, sxz = s[3] * i2, syz = s[4] * i2;
  v[0] = sxx * p[0] + sxy * p[1] + sxz * p[2];
  v[1] = sxy * p[0] + syy * p[1] + syz * p[2];
  v[2] = sxz * p[0] + syz * p[1] + szz * p[2];
}

}  // namespace pse
