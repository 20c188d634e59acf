// Device-side helpers shared by the libtem kernels: complex arithmetic,
// front metadata and launch helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tem {

template <typename R>
struct __align__(2 * sizeof(R)) cx {
  R x, y;
};
using c64 = cx<float>;
using c128 = cx<double>;

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) {
  cx<R> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk<R>(s * a.x, s * a.y); }
// acc += a * b
template <typename R>
__device__ __forceinline__ void cfma(cx<R> &acc, cx<R> a, cx<R> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b
template <typename R>
__device__ __forceinline__ void cfms(cx<R> &acc, cx<R> a, cx<R> b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// 1 / (a + i b) by Smith's scaling (1962): avoids overflow of a^2 + b^2.
template <typename R>
__device__ __forceinline__ cx<R> crecip(cx<R> z) {
  R a = z.x, b = z.y;
  if (fabs(a) >= fabs(b)) {
    R r = b / a;
    R d = a + b * r;
    return mk<R>(R(1) / d, -r / d);
  } else {
    R r = a / b;
    R d = a * r + b;
    return mk<R>(r / d, R(-1) / d);
  }
}
template <typename R>
__device__ __forceinline__ R cabs1(cx<R> z) { return fabs(z.x) + fabs(z.y); }

template <typename R>
__device__ __forceinline__ void atomic_add_cx(cx<R> *p, cx<R> v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}
// complex FP32: one 8-byte vector atomic (sm_90 and later)
template <>
__device__ __forceinline__ void atomic_add_cx<float>(cx<float> *p, cx<float> v) {
  atomicAdd(reinterpret_cast<float2 *>(p), make_float2(v.x, v.y));
}

// Front metadata as seen by the kernels.
struct FrontDev {
  int64_t lofs;    // factor block offset (n x k, column-major, column stride ld)
  int64_t uofs;    // update block offset in the arena (b x b, ld b), -1 if b == 0
  int64_t rows_off;
  int64_t rel_off;
  int64_t inv_off;  // first NB x NB diagonal-block inverse of this front (in blocks)
  int32_t n, k, c0, parent;
  int32_t ld;       // column stride: n rounded up to even (16-byte aligned columns)
  int32_t pad_;
};

// Device status words of one context.
struct DevStatus {
  int32_t pivot_fail;       // 1 if a pivot underflowed
  int32_t pivot_front;      // front of the first failure
  int32_t tc_timeout;       // 1 if a tensor-core completion wait gave up
  int32_t pad_;
  unsigned long long min_pivot_bits;  // bits of the smallest |d_kk| (positive double)
};

inline int div_up(int64_t a, int64_t b) { return int((a + b - 1) / b); }

// Pole of grid slot i: the identity, or the list of poles still refining.
__device__ __forceinline__ int pole_of(int i, const int *pmap) { return pmap ? pmap[i] : i; }

}  // namespace tem
