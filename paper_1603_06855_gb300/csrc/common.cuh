// Shared device helpers: complex arithmetic templated on the real type, launch
// checks, device status codes.
#pragma once
#include <atomic>
#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/phononic.h"

template <typename R> struct cplx_t;
template <> struct cplx_t<double> { typedef double2 type; };
template <> struct cplx_t<float>  { typedef float2 type; };

template <typename R> __host__ __device__ __forceinline__ typename cplx_t<R>::type mk(R x, R y) {
  typename cplx_t<R>::type c; c.x = x; c.y = y; return c;
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2  cadd(float2 a, float2 b)   { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2  csub(float2 a, float2 b)   { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ float2  cmul(float2 a, float2 b)   { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__host__ __device__ __forceinline__ float2  cmulc(float2 a, float2 b)   { return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2  cscale(float2 a, float s)   { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2  cconj(float2 a)  { return make_float2(a.x, -a.y); }
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
}
template <typename R> __device__ __forceinline__ R cabs2(typename cplx_t<R>::type a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
template <typename R> __device__ __forceinline__ typename cplx_t<R>::type from_d2(double2 a);
template <> __device__ __forceinline__ double2 from_d2<double>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d2<float>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// exp(i * pi * t / n) for an integer t reduced exactly modulo 2n: the phases of the
// plane waves at voxel centroids are exact rationals, so no argument error enters.
__device__ __forceinline__ double2 phase_pi_over(long long t, int n) {
  long long tm = t % (2LL * n);
  if (tm < 0) tm += 2LL * n;
  double s, c;
  sincospi((double)tm / (double)n, &s, &c);
  return make_double2(c, s);
}

// Device status word: first error wins.
__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

#define PC_CUDA_TRY(expr)                          \
  do {                                             \
    cudaError_t e__ = (expr);                      \
    if (e__ != cudaSuccess) return PC_ECUDA;       \
  } while (0)

// Every kernel launch is followed by this check, which also counts the launch.
extern std::atomic<long long> g_pc_launches;  // kernel launches (two host threads may launch)
#define PC_LAUNCH_CHECK()        \
  do {                           \
    ++g_pc_launches;             \
    PC_CUDA_TRY(cudaGetLastError()); \
  } while (0)

static inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }
