// dense.cuh -- element types and helpers of the dense (K) kernels.
#pragma once
#include "df64.cuh"

namespace tw {

constexpr int NB_ = 64;   // block size of K's tiles, the packed factor and the solves

// Scalar policy for the dense kernels: dd (FP64-class) or float (FP32 path).
template <class T> struct DS;
template <> struct DS<dd> {
  typedef dacc acc;
  static __device__ __forceinline__ acc zero() { return dacc_zero(); }
  static __device__ __forceinline__ void mac(acc &a, dd x, dd y) { dacc_mac(a, x, y); }
  static __device__ __forceinline__ dd get(acc a) { return dacc_get(a); }
  static __device__ __forceinline__ void fold(dd &tot, acc &a) { dacc_fold(tot, a); }
  static __device__ __forceinline__ dd add(dd a, dd b) { return dd_add(a, b); }
  static __device__ __forceinline__ dd sub(dd a, dd b) { return dd_sub(a, b); }
  static __device__ __forceinline__ dd mul(dd a, dd b) { return dd_mul(a, b); }
  static __device__ __forceinline__ dd neg(dd a) { return dd_neg(a); }
  static __device__ __forceinline__ dd zerov() { return dd_zero(); }
  static __device__ __forceinline__ dd one() { dd r; r.hi = 1.f; r.lo = 0.f; return r; }
  static __device__ __forceinline__ dd sqrtv(dd a) { return dd_sqrt(a); }
  static __device__ __forceinline__ dd div(dd a, dd b) { return dd_div(a, b); }
  static __device__ __forceinline__ float lead(dd a) { return a.hi; }
  static __device__ __forceinline__ dd from_d(double x) { return dd_from_double(x); }
  static __device__ __forceinline__ double to_d(dd a) { return dd_to_double(a); }
  static __device__ __forceinline__ dd shfl_xor(dd v, int m) {
    dd r; r.hi = __shfl_xor_sync(0xffffffffu, v.hi, m); r.lo = __shfl_xor_sync(0xffffffffu, v.lo, m); return r;
  }
};
template <> struct DS<float> {
  typedef float acc;
  static __device__ __forceinline__ acc zero() { return 0.f; }
  static __device__ __forceinline__ void mac(acc &a, float x, float y) { a = fmaf(x, y, a); }
  static __device__ __forceinline__ float get(acc a) { return a; }
  static __device__ __forceinline__ void fold(float &tot, acc &a) { tot += a; a = 0.f; }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
  static __device__ __forceinline__ float neg(float a) { return -a; }
  static __device__ __forceinline__ float zerov() { return 0.f; }
  static __device__ __forceinline__ float one() { return 1.f; }
  static __device__ __forceinline__ float sqrtv(float a) { return a > 0.f ? __fsqrt_rn(a) : 0.f; }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
  static __device__ __forceinline__ float lead(float a) { return a; }
  static __device__ __forceinline__ float from_d(double x) { return __double2float_rn(x); }
  static __device__ __forceinline__ double to_d(float a) { return (double)a; }
  static __device__ __forceinline__ float shfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
};

template <> struct DS<double> {
  typedef double acc;
  static __device__ __forceinline__ acc zero() { return 0.0; }
  static __device__ __forceinline__ void mac(acc &a, double x, double y) { a = fma(x, y, a); }
  static __device__ __forceinline__ double get(acc a) { return a; }
  static __device__ __forceinline__ void fold(double &tot, acc &a) { tot += a; a = 0.0; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
  static __device__ __forceinline__ double neg(double a) { return -a; }
  static __device__ __forceinline__ double zerov() { return 0.0; }
  static __device__ __forceinline__ double one() { return 1.0; }
  static __device__ __forceinline__ double sqrtv(double a) { return a > 0.0 ? sqrt(a) : 0.0; }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double lead(double a) { return a; }
  static __device__ __forceinline__ double from_d(double x) { return x; }
  static __device__ __forceinline__ double to_d(double a) { return a; }
  static __device__ __forceinline__ double shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
};

// index of block (I, J), J <= I, in the packed lower-triangular block array
__host__ __device__ __forceinline__ size_t packed_index(int I, int J) {
  return (size_t)I * (I + 1) / 2 + J;
}

}  // namespace tw
