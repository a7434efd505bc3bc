// Scalar arithmetic for the two-stage Householder kernels.
//
// Four element types: double and float (real), z64 and z32 (complex, interleaved
// re/im).  `S` below always names the storage/FP64 type (double or z64) and
// `B` the type of the bulk streaming products (S itself, or its FP32
// counterpart in the FP32-bulk variant).  Every complex multiply-add is four
// real FMAs; no operation here adds FP64 instructions beyond those.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tho {

struct __align__(16) z64 {
  double x, y;
};
struct __align__(8) z32 {
  float x, y;
};

template <class T> struct Tr;
template <> struct Tr<double> { using R = double; using F64 = double; static constexpr bool C = false; };
template <> struct Tr<float>  { using R = float;  using F64 = double; static constexpr bool C = false; };
template <> struct Tr<z64>    { using R = double; using F64 = z64;    static constexpr bool C = true; };
template <> struct Tr<z32>    { using R = float;  using F64 = z64;    static constexpr bool C = true; };

template <class T> __host__ __device__ __forceinline__ T zero();
template <> __host__ __device__ __forceinline__ double zero<double>() { return 0.0; }
template <> __host__ __device__ __forceinline__ float zero<float>() { return 0.0f; }
template <> __host__ __device__ __forceinline__ z64 zero<z64>() { return z64{0.0, 0.0}; }
template <> __host__ __device__ __forceinline__ z32 zero<z32>() { return z32{0.0f, 0.0f}; }

template <class T> __device__ __forceinline__ T from_real(double r);
template <> __device__ __forceinline__ double from_real<double>(double r) { return r; }
template <> __device__ __forceinline__ float from_real<float>(double r) { return (float)r; }
template <> __device__ __forceinline__ z64 from_real<z64>(double r) { return z64{r, 0.0}; }
template <> __device__ __forceinline__ z32 from_real<z32>(double r) { return z32{(float)r, 0.0f}; }

// ---- conversions between storage and bulk types --------------------------
template <class To, class From> __device__ __forceinline__ To cvt(From a);
template <> __device__ __forceinline__ double cvt<double, double>(double a) { return a; }
template <> __device__ __forceinline__ float cvt<float, double>(double a) { return __double2float_rn(a); }
template <> __device__ __forceinline__ double cvt<double, float>(float a) { return (double)a; }
template <> __device__ __forceinline__ float cvt<float, float>(float a) { return a; }
template <> __device__ __forceinline__ z64 cvt<z64, z64>(z64 a) { return a; }
template <> __device__ __forceinline__ z32 cvt<z32, z64>(z64 a) { return z32{__double2float_rn(a.x), __double2float_rn(a.y)}; }
template <> __device__ __forceinline__ z64 cvt<z64, z32>(z32 a) { return z64{(double)a.x, (double)a.y}; }
template <> __device__ __forceinline__ z32 cvt<z32, z32>(z32 a) { return a; }

// ---- arithmetic ---------------------------------------------------------------
__device__ __forceinline__ double madd(double c, double a, double b) { return fma(a, b, c); }
__device__ __forceinline__ float madd(float c, float a, float b) { return fmaf(a, b, c); }
__device__ __forceinline__ z64 madd(z64 c, z64 a, z64 b) {  // c + a b
  c.x = fma(a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ z32 madd(z32 c, z32 a, z32 b) {
  c.x = fmaf(a.x, b.x, c.x); c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y); c.y = fmaf(a.y, b.x, c.y);
  return c;
}

__device__ __forceinline__ double cmadd(double c, double a, double b) { return fma(a, b, c); }
__device__ __forceinline__ float cmadd(float c, float a, float b) { return fmaf(a, b, c); }
__device__ __forceinline__ z64 cmadd(z64 c, z64 a, z64 b) {  // c + conj(a) b
  c.x = fma(a.x, b.x, c.x); c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y); c.y = fma(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ z32 cmadd(z32 c, z32 a, z32 b) {
  c.x = fmaf(a.x, b.x, c.x); c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y); c.y = fmaf(-a.y, b.x, c.y);
  return c;
}

__device__ __forceinline__ double msub(double c, double a, double b) { return fma(-a, b, c); }
__device__ __forceinline__ float msub(float c, float a, float b) { return fmaf(-a, b, c); }
__device__ __forceinline__ z64 msub(z64 c, z64 a, z64 b) {  // c - a b
  c.x = fma(-a.x, b.x, c.x); c.x = fma(a.y, b.y, c.x);
  c.y = fma(-a.x, b.y, c.y); c.y = fma(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ z32 msub(z32 c, z32 a, z32 b) {
  c.x = fmaf(-a.x, b.x, c.x); c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(-a.x, b.y, c.y); c.y = fmaf(-a.y, b.x, c.y);
  return c;
}

__device__ __forceinline__ double cmsub(double c, double a, double b) { return fma(-a, b, c); }
__device__ __forceinline__ z64 cmsub(z64 c, z64 a, z64 b) {  // c - conj(a) b
  c.x = fma(-a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
  c.y = fma(-a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
  return c;
}

__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ z64 add(z64 a, z64 b) { return z64{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ z32 add(z32 a, z32 b) { return z32{a.x + b.x, a.y + b.y}; }

__device__ __forceinline__ double sub(double a, double b) { return a - b; }
__device__ __forceinline__ z64 sub(z64 a, z64 b) { return z64{a.x - b.x, a.y - b.y}; }

__device__ __forceinline__ double neg(double a) { return -a; }
__device__ __forceinline__ z64 neg(z64 a) { return z64{-a.x, -a.y}; }

__device__ __forceinline__ double conj_(double a) { return a; }
__device__ __forceinline__ float conj_(float a) { return a; }
__device__ __forceinline__ z64 conj_(z64 a) { return z64{a.x, -a.y}; }
__device__ __forceinline__ z32 conj_(z32 a) { return z32{a.x, -a.y}; }

__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ z64 mul(z64 a, z64 b) { return z64{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }

__device__ __forceinline__ double scale(double a, double r) { return a * r; }
__device__ __forceinline__ float scale(float a, double r) { return a * (float)r; }
__device__ __forceinline__ z64 scale(z64 a, double r) { return z64{a.x * r, a.y * r}; }
__device__ __forceinline__ z32 scale(z32 a, double r) { return z32{a.x * (float)r, a.y * (float)r}; }

// |a|^2 evaluated in FP64 whatever the element precision (reflector norms stay FP64).
__device__ __forceinline__ double abs2d(double a) { return a * a; }
__device__ __forceinline__ double abs2d(float a) { double d = a; return d * d; }
__device__ __forceinline__ double abs2d(z64 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double abs2d(z32 a) { double x = a.x, y = a.y; return fma(x, x, y * y); }

__device__ __forceinline__ double absd(double a) { return fabs(a); }
__device__ __forceinline__ double absd(z64 a) { return hypot(a.x, a.y); }

__device__ __forceinline__ double real_(double a) { return a; }
__device__ __forceinline__ double real_(z64 a) { return a.x; }

// Unit-modulus phase of a (phase(0) = 1), in FP64.
__device__ __forceinline__ double phase(double a) { return a < 0.0 ? -1.0 : 1.0; }
__device__ __forceinline__ z64 phase(z64 a) {
  double r = hypot(a.x, a.y);
  return r == 0.0 ? z64{1.0, 0.0} : z64{a.x / r, a.y / r};
}

__device__ __forceinline__ bool finite_(double a) { return isfinite(a); }
__device__ __forceinline__ bool finite_(z64 a) { return isfinite(a.x) && isfinite(a.y); }

// ---- warp reductions (butterfly; every lane gets the sum) -------------------
__device__ __forceinline__ double shfl_x(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ float shfl_x(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ z64 shfl_x(z64 v, int m) {
  return z64{__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}
__device__ __forceinline__ z32 shfl_x(z32 v, int m) {
  return z32{__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}
template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v = add(v, shfl_x(v, m));
  return v;
}

}  // namespace tho
