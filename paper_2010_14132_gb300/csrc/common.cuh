// Device helpers shared by the solver kernels: complex arithmetic, error-free
// float transformations, and integer-only conversions between double and float.
//
// On GB300 every FP64 instruction and every f32<->f64 conversion issues at about
// 1/65 of the FP32 rate (measured: 5.0e11 DFMA/s vs 3.3e13 FFMA/s), so the
// mixed-precision path never executes FP64 arithmetic per grid point.  Doubles
// are read and written as bit patterns and converted with integer operations;
// extra precision comes from pairs of floats (hi + lo, "double-float").
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pgb {

template <typename T> struct CT;
template <> struct CT<float> { using t = float2; };
template <> struct CT<double> { using t = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return {a.x, -a.y}; }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return {a.x * s, a.y * s}; }
// multiply by SIGN*i (SIGN = -1 for forward transforms, +1 for inverse)
template <int SIGN, typename C> __device__ __forceinline__ C cmul_si(C a) {
  if (SIGN < 0) return {a.y, -a.x};
  return {-a.y, a.x};
}
template <int SIGN, typename C> __device__ __forceinline__ C tw_apply(C a, C w) {
  // tables hold exp(-2 pi i m/n); the inverse uses the conjugate
  if (SIGN < 0) return cmul(a, w);
  return cmul(a, cconj(w));
}

template <typename T> __device__ __forceinline__ typename CT<T>::t make_c(T x, T y) {
  typename CT<T>::t r;
  r.x = x;
  r.y = y;
  return r;
}

// ---------------------------------------------------------------------------
// Error-free transformations (Knuth TwoSum, FMA-based TwoProduct; Dekker 1971,
// Ogita-Rump-Oishi 2005).  With hi = fl(a op b), the pair (hi, lo) is exact.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
// Fast two-sum, requires |a| >= |b| (or a == 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// ---------------------------------------------------------------------------
// Integer-only conversions (no FP64 pipe).
// ---------------------------------------------------------------------------

// double -> nearest float (ties to even); |x| < 2^-126 flushes to signed zero,
// |x| >= 2^128 gives infinity.  NaN inputs are not expected.
__device__ __forceinline__ float d2f_int(double x) {
  const unsigned long long b = __double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1fffffffu;
  uint32_t bits = ((uint32_t)(e - 896) << 23) + m;
  bits += (rem > 0x10000000u) | ((rem == 0x10000000u) & (m & 1u));
  bits = (e <= 896) ? 0u : bits;
  bits = (e >= 1151) ? 0x7f800000u : bits;
  return __uint_as_float(sign | bits);
}

// double -> (hi, lo) floats with hi = nearest float and hi + lo = x to about
// 2^-46 relative (lo keeps the top 22 bits of the rounding remainder).
__device__ __forceinline__ void d2ff_int(double x, float& h, float& l) {
  const unsigned long long b = __double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1fffffffu;
  const uint32_t up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (m & 1u));
  uint32_t bits = ((uint32_t)(e - 896) << 23) + m + up;
  const bool small = (e <= 896);
  bits = small ? 0u : bits;
  bits = (e >= 1151) ? 0x7f800000u : bits;
  h = __uint_as_float(sign | bits);
  // remainder x - h = (rem - up*2^29) * 2^(e-1075); keep its top bits: shift by 7
  // so it fits a float built by the 1.5*2^23 magic-number trick exactly.
  const int r = (int)rem - (int)(up << 29);            // |r| <= 2^28
  const int rs = (r + 64) >> 7;                        // |rs| <= 2^21 + 1, rounded
  const float rf = __int_as_float(0x4B400000 + rs) - 12582912.0f;   // == (float)rs exactly
  const int se = e - 1075 + 7 + 127;                   // biased exponent of 2^(e-1068)
  const float scale = (se >= 1 && se <= 254) ? __int_as_float(se << 23) : 0.0f;
  l = __uint_as_float(__float_as_uint(rf * scale) ^ sign);
  l = small ? 0.0f : l;
}

// float -> double, exact (denormal floats flush to zero).
__device__ __forceinline__ double f2d_int(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t m = u & 0x7fffffu;
  uint32_t hi = sign | ((e + 896u) << 20) | (m >> 3);
  uint32_t lo = m << 29;
  hi = (e == 0u) ? sign : hi;
  lo = (e == 0u) ? 0u : lo;
  hi = (e == 255u) ? (sign | 0x7ff00000u | (m ? 0x80000u : 0u)) : hi;
  return __longlong_as_double(((long long)hi << 32) | lo);
}

// Normalised double-float pair (s, t), |t| <= ulp(s)/2, -> the double nearest
// s + t (truncating bits of t below 2^-53 |s|).  Integer-only.
__device__ __forceinline__ double ff2d_int(float s, float t) {
  const uint32_t sb = __float_as_uint(s), tb = __float_as_uint(t);
  const int es = (int)((sb >> 23) & 0xffu);
  const int et = (int)((tb >> 23) & 0xffu);
  if (es == 0) return f2d_int(t);
  long long ms = (long long)((sb & 0x7fffffu) | 0x800000u) << 29;   // s in units of 2^(es-179)
  long long mt = (long long)((tb & 0x7fffffu) | (et ? 0x800000u : 0u));
  const int sh = (et ? et : 1) - es + 29;                            // t in the same units
  long long tv = (sh >= 0) ? (mt << (sh > 40 ? 40 : sh)) : ((sh > -40) ? (mt >> (-sh)) : 0);
  if ((sb ^ tb) & 0x80000000u) tv = -tv;
  long long m = ms + tv;
  int e = es + 896;
  if (m >= (1LL << 53)) { m >>= 1; e += 1; }
  if (m < (1LL << 52)) { m <<= 1; e -= 1; }
  const unsigned long long bits = ((unsigned long long)(sb & 0x80000000u) << 32) |
                                  ((unsigned long long)e << 52) |
                                  ((unsigned long long)m & ((1ULL << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// Normalised double-float pair (s, t), |t| <= ulp(s)/2 -> a double within
// 2^-47 |s + t| of s + t, in fewer integer steps than ff2d_int: the double bits
// of s plus t counted in units of 2^6 double ulps of s (half that unit below a
// power of two whose magnitude t lowers).  |s| < 2^-81 returns s alone.
__device__ __forceinline__ double ff2d_fast(float s, float t) {
  const uint32_t sb = __float_as_uint(s);
  const uint32_t es = (sb >> 23) & 0xffu;
  const uint32_t hi = (sb & 0x80000000u) | ((es + 896u) << 20) | ((sb >> 3) & 0xfffffu);
  const uint32_t lo = sb << 29;
  unsigned long long bits = ((unsigned long long)hi << 32) | lo;
  bits = (es == 0u) ? ((unsigned long long)(sb & 0x80000000u) << 32) : bits;   // zero (no denormal floats)
  // t / (2^6 ulp_d(s)) = t * 2^(173 - e_s), |.| <= 2^22: exact scaling, rounded to an integer
  const int sc = 300 - (int)es;
  const float scale = __uint_as_float((uint32_t)(sc > 0 && sc < 255 ? sc : 0) << 23);
  const int ti = __float_as_int(__fmul_rn(t, scale) + 12582912.0f) - 0x4B400000;
  const int delta = (sb & 0x80000000u) ? -ti : ti;   // change of the magnitude, in units
  const int shift = ((sb & 0x7fffffu) == 0u && delta < 0) ? 7 : 6;
  bits += (unsigned long long)((long long)delta << shift);
  return __longlong_as_double((long long)bits);
}

// ---------------------------------------------------------------------------
// Loads/stores of the solver's element types with conversion to compute type.
// ---------------------------------------------------------------------------
template <typename TI, typename T> struct Cvt;
template <> struct Cvt<double, double> { static __device__ __forceinline__ double f(double x) { return x; } };
template <> struct Cvt<float, float> { static __device__ __forceinline__ float f(float x) { return x; } };
template <> struct Cvt<double, float> { static __device__ __forceinline__ float f(double x) { return d2f_int(x); } };
template <> struct Cvt<float, double> { static __device__ __forceinline__ double f(float x) { return f2d_int(x); } };

// Device-side error word bits (workspace stats area).
enum : unsigned { ERR_WAIT_TIMEOUT = 1u, ERR_BAD_SIZE = 2u };

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of the solve chain are launched
// with pdl_launch: the next kernel's CTAs may start (and build their shared
// tables from the plan's constant tables) while the previous kernel drains
// (outside stream capture; captured launches keep ordinary stream order).
// Every such kernel calls pdl_wait() before it touches memory that an earlier
// kernel of the stream writes or reads: the wait returns once those kernels
// have completed and their writes are visible.  pdl_trigger() lets the next
// kernel launch early; its CTAs take SM resources only as this kernel's leave.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... P, typename... A>
inline cudaError_t pdl_launch(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
#ifdef PGB_NO_PDL
  at[0].val.programmaticStreamSerializationAllowed = 0;
#else
  // not inside a stream capture: the batched graphs run many small domains on concurrent branches,
  // where plain edges measured faster (FP32 batch of 64 domains: 4.30 against 4.46 ms)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusActive;
  at[0].val.programmaticStreamSerializationAllowed = (cs == cudaStreamCaptureStatusNone) ? 1 : 0;
#endif
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

}  // namespace pgb
