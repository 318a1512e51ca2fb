// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits.  Built from the
// error-free transformations of Dekker (Numer. Math. 18, 1971) and Knuth
// (TAOCP vol. 2): the exact sum of two floats (two_sum, fast_two_sum when
// |a| >= |b|) and the exact product through a fused multiply-add.  Used where
// FP64 accuracy is needed but FP64 throughput (1/64 of the FP32 rate on
// GB300) would bound the kernel.  Requires IEEE float semantics (no fast-math
// reassociation), which the build keeps.
#pragma once

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ df df_from(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}

__device__ __forceinline__ df df_from2(float2 v) { return {v.x, v.y}; }

__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  df s = df_two_sum(p, c.hi);
  return df_fast_two_sum(s.hi, s.lo + (e + c.lo));
}

__device__ __forceinline__ df df_abs(df a) { return a.hi < 0.f ? df_neg(a) : a; }

// larger of two non-negative values (ordered by hi, then lo); a NaN wins, so
// that it reaches the statistics built from these maxima
__device__ __forceinline__ df df_max_nonneg(df a, df b) {
  if (!(a.hi == a.hi)) return a;
  if (!(b.hi == b.hi)) return b;
  return (a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo)) ? a : b;
}

// Arithmetic shared by float and double-float code paths (the compute type
// of a kernel instantiated for FP32 or for FP64 accuracy).
__device__ __forceinline__ float ct_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ df ct_fma(df a, df b, df c) { return df_fma(a, b, c); }
__device__ __forceinline__ float ct_add(float a, float b) { return a + b; }
__device__ __forceinline__ float ct_mul(float a, float b) { return a * b; }
__device__ __forceinline__ df ct_mul(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ float ct_neg(float a) { return -a; }
__device__ __forceinline__ df ct_neg(df a) { return df_neg(a); }
__device__ __forceinline__ df ct_add(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ float ct_shfl_up(float v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ df ct_shfl_up(df v, int d) {
  return {__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d)};
}
__device__ __forceinline__ float ct_shfl_down(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ df ct_shfl_down(df v, int d) {
  return {__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d)};
}
template <typename CT> __device__ __forceinline__ CT ct_zero();
template <> __device__ __forceinline__ float ct_zero<float>() { return 0.f; }
template <> __device__ __forceinline__ df ct_zero<df>() { return {0.f, 0.f}; }
template <typename CT> __device__ __forceinline__ CT ct_from(float v);
template <> __device__ __forceinline__ float ct_from<float>(float v) { return v; }
template <> __device__ __forceinline__ df ct_from<df>(float v) { return {v, 0.f}; }
template <typename CT> __device__ __forceinline__ CT ct_from(double v);
template <> __device__ __forceinline__ float ct_from<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ df ct_from<df>(double v) { return df_from(v); }
template <typename CT> __device__ __forceinline__ CT ct_from(float2 v);
template <> __device__ __forceinline__ df ct_from<df>(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ void ct_store(float *p, float v) { *p = v; }
__device__ __forceinline__ void ct_store(double *p, df v) { *p = df_to(v); }
__device__ __forceinline__ void ct_store(float2 *p, df v) { *p = make_float2(v.hi, v.lo); }
