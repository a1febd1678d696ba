// Shared device helpers: 2x2 complex algebra, baseline map, phase setup.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rts {

constexpr double kCLight = 299792458.0;
constexpr double kTwo64 = 18446744073709551616.0;      // 2^64
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kTwoM32F = 2.3283064365386963e-10f;     // 2^-32

// ---- baselines: bl(i, j) = i*N - i(i+1)/2 + (j - i - 1), i < j -----------------
__host__ __device__ inline int64_t bl_index(int n_ant, int i, int j) {
  return (int64_t)i * n_ant - (int64_t)i * (i + 1) / 2 + (j - i - 1);
}

// ---- complex scalars --------------------------------------------------------------
template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };

template <typename C> __host__ __device__ inline C cmk(double re, double im) {
  C r; r.x = re; r.y = im; return r;
}
template <typename C> __device__ inline C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ inline C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ inline C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ inline C cconj(C a) { a.y = -a.y; return a; }
// a * conj(b)
template <typename C> __device__ inline C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
// conj(a) * b
template <typename C> __device__ inline C cconjmul(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}

// packed FP32x2 fused multiply-add (one instruction for two lanes): a * b + c
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long ra, rb, rc, rd;
  ra = (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
  rb = (unsigned long long)__float_as_uint(b.x) | ((unsigned long long)__float_as_uint(b.y) << 32);
  rc = (unsigned long long)__float_as_uint(c.x) | ((unsigned long long)__float_as_uint(c.y) << 32);
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  return make_float2(__uint_as_float((unsigned)rd), __uint_as_float((unsigned)(rd >> 32)));
}

// packed FP32x2 multiply: a * b
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  ra = (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
  rb = (unsigned long long)__float_as_uint(b.x) | ((unsigned long long)__float_as_uint(b.y) << 32);
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  return make_float2(__uint_as_float((unsigned)rd), __uint_as_float((unsigned)(rd >> 32)));
}

// ---- 2x2 complex matrices [0 1; 2 3] -------------------------------------------
template <typename C> struct M22 { C e[4]; };

template <typename C> __device__ inline M22<C> mmul(const M22<C>& a, const M22<C>& b) {
  M22<C> r;
  r.e[0] = cadd(cmul(a.e[0], b.e[0]), cmul(a.e[1], b.e[2]));
  r.e[1] = cadd(cmul(a.e[0], b.e[1]), cmul(a.e[1], b.e[3]));
  r.e[2] = cadd(cmul(a.e[2], b.e[0]), cmul(a.e[3], b.e[2]));
  r.e[3] = cadd(cmul(a.e[2], b.e[1]), cmul(a.e[3], b.e[3]));
  return r;
}
// a * b^H
template <typename C> __device__ inline M22<C> mmul_h(const M22<C>& a, const M22<C>& b) {
  M22<C> r;
  r.e[0] = cadd(cmulc(a.e[0], b.e[0]), cmulc(a.e[1], b.e[1]));
  r.e[1] = cadd(cmulc(a.e[0], b.e[2]), cmulc(a.e[1], b.e[3]));
  r.e[2] = cadd(cmulc(a.e[2], b.e[0]), cmulc(a.e[3], b.e[1]));
  r.e[3] = cadd(cmulc(a.e[2], b.e[2]), cmulc(a.e[3], b.e[3]));
  return r;
}
template <typename C> __device__ inline M22<C> mherm(const M22<C>& a) {
  M22<C> r;
  r.e[0] = cconj(a.e[0]); r.e[1] = cconj(a.e[2]);
  r.e[2] = cconj(a.e[1]); r.e[3] = cconj(a.e[3]);
  return r;
}

// ---- phase setup ------------------------------------------------------------------
// Per (time, baseline, source) the delay tau = u l + v m + w (n - 1) metres is
// formed in FP64 and turned into two unsigned Q0.64 fixed-point phases:
//   A = frac(tau nu_0 / c),  B = frac(tau dnu / c).
// Channel c then has phase A + c B (mod 2^64) exactly in integer arithmetic
// (integer wrap = reduction modulo one turn); this needs uniform channels.
struct SrcDir {
  double l, m, nm1;   // nm1 = n - 1 = -(l^2 + m^2) / (1 + n)
  double S;
};

__host__ inline SrcDir make_dir(double l, double m, double S) {
  double r2 = l * l + m * m;
  double n = sqrt(1.0 - r2);
  SrcDir d; d.l = l; d.m = m; d.nm1 = -r2 / (1.0 + n); d.S = S;
  return d;
}

__device__ inline unsigned long long frac_q64(double x) {
  double f = x - floor(x);
  if (!(f < 1.0)) f = 0.0;           // x just below an integer
  return __double2ull_rz(f * kTwo64);
}

__device__ inline double delay_m(const double* __restrict__ uvw, int n_ant, int t, int i, int j,
                                 const SrcDir& d) {
  const double* a = uvw + ((size_t)t * n_ant + i) * 3;
  const double* b = uvw + ((size_t)t * n_ant + j) * 3;
  double u = a[0] - b[0], v = a[1] - b[1], w = a[2] - b[2];
  return u * d.l + v * d.m + w * d.nm1;
}

// turns in [-1/2, 1/2) from a Q0.64 phase, rounded to Q0.32 first
__device__ inline float q64_to_turns(unsigned long long ph) {
  int hi = (int)((ph + 0x80000000ull) >> 32);
  return (float)hi * kTwoM32F;
}

// exp(+2 pi i turns) in FP32 (hardware sin/cos approximation on [-pi, pi))
__device__ inline float2 phasor_f(float turns) {
  float s, c;
  __sincosf(turns * kTwoPiF, &s, &c);
  return make_float2(c, s);
}

// exp(+2 pi i x) in FP64, x reduced by x - rint(x) first
__device__ inline double2 phasor_d(double x) {
  double f = x - rint(x);
  double s, c;
  sincospi(2.0 * f, &s, &c);
  return make_double2(c, s);
}

}  // namespace rts
