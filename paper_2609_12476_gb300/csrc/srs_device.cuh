// srs_device.cuh -- device functions shared by the kernels of libsrs: the
// FP64 anchors of the resampled time and the per-sample fixed-point phase.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "srs_internal.h"
#include "srs_kernels.h"

namespace srs {

__device__ __forceinline__ uint32_t frac_to_u32(double f) {  // f in [0, 1)
  long long v = __double2ll_rn(f * 4294967296.0);
  return (uint32_t)(v & 0xffffffffLL);
}

// f in [0, 1) as 64-bit fixed point (the double's 53 bits), high and low words.
__device__ __forceinline__ void frac_to_u64(double f, uint32_t& hi, uint32_t& lo) {
  const double h = floor(f * 4294967296.0);
  const double r = f * 4294967296.0 - h;                       // exact: f 2^32 has the same ulp as f
  long long l = __double2ll_rn(r * 4294967296.0);
  long long hh = (long long)h;
  if (l >= 4294967296LL) { l -= 4294967296LL; ++hh; }
  hi = (uint32_t)(hh & 0xffffffffLL);
  lo = (uint32_t)l;
}

// Coefficients of the two binomial series of the time map in y = 8/3 beta s / A
// (Eq. new_t around a point where 1 - 8/3 beta t = A):
//   1 - (1 - y)^(5/8) = sum_{k>=1} c_k y^k,  c_1 = 5/8, c_{k+1} = c_k (k - 5/8) / (k + 1)
//   (1 - y)^(-3/8)    = sum_{k>=0} d_k y^k,  d_0 = 1,   d_{k+1} = d_k (k + 3/8) / (k + 1)
// Seventeen terms reach double precision for y <= 1/8.
constexpr int kSeriesTerms = 17;
struct TimeSeries {
  double c[kSeriesTerms + 1], d[kSeriesTerms + 1];
  constexpr TimeSeries() : c(), d() {
    c[0] = 0.0;
    c[1] = 0.625;
    d[0] = 1.0;
    for (int k = 1; k < kSeriesTerms; ++k) c[k + 1] = c[k] * ((double)k - 0.625) / (double)(k + 1);
    for (int k = 0; k < kSeriesTerms; ++k) d[k + 1] = d[k] * ((double)k + 0.375) / (double)(k + 1);
  }
};
constexpr double kSeriesMaxY = 0.125;

// Anchor ai of segment i of a template with chirp parameter b (Eq. new_t
// expanded around the anchor sample l_a = ai * span): the segment-local
// resampled time delta(s) = tau(t_i0 + s) - tau(t_i0) at s0 = l_a / fs, written
// without cancellation, its derivative A^(-3/8) (= f / f0, Eq. f), and the
// Taylor coefficients of delta in the sample index.
__device__ __forceinline__ Anchor compute_anchor(double b, int i, int ai, const AnchorArgs& aa) {
  const double inv_fs = 1.0 / aa.fs, inv_t = 1.0 / aa.t_coh;
  // local: the segment's own 0PN template starts at its first sample
  const double t_i0 = aa.local ? 0.0 : (double)i * (double)aa.n_s * inv_fs;
  const double a = 1.0 - (8.0 / 3.0) * b * t_i0;
  const double inv_a = 1.0 / a;
  const double a58 = exp(0.625 * log(a));                       // a^(5/8)
  const double s0 = (double)ai * (double)aa.span * inv_fs;
  const double x = (8.0 / 3.0) * b * s0 * inv_a;
  const double k0 = 0.6 * a58 / b;                                // 3 a^(5/8) / (5 beta)
  double d0, e1;                                                  // delta(s0), A^(-3/8)
  if (x <= kSeriesMaxY) {
    constexpr TimeSeries ts;
    double sc = ts.c[kSeriesTerms], sd = ts.d[kSeriesTerms];
#pragma unroll
    for (int k = kSeriesTerms - 1; k >= 0; --k) {
      sc = fma(sc, x, ts.c[k]);
      sd = fma(sd, x, ts.d[k]);
    }
    d0 = k0 * sc;
    e1 = a58 * inv_a * sd;
  } else {
    const double L = log1p(-x);                                   // log(A / a)
    d0 = k0 * (-expm1(0.625 * L));
    e1 = a58 * inv_a * exp(-0.375 * L);
  }
  const double A = a * (1.0 - x);                                 // 1 - 8/3 beta (t_i0 + s0)
  Anchor an;
  double psi = d0 * inv_t;
  frac_to_u64(psi - floor(psi), an.psi0, an.psi0lo);
  const double E1 = e1 * inv_fs;                                  // d delta / d sample
  double P1 = E1 * inv_t;
  double P1f = P1 - floor(P1);
  double N1 = rint(P1f * 4294967296.0);
  an.n1 = (uint32_t)((long long)N1 & 0xffffffffLL);
  an.p1lo = (float)(P1f - N1 * 2.3283064365386962890625e-10);
  double th = aa.f_c * d0;
  frac_to_u64(th - floor(th), an.th0, an.th0lo);
  double M1 = aa.f_c * E1;
  double M1f = M1 - floor(M1);
  double Mr = rint(M1f * 4294967296.0);
  an.m1 = (uint32_t)((long long)Mr & 0xffffffffLL);
  an.m1lo = (float)(M1f - Mr * 2.3283064365386962890625e-10);
  // E_{k+1} = E_k * (8/3)(3/8 + k - 1) beta / (A fs (k + 1)), per sample, in periods
  const double r = b * inv_fs / A;
  const double E2 = E1 * r * 0.5;
  const double E3 = E2 * r * (11.0 / 9.0);
  const double E4 = E3 * r * (19.0 / 12.0);
  const double E5 = E4 * r * (9.0 / 5.0);
  an.q2 = __double2ll_rn(E2 * inv_t * 18446744073709551616.0);       // 2^-64 periods / sample^2
  an.kq2 = __double2ll_rn(aa.f_c * E2 * 18446744073709551616.0);     // 2^-64 cycles / sample^2
  an.p3 = (float)(E3 * inv_t);
  an.p4 = (float)(E4 * inv_t);
  an.p5 = (float)(E5 * inv_t);
  an.pad = 0u;
  return an;
}

// A small FP32 value (periods or cycles) in 2^-64 fixed point, two's complement.
__device__ __forceinline__ unsigned long long fix64(float v) {
  return (unsigned long long)__float2ll_rn(v * 18446744073709551616.0f);
}

// One phase of an anchor's span in 64-bit fixed point (2^-64 of a period or
// cycle, wrapping at whole periods): value at sample l of
//   c0 + l c1 + q l^2 + s (P3 l^3 + P4 l^4 + P5 l^5)
// with c0 64-bit and c1 32-bit fixed point, c1lo the FP32 residual of c1, q the 64-bit
// quadratic coefficient and s a scale of the higher FP32 terms (1 for the
// fine-grid phase, k_c for the demodulation phase).
__device__ __forceinline__ unsigned long long anchor_phase64(const Anchor& A, unsigned long long c0, uint32_t c1,
                                                             float c1lo, long long q, float s, int l) {
  const float lf = (float)l;
  const float q3 = s * fmaf(fmaf(A.p5, lf, A.p4), lf, A.p3) * (lf * lf * lf);
  // unsigned products: the phase wraps at whole periods (mod 2^64)
  const unsigned long long L = (unsigned long long)l;
  return c0 + ((unsigned long long)((uint32_t)l * c1) << 32) + L * fix64(c1lo) +
         (unsigned long long)q * (L * L) + fix64(q3);
}

// The anchor's phases at its own sample in 64-bit fixed point.
__device__ __forceinline__ unsigned long long anchor_psi0(const Anchor& A) {
  return ((unsigned long long)A.psi0 << 32) | A.psi0lo;
}
__device__ __forceinline__ unsigned long long anchor_th0(const Anchor& A) {
  return ((unsigned long long)A.th0 << 32) | A.th0lo;
}

// Phase of sample l (0 <= l < span) of an anchor's span: the fine-grid phase
// Psi (unsigned 32-bit fixed point, periods of t_coh) and the demodulation
// phase f_c delta mod 1 (unsigned 32-bit fixed point, cycles).
__device__ __forceinline__ void mixed_phase_fix(const Anchor& A, int l, float kc, uint32_t& Psi, uint32_t& Th) {
  const unsigned long long p = anchor_phase64(A, anchor_psi0(A), A.n1, A.p1lo, A.q2, 1.0f, l);
  const unsigned long long t = anchor_phase64(A, anchor_th0(A), A.m1, A.m1lo, A.kq2, kc, l);
  Psi = (uint32_t)((p + 0x80000000ull) >> 32);
  Th = (uint32_t)((t + 0x80000000ull) >> 32);
}

// The same with the demodulation phase as th in [-0.5, 0.5) cycles.
__device__ __forceinline__ void mixed_phase(const Anchor& A, int l, float kc, uint32_t& Psi, float& th) {
  uint32_t Th;
  mixed_phase_fix(A, l, kc, Psi, Th);
  th = (float)(int32_t)Th * 2.3283064365386963e-10f;
}

// Per-lane time map of the spreader.  A lane walks consecutive samples; from
// the anchor it takes one phase at its first sample and the phase's first,
// second and third forward differences, all in 64-bit fixed point (2^-64 of
// a period or cycle), and then steps sample by sample with integer adds
// (exact apart from the fourth and higher differences of the anchor's
// polynomial, below 1e-12 periods over a lane's run).
struct LaneMap {
  unsigned long long v, d1, d2, d3;
  __device__ __forceinline__ void step() {
    v += d1;
    d1 += d2;
    d2 += d3;
  }
};

// Seed a LaneMap at sample l of an anchor's span (see anchor_phase64 for the
// arguments): forward differences of the polynomial written out term by term,
//   D(l^2) = 2l + 1, D^2(l^2) = 2,
//   D(l^3) = 3l^2 + 3l + 1, D^2(l^3) = 6l + 6, D^3(l^3) = 6,
//   D(l^4) = 4l^3 + 6l^2 + 4l + 1, D^2(l^4) = 12l^2 + 24l + 14, D^3(l^4) = 24l + 36,
//   D(l^5) = 5l^4 + 10l^3 + 10l^2 + 5l + 1, D^2(l^5) = 20l^3 + 60l^2 + 70l + 30,
//   D^3(l^5) = 60l^2 + 180l + 150.
__device__ __forceinline__ LaneMap lane_map(const Anchor& A, unsigned long long c0, uint32_t c1, float c1lo,
                                            long long q, float s, int l) {
  const float lf = (float)l, l2 = lf * lf, l3 = l2 * lf;
  const float p3 = s * A.p3, p4 = s * A.p4, p5 = s * A.p5;
  const float d1 = p3 * fmaf(3.f, l2 + lf, 1.f) + p4 * fmaf(4.f, l3 + lf, fmaf(6.f, l2, 1.f)) +
                   p5 * fmaf(5.f, fmaf(l2, l2, lf), fmaf(10.f, l3 + l2, 1.f));
  const float d2 = p3 * fmaf(6.f, lf, 6.f) + p4 * fmaf(12.f, l2, fmaf(24.f, lf, 14.f)) +
                   p5 * fmaf(20.f, l3, fmaf(60.f, l2, fmaf(70.f, lf, 30.f)));
  const float d3 = 6.f * p3 + p4 * fmaf(24.f, lf, 36.f) + p5 * fmaf(60.f, l2, fmaf(180.f, lf, 150.f));
  const unsigned long long L = (unsigned long long)l, Q = (unsigned long long)q;
  LaneMap m;
  m.v = anchor_phase64(A, c0, c1, c1lo, q, s, l);
  m.d1 = ((unsigned long long)c1 << 32) + fix64(c1lo) + Q * (2 * L + 1) + fix64(d1);
  m.d2 = 2 * Q + fix64(d2);
  m.d3 = fix64(d3);
  return m;
}

// Top-k sort key of a map cell: larger value first, then smaller flat index
// (value bits made order-preserving as unsigned, flat index complemented).
__device__ __forceinline__ unsigned long long make_key(float v, uint32_t flat) {
  uint32_t u = __float_as_uint(v);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 32) | (unsigned long long)(~flat);
}
__device__ __forceinline__ float key_value(unsigned long long k) {
  uint32_t u = (uint32_t)(k >> 32);
  u = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  return __uint_as_float(u);
}

}  // namespace srs
