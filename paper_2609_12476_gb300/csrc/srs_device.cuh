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
  an.psi0 = frac_to_u32(psi - floor(psi));
  const double E1 = e1 * inv_fs;                                  // d delta / d sample
  double P1 = E1 * inv_t;
  double P1f = P1 - floor(P1);
  double N1 = rint(P1f * 4294967296.0);
  an.n1 = (uint32_t)((long long)N1 & 0xffffffffLL);
  an.p1lo = (float)(P1f - N1 * 2.3283064365386962890625e-10);
  double th = aa.f_c * d0;
  an.th0 = frac_to_u32(th - floor(th));
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
  an.p2 = (float)(E2 * inv_t);
  an.p3 = (float)(E3 * inv_t);
  an.p4 = (float)(E4 * inv_t);
  an.p5 = (float)(E5 * inv_t);
  an.pad0 = 0.f;
  an.pad1 = 0.f;
  return an;
}

// Phase of sample l (0 <= l < span) of an anchor's span: the fine-grid phase
// Psi (unsigned 32-bit fixed point, periods of t_coh) and the demodulation
// phase th = f_c delta mod 1 in [-0.5, 0.5] (cycles).
__device__ __forceinline__ void mixed_phase(const Anchor& A, int l, float kc, uint32_t& Psi, float& th) {
  const float lf = (float)l;
  const float cq = fmaf(fmaf(fmaf(A.p5, lf, A.p4), lf, A.p3), lf, A.p2) * (lf * lf);
  const float cpsi = fmaf(A.p1lo, lf, cq);
  Psi = A.psi0 + (uint32_t)l * A.n1 + (uint32_t)__float2int_rn(cpsi * 4294967296.0f);
  const float cth = fmaf(A.m1lo, lf, kc * cq);
  float t = (float)(int32_t)(A.th0 + (uint32_t)l * A.m1) * 2.3283064365386963e-10f + cth;
  th = t - rintf(t);
}

// The fine-grid phase alone (periods, 32-bit fixed point) of sample l.
__device__ __forceinline__ uint32_t mixed_psi(const Anchor& A, int l) {
  const float lf = (float)l;
  const float cq = fmaf(fmaf(fmaf(A.p5, lf, A.p4), lf, A.p3), lf, A.p2) * (lf * lf);
  const float cpsi = fmaf(A.p1lo, lf, cq);
  return A.psi0 + (uint32_t)l * A.n1 + (uint32_t)__float2int_rn(cpsi * 4294967296.0f);
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
