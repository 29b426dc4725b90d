// srs_slide.cu -- stack-slide over the per-segment power cube (Sec. III.C,
// Eqs. (weights) and (semicoherent_statistic) with equal weights; Sec. VI).
//
// Stage two of the two-stage search.  Stage one (k_mixed in spectra mode with
// per-segment templates) writes P[k][j][i]: bank entry k, bin j, segment i
// innermost.  A template theta = {Mc, t0 = (n + c) T} reads one power per
// segment of its track.  Rows r share (Mc, c) and differ only in the whole
// segment n of t0, so the tracks of one row are one (k_s, j_s) sequence
// shifted in i: a warp of 32 consecutive n reads 32 consecutive floats of
// the same cube row at every step, a coalesced 128-byte request.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "srs_device.cuh"
#include "srs_slide.h"

namespace srs {

namespace {

constexpr int kSlideThreads = 256;   // t0 columns per block
constexpr int kSlideStage = 2048;    // track cells staged in shared memory at a time
constexpr int kTrackThreads = 256;

// One (row, track segment) per thread.  The 0PN frequency at the segment's
// first sample, dt = (s + [c > 0] - c) T after t0 (Eq. f):
//   A = 1 - (8/3) beta0 dt,  f = f0 A^(-3/8),
// its nearest bin rint((f - f_lo) T), and the nearest bank entry to the local
// chirp parameter beta(Mc, f) = beta0 (f / f0)^(8/3) = beta0 / A (Eq. beta).
// A segment is on the track while A > 0 and its bin is inside the band; the
// frequency only rises, so the valid segments are a prefix of the row.
// Weight: A_s^2 ~ f^(4/3) = f0^(4/3) A^(-1/2) (Sec. II Eq. h0 with Eq. f); its
// mean over the segment, in units of f0^(4/3), is
//   (1/T) int A(u)^(-1/2) du = 2 / (sqrt(A_start) + sqrt(A_end)),
// written without the difference of square roots.
__global__ void k_slide_tracks(const double* __restrict__ beta0, const double* __restrict__ frac, int n_rows,
                               TrackArgs t, int* __restrict__ cell, float2* __restrict__ coef) {
  const long long total = (long long)n_rows * t.n_total;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / t.n_total);
    const int s = (int)(idx - (long long)r * t.n_total);
    const double b0 = beta0[r];
    const double c = frac[r];
    const double dt = ((double)s + (c > 0.0 ? 1.0 : 0.0) - c) * t.t_coh;
    const double A = 1.0 - (8.0 / 3.0) * b0 * dt;
    int out = -1;
    float2 cf = make_float2(0.f, 0.f);
    if (A > 0.0) {
      const double f = t.f0 * exp(-0.375 * log(A));
      const double jd = rint((f - t.f_lo) * t.t_coh);
      if (jd >= 0.0 && jd <= (double)(t.n_bins - 1)) {
        double kd = t.dbeta > 0.0 ? rint((b0 / A - t.beta_min) / t.dbeta) : 0.0;
        kd = fmin(fmax(kd, 0.0), (double)(t.n_beta - 1));
        out = (int)kd * t.n_bins + (int)jd;
        double a = 1.0;
        if (t.weighting == SRS_WEIGHT_AMPLITUDE) {
          const double A1 = fmax(1.0 - (8.0 / 3.0) * b0 * (dt + t.t_coh), 0.0);
          a = 2.0 / (sqrt(A) + sqrt(A1));
        }
        const double S = t.s_eff ? (double)t.s_eff[out] : 1.0;
        a /= S;
        // a whitened cube is divided by S already: S enters the weight alone
        const double Sp = t.s_in_weights_only ? 1.0 : S;
        cf = make_float2((float)(0.5 * a / Sp), (float)a);
      }
    }
    cell[idx] = out;
    coef[idx] = cf;
  }
}

// len[r] = index of the first -1 in row r, and w2[r][s] = sum_{s' < s} a_s'^2
// for s <= len[r] (an inclusive warp scan per 32 steps; one warp per row).
__global__ void k_slide_lengths(const int* __restrict__ cell, const float2* __restrict__ coef, int n_rows,
                                int n_total, int* __restrict__ len, double* __restrict__ w2) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n_rows) return;
  const int* row = cell + (long long)warp * n_total;
  const float2* crow = coef + (long long)warp * n_total;
  double* wrow = w2 + (long long)warp * (n_total + 1);
  if (lane == 0) wrow[0] = 0.0;
  int L = n_total;
  double run = 0.0;
  for (int s0 = 0; s0 < n_total; s0 += 32) {
    const int s = s0 + lane;
    const bool on = s < n_total && row[s] >= 0;
    const unsigned end = __ballot_sync(0xffffffffu, s < n_total && !on);
    const float a = on ? crow[s].y : 0.f;
    double v = (double)a * (double)a;
    for (int d = 1; d < 32; d <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += u;
    }
    const int stop = end ? s0 + __ffs(end) - 1 : n_total;   // first step past the track
    if (s < stop) wrow[s + 1] = run + v;
    run += __shfl_sync(0xffffffffu, v, 31);
    if (end) {
      L = stop;
      break;
    }
  }
  if (lane == 0) len[warp] = L;
}

// Block = (row r, tile of kSlideThreads t0 columns).  Thread n sums the
// powers of its track segments s whose segment i = first + s lies in the
// chunk, first = n + [c > 0], and s < min(len_r, n_total - first).  The
// row's track cells (and, WEIGHTED, their FMA coefficients) are staged in
// shared memory; four accumulators keep four loads in flight per thread.
// Without weights every term is P / 2 - 1.  OFF32: the staged value is the
// 32-bit cube offset cell_s * ld + s, and each thread adds it to its own
// base cube + first - seg_begin, so a power read is one shared load, one
// address multiply-add and the load.
template <bool WEIGHTED, bool OFF32>
__global__ void __launch_bounds__(kSlideThreads)
k_stack_slide(const float* __restrict__ cube, const int* __restrict__ cell, const float2* __restrict__ coef,
              const int* __restrict__ len, const double* __restrict__ w2, const double* __restrict__ frac,
              SlideArgs a, float* __restrict__ Z, float* __restrict__ map, unsigned long long* __restrict__ keys) {
  __shared__ int sc[kSlideStage];
  __shared__ float2 sw[WEIGHTED ? kSlideStage : 1];
  const int tiles = (a.n_t0 + kSlideThreads - 1) / kSlideThreads;
  const int r = blockIdx.x / tiles;
  const int tile = blockIdx.x - r * tiles;
  const int n0 = tile * kSlideThreads;
  const int n = n0 + threadIdx.x;
  const int e = frac[r] > 0.0 ? 1 : 0;
  const int L = len[r];
  const int first = n + e;
  const int Lp = max(0, min(L, a.n_total - first));           // N_seg(theta) inside the data
  const int s_lo = max(0, a.seg_begin - first);
  const int s_hi = n < a.n_t0 ? min(Lp, a.seg_end - first) : 0;
  // the block's union of track steps inside the chunk
  const int last_n = min(n0 + kSlideThreads, a.n_t0) - 1;
  const int S_lo = max(0, a.seg_begin - (last_n + e));
  const int S_hi = min(L, a.seg_end - (n0 + e));
  const int* __restrict__ crow = cell + (long long)r * a.n_total;
  const float2* __restrict__ wrow = coef + (long long)r * a.n_total;
  // cube index of track step s: cell_s * ld + (first + s - seg_begin)
  const long long c0 = (long long)first - a.seg_begin;
  // OFF32: this thread's base; every index it adds lands inside the cube
  const float* __restrict__ cb = cube + c0;
  const unsigned* __restrict__ so = reinterpret_cast<const unsigned*>(sc);
  float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
  for (int base = S_lo; base < S_hi; base += kSlideStage) {
    const int cnt = min(kSlideStage, S_hi - base);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += kSlideThreads) {
      if (OFF32) sc[t] = (int)((unsigned)crow[base + t] * (unsigned)a.ld + (unsigned)(base + t));
      else sc[t] = crow[base + t];
      if (WEIGHTED) sw[t] = wrow[base + t];
    }
    __syncthreads();
    const int lo = max(s_lo, base), hi = min(s_hi, base + cnt);
    int s = lo;
    if (OFF32) {
      for (; s + 3 < hi; s += 4) {
        const float p0 = __ldg(cb + so[s - base]);
        const float p1 = __ldg(cb + so[s + 1 - base]);
        const float p2 = __ldg(cb + so[s + 2 - base]);
        const float p3 = __ldg(cb + so[s + 3 - base]);
        if (WEIGHTED) {
          const float2 w0 = sw[s - base], w1 = sw[s + 1 - base], w2_ = sw[s + 2 - base], w3 = sw[s + 3 - base];
          z0 += fmaf(p0, w0.x, -w0.y);
          z1 += fmaf(p1, w1.x, -w1.y);
          z2 += fmaf(p2, w2_.x, -w2_.y);
          z3 += fmaf(p3, w3.x, -w3.y);
        } else {
          z0 += fmaf(p0, 0.5f, -1.0f);
          z1 += fmaf(p1, 0.5f, -1.0f);
          z2 += fmaf(p2, 0.5f, -1.0f);
          z3 += fmaf(p3, 0.5f, -1.0f);
        }
      }
      for (; s < hi; ++s) {
        const float2 w = WEIGHTED ? sw[s - base] : make_float2(0.5f, 1.0f);
        z0 += fmaf(__ldg(cb + so[s - base]), w.x, -w.y);
      }
      continue;
    }
    // term of track step s: a_s (P / S_s - 2) / 2 = sw.x P - sw.y
    for (; s + 3 < hi; s += 4) {
      const float p0 = __ldg(cube + ((long long)sc[s - base] * a.ld + c0 + s));
      const float p1 = __ldg(cube + ((long long)sc[s + 1 - base] * a.ld + c0 + s + 1));
      const float p2 = __ldg(cube + ((long long)sc[s + 2 - base] * a.ld + c0 + s + 2));
      const float p3 = __ldg(cube + ((long long)sc[s + 3 - base] * a.ld + c0 + s + 3));
      if (WEIGHTED) {
        const float2 w0 = sw[s - base], w1 = sw[s + 1 - base], w2_ = sw[s + 2 - base], w3 = sw[s + 3 - base];
        z0 += fmaf(p0, w0.x, -w0.y);
        z1 += fmaf(p1, w1.x, -w1.y);
        z2 += fmaf(p2, w2_.x, -w2_.y);
        z3 += fmaf(p3, w3.x, -w3.y);
      } else {
        z0 += fmaf(p0, 0.5f, -1.0f);
        z1 += fmaf(p1, 0.5f, -1.0f);
        z2 += fmaf(p2, 0.5f, -1.0f);
        z3 += fmaf(p3, 0.5f, -1.0f);
      }
    }
    for (; s < hi; ++s) {
      const float2 w = WEIGHTED ? sw[s - base] : make_float2(0.5f, 1.0f);
      z0 += fmaf(__ldg(cube + ((long long)sc[s - base] * a.ld + c0 + s)), w.x, -w.y);
    }
  }
  if (n >= a.n_t0) return;
  const long long o = (long long)r * a.n_t0 + n;
  float z = (z0 + z1) + (z2 + z3);
  if (!a.first) z += Z[o];
  if (!a.last) {
    Z[o] = z;
    return;
  }
  // FP32 from here: the FP64 units are few on this part
  // sum of a_s^2 over the track's segments in the data (N_seg itself without weights)
  const float norm = Lp <= 0 ? 0.f : WEIGHTED ? (float)w2[(long long)r * (a.n_total + 1) + Lp] : (float)Lp;
  const float v = norm > 0.f ? z / sqrtf(norm) : 0.f;
  if (map) map[o] = v;
  keys[o] = make_key(v, (uint32_t)o);
}

// Whitening (Sec. III.C: powers normalised by the effective PSD, background
// moments mu_i, sigma_i taken from the data).
// S[r] = mean over the row's n_seg segments of P / 2: one warp per row.
__global__ void k_cube_psd(const float* __restrict__ cube, long long rows, int ld, int n_seg, float* __restrict__ S) {
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const float* row = cube + r * ld;
  float s = 0.f;
  for (int i = lane; i < n_seg; i += 32) s += row[i];
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if (lane == 0) S[r] = fmaxf(s / (2.0f * (float)n_seg), 1e-30f);
}

// Per segment i: sum and sum of squares over rows of P / S.  Block = 256
// consecutive segments x a tile of rows (coalesced along i); FP32 within the
// tile, FP64 atomics across tiles.
__global__ void k_cube_moments(const float* __restrict__ cube, long long rows, int ld, int n_seg,
                               const float* __restrict__ S, int rows_per_block, double* __restrict__ sums) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const long long r0 = (long long)blockIdx.y * rows_per_block;
  const long long r1 = min(rows, r0 + rows_per_block);
  if (i >= n_seg) return;
  float s = 0.f, q = 0.f;
  for (long long r = r0; r < r1; ++r) {
    const float v = cube[r * ld + i] / S[r];
    s += v;
    q = fmaf(v, v, q);
  }
  atomicAdd(&sums[i], (double)s);
  atomicAdd(&sums[n_seg + i], (double)q);
}

// mu_i and 1 / sigma_i (population moments over all rows).
__global__ void k_cube_moments_finish(const double* __restrict__ sums, long long rows, int n_seg,
                                      float2* __restrict__ musig, float* __restrict__ mu, float* __restrict__ sigma) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_seg) return;
  const double m = sums[i] / (double)rows;
  const double var = fmax(sums[n_seg + i] / (double)rows - m * m, 1e-30);
  const double sd = sqrt(var);
  musig[i] = make_float2((float)m, (float)(1.0 / sd));
  if (mu) mu[i] = (float)m;
  if (sigma) sigma[i] = (float)sd;
}

// P <- 2 + 2 (P / S - mu_i) / sigma_i, in place.
__global__ void k_cube_apply(float* __restrict__ cube, long long rows, int ld, int n_seg,
                             const float* __restrict__ S, const float2* __restrict__ musig) {
  const long long total = rows * (long long)n_seg;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / n_seg;
    const int i = (int)(idx - r * n_seg);
    float* p = cube + r * ld + i;
    const float2 ms = musig[i];
    *p = fmaf(2.0f * ms.y, *p / S[r] - ms.x, 2.0f);
  }
}

}  // namespace

cudaError_t launch_cube_whiten(float* cube, long long rows, int ld, int n_seg, float* S, bool estimate_s,
                               double* sums, float2* musig, float* mu, float* sigma, int n_sm, cudaStream_t st) {
  if (rows <= 0 || n_seg <= 0) return cudaSuccess;
  cudaError_t e;
  if (estimate_s) {
    k_cube_psd<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(cube, rows, ld, n_seg, S);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = cudaMemsetAsync(sums, 0, (size_t)2 * n_seg * sizeof(double), st)) != cudaSuccess) return e;
  // tiles of 64 rows, more where the grid's y extent (65535) would not hold them
  const int per = (int)std::max<long long>(64, (rows + 65534) / 65535);
  const dim3 g((unsigned)((n_seg + 255) / 256), (unsigned)((rows + per - 1) / per));
  k_cube_moments<<<g, 256, 0, st>>>(cube, rows, ld, n_seg, S, per, sums);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_cube_moments_finish<<<(unsigned)((n_seg + 255) / 256), 256, 0, st>>>(sums, rows, n_seg, musig, mu, sigma);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  long long blocks = (rows * (long long)n_seg + 255) / 256;
  if (blocks > (long long)n_sm * 16) blocks = (long long)n_sm * 16;
  k_cube_apply<<<(unsigned)blocks, 256, 0, st>>>(cube, rows, ld, n_seg, S, musig);
  return cudaGetLastError();
}

cudaError_t launch_slide_tracks(const double* beta0, const double* frac, int n_rows, const TrackArgs& t,
                                int* cell, float2* coef, int* len, double* w2, int n_sm, cudaStream_t st) {
  const long long total = (long long)n_rows * t.n_total;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + kTrackThreads - 1) / kTrackThreads;
  if (blocks > (long long)n_sm * 32) blocks = (long long)n_sm * 32;
  k_slide_tracks<<<(unsigned)blocks, kTrackThreads, 0, st>>>(beta0, frac, n_rows, t, cell, coef);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long threads = (long long)n_rows * 32;
  k_slide_lengths<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(cell, coef, n_rows, t.n_total, len, w2);
  return cudaGetLastError();
}

cudaError_t launch_stack_slide(const float* cube, const int* cell, const float2* coef, const int* len,
                               const double* w2, const double* frac, const SlideArgs& a, float* Z, float* map,
                               unsigned long long* keys, cudaStream_t st) {
  const long long tiles = (a.n_t0 + kSlideThreads - 1) / kSlideThreads;
  const long long blocks = tiles * a.n_rows;
  if (blocks <= 0) return cudaSuccess;
  if (a.weighted && a.off32)
    k_stack_slide<true, true><<<(unsigned)blocks, kSlideThreads, 0, st>>>(cube, cell, coef, len, w2, frac, a, Z, map,
                                                                         keys);
  else if (a.weighted)
    k_stack_slide<true, false><<<(unsigned)blocks, kSlideThreads, 0, st>>>(cube, cell, coef, len, w2, frac, a, Z, map,
                                                                          keys);
  else if (a.off32)
    k_stack_slide<false, true><<<(unsigned)blocks, kSlideThreads, 0, st>>>(cube, cell, coef, len, w2, frac, a, Z, map,
                                                                          keys);
  else
    k_stack_slide<false, false><<<(unsigned)blocks, kSlideThreads, 0, st>>>(cube, cell, coef, len, w2, frac, a, Z, map,
                                                                           keys);
  return cudaGetLastError();
}

}  // namespace srs
