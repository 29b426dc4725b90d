// srs_learn.cu -- kernels of the learned proposal and its training data.
//
// The network proposes which fine (template, frequency) cells to compute in
// full from a coarse-template n_sigma map: input a 9 x 33 patch of the map
// (coarse templates m-4..m+4, bins b-16..b+16, zero outside the map), each
// value passed through asinh; a 297 -> 64 (ReLU) -> 1 MLP with FP16 weights
// and FP32 accumulation gives a logit; training minimises binary cross
// entropy with Adam on FP32 master weights.  Training maps come from the
// search itself run on seeded Gaussian noise with injected 0PN chirps
// (Sec. III.A Eqs. f, phi).  Refinement evaluates the proposed fine cells
// with a direct sum over the segment's samples at those bins (the transform
// the NUFFT approximates, Sec. III.B), accumulated into n_sigma like the
// full search.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "srs_internal.h"
#include "srs_kernels.h"
#include "srs_learn.h"
#include "srs_device.cuh"

namespace srs {

// ---------------------------------------------------------------------------
// Counter-based Gaussian noise: Philox-4x32 rounds (Salmon et al. 2011,
// "Parallel random numbers: as easy as 1, 2, 3"), 10 rounds, then Box-Muller.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// 4 N(0,1) values for counter `ctr` of stream `seed`.
__device__ __forceinline__ float4 gauss4(uint64_t seed, uint64_t ctr) {
  const uint4 r = philox4x32_10(make_uint4((uint32_t)ctr, (uint32_t)(ctr >> 32), 0x5352u, 0x5352u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  // uniforms in (0, 1]
  const float u0 = ((float)(r.x >> 8) + 1.0f) * 5.9604644775390625e-08f;
  const float u1 = ((float)(r.y >> 8) + 0.5f) * 5.9604644775390625e-08f;
  const float u2 = ((float)(r.z >> 8) + 1.0f) * 5.9604644775390625e-08f;
  const float u3 = ((float)(r.w >> 8) + 0.5f) * 5.9604644775390625e-08f;
  const float ra = sqrtf(-2.0f * logf(u0)), rb = sqrtf(-2.0f * logf(u2));
  float sa, ca, sb, cb;
  sincospif(2.0f * u1, &sa, &ca);
  sincospif(2.0f * u3, &sb, &cb);
  return make_float4(ra * ca, ra * sa, rb * cb, rb * sb);
}

// strain[j] = (noise ? N(0,1) : 0) + sum over injections of A cos(phi(t)), t = j / fs,
// phi(t) - phi0 = 2 pi f0 (3 / (5 beta)) (1 - (1 - 8/3 beta t)^(5/8)) for t < t_end
// (Eq. phi minus its value at t = 0; t_end is where the chirp leaves the band).
__global__ void k_make_strain(float* __restrict__ out, long long n, double fs, unsigned long long seed, int noise,
                              const InjectionDev* __restrict__ inj, int n_inj) {
  extern __shared__ InjectionDev s_inj[];
  for (int k = threadIdx.x; k < n_inj; k += blockDim.x) s_inj[k] = inj[k];
  __syncthreads();
  const long long quads = (n + 3) / 4;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < quads; q += (long long)gridDim.x * blockDim.x) {
    float4 z = noise ? gauss4(seed, (uint64_t)q) : make_float4(0.f, 0.f, 0.f, 0.f);
    float v[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const long long j = 4 * q + e;
      const double t = (double)j / fs;
      double acc = 0.0;
      for (int k = 0; k < n_inj; ++k) {
        const InjectionDev I = s_inj[k];
        if (t >= I.t_end) continue;
        const double x = (8.0 / 3.0) * I.beta * t;
        const double cyc = I.f0 * 3.0 / (5.0 * I.beta) * (-expm1(0.625 * log1p(-x))) + I.phi0_cyc;
        acc += I.amp * cospi(2.0 * (cyc - floor(cyc)));
      }
      v[e] += (float)acc;
    }
    for (int e = 0; e < 4; ++e)
      if (4 * q + e < n) out[4 * q + e] = v[e];
  }
}

// ---------------------------------------------------------------------------
// Patches and the MLP
// ---------------------------------------------------------------------------
__device__ __forceinline__ float feature(float x) { return asinhf(x); }

// out[k][r][c] = asinh(map[m_k + r - 4][b_k + c - 16]), zero outside the map.
__global__ void k_patches(const float* __restrict__ map, int n_templates, int n_bins, const int* __restrict__ cm,
                          const int* __restrict__ cb, int n, float* __restrict__ out) {
  const long long total = (long long)n * kPatchSize;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(f / kPatchSize);
    const int e = (int)(f - (long long)k * kPatchSize);
    const int r = e / kPatchBins, c = e - r * kPatchBins;
    const int m = cm[k] + r - kPatchTemplates / 2, b = cb[k] + c - kPatchBins / 2;
    float v = 0.f;
    if (m >= 0 && m < n_templates && b >= 0 && b < n_bins) v = feature(map[(long long)m * n_bins + b]);
    out[f] = v;
  }
}

// Forward pass: four samples per 256-thread block, one hidden unit per thread.
// z1 = W1 x + b1 (FP16 weights, FP32 sums), h = relu(z1), logit = w2 . h + b2.
__global__ void __launch_bounds__(256)
k_mlp_forward(const float* __restrict__ X, int n, const __half* __restrict__ W1h, const float* __restrict__ b1,
              const __half* __restrict__ w2h, const float* __restrict__ b2p, float* __restrict__ logits,
              float* __restrict__ Z1) {
  const float b2 = *b2p;
  __shared__ float sx[4][kPatchSize];
  __shared__ float sp[4][kHidden];
  const int g = threadIdx.x / kHidden, j = threadIdx.x % kHidden;
  for (long long s0 = (long long)blockIdx.x * 4; s0 < n; s0 += (long long)gridDim.x * 4) {
    for (int t = threadIdx.x; t < 4 * kPatchSize; t += blockDim.x) {
      const int gg = t / kPatchSize, e = t - gg * kPatchSize;
      const long long s = s0 + gg;
      sx[gg][e] = s < n ? X[s * kPatchSize + e] : 0.f;
    }
    __syncthreads();
    const long long s = s0 + g;
    const __half* w = W1h + (long long)j * kPatchSize;
    float acc = b1[j];
    for (int e = 0; e < kPatchSize; ++e) acc = fmaf(__half2float(w[e]), sx[g][e], acc);
    if (Z1 && s < n) Z1[s * kHidden + j] = acc;
    sp[g][j] = fmaxf(acc, 0.f) * __half2float(w2h[j]);
    __syncthreads();
    if (j < 32) {
      float v = sp[g][j] + sp[g][j + 32];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (j == 0 && s < n) logits[s] = v + b2;
    }
    __syncthreads();
  }
}

// dL/dlogit for L = mean_s softplus(z_s) - y_s z_s (binary cross entropy with
// logits), and each sample's loss term.
__global__ void k_bce(const float* __restrict__ logits, const float* __restrict__ y, int n, float* __restrict__ dz,
                      float* __restrict__ loss_terms) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const float z = logits[s];
    const float sg = 1.0f / (1.0f + expf(-z));
    dz[s] = (sg - y[s]) / (float)n;
    loss_terms[s] = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - y[s] * z;
  }
}

// Gradients of the batch, one thread per parameter (deterministic order):
// params are W1 [64][297], b1 [64], w2 [64], b2.
__global__ void k_mlp_grad(const float* __restrict__ X, int n, const float* __restrict__ Z1,
                           const float* __restrict__ dz, const __half* __restrict__ w2h, float* __restrict__ g) {
  const int total = kParams;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
    float acc = 0.f;
    if (p < kHidden * kPatchSize) {
      const int j = p / kPatchSize, e = p - j * kPatchSize;
      const float w2j = __half2float(w2h[j]);
      for (int s = 0; s < n; ++s) {
        const float zz = Z1[(long long)s * kHidden + j];
        if (zz > 0.f) acc = fmaf(dz[s] * w2j, X[(long long)s * kPatchSize + e], acc);
      }
    } else if (p < kHidden * kPatchSize + kHidden) {
      const int j = p - kHidden * kPatchSize;
      const float w2j = __half2float(w2h[j]);
      for (int s = 0; s < n; ++s)
        if (Z1[(long long)s * kHidden + j] > 0.f) acc += dz[s] * w2j;
    } else if (p < kHidden * kPatchSize + 2 * kHidden) {
      const int j = p - kHidden * kPatchSize - kHidden;
      for (int s = 0; s < n; ++s) acc = fmaf(dz[s], fmaxf(Z1[(long long)s * kHidden + j], 0.f), acc);
    } else {
      for (int s = 0; s < n; ++s) acc += dz[s];
    }
    g[p] = acc;
  }
}

// Adam (Kingma & Ba 2015) on FP32 master weights; FP16 copies of W1 and w2
// for the next forward pass.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, AdamArgs a, __half* __restrict__ W1h, __half* __restrict__ w2h) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kParams; p += gridDim.x * blockDim.x) {
    const float gg = g[p];
    const float mm = a.b1 * m1[p] + (1.f - a.b1) * gg;
    const float vv = a.b2 * m2[p] + (1.f - a.b2) * gg * gg;
    m1[p] = mm;
    m2[p] = vv;
    const float wn = w[p] - a.lr * (mm * a.c1) / (sqrtf(vv * a.c2) + a.eps);
    w[p] = wn;
    if (p < kHidden * kPatchSize) W1h[p] = __float2half_rn(wn);
    else if (p >= kHidden * kPatchSize + kHidden && p < kHidden * kPatchSize + 2 * kHidden)
      w2h[p - kHidden * kPatchSize - kHidden] = __float2half_rn(wn);
  }
}

__global__ void k_weights_to_half(const float* __restrict__ w, __half* __restrict__ W1h, __half* __restrict__ w2h) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kHidden * kPatchSize + 2 * kHidden; p += gridDim.x * blockDim.x) {
    if (p < kHidden * kPatchSize) W1h[p] = __float2half_rn(w[p]);
    else if (p >= kHidden * kPatchSize + kHidden) w2h[p - kHidden * kPatchSize - kHidden] = __float2half_rn(w[p]);
  }
}

// Gather rows idx[0..n) of X / y into a contiguous minibatch.
__global__ void k_gather_batch(const float* __restrict__ X, const float* __restrict__ y, const int* __restrict__ idx,
                               int n, float* __restrict__ Xb, float* __restrict__ yb) {
  const long long total = (long long)n * kPatchSize;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(f / kPatchSize);
    const int e = (int)(f - (long long)s * kPatchSize);
    Xb[f] = X[(long long)idx[s] * kPatchSize + e];
    if (e == 0) yb[s] = y[idx[s]];
  }
}

// ---------------------------------------------------------------------------
// Refinement: direct sums at a few bins of one template, accumulated over
// segments.  One CTA per work item (template, bin group, segment chunk); per
// segment, each lane walks a run of consecutive samples and steps the same
// 64-bit fixed-point phase as the spreader (a LaneMap seeded from the warp's
// FP64 anchor), adding x_j exp(-2 pi i (f_c + k/t_coh) delta_j) for each bin
// of the group: the demodulation phase k_c Psi (or its own map when k_c is
// not whole) plus k Psi, both mod 1 cycle; (P - 2) / 2 is summed over the
// chunk's segments.
// ---------------------------------------------------------------------------
template <bool INT_KC>
__global__ void __launch_bounds__(256)
k_sparse_bins(const float* __restrict__ strain, const SparseItem* __restrict__ items, int n_items,
              const double* __restrict__ betas, const int* __restrict__ bins, SparseArgs a,
              float* __restrict__ partial) {
  __shared__ Anchor anc[kSparseChunk][kSpreadWarps];   // every anchor of the item, computed up front
  __shared__ float red[kSparseMaxBins][2][kSpreadWarps];
  __shared__ float sZ[kSparseMaxBins];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int q = blockIdx.x; q < n_items; q += gridDim.x) {
    const SparseItem it = items[q];
    const int nb = it.nb;
    int kk[kSparseMaxBins];
#pragma unroll
    for (int u = 0; u < kSparseMaxBins; ++u) kk[u] = u < nb ? bins[it.b0 + u] - a.half_bins : 0;
    bool adjacent = false;                  // the group holds two neighbouring bins (uniform over the block)
#pragma unroll
    for (int u = 1; u < kSparseMaxBins; ++u) adjacent = adjacent || (u < nb && kk[u] == kk[u - 1] + 1);
    __syncthreads();   // the previous item is done with anc and sZ
    {
      const double b = betas[it.m];
      const int na = (it.i1 - it.i0) * a.aa.n_anchor;
      for (int t = tid; t < na; t += blockDim.x)
        anc[t / a.aa.n_anchor][t % a.aa.n_anchor] = compute_anchor(b, it.i0 + t / a.aa.n_anchor, t % a.aa.n_anchor, a.aa);
    }
    if (tid < kSparseMaxBins) sZ[tid] = 0.f;
    for (int i = it.i0; i < it.i1; ++i) {
      __syncthreads();   // anchors ready; red free again
      float re[kSparseMaxBins], im[kSparseMaxBins];
#pragma unroll
      for (int u = 0; u < kSparseMaxBins; ++u) { re[u] = 0.f; im[u] = 0.f; }
      const float* x = strain + (long long)i * a.n_s;
      // warp w walks anchor span w; lane l its run of consecutive samples
      const int j_lo = warp * a.span;
      const int j_hi = min(j_lo + a.span, a.n_s);
      const int j0 = j_lo + lane * a.run, j1 = min(j0 + a.run, j_hi);
      if (j0 < j1) {
        const Anchor A = anc[i - it.i0][warp];
        LaneMap m = lane_map(A, anchor_psi0(A), A.n1, A.p1lo, A.q2, 1.0f, j0 - j_lo);
        LaneMap mt;
        if (!INT_KC) mt = lane_map(A, anchor_th0(A), A.m1, A.m1lo, A.kq2, a.kc, j0 - j_lo);
        const uint32_t kc = (uint32_t)a.kc_int;
        for (int j = j0; j < j1; ++j) {
          const uint32_t ph = (uint32_t)(m.v >> 32), pl = (uint32_t)m.v;
          // f_b delta = f_c delta + k delta / t_coh: the k-term is k Psi (mod 1)
          const uint32_t T0 = INT_KC ? ph * kc + __umulhi(pl, kc) : (uint32_t)(mt.v >> 32);
          const uint32_t Psi = ph + (pl >> 31);            // rounded to 2^-32 periods
          const float xv = x[j];
          // the phasor of a bin next to the previous one is the previous one
          // turned by exp(-2 pi i Psi)
          float s1 = 0.f, c1 = 1.f;
          if (adjacent) __sincosf((float)(int32_t)Psi * 1.4629180792671596e-09f, &s1, &c1);  // 2 pi / 2^32
          float sn = 0.f, cs = 1.f;
#pragma unroll
          for (int u = 0; u < kSparseMaxBins; ++u) {
            if (u < nb) {
              if (u > 0 && kk[u] == kk[u - 1] + 1) {
                const float c = cs * c1 - sn * s1;
                sn = fmaf(sn, c1, cs * s1);
                cs = c;
              } else {
                const uint32_t Tb = T0 + (uint32_t)kk[u] * Psi;
                __sincosf((float)(int32_t)Tb * 1.4629180792671596e-09f, &sn, &cs);  // 2 pi / 2^32
              }
              re[u] = fmaf(xv, cs, re[u]);
              im[u] = fmaf(-xv, sn, im[u]);
            }
          }
          m.step();
          if (!INT_KC) mt.step();
        }
      }
#pragma unroll
      for (int u = 0; u < kSparseMaxBins; ++u) {
        if (u < nb) {   // uniform across the block
          float r = re[u], m_ = im[u];
          for (int o = 16; o > 0; o >>= 1) {
            r += __shfl_down_sync(0xffffffffu, r, o);
            m_ += __shfl_down_sync(0xffffffffu, m_, o);
          }
          if (lane == 0) { red[u][0][warp] = r; red[u][1][warp] = m_; }
        }
      }
      __syncthreads();
      if (tid < nb) {
        float r = 0.f, m_ = 0.f;
        for (int w = 0; w < kSpreadWarps; ++w) { r += red[tid][0][w]; m_ += red[tid][1][w]; }
        sZ[tid] += fmaf(r, r, m_ * m_) * a.inv_ns - 1.0f;   // (P - 2) / 2
      }
    }
    __syncthreads();
    if (tid < kSparseMaxBins) partial[(long long)q * kSparseMaxBins + tid] = sZ[tid];
  }
}

// n_sigma of each evaluated cell: cell c sums the partials of its items
// [cell_item0[c], cell_item0[c] + cell_nitems[c]) at slot cell_slot[c].
__global__ void k_sparse_reduce(const float* __restrict__ partial, const int* __restrict__ cell_item0,
                                const int* __restrict__ cell_nitems, const int* __restrict__ cell_slot,
                                const int* __restrict__ cell_nseg, int n_cells, float* __restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x) {
    double z = 0.0;
    const int q0 = cell_item0[c], nq = cell_nitems[c], u = cell_slot[c];
    for (int q = q0; q < q0 + nq; ++q) z += (double)partial[(long long)q * kSparseMaxBins + u];
    out[c] = (float)(z / sqrt((double)cell_nseg[c]));
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_make_strain(float* out, long long n, double fs, unsigned long long seed, int noise,
                               const InjectionDev* inj, int n_inj, int n_sm, cudaStream_t st) {
  long long quads = (n + 3) / 4;
  long long blocks = (quads + 255) / 256;
  if (blocks > (long long)n_sm * 16) blocks = (long long)n_sm * 16;
  k_make_strain<<<(unsigned)blocks, 256, (size_t)n_inj * sizeof(InjectionDev), st>>>(out, n, fs, seed, noise, inj, n_inj);
  return cudaGetLastError();
}

cudaError_t launch_patches(const float* map, int n_templates, int n_bins, const int* cm, const int* cb, int n,
                           float* out, int n_sm, cudaStream_t st) {
  long long total = (long long)n * kPatchSize;
  long long blocks = (total + 255) / 256;
  if (blocks > (long long)n_sm * 32) blocks = (long long)n_sm * 32;
  if (blocks < 1) blocks = 1;
  k_patches<<<(unsigned)blocks, 256, 0, st>>>(map, n_templates, n_bins, cm, cb, n, out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* X, int n, const __half* W1h, const float* b1, const __half* w2h,
                               const float* b2, float* logits, float* Z1, int n_sm, cudaStream_t st) {
  long long blocks = ((long long)n + 3) / 4;
  if (blocks > (long long)n_sm * 16) blocks = (long long)n_sm * 16;
  if (blocks < 1) blocks = 1;
  k_mlp_forward<<<(unsigned)blocks, 256, 0, st>>>(X, n, W1h, b1, w2h, b2, logits, Z1);
  return cudaGetLastError();
}

cudaError_t launch_bce(const float* logits, const float* y, int n, float* dz, float* loss_terms, cudaStream_t st) {
  k_bce<<<(n + 255) / 256, 256, 0, st>>>(logits, y, n, dz, loss_terms);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float* X, int n, const float* Z1, const float* dz, const __half* w2h, float* g,
                            cudaStream_t st) {
  k_mlp_grad<<<(kParams + 127) / 128, 128, 0, st>>>(X, n, Z1, dz, w2h, g);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* w, const float* g, float* m1, float* m2, const AdamArgs& a, __half* W1h, __half* w2h,
                        cudaStream_t st) {
  k_adam<<<(kParams + 255) / 256, 256, 0, st>>>(w, g, m1, m2, a, W1h, w2h);
  return cudaGetLastError();
}

cudaError_t launch_weights_to_half(const float* w, __half* W1h, __half* w2h, cudaStream_t st) {
  k_weights_to_half<<<(kParams + 255) / 256, 256, 0, st>>>(w, W1h, w2h);
  return cudaGetLastError();
}

cudaError_t launch_gather_batch(const float* X, const float* y, const int* idx, int n, float* Xb, float* yb,
                                int n_sm, cudaStream_t st) {
  long long total = (long long)n * kPatchSize;
  long long blocks = (total + 255) / 256;
  if (blocks > (long long)n_sm * 16) blocks = (long long)n_sm * 16;
  if (blocks < 1) blocks = 1;
  k_gather_batch<<<(unsigned)blocks, 256, 0, st>>>(X, y, idx, n, Xb, yb);
  return cudaGetLastError();
}

cudaError_t launch_sparse_bins(const float* strain, const SparseItem* items, int n_items, const double* betas,
                               const int* bins, const SparseArgs& a, float* partial, int n_sm, cudaStream_t st) {
  long long blocks = n_items;
  if (blocks > (long long)n_sm * 8) blocks = (long long)n_sm * 8;
  if (blocks < 1) blocks = 1;
  if (a.kc_int)
    k_sparse_bins<true><<<(unsigned)blocks, 256, 0, st>>>(strain, items, n_items, betas, bins, a, partial);
  else
    k_sparse_bins<false><<<(unsigned)blocks, 256, 0, st>>>(strain, items, n_items, betas, bins, a, partial);
  return cudaGetLastError();
}

cudaError_t launch_sparse_reduce(const float* partial, const int* cell_item0, const int* cell_nitems,
                                 const int* cell_slot, const int* cell_nseg, int n_cells, float* out, cudaStream_t st) {
  k_sparse_reduce<<<(n_cells + 255) / 256, 256, 0, st>>>(partial, cell_item0, cell_nitems, cell_slot, cell_nseg,
                                                         n_cells, out);
  return cudaGetLastError();
}

}  // namespace srs
