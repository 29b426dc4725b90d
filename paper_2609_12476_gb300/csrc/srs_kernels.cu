// srs_kernels.cu -- sm_103a kernels of the semicoherent NUFFT resampling search.
//
// Sec. III.B of arXiv:2609.12476: each coherent segment is resampled with the
// 0PN time tau(t; beta) of Eq. (new_t) and its spectrum is taken with a type-1
// NUFFT (spread onto an oversampled grid with an exponential-of-semicircle
// kernel, FFT, divide by the kernel's transform).  Sec. III.C: powers
// (Eq. normalized_power), equal-weight sum over segments into n_sigma
// (Eqs. weights, semicoherent_statistic), then top-k.
//
// Two forms:
//   mixed  -- k_mixed: a persistent kernel over (template, segment-chunk)
//             items with FP64 anchors of the time map (a few per segment),
//             FP32 spreading, shared-memory FFT and FP32 power/sum;
//             the reduction over items and the top-k are in srs_reduce.cu;
//   plain  -- k_plain: one CTA per spectrum, every step in FP64.
// k_anchors and k_time_map_* expose the time map itself.
#include <cuda_runtime.h>
#include <cstdint>

#include "srs_internal.h"
#include "srs_kernels.h"
#include "srs_device.cuh"

namespace srs {

// ---------------------------------------------------------------------------
// small complex helpers
// ---------------------------------------------------------------------------
template <typename R> struct cplx;
template <> struct cplx<float> { using T = float2; };
template <> struct cplx<double> { using T = double2; };

template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) { C c; c.x = a; c.y = b; return c; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
// i * a
template <typename C> __device__ __forceinline__ C cmuli(C a) { return cmk<C>(-a.y, a.x); }

// ---------------------------------------------------------------------------
// R-point forward DFTs, y_k = sum_r v_r exp(-2 pi i r k / R)
// ---------------------------------------------------------------------------
template <typename C, int R> struct Dft;
template <typename C> struct Dft<C, 2> {
  static __device__ __forceinline__ void run(C* v) { C a = v[0], b = v[1]; v[0] = cadd(a, b); v[1] = csub(a, b); }
};
template <typename C> struct Dft<C, 3> {
  static __device__ __forceinline__ void run(C* v) {
    using R_ = decltype(C::x);
    const R_ c = R_(-0.5), s = R_(-0.86602540378443864676);   // cos, sin of -2pi/3... sin(-2pi/3)
    C t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    C m = cadd(v[0], cscale(t1, c));
    C is = cmuli(cscale(t2, s));
    v[0] = cadd(v[0], t1);
    v[1] = cadd(m, is);
    v[2] = csub(m, is);
  }
};
template <typename C> struct Dft<C, 4> {
  static __device__ __forceinline__ void run(C* v) {
    C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    C c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    C id = cmuli(d);
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = csub(b, id);   // b - i d
    v[3] = cadd(b, id);   // b + i d
  }
};
template <typename C> struct Dft<C, 5> {
  static __device__ __forceinline__ void run(C* v) {
    using R_ = decltype(C::x);
    // cos(2pi/5), cos(4pi/5), -sin(2pi/5), -sin(4pi/5)
    const R_ c1 = R_(0.30901699437494742410), c2 = R_(-0.80901699437494742410);
    const R_ s1 = R_(-0.95105651629515357212), s2 = R_(-0.58778525229247312917);
    C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    C t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    C a1 = cadd(v[0], cadd(cscale(t1, c1), cscale(t2, c2)));
    C a2 = cadd(v[0], cadd(cscale(t1, c2), cscale(t2, c1)));
    C b1 = cmuli(cadd(cscale(t3, s1), cscale(t4, s2)));
    C b2 = cmuli(csub(cscale(t3, s2), cscale(t4, s1)));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
  }
};

// Composite radices by the prime-factor (Good-Thomas) map, N = N1 N2 with
// gcd(N1, N2) = 1: x[(N2 n1 + N1 n2) mod N] forms an N1 x N2 array; DFT-N1
// down its columns, then DFT-N2 along its rows, gives X[k] at
// k = (N2 (N2^-1 mod N1) k1 + N1 (N1^-1 mod N2) k2) mod N.  The index maps
// are compile-time register renamings: no twiddle factors between the two.
template <typename C, int N1, int N2, int A1, int A2>
__device__ __forceinline__ void dft_pfa(C* v) {
  constexpr int N = N1 * N2;
  C a[N1][N2];
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1)
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) a[n1][n2] = v[(N2 * n1 + N1 * n2) % N];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) {
    C t[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) t[n1] = a[n1][n2];
    Dft<C, N1>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) a[k1][n2] = t[k1];
  }
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    Dft<C, N2>::run(a[k1]);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) v[(A1 * k1 + A2 * k2) % N] = a[k1][k2];
  }
}
// 12 = 4 x 3: 3^-1 mod 4 = 3, 4^-1 mod 3 = 1, so k = (9 k1 + 4 k2) mod 12.
template <typename C> struct Dft<C, 12> {
  static __device__ __forceinline__ void run(C* v) { dft_pfa<C, 4, 3, 9, 4>(v); }
};
// 10 = 5 x 2: 2^-1 mod 5 = 3, 5^-1 mod 2 = 1, so k = (6 k1 + 5 k2) mod 10.
template <typename C> struct Dft<C, 10> {
  static __device__ __forceinline__ void run(C* v) { dft_pfa<C, 5, 2, 6, 5>(v); }
};

// One Stockham autosort pass of radix R over n points (Ns = product of the
// radices already applied).  Butterfly j reads in[j + r n/R], multiplies by
// the twiddles exp(-2 pi i (j mod Ns) r / (Ns R)), transforms, and writes
// out[(j - j mod Ns) R + j mod Ns + r Ns].
template <typename C, int R>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ in, C* __restrict__ out, int n, int Ns,
                                              const C* __restrict__ tw) {
  const int nR = n / R;
  const int step = n / (Ns * R);
  for (int j = threadIdx.x; j < nR; j += blockDim.x) {
    const int jm = j % Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[j + r * nR];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[jm * r * step]);
    }
    Dft<C, R>::run(v);
    const int idxD = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) out[idxD + r * Ns] = v[r];
  }
}

// One in-place decimation-in-frequency pass of radix R over sub-transforms of
// length M (Gentleman-Sande): butterfly (block c, k < L = M / R) takes
// x[cM + k + sL] for s < R, forms y_r = sum_s x_s exp(-2 pi i rs / R) and
// writes y_r exp(-2 pi i rk / M) back to x[cM + k + rL].  Every butterfly
// reads and writes its own R elements, so the pass needs no second buffer.
template <typename C, int R, int M, int N>
__device__ __forceinline__ void dif_pass(C* a, const C* __restrict__ tw) {
  constexpr int L = M / R;
  for (int j = threadIdx.x; j < N / R; j += blockDim.x) {
    const int c = j / L, k = j - c * L;
    const int base = c * M + k;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = a[base + r * L];
    Dft<C, R>::run(v);
    a[base] = v[0];
#pragma unroll
    for (int r = 1; r < R; ++r) a[base + r * L] = L > 1 ? cmul(v[r], tw[r * k * (N / M)]) : v[r];
  }
  __syncthreads();
}

// n = 1200 in place: DIF passes of radix 10, 10, 12 (each a prime-factor
// DFT in registers; three passes and two twiddle stages instead of five and
// four with radices 4, 4, 3, 5, 5).  Frequency f ends at position
// dif_1200_pos(f): with f = r1 + 10 (r2 + 10 r3), the position is
// r1 120 + r2 12 + r3.
template <typename C>
__device__ __forceinline__ void fft_1200_dif(C* a, const C* __restrict__ tw) {
  dif_pass<C, 10, 1200, 1200>(a, tw);
  dif_pass<C, 10, 120, 1200>(a, tw);
  dif_pass<C, 12, 12, 1200>(a, tw);
}
__device__ __forceinline__ int dif_1200_pos(int f) {
  const int f1 = f / 10, r1 = f - 10 * f1;
  const int r3 = f1 / 10, r2 = f1 - 10 * r3;
  return r1 * 120 + r2 * 12 + r3;
}

// Forward FFT of a[0..n) in shared memory, ping-ponging with b.  Returns the
// buffer that holds the result.  Every thread of the block must call it.
template <typename C>
__device__ C* fft_smem(C* a, C* b, int n, const int8_t* radices, int n_pass, const C* __restrict__ tw) {
  int Ns = 1;
  for (int p = 0; p < n_pass; ++p) {
    const int R = radices[p];
    switch (R) {
      case 2: stockham_pass<C, 2>(a, b, n, Ns, tw); break;
      case 3: stockham_pass<C, 3>(a, b, n, Ns, tw); break;
      case 4: stockham_pass<C, 4>(a, b, n, Ns, tw); break;
      default: stockham_pass<C, 5>(a, b, n, Ns, tw); break;
    }
    __syncthreads();
    C* t = a; a = b; b = t;
    Ns *= R;
  }
  return a;
}

// ---------------------------------------------------------------------------
// PTX helpers (documented single instructions)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------
// K1: FP64 anchors of the resampled time (Eq. new_t), one thread per
// (segment, anchor).  Segment g belongs to the item with the largest g0 <= g.
// ---------------------------------------------------------------------------
__global__ void k_anchors(const Item* __restrict__ items, int n_items, const double* __restrict__ betas,
                          AnchorArgs aa, Anchor* __restrict__ out, long long total) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long g = idx / aa.n_anchor;
    const int ai = (int)(idx - g * aa.n_anchor);
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {  // largest q with items[q].g0 <= g
      int mid = (lo + hi + 1) >> 1;
      if (items[mid].g0 <= g) lo = mid; else hi = mid - 1;
    }
    const Item it = items[lo];
    out[idx] = compute_anchor(betas[it.m], it.i0 + (int)(g - it.g0), ai, aa);
  }
}

// ---------------------------------------------------------------------------
// Mixed form: persistent spread + FFT + deconvolution + power/segment sum.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One TMA bulk copy global -> shared completing on `bar` (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(d), "l"(src), "r"(bytes), "r"(b) : "memory");
}
// Wait for phase `parity` of `bar`, giving up after ~2^31 cycles (about a second).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(b), "r"(parity) : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

// Self-test of the bounded staging wait: one thread arms an mbarrier for a
// 16-byte transfer that is never issued and waits on it exactly as k_mixed
// does; the wait gives up after its cycle limit and the error flag records
// it.  Nothing faults and nothing hangs.
__global__ void k_wait_selftest(int* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               ::"r"((uint32_t)__cvta_generic_to_shared(&bar)), "r"(16u) : "memory");
  if (!mbar_wait(&bar, 0u) && atomicExch(err, 1) == 0) {
    err[1] = -1;
    err[2] = -1;
    err[3] = 0;
    err[4] = (int)blockIdx.x;
  }
}

// Spread the samples [j_begin, j_end) of one lane into `grid`.
//
// Time map.  The lane's phases come from a LaneMap seeded at its first sample
// (64-bit fixed point, integer steps): Psi' = Psi - W/(2n) - base/n periods,
// where base is the lane's base cell (one cell before its first sample's
// first tap), so that s = Psi' n is the position of the first tap relative
// to base and never wraps within the lane's run.  A sample is keyed by
// floor(s): its taps go to cells floor(s) + 1 ... floor(s) + W.  (At an
// exact integer s, W + 1 cells are in reach and both end cells carry the
// kernel's edge value 2^-E; the walk takes the last W.)  The demodulation phase is
// k_c Psi mod 1 from the same Psi when k_c is a whole number, else a second
// LaneMap.
//
// Taps.  The ES kernel is phi(z) = 2^(E sqrt(1 - z^2)) 2^-E with E = beta
// log2 e; the constant 2^-E is left to the deconvolution factors.  With
// Z = E z, E sqrt(1 - z^2) = sqrt(E^2 - Z^2), and tap t of a sample sits at
// Z = Z0 + t H (H = 2E/W); taps are evaluated in pairs on the packed FP32x2
// pipe.  The first pair sits at (Z0, Z0 + H) and each further pair is one
// packed add of 2H on, so every operand is an ordinary register: packed
// multiply-adds by the tap numbers (Z = (t, t + 1) H + Z0) left the compiler
// moving those constants out of uniform registers for every sample.
//
// Cell walk.  The lane keeps the W cells [Bm + 1, Bm + 1 + W) of its kernel
// footprint in registers.  The warp walks cell by cell: each lane adds all
// of its samples keyed Bm, then every lane flushes cell Bm + 1
// with a shared-memory atomic and moves its window one cell on, so the step
// is warp-uniform.  The window is a ring: the walk is unrolled W times so
// that, at step R of the unrolled loop, cell Bm + 1 + t lives in register
// acc[(t + R) % W] and moving on renames registers instead of copying them.
// The per-sample step has no branch: the next sample's load index is clamped
// to the run, and a step past the run's end computes inputs nobody reads.
//
// The walk ends when every lane has used its run.  That needs a time map that
// never steps back a cell, which the planner's range guarantees; as a guard
// against anything else spread_run also stops the walk once no live lane is
// below cell n + W + 2 (a lane's run spans about n / threads + W cells),
// checked once per turn of the ring so the check stays off the per-cell path,
// and reports the lanes left with samples.
template <int W, bool INT_KC>
struct CellWalk {
  float2 acc[W];
  int l0;
  float z0, cre, cim;
  LaneMap m;
  LaneMap mt;
  uint32_t thofs, kc, n;
  int base, j, j_end, Bm;
  float x_next, H, eh32, E, EH1, H2, mE2;
  bool live;
  unsigned mask;
  const float* __restrict__ xs;
  float2* __restrict__ grid;

  __device__ __forceinline__ void inputs(float x) {
    const uint32_t ph = (uint32_t)(m.v >> 32), pl = (uint32_t)m.v;
    uint32_t th;
    if (INT_KC) {
      th = ph * kc + __umulhi(pl, kc) + thofs;
    } else {
      th = (uint32_t)(mt.v >> 32);
      mt.step();
    }
    float sn, cs;
    __sincosf((float)(int32_t)th * 1.4629180792671596e-09f, &sn, &cs);
    const unsigned long long sp = (unsigned long long)ph * n + __umulhi(pl, n);
    const uint32_t sl = (uint32_t)sp;
    l0 = (int)(sp >> 32);
    z0 = fmaf(-eh32, (float)sl, EH1);
    cre = x * cs;
    cim = -x * sn;
    m.step();
  }

  __device__ __forceinline__ void next() {
    ++j;
    live = j < j_end;
    const float x = x_next;
    x_next = xs[min(j + 1, j_end - 1)];
    inputs(x);
  }

  __device__ __forceinline__ void flush_cell(int c_rel, float2 v) {
    int c = base + c_rel;
    while (c >= (int)n) c -= n;
    atomicAdd(&grid[c].x, v.x);
    atomicAdd(&grid[c].y, v.y);
  }

  template <int R>
  __device__ __forceinline__ bool cell() {
    if (!__any_sync(mask, live)) return false;
    const float2 H2H2 = make_float2(H2, H2), mEE = make_float2(mE2, mE2);
    while (live && l0 == Bm) {
      const float2 cv = make_float2(cre, cim);
      float2 Z = make_float2(z0, z0 + H);   // taps 0 and 1; each further pair 2H on
#pragma unroll
      for (int t = 0; t + 1 < W; t += 2) {
        if (t > 0) Z = __fadd2_rn(Z, H2H2);
        const float2 q = __ffma2_rn(Z, Z, mEE);
        const float p0 = ex2_approx(sqrt_approx(fabsf(q.x)));
        const float p1 = ex2_approx(sqrt_approx(fabsf(q.y)));
        acc[(t + R) % W] = __ffma2_rn(make_float2(p0, p0), cv, acc[(t + R) % W]);
        acc[(t + 1 + R) % W] = __ffma2_rn(make_float2(p1, p1), cv, acc[(t + 1 + R) % W]);
      }
      if (W & 1) {
        const float Zl = W == 1 ? z0 : Z.x + H2;
        const float pl = ex2_approx(sqrt_approx(fabsf(fmaf(Zl, Zl, mE2))));
        acc[(W - 1 + R) % W] = __ffma2_rn(make_float2(pl, pl), cv, acc[(W - 1 + R) % W]);
      }
      next();
    }
    flush_cell(Bm, acc[R % W]);
    acc[R % W] = make_float2(0.f, 0.f);
    ++Bm;
    return true;
  }

  template <int R>
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int t = 0; t < W - 1; ++t) {
      const float2 v = acc[(t + R) % W];
      if (v.x != 0.f || v.y != 0.f) flush_cell(Bm + t, v);
    }
  }

  template <int R>
  __device__ __forceinline__ bool turn() {
    if constexpr (R == W) {
      return true;
    } else {
      if (!cell<R>()) {
        flush<R>();
        return false;
      }
      return turn<R + 1>();
    }
  }
};

// Returns false when the walk stopped at its cell bound with samples unused.
template <int W, bool INT_KC>
__device__ __forceinline__ bool spread_run(const float* __restrict__ xs, float2* __restrict__ grid,
                                           const Anchor& A, int j_begin, int j_end, int l_base,
                                           const MixedArgs& a) {
  CellWalk<W, INT_KC> w;
#pragma unroll
  for (int c = 0; c < W; ++c) w.acc[c] = make_float2(0.f, 0.f);
  const float E = a.es_beta_log2e;
  w.E = E;
  w.H = E * a.two_over_w;
  w.eh32 = w.H * 2.3283064365386963e-10f;
  w.EH1 = w.H - E;
  w.H2 = 2.f * w.H;
  w.mE2 = -E * E;
  w.n = (uint32_t)a.n_fine;
  w.kc = (uint32_t)a.kc_int;
  w.mask = __activemask();
  w.xs = xs;
  w.grid = grid;
  w.j = j_begin;
  w.j_end = j_end;
  w.live = j_begin < j_end;
  w.Bm = 0;
  if (w.live) {
    const int l = j_begin - l_base;
    // Psi - W/(2n) at the first sample, and the lane's base cell
    w.m = lane_map(A, anchor_psi0(A), A.n1, A.p1lo, A.q2, 1.0f, l);
    w.m.v -= a.wofs;
    const uint32_t ph = (uint32_t)(w.m.v >> 32), pl = (uint32_t)w.m.v;
    const unsigned long long sp = (unsigned long long)ph * w.n + __umulhi(pl, w.n);
    int base = (int)(sp >> 32) - 1;
    if (base < 0) base += (int)w.n;
    w.base = base;
    const unsigned long long off = (unsigned long long)base * a.inv_n64;   // base / n periods
    w.m.v -= off;
    const unsigned long long o = a.wofs + off;
    w.thofs = (uint32_t)(o >> 32) * w.kc + __umulhi((uint32_t)o, w.kc);  // k_c (W/(2n) + base/n) mod 1
    w.base = base + 1;   // flushes address cell base + 1 + c_rel: a sample keyed l0 has its first tap at l0 + 1
    if (!INT_KC) w.mt = lane_map(A, anchor_th0(A), A.m1, A.m1lo, A.kq2, a.kc, l);
    const float x0 = xs[j_begin];
    w.x_next = j_begin + 1 < j_end ? xs[j_begin + 1] : 0.f;
    w.inputs(x0);
    w.Bm = w.l0;
  }
  // each turn walks W cells; the bound is checked once per turn, and leaving
  // there flushes the window as the walk's own end (cell<0> finding no live
  // lane) would
  while (w.template turn<0>()) {
    if (!__any_sync(w.mask, w.live && w.Bm < a.n_fine + W + 2)) {
      w.template flush<0>();
      break;
    }
  }
  return !w.live;
}

// Persistent CTAs take (template, segment-chunk) items from `queue` (in the
// order `a.order` gives, if any).  Per item: FP64 anchors of all its
// segments; per segment: samples staged in shared memory by a TMA bulk copy
// (the next segment's copy overlaps this segment's FFT) or read from global
// memory (GLOBAL_X), spread, FFT, deconvolve, then either write F (SPECTRA)
// or add (P - 2) / 2 into the item's running sum Z.
template <int W, bool SPECTRA, bool INT_KC, bool GLOBAL_X>
__global__ void __launch_bounds__(kSpreadThreads, 4)
k_mixed(const float* __restrict__ strain, const Item* __restrict__ items, int n_items,
        const double* __restrict__ betas, int* __restrict__ queue, MixedArgs a,
        float* __restrict__ partial, double2* __restrict__ Fout, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  // GLOBAL_X: samples are read straight from the (L2-resident) strain;
  // otherwise a TMA bulk copy stages each segment in shared memory
  float* xs = reinterpret_cast<float*>(smem);                       // [ns4] unless GLOBAL_X
  float2* g0 = reinterpret_cast<float2*>(xs + (GLOBAL_X ? 0 : a.ns4));  // [n_fine]
  // the generic FFT ping-pongs with a second buffer; the 1200-point one runs in place
  float2* g1 = g0 + a.n_fine;                                       // [n_fine] unless 1200
  float* Z = reinterpret_cast<float*>(a.fft_fixed == 1200 ? g1 : g1 + a.n_fine);   // [nb4]
  Anchor* anc = reinterpret_cast<Anchor*>(Z + a.nb4);               // [chunk * n_anchor]
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_item, s_abort;
  __shared__ int8_t s_rad[16];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < 16) s_rad[tid] = a.radices[tid];
  if (tid == 0) { mbar_init(&s_bar); s_abort = 0; }
  __syncthreads();
  const float2* __restrict__ tw = reinterpret_cast<const float2*>(a.tw);
  const uint32_t seg_bytes = (uint32_t)a.n_s * 4u;
  uint32_t parity = 0;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int q = s_item;
    if (q >= n_items) break;
    const int qi = a.order ? a.order[q] : q;   // the item this queue position runs
    const Item it = items[qi];
    if (!GLOBAL_X && tid == 0) bulk_load(xs, strain + (long long)it.i0 * a.n_s, seg_bytes, &s_bar);
    {
      const int na = (it.i1 - it.i0) * a.n_anchor;
      const double b = betas[it.m];
      for (int t = tid; t < na; t += blockDim.x)
        anc[t] = compute_anchor(b, it.i0 + t / a.n_anchor, t % a.n_anchor, a.aa);
    }
    if (!SPECTRA)
      for (int b = tid; b < a.n_bins; b += blockDim.x) Z[b] = 0.f;
    for (int i = it.i0; i < it.i1; ++i) {
      for (int j = tid; j < a.n_fine; j += blockDim.x) g0[j] = make_float2(0.f, 0.f);
      if (!GLOBAL_X) {
        if (tid == 0 && !mbar_wait(&s_bar, parity)) {
          // record where the wait gave up: flag, item, segment, parity, block
          s_abort = 1;
          if (atomicCAS(err, 0, 1) == 0) { err[1] = q; err[2] = i; err[3] = (int)parity; err[4] = blockIdx.x; }
        }
        parity ^= 1u;
      }
      __syncthreads();
      if (s_abort) {
        // give the copy in flight one more bounded wait before leaving
        if (tid == 0) mbar_wait(&s_bar, parity ^ 1u);
        __syncthreads();
        return;
      }
      {
        const int j0 = (warp * 32 + lane) * a.run;
        const int j1 = min(j0 + a.run, a.n_s);
        const float* xsrc = GLOBAL_X ? strain + (long long)i * a.n_s : xs;
        // the anchor of this lane's span (one per warp, or per half-warp)
        const int ai = j0 / a.span;
        if (j0 < a.n_s && !spread_run<W, INT_KC>(xsrc, g0, anc[(i - it.i0) * a.n_anchor + ai], j0, j1, ai * a.span, a)
            && atomicCAS(err, 0, 2) == 0) {
          // the cell walk hit its bound: flag 2, item, segment, first sample of the lane, block
          err[1] = q; err[2] = i; err[3] = j0; err[4] = blockIdx.x;
        }
      }
      __syncthreads();
      if (!GLOBAL_X && tid == 0 && i + 1 < it.i1) bulk_load(xs, strain + (long long)(i + 1) * a.n_s, seg_bytes, &s_bar);
      if (SPECTRA && a.grid_out) {
        // the spread grid alone, for an FFT outside this kernel
        float2* go = a.grid_out + ((long long)it.m * a.seg_range + (i - a.seg_begin)) * a.n_fine;
        for (int j = tid; j < a.n_fine; j += blockDim.x) go[j] = g0[j];
        __syncthreads();
        continue;
      }
      const bool dif = a.fft_fixed == 1200;
      float2* res = g0;
      if (dif) fft_1200_dif<float2>(g0, tw);
      else res = fft_smem<float2>(g0, g1, a.n_fine, s_rad, a.n_pass, tw);
      for (int b = tid; b < a.n_bins; b += blockDim.x) {
        int k = b - a.half_bins;
        int idx = k < 0 ? k + a.n_fine : k;
        if (dif) idx = dif_1200_pos(idx);
        const float2 G = res[idx];
        const float c = a.corr[b];
        const float fx = G.x * c, fy = G.y * c;
        if (SPECTRA) {
          if (a.cube_out)
            a.cube_out[((long long)it.m * a.n_bins + b) * a.seg_range + (i - a.seg_begin)] =
                2.0f * fmaf(fx, fx, fy * fy) * a.inv_ns;
          else
            Fout[((long long)it.m * a.seg_range + (i - a.seg_begin)) * a.n_bins + b] = make_double2(fx, fy);
        } else {
          // (P - 2) / 2 with P = 2 |F|^2 / n_s (mu = sigma = 2)
          Z[b] += fmaf(fx, fx, fy * fy) * a.inv_ns - 1.0f;
        }
      }
      __syncthreads();
    }
    if (!SPECTRA)
      for (int b = tid; b < a.n_bins; b += blockDim.x) partial[(long long)qi * a.n_bins + b] = Z[b];
  }
}

// Deconvolution and band selection of externally transformed grids.
__global__ void k_grid_deconv(const float2* __restrict__ grid, long long n_spec, int n_fine, int n_bins,
                              int half_bins, const float* __restrict__ corr, double2* __restrict__ F) {
  const long long total = n_spec * n_bins;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total;
       f += (long long)gridDim.x * blockDim.x) {
    const long long sp = f / n_bins;
    const int b = (int)(f - sp * n_bins);
    const int k = b - half_bins;
    const float2 G = grid[sp * n_fine + (k < 0 ? k + n_fine : k)];
    const float c = corr[b];
    F[f] = make_double2(G.x * c, G.y * c);
  }
}

// Strain as FP32 (the mixed form's working precision for samples).
__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    out[k] = (float)in[k];
}

// ---------------------------------------------------------------------------
// Plain FP64 form: one CTA per (template, segment) spectrum.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void plain_phase(double b, double a, double pre, double s, const PlainArgs& p,
                                            double& psi, double& th) {
  const double x = (8.0 / 3.0) * b * s / a;
  const double d = pre * (-expm1(0.625 * log1p(-x)));   // delta(s), Eq. (new_t) referenced to t_i0
  psi = d / p.t_coh;
  psi -= floor(psi);
  th = p.f_c * d;
  th -= floor(th);
}

template <typename TIN, bool SPECTRA>
__global__ void __launch_bounds__(256)
k_plain(const TIN* __restrict__ strain, const double* __restrict__ betas, const int* __restrict__ nseg,
        PlainArgs p, double* __restrict__ S, double2* __restrict__ Fout) {
  extern __shared__ __align__(128) unsigned char smem[];
  double2* g0 = reinterpret_cast<double2*>(smem);
  double2* g1 = g0 + p.n_fine;
  __shared__ int8_t s_rad[16];
  const int m = blockIdx.y;
  const int i = blockIdx.x + p.seg_begin;
  if (!SPECTRA && i >= nseg[m]) return;
  const int tid = threadIdx.x;
  if (tid < 16) s_rad[tid] = p.radices[tid];
  const int n = p.n_fine;
  for (int j = tid; j < n; j += blockDim.x) g0[j] = make_double2(0.0, 0.0);
  __syncthreads();
  const double b = betas[m];
  const double t_i0 = (double)i * (double)p.n_s / p.fs;
  const double a = 1.0 - (8.0 / 3.0) * b * t_i0;
  const double pre = 3.0 * pow(a, 0.625) / (5.0 * b);
  const TIN* src = strain + (long long)i * p.n_s;
  const double hw = 0.5 * p.w;
  for (int j = tid; j < p.n_s; j += blockDim.x) {
    double psi, th;
    plain_phase(b, a, pre, (double)j / p.fs, p, psi, th);
    double sn, cs;
    sincospi(2.0 * th, &sn, &cs);
    const double xv = (double)src[j];
    const double cre = xv * cs, cim = -xv * sn;
    const double U = psi * n;
    const double l0 = ceil(U - hw);
    int cell = (int)l0;
    if (cell < 0) cell += n;
    for (int t = 0; t < p.w; ++t) {
      const double z = (l0 + t - U) / hw;
      const double ph = exp(p.beta_es * (sqrt(fmax(1.0 - z * z, 0.0)) - 1.0));
      int c = cell + t;
      if (c >= n) c -= n;
      atomicAdd(&g0[c].x, ph * cre);
      atomicAdd(&g0[c].y, ph * cim);
    }
  }
  __syncthreads();
  const double2* __restrict__ tw = reinterpret_cast<const double2*>(p.tw);
  double2* res = fft_smem<double2>(g0, g1, n, s_rad, p.n_pass, tw);
  for (int bb = tid; bb < p.n_bins; bb += blockDim.x) {
    int k = bb - p.half_bins;
    int idx = k < 0 ? k + n : k;
    const double2 G = res[idx];
    const double c = p.corr[bb];
    const double fx = G.x * c, fy = G.y * c;
    if (SPECTRA) {
      Fout[((long long)m * p.seg_range + (i - p.seg_begin)) * p.n_bins + bb] = make_double2(fx, fy);
    } else {
      atomicAdd(&S[(long long)m * p.n_bins + bb], 2.0 * (fx * fx + fy * fy) / (double)p.n_s);
    }
  }
}

// ---------------------------------------------------------------------------
// Time map alone (the same per-sample arithmetic as the spreaders)
// ---------------------------------------------------------------------------
__global__ void k_time_map_mixed(const Anchor* __restrict__ anchors, int n_items, MixedArgs a,
                                 double* __restrict__ psi_out, double* __restrict__ th_out) {
  // one thread per lane run of the spreader (samples [r run, (r + 1) run)),
  // stepping the same LaneMaps: Psi' plus the offsets the spreader removed,
  // and the demodulation phase exactly as the spreader forms it
  const int runs = (a.n_s + a.run - 1) / a.run;
  const long long total = (long long)n_items * runs;
  const uint32_t n = (uint32_t)a.n_fine, kc = (uint32_t)a.kc_int;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total;
       f += (long long)gridDim.x * blockDim.x) {
    const long long it = f / runs;
    const int r = (int)(f - it * runs);
    const int j0 = r * a.run, j1 = min(j0 + a.run, a.n_s);
    const int ai = j0 / a.span;
    const Anchor A = anchors[it * a.n_anchor + ai];
    const int l = j0 - ai * a.span;
    LaneMap m = lane_map(A, anchor_psi0(A), A.n1, A.p1lo, A.q2, 1.0f, l);
    m.v -= a.wofs;
    const uint32_t ph0 = (uint32_t)(m.v >> 32), pl0 = (uint32_t)m.v;
    const unsigned long long sp = (unsigned long long)ph0 * n + __umulhi(pl0, n);
    int base = (int)(sp >> 32) - 1;
    if (base < 0) base += (int)n;
    const unsigned long long off = (unsigned long long)base * a.inv_n64;
    m.v -= off;
    const unsigned long long o = a.wofs + off;
    const uint32_t thofs = (uint32_t)(o >> 32) * kc + __umulhi((uint32_t)o, kc);
    LaneMap mt = lane_map(A, anchor_th0(A), A.m1, A.m1lo, A.kq2, a.kc, l);
    for (int j = j0; j < j1; ++j) {
      const unsigned long long v = m.v + o;           // Psi, 2^-64 periods
      uint32_t th;
      if (kc) th = (uint32_t)(m.v >> 32) * kc + __umulhi((uint32_t)m.v, kc) + thofs;
      else th = (uint32_t)(mt.v >> 32);
      const long long out = it * a.n_s + j;
      psi_out[out] = (double)(v >> 11) * 1.1102230246251565404e-16;   // 2^-53
      th_out[out] = (double)th * 2.3283064365386962890625e-10;
      m.step();
      mt.step();
    }
  }
}

__global__ void k_time_map_plain(const int* __restrict__ item_m, const int* __restrict__ item_i, int n_items,
                                 const double* __restrict__ betas, PlainArgs p, double* __restrict__ psi_out,
                                 double* __restrict__ th_out) {
  const long long total = (long long)n_items * p.n_s;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total;
       f += (long long)gridDim.x * blockDim.x) {
    const long long it = f / p.n_s;
    const int j = (int)(f - it * p.n_s);
    const double b = betas[item_m[it]];
    const double t_i0 = (double)item_i[it] * (double)p.n_s / p.fs;
    const double a = 1.0 - (8.0 / 3.0) * b * t_i0;
    const double pre = 3.0 * pow(a, 0.625) / (5.0 * b);
    double psi, th;
    plain_phase(b, a, pre, (double)j / p.fs, p, psi, th);
    psi_out[f] = psi;
    th_out[f] = th;
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
size_t mixed_smem_bytes(const MixedArgs& a) {
  size_t s = a.use_tma ? (size_t)a.ns4 * sizeof(float) : 0;
  s += (size_t)a.n_fine * (a.fft_fixed == 1200 ? 1 : 2) * sizeof(float2);
  s += (size_t)a.nb4 * sizeof(float);
  s += (size_t)a.chunk * a.n_anchor * sizeof(Anchor);
  return s;
}

cudaError_t launch_anchors(const Item* items, int n_items, const double* betas, const AnchorArgs& aa,
                           Anchor* out, long long total, int n_sm, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > (long long)n_sm * 32) blocks = (long long)n_sm * 32;
  k_anchors<<<(unsigned)blocks, 256, 0, st>>>(items, n_items, betas, aa, out, total);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* in, float* out, long long n, int n_sm, cudaStream_t st) {
  long long blocks = (n + 255) / 256;
  if (blocks > (long long)n_sm * 16) blocks = (long long)n_sm * 16;
  k_to_f32<<<(unsigned)blocks, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

template <int W, bool SP>
static cudaError_t launch_mixed_t(const float* strain, const Item* items, int n_items, const double* betas,
                                  int* queue, const MixedArgs& a, float* partial, double2* Fout, int* err, int n_sm,
                                  int ctas_per_sm, cudaStream_t st) {
  const size_t smem = mixed_smem_bytes(a);
  auto kern = a.kc_int > 0 ? (a.use_tma ? k_mixed<W, SP, true, false> : k_mixed<W, SP, true, true>)
                           : (a.use_tma ? k_mixed<W, SP, false, false> : k_mixed<W, SP, false, true>);
  const int threads = a.threads > 0 ? a.threads : kSpreadThreads;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  // With fewer resident CTAs than shared memory allows, hand the rest of the
  // SM's 256 KB to L1 (global-load sample reads live there); a launch
  // attribute, so that a captured graph keeps it.
  cudaLaunchAttribute attr[1];
  int n_attr = 0;
  if (ctas_per_sm > 0 && ctas_per_sm < occ) {
    occ = ctas_per_sm;
    const size_t need = (size_t)occ * (smem + 1024);
    unsigned carveout = (unsigned)((100 * need + 228 * 1024 - 1) / (228 * 1024));
    attr[0].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    attr[0].val.sharedMemCarveout = carveout > 100 ? 100u : carveout;
    n_attr = 1;
  }
  long long grid = (long long)n_sm * occ;
  if (grid > n_items) grid = n_items;
  if (grid < 1) grid = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = n_attr ? attr : nullptr;
  cfg.numAttrs = (unsigned)n_attr;
  return cudaLaunchKernelEx(&cfg, kern, strain, items, n_items, betas, queue, a, partial, Fout, err);
}

cudaError_t launch_mixed(bool spectra, int w, const float* strain, const Item* items, int n_items,
                         const double* betas, int* queue, const MixedArgs& a, float* partial, double2* Fout,
                         int* err, int n_sm, int ctas_per_sm, cudaStream_t st) {
  switch (w) {
#define SRS_W(WW)                                                                                          \
  case WW:                                                                                                 \
    return spectra ? launch_mixed_t<WW, true>(strain, items, n_items, betas, queue, a, partial, Fout, err,  \
                                              n_sm, ctas_per_sm, st)                                       \
                   : launch_mixed_t<WW, false>(strain, items, n_items, betas, queue, a, partial, Fout, err, \
                                               n_sm, ctas_per_sm, st);
    SRS_W(2) SRS_W(3) SRS_W(4) SRS_W(5) SRS_W(6) SRS_W(7) SRS_W(8)
#undef SRS_W
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_plain(bool f64_in, bool spectra, const void* strain, const double* betas, const int* nseg,
                         const PlainArgs& p, int grid_x, int n_templates, double* S, double2* Fout,
                         cudaStream_t st) {
  const size_t smem = (size_t)p.n_fine * 2 * sizeof(double2);
  dim3 grid(grid_x, n_templates);
  cudaError_t e;
#define SRS_PLAIN(TIN, SP)                                                                              \
  do {                                                                                                  \
    auto kern = k_plain<TIN, SP>;                                                                       \
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);             \
    if (e != cudaSuccess) return e;                                                                     \
    kern<<<grid, 256, smem, st>>>(static_cast<const TIN*>(strain), betas, nseg, p, S, Fout);            \
  } while (0)
  if (f64_in) {
    if (spectra) SRS_PLAIN(double, true); else SRS_PLAIN(double, false);
  } else {
    if (spectra) SRS_PLAIN(float, true); else SRS_PLAIN(float, false);
  }
#undef SRS_PLAIN
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int* err, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(err);
  return cudaGetLastError();
}

cudaError_t launch_grid_deconv(const float2* grid, long long n_spec, int n_fine, int n_bins, int half_bins,
                               const float* corr, double2* F, int n_sm, cudaStream_t st) {
  const long long total = n_spec * n_bins;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > (long long)n_sm * 16) blocks = (long long)n_sm * 16;
  k_grid_deconv<<<(unsigned)blocks, 256, 0, st>>>(grid, n_spec, n_fine, n_bins, half_bins, corr, F);
  return cudaGetLastError();
}

cudaError_t launch_time_map_mixed(const Anchor* anchors, int n_items, const MixedArgs& a, double* psi,
                                  double* th, cudaStream_t st) {
  k_time_map_mixed<<<1024, 256, 0, st>>>(anchors, n_items, a, psi, th);
  return cudaGetLastError();
}

cudaError_t launch_time_map_plain(const int* item_m, const int* item_i, int n_items, const double* betas,
                                  const PlainArgs& p, double* psi, double* th, cudaStream_t st) {
  k_time_map_plain<<<1024, 256, 0, st>>>(item_m, item_i, n_items, betas, p, psi, th);
  return cudaGetLastError();
}

}  // namespace srs
