// msp_fft.cuh -- shared-memory-resident 2-D FFT building blocks for sm_103a.
//
// The Fourier operator F of the multislice model (Sec. 2.1 / 2.2) is the
// unnormalised 2-D DFT of a W x W wave.  A W-point line transform is split
// W = N1 * 8 (four-step Cooley-Tukey): eight threads share one line, thread j
// holds the line elements j, j+8, j+16, ...  (N1 complex values in registers),
//   step A: an N1-point DFT in registers over those elements,
//   step B: twiddle by w_W^(j k1),
//   exchange through a small shared buffer private to the group (warp-synchronous),
//   step C: N1/8 eight-point DFTs in registers.
// (W = 256 uses sixteen threads per line and sixteen-point DFTs in both steps.)
// The output indices k1 + N1 k2 held by thread j are again exactly the set
// {j + 8m}, so every line transform starts and ends with the same thread/index
// ownership and consecutive passes need no re-distribution beyond the row <->
// column transpose through shared memory.
//
// The inverse transform is conj(F(conj(x))) (unnormalised); negations fold into
// the arithmetic, so one forward kernel of small DFTs serves both directions.
//
// Shared-memory layout of the wave: element (r, c) lives at r*W + (c ^ swz(r)),
// swz(r) = ((r & 1) << 3) | (r & 6).  With eight threads per line and four lines
// per warp this makes every row and column access of the wave free of bank
// conflicts for 8-byte elements.
#pragma once
#include <cuda_runtime.h>

namespace msp {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// cos(2 pi k / 16) and sin(2 pi k / 16) for k = 0..3 (exact values of the regular 16-gon).
constexpr float kC1 = 0.92387953251128675613f;   // cos(pi/8)
constexpr float kS1 = 0.38268343236508977173f;   // sin(pi/8)
constexpr float kR2 = 0.70710678118654752440f;   // cos(pi/4)

// v * w_16^K with w_16 = exp(-2 pi i / 16); K in [0, 16).  Trivial factors are
// special-cased so that no multiplication by 0 or 1 is issued.
template <int K>
__device__ __forceinline__ float2 tw16(float2 v) {
  constexpr int k = K & 15;
  if constexpr (k == 0) return v;
  else if constexpr (k == 4) return make_float2(v.y, -v.x);           // * (-i)
  else if constexpr (k == 8) return make_float2(-v.x, -v.y);          // * (-1)
  else if constexpr (k == 12) return make_float2(-v.y, v.x);          // * (+i)
  else if constexpr (k == 2) return make_float2(kR2 * (v.x + v.y), kR2 * (v.y - v.x));
  else if constexpr (k == 6) return make_float2(kR2 * (v.y - v.x), -kR2 * (v.x + v.y));
  else if constexpr (k == 10) return make_float2(-kR2 * (v.x + v.y), kR2 * (v.x - v.y));
  else if constexpr (k == 14) return make_float2(kR2 * (v.x - v.y), kR2 * (v.x + v.y));
  else {
    // general: (a + ib)(c - is) with c = cos(2 pi k/16), s = sin(2 pi k/16)
    constexpr float c = (k == 1 || k == 15) ? kC1 : (k == 3 || k == 13) ? kS1 : (k == 5 || k == 11) ? -kS1 : -kC1;
    constexpr float s = (k == 1 || k == 7) ? kS1 : (k == 3 || k == 5) ? kC1 : (k == 9 || k == 15) ? -kS1 : -kC1;
    return make_float2(fmaf(v.x, c, v.y * s), fmaf(v.y, c, -v.x * s));
  }
}

// Radix-2 decimation-in-time butterflies of an N-point DFT, N <= 16.
template <int N, int K>
__device__ __forceinline__ void dit_bfly(const float2* E, const float2* O, float2* X) {
  if constexpr (K < N / 2) {
    const float2 t = tw16<(K * 16) / N>(O[K]);
    X[K] = cadd(E[K], t);
    X[K + N / 2] = csub(E[K], t);
    dit_bfly<N, K + 1>(E, O, X);
  }
}

// X[k] = sum_n x[n*S] w_N^(n k), forward DFT in registers (all indices compile-time).
template <int N, int S>
__device__ __forceinline__ void dft(const float2* x, float2* X) {
  if constexpr (N == 1) {
    X[0] = x[0];
  } else if constexpr (N == 2) {
    X[0] = cadd(x[0], x[S]);
    X[1] = csub(x[0], x[S]);
  } else {
    float2 E[N / 2], O[N / 2];
    dft<N / 2, 2 * S>(x, E);
    dft<N / 2, 2 * S>(x + S, O);
    dit_bfly<N, 0>(E, O, X);
  }
}

__device__ __forceinline__ int swz(int r) { return ((r & 1) << 3) | (r & 6); }

// Twiddles w_W^(j k1) of thread j (of T per line), read from the shared table [k1 * T + j].
template <int T = 8>
struct SharedTwiddles {
  const float2* __restrict__ t;
  int j;
  template <int K1>
  __device__ __forceinline__ float2 get() const { return t[K1 * T + j]; }
};

// Twiddles of thread j held in registers: w^(j k) for k < 8, and w^(j k) = w^(8j) w^(j (k - 8))
// for k >= 8 (one extra rounded product).  `t` is the shared table [k1 * T + j].
template <int W, int T = 8>
struct RegisterTwiddles {
  float2 r[8];   // r[0] unused (k1 = 0 is never multiplied); r[k] = w^(j k), k = 1..7
  float2 w8;     // w^(8 j)
  __device__ __forceinline__ RegisterTwiddles(const float2* __restrict__ t, int j) {
#pragma unroll
    for (int k = 1; k < 8; ++k) r[k] = t[k * T + j];
    w8 = (W / T > 8) ? t[8 * T + j] : make_float2(1.f, 0.f);
  }
  template <int K1>
  __device__ __forceinline__ float2 get() const {
    if constexpr (K1 < 8) return r[K1];
    else if constexpr (K1 == 8) return w8;
    else return cmul(w8, r[K1 - 8]);
  }
};

template <int K1, int N1, typename Tw, int STRIDE = 1>
__device__ __forceinline__ void twiddle_store(const float2* y, float2* xw, const Tw& tw) {
  if constexpr (K1 < N1) {
    xw[K1 * STRIDE] = (K1 == 0) ? y[K1] : cmul(y[K1], tw.template get<K1>());
    twiddle_store<K1 + 1, N1, Tw, STRIDE>(y, xw, tw);
  }
}

// Line transform of a W-point line held by T threads (lane group, T = 8 or 16), in place
// in `v`: on entry v[m] is line element j + T m, on exit v[m] is spectrum element j + T m.
// W = N1 T (four-step): step A is an N1-point DFT in registers over x[T n1 + j], step B
// the twiddles w_W^(j k1), then an exchange, then step C, N1/T T-point DFTs.
// `xb` is the group's private exchange buffer of T * (N1 + 1) float2: thread j writes
// its step-A results Y[j][k1] at xb[j (N1 + 1) + k1] and reads Y[n2][k1] at
// xb[n2 (N1 + 1) + k1]; the odd stride N1 + 1 spreads both patterns over distinct banks
// (and, for T = 8, consecutive groups' buffers start half a bank row apart), so the
// exchange is conflict-free and its addresses are a per-thread base plus immediate offsets.
// `tw.get<k1>()` = w_W^(j k1) (forward sign).  INV selects the unnormalised inverse.
// Exchange layout with the step-A results transposed (eight threads per line): row k1 of
// the group's buffer holds Y[0..7][k1] at stride kXRow, so thread j writes Y[j][k1] at
// xb[k1 kXRow + j] (64-bit stores) and reads its step-C operands Y[0..7][k1] for
// k1 = j + 8 mc as four 128-bit loads per row.  With kXRow = 10 and group buffers
// kXGroup(N1) apart (an odd multiple of eight float2) both patterns are conflict-free.
constexpr int kXRow = 10;
__host__ __device__ constexpr int kXGroup(int n1) { return n1 * kXRow + 8; }

template <int W, bool INV, typename Tw>
__device__ __forceinline__ void line_fft_t(float2 (&v)[W / 8], const Tw& tw, float2* xb, int j) {
  constexpr int N1 = W / 8;
  constexpr int NC = N1 / 8;
  float2 y[N1];
  if constexpr (INV) {
#pragma unroll
    for (int m = 0; m < N1; ++m) v[m] = cconj(v[m]);
  }
  dft<N1, 1>(v, y);
  twiddle_store<0, N1, Tw, kXRow>(y, xb + j, tw);
  __syncwarp();
  float2 b[NC][8];
#pragma unroll
  for (int mc = 0; mc < NC; ++mc) {
    const float4* row = reinterpret_cast<const float4*>(xb + (j + 8 * mc) * kXRow);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 f = row[q];
      b[mc][2 * q] = make_float2(f.x, f.y);
      b[mc][2 * q + 1] = make_float2(f.z, f.w);
    }
  }
  __syncwarp();
#pragma unroll
  for (int mc = 0; mc < NC; ++mc) {
    float2 X[8];
    dft<8, 1>(b[mc], X);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) v[mc + NC * k2] = INV ? cconj(X[k2]) : X[k2];
  }
}

template <int W, bool INV, typename Tw, int T = 8>
__device__ __forceinline__ void line_fft(float2 (&v)[W / T], const Tw& tw, float2* xb, int j) {
  constexpr int N1 = W / T;
  constexpr int NC = N1 / T;
  constexpr int XS = N1 + 1;
  static_assert(N1 % T == 0, "W / T must be a multiple of T");
  float2 y[N1];
  if constexpr (INV) {
#pragma unroll
    for (int m = 0; m < N1; ++m) v[m] = cconj(v[m]);
  }
  // step A: DFT over n1 of x[T n1 + j]
  dft<N1, 1>(v, y);
  // step B: twiddles, then exchange Y[n2 = j][k1]
  float2* xw = xb + j * XS;
  twiddle_store<0, N1>(y, xw, tw);
  __syncwarp();
  float2 b[NC][T];
  const float2* xr = xb + j;
#pragma unroll
  for (int mc = 0; mc < NC; ++mc) {
#pragma unroll
    for (int n2 = 0; n2 < T; ++n2) b[mc][n2] = xr[n2 * XS + T * mc];
  }
  __syncwarp();   // the buffer is reused by this group's next transform
  // step C: T-point DFTs over n2; X[k1 + N1 k2] with k1 = j + T mc is v[mc + NC k2]
#pragma unroll
  for (int mc = 0; mc < NC; ++mc) {
    float2 X[T];
    dft<T, 1>(b[mc], X);
#pragma unroll
    for (int k2 = 0; k2 < T; ++k2) v[mc + NC * k2] = INV ? cconj(X[k2]) : X[k2];
  }
}

}  // namespace msp
