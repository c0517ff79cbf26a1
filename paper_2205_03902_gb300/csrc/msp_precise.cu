// msp_precise.cu -- the precise-forward modes (MSP_PRECISION_FP64_FORWARD, MSP_PRECISION_DF_FORWARD).
//
// The gradients of Sec. 3.2 are linear in the far-field residual R = Psi - sqrt(I) Psi/|Psi|.
// Near a fit (the states a reconstruction visits), ||R|| is a small fraction of ||Psi||, so
// the forward model's rounding, an absolute error of a few units in the last place of Psi,
// becomes a relative error of R amplified by ||Psi|| / ||R|| (hundreds at the workloads'
// starting points).  That amplification happens in the forward model alone: the adjoint
// recursion chi_{m-1} = G^H (conj(X_m) o chi_m) (Sec. 3.3) is linear in R, so its own
// rounding stays relative to ||R||.  This mode therefore runs the forward model (every
// transmit, Fresnel propagation and the far-field transform of Sec. 2.1) in FP64, forms R
// and the loss in FP64, rounds R and the stored exit waves to FP32 once, and runs the
// adjoint in FP32.  Rounding the far field alone to higher precision does not help: the
// error is already in the exit wave of the last slice.
//
// Layout: positions are taken in batches of B, sized so that one batch's FP64 waves
// (B W^2 x 16 bytes) stay resident in L2 across the passes over them.  The line transforms
// (W-point DFTs of rows or columns, the fast path's four-step W = N1 x 8 split in registers)
// carry the operators next to them, so that a pass over the batch is one of
//   [probe o X_1, rows F]                         start of the forward model
//   [columns F, x h(ky) h(kx), columns F^-1]       a Fresnel propagation's middle (G or G^H)
//   [rows F^-1, o X_l and the stash, rows F]       a transmit between two propagations
//   [columns F, loss, R, columns F^-1 (FP32)]      the far field, the residual, chi_L's columns
//   [rows F^-1, adjoint step, rows F]              window gradients, conj(X_m) o chi_m, the probe term
// (double-float or FP64 up to R, FP32 after it).  The FP64 mode is this structure in FP64;
// the double-float mode (MSP_PRECISION_DF_FORWARD) in unevaluated pairs of FP32 numbers.
// The window gradients land in the same per-position buffers as the fused kernel's, so the
// overlap-add, the reductions and the updates downstream are shared with the fast path.
//
// The split-BF16 precision form (MSP_PRECISION_BF16X3_DFT) runs the same steps one operator per
// pass: every 2-D transform of the forward and of the adjoint is two tensor-core passes of the
// W-point DFT as a matrix product with 3-term split-BF16 operands (msp_tcdft.cu), with separate
// transmit, propagator, residual and adjoint kernels; the waves are FP32, and the loss and the
// probe-gradient sum accumulate in FP64.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <type_traits>

#include "msp.h"
#include "msp_kernels.cuh"

namespace msp {
namespace precise {

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2
// ---------------------------------------------------------------------------
template <typename C> struct Real;
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };

template <typename C>
__device__ __forceinline__ C mk(typename Real<C>::type a, typename Real<C>::type b) {
  C c;
  c.x = a;
  c.y = b;
  return c;
}
template <typename C>
__device__ __forceinline__ C add(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C>
__device__ __forceinline__ C sub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C>
__device__ __forceinline__ C mul(C a, C b) { return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C>   // a * conj(b)
__device__ __forceinline__ C mulc(C a, C b) { return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }

__device__ __forceinline__ double2 widen(float2 a) { return make_double2((double)a.x, (double)a.y); }
__device__ __forceinline__ float2 narrow(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 widen(double2 a) { return a; }
__device__ __forceinline__ float2 narrow(float2 a) { return a; }
template <typename C> __device__ __forceinline__ C from_f2(float2 a);
template <> __device__ __forceinline__ float2 from_f2<float2>(float2 a) { return a; }
template <> __device__ __forceinline__ double2 from_f2<double2>(float2 a) { return widen(a); }
template <typename C> __device__ __forceinline__ C from_d(double re, double im);
template <> __device__ __forceinline__ float2 from_d<float2>(double re, double im) { return make_float2((float)re, (float)im); }
template <> __device__ __forceinline__ double2 from_d<double2>(double re, double im) { return make_double2(re, im); }

// ---------------------------------------------------------------------------
// double-float arithmetic: a value is an unevaluated sum h + l of two FP32 numbers with
// |l| <= ulp(h) / 2 (about 48 significand bits), operated on with the error-free
// transformations of Knuth (two-sum) and of the fused multiply-add (two-product).  Additions
// use the short form, whose error is bounded relative to the operands' magnitudes, as the
// error of an FP64 addition is; that is the bound an FFT's error analysis uses.  Every
// operation runs on the FP32 pipe.
// ---------------------------------------------------------------------------
struct dff {
  float h, l;
};
struct dfc {   // complex: re, im
  dff re, im;
};
__device__ __forceinline__ dff two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dff fast_two_sum(float a, float b) {   // |a| >= |b| or a = 0
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dff df_add(dff x, dff y) {
  const dff s = two_sum(x.h, y.h);
  return fast_two_sum(s.h, s.l + (x.l + y.l));
}
__device__ __forceinline__ dff df_neg(dff x) { return {-x.h, -x.l}; }
__device__ __forceinline__ dff df_mul(dff x, dff y) {
  const float p = x.h * y.h;
  float e = fmaf(x.h, y.h, -p);
  e = fmaf(x.h, y.l, e);
  e = fmaf(x.l, y.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dff df_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(dff x) { return (double)x.h + (double)x.l; }
// Square root and quotient: an FP32 seed corrected by one Newton step whose residual is formed
// exactly (Karp and Markstein, ACM TOMS 1997); about 46 significand bits.
__device__ __forceinline__ dff df_sqrt(dff x) {
  if (!(x.h > 0.f)) return {0.f, 0.f};
  const float s = sqrtf(x.h);
  const float p = s * s, e = fmaf(s, s, -p);   // s^2 = p + e exactly
  const float r = ((x.h - p) - e) + x.l;       // x - s^2 (x.h - p exact: p is within a factor 2 of x.h)
  return fast_two_sum(s, r * (0.5f / s));
}
__device__ __forceinline__ dff df_div(dff a, dff b) {   // a / b, b != 0
  const float q0 = a.h / b.h;
  const float p = q0 * b.h, e = fmaf(q0, b.h, -p);   // q0 b.h = p + e exactly
  const float r = (((a.h - p) - e) + a.l) - q0 * b.l; // a - q0 b
  return fast_two_sum(q0, r / b.h);
}

__device__ __forceinline__ dfc add(dfc a, dfc b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dfc sub(dfc a, dfc b) { return {df_add(a.re, df_neg(b.re)), df_add(a.im, df_neg(b.im))}; }
__device__ __forceinline__ dfc mul(dfc a, dfc b) {
  return {df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ dfc mulc(dfc a, dfc b) {   // a * conj(b)
  return {df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.im, b.re), df_neg(df_mul(a.re, b.im)))};
}
__device__ __forceinline__ double2 widen(dfc a) { return make_double2(df_to(a.re), df_to(a.im)); }
__device__ __forceinline__ float2 narrow(dfc a) { return make_float2((float)df_to(a.re), (float)df_to(a.im)); }
template <> __device__ __forceinline__ dfc from_f2<dfc>(float2 a) { return {{a.x, 0.f}, {a.y, 0.f}}; }
template <> __device__ __forceinline__ dfc from_d<dfc>(double re, double im) { return {df_from(re), df_from(im)}; }

__device__ __forceinline__ bool window_ok(int2 ps, int Ny, int Nx, int W) {
  return ps.x >= 0 && ps.y >= 0 && ps.x <= Ny - W && ps.y <= Nx - W;
}

// ---------------------------------------------------------------------------
// batched line DFTs: the four-step split W = N1 x 8 of the fast path in registers, for the
// three arithmetics (FP32, FP64, double-float)
// ---------------------------------------------------------------------------
template <typename C> __device__ __forceinline__ C from_h(C h) { return h; }
template <typename C> __device__ __forceinline__ C conj_(C a) { return mk<C>(a.x, -a.y); }
template <> __device__ __forceinline__ dfc conj_<dfc>(dfc a) { return {a.re, df_neg(a.im)}; }
template <typename C> __device__ __forceinline__ C rot_mi(C a) { return mk<C>(a.y, -a.x); }   // a (-i)
template <> __device__ __forceinline__ dfc rot_mi<dfc>(dfc a) { return {a.im, df_neg(a.re)}; }
template <typename C> __device__ __forceinline__ C neg_(C a) { return mk<C>(-a.x, -a.y); }
template <> __device__ __forceinline__ dfc neg_<dfc>(dfc a) { return {df_neg(a.re), df_neg(a.im)}; }

// cos and sin of 2 pi k / 16, k = 0..3, as exact decimal expansions of the regular 16-gon
constexpr double kCos16[4] = {1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173};

// w_16^K = exp(-2 pi i K / 16) in the type's arithmetic (constants folded at compile time)
template <typename C, int K> __device__ __forceinline__ C w16c();
template <int K>
__device__ __forceinline__ constexpr double cos16() {
  return (K % 16) <= 4 ? kCos16[K % 16] : (K % 16) <= 8 ? -kCos16[8 - K % 16] : (K % 16) <= 12 ? -kCos16[K % 16 - 8]
                                                                                        : kCos16[16 - K % 16];
}
template <int K>
__device__ __forceinline__ constexpr double sin16() { return cos16<K + 12>(); }   // sin x = cos(x - pi/2)
template <> __device__ __forceinline__ float2 w16c<float2, 0>() { return make_float2(1.f, 0.f); }
#define MSP_W16(K)                                                                                        \
  template <> __device__ __forceinline__ float2 w16c<float2, K>() {                                      \
    return make_float2((float)cos16<K>(), (float)-sin16<K>());                                           \
  }                                                                                                       \
  template <> __device__ __forceinline__ double2 w16c<double2, K>() { return make_double2(cos16<K>(), -sin16<K>()); } \
  template <> __device__ __forceinline__ dfc w16c<dfc, K>() {                                            \
    constexpr double c = cos16<K>(), sn = -sin16<K>();                                                    \
    constexpr float ch = (float)c, sh = (float)sn;                                                        \
    return {{ch, (float)(c - (double)ch)}, {sh, (float)(sn - (double)sh)}};                               \
  }
MSP_W16(1) MSP_W16(2) MSP_W16(3) MSP_W16(5) MSP_W16(6) MSP_W16(7) MSP_W16(9) MSP_W16(10) MSP_W16(11)
MSP_W16(13) MSP_W16(14) MSP_W16(15)
#undef MSP_W16

template <typename C, int K>
__device__ __forceinline__ C tw16g(C v) {   // v w_16^K; the quarter turns are exact
  constexpr int k = K & 15;
  if constexpr (k == 0) return v;
  else if constexpr (k == 4) return rot_mi(v);
  else if constexpr (k == 8) return neg_(v);
  else if constexpr (k == 12) return neg_(rot_mi(v));
  else return mul(v, w16c<C, k>());
}
template <typename C, int N, int K>
__device__ __forceinline__ void dit_bfly_g(const C* E, const C* O, C* X) {
  if constexpr (K < N / 2) {
    const C t = tw16g<C, (K * 16) / N>(O[K]);
    X[K] = add(E[K], t);
    X[K + N / 2] = sub(E[K], t);
    dit_bfly_g<C, N, K + 1>(E, O, X);
  }
}
// X[k] = sum_n x[n S] w_N^(n k), N <= 16, in registers
template <typename C, int N, int S>
__device__ __forceinline__ void dft_g(const C* x, C* X) {
  if constexpr (N == 1) {
    X[0] = x[0];
  } else if constexpr (N == 2) {
    X[0] = add(x[0], x[S]);
    X[1] = sub(x[0], x[S]);
  } else {
    C E[N / 2], O[N / 2];
    dft_g<C, N / 2, 2 * S>(x, E);
    dft_g<C, N / 2, 2 * S>(x + S, O);
    dit_bfly_g<C, N, 0>(E, O, X);
  }
}
// N1-point DFTs for N1 = 32 (W = 256): two 16-point DFTs and one radix-2 combination with the
// twiddles w_32^k = from the line's table (tw32[k] = w_W^(k W / 32)).
template <typename C, int N1>
__device__ __forceinline__ void dft_n1(const C* x, C* X, const C* __restrict__ tw32) {
  if constexpr (N1 <= 16) {
    dft_g<C, N1, 1>(x, X);
  } else {
    C E[16], O[16];
    dft_g<C, 16, 2>(x, E);
    dft_g<C, 16, 2>(x + 1, O);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const C t = k == 0 ? O[0] : mul(O[k], tw32[k]);
      X[k] = add(E[k], t);
      X[k + 16] = sub(E[k], t);
    }
  }
}

constexpr int kT = 8;   // threads per line

// Lines per CTA of type C and size W: as many as keep the exchange buffers within 40 KB of
// static shared memory (at most 32).
template <typename C, int W>
struct LinesCfg {
  static constexpr int N1 = W / kT;
  static constexpr int XS = N1 + 1;
  static constexpr int fit = 40960 / (kT * XS * (int)sizeof(C));
  static constexpr int LPC = fit >= 32 ? 32 : fit >= 16 ? 16 : fit >= 8 ? 8 : 4;
  static constexpr int THREADS = LPC * kT;
};

// Forward unnormalised W-point DFT of one line held by eight threads: thread j holds elements
// j + 8m on entry and spectrum elements j + 8m on exit.  Step A is an N1-point DFT in registers,
// step B the twiddles w_W^(j k1) (s_tw[k1 kT + j]), an exchange through the group's shared
// buffer xb, step C N1/8 eight-point DFTs.
template <typename C, int W>
__device__ __forceinline__ void line_dft(C (&v)[W / kT], const C* __restrict__ s_tw, const C* __restrict__ s_t32,
                                         C* xb, int j) {
  constexpr int N1 = W / kT, XS = N1 + 1, NC = N1 / kT;
  C y[N1];
  dft_n1<C, N1>(v, y, s_t32);
  __syncwarp();   // the group's previous transform has read the buffer
  C* xw = xb + j * XS;
  xw[0] = y[0];
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) xw[k1] = mul(y[k1], s_tw[k1 * kT + j]);
  __syncwarp();
  C b[NC][kT];
  const C* xr = xb + j;
#pragma unroll
  for (int mc = 0; mc < NC; ++mc)
#pragma unroll
    for (int n2 = 0; n2 < kT; ++n2) b[mc][n2] = xr[n2 * XS + kT * mc];
#pragma unroll
  for (int mc = 0; mc < NC; ++mc) {
    C X[kT];
    dft_g<C, kT, 1>(b[mc], X);
#pragma unroll
    for (int k2 = 0; k2 < kT; ++k2) v[mc + NC * k2] = X[k2];   // spectrum element k1 + N1 k2, k1 = j + kT mc
  }
}

// The twiddle tables of a CTA's line transforms: s_tw[k1 kT + j] = w_W^(j k1) and, for N1 = 32,
// s_t32[k] = w_32^k, from wtab[k] = w_256^k.
template <typename C, int W, int NT>
__device__ __forceinline__ void load_twiddles(C* s_tw, C* s_t32, const C* __restrict__ wtab) {
  constexpr int N1 = W / kT, STEP = 256 / W;
  for (int i = threadIdx.x; i < N1 * kT; i += NT) s_tw[i] = wtab[((i / kT) * (i % kT) * STEP) % 256];
  if (N1 > 16 && threadIdx.x < 16) s_t32[threadIdx.x] = wtab[threadIdx.x * 8];
}

// The column half of a Fresnel propagation of row-transformed waves: every column is
// transformed, multiplied by the separable propagator h1(ky) h1(kx) (CONJ: its conjugate, for
// G^H) and transformed back (unnormalised inverse); with row transforms before and after this
// is F^-1 (H o F x) up to the normalisation that h1 carries.  Grid: (W / LPC, nb).
template <typename C, typename H, int W, bool CONJ>
__global__ void __launch_bounds__(LinesCfg<C, W>::THREADS) cols_propagate_kernel(C* __restrict__ data,
                                                                                const C* __restrict__ wtab,
                                                                                const H* __restrict__ h1) {
  using Cfg = LinesCfg<C, W>;
  constexpr int N1 = Cfg::N1, XS = Cfg::XS, LPC = Cfg::LPC;
  __shared__ C s_tw[N1 * kT];
  __shared__ C s_t32[16];
  __shared__ C xbuf[LPC][kT * XS];
  load_twiddles<C, W, Cfg::THREADS>(s_tw, s_t32, wtab);
  __syncthreads();
  const int tid = threadIdx.x, j = tid % kT, grp = tid / kT;
  const int line = blockIdx.x * LPC + grp;   // column kx
  C* img = data + (size_t)blockIdx.y * W * W;
  C v[N1];
#pragma unroll
  for (int m = 0; m < N1; ++m) v[m] = img[(size_t)(j + kT * m) * W + line];
  line_dft<C, W>(v, s_tw, s_t32, xbuf[grp], j);
  const C hx = from_h<C>(h1[line]);
#pragma unroll
  for (int m = 0; m < N1; ++m) {
    const C h = mul(from_h<C>(h1[j + kT * m]), hx);   // ky = j + kT m
    v[m] = conj_(CONJ ? mulc(v[m], h) : mul(v[m], h));   // conj: the inverse transform follows
  }
  line_dft<C, W>(v, s_tw, s_t32, xbuf[grp], j);
#pragma unroll
  for (int m = 0; m < N1; ++m) img[(size_t)(j + kT * m) * W + line] = conj_(v[m]);
}

// wtab[k] = exp(-2 pi i k / 256), evaluated in double, rounded (FP32) or split (double-float) once
template <typename C>
__global__ void wtab_kernel(C* __restrict__ wtab) {
  const int k = threadIdx.x;
  double sn, cs;
  sincospi(2.0 * (double)k / 256.0, &sn, &cs);
  wtab[k] = from_d<C>(cs, -sn);
}

// ---------------------------------------------------------------------------
// element-wise kernels over a batch [nb][W][W]
// ---------------------------------------------------------------------------

// FP64 slice transmissions: exp(i sigma V) from the FP32 potentials, or the caller's complex
// slices widened.
template <typename C>
__global__ void table64_kernel(const float* __restrict__ V, const float2* __restrict__ X, C* __restrict__ T, size_t n,
                               double sigma) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (X) {
      T[i] = from_f2<C>(X[i]);
    } else {
      double sn, cs;
      sincos(sigma * (double)V[i], &sn, &cs);
      T[i] = from_d<C>(cs, sn);
    }
  }
}

// h1(k) = exp(-i pi dz lambda q_k^2) / W in double (the propagator factor of the fast path
// before its rounding to single).
template <typename C>
__global__ void h1_64_kernel(C* __restrict__ h1, int W, double dzlam, double dq) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= W) return;
  const double q = (double)(k < W / 2 ? k : k - W) * dq;
  double t = dzlam * q * q;
  t = t - 2.0 * floor(t * 0.5);
  double sn, cs;
  sincospi(t, &sn, &cs);
  h1[k] = from_d<C>(cs / W, -sn / W);
}

struct Batch {
  const int2* pos;     // positions of this batch (pos + b0)
  int nb, W, Ny, Nx, L;
  size_t plane;
};

// Slice `l` (0: the probe itself is the incident wave) : E = psi o X_l, stashed for the adjoint
// (the incident psi in transmission mode), in FP32.  A window outside the object gives zeros.
template <typename C>
__global__ void transmit_kernel(Batch bt, int l, const float2* __restrict__ probe, const C* __restrict__ T,
                                C* __restrict__ wave, float2* __restrict__ stash, int stash_l0, int keep, int cplx) {
  const int W = bt.W;
  const size_t WW = (size_t)W * W, n = (size_t)bt.nb * WW;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / WW);
    const int r = (int)((i % WW) / W), c = (int)(i % W);
    const int2 ps = bt.pos[b];
    C e = from_d<C>(0.0, 0.0), psi = e;
    if (window_ok(ps, bt.Ny, bt.Nx, W)) {
      psi = l == 0 ? from_f2<C>(probe[i % WW]) : wave[i];
      e = mul(psi, T[(size_t)l * bt.plane + (size_t)(ps.x + r) * bt.Nx + ps.y + c]);
    }
    wave[i] = e;
    if (keep) stash[((size_t)b * bt.L + (l - stash_l0)) * WW + (i % WW)] = narrow(cplx ? psi : e);
  }
}

// Row pass of the forward model at slice l, fused: the inverse row transform that ends the
// propagation of slice l - 1 (START: none, the probe is the incident wave of slice 0), the
// transmit E = psi o X_l with its stash for the adjoint (the incident psi in transmission mode),
// and the forward row transform that starts the next propagation or the far field.  A window
// outside the object gives zeros.  Grid: (W / LPC, nb).
template <typename C, int W, bool START>
__global__ void __launch_bounds__(LinesCfg<C, W>::THREADS) rows_transmit_kernel(
    C* __restrict__ wave, const C* __restrict__ wtab, Batch bt, int l, const float2* __restrict__ probe,
    const C* __restrict__ T, float2* __restrict__ stash, int keep, int cplx) {
  using Cfg = LinesCfg<C, W>;
  constexpr int N1 = Cfg::N1, XS = Cfg::XS, LPC = Cfg::LPC;
  constexpr size_t WW = (size_t)W * W;
  __shared__ C s_tw[N1 * kT];
  __shared__ C s_t32[16];
  __shared__ C xbuf[LPC][kT * XS];
  load_twiddles<C, W, Cfg::THREADS>(s_tw, s_t32, wtab);
  __syncthreads();
  const int tid = threadIdx.x, j = tid % kT, grp = tid / kT;
  const int r = blockIdx.x * LPC + grp, b = blockIdx.y;
  C* row = wave + (size_t)b * WW + (size_t)r * W;
  const int2 ps = bt.pos[b];
  const bool ok = window_ok(ps, bt.Ny, bt.Nx, W);
  C v[N1];
  if (START) {
#pragma unroll
    for (int m = 0; m < N1; ++m) v[m] = from_f2<C>(probe[(size_t)r * W + j + kT * m]);
  } else {
#pragma unroll
    for (int m = 0; m < N1; ++m) v[m] = conj_(row[j + kT * m]);
    line_dft<C, W>(v, s_tw, s_t32, xbuf[grp], j);
#pragma unroll
    for (int m = 0; m < N1; ++m) v[m] = conj_(v[m]);   // unnormalised inverse row transform
  }
  const C* Tr = T + (size_t)l * bt.plane + (size_t)(ps.x + r) * bt.Nx + ps.y;
  float2* st = stash + ((size_t)b * bt.L + l) * WW + (size_t)r * W;
#pragma unroll
  for (int m = 0; m < N1; ++m) {
    const int c = j + kT * m;
    const C psi = ok ? v[m] : from_d<C>(0.0, 0.0);
    const C e = ok ? mul(psi, Tr[c]) : psi;
    if (keep) st[c] = narrow(cplx ? psi : e);
    v[m] = e;
  }
  line_dft<C, W>(v, s_tw, s_t32, xbuf[grp], j);
#pragma unroll
  for (int m = 0; m < N1; ++m) row[j + kT * m] = v[m];
}

// x h1(ky) h1(kx) (CONJ: the conjugate, for G^H) on the spectrum of every wave.
template <typename C, typename H>
__global__ void propagator_kernel(Batch bt, const H* __restrict__ h1, C* __restrict__ data, int conj) {
  const int W = bt.W;
  const size_t WW = (size_t)W * W, n = (size_t)bt.nb * WW;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)((i % WW) / W), kx = (int)(i % W);
    const C h = mul(h1[ky], h1[kx]);
    data[i] = conj ? mulc(data[i], h) : mul(data[i], h);
  }
}

// Far field Psi (FP32 waves of the split-BF16 form) -> the loss of each position,
// R = Psi - sqrt(I) Psi / |Psi| (the fraction 0 where |Psi|^2 <= thr2) in FP64 and rounded to
// FP32, or the intensities |Psi|^2.  One CTA per position.  (The FP64 and double-float forms
// compute these in cols_farfield_kernel.)
template <typename C>
__global__ void __launch_bounds__(256) residual_kernel(Batch bt, const C* __restrict__ psi,
                                                       const float* __restrict__ I_meas, const double* __restrict__ zthr2,
                                                       float2* __restrict__ R, double* __restrict__ loss_part,
                                                       float* __restrict__ I_out) {
  __shared__ double red[8];
  const int W = bt.W;
  const size_t WW = (size_t)W * W;
  const int b = blockIdx.x, tid = threadIdx.x;
  const bool ok = window_ok(bt.pos[b], bt.Ny, bt.Nx, W);
  const double thr2 = I_out ? 0.0 : zthr2[0];
  double acc = 0.0;
  for (size_t k = tid; k < WW; k += 256) {
    const double2 v = widen(psi[(size_t)b * WW + k]);
    const double a2 = v.x * v.x + v.y * v.y;
    if (I_out) {
      I_out[(size_t)b * WW + k] = (float)a2;
      continue;
    }
    const double a = sqrt(a2), rt = sqrt((double)I_meas[(size_t)b * WW + k]);
    const double d = rt - a;
    acc += d * d;
    const double f = (a2 > thr2) ? 1.0 - rt / a : 1.0;
    R[(size_t)b * WW + k] = make_float2((float)(v.x * f), (float)(v.y * f));
  }
  if (I_out) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    loss_part[b] = ok ? s : 0.0;   // a skipped position contributes nothing (as in the fused kernel)
  }
}

// One far-field value: R = Psi (1 - sqrt(I) / |Psi|) (the fraction 0 where |Psi|^2 <= thr2) in
// FP32, and (sqrt(I) - |Psi|)^2 added to acc; FP64 or double-float arithmetic, as the residual
// kernel.
__device__ __forceinline__ float2 residual_value(double2 v, float I, double thr2, double& acc) {
  const double a2 = v.x * v.x + v.y * v.y;
  const double a = sqrt(a2), rt = sqrt((double)I);
  const double d = rt - a;
  acc += d * d;
  const double f = (a2 > thr2) ? 1.0 - rt / a : 1.0;
  return make_float2((float)(v.x * f), (float)(v.y * f));
}
__device__ __forceinline__ float2 residual_value(dfc v, float I, double thr2, double& acc) {
  const dff a2 = df_add(df_mul(v.re, v.re), df_mul(v.im, v.im));
  const dff a = df_sqrt(a2), rt = df_sqrt(dff{I, 0.f});
  const double dd = df_to(df_add(rt, df_neg(a)));
  acc += dd * dd;
  const dff f = df_to(a2) > thr2 ? df_add(dff{1.f, 0.f}, df_neg(df_div(rt, a))) : dff{1.f, 0.f};
  const dff rx = df_mul(v.re, f), ry = df_mul(v.im, f);
  return make_float2(rx.h + rx.l, ry.h + ry.l);
}
__device__ __forceinline__ float intensity_value(double2 v) { return (float)(v.x * v.x + v.y * v.y); }
__device__ __forceinline__ float intensity_value(dfc v) {
  const dff a2 = df_add(df_mul(v.re, v.re), df_mul(v.im, v.im));
  return a2.h + a2.l;
}

// Column pass of the far field, fused (FP64 or double-float forward): every column of the
// row-transformed exit wave is transformed (Psi = F E_L), then either the intensities |Psi|^2
// are written (I_out), or the residual R is formed (as residual_kernel does) and transformed back
// by the FP32 inverse column DFT, which leaves the columns of chi_L = F^-1 R for the adjoint's
// first row pass; part[b][blockIdx.x] receives the CTA's share of the loss of position b (0 for
// a window outside the object).  Grid: (W / LPC, nb).
template <typename C, int W>
__global__ void __launch_bounds__(LinesCfg<C, W>::THREADS) cols_farfield_kernel(
    const C* __restrict__ wave, const C* __restrict__ wtab, const float2* __restrict__ wtab8, Batch bt,
    const float* __restrict__ I_meas, const double* __restrict__ zthr2, float2* __restrict__ chi,
    double* __restrict__ part, float* __restrict__ I_out) {
  using Cfg = LinesCfg<C, W>;
  constexpr int N1 = Cfg::N1, XS = Cfg::XS, LPC = Cfg::LPC, NT = Cfg::THREADS;
  constexpr size_t WW = (size_t)W * W;
  __shared__ C s_tw[N1 * kT];
  __shared__ C s_t32[16];
  __shared__ float2 s_tw8[N1 * kT];
  __shared__ float2 s_t328[16];
  __shared__ C xbuf[LPC][kT * XS];
  __shared__ double red[NT / 32];
  load_twiddles<C, W, NT>(s_tw, s_t32, wtab);
  load_twiddles<float2, W, NT>(s_tw8, s_t328, wtab8);
  __syncthreads();
  const int tid = threadIdx.x, j = tid % kT, grp = tid / kT;
  const int c = blockIdx.x * LPC + grp, b = blockIdx.y;
  C v[N1];
#pragma unroll
  for (int m = 0; m < N1; ++m) v[m] = wave[(size_t)b * WW + (size_t)(j + kT * m) * W + c];
  line_dft<C, W>(v, s_tw, s_t32, xbuf[grp], j);   // Psi at (ky = j + kT m, kx = c)
  if (I_out) {
#pragma unroll
    for (int m = 0; m < N1; ++m) I_out[(size_t)b * WW + (size_t)(j + kT * m) * W + c] = intensity_value(v[m]);
    return;
  }
  const double thr2 = zthr2[0];
  double acc = 0.0;
  float2 r[N1];
#pragma unroll
  for (int m = 0; m < N1; ++m)
    r[m] = conj_(residual_value(v[m], I_meas[(size_t)b * WW + (size_t)(j + kT * m) * W + c], thr2, acc));
  line_dft<float2, W>(r, s_tw8, s_t328, reinterpret_cast<float2*>(xbuf[grp]), j);   // conj(F conj R) = F^-1 R
#pragma unroll
  for (int m = 0; m < N1; ++m) chi[(size_t)b * WW + (size_t)(j + kT * m) * W + c] = conj_(r[m]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) sum += red[w];
    part[(size_t)b * gridDim.x + blockIdx.x] = window_ok(bt.pos[b], bt.Ny, bt.Nx, W) ? sum : 0.0;
  }
}

// loss_part[b] = sum of the far-field kernel's nparts partials of position b, in order.
__global__ void loss_parts_kernel(const double* __restrict__ part, int nb, int nparts, double* __restrict__ loss_part) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double sum = 0.0;
  for (int i = 0; i < nparts; ++i) sum += part[(size_t)b * nparts + i];
  loss_part[b] = sum;
}

// Adjoint at slice l on chi = dL/dconj(E_l) (FP32): the window gradient of slice l
//   potential mode 2 sigma Im(conj(E_l) chi)  -> wgrad (float), transmission mode conj(psi_l) chi (float2),
// the illumination |psi_in,l|^2 of a layer step, then chi <- conj(X_l) o chi (if go_on), and at
// l = 0 the probe-gradient term conj(X_1) o chi_1 of each position.
struct AdjOut {
  float* wgrad;        // this slice's window gradients of position s at wgrad + wstride * s (or NULL)
  size_t wstride;      // floats between consecutive positions' windows
  float* willum;       // [S][W][W] (layer step) or NULL
  float2* contrib;     // [nb][W][W] probe-gradient terms (l = 0) or NULL
  int s0;              // scan index of the batch's first position
};
__global__ void adjoint_kernel(Batch bt, int l, float2* __restrict__ chi, const float2* __restrict__ stash_l,
                               const float2* __restrict__ X, AdjOut o, int go_on, int cplx, float two_sigma) {
  const int W = bt.W;
  const size_t WW = (size_t)W * W, n = (size_t)bt.nb * WW;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / WW);
    const size_t k = i % WW;
    const int r = (int)(k / W), c = (int)(k % W);
    const int2 ps = bt.pos[b];
    const bool ok = window_ok(ps, bt.Ny, bt.Nx, W);
    float2 v = chi[i];
    if (!ok) v = make_float2(0.f, 0.f);
    const size_t s = (size_t)(o.s0 + b);
    if (o.wgrad || o.willum) {
      const float2 e = stash_l[(size_t)b * bt.L * WW + k];   // stash_l points at slice l of position 0
      if (o.wgrad) {
        if (cplx) reinterpret_cast<float2*>(o.wgrad)[(o.wstride / 2) * s + k] = mulc(v, e);
        else o.wgrad[o.wstride * s + k] = two_sigma * (e.x * v.y - e.y * v.x);
      }
      if (o.willum) o.willum[s * WW + k] = e.x * e.x + e.y * e.y;
    }
    if (go_on) {
      const float2 t = ok ? X[(size_t)l * bt.plane + (size_t)(ps.x + r) * bt.Nx + ps.y + c] : make_float2(0.f, 0.f);
      v = mulc(v, t);
      if (l == 0) {
        if (o.contrib) o.contrib[i] = v;
      } else {
        chi[i] = v;
      }
    }
  }
}

// Row pass of the adjoint at slice l, fused: the inverse row transform that ends chi_l's
// transform (a propagation, or F^-1 of the residual), the adjoint step of adjoint_kernel, and
// (NEXT) the forward row transform that starts the propagation by G^H.  Grid: (W / LPC, nb).
template <int W, bool NEXT>
__global__ void __launch_bounds__(LinesCfg<float2, W>::THREADS) rows_adjoint_kernel(
    float2* __restrict__ chi, const float2* __restrict__ wtab, Batch bt, int l, const float2* __restrict__ stash_l,
    const float2* __restrict__ X, AdjOut o, int go_on, int cplx, float two_sigma) {
  using Cfg = LinesCfg<float2, W>;
  constexpr int N1 = Cfg::N1, XS = Cfg::XS, LPC = Cfg::LPC;
  constexpr size_t WW = (size_t)W * W;
  __shared__ float2 s_tw[N1 * kT];
  __shared__ float2 s_t32[16];
  __shared__ float2 xbuf[LPC][kT * XS];
  load_twiddles<float2, W, Cfg::THREADS>(s_tw, s_t32, wtab);
  __syncthreads();
  const int tid = threadIdx.x, j = tid % kT, grp = tid / kT;
  const int r = blockIdx.x * LPC + grp, b = blockIdx.y;
  float2* row = chi + (size_t)b * WW + (size_t)r * W;
  const int2 ps = bt.pos[b];
  const bool ok = window_ok(ps, bt.Ny, bt.Nx, W);
  const size_t s = (size_t)(o.s0 + b);
  float2 v[N1];
#pragma unroll
  for (int m = 0; m < N1; ++m) v[m] = conj_(row[j + kT * m]);
  line_dft<float2, W>(v, s_tw, s_t32, xbuf[grp], j);
#pragma unroll
  for (int m = 0; m < N1; ++m) {
    const int c = j + kT * m;
    const size_t k = (size_t)r * W + c;
    float2 u = ok ? conj_(v[m]) : make_float2(0.f, 0.f);   // chi_l at (r, c)
    if (o.wgrad || o.willum) {
      const float2 e = stash_l[(size_t)b * bt.L * WW + k];
      if (o.wgrad) {
        if (cplx) reinterpret_cast<float2*>(o.wgrad)[(o.wstride / 2) * s + k] = mulc(u, e);
        else o.wgrad[o.wstride * s + k] = two_sigma * (e.x * u.y - e.y * u.x);
      }
      if (o.willum) o.willum[s * WW + k] = e.x * e.x + e.y * e.y;
    }
    if (go_on) {
      const float2 t = ok ? X[(size_t)l * bt.plane + (size_t)(ps.x + r) * bt.Nx + ps.y + c] : make_float2(0.f, 0.f);
      u = mulc(u, t);
      if (l == 0 && o.contrib) o.contrib[(size_t)b * WW + k] = u;
    }
    v[m] = u;
  }
  if (NEXT) {
    line_dft<float2, W>(v, s_tw, s_t32, xbuf[grp], j);
#pragma unroll
    for (int m = 0; m < N1; ++m) row[j + kT * m] = v[m];
  }
}

// dp64[k] += sum_{b < nb} contrib[b][k], b ascending (FP64, fixed order); eight loads in flight
// per thread, added in the same order.
__global__ void dprobe_accumulate_kernel(const float2* __restrict__ contrib, int nb, int WW, double2* __restrict__ dp64,
                                         int first) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= WW) return;
  double2 a = first ? make_double2(0.0, 0.0) : dp64[k];
  int b = 0;
  for (; b + 8 <= nb; b += 8) {
    float2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = contrib[(size_t)(b + u) * WW + k];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      a.x += v[u].x;
      a.y += v[u].y;
    }
  }
  for (; b < nb; ++b) {
    const float2 v = contrib[(size_t)b * WW + k];
    a.x += v.x;
    a.y += v.y;
  }
  dp64[k] = a;
}

__global__ void dprobe_finish_kernel(const double2* __restrict__ dp64, int WW, float2* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < WW) out[k] = narrow(dp64[k]);
}

__global__ void flag_windows_kernel(const int2* __restrict__ pos, int S, int Ny, int Nx, int W, int* err) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x)
    if (!window_ok(pos[s], Ny, Nx, W)) atomicMax(err, 1);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <typename C, int W>
static void rows_transmit(bool start, C* wave, const C* wtab, const Batch& bt, int l, const float2* probe, const C* T,
                          float2* stash, int keep, int cplx, cudaStream_t st) {
  const dim3 grid(W / LinesCfg<C, W>::LPC, bt.nb);
  constexpr int NT = LinesCfg<C, W>::THREADS;
  if (start) rows_transmit_kernel<C, W, true><<<grid, NT, 0, st>>>(wave, wtab, bt, l, probe, T, stash, keep, cplx);
  else rows_transmit_kernel<C, W, false><<<grid, NT, 0, st>>>(wave, wtab, bt, l, probe, T, stash, keep, cplx);
}
template <typename C>
static void rows_transmit_w(bool start, C* wave, const C* wtab, const Batch& bt, int l, const float2* probe,
                            const C* T, float2* stash, int keep, int cplx, cudaStream_t st) {
  if (bt.W == 64) rows_transmit<C, 64>(start, wave, wtab, bt, l, probe, T, stash, keep, cplx, st);
  else if (bt.W == 128) rows_transmit<C, 128>(start, wave, wtab, bt, l, probe, T, stash, keep, cplx, st);
  else rows_transmit<C, 256>(start, wave, wtab, bt, l, probe, T, stash, keep, cplx, st);
}
// The fused far-field column pass; returns the loss partials per position (0 in the forward mode).
template <typename C>
static int cols_farfield_w(int W, const C* wave, const C* wtab, const float2* wtab8, const Batch& bt,
                           const float* I_meas, const double* zthr2, float2* chi, double* part, float* I_out,
                           cudaStream_t st) {
#define MSP_FAR(WW_)                                                                                             \
  if (W == WW_) {                                                                                                \
    const dim3 grid(WW_ / LinesCfg<C, WW_>::LPC, bt.nb);                                                         \
    cols_farfield_kernel<C, WW_><<<grid, LinesCfg<C, WW_>::THREADS, 0, st>>>(wave, wtab, wtab8, bt, I_meas, zthr2, \
                                                                             chi, part, I_out);                  \
    return WW_ / LinesCfg<C, WW_>::LPC;                                                                          \
  }
  MSP_FAR(64)
  MSP_FAR(128)
  MSP_FAR(256)
#undef MSP_FAR
  return 0;
}

// The column half of a propagation (the rows are fused with the transmit or the adjoint step);
// CONJ: by G^H.
template <typename C, bool CONJ = false>
static void cols_propagate_w(int W, C* data, const C* wtab, const C* h1, int nb, cudaStream_t st) {
#define MSP_COLS(WW_)                                                                                   \
  if (W == WW_) {                                                                                       \
    cols_propagate_kernel<C, C, WW_, CONJ>                                                              \
        <<<dim3(WW_ / LinesCfg<C, WW_>::LPC, nb), LinesCfg<C, WW_>::THREADS, 0, st>>>(data, wtab, h1);  \
    return;                                                                                             \
  }
  MSP_COLS(64)
  MSP_COLS(128)
  MSP_COLS(256)
#undef MSP_COLS
}

static void rows_adjoint_w(bool next, float2* chi, const float2* wtab, const Batch& bt, int l, const float2* stash_l,
                           const float2* X, const AdjOut& o, int go_on, int cplx, float two_sigma, cudaStream_t st) {
#define MSP_ROWA(WW_)                                                                                             \
  if (bt.W == WW_) {                                                                                              \
    const dim3 grid(WW_ / LinesCfg<float2, WW_>::LPC, bt.nb);                                                     \
    constexpr int NT = LinesCfg<float2, WW_>::THREADS;                                                            \
    if (next) rows_adjoint_kernel<WW_, true><<<grid, NT, 0, st>>>(chi, wtab, bt, l, stash_l, X, o, go_on, cplx, two_sigma); \
    else rows_adjoint_kernel<WW_, false><<<grid, NT, 0, st>>>(chi, wtab, bt, l, stash_l, X, o, go_on, cplx, two_sigma);    \
    return;                                                                                                       \
  }
  MSP_ROWA(64)
  MSP_ROWA(128)
  MSP_ROWA(256)
#undef MSP_ROWA
}

static int elem_blocks(size_t n, int sms) {
  const size_t b = (n + 255) / 256, cap = (size_t)sms * 8;
  return (int)(b < cap ? (b ? b : 1) : cap);
}

}  // namespace precise

cudaError_t tcdft_prepare(int W, int inverse, void* mat, cudaStream_t st);
cudaError_t tcdft_pass(int W, const float2* in, float2* out, int nb, const void* mat, int* err, int wait_limit,
                       cudaStream_t st);
size_t tcdft_matrix_bytes(int W);

// Positions per batch of the batched modes: one batch's FP64 waves take 64 MiB (the split-BF16
// mode uses the same batches of FP32 waves and a second buffer of the same size).
int precise_batch(int W, int S) {
  const int b = (int)((size_t(64) << 20) / ((size_t)W * W * sizeof(double2)));
  return S < b ? (S > 0 ? S : 1) : b;
}

namespace {
struct Segs {
  double2* T64 = nullptr;     // transmissions of the FP64 / double-float forward
  double2* h1d = nullptr;     // propagator factor of the FP64 / double-float forward
  void* wave = nullptr;       // [B][W][W] forward waves: double2, double-float or float2 (split BF16)
  float2* tmp = nullptr;      // [B][W][W] second buffer of the tensor-core passes (split BF16)
  float2* chi = nullptr;      // [B][W][W] adjoint waves
  float2* stash = nullptr;    // [B][L][W][W] exit (or incident) waves kept for the adjoint
  float2* contrib = nullptr;  // [B][W][W] probe-gradient terms of the batch
  double2* dp64 = nullptr;    // [W][W] probe-gradient sum
  void* mat_f = nullptr;      // split-BF16 DFT matrices, forward and inverse (split BF16)
  void* mat_i = nullptr;
  void* wtab16 = nullptr;     // [256] exp(-2 pi i k / 256), FP64 or double-float (the forward's type)
  double* lpart = nullptr;    // [B][W / 4] loss partials of the fused far-field pass
  float2* wtab8 = nullptr;    // [256] the same rounded to FP32 (the adjoint)
  size_t bytes = 0;
};

Segs carve(int precision, int W, int L, int Ny, int Nx, int S, char* base) {
  auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
  Segs g;
  size_t off = 0;
  auto take = [&](size_t b) { char* q = base ? base + off : nullptr; off += a(b); return (void*)q; };
  const size_t WW = (size_t)W * W, B = (size_t)precise_batch(W, S);
  const bool tc = precision == MSP_PRECISION_BF16X3_DFT;
  static_assert(sizeof(precise::dfc) == sizeof(double2), "double-float and FP64 complex share the segments");
  if (!tc) {   // FP64 or double-float (both 16 bytes per complex value)
    g.T64 = (double2*)take((size_t)L * Ny * Nx * sizeof(double2));
    g.h1d = (double2*)take(W * sizeof(double2));
  }
  g.wave = take(B * WW * (tc ? sizeof(float2) : sizeof(double2)));
  if (tc) g.tmp = (float2*)take(B * WW * sizeof(float2));
  g.chi = (float2*)take(B * WW * sizeof(float2));
  g.stash = (float2*)take(B * L * WW * sizeof(float2));
  g.contrib = (float2*)take(B * WW * sizeof(float2));
  g.dp64 = (double2*)take(WW * sizeof(double2));
  if (tc) {
    g.mat_f = take(tcdft_matrix_bytes(W));
    g.mat_i = take(tcdft_matrix_bytes(W));
  } else {
    g.wtab16 = take(256 * sizeof(double2));
    g.wtab8 = (float2*)take(256 * sizeof(float2));
    g.lpart = (double*)take(B * (W / 4) * sizeof(double));
  }
  g.bytes = off;
  return g;
}
}  // namespace

// Workspace of the batched modes beyond the fast path's (every segment 256-byte aligned).
size_t precise_extra_bytes(int precision, int W, int L, int Ny, int Nx, int S) {
  return carve(precision, W, L, Ny, Nx, S, nullptr).bytes;
}

// The forward model and the adjoint of `mode` over all positions in batches, writing what the
// fused kernel writes: I_out (forward), loss_part, the window gradients and illumination, and
// the probe gradient into dprobe_part[0] (one partial).  FP64-forward mode: FP64 forward with the
// four-step line FFT, FP32 adjoint.  Double-float mode: the same with the forward in double-float.  Split-BF16 mode: every 2-D transform as two tensor-core passes,
// FP32 waves.  Reports the number of kernels launched.
cudaError_t run_precise(int mode, const PosParams& p, int W, const PreciseIn& in, cudaStream_t st, long long* launches) {
  using namespace precise;
  const int L = p.L, S = p.S;
  const size_t WW = (size_t)W * W, plane = (size_t)p.Ny * p.Nx;
  const int B = precise_batch(W, S);
  const bool tc = in.precision == MSP_PRECISION_BF16X3_DFT;
  const bool df = in.precision == MSP_PRECISION_DF_FORWARD;
  const Segs g = carve(in.precision, W, L, p.Ny, p.Nx, S, in.extra);
  long long n_launch = 0;
  cudaError_t err = cudaSuccess;

  if (tc) {
    if ((err = tcdft_prepare(W, 0, g.mat_f, st)) != cudaSuccess) return err;
    if ((err = tcdft_prepare(W, 1, g.mat_i, st)) != cudaSuccess) return err;
    n_launch += 2;
  } else if (df) {
    table64_kernel<dfc><<<elem_blocks((size_t)L * plane, in.sms), 256, 0, st>>>(in.X ? nullptr : in.V, in.X,
                                                                                 (dfc*)g.T64, (size_t)L * plane,
                                                                                 in.sigma);
    h1_64_kernel<dfc><<<(W + 255) / 256, 256, 0, st>>>((dfc*)g.h1d, W, in.dzlam, in.dq);
    wtab_kernel<dfc><<<1, 256, 0, st>>>((dfc*)g.wtab16);
    wtab_kernel<float2><<<1, 256, 0, st>>>(g.wtab8);
    n_launch += 4;
  } else {
    table64_kernel<double2><<<elem_blocks((size_t)L * plane, in.sms), 256, 0, st>>>(in.X ? nullptr : in.V, in.X,
                                                                                     g.T64, (size_t)L * plane, in.sigma);
    h1_64_kernel<double2><<<(W + 255) / 256, 256, 0, st>>>(g.h1d, W, in.dzlam, in.dq);
    wtab_kernel<double2><<<1, 256, 0, st>>>((double2*)g.wtab16);
    wtab_kernel<float2><<<1, 256, 0, st>>>(g.wtab8);
    n_launch += 4;
  }
  flag_windows_kernel<<<(S + 255) / 256, 256, 0, st>>>(p.pos, S, p.Ny, p.Nx, W, p.err);
  ++n_launch;

  // 2-D transforms: unnormalised, forward or inverse
  auto keep_first = [&](cudaError_t e) {
    if (err == cudaSuccess) err = e;
  };
  // split-BF16 form: a 2-D transform is two tensor-core DFT passes (each transposes the waves)
  auto fwd2 = [&](int nb, bool inverse) {   // the forward model's waves
    keep_first(tcdft_pass(W, (float2*)g.wave, g.tmp, nb, inverse ? g.mat_i : g.mat_f, p.err, in.wait_limit, st));
    keep_first(tcdft_pass(W, g.tmp, (float2*)g.wave, nb, inverse ? g.mat_i : g.mat_f, p.err, in.wait_limit, st));
    n_launch += 2;
  };
  auto adj2 = [&](int nb, bool inverse) {   // the adjoint's waves
    keep_first(tcdft_pass(W, g.chi, g.tmp, nb, inverse ? g.mat_i : g.mat_f, p.err, in.wait_limit, st));
    keep_first(tcdft_pass(W, g.tmp, g.chi, nb, inverse ? g.mat_i : g.mat_f, p.err, in.wait_limit, st));
    n_launch += 2;
  };

  const bool fwd = mode == MODE_FORWARD;
  const bool loss_only = mode == MODE_LOSS_GRAD && p.loss_only;   // the forward and the loss only
  const int lowest = mode == MODE_LAYER ? p.layer : 0;
  const bool want_dprobe = mode != MODE_LAYER && !fwd && p.want_dprobe;
  const int CW = p.cplx ? 2 : 1;
  for (int b0 = 0; b0 < S; b0 += B) {
    const int nb = S - b0 < B ? S - b0 : B;
    Batch bt{p.pos + b0, nb, W, p.Ny, p.Nx, L, plane};
    const int eb = elem_blocks((size_t)nb * WW, in.sms);
    // forward: slice 0, then (propagate, transmit) for every later slice
    if (tc) {
      for (int l = 0; l < L; ++l) {
        const int keep = !fwd && !loss_only && l >= lowest;
        if (l > 0) {
          fwd2(nb, false);
          propagator_kernel<float2, float2><<<eb, 256, 0, st>>>(bt, p.h1, (float2*)g.wave, 0);
          fwd2(nb, true);
          ++n_launch;
        }
        transmit_kernel<float2><<<eb, 256, 0, st>>>(bt, l, p.probe, p.T, (float2*)g.wave, g.stash, 0, keep, p.cplx);
        ++n_launch;
      }
      fwd2(nb, false);   // far field Psi = F(E_L)
    } else {
      // row passes fused with the transmits: [start: probe o X_1, rows F], then per slice
      // [columns F, x H, F^-1] [rows F^-1, o X_l, rows F]; the far field's columns follow
      auto fused = [&](auto* wave, const auto* wtab, const auto* T, const auto* h1d) {
        for (int l = 0; l < L; ++l) {
          const int keep = !fwd && !loss_only && l >= lowest;
          if (l > 0) {
            cols_propagate_w(W, wave, wtab, h1d, nb, st);
            ++n_launch;
          }
          rows_transmit_w(l == 0, wave, wtab, bt, l, p.probe, T, g.stash, keep, p.cplx, st);
          ++n_launch;
        }
      };
      if (df) fused((dfc*)g.wave, (const dfc*)g.wtab16, (const dfc*)g.T64, (const dfc*)g.h1d);
      else fused((double2*)g.wave, (const double2*)g.wtab16, (const double2*)g.T64, (const double2*)g.h1d);
    }
    const float* Im = fwd ? nullptr : p.I_meas + (size_t)b0 * WW;
    double* lp = fwd ? nullptr : p.loss_part + b0;
    float* Io = fwd ? p.I_out + (size_t)b0 * WW : nullptr;
    if (tc) {
      residual_kernel<float2><<<nb, 256, 0, st>>>(bt, (const float2*)g.wave, Im, p.zthr2, g.chi, lp, Io);
      ++n_launch;
    } else {
      // [columns F of the far field, the residual, columns F^-1 of R]: chi_L's columns
      const int np = df ? cols_farfield_w(W, (const dfc*)g.wave, (const dfc*)g.wtab16, g.wtab8, bt, Im, p.zthr2, g.chi,
                                          g.lpart, Io, st)
                        : cols_farfield_w(W, (const double2*)g.wave, (const double2*)g.wtab16, g.wtab8, bt, Im,
                                          p.zthr2, g.chi, g.lpart, Io, st);
      ++n_launch;
      if (!fwd) {
        loss_parts_kernel<<<(nb + 127) / 128, 128, 0, st>>>(g.lpart, nb, np, lp);
        ++n_launch;
      }
    }
    if (fwd || loss_only) continue;
    // adjoint: chi_L = F^H R, then down the slices
    if (tc) {
      adj2(nb, true);
      for (int l = L - 1; l >= lowest; --l) {
        const bool grad_here = mode == MODE_LOSS_GRAD || (mode == MODE_LAYER && l == p.layer);
        const bool go_on = (l > lowest) || (l == 0 && want_dprobe);
        AdjOut o{};
        o.s0 = b0;
        if (grad_here) {
          o.wgrad = mode == MODE_LOSS_GRAD ? p.wgrad + (size_t)CW * l * WW : p.wgrad;
          o.wstride = (size_t)CW * WW * (mode == MODE_LOSS_GRAD ? L : 1);
          if (mode == MODE_LAYER) o.willum = p.willum;
        }
        if (l == 0 && want_dprobe) o.contrib = g.contrib;
        adjoint_kernel<<<eb, 256, 0, st>>>(bt, l, g.chi, g.stash + (size_t)l * WW, p.T, o, go_on ? 1 : 0, p.cplx,
                                           p.two_sigma);
        ++n_launch;
        if (!go_on || l == 0) break;
        adj2(nb, false);
        propagator_kernel<float2, float2><<<eb, 256, 0, st>>>(bt, p.h1, g.chi, 1);
        adj2(nb, true);
        ++n_launch;
      }
    } else {
      // the row passes fused with the adjoint steps (the columns of F^-1 R came with the far
      // field): per slice [rows F^-1, adjoint step, rows F] [columns F, x conj H, F^-1], the last
      // slice's row pass without the forward transform
      for (int l = L - 1; l >= lowest; --l) {
        const bool grad_here = mode == MODE_LOSS_GRAD || (mode == MODE_LAYER && l == p.layer);
        const bool go_on = (l > lowest) || (l == 0 && want_dprobe);
        const bool next = go_on && l > 0;
        AdjOut o{};
        o.s0 = b0;
        if (grad_here) {
          o.wgrad = mode == MODE_LOSS_GRAD ? p.wgrad + (size_t)CW * l * WW : p.wgrad;
          o.wstride = (size_t)CW * WW * (mode == MODE_LOSS_GRAD ? L : 1);
          if (mode == MODE_LAYER) o.willum = p.willum;
        }
        if (l == 0 && want_dprobe) o.contrib = g.contrib;
        rows_adjoint_w(next, g.chi, g.wtab8, bt, l, g.stash + (size_t)l * WW, p.T, o, go_on ? 1 : 0, p.cplx,
                       p.two_sigma, st);
        ++n_launch;
        if (!next) break;
        cols_propagate_w<float2, true>(W, g.chi, g.wtab8, p.h1, nb, st);
        ++n_launch;
      }
    }
    if (want_dprobe) {
      dprobe_accumulate_kernel<<<(int)((WW + 255) / 256), 256, 0, st>>>(g.contrib, nb, (int)WW, g.dp64, b0 == 0);
      ++n_launch;
    }
  }
  if (want_dprobe) {
    dprobe_finish_kernel<<<(int)((WW + 255) / 256), 256, 0, st>>>(g.dp64, (int)WW, p.dprobe_part);
    ++n_launch;
  }
  *launches = n_launch;
  const cudaError_t last = cudaGetLastError();
  return err != cudaSuccess ? err : last;
}

}  // namespace msp
