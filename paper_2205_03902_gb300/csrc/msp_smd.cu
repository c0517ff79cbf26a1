// msp_smd.cu -- Sparse Matrix Decomposition (Sec. 3.4, Algorithm 2) on sm_103a.
//
// Algorithm 2 alternates two problems on the paper's full-field model (an N x N
// object, the probe shifted cyclically, dense N^2 x N^2 matrices):
//
//   matrix estimate   A <- A - mu F^H ((|FAP| - sqrt I) o FAP/|FAP|) P^H
//                     Two dense complex contractions (A P and the rank-S update by P^H)
//                     run in `cgemm_kernel`; between them `farfield_kernel` takes every
//                     column of A P through the 2-D DFT, forms the amplitude-flow
//                     residual and takes it back (F^H), one CTA per column.
//   decomposition     The proximal step of every slice needs diag(R_l^H M S_l^H) with
//                     M = lambda A(o) - Ahat.  Column j of A(o) is the multislice exit
//                     wave of a unit impulse at object pixel j, S_l e_j is the wave that
//                     impulse makes incident on slice l and R_l^H m_j is the adjoint wave
//                     at slice l, so the diagonal is sum_j (R_l^H m_j) o conj(S_l e_j):
//                     one forward and one adjoint multislice pass per column, with the
//                     per-slice products summed over columns (`grad_kernel`).  No dense
//                     R_l or S_l is formed.  `transfer_kernel` rebuilds A(o) column by
//                     column for the lambda update (Eq. Update Lambda) and for A^{t+1}.
//
// N is not a power of two in the paper's own setting (40 x 40 detector and scan,
// Table 1).  The 2-D DFT of an N x N image is two passes over its rows in shared memory,
// each the product with the N-point DFT matrix (Y = W X W), factored once as N = N1 N2
// (Cooley-Tukey): a length-N1 DFT over the N2 decimated sub-sequences, a twiddle, then a
// length-N2 DFT, N1 + N2 + 1 complex multiply-adds per output instead of N.  A thread owns
// two rows and one bin c0 < N1 of the short DFT, i.e. the N2 columns c0 + N1 j: every step
// of the factored pass stays in its registers.  Every pass stores its result transposed,
// so after the two passes of a 2-D DFT the image is back in row-major order and every
// elementwise step (propagator, slice, residual) works on the same 2 N2 pixels per
// thread, held in registers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <mutex>
#include <string>

#include "msp.h"
#include "msp_smd.h"
#include "msp_cgemm.cuh"

namespace msp {

msp_status set_last_error(msp_status s, const std::string& m);   // shown by msp_last_error_message()
msp_status refuse_untrusted_device();                            // MSP_EDEVICE once a drain wait ran out
void count_launches(int n);
int tc_wait_limit();
msp_status profiled_launch(cudaStream_t st, const std::function<cudaError_t()>& launch);

namespace smd {

constexpr double kZeroTau = 1e-5;   // zero rule: |U| <= 1e-5 sqrt(mean I) counts as U = 0
constexpr int kMaxSlices = 5;
constexpr int kPartSlots = 4096;    // FP64 partial sums per reduction

// scalar slots in the workspace
enum { S_OBJ = 0, S_MU = 1, S_SPEC = 2, S_SUMI = 3, S_THR2 = 4, S_DOBJ = 5 };

__host__ __device__ constexpr int ld_of(int N) { return N + 2; }   // padded row of an image buffer
// N = N1 N2 with N1 = 8 (4 at N = 16); the kernels' images need N in {16, 24, 32, 40, 48, 64}
__host__ __device__ constexpr int fac1(int N) { return N == 16 ? 4 : 8; }
__host__ __device__ constexpr int fac2(int N) { return N / fac1(N); }
__host__ __device__ constexpr int threads_of(int N) { return (N / 2) * fac1(N); }
// float2 slots of the twiddle tables: N base values, the N2 x N2 matrix and its conjugate (N2 <= 8)
__host__ __device__ constexpr int tw_elems(int N) { return N + 128; }
__host__ __device__ constexpr int max_slices(int N) { return N == 64 ? 3 : kMaxSlices; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// acc += d * w (CONJ: d * conj(w))
template <bool CONJ>
__device__ __forceinline__ void cmac(float2& acc, float2 d, float2 w) {
  if (!CONJ) {
    acc.x = fmaf(d.x, w.x, acc.x);
    acc.x = fmaf(-d.y, w.y, acc.x);
    acc.y = fmaf(d.x, w.y, acc.y);
    acc.y = fmaf(d.y, w.x, acc.y);
  } else {
    acc.x = fmaf(d.x, w.x, acc.x);
    acc.x = fmaf(d.y, w.y, acc.x);
    acc.y = fmaf(d.y, w.x, acc.y);
    acc.y = fmaf(-d.x, w.y, acc.y);
  }
}

// Wt[m] = exp(-2 pi i m / N) for m < N, computed in double and rounded once; then
// Wt[N + k2 N2 + c2] = Wt[(N1 k2 c2) mod N], the N2-point DFT matrix, and at Wt[N + 64 + ...]
// its conjugate.  Ends with a barrier.
template <int N>
__device__ void fill_twiddles(float2* Wt) {
  constexpr int N1 = fac1(N), N2 = fac2(N);
  for (int m = threadIdx.x; m < N; m += blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)m / (double)N, &s, &c);
    Wt[m] = make_float2((float)c, (float)s);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N2 * N2; e += blockDim.x) {
    const float2 w = Wt[(N1 * (e / N2) * (e % N2)) % N];
    Wt[N + e] = w;
    Wt[N + 64 + e] = make_float2(w.x, -w.y);
  }
  __syncthreads();
}

// The twiddles of one thread's bin c0: its row of the N1-point DFT and the twiddles between
// the two short DFTs in registers, the N2-point DFT matrix (the same for every thread) in
// shared memory.  conjugate() turns them into those of F^H (and back).
template <int N>
struct Twiddles {
  float2 w1[fac1(N)];   // exp(-2 pi i N2 k1 c0 / N), k1 < N1
  float2 tw[fac2(N)];   // exp(-2 pi i k2 c0 / N), k2 < N2
  const float2* w2;     // [k2][c2]: exp(-2 pi i N1 k2 c2 / N)
  const float2* w2c;    // its conjugate
  __device__ Twiddles(const float2* Wt, int c0) {
#pragma unroll
    for (int k1 = 0; k1 < fac1(N); ++k1) w1[k1] = Wt[(fac2(N) * k1 * c0) % N];
#pragma unroll
    for (int k2 = 0; k2 < fac2(N); ++k2) tw[k2] = Wt[(k2 * c0) % N];
    w2 = Wt + N;
    w2c = Wt + N + 64;
  }
  __device__ __forceinline__ void conjugate() {
#pragma unroll
    for (int k1 = 0; k1 < fac1(N); ++k1) w1[k1].y = -w1[k1].y;
#pragma unroll
    for (int k2 = 0; k2 < fac2(N); ++k2) tw[k2].y = -tw[k2].y;
    const float2* t = w2;
    w2 = w2c;
    w2c = t;
  }
};

// One pass: a[i][j] = element (r0 + i, c0 + N1 j) of D W, through
// X[c0 + N1 c2] = sum_k2 W_N2^(k2 c2) W_N^(k2 c0) sum_k1 W_N1^(k1 c0) x[N2 k1 + k2],
// with W_n = exp(-2 pi i / n) (conjugated twiddles: D conj(W)).  The threads of a bin read
// the same row words (broadcast).
template <int N>
__device__ __forceinline__ void dft_pass(const float2* __restrict__ D, const Twiddles<N>& tw,
                                         float2 (&a)[2][fac2(N)], int r0) {
  constexpr int LD = ld_of(N), N2 = fac2(N);
  float2 y[2][N2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int q = 0; q < N2; ++q) y[i][q] = make_float2(0.f, 0.f);
  const float2* d0 = D + r0 * LD;
  const float2* d1 = d0 + LD;
#pragma unroll
  for (int k = 0; k < N; k += 2) {   // x[k] = x[N2 k1 + k2]: k1 = k / N2, k2 = k % N2
    const float4 x0 = *reinterpret_cast<const float4*>(d0 + k);
    const float4 x1 = *reinterpret_cast<const float4*>(d1 + k);
    cmac<false>(y[0][k % N2], make_float2(x0.x, x0.y), tw.w1[k / N2]);
    cmac<false>(y[1][k % N2], make_float2(x1.x, x1.y), tw.w1[k / N2]);
    cmac<false>(y[0][(k + 1) % N2], make_float2(x0.z, x0.w), tw.w1[(k + 1) / N2]);
    cmac<false>(y[1][(k + 1) % N2], make_float2(x1.z, x1.w), tw.w1[(k + 1) / N2]);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int q = 0; q < N2; ++q) y[i][q] = cmul(y[i][q], tw.tw[q]);
#pragma unroll
  for (int c2 = 0; c2 < N2; ++c2) {
    float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < N2; ++q) {
      const float2 w = tw.w2[q * N2 + c2];
      cmac<false>(s0, y[0][q], w);
      cmac<false>(s1, y[1][q], w);
    }
    a[0][c2] = s0;
    a[1][c2] = s1;
  }
}

// O[c0 + N1 j][r0 + i] = a[i][j]: the transposed store that follows every pass.
template <int N>
__device__ __forceinline__ void store_t(float2* O, const float2 (&a)[2][fac2(N)], int r0, int c0) {
  constexpr int LD = ld_of(N);
#pragma unroll
  for (int j = 0; j < fac2(N); ++j)
    *reinterpret_cast<float4*>(O + (c0 + fac1(N) * j) * LD + r0) =
        make_float4(a[0][j].x, a[0][j].y, a[1][j].x, a[1][j].y);
}

// 2-D DFT of the image whose pixels (y, x) = (c0 + N1 j, r0 + i) are held in v (the pixels
// this thread owns); the result comes back in v at the same pixels.  inv: conjugate kernel
// (F^H, unnormalised).  Uses X (first pass) and Y (second) as scratch; begins and ends with
// all threads free to overwrite X.  The two passes share one copy of the pass code and the
// direction is a run-time flag: a kernel inlines this a few times only, which keeps its
// code within the instruction cache.
template <int N>
__device__ __forceinline__ void dft2(float2 (&v)[2][fac2(N)], float2* X, float2* Y, Twiddles<N>& tw, bool inv,
                                     int r0, int c0) {
  if (inv) tw.conjugate();
#pragma unroll 1
  for (int p = 0; p < 2; ++p) {
    float2* B = p ? Y : X;
    store_t<N>(B, v, r0, c0);
    __syncthreads();
    dft_pass<N>(B, tw, v, r0);
  }
  if (inv) tw.conjugate();
}

__host__ __device__ constexpr int owned(int N, int r0, int c0, int i, int j) { return (c0 + fac1(N) * j) * N + r0 + i; }

// v <- G v (adj: G^H v), G = F^-1 diag(h) F; h carries the 1/N^2 of F^-1.  One inlined
// 2-D DFT, run forward, then (after diag(h), or diag(conj h)) inverse.
template <int N>
__device__ __forceinline__ void propagate(float2 (&v)[2][fac2(N)], float2* X, float2* Y, Twiddles<N>& tw,
                                          const float2* __restrict__ h, bool adj, int r0, int c0) {
  const float hs = adj ? -1.f : 1.f;
#pragma unroll 1
  for (int d = 0; d < 2; ++d) {
    dft2<N>(v, X, Y, tw, d == 1, r0, c0);
    if (d == 0) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < fac2(N); ++j) {
          const float2 hv = __ldg(&h[owned(N, r0, c0, i, j)]);
          v[i][j] = cmul(v[i][j], make_float2(hv.x, hs * hv.y));
        }
    }
  }
}

// Fixed-order FP64 block sum (at least 32 threads): the first warp adds strided values in
// order, then a butterfly; every thread receives the total.  sh: blockDim.x + 1 doubles.
template <bool MAX = false>
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = MAX ? sh[threadIdx.x] : 0.0;
    for (int i = threadIdx.x + (MAX ? 32 : 0); i < (int)blockDim.x; i += 32) s = MAX ? fmax(s, sh[i]) : s + sh[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_xor_sync(0xffffffffu, s, off);
      s = MAX ? fmax(s, o) : s + o;
    }
    if (threadIdx.x == 0) sh[blockDim.x] = s;
  }
  __syncthreads();
  const double t = sh[blockDim.x];
  __syncthreads();
  return t;
}

template <int N>
constexpr size_t image_bytes() { return (size_t)N * ld_of(N) * sizeof(float2); }

// ---------------------------------------------------------------------------
// per-column kernels
// ---------------------------------------------------------------------------

// Matrix step, between the two contractions: for every column s of A P (summed over its
// `splits` partial products), U = F (A P)_s, the objective term and R = U - sqrt(I) U/|U|
// (U where |U|^2 <= thr2), then C_s = F^H R written over partial 0.
template <int N>
__global__ void __launch_bounds__(threads_of(N)) farfield_kernel(float2* BC, int splits, size_t split_stride,
                                                                 const float* __restrict__ I, int S,
                                                                 const double* __restrict__ scal,
                                                                 double* __restrict__ obj_part) {
  extern __shared__ float4 smem4[];
  float2* X = reinterpret_cast<float2*>(smem4);
  float2* Y = X + N * ld_of(N);
  float2* Wt = Y + N * ld_of(N);
  double* red = reinterpret_cast<double*>(Wt + tw_elems(N));
  constexpr int n2 = N * N;
  const int t = threadIdx.x, r0 = 2 * (t / fac1(N)), c0 = t % fac1(N);
  fill_twiddles<N>(Wt);
  Twiddles<N> tw(Wt, c0);
  const float thr2 = (float)scal[S_THR2];
  double obj = 0.0;
  for (int s = blockIdx.x; s < S; s += gridDim.x) {
    float2 v[2][fac2(N)];
    float4 acc[fac2(N)];   // the partials in split order, every split's loads in flight together
#pragma unroll
    for (int j = 0; j < fac2(N); ++j)
      acc[j] = *reinterpret_cast<const float4*>(BC + (size_t)s * n2 + owned(N, r0, c0, 0, j));
    for (int z = 1; z < splits; ++z) {
      const float2* Bz = BC + z * split_stride + (size_t)s * n2;
#pragma unroll
      for (int j = 0; j < fac2(N); ++j) {
        const float4 q = *reinterpret_cast<const float4*>(Bz + owned(N, r0, c0, 0, j));
        acc[j].x += q.x; acc[j].y += q.y; acc[j].z += q.z; acc[j].w += q.w;
      }
    }
#pragma unroll
    for (int j = 0; j < fac2(N); ++j) {
      v[0][j] = make_float2(acc[j].x, acc[j].y);
      v[1][j] = make_float2(acc[j].z, acc[j].w);
    }
    dft2<N>(v, X, Y, tw, false, r0, c0);
    float o = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < fac2(N); ++j) {
        const float meas = __ldg(&I[(size_t)s * n2 + owned(N, r0, c0, i, j)]);
        const float2 u = v[i][j];
        const float a2 = fmaf(u.x, u.x, u.y * u.y);
        const float a = sqrtf(a2);
        const float rt = sqrtf(meas);
        o = fmaf(rt - a, rt - a, o);
        const float f = (a2 > thr2) ? 1.f - rt / a : 1.f;
        v[i][j] = make_float2(u.x * f, u.y * f);
      }
    obj += (double)o;
    dft2<N>(v, X, Y, tw, true, r0, c0);
#pragma unroll
    for (int j = 0; j < fac2(N); ++j)
      *reinterpret_cast<float4*>(BC + (size_t)s * n2 + owned(N, r0, c0, 0, j)) =
          make_float4(v[0][j].x, v[0][j].y, v[1][j].x, v[1][j].y);
  }
  const double tot = block_sum(obj, red);
  if (threadIdx.x == 0) obj_part[blockIdx.x] = 0.5 * tot;
}

// Fixed-order sum of one complex value per thread (block of at least 32 threads); every
// thread receives the total.  red: blockDim.x + 1 float2.
__device__ float2 block_sum2(float2 v, float2* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float2 s = make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) {
      s.x += red[i].x;
      s.y += red[i].y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
    }
    if (threadIdx.x == 0) red[blockDim.x] = s;
  }
  __syncthreads();
  return red[blockDim.x];
}

// Index of pixel e = (y, x) relative to pixel col, cyclically: (y - yc) mod N, (x - xc) mod N.
__device__ __forceinline__ int rel_index(int N, int e, int col) {
  const int y = e / N - col / N, x = e % N - col % N;
  return (y < 0 ? y + N : y) * N + (x < 0 ? x + N : x);
}

// Multislice pass of a unit impulse at object pixel `col` through the slices o (M of them):
// v ends as column col of A(o) = O_M G ... G O_1.  The first propagation needs no DFT:
// G (o_1[col] e_col) = o_1[col] gk(. - col), gk = G e_0 the propagator's real-space kernel.
// Incident waves on slices 1..M-1 go to stash.
template <int N, bool STASH>
__device__ __forceinline__ void impulse_forward(float2 (&v)[2][fac2(N)], int col, int M, const float2* __restrict__ o,
                                                const float2* __restrict__ gk, const float2* __restrict__ h,
                                                float2* X, float2* Y, Twiddles<N>& tw, float2* stash,
                                                int r0, int c0) {
  constexpr int n2 = N * N;
  const float2 o0 = __ldg(&o[col]);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < fac2(N); ++j) {
      const int e = owned(N, r0, c0, i, j);
      v[i][j] = M == 1 ? (e == col ? o0 : make_float2(0.f, 0.f)) : cmul(o0, __ldg(&gk[rel_index(N, e, col)]));
    }
  for (int m = 1; m < M; ++m) {
    if (m > 1) propagate<N>(v, X, Y, tw, h, false, r0, c0);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < fac2(N); ++j) {
        const int e = owned(N, r0, c0, i, j);
        if (STASH) stash[(m - 1) * n2 + (i * fac2(N) + j) * threads_of(N) + threadIdx.x] = v[i][j];
        v[i][j] = cmul(v[i][j], __ldg(&o[(size_t)m * n2 + e]));
      }
  }
}

// Decomposition gradient: for every column j, m_j = lambda A(o)_j - Ahat_j and, for every
// slice l, the column's share (R_l^H m_j) o conj(S_l e_j) of diag(R_l^H M S_l^H).  Slice 0
// (S_0 = I) receives from column j one value only, at pixel j: it is written to g0[j].  The
// per-CTA sums of slices 1..M-1 go to gpart[cta][l-1][k]; the objective 1/2 sum |m_j|^2 to
// obj_part[cta].  Each CTA also writes max |o_m|^2 over its share of the pixels to
// maxpart[cta][m], for the proximal step sizes.
template <int N, int M>
__global__ void __launch_bounds__(threads_of(N)) grad_kernel(const float2* __restrict__ A,
                                                             const float2* __restrict__ o,
                                                             const float2* __restrict__ gk,
                                                             const float2* __restrict__ h,
                                                             const double* __restrict__ lam_p,
                                                             float2* __restrict__ g0,
                                                             float2* __restrict__ gpart,
                                                             double* __restrict__ obj_part,
                                                             float* __restrict__ maxpart) {
  constexpr int NA = M > 1 ? M - 1 : 1;   // accumulated slices 1..M-1
  extern __shared__ float4 smem4[];
  float2* X = reinterpret_cast<float2*>(smem4);
  float2* Y = X + N * ld_of(N);
  float2* Wt = Y + N * ld_of(N);
  float2* stash = Wt + tw_elems(N);   // [M-1][pixel slot (i, j)][thread]: each thread reads back its own
  double* red = reinterpret_cast<double*>(stash + (M - 1) * N * N);
  float2* red2 = reinterpret_cast<float2*>(red);
  constexpr int n2 = N * N;
  const int t = threadIdx.x, r0 = 2 * (t / fac1(N)), c0 = t % fac1(N);
  fill_twiddles<N>(Wt);
  Twiddles<N> tw(Wt, c0);
  {
    const int chunk = (n2 + gridDim.x - 1) / gridDim.x;
    const int k0 = blockIdx.x * chunk, k1 = min(n2, k0 + chunk);
    for (int m = 0; m < M; ++m) {
      float a = 0.f;
      for (int k = k0 + t; k < k1; k += blockDim.x) {
        const float2 v = __ldg(&o[(size_t)m * n2 + k]);
        a = fmaxf(a, fmaf(v.x, v.x, v.y * v.y));
      }
      const double mx = block_sum<true>((double)a, red);
      if (t == 0) maxpart[blockIdx.x * M + m] = (float)mx;
    }
  }
  const float lam = (float)lam_p[0];
  float2 acc[NA][2][fac2(N)];
#pragma unroll
  for (int q = 0; q < NA; ++q)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < fac2(N); ++j) acc[q][i][j] = make_float2(0.f, 0.f);
  double obj = 0.0;
  for (int col = blockIdx.x; col < n2; col += gridDim.x) {
    float2 v[2][fac2(N)];
    impulse_forward<N, true>(v, col, M, o, gk, h, X, Y, tw, stash, r0, c0);
    const float2* Aj = A + (size_t)col * n2;
    float ob = 0.f;
#pragma unroll
    for (int j = 0; j < fac2(N); ++j) {
      const float4 a = *reinterpret_cast<const float4*>(Aj + owned(N, r0, c0, 0, j));
      const float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
      v[0][j] = make_float2(fmaf(lam, v[0][j].x, -a0.x), fmaf(lam, v[0][j].y, -a0.y));
      v[1][j] = make_float2(fmaf(lam, v[1][j].x, -a1.x), fmaf(lam, v[1][j].y, -a1.y));
      ob = fmaf(v[0][j].x, v[0][j].x, fmaf(v[0][j].y, v[0][j].y, ob));
      ob = fmaf(v[1][j].x, v[1][j].x, fmaf(v[1][j].y, v[1][j].y, ob));
    }
    obj += (double)ob;
    // adjoint: chi_l = R_l^H m_j, from slice M-1 down to slice 1
#pragma unroll
    for (int l = M - 1; l >= 1; --l) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < fac2(N); ++j) {
          const int e = owned(N, r0, c0, i, j);
          const float2 g = cmulc(v[i][j], stash[(l - 1) * n2 + (i * fac2(N) + j) * threads_of(N) + threadIdx.x]);
          acc[l - 1][i][j].x += g.x;
          acc[l - 1][i][j].y += g.y;
          v[i][j] = cmulc(v[i][j], __ldg(&o[(size_t)l * n2 + e]));
        }
      if (l > 1) propagate<N>(v, X, Y, tw, h, true, r0, c0);
    }
    // slice 0: (G^H conj(o_1) chi_1)[col] = <G e_col, conj(o_1) chi_1>, or m_j[col] when M = 1
    float2 chi0 = make_float2(0.f, 0.f);
    if (M > 1) {
      float2 d = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < fac2(N); ++j) {
          const float2 p = cmulc(v[i][j], __ldg(&gk[rel_index(N, owned(N, r0, c0, i, j), col)]));
          d.x += p.x;
          d.y += p.y;
        }
      chi0 = block_sum2(d, red2);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < fac2(N); ++j)
        if (owned(N, r0, c0, i, j) == col) g0[col] = M > 1 ? chi0 : v[i][j];
  }
  if (M > 1) {
#pragma unroll
    for (int q = 0; q < NA; ++q)
#pragma unroll
      for (int j = 0; j < fac2(N); ++j)
        *reinterpret_cast<float4*>(gpart + ((size_t)blockIdx.x * NA + q) * n2 + owned(N, r0, c0, 0, j)) =
            make_float4(acc[q][0][j].x, acc[q][0][j].y, acc[q][1][j].x, acc[q][1][j].y);
  }
  const double tot = block_sum(obj, red);
  if (threadIdx.x == 0) obj_part[blockIdx.x] = 0.5 * tot;
}

// A(o) column by column, written as scale * A(o) into A.  HAVE_AHAT: A holds Ahat on entry;
// per CTA, Re <Ahat_j, A(o)_j> and ||A(o)_j||^2 are summed for the lambda update.
template <int N, bool HAVE_AHAT>
__global__ void __launch_bounds__(threads_of(N)) transfer_kernel(float2* A, const float2* __restrict__ o,
                                                                 const float2* __restrict__ gk,
                                                                 const float2* __restrict__ h, int M, float scale,
                                                                 double* __restrict__ dot_part,
                                                                 double* __restrict__ nrm_part) {
  extern __shared__ float4 smem4[];
  float2* X = reinterpret_cast<float2*>(smem4);
  float2* Y = X + N * ld_of(N);
  float2* Wt = Y + N * ld_of(N);
  double* red = reinterpret_cast<double*>(Wt + tw_elems(N));
  constexpr int n2 = N * N;
  const int t = threadIdx.x, r0 = 2 * (t / fac1(N)), c0 = t % fac1(N);
  fill_twiddles<N>(Wt);
  Twiddles<N> tw(Wt, c0);
  double dot = 0.0, nrm = 0.0;
  for (int col = blockIdx.x; col < n2; col += gridDim.x) {
    float2 v[2][fac2(N)];
    impulse_forward<N, false>(v, col, M, o, gk, h, X, Y, tw, nullptr, r0, c0);
    float2* Aj = A + (size_t)col * n2;
    float d = 0.f, q = 0.f;
#pragma unroll
    for (int j = 0; j < fac2(N); ++j) {
      float4* p = reinterpret_cast<float4*>(Aj + owned(N, r0, c0, 0, j));
      if (HAVE_AHAT) {
        const float4 a = *p;
        d = fmaf(a.x, v[0][j].x, fmaf(a.y, v[0][j].y, d));
        d = fmaf(a.z, v[1][j].x, fmaf(a.w, v[1][j].y, d));
        q = fmaf(v[0][j].x, v[0][j].x, fmaf(v[0][j].y, v[0][j].y, q));
        q = fmaf(v[1][j].x, v[1][j].x, fmaf(v[1][j].y, v[1][j].y, q));
      }
      *p = make_float4(scale * v[0][j].x, scale * v[0][j].y, scale * v[1][j].x, scale * v[1][j].y);
    }
    dot += (double)d;
    nrm += (double)q;
  }
  if (HAVE_AHAT) {
    const double td = block_sum(dot, red);
    const double tn = block_sum(nrm, red);
    if (threadIdx.x == 0) {
      dot_part[blockIdx.x] = td;
      nrm_part[blockIdx.x] = tn;
    }
  }
}

// Matrix-step set-up (one CTA): max_k |(F p)_k|^2, the sum of I from its partials, the
// squared zero-rule threshold and mu.
template <int N>
__global__ void __launch_bounds__(threads_of(N)) setup_kernel(const float2* __restrict__ probe,
                                                              const double* __restrict__ sum_part, int n_part,
                                                              double count, double step, double* scal,
                                                              double* mu_out) {
  extern __shared__ float4 smem4[];
  float2* X = reinterpret_cast<float2*>(smem4);
  float2* Y = X + N * ld_of(N);
  float2* Wt = Y + N * ld_of(N);
  double* red = reinterpret_cast<double*>(Wt + tw_elems(N));
  const int t = threadIdx.x, r0 = 2 * (t / fac1(N)), c0 = t % fac1(N);
  fill_twiddles<N>(Wt);
  Twiddles<N> tw(Wt, c0);
  float2 v[2][fac2(N)];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < fac2(N); ++j) v[i][j] = probe[owned(N, r0, c0, i, j)];
  dft2<N>(v, X, Y, tw, false, r0, c0);
  double mx = 0.0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < fac2(N); ++j) mx = fmax(mx, (double)v[i][j].x * v[i][j].x + (double)v[i][j].y * v[i][j].y);
  const double m = block_sum<true>(mx, red);
  double a = 0.0;
  for (int i = t; i < n_part; i += blockDim.x) a += sum_part[i];
  const double s = block_sum(a, red);
  if (t == 0) {
    scal[S_SPEC] = m;
    scal[S_SUMI] = s;
    scal[S_THR2] = kZeroTau * kZeroTau * s / count;
    const double mu = step > 0.0 ? step : (m > 0.0 ? 1.0 / ((double)(N * N) * m) : 0.0);
    scal[S_MU] = mu;
    if (mu_out) mu_out[0] = mu;
  }
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------

// P[:, s] = vec of the probe shifted cyclically by shifts[s] (Sec. 2.1).
// Grid: x over the pixels k of a column, y over the shifts s (each thread takes every
// gridDim.y-th shift).  The block first reduces its shifts modulo N into shared memory.
constexpr int kProbeShifts = 128;   // shifts per block at most: S <= 128 gridDim.y
__global__ void probe_matrix_kernel(const float2* __restrict__ probe, const int2* __restrict__ shifts, int N, int S,
                                    float2* __restrict__ P) {
  __shared__ int2 sh[kProbeShifts];
  const int mine = (S - (int)blockIdx.y + (int)gridDim.y - 1) / (int)gridDim.y;   // shifts of this block
  for (int i = threadIdx.x; i < mine; i += blockDim.x) {
    const int2 v = shifts[blockIdx.y + i * gridDim.y];
    int ys = v.x % N, xs = v.y % N;
    if (ys < 0) ys += N;
    if (xs < 0) xs += N;
    sh[i] = make_int2(ys, xs);
  }
  __syncthreads();
  const int n2 = N * N, k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n2) return;
  const int y = k / N, x = k - y * N;
#pragma unroll 4
  for (int i = 0; i < mine; ++i) {
    const int2 v = sh[i];
    int yy = y - v.x, xx = x - v.y;
    if (yy < 0) yy += N;
    if (xx < 0) xx += N;
    P[(size_t)(blockIdx.y + i * gridDim.y) * n2 + k] = __ldg(&probe[yy * N + xx]);
  }
}

// The propagator h[ky][kx] = exp(-i pi dz lambda (qy^2 + qx^2)) / N^2 = h1(ky) h1(kx) / N^2 and
// its real-space kernel gk = G e_0, gk[y][x] = g1(y) g1(x), g1(y) = (1/N) sum_k h1(k)
// exp(2 pi i k y / N), are outer products of one-dimensional factors: this kernel forms g1[y]
// and h1[y] in double (one block of one warp per y, spreading the FP64 work over N SMs: lanes
// take k = lane, lane + 32, then a butterfly sum), `kernel_column_kernel` the products.
__global__ void __launch_bounds__(32) kernel_row_kernel(double2* __restrict__ g1, double2* __restrict__ h1, int N,
                                                        double dzlam, double dq) {
  const int y = blockIdx.x, lane = threadIdx.x;
  double re = 0.0, im = 0.0;
  for (int k = lane; k < N; k += 32) {
    const double q = (k < N / 2 ? k : k - N) * dq;
    double s, c;
    sincospi(-dzlam * q * q + 2.0 * (double)((k * y) % N) / N, &s, &c);
    re += c;
    im += s;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  if (lane == 0) {
    g1[y] = make_double2(re / N, im / N);
    const double q = (y < N / 2 ? y : y - N) * dq;
    double s, c;
    sincospi(-dzlam * q * q, &s, &c);
    h1[y] = make_double2(c, s);
  }
}

// gk[y][x] = g1(y) g1(x) and h[ky][kx] = h1(ky) h1(kx) / N^2, in double, each rounded once.
__global__ void kernel_column_kernel(float2* __restrict__ gk, float2* __restrict__ h, const double2* __restrict__ g1,
                                     const double2* __restrict__ h1, int N) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const double2 a = g1[e / N], b = g1[e % N];
  gk[e] = make_float2((float)(a.x * b.x - a.y * b.y), (float)(a.x * b.y + a.y * b.x));
  const double2 u = h1[e / N], v = h1[e % N];
  const double inv = 1.0 / ((double)N * N);
  h[e] = make_float2((float)((u.x * v.x - u.y * v.y) * inv), (float)((u.x * v.y + u.y * v.x) * inv));
}

// Block partial sums of a float array over fixed chunks: FP32 within a thread (a few dozen
// terms), FP64 across the block.  Only the zero-rule threshold uses the total.
__global__ void __launch_bounds__(256) sum_part_kernel(const float* __restrict__ x, size_t n, double* __restrict__ part) {
  __shared__ double sh[257];
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  float a = 0.f;
#pragma unroll 8
  for (size_t i = b0 + threadIdx.x; i < b1; i += 256) a += __ldg(&x[i]);
  const double tot = block_sum((double)a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// out = sum of part[0..n) in a fixed order (one block of 256), written to scal[slot] and copy.
__global__ void __launch_bounds__(256) finish_sum_kernel(const double* __restrict__ part, int n, double* scal,
                                                         int slot, double* copy) {
  __shared__ double sh[257];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) a += part[i];
  const double s = block_sum(a, sh);
  if (threadIdx.x == 0) {
    scal[slot] = s;
    if (copy) copy[0] = s;
  }
}

// A += -mu * sum_z part_z (the rank-S update of the matrix step), float4 over element pairs.
__global__ void combine_kernel(float2* __restrict__ A, const float2* __restrict__ part, int splits, size_t stride,
                               size_t n_pairs, const double* __restrict__ scal) {
  const float a = (float)(-scal[S_MU]);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n_pairs; e += (size_t)gridDim.x * blockDim.x) {
    float4 s = reinterpret_cast<const float4*>(part)[e];
    for (int z = 1; z < splits; ++z) {
      const float4 q = reinterpret_cast<const float4*>(part + z * stride)[e];
      s.x += q.x; s.y += q.y; s.z += q.z; s.w += q.w;
    }
    float4 v = reinterpret_cast<float4*>(A)[e];
    v.x = fmaf(a, s.x, v.x);
    v.y = fmaf(a, s.y, v.y);
    v.z = fmaf(a, s.z, v.z);
    v.w = fmaf(a, s.w, v.w);
    reinterpret_cast<float4*>(A)[e] = v;
  }
}

// The proximal step (Eq. Prox_Min) before its normalisation.  Element e = l n2 + k of the
// slices (a block: 32 elements of one slice; n2 is a multiple of 32):
//   g_l[k]: slice 0 from g0, slices 1..M-1 summed in FP64 over the CTAs' partials in a fixed
//           order (8 groups of CTAs, cta mod 8, then the groups in order);
//   x = o_l[k] - mu_l lambda g_l[k] in FP64, mu_l = 1 / (lambda prod_{m != l} max|o_m|)^2,
//       written over o_l[k];
//   normpart[block] = sum of |x|^2 over the block's 32 elements (fixed order).
// max|o_m| comes from the CTAs' maxima (every block reduces them alike).  Block 0 also sums the
// decomposition objective into scal[S_DOBJ] (and obj_out).
__global__ void __launch_bounds__(256) grad_step_kernel(float2* __restrict__ o, const float2* __restrict__ g0,
                                                        const float2* __restrict__ gpart,
                                                        const float* __restrict__ maxpart, int n_cta, int M, int n2,
                                                        const double* __restrict__ lam_p,
                                                        const double* __restrict__ obj_part,
                                                        double* __restrict__ normpart, double* scal,
                                                        double* obj_out) {
  __shared__ double2 sh[8][32];
  __shared__ double red[257];
  __shared__ double maxo[kMaxSlices];
  const int t = threadIdx.x, lane = t & 31, grp = t >> 5;
  for (int m = 0; m < M; ++m) {
    float a = 0.f;
    for (int c = t; c < n_cta; c += 256) a = fmaxf(a, maxpart[c * M + m]);
    const double mx = block_sum<true>((double)a, red);
    if (t == 0) maxo[m] = sqrt(mx);
  }
  const int l = (blockIdx.x * 32) / n2, k = blockIdx.x * 32 - l * n2 + lane;
  const size_t na = (size_t)(M - 1) * n2;
  double re = 0.0, im = 0.0;
  if (l > 0)
#pragma unroll 4
    for (int c = grp; c < n_cta; c += 8) {
      const float2 v = gpart[(size_t)c * na + (size_t)(l - 1) * n2 + k];
      re += v.x;
      im += v.y;
    }
  sh[grp][lane] = make_double2(re, im);
  __syncthreads();
  if (grp == 0) {
    double2 g;
    if (l == 0) {
      g = make_double2(g0[k].x, g0[k].y);
    } else {
      g = sh[0][lane];
      for (int q = 1; q < 8; ++q) {
        g.x += sh[q][lane].x;
        g.y += sh[q][lane].y;
      }
    }
    const double lam = lam_p[0];
    double bound = fabs(lam);
    for (int m = 0; m < M; ++m)
      if (m != l) bound *= maxo[m];
    const double cstep = (bound > 0.0 ? 1.0 / (bound * bound) : 0.0) * lam;
    float2* p = o + (size_t)l * n2 + k;
    const double xr = (double)p->x - cstep * g.x, xi = (double)p->y - cstep * g.y;
    *p = make_float2((float)xr, (float)xi);
    double ss = xr * xr + xi * xi;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
    if (lane == 0) normpart[blockIdx.x] = ss;
  }
  if (blockIdx.x == 0) {
    double a = 0.0;
    for (int i = t; i < n_cta; i += 256) a += obj_part[i];
    const double tot = block_sum(a, red);
    if (t == 0) {
      scal[S_DOBJ] = tot;
      if (obj_out) obj_out[0] = tot;
    }
  }
}

// o_l = x_l / ||x_l||_F (Eq. Prox_Min) for slice l = blockIdx.y, ||x_l||^2 the fixed-order sum
// of its blocks' partials.
__global__ void __launch_bounds__(256) prox_kernel(float2* __restrict__ o, const double* __restrict__ normpart,
                                                   int n2) {
  __shared__ double red[257];
  const int l = blockIdx.y, nb = n2 / 32;
  double a = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) a += normpart[l * nb + i];
  const double nrm2 = block_sum(a, red);
  const float inv = nrm2 > 0.0 ? (float)(1.0 / sqrt(nrm2)) : 1.f;
  for (int k = blockIdx.x * 256 + threadIdx.x; k < n2; k += gridDim.x * 256) {
    float2* p = o + (size_t)l * n2 + k;
    *p = make_float2(p->x * inv, p->y * inv);
  }
}

// lambda = sum dot / sum nrm (Eq. Update Lambda, real part), partials in CTA order.
__global__ void __launch_bounds__(256) lambda_kernel(const double* __restrict__ dot_part,
                                                     const double* __restrict__ nrm_part, int n, double* lam) {
  __shared__ double sh[257];
  double d = 0.0, q = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    d += dot_part[i];
    q += nrm_part[i];
  }
  d = block_sum(d, sh);
  q = block_sum(q, sh);
  if (threadIdx.x == 0) lam[0] = q > 0.0 ? d / q : 0.0;
}

__global__ void scale_kernel(float4* __restrict__ A, size_t n4, const double* __restrict__ lam) {
  const float s = (float)lam[0];
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n4; e += (size_t)gridDim.x * blockDim.x) {
    float4 v = A[e];
    v.x *= s; v.y *= s; v.z *= s; v.w *= s;
    A[e] = v;
  }
}

// out_m = lambda^(1/M) o_m, principal root.
__global__ void final_slices_kernel(const float2* o, const double* __restrict__ lam, int M, size_t n, float2* out) {
  const double l = lam[0];
  const double r = pow(fabs(l), 1.0 / M);
  double s = 0.0, c = 1.0;
  if (l < 0.0) sincospi(1.0 / M, &s, &c);
  const float2 root = make_float2((float)(r * c), (float)(r * s));
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = cmul(o[e], root);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static msp_status fail(msp_status s, const std::string& m) { return set_last_error(s, m); }

#define SMD_CK(call)                                                                                  \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return fail(MSP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define SMD_LAUNCHED(n)                                                                                    \
  do {                                                                                                     \
    cudaError_t e_ = cudaGetLastError();                                                                   \
    if (e_ != cudaSuccess) return fail(MSP_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    count_launches(n);                                                                                     \
  } while (0)
#define SMD_TRY(expr)            \
  do {                           \
    msp_status s_ = (expr);      \
    if (s_ != MSP_OK) return s_; \
  } while (0)

static bool supported_n(int n) { return n == 16 || n == 24 || n == 32 || n == 40 || n == 48 || n == 64; }

static msp_status check(const msp_smd_geometry* g) {
  if (!g) return fail(MSP_EINVAL, "geometry is NULL");
  if (!supported_n(g->n)) return fail(MSP_EUNSUPPORTED, "N = " + std::to_string(g->n) + " (supported: 16, 24, 32, 40, 48, 64)");
  if (g->n_slices < 1) return fail(MSP_EINVAL, "n_slices < 1");
  if (g->n_slices > max_slices(g->n))
    return fail(MSP_EUNSUPPORTED, "at most " + std::to_string(max_slices(g->n)) + " slices for N = " + std::to_string(g->n));
  if (g->n_pos < 1) return fail(MSP_EINVAL, "n_pos < 1");
  if (!(std::isfinite(g->wavelength_A) && g->wavelength_A > 0)) return fail(MSP_EINVAL, "wavelength must be > 0");
  if (!(std::isfinite(g->pixel_A) && g->pixel_A > 0)) return fail(MSP_EINVAL, "pixel size must be > 0");
  if (!(std::isfinite(g->dz_A) && g->dz_A >= 0)) return fail(MSP_EINVAL, "propagation distance must be >= 0");
  if ((double)g->n * g->n * g->n_pos > 2.0e9) return fail(MSP_EUNSUPPORTED, "N^2 S too large");
  return MSP_OK;
}

// Dynamic shared memory of the per-column kernels.
static size_t image_smem(int N, int stash_planes, int threads) {
  return 2 * (size_t)N * ld_of(N) * sizeof(float2) + (size_t)tw_elems(N) * sizeof(float2) +
         (size_t)stash_planes * N * N * sizeof(float2) + (size_t)(threads + 1) * sizeof(double);
}

struct Dev {
  bool init = false;
  int sms = 0;
  int gemm_per_sm = 1;
};
static Dev g_dev[64];
static std::mutex g_mu;

template <int N>
struct Kernels {
  static constexpr int T = threads_of(N);
  static constexpr int MM = max_slices(N);
  static size_t smem_plain() { return image_smem(N, 0, T); }
  static size_t smem_grad(int M) { return image_smem(N, M - 1, T); }
  template <int M>
  static cudaError_t grad_attr(int* per_sm) {
    if constexpr (M <= max_slices(N)) {
      cudaError_t e = cudaFuncSetAttribute(grad_kernel<N, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem_grad(M));
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, grad_kernel<N, M>, T, smem_grad(M));
      return e;
    }
    return cudaSuccess;
  }
  static cudaError_t attrs(int* grad_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(farfield_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_plain());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(transfer_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_plain());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(transfer_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_plain());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(setup_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_plain());
    if (e == cudaSuccess) e = grad_attr<1>(&grad_per_sm[1]);
    if (e == cudaSuccess) e = grad_attr<2>(&grad_per_sm[2]);
    if (e == cudaSuccess) e = grad_attr<3>(&grad_per_sm[3]);
    if (e == cudaSuccess) e = grad_attr<4>(&grad_per_sm[4]);
    if (e == cudaSuccess) e = grad_attr<5>(&grad_per_sm[5]);
    return e;
  }
  static int per_sm_plain() {
    int k = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, farfield_kernel<N>, T, smem_plain());
    int k2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k2, transfer_kernel<N, true>, T, smem_plain());
    return std::max(1, std::min(k, k2));
  }
};

struct PerN {
  bool init = false;
  int plain = 1;                       // resident CTAs per SM of the plain per-column kernels
  int grad[kMaxSlices + 1] = {};       // ... of grad_kernel<N, M>
};
static PerN g_pern[64][65];

template <int N>
static msp_status init_n(int dev, PerN* out) {
  PerN& p = g_pern[dev][N];
  if (!p.init) {
    SMD_CK(Kernels<N>::attrs(p.grad));
    p.plain = Kernels<N>::per_sm_plain();
    for (int m = 1; m <= kMaxSlices; ++m) p.grad[m] = std::max(1, p.grad[m]);
    p.init = true;
  }
  *out = p;
  return MSP_OK;
}

static msp_status device(Dev* d, PerN* pn, int N) {
  int dev = 0;
  SMD_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(MSP_EUNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lk(g_mu);
  Dev& D = g_dev[dev];
  if (!D.init) {
    SMD_CK(cudaDeviceGetAttribute(&D.sms, cudaDevAttrMultiProcessorCount, dev));
    SMD_CK(cudaFuncSetAttribute(cgemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm::SMEM_BYTES));
    SMD_CK(cudaFuncSetAttribute(cgemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm::SMEM_BYTES));
    int k = 0, k2 = 0;
    SMD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, cgemm_kernel<false>, gemm::NTHREADS, gemm::SMEM_BYTES));
    SMD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k2, cgemm_kernel<true>, gemm::NTHREADS, gemm::SMEM_BYTES));
    D.gemm_per_sm = std::max(1, std::min(k, k2));
    // resident CTAs must never ask for more than the 512 TMEM columns of an SM (an allocation
    // that cannot be met waits)
    if (std::max(k, k2) * (int)gemm::TMEM_COLS > 512)
      return fail(MSP_EUNSUPPORTED, "tensor-memory budget: more resident contraction CTAs than TMEM allows");
    D.init = true;
  }
  *d = D;
  switch (N) {
    case 16: return init_n<16>(dev, pn);
    case 24: return init_n<24>(dev, pn);
    case 32: return init_n<32>(dev, pn);
    case 40: return init_n<40>(dev, pn);
    case 48: return init_n<48>(dev, pn);
    case 64: return init_n<64>(dev, pn);
  }
  return fail(MSP_EUNSUPPORTED, "N");
}

// Split of the K range of a contraction over `tiles` output tiles: the split count that
// minimises waves x (K-chunk + the cost of writing one partial tile, counted as 64 K),
// fewest splits on ties.
struct Split {
  int splits = 1, chunk = 0;
};
static Split choose_split(int tiles, int K, int slots, int max_splits) {
  Split best;
  long long best_cost = -1;
  for (int s = 1; s <= max_splits; ++s) {
    int chunk = (K + s - 1) / s;
    chunk = (chunk + gemm::TK - 1) / gemm::TK * gemm::TK;
    const int real = (K + chunk - 1) / chunk;
    if (real != s) continue;
    const long long waves = ((long long)tiles * s + slots - 1) / slots;
    const long long cost = waves * (chunk + 64);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best.splits = s;
      best.chunk = chunk;
    }
  }
  return best;
}

static int tiles_of(int M, int N) { return ((M + gemm::TM - 1) / gemm::TM) * ((N + gemm::TN - 1) / gemm::TN); }

struct Layout {
  int* err = nullptr;        // first word of the workspace: 2 = a tensor-core wait timed out
  double* scal = nullptr;
  double* part = nullptr;    // kPartSlots
  double* part2 = nullptr;   // kPartSlots
  float2* h = nullptr;
  float2* gk = nullptr;      // G e_0
  double2* g1 = nullptr;     // its separable factor, N values; the propagator's, N values from g1 + 64
  float2* P = nullptr;
  float2* BC = nullptr;      // splits1 * n2 * S
  float2* U = nullptr;       // splits2 * n2 * n2 (rank-S update partials)
  float2* g0 = nullptr;      // n2: slice-0 gradient, one value per column
  float2* gpart = nullptr;   // grid_grad * (M - 1) * n2
  float* maxpart = nullptr;  // grid_grad * M: per-CTA max |o_m|^2
  double* normpart = nullptr;  // M * n2 / 32: per-block |x|^2 of the proximal step
  Split s1, s2;
  int grid_plain = 1, grid_grad = 1, grid_ff = 1;
  size_t bytes = 0;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static Layout layout(const msp_smd_geometry* g, const Dev& d, const PerN& pn, char* base) {
  Layout w;
  const size_t n2 = (size_t)g->n * g->n, S = g->n_pos, M = g->n_slices;
  const int slots = d.gemm_per_sm * d.sms;
  w.s1 = choose_split(tiles_of((int)n2, (int)S), (int)n2, slots, 16);
  w.s2 = choose_split(tiles_of((int)n2, (int)n2), (int)S, slots, 4);
  const size_t cap = kPartSlots;
  w.grid_plain = (int)std::min({n2, (size_t)pn.plain * d.sms, cap});
  w.grid_grad = (int)std::min({n2, (size_t)pn.grad[M] * d.sms, cap});
  w.grid_ff = (int)std::min({S, (size_t)pn.plain * d.sms, cap});
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = base ? base + off : nullptr; off += align256(bytes); return p; };
  w.err = (int*)take(sizeof(int));
  w.scal = (double*)take(32 * sizeof(double));
  w.part = (double*)take(kPartSlots * sizeof(double));
  w.part2 = (double*)take(kPartSlots * sizeof(double));
  w.h = (float2*)take(n2 * sizeof(float2));
  w.gk = (float2*)take(n2 * sizeof(float2));
  w.g1 = (double2*)take(128 * sizeof(double2));
  w.P = (float2*)take(n2 * S * sizeof(float2));
  w.BC = (float2*)take((size_t)w.s1.splits * n2 * S * sizeof(float2));
  w.U = (float2*)take(w.s2.splits > 1 ? (size_t)w.s2.splits * n2 * n2 * sizeof(float2) : n2 * n2 * sizeof(float2));
  w.g0 = (float2*)take(n2 * sizeof(float2));
  w.gpart = (float2*)take((size_t)w.grid_grad * std::max<size_t>(M - 1, 1) * n2 * sizeof(float2));
  w.maxpart = (float*)take((size_t)w.grid_grad * M * sizeof(float));
  w.normpart = (double*)take(M * n2 / 32 * sizeof(double));
  w.bytes = off;
  return w;
}

struct Call {
  Dev dev;
  PerN pn;
  Layout w;
  cudaStream_t st = nullptr;
};

static bool misaligned(const void* p, size_t a) { return ((uintptr_t)p) % a != 0; }

static msp_status need(const void* p, const char* name) {
  if (!p) return fail(MSP_EINVAL, std::string(name) + " is NULL");
  if (misaligned(p, 16)) return fail(MSP_EINVAL, std::string(name) + " must be 16-byte aligned");
  return MSP_OK;
}

static msp_status begin(const msp_smd_geometry* g, void* ws, size_t ws_bytes, void* stream, Call* c) {
  SMD_TRY(check(g));
  SMD_TRY(refuse_untrusted_device());
  SMD_TRY(device(&c->dev, &c->pn, g->n));
  const size_t need_b = layout(g, c->dev, c->pn, nullptr).bytes;
  if (!ws) return fail(MSP_EINVAL, "workspace is NULL");
  if (misaligned(ws, 256)) return fail(MSP_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < need_b)
    return fail(MSP_EINVAL, "workspace too small: " + std::to_string(ws_bytes) + " < " + std::to_string(need_b));
  c->w = layout(g, c->dev, c->pn, (char*)ws);
  c->st = (cudaStream_t)stream;
  return MSP_OK;
}

static msp_status launch_propagator(const msp_smd_geometry* g, Call& c) {
  const int N = g->n;
  kernel_row_kernel<<<N, 32, 0, c.st>>>(c.w.g1, c.w.g1 + 64, N, g->dz_A * g->wavelength_A,
                                        1.0 / ((double)N * g->pixel_A));
  SMD_LAUNCHED(1);
  kernel_column_kernel<<<(N * N + 255) / 256, 256, 0, c.st>>>(c.w.gk, c.w.h, c.w.g1, c.w.g1 + 64, N);
  SMD_LAUNCHED(1);
  return MSP_OK;
}

template <int N>
static msp_status launch_transfer(const msp_smd_geometry* g, Call& c, float2* A, const float2* o, float scale,
                                  bool have_ahat) {
  const size_t sm = Kernels<N>::smem_plain();
  if (have_ahat)
    transfer_kernel<N, true><<<c.w.grid_plain, threads_of(N), sm, c.st>>>(A, o, c.w.gk, c.w.h, g->n_slices, scale,
                                                                          c.w.part, c.w.part2);
  else
    transfer_kernel<N, false><<<c.w.grid_plain, threads_of(N), sm, c.st>>>(A, o, c.w.gk, c.w.h, g->n_slices, scale,
                                                                           nullptr, nullptr);
  SMD_LAUNCHED(1);
  return MSP_OK;
}

template <int N>
static msp_status matrix_step_n(const msp_smd_geometry* g, Call& c, float2* A, const float2* probe,
                                const int2* shifts, const float* I, double step, double* obj_out) {
  const size_t n2 = (size_t)N * N, S = g->n_pos;
  const Layout& w = c.w;
  SMD_CK(cudaMemsetAsync(w.err, 0, sizeof(int), c.st));   // the call's own error word
  // every block takes at most kProbeShifts shifts: gridDim.y >= S / kProbeShifts
  const unsigned gy = (unsigned)std::min<size_t>(S, std::max<size_t>(128, (S + kProbeShifts - 1) / kProbeShifts));
  probe_matrix_kernel<<<dim3((unsigned)((n2 + 255) / 256), gy), 256, 0, c.st>>>(
      probe, shifts, N, (int)S, w.P);
  SMD_LAUNCHED(1);
  const int nsum = std::min(kPartSlots, 4 * c.dev.sms);
  sum_part_kernel<<<nsum, 256, 0, c.st>>>(I, n2 * S, w.part2);
  SMD_LAUNCHED(1);
  setup_kernel<N><<<1, threads_of(N), Kernels<N>::smem_plain(), c.st>>>(probe, w.part2, nsum, (double)(n2 * S), step,
                                                                        w.scal, nullptr);
  SMD_LAUNCHED(1);
  // A P: M = N^2, N = S, K = N^2
  dim3 g1((unsigned)((n2 + gemm::TM - 1) / gemm::TM), (unsigned)((S + gemm::TN - 1) / gemm::TN), (unsigned)w.s1.splits);
  SMD_TRY(profiled_launch(c.st, [&] {
    cgemm_kernel<false><<<g1, gemm::NTHREADS, gemm::SMEM_BYTES, c.st>>>((int)n2, (int)S, (int)n2, w.s1.chunk, A, n2,
                                                                         w.P, n2, w.BC, n2, n2 * S, w.err, tc_wait_limit());
    return cudaGetLastError();
  }));
  farfield_kernel<N><<<w.grid_ff, threads_of(N), Kernels<N>::smem_plain(), c.st>>>(w.BC, w.s1.splits, n2 * S, I,
                                                                                   (int)S, w.scal, w.part);
  SMD_LAUNCHED(1);
  finish_sum_kernel<<<1, 256, 0, c.st>>>(w.part, w.grid_ff, w.scal, S_OBJ, obj_out);
  SMD_LAUNCHED(1);
  // C P^H: M = N^2, N = N^2, K = S
  dim3 g2((unsigned)((n2 + gemm::TM - 1) / gemm::TM), (unsigned)((n2 + gemm::TN - 1) / gemm::TN), (unsigned)w.s2.splits);
  SMD_TRY(profiled_launch(c.st, [&] {
    cgemm_kernel<true><<<g2, gemm::NTHREADS, gemm::SMEM_BYTES, c.st>>>((int)n2, (int)n2, (int)S, w.s2.chunk, w.BC, n2,
                                                                        w.P, n2, w.U, n2, n2 * n2, w.err, tc_wait_limit());
    return cudaGetLastError();
  }));
  const size_t pairs = n2 * n2 / 2;
  combine_kernel<<<(int)std::min<size_t>((pairs + 255) / 256, (size_t)c.dev.sms * 16), 256, 0, c.st>>>(
      A, w.U, w.s2.splits, n2 * n2, pairs, w.scal);
  SMD_LAUNCHED(1);
  return MSP_OK;
}

template <int N, int M>
static cudaError_t launch_grad_m(Call& c, const float2* A, const float2* o, const double* lam) {
  if constexpr (M <= max_slices(N)) {
    const Layout& w = c.w;
    grad_kernel<N, M><<<w.grid_grad, threads_of(N), Kernels<N>::smem_grad(M), c.st>>>(A, o, w.gk, w.h, lam, w.g0,
                                                                                      w.gpart, w.part, w.maxpart);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

template <int N>
static msp_status launch_grad(int M, Call& c, const float2* A, const float2* o, const double* lam) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (M) {
    case 1: e = launch_grad_m<N, 1>(c, A, o, lam); break;
    case 2: e = launch_grad_m<N, 2>(c, A, o, lam); break;
    case 3: e = launch_grad_m<N, 3>(c, A, o, lam); break;
    case 4: e = launch_grad_m<N, 4>(c, A, o, lam); break;
    case 5: e = launch_grad_m<N, 5>(c, A, o, lam); break;
  }
  if (e != cudaSuccess) return fail(MSP_ECUDA, std::string("grad_kernel: ") + cudaGetErrorString(e));
  return MSP_OK;
}

template <int N>
static msp_status decompose_n(const msp_smd_geometry* g, Call& c, float2* A, float2* o, double* lam, double* obj_out) {
  const size_t n2 = (size_t)N * N;
  const int M = g->n_slices;
  const Layout& w = c.w;
  SMD_TRY(launch_propagator(g, c));
  SMD_TRY(launch_grad<N>(M, c, A, o, lam));
  SMD_LAUNCHED(1);
  grad_step_kernel<<<(int)(M * n2 / 32), 256, 0, c.st>>>(o, w.g0, w.gpart, w.maxpart, w.grid_grad, M, (int)n2, lam,
                                                        w.part, w.normpart, w.scal, obj_out);
  SMD_LAUNCHED(1);
  prox_kernel<<<dim3((unsigned)((n2 + 255) / 256), (unsigned)M), 256, 0, c.st>>>(o, w.normpart, (int)n2);
  SMD_LAUNCHED(1);
  SMD_TRY(launch_transfer<N>(g, c, A, o, 1.f, true));
  lambda_kernel<<<1, 256, 0, c.st>>>(w.part, w.part2, w.grid_plain, lam);
  SMD_LAUNCHED(1);
  const size_t n4 = n2 * n2 / 2;
  scale_kernel<<<(int)std::min<size_t>((n4 + 255) / 256, (size_t)c.dev.sms * 16), 256, 0, c.st>>>((float4*)A, n4, lam);
  SMD_LAUNCHED(1);
  return MSP_OK;
}

}  // namespace smd
}  // namespace msp

using namespace msp;
using namespace msp::smd;

#define SMD_DISPATCH(N_, CALL)          \
  switch (N_) {                         \
    case 16: { constexpr int N = 16; return CALL; } \
    case 24: { constexpr int N = 24; return CALL; } \
    case 32: { constexpr int N = 32; return CALL; } \
    case 40: { constexpr int N = 40; return CALL; } \
    case 48: { constexpr int N = 48; return CALL; } \
    case 64: { constexpr int N = 64; return CALL; } \
  }                                     \
  return fail(MSP_EUNSUPPORTED, "N");

extern "C" {

msp_status msp_smd_validate_geometry(const msp_smd_geometry* g) {
  set_last_error(MSP_OK, "");
  return check(g);
}

size_t msp_smd_workspace_bytes(const msp_smd_geometry* g) {
  if (check(g) != MSP_OK) return 0;
  Dev d;
  PerN pn;
  if (device(&d, &pn, g->n) != MSP_OK) return 0;
  return layout(g, d, pn, nullptr).bytes;
}

msp_status msp_smd_transfer(const msp_smd_geometry* g, const float* o, double lambda, float* A, void* ws,
                            size_t ws_bytes, void* stream) {
  set_last_error(MSP_OK, "");
  Call c;
  SMD_TRY(begin(g, ws, ws_bytes, stream, &c));
  SMD_TRY(need(o, "o"));
  SMD_TRY(need(A, "A"));
  if (!std::isfinite(lambda)) return fail(MSP_EINVAL, "lambda must be finite");
  SMD_TRY(launch_propagator(g, c));
  SMD_DISPATCH(g->n, (launch_transfer<N>(g, c, (float2*)A, (const float2*)o, (float)lambda, false)));
}

msp_status msp_smd_matrix_step(const msp_smd_geometry* g, float* A, const float* probe, const int32_t* shifts,
                               const float* I, double step, double* objective_before, double* mu_out, void* ws,
                               size_t ws_bytes, void* stream) {
  set_last_error(MSP_OK, "");
  Call c;
  SMD_TRY(begin(g, ws, ws_bytes, stream, &c));
  SMD_TRY(need(A, "A"));
  SMD_TRY(need(probe, "probe"));
  SMD_TRY(need(shifts, "shifts"));
  SMD_TRY(need(I, "I"));
  if (objective_before && misaligned(objective_before, 8)) return fail(MSP_EINVAL, "objective_before must be 8-byte aligned");
  if (mu_out && misaligned(mu_out, 8)) return fail(MSP_EINVAL, "mu_out must be 8-byte aligned");
  if (!std::isfinite(step)) return fail(MSP_EINVAL, "step must be finite");
  msp_status s = MSP_OK;
  switch (g->n) {
    case 16: s = matrix_step_n<16>(g, c, (float2*)A, (const float2*)probe, (const int2*)shifts, I, step, objective_before); break;
    case 24: s = matrix_step_n<24>(g, c, (float2*)A, (const float2*)probe, (const int2*)shifts, I, step, objective_before); break;
    case 32: s = matrix_step_n<32>(g, c, (float2*)A, (const float2*)probe, (const int2*)shifts, I, step, objective_before); break;
    case 40: s = matrix_step_n<40>(g, c, (float2*)A, (const float2*)probe, (const int2*)shifts, I, step, objective_before); break;
    case 48: s = matrix_step_n<48>(g, c, (float2*)A, (const float2*)probe, (const int2*)shifts, I, step, objective_before); break;
    case 64: s = matrix_step_n<64>(g, c, (float2*)A, (const float2*)probe, (const int2*)shifts, I, step, objective_before); break;
  }
  if (s != MSP_OK) return s;
  if (mu_out) SMD_CK(cudaMemcpyAsync(mu_out, c.w.scal + S_MU, sizeof(double), cudaMemcpyDeviceToDevice, c.st));
  return MSP_OK;
}

msp_status msp_smd_decompose(const msp_smd_geometry* g, float* A, float* o, double* lambda, double* objective_before,
                             void* ws, size_t ws_bytes, void* stream) {
  set_last_error(MSP_OK, "");
  Call c;
  SMD_TRY(begin(g, ws, ws_bytes, stream, &c));
  SMD_TRY(need(A, "A"));
  SMD_TRY(need(o, "o"));
  if (!lambda || misaligned(lambda, 8)) return fail(MSP_EINVAL, "lambda must be a non-NULL 8-byte aligned device double");
  if (objective_before && misaligned(objective_before, 8)) return fail(MSP_EINVAL, "objective_before must be 8-byte aligned");
  SMD_DISPATCH(g->n, (decompose_n<N>(g, c, (float2*)A, (float2*)o, lambda, objective_before)));
}

msp_status msp_smd_final_slices(const msp_smd_geometry* g, const float* o, const double* lambda, float* out,
                                void* stream) {
  set_last_error(MSP_OK, "");
  SMD_TRY(check(g));
  SMD_TRY(need(o, "o"));
  SMD_TRY(need(out, "out"));
  if (!lambda || misaligned(lambda, 8)) return fail(MSP_EINVAL, "lambda must be a non-NULL 8-byte aligned device double");
  const size_t n = (size_t)g->n_slices * g->n * g->n;
  final_slices_kernel<<<(int)std::min<size_t>((n + 255) / 256, 4096), 256, 0, (cudaStream_t)stream>>>(
      (const float2*)o, lambda, g->n_slices, n, (float2*)out);
  SMD_LAUNCHED(1);
  return MSP_OK;
}

}  // extern "C"
