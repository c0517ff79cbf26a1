// msp_learn.cu -- the learned-proposal form (include/msp_learn.h): a six-layer 3 x 3
// convolutional network in BF16 with FP32 accumulation on the tensor cores, its training step
// (backward pass and Adam) and its proposal.
//
// Every convolution is an implicit GEMM on tcgen05 (kind::f16, bf16 operands, FP32 accumulator
// in tensor memory):
//   forward / data gradient:  D[pixel][c_out] = sum_k A[pixel][k] B[c_out][k], k = 9-tap x c_in,
//     A gathered per K chunk of 64 from the NHWC activations (8 channels of one tap are 16
//     contiguous bytes), zero outside the image; B the packed weights.  One CTA per 128 pixels
//     of an image row.  The data gradient is the forward convolution of the gradient with the
//     weights mirrored in the taps and transposed in the channels.
//   weight gradient:  D[c_out][(tap, c_in)] = sum_p dPre[c_out][p] in[c_in][p + tap], K = the
//     pixels of one image row per CTA, operands from the channel-major (CHW) copies every
//     layer also writes; the per-row partial sums are added in a fixed order.
// Operands are staged through shared memory in the canonical no-swizzle K-major layout
// (core matrices of 8 rows x 16 bytes); one thread issues the MMAs and commits them to an
// mbarrier whose bounded wait records a timeout in the error word.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "msp.h"
#include "msp_learn.h"
#include "msp_tc.cuh"

namespace msp {

msp_status set_last_error(msp_status s, const std::string& m);
msp_status refuse_untrusted_device();
void count_launches(int n);
int tc_wait_limit();

namespace learn {

using bf16 = __nv_bfloat16;
constexpr int kLayers = 6;
constexpr int kHid = 64;
constexpr int kPix = 128;      // pixels per CTA (M)
constexpr int kKC = 64;        // K per chunk
constexpr int kThreads = 256;
constexpr int kDrainLimit = 1 << 20;

enum Epi { EPI_NONE = 0, EPI_GELU = 1, EPI_GELU_GRAD = 2 };

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__host__ __device__ constexpr int kchunks(int cin) { return (9 * cin + kKC - 1) / kKC; }

// ---------------------------------------------------------------------------
// forward / data-gradient convolution
// ---------------------------------------------------------------------------
// in  [H][Wd][CIN] bf16; B packed: kchunks(CIN) blocks of COUT x 64 bf16 (canonical layout).
// pre (FP32 [H][Wd][COUT], may be NULL) receives D + bias (bias[c] for c < nbias, else 0).  EPI_GELU: out = gelu(pre) in bf16,
// NHWC and CHW.  EPI_GELU_GRAD: out = D * gelu'(aux) (aux FP32 [H][Wd][COUT]), NHWC and CHW.
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(kThreads, 1) conv_kernel(const bf16* __restrict__ in, const bf16* __restrict__ Bp,
                                                           const float* __restrict__ bias, const float* __restrict__ aux,
                                                           float* __restrict__ pre, bf16* __restrict__ out,
                                                           bf16* __restrict__ out_chw, int nbias, int H, int Wd,
                                                           int* err, int wait_limit) {
  constexpr int NC = kchunks(CIN);
  constexpr uint32_t A_BYTES = kPix * kKC * 2, B_BYTES = COUT * kKC * 2;
  constexpr uint32_t TCOLS = COUT < 32 ? 32 : COUT;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sa = smem;
  uint8_t* sb = sa + A_BYTES;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sb + B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  volatile int* flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int y = blockIdx.y, x0 = blockIdx.x * kPix;
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
    *flag = 0;
  }
  if (warp == 0) tc::tmem_alloc(tslot, TCOLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::idesc_bf16(kPix, COUT);
  int issued = -1;
#pragma unroll 1
  for (int c = 0; c < NC; ++c) {
    if (c > 0) {
      if (tid == 0 && !tc::wait_phase(bar, (uint32_t)((c - 1) & 1), wait_limit)) *flag = 2;
      __syncthreads();
      if (*flag) break;
    }
    // A: 128 pixels x 64 K, 16-byte pieces (8 channels of one tap)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // 1024 pieces; eight consecutive threads take eight rows of one core matrix (no bank conflict)
      const int piece = tid + kThreads * i;
      const int r = (piece & 7) | ((piece >> 6) << 3), q = (piece >> 3) & 7;
      const int k0 = c * kKC + 8 * q;
      const int t = k0 / CIN, ci = k0 % CIN;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (t < 9) {
        const int yy = y + t / 3 - 1, xx = x0 + r + t % 3 - 1;
        if (yy >= 0 && yy < H && xx >= 0 && xx < Wd)
          v = *reinterpret_cast<const uint4*>(in + ((size_t)yy * Wd + xx) * CIN + ci);
      }
      *reinterpret_cast<uint4*>(sa + tc::kmaj16(r, 8 * q)) = v;
    }
    // B: the packed chunk
    {
      const uint4* src = reinterpret_cast<const uint4*>(Bp + (size_t)c * COUT * kKC);
      for (int i = tid; i < (int)(B_BYTES / 16); i += kThreads) reinterpret_cast<uint4*>(sb)[i] = src[i];
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t a = tc::smem_u32(sa), b = tc::smem_u32(sb);
#pragma unroll
      for (int s = 0; s < kKC / 16; ++s)
        tc::mma_bf16(tmem, tc::smem_desc(a + s * 256, 128, 1024), tc::smem_desc(b + s * 256, 128, 1024), idesc,
                     (c > 0 || s > 0) ? 1u : 0u);
      tc::commit(bar);
    }
    issued = c;
  }
  if (!*flag && issued == NC - 1) {
    if (tid == 0 && !tc::wait_phase(bar, (uint32_t)((NC - 1) & 1), wait_limit)) *flag = 2;
  }
  __syncthreads();
  tc::fence_after();
  if (!*flag && warp < 4) {
    const int r = 32 * warp + lane;
    const int x = x0 + r;
    const bool ok = x < Wd;
    const size_t p = (size_t)y * Wd + x;
#pragma unroll 1
    for (int j0 = 0; j0 < COUT; j0 += 16) {
      uint32_t d[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)j0, d);
      tc::tmem_wait_ld();
      if (!ok) continue;
      float v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = __uint_as_float(d[u]) + (j0 + u < nbias ? bias[j0 + u] : 0.f);
      if (pre) {
        float4* dst = reinterpret_cast<float4*>(pre + p * COUT + j0);
#pragma unroll
        for (int u = 0; u < 4; ++u) dst[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
      }
      if (EPI != EPI_NONE) {
        __align__(16) bf16 o[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const float a = EPI == EPI_GELU ? gelu(v[u]) : v[u] * gelu_grad(aux[p * COUT + j0 + u]);
          o[u] = __float2bfloat16_rn(a);
          out_chw[(size_t)(j0 + u) * H * Wd + p] = o[u];
        }
        uint4* dst = reinterpret_cast<uint4*>(out + p * COUT + j0);
        dst[0] = reinterpret_cast<const uint4*>(o)[0];
        dst[1] = reinterpret_cast<const uint4*>(o)[1];
      }
    }
  }
  if (tid == 0 && *flag && issued >= 0 && !tc::wait_phase(bar, (uint32_t)(issued & 1), kDrainLimit)) *flag = 3;
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, TCOLS);
  }
  if (tid == 0 && *flag) atomicMax(err, *flag);
}

template <int CIN, int COUT>
constexpr size_t conv_smem() {
  return 1024 + (size_t)kPix * kKC * 2 + (size_t)COUT * kKC * 2 + 64;
}

// ---------------------------------------------------------------------------
// weight gradient: D[c_out][n = tap CIN + c_in] over the pixels of one image row
// ---------------------------------------------------------------------------
// g_chw [COUT][H Wd], in_chw [CIN][H Wd] (bf16).  Partial sums [H][COUT][9 CIN] (FP32): row y of
// the image contributes its pixels.  N tile NT = 9 CIN / n_tiles, rows of A beyond COUT are zero.
template <int CIN, int COUT>
struct WG {
  static constexpr int N = 9 * CIN;
  static constexpr int NTILES = N <= 256 ? 1 : 3;
  static constexpr int NT = N / NTILES;   // 144 (CIN = 16) or 192 (CIN = 64)
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads, 1) wgrad_kernel(const bf16* __restrict__ g_chw, const bf16* __restrict__ in_chw,
                                                            float* __restrict__ part, int H, int Wd, int* err,
                                                            int wait_limit) {
  constexpr int NT = WG<CIN, COUT>::NT, N = WG<CIN, COUT>::N;
  constexpr uint32_t A_BYTES = kPix * kKC * 2, B_BYTES = NT * kKC * 2;
  constexpr uint32_t TCOLS = 256;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sa = smem;
  uint8_t* sb = sa + A_BYTES;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sb + B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  volatile int* flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int y = blockIdx.x, tile = blockIdx.y;
  const size_t P = (size_t)H * Wd;
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
    *flag = 0;
  }
  // rows of A beyond COUT stay zero for the whole kernel
  for (int i = tid; i < (int)(A_BYTES / 16); i += kThreads) reinterpret_cast<uint4*>(sa)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) tc::tmem_alloc(tslot, TCOLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::idesc_bf16(kPix, NT);
  const int NC = Wd / kKC;
  int issued = -1;
#pragma unroll 1
  for (int c = 0; c < NC; ++c) {
    if (c > 0) {
      if (tid == 0 && !tc::wait_phase(bar, (uint32_t)((c - 1) & 1), wait_limit)) *flag = 2;
      __syncthreads();
      if (*flag) break;
    }
    const int p0 = c * kKC;   // column of the image row
    // A: rows c_out < COUT, 64 pixels: 8 pieces of 16 bytes each
    for (int piece = tid; piece < COUT * 8; piece += kThreads) {
      const int r = piece >> 3, q = piece & 7;
      const uint4 v = *reinterpret_cast<const uint4*>(g_chw + (size_t)r * P + (size_t)y * Wd + p0 + 8 * q);
      *reinterpret_cast<uint4*>(sa + tc::kmaj16(r, 8 * q)) = v;
    }
    // B: rows n = tap CIN + c_in of this tile, 64 pixels shifted by the tap (zero outside)
    for (int piece = tid; piece < NT * 8; piece += kThreads) {
      const int rr = piece >> 3, q = piece & 7;
      const int n = tile * NT + rr;
      const int t = n / CIN, ci = n % CIN;
      const int yy = y + t / 3 - 1, dx = t % 3 - 1;
      __align__(16) bf16 v[8];
      const int xs = p0 + 8 * q + dx;
      if (yy < 0 || yy >= H) {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16_rn(0.f);
      } else if (dx == 0) {
        *reinterpret_cast<uint4*>(v) = *reinterpret_cast<const uint4*>(in_chw + (size_t)ci * P + (size_t)yy * Wd + xs);
      } else {
        const bf16* row = in_chw + (size_t)ci * P + (size_t)yy * Wd;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int xx = xs + e;
          v[e] = (xx >= 0 && xx < Wd) ? row[xx] : __float2bfloat16_rn(0.f);
        }
      }
      *reinterpret_cast<uint4*>(sb + tc::kmaj16(rr, 8 * q)) = *reinterpret_cast<const uint4*>(v);
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t a = tc::smem_u32(sa), b = tc::smem_u32(sb);
#pragma unroll
      for (int s = 0; s < kKC / 16; ++s)
        tc::mma_bf16(tmem, tc::smem_desc(a + s * 256, 128, 1024), tc::smem_desc(b + s * 256, 128, 1024), idesc,
                     (c > 0 || s > 0) ? 1u : 0u);
      tc::commit(bar);
    }
    issued = c;
  }
  if (!*flag && issued == NC - 1) {
    if (tid == 0 && !tc::wait_phase(bar, (uint32_t)((NC - 1) & 1), wait_limit)) *flag = 2;
  }
  __syncthreads();
  tc::fence_after();
  if (!*flag && warp < 4 && 32 * warp < COUT) {
    const int co = 32 * warp + lane;
#pragma unroll 1
    for (int j0 = 0; j0 < NT; j0 += 16) {
      uint32_t d[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)j0, d);
      tc::tmem_wait_ld();
      if (co < COUT) {
        float* dst = part + ((size_t)y * COUT + co) * N + tile * NT + j0;
#pragma unroll
        for (int u = 0; u < 16; ++u) dst[u] = __uint_as_float(d[u]);
      }
    }
  }
  if (tid == 0 && *flag && issued >= 0 && !tc::wait_phase(bar, (uint32_t)(issued & 1), kDrainLimit)) *flag = 3;
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, TCOLS);
  }
  if (tid == 0 && *flag) atomicMax(err, *flag);
}

// At least 90 KB so that no more than two CTAs (2 x 256 TMEM columns) share an SM.
template <int CIN>
constexpr size_t wgrad_smem() {
  return 1024 + (size_t)kPix * kKC * 2 + (size_t)WG<CIN, 16>::NT * kKC * 2 + 64 > 90 * 1024
             ? 1024 + (size_t)kPix * kKC * 2 + (size_t)WG<CIN, 16>::NT * kKC * 2 + 64
             : 90 * 1024;
}

// dW[co][n] (n = tap CIN + c_in, valid c_in < cin_true) = sum over image rows of part, in row order;
// written to the parameter layout [co][9][cin_true] of rows co < cout_true.
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int H, int COUT, int CIN, int cout_true,
                                    int cin_true, float* __restrict__ dW) {
  const int N = 9 * CIN;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= cout_true * N) return;
  const int co = idx / N, n = idx % N;
  const int t = n / CIN, ci = n % CIN;
  if (ci >= cin_true) return;
  float s = 0.f;
  for (int y = 0; y < H; ++y) s += part[((size_t)y * COUT + co) * N + n];
  dW[((size_t)co * 9 + t) * cin_true + ci] = s;
}

// db[co] = sum over pixels of g[p][co] (NHWC bf16, COUT channels), per-block partials in a fixed
// order: block b sums rows of pixels b, b + gridDim.x, ... into part[b][co]; then row order.
__global__ void bias_grad_part_kernel(const bf16* __restrict__ g, size_t P, int COUT, float* __restrict__ part) {
  __shared__ float acc[256];
  const int co = threadIdx.x % COUT, lanes = blockDim.x / COUT, li = threadIdx.x / COUT;
  float s = 0.f;
  for (size_t p = (size_t)blockIdx.x * lanes + li; p < P; p += (size_t)gridDim.x * lanes)
    s += __bfloat162float(g[p * COUT + co]);
  acc[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < COUT) {
    float t = 0.f;
    for (int i = 0; i < lanes; ++i) t += acc[i * COUT + threadIdx.x];
    part[(size_t)blockIdx.x * COUT + threadIdx.x] = t;
  }
}
__global__ void bias_grad_sum_kernel(const float* __restrict__ part, int nb, int COUT, int cout_true, float* __restrict__ db) {
  const int co = threadIdx.x;
  if (co >= cout_true) return;
  float s = 0.f;
  for (int b = 0; b < nb; ++b) s += part[(size_t)b * COUT + co];
  db[co] = s;
}

// ---------------------------------------------------------------------------
// packing, input, output, loss, Adam, initialisation
// ---------------------------------------------------------------------------

// B operand of the forward convolution from w [cout_true][9][cin_true] FP32: chunk c, row co
// (< COUT), k = tap CIN + ci; zero for padded channels and taps >= 9.
__global__ void pack_fwd_kernel(const float* __restrict__ w, int cin_true, int cout_true, int CIN, int COUT,
                                bf16* __restrict__ Bp) {
  const int NC = (9 * CIN + kKC - 1) / kKC;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NC * COUT * kKC) return;
  const int c = idx / (COUT * kKC), rem = idx % (COUT * kKC);
  const int co = rem / kKC, kk = rem % kKC;
  const int k = c * kKC + kk, t = k / CIN, ci = k % CIN;
  float v = 0.f;
  if (t < 9 && ci < cin_true && co < cout_true) v = w[((size_t)co * 9 + t) * cin_true + ci];
  Bp[(size_t)c * COUT * kKC + tc::kmaj16(co, kk) / 2] = __float2bfloat16_rn(v);
}

// B operand of the data-gradient convolution: rows ci (< CIN of the layer), k = tap' COUT + co,
// value w[co][8 - tap'][ci] (taps mirrored, channels transposed).
__global__ void pack_dgrad_kernel(const float* __restrict__ w, int cin_true, int cout_true, int CIN, int COUT,
                                  bf16* __restrict__ Bp) {
  const int NC = (9 * COUT + kKC - 1) / kKC;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NC * CIN * kKC) return;
  const int c = idx / (CIN * kKC), rem = idx % (CIN * kKC);
  const int ci = rem / kKC, kk = rem % kKC;
  const int k = c * kKC + kk, t = k / COUT, co = k % COUT;
  float v = 0.f;
  if (t < 9 && ci < cin_true && co < cout_true) v = w[((size_t)co * 9 + (8 - t)) * cin_true + ci];
  Bp[(size_t)c * CIN * kKC + tc::kmaj16(ci, kk) / 2] = __float2bfloat16_rn(v);
}

// Network input: x[p][c] = s_V V_c (c < L), s_G G_{c-L} (L <= c < 2L), 0 up to 16; NHWC and CHW.
__global__ void input_kernel(const float* __restrict__ V, const float* __restrict__ G, int L, size_t P, float sv,
                             float sg, bf16* __restrict__ x, bf16* __restrict__ x_chw) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * 16; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i / 16;
    const int c = (int)(i % 16);
    float v = 0.f;
    if (c < L) v = sv * V[(size_t)c * P + p];
    else if (c < 2 * L) v = sg * G[(size_t)(c - L) * P + p];
    const bf16 b = __float2bfloat16_rn(v);
    x[i] = b;
    x_chw[(size_t)c * P + p] = b;
  }
}

// Proposal dV[l][p] = s_D pre[p][l] (l < L) from the last layer's FP32 pre-activation [P][16].
__global__ void output_kernel(const float* __restrict__ pre, int L, size_t P, float sd, float* __restrict__ dV) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * L; i += (size_t)gridDim.x * blockDim.x) {
    const size_t l = i / P, p = i % P;
    dV[i] = sd * pre[p * 16 + l];
  }
}

// Mean squared error against target / s_D and its gradient with respect to the last layer's
// pre-activation (bf16, NHWC and CHW, padded channels 0); per-block loss partials (FP64).
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ pre, const float* __restrict__ target, int L,
                                                   size_t P, float inv_sd, bf16* __restrict__ g, bf16* __restrict__ g_chw,
                                                   double* __restrict__ part) {
  __shared__ double red[8];
  const double inv_n = 1.0 / ((double)P * L);
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * 16; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i / 16;
    const int c = (int)(i % 16);
    float gv = 0.f;
    if (c < L) {
      const float d = pre[i] - inv_sd * target[(size_t)c * P + p];
      acc += (double)d * d;
      gv = (float)(2.0 * inv_n) * d;
    }
    const bf16 b = __float2bfloat16_rn(gv);
    g[i] = b;
    g_chw[(size_t)c * P + p] = b;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    part[blockIdx.x] = s * inv_n;
  }
}

__global__ void loss_sum_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    out[0] = s;
  }
}

// NHWC -> CHW copy of a bf16 image (the weight-gradient test hook).
__global__ void to_chw_kernel(const bf16* __restrict__ in, size_t P, int C, bf16* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P * C; i += (size_t)gridDim.x * blockDim.x)
    out[(i % C) * P + i / C] = in[i];
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, size_t n, float lr, float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
  }
}

// Counter-based uniform in [-1, 1) from (seed, index): the 64-bit finaliser of splitmix64.
__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}
__global__ void init_kernel(float* __restrict__ params, size_t off, size_t nw, size_t nb, float bound, uint64_t seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nw + nb; i += (size_t)gridDim.x * blockDim.x)
    params[off + i] = i < nw ? bound * hash_uniform(seed, off + i) : 0.f;
}

// Candidate potentials Vc = V + dV.
__global__ void candidate_kernel(const float* __restrict__ V, const float* __restrict__ dV, size_t n,
                                 float* __restrict__ Vc) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    Vc[i] = V[i] + dV[i];
}

// The acceptance rule: V <- Vc where the loss at Vc is below the loss at V (loss[1] < loss[0];
// a NaN loss is never below), and accepted = 1 or 0.
__global__ void select_kernel(const double* __restrict__ loss, const float* __restrict__ Vc, size_t n,
                              float* __restrict__ V, int32_t* __restrict__ accepted) {
  const bool take = loss[1] < loss[0];
  if (blockIdx.x == 0 && threadIdx.x == 0 && accepted) *accepted = take ? 1 : 0;
  if (!take) return;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    V[i] = Vc[i];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Layer {
  int cin_true, cout_true;   // channels in the parameter layout
  int cin, cout;             // padded channels of the kernels (16 or 64)
  size_t w_off, b_off;       // offsets in the parameter array
};

struct Net {
  Layer layer[kLayers];
  size_t n_params = 0;
};

Net make_net(int L) {
  Net n;
  const int ct[kLayers + 1] = {2 * L, kHid, kHid, kHid, kHid, kHid, L};
  size_t off = 0;
  for (int i = 0; i < kLayers; ++i) {
    Layer& l = n.layer[i];
    l.cin_true = ct[i];
    l.cout_true = ct[i + 1];
    l.cin = ct[i] <= 16 ? 16 : 64;
    l.cout = ct[i + 1] <= 16 ? 16 : 64;
    l.w_off = off;
    off += (size_t)l.cout_true * 9 * l.cin_true;
    l.b_off = off;
    off += (size_t)l.cout_true;
  }
  n.n_params = off;
  return n;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
size_t packed_fwd_elems(const Layer& l) { return (size_t)kchunks(l.cin) * l.cout * kKC; }
size_t packed_dgrad_elems(const Layer& l) { return (size_t)kchunks(l.cout) * l.cin * kKC; }

struct Ws {
  int* err;
  double* loss_part;            // [512]
  bf16* x;                      // [P][16] input, NHWC
  bf16* x_chw;                  // [16][P]
  bf16* act[kLayers - 1];       // [P][64] outputs of the hidden layers (gelu), NHWC
  bf16* act_chw[kLayers - 1];   // [64][P]
  float* pre[kLayers];          // [P][cout] pre-activations (FP32)
  bf16* g[2];                   // [P][64] gradients of a pre-activation, NHWC (ping-pong)
  bf16* g_chw[2];               // [64][P]
  bf16* Bf[kLayers];            // packed forward weights
  bf16* Bd[kLayers];            // packed data-gradient weights
  float* part;                  // [H][64][576] weight-gradient partials
  float* bpart;                 // [512][64] bias-gradient partials
  float* grad;                  // [n_params]
  size_t bytes;
};

Ws carve(const Net& n, int H, int Wd, char* base) {
  Ws w{};
  size_t off = 0;
  auto take = [&](size_t b) { char* q = base ? base + off : nullptr; off += align256(b); return (void*)q; };
  const size_t P = (size_t)H * Wd;
  w.err = (int*)take(sizeof(int));
  w.loss_part = (double*)take(512 * sizeof(double));
  w.x = (bf16*)take(P * 16 * 2);
  w.x_chw = (bf16*)take(P * 16 * 2);
  for (int i = 0; i < kLayers - 1; ++i) {
    w.act[i] = (bf16*)take(P * kHid * 2);
    w.act_chw[i] = (bf16*)take(P * kHid * 2);
  }
  for (int i = 0; i < kLayers; ++i) w.pre[i] = (float*)take(P * n.layer[i].cout * 4);
  for (int i = 0; i < 2; ++i) {
    w.g[i] = (bf16*)take(P * kHid * 2);
    w.g_chw[i] = (bf16*)take(P * kHid * 2);
  }
  for (int i = 0; i < kLayers; ++i) {
    w.Bf[i] = (bf16*)take(packed_fwd_elems(n.layer[i]) * 2);
    w.Bd[i] = (bf16*)take(packed_dgrad_elems(n.layer[i]) * 2);
  }
  w.part = (float*)take((size_t)H * kHid * 9 * kHid * 4);
  w.bpart = (float*)take(512 * kHid * 4);
  w.grad = (float*)take(n.n_params * 4);
  w.bytes = off;
  return w;
}

msp_status fail(msp_status s, const std::string& m) { return set_last_error(s, m); }

template <int CIN, int COUT, int EPI>
cudaError_t launch_conv(const bf16* in, const bf16* Bp, const float* bias, const float* aux, float* pre, bf16* out,
                        bf16* out_chw, int nbias, int H, int Wd, int* err, cudaStream_t st) {
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(conv_kernel<CIN, COUT, EPI>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem<CIN, COUT>());
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  conv_kernel<CIN, COUT, EPI><<<dim3((unsigned)(Wd / kPix), (unsigned)H), kThreads, conv_smem<CIN, COUT>(), st>>>(
      in, Bp, bias, aux, pre, out, out_chw, nbias, H, Wd, err, tc_wait_limit());
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t conv(int cin, int cout, int epi, const bf16* in, const bf16* Bp, const float* bias, const float* aux,
                 float* pre, bf16* out, bf16* out_chw, int nbias, int H, int Wd, int* err, cudaStream_t st) {
#define MSP_CONV(CI, CO, E) \
  if (cin == CI && cout == CO && epi == E) return launch_conv<CI, CO, E>(in, Bp, bias, aux, pre, out, out_chw, nbias, H, Wd, err, st);
  MSP_CONV(16, 64, EPI_GELU)
  MSP_CONV(64, 64, EPI_GELU)
  MSP_CONV(64, 16, EPI_NONE)
  MSP_CONV(64, 64, EPI_GELU_GRAD)
  MSP_CONV(16, 64, EPI_GELU_GRAD)
  MSP_CONV(16, 64, EPI_NONE)
  MSP_CONV(64, 64, EPI_NONE)
  MSP_CONV(16, 16, EPI_NONE)
#undef MSP_CONV
  return cudaErrorInvalidValue;
}

template <int CIN, int COUT>
cudaError_t launch_wgrad(const bf16* g_chw, const bf16* in_chw, float* part, int H, int Wd, int* err, cudaStream_t st) {
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(wgrad_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)wgrad_smem<CIN>());
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  wgrad_kernel<CIN, COUT><<<dim3((unsigned)H, (unsigned)WG<CIN, COUT>::NTILES), kThreads, wgrad_smem<CIN>(), st>>>(
      g_chw, in_chw, part, H, Wd, err, tc_wait_limit());
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t wgrad(int cin, int cout, const bf16* g_chw, const bf16* in_chw, float* part, int H, int Wd, int* err,
                  cudaStream_t st) {
  if (cin == 16 && cout == 64) return launch_wgrad<16, 64>(g_chw, in_chw, part, H, Wd, err, st);
  if (cin == 64 && cout == 64) return launch_wgrad<64, 64>(g_chw, in_chw, part, H, Wd, err, st);
  if (cin == 64 && cout == 16) return launch_wgrad<64, 16>(g_chw, in_chw, part, H, Wd, err, st);
  if (cin == 16 && cout == 16) return launch_wgrad<16, 16>(g_chw, in_chw, part, H, Wd, err, st);
  return cudaErrorInvalidValue;
}

int grid1d(size_t n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

// Packs every layer's forward (and, for training, data-gradient) operand from the FP32 weights.
cudaError_t pack_all(const Net& n, const float* params, const Ws& w, bool dgrad, cudaStream_t st) {
  for (int i = 0; i < kLayers; ++i) {
    const Layer& l = n.layer[i];
    pack_fwd_kernel<<<grid1d(packed_fwd_elems(l)), 256, 0, st>>>(params + l.w_off, l.cin_true, l.cout_true, l.cin,
                                                                  l.cout, w.Bf[i]);
    count_launches(1);
    if (dgrad && i > 0) {
      pack_dgrad_kernel<<<grid1d(packed_dgrad_elems(l)), 256, 0, st>>>(params + l.w_off, l.cin_true, l.cout_true,
                                                                        l.cin, l.cout, w.Bd[i]);
      count_launches(1);
    }
  }
  return cudaGetLastError();
}

// Forward through the six layers from the packed input; keeps every pre-activation.
cudaError_t forward(const Net& n, const float* params, const Ws& w, int H, int Wd, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < kLayers && e == cudaSuccess; ++i) {
    const Layer& l = n.layer[i];
    const bf16* in = i == 0 ? w.x : w.act[i - 1];
    const bool last = i == kLayers - 1;
    e = conv(l.cin, l.cout, last ? EPI_NONE : EPI_GELU, in, w.Bf[i], params + l.b_off, nullptr, w.pre[i],
             last ? nullptr : w.act[i], last ? nullptr : w.act_chw[i], l.cout_true, H, Wd, w.err, st);
  }
  return e;
}

}  // namespace learn
}  // namespace msp

using namespace msp;
using namespace msp::learn;

static msp_status check_shape(const msp_net_shape* s) {
  if (!s) return fail(MSP_EINVAL, "shape is NULL");
  if (s->n_slices < 1 || s->n_slices > 8) return fail(MSP_EUNSUPPORTED, "n_slices must be 1 .. 8");
  if (s->height < 1 || s->height > 65535 || s->width < kPix || s->width % kPix != 0)
    return fail(MSP_EUNSUPPORTED, "width must be a positive multiple of 128 and height 1 .. 65535");
  if ((size_t)s->height * s->width > ((size_t)1 << 26)) return fail(MSP_EUNSUPPORTED, "image too large");
  if (!(s->scale_v > 0 && s->scale_g > 0 && s->scale_d > 0)) return fail(MSP_EINVAL, "scales must be > 0");
  return MSP_OK;
}

#define LEARN_CK(call)                                                                        \
  do {                                                                                        \
    const cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(MSP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" {

msp_status msp_net_validate(const msp_net_shape* s) {
  set_last_error(MSP_OK, "");
  return check_shape(s);
}

size_t msp_net_param_count(const msp_net_shape* s) {
  if (check_shape(s) != MSP_OK) return 0;
  return make_net(s->n_slices).n_params;
}

size_t msp_net_workspace_bytes(const msp_net_shape* s) {
  if (check_shape(s) != MSP_OK) return 0;
  return carve(make_net(s->n_slices), s->height, s->width, nullptr).bytes;
}

msp_status msp_net_init(const msp_net_shape* s, float* params, uint64_t seed, void* stream) {
  set_last_error(MSP_OK, "");
  msp_status st = check_shape(s);
  if (st != MSP_OK) return st;
  if (!params) return fail(MSP_EINVAL, "params is NULL");
  const Net n = make_net(s->n_slices);
  for (int i = 0; i < kLayers; ++i) {
    const Layer& l = n.layer[i];
    float bound = (float)sqrt(6.0 / (9.0 * l.cin_true + 9.0 * l.cout_true));
    if (i == kLayers - 1) bound *= 0.1f;
    const size_t nw = (size_t)l.cout_true * 9 * l.cin_true;
    init_kernel<<<grid1d(nw), 256, 0, (cudaStream_t)stream>>>(params, l.w_off, nw, (size_t)l.cout_true, bound, seed);
    count_launches(1);
  }
  LEARN_CK(cudaGetLastError());
  return MSP_OK;
}

static msp_status net_begin(const msp_net_shape* s, void* ws, size_t ws_bytes, Net* n, Ws* w) {
  msp_status st = check_shape(s);
  if (st != MSP_OK) return st;
  st = refuse_untrusted_device();
  if (st != MSP_OK) return st;
  *n = make_net(s->n_slices);
  const size_t need = carve(*n, s->height, s->width, nullptr).bytes;
  if (!ws || ((uintptr_t)ws) % 256) return fail(MSP_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) return fail(MSP_EINVAL, "workspace too small: " + std::to_string(ws_bytes) + " < " + std::to_string(need));
  *w = carve(*n, s->height, s->width, (char*)ws);
  return MSP_OK;
}

msp_status msp_net_forward(const msp_net_shape* s, const float* params, const float* V, const float* G, float* dV_prop,
                           void* ws, size_t ws_bytes, void* stream) {
  set_last_error(MSP_OK, "");
  Net n;
  Ws w;
  msp_status st = net_begin(s, ws, ws_bytes, &n, &w);
  if (st != MSP_OK) return st;
  if (!params || !V || !G || !dV_prop) return fail(MSP_EINVAL, "params, V, G and dV_prop must be non-NULL");
  cudaStream_t cs = (cudaStream_t)stream;
  const int H = s->height, Wd = s->width, L = s->n_slices;
  const size_t P = (size_t)H * Wd;
  LEARN_CK(cudaMemsetAsync(w.err, 0, sizeof(int), cs));
  LEARN_CK(pack_all(n, params, w, false, cs));
  input_kernel<<<grid1d(P * 16), 256, 0, cs>>>(V, G, L, P, (float)s->scale_v, (float)s->scale_g, w.x, w.x_chw);
  count_launches(1);
  LEARN_CK(forward(n, params, w, H, Wd, cs));
  output_kernel<<<grid1d(P * L), 256, 0, cs>>>(w.pre[kLayers - 1], L, P, (float)s->scale_d, dV_prop);
  count_launches(1);
  LEARN_CK(cudaGetLastError());
  return MSP_OK;
}

}  // extern "C"

// Loss of the proposal against `target` and its gradient with respect to the parameters (into
// `grad`, FP32 parameter layout); `loss_out` may be NULL.
static msp_status net_loss_grad(const msp_net_shape* s, const Net& n, const Ws& w, const float* params, const float* V,
                                const float* G, const float* target, float* grad, double* loss_out, cudaStream_t cs) {
  const int H = s->height, Wd = s->width, L = s->n_slices;
  const size_t P = (size_t)H * Wd;
  LEARN_CK(cudaMemsetAsync(w.err, 0, sizeof(int), cs));
  LEARN_CK(pack_all(n, params, w, true, cs));
  input_kernel<<<grid1d(P * 16), 256, 0, cs>>>(V, G, L, P, (float)s->scale_v, (float)s->scale_g, w.x, w.x_chw);
  count_launches(1);
  LEARN_CK(forward(n, params, w, H, Wd, cs));
  const int lb = 512;
  loss_kernel<<<lb, 256, 0, cs>>>(w.pre[kLayers - 1], target, L, P, (float)(1.0 / s->scale_d), w.g[0], w.g_chw[0],
                                  w.loss_part);
  count_launches(1);
  if (loss_out) {
    loss_sum_kernel<<<1, 32, 0, cs>>>(w.loss_part, lb, loss_out);
    count_launches(1);
  }
  // backward, last layer first: g[cur] holds the gradient of layer i's pre-activation
  int cur = 0;
  for (int i = kLayers - 1; i >= 0; --i) {
    const Layer& l = n.layer[i];
    const bf16* in_chw = i == 0 ? w.x_chw : w.act_chw[i - 1];
    LEARN_CK(wgrad(l.cin, l.cout, w.g_chw[cur], in_chw, w.part, H, Wd, w.err, cs));
    const int nred = l.cout_true * 9 * l.cin;
    wgrad_reduce_kernel<<<(nred + 255) / 256, 256, 0, cs>>>(w.part, H, l.cout, l.cin, l.cout_true, l.cin_true,
                                                            grad + l.w_off);
    bias_grad_part_kernel<<<lb, 256, 0, cs>>>(w.g[cur], P, l.cout, w.bpart);
    bias_grad_sum_kernel<<<1, 64, 0, cs>>>(w.bpart, lb, l.cout, l.cout_true, grad + l.b_off);
    count_launches(3);
    if (i > 0) {   // gradient of the previous layer's pre-activation: conv with mirrored weights x gelu'
      LEARN_CK(conv(l.cout, l.cin, EPI_GELU_GRAD, w.g[cur], w.Bd[i], nullptr, w.pre[i - 1], nullptr, w.g[1 - cur],
                    w.g_chw[1 - cur], 0, H, Wd, w.err, cs));
      cur = 1 - cur;
    }
  }
  LEARN_CK(cudaGetLastError());
  return MSP_OK;
}

extern "C" {

msp_status msp_net_loss_grad(const msp_net_shape* s, const float* params, const float* V, const float* G,
                             const float* target, float* grad, double* loss_out, void* ws, size_t ws_bytes,
                             void* stream) {
  set_last_error(MSP_OK, "");
  Net n;
  Ws w;
  msp_status st = net_begin(s, ws, ws_bytes, &n, &w);
  if (st != MSP_OK) return st;
  if (!params || !V || !G || !target || !grad) return fail(MSP_EINVAL, "params, V, G, target and grad must be non-NULL");
  return net_loss_grad(s, n, w, params, V, G, target, grad, loss_out, (cudaStream_t)stream);
}

msp_status msp_net_train_step(const msp_net_shape* s, float* params, float* adam_m, float* adam_v, int32_t step,
                              double lr, const float* V, const float* G, const float* target, double* loss_out,
                              void* ws, size_t ws_bytes, void* stream) {
  set_last_error(MSP_OK, "");
  Net n;
  Ws w;
  msp_status st = net_begin(s, ws, ws_bytes, &n, &w);
  if (st != MSP_OK) return st;
  if (!params || !adam_m || !adam_v || !V || !G || !target)
    return fail(MSP_EINVAL, "params, adam_m, adam_v, V, G and target must be non-NULL");
  if (step < 1 || !(lr > 0)) return fail(MSP_EINVAL, "step must be >= 1 and lr > 0");
  cudaStream_t cs = (cudaStream_t)stream;
  st = net_loss_grad(s, n, w, params, V, G, target, w.grad, loss_out, cs);
  if (st != MSP_OK) return st;
  const double c1 = 1.0 / (1.0 - pow(0.9, step)), c2 = 1.0 / (1.0 - pow(0.999, step));
  adam_kernel<<<grid1d(n.n_params), 256, 0, cs>>>(params, adam_m, adam_v, w.grad, n.n_params, (float)lr, (float)c1,
                                                  (float)c2);
  count_launches(1);
  LEARN_CK(cudaGetLastError());
  return MSP_OK;
}

static size_t planes_bytes(const msp_net_shape* s) {
  return align256((size_t)s->n_slices * s->height * s->width * sizeof(float));
}

static msp_status check_pair(const msp_geometry* g, const msp_net_shape* s) {
  if (!g) return fail(MSP_EINVAL, "geometry is NULL");
  msp_status st = check_shape(s);
  if (st != MSP_OK) return st;
  st = msp_validate_geometry(g);
  if (st != MSP_OK) return st;
  if (g->param != MSP_PARAM_POTENTIAL) return fail(MSP_EUNSUPPORTED, "the proposal acts on potentials");
  if (s->n_slices != g->n_slices || s->height != g->obj_ny || s->width != g->obj_nx)
    return fail(MSP_EINVAL, "network shape and geometry disagree (n_slices, height = obj_ny, width = obj_nx)");
  return MSP_OK;
}

size_t msp_learned_workspace_bytes(const msp_geometry* g, const msp_net_shape* s) {
  if (check_pair(g, s) != MSP_OK) return 0;
  return carve(make_net(s->n_slices), s->height, s->width, nullptr).bytes + 3 * planes_bytes(s);
}

msp_status msp_learned_propose(const msp_geometry* g, const msp_net_shape* s, const float* params,
                               const float* probe, float* V, const int32_t* pos, const float* I_meas,
                               int32_t* accepted, double* loss, void* ws, size_t ws_bytes, void* learn_ws,
                               size_t learn_ws_bytes, void* stream) {
  set_last_error(MSP_OK, "");
  msp_status st = check_pair(g, s);
  if (st != MSP_OK) return st;
  if (!params || !probe || !V || !pos || !I_meas || !loss)
    return fail(MSP_EINVAL, "params, probe, V, pos, I_meas and loss must be non-NULL");
  const size_t net_bytes = carve(make_net(s->n_slices), s->height, s->width, nullptr).bytes;
  if (!learn_ws || ((uintptr_t)learn_ws) % 256 || learn_ws_bytes < net_bytes + 3 * planes_bytes(s))
    return fail(MSP_EINVAL, "learned workspace must be 256-byte aligned and msp_learned_workspace_bytes long");
  char* base = (char*)learn_ws;
  float* G = (float*)(base + net_bytes);
  float* dV = (float*)(base + net_bytes + planes_bytes(s));
  float* Vc = (float*)(base + net_bytes + 2 * planes_bytes(s));
  cudaStream_t cs = (cudaStream_t)stream;
  const size_t n = (size_t)s->n_slices * s->height * s->width;
  st = msp_loss_grad(g, probe, V, pos, I_meas, loss, G, nullptr, ws, ws_bytes, stream);
  if (st != MSP_OK) return st;
  st = msp_net_forward(s, params, V, G, dV, learn_ws, net_bytes, stream);
  if (st != MSP_OK) return st;
  candidate_kernel<<<grid1d(n), 256, 0, cs>>>(V, dV, n, Vc);
  count_launches(1);
  LEARN_CK(cudaGetLastError());
  st = msp_loss_grad(g, probe, Vc, pos, I_meas, loss + 1, nullptr, nullptr, ws, ws_bytes, stream);
  if (st != MSP_OK) return st;
  select_kernel<<<grid1d(n), 256, 0, cs>>>(loss, Vc, n, V, accepted);
  count_launches(1);
  LEARN_CK(cudaGetLastError());
  return MSP_OK;
}

size_t msp_conv3x3_test_workspace_bytes(int32_t height, int32_t width, int32_t c_in, int32_t c_out) {
  if (height < 1 || height > 65535 || width < kPix || width % kPix || (c_in != 16 && c_in != 64) ||
      (c_out != 16 && c_out != 64))
    return 0;
  const size_t P = (size_t)height * width;
  return align256(sizeof(int)) + align256((size_t)kchunks(c_in) * c_out * kKC * 2) +
         align256((size_t)height * c_out * 9 * c_in * 4) + align256(512 * 64 * 4) + align256(2 * P * 64 * 2);
}

msp_status msp_conv3x3_test(int32_t height, int32_t width, int32_t c_in, int32_t c_out, const void* in_bf16,
                            const float* w, const float* bias, float* pre_out, void* ws, size_t ws_bytes, void* stream) {
  set_last_error(MSP_OK, "");
  const size_t need = msp_conv3x3_test_workspace_bytes(height, width, c_in, c_out);
  if (need == 0) return fail(MSP_EUNSUPPORTED, "c_in, c_out in {16, 64}, width a positive multiple of 128");
  if (!ws || ((uintptr_t)ws) % 256 || ws_bytes < need) return fail(MSP_EINVAL, "workspace");
  if (!in_bf16 || !w || !pre_out) return fail(MSP_EINVAL, "in, w and pre_out must be non-NULL");
  cudaStream_t cs = (cudaStream_t)stream;
  char* b = (char*)ws;
  int* err = (int*)b;
  bf16* Bp = (bf16*)(b + align256(sizeof(int)));
  LEARN_CK(cudaMemsetAsync(err, 0, sizeof(int), cs));
  const size_t ne = (size_t)kchunks(c_in) * c_out * kKC;
  pack_fwd_kernel<<<grid1d(ne), 256, 0, cs>>>(w, c_in, c_out, c_in, c_out, Bp);
  count_launches(1);
  LEARN_CK(conv(c_in, c_out, EPI_NONE, (const bf16*)in_bf16, Bp, bias, nullptr, pre_out, nullptr, nullptr,
                bias ? c_out : 0, height, width, err, cs));
  return MSP_OK;
}

msp_status msp_conv3x3_wgrad_test(int32_t height, int32_t width, int32_t c_in, int32_t c_out, const void* in_bf16,
                                  const void* grad_pre_bf16, float* dW, float* db, void* ws, size_t ws_bytes,
                                  void* stream) {
  set_last_error(MSP_OK, "");
  const size_t need = msp_conv3x3_test_workspace_bytes(height, width, c_in, c_out);
  if (need == 0) return fail(MSP_EUNSUPPORTED, "c_in, c_out in {16, 64}, width a positive multiple of 128");
  if (!ws || ((uintptr_t)ws) % 256 || ws_bytes < need) return fail(MSP_EINVAL, "workspace");
  if (!in_bf16 || !grad_pre_bf16 || !dW || !db) return fail(MSP_EINVAL, "in, grad_pre, dW and db must be non-NULL");
  cudaStream_t cs = (cudaStream_t)stream;
  const size_t P = (size_t)height * width;
  char* b = (char*)ws;
  int* err = (int*)b;
  size_t off = align256(sizeof(int)) + align256((size_t)kchunks(c_in) * c_out * kKC * 2);
  float* part = (float*)(b + off);
  off += align256((size_t)height * c_out * 9 * c_in * 4);
  float* bpart = (float*)(b + off);
  off += align256(512 * 64 * 4);
  bf16* in_chw = (bf16*)(b + off);
  bf16* g_chw = in_chw + P * 64;
  LEARN_CK(cudaMemsetAsync(err, 0, sizeof(int), cs));
  // channel-major copies of the NHWC operands
  {
    const bf16* src = (const bf16*)in_bf16;
    const bf16* gs = (const bf16*)grad_pre_bf16;
    const size_t n1 = P * c_in, n2 = P * c_out;
    to_chw_kernel<<<grid1d(n1), 256, 0, cs>>>(src, P, c_in, in_chw);
    to_chw_kernel<<<grid1d(n2), 256, 0, cs>>>(gs, P, c_out, g_chw);
    count_launches(2);
  }
  LEARN_CK(wgrad(c_in, c_out, g_chw, in_chw, part, height, width, err, cs));
  wgrad_reduce_kernel<<<(c_out * 9 * c_in + 255) / 256, 256, 0, cs>>>(part, height, c_out, c_in, c_out, c_in, dW);
  bias_grad_part_kernel<<<512, 256, 0, cs>>>((const bf16*)grad_pre_bf16, P, c_out, bpart);
  bias_grad_sum_kernel<<<1, 64, 0, cs>>>(bpart, 512, c_out, c_out, db);
  count_launches(3);
  LEARN_CK(cudaGetLastError());
  return MSP_OK;
}

}  // extern "C"
