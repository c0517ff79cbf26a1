// msp_learn.cu -- the learned-proposal form (include/msp_learn.h): a six-layer 3 x 3
// convolutional network in BF16 with FP32 accumulation on the tensor cores, its training step
// (backward pass and Adam) and its proposal.
//
// Every convolution is an implicit GEMM on tcgen05 (kind::f16, bf16 operands, FP32 accumulator
// in tensor memory):
//   forward / data gradient:  D[pixel][c_out] = sum over taps and c_in of in[pixel + tap][c_in]
//     w[c_out][tap][c_in], 128 pixels of an image row per accumulator; persistent CTAs stage each
//     input row once (NHWC, 8 channels of a pixel are 16 contiguous bytes, zero outside the
//     image) and read all nine taps from it; the weights stay resident.  The data gradient is
//     the forward convolution of the gradient with the weights mirrored in the taps and
//     transposed in the channels.
//   weight gradient:  D_tap[c_in][c_out] = sum_p in[p + tap][c_in] dPre[p][c_out], K = the pixels
//     of a CTA's rows, both operands MN-major from the same staged NHWC rows; the bias gradient
//     is one more row of it (a constant group of ones); the per-CTA partial sums are added in a
//     fixed order.
// Operands are staged through shared memory in the canonical no-swizzle layouts (core matrices
// of 8 rows x 16 bytes): the image rows by tensor loads (TMA) that complete on mbarriers, the
// convolution's resident weights once per CTA with cp.async.  One thread issues the MMAs and
// commits them to mbarriers; every wait is bounded and records a timeout in the error word.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
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
constexpr int kThreads = 256;
constexpr int kDrainLimit = 1 << 20;

enum Epi { EPI_NONE = 0, EPI_GELU = 1, EPI_GELU_GRAD = 2 };

// The normal CDF Phi(x) = erfc(-x / sqrt 2) / 2, branch-free: with z = min(|x| / sqrt 2, 6) and
// g(z) = -log erfc(z) = z h(z), Phi = exp(-g) / 2 for x < 0 and 1 - exp(-g) / 2 otherwise, so
// both tails keep their accuracy.  h is a degree-11 least-squares fit in the Chebyshev basis of
// u = z / 3 - 1, written as monomials in u (csrc/gen_phi_fit.py prints them and the error:
// |Phi error| < 1e-7 in FP32).  One exponential and twelve fused multiply-adds.
__device__ __forceinline__ float phi_cdf(float x) {
  const float z = fminf(fabsf(x) * 0.70710678118654752f, 6.f);
  const float u = fmaf(z, 1.f / 3.f, -1.f);
  float h = 7.291426300e-04f;
  h = fmaf(h, u, -1.261031372e-03f);
  h = fmaf(h, u, -2.603480243e-04f);
  h = fmaf(h, u, 1.729566371e-03f);
  h = fmaf(h, u, -2.867543837e-03f);
  h = fmaf(h, u, 7.777833380e-03f);
  h = fmaf(h, u, -1.878948696e-02f);
  h = fmaf(h, u, 3.874455020e-02f);
  h = fmaf(h, u, -7.517043501e-02f);
  h = fmaf(h, u, 1.418747455e-01f);
  h = fmaf(h, u, 2.730299234e+00f);
  h = fmaf(h, u, 3.573454380e+00f);
  const float t = 0.5f * exp2f(-1.44269504088896341f * (h * z));   // exp(-g) / 2
  return x < 0.f ? t : 1.f - t;
}
// GELU(x) = x Phi(x), GELU'(x) = Phi(x) + x phi(x), from p = Phi(x)
__device__ __forceinline__ float gelu_from(float x, float p) { return x * p; }
__device__ __forceinline__ float gelu_grad_from(float x, float p) {
  return p + x * 0.39894228040143268f * expf(-0.5f * x * x);
}


// ---------------------------------------------------------------------------
// forward / data-gradient convolution
// ---------------------------------------------------------------------------
// A persistent CTA owns a strip of 128 output columns and a run of output rows.  It stages
// every input row it needs once in shared memory (130 pixels with the halo, zero outside the
// image) and keeps all nine taps of the weights resident; the nine taps of an output row then
// read the staged rows through matrix descriptors whose start is offset by the tap (dx pixels
// = dx x 16 bytes: pixels are consecutive 16-byte rows of the K-major core matrices, the 8-channel
// groups are kTRows x 16 bytes apart).  Warp roles: one thread of warp 8 fetches rows with tensor
// loads, one thread of warp 9 issues the MMAs, warps 0-7 run the epilogue.  The accumulator is
// double-buffered in tensor memory: the MMAs of row k run while the epilogue warps drain the
// other buffer (row k - 1) and the next rows are in flight.
constexpr int kTRows = 136;  // staged pixels per channel group (130 used); 136 x 16 B keeps every
                             // group 128-byte aligned for the tensor loads
constexpr uint32_t kBox = 130 * 16;   // bytes of one tensor-load box: 8 channels x 130 pixels
constexpr int kFSlots = 5;   // staged input rows of the convolution: three in use, two in flight
constexpr int kCSlots = 5;   // staged input rows of the weight-gradient kernel
constexpr int kGSlots = 3;   // staged gradient rows of the weight-gradient kernel
constexpr int kWSteps = 3;   // row steps of the weight-gradient kernel in flight (one barrier pair each)

// packed weights of conv2_kernel: [9 taps][CIN / 8 channel groups][COUT rows][8 channels]
__host__ __device__ constexpr size_t packed_off(int t, int n, int k, int CIN, int COUT) {
  return (size_t)t * COUT * CIN + (size_t)(k >> 3) * COUT * 8 + (size_t)n * 8 + (k & 7);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
// Tensor memory access (TMA): a tiled load of a box of the tensor described by `tmap` into
// shared memory, completing on an mbarrier by transaction count.  Coordinates are elements,
// innermost first; boxes reaching outside the tensor are filled with zeros.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tmap, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(tc::smem_u32(bar))
      : "memory");
}

// Programmatic dependent launch: wait for the preceding kernel of the stream to complete (its
// writes visible), and allow the next one to be scheduled.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int CIN, int COUT>
struct Conv {
  static constexpr int G = CIN / 8;                                  // channel groups
  static constexpr uint32_t GRP = kTRows * 16;                       // bytes of one group of a staged row
  static constexpr uint32_t SLOT = (uint32_t)G * GRP;                // bytes of one staged row
  static constexpr uint32_t WB = 9u * COUT * CIN * 2;                // bytes of the weights
  static constexpr uint32_t TC = COUT < 32 ? 32 : COUT;              // TMEM columns per accumulator
  static constexpr size_t SMEM = 1024 + (size_t)WB + (size_t)kFSlots * SLOT + 2 * 8 * kFSlots + 4 * 8 + 16;
};

// in  [H][Wd][CIN] bf16 (NHWC); Bp packed as packed_off.  Output rows [y0, y0 + rows_per_cta)
// of column strip blockIdx.x, with y0 = blockIdx.y * rows_per_cta.
// pre (FP32 [H][Wd][COUT], may be NULL) receives, with EPI_NONE, the pre-activation D + bias
// (bias[c] for c < nbias, else 0) and, with EPI_GELU, the derivative gelu'(D + bias) that the
// backward pass multiplies by (computed once here instead of from the pre-activation there).
// EPI_GELU: out = gelu(D + bias) in bf16 (NHWC).
// EPI_GELU_GRAD: out = D * aux (aux FP32 [H][Wd][COUT], gelu' of the forward's pre-activation)
// in bf16 (NHWC).
//
// Roles, synchronised by mbarriers only:
//   warp 8, one thread (producer): fetches input row i into slot i % kFSlots by tensor loads
//     once the MMAs of output row i - kFSlots released it (empty[slot]); the loads complete on
//     full[slot] by transaction count;
//   warp 9, one thread (MMA): for output row k waits for staged row k + 2 (full) and for the
//     epilogue to have drained accumulator k & 1 (acc_empty), issues the 9 x CIN / 16 MMAs,
//     commits to acc_full[k & 1] and to empty[k % kFSlots] (row k has no later reader);
//   warps 0..7 (epilogue): wait for acc_full, read the accumulator, write the outputs, arrive on
//     acc_empty.
// Every wait is bounded: the first that runs out raises the flag, the other roles see it and
// stop, the producer waits for the loads it issued, and the MMA thread waits for its last
// commit before the tensor memory is released.
constexpr int kConvThreads = 320;

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(kConvThreads, 1) conv_kernel(const bf16* __restrict__ in, const bf16* __restrict__ Bp,
                                                               const float* __restrict__ bias,
                                                               const float* __restrict__ aux, float* __restrict__ pre,
                                                               bf16* __restrict__ out, int nbias, int H, int Wd,
                                                               int rows_per_cta, int* err, int wait_limit,
                                                               const __grid_constant__ CUtensorMap tmap) {
  using C = Conv<CIN, COUT>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sw = smem;                 // weights
  uint8_t* srow = sw + C::WB;         // staged rows
  uint64_t* full = reinterpret_cast<uint64_t*>(srow + kFSlots * C::SLOT);
  uint64_t* empty = full + kFSlots;
  uint64_t* acc_full = empty + kFSlots;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * kPix;
  const int y0 = blockIdx.y * rows_per_cta;
  const int n = min(rows_per_cta, H - y0);   // output rows of this CTA
  if (n <= 0) return;

  if (tid == 0) {
    for (int i = 0; i < kFSlots; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], 8);
    }
    tc::fence_mbar_init();
    *flag = 0;
  }
  // the weights, once, by all threads
  for (int i = tid; i < (int)(C::WB / 16); i += kConvThreads)
    cp_async16(tc::smem_u32(sw) + 16u * i, reinterpret_cast<const uint4*>(Bp) + i, true);
  cp_async_commit();
  if (warp == 0) tc::tmem_alloc(tslot, 2 * C::TC);
  cp_async_wait_all();
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 8) {
    // ---- producer, one thread: staged rows 0 .. n + 1 (input rows y0 - 1 .. y0 + n) by tensor
    // loads, one box of 8 channels x 130 pixels per channel group, completing on full[slot] ----
    // The prologue above (barriers, tensor memory, weights packed by an earlier kernel) may
    // overlap the preceding kernel; the input it wrote is read only after it has completed.
    if (lane == 0) {
      grid_dependency_wait();
      grid_dependents_launch();
      int i = 0;
      for (; i < n + 2 && !*flag; ++i) {
        const int slot = i % kFSlots;
        if (i >= kFSlots && !tc::wait_phase(&empty[slot], (uint32_t)((i / kFSlots - 1) & 1), wait_limit)) {
          *flag = 2;
          break;
        }
        mbar_expect_tx(&full[slot], (uint32_t)C::G * kBox);   // G boxes of 130 pixels x 16 B
        const uint32_t dst = tc::smem_u32(srow + slot * C::SLOT);
#pragma unroll 1
        for (int j = 0; j < C::G; ++j) tma_load_3d(dst + (uint32_t)j * C::GRP, &tmap, 8 * j, x0 - 1, y0 - 1 + i, &full[slot]);
      }
      // after an abort, the loads in flight land before the shared memory is released: the latest
      // load of each slot is the last completion of its barrier
      if (*flag)
        for (int r = max(0, i - kFSlots); r < i; ++r)
          if (!tc::wait_phase(&full[r % kFSlots], (uint32_t)((r / kFSlots) & 1), kDrainLimit)) *flag = 3;
    }
  } else if (warp == 9) {
    // ---- MMA issuer ----
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16(kPix, COUT);
      const uint32_t a0 = tc::smem_u32(srow), b0 = tc::smem_u32(sw);
      int issued = -1;
      for (int k = 0; k < n && !*flag; ++k) {
        bool ok = true;
        for (int i = (k == 0 ? 0 : k + 2); i <= k + 2 && ok; ++i)
          ok = tc::wait_phase(&full[i % kFSlots], (uint32_t)((i / kFSlots) & 1), wait_limit);
        if (ok && k >= 2) ok = tc::wait_phase(&acc_empty[k & 1], (uint32_t)(((k - 2) >> 1) & 1), wait_limit);
        if (!ok) {
          *flag = 2;
          break;
        }
        tc::fence_after();
        const uint32_t dcol = tmem + (uint32_t)(k & 1) * C::TC;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const int dy = t / 3, dx = t % 3;   // staged row k + dy, pixel offset dx
          const uint32_t a = a0 + (uint32_t)((k + dy) % kFSlots) * C::SLOT + (uint32_t)dx * 16u;
          const uint32_t b = b0 + (uint32_t)t * (COUT * CIN * 2);
#pragma unroll
          for (int s = 0; s < CIN / 16; ++s)
            tc::mma_bf16(dcol, tc::smem_desc(a + (uint32_t)(2 * s) * C::GRP, C::GRP, 128),
                         tc::smem_desc(b + (uint32_t)(2 * s) * (COUT * 16), COUT * 16, 128), idesc,
                         (t > 0 || s > 0) ? 1u : 0u);
        }
        tc::commit(&acc_full[k & 1]);
        tc::commit(&empty[k % kFSlots]);
        issued = k;
      }
      // Before the CTA exits, every commit has arrived: the latest one on each staging slot (rows
      // issued - 4 .. issued, which the producer may never have waited for) and, after an
      // abort, on both accumulators.  Each is the last completion of its barrier, so the
      // parity names it without ambiguity.
      for (int k = max(0, issued - (kFSlots - 1)); k <= issued; ++k)
        if (!tc::wait_phase(&empty[k % kFSlots], (uint32_t)((k / kFSlots) & 1), kDrainLimit)) *flag = 3;
      if (*flag)
        for (int k = max(0, issued - 1); k <= issued; ++k)
          if (!tc::wait_phase(&acc_full[k & 1], (uint32_t)((k >> 1) & 1), kDrainLimit)) *flag = 3;
    }
  } else {
    // ---- epilogue: warps w and w + 4 read TMEM lanes 32 (w % 4) .., the lower and the upper
    // half of the channels (warps 0..3 all of them if COUT = 16) ----
    constexpr int HALF = COUT >= 32 ? COUT / 2 : COUT;
    constexpr int NCH = HALF / 16;   // 16-column chunks of a thread's accumulator row
    const bool active = !(COUT < 32 && warp >= 4);
    const int q = warp & 3, c0 = (warp >> 2) * HALF;
    // this thread's biases, in registers (written by an earlier kernel: read after the wait)
    grid_dependency_wait();
    float bsum[HALF];
#pragma unroll
    for (int u = 0; u < HALF; ++u) bsum[u] = (c0 + u < nbias) ? bias[c0 + u] : 0.f;
    for (int k = 0; k < n; ++k) {
      if (lane == 0 && !tc::wait_phase(&acc_full[k & 1], (uint32_t)((k >> 1) & 1), wait_limit)) *flag = 2;
      __syncwarp();
      if (*flag) break;
      tc::fence_after();
      if (active) {
        const int y = y0 + k, r = 32 * q + lane, x = x0 + r;
        const size_t p = (size_t)y * Wd + x;
        const uint32_t acc = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(k & 1) * C::TC;
        // the next chunk's tensor-memory load is in flight while this chunk is processed
        uint32_t d[2][16];
        tc::tmem_ld16(acc + (uint32_t)c0, d[0]);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          const int j0 = c0 + 16 * ch;
          tc::tmem_wait_ld();
          tc::tmem_ready(d[ch & 1]);
          if (ch + 1 < NCH) tc::tmem_ld16(acc + (uint32_t)(j0 + 16), d[(ch + 1) & 1]);
          float v[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) v[u] = __uint_as_float(d[ch & 1][u]) + bsum[16 * ch + u];
          float ph[16];   // Phi of the pre-activations (GELU)
          if (EPI == EPI_GELU) {
#pragma unroll
            for (int u = 0; u < 16; ++u) ph[u] = phi_cdf(v[u]);
          }
          if (pre) {   // the pre-activation, or with GELU its derivative there
            float4* dst = reinterpret_cast<float4*>(pre + p * COUT + j0);
            float q[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) q[u] = EPI == EPI_GELU ? gelu_grad_from(v[u], ph[u]) : v[u];
#pragma unroll
            for (int u = 0; u < 4; ++u) dst[u] = make_float4(q[4 * u], q[4 * u + 1], q[4 * u + 2], q[4 * u + 3]);
          }
          if (EPI != EPI_NONE) {
            float g[16];
            if (EPI == EPI_GELU_GRAD) {
              const float4* ap = reinterpret_cast<const float4*>(aux + p * COUT + j0);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float4 a = ap[u];
                g[4 * u] = a.x, g[4 * u + 1] = a.y, g[4 * u + 2] = a.z, g[4 * u + 3] = a.w;
              }
            }
            __align__(16) bf16 o[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) o[u] = __float2bfloat16_rn(EPI == EPI_GELU ? gelu_from(v[u], ph[u]) : v[u] * g[u]);
            uint4* dst = reinterpret_cast<uint4*>(out + p * COUT + j0);
            dst[0] = reinterpret_cast<const uint4*>(o)[0];
            dst[1] = reinterpret_cast<const uint4*>(o)[1];
          }
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty[k & 1]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 2 * C::TC);
  }
  if (tid == 0 && *flag) atomicMax(err, *flag);
}

template <int CIN, int COUT>
constexpr size_t conv_smem() {
  return Conv<CIN, COUT>::SMEM;
}

// ---------------------------------------------------------------------------
// weight and bias gradients
// ---------------------------------------------------------------------------
// D_t[ci][co] = sum_p in[p + off(t)][ci] g[p][co] over the pixels of a CTA's strip and rows, on
// the tensor core with M = 128 rows of c_in (the first CIN real) and N = COUT, K = 16 pixels per
// MMA.  Both operands come from staged NHWC rows exactly as in the convolution: for one pixel the
// channels are 16 contiguous bytes, so they are MN-major operands (channel groups kTRows x 16
// bytes apart, 8-pixel groups 128 bytes apart) and a tap's pixel shift is again a start offset.
// Row CIN of the input operand reads a constant group of ones, which turns the centre tap's row
// CIN into the bias gradient sum_p g[p][co].  Each CTA accumulates all its rows in tensor memory
// (five or four taps x COUT columns: the taps are split over two CTA groups) and writes one
// partial sum; the partials are then added in a fixed order.
//
// Roles: one thread of warp 4 fetches rows by tensor loads, one thread of warp 5 issues the MMAs,
// warps 0-3 read the accumulator at the end.  Row step k (output row y0 + k) needs input rows
// k .. k + 2 and gradient row k; its loads (rows 0 .. 2 at k = 0, row k + 2 after) complete on
// full[k % kWSteps], its MMAs commit to done[k % kWSteps].  The slots step k fills held input and
// gradient rows k - 3, which step k - 3 was the last to read, so the fetch of step k waits for
// done of step k - 3 and three steps are in flight.
constexpr int kMaxSpatial = 512;   // spatial CTAs of one weight-gradient launch at most
// MN-major operands without swizzle: the descriptor's LBO is the stride between 8-row K groups and
// its SBO the stride between 8-element MN groups (the reverse of the K-major roles).
constexpr uint32_t kMnStrideLbo = 0;

template <int CIN, int COUT>
struct WGrad {
  static constexpr int G = CIN / 8, GO = COUT / 8;
  static constexpr uint32_t GRP = kTRows * 16;             // bytes of one channel group of a staged row
  static constexpr uint32_t ISLOT = (G + 1) * GRP;         // an input row and a group of ones
  static constexpr uint32_t GSLOT = GO * GRP;              // a gradient row
  static constexpr uint32_t PAD = (16 - G - 1) * GRP;      // the M = 128 operand spans 16 groups
  static constexpr int TAPS = 5;                           // taps [0, 5) or [5, 9) per CTA
  static constexpr uint32_t TC = TAPS * COUT <= 128 ? 128 : (TAPS * COUT <= 256 ? 256 : 512);
  static constexpr size_t SMEM = 1024 + (size_t)kCSlots * ISLOT + PAD + kGSlots * (size_t)GSLOT + 64;
  static_assert(kCSlots == kWSteps + 2 && kGSlots == kWSteps, "slot reuse follows the step pipeline");
};

// imap: tensor map of in [H][Wd][CIN], gmap: of g [H][Wd][COUT] (bf16 NHWC, boxes of 8 channels
// x 130 pixels x 1 row).  CTA (strip blockIdx.x, rows blockIdx.y, taps blockIdx.z) writes
// part[sp][t][co][ci] for its taps (sp = blockIdx.y * gridDim.x + blockIdx.x) and, for the
// centre tap's group, bpart[sp][co].
template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads, 1) wgrad_kernel(float* __restrict__ part, float* __restrict__ bpart,
                                                            int H, int rows_per_cta, int* err, int wait_limit,
                                                            const __grid_constant__ CUtensorMap gmap,
                                                            const __grid_constant__ CUtensorMap imap) {
  using C = WGrad<CIN, COUT>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sin = smem;
  uint8_t* sg = sin + kCSlots * C::ISLOT + C::PAD;
  uint64_t* full = reinterpret_cast<uint64_t*>(sg + kGSlots * C::GSLOT);
  uint64_t* done = full + kWSteps;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + kWSteps);
  volatile int* flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * kPix, y0 = blockIdx.y * rows_per_cta;
  const int t0 = blockIdx.z * C::TAPS, nt = blockIdx.z == 0 ? C::TAPS : 9 - C::TAPS;
  const int sp = blockIdx.y * gridDim.x + blockIdx.x;
  const int n = min(rows_per_cta, H - y0);
  if (n <= 0) return;

  if (tid == 0) {
    for (int i = 0; i < kWSteps; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&done[i], 1);
    }
    tc::fence_mbar_init();
    *flag = 0;
  }
  {   // the group of ones after every input slot; the padding after the last slot is zero
    const uint4 ones = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);   // bf16 1.0 x 8
    for (int i = tid; i < kCSlots * kTRows; i += kThreads)
      *reinterpret_cast<uint4*>(sin + (i / kTRows) * C::ISLOT + C::G * C::GRP + (i % kTRows) * 16) = ones;
    for (int i = tid; i < (int)(C::PAD / 16); i += kThreads)
      reinterpret_cast<uint4*>(sin + kCSlots * C::ISLOT)[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (warp == 0) tc::tmem_alloc(tslot, C::TC);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 4) {
    if (lane == 0) {   // ---- producer ----
      grid_dependency_wait();   // the gradient rows come from the preceding kernel
      grid_dependents_launch();
      int k = 0;
      for (; k < n && !*flag; ++k) {
        const int b = k % kWSteps;
        if (k >= kWSteps && !tc::wait_phase(&done[b], (uint32_t)((k / kWSteps - 1) & 1), wait_limit)) {
          *flag = 2;
          break;
        }
        const int i0 = k == 0 ? 0 : k + 2;
        mbar_expect_tx(&full[b], (uint32_t)((k + 3 - i0) * C::G + C::GO) * kBox);
#pragma unroll 1
        for (int i = i0; i <= k + 2; ++i) {   // staged input row i = image row y0 - 1 + i
          const uint32_t dst = tc::smem_u32(sin + (i % kCSlots) * C::ISLOT);
#pragma unroll 1
          for (int j = 0; j < C::G; ++j) tma_load_3d(dst + (uint32_t)j * C::GRP, &imap, 8 * j, x0 - 1, y0 - 1 + i, &full[b]);
        }
        const uint32_t dst = tc::smem_u32(sg + (k % kGSlots) * C::GSLOT);
#pragma unroll 1
        for (int j = 0; j < C::GO; ++j) tma_load_3d(dst + (uint32_t)j * C::GRP, &gmap, 8 * j, x0 - 1, y0 + k, &full[b]);
      }
      // after an abort, the loads in flight land before the shared memory is released
      if (*flag)
        for (int r = max(0, k - kWSteps); r < k; ++r)
          if (!tc::wait_phase(&full[r % kWSteps], (uint32_t)((r / kWSteps) & 1), kDrainLimit)) *flag = 3;
    }
  } else if (warp == 5) {
    if (lane == 0) {   // ---- MMA issuer ----
      constexpr uint32_t idesc = tc::idesc_bf16(kPix, COUT) | (1u << 15) | (1u << 16);   // A and B MN-major
      constexpr uint32_t LBO = kMnStrideLbo ? C::GRP : 128u, SBO = kMnStrideLbo ? 128u : C::GRP;
      const uint32_t a0 = tc::smem_u32(sin), b0 = tc::smem_u32(sg);
      int issued = -1;
#pragma unroll 1
      for (int k = 0; k < n && !*flag; ++k) {
        if (!tc::wait_phase(&full[k % kWSteps], (uint32_t)((k / kWSteps) & 1), wait_limit)) {
          *flag = 2;
          break;
        }
        tc::fence_after();
        const uint32_t b = b0 + (uint32_t)(k % kGSlots) * C::GSLOT + 16u;   // gradient pixel r at staged index r + 1
#pragma unroll 1
        for (int tl = 0; tl < nt; ++tl) {
          const int t = t0 + tl, dy = t / 3, dx = t % 3;
          const uint32_t a = a0 + (uint32_t)((k + dy) % kCSlots) * C::ISLOT + (uint32_t)dx * 16u;
#pragma unroll
          for (int s = 0; s < kPix / 16; ++s)
            tc::mma_bf16(tmem + (uint32_t)(tl * COUT), tc::smem_desc(a + (uint32_t)s * 256u, LBO, SBO),
                         tc::smem_desc(b + (uint32_t)s * 256u, LBO, SBO), idesc, (k > 0 || s > 0) ? 1u : 0u);
        }
        tc::commit(&done[k % kWSteps]);
        issued = k;
      }
      // the last commit covers every MMA issued; it is the latest completion of its barrier
      if (issued >= 0) {
        const bool aborted = *flag != 0;
        if (!tc::wait_phase(&done[issued % kWSteps], (uint32_t)((issued / kWSteps) & 1),
                            aborted ? kDrainLimit : wait_limit))
          *flag = aborted ? 3 : 2;
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (!*flag && warp < 4) {   // lane = row of D: c_in (< CIN) or the bias row (CIN)
    const int row = 32 * warp + lane;
    const bool active = __any_sync(0xffffffffu, row <= CIN);
    if (active) {
#pragma unroll 1
      for (int tl = 0; tl < nt; ++tl) {
        const int t = t0 + tl;
#pragma unroll 1
        for (int j0 = 0; j0 < COUT; j0 += 16) {
          uint32_t d[16];
          tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(tl * COUT + j0), d);
          tc::tmem_wait_ld();
          if (row < CIN) {
            float* dst = part + (((size_t)sp * 9 + t) * COUT + j0) * CIN + row;
#pragma unroll
            for (int u = 0; u < 16; ++u) dst[(size_t)u * CIN] = __uint_as_float(d[u]);
          } else if (row == CIN && t == 4) {
#pragma unroll
            for (int u = 0; u < 16; ++u) bpart[(size_t)sp * COUT + j0 + u] = __uint_as_float(d[u]);
          }
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, C::TC);
  }
  if (tid == 0 && *flag) atomicMax(err, *flag);
}

// x[0] + x[stride] + ... + x[(n - 1) stride], added in that order, eight loads in flight.
__device__ __forceinline__ float sum_in_order(const float* __restrict__ x, int stride, int n) {
  float s = 0.f;
  int i = 0;
  for (; i + 8 <= n; i += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = x[(size_t)(i + u) * stride];
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  for (; i < n; ++i) s += x[(size_t)i * stride];
  return s;
}

// dW[co][t][ci] (co < cout_true, ci < cin_true, the parameter layout) = sum over the nsp spatial
// partials in order; db[co] likewise.
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, const float* __restrict__ bpart, int nsp, int COUT,
                                    int CIN, int cout_true, int cin_true, float* __restrict__ dW,
                                    float* __restrict__ db) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nw = 9 * COUT * CIN;
  if (idx < nw) {
    const int t = idx / (COUT * CIN), co = (idx / CIN) % COUT, ci = idx % CIN;
    if (co >= cout_true || ci >= cin_true) return;
    dW[((size_t)co * 9 + t) * cin_true + ci] = sum_in_order(part + idx, nw, nsp);
  } else if (idx < nw + cout_true) {
    const int co = idx - nw;
    db[co] = sum_in_order(bpart + co, COUT, nsp);
  }
}

// ---------------------------------------------------------------------------
// packing, input, output, loss, Adam, initialisation
// ---------------------------------------------------------------------------

// B operand of the forward convolution from w [cout_true][9][cin_true] FP32: tap t, row co (< COUT),
// channel ci (< CIN), at packed_off; zero for padded channels.
__global__ void pack_fwd_kernel(const float* __restrict__ w, int cin_true, int cout_true, int CIN, int COUT,
                                bf16* __restrict__ Bp) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 9 * COUT * CIN) return;
  const int t = idx / (COUT * CIN), co = (idx / CIN) % COUT, ci = idx % CIN;
  float v = 0.f;
  if (ci < cin_true && co < cout_true) v = w[((size_t)co * 9 + t) * cin_true + ci];
  Bp[packed_off(t, co, ci, CIN, COUT)] = __float2bfloat16_rn(v);
}

// B operand of the data-gradient convolution (a forward convolution from COUT channels to CIN):
// tap t', row ci (< CIN), channel co (< COUT): w[co][8 - t'][ci] (taps mirrored, channels
// transposed).
__global__ void pack_dgrad_kernel(const float* __restrict__ w, int cin_true, int cout_true, int CIN, int COUT,
                                  bf16* __restrict__ Bp) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 9 * COUT * CIN) return;
  const int t = idx / (COUT * CIN), ci = (idx / COUT) % CIN, co = idx % COUT;
  float v = 0.f;
  if (ci < cin_true && co < cout_true) v = w[((size_t)co * 9 + (8 - t)) * cin_true + ci];
  Bp[packed_off(t, ci, co, COUT, CIN)] = __float2bfloat16_rn(v);
}

// Network input: x[p][c] = s_V V_c (c < L), s_G G_{c-L} (L <= c < 2L), 0 up to 16 (NHWC); one
// thread per pixel (the planes are read coalesced, the 16 channels written as 32 bytes).
__global__ void input_kernel(const float* __restrict__ V, const float* __restrict__ G, int L, size_t P, float sv,
                             float sg, bf16* __restrict__ x) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
    __align__(16) bf16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      float a = 0.f;
      if (c < L) a = sv * V[(size_t)c * P + p];
      else if (c < 2 * L) a = sg * G[(size_t)(c - L) * P + p];
      v[c] = __float2bfloat16_rn(a);
    }
    uint4* dst = reinterpret_cast<uint4*>(x + p * 16);
    dst[0] = reinterpret_cast<const uint4*>(v)[0];
    dst[1] = reinterpret_cast<const uint4*>(v)[1];
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
// pre-activation (bf16 NHWC, padded channels 0); per-block loss partials (FP64).
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ pre, const float* __restrict__ target, int L,
                                                   size_t P, float inv_sd, bf16* __restrict__ g,
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
    g[i] = __float2bfloat16_rn(gv);
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

// out = sum of the 512 loss partials: a fixed-order tree over one block of 512 threads.
__global__ void __launch_bounds__(512) loss_sum_kernel(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double s[512];
  s[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int h = 256; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = s[0];
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
size_t packed_fwd_elems(const Layer& l) { return (size_t)9 * l.cin * l.cout; }
size_t packed_dgrad_elems(const Layer& l) { return (size_t)9 * l.cin * l.cout; }

struct Ws {
  int* err;
  double* loss_part;            // [512]
  bf16* x;                      // [P][16] input, NHWC
  bf16* act[kLayers - 1];       // [P][64] outputs of the hidden layers (gelu), NHWC
  float* pre[kLayers];          // [P][cout] FP32: gelu' of the hidden layers' pre-activations (training),
                                // the last layer's pre-activation
  bf16* g[2];                   // [P][64] gradients of a pre-activation, NHWC (ping-pong)
  bf16* Bf[kLayers];            // packed forward weights
  bf16* Bd[kLayers];            // packed data-gradient weights
  float* part;                  // [kMaxSpatial][9][64][64] weight-gradient partials
  float* bpart;                 // [kMaxSpatial][64] bias-gradient partials
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
  for (int i = 0; i < kLayers - 1; ++i) w.act[i] = (bf16*)take(P * kHid * 2);
  for (int i = 0; i < kLayers; ++i) w.pre[i] = (float*)take(P * n.layer[i].cout * 4);
  for (int i = 0; i < 2; ++i) w.g[i] = (bf16*)take(P * kHid * 2);
  for (int i = 0; i < kLayers; ++i) {
    w.Bf[i] = (bf16*)take(packed_fwd_elems(n.layer[i]) * 2);
    w.Bd[i] = (bf16*)take(packed_dgrad_elems(n.layer[i]) * 2);
  }
  w.part = (float*)take((size_t)kMaxSpatial * 9 * kHid * kHid * 4);
  w.bpart = (float*)take((size_t)kMaxSpatial * kHid * 4);
  w.grad = (float*)take(n.n_params * 4);
  w.bytes = off;
  return w;
}

msp_status fail(msp_status s, const std::string& m) { return set_last_error(s, m); }

// Tensor map of an NHWC bf16 image [H][Wd][C] for the convolution's row loads: boxes of
// 8 channels x 130 pixels x 1 row, zero fill outside.  The encoder comes from the driver
// through the runtime's entry-point query.
cudaError_t encode_rows_map(CUtensorMap* map, const bf16* img, int C, int Wd, int H) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static const Encode encode = [] {   // looked up once (thread-safe static initialisation)
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? reinterpret_cast<Encode>(fn) : nullptr;
  }();
  if (!encode) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)Wd, (cuuint64_t)H};
  const cuuint64_t strides[2] = {(cuuint64_t)C * 2, (cuuint64_t)Wd * C * 2};
  const cuuint32_t box[3] = {8, 130, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(img), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CIN, int COUT, int EPI>
cudaError_t launch_conv(const bf16* in, const bf16* Bp, const float* bias, const float* aux, float* pre, bf16* out,
                        int nbias, int H, int Wd, int* err, cudaStream_t st) {
  static int resident[64] = {};   // co-resident CTAs per SM (shared memory, threads, tensor memory)
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!resident[dev]) {
    cudaError_t e = cudaFuncSetAttribute(conv_kernel<CIN, COUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)conv_smem<CIN, COUT>());
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv_kernel<CIN, COUT, EPI>, kConvThreads,
                                                      conv_smem<CIN, COUT>());
    if (e != cudaSuccess) return e;
    resident[dev] = std::max(1, std::min(occ, (int)(512 / (2 * Conv<CIN, COUT>::TC))));
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int strips = Wd / kPix;
  const int want = std::max(1, sms * resident[dev] / strips);   // CTAs along the rows
  const int rows = (H + std::min(want, H) - 1) / std::min(want, H);
  const int ny = (H + rows - 1) / rows;
  alignas(64) CUtensorMap tmap;
  const cudaError_t me = encode_rows_map(&tmap, in, CIN, Wd, H);
  if (me != cudaSuccess) return me;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3((unsigned)strips, (unsigned)ny);
  cfg.blockDim = dim3(kConvThreads);
  cfg.dynamicSmemBytes = conv_smem<CIN, COUT>();
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, conv_kernel<CIN, COUT, EPI>, in, Bp, bias, aux, pre, out, nbias, H, Wd,
                                           rows, err, tc_wait_limit(), tmap);
  count_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t conv(int cin, int cout, int epi, const bf16* in, const bf16* Bp, const float* bias, const float* aux,
                 float* pre, bf16* out, int nbias, int H, int Wd, int* err, cudaStream_t st) {
#define MSP_CONV(CI, CO, E) \
  if (cin == CI && cout == CO && epi == E) return launch_conv<CI, CO, E>(in, Bp, bias, aux, pre, out, nbias, H, Wd, err, st);
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

// Weight and bias gradients of one convolution into the parameter layout (dW [cout_true][9]
// [cin_true], db [cout_true]): the partial-sum kernel over (strips x row runs x 2 tap groups), then
// the fixed-order reduction.
template <int CIN, int COUT>
cudaError_t launch_wgrad(const bf16* g, const bf16* in, float* part, float* bpart, int cout_true, int cin_true,
                         float* dW, float* db, int H, int Wd, int* err, cudaStream_t st) {
  using C = WGrad<CIN, COUT>;
  static int resident[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!resident[dev]) {
    cudaError_t e = cudaFuncSetAttribute(wgrad_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, wgrad_kernel<CIN, COUT>, kThreads, C::SMEM);
    if (e != cudaSuccess) return e;
    resident[dev] = std::max(1, std::min(occ, (int)(512 / C::TC)));
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int strips = Wd / kPix;
  int want = std::max(1, std::min(sms * resident[dev] / 2, kMaxSpatial) / strips);
  want = std::min(want, H);
  const int rows = (H + want - 1) / want;
  const int ny = (H + rows - 1) / rows;
  alignas(64) CUtensorMap gmap, imap;
  cudaError_t me = encode_rows_map(&gmap, g, COUT, Wd, H);
  if (me == cudaSuccess) me = encode_rows_map(&imap, in, CIN, Wd, H);
  if (me != cudaSuccess) return me;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3((unsigned)strips, (unsigned)ny, 2u);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, wgrad_kernel<CIN, COUT>, part, bpart, H, rows, err, tc_wait_limit(),
                                     gmap, imap);
  if (e != cudaSuccess) return e;
  const int nred = 9 * COUT * CIN + cout_true;
  wgrad_reduce_kernel<<<(nred + 255) / 256, 256, 0, st>>>(part, bpart, strips * ny, COUT, CIN, cout_true, cin_true,
                                                          dW, db);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t wgrad(int cin, int cout, const bf16* g, const bf16* in, float* part, float* bpart, int cout_true,
                  int cin_true, float* dW, float* db, int H, int Wd, int* err, cudaStream_t st) {
#define MSP_WGRAD(CI, CO) \
  if (cin == CI && cout == CO) return launch_wgrad<CI, CO>(g, in, part, bpart, cout_true, cin_true, dW, db, H, Wd, err, st);
  MSP_WGRAD(16, 64)
  MSP_WGRAD(64, 64)
  MSP_WGRAD(64, 16)
  MSP_WGRAD(16, 16)
#undef MSP_WGRAD
  return cudaErrorInvalidValue;
}

int grid1d(size_t n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

// Packs every layer's forward (and, for training, data-gradient) operand from the FP32 weights,
// in one launch: blockIdx.y is the layer, blockIdx.z the operand.
struct PackJob {
  const float* w[kLayers];
  bf16* Bf[kLayers];
  bf16* Bd[kLayers];
  int cin_true[kLayers], cout_true[kLayers], cin[kLayers], cout[kLayers];
};

__global__ void pack_all_kernel(PackJob job) {
  const int i = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int CIN = job.cin[i], COUT = job.cout[i], cit = job.cin_true[i], cot = job.cout_true[i];
  if (idx >= 9 * COUT * CIN) return;
  const float* w = job.w[i];
  if (blockIdx.z == 0) {
    const int t = idx / (COUT * CIN), co = (idx / CIN) % COUT, ci = idx % CIN;
    const float v = (ci < cit && co < cot) ? w[((size_t)co * 9 + t) * cit + ci] : 0.f;
    job.Bf[i][packed_off(t, co, ci, CIN, COUT)] = __float2bfloat16_rn(v);
  } else if (i > 0) {
    const int t = idx / (COUT * CIN), ci = (idx / COUT) % CIN, co = idx % COUT;
    const float v = (ci < cit && co < cot) ? w[((size_t)co * 9 + (8 - t)) * cit + ci] : 0.f;
    job.Bd[i][packed_off(t, ci, co, COUT, CIN)] = __float2bfloat16_rn(v);
  }
}

cudaError_t pack_all(const Net& n, const float* params, const Ws& w, bool dgrad, cudaStream_t st) {
  PackJob job{};
  int most = 0;
  for (int i = 0; i < kLayers; ++i) {
    const Layer& l = n.layer[i];
    job.w[i] = params + l.w_off;
    job.Bf[i] = w.Bf[i];
    job.Bd[i] = w.Bd[i];
    job.cin_true[i] = l.cin_true;
    job.cout_true[i] = l.cout_true;
    job.cin[i] = l.cin;
    job.cout[i] = l.cout;
    most = std::max(most, 9 * l.cin * l.cout);
  }
  pack_all_kernel<<<dim3((unsigned)((most + 255) / 256), (unsigned)kLayers, dgrad ? 2u : 1u), 256, 0, st>>>(job);
  count_launches(1);
  return cudaGetLastError();
}

// Forward through the six layers from the packed input.  For training (`train`) every layer also
// keeps its FP32 pre-activation (the backward pass reads it); the proposal alone needs only the
// last layer's.
cudaError_t forward(const Net& n, const float* params, const Ws& w, int H, int Wd, bool train, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < kLayers && e == cudaSuccess; ++i) {
    const Layer& l = n.layer[i];
    const bf16* in = i == 0 ? w.x : w.act[i - 1];
    const bool last = i == kLayers - 1;
    e = conv(l.cin, l.cout, last ? EPI_NONE : EPI_GELU, in, w.Bf[i], params + l.b_off, nullptr,
             (last || train) ? w.pre[i] : nullptr, last ? nullptr : w.act[i], l.cout_true, H, Wd, w.err, st);
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
  input_kernel<<<grid1d(P), 256, 0, cs>>>(V, G, L, P, (float)s->scale_v, (float)s->scale_g, w.x);
  count_launches(1);
  LEARN_CK(forward(n, params, w, H, Wd, false, cs));
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
  input_kernel<<<grid1d(P), 256, 0, cs>>>(V, G, L, P, (float)s->scale_v, (float)s->scale_g, w.x);
  count_launches(1);
  LEARN_CK(forward(n, params, w, H, Wd, true, cs));
  const int lb = 512;
  loss_kernel<<<lb, 256, 0, cs>>>(w.pre[kLayers - 1], target, L, P, (float)(1.0 / s->scale_d), w.g[0],
                                  w.loss_part);
  count_launches(1);
  if (loss_out) {
    loss_sum_kernel<<<1, lb, 0, cs>>>(w.loss_part, loss_out);
    count_launches(1);
  }
  // backward, last layer first: g[cur] holds the gradient of layer i's pre-activation
  int cur = 0;
  for (int i = kLayers - 1; i >= 0; --i) {
    const Layer& l = n.layer[i];
    const bf16* in = i == 0 ? w.x : w.act[i - 1];
    LEARN_CK(wgrad(l.cin, l.cout, w.g[cur], in, w.part, w.bpart, l.cout_true, l.cin_true, grad + l.w_off,
                   grad + l.b_off, H, Wd, w.err, cs));
    if (i > 0) {   // gradient of the previous layer's pre-activation: conv with mirrored weights x gelu'
      LEARN_CK(conv(l.cout, l.cin, EPI_GELU_GRAD, w.g[cur], w.Bd[i], nullptr, w.pre[i - 1], nullptr, w.g[1 - cur],
                    0, H, Wd, w.err, cs));
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
  return align256(sizeof(int)) + align256((size_t)9 * c_in * c_out * 2) +
         align256((size_t)kMaxSpatial * 9 * c_out * c_in * 4) + align256((size_t)kMaxSpatial * 64 * 4);
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
  const size_t ne = (size_t)9 * c_in * c_out;
  pack_fwd_kernel<<<grid1d(ne), 256, 0, cs>>>(w, c_in, c_out, c_in, c_out, Bp);
  count_launches(1);
  LEARN_CK(conv(c_in, c_out, EPI_NONE, (const bf16*)in_bf16, Bp, bias, nullptr, pre_out, nullptr,
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
  char* b = (char*)ws;
  int* err = (int*)b;
  size_t off = align256(sizeof(int)) + align256((size_t)9 * c_in * c_out * 2);
  float* part = (float*)(b + off);
  off += align256((size_t)kMaxSpatial * 9 * c_out * c_in * 4);
  float* bpart = (float*)(b + off);
  LEARN_CK(cudaMemsetAsync(err, 0, sizeof(int), cs));
  LEARN_CK(wgrad(c_in, c_out, (const bf16*)grad_pre_bf16, (const bf16*)in_bf16, part, bpart, c_out, c_in, dW, db,
                 height, width, err, cs));
  LEARN_CK(cudaGetLastError());
  return MSP_OK;
}

}  // extern "C"
