// msp_tcdft.cu -- the W-point DFT as a matrix product on the 5th-generation tensor cores, with
// 3-term split-BF16 operands and FP32 accumulation (the split-BF16 precision form).
//
// Sec. 6 of the paper proposes replacing the successive Fourier transforms of the multislice
// model by matrix products.  One pass here transforms every row of a batch of W x W waves:
//   Y[l][n] = sum_m X[l][m] exp(-+2 pi i m n / W)        (l: line, all rows of all waves)
// and stores each wave's result transposed, so two passes are the 2-D DFT with the result back
// in row-major order (Y = F X F, F symmetric).
//
// Real form.  With the complex inputs interleaved (re, im) along K, row l of A is the line as
// stored, K = 2W, and the real output columns of one N tile are [Re y_n | Im y_n] for n in the
// tile:  B'[Re n][2m] = Fr[m][n], B'[Re n][2m+1] = -Fi[m][n], B'[Im n][2m] = Fi[m][n],
// B'[Im n][2m+1] = Fr[m][n], so that D = A B'^T (tcgen05: D in tensor memory, A and B K-major).
//
// Precision.  x = x_hi + x_lo with x_hi = bf16(x) and x_lo = bf16(x - x_hi) (16 mantissa bits of
// x kept); D accumulates A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 (the tensor core's
// accumulation); the neglected A_lo B_lo term and the bits of x beyond x_lo leave about 2^-16
// relative error per product.  B' is formed in double and split once per call.
//
// Structure (one CTA of 256 threads per 128 lines and N tile; one tcgen05.mma issuer):
//   for each K chunk of 64 (32 complex inputs): the threads split the lines' chunk into
//   bf16 (hi, lo) parts and store them, with the chunk of B', in the canonical no-swizzle
//   K-major layout (core matrices of 8 rows x 16 bytes); one thread issues 4 K-steps x 3
//   products of M = 128, N = NT, K = 16 (kind::f16, bf16 operands) and commits them to an
//   mbarrier that the next chunk waits for (bounded: the error word records a timeout).
//   Then every warp reads its lanes' accumulators (tcgen05.ld) and stores the transposed result.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "msp_tc.cuh"

namespace msp {
namespace tcdft {

using tc::kmaj16;
using tc::idesc_bf16;
using tc::mma_bf16;
using tc::wait_phase;

constexpr int kM = 128;        // lines per CTA
constexpr int kKC = 64;        // real K per chunk (32 complex inputs)
constexpr int kThreads = 256;
constexpr int kDrainLimit = 1 << 20;

__host__ __device__ constexpr int n_tile(int W) { return 2 * W < 256 ? 2 * W : 256; }   // real columns per N tile
__host__ __device__ constexpr int n_tiles(int W) { return 2 * W / n_tile(W); }
__host__ __device__ constexpr int n_chunks(int W) { return 2 * W / kKC; }
// bf16 elements of one (tile, chunk, part) block of B': NT rows x kKC
__host__ __device__ constexpr size_t block_elems(int W) { return (size_t)n_tile(W) * kKC; }


// B' of the W-point DFT (sign -1: forward, +1: inverse) as split bf16, laid out block by block:
// block (tile t, chunk c, part p) at ((t * n_chunks + c) * 2 + p) * block_elems, each block in
// the canonical layout above.  One thread per (row, complex input m) of the full 2W x 2W matrix.
__global__ void matrix_kernel(__nv_bfloat16* __restrict__ mat, int W, int sign) {
  const int NT = n_tile(W), NC = n_chunks(W);
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * W * W) return;
  const int row = idx / W, m = idx % W;            // row of B' (over all tiles), complex input m
  const int t = row / NT, i = row % NT;            // tile, row within the tile
  const int n = t * (NT / 2) + (i % (NT / 2));     // complex output of this row
  const bool im_row = i >= NT / 2;
  double s, c;
  sincospi(2.0 * sign * (double)((m * n) % W) / (double)W, &s, &c);
  // (value at K = 2m, value at K = 2m + 1)
  const double v0 = im_row ? s : c, v1 = im_row ? c : -s;
  const int k0 = 2 * m, chunk = k0 / kKC, kk = k0 % kKC;
  const double vals[2] = {v0, v1};
  for (int q = 0; q < 2; ++q) {
    const float x = (float)vals[q];
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    const size_t b0 = ((size_t)(t * NC + chunk) * 2) * block_elems(W);
    const uint32_t off = kmaj16(i, kk + q) / 2;
    mat[b0 + off] = hi;
    mat[b0 + block_elems(W) + off] = lo;
  }
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}


// One pass: out[b][n][r] = sum_m in[b][r][m] w^(m n) for every wave b < nb (see the file comment).
// `in` and `out` must not overlap.  err: 2 = a wait for the tensor core ran out (results invalid),
// 3 = the wait for the CTA's own MMAs before releasing tensor memory ran out as well.
template <int W>
__global__ void __launch_bounds__(kThreads, 1) pass_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                           int nb, const __nv_bfloat16* __restrict__ mat,
                                                           int* __restrict__ err, int wait_limit) {
  constexpr int NT = n_tile(W), NC = n_chunks(W);
  constexpr uint32_t A_BYTES = kM * kKC * 2, B_BYTES = NT * kKC * 2;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* a_hi = smem;
  uint8_t* a_lo = a_hi + A_BYTES;
  uint8_t* b_hi = a_lo + A_BYTES;
  uint8_t* b_lo = b_hi + B_BYTES;
  uint64_t* bar = reinterpret_cast<uint64_t*>(b_lo + B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  volatile int* flag = reinterpret_cast<volatile int*>(tslot + 1);   // 0 ok, 2 timed out

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lines = nb * W;
  const int row0 = blockIdx.x * kM;
  const int tile = blockIdx.y;
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
    *flag = 0;
  }
  if (warp == 0) tc::tmem_alloc(tslot, NT);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = idesc_bf16(kM, NT);

  // this thread's share of the A chunk: line r, complex inputs 16 h .. 16 h + 15 of the chunk
  const int r = tid >> 1, h = tid & 1;
  const int line = row0 + r;
  const bool live = line < lines;
  int issued = -1;
#pragma unroll 1
  for (int c = 0; c < NC; ++c) {
    if (c > 0) {   // the previous chunk's MMAs must be done reading shared memory
      if (tid == 0 && !wait_phase(bar, (uint32_t)((c - 1) & 1), wait_limit)) *flag = 2;
      __syncthreads();
      if (*flag) break;
    }
    // A: split the chunk's 16 complex values of line r into bf16 (hi, lo), 4 x 16 bytes per part
    {
      const float4* src = reinterpret_cast<const float4*>(in + (size_t)line * W + c * (kKC / 2) + 16 * h);
#pragma unroll
      for (int q = 0; q < 4; ++q) {   // 8 consecutive real K = 4 complex values per 16-byte row piece
        float v[8];
        if (live) {
          const float4 f0 = src[2 * q], f1 = src[2 * q + 1];
          v[0] = f0.x; v[1] = f0.y; v[2] = f0.z; v[3] = f0.w;
          v[4] = f1.x; v[5] = f1.y; v[6] = f1.z; v[7] = f1.w;
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = 0.f;
        }
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * e]), h1 = __float2bfloat16_rn(v[2 * e + 1]);
          const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * e] - __bfloat162float(h0));
          const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * e + 1] - __bfloat162float(h1));
          hi[e] = pack2(h0, h1);
          lo[e] = pack2(l0, l1);
        }
        const uint32_t off = kmaj16(r, 32 * h + 8 * q);
        *reinterpret_cast<uint4*>(a_hi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(a_lo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
    // B: the chunk's blocks of B' are stored in the layout the MMA reads; copy them
    {
      const uint4* bh = reinterpret_cast<const uint4*>(mat + ((size_t)(tile * NC + c) * 2) * block_elems(W));
      const uint4* bl = bh + block_elems(W) / 8;
      for (int i = tid; i < (int)(B_BYTES / 16); i += kThreads) {
        reinterpret_cast<uint4*>(b_hi)[i] = bh[i];
        reinterpret_cast<uint4*>(b_lo)[i] = bl[i];
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t ah = tc::smem_u32(a_hi), al = tc::smem_u32(a_lo);
      const uint32_t bh = tc::smem_u32(b_hi), bl = tc::smem_u32(b_lo);
#pragma unroll
      for (int s = 0; s < kKC / 16; ++s) {   // K = 16 bf16 (two core matrices) per MMA
        const uint32_t ko = s * 256;
        const uint64_t dah = tc::smem_desc(ah + ko, 128, 1024), dal = tc::smem_desc(al + ko, 128, 1024);
        const uint64_t dbh = tc::smem_desc(bh + ko, 128, 1024), dbl = tc::smem_desc(bl + ko, 128, 1024);
        mma_bf16(tmem, dah, dbh, idesc, (c > 0 || s > 0) ? 1u : 0u);
        mma_bf16(tmem, dah, dbl, idesc, 1u);
        mma_bf16(tmem, dal, dbh, idesc, 1u);
      }
      tc::commit(bar);
    }
    issued = c;
  }
  // the last chunk's MMAs
  if (!*flag && issued == NC - 1) {
    if (tid == 0 && !wait_phase(bar, (uint32_t)((NC - 1) & 1), wait_limit)) *flag = 2;
  }
  __syncthreads();
  tc::fence_after();
  if (!*flag) {
    // epilogue: warp w reads lanes 32 (w % 4) .. + 31 (lines), complex outputs of half w / 4
    const int q = warp & 3, half = warp >> 2;
    const int l = row0 + 32 * q + lane;
    const bool ok = l < lines;
    const int b = l / W, rr = l % W;
#pragma unroll 1
    for (int j0 = half * (NT / 4); j0 < (half + 1) * (NT / 4); j0 += 16) {
      uint32_t re[16], im[16];
      const uint32_t base = tmem + ((uint32_t)(32 * q) << 16);
      tc::tmem_ld16(base + (uint32_t)j0, re);
      tc::tmem_ld16(base + (uint32_t)(NT / 2 + j0), im);
      tc::tmem_wait_ld();
      if (ok) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int n = tile * (NT / 2) + j0 + u;
          out[((size_t)b * W + n) * W + rr] = make_float2(__uint_as_float(re[u]), __uint_as_float(im[u]));
        }
      }
    }
  }
  // no MMA may still write tensor memory when it is released
  if (tid == 0 && *flag && issued >= 0 && !wait_phase(bar, (uint32_t)(issued & 1), kDrainLimit)) *flag = 3;
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, NT);
  }
  if (tid == 0 && *flag) atomicMax(err, *flag);
}

template <int W>
constexpr size_t smem_bytes() {
  return 1024 + 2 * (size_t)kM * kKC * 2 + 2 * (size_t)n_tile(W) * kKC * 2 + 64;
}

template <int W>
static cudaError_t launch_pass(const float2* in, float2* out, int nb, const __nv_bfloat16* mat, int* err, int wait_limit,
                               cudaStream_t st) {
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_done[dev]) {
    const cudaError_t e =
        cudaFuncSetAttribute(pass_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<W>());
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  const dim3 grid((unsigned)((nb * W + kM - 1) / kM), (unsigned)n_tiles(W));
  pass_kernel<W><<<grid, kThreads, smem_bytes<W>(), st>>>(in, out, nb, mat, err, wait_limit);
  return cudaGetLastError();
}

}  // namespace tcdft

// Bytes of the split-bf16 DFT matrix of one direction for window W.
size_t tcdft_matrix_bytes(int W) { return (size_t)tcdft::n_tiles(W) * tcdft::n_chunks(W) * 2 * tcdft::block_elems(W) * 2; }

// Builds the split-bf16 DFT matrix of one direction (inverse: the unnormalised inverse).
cudaError_t tcdft_prepare(int W, int inverse, void* mat, cudaStream_t st) {
  const int n = 2 * W * W;
  tcdft::matrix_kernel<<<(n + 255) / 256, 256, 0, st>>>((__nv_bfloat16*)mat, W, inverse ? 1 : -1);
  return cudaGetLastError();
}

// out[b][n][r] = sum_m in[b][r][m] w^(m n) over nb waves (one tensor-core pass; see above).
cudaError_t tcdft_pass(int W, const float2* in, float2* out, int nb, const void* mat, int* err, int wait_limit,
                       cudaStream_t st) {
  const __nv_bfloat16* m = (const __nv_bfloat16*)mat;
  if (W == 64) return tcdft::launch_pass<64>(in, out, nb, m, err, wait_limit, st);
  if (W == 128) return tcdft::launch_pass<128>(in, out, nb, m, err, wait_limit, st);
  return tcdft::launch_pass<256>(in, out, nb, m, err, wait_limit, st);
}

}  // namespace msp
