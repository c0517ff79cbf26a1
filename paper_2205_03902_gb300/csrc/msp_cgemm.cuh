// msp_cgemm.cuh -- dense complex contraction on the 5th-generation tensor cores (tcgen05,
// kind::tf32 with operands split into tf32 pairs), shared by the sparse-decomposition matrix
// step and the batched 2-D DFT.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "msp_tc.cuh"

namespace msp {

// ---------------------------------------------------------------------------
// dense complex contraction on the tensor cores (tcgen05, 3xTF32)
// ---------------------------------------------------------------------------
// C_z = A[:, K_z] op(B)[K_z, :] for the K range K_z of blockIdx.z.  A: M x K column-major.
// op(B) = B (K x N column-major) or, with B_CONJ_T, B^H for B stored N x K column-major.
// C: M x N column-major, partial z at C + z * c_stride.
//
// One CTA computes a 128 x 128 complex tile as two real products sharing one B operand,
//   Re C = [Ar, -Ai] B'^T,  Im C = [Ai, Ar] B'^T,  B' rows n: [Br, Bi],
// each an M = 128, N = 128 MMA per 8 real K into its own TMEM accumulator (columns 0..127 Re,
// 128..255 Im).  Both A operands are windows of one TMEM layout per row, [Ai | Ar | -Ai], so B
// is split and stored once, without duplicates.  Every real operand x is split into tf32
// parts x = big + small and D accumulates big*big + big*small + small*big, which keeps the
// product error near FP32's.  The tensor core's FP32 accumulation does not round to
// nearest, so D accumulates over groups of GROUP K-tiles only; after each group the
// producers add D into FP32 registers (128 per thread) and release it (`dfree` mbarrier)
// before the next group overwrites it.
//
// Warps 0..7 are producers.  They copy the raw complex K-tiles of A and B into shared
// memory with cp.async, one tile ahead of the one they convert, so that no register waits
// on a global load.  They split each tile and write [Ai | Ar | -Ai] into tensor memory (row m
// in lane m, its K in consecutive columns; tcgen05.st) and B' in the canonical no-swizzle
// K-major layout into shared memory: a 2-stage ring (`full` mbarriers, one arrival per
// producer thread).  A read from tensor memory costs no shared-memory bandwidth.  Warp 8
// allocates TMEM and one of its threads issues the MMAs; a tcgen05.commit to the stage's
// `empty` mbarrier hands the stage back once the MMAs have read it.  Every wait is bounded
// (by `wait_limit` polls): on timeout the CTA raises *err = 2 and stops; the MMA thread
// still waits, bounded, for the MMAs it issued before the TMEM is freed.  If that drain wait
// runs out too, the CTA raises *err = 3 instead: tensor memory may then be released while
// MMAs still write it, and the host treats the device as untrusted.
namespace gemm {
constexpr int TM = 128, TN = 128, TK = 16;                  // complex tile and K-tile
constexpr int KR = 2 * TK;                                  // real K per tile
constexpr uint32_t B_BYTES = TN * KR * 4;                   // one tf32 part of B': 16 KB
constexpr uint32_t STAGE_BYTES = 2 * B_BYTES;               // 32 KB of shared memory
constexpr int STAGES = 2;
constexpr int GROUP = 8;
constexpr int NPROD = 256;
constexpr int NTHREADS = NPROD + 32;
constexpr int CPT = TN / 2;                                 // complex columns of C per producer thread
constexpr uint32_t DCOLS = 2 * TN;                          // f32 columns of the accumulators (Re, Im)
constexpr uint32_t ACOL = DCOLS;                            // first TMEM column of the A stages
constexpr uint32_t APART = 3 * TK;                          // columns of one tf32 part: [Ai | Ar | -Ai]
constexpr uint32_t TMEM_COLS = 512;                         // accumulators + STAGES x (big, small) A
static_assert(ACOL + STAGES * 2 * APART <= TMEM_COLS, "tensor memory of one CTA");
// raw complex K-tiles as they come from global memory: RAW slots, RAW - 1 tiles in flight
constexpr int RAW = 2;
constexpr int RB_LD = TK + 2;                               // padded row of a raw B tile [j][k]
constexpr uint32_t RAW_A_BYTES = TK * TM * 8;               // [k][i] float2: 16 KB
constexpr uint32_t RAW_B_BYTES = (TN * RB_LD > TK * TN ? TN * RB_LD : TK * TN) * 8;
constexpr uint32_t RAW_BYTES = RAW_A_BYTES + RAW_B_BYTES;
constexpr uint32_t SMEM_BYTES = STAGES * STAGE_BYTES + RAW * RAW_BYTES + 1024 + 128;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory of one CTA");
constexpr int kWaitLimit = 1 << 20;   // default polls (with 32 ns pauses) per wait: well under a second

// Bounded wait of at most `limit` polls; gives up early once another thread has raised the
// abort flag, and raises it when the limit runs out.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int limit) {
  for (int i = 0; i < limit; ++i) {
    if (tc::mbar_test(bar, parity)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
    if (i > 64) __nanosleep(32);
  }
  *abort_flag = 1;
  return false;
}

// Warp-uniform wait: lane 0 waits, every lane gets the verdict.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int limit) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = wait_or_abort(bar, parity, abort_flag, limit) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Bounded wait that ignores the abort flag: the MMA thread's wait for its own last commit,
// so that no MMA is still writing tensor memory when it is freed.
__device__ __forceinline__ bool drain_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kWaitLimit; ++i) {
    if (tc::mbar_test(bar, parity)) return true;
    if (i > 64) __nanosleep(32);
  }
  return false;
}

// Byte offset of real element (row, k) in a K-major operand: core matrices of 8 rows x 4
// tf32, 128 bytes apart along K, KR/4 * 128 bytes apart along rows.
__device__ __forceinline__ uint32_t kmaj(int row, int k) {
  return (uint32_t)((k >> 2) * 128 + (row >> 3) * (KR / 4) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

struct Split4 {
  uint4 big, small;
};

// big = x rounded to tf32 (nearest, ties away: add half a tf32 ulp, clear the 13 low bits, two
// integer operations instead of the conversion unit); small = x - big, exact in FP32, handed
// over unrounded (the tensor core reads the 19 high bits of a tf32 operand, so small loses at
// most 2^-10 of itself, 2^-21 of x).
__device__ __forceinline__ uint32_t tf32_big(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }

__device__ __forceinline__ Split4 split4(float x0, float x1, float x2, float x3) {
  Split4 r;
  r.big = make_uint4(tf32_big(x0), tf32_big(x1), tf32_big(x2), tf32_big(x3));
  r.small = make_uint4(__float_as_uint(x0 - __uint_as_float(r.big.x)), __float_as_uint(x1 - __uint_as_float(r.big.y)),
                       __float_as_uint(x2 - __uint_as_float(r.big.z)), __float_as_uint(x3 - __uint_as_float(r.big.w)));
  return r;
}

__device__ __forceinline__ Split4 neg(const Split4& v) {   // rounding is symmetric: split(-x) = -split(x)
  Split4 r;
  r.big = make_uint4(v.big.x ^ 0x80000000u, v.big.y ^ 0x80000000u, v.big.z ^ 0x80000000u, v.big.w ^ 0x80000000u);
  r.small = make_uint4(v.small.x ^ 0x80000000u, v.small.y ^ 0x80000000u, v.small.z ^ 0x80000000u,
                       v.small.w ^ 0x80000000u);
  return r;
}

__device__ __forceinline__ void put(uint8_t* big, uint8_t* small, uint32_t off, const Split4& v) {
  *reinterpret_cast<uint4*>(big + off) = v.big;
  *reinterpret_cast<uint4*>(small + off) = v.small;
}

// Copies `bytes` (0, 8 or 16) from global src into 16 bytes at shared dst, zero-filling the
// rest; vec16: one 16-byte copy (src and dst 16-byte aligned), else two 8-byte copies.
__device__ __forceinline__ void copy_pair(uint8_t* dst, const float2* src, const float2* safe, int bytes, bool vec16) {
  const uint32_t d = tc::smem_u32(dst);
  if (vec16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(bytes > 0 ? src : safe), "r"(bytes)
                 : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(bytes >= 8 ? src : safe),
                 "r"(bytes >= 8 ? 8 : 0)
                 : "memory");
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d + 8), "l"(bytes >= 16 ? src + 1 : safe),
                 "r"(bytes >= 16 ? 8 : 0)
                 : "memory");
  }
}
__device__ __forceinline__ void copy_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// this thread's copies of all but the newest `pending` groups are complete
template <int pending>
__device__ __forceinline__ void copy_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(pending) : "memory"); }
__device__ __forceinline__ void copy_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// barrier of the NPROD producer threads only (the MMA warp never joins it)
__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NPROD) : "memory"); }

// Adds the accumulator into this thread's registers: TMEM lane (row) 32 (warp & 3) + lane,
// columns CPT (warp >> 2) + q (Re) and TN + CPT (warp >> 2) + q (Im), q < CPT.
__device__ __forceinline__ void flush(uint32_t tmem, int warp, float (&re)[CPT], float (&im)[CPT]) {
  const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(CPT * (warp >> 2));
#pragma unroll
  for (int part = 0; part < CPT / 16; ++part) {
    uint32_t r[16], u[16];
    tc::tmem_ld16(base + 16 * part, r);
    tc::tmem_ld16(base + TN + 16 * part, u);
    tc::tmem_wait_ld();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      re[16 * part + q] += __uint_as_float(r[q]);
      im[16 * part + q] += __uint_as_float(u[q]);
    }
  }
}
}  // namespace gemm

// STORE_T: element (i, j) of C goes to C[((j / ldc) * ldc + i) * ldc + j % ldc] instead of
// C[j * ldc + i]: with ldc = W and the columns j = (image s, row r) of a batch of W x W
// images, each W x W block is stored transposed (used by the batched 2-D DFT).
template <bool B_CONJ_T, bool STORE_T = false>
__global__ void __launch_bounds__(gemm::NTHREADS, 1) cgemm_kernel(int M, int N, int K, int k_chunk,
                                                                  const float2* __restrict__ A, size_t lda,
                                                                  const float2* __restrict__ B, size_t ldb,
                                                                  float2* __restrict__ C, size_t ldc,
                                                                  size_t c_stride, int* err, int wait_limit) {
  using namespace gemm;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* raw = smem + STAGES * STAGE_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(raw + RAW * RAW_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* dfree = empty + STAGES;   // the producers have read the accumulator out
  uint32_t* tslot = reinterpret_cast<uint32_t*>(dfree + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* drain_fail = reinterpret_cast<volatile int*>(tslot + 2);   // the MMA thread's drain ran out
  const int t = threadIdx.x, warp = t >> 5;
  const int i0 = blockIdx.x * TM, j0 = blockIdx.y * TN;
  const int kb = blockIdx.z * k_chunk;
  const int ke = min(K, kb + k_chunk);
  const int ntiles = max(0, (ke - kb + TK - 1) / TK);

  if (t == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], NPROD);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(dfree, NPROD);
    tc::fence_mbar_init();
    *abort_flag = 0;
    *drain_fail = 0;
  }
  if (warp == 8) tc::tmem_alloc(tslot, TMEM_COLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 8) {
    if ((t & 31) == 0) {   // MMA issuer
      constexpr uint32_t idesc = tc::idesc_tf32(128, TN);
      int last = -1;   // last tile whose MMAs were committed
      for (int it = 0; it < ntiles; ++it) {
        const int s = it % STAGES;
        // a new group overwrites the accumulator: wait until the last one has been read out
        if (it >= GROUP && it % GROUP == 0 &&
            !wait_or_abort(dfree, ((it / GROUP) - 1) & 1, abort_flag, wait_limit))
          break;
        if (!wait_or_abort(&full[s], (it / STAGES) & 1, abort_flag, wait_limit)) break;
        tc::fence_after();
        const uint32_t bb = tc::smem_u32(smem + s * STAGE_BYTES), bs = bb + B_BYTES;
        // A big and small parts, each [Ai | Ar | -Ai]: Re uses columns TK.., Im columns 0..
        const uint32_t ab = tmem + ACOL + (uint32_t)(s * 2 * APART), as = ab + APART;
        const uint32_t dre = tmem, dim = tmem + TN;
#pragma unroll
        for (int kk = 0; kk < KR / 8; ++kk) {   // K = 8 tf32 (two core matrices) per MMA
          const uint32_t koff = kk * 256;
          const uint64_t dbb = tc::smem_desc(bb + koff, 128, (KR / 4) * 128);
          const uint64_t dbs = tc::smem_desc(bs + koff, 128, (KR / 4) * 128);
          const uint32_t acc = (it % GROUP > 0 || kk > 0) ? 1u : 0u;
          tc::mma_tf32_ta(dre, ab + TK + 8 * kk, dbb, idesc, acc);
          tc::mma_tf32_ta(dre, ab + TK + 8 * kk, dbs, idesc, 1u);
          tc::mma_tf32_ta(dre, as + TK + 8 * kk, dbb, idesc, 1u);
          tc::mma_tf32_ta(dim, ab + 8 * kk, dbb, idesc, acc);
          tc::mma_tf32_ta(dim, ab + 8 * kk, dbs, idesc, 1u);
          tc::mma_tf32_ta(dim, as + 8 * kk, dbb, idesc, 1u);
        }
        tc::commit(&empty[s]);
        last = it;
      }
      // every MMA issued must be done before tensor memory is freed, aborted or not
      if (last >= 0 && !drain_wait(&empty[last % STAGES], (last / STAGES) & 1)) {
        *drain_fail = 1;
        *abort_flag = 1;
      }
    }
  } else {
    float re[CPT], im[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) re[q] = im[q] = 0.f;
    int flushed = 0;
    const int am = t & 127, aq = t >> 7;   // A: row am, complex K 8 aq .. 8 aq + 7 of the tile
    const int bn = t & 127, bq = t >> 7;   // B: column bn, complex K 8 bq .. 8 bq + 7
    // 16-byte copies need 16-byte aligned rows and even offsets of every copied pair
    const bool vec16 = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) == 0 &&
                       (lda & 1) == 0 && (ldb & 1) == 0 && (kb & 1) == 0;
    // copies: A row pair ia, ia + 1 at K rows ka + 4 u of each tile; B four pairs u = 0..3
    const int ka = t >> 6, ia = i0 + 2 * (t & 63);
    const int na = max(0, min(2, M - ia));
    const float2* a_src = A + (na > 0 ? (size_t)(kb + ka) * lda + ia : 0);
    const uint32_t a_dst = (uint32_t)(ka * TM + 2 * (t & 63)) * 8;
    // B^H: K rows kbk + 4 u, columns jb, jb + 1 (nb of them);  B: columns jb + 32 u, K pair kbk
    const int kbk = B_CONJ_T ? (t >> 6) : 2 * (t & 7);
    const int jb = B_CONJ_T ? j0 + 2 * (t & 63) : j0 + (t >> 3);
    const int nb = B_CONJ_T ? max(0, min(2, N - jb)) : 0;
    const float2* b_src = B_CONJ_T ? B + (nb > 0 ? (size_t)(kb + kbk) * ldb + jb : 0) : B + (size_t)jb * ldb + kb + kbk;
    const uint32_t b_dst = B_CONJ_T ? (uint32_t)(kbk * TN + 2 * (t & 63)) * 8 : (uint32_t)((t >> 3) * RB_LD + kbk) * 8;
    // starts the copies of K-tile it into raw slot it % RAW (one commit group, empty past the end)
    auto issue = [&](int it) {
      if (it < ntiles) {
        uint8_t* ra = raw + (it % RAW) * RAW_BYTES;
        uint8_t* rb = ra + RAW_A_BYTES;
        const int k0 = kb + it * TK;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int n = k0 + ka + 4 * u < ke ? na : 0;
          copy_pair(ra + a_dst + u * 4 * TM * 8, n > 0 ? a_src + (size_t)(it * TK + 4 * u) * lda : A, A, 8 * n,
                    vec16);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (B_CONJ_T) {
            const int n = k0 + kbk + 4 * u < ke ? nb : 0;
            copy_pair(rb + b_dst + u * 4 * TN * 8, n > 0 ? b_src + (size_t)(it * TK + 4 * u) * ldb : B, B, 8 * n,
                      vec16);
          } else {
            const int n = jb + 32 * u < N ? max(0, min(2, ke - (k0 + kbk))) : 0;
            copy_pair(rb + b_dst + u * 32 * RB_LD * 8, n > 0 ? b_src + (size_t)32 * u * ldb + it * TK : B, B, 8 * n,
                      vec16);
          }
        }
      }
      copy_commit();
    };
    bool ok = true;
#pragma unroll
    for (int it = 0; it < RAW - 1; ++it) issue(it);
    // Every producer passes producers_sync once per tile, aborted or not, so that none waits
    // at it for a warp that has left.
    for (int it = 0; it < ntiles; ++it) {
      copy_wait<RAW - 2>();  // this thread's copies of tile it have landed
      producers_sync();      // everyone's have; everyone has converted tile it - 1
      issue(it + RAW - 1);   // into the slot tile it - 1 came from
      if (!ok) continue;
      const int s = it % STAGES;
      if (it >= STAGES) {
        ok = warp_wait(&empty[s], ((it / STAGES) - 1) & 1, abort_flag, wait_limit);
        if (!ok) continue;
        tc::fence_after();
      }
      const float2* ra = reinterpret_cast<const float2*>(raw + (it % RAW) * RAW_BYTES);
      const float2* rb = reinterpret_cast<const float2*>(raw + (it % RAW) * RAW_BYTES + RAW_A_BYTES);
      {
        float2 a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = ra[(8 * aq + q) * TM + am];
        const Split4 r0 = split4(a[0].x, a[1].x, a[2].x, a[3].x), r1 = split4(a[4].x, a[5].x, a[6].x, a[7].x);
        const Split4 m0 = split4(a[0].y, a[1].y, a[2].y, a[3].y), m1 = split4(a[4].y, a[5].y, a[6].y, a[7].y);
        // row am, [Ai | Ar | -Ai] per part: this warp's TMEM lanes are 32 (warp & 3) .. + 31
        const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + ACOL + (uint32_t)(s * 2 * APART);
        const Split4 n0 = neg(m0), n1 = neg(m1);
        tc::tmem_st8(ta + 8 * aq, m0.big, m1.big);
        tc::tmem_st8(ta + TK + 8 * aq, r0.big, r1.big);
        tc::tmem_st8(ta + 2 * TK + 8 * aq, n0.big, n1.big);
        tc::tmem_st8(ta + APART + 8 * aq, m0.small, m1.small);
        tc::tmem_st8(ta + APART + TK + 8 * aq, r0.small, r1.small);
        tc::tmem_st8(ta + APART + 2 * TK + 8 * aq, n0.small, n1.small);
      }
      uint8_t* Bb = smem + s * STAGE_BYTES;
      uint8_t* Bs = Bb + B_BYTES;
#pragma unroll
      for (int hq = 0; hq < 2; ++hq) {   // complex K 8 bq + 4 hq .. + 3
        float2 b[4];
        if (B_CONJ_T) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 v = rb[(8 * bq + 4 * hq + q) * TN + bn];
            b[q] = make_float2(v.x, -v.y);
          }
        } else {
          const float4 v0 = *reinterpret_cast<const float4*>(rb + bn * RB_LD + 8 * bq + 4 * hq);
          const float4 v1 = *reinterpret_cast<const float4*>(rb + bn * RB_LD + 8 * bq + 4 * hq + 2);
          b[0] = make_float2(v0.x, v0.y);
          b[1] = make_float2(v0.z, v0.w);
          b[2] = make_float2(v1.x, v1.y);
          b[3] = make_float2(v1.z, v1.w);
        }
        const int k4 = 8 * bq + 4 * hq;
        put(Bb, Bs, kmaj(bn, k4), split4(b[0].x, b[1].x, b[2].x, b[3].x));        // row n: Br
        put(Bb, Bs, kmaj(bn, TK + k4), split4(b[0].y, b[1].y, b[2].y, b[3].y));   //        Bi
      }
      tc::tmem_wait_st();
      tc::fence_proxy_async();
      tc::fence_before();
      tc::mbar_arrive(&full[s]);
      // tile it opens a new group: once the MMAs of the last group are done (the commit of
      // tile it - 1), fold the accumulator in and hand it back to the MMAs of tile it
      if (it >= GROUP && it % GROUP == 0) {
        const int lt = it - 1;
        ok = warp_wait(&empty[lt % STAGES], (lt / STAGES) & 1, abort_flag, wait_limit);
        if (!ok) continue;
        tc::fence_after();
        flush(tmem, warp, re, im);
        tc::fence_before();
        tc::mbar_arrive(dfree);
        ++flushed;
      }
    }
    copy_wait_all();   // no copy may still be writing shared memory when the CTA ends
    // the last tile's commit covers every MMA of the CTA
    if (ok && ntiles > 0) ok = warp_wait(&empty[(ntiles - 1) % STAGES], ((ntiles - 1) / STAGES) & 1, abort_flag, wait_limit);
    tc::fence_after();
    if (ok) {
      const int groups = (ntiles + GROUP - 1) / GROUP;
      while (flushed < groups) {
        flush(tmem, warp, re, im);
        ++flushed;
      }
    }
    const int i = i0 + 32 * (warp & 3) + (t & 31);
    float2* Cz = C + (size_t)blockIdx.z * c_stride;
    if (i < M) {
#pragma unroll
      for (int q = 0; q < CPT; ++q) {
        const int j = j0 + CPT * (warp >> 2) + q;
        if (j < N) {
          const size_t e = STORE_T ? ((size_t)(j / ldc) * ldc + i) * ldc + (size_t)(j % ldc) : (size_t)j * ldc + i;
          Cz[e] = make_float2(re[q], im[q]);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 8) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
  // the most severe outcome wins across CTAs: 3 (drain ran out) over 2 (pipeline wait ran out)
  if (t == 0 && *abort_flag) atomicMax(err, *drain_fail ? 3 : 2);
}

}  // namespace msp
