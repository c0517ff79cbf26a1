// msp_peaks.cu -- stand-alone micro-benchmarks of the two compute pipes the kernels are
// measured against (not part of libmsp; `python bench.py --config peaks` builds and runs it):
//   * FP32 FFMA throughput: every thread of 8 CTAs per SM runs 8 independent FMA chains;
//   * tcgen05.mma kind::tf32 rate, M = 128 and N = 64 / 128 / 256, with A in tensor memory
//     or in shared memory: one CTA per SM, one thread issues R MMAs back to back on fixed
//     operands, then waits (bounded) for their commit.
// Prints one JSON object.
#include <cstdio>
#include <cstdlib>

#include "msp_tc.cuh"

using namespace msp;

#define PK_CK(x)                                                              \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) {                                                  \
      printf("{\"error\": \"%s line %d\"}\n", cudaGetErrorString(e_), __LINE__); \
      exit(2);                                                                \
    }                                                                         \
  } while (0)

constexpr int kFmaIters = 4096;

__global__ void __launch_bounds__(256) ffma_kernel(float* out, float b, float c) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3f + i;
  for (int k = 0; k < kFmaIters; ++k) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == 12345.678f) out[0] = s;   // keeps the chains live
}

constexpr int kMmas = 768;
constexpr int kMmaSmem = 120 * 1024;   // more than half an SM's shared memory: one CTA per SM

// Shared memory: A (128 x 32 tf32, 16 KB) and B (up to 256 x 32 tf32, 32 KB) in the canonical
// no-swizzle K-major layout (core matrices 128 bytes apart along K, 1024 bytes along rows),
// then the mbarrier and the TMEM address slot.  TMEM: D in columns 0..N-1, A at column 256.
template <int N, bool ATMEM>
__global__ void __launch_bounds__(128, 1) mma_rate_kernel(unsigned long long* cycles, int* err) {
  extern __shared__ uint8_t sm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* As = smem;
  uint8_t* Bs = smem + 16384;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 16384 + 32768);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int t = threadIdx.x;
  for (int i = t; i < (16384 + 32768) / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(smem)[i] = 0x3f800000u;
  if (t == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  if (t < 32) tc::tmem_alloc(slot, 512);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  if (t == 0) {
    constexpr uint32_t idesc = tc::idesc_tf32(128, N);
    const uint32_t a = tc::smem_u32(As), b = tc::smem_u32(Bs);
    const unsigned long long c0 = clock64();
    for (int r = 0; r < kMmas; ++r) {
      const int kk = r & 3;
      const uint64_t db = tc::smem_desc(b + kk * 256, 128, 1024);
      if (ATMEM) {
        tc::mma_tf32_ta(tmem, tmem + 256 + 8 * kk, db, idesc, r > 0 ? 1u : 0u);
      } else {
        const uint64_t da = tc::smem_desc(a + kk * 256, 128, 1024);
        tc::mma_tf32(tmem, da, db, idesc, r > 0 ? 1u : 0u);
      }
    }
    const unsigned long long c1 = clock64();
    tc::commit(bar);
    bool done = false;
    for (int i = 0; i < (1 << 22) && !done; ++i) done = tc::mbar_test(bar, 0);
    const unsigned long long c2 = clock64();
    if (!done) atomicExch(err, 1);
    if (blockIdx.x == 0) {
      cycles[0] = c1 - c0;
      cycles[1] = c2 - c0;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (t < 32) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

template <int N, bool ATMEM>
static void mma_rate(unsigned long long* d, int* err, int sms, bool first) {
  PK_CK(cudaFuncSetAttribute(mma_rate_kernel<N, ATMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem));
  for (int i = 0; i < 3; ++i) mma_rate_kernel<N, ATMEM><<<sms, 128, kMmaSmem>>>(d, err);
  PK_CK(cudaGetLastError());
  PK_CK(cudaDeviceSynchronize());
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a);
  mma_rate_kernel<N, ATMEM><<<sms, 128, kMmaSmem>>>(d, err);
  cudaEventRecord(b);
  PK_CK(cudaEventSynchronize(b));
  float ms;
  cudaEventElapsedTime(&ms, a, b);
  unsigned long long h[2];
  int e;
  PK_CK(cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost));
  PK_CK(cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost));
  const double flop = 2.0 * 128 * N * 8 * (double)kMmas * sms;
  printf("%s{\"N\": %d, \"a_operand\": \"%s\", \"issue_cycles_per_mma\": %.1f, \"complete_cycles_per_mma\": %.1f, "
         "\"tflops_incl_launch\": %.1f, \"timed_out\": %d}",
         first ? "" : ", ", N, ATMEM ? "tmem" : "smem", (double)h[0] / kMmas, (double)h[1] / kMmas,
         flop / (ms * 1e-3) / 1e12, e);
}

int main() {
  setvbuf(stdout, nullptr, _IONBF, 0);
  int sms;
  PK_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  float* f;
  PK_CK(cudaMalloc(&f, sizeof(float)));
  const int blocks = sms * 8, threads = 256, reps = 20;
  for (int w = 0; w < 3; ++w) ffma_kernel<<<blocks, threads>>>(f, 0.999f, 1e-3f);
  PK_CK(cudaGetLastError());
  PK_CK(cudaDeviceSynchronize());
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  for (int r = 0; r < reps; ++r) ffma_kernel<<<blocks, threads>>>(f, 0.999f, 1e-3f);
  cudaEventRecord(e1);
  PK_CK(cudaEventSynchronize(e1));
  float ms;
  cudaEventElapsedTime(&ms, e0, e1);
  const double flop = 2.0 * 8 * kFmaIters * (double)blocks * threads * reps;
  printf("{\"sms\": %d, \"ffma_tflops\": %.2f, \"tf32_mma\": [", sms, flop / (ms * 1e-3) / 1e12);
  unsigned long long* d;
  int* err;
  PK_CK(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
  PK_CK(cudaMalloc(&err, sizeof(int)));
  PK_CK(cudaMemset(err, 0, sizeof(int)));
  mma_rate<64, true>(d, err, sms, true);
  mma_rate<128, true>(d, err, sms, false);
  mma_rate<128, false>(d, err, sms, false);
  mma_rate<256, true>(d, err, sms, false);
  mma_rate<256, false>(d, err, sms, false);
  printf("]}\n");
  return 0;
}
