// msp_dft.cu -- batched 2-D DFT as two tensor-core contractions (msp_dft.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <mutex>
#include <string>

#include "msp.h"
#include "msp_cgemm.cuh"
#include "msp_dft.h"

namespace msp {

msp_status set_last_error(msp_status s, const std::string& m);
msp_status refuse_untrusted_device();
void count_launches(int n);
int tc_wait_limit();
msp_status profiled_launch(cudaStream_t st, const std::function<cudaError_t()>& launch);

namespace {

// F[k + x W] = exp(sign 2 pi i (k x mod W) / W), column-major (F is symmetric), in double.
__global__ void dft_matrix_kernel(float2* __restrict__ F, int W, int sign) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= W * W) return;
  const int k = e % W, x = e / W;
  double s, c;
  sincospi(2.0 * sign * (double)((k * x) % W) / W, &s, &c);
  F[e] = make_float2((float)c, (float)s);
}

msp_status fail(msp_status s, const std::string& m) { return set_last_error(s, m); }

bool supported(int W, int S) {
  return (W == 32 || W == 64 || W == 128 || W == 256) && S >= 1 && (long long)S * W <= 65535LL * gemm::TN;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  int* err;
  float2* F;
  float2* tmp;
  size_t bytes;
};

Layout layout(int W, int S, char* base) {
  Layout l{};
  size_t off = 0;
  auto take = [&](size_t b) { char* p = base ? base + off : nullptr; off += align256(b); return p; };
  l.err = (int*)take(sizeof(int));
  l.F = (float2*)take((size_t)W * W * sizeof(float2));
  l.tmp = (float2*)take((size_t)S * W * W * sizeof(float2));
  l.bytes = off;
  return l;
}

std::mutex g_mu;
bool g_attr[64] = {};

}  // namespace
}  // namespace msp

using namespace msp;

extern "C" {

size_t msp_dft2_tc_workspace_bytes(int32_t W, int32_t S) {
  if (!supported(W, S)) return 0;
  return layout(W, S, nullptr).bytes;
}

msp_status msp_dft2_tc(int32_t W, int32_t S, int32_t inverse, const float* in, float* out, void* ws, size_t ws_bytes,
                       void* stream) {
  set_last_error(MSP_OK, "");
  if (!supported(W, S)) return fail(MSP_EUNSUPPORTED, "W must be 32, 64, 128 or 256 and 1 <= S, S W <= 8388480");
  {
    const msp_status u = refuse_untrusted_device();
    if (u != MSP_OK) return u;
  }
  if (!in || !out || ((uintptr_t)in | (uintptr_t)out) % 16) return fail(MSP_EINVAL, "in and out must be non-NULL and 16-byte aligned");
  if (!ws || (uintptr_t)ws % 256) return fail(MSP_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  const Layout l = layout(W, S, (char*)ws);
  if (ws_bytes < l.bytes) return fail(MSP_EINVAL, "workspace too small: " + std::to_string(ws_bytes) + " < " + std::to_string(l.bytes));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return fail(MSP_ECUDA, "no current CUDA device");
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_attr[dev]) {
      e = cudaFuncSetAttribute(cgemm_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm::SMEM_BYTES);
      int k = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, cgemm_kernel<false, true>, gemm::NTHREADS, gemm::SMEM_BYTES);
      if (e != cudaSuccess) return fail(MSP_ECUDA, std::string("contraction set-up: ") + cudaGetErrorString(e));
      if (k * (int)gemm::TMEM_COLS > 512) return fail(MSP_EUNSUPPORTED, "tensor-memory budget exceeded");
      g_attr[dev] = true;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  e = cudaMemsetAsync(l.err, 0, sizeof(int), st);
  if (e != cudaSuccess) return fail(MSP_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  dft_matrix_kernel<<<(W * W + 255) / 256, 256, 0, st>>>(l.F, W, inverse ? 1 : -1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MSP_ECUDA, std::string("dft_matrix_kernel: ") + cudaGetErrorString(e));
  count_launches(1);
  // pass 1: columns j = (s, y) of the images' rows; C[k, (s, y)] = sum_x F[k, x] X[s][y][x],
  // stored transposed per image: tmp[s][k][y].  pass 2 repeats it on tmp, giving out[s][ky][kx].
  const int N = S * W;
  dim3 grid((unsigned)((W + gemm::TM - 1) / gemm::TM), (unsigned)((N + gemm::TN - 1) / gemm::TN), 1u);
  const float2* src[2] = {(const float2*)in, l.tmp};
  float2* dst[2] = {l.tmp, (float2*)out};
  for (int pass = 0; pass < 2; ++pass) {
    msp_status s = profiled_launch(st, [&] {
      cgemm_kernel<false, true><<<grid, gemm::NTHREADS, gemm::SMEM_BYTES, st>>>(W, N, W, W, l.F, (size_t)W, src[pass],
                                                                               (size_t)W, dst[pass], (size_t)W, 0, l.err,
                                                                               tc_wait_limit());
      return cudaGetLastError();
    });
    if (s != MSP_OK) return s;
  }
  return MSP_OK;
}

}  // extern "C"
