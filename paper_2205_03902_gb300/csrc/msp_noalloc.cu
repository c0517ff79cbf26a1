// msp_noalloc.cu -- msp_forward_noalloc: the forward model without a caller
// workspace and without any device allocation.
//
// Some callers cannot call cudaMalloc: a host application that owns all device
// memory through its own pool and forbids any other allocation, or an
// acquisition loop that must not allocate once it runs, because an allocation
// can synchronise the whole device and has no bounded latency.  Such callers
// cannot hand the other entry points a workspace either.  This file gives them
// the fused forward kernel with its scratch (the slice transmissions, the
// propagator factor and an error word) in one file-scope device array of fixed
// size.  The array belongs to this library's device code: it is reserved on a
// device when that code is loaded there (under CUDA's lazy module loading, by the
// first call made on that device) and held until the process exits.
//
// Host code must not pass `g_noalloc_scratch` itself to a kernel: in host code
// that name is a host-side stand-in, not a device address.  Every call looks the
// device address up with cudaGetSymbolAddress, with the calling device current.
// The lookup allocates nothing once the module is loaded; doing it on every call
// (rather than caching an address per device index) keeps the address right after
// a cudaDeviceReset, which reloads the module, and in a caller's own driver-API
// context, where the same device holds a different copy of the array.
#include <cuda_runtime.h>

#include <string>

#include "msp.h"
#include "msp_kernels.cuh"

namespace msp {

cudaError_t launch_position_kernel(int win, int mode, const PosParams& p, int grid, cudaStream_t st);
int position_slots(int win);
__global__ void transmission_kernel(const float* __restrict__ V, float2* __restrict__ T, size_t n, float sigma);
__global__ void propagator_kernel(float2* __restrict__ h1, int W, double dzlam, double dq);

// 16 MiB: a 4 KiB header (error word, propagator factor), then the transmissions.
constexpr size_t kNoallocBytes = size_t(16) << 20;
constexpr size_t kNoallocHeader = 4096;
constexpr size_t kNoallocMaxCells = (kNoallocBytes - kNoallocHeader) / sizeof(float2);   // L * Ny * Nx

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

msp_status set_last_error(msp_status s, const std::string& m);   // shown by msp_last_error_message()
msp_status refuse_untrusted_device();                            // MSP_EDEVICE once a drain wait ran out

static msp_status noalloc_fail(msp_status s, const std::string& m) { return set_last_error(s, m); }

// Device address of the scratch array in the current context, looked up on every call.
static msp_status noalloc_scratch(unsigned char** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr)
    return noalloc_fail(MSP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = (unsigned char*)ptr;
  return MSP_OK;
}

}  // namespace msp

using namespace msp;

extern "C" msp_status msp_forward_noalloc(const msp_geometry* g, const float* probe, const float* V,
                                          const int32_t* pos, float* I_out, int32_t* window_error,
                                          void* stream) {
  msp_status s = msp_validate_geometry(g);   // also clears this thread's error message
  if (s != MSP_OK) return s;
  s = refuse_untrusted_device();
  if (s != MSP_OK) return s;
  if (g->precision != MSP_PRECISION_FP32)
    return noalloc_fail(MSP_EUNSUPPORTED, "msp_forward_noalloc runs the FP32 forward only; use msp_forward");
  if (g->param != MSP_PARAM_POTENTIAL)
    return noalloc_fail(MSP_EUNSUPPORTED, "msp_forward_noalloc takes potentials only; use msp_forward");
  const size_t cells = (size_t)g->n_slices * g->obj_ny * g->obj_nx;
  if (cells > kNoallocMaxCells)
    return noalloc_fail(MSP_EUNSUPPORTED, "L * Ny * Nx = " + std::to_string(cells) + " exceeds the " +
                                              std::to_string(kNoallocMaxCells) +
                                              " cells of the fixed 16 MiB scratch; use msp_forward");
  auto bad = [](const void* p) { return !p || ((uintptr_t)p) % 16 != 0; };
  if (bad(probe) || bad(V)) return noalloc_fail(MSP_EINVAL, "probe and V must be non-NULL and 16-byte aligned");
  if (g->n_pos > 0 && (bad(pos) || bad(I_out)))
    return noalloc_fail(MSP_EINVAL, "pos and I_out must be non-NULL and 16-byte aligned");
  if (window_error && ((uintptr_t)window_error) % 4 != 0)
    return noalloc_fail(MSP_EINVAL, "window_error must be 4-byte aligned");

  unsigned char* base = nullptr;
  s = noalloc_scratch(&base);
  if (s != MSP_OK) return s;
  int* err = window_error ? (int*)window_error : (int*)base;
  float2* h1 = (float2*)(base + 256);
  float2* T = (float2*)(base + kNoallocHeader);
  cudaStream_t st = (cudaStream_t)stream;

  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);   // the only value that must start at zero
  if (e != cudaSuccess) return noalloc_fail(MSP_ECUDA, std::string("set-up: ") + cudaGetErrorString(e));

  const int W = g->win;
  propagator_kernel<<<(W + 255) / 256, 256, 0, st>>>(h1, W, g->dz_A * g->wavelength_A, 1.0 / ((double)W * g->pixel_A));
  const int blocks = (int)((cells + 255) / 256 < (size_t)sms * 16 ? (cells + 255) / 256 : (size_t)sms * 16);
  transmission_kernel<<<blocks, 256, 0, st>>>(V, T, cells, (float)g->sigma);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(MSP_ECUDA, std::string("table kernels: ") + cudaGetErrorString(e));
  if (g->n_pos == 0) return MSP_OK;

  PosParams p{};
  p.probe = (const float2*)probe;
  p.T = T;
  p.h1 = h1;
  p.pos = (const int2*)pos;
  p.I_out = I_out;
  p.err = err;
  p.L = g->n_slices;
  p.Ny = g->obj_ny;
  p.Nx = g->obj_nx;
  p.S = g->n_pos;
  const int cap = position_slots(W);
  e = launch_position_kernel(W, MODE_FORWARD, p, g->n_pos < cap ? g->n_pos : cap, st);
  if (e != cudaSuccess) return noalloc_fail(MSP_ECUDA, std::string("forward kernel: ") + cudaGetErrorString(e));
  return MSP_OK;
}
