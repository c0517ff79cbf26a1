// msp_kernels.cuh -- kernel parameter blocks and launch helpers shared by the
// translation units of libmsp.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace msp {

enum Mode { MODE_FORWARD = 0, MODE_LOSS_GRAD = 1, MODE_LAYER = 2, MODE_PROBE = 3 };

// Everything the fused per-position kernel reads or writes.
struct PosParams {
  const float2* probe;     // [W][W]
  const float2* T;         // [L][Ny][Nx] slice transmissions exp(i sigma V)
  const float2* h1;        // [W] separable propagator factor exp(-i pi dz lambda q_k^2) / W
  const int2* pos;         // [S] window top-left (y, x)
  const float* I_meas;     // [S][W][W]
  float* I_out;            // [S][W][W]                (forward)
  float2* stash;           // [G][Ls][W][W] exit waves kept for the adjoint
  float* wgrad;            // [S][Lg][W][W] per-position window gradients (float2 in transmission mode)
  float* willum;           // [S][W][W] per-position |psi_in,l|^2 (layer step)
  float* dVred;            // [L][Ny][Nx] (loss and gradients) or [Ny][Nx] (layer step), float2 in
                           // transmission mode, zeroed: when set, the kernel adds every window
                           // gradient into it with reductions in L2 instead of writing wgrad (the
                           // order of the additions is not fixed)
  float* illumred;         // [Ny][Nx], zeroed: the layer step's |psi_in,l|^2 likewise, instead of willum
  float2* dprobe_part;     // [G][W][W] per-CTA probe-gradient partial sums
  double* loss_part;       // [S] per-position loss
  const double* zthr2;     // [1] squared far-field amplitude that counts as zero
  int* err;                // error flags
  int L, Ny, Nx, S;
  int layer;               // slice of a layer step
  int want_dprobe;
  int loss_only;           // loss-and-gradient pass with neither gradient wanted: forward and loss only
  int cplx;                // transmission mode: T is the caller's complex slices, gradients complex
  float two_sigma;
};

// Workspace carve-up (all offsets 256-byte aligned).
struct Workspace {
  int* err;
  double* scal;            // [16] scalars: 0 loss, 1 mu, 2 max illum, 3 sum I, 5 zero-rule threshold^2
  double* red;             // [kRedSlots] block partials of FP64 reductions
  float2* h1;              // [W]
  float2* T;
  float2* stash;
  float* wgrad;
  float* willum;
  float2* dprobe_part;
  float2* dprobe_sum;      // [W][W]
  double* loss_part;       // [S]
  float* map0;             // [Ny][Nx] layer gradient map
  float* map1;             // [Ny][Nx] illumination map
  char* precise;           // the precise-forward mode's buffers (NULL in the FP32 mode)
  size_t bytes;
};

// Inputs of the batched modes (FP64 forward, split-BF16 DFT) beyond the fused kernel's parameters.
struct PreciseIn {
  const float* V;        // FP32 potentials (potential mode) or NULL
  const float2* X;       // the caller's complex slices (transmission mode) or NULL
  double sigma;          // interaction constant
  double dzlam, dq;      // dz lambda and the reciprocal pixel 1 / (W pixel) of the propagator
  char* extra;           // the batched modes' workspace segment
  int sms;               // SMs of the device (grid sizes of the element-wise kernels)
  int precision;         // MSP_PRECISION_FP64_FORWARD or MSP_PRECISION_BF16X3_DFT
  int wait_limit;        // poll bound of the tensor-core waits
};

constexpr int kRedSlots = 8192;

// Zero rule of the amplitude-flow gradient (Sec. 3.2: Qz/|Qz| := 0 where Qz = 0),
// resolved at the arithmetic's resolution: a far-field value counts as zero when
// |Psi_k| <= kZeroRuleTau * ||p||_2, the probe norm being the RMS far-field amplitude
// of every pattern of pure-phase slices (Parseval).
constexpr double kZeroRuleTau = 1e-5;

}  // namespace msp
