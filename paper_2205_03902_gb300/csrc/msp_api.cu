// msp_api.cu -- C ABI of libmsp: argument checks, workspace carve-up, and the
// element-wise / reduction kernels around the fused per-position kernel.
//
//   transmission      X_m = exp(i sigma V_m) over the whole object (Sec. 2.1)
//   propagator        separable factor of H / W^2, Eq. (fresnel_element), zero tilt
//   gather            atomic-free overlap-add of per-position window gradients
//                     into object-frame maps, every pixel summing its covering
//                     positions in ascending scan order (the sum over s of
//                     Eq. Opt_Prob_Layerwise)
//   reductions        FP64, fixed order: loss, illumination maximum, pattern sums
//   updates           the gradient steps of Algorithm 1 and of Sec. 3.5
#include <cuda_runtime.h>
#include <type_traits>

#include <algorithm>
#include <atomic>
#include <vector>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>

#include "msp.h"
#include "msp_kernels.cuh"

namespace msp {

cudaError_t launch_position_kernel(int win, int mode, const PosParams& p, int grid, cudaStream_t st);
int position_slots(int win);

// the precise-forward mode (msp_precise.cu)
size_t precise_extra_bytes(int precision, int W, int L, int Ny, int Nx, int S);
cudaError_t run_precise(int mode, const PosParams& p, int W, const PreciseIn& in, cudaStream_t st, long long* launches);

// ---------------------------------------------------------------------------
// element-wise kernels
// ---------------------------------------------------------------------------

__global__ void transmission_kernel(const float* __restrict__ V, float2* __restrict__ T, size_t n, float sigma) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float sn, cs;
    sincosf(sigma * V[i], &sn, &cs);
    T[i] = make_float2(cs, sn);
  }
}

// Separable Fresnel propagator, Eq. (fresnel_element) with zero tilt:
// h(ky, kx) = exp(-i pi dz lambda (qy^2 + qx^2)) / W^2 = h1(ky) h1(kx) with
// h1(k) = exp(-i pi dz lambda q_k^2) / W, evaluated in double precision and rounded
// once to single (the table's rounding is shared by every position, so it is kept at
// half a unit in the last place).
__global__ void propagator_kernel(float2* __restrict__ h1, int W, double dzlam, double dq) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= W) return;
  const double q = (double)(k < W / 2 ? k : k - W) * dq;
  double t = dzlam * q * q;   // phase / pi
  t = t - 2.0 * floor(t * 0.5);
  double sn, cs;
  sincospi(t, &sn, &cs);
  h1[k] = make_float2((float)(cs / W), (float)(-sn / W));
}

// Overlap-add of per-position window arrays into object-frame maps.  One CTA of 256
// threads owns a 32 x 8 object tile (one pixel per thread, one warp per tile row, so a warp
// reads 128 contiguous bytes of a window per position) and a run of slices.  Positions are
// scanned in chunks of 256: the chunk's positions whose window overlaps the tile are
// appended (ballot, order kept) to a shared list of up to kGatherList entries, which serves
// every slice of the run (the covering positions do not depend on the slice).  The CTA then
// adds the listed windows' values in list order, i.e. ascending scan order, LG slices at a
// time, with the loads of the next batch of positions issued before the sums of the current
// one.  Every pixel of every slice therefore sums its covering positions in a fixed order
// (bit-reproducible, no atomics) and no thread spends time on positions that miss its tile.
constexpr int kGatherTX = 32, kGatherTY = 8;   // object tile of one CTA: one warp per tile row
constexpr int kGatherList = 1024;              // listed positions per pass over the list
constexpr int kGatherSlices = 4;               // slices summed together by the loss-and-gradient gather

__device__ __forceinline__ void accum(float& a, float v) { a += v; }
__device__ __forceinline__ void accum(float2& a, float2 v) {
  a.x += v.x;
  a.y += v.y;
}

// CPLX: the gathered channel is complex (float2, transmission mode); ILLUM: a second, real
// channel (the illumination windows of a layer step) is gathered too and its per-tile
// maximum written to `blockmax` (one slice, LG = 1).  The tile (bx, by) of slices l_first ..
// l_first + n_l - 1; gx tiles per row (the block-maximum index is by gx + bx).
template <bool CPLX, bool ILLUM, int LG>
__device__ __forceinline__ void gather_tile(const float* __restrict__ src0, const float* __restrict__ src1,
                                            int nl_src, const int2* __restrict__ pos, int S, int W, int Ny, int Nx,
                                            float* __restrict__ out0, float* __restrict__ out1,
                                            double* __restrict__ blockmax, int bx, int by, int l_first, int n_l,
                                            int gx) {
  static_assert(!ILLUM || LG == 1, "the illumination channel is gathered for one slice");
  using Val = typename std::conditional<CPLX, float2, float>::type;
  constexpr int TX = kGatherTX, TY = kGatherTY;
  constexpr int U = LG == 1 ? 16 : 8;   // positions per batch of loads
  __shared__ int2 spos[kGatherList];
  // per listed position, the element offsets of window pixel (0, 0) of slice l_first moved to
  // the object origin: window value (dy, dx) of object pixel (py, px) sits at base + py W + px
  __shared__ long long sbase0[kGatherList], sbase1[ILLUM ? kGatherList : 1];
  __shared__ int wcount[8];
  __shared__ float wmax[8];
  const int tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;
  const int tx0 = bx * TX, ty0 = by * TY;
  const int px = tx0 + (tid % TX), py = ty0 + (tid / TX);
  const size_t WW = (size_t)W * W;
  const long long pix = (long long)py * W + px;   // this thread's pixel, window-row stride
  const Val zero = Val();
  float acc1 = 0.f;

  // the values of list entries q0 .. q0 + U - 1 at this thread's pixel, slices lg .. lg + LG - 1
  // of the run (zero past the list's end, past the run and where the window misses the pixel)
  auto fetch = [&](int q0, int total, int lg, Val (&v0)[U][LG], float (&v1)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + u;
      const bool live = q < total;   // the list has `total` entries; nothing past it is read
      int2 pq = make_int2(-(1 << 29), -(1 << 29));
      long long o0 = 0, o1 = 0;
      if (live) {
        pq = spos[q];
        o0 = sbase0[q] + pix;
        if (ILLUM) o1 = sbase1[q] + pix;
      }
      const bool in = ((unsigned)(px - pq.y) < (unsigned)W) && ((unsigned)(py - pq.x) < (unsigned)W);
#pragma unroll
      for (int k = 0; k < LG; ++k) {
        const bool ok = in && lg + k < n_l;
        const long long o = o0 + (long long)(lg + k) * (long long)WW;
        if constexpr (CPLX) v0[u][k] = ok ? __ldcs(reinterpret_cast<const float2*>(src0) + o) : zero;
        else v0[u][k] = ok ? __ldcs(src0 + o) : zero;
      }
      v1[u] = (ILLUM && in) ? __ldcs(src1 + o1) : 0.f;
    }
  };
  auto add = [&](Val (&acc)[LG], const Val (&v0)[U][LG], const float (&v1)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int k = 0; k < LG; ++k) accum(acc[k], v0[u][k]);
      if (ILLUM) acc1 += v1[u];
    }
  };
  // sums the list's `total` entries in order, two batches of U in flight
  auto drain = [&](int total, int lg, Val (&acc)[LG]) {
    Val a0[U][LG], b0[U][LG];
    float a1[U], b1[U];
    fetch(0, total, lg, a0, a1);
    for (int q0 = 0; q0 < total; q0 += 2 * U) {
      fetch(q0 + U, total, lg, b0, b1);
      add(acc, a0, a1);
      fetch(q0 + 2 * U, total, lg, a0, a1);
      add(acc, b0, b1);
    }
  };

  for (int lg = 0; lg < n_l; lg += LG) {
    Val acc[LG];
#pragma unroll
    for (int k = 0; k < LG; ++k) acc[k] = zero;
    int listed = 0;   // entries in the list (the same in every thread)
    for (int base = 0; base < S; base += 256) {
      const int n = min(256, S - base);
      int2 ps = make_int2(0, 0);
      bool ov = false;
      if (tid < n) {
        ps = pos[base + tid];
        ov = ps.x < ty0 + TY && ps.x + W > ty0 && ps.y < tx0 + TX && ps.y + W > tx0;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, ov);
      __syncthreads();                      // the previous chunk's counts and the list are no longer read
      if (lane == 0) wcount[w] = __popc(mask);
      __syncthreads();
      int off = 0, total = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        off += (i < w) ? wcount[i] : 0;
        total += wcount[i];
      }
      if (listed + total > kGatherList) {   // full: sum the list so far, then start it again
        drain(listed, lg, acc);
        listed = 0;
        __syncthreads();                    // the list is no longer read
      }
      if (ov) {
        const int q = listed + off + __popc(mask & ((1u << lane) - 1u));
        const long long sq = base + tid, shift = (long long)ps.x * W + ps.y;
        spos[q] = ps;
        sbase0[q] = (sq * nl_src + l_first) * (long long)WW - shift;
        if (ILLUM) sbase1[q] = sq * (long long)WW - shift;
      }
      listed += total;
    }
    __syncthreads();
    drain(listed, lg, acc);
    if (py < Ny && px < Nx) {
#pragma unroll
      for (int k = 0; k < LG; ++k)
        if (lg + k < n_l) {
          const size_t oi = ((size_t)(l_first + lg + k) * Ny + py) * Nx + px;
          if constexpr (CPLX) reinterpret_cast<float2*>(out0)[oi] = acc[k];
          else out0[oi] = acc[k];
        }
    }
  }
  if (ILLUM) {
    float m = 0.f;
    if (py < Ny && px < Nx) {
      out1[(size_t)py * Nx + px] = acc1;
      m = acc1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) wmax[w] = m;
    __syncthreads();
    if (tid == 0) {
      float b = 0.f;
      for (int i = 0; i < 8; ++i) b = fmaxf(b, wmax[i]);
      blockmax[by * gx + bx] = (double)b;
    }
  }
}

template <bool CPLX, bool ILLUM>
__global__ void __launch_bounds__(256) gather_kernel(const float* __restrict__ src0, const float* __restrict__ src1,
                                                     int nl_src, const int2* __restrict__ pos, int S, int W,
                                                     int Ny, int Nx, float* __restrict__ out0,
                                                     float* __restrict__ out1, double* __restrict__ blockmax) {
  gather_tile<CPLX, ILLUM, 1>(src0, src1, nl_src, pos, S, W, Ny, Nx, out0, out1, blockmax, blockIdx.x, blockIdx.y,
                              blockIdx.z, 1, gridDim.x);
}

// Per 32 x 8 object tile, the maximum of `map` (the gather's tiles and block-maximum layout):
// the illumination maximum when the fused kernel summed the illumination map itself.
__global__ void __launch_bounds__(256) tile_max_kernel(const float* __restrict__ map, int Ny, int Nx,
                                                       double* __restrict__ blockmax) {
  __shared__ float wmax[8];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int px = blockIdx.x * kGatherTX + (tid % kGatherTX), py = blockIdx.y * kGatherTY + (tid / kGatherTX);
  float m = (py < Ny && px < Nx) ? map[(size_t)py * Nx + px] : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) wmax[w] = m;
  __syncthreads();
  if (tid == 0) {
    float b = 0.f;
    for (int i = 0; i < 8; ++i) b = fmaxf(b, wmax[i]);
    blockmax[blockIdx.y * gridDim.x + blockIdx.x] = (double)b;
  }
}

// prod_{m > layer} max_pixel |o_m|^2 (FP64; 1 when layer is the last slice): the factor by
// which non-unimodular later slices can enlarge ||Q_l||^2 (transmission-mode step size).
__global__ void __launch_bounds__(1024) later_slices_gain_kernel(const float2* __restrict__ X, int L, size_t plane,
                                                                 int layer, double* __restrict__ out) {
  __shared__ float sh[1024];
  const int tid = threadIdx.x;
  double prod = 1.0;
  for (int m = layer + 1; m < L; ++m) {
    float a = 0.f;
    for (size_t i = tid; i < plane; i += 1024) {
      const float2 v = X[(size_t)m * plane + i];
      a = fmaxf(a, fmaf(v.x, v.x, v.y * v.y));
    }
    sh[tid] = a;
    __syncthreads();
    for (int k = 512; k > 0; k >>= 1) {
      if (tid < k) sh[tid] = fmaxf(sh[tid], sh[tid + k]);
      __syncthreads();
    }
    prod *= (double)sh[0];
    __syncthreads();
  }
  if (tid == 0) out[0] = prod;
}

// Single-block FP64 reduction in a fixed order.  op 0: sum, 1: max.
__global__ void __launch_bounds__(1024) reduce_kernel(const double* __restrict__ in, int n, int op,
                                                      double* __restrict__ out, double* __restrict__ out2) {
  __shared__ double sh[1024];
  const int tid = threadIdx.x;
  double a = 0.0;
  for (int i = tid; i < n; i += 1024) a = (op == 0) ? a + in[i] : fmax(a, in[i]);
  sh[tid] = a;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (tid < s) sh[tid] = (op == 0) ? sh[tid] + sh[tid + s] : fmax(sh[tid], sh[tid + s]);
    __syncthreads();
  }
  if (tid == 0) {
    out[0] = sh[0];
    if (out2) out2[0] = sh[0];
  }
}

// Block partial sums (FP64) of a float array; grid size fixed by the caller.
__global__ void __launch_bounds__(256) sum_blocks_kernel(const float* __restrict__ x, size_t n,
                                                         double* __restrict__ part) {
  __shared__ double sh[256];
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t b0 = blockIdx.x * chunk;
  const size_t b1 = min(n, b0 + chunk);
  double a = 0.0;
  for (size_t i = b0 + threadIdx.x; i < b1; i += 256) a += (double)x[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// dprobe[i] = sum_b part[b][i] (FP64 accumulation, fixed order).  A block of 256 threads owns 32
// consecutive probe values: warp g sums the partials b = g, g + 8, g + 16, ... (lane = value, so
// every load is 256 contiguous bytes), all of them in flight at once, and the eight warp sums
// are added in warp order.  512 blocks for W = 128 keep every SM loading.
constexpr int kDprobeVals = 32;
__device__ __forceinline__ void dprobe_block(const float2* __restrict__ part, int G, int WW, float2* __restrict__ out,
                                             int blk) {
  __shared__ double2 acc_w[8][kDprobeVals];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int i = blk * kDprobeVals + lane;
  double re = 0.0, im = 0.0;
  if (i < WW) {
    // all of a warp's partials (up to 24 at once) in flight, then added in ascending order
    constexpr int kBatch = 24;
    for (int b0 = g; b0 < G; b0 += 8 * kBatch) {
      float2 v[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u)   // past the last partial: a repeat of it, added as zero below
        v[u] = __ldcs(part + (size_t)min(b0 + 8 * u, G - 1) * WW + i);
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const bool live = b0 + 8 * u < G;
        re += live ? (double)v[u].x : 0.0;
        im += live ? (double)v[u].y : 0.0;
      }
    }
  }
  acc_w[g][lane] = make_double2(re, im);
  __syncthreads();
  if (g == 0 && i < WW) {
    double2 t = acc_w[0][lane];
    for (int w = 1; w < 8; ++w) {
      t.x += acc_w[w][lane].x;
      t.y += acc_w[w][lane].y;
    }
    out[i] = make_float2((float)t.x, (float)t.y);
  }
}

__global__ void __launch_bounds__(256) dprobe_reduce_kernel(const float2* __restrict__ part, int G, int WW,
                                                            float2* __restrict__ out) {
  dprobe_block(part, G, WW, out, blockIdx.x);
}

// The loss: the sum of n FP64 values in reduce_kernel's order (1024 strided partial sums, then
// a halving tree), by one block of 256 threads.
__device__ __forceinline__ void loss_block(const double* __restrict__ in, int n, double* __restrict__ out,
                                           double* __restrict__ out2) {
  __shared__ double sh[1024];
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int t = tid + 256 * k;
    double a = 0.0;
    for (int i = t; i < n; i += 1024) a = a + in[i];
    sh[t] = a;
  }
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    for (int t = tid; t < h; t += 256) sh[t] = sh[t] + sh[t + h];
    __syncthreads();
  }
  if (tid == 0) {
    out[0] = sh[0];
    if (out2) out2[0] = sh[0];
  }
}

// What follows the fused kernel in a loss-and-gradient pass, in one launch: blocks [0, n_gather)
// gather dV (one tile and up to kGatherSlices slices each), the next n_dprobe blocks sum the
// probe-gradient partials, and the last block sums the loss.  The three parts are independent
// of one another.
template <bool CPLX>
__global__ void __launch_bounds__(256) loss_grad_finish_kernel(const float* __restrict__ wgrad, const int2* __restrict__ pos,
                                                               int S, int W, int L, int Ny, int Nx, int gx, int gy,
                                                               float* __restrict__ dV, int n_gather,
                                                               const float2* __restrict__ dprobe_part, int G,
                                                               float2* __restrict__ dprobe, int n_dprobe,
                                                               const double* __restrict__ loss_part, int n_loss,
                                                               double* __restrict__ loss, double* __restrict__ loss2) {
  const int b = blockIdx.x;
  if (b < n_gather) {
    // the tile (bx, by) of slices l0 .. l0 + LG - 1 (LG = kGatherSlices, two if complex)
    constexpr int LG = CPLX ? 2 : kGatherSlices;
    const int t = b % (gx * gy), l0 = (b / (gx * gy)) * LG;
    gather_tile<CPLX, false, LG>(wgrad, nullptr, L, pos, S, W, Ny, Nx, dV, nullptr, nullptr, t % gx, t / gx, l0,
                                 min(LG, L - l0), gx);
  } else if (b < n_gather + n_dprobe) {
    dprobe_block(dprobe_part, G, W * W, dprobe, b - n_gather);
  } else {
    loss_block(loss_part, n_loss, loss, loss2);
  }
}

// Step size of a layer step: mu = step, or 1 / (c W^2 max illumination) with c = 2 sigma^2
// (potential mode) or c = prod_{m > l} max |o_m|^2 (scal[6], transmission mode).
// Set-up of every pass in one launch.  Block 0 clears the error word, forms the squared
// zero-rule threshold tau^2 ||p||^2 (fixed-order sums) and the propagator factor
// h1 (as propagator_kernel); every block converts its share of the potentials into
// transmissions exp(i sigma V) (potential mode; n = 0 in transmission mode).
__global__ void __launch_bounds__(1024) prepare_kernel(const float2* __restrict__ probe, int W, double tau2,
                                                       double* __restrict__ zthr2, float2* __restrict__ h1,
                                                       double dzlam, double dq, int* __restrict__ err,
                                                       const float* __restrict__ V, float2* __restrict__ T, size_t n,
                                                       float sigma) {
  if (blockIdx.x == 0) {
    // the squared zero-rule threshold tau^2 sum |p|^2: FP32 partials per thread and warp, the
    // 32 warp sums in FP64 in a fixed order (FP64 throughput is low; a threshold needs no more)
    __shared__ float wsum[32];
    const int tid = threadIdx.x;
    float a = 0.f;
    for (int i = tid; i < W * W; i += 1024) {
      const float2 v = probe[i];
      a = fmaf(v.x, v.x, fmaf(v.y, v.y, a));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((tid & 31) == 0) wsum[tid >> 5] = a;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < 32; ++i) t += (double)wsum[i];
      zthr2[0] = tau2 * t;
      err[0] = 0;
    }
    for (int k = tid; k < W; k += 1024) {
      const double q = (double)(k < W / 2 ? k : k - W) * dq;
      double t = dzlam * q * q;   // phase / pi
      t = t - 2.0 * floor(t * 0.5);
      double sn, cs;
      sincospi(t, &sn, &cs);
      h1[k] = make_float2((float)(cs / W), (float)(-sn / W));
    }
  }
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float sn, cs;
    sincosf(sigma * V[i], &sn, &cs);
    T[i] = make_float2(cs, sn);
  }
}

// End of a layer step's reductions in one launch, each in a fixed order (strided partials per
// thread, a butterfly within each warp, the 32 warp values in order): the illumination
// maximum (scal[2]) from the gather's per-tile maxima, the loss (scal[0], loss_out) from the
// per-position partials, and the step mu (scal[1], mu_out) as layer_mu_kernel forms it.
__global__ void __launch_bounds__(1024) layer_finish_kernel(const double* __restrict__ blockmax, int nblk,
                                                            const double* __restrict__ loss_part, int nloss,
                                                            double step, double c_w2, int cplx, double* scal,
                                                            double* mu_out, double* loss_out) {
  __shared__ double wm[32], ws[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  double m = 0.0, a = 0.0;
  for (int i = tid; i < nblk; i += 1024) m = fmax(m, blockmax[i]);
  for (int i = tid; i < nloss; i += 1024) a += loss_part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    a += __shfl_xor_sync(0xffffffffu, a, o);
  }
  if (lane == 0) {
    wm[w] = m;
    ws[w] = a;
  }
  __syncthreads();
  if (tid == 0) {
    double illum = 0.0, loss = 0.0;
    for (int i = 0; i < 32; ++i) {
      illum = fmax(illum, wm[i]);
      loss += ws[i];
    }
    scal[2] = illum;
    scal[0] = loss;
    if (loss_out) loss_out[0] = loss;
    double mu = step;
    if (!(step > 0.0)) {
      const double mm = illum * (cplx ? scal[6] : 1.0);
      mu = (mm > 0.0) ? 1.0 / (c_w2 * mm) : 0.0;
    }
    scal[1] = mu;
    if (mu_out) mu_out[0] = mu;
  }
}

__global__ void layer_mu_kernel(double* scal, double step, double two_sig2_w2, double* mu_out, int cplx) {
  double mu = step;
  if (!(step > 0.0)) {
    const double m = scal[2] * (cplx ? scal[6] : 1.0);
    mu = (m > 0.0) ? 1.0 / (two_sig2_w2 * m) : 0.0;
  }
  scal[1] = mu;
  if (mu_out) mu_out[0] = mu;
}

__global__ void layer_update_kernel(float* __restrict__ V, const float* __restrict__ dV, size_t n,
                                    const double* __restrict__ scal) {
  const double mu = scal[1];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    V[i] = (float)((double)V[i] - mu * (double)dV[i]);
}

// Probe step p <- p - mu dprobe, optionally rescaled so that W^2 ||p||^2 = mean pattern sum.
__global__ void __launch_bounds__(1024) probe_update_kernel(float2* __restrict__ probe, const float2* __restrict__ d,
                                                            int WW, double mu, int normalize, double target,
                                                            const double* __restrict__ sumI, int S,
                                                            double* __restrict__ mu_out) {
  __shared__ double sh[1024];
  const int tid = threadIdx.x;
  double a = 0.0;
  for (int i = tid; i < WW; i += 1024) {
    const float2 p = probe[i], g = d[i];
    const double re = (double)p.x - mu * (double)g.x;
    const double im = (double)p.y - mu * (double)g.y;
    probe[i] = make_float2((float)re, (float)im);
    a += re * re + im * im;
  }
  if (tid == 0 && mu_out) mu_out[0] = mu;
  if (!normalize) return;
  sh[tid] = a;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (tid < s) sh[tid] += sh[tid + s];
    __syncthreads();
  }
  const double cur = (double)WW * sh[0];
  const double tgt = (S > 0) ? sumI[0] / (double)S : target;
  const double scale = (cur > 0.0 && tgt > 0.0) ? sqrt(tgt / cur) : 1.0;
  for (int i = tid; i < WW; i += 1024) {
    const float2 p = probe[i];
    probe[i] = make_float2((float)(p.x * scale), (float)(p.y * scale));
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static thread_local std::string g_err;

// ---- profiling: launch counter and optional events around the fused kernel ----
static std::atomic<long long> g_launches{0};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<cudaEvent_t> g_ev_pool;   // pairs (start, stop)
static size_t g_ev_used = 0;                 // pairs recorded since the last read
static double g_prof_ms = 0.0;
static long long g_prof_n = 0;

static inline void counted(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Drains recorded event pairs into the running sum (caller holds g_prof_mu).
static cudaError_t prof_drain() {
  for (size_t i = 0; i < g_ev_used; ++i) {
    cudaError_t e = cudaEventSynchronize(g_ev_pool[2 * i + 1]);
    if (e != cudaSuccess) return e;
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, g_ev_pool[2 * i], g_ev_pool[2 * i + 1]);
    if (e != cudaSuccess) return e;
    g_prof_ms += ms;
    ++g_prof_n;
  }
  g_ev_used = 0;
  return cudaSuccess;
}

static msp_status fail(msp_status s, const std::string& m) {
  g_err = m;
  return s;
}

// For entry points defined in other translation units.
msp_status set_last_error(msp_status s, const std::string& m) { return fail(s, m); }
void count_launches(int n) { counted(n); }

// Poll bound of the tensor-core kernels' mbarrier waits (msp_set_wait_limit).
static std::atomic<int> g_wait_limit{1 << 20};
// Overlap-add of msp_loss_grad's window gradients (msp_set_overlap_add).
static std::atomic<int> g_overlap{MSP_OVERLAP_FIXED_ORDER};
int tc_wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

// Devices on which a tensor-core kernel reported that its drain wait ran out (workspace
// flag 3): tensor memory may have been released under running MMAs, so no later result
// from that device is trusted for the rest of the process.
static std::atomic<bool> g_untrusted[64];

static int current_device() {
  int dev = -1;
  return (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) ? dev : -1;
}

// MSP_EDEVICE if the current device has been marked untrusted; every compute entry point
// calls this before it launches anything.
msp_status refuse_untrusted_device() {
  const int dev = current_device();
  if (dev >= 0 && g_untrusted[dev].load())
    return fail(MSP_EDEVICE, "this device reported a tensor-core drain timeout earlier in the process; "
                             "its results are no longer trusted (end the process or reset the device)");
  return MSP_OK;
}

#define MSP_CK(call)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(MSP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct DevInfo {
  bool init = false;
  int sms = 0;
  int slots64 = 1, slots128 = 1, slots256 = 1;   // persistent-grid slots per window size
};
static DevInfo g_dev[64];
static std::mutex g_dev_mu;

static bool device_info(DevInfo* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DevInfo& d = g_dev[dev];
  if (!d.init) {
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    d.slots64 = position_slots(64);
    d.slots128 = position_slots(128);
    d.slots256 = position_slots(256);
    d.init = true;
  }
  *out = d;
  return true;
}

static msp_status check_geometry(const msp_geometry* g) {
  if (!g) return fail(MSP_EINVAL, "geometry is NULL");
  if (g->win != 64 && g->win != 128 && g->win != 256)
    return fail(MSP_EUNSUPPORTED, "window size " + std::to_string(g->win) + " (supported: 64, 128, 256)");
  if (g->param != MSP_PARAM_POTENTIAL && g->param != MSP_PARAM_TRANSMISSION)
    return fail(MSP_EINVAL, "param must be MSP_PARAM_POTENTIAL or MSP_PARAM_TRANSMISSION");
  if (g->n_slices < 1) return fail(MSP_EINVAL, "n_slices < 1");
  if (g->obj_ny < g->win || g->obj_nx < g->win) return fail(MSP_EINVAL, "object smaller than the window");
  if (g->n_pos < 0) return fail(MSP_EINVAL, "n_pos < 0");
  if (!(std::isfinite(g->wavelength_A) && g->wavelength_A > 0)) return fail(MSP_EINVAL, "wavelength must be > 0");
  if (!(std::isfinite(g->pixel_A) && g->pixel_A > 0)) return fail(MSP_EINVAL, "pixel size must be > 0");
  if (!(std::isfinite(g->dz_A) && g->dz_A >= 0)) return fail(MSP_EINVAL, "slice thickness must be >= 0");
  if (!std::isfinite(g->sigma)) return fail(MSP_EINVAL, "sigma must be finite");
  if (g->precision < MSP_PRECISION_FP32 || g->precision > MSP_PRECISION_DF_FORWARD)
    return fail(MSP_EINVAL, "precision must be MSP_PRECISION_FP32, _FP64_FORWARD, _BF16X3_DFT or _DF_FORWARD");
  const double cells = (double)g->n_slices * g->obj_ny * g->obj_nx;
  if (cells > 4.0e9) return fail(MSP_EUNSUPPORTED, "object too large");
  if ((size_t)((g->obj_nx + kGatherTX - 1) / kGatherTX) * ((g->obj_ny + kGatherTY - 1) / kGatherTY) > (size_t)kRedSlots)
    return fail(MSP_EUNSUPPORTED, "object too large for the illumination reduction");
  return MSP_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int grid_cap(const DevInfo& d, int win) {
  return win == 64 ? d.slots64 : (win == 128 ? d.slots128 : d.slots256);
}

// Loss partials per position: one per CTA that holds part of the wave.
static int loss_slots(const msp_geometry* g) {
  return (g->win == 256 && g->precision == MSP_PRECISION_FP32) ? 4 : 1;
}
// The FP64-forward and split-BF16 modes run the batched path (msp_precise.cu).
static bool precise(const msp_geometry* g) { return g->precision != MSP_PRECISION_FP32; }

// Carve the workspace; with base == nullptr only the size is computed.
static Workspace layout(const msp_geometry* g, int gcap, char* base) {
  Workspace w{};
  const size_t W = g->win, WW = W * W, S = (size_t)g->n_pos, L = g->n_slices;
  const size_t plane = (size_t)g->obj_ny * g->obj_nx;
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = base ? base + off : nullptr; off += align256(bytes); return p; };
  w.err = (int*)take(sizeof(int));
  w.scal = (double*)take(16 * sizeof(double));
  w.red = (double*)take(kRedSlots * sizeof(double));
  w.h1 = (float2*)take(W * sizeof(float2));
  w.T = (float2*)take(L * plane * sizeof(float2));
  w.stash = (float2*)take((size_t)gcap * L * WW * sizeof(float2));
  // window gradients (float2 in transmission mode), then the illumination windows of a layer step
  const size_t cw = g->param == MSP_PARAM_TRANSMISSION ? 2 : 1;
  w.wgrad = (float*)take(S * std::max(L * cw, cw + 1) * WW * sizeof(float));
  w.willum = base ? w.wgrad + cw * S * WW : nullptr;
  w.dprobe_part = (float2*)take((size_t)gcap * WW * sizeof(float2));
  w.dprobe_sum = (float2*)take(WW * sizeof(float2));
  w.loss_part = (double*)take((S > 0 ? S : 1) * loss_slots(g) * sizeof(double));
  w.map0 = (float*)take(2 * plane * sizeof(float));   // complex in transmission mode
  w.map1 = (float*)take(plane * sizeof(float));
  w.precise = precise(g) ? (char*)take(precise_extra_bytes(g->precision, (int)W, (int)L, g->obj_ny, g->obj_nx, (int)S))
                         : nullptr;
  w.bytes = off;
  return w;
}

static bool misaligned(const void* p, size_t a) { return ((uintptr_t)p) % a != 0; }

struct Call {
  DevInfo dev;
  Workspace ws;
  int gcap = 0;
  int grid = 0;
  int parts = 0;               // per-CTA probe-gradient partials the fused pass leaves
  const float* V = nullptr;    // the caller's slices (potentials, or complex in transmission mode)
  cudaStream_t st = nullptr;
};

static msp_status begin(const msp_geometry* g, void* ws, size_t ws_bytes, void* stream, Call* c) {
  msp_status s = check_geometry(g);
  if (s != MSP_OK) return s;
  s = refuse_untrusted_device();
  if (s != MSP_OK) return s;
  if (!device_info(&c->dev)) return fail(MSP_ECUDA, "no current CUDA device");
  c->gcap = grid_cap(c->dev, g->win);
  const size_t need = layout(g, c->gcap, nullptr).bytes;
  if (!ws) return fail(MSP_EINVAL, "workspace is NULL");
  if (misaligned(ws, 256)) return fail(MSP_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < need)
    return fail(MSP_EINVAL, "workspace too small: " + std::to_string(ws_bytes) + " < " + std::to_string(need));
  c->ws = layout(g, c->gcap, (char*)ws);
  c->grid = g->n_pos < c->gcap ? g->n_pos : c->gcap;
  c->parts = precise(g) ? 1 : c->grid;
  c->st = (cudaStream_t)stream;
  return MSP_OK;
}

static msp_status need_ptr(const void* p, const char* name) {
  if (!p) return fail(MSP_EINVAL, std::string(name) + " is NULL");
  if (misaligned(p, 16)) return fail(MSP_EINVAL, std::string(name) + " must be 16-byte aligned");
  return MSP_OK;
}

#define MSP_TRY(expr)            \
  do {                           \
    msp_status s_ = (expr);      \
    if (s_ != MSP_OK) return s_; \
  } while (0)

static msp_status prepare(const msp_geometry* g, const float* probe, const float* V, Call& c) {
  const int W = g->win;
  const bool pot = g->param != MSP_PARAM_TRANSMISSION;   // transmission mode uses the caller's slices as given
  const size_t n = pot ? (size_t)g->n_slices * g->obj_ny * g->obj_nx : 0;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((n + 1023) / 1024, (size_t)c.dev.sms * 4));
  prepare_kernel<<<blocks, 1024, 0, c.st>>>((const float2*)probe, W, kZeroRuleTau * kZeroRuleTau, c.ws.scal + 5,
                                            c.ws.h1, g->dz_A * g->wavelength_A, 1.0 / ((double)W * g->pixel_A),
                                            c.ws.err, V, c.ws.T, n, (float)g->sigma);
  MSP_CK(cudaGetLastError());
  counted();
  return MSP_OK;
}

static PosParams base_params(const msp_geometry* g, const float* probe, const float* V, const int32_t* pos,
                             Call& c) {
  c.V = V;
  PosParams p{};
  p.probe = (const float2*)probe;
  p.cplx = g->param == MSP_PARAM_TRANSMISSION;
  p.T = p.cplx ? (const float2*)V : c.ws.T;   // transmission mode: the caller's complex slices
  p.h1 = c.ws.h1;
  p.pos = (const int2*)pos;
  p.stash = c.ws.stash;
  p.wgrad = c.ws.wgrad;
  p.willum = c.ws.willum;
  p.dprobe_part = c.ws.dprobe_part;
  p.loss_part = c.ws.loss_part;
  p.err = c.ws.err;
  p.zthr2 = c.ws.scal + 5;
  p.L = g->n_slices;
  p.Ny = g->obj_ny;
  p.Nx = g->obj_nx;
  p.S = g->n_pos;
  p.two_sigma = (float)(2.0 * g->sigma);
  return p;
}

// Launches one kernel through `launch`; while profiling is on, brackets it with an event
// pair on `st` (the dominant kernel of each call: the fused per-position kernel here, the
// dense contraction of the sparse-decomposition matrix step).
msp_status profiled_launch(cudaStream_t st, const std::function<cudaError_t()>& launch) {
  std::unique_lock<std::mutex> lk(g_prof_mu);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (g_prof_on) {
    if (g_ev_used * 2 + 2 > g_ev_pool.size()) {
      if (g_ev_pool.size() >= 8192) {
        MSP_CK(prof_drain());
      } else {
        for (int k = 0; k < 2; ++k) {
          cudaEvent_t ev;
          MSP_CK(cudaEventCreate(&ev));
          g_ev_pool.push_back(ev);
        }
      }
    }
    e0 = g_ev_pool[2 * g_ev_used];
    e1 = g_ev_pool[2 * g_ev_used + 1];
    MSP_CK(cudaEventRecord(e0, st));
  }
  MSP_CK(launch());
  counted();
  if (g_prof_on) {
    MSP_CK(cudaEventRecord(e1, st));
    ++g_ev_used;
  }
  return MSP_OK;
}

static msp_status run_position(const msp_geometry* g, int mode, const PosParams& p, Call& c) {
  if (g->n_pos == 0) return MSP_OK;
  if (precise(g)) {
    PreciseIn in{};
    in.V = p.cplx ? nullptr : c.V;
    in.X = p.cplx ? (const float2*)c.V : nullptr;
    in.sigma = g->sigma;
    in.dzlam = g->dz_A * g->wavelength_A;
    in.dq = 1.0 / ((double)g->win * g->pixel_A);
    in.extra = c.ws.precise;
    in.sms = c.dev.sms;
    in.precision = g->precision;
    in.wait_limit = tc_wait_limit();
    long long n = 0;
    const msp_status s = profiled_launch(c.st, [&] { return run_precise(mode, p, g->win, in, c.st, &n); });
    if (n > 1) counted((int)(n - 1));   // profiled_launch counted one
    return s;
  }
  return profiled_launch(c.st, [&] { return launch_position_kernel(g->win, mode, p, c.grid, c.st); });
}

static msp_status reduce_loss(const msp_geometry* g, Call& c, double* extra) {
  if (g->n_pos == 0) {
    MSP_CK(cudaMemsetAsync(c.ws.scal, 0, sizeof(double), c.st));
    if (extra) MSP_CK(cudaMemsetAsync(extra, 0, sizeof(double), c.st));
    return MSP_OK;
  }
  reduce_kernel<<<1, 1024, 0, c.st>>>(c.ws.loss_part, g->n_pos * loss_slots(g), 0, c.ws.scal, extra);
  MSP_CK(cudaGetLastError());
  counted();
  return MSP_OK;
}

}  // namespace msp

using namespace msp;

extern "C" {

msp_status msp_validate_geometry(const msp_geometry* g) {
  g_err.clear();
  return check_geometry(g);
}

size_t msp_workspace_bytes(const msp_geometry* g) {
  if (check_geometry(g) != MSP_OK) return 0;
  DevInfo d;
  if (!device_info(&d)) return 0;
  return layout(g, grid_cap(d, g->win), nullptr).bytes;
}

msp_status msp_forward(const msp_geometry* g, const float* probe, const float* V, const int32_t* pos, float* I_out,
                       void* ws, size_t ws_bytes, void* stream) {
  g_err.clear();
  Call c;
  MSP_TRY(begin(g, ws, ws_bytes, stream, &c));
  MSP_TRY(need_ptr(probe, "probe"));
  MSP_TRY(need_ptr(V, "V"));
  if (g->n_pos > 0) {
    MSP_TRY(need_ptr(pos, "pos"));
    MSP_TRY(need_ptr(I_out, "I_out"));
  }
  MSP_TRY(prepare(g, probe, V, c));
  PosParams p = base_params(g, probe, V, pos, c);
  p.I_out = I_out;
  return run_position(g, MODE_FORWARD, p, c);
}

msp_status msp_loss_grad(const msp_geometry* g, const float* probe, const float* V, const int32_t* pos,
                         const float* I_meas, double* loss, float* dV, float* dprobe, void* ws, size_t ws_bytes,
                         void* stream) {
  g_err.clear();
  Call c;
  MSP_TRY(begin(g, ws, ws_bytes, stream, &c));
  MSP_TRY(need_ptr(probe, "probe"));
  MSP_TRY(need_ptr(V, "V"));
  if (g->n_pos > 0) {
    MSP_TRY(need_ptr(pos, "pos"));
    MSP_TRY(need_ptr(I_meas, "I_meas"));
  }
  if (loss && misaligned(loss, 8)) return fail(MSP_EINVAL, "loss must be 8-byte aligned");
  if (dV) MSP_TRY(need_ptr(dV, "dV"));
  if (dprobe) MSP_TRY(need_ptr(dprobe, "dprobe"));
  MSP_TRY(prepare(g, probe, V, c));
  const int W = g->win;
  const size_t WW = (size_t)W * W;
  const size_t plane = (size_t)g->obj_ny * g->obj_nx;
  PosParams p = base_params(g, probe, V, pos, c);
  p.I_meas = I_meas;
  p.want_dprobe = dprobe != nullptr;
  p.loss_only = !dV && !dprobe;   // the adjoint is skipped
  const size_t dV_bytes = (size_t)g->n_slices * plane * sizeof(float) * (p.cplx ? 2 : 1);
  if (g->n_pos == 0) {
    if (dV) MSP_CK(cudaMemsetAsync(dV, 0, dV_bytes, c.st));
    if (dprobe) MSP_CK(cudaMemsetAsync(dprobe, 0, WW * sizeof(float2), c.st));
    return reduce_loss(g, c, loss);
  }
  // in the FP32 mode the fused kernels can add the window gradients into dV themselves
  const bool l2_reduce = dV && !precise(g) && g_overlap.load(std::memory_order_relaxed) == MSP_OVERLAP_L2_REDUCE;
  if (l2_reduce) {
    if (misaligned(dV, p.cplx ? 8 : 4)) return fail(MSP_EINVAL, "dV must be aligned to its element");
    MSP_CK(cudaMemsetAsync(dV, 0, dV_bytes, c.st));
    p.dVred = dV;
  }
  MSP_TRY(run_position(g, MODE_LOSS_GRAD, p, c));
  // the gather of dV, the probe-gradient sum and the loss sum, in one launch
  const int gx = (g->obj_nx + kGatherTX - 1) / kGatherTX, gy = (g->obj_ny + kGatherTY - 1) / kGatherTY;
  const int lg = p.cplx ? 2 : kGatherSlices;   // slices per gather block
  const int n_gather = (dV && !l2_reduce) ? gx * gy * ((g->n_slices + lg - 1) / lg) : 0;
  const int n_dprobe = dprobe ? (int)((WW + kDprobeVals - 1) / kDprobeVals) : 0;
  const int nblk = n_gather + n_dprobe + 1;
  if (p.cplx)
    loss_grad_finish_kernel<true><<<nblk, 256, 0, c.st>>>(
        c.ws.wgrad, (const int2*)pos, g->n_pos, W, g->n_slices, g->obj_ny, g->obj_nx, gx, gy, dV, n_gather,
        c.ws.dprobe_part, c.parts, (float2*)dprobe, n_dprobe, c.ws.loss_part, g->n_pos * loss_slots(g), c.ws.scal,
        loss);
  else
    loss_grad_finish_kernel<false><<<nblk, 256, 0, c.st>>>(
        c.ws.wgrad, (const int2*)pos, g->n_pos, W, g->n_slices, g->obj_ny, g->obj_nx, gx, gy, dV, n_gather,
        c.ws.dprobe_part, c.parts, (float2*)dprobe, n_dprobe, c.ws.loss_part, g->n_pos * loss_slots(g), c.ws.scal,
        loss);
  MSP_CK(cudaGetLastError());
  counted();
  return MSP_OK;
}

msp_status msp_layer_step(const msp_geometry* g, const float* probe, float* V, const int32_t* pos,
                          const float* I_meas, int32_t layer, double step, double* loss_before, double* mu_out,
                          void* ws, size_t ws_bytes, void* stream) {
  g_err.clear();
  Call c;
  MSP_TRY(begin(g, ws, ws_bytes, stream, &c));
  MSP_TRY(need_ptr(probe, "probe"));
  MSP_TRY(need_ptr(V, "V"));
  if (layer < 0 || layer >= g->n_slices) return fail(MSP_EINVAL, "layer out of range");
  if (!std::isfinite(step)) return fail(MSP_EINVAL, "step must be finite");
  if (g->n_pos > 0) {
    MSP_TRY(need_ptr(pos, "pos"));
    MSP_TRY(need_ptr(I_meas, "I_meas"));
  }
  if (loss_before && misaligned(loss_before, 8)) return fail(MSP_EINVAL, "loss_before must be 8-byte aligned");
  if (mu_out && misaligned(mu_out, 8)) return fail(MSP_EINVAL, "mu_out must be 8-byte aligned");
  MSP_TRY(prepare(g, probe, V, c));
  const int W = g->win;
  const size_t plane = (size_t)g->obj_ny * g->obj_nx;
  if (g->n_pos == 0) {
    MSP_CK(cudaMemsetAsync(c.ws.scal, 0, 16 * sizeof(double), c.st));
    layer_mu_kernel<<<1, 1, 0, c.st>>>(c.ws.scal, step, 0.0, mu_out, 0);
    MSP_CK(cudaGetLastError());
  counted();
    return reduce_loss(g, c, loss_before);
  }
  PosParams p = base_params(g, probe, V, pos, c);
  p.I_meas = I_meas;
  p.layer = layer;
  dim3 grid((g->obj_nx + kGatherTX - 1) / kGatherTX, (g->obj_ny + kGatherTY - 1) / kGatherTY, 1);
  const int nblk = (int)(grid.x * grid.y);
  if (nblk > kRedSlots) return fail(MSP_EUNSUPPORTED, "object too large for the illumination reduction");
  // in the FP32 mode the fused kernels can add the gradient and illumination windows into the maps
  const bool l2_reduce = !precise(g) && g_overlap.load(std::memory_order_relaxed) == MSP_OVERLAP_L2_REDUCE;
  if (l2_reduce) {
    MSP_CK(cudaMemsetAsync(c.ws.map0, 0, plane * sizeof(float) * (p.cplx ? 2 : 1), c.st));
    MSP_CK(cudaMemsetAsync(c.ws.map1, 0, plane * sizeof(float), c.st));
    p.dVred = c.ws.map0;
    p.illumred = c.ws.map1;
  }
  MSP_TRY(run_position(g, MODE_LAYER, p, c));
  if (l2_reduce)
    tile_max_kernel<<<grid, 256, 0, c.st>>>(c.ws.map1, g->obj_ny, g->obj_nx, c.ws.red);
  else if (p.cplx)
    gather_kernel<true, true><<<grid, 256, 0, c.st>>>(c.ws.wgrad, c.ws.willum, 1, (const int2*)pos, g->n_pos, W,
                                                      g->obj_ny, g->obj_nx, c.ws.map0, c.ws.map1, c.ws.red);
  else
    gather_kernel<false, true><<<grid, 256, 0, c.st>>>(c.ws.wgrad, c.ws.willum, 1, (const int2*)pos, g->n_pos, W,
                                                       g->obj_ny, g->obj_nx, c.ws.map0, c.ws.map1, c.ws.red);
  MSP_CK(cudaGetLastError());
  counted();
  if (p.cplx) {
    later_slices_gain_kernel<<<1, 1024, 0, c.st>>>((const float2*)V, g->n_slices, plane, layer, c.ws.scal + 6);
    MSP_CK(cudaGetLastError());
    counted();
  }
  // potential mode: mu = 1 / (2 sigma^2 W^2 max illum); transmission: 1 / (W^2 max illum prod max|o_m|^2)
  const double c_w2 = (p.cplx ? 1.0 : 2.0 * g->sigma * g->sigma) * (double)W * (double)W;
  layer_finish_kernel<<<1, 1024, 0, c.st>>>(c.ws.red, nblk, c.ws.loss_part, g->n_pos * loss_slots(g), step, c_w2,
                                            p.cplx, c.ws.scal, mu_out, loss_before);
  MSP_CK(cudaGetLastError());
  counted();
  // V_l (or the complex o_l, as interleaved floats) -= mu * gradient map
  const size_t nupd = plane * (p.cplx ? 2 : 1);
  const int blocks = (int)std::min<size_t>((nupd + 255) / 256, (size_t)c.dev.sms * 8);
  layer_update_kernel<<<blocks, 256, 0, c.st>>>(V + (size_t)layer * nupd, c.ws.map0, nupd, c.ws.scal);
  MSP_CK(cudaGetLastError());
  counted();
  return MSP_OK;
}

msp_status msp_probe_step(const msp_geometry* g, float* probe, const float* V, const int32_t* pos,
                          const float* I_meas, double step, int32_t normalize, double* loss_before, double* mu_out,
                          void* ws, size_t ws_bytes, void* stream) {
  g_err.clear();
  Call c;
  MSP_TRY(begin(g, ws, ws_bytes, stream, &c));
  MSP_TRY(need_ptr(probe, "probe"));
  MSP_TRY(need_ptr(V, "V"));
  if (!std::isfinite(step)) return fail(MSP_EINVAL, "step must be finite");
  if (g->n_pos > 0) {
    MSP_TRY(need_ptr(pos, "pos"));
    MSP_TRY(need_ptr(I_meas, "I_meas"));
  }
  if (loss_before && misaligned(loss_before, 8)) return fail(MSP_EINVAL, "loss_before must be 8-byte aligned");
  if (mu_out && misaligned(mu_out, 8)) return fail(MSP_EINVAL, "mu_out must be 8-byte aligned");
  MSP_TRY(prepare(g, probe, V, c));
  const int W = g->win;
  const size_t WW = (size_t)W * W;
  const int S = g->n_pos;
  const double mu = (step > 0.0) ? step : (S > 0 ? 1.0 / ((double)S * (double)WW) : 0.0);
  if (S == 0) {
    MSP_CK(cudaMemsetAsync(c.ws.dprobe_sum, 0, WW * sizeof(float2), c.st));
  } else {
    PosParams p = base_params(g, probe, V, pos, c);
    p.I_meas = I_meas;
    p.want_dprobe = 1;
    MSP_TRY(run_position(g, MODE_PROBE, p, c));
    dprobe_reduce_kernel<<<(int)((WW + kDprobeVals - 1) / kDprobeVals), 256, 0, c.st>>>(c.ws.dprobe_part, c.parts, (int)WW,
                                                                   c.ws.dprobe_sum);
    MSP_CK(cudaGetLastError());
  counted();
  }
  MSP_TRY(reduce_loss(g, c, loss_before));
  if (normalize && S > 0) {
    const int nb = 1024;
    sum_blocks_kernel<<<nb, 256, 0, c.st>>>(I_meas, (size_t)S * WW, c.ws.red);
    MSP_CK(cudaGetLastError());
  counted();
    reduce_kernel<<<1, 1024, 0, c.st>>>(c.ws.red, nb, 0, c.ws.scal + 3, nullptr);
    MSP_CK(cudaGetLastError());
  counted();
  }
  probe_update_kernel<<<1, 1024, 0, c.st>>>((float2*)probe, c.ws.dprobe_sum, (int)WW, mu,
                                            (normalize && S > 0) ? 1 : 0, 0.0, c.ws.scal + 3, S, mu_out);
  MSP_CK(cudaGetLastError());
  counted();
  return MSP_OK;
}

static msp_status check_plan(const msp_geometry* g, const msp_plan* plan) {
  MSP_TRY(check_geometry(g));
  if (!plan) return fail(MSP_EINVAL, "plan is NULL");
  if (plan->sweeps < 0 || plan->steps_per_layer < 0 || plan->probe_steps < 0)
    return fail(MSP_EINVAL, "sweeps, steps_per_layer and probe_steps must be >= 0");
  if (!std::isfinite(plan->layer_step) || !std::isfinite(plan->probe_step))
    return fail(MSP_EINVAL, "step sizes must be finite");
  const double steps = (double)plan->sweeps * ((double)g->n_slices * plan->steps_per_layer + plan->probe_steps);
  if (steps > 1.0e9) return fail(MSP_EINVAL, "plan has more than 1e9 steps");
  return MSP_OK;
}

size_t msp_reconstruct_history_length(const msp_geometry* g, const msp_plan* plan) {
  if (check_plan(g, plan) != MSP_OK) return 0;
  return (size_t)plan->sweeps * ((size_t)g->n_slices * plan->steps_per_layer + plan->probe_steps) + 1;
}

msp_status msp_reconstruct(const msp_geometry* g, const msp_plan* plan, float* probe, float* V, const int32_t* pos,
                           const float* I_meas, double* loss_history, void* ws, size_t ws_bytes, void* stream) {
  g_err.clear();
  MSP_TRY(check_plan(g, plan));
  if (loss_history && misaligned(loss_history, 8)) return fail(MSP_EINVAL, "loss_history must be 8-byte aligned");
  {
    // every argument the steps take is checked once here, before the first launch
    Call c;
    MSP_TRY(begin(g, ws, ws_bytes, stream, &c));
    MSP_TRY(need_ptr(probe, "probe"));
    MSP_TRY(need_ptr(V, "V"));
    if (g->n_pos > 0) {
      MSP_TRY(need_ptr(pos, "pos"));
      MSP_TRY(need_ptr(I_meas, "I_meas"));
    }
  }
  size_t k = 0;
  auto slot = [&]() { return loss_history ? loss_history + k++ : nullptr; };
  for (int t = 0; t < plan->sweeps; ++t) {
    for (int l = 0; l < g->n_slices; ++l)
      for (int i = 0; i < plan->steps_per_layer; ++i)
        MSP_TRY(msp_layer_step(g, probe, V, pos, I_meas, l, plan->layer_step, slot(), nullptr, ws, ws_bytes, stream));
    for (int i = 0; i < plan->probe_steps; ++i)
      MSP_TRY(msp_probe_step(g, (float*)probe, V, pos, I_meas, plan->probe_step, plan->normalize_probe, slot(),
                             nullptr, ws, ws_bytes, stream));
  }
  if (loss_history) MSP_TRY(msp_loss_grad(g, probe, V, pos, I_meas, slot(), nullptr, nullptr, ws, ws_bytes, stream));
  return MSP_OK;
}

msp_status msp_set_wait_limit(int32_t polls) {
  g_err.clear();
  g_wait_limit.store(polls >= 1 ? polls : polls == 0 ? (1 << 20) : 0, std::memory_order_relaxed);
  return MSP_OK;
}

msp_status msp_set_overlap_add(int32_t mode) {
  g_err.clear();
  if (mode != MSP_OVERLAP_FIXED_ORDER && mode != MSP_OVERLAP_L2_REDUCE)
    return fail(MSP_EINVAL, "overlap-add mode must be MSP_OVERLAP_FIXED_ORDER or MSP_OVERLAP_L2_REDUCE");
  g_overlap.store(mode, std::memory_order_relaxed);
  return MSP_OK;
}

msp_status msp_profile_enable(int32_t on) {
  g_err.clear();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return MSP_OK;
}

msp_status msp_profile_read(double* fused_ms, int64_t* fused_launches, int64_t* all_launches, int32_t reset) {
  g_err.clear();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  MSP_CK(prof_drain());
  if (fused_ms) *fused_ms = g_prof_ms;
  if (fused_launches) *fused_launches = g_prof_n;
  if (all_launches) *all_launches = g_launches.load();
  if (reset) {
    g_prof_ms = 0.0;
    g_prof_n = 0;
    g_launches.store(0);
  }
  return MSP_OK;
}

msp_status msp_check_workspace(void* ws, void* stream) {
  g_err.clear();
  if (!ws) return fail(MSP_EINVAL, "workspace is NULL");
  MSP_CK(cudaStreamSynchronize((cudaStream_t)stream));
  int flag = 0;
  MSP_CK(cudaMemcpy(&flag, ws, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    MSP_CK(cudaMemset(ws, 0, sizeof(int)));
    if (flag == 3) {
      const int dev = current_device();
      if (dev >= 0) g_untrusted[dev].store(true);
      return fail(MSP_EDEVICE, "a tensor-core wait timed out and the kernel could not confirm that its own MMAs "
                               "had finished before it released tensor memory; the device is no longer trusted");
    }
    if (flag == 2) return fail(MSP_ETIMEOUT, "a wait for the tensor core timed out; the call's results are not valid");
    return fail(MSP_EINVAL, "a scan window lies outside the object (position skipped)");
  }
  return refuse_untrusted_device();
}

const char* msp_status_string(msp_status s) {
  switch (s) {
    case MSP_OK: return "MSP_OK";
    case MSP_EINVAL: return "MSP_EINVAL";
    case MSP_ENOMEM: return "MSP_ENOMEM";
    case MSP_ECUDA: return "MSP_ECUDA";
    case MSP_EUNSUPPORTED: return "MSP_EUNSUPPORTED";
    case MSP_ETIMEOUT: return "MSP_ETIMEOUT";
    case MSP_EDEVICE: return "MSP_EDEVICE";
  }
  return "MSP_UNKNOWN";
}

const char* msp_last_error_message(void) { return g_err.c_str(); }

}  // extern "C"
