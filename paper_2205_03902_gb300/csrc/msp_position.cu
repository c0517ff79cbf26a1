// msp_position.cu -- the fused per-position multislice forward / adjoint kernel.
//
// One CTA owns one scan position at a time (persistent grid, positions
// s = blockIdx.x, blockIdx.x + gridDim.x, ...).  The W x W complex wave stays
// in shared memory for the whole position: every slice's transmit (Sec. 2.1,
// E_m = V_z(E_{m-1}) o X_m), Fresnel propagation F^-1(H o F .) and the far-field
// transform F(E_M) run on it in place, then the amplitude-flow residual
// (Sec. 3.2) and the adjoint recursion chi_{m-1} = G^H (conj(X_m) o chi_m)
// (Sec. 3.3, the prefix / suffix products R_l and S_l applied matrix-free).
//
// Each eight-thread line group owns a small padded exchange buffer next to the
// wave, so the in-line exchange never touches the wave itself.
//
// A propagation is  rows F -> [columns F, x H, columns F^-1] -> rows F^-1: the
// column transforms and the propagator run back to back in registers, and the
// inverse row transform of one slice, the transmit of the next slice and its
// forward row transform also run back to back in registers.  Each phase is one
// read and one write of the wave in shared memory plus the in-line exchange.
//
// The propagator is separable, h(ky, kx) = h1(ky) h1(kx) with
// h1(k) = exp(-i pi dz lambda q_k^2) / W (the 1/W^2 of F^-1 folded in), so it is
// a W-entry shared table.  Global operands of a phase (transmission window,
// measured intensities, stashed exit waves) are loaded before the line transform
// that precedes their use, so their latency hides behind the arithmetic.
//
// The only per-slice global traffic is the transmission window (read), the exit
// wave of each slice (written to this CTA's stash slot on the way forward, read
// back on the way down; the slots are reused position after position so they
// stay L2-resident) and the per-position window gradient.  The data each position
// touches once (measured pattern, window gradients, illumination) is loaded and
// stored with the evict-first (streaming) cache hint, so that it does not push the
// stash slots out of L2.
#include "msp_fft.cuh"
#include "msp_kernels.cuh"
#include "msp_tc.cuh"

// Twiddles of the line transforms from shared memory (0) or registers (1).
#ifndef MSP_TWIDDLE_REGISTERS
#define MSP_TWIDDLE_REGISTERS 1
#endif
// In-line exchange with row-major (0) or transposed (1) step-A results.
#ifndef MSP_TRANSPOSED_EXCHANGE
#define MSP_TRANSPOSED_EXCHANGE 1
#endif

namespace msp {

// Exit-wave stash in tensor memory (W = 128, one CTA per SM).  The fused kernel issues no MMAs,
// so the SM's 256 KB of tensor memory is free: each thread keeps the values it stashes for two
// slices in its own TMEM lane (warp w: lanes 32 (w % 4) .., columns 128 (w / 4) .. + 127; a
// slice takes 2 row iterations x 16 complex values = 64 columns).  Those slices neither pass
// through the L1 data pipe nor compete for L2 with the streaming window gradients; the others
// use the CTA's global stash slot.  Loss and gradients: the last two slices (the first ones
// the adjoint reads back); layer step: the one stashed slice.
#ifndef MSP_TMEM_STASH
#define MSP_TMEM_STASH 1
#endif
struct TmemStash {
  uint32_t base;   // this thread's lane and its warp's first column
  // 16 complex values of row iteration `it` of stash slot `slot` (0 or 1)
  __device__ __forceinline__ uint32_t addr(int slot, int it) const { return base + (uint32_t)(64 * slot + 32 * it); }
  __device__ __forceinline__ void store(int slot, int it, const float2 (&v)[16]) const {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(addr(slot, it)),
        "f"(v[0].x), "f"(v[0].y), "f"(v[1].x), "f"(v[1].y), "f"(v[2].x), "f"(v[2].y), "f"(v[3].x), "f"(v[3].y),
        "f"(v[4].x), "f"(v[4].y), "f"(v[5].x), "f"(v[5].y), "f"(v[6].x), "f"(v[6].y), "f"(v[7].x), "f"(v[7].y),
        "f"(v[8].x), "f"(v[8].y), "f"(v[9].x), "f"(v[9].y), "f"(v[10].x), "f"(v[10].y), "f"(v[11].x), "f"(v[11].y),
        "f"(v[12].x), "f"(v[12].y), "f"(v[13].x), "f"(v[13].y), "f"(v[14].x), "f"(v[14].y), "f"(v[15].x),
        "f"(v[15].y)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  __device__ __forceinline__ void load(int slot, int it, float2 (&v)[16]) const {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y), "=f"(v[2].x), "=f"(v[2].y), "=f"(v[3].x),
          "=f"(v[3].y), "=f"(v[4].x), "=f"(v[4].y), "=f"(v[5].x), "=f"(v[5].y), "=f"(v[6].x), "=f"(v[6].y),
          "=f"(v[7].x), "=f"(v[7].y), "=f"(v[8].x), "=f"(v[8].y), "=f"(v[9].x), "=f"(v[9].y), "=f"(v[10].x),
          "=f"(v[10].y), "=f"(v[11].x), "=f"(v[11].y), "=f"(v[12].x), "=f"(v[12].y), "=f"(v[13].x), "=f"(v[13].y),
          "=f"(v[14].x), "=f"(v[14].y), "=f"(v[15].x), "=f"(v[15].y)
        : "r"(addr(slot, it))
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  }
};

#if MSP_TRANSPOSED_EXCHANGE
#define LINE_FFT line_fft_t
#else
#define LINE_FFT line_fft
#endif

template <int W>
struct Geo {
  static constexpr int NT = 4 * W;        // threads per CTA
  static constexpr int N1 = W / 8;        // values per thread per line
  static constexpr int GROUPS = NT / 8;   // eight-thread line groups
  static constexpr int LPG = W / GROUPS;  // lines per group per pass
};

// Shared-memory offset of element j + 8m of wave row r: (j + 8m) ^ swz(r) flips bits 0-2
// by swz(r) & 7 and bit 3 by swz(r) & 8, i.e. adds +-8 for even / odd m.
template <int W>
struct RowIdx {
  int be, bo;
  __device__ __forceinline__ RowIdx(int r, int j) {
    const int sw = swz(r);
    const int base = r * W + (j ^ (sw & 7));
    be = base + (sw & 8);
    bo = base - (sw & 8);
  }
  __device__ __forceinline__ int operator()(int m) const { return ((m & 1) ? bo : be) + 8 * m; }
};
// Element j + 8m of wave column c: swz depends on the row's low three bits only (= j).
template <int W>
struct ColIdx {
  int b;
  __device__ __forceinline__ ColIdx(int c, int j) : b(j * W + (c ^ swz(j))) {}
  __device__ __forceinline__ int operator()(int m) const { return b + 8 * m * W; }
};

// Dynamic shared memory: the wave, then one exchange buffer per eight-thread line group.
template <int W>
__host__ __device__ constexpr int exchange_floats2() {
  return MSP_TRANSPOSED_EXCHANGE ? kXGroup(W / 8) : 8 * (W / 8 + 1);
}
template <int W>
constexpr size_t position_smem_bytes() {
  return ((size_t)W * W + (size_t)(W / 2) * exchange_floats2<W>()) * sizeof(float2);
}

// CPLX: transmission mode (the paper's complex slices o_l).  The stash then holds the wave
// incident on each slice and the window gradient is dL/dconj(o_l) = conj(psi_in,l) o chi_l;
// in potential mode it holds the exit wave and the gradient is 2 sigma Im(conj(E_l) chi_l).
template <int W, int MODE, bool CPLX = false>
__global__ void __launch_bounds__(4 * W, 1) position_kernel(const PosParams p) {
  using G = Geo<W>;
  constexpr int N1 = G::N1;
  extern __shared__ float2 sm[];
  __shared__ float2 s_tw[N1 * 8];   // w_W^(j k1) at [k1 * 8 + j]
  __shared__ float2 s_h1[W];        // h1(k) = exp(-i pi dz lambda q_k^2) / W
  __shared__ float red[G::NT / 32];

  const int tid = threadIdx.x;
  const int j = tid & 7;
  const int grp = tid >> 3;
  const size_t WW = (size_t)W * W;
  const size_t plane = (size_t)p.Ny * p.Nx;
  float2* xb = sm + W * W + grp * exchange_floats2<W>();   // this group's exchange buffer

  if (tid < N1 * 8) {   // evaluated in double, rounded once
    const int k1 = tid >> 3, jj = tid & 7;
    double sn, cs;
    sincospi(2.0 * (double)((jj * k1) % W) / (double)W, &sn, &cs);
    s_tw[tid] = make_float2((float)cs, (float)-sn);
  }
  if (tid < W) s_h1[tid] = p.h1[tid];
  __syncthreads();
#if MSP_TWIDDLE_REGISTERS
  const RegisterTwiddles<W, 8> tw(s_tw, j);
#else
  const SharedTwiddles<8> tw{s_tw, j};
#endif

  const int L = p.L;
  const float zthr2 = (MODE == MODE_FORWARD) ? 0.f : (float)p.zthr2[0];
  const bool need_stash = (MODE == MODE_LOSS_GRAD && !p.loss_only) || (MODE == MODE_LAYER);
  const int lowest = (MODE == MODE_LAYER) ? p.layer : 0;
  bool first_dprobe = true;
  // TMEM stash (W = 128 only): slot of slice l, or -1 for the global stash
  constexpr bool kTmem = MSP_TMEM_STASH && W == 128 && (MODE == MODE_LOSS_GRAD || MODE == MODE_LAYER);
  __shared__ uint32_t s_tmem;
  TmemStash ts{0};
  if constexpr (kTmem) {
    if (tid < 32) tc::tmem_alloc(&s_tmem, 512);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const int warp = tid >> 5;
    ts.base = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(128 * (warp >> 2));
  }
  auto tslot = [&](int l) -> int {
    if constexpr (!kTmem) return -1;
    if (MODE == MODE_LAYER) return 0;
    return l >= L - 2 ? l - (L - 2 > 0 ? L - 2 : 0) : -1;
  };

  for (int s = blockIdx.x; s < p.S; s += gridDim.x) {
    const int2 ps = p.pos[s];
    const int y0 = ps.x, x0 = ps.y;
    const bool ok = (y0 >= 0) && (x0 >= 0) && (y0 <= p.Ny - W) && (x0 <= p.Nx - W);
    if (!ok) {
      if (tid == 0) atomicMax(p.err, 1);
      // outputs of a skipped position are zero
      if (MODE == MODE_FORWARD) {
        for (size_t i = tid; i < WW; i += G::NT) p.I_out[s * WW + i] = 0.f;
      } else {
        if (tid == 0) p.loss_part[s] = 0.0;
        constexpr int CW = CPLX ? 2 : 1;
        if (MODE == MODE_LOSS_GRAD && !p.dVred)
          for (size_t i = tid; i < CW * WW * L; i += G::NT) p.wgrad[CW * s * WW * L + i] = 0.f;
        if (MODE == MODE_LAYER && !p.dVred) {
          for (size_t i = tid; i < CW * WW; i += G::NT) p.wgrad[CW * s * WW + i] = 0.f;
          for (size_t i = tid; i < WW; i += G::NT) p.willum[s * WW + i] = 0.f;
        }
      }
      continue;  // uniform across the CTA
    }
    const size_t win0 = (size_t)y0 * p.Nx + x0;
    float2* stash = p.stash + (size_t)blockIdx.x * (MODE == MODE_LOSS_GRAD ? L : 1) * WW;

    // ---------------- forward: slice 0, rows ----------------
#pragma unroll 1
    for (int it = 0; it < G::LPG; ++it) {
      const int r = grp + G::GROUPS * it;
      float2 v[N1];
      const float2* T0 = p.T + win0 + (size_t)r * p.Nx;
#pragma unroll
      for (int m = 0; m < N1; ++m) v[m] = p.probe[r * W + j + 8 * m];
      const bool keep0 = need_stash && (MODE == MODE_LOSS_GRAD || p.layer == 0);
      if (CPLX && keep0) {
        if constexpr (kTmem) {
          if (tslot(0) >= 0) ts.store(tslot(0), it, v);   // incident wave
        }
        if (tslot(0) < 0) {
#pragma unroll
          for (int m = 0; m < N1; ++m) stash[r * W + j + 8 * m] = v[m];   // incident wave
        }
      }
#pragma unroll
      for (int m = 0; m < N1; ++m) v[m] = cmul(v[m], T0[j + 8 * m]);
      if (!CPLX && keep0) {
        if constexpr (kTmem) {
          if (tslot(0) >= 0) ts.store(tslot(0), it, v);   // exit wave
        }
        if (tslot(0) < 0) {
#pragma unroll
          for (int m = 0; m < N1; ++m) stash[r * W + j + 8 * m] = v[m];   // exit wave
        }
      }
      LINE_FFT<W, false>(v, tw, xb, j);
#pragma unroll
      for (int m = 0; m < N1; ++m) sm[RowIdx<W>(r, j)(m)] = v[m];
    }
    __syncthreads();

    float lsum = 0.f;
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
      if (l < L - 1) {
        // columns: F, x H / W^2, F^-1 (unnormalised)
#pragma unroll 1
        for (int it = 0; it < G::LPG; ++it) {
          const int c = grp + G::GROUPS * it;
          const ColIdx<W> ca(c, j);
          float2 v[N1];
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = sm[ca(m)];
          LINE_FFT<W, false>(v, tw, xb, j);
          const float2 hx = s_h1[c];
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = cmul(v[m], cmul(s_h1[j + 8 * m], hx));
          LINE_FFT<W, true>(v, tw, xb, j);
#pragma unroll
          for (int m = 0; m < N1; ++m) sm[ca(m)] = v[m];
        }
        __syncthreads();
        // rows: F^-1, transmit slice l+1, keep the exit wave, F
        const float2* Tl = p.T + (size_t)(l + 1) * plane + win0;
        const bool keep = need_stash && (MODE == MODE_LOSS_GRAD || p.layer == l + 1);
        float2* st = stash + (MODE == MODE_LOSS_GRAD ? (size_t)(l + 1) * WW : 0);
#pragma unroll 1
        for (int it = 0; it < G::LPG; ++it) {
          const int r = grp + G::GROUPS * it;
          const RowIdx<W> ra(r, j);
          float2 t[N1], v[N1];
          const float2* Tr = Tl + (size_t)r * p.Nx;
#pragma unroll
          for (int m = 0; m < N1; ++m) t[m] = Tr[j + 8 * m];     // in flight during the transform
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = sm[ra(m)];
          LINE_FFT<W, true>(v, tw, xb, j);
          if (CPLX && keep) {
            if constexpr (kTmem) {
              if (tslot(l + 1) >= 0) ts.store(tslot(l + 1), it, v);   // incident wave
            }
            if (tslot(l + 1) < 0) {
#pragma unroll
              for (int m = 0; m < N1; ++m) st[r * W + j + 8 * m] = v[m];   // incident wave
            }
          }
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = cmul(v[m], t[m]);
          if (!CPLX && keep) {
            if constexpr (kTmem) {
              if (tslot(l + 1) >= 0) ts.store(tslot(l + 1), it, v);   // exit wave
            }
            if (tslot(l + 1) < 0) {
#pragma unroll
              for (int m = 0; m < N1; ++m) st[r * W + j + 8 * m] = v[m];   // exit wave
            }
          }
          LINE_FFT<W, false>(v, tw, xb, j);
#pragma unroll
          for (int m = 0; m < N1; ++m) sm[ra(m)] = v[m];
        }
        __syncthreads();
      } else {
        // far field Psi = F(E_L): finish with the column transforms
#pragma unroll 1
        for (int it = 0; it < G::LPG; ++it) {
          const int c = grp + G::GROUPS * it;
          const ColIdx<W> ca(c, j);
          float2 v[N1];
          float im[N1];
          if (MODE != MODE_FORWARD) {
            const float* ip = p.I_meas + s * WW + c;
#pragma unroll
            for (int m = 0; m < N1; ++m) im[m] = __ldcs(ip + (j + 8 * m) * W);   // read once: evict first; in flight during the transform
          }
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = sm[ca(m)];
          LINE_FFT<W, false>(v, tw, xb, j);
          if (MODE == MODE_FORWARD) {
            float* out = p.I_out + s * WW + c;
#pragma unroll
            for (int m = 0; m < N1; ++m) out[(j + 8 * m) * W] = fmaf(v[m].x, v[m].x, v[m].y * v[m].y);
          } else {
            // amplitude-flow residual R = Psi - sqrt(I) Psi / |Psi| (fraction 0 where Psi counts as 0)
#pragma unroll
            for (int m = 0; m < N1; ++m) {
              const float a2 = fmaf(v[m].x, v[m].x, v[m].y * v[m].y);
              const float a = sqrtf(a2);
              const float rt = sqrtf(im[m]);
              const float d = rt - a;
              lsum = fmaf(d, d, lsum);
              // below the threshold the fraction is 0, so R = Psi (f = 1); a2 > zthr2 >= 0 implies a > 0
              const float f = (a2 > zthr2) ? (1.f - rt / a) : 1.f;
              v[m] = make_float2(v[m].x * f, v[m].y * f);
            }
            // chi = F^H R: inverse column transforms now, rows below
            if (!p.loss_only) {
              LINE_FFT<W, true>(v, tw, xb, j);
#pragma unroll
              for (int m = 0; m < N1; ++m) sm[ca(m)] = v[m];
            }
          }
        }
        if (MODE != MODE_FORWARD) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
          if ((tid & 31) == 0) red[tid >> 5] = lsum;
        }
        __syncthreads();
        if (MODE != MODE_FORWARD && tid == 0) {
          double acc = 0.0;
#pragma unroll 1
          for (int w = 0; w < G::NT / 32; ++w) acc += (double)red[w];
          p.loss_part[s] = acc;
        }
      }
    }
    if (MODE == MODE_FORWARD || p.loss_only) {
      __syncthreads();
      continue;
    }

    // ---------------- adjoint: slices L-1 .. lowest ----------------
#pragma unroll 1
    for (int l = L - 1; l >= lowest; --l) {
      const bool grad_here = (MODE == MODE_LOSS_GRAD) || (MODE == MODE_LAYER && l == p.layer);
      const bool go_on = (l > lowest) || (l == 0 && MODE != MODE_LAYER && p.want_dprobe);
      const float2* Tl = p.T + (size_t)l * plane + win0;
      const float2* st = stash + (MODE == MODE_LOSS_GRAD ? (size_t)l * WW : 0);
      // window gradients: [S][L][W][W] (LOSS_GRAD) or [S][W][W] (LAYER), float2 in transmission mode
      float* wg = p.wgrad + (CPLX ? 2 : 1) * (MODE == MODE_LOSS_GRAD ? ((size_t)s * L + l) * WW : (size_t)s * WW);
#pragma unroll 1
      for (int it = 0; it < G::LPG; ++it) {
        const int r = grp + G::GROUPS * it;
        const RowIdx<W> ra(r, j);
        float2 e[N1], v[N1];
        if (grad_here) {
          if constexpr (kTmem) {
            if (tslot(l) >= 0) ts.load(tslot(l), it, e);
          }
          if (tslot(l) < 0) {
#pragma unroll
            for (int m = 0; m < N1; ++m) e[m] = st[r * W + j + 8 * m];   // in flight during the transform
          }
        }
#pragma unroll
        for (int m = 0; m < N1; ++m) v[m] = sm[ra(m)];
        LINE_FFT<W, true>(v, tw, xb, j);   // v = chi_l (row r)
        if (grad_here) {
          // object-frame offset of this row's first element (the layer step's map is one slice)
          const size_t o = (MODE == MODE_LOSS_GRAD ? (size_t)l * plane : 0) + win0 + (size_t)r * p.Nx + j;
          if (p.dVred) {
            // added into the object-frame gradient at once (reductions in L2)
            if (CPLX) {
#pragma unroll
              for (int m = 0; m < N1; ++m) atomicAdd(reinterpret_cast<float2*>(p.dVred) + o + 8 * m, cmulc(v[m], e[m]));
            } else {
#pragma unroll
              for (int m = 0; m < N1; ++m) atomicAdd(p.dVred + o + 8 * m, p.two_sigma * fmaf(e[m].x, v[m].y, -e[m].y * v[m].x));
            }
          } else if (CPLX) {
            // dL/dconj(o_l) on the window: conj(psi_in,l) o chi_l
            float2* wg2 = reinterpret_cast<float2*>(wg) + r * W + j;
#pragma unroll
            for (int m = 0; m < N1; ++m) __stcs(wg2 + 8 * m, cmulc(v[m], e[m]));
          } else {
            // dL/dV_l on the window: 2 sigma Im(conj(E_l) chi_l)
#pragma unroll
            for (int m = 0; m < N1; ++m) __stcs(wg + r * W + j + 8 * m, p.two_sigma * fmaf(e[m].x, v[m].y, -e[m].y * v[m].x));
          }
          if (MODE == MODE_LAYER) {   // |psi_in,l|^2 (= |E_l|^2 for unimodular slices)
            if (p.illumred) {
#pragma unroll
              for (int m = 0; m < N1; ++m) atomicAdd(p.illumred + o + 8 * m, fmaf(e[m].x, e[m].x, e[m].y * e[m].y));
            } else {
#pragma unroll
              for (int m = 0; m < N1; ++m) __stcs(p.willum + s * WW + r * W + j + 8 * m, fmaf(e[m].x, e[m].x, e[m].y * e[m].y));
            }
          }
        }
        if (go_on) {
          const float2* Tr = Tl + (size_t)r * p.Nx;
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = cmulc(v[m], Tr[j + 8 * m]);   // conj(X_l) o chi_l
          if (l == 0) {
            float2* dp = p.dprobe_part + (size_t)blockIdx.x * WW + r * W;
            if (first_dprobe) {
#pragma unroll
              for (int m = 0; m < N1; ++m) dp[j + 8 * m] = v[m];
            } else {
#pragma unroll
              for (int m = 0; m < N1; ++m) dp[j + 8 * m] = cadd(dp[j + 8 * m], v[m]);
            }
          } else {
            LINE_FFT<W, false>(v, tw, xb, j);
#pragma unroll
            for (int m = 0; m < N1; ++m) sm[ra(m)] = v[m];
          }
        }
      }
      if (l == 0 && go_on) first_dprobe = false;
      if (!go_on || l == 0) break;
      __syncthreads();
      // columns of G^H: F, x conj(H) / W^2, F^-1
#pragma unroll 1
      for (int it = 0; it < G::LPG; ++it) {
        const int c = grp + G::GROUPS * it;
        const ColIdx<W> ca(c, j);
        float2 v[N1];
#pragma unroll
        for (int m = 0; m < N1; ++m) v[m] = sm[ca(m)];
        LINE_FFT<W, false>(v, tw, xb, j);
        const float2 hx = s_h1[c];
#pragma unroll
        for (int m = 0; m < N1; ++m) v[m] = cmulc(v[m], cmul(s_h1[j + 8 * m], hx));
        LINE_FFT<W, true>(v, tw, xb, j);
#pragma unroll
        for (int m = 0; m < N1; ++m) sm[ca(m)] = v[m];
      }
      __syncthreads();
    }
    __syncthreads();
  }

  // a CTA whose every position was skipped still owns a (zero) probe partial
  if ((MODE == MODE_LOSS_GRAD || MODE == MODE_PROBE) && p.want_dprobe && first_dprobe) {
    float2* dp = p.dprobe_part + (size_t)blockIdx.x * WW;
    for (size_t i = tid; i < WW; i += G::NT) dp[i] = make_float2(0.f, 0.f);
  }
  if constexpr (kTmem) {
    tc::fence_before();
    __syncthreads();
    if (tid < 32) {
      tc::fence_after();
      tc::tmem_dealloc(s_tmem, 512);
    }
  }
}

// ----------------------------------------------------------------------------
// launch helpers
// ----------------------------------------------------------------------------

template <int W, int MODE, bool CPLX>
static cudaError_t launch_one(const PosParams& p, int grid, cudaStream_t st) {
  const size_t smem = position_smem_bytes<W>();
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(position_kernel<W, MODE, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  position_kernel<W, MODE, CPLX><<<grid, 4 * W, smem, st>>>(p);
  return cudaGetLastError();
}

template <int W, bool CPLX>
static cudaError_t launch_wc(int mode, const PosParams& p, int grid, cudaStream_t st) {
  switch (mode) {
    case MODE_FORWARD: return launch_one<W, MODE_FORWARD, CPLX>(p, grid, st);
    case MODE_LOSS_GRAD: return launch_one<W, MODE_LOSS_GRAD, CPLX>(p, grid, st);
    case MODE_LAYER: return launch_one<W, MODE_LAYER, CPLX>(p, grid, st);
    default: return launch_one<W, MODE_PROBE, CPLX>(p, grid, st);
  }
}

template <int W>
static cudaError_t launch_w(int mode, const PosParams& p, int grid, cudaStream_t st) {
  // the forward model reads the slices the same way in both parametrisations
  if (p.cplx && mode != MODE_FORWARD) return launch_wc<W, true>(mode, p, grid, st);
  return launch_wc<W, false>(mode, p, grid, st);
}

cudaError_t launch_position_cluster_kernel(int mode, const PosParams& p, int clusters, cudaStream_t st);
int position_clusters_resident();

// `grid` counts position slots: CTAs for W = 64 / 128, four-CTA clusters for W = 256.
cudaError_t launch_position_kernel(int win, int mode, const PosParams& p, int grid, cudaStream_t st) {
  if (win == 64) return launch_w<64>(mode, p, grid, st);
  if (win == 128) return launch_w<128>(mode, p, grid, st);
  return launch_position_cluster_kernel(mode, p, grid, st);
}

// CTAs of the fused kernel that fit on one SM (same for every mode of a window size).
static int position_ctas_per_sm(int win) {
  int n = 0;
  const size_t smem = win == 64 ? position_smem_bytes<64>() : position_smem_bytes<128>();
  if (win == 64) {
    cudaFuncSetAttribute(position_kernel<64, MODE_LOSS_GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, position_kernel<64, MODE_LOSS_GRAD>, 4 * 64, smem);
  } else {
    cudaFuncSetAttribute(position_kernel<128, MODE_LOSS_GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, position_kernel<128, MODE_LOSS_GRAD>, 4 * 128, smem);
  }
  return n < 1 ? 1 : n;
}

// Positions the fused kernel processes at once on the current device (its persistent
// grid): resident CTAs for W = 64 / 128, resident four-CTA clusters for W = 256.
int position_slots(int win) {
  if (win == 256) return position_clusters_resident();
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * position_ctas_per_sm(win);
}

}  // namespace msp
