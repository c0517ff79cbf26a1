// msp_position_cluster.cu -- the fused per-position forward / adjoint kernel for
// W = 256, resident in the distributed shared memory of a four-CTA cluster.
//
// A 256 x 256 complex wave (512 KB) does not fit one SM's shared memory, so each
// scan position is owned by a cluster of four CTAs on four SMs: CTA k keeps wave
// rows 64k .. 64k+63 in its own shared memory (128 KB).  Row phases (the row
// transforms, the transmit of the next slice, the stash of exit waves, the window
// gradients) work on local rows only.  Column phases (the column transforms with
// the propagator between them, the far-field residual) take CTA k through columns
// 64k .. 64k+63, reading and writing the rows of all four CTAs through distributed
// shared memory.  A cluster barrier separates the phases.  The arithmetic is the
// same as position_kernel's (Sec. 2.1 recursion, Sec. 3.2 residual, Sec. 3.3
// adjoint), with sixteen-thread line groups and 16 x 16 four-step line transforms.
//
// Local layout: wave element (rl, c) of CTA-local row rl lives at rl * 256 + (c ^ (rl & 15)),
// which keeps the row accesses and the (local or remote) column accesses of a
// half-warp on sixteen distinct banks.  Column accesses use explicit shared::cluster
// addresses (mapa, ld/st.shared::cluster), which keep them on the shared-memory path;
// generic pointers into another CTA's shared memory take the global load/store path.
#include <cooperative_groups.h>

#include "msp_fft.cuh"
#include "msp_kernels.cuh"

namespace cg = cooperative_groups;

namespace msp {

// 8-byte access to the shared memory of a CTA of this cluster, by shared::cluster address
__device__ __forceinline__ uint32_t cluster_addr(const void* local, int rank) {
  uint32_t a;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
  return a;
}
__device__ __forceinline__ float2 ld_cluster(uint32_t a) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_cluster(uint32_t a, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}

namespace c256 {
constexpr int W = 256;
constexpr int CL = 4;             // CTAs per cluster
constexpr int RW = W / CL;        // wave rows (and columns processed) per CTA
constexpr int T = 16;             // threads per line
constexpr int N1 = W / T;         // values per thread per line
constexpr int NT = 512;           // threads per CTA
constexpr int GROUPS = NT / T;    // line groups per CTA
constexpr int LPG = RW / GROUPS;  // lines per group per phase
constexpr int XS = N1 + 1;        // exchange-buffer stride
constexpr size_t SMEM = ((size_t)RW * W + (size_t)GROUPS * T * XS) * sizeof(float2);
}  // namespace c256

// CPLX: transmission mode, as in position_kernel.
template <int MODE, bool CPLX = false>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(512, 1) position_cluster_kernel(const PosParams p) {
  using namespace c256;
  extern __shared__ float2 sm[];
  __shared__ float2 s_tw[N1 * T];   // w_256^(j k1) at [k1 * 16 + j]
  __shared__ float2 s_h1[W];        // h1(k) = exp(-i pi dz lambda q_k^2) / W
  __shared__ float red[NT / 32];

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cl = blockIdx.x / CL;
  const int ncl = gridDim.x / CL;
  const int tid = threadIdx.x;
  const int j = tid & (T - 1);
  const int grp = tid / T;
  const size_t WW = (size_t)W * W;
  const size_t plane = (size_t)p.Ny * p.Nx;
  float2* xb = sm + RW * W + grp * T * XS;

  if (tid < N1 * T) {   // evaluated in double, rounded once
    const int k1 = tid / T, jj = tid % T;
    double sn, cs;
    sincospi(2.0 * (double)((jj * k1) % W) / (double)W, &sn, &cs);
    s_tw[tid] = make_float2((float)cs, (float)-sn);
  }
  if (tid < W) s_h1[tid] = p.h1[tid];
  __syncthreads();
  const RegisterTwiddles<W, T> tw(s_tw, j);

  // Rows of the wave on every CTA of the cluster (shared::cluster addresses of element 0).
  uint32_t rows[CL];
#pragma unroll
  for (int k = 0; k < CL; ++k) rows[k] = cluster_addr(sm, k);

  // local row rl, element j + 16m
  auto rix = [&](int rl, int m) { return rl * W + ((j ^ (rl & 15)) + T * m); };
  // column c, global row j + 16m: CTA m >> 2, local row j + 16 (m & 3)
  auto cix = [&](int c, int m) { return (j + T * (m & 3)) * W + (c ^ j); };
  auto col_ld = [&](int c, int m) { return ld_cluster(rows[m >> 2] + 8u * (uint32_t)cix(c, m)); };
  auto col_st = [&](int c, int m, float2 v) { st_cluster(rows[m >> 2] + 8u * (uint32_t)cix(c, m), v); };

  const int L = p.L;
  const float zthr2 = (MODE == MODE_FORWARD) ? 0.f : (float)p.zthr2[0];
  const bool need_stash = (MODE == MODE_LOSS_GRAD && !p.loss_only) || (MODE == MODE_LAYER);
  const int lowest = (MODE == MODE_LAYER) ? p.layer : 0;
  const size_t slot = (MODE == MODE_LOSS_GRAD ? (size_t)L : 1) * WW;   // stash per cluster
  bool first_dprobe = true;

  for (int s = cl; s < p.S; s += ncl) {
    const int2 ps = p.pos[s];
    const int y0 = ps.x, x0 = ps.y;
    const bool ok = (y0 >= 0) && (x0 >= 0) && (y0 <= p.Ny - W) && (x0 <= p.Nx - W);
    if (!ok) {   // the same decision on every CTA of the cluster
      if (tid == 0 && rank == 0) atomicMax(p.err, 1);
      const size_t r0 = (size_t)rank * RW * W, r1 = r0 + (size_t)RW * W;
      if (MODE == MODE_FORWARD) {
        for (size_t i = r0 + tid; i < r1; i += NT) p.I_out[s * WW + i] = 0.f;
      } else {
        if (tid == 0) p.loss_part[(size_t)s * CL + rank] = 0.0;
        constexpr int CW = CPLX ? 2 : 1;
        if (MODE == MODE_LOSS_GRAD && !p.dVred)
          for (int l = 0; l < L; ++l)
            for (size_t i = CW * r0 + tid; i < CW * r1; i += NT) p.wgrad[CW * ((size_t)s * L + l) * WW + i] = 0.f;
        if (MODE == MODE_LAYER && !p.dVred) {
          for (size_t i = CW * r0 + tid; i < CW * r1; i += NT) p.wgrad[CW * s * WW + i] = 0.f;
          for (size_t i = r0 + tid; i < r1; i += NT) p.willum[s * WW + i] = 0.f;
        }
      }
      continue;
    }
    const size_t win0 = (size_t)y0 * p.Nx + x0;
    float2* stash = p.stash + (size_t)cl * slot;

    // ---------------- forward: slice 0, local rows ----------------
#pragma unroll 1
    for (int it = 0; it < LPG; ++it) {
      const int rl = grp + GROUPS * it, gr = rank * RW + rl;
      float2 v[N1];
      const float2* T0 = p.T + win0 + (size_t)gr * p.Nx + j;
      const float2* pr = p.probe + (size_t)gr * W + j;
#pragma unroll
      for (int m = 0; m < N1; ++m) v[m] = pr[T * m];
      if (CPLX && need_stash && (MODE == MODE_LOSS_GRAD || p.layer == 0)) {
#pragma unroll
        for (int m = 0; m < N1; ++m) stash[(size_t)gr * W + j + T * m] = v[m];   // incident wave
      }
#pragma unroll
      for (int m = 0; m < N1; ++m) v[m] = cmul(v[m], T0[T * m]);
      if (!CPLX && need_stash && (MODE == MODE_LOSS_GRAD || p.layer == 0)) {
#pragma unroll
        for (int m = 0; m < N1; ++m) stash[(size_t)gr * W + j + T * m] = v[m];   // exit wave
      }
      line_fft<W, false, RegisterTwiddles<W, T>, T>(v, tw, xb, j);
#pragma unroll
      for (int m = 0; m < N1; ++m) sm[rix(rl, m)] = v[m];
    }
    cluster.sync();

    float lsum = 0.f;
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
      if (l < L - 1) {
        // columns 64 rank .. : F, x H / W^2, F^-1 across the cluster
#pragma unroll 1
        for (int it = 0; it < LPG; ++it) {
          const int c = rank * RW + grp + GROUPS * it;
          float2 v[N1];
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = col_ld(c, m);
          line_fft<W, false, RegisterTwiddles<W, T>, T>(v, tw, xb, j);
          const float2 hx = s_h1[c];
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = cmul(v[m], cmul(s_h1[j + T * m], hx));
          line_fft<W, true, RegisterTwiddles<W, T>, T>(v, tw, xb, j);
#pragma unroll
          for (int m = 0; m < N1; ++m) col_st(c, m, v[m]);
        }
        cluster.sync();
        // local rows: F^-1, transmit slice l+1, keep the exit wave, F
        const float2* Tl = p.T + (size_t)(l + 1) * plane + win0;
        const bool keep = need_stash && (MODE == MODE_LOSS_GRAD || p.layer == l + 1);
        float2* st = stash + (MODE == MODE_LOSS_GRAD ? (size_t)(l + 1) * WW : 0);
#pragma unroll 1
        for (int it = 0; it < LPG; ++it) {
          const int rl = grp + GROUPS * it, gr = rank * RW + rl;
          float2 t[N1], v[N1];
          const float2* Tr = Tl + (size_t)gr * p.Nx + j;
#pragma unroll
          for (int m = 0; m < N1; ++m) t[m] = Tr[T * m];     // in flight during the transform
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = sm[rix(rl, m)];
          line_fft<W, true, RegisterTwiddles<W, T>, T>(v, tw, xb, j);
          if (CPLX && keep) {
#pragma unroll
            for (int m = 0; m < N1; ++m) st[(size_t)gr * W + j + T * m] = v[m];   // incident wave
          }
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = cmul(v[m], t[m]);
          if (!CPLX && keep) {
#pragma unroll
            for (int m = 0; m < N1; ++m) st[(size_t)gr * W + j + T * m] = v[m];   // exit wave
          }
          line_fft<W, false, RegisterTwiddles<W, T>, T>(v, tw, xb, j);
#pragma unroll
          for (int m = 0; m < N1; ++m) sm[rix(rl, m)] = v[m];
        }
        cluster.sync();
      } else {
        // far field Psi = F(E_L): the column transforms of this CTA's columns
#pragma unroll 1
        for (int it = 0; it < LPG; ++it) {
          const int c = rank * RW + grp + GROUPS * it;
          float2 v[N1];
          float im[N1];
          if (MODE != MODE_FORWARD) {
            const float* ip = p.I_meas + s * WW + c;
#pragma unroll
            for (int m = 0; m < N1; ++m) im[m] = __ldcs(ip + (size_t)(j + T * m) * W);   // read once: evict first
          }
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = col_ld(c, m);
          line_fft<W, false, RegisterTwiddles<W, T>, T>(v, tw, xb, j);
          if (MODE == MODE_FORWARD) {
            float* out = p.I_out + s * WW + c;
#pragma unroll
            for (int m = 0; m < N1; ++m) out[(size_t)(j + T * m) * W] = fmaf(v[m].x, v[m].x, v[m].y * v[m].y);
          } else {
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
            if (!p.loss_only) {
              line_fft<W, true, RegisterTwiddles<W, T>, T>(v, tw, xb, j);
#pragma unroll
              for (int m = 0; m < N1; ++m) col_st(c, m, v[m]);
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
          for (int w = 0; w < NT / 32; ++w) acc += (double)red[w];
          p.loss_part[(size_t)s * CL + rank] = acc;
        }
        cluster.sync();
      }
    }
    if (MODE == MODE_FORWARD || p.loss_only) continue;   // the far-field phase ended with a cluster barrier

    // ---------------- adjoint: slices L-1 .. lowest ----------------
#pragma unroll 1
    for (int l = L - 1; l >= lowest; --l) {
      const bool grad_here = (MODE == MODE_LOSS_GRAD) || (MODE == MODE_LAYER && l == p.layer);
      const bool go_on = (l > lowest) || (l == 0 && MODE != MODE_LAYER && p.want_dprobe);
      const float2* Tl = p.T + (size_t)l * plane + win0;
      const float2* st = stash + (MODE == MODE_LOSS_GRAD ? (size_t)l * WW : 0);
      float* wg = p.wgrad + (CPLX ? 2 : 1) * (MODE == MODE_LOSS_GRAD ? ((size_t)s * L + l) * WW : (size_t)s * WW);
#pragma unroll 1
      for (int it = 0; it < LPG; ++it) {
        const int rl = grp + GROUPS * it, gr = rank * RW + rl;
        float2 e[N1], v[N1];
        if (grad_here) {
#pragma unroll
          for (int m = 0; m < N1; ++m) e[m] = st[(size_t)gr * W + j + T * m];
        }
#pragma unroll
        for (int m = 0; m < N1; ++m) v[m] = sm[rix(rl, m)];
        line_fft<W, true, RegisterTwiddles<W, T>, T>(v, tw, xb, j);   // v = chi_l (row gr)
        if (grad_here) {
          // object-frame offset of this row's first element (the layer step's map is one slice)
          const size_t o = (MODE == MODE_LOSS_GRAD ? (size_t)l * plane : 0) + win0 + (size_t)gr * p.Nx + j;
          if (p.dVred) {
            // added into the object-frame gradient at once (reductions in L2)
            if (CPLX) {
#pragma unroll
              for (int m = 0; m < N1; ++m) atomicAdd(reinterpret_cast<float2*>(p.dVred) + o + T * m, cmulc(v[m], e[m]));
            } else {
#pragma unroll
              for (int m = 0; m < N1; ++m) atomicAdd(p.dVred + o + T * m, p.two_sigma * fmaf(e[m].x, v[m].y, -e[m].y * v[m].x));
            }
          } else if (CPLX) {
            float2* wg2 = reinterpret_cast<float2*>(wg) + (size_t)gr * W + j;
#pragma unroll
            for (int m = 0; m < N1; ++m) __stcs(wg2 + T * m, cmulc(v[m], e[m]));
          } else {
#pragma unroll
            for (int m = 0; m < N1; ++m)
              __stcs(wg + (size_t)gr * W + j + T * m, p.two_sigma * fmaf(e[m].x, v[m].y, -e[m].y * v[m].x));
          }
          if (MODE == MODE_LAYER && p.illumred) {
#pragma unroll
            for (int m = 0; m < N1; ++m) atomicAdd(p.illumred + o + T * m, fmaf(e[m].x, e[m].x, e[m].y * e[m].y));
          } else if (MODE == MODE_LAYER) {
#pragma unroll
            for (int m = 0; m < N1; ++m)
              __stcs(p.willum + s * WW + (size_t)gr * W + j + T * m, fmaf(e[m].x, e[m].x, e[m].y * e[m].y));
          }
        }
        if (go_on) {
          const float2* Tr = Tl + (size_t)gr * p.Nx + j;
#pragma unroll
          for (int m = 0; m < N1; ++m) v[m] = cmulc(v[m], Tr[T * m]);   // conj(X_l) o chi_l
          if (l == 0) {
            float2* dp = p.dprobe_part + (size_t)cl * WW + (size_t)gr * W + j;
            if (first_dprobe) {
#pragma unroll
              for (int m = 0; m < N1; ++m) dp[T * m] = v[m];
            } else {
#pragma unroll
              for (int m = 0; m < N1; ++m) dp[T * m] = cadd(dp[T * m], v[m]);
            }
          } else {
            line_fft<W, false, RegisterTwiddles<W, T>, T>(v, tw, xb, j);
#pragma unroll
            for (int m = 0; m < N1; ++m) sm[rix(rl, m)] = v[m];
          }
        }
      }
      if (l == 0 && go_on) first_dprobe = false;
      if (!go_on || l == 0) break;
      cluster.sync();
      // columns of G^H: F, x conj(H) / W^2, F^-1 across the cluster
#pragma unroll 1
      for (int it = 0; it < LPG; ++it) {
        const int c = rank * RW + grp + GROUPS * it;
        float2 v[N1];
#pragma unroll
        for (int m = 0; m < N1; ++m) v[m] = col_ld(c, m);
        line_fft<W, false, RegisterTwiddles<W, T>, T>(v, tw, xb, j);
        const float2 hx = s_h1[c];
#pragma unroll
        for (int m = 0; m < N1; ++m) v[m] = cmulc(v[m], cmul(s_h1[j + T * m], hx));
        line_fft<W, true, RegisterTwiddles<W, T>, T>(v, tw, xb, j);
#pragma unroll
        for (int m = 0; m < N1; ++m) col_st(c, m, v[m]);
      }
      cluster.sync();
    }
    cluster.sync();   // no CTA starts the next position while another still reads its rows
  }

  // a cluster whose every position was skipped still owns a (zero) probe partial
  if ((MODE == MODE_LOSS_GRAD || MODE == MODE_PROBE) && p.want_dprobe && first_dprobe) {
    float2* dp = p.dprobe_part + (size_t)cl * WW + (size_t)rank * RW * W;
    for (int i = tid; i < RW * W; i += NT) dp[i] = make_float2(0.f, 0.f);
  }
  cluster.sync();   // shared memory must outlive every remote access
}

template <int MODE, bool CPLX>
static cudaError_t launch_cluster_one(const PosParams& p, int clusters, cudaStream_t st) {
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(position_cluster_kernel<MODE, CPLX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c256::SMEM);
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  position_cluster_kernel<MODE, CPLX><<<clusters * c256::CL, c256::NT, c256::SMEM, st>>>(p);
  return cudaGetLastError();
}

template <bool CPLX>
static cudaError_t launch_cluster_c(int mode, const PosParams& p, int clusters, cudaStream_t st) {
  switch (mode) {
    case MODE_FORWARD: return launch_cluster_one<MODE_FORWARD, CPLX>(p, clusters, st);
    case MODE_LOSS_GRAD: return launch_cluster_one<MODE_LOSS_GRAD, CPLX>(p, clusters, st);
    case MODE_LAYER: return launch_cluster_one<MODE_LAYER, CPLX>(p, clusters, st);
    default: return launch_cluster_one<MODE_PROBE, CPLX>(p, clusters, st);
  }
}

cudaError_t launch_position_cluster_kernel(int mode, const PosParams& p, int clusters, cudaStream_t st) {
  if (p.cplx && mode != MODE_FORWARD) return launch_cluster_c<true>(mode, p, clusters, st);
  return launch_cluster_c<false>(mode, p, clusters, st);
}

// Four-CTA clusters of the W = 256 kernel that can be resident at once on this device.
int position_clusters_resident() {
  cudaFuncSetAttribute(position_cluster_kernel<MODE_LOSS_GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)c256::SMEM);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c256::CL, 1, 1);
  cfg.blockDim = dim3(c256::NT, 1, 1);
  cfg.dynamicSmemBytes = c256::SMEM;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = c256::CL;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, position_cluster_kernel<MODE_LOSS_GRAD>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  return n < 1 ? 1 : n;
}

}  // namespace msp
