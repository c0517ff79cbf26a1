/*
 * msp_smd.h -- C ABI of libmsp for Sparse Matrix Decomposition, the paper's second
 * method (arXiv 2205.03902, Sec. 3.4, Algorithm 2).
 *
 * Algorithm 2 works on the paper's own full-field model (Sec. 2.1 / 2.2): an N x N
 * object, an N x N probe shifted cyclically to S scan positions, an N x N detector.
 * The specimen is the dense transfer matrix A = O_M G O_{M-1} ... G O_1 (N^2 x N^2,
 * Eq. exit_wave_mslices) and the measurements are I = |F_2D A P|^2, P = (p^1 .. p^S)
 * the shifted probes.  One iteration of Algorithm 2 is
 *   1. gradient steps on A for Eq. (Opt_Prob_Matrix)     -> msp_smd_matrix_step
 *   2. a proximal step on every slice (Eq. Prox_Min), the lambda update of
 *      Eq. (Update Lambda) and A = lambda O_M prod G O   -> msp_smd_decompose
 * and the slices returned at the end are lambda^(1/M) O_m   -> msp_smd_final_slices.
 *
 * Conventions (shared with msp.h where they overlap)
 *   - F_2D is the unnormalised 2-D DFT of an N x N array vectorised row-major,
 *     kernel exp(-2 pi i k.n / N); ||F_2D||^2 = N^2.
 *   - G = F^-1 diag(h) F with h = exp(-i pi dz lambda (qy^2 + qx^2)) on the N-point
 *     grid q_k = k / (N pixel) for k < N/2, (k - N) / (N pixel) otherwise.
 *   - Slices o are complex, [M][N][N] interleaved (re, im) floats.  The probe is
 *     complex [N][N].  A is complex N^2 x N^2 stored COLUMN-MAJOR: column j (the
 *     exit wave of a unit impulse at object pixel j) is the contiguous N x N image
 *     A[j * N^2 .. j * N^2 + N^2 - 1].
 *   - Shift s = (ys, xs) puts the probe at p^s[y][x] = p[(y - ys) mod N][(x - xs) mod N];
 *     shifts are int32 [S][2] in 0 <= ys, xs < N.  Measurements are [S][N][N] floats,
 *     unshifted FFT order.
 *   - The matrix objective is 1/2 sum (sqrt(I) - |F A P|)^2 (Eq. Opt_Prob_Matrix, with
 *     its 1/2); U/|U| is taken as 0 where |U| <= 1e-5 sqrt(mean I).
 *   - Step of the matrix estimate: mu = 1 / (N^2 ||P||^2) with ||P|| = max_k |(F p)_k|,
 *     the exact spectral norm for the full raster scan (all N^2 shifts, the scan of the
 *     paper's Table 1) and an upper bound for any other set of distinct shifts.
 *   - Every slice takes its proximal step from the slices and lambda of iteration t
 *     (Eq. Prox_Min prints R_l^t, S_l^t, lambda^t), with mu_l = 1/c_l,
 *     c_l = (lambda prod_{m != l} max|o_m|)^2 >= (lambda ||R_l|| ||S_l||)^2, then the
 *     projection onto unit Frobenius norm.  lambda is real: the real part of the ratio
 *     of Eq. (Update Lambda), which is its least-squares value.
 *
 * Supported sizes: N in {16, 24, 32, 40, 48, 64}; 1 <= M <= 5 (M <= 3 for N = 64);
 * S >= 1.  Memory, ownership, errors and determinism as in msp.h: device pointers
 * owned by the caller, 16-byte aligned; scratch in the caller's workspace (256-byte
 * aligned, msp_smd_workspace_bytes); asynchronous on `stream`; nothing allocated;
 * fixed-order sums, so repeated calls give bit-identical results.
 */
#ifndef MSP_SMD_H
#define MSP_SMD_H

#include <stddef.h>
#include <stdint.h>

#include "msp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n;            /* N: object side = probe side = detector side            */
  int32_t n_slices;     /* M                                                      */
  int32_t n_pos;        /* S: probe shifts                                        */
  double  wavelength_A; /* electron wavelength (angstrom)                         */
  double  dz_A;         /* Fresnel propagation distance between slices (angstrom) */
  double  pixel_A;      /* object pixel size (angstrom)                           */
} msp_smd_geometry;

/* MSP_OK, MSP_EINVAL (NULL, non-positive or non-finite values, M < 1, S < 1) or
 * MSP_EUNSUPPORTED (N or M outside the supported sizes). */
msp_status msp_smd_validate_geometry(const msp_smd_geometry* g);

/* Workspace bytes for every msp_smd_* call with this geometry; 0 if invalid. */
size_t msp_smd_workspace_bytes(const msp_smd_geometry* g);

/* A = lambda * O_M prod_{m<M} G O_m (Eq. Initial), the initial matrix of Algorithm 2.
 * o: [M][N][N] complex (device, read); lambda: host scalar; A: N^2 x N^2 complex,
 * column-major (device, written). */
msp_status msp_smd_transfer(const msp_smd_geometry* g, const float* o, double lambda, float* A,
                            void* ws, size_t ws_bytes, void* stream);

/* One gradient step of Eq. (Opt_Prob_Matrix) (Sec. 3.4):
 *   A <- A - mu F^H ((|F A P| - sqrt(I)) o F A P / |F A P|) P^H.
 * A: in/out; probe [N][N] complex; shifts [S][2] int32; I [S][N][N] float.
 * step > 0 sets mu, step <= 0 takes mu = 1 / (N^2 ||P||^2).  objective_before (device
 * double, or NULL) receives the objective at the incoming A; mu_out (device double or
 * NULL) the step used.  The two contractions run on the tensor cores (tcgen05, operands
 * split into tf32 pairs); their waits are bounded, and a wait that runs out leaves A
 * invalid and raises the workspace flag, which msp_check_workspace(ws, stream) reports
 * as MSP_ETIMEOUT. */
msp_status msp_smd_matrix_step(const msp_smd_geometry* g, float* A, const float* probe,
                               const int32_t* shifts, const float* I, double step,
                               double* objective_before, double* mu_out,
                               void* ws, size_t ws_bytes, void* stream);

/* The decomposition half of one Algorithm 2 iteration, from the estimate Ahat held in A:
 * every slice takes the proximal step of Eq. (Prox_Min) from (o, lambda) of iteration t,
 * lambda becomes Re Tr(Ahat^H Atilde) / Tr(Atilde^H Atilde) with Atilde = A(o^{t+1})
 * (Eq. Update Lambda), and A becomes lambda Atilde.
 * A: in Ahat, out lambda Atilde; o: in/out [M][N][N] complex; lambda: device double,
 * in/out; objective_before (device double or NULL) receives 1/2 ||Ahat - lambda A(o^t)||_F^2. */
msp_status msp_smd_decompose(const msp_smd_geometry* g, float* A, float* o, double* lambda,
                             double* objective_before, void* ws, size_t ws_bytes, void* stream);

/* The slices Algorithm 2 returns: out_m = lambda^(1/M) o_m, with the principal complex
 * root (a negative lambda gives the phase pi/M), so that A(out) = lambda A(o).
 * o, out: [M][N][N] complex (device; may alias); lambda: device double. */
msp_status msp_smd_final_slices(const msp_smd_geometry* g, const float* o, const double* lambda,
                                float* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MSP_SMD_H */
