/*
 * msp.h -- C ABI of libmsp, the GB300 (sm_103a) hot path of inverse multislice
 * ptychography by layer-wise optimisation (arXiv 2205.03902).
 *
 * The library computes, for S scan positions at once, the multislice forward
 * model of Sec. 2.1 (E_1 = P o X_1, E_m = V_z(E_{m-1}) o X_m, I = |F(E_M)|^2),
 * the amplitude-flow loss and its Wirtinger gradient of Sec. 3.2, and the
 * gradient steps of Algorithm 1 (Sec. 3.3) and of the probe problem (Sec. 3.5).
 *
 * Conventions shared by every entry point
 *   - Slices are given as real projected potentials V (V*angstrom), the slice
 *     transmission being X_m = exp(i sigma V_m) (the phase grating of Sec. 2.1); or,
 *     with param = MSP_PARAM_TRANSMISSION, as the complex slices o_m themselves (the
 *     paper's own unknowns, Sec. 2.2 / 3.3).  In transmission mode every argument named
 *     V or dV below is complex, [L][Ny][Nx] interleaved (re, im) pairs, and gradients
 *     are the Wirtinger derivatives dL/dconj(o).
 *   - Window model: scan position s uses the W x W window of every slice whose
 *     top-left object pixel is pos[s] = (y, x); the probe is one W x W array.
 *     Every window must lie inside the object: 0 <= y <= Ny - W, 0 <= x <= Nx - W.
 *   - F is the unnormalised 2-D DFT (kernel exp(-2 pi i k.n / W)), F^-1 = F^H / W^2.
 *     Intensities are in unshifted FFT order (zero frequency at [0][0]).
 *   - Fresnel propagator h = exp(-i pi dz lambda (qy^2 + qx^2)), Eq. (fresnel_element)
 *     with zero tilt, q_k = k / (W pixel) for k < W/2 and (k - W) / (W pixel) otherwise.
 *     The slices are separated by dz; no propagation follows the last slice.
 *   - Loss: L = sum_s sum_k (sqrt(I_meas) - |Psi|)^2 (Sec. 3.2, no factor 1/2).  The
 *     gradient's residual is R = Psi - sqrt(I_meas) Psi/|Psi|, with the fraction Psi/|Psi|
 *     taken as 0 (so R = Psi) where the far-field value counts as zero (Sec. 3.2 sets the
 *     fraction to 0 where Qz = 0): where |Psi_k| <= 1e-5 ||p||_2, ||p||_2 being the probe's
 *     L2 norm (by Parseval the RMS far-field amplitude of a pattern of pure-phase slices).
 *     The threshold resolves "Psi = 0" above FP32 round-off and far below physical
 *     amplitudes; a literal Psi == 0 test would let round-off choose the residual's phase
 *     wherever the exact far field vanishes (outside the probe aperture at V = 0).
 *   - Complex arrays are interleaved float pairs (re, im), row-major.
 *
 * Memory and ownership
 *   - Every array argument is a DEVICE pointer owned by the caller, 16-byte aligned.
 *     Scalars written by the library (loss, step size) are device doubles.
 *   - The library allocates nothing.  Scratch space is the caller's workspace `ws`
 *     of at least msp_workspace_bytes(geometry) bytes (256-byte aligned), valid
 *     for the current device; one workspace serves one call at a time.
 *   - All compute calls are asynchronous on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream).  Results are valid once the stream has reached them.
 *
 * Errors
 *   - Every entry point returns an msp_status.  Argument errors are found on the
 *     host before anything is launched (MSP_EINVAL / MSP_EUNSUPPORTED); a failed
 *     launch returns MSP_ECUDA.  Nothing throws or exits across the ABI.
 *   - A scan window outside the object cannot be seen on the host (positions live
 *     on the device): the kernels skip such a position (its outputs are zero) and
 *     raise a flag in the workspace, which msp_check_workspace reports as MSP_EINVAL.
 *   - msp_last_error_message() describes the most recent failure of this thread.
 *
 * Results are deterministic by default: no atomics are used on data, every sum runs in a
 * fixed order, so repeated calls on the same device give bit-identical results.  The one
 * exception is opt-in: msp_set_overlap_add(MSP_OVERLAP_L2_REDUCE) trades the fixed order of
 * the sums over positions for reductions in L2 (results then agree to rounding).
 */
#ifndef MSP_H
#define MSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MSP_OK = 0,
  MSP_EINVAL = 1,        /* bad argument, null pointer, workspace too small, window outside object */
  MSP_ENOMEM = 2,        /* reserved: the library never allocates */
  MSP_ECUDA = 3,         /* a CUDA launch or runtime call failed */
  MSP_EUNSUPPORTED = 4,  /* valid but not implemented here (window size, parametrisation) */
  MSP_ETIMEOUT = 5,      /* a bounded device-side wait ran out (msp_check_workspace) */
  MSP_EDEVICE = 6        /* a tensor-core kernel could not confirm that its own MMAs had finished
                            before it released tensor memory: the device is no longer trusted
                            (msp_check_workspace; every later call on that device returns this) */
} msp_status;

/* Slice parametrisation: real potentials (X_m = exp(i sigma V_m)) or complex
 * transmissions o_m (the paper's parametrisation). */
enum { MSP_PARAM_POTENTIAL = 0, MSP_PARAM_TRANSMISSION = 1 };

/* Arithmetic of the forward model, the residual and the adjoint.
 *   MSP_PRECISION_FP32: everything in FP32 in the fused per-position kernel (the fast path).
 *   MSP_PRECISION_FP64_FORWARD: the forward model (transmit, Fresnel propagation, far field,
 *     Sec. 2.1) and the residual R = Psi - sqrt(I) Psi/|Psi| and loss (Sec. 3.2) in FP64, R
 *     and the stored exit waves rounded to FP32 once, the adjoint in FP32.  Near a fit the
 *     gradient is a small difference of far-field amplitudes, so the FP32 forward's rounding
 *     is amplified by ||Psi|| / ||R||; this mode removes that amplification.  Slower (GB300's
 *     FP64 rate is 1/64 of its FP32 rate) and with a larger workspace.
 *   MSP_PRECISION_BF16X3_DFT: the split-BF16 precision form.  Every 2-D Fourier transform of
 *     the forward model and of the adjoint is two passes of the W-point DFT as a matrix
 *     product on the tensor cores (the matrix-product form of the propagation that Sec. 6
 *     suggests), operands split into bf16 pairs x = hi + lo and multiplied as
 *     hi*hi + hi*lo + lo*hi with FP32 accumulation; waves in FP32, loss and probe-gradient
 *     sums in FP64.  About 2^-16 relative error per product.
 *   MSP_PRECISION_DF_FORWARD: MSP_PRECISION_FP64_FORWARD with the forward model in
 *     double-float arithmetic (each value an unevaluated sum of two FP32 numbers, about 48
 *     significand bits, operated on by error-free sums and fused-multiply-add products) on the
 *     FP32 pipe instead of the FP64 pipe: the same residual accuracy at a fraction of the cost. */
enum {
  MSP_PRECISION_FP32 = 0,
  MSP_PRECISION_FP64_FORWARD = 1,
  MSP_PRECISION_BF16X3_DFT = 2,
  MSP_PRECISION_DF_FORWARD = 3
};

/* Statement of the problem (Sec. 2.1).  Supported windows: W = 64, 128 or 256 (W = 256 runs
 * each position on a four-CTA thread-block cluster). */
typedef struct {
  int32_t n_slices;     /* L (the paper's M), >= 1                                 */
  int32_t obj_ny;       /* object rows Ny >= W                                     */
  int32_t obj_nx;       /* object columns Nx >= W                                  */
  int32_t win;          /* W: probe window side = detector side (64, 128, 256)    */
  int32_t n_pos;        /* S: scan positions, >= 0                                 */
  int32_t param;        /* MSP_PARAM_POTENTIAL or MSP_PARAM_TRANSMISSION          */
  double wavelength_A;  /* electron wavelength lambda in angstrom (Sec. 5.3.2)    */
  double sigma;         /* interaction constant, rad / (V angstrom)               */
  double dz_A;          /* slice separation = Fresnel distance Delta (Eq. fresnel_element) */
  double pixel_A;       /* real-space pixel size in angstrom                       */
  int32_t precision;    /* MSP_PRECISION_FP32, _FP64_FORWARD, _BF16X3_DFT, _DF_FORWARD */
} msp_geometry;

/* Checks a geometry on the host.  MSP_OK, MSP_EINVAL or MSP_EUNSUPPORTED. */
msp_status msp_validate_geometry(const msp_geometry* g);

/* Workspace bytes every compute call on `g` needs on the current device
 * (0 if the geometry is invalid). */
size_t msp_workspace_bytes(const msp_geometry* g);

/* Forward model (Sec. 2.1, Eq. intensity measurements):
 *   probe  [W][W] complex   incident probe P
 *   V      [L][Ny][Nx] float projected potentials
 *   pos    [S][2] int32     window top-left (y, x) per scan position
 *   I_out  [S][W][W] float  far-field intensities |F(E_M^s)|^2 (written) */
msp_status msp_forward(const msp_geometry* g, const float* probe, const float* V,
                       const int32_t* pos, float* I_out,
                       void* ws, size_t ws_bytes, void* stream);

/* Loss and gradients (Sec. 3.2 applied to Eq. Opt_Prob_Layerwise):
 *   I_meas  [S][W][W] float     measured intensities
 *   loss    device double [1]   L (written; may be NULL)
 *   dV      [L][Ny][Nx] float   dL/dV = 2 sigma Im(conj(X) o dL/dconj(X)), overlap-added
 *                               over all positions (written; may be NULL)
 *   dprobe  [W][W] complex      dL/dconj(P) = sum_s conj(X_1[win_s]) o chi_1^s (may be NULL) */
msp_status msp_loss_grad(const msp_geometry* g, const float* probe, const float* V,
                         const int32_t* pos, const float* I_meas,
                         double* loss, float* dV, float* dprobe,
                         void* ws, size_t ws_bytes, void* stream);

/* One gradient step of Algorithm 1 on slice `layer` (0-based), Eq.
 * (Opt_Prob_Amplitude_Flow_Step) with the other slices fixed:
 *   V[layer] <- V[layer] - mu dL/dV[layer]
 * step > 0 sets mu; step <= 0 takes mu = 1 / (2 sigma^2 W^2 max_pixel sum_s |psi_in,l^s|^2),
 * the spectral step ||Q_l||^-2 of Sec. 3.2 carried to the potential.  In transmission mode
 * o_l <- o_l - mu dL/dconj(o_l) with mu = 1 / (W^2 max_pixel sum_s |psi_in,l^s|^2
 * prod_{m > l} max_pixel |o_m|^2), ||Q_l||^-2 or, for non-unimodular later slices, a bound on it.
 *   V          [L][Ny][Nx] float, updated in place (only slice `layer` changes)
 *   loss_before device double [1], loss at the incoming V (may be NULL)
 *   mu_out      device double [1], step size used (may be NULL) */
msp_status msp_layer_step(const msp_geometry* g, const float* probe, float* V,
                          const int32_t* pos, const float* I_meas, int32_t layer,
                          double step, double* loss_before, double* mu_out,
                          void* ws, size_t ws_bytes, void* stream);

/* One amplitude-flow step on the probe (Sec. 3.5, Eq. Opt_Est_Probe, all positions):
 *   probe <- probe - mu sum_s conj(X_1[win_s]) o chi_1^s
 * step > 0 sets mu; step <= 0 takes mu = 1 / (S W^2) (= ||Q_p||^-2 for pure-phase slices).
 * normalize != 0 then rescales the probe so that W^2 ||p||^2 = mean_s sum_k I_meas^s.
 *   probe  [W][W] complex, updated in place; loss_before / mu_out as above. */
msp_status msp_probe_step(const msp_geometry* g, float* probe, const float* V,
                          const int32_t* pos, const float* I_meas, double step,
                          int32_t normalize, double* loss_before, double* mu_out,
                          void* ws, size_t ws_bytes, void* stream);

/* The plain method: Algorithm 1 (Layer-wise Estimation, Sec. 3.3) with optional probe
 * estimation (Sec. 3.5), run entirely on `stream` without host synchronisation.
 *   for t in [T]:  for l = 0 .. L-1 (ascending; each slice's prefix uses the slices already
 *                  updated in this sweep, Gauss-Seidel):  K steps of msp_layer_step on l
 *                  then P steps of msp_probe_step
 * The paper estimates the probe after the object (Sec. 3.5); P > 0 alternates the two,
 * which an initial probe with a defocus error needs; K = 0 runs probe steps only, so
 * "object, then probe" is two calls. */
typedef struct {
  int32_t sweeps;            /* T >= 0: iterations of Algorithm 1                         */
  int32_t steps_per_layer;   /* K >= 0: gradient steps per slice per sweep                */
  int32_t probe_steps;       /* P >= 0: probe steps after each sweep (0: probe known)     */
  int32_t normalize_probe;   /* != 0: rescale the probe after each probe step (msp_probe_step) */
  double layer_step;         /* mu of the slice steps; <= 0: the spectral step (msp_layer_step) */
  double probe_step;         /* mu of the probe steps; <= 0: 1 / (S W^2) (msp_probe_step)      */
} msp_plan;

/* Entries of the loss history of msp_reconstruct: T (L K + P) + 1 (0 if g or plan is invalid). */
size_t msp_reconstruct_history_length(const msp_geometry* g, const msp_plan* plan);

/* Runs `plan` from the caller's probe and slices, both updated in place (the probe only when
 * P > 0).  loss_history (device double [msp_reconstruct_history_length], may be NULL) receives
 * the loss before every step, in the order the steps run, and last the loss after the final
 * step.  pos, I_meas and the workspace are as for msp_layer_step (its workspace size covers
 * this call).  Argument errors return before anything is launched; a launch failure returns
 * MSP_ECUDA with the steps issued so far left queued on the stream. */
msp_status msp_reconstruct(const msp_geometry* g, const msp_plan* plan, float* probe, float* V,
                           const int32_t* pos, const float* I_meas, double* loss_history,
                           void* ws, size_t ws_bytes, void* stream);

/* msp_forward for callers that cannot allocate device memory.  The paper has no
 * counterpart; it exists because some callers cannot call cudaMalloc (a host
 * application that owns all device memory through its own pool, or a loop that
 * must not allocate once running, since an allocation can synchronise the device)
 * and so cannot provide the workspace msp_forward takes.  Same arguments and
 * results as msp_forward except:
 *   - no workspace: the scratch (slice transmissions, propagator factor, an error
 *     word) is one 16 MiB file-scope device array that every GPU loading the library
 *     holds until the process exits; L * Ny * Nx may not exceed 2,096,640 (returns
 *     MSP_EUNSUPPORTED, with the reason in msp_last_error_message(), otherwise);
 *   - potentials only (MSP_PARAM_TRANSMISSION returns MSP_EUNSUPPORTED) and the FP32
 *     forward only (other precisions return MSP_EUNSUPPORTED);
 *   - window_error (device int32, may be NULL) is set to 0, or to 1 if a window lay
 *     outside the object (that position's pattern is then zero);
 *   - every call looks the array's device address up (cudaGetSymbolAddress, with the
 *     calling device current), so the address stays right after a device reset and in
 *     a caller's own driver-API context;
 *   - the array is part of the library's device code, which CUDA loads on a device when
 *     it is first used there (lazy module loading): the FIRST call on each device loads
 *     it, which reserves the array and may synchronise that device.  Make one warm-up
 *     call on each device before any loop that must not allocate and before any stream
 *     capture; later calls allocate nothing;
 *   - every call uses the same array: calls that may overlap on the GPU (other
 *     streams, other host threads) race and must be serialised by the caller.
 * Apart from that one-time load, nothing is allocated or freed, by this library or on
 * its behalf. */
msp_status msp_forward_noalloc(const msp_geometry* g, const float* probe, const float* V,
                               const int32_t* pos, float* I_out, int32_t* window_error,
                               void* stream);

/* Synchronises `stream`, then reports (and clears) the workspace flag raised by the
 * most recent compute call on `ws` (every call that can raise it clears it when it
 * starts): MSP_OK; MSP_EINVAL when a scan window lay outside the object; MSP_ETIMEOUT
 * when a bounded wait for the tensor core's pipeline ran out (msp_smd_matrix_step,
 * msp_dft2_tc: the call's results are invalid, the device stays usable); MSP_EDEVICE when,
 * after such a timeout, the kernel's bounded wait for its own issued MMAs also ran out, so
 * tensor memory may have been released under running MMAs.  MSP_EDEVICE marks the current
 * device as untrusted for the rest of the process: every later compute call on it returns
 * MSP_EDEVICE (end the process or reset the device). */
msp_status msp_check_workspace(void* ws, void* stream);

/* Failure-detection hook: the number of polls after which a wait of the tensor-core
 * kernels (msp_smd_matrix_step, msp_dft2_tc, the split-BF16 mode, the convolutions of
 * msp_learn.h) for their own pipeline gives up, for every later call of this process.
 * polls = 0 restores the default, 2^20 polls, well under a second; polls < 0 makes every
 * such wait give up without polling.  A tiny or negative bound makes the waits run out on
 * purpose, which the kernels report through the workspace flag (msp_check_workspace:
 * MSP_ETIMEOUT) after waiting (with their own fixed bound) for the MMAs they issued and
 * freeing their tensor memory, leaving the device usable. */
msp_status msp_set_wait_limit(int32_t polls);

/* How msp_loss_grad forms dV, the sum over scan positions of the window gradients (the sum
 * over s in the gradient of Eq. Opt_Prob_Layerwise), and msp_layer_step (so also
 * msp_reconstruct) its slice's gradient and illumination maps, for every later call of this
 * process:
 *   MSP_OVERLAP_FIXED_ORDER (default): the fused kernel writes each position's windows to the
 *     workspace and a gather adds them per object pixel in ascending scan order: the results
 *     are bit-reproducible.
 *   MSP_OVERLAP_L2_REDUCE: the fused kernel adds each window into the object-frame map as it
 *     is produced, with FP32 reductions performed in L2 (the map is zeroed first); no
 *     per-position buffer is written and no gather runs.  The order of the additions depends
 *     on the schedule, so results agree between runs only to rounding.  Applies to the FP32
 *     mode (MSP_PRECISION_FP32); the other modes keep the fixed order.
 * Returns MSP_EINVAL for any other value. */
enum { MSP_OVERLAP_FIXED_ORDER = 0, MSP_OVERLAP_L2_REDUCE = 1 };
msp_status msp_set_overlap_add(int32_t mode);

/* Profiling hooks, off by default.  While enabled, every launch of the dominant
 * kernel of a call is bracketed by CUDA events recorded on its stream: the fused
 * per-position kernel (the forward / adjoint of all positions) of the calls above,
 * and the two dense complex contractions of msp_smd_matrix_step (msp_smd.h). */
msp_status msp_profile_enable(int32_t on);

/* Waits for the recorded events and returns, since the last reset: the summed
 * duration in ms and the number of dominant-kernel launches timed, and the number of
 * kernels libmsp launched in total (counted whether or not timing is enabled).
 * Any output pointer may be NULL (host pointers); reset != 0 starts a new interval. */
msp_status msp_profile_read(double* fused_ms, int64_t* fused_launches, int64_t* all_launches,
                            int32_t reset);

/* Human-readable status name; never NULL. */
const char* msp_status_string(msp_status s);

/* Detail of this thread's most recent failure ("" if none); never NULL. */
const char* msp_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* MSP_H */
