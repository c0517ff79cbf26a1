/*
 * msp_dft.h -- batched 2-D DFT as dense contractions on the tensor cores: the
 * "DFT as a matrix product" route that the paper names for faster multislice forward
 * passes (Sec. 6), built as a study next to the FFT of the fused multislice kernels.
 *
 * Y_s = F X_s F for S complex W x W images X_s (row-major, interleaved (re, im) floats),
 * F[k][x] = exp(-2 pi i k x / W) (inverse != 0: the conjugate kernel, unnormalised, so the
 * inverse transform is F^H Y F^H / W^2 after scaling by the caller).  Each of the two passes
 * is one contraction F (W x W) times all images' rows (W x S W) on the tensor cores
 * (tcgen05 kind::tf32, every operand split into a tf32 pair, FP32 accumulation over groups
 * of 128 K), whose epilogue stores every image transposed, so the second pass transforms
 * the columns and the result comes back in row-major order.
 *
 * Supported: W in {32, 64, 128, 256}, 1 <= S and S W <= 8,388,480 (65535 column tiles
 * of 128).  Device pointers, 16-byte aligned, in and out may alias; the caller's
 * workspace (256-byte aligned, msp_dft2_tc_workspace_bytes) holds F and the
 * intermediate.  Asynchronous on `stream`;
 * a tensor-core wait that runs out raises the workspace flag (msp_check_workspace:
 * MSP_ETIMEOUT).
 */
#ifndef MSP_DFT_H
#define MSP_DFT_H

#include <stddef.h>
#include <stdint.h>

#include "msp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Workspace bytes for msp_dft2_tc(W, S); 0 if (W, S) is not supported. */
size_t msp_dft2_tc_workspace_bytes(int32_t W, int32_t S);

/* out[s] = F in[s] F (inverse: conj(F) in[s] conj(F)), s < S.  MSP_EINVAL / MSP_EUNSUPPORTED
 * for bad arguments (checked on the host), MSP_ECUDA for a failed launch. */
msp_status msp_dft2_tc(int32_t W, int32_t S, int32_t inverse, const float* in, float* out, void* ws,
                       size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MSP_DFT_H */
