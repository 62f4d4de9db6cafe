/*
 * hcran_mlp.h -- C ABI of the warm-start network's tensor-core kernels
 * (sm_103a, tcgen05 BF16 x BF16 -> FP32).
 *
 * The learned warm start maps per-link features to an initial log-power and
 * to the dual multipliers the solver starts from.  Its layers are dense:
 * out[t][p] = epi( sum_q A[t][q] * Bt[p][q] ), on the 5th-generation tensor
 * cores with the accumulators in tensor memory.
 *
 * Conventions: every pointer is a device pointer, 16-byte aligned; matrices
 * are row-major; BF16 values are 16-bit words; Q and P are multiples of 16
 * in [16, 256]; calls are asynchronous on `stream` (NULL: the legacy default
 * stream) and borrow their arguments until the stream reaches them.
 */
#ifndef HCRAN_MLP_H
#define HCRAN_MLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { HCRAN_MLP_OK = 0, HCRAN_MLP_EINVAL = 1, HCRAN_MLP_ECUDA = 3 };

/* Epilogues of hcran_mlp_dense. */
enum {
  HCRAN_MLP_EPI_BIAS_RELU = 0, /* out (BF16) = relu(acc + bias)          layer forward, hidden  */
  HCRAN_MLP_EPI_BIAS_F32 = 1,  /* out (FP32) = acc + bias                layer forward, output  */
  HCRAN_MLP_EPI_RELU_MASK = 2, /* out (BF16) = acc * (H > 0)             input gradient through a ReLU */
  HCRAN_MLP_EPI_F32 = 3        /* out (FP32) = acc                                               */
};

/* One dense layer: A [T][Q] BF16, Bt [P][Q] BF16 (weights as [out][in] for a
 * forward, the transposed weights for an input gradient), bias [P] FP32 or
 * NULL, H [T][P] BF16 (the layer's forward output; only for the RELU_MASK
 * epilogue), out [T][P] BF16 or FP32 by epilogue.  Returns
 * HCRAN_MLP_EINVAL for a bad size, pointer or epilogue, HCRAN_MLP_ECUDA on a
 * launch error.  A tensor-core wait that gives up sets the flag read by
 * hcran_mlp_tc_status. */
int hcran_mlp_dense(const void *A, const void *Bt, const float *bias, const void *H, int64_t T, int32_t Q,
                    int32_t P, int32_t epi, void *out, void *stream);

/* Synchronises the device, then reports (*failed = 1) and clears the flag a
 * bounded tensor-core wait sets when it gives up. */
int hcran_mlp_tc_status(int32_t *failed);

#ifdef __cplusplus
}
#endif

#endif /* HCRAN_MLP_H */
