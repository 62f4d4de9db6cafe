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

enum { HCRAN_MLP_OK = 0, HCRAN_MLP_EINVAL = 1, HCRAN_MLP_ENOMEM = 2, HCRAN_MLP_ECUDA = 3 };

/* Network shape: HCRAN_MLP_FEATURES features per link (padded with zeros to
 * HCRAN_MLP_IN columns), three hidden layers of HCRAN_MLP_HIDDEN with ReLU,
 * HCRAN_MLP_OUT output columns of which the first three are used. */
enum {
  HCRAN_MLP_FEATURES = 4,
  HCRAN_MLP_IN = 16,
  HCRAN_MLP_HIDDEN = 256,
  HCRAN_MLP_OUT = 16,
  HCRAN_MLP_LAYERS = 4
};

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

/* ---- the network: FP32 master weights, BF16 copies for the tensor cores ----
 * Layer i maps HCRAN dims[i] -> dims[i+1], dims = {16, 256, 256, 256, 16};
 * out = W4 relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4, weights stored
 * [out][in].  The handle owns its device buffers (allocated on the current
 * device at create); calls on one handle must not overlap. */
typedef struct hcran_mlp_s *hcran_mlp_t;

/* He-initialised network (seeded splitmix64 / Box-Muller; biases 0) with
 * activation buffers for max_rows rows (the largest T of a training step).
 * HCRAN_MLP_EINVAL: NULL out, max_rows < 1 or > 2^28; HCRAN_MLP_ENOMEM. */
int hcran_mlp_create(hcran_mlp_t *out, uint64_t seed, int64_t max_rows);
void hcran_mlp_destroy(hcran_mlp_t h);

/* Parameters (and gradients of the last backward) as one packed FP32 host
 * array [W1 b1 W2 b2 W3 b3 W4 b4]; *n = its length.  Synchronous. */
int hcran_mlp_param_count(hcran_mlp_t h, int64_t *n);
int hcran_mlp_get_params(hcran_mlp_t h, float *host);
int hcran_mlp_set_params(hcran_mlp_t h, const float *host);
int hcran_mlp_get_grads(hcran_mlp_t h, float *host);

/* Forward of x [T][16] BF16 into out [T][16] FP32, in chunks of max_rows rows;
 * the hidden activations of the last chunk stay for hcran_mlp_backward. */
int hcran_mlp_forward(hcran_mlp_t h, const void *x, int64_t T, float *out, void *stream);

/* Masked squared error of the first nout columns, averaged over the T rows:
 * *loss (device) = (1/T) sum mask (out - target)^2, and its gradient with
 * respect to out kept for the backward.  out, target, mask: [T][16] FP32
 * device arrays; T <= max_rows. */
int hcran_mlp_loss_grad(hcran_mlp_t h, const float *out, const float *target, const float *mask, int64_t T,
                        int32_t nout, float *loss, void *stream);

/* Gradients of that loss with respect to every parameter, for the x and T of
 * the last forward (T <= max_rows): every matrix product on the tensor cores
 * (input gradients as dense layers with the transposed weights, weight
 * gradients as sums of outer products over the rows), fixed-order sums. */
int hcran_mlp_backward(hcran_mlp_t h, const void *x, int64_t T, void *stream);

/* One Adam step (bias-corrected) on the FP32 master weights with the last
 * gradients, then the BF16 copies. */
int hcran_mlp_adam(hcran_mlp_t h, float lr, float beta1, float beta2, float eps, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HCRAN_MLP_H */
