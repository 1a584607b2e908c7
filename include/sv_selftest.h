/*
 * libsv self-test entry points (not part of the simulation API).  They check
 * the hardware building blocks the simulator's kernels rely on, with inputs
 * the caller supplies, so a test can compare against its own computation.
 */
#ifndef SV_SELFTEST_H_
#define SV_SELFTEST_H_

#ifdef __cplusplus
extern "C" {
#endif

/* One 5th-generation tensor-core product on the current device, the building
 * block of the tensor-core dense apply (fused blocks of 4-5 qubits as dense
 * 2^k x 2^k products, App. D.2 "gate fusion = 5"):
 *   D[m][n] = sum_k A[m][k] * B[n][k],  m < 128, n < 64, k < 64,
 * with A (host, 128 x 64 row-major) held in tensor memory, B (host, 64 x 64
 * row-major, n-th row = K values) placed in shared memory in the no-swizzle
 * K-major core-matrix layout with byte strides kstride (between 4-element K
 * groups) and nstride (between 8-row groups), kind::tf32 inputs, FP32
 * accumulation.  swap_fields = 1 puts the two strides into the descriptor's
 * fields the other way round (for diagnosing the layout).  D (host, 128 x 64)
 * receives the result; *host_status = 0 on success, 1 if the bounded wait for
 * the tensor core gave up.  Returns SV_OK, SV_EINVAL (strides out of range)
 * or SV_ECUDA. */
int sv_selftest_tc_tf32(const float *host_a, const float *host_b, float *host_d, int kstride, int nstride,
                        int swap_fields, int *host_status);

/* The kind::f16 tensor-core product of the register passes' dense op:
 *   D[m][n] = sum_k A[m][k] * B[n][k],  m < 128, n < 64, k < 64,
 * A and B given as IEEE binary16 bit patterns (host, row-major), A held in
 * tensor memory two values per 32-bit column (value 2j in the low half of
 * column j; swap_halves = 1 puts it in the high half, for diagnosing the
 * layout), B in shared memory in the no-swizzle K-major layout (core matrices
 * of 8 rows x 8 values, 128 bytes apart along K, 1024 bytes between 8-row
 * groups), FP32 accumulation.  D (host, 128 x 64 floats) receives the result;
 * *host_status = 0 on success, 1 if the bounded wait gave up.  Returns SV_OK
 * or SV_ECUDA. */
int sv_selftest_tc_f16(const unsigned short *host_a, const unsigned short *host_b, float *host_d,
                       int swap_halves, int *host_status);

/* Failure detection without a GPU fault: a one-CTA kernel waits on an
 * mbarrier that nothing ever arrives at, with the bounded wait of the
 * tensor-core pass (limit try-wait rounds, 1..2^22), then records the expiry
 * in a device status word and returns normally, so the context stays usable.
 * *host_status = 1 when the wait gave up (the expected outcome), 0 if it
 * completed.  Returns SV_OK, SV_EINVAL or SV_ECUDA.  The simulator's own
 * passes report such an expiry as SV_ETIMEOUT from the next call that
 * synchronises. */
int sv_selftest_wait_timeout(unsigned limit, int *host_status);

/* Failure detection in the batch executor's persistent wave kernel
 * (sv_batch_run), without a GPU fault: a wave of one 14-qubit circuit whose
 * first work item is made to wait for more finished items of its circuit
 * than there can be; the wait gives up after limit polls (1..2^22, about 128 ns
 * each), the kernel records it and returns, and the wave reports
 * SV_ETIMEOUT.  *host_status = 1 when the wait gave up (the expected
 * outcome), 0 otherwise.  Returns SV_OK, SV_EINVAL or SV_ECUDA. */
int sv_selftest_wave_timeout(unsigned limit, int *host_status);

/* The cost-model network's loss and gradient on the GPU (the training
 * kernels' forward and backward passes) for flat parameters params
 * (sv_mlp_param_count() floats: W1 64x32 row-major | b1 | W2 64x64 | b2 |
 * w3 | b3), inputs x (B x 32) and standardised targets t (B).  Writes the mean
 * squared error to *loss and the gradient to grads. */
int sv_mlp_gradient(const float *params, const float *x, const float *t, int B, double *loss, float *grads);

/* steps Adam updates (beta1 0.9, beta2 0.999, eps 1e-8, zero initial moments)
 * with the fixed gradient grads, on the GPU; params updated in place. */
int sv_mlp_adam(float *params, const float *grads, int steps, double lr);

/* Number of network parameters (6337). */
int sv_mlp_param_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SV_SELFTEST_H_ */
