/* Testing hooks of the rflbm library (not for production use).
 *
 * They let a test drive the library's failure paths on a GPU without faulting it: every
 * wait inside a kernel is bounded (in polls and in time, about one second), after which
 * the kernel sets the handle's error flag, lets its copies in flight land and exits, and
 * the next synchronising call reports RFLBM_ETIMEOUT. The paper has no counterpart.
 */
#ifndef RFLBM_TESTING_H
#define RFLBM_TESTING_H

#include <stdint.h>

#include "rflbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Every later step launch of h on the TMA path (either streaming pattern, one-site and
 * two-site forms) expects `bytes` more
 * bytes on its copy barrier than its copies deliver, so that barrier never completes and
 * each CTA's bounded wait runs out (about one second per wait). 0 restores normal
 * operation. bytes <= 2^20, else RFLBM_EINVAL. The state after such a step is undefined;
 * re-initialise it. */
int rflbm_testing_expect_extra_bytes(rflbm_t* h, uint32_t bytes);

/* rflbm_slab_exchange moves a face as one 3-D copy only while its plane pitch is at most
 * `bytes` (and the device's maximum copy pitch); above it, one copy per plane row. The limit
 * is process-wide; 0 restores the default (the device's maximum). bytes < 0: RFLBM_EINVAL. */
int rflbm_testing_slab_copy_pitch_limit(int64_t bytes);

/* Measurement of a design choice, not a production path: the back transform of Eq. 11,
 * f_i = w_i sum_k e_ki m_k / b_k (Table II modes, scaled moments M_k = m_k / b_k as input),
 * on its own, computed either as the step kernels compute it (method 0: sum-factorised
 * float32 FMAs, one thread per site) or on the tensor cores (method 1: one tcgen05 MMA tile of
 * 128 sites x 32 populations x 32 modes per CTA, split-bfloat16 moments, float32 accumulator
 * in tensor memory; about 16 significant bits of M survive the split).
 * rflbm_testing_backtransform: m holds 27 planes of n scaled moments (host memory, element
 *   [k n + s], k = 9 p + 3 q + r for the exponents (p, q, r) of the mode), f receives 27
 *   planes of n populations (host, element [i n + s], i = 9 (c_x + 1) + 3 (c_y + 1) + c_z + 1).
 *   n must be a positive multiple of 128. Synchronous; allocates device memory.
 * rflbm_testing_backtransform_time: *ms receives the time of one launch over `tiles` tiles of
 *   128 sites, each site transforming `reps` sets of synthetic moments held in registers
 *   (one untimed launch first). Synchronous; allocates device memory.
 * A bounded wait for the MMA that expires returns RFLBM_ETIMEOUT. */
int rflbm_testing_backtransform(int method, const float* m, int64_t n, float* f);
int rflbm_testing_backtransform_time(int method, int64_t tiles, int reps, float* ms);

/* Measurement of a design choice, not a production path: the forward projection of Eq. 5 for
 * the moments the step uses (order <= 2), on its own, as the ten raw moments
 * m_k = sum_i f_i c_x^p c_y^q c_z^r in the order 1, c_x, c_y, c_z, c_x^2, c_y^2, c_z^2, c_x c_y,
 * c_x c_z, c_y c_z, computed either as the step kernels compute them (method 0: sum-factorised
 * float32 FMAs) or on the tensor cores (method 1: one tcgen05 MMA tile of 128 sites x 16 moments
 * x 32 populations per CTA with float16 operands, float32 accumulator in tensor memory: exact
 * for populations that are float16 values, as 16-bit storage gives them).
 * rflbm_testing_forward: f holds 27 planes of n populations (host, element [i n + s],
 *   i = 9 (c_x + 1) + 3 (c_y + 1) + c_z + 1; method 1 rounds them to float16), m receives 10
 *   planes of n moments (host). n must be a positive multiple of 128. Synchronous; allocates
 *   device memory.
 * rflbm_testing_forward_time: *ms receives the time of one launch over `tiles` tiles of 128
 *   sites, each site projecting `reps` sets of synthetic float16 populations held in registers
 *   (one untimed launch first). Synchronous; allocates device memory.
 * A bounded wait for the MMA that expires returns RFLBM_ETIMEOUT. */
int rflbm_testing_forward(int method, const float* f, int64_t n, float* m);
int rflbm_testing_forward_time(int method, int64_t tiles, int reps, float* ms);

/* Measurement of the noise draw of a step alone (the r_k of Eq. 9 by the generator stated in
 * rflbm.h: 6 Philox4x32-10 calls and 12 Box-Muller pairs per site), two sites per thread as in
 * the 16-bit step kernels, with nothing else done: *ms receives the time of one launch over
 * nsites sites (2 <= nsites < 2^31; one untimed launch first). Synchronous. */
int rflbm_testing_noise_time(int64_t nsites, float* ms);

#ifdef __cplusplus
}
#endif

#endif /* RFLBM_TESTING_H */
