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

#ifdef __cplusplus
}
#endif

#endif /* RFLBM_TESTING_H */
