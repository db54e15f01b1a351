/*
 * libturtle failure injection, for tests of the error paths (no counterpart in the paper).
 *
 * Every injection acts on the host side of the library or on launch arguments; none makes a
 * device fault, trap or wait without bound. An armed injection fires once, on the first call
 * that reaches its point, and is then disarmed. Injections are process-wide; arm them only while
 * no other thread is inside the library.
 */
#ifndef TURTLE_TESTING_H
#define TURTLE_TESTING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TURTLE_INJECT_NONE 0        /* disarm every injection */
#define TURTLE_INJECT_DEVICE_ALLOC 1 /* value n: the (n+1)-th device scratch allocation from now fails as if the
                                        device were out of memory; the call returns TURTLE_E_NOMEM and frees
                                        what it had allocated */
#define TURTLE_INJECT_HOST_ALLOC 2   /* value n: the (n+1)-th host result allocation from now fails
                                        (TURTLE_E_NOMEM) */
#define TURTLE_INJECT_LOOKBACK 3     /* value n (> 0): the next merge of the lazy form (compact = 3) hands its
                                        tiles tickets from 1, so tile 0 never runs and the look-back waits of
                                        the others run out after n rounds; the kernel sets its error word and
                                        returns, and the call returns TURTLE_E_DEVICE */
#define TURTLE_INJECT_CAND_CAP 4     /* value n: pass 1 of the next call may emit at most n candidates (the
                                        buffer keeps its full size); more set the overflow bit and the call
                                        returns TURTLE_E_CAPACITY */

/* Arm injection `what` with `value` (TURTLE_INJECT_NONE: disarm all). TURTLE_E_ARG for an unknown kind. */
int turtle_test_inject(int what, uint64_t value);

#ifdef __cplusplus
}
#endif
#endif /* TURTLE_TESTING_H */
