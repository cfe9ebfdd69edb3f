/*
 * galnb_testing.h -- test hooks of libgalnb.so, kept out of the public
 * interface in galnb.h.  They exercise failure paths that normal inputs never
 * reach; an application has no use for them.
 */
#ifndef GALNB_TESTING_H
#define GALNB_TESTING_H

#include "galnb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Failure path of the tensor-core convolutions (no counterpart in the
 * paper): runs one forward pass on zeros in which the first convolution's
 * halo barriers expect 16 bytes more than its TMA loads deliver, so none of
 * its halo waits can complete.  Each bounded wait (1 s) runs out, the kernel
 * drains its copies and MMAs, frees TMEM and exits, and the call returns
 * GNB_ETIMEOUT; the network and the CUDA context stay usable.  Takes a few
 * seconds.  Errors: GNB_EINVAL (NULL, or the mma.sync path selected). */
int gnb_unet_test_wait_timeout(gnb_unet *net);

#ifdef __cplusplus
}
#endif

#endif /* GALNB_TESTING_H */
