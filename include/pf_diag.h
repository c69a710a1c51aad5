/*
 * pf_diag.h -- diagnostic entry points of libpf.so for failure-detection
 * tests.  They are not part of the particle-learning method: the paper has
 * no counterpart.  They exercise the library's failure handling without
 * faulting or hanging a GPU, by making one of its bounded device waits run
 * out on purpose.
 */
#ifndef PF_DIAG_H
#define PF_DIAG_H

#include <stddef.h>
#include <stdint.h>

#include "pf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* pf_cdf (the exact fixed-point CDF of float weights, a single-pass scan with
 * decoupled look-back over 4096-element tiles) with test settings of the
 * look-back's bounded wait.  The tile that takes ticket `withhold_tile`
 * publishes neither its aggregate nor its prefix, so the next tile polls its
 * status word until `spin_limit` polls have passed, gives up and raises the
 * timeout bit of the error word; the call then returns PF_ERR_TIMEOUT and
 * Q_dev holds no valid CDF.  withhold_tile = 0xffffffff withholds nothing
 * (the call is then pf_cdf with a wait of spin_limit polls; pf_cdf itself
 * waits up to 2^22 polls).  Every wait is bounded, so the call always
 * returns, and nothing persists between calls: a later pf_cdf on the same
 * stream works normally.  Arguments otherwise as pf_cdf (device pointers,
 * n in [1, 2^26], spin_limit >= 1); synchronises `stream`. */
pf_status pf_diag_cdf_wait(const float* w_dev, uint64_t n, uint32_t withhold_tile,
                           uint32_t spin_limit, uint64_t* Q_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PF_DIAG_H */
