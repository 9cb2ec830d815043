/*
 * coll_debug.h -- inspection and failure-injection entry points of libcoll.so.
 *
 * coll_plan_tables_host builds, on the host and without touching any GPU, the
 * multiplier tables a plan would upload (sec. 4.4.1, separated kernel
 * beta_F ~ sum_t alpha_t alpha'_t): n_terms * N * N * (N/2) pairs
 * (A_t, B_t) = (c_t alpha_t / (s_t N^3), s_t alpha'_t / N^3), the last term
 * being the loss (-Lambda / (s N^3), s / N^3), where s_t is a power of two
 * that balances the two factors (A_t B_t does not depend on it); layout
 * [t][k0][k1][k2 < N/2][2], k0 and k1 in FFT order.  out may be NULL to query *n_terms and *n_doubles only.
 * Returns COLL_EINVAL / COLL_EUNSUPPORTED like coll_plan_create, and
 * COLL_ENOMEM if cap (in doubles) is too small.
 */
#ifndef COLL_DEBUG_H
#define COLL_DEBUG_H

#include "coll.h"

#ifdef __cplusplus
extern "C" {
#endif

coll_status coll_plan_tables_host(const coll_plan_desc* desc, double* out, size_t cap, int32_t* n_terms,
                                  size_t* n_doubles);

/*
 * coll_m2d_tables_host -- the table a 2D Maxwell plan would upload, built on
 * the host without a GPU: (A + 1) * N * (N/2) pairs (A_t, B_t), layout
 * [t][k0][k1 < N/2][2], k0 in FFT order, the loss pair last (see
 * coll_m2d_plan_create).  out may be NULL to query the sizes; COLL_ENOMEM if
 * cap (in doubles) is too small; COLL_EINVAL / COLL_EUNSUPPORTED like
 * coll_m2d_plan_create.
 */
coll_status coll_m2d_tables_host(const coll_m2d_plan_desc* desc, double* out, size_t cap, int32_t* n_terms,
                                 size_t* n_doubles);

/*
 * coll_debug_mixed_drop_commit -- failure injection for the bounded waits of
 * the tensor-core path (COLL_MIXED_F16X2).  With on != 0, in every later
 * launch warpgroup 0 of each CTA omits the completion signal of its first MMA
 * batch: its wait expires after about one second of SM clocks, the CTA stops,
 * waits (bounded) on a fresh completion signal for the MMAs it started, frees
 * its tensor memory and returns, and the plan's sticky status reads
 * COLL_ETIMEOUT (coll_device_status).  Nothing faults or hangs; the launch
 * takes about one second.  on = 0 restores normal
 * operation.  Applies to the current device.  Returns COLL_ECUDA if the switch
 * cannot be written.
 */
coll_status coll_debug_mixed_drop_commit(int32_t on);

#ifdef __cplusplus
}
#endif

#endif /* COLL_DEBUG_H */
