/*
 * fks_testing.h -- test hooks of the FKS library (not for production use).
 *
 * fks_test_hold_first_partition(on): while `on` is non-zero, builds started
 * on the calling thread make their first level-one partition withhold its
 * slot prefix from the cross-partition scan, so that the next partition's
 * bounded wait runs out and the build returns FKS_ERR_TIMEOUT.  This
 * exercises the device-side timeout path without faulting or hanging the
 * GPU (every device wait in the library is bounded by
 * fks_build_opts.spin_limit polls).  The paper has no counterpart; it is a
 * failure-injection hook of this library.
 *
 * fks_test_fail_serve_launches(n): the next n lookup batches that a batched
 * server (FKS_SERVE_BATCHED) would launch are not launched; each reports
 * the launch error a failed kernel launch returns (cudaErrorLaunchFailure),
 * so that every request of those batches completes with FKS_ERR_CUDA while
 * the CUDA context stays usable.  A host-side fake of the failing call: no
 * kernel faults.  n = 0 clears it.  Process-wide.
 */
#ifndef FKS_TESTING_H_
#define FKS_TESTING_H_
#ifdef __cplusplus
extern "C" {
#endif

void fks_test_hold_first_partition(int on);
void fks_test_fail_serve_launches(int n);

#ifdef __cplusplus
}
#endif
#endif /* FKS_TESTING_H_ */
