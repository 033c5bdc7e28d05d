/*
 * sho_fault.h -- fault injection for tests of libsho's failure detection (part of libsho.so).
 *
 * The paper has no counterpart: these calls exist so that the library's bounded waits and the serving
 * loop's handling of stuck and failed requests can be exercised without faulting, trapping or hanging
 * a GPU.  Every injected failure ends by itself: device waits keep an iteration bound and return an
 * error status, held requests finish once released.  Production code leaves these at their defaults.
 */
#ifndef SHO_FAULT_H
#define SHO_FAULT_H

#include "sho.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Limit, in SM clock cycles, of every bounded wait the handle's kernels make on their own data pipeline
 * (the plane-sweep projection's mbarrier waits on its TMA row ring; the tensor-core expansions' waits on
 * their bulk-copy staging and MMA commits).  0 restores the default of about
 * 2 s (4e9 cycles); a negative value returns SHO_ERR_ARG.  When a wait runs out the kernel records
 * SHO_ERR_TIMEOUT in the handle's status word, leaves its loop (its results are incomplete) and
 * returns; sho_sync then reports SHO_ERR_TIMEOUT. */
int sho_fault_wait_limit(sho_handle* handle, long long cycles);

/* Make the plane-sweep projection's producer warps issue only the first `rows` rows of each sweep, and
 * the FP64-accurate tensor-core expansion stage the z-pass slices of only the first `rows` atoms of each
 * tile (a pipeline stage that never arrives), so that the consumers' bounded waits run out.  Each kernel
 * still waits for the copies it did issue before it returns, so nothing is in flight when its block
 * exits.  A negative value restores normal operation. */
int sho_fault_stop_rows(sho_handle* handle, int rows);

/* Make the device checks (sho_set_device_checks) take psi's extent as at most `psi_elems` elements, so
 * that indices at and above it count as out of bounds while every access stays inside the real buffer
 * (the checked access is skipped).  A negative value restores the real extent. */
int sho_fault_check_extent(sho_handle* handle, long long psi_elems);

/* Apply sho_fault_wait_limit(cycles) and sho_fault_stop_rows(rows) to every execution slot of a server
 * (its requests' kernels), so that served requests meet the same injected pipeline failure. */
int sho_fault_server_pipeline(sho_server* server, long long cycles, int rows);

/* Hold (hold != 0) or release the requests of one system in a server: while held, a running request
 * of that system is not retired even after its GPU work completed -- a stuck request as the scheduler
 * sees it.  Other systems' requests keep running; sho_wait on the held ticket runs into its timeout;
 * queued requests of the same system stay queued (they may be cancelled).  Release retires it.
 * Returns SHO_ERR_STATE for an unknown system. */
int sho_fault_hold(sho_server* server, int system_id, int hold);

#ifdef __cplusplus
}
#endif

#endif /* SHO_FAULT_H */
