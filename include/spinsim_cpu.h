/* spinsim_cpu.h -- the same method on the host's cores (multicore CPU backend).
 *
 * The paper's integrator also runs, with the same algorithm, in parallel on a
 * multicore CPU when no GPU is used (Sec. 1.2.6, 1.2.7; device comparison in
 * Sec. 1.3.3).  This library computes every sample operator U_k with the same
 * per-sample arithmetic as the GPU kernels (the shared device-math headers
 * compiled for the host; FP32-bulk or FP64 exactly as configured), spread
 * over host threads, then chains each simulation's operators in order on the
 * host in FP64, writing psi_k, <J>_k and optionally U_k.
 *
 * It is a separate shared library, libspinsim_cpu.so, with this one entry
 * point.  Nothing selects it automatically: the GPU library (spinsim.h) never
 * calls it and fails on its own when no GPU is present.
 *
 * The request, result and configuration types are those of spinsim.h.
 */
#ifndef SPINSIM_CPU_H
#define SPINSIM_CPU_H

#include "spinsim.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Run n requests on the host.
 *
 * cfg:     method, precision, rotating_frame and trotter_squares are used as
 *          in spinsim_create (NULL = CF4, FP32-bulk, frame on, automatic tau);
 *          the GPU-only fields are ignored.
 * reqs:    n requests (host memory, read only), validated as by spinsim_simulate.
 * res:     n results; states (required), spin and ops (optional) must be HOST
 *          buffers of at least K samples (capacity >= K), laid out as in
 *          spinsim_result.  status, flags, n_samples and trotter_squares are
 *          written for every request.
 * threads: worker threads; 0 = every core the process may use.
 *
 * Returns SPINSIM_OK, or the first request's error status (the other valid
 * requests are still computed); SPINSIM_E_ARG for n < 0, a NULL reqs/res with
 * n > 0 or threads < 0; SPINSIM_E_NOMEM when the operator scratch cannot be
 * allocated.  Blocks until every result is written. */
int spinsim_cpu_simulate(const spinsim_config* cfg, const spinsim_request* reqs, spinsim_result* res, int64_t n,
                         int32_t threads);

#ifdef __cplusplus
}
#endif

#endif /* SPINSIM_CPU_H */
