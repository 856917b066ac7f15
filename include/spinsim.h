/*
 * spinsim.h -- C ABI of the GB300-native spin-half / spin-one CF4 integrator.
 *
 * The library integrates the time-dependent Schroedinger equation
 * i dpsi/dt = H(t) psi (hbar = 1) for spin-half (N = 2) and spin-one (N = 3)
 * systems, H(t) = w_x J_x + w_y J_y + w_z J_z (+ w_q Q for spin-one), as in
 * Tritt et al., arXiv 2204.05586:
 *   - each output interval [t_{k-1}, t_k] gets its own time-evolution operator
 *     U_k built from L integration steps of the commutator-free fourth-order
 *     Magnus method CF4 (Sec. 1.2.2, Eqs. cf4_sample_1/2, cf4_implementation),
 *   - spin-half exponentials in closed SU(2) form, spin-one exponentials by
 *     Lie-Trotter with 2^tau residual squarings (Sec. 1.2.3, Eq. lie_trotter_4),
 *   - optionally inside a per-interval rotating frame (Sec. 1.2.5,
 *     Eq. exit_rotating_frame),
 *   - the U_k are chained psi_k = U_k psi_{k-1} (Sec. 1.2.4,
 *     Eq. integration_compilation) by a parallel ordered prefix product in FP64,
 *     and psi_k plus <J_x, J_y, J_z>_k (Sec. 1.2.1) are written for every k.
 *
 * Conventions used throughout:
 *   - basis order m = +j ... -j; J = sigma/2 for spin-half; Q = diag(1,-2,1)/3.
 *   - complex numbers are stored as interleaved (re, im) doubles.
 *   - K = (t_end - t_start)/dt_out output samples, sample k at
 *     t_k = t_start + k dt_out, psi_0 = psi0 (the initial state), no sample at
 *     t_end; L = dt_out/dt integration steps per sample, delta_t = dt_out / L.
 *   - U_0 is defined as the identity.
 *
 * Threading: a handle may be used by one host thread at a time.  All work is
 * enqueued on the CUDA stream passed in (NULL = the legacy default stream);
 * results and the per-request status are final once that stream is
 * synchronised.  No call aborts or exits the process; errors are returned.
 */
#ifndef SPINSIM_H
#define SPINSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPINSIM_ABI_VERSION 2
#define SPINSIM_MAX_PULSES 4
#define SPINSIM_MAX_TONES 3

/* Status codes (negative = error).  A call returns the first error it meets;
 * spinsim_result.status carries each request's own status. */
typedef enum {
    SPINSIM_OK = 0,
    SPINSIM_PENDING = 1,          /* spinsim_poll: the request has not finished yet          */
    SPINSIM_E_ARG = -1,           /* NULL pointer, unknown enum value, non-positive step...  */
    SPINSIM_E_STEP_RATIO = -2,    /* (t_end-t_start)/dt_out or dt_out/dt not an integer (1e-9) */
    SPINSIM_E_NORM = -3,          /* | ||psi0|| - 1 | > 1e-10 (the state must be normalised)  */
    SPINSIM_E_NOMEM = -4,         /* scratch over the handle's budget, or cudaMalloc failed   */
    SPINSIM_E_CUDA = -5,          /* a CUDA runtime call or kernel launch failed              */
    SPINSIM_E_TIMEOUT = -6,       /* spinsim_poll: waited wait_us without completion          */
    SPINSIM_E_CAPACITY = -7,      /* result capacity smaller than the request's K             */
    SPINSIM_E_UNSUPPORTED = -8    /* valid but not provided (graphs while capturing, su(3) FP32) */
} spinsim_status;

/* spinsim_result.flags bits (warnings; the request still ran). */
#define SPINSIM_WARN_MAGNUS 1     /* an upper bound of ||H||_2 delta_t reaches the Magnus
                                     convergence radius xi = 1.0868687 (Sec. 1.2.2)       */
#define SPINSIM_WARN_FP32_LAB 2   /* FP32-bulk with the rotating frame off and a z field: each
                                     sample then turns by w_z dt_out and the FP32 rounding of
                                     that rotation, alike in every sample, adds up over the
                                     run; the 1e-5 FP32-bulk accuracy is held only in the
                                     rotating frame (Sec. 1.2.5)                          */

typedef enum {
    SPINSIM_METHOD_CF4 = 0,       /* Sec. 1.2.2 (default)                                    */
    SPINSIM_METHOD_MIDPOINT = 1,  /* midpoint Euler sampling, Sec. 1.3.1                     */
    SPINSIM_METHOD_HEUN = 2       /* Heun-Euler sampling, Sec. 1.3.1                         */
} spinsim_method;

typedef enum {
    SPINSIM_PREC_FP64 = 0,        /* every step in FP64                                      */
    SPINSIM_PREC_FP32_BULK = 1    /* field, exponentials and step products in FP32; first
                                     order, frame exit and chain in FP64; U_k stored as
                                     computed (not re-unitarised), every written psi_k
                                     renormalised in FP64                                  */
} spinsim_precision;

/* Handle configuration.  Zero-initialise, or call spinsim_config_default. */
typedef struct {
    int32_t method;               /* spinsim_method                                          */
    int32_t precision;            /* spinsim_precision                                       */
    int32_t rotating_frame;       /* 1: per-interval rotating frame (default), 0: lab frame  */
    int32_t trotter_squares;      /* tau, n = 2^tau Lie-Trotter factors (spin-one), 0..40;
                                     -1 = default: 24 for FP64 (Sec. 1.2.3); for FP32-bulk,
                                     per request the fewest squarings whose splitting-error
                                     bound, summed over all steps of the request, is <= 1e-6 */
    int32_t lanes_per_sample;     /* 0 = default (1); else 1, 2, 4 or 8 threads share one U_k
                                     in the whole waves of a launch (the samples after the
                                     last whole wave use one lane per segment of a sample).
                                     Results do not depend on it (fixed reduction tree).   */
    int32_t threads_per_block;    /* 0 = autotune; else 64, 128 or 256                        */
    int32_t use_graphs;           /* 1: replay repeated identical batch shapes as a CUDA graph
                                     on the caller's stream (the first call of a shape runs
                                     eagerly and captures it); calls stay in issue order.
                                     A call that repeats the previous one byte for byte
                                     (requests and result buffers) replays the graph without
                                     validating and refilling the parameter tables again  */
    int32_t device;               /* CUDA device ordinal                                      */
    int64_t mem_budget;           /* bytes of device memory the handle may hold in total
                                     (its arena for spinsim_simulate and ranges plus its
                                     serving pool); 0 = 90% of the free memory at
                                     spinsim_create                                        */
    int32_t profile;              /* 1: time the integrate and chain kernels of each call
                                     with CUDA events (read by spinsim_last_launch)         */
    int32_t blocks_per_sm;        /* 0 = autotune; else resident integrate blocks per SM
                                     (1..32, capped at what the kernel's registers allow).
                                     Results do not depend on it.                          */
    int32_t chain_precision;      /* 0 = FP64 (default): the cross-sample product and the
                                     state propagation in double precision; 1 = FP32: the
                                     same kernels with every product rounded to single
                                     precision, a control for precision studies (it shows
                                     why the product stays FP64); ignored by the CPU backend */
    int32_t direct_host_outputs;  /* 0: host-resident result buffers are staged in
                                     device memory and copied back after the kernels; 1: the
                                     kernels write them directly when they are pinned host
                                     memory the device can address (cudaHostAlloc /
                                     cudaHostRegister, mapped), so the output crosses the
                                     host link while the chain runs and no copy follows
                                     (the default of spinsim_config_default).  Other host
                                     memory is staged either way.                          */
} spinsim_config;

/* The fixed parameterised field family (Hz, seconds, radians):
 *   w_x(t) = 2 pi drive_x_hz cos(2 pi drive_hz t + drive_phase)
 *            + sum_j 2 pi tone_x_hz[j] cos(2 pi tone_hz[j] t + tone_phase[j])
 *   w_y(t) = 2 pi drive_y_hz sin(2 pi drive_hz t + drive_phase)
 *            + sum_j 2 pi tone_y_hz[j] sin(2 pi tone_hz[j] t + tone_phase[j])
 *   w_z(t) = 2 pi (bias_hz + sum_p pulse_amp_hz[p] shape_p(t))
 *   w_q(t) = 2 pi quad_hz                       (spin-one only; ignored for spin-half)
 * with, for pulse p (c = pulse_centre_s[p], w = pulse_width_s[p] > 0):
 *   Gaussian (bit p of pulse_sine_mask clear): shape_p(t) = exp(-(t - c)^2 / (2 w^2));
 *   single sine cycle (bit p set; the "sinp" signal pulse of the paper's benchmark
 *   field, Eq. neural_pulse): shape_p(t) = sin(2 pi (t - c) / w) for c <= t < c + w,
 *   else 0 (c is the start of the cycle, w its period).
 * A linearly polarised drive "2 R cos(2 pi f t)" is drive_x_hz = 2R, drive_y_hz = 0;
 * a circularly polarised one has drive_x_hz = drive_y_hz.  The detuning of the
 * drive is drive_hz - bias_hz.  Tones j < n_tones are further drive terms of the
 * same form (a multi-tone drive of any polarisations, Sec. 3.1); requests with
 * tones run on a kernel variant that evaluates them, the others are unaffected.
 *
 * Full su(3) spin-one Hamiltonians (Sec. 1.2.1): with qd_on = 1 two quadrupole
 * drives of the same form act on the symmetric products of the spin matrices
 * D_xz = J_x J_z + J_z J_x, D_yz = J_y J_z + J_z J_y (pair 0) and
 * D_x2y2 = J_x^2 - J_y^2, D_xy = J_x J_y + J_y J_x (pair 1):
 *   w_xz = 2 pi qd_x_hz[0] cos(ph_0), w_yz = 2 pi qd_y_hz[0] sin(ph_0),
 *   w_x2y2 = 2 pi qd_x_hz[1] cos(ph_1), w_xy = 2 pi qd_y_hz[1] sin(ph_1),
 *   ph_p = 2 pi qd_hz[p] t + qd_phase[p];
 * with J_x, J_y, J_z and Q they span su(3).  Spin-one and SPINSIM_PREC_FP64
 * only (SPINSIM_E_ARG for spin-half, SPINSIM_E_UNSUPPORTED in FP32-bulk). */
typedef struct {
    double bias_hz;
    double drive_x_hz;
    double drive_y_hz;
    double drive_hz;
    double drive_phase;
    double quad_hz;
    int32_t n_pulses;             /* 0..SPINSIM_MAX_PULSES                                   */
    int32_t pulse_sine_mask;      /* bit p: pulse p is a single sine cycle, else a Gaussian  */
    double pulse_amp_hz[SPINSIM_MAX_PULSES];
    double pulse_centre_s[SPINSIM_MAX_PULSES];
    double pulse_width_s[SPINSIM_MAX_PULSES];   /* standard deviation, > 0 when used       */
    int32_t n_tones;              /* 0..SPINSIM_MAX_TONES further drive tones                */
    int32_t reserved;             /* ignored                                                 */
    double tone_x_hz[SPINSIM_MAX_TONES];
    double tone_y_hz[SPINSIM_MAX_TONES];
    double tone_hz[SPINSIM_MAX_TONES];
    double tone_phase[SPINSIM_MAX_TONES];
    int32_t qd_on;                /* 1: the two quadrupole drives below are on (spin-one)     */
    int32_t reserved2;            /* ignored                                                 */
    double qd_x_hz[2];
    double qd_y_hz[2];
    double qd_hz[2];
    double qd_phase[2];
} spinsim_field;

/* One simulation (Sec. 1.2.4 problem statement). */
typedef struct {
    int32_t spin_x2;              /* 1 = spin-half (N = 2), 2 = spin-one (N = 3)             */
    int32_t reserved;
    spinsim_field field;
    double t_start, t_end;        /* seconds, t_end >= t_start                               */
    double dt;                    /* integration step delta_t (> 0)                          */
    double dt_out;                /* output step Delta_t (> 0), an integer multiple of dt    */
    double psi0[6];               /* initial state, N complex (re, im), normalised           */
} spinsim_request;

/* Caller-owned output buffers of one request.  Each pointer may be device
 * memory (written in place) or host memory (the library stages it through
 * device scratch and copies back on the stream; with direct_host_outputs,
 * pinned mapped host memory is written in place).  The library never frees
 * them. */
typedef struct {
    double* states;               /* [capacity][N] complex psi_k, required                   */
    double* spin;                 /* [capacity][3] <J_x>, <J_y>, <J_z>; NULL = not written   */
    double* ops;                  /* [capacity][N][N] complex U_k (row-major); NULL = not written */
    int64_t capacity;             /* samples the buffers can hold (>= K)                     */
    int64_t n_samples;            /* out: K                                                  */
    int32_t status;               /* out: this request's spinsim_status                      */
    int32_t flags;                /* out: SPINSIM_WARN_* bits                                */
    int32_t trotter_squares;      /* out: tau used for this request (0 for spin-half)        */
    int32_t reserved;             /* set to 0                                                */
} spinsim_result;

typedef struct spinsim_s* spinsim_handle;

/* Fill *cfg with defaults: CF4, FP32-bulk, rotating frame on, default tau,
 * autotuned launch shape, graphs off, device 0, budget 0 (90% of free),
 * FP64 chain, pinned host outputs written directly (direct_host_outputs = 1). */
int spinsim_config_default(spinsim_config* cfg);

/* Create a handle on cfg->device.  The handle owns device scratch (operator
 * buffer, chain aggregates, parameter tables), pinned staging memory, the
 * autotuner's cache and the serving queue.  Returns SPINSIM_E_ARG for a bad
 * configuration, SPINSIM_E_CUDA when the device cannot be used.
 *
 * Fault injection for testing failure handling without a GPU fault: when the
 * environment variable SPINSIM_FAIL_ALLOC (SPINSIM_FAIL_LAUNCH) holds a
 * positive integer n at spinsim_create, the handle's n-th device allocation
 * (n-th kernel launch of a batch, counting the integrate and chain launches)
 * is not made and reports failure as cudaMalloc (a launch) would:
 * SPINSIM_E_NOMEM (SPINSIM_E_CUDA) for the batch and its requests.  Later
 * calls on the handle run normally. */
int spinsim_create(const spinsim_config* cfg, spinsim_handle* out);

/* Release everything the handle owns (after synchronising its work). */
void spinsim_destroy(spinsim_handle h);

/* K and L of a request, with the same validation spinsim_simulate applies. */
int spinsim_counts(const spinsim_request* req, int64_t* K, int64_t* L);

/* Bytes of device scratch spinsim_simulate needs for these n requests with
 * device-resident outputs (host-resident or unaligned outputs add their own
 * size, staged); -SPINSIM_E_* on invalid input.  A batch whose footprint
 * exceeds the handle's mem_budget gets SPINSIM_E_NOMEM from spinsim_simulate,
 * and a single request whose footprint exceeds it gets SPINSIM_E_NOMEM from
 * spinsim_submit. */
int64_t spinsim_footprint(spinsim_handle h, const spinsim_request* reqs, int64_t n);

/* Simulate n independent requests as one batch on `stream` (a cudaStream_t).
 * Every request is validated first; requests that fail validation get their
 * status set and are skipped, the others run.  Returns SPINSIM_OK when every
 * request is valid and all launches were enqueued, else the first error.
 * res[i].states/spin/ops receive psi_k, <J>_k and U_k for k = 0..K-1.  The
 * batch runs as one launch per spin and kernel variant, so each request's
 * results are bit-identical to running it alone, whatever it is batched with. */
int spinsim_simulate(spinsim_handle h, const spinsim_request* reqs, spinsim_result* res, int64_t n,
                     void* stream);

/* Continuous-batching serving interface (Sec. 1.2.7's "many simulations from
 * one compiled simulator", served as they arrive).  spinsim_submit copies the
 * request and queues it; pending requests are launched in arrival order as
 * one batch on a free internal stream (four) while earlier batches are still
 * running.  A batch's device scratch is a piece of one serving pool: the
 * queue's head waits until a stream is free and its scratch fits in the
 * pool's free memory.  The pool grows only while no served batch is in
 * flight (so no allocation stalls work on the device), and the pool plus the
 * handle's arena never exceed mem_budget (spinsim_memory).  A request whose
 * own footprint (spinsim_footprint, plus staging of host outputs) exceeds
 * mem_budget is refused with SPINSIM_E_NOMEM and completes at once.  The
 * result buffers must stay valid until spinsim_poll or spinsim_poll_any
 * reports completion.  *ticket identifies the request. */
int spinsim_submit(spinsim_handle h, const spinsim_request* req, spinsim_result* res, int64_t* ticket);

/* Drive the serving queue and report a ticket: SPINSIM_OK when its results
 * are complete (res->status holds the request status), SPINSIM_PENDING when
 * not yet (wait_us = 0), SPINSIM_E_TIMEOUT when wait_us > 0 elapsed first, or
 * SPINSIM_E_ARG for an unknown ticket.  Completed tickets are forgotten. */
int spinsim_poll(spinsim_handle h, int64_t ticket, int32_t wait_us);

/* Drive the serving queue and report completed tickets in order of
 * completion: up to `capacity` of them are written to tickets[] (and
 * forgotten), *n_done receives their number.  Returns SPINSIM_OK when at
 * least one was written (or capacity = 0), SPINSIM_PENDING when none had
 * completed (wait_us = 0), SPINSIM_E_TIMEOUT when wait_us > 0 elapsed first.
 * Tickets already reported by spinsim_poll are not reported again. */
int spinsim_poll_any(spinsim_handle h, int64_t* tickets, int64_t capacity, int32_t wait_us, int64_t* n_done);

/* Device memory of a handle (bytes), read on the host without waiting. */
typedef struct {
    int64_t budget;               /* mem_budget in effect                                    */
    int64_t held;                 /* arena + serving pool now held                           */
    int64_t peak_held;            /* the most held at any time since spinsim_create          */
    int64_t arena;                /* main arena (spinsim_simulate, ranges)                   */
    int64_t pool;                 /* serving pool                                            */
    int64_t pool_in_use;          /* pool bytes carved for served batches in flight          */
    int64_t pending;              /* submitted requests waiting for a stream or memory       */
    int64_t in_flight;            /* submitted requests in batches on the device             */
} spinsim_memory_info;
int spinsim_memory(spinsim_handle h, spinsim_memory_info* info);

/* Launch shape the last spinsim_simulate call used for its integration
 * kernel, how many kernels it launched, the bytes it copied between host and
 * device, and (with cfg.profile = 1, not for graph replays) the device time
 * of its integrate and chain kernels.  Reading the times waits for them. */
typedef struct {
    int32_t lanes_per_sample;
    int32_t threads_per_block;
    int32_t grid_blocks;
    int32_t kernels_launched;
    int32_t trotter_squares;
    int32_t graph_replayed;
    int64_t h2d_bytes;            /* parameter tables uploaded                               */
    int64_t d2h_bytes;            /* outputs that reached host buffers (copied back, or
                                     written directly with direct_host_outputs)             */
    double integrate_ms;          /* -1 when not profiled                                    */
    double chain_ms;
} spinsim_launch_info;
int spinsim_last_launch(spinsim_handle h, spinsim_launch_info* info);

/* Allocation-free variant of spinsim_simulate for one request (the paper has
 * no counterpart; it exists for callers that cannot let a library allocate:
 * real-time loops where cudaMalloc/cudaFree would synchronise the device,
 * frameworks whose pooled allocator already owns all device memory, hosts
 * that must not allocate while building their own work).
 * It needs no handle, creates no stream, event or buffer and calls no
 * allocator: all scratch lives in one file-scope device array of 16 MiB,
 * which the CUDA runtime places on a GPU when the library's device code is
 * loaded there (at the latest at the first call on that device) and which
 * stays until the process exits.  That bounds
 * the request: up to about 99,000 output samples for spin-one and 460,000
 * for spin-half; a larger K returns SPINSIM_E_NOMEM without launching.
 * res->states (and res->spin, res->ops when not NULL) must be 16-byte
 * aligned device memory, else SPINSIM_E_ARG.  cfg selects method, precision,
 * frame, tau and the launch shape (0 = lanes 1, 128 threads, as many resident
 * blocks per SM as fit; no autotuning); use_graphs, mem_budget and profile are
 * ignored; res->flags receives the request's warning bits.
 * The first call on a device looks up the device address of the array; make
 * it before any stream capture.  Every call uses the same array and leaves
 * its contents behind, so calls that overlap on the GPU (on different
 * streams, or unsynchronised host threads) race: serialise them, e.g. on one
 * stream.  Results equal those of spinsim_simulate with the same
 * configuration. */
int spinsim_simulate_static(const spinsim_config* cfg, const spinsim_request* req, spinsim_result* res,
                            void* stream);

/* One long simulation split into contiguous ranges of output samples, for
 * example one range per process (Sec. 1.2.4: the U_k are independent, so a
 * range's operators need nothing from the others; only the ordered product
 * across ranges is shared, in one exchange of one N x N matrix per range).
 *
 * spinsim_range_begin computes the sample operators of one request and their
 * ordered product agg = U_{K-1} ... U_1 U_0 (U_0 = I): the propagator from
 * t_start to t_start + (K-1) dt_out, FP64 complex [N][N] row-major, re/im
 * interleaved (2 N N doubles), written to host memory agg.  It validates the
 * request like spinsim_simulate (res->status, res->flags, res->n_samples = K;
 * req->psi0 must be normalised but is not used), runs on `stream` and waits
 * for it.  The operators stay in the handle's device memory.
 *
 * spinsim_range_finish then writes the outputs of that request (res->states,
 * and res->spin / res->ops when not NULL, as at begin) from the entering
 * state psi_in (N complex, re/im interleaved, normalised to 1e-10, else
 * SPINSIM_E_NORM), asynchronously on `stream`.  res must stay valid until then.
 *
 * A range whose request ends at t_start + (K-1) dt_out = the next range's
 * t_start therefore gives that range's entering state as agg applied to its
 * own.  finish closes the range whatever its result (after SPINSIM_E_NORM the
 * range must be begun again).  Any other call on the handle between begin and
 * finish (simulate, submit, another begin) discards the open range; finish
 * then returns SPINSIM_E_ARG.  Not for use during stream capture. */
int spinsim_range_begin(spinsim_handle h, const spinsim_request* req, spinsim_result* res, double* agg,
                        void* stream);
int spinsim_range_finish(spinsim_handle h, const double* psi_in, void* stream);

/* The exchange step between ranges (Sec. 1.2.4, Eq. integration_compilation
 * applied range by range): the state entering range `rank`,
 *   psi_out = A_{rank-1} ... A_1 A_0 psi_init,
 * from the propagators A_r that spinsim_range_begin returned for ranges
 * r = 0 .. rank - 1 (aggs: rank consecutive FP64 complex [N][N] matrices,
 * row-major, re/im interleaved; may be NULL for rank 0) and the simulation's
 * initial state psi_init (N complex).  Host arithmetic in FP64, in range
 * order, the state renormalised after each range (FP32-bulk operators are
 * not exactly unitary; the library renormalises every state it writes).
 * psi_out receives N complex.  Needs no handle and no GPU.  Returns
 * SPINSIM_E_ARG for a bad spin, rank < 0, NULL pointers or non-finite
 * values, SPINSIM_E_NORM when psi_init is not normalised to 1e-10. */
int spinsim_range_entering_state(int32_t spin_x2, const double* aggs, int32_t rank, const double* psi_init,
                                 double* psi_out);

/* The debug build's range checks (a library compiled with -DSPINSIM_BOUNDS,
 * libspinsim_bounds.so): every checked global-memory index of the kernels
 * that fell outside its buffer sets a bit of an error word on the device and
 * the access is skipped (no trap).  This call waits for the device's work,
 * writes the word of `device` into *word (0: every index was in range; bits
 * 0-1 integrate kernel, 2 drive phasor tables, 8-15 chain kernels) and
 * clears it.  The normal
 * library has no checks: it writes 0 and returns SPINSIM_E_UNSUPPORTED.
 * The paper has no counterpart: this exists to test the kernels' indexing. */
int spinsim_debug_bounds(int32_t device, uint64_t* word);

/* Static description of a status code. */
const char* spinsim_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* SPINSIM_H */
