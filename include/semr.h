/*
 * semr.h -- C ABI of libsemr: in-situ reduction of spectral-element (SEM)
 * field snapshots on one NVIDIA B300 GPU (sm_103a).
 *
 * The operation is the GPU lossy compression step of the in-situ workflow in
 * arXiv 2407.20731 (Sec. IV-B, "Turbulence with data compression"): each
 * element's lx^3 block of nodal values on Gauss-Lobatto-Legendre (GLL) points
 * is transformed to a discretely orthonormal Legendre basis, the modes whose
 * energy is below tau times the element's energy are dropped (the paper keeps
 * only the most energetic part of the data, with the amount set by a maximal
 * allowed error), the rest are quantised with a power-of-two step, written
 * to a compact payload, reconstructed, and the mass-weighted L2 and the Linf
 * errors are reported per element and per field.  The compression ratio is
 * the paper's Eq. 1, CR = (original - compressed) / original.
 *
 * Conventions of every entry point:
 *   - Return value: SEMR_OK (0) or one of the SEMR_E* codes below.  No entry
 *     point aborts, throws or prints.  semr_strerror() names a code.
 *   - Device pointers are CUDA device addresses on the device that is current
 *     when the call is made (stream ordered on the stream passed in);
 *     host pointers are ordinary host memory.
 *   - The caller owns every buffer it passes in.  Inputs must stay valid and
 *     unmodified until the work is complete (the stream has passed the
 *     launch, or semr_query returns SEMR_OK for the ticket).
 *   - Field layout: one FP64 array per field, n_elem blocks of lx^3 values,
 *     element block e at offset e*lx^3, value (i, j, k) at i + lx*(j + lx*k)
 *     (i fastest).  Modal index m = p + lx*(q + lx*r).  Field pointers
 *     16-byte aligned for even lx, 8-byte aligned for odd lx; every other
 *     FP64 pointer 8-byte aligned; payload 16-byte, scratch 256-byte aligned.
 *
 * Payload format (version 1, little-endian, all section starts 16-aligned):
 *   header : "SEMR", u16 version, u16 lx, u16 n_fields, u16 flags,
 *            u32 header_bytes, u64 n_elem, f64 tau, u64 code_base,
 *            u64 code_total, u64 code_count[n_fields], padded to 16 bytes
 *   field f: mask  n_elem x ceil(lx^3/8) bytes (mode m of element e is bit
 *                  (m & 7) of byte e*ceil(lx^3/8) + (m >> 3)), padded
 *            step  int16[n_elem]  s_e (INT16_MIN: element keeps nothing), padded
 *            count uint16[n_elem] n_e, number of kept modes, padded
 *   codes  : code_total entries from byte code_base, ordered by (field,
 *            element, mode); int16 (flags & SEMR_PAYLOAD_CODE32 == 0),
 *            int32 (SEMR_PAYLOAD_CODE32), or the raw FP64 coefficient in
 *            lossless mode (SEMR_PAYLOAD_LOSSLESS, tau == 0).
 *   Kept mode m of element e is reconstructed as a~_m = code * 2^{s_e}.
 *   Quantisation: t = tau * S_e with S_e = sum_m a_m^2; mode m kept iff
 *   a_m^2 >= t; s_e = floor((ex - 1) / 2) for t = mu * 2^ex, mu in [1/2, 1);
 *   code = rint(a_m * 2^{-s_e}), ties to even.  Codes are int16 when
 *   tau * 32767^2 > 4 (then |code| <= 2 / sqrt(tau) < 32767), else int32.
 *   An element with t below the smallest normal double keeps nothing.
 *   The result depends on the field's magnitude only through exact powers of
 *   two: every element is read as u * 2^-k, k the binary exponent of its
 *   largest |u|, so scaling a field by 2^j leaves masks, counts and codes
 *   unchanged and shifts every step by j (for magnitudes 2^-1022 <= |u| <
 *   2^500; the status bits below flag elements outside that range).
 */
#ifndef SEMR_H
#define SEMR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define SEMR_OK 0
#define SEMR_EINVAL 1         /* bad argument: null pointer, size, alignment, lx, tau */
#define SEMR_ENOMEM 2         /* a device or pinned-host allocation failed */
#define SEMR_EBUDGET 3        /* the request does not fit the stream's memory budget now */
#define SEMR_EAGAIN 4         /* the ticket's work has not finished yet */
#define SEMR_ETIMEDOUT 5      /* a bounded device-side wait gave up (result invalid) */
#define SEMR_ECUDA 6          /* a CUDA runtime call failed */
#define SEMR_ENOSPACE 7       /* an output buffer is smaller than the result */
#define SEMR_ENONFINITE 8     /* an element held a NaN or an infinity (that element keeps nothing) */
#define SEMR_EUNSUPPORTED 9   /* lx or precision not built into this library */

/* ------------------------------------------------------------- parameters */
#define SEMR_MAX_FIELDS 16
#define SEMR_LX_MIN 2
#define SEMR_LX_MAX 12

/* precision of the transforms */
#define SEMR_FP64 0          /* FP64 accuracy on the FP32 pipes: an FP32 forward transform under a
                                proven error bound settles most decisions, the few it cannot are
                                recomputed in hardware FP64; energies, reconstruction and norms are
                                float pairs (about 48 significant bits).  Payloads match an FP64
                                computation bit for bit outside decisions within 1e-9 of a tie */
#define SEMR_FP32 1          /* the precision form: transforms in FP32 with FP32 accumulation; the
                                threshold test is exactly the FP64 comparison; element and field
                                sums are float-pair tree sums finished in FP64 */
#define SEMR_FP64_NATIVE 2   /* every operation in hardware FP64 (slow on B300: its FP64 pipe runs
                                under 1 TFLOP/s); kept as a reference path */

/* fieldset flags */
#define SEMR_WRITE_RECON 1   /* also write the reconstruction to fieldset.recon[f] */
#define SEMR_CUMULATIVE 2    /* cumulative-energy truncation (the sort-based reading of Sec. IV-B's
                                maximal allowed error as a budget on the discarded energy): drop the
                                least energetic modes while their summed energy stays <= tau S_e,
                                keep every mode whose energy is at least the smallest one not
                                dropped (equal energies together).  Step and codes as in the
                                threshold form.  SEMR_FP64 and SEMR_FP32 only, single launches and
                                the stream API (SEMR_EUNSUPPORTED with SEMR_FP64_NATIVE or in a
                                batch); ignored in lossless mode (tau == 0). */

/* payload header flag bits */
#define SEMR_PAYLOAD_LOSSLESS 1
#define SEMR_PAYLOAD_CODE32 2
#define SEMR_PAYLOAD_FP32 4
#define SEMR_PAYLOAD_CUMULATIVE 8  /* modes selected by SEMR_CUMULATIVE */

/* summary.status bits (device-written) */
#define SEMR_STATUS_OVERFLOW 1    /* payload_cap too small: codes not written */
#define SEMR_STATUS_TIMEOUT 2     /* look-back wait gave up */
#define SEMR_STATUS_NONFINITE 4   /* an element held a NaN, an infinity or a magnitude of 2^500 or more
                                     (its energy would overflow FP64 arithmetic): that element keeps
                                     nothing */
#define SEMR_STATUS_STAGE 16      /* after a timed-out wait for an element block's TMA copy, a second
                                     bounded wait for that copy gave up too: the copy may have landed in
                                     shared memory after the kernel stopped using it (results invalid,
                                     as with SEMR_STATUS_TIMEOUT, which is also set; treat the device as
                                     suspect) */
#define SEMR_STATUS_TINY 8        /* informational, not an error: an element held only subnormal values
                                     (every |u| < 2^-1022).  It keeps nothing, as an FP64 evaluation
                                     does (its t = tau S_e underflows), and its e2_e, E_e and Linf_e
                                     are reported as 0 where FP64 gives values below 2^-1022 */
#define SEMR_STATUS_BOUNDS 32     /* only in a library built with -DSEMR_BOUNDS (a checking build, see
                                     semr_build_flags): a kernel computed an index or a byte range outside
                                     the buffer it was about to read or write; that access was skipped
                                     (results invalid) */

typedef struct {
    int32_t lx;            /* GLL points per direction, SEMR_LX_MIN..SEMR_LX_MAX */
    int32_t pad_;
    int64_t n_elem;        /* number of elements, >= 1, n_elem * lx^3 < 2^40 */
    const double* jac;     /* device, n_elem element Jacobians (mass scale), finite */
} semr_mesh;

typedef struct {
    int32_t n_fields;                 /* 1..SEMR_MAX_FIELDS */
    int32_t precision;                /* SEMR_FP64 or SEMR_FP32 */
    double tau;                       /* threshold: 0 (lossless mode) or 2^-60 < tau <= 2^64 (for smaller
                                         tau a code 2/sqrt(tau) would not fit int32) */
    int32_t flags;                    /* SEMR_WRITE_RECON | SEMR_CUMULATIVE, or 0 */
    int32_t pad_;
    const double* fields[SEMR_MAX_FIELDS];  /* device, n_elem*lx^3 FP64 each */
    double* recon[SEMR_MAX_FIELDS];         /* device outputs when SEMR_WRITE_RECON, else ignored */
} semr_fieldset;

/* Per-field error report (Sec. IV-B's "sufficient accuracy" check and Eq. 1). */
typedef struct {
    double l2_abs;      /* sqrt(sum_e e2_e), e2_e = J_e sum w_i w_j w_k (u - u~)^2 */
    double l2_rel;      /* sqrt(sum e2 / sum E), E_e = J_e sum w_i w_j w_k u^2; 0 if sum E == 0 */
    double linf_abs;    /* max |u - u~| over all GLL points (unweighted) */
    double linf_rel;    /* linf_abs / max|u|; 0 if max|u| == 0 */
    double sum_err2;    /* sum_e e2_e */
    double sum_energy;  /* sum_e E_e */
    double umax;        /* max |u| */
    uint64_t kept;      /* number of codes of this field */
    uint64_t bytes;     /* fixed sections + codes of this field */
    double cr;          /* Eq. 1 for this field: 1 - bytes / (8 lx^3 n_elem) */
} semr_field_report;

/* Device-written result summary of one reduction. */
typedef struct {
    uint64_t payload_bytes;   /* total payload size */
    uint64_t code_total;      /* codes over all fields */
    uint32_t status;          /* SEMR_STATUS_* bits, 0 when everything is valid */
    uint32_t n_fields;
    double cr;                /* Eq. 1 over the whole snapshot */
    uint64_t recomputed;      /* FP64 mode: coefficients whose FP32 value could not settle a
                                 decision and were recomputed exactly */
    semr_field_report field[SEMR_MAX_FIELDS];
} semr_summary;

/* Buffer sizes of one reduction (host-computed, exact). */
typedef struct {
    uint64_t header_bytes;       /* payload header */
    uint64_t code_base;          /* header + fixed sections: minimum payload capacity */
    uint64_t payload_worst;      /* code_base + every mode kept: always sufficient */
    uint64_t scratch_bytes;      /* device scratch for semr_reduce_async (recommended size) */
    uint64_t elem_report_bytes;  /* n_fields * n_elem * 3 doubles */
    uint32_t code_width;         /* 2, 4 or 8 bytes */
    uint32_t tiles;              /* work tiles of the CTA-per-tile kernels (saturates at 2^32-1) */
    uint64_t scratch_min_bytes;  /* smallest scratch semr_reduce_async accepts (<= scratch_bytes);
                                    at lx = 8 a scratch between the two runs the kernel on fewer
                                    CTAs, with the same results */
} semr_sizes;

/* Device buffers of one reduction (all caller-owned device memory). */
typedef struct {
    uint8_t* payload;          /* device, payload_cap bytes; the complete payload */
    uint64_t payload_cap;      /* >= semr_sizes.code_base; codes beyond it set SEMR_STATUS_OVERFLOW */
    double* elem_report;       /* device [n_fields][n_elem][3] = (e2_e, E_e, Linf_e), or NULL */
    semr_summary* summary;     /* device, one semr_summary */
    void* scratch;             /* device, semr_sizes.scratch_bytes, 256-byte aligned */
    uint64_t scratch_bytes;
} semr_outputs;

typedef struct semr_stream semr_stream;

/*
 * semr_sizes_for: sizes of the buffers one reduction needs.
 *   lx, n_elem, n_fields, tau as in semr_mesh / semr_fieldset.
 * Errors: SEMR_EINVAL (out-of-range argument or null out).
 */
int semr_sizes_for(int32_t lx, int64_t n_elem, int32_t n_fields, double tau, semr_sizes* out);

/*
 * semr_reduce_async: the hot path.  Launches the fused reduce kernel (forward
 * transform, energy, truncation mask, quantisation, one-pass global
 * compaction of the codes, reconstruction, error norms) and the finalize
 * kernel on `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 * Writes the complete payload, the optional element report and the summary.
 * Asynchronous: returns after the launches; results are valid once the
 * stream passes this point and summary->status == 0.  Allocates nothing.
 * Errors: SEMR_EINVAL (null/misaligned pointer, bad size or tau, scratch or
 * payload_cap too small), SEMR_EUNSUPPORTED (lx or precision), SEMR_ECUDA
 * (launch failure).
 */
int semr_reduce_async(const semr_fieldset* fs, const semr_mesh* mesh, const semr_outputs* out,
                      void* cuda_stream);

/*
 * semr_reduce_async_timed: semr_reduce_async that also records two CUDA
 * events (cudaEvent_t handles, either may be NULL) on `cuda_stream`
 * immediately before and immediately after the fused reduce kernel, so that
 * a caller can time that kernel alone (the scratch clear and the finalize
 * kernel fall outside the pair).  Same arguments, errors and effects as
 * semr_reduce_async; SEMR_ECUDA if an event record fails.
 */
int semr_reduce_async_timed(const semr_fieldset* fs, const semr_mesh* mesh, const semr_outputs* out,
                            void* cuda_stream, void* ev_begin, void* ev_end);

/*
 * semr_open: a reduction stream with library-owned buffers (the hand-over of
 * a snapshot from the simulation to the in-situ reduction, Sec. III-A: the
 * producer submits and goes on; results are fetched when ready).
 *   device: CUDA device ordinal.  cuda_stream: cudaStream_t to order work on
 *   (NULL: the library creates its own non-blocking stream).
 *   mem_budget_bytes: upper bound on device memory that unfetched tickets may
 *   hold (payload + scratch + reports); 0 = no bound.
 * A ticket's payload is sized for an estimate of its codes: twice the
 * largest share of modes kept by the stream's completed tickets (1/16 of all
 * modes before the first completes), plus 4096 codes, at most every mode.  A
 * ticket whose codes do not fit is re-run once, at the exact size its first
 * run reports, when its completion is next observed (semr_query or
 * semr_fetch), unless that run also reported SEMR_STATUS_TIMEOUT, _STAGE or
 * _BOUNDS (the input flags _TINY and _NONFINITE recur in the re-run); the field and Jacobian buffers must therefore stay valid
 * until semr_query returns SEMR_OK or semr_fetch succeeds.  The stream's
 * calls are thread-safe with respect to each other, except semr_close,
 * which must not overlap any other call on the stream.  No call holds the
 * stream's lock while it waits for the device or copies.
 * Errors: SEMR_EINVAL, SEMR_ECUDA, SEMR_ENOMEM.
 */
int semr_open(semr_stream** s, int device, void* cuda_stream, uint64_t mem_budget_bytes);

/*
 * semr_submit: queue the reduction of one snapshot; returns at once with a
 * ticket.  Allocates the ticket's device buffers (stream-ordered) within the
 * budget.  The field and Jacobian buffers must stay valid until the ticket
 * completes.  Errors: SEMR_EINVAL, SEMR_EUNSUPPORTED, SEMR_EBUDGET (does
 * not fit next to the tickets in flight: fetch some first), SEMR_ENOMEM,
 * SEMR_ECUDA.
 */
int semr_submit(semr_stream* s, const semr_fieldset* fs, const semr_mesh* mesh, uint64_t* ticket);

/* semr_query: SEMR_OK when the ticket's results are final, SEMR_EAGAIN if
 * its work (or its exact-size re-run, started by this call) is still running,
 * SEMR_EBUDGET if that re-run does not fit the budget next to the other
 * unfetched tickets (fetch some, then query again), SEMR_EINVAL for an unknown
 * ticket, SEMR_ENOMEM / SEMR_ECUDA if the re-run could not be started. */
int semr_query(semr_stream* s, uint64_t ticket);

/*
 * semr_fetch: copy a ticket's results to host memory and release the ticket.
 *   wait: nonzero blocks until the results are final (through a re-run, if
 *   one is needed); zero returns SEMR_EAGAIN if they are not.
 *   payload (host, cap bytes) or NULL; *payload_bytes gets the size.
 *   reports (host, n_fields entries) or NULL; elem_report (host, n_fields *
 *   n_elem * 3 doubles) or NULL.
 * The copies run on a copy stream of the library's, ordered after this
 * ticket's work only.
 * Errors: SEMR_EAGAIN (not final, or another fetch of the ticket is in
 * progress), SEMR_EINVAL (unknown ticket), SEMR_EBUDGET (as semr_query),
 * SEMR_ENOSPACE (cap too small: nothing copied, ticket kept; *payload_bytes
 * holds the size needed), SEMR_ETIMEDOUT / SEMR_ENONFINITE (device status;
 * results copied, ticket released), SEMR_ECUDA.
 */
int semr_fetch(semr_stream* s, uint64_t ticket, int wait, void* payload, uint64_t cap,
               uint64_t* payload_bytes, semr_field_report* reports, double* elem_report);

/* semr_close: wait for the stream's work, free everything it owns. */
void semr_close(semr_stream* s);

/*
 * semr_decode: rebuild the fields from a payload on the host (FP64).
 *   out: host, n_fields * n_elem * lx^3 doubles (cap_doubles), layout as the input.
 *   hdr_out (optional): lx, n_fields, n_elem of the payload.
 * Errors: SEMR_EINVAL (malformed payload), SEMR_ENOSPACE.
 */
int semr_decode(const void* payload, uint64_t bytes, double* out, uint64_t cap_doubles,
                int32_t* lx_out, int32_t* n_fields_out, int64_t* n_elem_out);

/* semr_gll: the library's GLL nodes and weights (host, lx entries each). */
int semr_gll(int32_t lx, double* nodes, double* weights);

/*
 * semr_reduce_async_noalloc: semr_reduce_async for callers that cannot
 * allocate device memory -- for example a solver that hands nearly all of
 * the GPU's memory to its own pool at start-up, or in-situ code that runs
 * between time steps where no allocator call is allowed.  The paper has no
 * counterpart to this entry point.
 *
 * The caller still passes the inputs and the outputs (payload of
 * payload_cap bytes, optional elem_report, summary), all device memory, as
 * in semr_outputs.  The kernel's scratch comes from one file-scope device
 * array of SEMR_NOALLOC_SCRATCH_BYTES (64 MiB) that every GPU loading the
 * library holds until the process exits; nothing is allocated or freed
 * (no cudaMalloc, cudaFree or allocating library routine).  A snapshot
 * whose smallest usable scratch (semr_sizes.scratch_min_bytes) exceeds the
 * array is rejected with SEMR_EBUDGET, before any pointer is looked at.
 * At lx = 8 that is about 10 bytes per element-field (the CTA-per-tile
 * kernel's 40 bytes per 4-element tile, which also covers the warp kernel's
 * 4.3 bytes per element-field plus one CTA's 67,840-byte code staging), so
 * snapshots up to about 6.7 million element-fields are accepted (e.g. 128^3
 * elements x 3 fields).  The array holds code staging for every CTA the warp
 * kernel can keep resident up to about 6.2 million (SEMR_FP64) or 1.6 million
 * (SEMR_FP32) element-fields; beyond that it runs on the CTAs it can stage
 * for (same results, less throughput).
 *
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it: make that first call before any stream
 * capture.  Every call on a device shares the one array, whose contents
 * persist between calls; each call clears the part that must start at zero.
 * Calls that overlap on the GPU (on different streams, or not yet finished
 * on another stream) race on the array and corrupt each other's results:
 * order them on one stream.  Errors as semr_reduce_async, plus SEMR_EBUDGET
 * (above) and SEMR_ECUDA if the address lookup fails.
 */
#define SEMR_NOALLOC_SCRATCH_BYTES (64ull << 20)
int semr_reduce_async_noalloc(const semr_fieldset* fs, const semr_mesh* mesh, uint8_t* payload,
                              uint64_t payload_cap, double* elem_report, semr_summary* summary,
                              void* cuda_stream);

/* Self-test of the bounded device-side waits, with no fault and no hang: one
 * warp runs (0) the decoupled look-back of a tile whose predecessor never
 * publishes its state, and (1) the wait for a phase of an mbarrier that never
 * completes, the two waits every reduction kernel bounds, followed (as in the
 * reduce kernel's abort path) by the second bounded wait for a copy that
 * might still be in flight.  Each wait gives up at its bound (the look-back
 * after 2^22 polls, about 2-3 s; the barrier after 1000 polls of at most 1 ms
 * each, twice) and records what the kernel records: SEMR_STATUS_TIMEOUT for
 * (0), SEMR_STATUS_TIMEOUT | SEMR_STATUS_STAGE for (1).  The kernel then
 * returns and the context stays usable.  status_out: host uint32_t[2],
 * receives the status word of each wait.  Blocks until done (current device,
 * legacy default stream).  Returns SEMR_OK, SEMR_EINVAL (null status_out),
 * SEMR_ENOMEM or SEMR_ECUDA. */
int semr_selftest_waits(uint32_t* status_out);

/* ------------------------------------------------------ batched launches */

/* One snapshot of a batch: as for semr_reduce_async; out.scratch is ignored
 * (the batch owns the scratch).  Precision SEMR_FP64 or SEMR_FP32 (FP64 mode
 * not lossless); SEMR_CUMULATIVE at lx = 6, 8 and 10 with int16 codes (the
 * orders the warp-level kernels serve), SEMR_EUNSUPPORTED otherwise. */
typedef struct {
    semr_fieldset fs;
    semr_mesh mesh;
    semr_outputs out;
} semr_batch_item;

#define SEMR_BATCH_AUTOTUNE 1  /* time every tile variant per (lx, precision) group, keep the fastest */

typedef struct semr_batch semr_batch;

/*
 * semr_batch_create: plan the reduction of n_items snapshots of any sizes and
 * orders in one launch sequence (many uneven snapshots per launch, the
 * batched form of the in-situ reduction).  Snapshots are grouped by (lx,
 * precision, truncation); each group runs one persistent kernel over a single work queue
 * of all its snapshots' tiles, then one finalize kernel.  With
 * SEMR_BATCH_AUTOTUNE the elements per CTA of each group are chosen by timing
 * every compiled variant on the group's largest snapshot (this runs kernels
 * and writes that snapshot's outputs).  Allocates one device workspace and
 * uploads the descriptors (synchronises `cuda_stream`).  The item buffers
 * must stay valid for the plan's lifetime.
 * Errors: SEMR_EINVAL, SEMR_EUNSUPPORTED, SEMR_ENOMEM, SEMR_ECUDA.
 */
int semr_batch_create(semr_batch** b, const semr_batch_item* items, int n_items, int flags, void* cuda_stream);

/* semr_batch_launch: enqueue the whole batch on `cuda_stream` (scratch
 * clears, kernels).  Asynchronous; may itself be captured into a graph. */
int semr_batch_launch(semr_batch* b, void* cuda_stream);

/* semr_batch_capture: capture the launch sequence into a CUDA graph owned by
 * the plan; semr_batch_replay launches it on `cuda_stream` (one graph launch
 * for the whole batch). */
int semr_batch_capture(semr_batch* b, void* cuda_stream);
int semr_batch_replay(semr_batch* b, void* cuda_stream);

/* semr_batch_schedule: group < 0 returns the number of groups; else fills the
 * group's lx, precision, chosen elements per tile, item count, and the tuned
 * time (ms, -1 if the variant could not run) of each of up to `cap` variants. */
int semr_batch_schedule(const semr_batch* b, int group, int* lx, int* precision, int* tile, int* n_items,
                        float* variant_ms, int* variant_tiles, int cap);

/* semr_batch_destroy: wait for the device, free the workspace and graph. */
void semr_batch_destroy(semr_batch* b);

/* ------------------------------------------------------------ serving */

/*
 * A continuous-batching server for in-situ reductions (the paper's
 * asynchronous approach, Sec. III-A, realised with streams in one process).
 * Producers on any thread submit reductions of snapshots already in device
 * memory.  A dispatcher thread admits queued requests in arrival order into
 * `slots` device slots (one CUDA stream each) whenever a slot is free and the
 * request's device memory (payload + scratch + reports) fits `mem_budget_bytes`
 * (0: no bound) next to every admitted, unreleased request.  The payload is
 * sized for an estimate of the request's codes: twice the largest share of
 * modes kept by the requests completed so far (1/16 of all modes before the
 * first), plus 4096 codes, at most every mode kept.  A request whose codes do
 * not fit is re-run once on its slot at the exact size its first run reports
 * (when that fits the budget, and unless that run also reported
 * SEMR_STATUS_TIMEOUT, _STAGE or _BOUNDS), so its completion comes later but
 * its result is the same.  Admitted requests run concurrently and overlap on the GPU;
 * results stay on the device until released.  The input buffers must stay
 * valid until the request completes.
 */
typedef struct semr_server semr_server;

typedef struct {
    double t_submit, t_admit, t_done;  /* host steady-clock seconds (completion from a stream callback) */
    int32_t slot;                      /* device slot that ran the request */
    int32_t status;                    /* SEMR_OK, or the error that stopped the launch */
    uint64_t device_bytes;             /* device memory the request held (after a re-run: its exact size) */
    semr_summary summary;              /* as written by the reduction */
} semr_request_info;

/* Errors: SEMR_EINVAL (device, slots outside 1..64), SEMR_ECUDA, SEMR_ENOMEM. */
int semr_server_create(semr_server** s, int device, uint32_t slots, uint64_t mem_budget_bytes);
/* Queue one reduction (thread-safe, returns at once).  SEMR_EBUDGET if the
 * request alone exceeds the budget; SEMR_EINVAL for bad sizes. */
int semr_server_submit(semr_server* s, const semr_fieldset* fs, const semr_mesh* mesh, uint64_t* id);
/* State of a request: SEMR_EAGAIN while queued or running (wait = 0), else
 * its result status; fills `info` when done.  wait != 0 blocks until done. */
int semr_server_wait(semr_server* s, uint64_t id, int wait, semr_request_info* info);
/* Wait for the request, copy its payload to `payload` (host, cap bytes; may
 * be NULL), free its device memory and forget it.  SEMR_ENOSPACE if cap is
 * too small (the request is released all the same). */
int semr_server_release(semr_server* s, uint64_t id, void* payload, uint64_t cap, uint64_t* bytes);
/* Counters: admitted, completed, still queued, device bytes held, seconds
 * from the first admission to the last completion, input bytes completed. */
int semr_server_stats(semr_server* s, uint64_t* admitted, uint64_t* completed, uint64_t* queued,
                      uint64_t* held_bytes, double* busy_seconds, uint64_t* bytes_done);
/* Stop the dispatcher, wait for running requests, free everything. */
void semr_server_destroy(semr_server* s);

/* ------------------------------------------------- in-situ slice image
 *
 * The other in-situ task of arXiv 2407.20731 (Sec. IV-A): an image of a
 * slice through the fields, rendered while the simulation runs (there by
 * ParaView/Catalyst on the host, with a pipeline that fixes the camera, the
 * image size and the slice position).  Here one call renders the slice into
 * a headless RGBA8 device buffer:
 *   1. pixel (column c, row r) of a W x H image sits at the world point
 *        p = (origin + ((c + 0.5)/W) axis_u) + ((r + 0.5)/H) axis_v
 *      (row 0 nearest origin along axis_v, each operation rounded once);
 *   2. per axis q = (p - mesh.origin) / mesh.h, element index floor(q) (the
 *      top face q == n belongs to the last element), reference coordinate
 *      2 (q - floor(q)) - 1; points outside the lattice get `background`;
 *   3. the value is the element's tensor-product Lagrange interpolant
 *      through its lx^3 GLL nodal values (the spectral-element field itself),
 *      or with n_comp = 2 or 3 the magnitude of the interpolated vector;
 *   4. t = clamp((s - vmin)/(vmax - vmin), 0, 1), each colour channel
 *      linear in t between the control points (t_k, r_k, g_k, b_k) of the
 *      segment that holds t, byte = floor(255 c + 0.5), alpha 255.
 * Steps 1-2 run in FP64 (they decide which element owns a pixel); steps 3-4
 * in FP32 (ample for 8-bit colour): a channel may differ by one from an FP64
 * evaluation only where 255 c lies within the FP32 error of a rounding tie.
 * A slice whose axis_u and axis_v each lie along one (different) lattice
 * axis is rendered one element per thread block (the element is contracted
 * along the slice normal once, then each pixel costs lx^2 + lx FMAs per
 * component); any other plane takes the per-pixel lx^3 path.
 */
typedef struct {
    int32_t lx;            /* GLL points per direction, SEMR_LX_MIN..SEMR_LX_MAX */
    int32_t nx, ny, nz;    /* element lattice, >= 1 each; element e = ex + nx*(ey + ny*ez), nx*ny*nz < 2^31 */
    double origin[3];      /* lower corner of the box */
    double h[3];           /* element edge lengths, > 0 (affine, axis-aligned hexahedra) */
} semr_lattice;

#define SEMR_SLICE_MAX_CTRL 16
#define SEMR_SLICE_MAX_COMP 3
#define SEMR_SLICE_MAX_SIDE 16384

typedef struct {
    double origin[3];      /* world point of the image corner (pixel (0,0) is half a pixel inside) */
    double axis_u[3];      /* world vector along the image width (columns) */
    double axis_v[3];      /* world vector along the image height (rows) */
    int32_t width, height; /* pixels, 1..SEMR_SLICE_MAX_SIDE each */
    int32_t n_comp;        /* 1: colour by fields[0]; 2-3: by the magnitude of (fields[0], ...) */
    int32_t n_ctrl;        /* colour-table control points, 2..SEMR_SLICE_MAX_CTRL */
    double vmin, vmax;     /* scalar range mapped to t in [0, 1], vmax > vmin, finite */
    double ctrl[SEMR_SLICE_MAX_CTRL][4];  /* (t, r, g, b): t_0 = 0 < t_1 < ... < t_{n-1} = 1, r, g, b in [0, 1] */
    uint32_t background;   /* RGBA8 of pixels outside the mesh, R in the low byte */
    int32_t pad_;
} semr_slice;

/* Render one slice image, stream ordered on cuda_stream; allocates nothing.
 *   fields  host array of n_comp device pointers, each lattice n_elem*lx^3
 *           FP64 values in the layout of semr_fieldset (16-byte aligned for
 *           even lx, 8-byte for odd)
 *   rgba    device, width*height*4 bytes: pixel (c, r) at 4 (r width + c),
 *           bytes R, G, B, A
 *   values  device, width*height floats, the coloured scalar (NaN outside
 *           the mesh), or NULL
 * Errors: SEMR_EINVAL (null pointer, sizes, non-finite or non-positive
 * geometry, colour table not as above, vmax <= vmin), SEMR_EUNSUPPORTED (lx),
 * SEMR_ECUDA (launch).  Inputs are read only; caller owns every buffer. */
int semr_slice_rgba(const semr_lattice* mesh, const double* const* fields, const semr_slice* sl,
                    uint8_t* rgba, float* values, void* cuda_stream);

/* semr_strerror: static text for a status code. */
const char* semr_strerror(int code);

/* semr_build_flags: how this copy of the library was built.  SEMR_BUILD_BOUNDS:
 * compiled with -DSEMR_BOUNDS, a checking build in which every kernel tests
 * the index or byte range of each global access (payload, element report,
 * reconstruction, scratch, slice image, staged codes) against its buffer
 * before making it; an access outside is skipped and sets SEMR_STATUS_BOUNDS.
 * The checks never trap.  Slower than the default build; for testing. */
#define SEMR_BUILD_BOUNDS 1
int semr_build_flags(void);

/* semr_bounds_status: SEMR_STATUS_BOUNDS if, since the last reset, a kernel
 * without a status word of its own (the slice kernels) skipped an access in
 * a bounds build; 0 otherwise, and always 0 in the default build.  reset != 0
 * clears it.  Synchronous (waits for the device); 0xffffffff on a CUDA error. */
uint32_t semr_bounds_status(int reset);

/* semr_selftest_bounds: checking build only (SEMR_EUNSUPPORTED otherwise).
 * Shows that the range tests fire: reduces a 300-element lx = 8 field (FP64
 * mode, tau = 1e-3) into buffers of the full size while the kernels are told
 * a payload capacity 64 bytes short of the fixed sections, so every element's
 * payload range test fails and its writes are skipped (none leaves the
 * buffers the call allocated).  *status_out gets the summary's status word,
 * which must hold SEMR_STATUS_BOUNDS.  Synchronous; allocates and frees its
 * own device memory. */
int semr_selftest_bounds(uint32_t* status_out);

#ifdef __cplusplus
}
#endif
#endif /* SEMR_H */
