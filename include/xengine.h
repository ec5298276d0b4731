/*
 * xengine.h -- C ABI of the B300 (sm_103a) FX-correlator X-engine.
 *
 * The X-engine takes gulps of 4+4-bit complex voltages laid out as
 * (time, channel, input) and, for every frequency channel c, accumulates the
 * Hermitian visibility matrix
 *
 *     V_c[i][j] = sum_t x[t][c][i] * conj(x[t][c][j]),        i >= j,
 *
 * emitting the packed lower triangle.  The pieces come from arXiv 1708.00720
 * (Bifrost): the sample format is the F-engine's 4+4-bit complex signed
 * integers (section "Packet capture implementation"); the unpack, the
 * accumulate and the linear-algebra product are the unpack block, the
 * accumulate block (section "Some included blocks") and the linear-algebra
 * module (section "Back end"); a gulp is the span of data a block reads
 * from its ring buffer in one step (section "Memory management and ring
 * buffers").
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Sample byte: real part in the high nibble, imaginary part in the low
 *    nibble, each 4-bit two's complement in [-8, 7] (0x80 = -8 + 0i,
 *    0x0F = 0 - 1i).
 *  - Gulp layout: uint8 x[ntime][n_chan][n_input], input fastest.  Element
 *    (t, c, i) is at byte t*n_chan*n_input + c*n_input + i.
 *  - Visibility layout: [n_chan][n_input*(n_input+1)/2] complex values,
 *    channel slowest; baseline (i, j), i >= j, at i*(i+1)/2 + j; each value
 *    is an (re, im) pair of int32 (XE_OUT_CI32) or float (XE_OUT_CF32).
 *    Every value is an exact integer below 2^31 in magnitude (CI32) and below
 *    2^24 for any integration the plan accepts, so CF32 is exact too.
 *  - Pointers named d_* are CUDA device pointers on the plan's device; h_*
 *    are host pointers (pinned memory gives full copy speed).  The caller
 *    owns every buffer it passes and must keep it alive until the stream work
 *    that uses it has completed.  The plan owns its accumulator and
 *    workspace.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued asynchronously on it; argument
 *    checks happen synchronously on the host and a call that fails a check
 *    enqueues nothing.
 *  - Calls never throw and never abort; they return an xe_status.  After
 *    XE_ERR_CUDA, xe_plan_last_error() holds the CUDA error text.
 *  - A plan is not thread-safe: calls on one plan must be serialised by the
 *    caller, and their device work must not overlap (use one stream per
 *    plan, or order the streams): the correlation kernels of a plan share
 *    its accumulator and its scratch, also for xe_correlate_emit.
 *    Different plans are independent.
 */
#ifndef XENGINE_H
#define XENGINE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define XE_API __attribute__((visibility("default")))
#else
#define XE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    XE_OK = 0,
    XE_ERR_INVALID_ARG = 1,        /* null pointer, negative size, bad enum */
    XE_ERR_ALIGNMENT = 2,          /* pointer not 16-byte aligned, or n_input % 16 != 0 */
    XE_ERR_SHAPE = 3,              /* size beyond what the plan was created for */
    XE_ERR_ACCUM_BOUND = 4,        /* integration would lose exactness (see xe_correlate) */
    XE_ERR_NOMEM = 5,              /* device allocation failed */
    XE_ERR_CUDA = 6,               /* a CUDA runtime/driver call failed */
    XE_ERR_DEVICE_UNSUPPORTED = 7, /* current device is not sm_103 */
    XE_ERR_TIMEOUT = 8,            /* a bounded device-side wait gave up */
    XE_ERR_BUSY = 9,               /* resource in use (serving layer) */
    XE_ERR_DEVICE_INDEX = 10       /* debug build only: a kernel's global index fell outside its
                                      buffer; the access was skipped (see xe_plan_check) */
} xe_status;

/* Operand type the contraction runs in.  All three give identical, exact
 * results; they differ only in speed.
 *  XE_OPERAND_FP8_E4M3        tcgen05 tensor cores, kind::f8f6f4 (fastest)
 *  XE_OPERAND_FP16            tcgen05 tensor cores, kind::f16
 *  XE_OPERAND_INT32_CUDACORE  plain CUDA-core int8 dot products into int32
 *                             (the comparison baseline) */
typedef enum {
    XE_OPERAND_FP8_E4M3 = 0,
    XE_OPERAND_FP16 = 1,
    XE_OPERAND_INT32_CUDACORE = 2
} xe_operand;

/* Element type of emitted visibilities. */
typedef enum {
    XE_OUT_CI32 = 0,   /* int32 (re, im) pairs */
    XE_OUT_CF32 = 1    /* float (re, im) pairs, exact integers */
} xe_out;

typedef struct xe_plan *xe_plan_t;

/* Largest number of time samples one integration may hold (from the last
 * xe_reset or non-accumulating xe_correlate): every visibility is at most
 * 128 per sample in magnitude, so 128 * samples must stay below 2^31 for the
 * int32 accumulator (XE_OUT_CI32) and at most 2^24 for exact float32 output
 * (XE_OUT_CF32).  Inside one gulp the tensor-core kernels keep every float32
 * partial sum exact by splitting the gulp into launches of at most 32768
 * samples (450 * 32768 < 2^24), each adding into the int32 accumulator. */
#define XE_MAX_SAMPLES_CI32 16777215LL
#define XE_MAX_SAMPLES_CF32 131072LL

/*
 * Create a plan on the current CUDA device for n_input inputs (n_input %
 * 16 == 0, 16 <= n_input <= 8192), n_chan channels (>= 1) and gulps of at
 * most max_ntime samples (>= 1).  Allocates the int32
 * integration accumulator (n_chan * n_input*(n_input+1)/2 * 8 bytes),
 * zeroes it, and sets the sample counter to 0.  On failure *out is NULL.
 * Errors: XE_ERR_INVALID_ARG, XE_ERR_ALIGNMENT (n_input % 16), XE_ERR_NOMEM,
 * XE_ERR_DEVICE_UNSUPPORTED, XE_ERR_CUDA.
 */
XE_API xe_status xe_plan_create(xe_plan_t *out, int n_input, int n_chan, int max_ntime,
                         xe_operand op, xe_out out_type);

/* Free the plan and its device memory (synchronises its device first).
 * NULL is accepted and ignored. */
XE_API xe_status xe_plan_destroy(xe_plan_t plan);

/*
 * Unpack (section "Some included blocks", unpack; the TBN pipeline's 4+4 to
 * 8+8 conversion): d_ci8[k][0] = real, d_ci8[k][1] = imaginary part of
 * d_packed[k], for k < ntime * n_chan * n_input.  d_packed must be 16-byte
 * aligned.  Does not touch the accumulator.
 */
XE_API xe_status xe_unpack(xe_plan_t plan, const uint8_t *d_packed, int8_t *d_ci8,
                    int ntime, void *stream);

/*
 * Correlate one gulp d_gulp[ntime][n_chan][n_input] (16-byte aligned) into
 * the plan's accumulator: accumulate = 0 replaces the accumulator with this
 * gulp's visibilities and sets the sample counter to ntime; accumulate = 1
 * adds them and adds ntime to the counter (the accumulate block).
 * ntime = 0 is allowed (adds nothing / zeroes the accumulator); d_gulp may
 * then be NULL.
 * Errors: XE_ERR_SHAPE (ntime > max_ntime), XE_ERR_ACCUM_BOUND (the
 * integration would hold more than XE_MAX_SAMPLES_CI32 / _CF32 samples),
 * XE_ERR_ALIGNMENT, XE_ERR_INVALID_ARG, XE_ERR_CUDA.  A rejected call
 * changes neither the accumulator nor the counter.
 */
XE_API xe_status xe_correlate(xe_plan_t plan, const uint8_t *d_gulp, int ntime,
                       int accumulate, void *stream);

/* Emit the accumulator as visibilities into d_vis (layout above, element
 * type = the plan's xe_out).  d_vis must be 8-byte aligned. */
XE_API xe_status xe_integrate(xe_plan_t plan, void *d_vis, void *stream);

/*
 * Several independent correlations in ONE launch: plan k correlates
 * d_gulps[k][ntime[k]][C_k][N_k] into its own accumulator exactly as
 * xe_correlate(plans[k], d_gulps[k], ntime[k], accumulate[k], stream)
 * would, while one persistent grid of CTA pairs works through the
 * concatenated tile-pair units of all problems.  This is how the streaming
 * service batches the gulps of different streams (arrays of different
 * sizes) that are ready at the same time ("Memory management and ring
 * buffers": every reader of a ring processes its own span of data; here
 * several readers share one launch).
 *  - 1 <= n <= 8 distinct plans, all XE_OPERAND_FP8_E4M3 and created on the
 *    current device; each ntime[k] <= 32768 (one launch per problem:
 *    XE_ERR_SHAPE beyond) and within its plan's max_ntime and integration
 *    bounds; the other rules and errors as for xe_correlate.  Nothing is
 *    launched if any problem fails a check.
 *  - Each plan's sample counter and launch count are updated as by
 *    xe_correlate; a device wait that times out is reported by
 *    xe_plan_check of every plan of the batch.
 */
XE_API xe_status xe_correlate_batch(int n, const xe_plan_t *plans, const uint8_t *const *d_gulps,
                                    const int *ntime, const int *accumulate, void *stream);

/* A one-gulp integration in one call (sections "Some included blocks" and
 * "Memory management and ring buffers": correlate, accumulate and emit when
 * the integration is a single gulp): the visibilities of this gulp alone,
 * written by the correlation kernels straight into d_vis, the same values
 * as xe_reset + xe_correlate (accumulate 0) + xe_integrate but without the
 * copy out of the plan's accumulator.  The plan's accumulator and sample
 * count are left untouched.  ci32 plans only (XE_ERR_INVALID_ARG for cf32);
 * d_vis int32 [C][N(N+1)/2][2], 8-byte aligned, caller-owned; d_gulp as for
 * xe_correlate (ntime = 0 zeroes d_vis).  Errors as for xe_correlate.
 * Asynchronous on stream. */
XE_API xe_status xe_correlate_emit(xe_plan_t plan, const uint8_t *d_gulp, int ntime, void *d_vis,
                                   void *stream);

/* Zero the accumulator and the sample counter. */
XE_API xe_status xe_reset(xe_plan_t plan, void *stream);

/* Time samples in the current integration (host-side counter). */
XE_API xe_status xe_samples_integrated(xe_plan_t plan, long long *out);

/*
 * End-to-end call on HOST buffers: copies h_gulp[ntime][n_chan][n_input] to
 * the device, correlates it (accumulate as in xe_correlate), emits the
 * accumulator into h_vis and waits for completion.  Copies and compute are
 * pipelined over time slices on the plan's internal streams.  The device
 * staging buffers are allocated on first use and kept by the plan.
 * Synchronous: returns once h_vis holds the result.
 */
XE_API xe_status xe_correlate_host(xe_plan_t plan, const uint8_t *h_gulp, int ntime,
                            int accumulate, void *h_vis);

/*
 * Allocation-free correlation of one gulp, for callers that cannot allocate
 * device memory: a host framework that owns every device allocation through
 * its own pool, or a real-time stream processor that reserves all of its
 * memory at start-up and must not call cudaMalloc / cudaFree while observing.
 * (The paper has no counterpart: this is a deployment convenience.)
 *
 * Same computation and result as a plan's xe_correlate(accumulate = 0)
 * followed by xe_integrate, on the e4m3 tensor-core path: d_vis receives the
 * visibilities of d_gulp[ntime][n_chan][n_input] (layout and element type as
 * for xe_integrate).  No plan is needed and nothing is allocated: the int32
 * scratch and the device error word live in a fixed 16 MiB + 256 B
 * __device__ array of the library, which every GPU that loads the library
 * keeps until the process exits.
 *  - Limit: n_chan * n_input (n_input + 1) / 2 <= 2^21 complex values;
 *    larger problems return XE_ERR_SHAPE without launching anything.
 *  - ntime as for xe_correlate (XE_ERR_ACCUM_BOUND beyond XE_MAX_SAMPLES_*);
 *    ntime = 0 writes zeros.  Same alignment rules as the plan calls.
 *  - The first call on a device looks up the scratch's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept for the life of the
 *    process: do not use these calls across a cudaDeviceReset.
 *  - Every call shares the scratch and overwrites the integration buffer
 *    before adding to it; calls whose GPU work overlaps, e.g. on different
 *    streams, race on it and must be serialised by the caller.
 *  - Asynchronous on `stream`.  Argument errors and launch failures are
 *    returned at once, as for the plan calls.  A device wait that times out
 *    (XE_ERR_TIMEOUT for a plan, through xe_plan_check) is recorded in the
 *    scratch's error word, which only xe_correlate_noalloc_check reads:
 *    call it once the stream has drained the work, before trusting d_vis.
 */
XE_API xe_status xe_correlate_noalloc(const uint8_t *d_gulp, int ntime, int n_chan,
                                      int n_input, xe_out out_type, void *d_vis,
                                      void *stream);

/*
 * Outcome of the allocation-free calls so far: synchronises `stream`, reads
 * the scratch's error word and clears it.  XE_OK if no device wait of any
 * xe_correlate_noalloc call since the previous check timed out, else
 * XE_ERR_TIMEOUT (the visibilities of those calls are not to be trusted);
 * XE_ERR_CUDA if the synchronisation or the copy fails.  Allocates nothing.
 * (No counterpart in the paper.)
 */
XE_API xe_status xe_correlate_noalloc_check(void *stream);

/* ------------------------------------------------------------------------
 * Gain calibration on emitted visibilities (weighted chi^2 and its adjoint).
 *
 *   r_ij = V_ij - g_i conj(g_j) C_ij   for every channel c and baseline i >= j
 *   chi2 = sum_c sum_{i>=j} w_ij |r_ij|^2           (i = j terms only if include_autos)
 *   grad_k = dchi2/dRe g_k + i dchi2/dIm g_k
 *          = -2 [ sum_{j<=k} w_kj r_kj g_j conj(C_kj) + sum_{i>=k} w_ik conj(r_ik) g_i C_ik ]
 *
 * Layouts (all device memory, interleaved (re, im) float32 pairs): d_g
 * [n_chan][n_input]; d_model (C_ij) and d_vobs (V_ij) [n_chan][n_input *
 * (n_input + 1) / 2] in the visibility layout above; d_w float32 weights in
 * the same layout, or NULL for all ones.  Complex pointers must be 8-byte
 * aligned.  Per-baseline terms are float32; chi^2 is summed in float32 with a
 * compensation term (per thread, per warp and over the warps) and in float64
 * only over the final 8 partial totals; both
 * results are deterministic.  The object owns its scratch (per-CTA chi^2
 * partials and the adjoint's partial sums); calls on one object must not
 * overlap.  Errors: XE_ERR_INVALID_ARG for a NULL handle or required pointer
 * or include_autos not 0/1, XE_ERR_ALIGNMENT for a misaligned pointer,
 * XE_ERR_CUDA if a launch fails; nothing is launched on an error.
 * (The paper's pipelines stop at the correlator; this is the calibration
 * step that consumes its output.)
 * ---------------------------------------------------------------------- */
typedef struct xe_calib *xe_calib_t;

/* n_input in 1..8192, n_chan in 1..2^20; allocates the scratch
 * (about n_chan * n_input * (n_input / 4 + 8) bytes) on the current device. */
XE_API xe_status xe_calib_create(xe_calib_t *out, int n_input, int n_chan);
XE_API xe_status xe_calib_destroy(xe_calib_t calib);

/* *d_chisq (one float64 in device memory) = chi2.  Asynchronous on stream. */
XE_API xe_status xe_calib_chisq(xe_calib_t calib, const float *d_g, const float *d_model,
                                const float *d_vobs, const float *d_w, int include_autos,
                                double *d_chisq, void *stream);

/* d_grad [n_chan][n_input] complex float32 = (*d_scale) * grad, d_scale a
 * float64 in device memory (the incoming gradient of chi2) or NULL for 1. */
XE_API xe_status xe_calib_grad(xe_calib_t calib, const float *d_g, const float *d_model,
                               const float *d_vobs, const float *d_w, int include_autos,
                               const double *d_scale, float *d_grad, void *stream);

/* chi2 and the (unscaled) gradient from one pass over the visibilities: the
 * same results as the two calls above, at half their memory traffic. */
XE_API xe_status xe_calib_chisq_grad(xe_calib_t calib, const float *d_g, const float *d_model,
                                     const float *d_vobs, const float *d_w, int include_autos,
                                     double *d_chisq, float *d_grad, void *stream);

/* d_out[k] = (*d_scale) * d_in[k] for the n_chan * n_input complex float32
 * values of a gradient (d_in == d_out allowed); d_scale a float64 in device
 * memory.  Applies an incoming gradient to a saved unscaled one. */
XE_API xe_status xe_calib_scale(xe_calib_t calib, const float *d_in, const double *d_scale,
                                float *d_out, void *stream);

/* ------------------------------------------------------------------------
 * Streaming service: several independent streams of gulps, each with a
 * device ring, correlated and integrated as the gulps arrive (the paper's
 * ring buffers, gulps, buffer factor and guaranteed / unguaranteed readers,
 * section "Memory management and ring buffers" and "Guarantees").
 *
 * A writer (the capture side) reserves the next slot of a stream's pinned
 * staging ring, fills it with one gulp uint8[gulp_ntime][n_chan][n_input],
 * and commits it with its sequence number (strictly increasing; gaps are
 * gulps that never arrived).  Committed gulps are copied to the device ring
 * in 32 MB pieces, at most 4 in flight per direction with the streams
 * taking turns (whole when the service has one stream); pending gulps whose
 * copies are issued and that are contiguous in the ring are correlated in
 * one launch whenever the stream has fewer than two launches in flight and
 * the GPU fewer than two in all (an idle GPU takes a gulp at once; a busy
 * one lets ready gulps gather).
 * When several e4m3 streams have such runs ready at the same time (each of
 * at most 32768 samples), their runs share ONE launch (xe_correlate_batch)
 * on the service's own CUDA stream, up to 8 streams per launch; each
 * stream's integrations still come out in order and unchanged.  The flag
 * XE_SERVICE_NO_BATCH keeps every launch to one stream.
 * Integration k covers sequence numbers [k G, (k+1) G), G = integrate_gulps;
 * it is emitted when its last gulp has been correlated, when a later gulp is
 * committed, or on flush (which closes the integration holding the gulps
 * committed before it), into one of two pinned output buffers per stream
 * that the consumer gets from xe_service_poll and hands back with
 * xe_service_release.  Ring full: a guaranteed stream makes reserve wait (up
 * to timeout_ms; back-pressure), an unguaranteed one returns XE_ERR_BUSY at
 * once and counts the gulp as skipped.
 *
 * Admission: xe_service_add_stream returns XE_ERR_NOMEM when the stream's
 * device memory (ring + accumulator + visibility buffer + 1 MiB) would take
 * the service above its cap (mem_cap_bytes, or half the free device memory
 * at creation when mem_cap_bytes <= 0).
 *
 * Calls on one service are thread-safe; each stream takes one writer and one
 * consumer.  Errors: XE_ERR_INVALID_ARG (bad handle, id, sizes, sequence
 * number), XE_ERR_ALIGNMENT (n_chan * n_input not a multiple of 16),
 * XE_ERR_ACCUM_BOUND (integrate_gulps * gulp_ntime above the output type's
 * sample bound), XE_ERR_NOMEM, XE_ERR_BUSY, XE_ERR_CUDA (a failed stream
 * keeps returning it; other streams are unaffected).
 * ---------------------------------------------------------------------- */
typedef struct xe_service *xe_service_t;

#define XE_SERVICE_DRYRUN 1  /* host bookkeeping only: no CUDA call, visibilities are zeros */
#define XE_SERVICE_MANUAL 2  /* with DRYRUN: work stays in flight until xe_service_dryrun_complete */
#define XE_SERVICE_NO_BATCH 4 /* every launch serves one stream (no cross-stream launches) */

#define XE_FAULT_LAUNCH 1    /* the stream's next launch fails as a failing CUDA call would */
#define XE_FAULT_DROP_GULP 2 /* the next committed gulp is lost in transit */

typedef struct {
  int n_input, n_chan;
  int gulp_ntime;       /* samples per gulp */
  int ring_gulps;       /* buffer factor: ring size in gulps, 1..1024 */
  int integrate_gulps;  /* gulps per integration */
  int guaranteed;       /* 1: back-pressure on a full ring; 0: skip */
  int operand;          /* xe_operand */
  int out_type;         /* xe_out */
} xe_stream_config;

typedef struct {
  int stream;
  long long index;      /* integration number k */
  long long first_seq;  /* k * integrate_gulps */
  int gulps;            /* gulps correlated into it */
  int skipped;          /* integrate_gulps - gulps */
  long long samples;    /* gulps * gulp_ntime */
  double latency_ms;    /* commit of its last gulp -> visibilities in host memory */
  const void *vis;      /* host [n_chan][n_input (n_input + 1) / 2] ci32 / cf32 pairs, valid until released */
  long long vis_bytes;
  int status;           /* XE_OK or the error that ended it */
} xe_integration;

typedef struct {
  long long committed, skipped_full, dropped, launches, gulps_correlated, integrations, max_batch;
  long long device_bytes, host_bytes;
  int state;            /* XE_OK, or the error that stopped the stream */
  int pending, inflight;
  long long shared_launches;   /* launches this stream shared with other streams */
} xe_stream_stats;

XE_API xe_status xe_service_create(xe_service_t *out, long long mem_cap_bytes, int flags);
XE_API xe_status xe_service_destroy(xe_service_t svc);   /* waits for the stream's work */
XE_API xe_status xe_service_add_stream(xe_service_t svc, const xe_stream_config *cfg, int *stream_id);
/* *h_slot = the next staging slot (gulp bytes, pinned host memory). */
XE_API xe_status xe_service_reserve(xe_service_t svc, int stream, int timeout_ms, void **h_slot);
XE_API xe_status xe_service_commit(xe_service_t svc, int stream, long long seq);
/* reserve + copy from h_gulp + commit */
XE_API xe_status xe_service_submit(xe_service_t svc, int stream, const void *h_gulp, long long seq,
                                   int timeout_ms);
/* Close the current integration even if gulps of it are missing. */
XE_API xe_status xe_service_flush(xe_service_t svc, int stream);
/* The oldest finished integration (XE_ERR_BUSY if none within timeout_ms). */
XE_API xe_status xe_service_poll(xe_service_t svc, int stream, int timeout_ms, xe_integration *out);
XE_API xe_status xe_service_release(xe_service_t svc, int stream, long long index);
XE_API xe_status xe_service_stats(xe_service_t svc, int stream, xe_stream_stats *out);
XE_API xe_status xe_service_inject(xe_service_t svc, int stream, int fault);   /* host-side fault injection */
XE_API xe_status xe_service_dryrun_complete(xe_service_t svc, int stream);   /* -1: every stream */
XE_API const char *xe_service_last_error(xe_service_t svc);

/* Bounded device-side wait (failure detection): one thread waits until
 * *d_flag == expected or timeout_ns (at most 60 s) passes, then writes
 * *d_status = 0 (flag seen) or 1 (timed out) and the kernel ends; the
 * context stays usable either way.  Asynchronous on stream. */
XE_API xe_status xe_wait_flag(const int *d_flag, int expected, long long timeout_ns, int *d_status,
                              void *stream);

/* ------------------------------------------------------------------------
 * Beamformer on 4+4-bit voltages (the DRX pipeline's phase-and-sum GPU
 * beamformer, section "LWA Sevilleta implementation", which works directly
 * on the 4+4-bit samples):  y[t][c][b] = sum_i w[c][b][i] x[t][c][i].
 *
 * d_w: complex64 (interleaved float pairs) weights [n_chan][n_beam][n_input]
 * in device memory; xe_beam_set_weights rounds their real and imaginary
 * parts to float16 (the operand precision) and converts them into the
 * kernel's operand form, held by the object with per-output bias sums: for
 * n_beam <= 16 and n_input <= 512, four e4m3 terms per coefficient after a
 * per-channel power-of-two scale (exact for every coefficient of at least
 * 2^-18 of the channel's largest; others err by less than 2^-28 of it),
 * otherwise float16 tiles.  xe_beam_form reads a gulp
 * uint8[ntime][n_chan][n_input] (same layout as xe_correlate) and writes
 * d_out complex64 [ntime][n_chan][n_beam]; products are accumulated in
 * float32 on the tensor cores.  n_beam in 8..64, a multiple of 8; n_input
 * a multiple of 16 (XE_ERR_ALIGNMENT otherwise); d_gulp and d_out 16-byte
 * aligned.
 * Asynchronous on stream; xe_beam_check reports XE_ERR_TIMEOUT if a bounded
 * device wait gave up.  (The paper gives no beamformer algorithm beyond
 * phase-and-sum; this is its definition.)
 * ---------------------------------------------------------------------- */
typedef struct xe_beam *xe_beam_t;

XE_API xe_status xe_beam_create(xe_beam_t *out, int n_input, int n_chan, int n_beam, int max_ntime);
XE_API xe_status xe_beam_destroy(xe_beam_t beam);
XE_API xe_status xe_beam_set_weights(xe_beam_t beam, const float *d_w, void *stream);
XE_API xe_status xe_beam_form(xe_beam_t beam, const uint8_t *d_gulp, int ntime, float *d_out, void *stream);
XE_API xe_status xe_beam_check(xe_beam_t beam);
XE_API const char *xe_beam_last_error(xe_beam_t beam);

/* Wait for all device work, then report whether any bounded device-side
 * wait of this plan's kernels gave up since the last check
 * (XE_ERR_TIMEOUT; the code is in xe_plan_last_error and is then cleared).
 * In the debug build of the library (libxengine_debug.so, compiled with
 * XE_DEBUG_CHECKS) the X-engine kernels also check every global index they
 * store to against its buffer, skip an access outside it and record it
 * here as XE_ERR_DEVICE_INDEX: the stand-in for a memory checker, without
 * faulting the GPU. */
XE_API xe_status xe_plan_check(xe_plan_t plan);

/* Number of kernel launches this plan has enqueued since creation. */
XE_API xe_status xe_plan_launch_count(xe_plan_t plan, long long *out);

/* Static text for a status code. */
XE_API const char *xe_status_string(xe_status s);

/* Text of the last CUDA error seen by the plan ("" if none).  Valid until
 * the next call on the plan. */
XE_API const char *xe_plan_last_error(xe_plan_t plan);

/* Library version string. */
XE_API const char *xe_version(void);

/* ------------------------------------------------------------------------
 * Measurement aid (no counterpart in the paper): the CUDA cores' dp4a issue
 * rate, the arithmetic ceiling of the plain int32 X-engine
 * (XE_OPERAND_INT32_CUDACORE), which spends one dp4a per complex
 * multiply-accumulate.  Launches `ctas` CTAs of 256 threads; every thread
 * issues iters * 256 dp4a in 8 independent chains on register operands.
 * d_cycles[ctas] (int64) receives each CTA's clock64 cycles, d_sink[ctas *
 * 256] (int32) the threads' sums; *dp4a_per_cta is set on the host.  Launch
 * one CTA per SM (ctas = the SM count; at most one is resident per SM): the
 * rate per SM and clock is then dp4a_per_cta / cycles.  Asynchronous on
 * `stream`; XE_ERR_INVALID_ARG for iters outside 1..2^20, ctas outside
 * 1..2^16 or a NULL pointer.
 * ---------------------------------------------------------------------- */
XE_API xe_status xe_probe_dp4a_rate(int iters, int ctas, long long *d_cycles, int *d_sink,
                                    long long *dp4a_per_cta, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* XENGINE_H */
