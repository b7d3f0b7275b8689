/*
 * sdft.h -- C ABI of the planar split-complex DFT library (libsdft.so) for
 * NVIDIA GB300 (sm_103a).
 *
 * The library computes the batched complex N-point discrete Fourier
 * transform of A. Cariow, "Fast algorithms for complex-valued discrete
 * Fourier transform with separate real and imaginary inputs/outputs"
 * (arXiv 2504.07264), with real and imaginary parts kept in separate
 * (planar) arrays from input to output:
 *
 *   forward  (Eq. (1), split form Eq. (3), block form Eqs. (4)-(5)):
 *     y_k = sum_n x_n exp(-j 2 pi n k / N),
 *     y^r = C x^r + S x^i,   y^i = C x^i - S x^r,
 *     c_{k,n} = cos(2 pi k n / N),  s_{k,n} = sin(2 pi k n / N).
 *   adjoint (the transpose of E_2N of Eq. (5), i.e. the conjugate transpose
 *     of the DFT matrix, the unnormalised inverse DFT):
 *     y^r = C x^r - S x^i,   y^i = S x^r + C x^i.
 *
 * Neither direction normalises (no 1/N): adjoint(forward(x)) = N x.
 *
 * Domain: N = 2^m with 1 <= m <= 16 (Section III takes N = 2^m, m >= 2; the
 * same formulas hold for N = 2).  Other N: SDFT_ERR_UNSUPPORTED_N.
 *
 * Layout: each of xr, xi, yr, yi is a contiguous row-major float32 array of
 * shape [batch][N] in device memory (transform b occupies elements
 * b*N .. b*N+N-1).  Ragged plans use the transforms' rows concatenated in the
 * order given, transform t starting at the exclusive prefix sum of the
 * lengths before it.  The caller owns every buffer.  All four pointers must be
 * 16-byte aligned.  Out-of-place, or fully in-place (yr == xr and yi == xi),
 * are accepted; any other overlap among the four arrays is SDFT_ERR_ALIAS.
 *
 * Arithmetic: dtype SDFT_F32 computes in float32 with twiddle factors
 * computed in float64 and rounded once to float32.  SDFT_F32_SPLIT_BF16 and
 * SDFT_F32_SPLIT_FP16 run the dense radix blocks on tensor cores from hi/lo
 * splits of the data and of the block (three products accumulated in
 * float32); their input and output arrays are still float32.
 *
 * Streams and errors: every compute call is asynchronous on `stream` (a
 * cudaStream_t passed as void*; NULL = the legacy default stream).  Each
 * function returns an sdft status; argument errors are detected on the host
 * before anything is enqueued.  A CUDA launch failure returns SDFT_ERR_CUDA.
 * Calls must be made with the plan's device current (the device current at
 * sdft_plan_create), otherwise SDFT_ERR_INVALID_ARG.
 *
 * Thread safety: a plan is immutable after creation; concurrent calls on one
 * plan from several host threads or streams are safe, with two exceptions:
 * plans on the two-pass CTA schedule of N >= 32768 own one scratch area that
 * every call uses, so their calls must be ordered on one stream; and the
 * *_host calls share the plan's staging buffers, so they must be serialised.
 */
#ifndef SDFT_H_
#define SDFT_H_

#include <stdint.h>

#if defined(__GNUC__)
#define SDFT_API __attribute__((visibility("default")))
#else
#define SDFT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SDFT_OK                    0
#define SDFT_ERR_INVALID_ARG       1  /* null pointer, batch < 1, bad direction, wrong device */
#define SDFT_ERR_UNSUPPORTED_N     2  /* N not a power of two in [2, 65536] */
#define SDFT_ERR_MISALIGNED        3  /* a data pointer not 16-byte aligned */
#define SDFT_ERR_ALIAS             4  /* partial overlap of input and output arrays */
#define SDFT_ERR_BAD_PLAN          5  /* NULL, destroyed or foreign plan handle */
#define SDFT_ERR_CUDA              6  /* a CUDA runtime call failed */
#define SDFT_ERR_ALLOC             7  /* host or device allocation failed */
#define SDFT_ERR_TIMEOUT           8  /* a bounded device-side wait expired */
#define SDFT_ERR_UNSUPPORTED_DTYPE 9  /* unknown dtype, or not offered for this N */

/* ---- arithmetic paths (input/output are always float32 planar) ------- */
#define SDFT_F32             0
#define SDFT_F32_SPLIT_BF16  1
#define SDFT_F32_SPLIT_FP16  2

/* ---- directions -------------------------------------------------------- */
#define SDFT_FORWARD 0   /* Eq. (1): E_2N of Eq. (5) */
#define SDFT_ADJOINT 1   /* transpose of E_2N */

typedef struct sdft_plan sdft_plan;

/* Create a plan for `batch` transforms of length `n` (Section III: n = 2^m).
 * Allocates the plan's device twiddle tables on the current device and
 * synchronises that device once.  Returns NULL on error; sdft_last_error()
 * then gives the status (SDFT_ERR_UNSUPPORTED_N, SDFT_ERR_INVALID_ARG,
 * SDFT_ERR_UNSUPPORTED_DTYPE, SDFT_ERR_ALLOC, SDFT_ERR_CUDA). */
SDFT_API sdft_plan* sdft_plan_create(int64_t n, int64_t batch, int dtype);

/* Create a plan for a ragged batch: `count` transforms whose lengths
 * lengths[0..count-1] (host array, read during the call only) are each a
 * power of two in [4, 65536].  Rows are concatenated in the order given.
 * Forward and adjoint calls on such a plan run as one persistent kernel
 * launch (thread-block clusters of 8 CTAs, replayed from a CUDA graph) that
 * claims work from device queues, largest transforms first.  Every length
 * runs one of its compiled forms (see sdft_ragged_form_count): a transform of
 * N >= 8192 may be held in the distributed shared memory of 8, 4 or 2 CTAs,
 * a shorter one (and N = 8192 in its row form) runs in a tile of one CTA.  The
 * plan starts with the forms selected by sdft_ragged_form_select (form 0 if
 * none) and allocates the twiddle tables of every form of its lengths.
 * Returns NULL on error (see sdft_last_error). */
SDFT_API sdft_plan* sdft_plan_create_ragged(const int64_t* lengths, int64_t count, int dtype);

/* Release a plan and its device memory.  NULL is ignored.  The caller must
 * ensure no work using the plan is still in flight. */
SDFT_API void sdft_plan_destroy(sdft_plan* plan);

/* Forward transform (Eq. (1)/(3)) of every row: [yr; yi] = E_2N [xr; xi].
 * xr, xi: input planes (device, float32, read only);
 * yr, yi: output planes (device, float32, written);
 * stream: cudaStream_t, or NULL.  Returns SDFT_OK or an error status. */
SDFT_API int sdft_forward(const sdft_plan* plan, const float* xr, const float* xi,
                 float* yr, float* yi, void* stream);

/* Adjoint transform of every row: [yr; yi] = E_2N^T [xr; xi]
 * (conjugate-transpose DFT, unnormalised).  Same arguments as sdft_forward. */
SDFT_API int sdft_adjoint(const sdft_plan* plan, const float* xr, const float* xi,
                 float* yr, float* yi, void* stream);

/* Either direction (SDFT_FORWARD or SDFT_ADJOINT) through one entry point. */
SDFT_API int sdft_execute(const sdft_plan* plan, int direction, const float* xr, const float* xi,
                 float* yr, float* yi, void* stream);

/* The same transform on HOST buffers; returns after the result is in yr, yi.
 * Two ways, chosen by sdft_plan_set_host_mode:
 *   zero copy (default when all four buffers are page-locked host memory the
 *     GPU can address, e.g. from cudaHostAlloc): the kernel reads xr, xi and
 *     writes yr, yi directly over the CPU-GPU link, on `stream`;
 *   staged (otherwise): xr, xi are copied to plan-owned device staging
 *     buffers, transformed, and copied back, in chunks pipelined over the
 *     plan's two internal streams, ordered after prior work on `stream`.  The
 *     staging buffers (two chunks of ~32 MiB per plane, not the whole batch)
 *     are allocated by the first staged call on a plan. */
SDFT_API int sdft_execute_host(sdft_plan* plan, int direction, const float* xr, const float* xi,
                      float* yr, float* yi, void* stream);

#define SDFT_HOST_AUTO      0   /* zero copy if every buffer is page-locked, else staged */
#define SDFT_HOST_STAGED    1   /* always staged */
#define SDFT_HOST_ZERO_COPY 2   /* always zero copy (SDFT_ERR_INVALID_ARG if impossible) */
/* Choose how sdft_execute_host moves data (default SDFT_HOST_AUTO). */
SDFT_API int sdft_plan_set_host_mode(sdft_plan* plan, int mode);

/* Launch grid (CTAs) of a uniform plan's kernel.  The default is the
 * kernel's occupancy times the SM count (for cluster kernels: the clusters
 * that fit at once, times their size); a persistent grid-stride loop makes
 * any grid >= 1 correct (cluster kernels round it down to whole clusters, at
 * least one).  Plans whose kernel owns per-CTA scratch and work-queue plans
 * keep their grid: SDFT_ERR_INVALID_ARG. */
SDFT_API int sdft_plan_set_grid(sdft_plan* plan, int grid);
SDFT_API int sdft_plan_grid(const sdft_plan* plan);

/* Bound of the device-side waits of a work-queue plan (ragged plans, and
 * uniform plans on a work-queue schedule).  Their kernel needs no waits to
 * compute; the only one is the wait added by the testing hook below.  Every such wait polls at most `polls` times (default 2^23); past
 * that the kernel records SDFT_ERR_TIMEOUT in the status word, stops waiting
 * anywhere and carries on (the results of that call are then undefined).  The status stays set, and later
 * calls skip their waits too, until sdft_plan_sync_status reads and clears it.
 * SDFT_ERR_INVALID_ARG for other plans or polls < 1. */
SDFT_API int sdft_plan_set_wait_limit(sdft_plan* plan, int polls);
/* Testing hook: make every transform a work-queue plan holds in the shared
 * memory of several CTAs first wait for a device word that nothing sets
 * (on != 0), or not (on == 0), so that the bounded-wait path can be exercised
 * without any fault on the GPU.  SDFT_ERR_INVALID_ARG for plans with no such
 * transform under their current forms. */
SDFT_API int sdft_plan_inject_unreachable_wait(sdft_plan* plan, int on);

/* ---- forms of the work-queue kernel (ragged plans) ----------------------
 * Each length N = 4 .. 65536 has one or more compiled forms in the persistent
 * kernel of ragged plans: the radix split, values per thread and transforms
 * per tile of a one-CTA row tile, or the number of CTAs (8, 4, 2) whose shared
 * memory holds one transform of N >= 8192.  Every form computes the same
 * transform (results agree within rounding).  Functions returning a count or
 * index return a negative status on error. */
/* Number of forms of length n (SDFT_ERR_UNSUPPORTED_N outside 4 .. 65536). */
SDFT_API int sdft_ragged_form_count(int64_t n);
/* Describe form `form` of length n into buf (snprintf convention). */
SDFT_API int sdft_ragged_form_describe(int64_t n, int form, char* buf, int64_t len);
/* Process-wide choice of the form of length n for work-queue plans created
 * later (SDFT_OK, or SDFT_ERR_INVALID_ARG / SDFT_ERR_UNSUPPORTED_N). */
SDFT_API int sdft_ragged_form_select(int64_t n, int form);
SDFT_API int sdft_ragged_form_selected(int64_t n);
/* Run length n of a work-queue plan (ragged plans, and uniform plans on a
 * work-queue schedule) in form `form`: rebuilds the plan's work items and
 * synchronises the device.  No work using the plan may be in flight.
 * SDFT_ERR_INVALID_ARG for other plans, lengths the plan does not hold, or an
 * unknown form. */
SDFT_API int sdft_plan_set_ragged_form(sdft_plan* plan, int64_t n, int form);
/* The form length n runs in on this plan (>= 0), or -status. */
SDFT_API int sdft_plan_ragged_form(const sdft_plan* plan, int64_t n);
/* Host-only view of the work a ragged plan of these lengths (as for
 * sdft_plan_create_ragged) would run with the process-wide forms, without
 * touching any GPU: for every transform t, phase_of[t] (0, 1, 2: a transform
 * held by 8, 4 or 2 CTAs; 3: a row tile) and item_of[t] (its work item within
 * that phase); nitems[0..3] receives the number of items of each phase.  Items
 * of a phase are ordered longest transforms first; a group item holds one
 * transform, a row tile up to the form's transforms per tile, all of one
 * length.  phase_of and item_of have room for `count` entries.  Returns
 * SDFT_OK, SDFT_ERR_INVALID_ARG or SDFT_ERR_UNSUPPORTED_N. */
SDFT_API int sdft_ragged_work_layout(const int64_t* lengths, int64_t count, int32_t* phase_of,
                                     int32_t* item_of, int64_t* nitems);
/* Autotune a work-queue plan on the caller's device buffers (the plan's
 * layout, read xr/xi, written yr/yi): one length at a time, longest first,
 * time the plan's forward call with each form of that length (`reps` timed
 * calls per trial after one untimed call, CUDA events on `stream`) and keep
 * another form only where it is faster by more than 1 %.  Rebuilds the work
 * items between trials, so it synchronises the device.  Leaves the chosen
 * forms set and returns a mask with bit l set for every length 2^l that runs
 * a form other than form 0 (>= 0), or -status. */
SDFT_API int sdft_plan_ragged_autotune(sdft_plan* plan, const float* xr, const float* xi,
                                       float* yr, float* yi, int reps, void* stream);

/* Wait for `stream`, then read and clear the plan's device status word:
 * SDFT_OK, or SDFT_ERR_TIMEOUT if a bounded device-side wait gave up. */
SDFT_API int sdft_plan_sync_status(const sdft_plan* plan, void* stream);

/* ---- schedules and autotuning ------------------------------------------- */
/* Each length has one or more compiled schedules (radix split, threads per
 * transform, transforms per CTA, register-DFT order).  sdft_plan_create uses
 * the schedule currently selected for its length (index 0 until something is
 * selected); the selection is process-wide and affects plans created later.
 * Functions returning a count or index return a negative status on error. */
SDFT_API int sdft_schedule_count(int64_t n, int dtype);
/* Describe schedule `index` of length n into buf (snprintf convention). */
SDFT_API int sdft_schedule_describe(int64_t n, int dtype, int index, char* buf, int64_t len);
/* Select schedule `index` for length n (SDFT_OK, or SDFT_ERR_INVALID_ARG). */
SDFT_API int sdft_schedule_select(int64_t n, int dtype, int index);
SDFT_API int sdft_schedule_selected(int64_t n, int dtype);
/* Time every schedule of length n on the caller's device buffers (`batch`
 * transforms, forward, `reps` timed launches after two warm-up launches, CUDA
 * events on `stream`), write the mean milliseconds per launch of schedule i to
 * ms_out[i] (may be NULL; room for sdft_schedule_count entries), select the
 * fastest and return its index.  Creates and destroys one temporary plan per
 * schedule, so it allocates device memory and synchronises `stream`. */
SDFT_API int sdft_autotune(int64_t n, int64_t batch, int dtype, const float* xr, const float* xi,
                           float* yr, float* yi, int reps, float* ms_out, void* stream);

/* ---- allocation-free long transforms ---------------------------------- */
/* The paper has no counterpart to this entry point.
 * For callers that cannot allocate device memory (their memory is owned by
 * another allocator or capped, or they must avoid the synchronisation that
 * cudaMalloc/cudaFree can cause): transform `batch` rows of length n = 32768
 * or 65536 -- the lengths whose kernel needs global scratch -- without a plan
 * and without any allocation.  Scratch and twiddle tables live in file-scope
 * device arrays of libsdft.so that every GPU loading the library holds until
 * the process exits; the scratch is 8 MiB (16 slots of 65536 or 32 of 32768
 * complex values).  Arguments as sdft_execute; n other than 32768 or 65536:
 * SDFT_ERR_UNSUPPORTED_N.  The first call on a device sets up that device
 * (resolves the arrays, fills the tables, synchronises the device): make it
 * before any stream capture.  All calls share the arrays, so calls that
 * overlap on the GPU race; order them on one stream. */
SDFT_API int sdft_execute_noalloc(int64_t n, int64_t batch, int direction, const float* xr,
                                  const float* xi, float* yr, float* yi, void* stream);

/* ---- introspection ----------------------------------------------------- */
SDFT_API int64_t sdft_plan_n(const sdft_plan* plan);        /* N, or 0 for ragged plans */
SDFT_API int64_t sdft_plan_batch(const sdft_plan* plan);    /* number of transforms */
SDFT_API int64_t sdft_plan_points(const sdft_plan* plan);   /* total complex points per call */
SDFT_API int     sdft_plan_dtype(const sdft_plan* plan);
/* Kernel launches one sdft_forward/sdft_adjoint call makes. */
SDFT_API int     sdft_plan_launches(const sdft_plan* plan, int direction);
/* Human-readable schedule (radices, threads, I/O mode) into buf; returns the
 * full length, like snprintf. */
SDFT_API int     sdft_plan_describe(const sdft_plan* plan, char* buf, int64_t len);

/* ---- errors ------------------------------------------------------------ */
/* Status of the last failing call on this host thread (SDFT_OK if none). */
SDFT_API int         sdft_last_error(void);
/* Static English description of a status code. */
SDFT_API const char* sdft_status_string(int status);
/* Library version, "major.minor.patch". */
SDFT_API const char* sdft_version(void);

#ifdef __cplusplus
}  /* extern "C" */
#endif

#endif  /* SDFT_H_ */
