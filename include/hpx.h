/*
 * hpx.h -- C ABI of libhpx: spherical harmonic transforms on RING-ordered
 * HEALPix grids, computed on one NVIDIA GB300 (sm_103a).
 *
 * Method: arXiv 2510.01785 (cuHPX).  Every transform is a per-ring Fourier
 * step over the variable-length rings followed by a Legendre step over the
 * rings (Sec. III-D, Eq. 12-14):
 *
 *   synthesis  p = Y a          p_xy = sum_m sum_l a_lm lambda_lm(theta_y)
 *                                      exp(i m phi_{0,y} + 2 pi i m x / N_y)
 *                                                              (Eq. 24-25)
 *   analysis   a = Y^dagger W p a_lm = sum_y sum_x p_xy w_y lambda_lm(theta_y)
 *                                      exp(-i m phi_{0,y} - 2 pi i m x / N_y)
 *                                                              (Eq. 26-27)
 *   adjoints   adjoint of synthesis = Y^dagger,
 *              adjoint of analysis  = W Y               (Sec. III-F)
 *
 * with lambda_lm the orthonormal associated Legendre functions including the
 * Condon-Shortley phase (Eq. 8, 15), generated by the three-term recurrence
 * in l (Eq. 16) in FP64, and equal-area weights w_y = 4 pi / Npix (Eq. 1).
 *
 * Data layout (all device buffers are owned by the caller):
 *   map : [nbatch][12 nside^2] real, RING order (rings north to south,
 *         pixels by increasing phi), contiguous.
 *   alm : [nbatch][nalm] complex, interleaved (re, im), packed m-major:
 *         index(l, m) = m (2 lmax + 1 - m) / 2 + l for 0 <= m <= mmax,
 *         m <= l <= lmax; nalm = hpx_nalm(lmax, mmax).  Only m >= 0 is
 *         stored: the fields are real, so a_{l,-m} = (-1)^m conj(a_lm).
 *         Synthesis reads Re(a_l0) only; analysis writes Im(a_l0) = 0.
 *   real type: double for HPX_F64, float for every other dtype.
 * Pointers must be 16-byte aligned; map and alm must not overlap.
 *
 * Calls are asynchronous and ordered on the stream passed in (NULL = the
 * legacy default stream).  From Nside 512 a ring-transform stage forks part
 * of its kernels onto a plan-owned second stream (one for analyses, one for
 * syntheses) and joins it back before the call's next work on the caller's
 * stream, so the call stays ordered there and a stream capture records the
 * fork and the join.  A plan owns device workspace: one part for its
 * analyses (hpx_map2alm, hpx_alm2map_adjoint, hpx_map2alm_n) and one for
 * its syntheses (hpx_alm2map, hpx_map2alm_adjoint, hpx_alm2map_n).  So one
 * analysis and one synthesis may run at the same time on two streams
 * (issued from one host thread);
 * two analyses, two syntheses, the host-buffer calls, hpx_map2alm_iter and
 * every call on an out-of-core plan must be ordered by the caller, or use
 * one plan per stream.  The device-buffer transforms of a resident plan
 * (hpx_map2alm, hpx_alm2map, their adjoints, gradients and _n forms)
 * allocate nothing and never wait on the host, so a stream capture may
 * record them into a CUDA graph after one call outside the capture; the
 * replays give the same results.
 *
 * Errors: every call returns an hpx_status; on failure hpx_last_error()
 * returns a message for the calling thread.  No exception crosses the ABI.
 */
#ifndef HPX_H
#define HPX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t / CUstream); declared here so the header needs
 * no CUDA include. */
struct CUstream_st;
typedef struct CUstream_st* hpx_stream_t;

typedef struct hpx_plan_s* hpx_plan;

/* I/O precision and contraction mode.
 *   HPX_F64        double maps/coefficients, FP64 contraction.
 *   HPX_F32        float maps/coefficients, FP32 contraction; lambda_lm still
 *                  comes from the FP64 recurrence.
 *   HPX_F32_BF16 / HPX_F32_FP16     float I/O (ring transforms in FP32);
 *                  both Legendre stages on tensor cores from plan-resident
 *                  BF16 / FP16 lambda tables (rounded from the FP64
 *                  recurrence) and BF16 / FP16 operands, FP32 accumulation.
 *                  FP16 operands are scaled per channel by a power of two
 *                  (from the largest component of the channel's spectra or
 *                  coefficients) to stay in range; the scale is undone on
 *                  output.
 *   HPX_F32_BF16X3 / HPX_F32_FP16X3 the same with split products: every
 *                  value is stored as hi + lo (lo = the remainder rounded
 *                  again) and hi*hi + hi*lo + lo*hi are accumulated.
 * The four 16-bit dtypes always build their tables and use the tensor-core
 * path (HPX_PLAN_LAMBDA_TABLE | HPX_PLAN_TENSOR_CORES are implied). */
typedef enum {
  HPX_F64 = 0,
  HPX_F32 = 1,
  HPX_F32_BF16 = 2,
  HPX_F32_BF16X3 = 3,
  HPX_F32_FP16 = 4,
  HPX_F32_FP16X3 = 5
} hpx_dtype;

typedef enum {
  HPX_OK = 0,
  HPX_ERR_INVALID = 1,     /* bad argument (plan parameters, pointer, size) */
  HPX_ERR_NOMEM = 2,       /* device allocation failed */
  HPX_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  HPX_ERR_TIMEOUT = 4,     /* a bounded device-side wait expired */
  HPX_ERR_UNSUPPORTED = 5  /* valid request this build does not provide */
} hpx_status;

/* Plan flags for hpx_plan_create_ex. */
#define HPX_PLAN_LAMBDA_RECOMPUTE 0u /* lambda_lm recomputed by the FP64
                                        recurrence inside every transform */
#define HPX_PLAN_LAMBDA_TABLE 1u     /* lambda_lm generated once at plan time
                                        by the same FP64 recurrence and kept
                                        in device memory (the precomputed
                                        Legendre tensor of Sec. III-D/III-G);
                                        results are identical to the
                                        recomputing plan.  Costs one value of
                                        the real type per significant
                                        (l, m, ring pair), about 30 GB in
                                        float at nside 1024, lmax 3071. */
#define HPX_PLAN_TENSOR_CORES 2u     /* with HPX_PLAN_LAMBDA_TABLE on an
                                        HPX_F32 plan: both Legendre stages
                                        (Eq. 24-27) run as tensor-core
                                        matrix products (tcgen05), fed by TMA
                                        from the table and from a second,
                                        transposed copy of it made at plan
                                        time (about twice the table memory).
                                        FP32 accuracy from split products:
                                        every table value and operand is
                                        stored as an FP16 pair hi + lo (4
                                        bytes, as a float; the operands per
                                        channel scaled by a power of two into
                                        FP16 range) and each term is
                                        hi*hi + hi*lo + lo*hi with FP32
                                        accumulation.  Results agree with
                                        the CUDA-core path to FP32 rounding,
                                        not bit for bit.  Other dtypes or a
                                        missing table flag: HPX_ERR_INVALID. */
#define HPX_PLAN_TC_TF32X3 8u        /* with HPX_PLAN_TENSOR_CORES: the
                                        products from TF32 splits instead
                                        ("3xTF32": the FP32 table, read as
                                        TF32 hi, with the TF32 remainders
                                        formed in the kernel); slower, kept
                                        for comparison. */

#define HPX_PLAN_LAMBDA_HOST 4u      /* with the tensor-core path: both
                                        lambda tables live in pinned host
                                        memory (out of core, Sec. III-G) and
                                        every transform streams them, block
                                        of m by block, through two device
                                        staging buffers, copies overlapped
                                        with the tile kernels.  For tables
                                        larger than HBM.  Same results as
                                        the resident plan. */
#define HPX_PLAN_LAMBDA_STREAM 16u   /* with the tensor-core path: no table
                                        is kept; every transform recomputes
                                        lambda by the FP64 recurrence (Eq.
                                        15-16), block of m by block, into two
                                        device staging buffers on a second
                                        stream, and each block is contracted
                                        on the tensor cores once it is
                                        filled, while the recurrence fills
                                        the other buffer.  One recurrence
                                        serves all channels of the transform,
                                        so the cost hardly grows with nbatch.
                                        Same results as the resident plan
                                        (the same fill kernels).  Not with
                                        HPX_PLAN_LAMBDA_HOST. */

/* Number of packed coefficients for (lmax, mmax). */
int64_t hpx_nalm(int lmax, int mmax);

/* Create a plan on the current CUDA device.
 *   nside  : HEALPix resolution, a power of two, 1 <= nside <= 2048
 *            (Sec. III-A: Npix = 12 nside^2, 4 nside - 1 rings).
 *   lmax, mmax : band limits, 0 <= mmax <= lmax <= 16384.
 *   nbatch : number of independent channels per call, 1 <= nbatch <= 65535.
 *   dtype  : see hpx_dtype.
 * Builds the ring-geometry table, the recurrence coefficients, the starting
 * state of every (m, ring) recurrence chain and the FFT tables on the device;
 * returns once they are complete.  *out receives the plan.
 * Errors: HPX_ERR_INVALID, HPX_ERR_NOMEM, HPX_ERR_CUDA, HPX_ERR_UNSUPPORTED. */
hpx_status hpx_plan_create(int nside, int lmax, int mmax, int nbatch,
                           hpx_dtype dtype, hpx_plan* out);

/* As hpx_plan_create, with HPX_PLAN_* flags. */
hpx_status hpx_plan_create_ex(int nside, int lmax, int mmax, int nbatch,
                              hpx_dtype dtype, unsigned flags, hpx_plan* out);

/* An out-of-core tensor-core plan (HPX_PLAN_LAMBDA_TABLE |
 * HPX_PLAN_TENSOR_CORES | HPX_PLAN_LAMBDA_HOST) whose two device staging
 * buffers hold stage_bytes per table part (hi, and lo for the x3 dtypes);
 * 0 selects 1 GiB, or the larger table part where that is smaller.  dtype: HPX_F32 or a 16-bit dtype.  The tables are built
 * on the device block by block and copied to pinned host memory
 * (hpx_plan_host_bytes).  HPX_ERR_INVALID if one m's table slice does not
 * fit a staging buffer. */
hpx_status hpx_plan_create_ooc(int nside, int lmax, int mmax, int nbatch,
                               hpx_dtype dtype, size_t stage_bytes,
                               hpx_plan* out);

/* A streamed tensor-core plan (HPX_PLAN_LAMBDA_TABLE |
 * HPX_PLAN_TENSOR_CORES | HPX_PLAN_LAMBDA_STREAM, plus `flags`: 0 or
 * HPX_PLAN_TC_TF32X3 for an HPX_F32 plan) whose two device staging buffers
 * hold stage_bytes per table part (hi, and lo for the x3 dtypes); 0 selects
 * 1 GiB, or the larger table part where that is smaller.  dtype: HPX_F32 or a 16-bit dtype.  No table is built at plan
 * time.  HPX_ERR_INVALID for other flags or if one m's table slice does not
 * fit a staging buffer. */
hpx_status hpx_plan_create_stream(int nside, int lmax, int mmax, int nbatch,
                                  hpx_dtype dtype, unsigned flags,
                                  size_t stage_bytes, hpx_plan* out);

/* Pinned host bytes of an out-of-core plan's tables (0 otherwise). */
size_t hpx_plan_host_bytes(hpx_plan plan);

/* Release the plan and all device memory it owns (after synchronising its
 * device).  NULL is accepted. */
hpx_status hpx_plan_destroy(hpx_plan plan);

/* a = Y^dagger W p: analysis, Eq. 26-27 with w_y = 4 pi / Npix (Eq. 1).
 *   map : device, [nbatch][npix] real (input).
 *   alm : device, [nbatch][nalm] complex (output, fully overwritten). */
hpx_status hpx_map2alm(hpx_plan plan, const void* map, void* alm,
                       hpx_stream_t stream);

/* p = Y a: synthesis, Eq. 24-25.
 *   alm : device, [nbatch][nalm] complex (input).
 *   map : device, [nbatch][npix] real (output, fully overwritten). */
hpx_status hpx_alm2map(hpx_plan plan, const void* alm, void* map,
                       hpx_stream_t stream);

/* p = W Y a: adjoint of the analysis (Sec. III-F), i.e. the synthesis with
 * every ring scaled by its weight.  Adjoint with respect to the real inner
 * product <a, b> = sum_l Re(conj a_l0 b_l0) + 2 sum_{m>=1} Re(conj a_lm b_lm)
 * on coefficients and the plain dot product on maps.
 *   alm : device input; map : device output. */
hpx_status hpx_map2alm_adjoint(hpx_plan plan, const void* alm, void* map,
                               hpx_stream_t stream);

/* a = Y^dagger p: adjoint of the synthesis (Sec. III-F), i.e. the analysis
 * sum with unit weights (same inner products as above).
 *   map : device input; alm : device output. */
hpx_status hpx_alm2map_adjoint(hpx_plan plan, const void* map, void* alm,
                               hpx_stream_t stream);

/* hpx_map2alm / hpx_alm2map on the first n channels only (1 <= n <= nbatch):
 * buffers hold n channels in the same layout.  Lets one plan serve batches
 * of varying size (continuous batching of requests). */
hpx_status hpx_map2alm_n(hpx_plan plan, int n, const void* map, void* alm,
                         hpx_stream_t stream);
hpx_status hpx_alm2map_n(hpx_plan plan, int n, const void* alm, void* map,
                         hpx_stream_t stream);

/* Gradients for automatic differentiation (Sec. III-F, IV-C).  The
 * coefficients are the real parameters (Re a_lm, Im a_lm) of a real field,
 * and a coefficient gradient holds dL/dRe + i dL/dIm (PyTorch's convention
 * for complex tensors).  With D = 1 for m = 0 and 2 for m >= 1:
 *   hpx_alm2map_grad:  grad_alm = D Y^dagger grad_map   (backward of
 *                      hpx_alm2map; Im of the m = 0 entries is 0, since the
 *                      synthesis reads Re a_l0 only);
 *   hpx_map2alm_grad:  grad_map = W Y D^-1 grad_alm     (backward of
 *                      hpx_map2alm; reads Re of the m = 0 entries).
 * lambda_lm is recomputed (or read from the plan's table), never stored by
 * the forward call.  Same layouts and stream semantics as the transforms. */
hpx_status hpx_alm2map_grad(hpx_plan plan, const void* grad_map, void* grad_alm,
                            hpx_stream_t stream);
hpx_status hpx_map2alm_grad(hpx_plan plan, const void* grad_alm, void* grad_map,
                            hpx_stream_t stream);

/* Pipelined host-buffer forms: the same transforms, queued without waiting.
 * The input is uploaded on a plan-owned host-to-device stream into one of
 * two plan-owned I/O slots (alternating per call; a slot is reused once its
 * previous result has been downloaded), the transform runs on `stream`
 * after the upload, and the result is downloaded on a plan-owned
 * device-to-host stream.  Consecutive calls thus overlap one call's copies
 * with the neighbouring calls' kernels.  host buffers: pinned, left
 * untouched (input) or unread (output) until hpx_plan_host_sync returns.
 * The slots (two map- and two alm-sized device buffers) are allocated on
 * the first call and counted by hpx_plan_device_bytes. */
hpx_status hpx_map2alm_host_async(hpx_plan plan, const void* host_map,
                                  void* host_alm, hpx_stream_t stream);
hpx_status hpx_alm2map_host_async(hpx_plan plan, const void* host_alm,
                                  void* host_map, hpx_stream_t stream);
/* Waits for every pipelined call's download (and reports the plan's
 * device-side wait status, as hpx_plan_device_status does). */
hpx_status hpx_plan_host_sync(hpx_plan plan);

/* Analysis with iterative refinement (Sec. II-A Eq. 4): a^0 = A f, then
 * niter times r = f - S a^k, a^{k+1} = a^k + A r, with A = map2alm and S =
 * alm2map of this plan.  Each step reduces the residual of a band-limited
 * map; the cost is (1 + 2 niter) transforms.
 *   map : device, [nbatch][npix] real (input f).
 *   alm : device, [nbatch][nalm] complex (output a^niter).
 *   niter : 0 .. 1000 (0: plain hpx_map2alm).
 * A map-sized and an alm-sized plan-owned buffer are allocated on the first
 * call with niter > 0 and counted by hpx_plan_device_bytes.  Same stream
 * semantics as the transforms. */
hpx_status hpx_map2alm_iter(hpx_plan plan, const void* map, void* alm, int niter,
                            hpx_stream_t stream);

/* Host-buffer forms of the two transforms: copy the input from host memory
 * (pinned or pageable) into plan-owned device buffers, run the transform on
 * the stream, copy the result back and wait for the stream.  The device I/O
 * buffers are allocated on the first such call and counted by
 * hpx_plan_device_bytes. */
hpx_status hpx_map2alm_host(hpx_plan plan, const void* host_map,
                            void* host_alm, hpx_stream_t stream);
hpx_status hpx_alm2map_host(hpx_plan plan, const void* host_alm,
                            void* host_map, hpx_stream_t stream);

/* a = Y^dagger W p, like hpx_map2alm, for callers that must not allocate
 * device memory when they transform (their device memory is owned by another
 * allocator or pool, or their loop cannot risk the device-wide
 * synchronisation that cudaMalloc / cudaFree may cause).  The paper has no
 * counterpart: this is a deployment variant of the same kernels.
 *   The intermediate ring spectra live in one fixed 16 MiB device array
 *   compiled into the library (held on every GPU where it was used, until
 *   the process exits) instead of the plan's workspace.  Plans needing
 *   more than 16 MiB of spectra (nbatch * (6 nside^2 + 4 nside - 1) complex
 *   values) get HPX_ERR_INVALID.
 *   The first call on a device (and the first after its context was reset)
 *   looks up the array's device address (cudaGetSymbolAddress) with that
 *   device current.  Under lazy module loading, the CUDA default, that
 *   lookup also loads the array, which may allocate and synchronise once:
 *   make the first call during set-up, outside the loop that must not
 *   allocate, and before any stream capture.  Later calls allocate nothing.
 *   All calls share the array: calls whose work overlaps on the GPU race and
 *   must be ordered by the caller.  Nothing in it needs to start at zero.
 *   The Legendre stage runs on the CUDA cores: on the plan's table if it
 *   holds one in the plan's real type, else recomputing lambda (FP32 plans
 *   with the FP16-split tensor-core tables).  16-bit dtypes:
 *   HPX_ERR_UNSUPPORTED.
 *   map : device input [nbatch][npix]; alm : device output [nbatch][nalm]. */
hpx_status hpx_map2alm_noalloc(hpx_plan plan, const void* map, void* alm,
                               hpx_stream_t stream);

/* Device bytes held by the plan (tables + workspace), for admission control. */
size_t hpx_plan_device_bytes(hpx_plan plan);

/* Copy the plan's ring-geometry table to host arrays of length 4 nside - 1:
 * first pixel, pixel count N_y, z = cos(theta_y), sin(theta_y) and the
 * half-pixel shift sigma_y (phi_{0,y} = sigma_y pi / N_y).  Synchronous. */
hpx_status hpx_plan_ring_table(hpx_plan plan, int64_t* start, int32_t* nphi,
                               double* z, double* sinth, int32_t* sigma);

/* Stage timing.  While enabled, every transform on the plan records a pair of
 * CUDA events on its stream around each stage: 0 ring analysis FFT, 1
 * Legendre analysis, 2 Legendre synthesis, 3 ring synthesis FFT, 4 and 5
 * the operand packs of the tensor-core analysis and synthesis
 * (HPX_PLAN_TENSOR_CORES plans only).  hpx_plan_stage_times waits for the
 * recorded events, adds their elapsed times (ms) and kernel launch counts
 * into ms[6] and launches[6] (either may be NULL), and clears the record.
 * Measurement support, not part of the transform. */
hpx_status hpx_plan_set_timing(hpx_plan plan, int enable);
hpx_status hpx_plan_stage_times(hpx_plan plan, double* ms, int64_t* launches);

/* Work of the Legendre stage per channel: *total = number of (l, m, ring
 * pair) triples, nalm * 2 nside; *active = triples from each chain's first
 * significant l on (the recurrence steps the kernels execute per chain).
 * Synchronous. */
hpx_status hpx_plan_chain_stats(hpx_plan plan, int64_t* active, int64_t* total);

/* Device bytes hpx_plan_create_ex would allocate for these arguments (an
 * upper bound for the lambda table), without allocating or touching the GPU;
 * 0 for invalid arguments.  For admission control. */
size_t hpx_plan_estimate_bytes(int nside, int lmax, int mmax, int nbatch,
                               hpx_dtype dtype, unsigned flags);

/* Bytes of the plan-resident lambda table (0 without HPX_PLAN_LAMBDA_TABLE);
 * hi and lo parts together for the x3 dtypes. */
size_t hpx_plan_table_bytes(hpx_plan plan);

/* Bytes of the transposed copy of the table the tensor-core synthesis reads
 * (0 without the tensor-core path). */
size_t hpx_plan_column_table_bytes(hpx_plan plan);

/* Per-ring quadrature weights (Sec. IV-A; NEXT to Eq. 1's equal 4 pi/Npix):
 * w[y] for the 4 nside - 1 rings, north to south (host array, copied).
 * Replaces the weight every later hpx_map2alm / hpx_map2alm_adjoint /
 * hpx_map2alm_grad of this plan applies to ring y (the unweighted operators
 * are unaffected).  Synchronises the device.  Pixel weights are applied by
 * weighting the map and calling hpx_alm2map_adjoint.
 * Errors: HPX_ERR_INVALID (count differs from the ring count, a weight not
 * finite). */
hpx_status hpx_plan_set_ring_weights(hpx_plan plan, const double* w, int n);

/* Status of the plan's device-side waits.  Synchronises the plan's device,
 * returns HPX_ERR_TIMEOUT if a bounded wait inside one of the plan's kernels
 * expired since the last call (that transform's output is incomplete) and
 * clears the record; HPX_OK otherwise.  The host-buffer entry points check
 * it themselves. */
hpx_status hpx_plan_device_status(hpx_plan plan);

/* Test support for the bounded waits (no counterpart in the paper).  While
 * withhold is nonzero, the tensor-core tile kernels of the plan's transforms
 * issue none of their copies, so the first wait of each CTA for a copy runs
 * out after its limit (1 s), with no copy or product in flight; the CTA
 * frees its tensor memory, writes no output and records HPX_ERR_TIMEOUT,
 * which the next hpx_plan_device_status returns.  Transforms that have no
 * tile kernel (CUDA-core plans) are unaffected.  0 restores normal work. */
hpx_status hpx_plan_test_withhold_copies(hpx_plan plan, int withhold);

/* Pixel layouts (Sec. III-B).
 *   HPX_RING   : rings north to south, pixels by increasing longitude.
 *   HPX_NESTED : face f (0..11) times nside^2 plus the Morton (Z-order)
 *                interleave of the face coordinates x (even bits) and y
 *                (odd bits); x + y grows northward, x - y eastward.
 *   HPX_FLAT   : f nside^2 + y nside + x (row-major face images).
 * Face f's rings and longitudes follow Gorski et al. 2005 (faces 0-3 north,
 * 4-7 equatorial, 8-11 south, each ordered eastward from longitude 0). */
typedef enum { HPX_RING = 0, HPX_NESTED = 1, HPX_FLAT = 2 } hpx_layout;

/* Reorders nbatch maps of 12 nside^2 elements of elem_bytes (4, 8 or 16)
 * bytes from layout `from` to layout `to` through the (x, y, f)
 * representation: out[b][t] = in[b][s(t)], s(t) the `from` index of the
 * pixel with `to` index t.  in, out: device, distinct, aligned to the
 * element size.  nside: power of two, 1..8192.  Allocates nothing, needs no
 * plan; stream-ordered. */
hpx_status hpx_reorder(int nside, int nbatch, size_t elem_bytes, hpx_layout from,
                       hpx_layout to, const void* in, void* out,
                       hpx_stream_t stream);

/* index[t] (device, 12 nside^2 int64) = the `from` index of the pixel whose
 * `to` index is t (the gather map hpx_reorder applies). */
hpx_status hpx_layout_index(int nside, hpx_layout from, hpx_layout to,
                            int64_t* index, hpx_stream_t stream);

/* Synchronises the current device and reports (HPX_ERR_INVALID) whether any
 * reorder or index kernel since the last call met an index without an
 * (x, y, f) representation (impossible for valid arguments); clears it. */
hpx_status hpx_layout_status(void);

/* Message describing the last failure on the calling thread ("" if none). */
const char* hpx_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HPX_H */
