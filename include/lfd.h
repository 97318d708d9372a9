/*
 * lfd.h - C ABI of the GB300 light-field Richardson-Lucy deconvolution library
 * (liblfd.so, CUDA for sm_103a).
 *
 * The library runs the data-parallel hot path of light-field microscopy
 * deconvolution that AutoDeconJ (Su et al., arXiv 2208.11422) accelerates:
 * Richardson-Lucy (RL) iterations on a light-field image with a depth- and
 * phase-dependent PSF (Sections 1 and 2.1), with the DCT-entropy image-quality
 * metric of Section 2.2 (Eqs. 1-12) evaluated on every iterate to predict the
 * iteration count. Intermediates stay on the GPU; only results come back
 * (Section 2.1, Fig. 1).
 *
 * Model. Volume v[z][i'][j'] (z < Nz, i' < H, j' < W), sensor image y[i][j],
 * PSF K[z][aa][bb][mi][mj] (aa, bb < Nnum lenslet phase, mi, mj < P, P odd,
 * centre c = (P-1)/2). The paper does not write the model out; it is the
 * Prevedel et al. 2014 model the paper builds on:
 *   forward   (Hv)[i][j]        = sum_{z,i',j'} v[z][i'][j'] K[z][i'%N][j'%N][i-i'+c][j-j'+c]
 *   backward  (H^T r)[z][i'][j'] = sum_{i,j}    r[i][j]     K[z][i'%N][j'%N][i-i'+c][j-j'+c]
 * (terms outside the PSF window or the sensor are zero). One RL iteration:
 *   r = y / (Hv + eps);  v <- max(0, v * (H^T r) / (H^T 1))  (0 where H^T 1 = 0).
 *
 * Conventions
 *   - All arrays are dense, row-major, FP32. Volumes are [Nz][H][W] (stack
 *     order), images [H][W], the PSF [Nz][Nnum][Nnum][P][P].
 *   - Pointers may be device or host memory; the library tells them apart with
 *     cudaPointerGetAttributes. Host buffers are staged through device memory
 *     owned by the context (pinned host memory makes those copies fast).
 *   - The caller owns every buffer it passes; the context owns its internal
 *     buffers and frees them in lfd_destroy.
 *   - Calls are ordered on the CUDA stream passed in (NULL = legacy default
 *     stream). lfd_forward / lfd_backward return after enqueueing when given
 *     device pointers; the others synchronise the stream before returning.
 *     Launch and argument errors are returned at once; asynchronous device
 *     faults surface at the next call that synchronises.
 *   - No function aborts the process. On error the status is returned and
 *     lfd_last_error(ctx) gives a message.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef LFD_H
#define LFD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lfd_ctx lfd_ctx;

typedef enum {
    LFD_OK = 0,
    LFD_EINVAL = 1,       /* invalid argument or shape                         */
    LFD_ENOMEM = 2,       /* a device or host allocation failed                 */
    LFD_ECUDA = 3,        /* a CUDA runtime/driver call failed                  */
    LFD_ENOTREADY = 4,    /* lfd_poll: the request has not finished yet         */
    LFD_ETIMEDOUT = 5,    /* a bounded device wait gave up (kernel error flag),
                             or lfd_poll's timeout passed                        */
    LFD_EBUSY = 6,        /* lfd_submit: queue full; lfd_cancel: request already
                             running; lfd_server_add_psf: server started        */
    LFD_EINTERNAL = 7,    /* internal consistency check failed                  */
    LFD_EUNSUPPORTED = 8, /* option not available for this shape / device       */
    LFD_ECANCELED = 9     /* the request was cancelled before it started        */
} lfd_status;

/* Arithmetic of the two projections (the ratio, update and metric are FP32 with
 * FP64 reductions in every mode). */
typedef enum {
    LFD_FP32 = 0,   /* FP32 inputs and FP32 FMA accumulation on the CUDA cores   */
    LFD_TF32 = 1,   /* TF32 on tcgen05 tensor cores, FP32 accumulation (LFD_DIRECT
                       only; LFD_EUNSUPPORTED with LFD_FFT): the PSF, the iterate
                       and the ratio image rounded to TF32 (10-bit mantissa,
                       round to nearest), one product per term               */
    LFD_BF16 = 2,   /* BF16 on tcgen05 tensor cores, FP32 accumulation. LFD_DIRECT:
                       PSF and data rounded to BF16, one product per term.
                       LFD_FFT: the PSF spectra rounded once to BF16 (4 bytes
                       per complex value), the transformed data split hi + lo,
                       two products per term                                     */
    LFD_BF16X3 = 3  /* split BF16: x = hi + lo, three products hi*hi + hi*lo +
                       lo*hi per term, FP32 accumulation (tensor cores)          */
} lfd_precision;

typedef struct {
    int precision;        /* lfd_precision                                          */
    float eps;            /* ratio guard: r = y / (Hv + eps); default 1e-6          */
    /* optics for the metric's region size (Eqs. 7, 9-11); defaults
       d_ML = 150 um, Q = 40, NA = 0.95, lambda = 0.525 um                          */
    double dML_um, Q, NA, lambda_um;
    int XS, YS;           /* region width / height; > 0 overrides the optics        */
    int l2_over_region;   /* 1: L2 norm of Eq. 12 over the region S (default);
                             0: over the whole DCT (= 2-norm of the MIP)            */
    int variant;          /* projection formulation, lfd_variant                     */
    int max_frames;       /* frames one lfd_rl_iterate_batch call may carry (>= 1;
                             more than 1 needs LFD_FFT); buffers are sized for it   */
    int use_graph;        /* 1 (default): replay each RL iteration as a captured CUDA
                             graph (not while profiling); 0: plain launches         */
    int fft_size;         /* LFD_FFT transform size per axis: 32 or 64; 0 (default)
                             picks by a bandwidth / arithmetic cost model (see
                             lfd_autotune for picking by measurement)               */
    float spectra_lo_tau; /* LFD_FFT with LFD_BF16X3: the lo planes of the PSF
                             spectra are kept only for the (frequency bin,
                             64-channel block) tiles whose largest hi value
                             reaches tau x the largest of all spectra; a dropped
                             lo part is below 2^-9 tau of that largest value.
                             0 keeps every lo plane; default 2^-8; [0, 1)        */
    int contraction_cols; /* LFD_FFT on the tensor cores: the widest column chunk of
                             one contraction pass (16, 32 or 64 columns = frames x
                             tiles; every chunk streams the PSF spectra once); 0
                             (default) the widest the frames need, up to 64.
                             Wider chunks stream the spectra fewer times with
                             fewer stages in flight (see lfd_autotune_options) */
} lfd_options;

/* How the two projections are computed (same results up to rounding). */
typedef enum {
    LFD_DIRECT = 0,  /* polyphase implicit GEMM: tcgen05 (BF16, split BF16, TF32) or
                        CUDA cores (FP32)                                           */
    LFD_FFT = 1      /* overlap-save FFT on the lenslet grid with cached PSF spectra,
                        FP32 transforms; complex contractions in FP32 on the CUDA
                        cores (LFD_FP32), or on tcgen05 in split BF16 (LFD_BF16X3)
                        or with BF16 PSF spectra (LFD_BF16)                      */
} lfd_variant;

/* Fills *opt with the defaults listed above. */
void lfd_default_options(lfd_options* opt);

/* Creates a context for one PSF and one sensor shape (Fig. 1: the PSF is moved
 * to the GPU once and reused by every reconstruction).
 *   psf     [Nz][Nnum][Nnum][P][P] FP32, host or device; copied, not kept.
 *   P       PSF window width in pixels: odd, a multiple of Nnum.
 *   Nnum    pixels per lenslet (odd, >= 1).  Nz >= 1 depths.
 *   H, W    sensor height / width in pixels, each a positive multiple of Nnum.
 *   opt     NULL for defaults.
 * Work done here: the PSF is repacked into the polyphase layout the projection
 * kernels read, H^T 1 is computed, and the metric's cosine tables are built.
 * Errors: LFD_EINVAL (shape rules above, NULL out), LFD_ENOMEM, LFD_ECUDA,
 * LFD_EUNSUPPORTED (precision needs tensor cores the device lacks; LFD_TF32
 * with LFD_FFT; max_frames > 1 with LFD_DIRECT).
 * On error *out is NULL. */
lfd_status lfd_create(const float* psf, int P, int Nnum, int Nz, int H, int W,
                      const lfd_options* opt, void* cuda_stream, lfd_ctx** out);

/* Forward projection y_out = H v (model above).
 *   v      [Nz][H][W], y_out [H][W]; host or device. */
lfd_status lfd_forward(lfd_ctx* ctx, const float* v, float* y_out, void* cuda_stream);

/* Backprojection v_out = H^T r (model above): the flipped-PSF sum of every
 * phase, sub-sampled into each depth.
 *   r      [H][W], v_out [Nz][H][W]; host or device. */
lfd_status lfd_backward(lfd_ctx* ctx, const float* r, float* v_out, void* cuda_stream);

/* Runs up to n RL iterations (model above) starting from the volume in v and
 * writes the result back into v. After each iteration the DCT entropy of the
 * z-maximum projection is computed (Section 2.2, Eqs. 1-12).
 *   y                 [H][W] light-field image (host or device)
 *   v                 [Nz][H][W] in: v^0 (e.g. all ones), out: result
 *   n                 iterations to run (>= 1)
 *   stop_at_predicted 0: run n iterations, v = v^n.
 *                     1: stop once the entropy decreases (E_{k+1} < E_k) and
 *                        return v = v^k, the iterate with the higher entropy
 *                        (Section 2.2: stop when the entropy starts to fall).
 *   iters_done        (may be NULL) iterations whose result is in v
 *   predicted         (may be NULL) predicted iteration n*: first k with
 *                     E_{k+1} < E_k, else the first argmax of E_1..E_ran
 *   entropy_hist      (may be NULL) host array of n doubles, E_1..E_ran
 *                     (entries past the last iteration run are set to NaN)
 *   flux_hist         (may be NULL) host array of n doubles:
 *                     sum(H^T1 * v^k), which equals sum(y * Hv/(Hv+eps))
 * Synchronises the stream. */
lfd_status lfd_rl_iterate(lfd_ctx* ctx, const float* y, float* v, int n,
                          int stop_at_predicted, int* iters_done, int* predicted,
                          double* entropy_hist, double* flux_hist, void* cuda_stream);

/* RL iterations on an iterate that stays in the context between calls, for a
 * caller that steps the deconvolution itself (e.g. one iteration at a time,
 * watching the entropy of Section 2.2 to decide when to stop): the volume is
 * repacked into the context's layout once, not on every call as with
 * lfd_rl_iterate.
 *   lfd_rl_load(ctx, v)       resident iterate <- v [Nz][H][W] (host or device)
 *   lfd_rl_step(ctx, y, n, entropy_hist, flux_hist)
 *                             n >= 1 RL iterations (model above) of the resident
 *                             iterate with the light-field image y [H][W] (host
 *                             or device; read by this call only); entropy_hist
 *                             and flux_hist (host arrays of n doubles, may be
 *                             NULL) get E_k and sum(H^T1 * v^k) of each
 *                             iteration. Synchronises the stream.
 *   lfd_rl_store(ctx, v)      v [Nz][H][W] (host or device) <- the resident
 *                             iterate; with a host v the stream is synchronised.
 * The resident iterate is the one of the lfd_split_* calls: lfd_split_load and
 * lfd_rl_load are interchangeable. lfd_forward, lfd_rl_iterate and
 * lfd_rl_iterate_batch reuse its buffers (after them lfd_rl_load is needed
 * again). Frame 0 of a context made for several frames.
 * Errors: LFD_EINVAL (NULL arguments, n < 1, no iterate loaded), LFD_ECUDA,
 * LFD_ETIMEDOUT (a tensor-core kernel gave up waiting). */
lfd_status lfd_rl_load(lfd_ctx* ctx, const float* v, void* cuda_stream);
lfd_status lfd_rl_step(lfd_ctx* ctx, const float* y, int n, double* entropy_hist, double* flux_hist,
                       void* cuda_stream);
lfd_status lfd_rl_store(lfd_ctx* ctx, float* v, void* cuda_stream);

/* lfd_rl_iterate for nframes frames that share the context's PSF and sensor
 * shape (e.g. a time-lapse), all advanced together: every stage of an
 * iteration is one launch over all frames, and the iteration is replayed as a
 * captured CUDA graph. Each frame keeps its own entropy history and, with
 * stop_at_predicted, stops at its own predicted iteration (the other frames
 * go on, up to n).
 *   nframes      1 .. max_frames given at lfd_create
 *   y            [nframes][H][W], v [nframes][Nz][H][W] (host or device)
 *   iters_done, predicted      arrays of nframes ints (may be NULL)
 *   entropy_hist, flux_hist    host arrays of nframes * n doubles (frame-major,
 *                              may be NULL); entries past a frame's last
 *                              iteration are NaN
 * The other arguments and the errors are those of lfd_rl_iterate, plus
 * LFD_EINVAL when nframes is outside 1 .. max_frames. Synchronises the stream. */
lfd_status lfd_rl_iterate_batch(lfd_ctx* ctx, int nframes, const float* y, float* v, int n,
                                int stop_at_predicted, int* iters_done, int* predicted,
                                double* entropy_hist, double* flux_hist, void* cuda_stream);

/* Picks the fastest LFD_FFT transform size for this PSF, sensor shape and
 * opt->max_frames by measurement (lfd_autotune_options, with the contraction's
 * column chunk opt->contraction_cols kept fixed): for each feasible size a
 * context is created, one RL iteration of max_frames frames of a constant
 * image is run to warm up and two more are timed with CUDA events; the
 * contexts are destroyed again.
 *   opt          options of the context to tune (variant must be LFD_FFT)
 *   best_size    (out) 32 or 64, to pass as opt->fft_size to lfd_create
 *   ms_per_iter  (out, may be NULL) measured time of one batched iteration of
 *                the winner, in milliseconds
 * Errors: LFD_EINVAL, LFD_EUNSUPPORTED (no size fits), and those of lfd_create.
 * Allocates and frees device memory; synchronises the stream. */
lfd_status lfd_autotune(const float* psf, int P, int Nnum, int Nz, int H, int W,
                        const lfd_options* opt, void* cuda_stream, int* best_size,
                        float* ms_per_iter);

/* Picks the LFD_FFT tiles for this PSF, sensor shape and opt->max_frames by
 * measurement: the transform size (fft_size 32 or 64) and the contraction's
 * column chunk (contraction_cols 16, 32 or 64, the chunks wider than the
 * frames' columns need left out) on the tensor cores. For each feasible pair
 * a context is created, one batched RL iteration of a constant image warms
 * it up and two more are timed with CUDA events. The winner is written into
 * *opt (fft_size, contraction_cols; the other fields are kept), ready for
 * lfd_create, and cached for the process: a later call with the same PSF
 * (pointer and a sample of its values), shape, frames, precision and lo-plane
 * threshold returns it without timing (*cached = 1).
 *   opt          in: options of the context to tune (variant LFD_FFT); out: the choice
 *   ms_per_iter  (out, may be NULL) measured time of one batched iteration of the winner
 *   cached       (out, may be NULL) 1 when the result came from the cache
 * Errors: LFD_EINVAL, LFD_EUNSUPPORTED (no pair fits), and those of lfd_create.
 * Allocates and frees device memory; synchronises the stream. */
lfd_status lfd_autotune_options(const float* psf, int P, int Nnum, int Nz, int H, int W,
                                lfd_options* opt, void* cuda_stream, float* ms_per_iter, int* cached);

/* DCT entropy (Eq. 12 over the region of Eq. 6) of the z-maximum projection of
 * the volume v [Nz][H][W] (host or device); result in *entropy (host).
 * Synchronises the stream. */
lfd_status lfd_quality(lfd_ctx* ctx, const float* v, double* entropy, void* cuda_stream);

/* Image-quality value of a z-maximum projection image, without allocating memory.
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot call cudaMalloc, for example a host application that owns all device
 * memory and gives a plug-in only fixed buffers, or a real-time acquisition loop
 * that cannot afford the device-wide synchronisation an allocation may cause.
 * It returns the same value as lfd_quality, computed from the projection image
 * instead of the volume, and needs no context.
 *   mip            [H][W] FP32 image in device (or managed) memory, e.g. the
 *                  maximum over z of a volume
 *   H, W           1..4096 each
 *   XS, YS         region width / height: 1..min(W, 128) and 1..min(H, 128)
 *                  (lfd_region_size gives the paper's values)
 *   l2_over_region as in lfd_options
 *   entropy        one double in device (or managed) memory; receives the value
 * Intermediates live in one static device array of about 4.2 MB that every
 * GPU loading the library holds until the process exits. Sizes beyond the
 * limits above, and host pointers (this function stages nothing), return
 * LFD_EINVAL with a message on stderr; nothing is allocated, by this function
 * or on its behalf. Every call looks up the array's device address
 * (cudaGetSymbolAddress) on the current device, so the first call on a device
 * should come before any stream capture. Every call shares the array and
 * leaves its contents behind (each call writes every entry it reads before
 * reading it), so calls that may overlap on the GPU (different streams, or
 * different host threads) race and must be serialised by the caller.
 * Asynchronous: the result is ready when the stream reaches it.
 * Errors: LFD_EINVAL, LFD_ECUDA (lookup or launch failure). */
lfd_status lfd_quality_mip_static(const float* mip, int H, int W, int XS, int YS,
                                  int l2_over_region, double* entropy, void* cuda_stream);

/* ------------------------------------------------------------ depth split --
 * Section 2.1 and Fig. 1 of the paper divide the depth layers (and the PSF
 * slices that belong to them) among several GPUs. A context made over the
 * depths [z0, z1) of a PSF (psf + z0 * Nnum * Nnum * P * P, Nz = z1 - z0)
 * owns that part of the volume; the forward projection is the sum over all
 * parts of their partial projections, the backprojection and the update are
 * per depth, the z-maximum projection is the maximum of the parts', and the
 * flux the sum of theirs. These calls cut one RL iteration (model above) at
 * those two exchange points; the caller does the reductions between them
 * (paper_2208_11422_gb300/depth_split.py does them with torch.distributed):
 *   lfd_split_load(ctx, v)         iterate <- v, this part's [Nz][H][W] (host or device)
 *   per iteration:
 *     lfd_split_forward(ctx, hv)   hv [H][W] (device) <- partial H v of the iterate
 *     (sum hv over all parts)
 *     lfd_split_update(ctx, y, hv, mip, flux)
 *                                  r = y / (hv + eps); v <- max(0, v H^T r / H^T 1);
 *                                  mip [H][W] <- max over this part's depths of the new v;
 *                                  *flux (one double) <- sum(H^T 1 * v) over this part
 *                                  (y, hv, mip, flux in device memory)
 *     (max of mip and sum of flux over all parts; lfd_quality_mip gives the
 *      entropy of the reduced mip, and the stopping rule of lfd_rl_iterate
 *      applies to the entropies)
 *   lfd_split_store(ctx, v, previous)  v <- the current iterate (previous = 0)
 *                                  or the one before the last update (1)
 * All calls are ordered on cuda_stream; lfd_split_store with a host v and
 * lfd_quality_mip synchronise it. lfd_forward and lfd_rl_iterate reuse the
 * iterate buffers: after them lfd_split_load is needed again.
 * Errors: LFD_EINVAL (NULL or host pointers where device memory is required,
 * no iterate loaded, no previous iterate), LFD_ECUDA, LFD_ETIMEDOUT. */
lfd_status lfd_split_load(lfd_ctx* ctx, const float* v, void* cuda_stream);
lfd_status lfd_split_forward(lfd_ctx* ctx, float* hv_part, void* cuda_stream);
lfd_status lfd_split_update(lfd_ctx* ctx, const float* y, const float* hv, float* mip_part,
                            double* flux_part, void* cuda_stream);
lfd_status lfd_split_store(lfd_ctx* ctx, float* v, int previous, void* cuda_stream);

/* DCT entropy (Eq. 12 over the region of Eq. 6) of a z-maximum projection
 * image mip [H][W] (host or device) with the context's region and tables; the
 * metric step of lfd_rl_iterate on an image reduced outside the library (the
 * depth split above). Synchronises the stream. */
lfd_status lfd_quality_mip(lfd_ctx* ctx, const float* mip, double* entropy, void* cuda_stream);

/* Frees the context and everything it owns. NULL is a no-op. */
void lfd_destroy(lfd_ctx* ctx);

/* Message of the last error on ctx ("" if none); static text if ctx is NULL. */
const char* lfd_last_error(const lfd_ctx* ctx);

/* Name of a status code. */
const char* lfd_status_string(lfd_status s);

/* Host-only helpers (no GPU needed). */

/* Region size of Eqs. 7, 9, 10, 11: P_u = d_ML / (Q Nnum),
 * d_psf = 1.22 lambda Nnum / NA, X_S = floor(P_u W / d_psf),
 * Y_S = floor(P_u H / d_psf), each clamped to [min(2, size), size].
 * Errors: LFD_EINVAL for non-positive sizes or optics, NULL outputs. */
lfd_status lfd_region_size(int Nnum, int H, int W, double dML_um, double Q,
                           double NA, double lambda_um, int* XS, int* YS);

/* Predicted iteration (1-based) from an entropy history E[0..n-1] = E_1..E_n:
 * the first k with E_{k+1} < E_k, else the first argmax; 0 when n < 1. */
int lfd_predict_stop(const double* E, int n);

/* Shape of the context's internal problem, for inspection and tests.
 * Each pointer may be NULL. taps = k + 2 where k = P / Nnum. */
lfd_status lfd_get_geometry(const lfd_ctx* ctx, int* XS, int* YS, int* taps,
                            int* precision, int64_t* device_bytes);

/* FFT tiling of an LFD_FFT context: transform size F (lenslets per patch side),
 * valid lenslets per tile side B = F - 2h, tiles per frame, and frequency bins
 * F*(F/2+1) per channel. All four are 0 for an LFD_DIRECT context. Any output
 * pointer may be NULL. LFD_EINVAL only for ctx == NULL. */
lfd_status lfd_get_fft_plan(const lfd_ctx* ctx, int* F, int* B, int* tiles, int* bins);

/* Low-sensitivity voxels of an LFD_FFT context (H^T 1 below 1e-3 of its
 * largest value), which every backprojection sums exactly over their PSF
 * windows instead of taking the transforms' value: how many there are
 * (n_low), how many are summed in runs along a sensor row or column (in_runs,
 * in `runs` blocks of at most 68 voxels) and how many one warp each
 * (single = n_low - in_runs). All 0 for an LFD_DIRECT context. Any output
 * pointer may be NULL. LFD_EINVAL only for ctx == NULL. */
lfd_status lfd_get_exact_plan(const lfd_ctx* ctx, int64_t* n_low, int64_t* in_runs, int64_t* runs,
                              int64_t* single);

/* PSF spectra of an LFD_FFT context on the tensor cores: device bytes of the
 * planes the contractions stream, and of the (frequency bin, 64-channel block)
 * tiles how many keep their lo planes (lo_tiles_kept) out of lo_tiles (all
 * tiles with full split BF16, none with LFD_BF16). All 0 for other contexts.
 * Any output pointer may be NULL. LFD_EINVAL only for ctx == NULL. */
lfd_status lfd_get_spectra(const lfd_ctx* ctx, int64_t* bytes, int64_t* lo_tiles_kept, int64_t* lo_tiles);

/* Test hooks (no counterpart in the paper).
 * lfd_debug_fail_allocs(n): the next n device allocations the library makes
 * (contexts, staging buffers, PSF sets, the serving arena) fail with
 * LFD_ENOMEM without calling the CUDA allocator; n <= 0 cancels. Host-side
 * fault injection: a call that fails this way leaves its context as it was.
 * lfd_selftest_bounded_wait(limit_ns, code): runs one kernel whose thread waits
 * on a shared-memory mbarrier that nothing arrives at, with the bounded wait of
 * the tensor-core kernels limited to limit_ns (1e6 .. 4e9); *code receives the
 * error word the kernel stored. LFD_ETIMEDOUT: the wait gave up (the expected
 * outcome); LFD_OK: it completed; LFD_EINVAL: limit out of range; LFD_ECUDA:
 * a launch or copy failed.
 * lfd_selftest_freelist(seed, steps): host only; runs `steps` random
 * allocations and releases on the first-fit free list of the serving arena and
 * checks it against a byte map: no overlap, 256-byte alignment, failure only
 * when no free run is large enough, exact accounting, full coalescing at the
 * end. LFD_OK, LFD_EINTERNAL on a violation, LFD_EINVAL for steps < 1.
 * lfd_selftest_exact_runs(seed, Nnum, Nz, k, L): host only; builds the plan
 * of runs for the exact low-sensitivity sums (lfd_get_exact_plan) from a
 * seeded synthetic voxel list on an L x L lenslet grid (Nnum, Nz depths, PSF
 * k lenslets wide): border bands, corner blocks and scattered voxels of each
 * channel. Checks that every listed voxel is summed exactly once, that a
 * piece holds voxels of one channel along one lenslet row or column in
 * increasing order within the piece and staging limits, that its PSF tile is
 * the voxel's (or its transposed copy), and the cost order. LFD_OK,
 * LFD_EINTERNAL on a violation, LFD_EINVAL for an invalid shape.
 * lfd_selftest_balanced_ranges(seed, n, grid): host only; splits n seeded
 * synthetic unit costs (stretches of units with and without lo planes, as in
 * the adjoint contraction) into grid contiguous ranges the way the adjoint's
 * blocks get theirs, and checks that they tile the units in order, that none
 * is empty, and that none exceeds the mean by the largest unit cost. LFD_OK,
 * LFD_EINTERNAL on a violation, LFD_EINVAL unless 1 <= grid <= n. */
void lfd_debug_fail_allocs(int n);
lfd_status lfd_selftest_bounded_wait(int64_t limit_ns, int* code);
lfd_status lfd_selftest_freelist(int seed, int steps);
lfd_status lfd_selftest_exact_runs(int seed, int Nnum, int Nz, int k, int L);
lfd_status lfd_selftest_balanced_ranges(int seed, int n, int grid);

/* Number of kernels the library has launched in this process (all contexts). */
uint64_t lfd_launch_count(void);

/* Per-stage device time of lfd_rl_iterate iterations, in milliseconds, measured
 * with CUDA events recorded on the call's stream around each stage:
 * [0] forward projection (FFT variant: ratio included), [1] ratio (direct
 * variant), [2] backprojection, [3] update + MIP + flux, [4] metric,
 * [5] forward contraction kernel alone, [6] backward contraction kernel alone,
 * [7] the FFT variant's transforms (0 for the direct variant), of which
 * [8] the forward projection's volume transform (R2C) and [9] the
 * backprojection's volume transform (C2R) alone, [10] the FFT variant's exact
 * backprojection of low-sensitivity voxels (part of [2]).
 * lfd_set_profiling(ctx, 1) turns the events on and resets the averages;
 * lfd_stage_times writes the mean over every iteration run since then (zeros
 * if none) into ms[0..n-1] (entries past 10 are 0). */
lfd_status lfd_stage_times(const lfd_ctx* ctx, float* ms, int n);

/* ------------------------------------------------------------------ serving --
 * A server reconstructs a stream of light-field frames with continuous
 * batching. Fig. 1 of the paper moves each PSF to the GPU once and reuses it
 * for every reconstruction; here several PSF sets stay resident (as FFT
 * spectra), frames of any sensor size up to a set's maximum are admitted when
 * their device footprint fits (Fig. 1 estimates the memory a reconstruction
 * needs before allocating it), frames of one set advance together through
 * one launch per stage, and each frame stops at its metric-predicted
 * iteration (Section 2.2) and leaves the batch while others join.
 *
 * Arithmetic is the LFD_FFT variant's (split BF16 or FP32), with the same
 * results as an lfd_ctx made for the frame's shape with the same options and
 * the same FFT size (up to rounding order).
 *
 * Threads: lfd_submit, lfd_poll, lfd_cancel and lfd_server_stats may be called
 * from any host thread. One scheduler thread per server owns the GPU work; it
 * runs on the device that was current in lfd_server_create. */
typedef struct lfd_server lfd_server;

typedef struct {
    lfd_options opt;          /* precision (LFD_BF16X3 default, LFD_BF16 or LFD_FP32), eps,
                                 optics, XS / YS, l2_over_region, fft_size; variant
                                 is LFD_FFT; max_frames and use_graph are ignored  */
    int64_t arena_bytes;      /* device memory for frames in flight; 0 (default):
                                 85 % of the free memory at the first submit        */
    int max_frames_per_set;   /* frames iterating together per PSF set (default 32) */
    int max_cols;             /* FFT tiles per contraction launch (default 128; a
                                 multiple of 16); larger batches take several
                                 launches                                          */
    int max_queue;            /* requests waiting for admission (default 4096)      */
    int max_iter;             /* iteration cap of a request with max_iter 0
                                 (default 40)                                       */
} lfd_server_options;

typedef struct {
    int set_id;               /* from lfd_server_add_psf                           */
    int H, W;                 /* sensor size in pixels: positive multiples of the
                                 set's Nnum, at most the set's max_H x max_W       */
    const float* y;           /* [H][W] light-field image, host or device           */
    float* v_out;             /* [Nz][H][W] result, host or device                   */
    int max_iter;             /* iteration cap (0: the server's)                     */
    int stop_at_predicted;    /* 1: stop at the predicted iteration, as in
                                 lfd_rl_iterate; 0: run max_iter iterations         */
    double* entropy_hist;     /* optional host array [max_iter]: E after each
                                 iteration run, NaN after the last                 */
} lfd_request;
/* The caller keeps y, v_out and entropy_hist alive and unchanged until
 * lfd_poll reports the request finished (or it is cancelled). The start volume
 * is all ones. Host buffers in page-locked memory are copied asynchronously;
 * pageable ones stall the scheduler while they are copied. */

typedef struct {
    int status;               /* lfd_status of the request: LFD_OK, LFD_ECANCELED,
                                 LFD_ECUDA, LFD_ETIMEDOUT                          */
    int iters_done;           /* iterations whose result v_out holds                */
    int iters_run;            /* iterations computed                                */
    int predicted;            /* lfd_predict_stop of the entropy history            */
    int64_t queue_us;         /* submit -> admission (device memory reserved)       */
    int64_t latency_us;       /* submit -> result in v_out                          */
} lfd_result;

typedef struct {
    int64_t submitted, admitted, completed, rejected, cancelled;
    int64_t frame_iterations; /* RL iterations over all frames                      */
    int64_t ticks;            /* batched steps over all sets                        */
    int64_t columns;          /* FFT tiles transformed in forward passes            */
    int64_t arena_bytes, arena_peak_bytes, resident_bytes;
    int queued, in_flight;
} lfd_server_stats;

/* Fills *opt with the defaults listed above. */
void lfd_server_default_options(lfd_server_options* opt);

/* Creates a server on the current device and starts its scheduler thread.
 * Errors: LFD_EINVAL (options), LFD_ENOMEM, LFD_ECUDA. */
lfd_status lfd_server_create(const lfd_server_options* opt, lfd_server** out);

/* Makes a PSF set resident: PSF [Nz][Nnum][Nnum][P][P] (host or device, copied)
 * for frames up to max_H x max_W pixels. Computes the PSF spectra (and keeps
 * the PSF for the exact backprojection of low-sensitivity voxels).
 * Only before the first lfd_submit (LFD_EBUSY after).
 * Errors: LFD_EINVAL (shape rules of lfd_create), LFD_ENOMEM, LFD_ECUDA,
 * LFD_EUNSUPPORTED (no FFT tiling fits, or split BF16 without tcgen05). */
lfd_status lfd_server_add_psf(lfd_server* srv, const float* psf, int P, int Nnum, int Nz,
                              int max_H, int max_W, int* set_id);

/* Queues a request; *ticket identifies it. Returns at once.
 * Errors: LFD_EINVAL (unknown set, shape, NULL y / v_out), LFD_ENOMEM (the
 * frame alone needs more than the arena), LFD_EBUSY (queue full). */
lfd_status lfd_submit(lfd_server* srv, const lfd_request* req, uint64_t* ticket);

/* Waits up to timeout_us microseconds (0: do not wait; < 0: no limit) for the
 * request to finish. LFD_OK: finished, *res filled, the ticket is released.
 * LFD_ENOTREADY (timeout_us == 0) or LFD_ETIMEDOUT: not finished yet.
 * LFD_EINVAL: unknown or released ticket. */
lfd_status lfd_poll(lfd_server* srv, uint64_t ticket, int64_t timeout_us, lfd_result* res);

/* Cancels a request that has not been admitted yet: LFD_OK (poll then reports
 * status LFD_ECANCELED), LFD_EBUSY if it is already running or finished,
 * LFD_EINVAL for an unknown ticket. */
lfd_status lfd_cancel(lfd_server* srv, uint64_t ticket);

lfd_status lfd_server_stats_get(const lfd_server* srv, lfd_server_stats* stats);

/* Last error message of the server (scheduler or API), "" if none. The text is
 * copied under the server's lock into a buffer of the calling thread, valid
 * until that thread calls lfd_server_last_error again. */
const char* lfd_server_last_error(const lfd_server* srv);

/* Finishes the requests already admitted, cancels the queued ones, stops the
 * scheduler and frees everything. Tickets not yet polled become invalid. */
void lfd_server_destroy(lfd_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* LFD_H */
