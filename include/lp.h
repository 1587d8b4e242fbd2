/*
 * lp.h -- C ABI of the GB300 light-pollution convolution library (liblp.so).
 *
 * The library computes artificial night-sky-brightness maps as the linear
 * two-dimensional convolution of a gridded ground-radiance map L1 with a
 * shift-invariant point spread function K (Bara et al., arXiv:1907.02891):
 *
 *   B(r) = integral of K(r - r') L1(r') d^2 r'          Sec. 2.3, Eq. (7)
 *
 * discretised on the pixel grid (Eq. (2) with the factorable source of
 * Eq. (3)) and evaluated through the convolution theorem, Sec. 2.3 Eq. (9):
 * zero-pad both to a common size of at least N_L + N_K - 1 (Sec. 2.5), take
 * the DFT of Eq. (10) by FFT, multiply pixel-wise, inverse FFT, crop.  The
 * pixel-area factor of Eq. (2) is not applied; fold it into K.
 *
 * With 0-based indices, for a map L (h x w) and a PSF K (hk x wk, both odd,
 * centre (cy, cx) = ((hk-1)/2, (wk-1)/2)):
 *
 *   Bfull[i][j] = sum_{i',j'} L[i'][j'] K[i-i'][j-j'],
 *                 0 <= i < h+hk-1, 0 <= j < w+wk-1            (LP_OUT_FULL)
 *   B[i][j]     = Bfull[i+cy][j+cx],  0 <= i < h, 0 <= j < w  (LP_OUT_SAME)
 *
 * LP_OUT_SAME puts every observer on a source pixel and keeps the map
 * region; the sources all around it still contribute (Sec. 3).
 *
 * Conventions
 *   - Pointers named "device" must be CUDA device pointers of the context's
 *     device; "host" pointers are ordinary (preferably pinned) host memory.
 *   - Matrices are row-major; ld* are leading dimensions in elements.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     All map calls are asynchronous on that stream.
 *   - Every call returns lp_status.  Arguments are validated before anything
 *     is launched; on error nothing is launched and lp_last_error() returns
 *     a message (thread-local, valid until the next call on that thread).
 *   - The caller owns L, K and out[]; the library owns plans, twiddle
 *     tables, spectra, workspaces and its internal streams.  Inputs are
 *     never written.  out[] must not overlap L.
 */
#ifndef LP_H
#define LP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lp_status {
    LP_OK = 0,
    LP_ERR_INVALID = 1,     /* bad argument (null, size, leading dimension, padding) */
    LP_ERR_OOM = 2,         /* device allocation failed or HBM budget exceeded */
    LP_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    LP_ERR_TIMEOUT = 4,     /* a bounded wait ran out */
    LP_ERR_UNSUPPORTED = 5, /* size or precision not built into this library */
    LP_ERR_BUSY = 6,        /* serving queue full / state does not allow the call */
    LP_ERR_DEVICE = 7,      /* a kernel reported an anomaly in the device status word */
    LP_ERR_CANCELLED = 8    /* a queued serving request was cancelled before it started */
} lp_status;

typedef enum lp_precision {
    LP_PREC_FP32 = 0,       /* FP32 FFT path */
    LP_PREC_SPLIT_BF16 = 1, /* column DFT stages on the tensor cores: operands split
                               into BF16 hi + lo, FP32 accumulation (row passes FP32) */
    LP_PREC_SPLIT_FP16 = 2  /* reserved: split-FP16 tensor-core DFT stages (not built) */
} lp_precision;

typedef enum lp_outmode {
    LP_OUT_SAME = 0, /* h x w: the map region, observers on the source grid */
    LP_OUT_FULL = 1  /* (h+hk-1) x (w+wk-1): the full linear convolution */
} lp_outmode;

typedef struct lp_ctx lp_ctx;
typedef struct lp_spectrum lp_spectrum;

/* Library version, major*10000 + minor*100 + patch. */
int lp_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char* lp_last_error(void);

/*
 * Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * device memory the context holds (spectra + workspaces + staging); 0 means
 * no cap.  Sets *ctx to NULL on failure.
 */
lp_status lp_create(lp_ctx** ctx, int device, size_t hbm_budget_bytes);

/* Release everything the context owns (waits for its work to finish). */
void lp_destroy(lp_ctx* ctx);

/* Device bytes currently held by the context. */
size_t lp_bytes_in_use(const lp_ctx* ctx);

/*
 * Supported padded FFT lengths (mixed radix, factors 2, 3, 5, 7).
 * lp_supported_size(n) returns the smallest supported length >= n, or -1.
 */
int lp_num_supported_sizes(void);
int lp_supported_size_at(int i);
int lp_supported_size(int n);

/*
 * 1 if the supported length n has the split-precision (LP_PREC_SPLIT_BF16)
 * column pass, else 0.  That precision needs it for the padded column count
 * pad_ny; its auto padding picks the smallest such length.  The pass runs
 * each radix-R stage of the column DFT (Eq. (10)) as a real 2R x 2R matrix
 * product on the tensor cores, D = A_hi F_hi + A_hi F_lo + A_lo F_hi, and
 * matches the FP32 path to about 1e-5 of the map maximum.
 */
int lp_split_supported(int n);

/*
 * Kernel spectrum (Sec. 2.3 Eq. (9)-(10), padding of Sec. 2.5): the DFT of
 * K zero-padded to pad_ny x pad_nx, computed in FP64 on the device and kept
 * device-resident in FP32, scaled so that lp_map returns Eq. (7) directly.
 *
 *   K          device, FP64, hk x wk row-major (ld = wk); hk, wk odd; the
 *              PSF centre is element ((hk-1)/2, (wk-1)/2).
 *   max_h/w    largest map this spectrum will be used with; used only when
 *              pad_ny / pad_nx is 0 (auto = smallest supported size
 *              >= max_h + hk - 1, resp. max_w + wk - 1).
 *   pad_ny/nx  explicit padded size (must be supported), or 0 for auto.
 *   prec       LP_PREC_FP32 or LP_PREC_SPLIT_BF16 (needs lp_split_supported(pad_ny));
 *              LP_PREC_SPLIT_FP16: LP_ERR_UNSUPPORTED.  lp_map must be called
 *              with the spectra's precision.
 *   stream     the spectrum is ready in stream order; the call itself
 *              synchronises the stream once (symmetry check).
 *   out        receives a handle (refcounted: an identical request --
 *              same values, sizes and precision -- returns the cached one).
 *              The cache is keyed by a 64-bit fingerprint of K's values
 *              and the sizes; a hit is confirmed by comparing K with a
 *              device copy kept with the spectrum, value by value, so a
 *              fingerprint collision builds a new spectrum instead of
 *              returning another PSF's.
 *
 * A point-symmetric K (K[cy+a][cx+b] == K[cy-a][cx-b] exactly) has a real
 * spectrum and is stored as 4 bytes per bin, otherwise 8.
 */
lp_status lp_kernel_spectrum(lp_ctx* ctx, const double* K, int hk, int wk, int max_h, int max_w,
                             int pad_ny, int pad_nx, lp_precision prec, void* stream,
                             lp_spectrum** out);

/* Shape of a spectrum.  Any out pointer may be NULL. */
lp_status lp_spectrum_info(const lp_spectrum* s, int* ny, int* nx, int* hk, int* wk,
                           int* is_real);

/*
 * Copy the stored spectrum (device -> device) for inspection: layout
 * (nx/2+1) rows x ny, row c holding the column-frequency c of every
 * row-frequency u; FP32 real (is_real) or interleaved complex, scaled by
 * 1/(2 ny nx).  dst_floats must be >= (nx/2+1)*ny*(is_real ? 1 : 2).
 */
lp_status lp_spectrum_copy(const lp_spectrum* s, float* dst, size_t dst_floats, void* stream);

/*
 * Drop one reference.  When the last one goes the handle becomes invalid at
 * once, but the device memory is freed in stream order: only after the
 * spectrum's build and every map call already enqueued with it (on any
 * stream) have completed.  The call never waits for the device; memory
 * still held is freed by a later lp_kernel_spectrum, lp_spectrum_release,
 * lp_map or lp_sync_status call, or by lp_destroy.
 */
lp_status lp_spectrum_release(lp_ctx* ctx, lp_spectrum* s);

/*
 * The map (steps S1-S6): B_k = K_k * L for each of the n spectra, from one
 * shared row transform of L; the column pass also shares its forward
 * transform across the spectra where the length's plan batches them (Sec. 3
 * computes several maps -- zenithal brightness and all-sky ratio -- from the
 * same radiance map).
 *
 *   L        device FP32, h x w, leading dimension ldl >= w.
 *   spectra  n >= 1 handles with identical (ny, nx), ny >= h + hk - 1 and
 *            nx >= w + wk - 1 for each (the padding rule of Sec. 2.5); in
 *            LP_OUT_FULL mode they must also share (hk, wk).
 *   out      n device FP32 pointers, caller-allocated: h x w (SAME) or
 *            (h+hk-1) x (w+wk-1) (FULL), leading dimension ldo.
 *   prec     LP_PREC_FP32, or LP_PREC_SPLIT_BF16 with spectra built in that
 *            precision (the column pass then runs on the tensor cores, one
 *            launch per spectrum; the row passes stay FP32).
 * Asynchronous on `stream`; use lp_sync_status to wait and collect device
 * anomalies.  Calls on different streams of one context may overlap; each
 * stream gets its own workspace.  The map waits, in stream order, for the
 * builds of its spectra (lp_kernel_spectrum is asynchronous on the stream it
 * is given, and a cache hit may return a spectrum still being built on
 * another stream); no wait is issued once a build has been seen complete.
 */
lp_status lp_map(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                 const lp_spectrum* const* spectra, int n, float* const* out, int ldo,
                 lp_outmode mode, lp_precision prec, void* stream);

/*
 * Same as lp_map with HOST buffers: copies L to the device, runs the map,
 * copies every out[k] back (the copies are asynchronous when the host memory
 * is pinned).  `stream` reaches the end of the call only when every out[k]
 * is in host memory; host buffers must stay valid until then
 * (lp_sync_status).  The downloads into out[] wait for the caller's earlier
 * work on `stream`.  The upload of L and the passes do not: they run on the
 * context's internal streams and wait only for the previous host map's use of
 * the context's staging buffers and for the spectra's builds.  So L_host must
 * hold its data when the call is made, and consecutive host maps overlap (one
 * map's passes and upload with the previous map's download).
 */
lp_status lp_map_host(lp_ctx* ctx, const float* L_host, int h, int w, int ldl,
                      const lp_spectrum* const* spectra, int n, float* const* out_host, int ldo,
                      lp_outmode mode, lp_precision prec, void* stream);

/*
 * Multi-class sources, Sec. 2.2 Eq. (4): B = sum_t K_t * L_t for T maps
 * (device FP32, each h x w with leading dimension ldl) and T spectra (same
 * rules as lp_map).  The spectrum products are summed before one inverse
 * transform.  out: device FP32, leading dimension ldo.  Only LP_PREC_FP32 is
 * built here (other precisions: LP_ERR_UNSUPPORTED).
 */
lp_status lp_map_multiclass(lp_ctx* ctx, const float* const* L, int T, int h, int w, int ldl,
                            const lp_spectrum* const* spectra, float* out, int ldo,
                            lp_outmode mode, lp_precision prec, void* stream);

/*
 * lp_map without any allocation.  There is no counterpart in the paper: this
 * is for callers that cannot let the library call cudaMalloc while they run
 * -- a host framework that owns all device memory through its own pool and
 * budget, or a latency-bound loop that cannot afford an allocation and the
 * device synchronisation it brings.  Arguments, layouts, results and errors
 * are those of lp_map, except:
 *   - the intermediate spectra live in one static device array of
 *     LP_NOALLOC_SCRATCH_BYTES (64 MiB) that every GPU loading this code
 *     holds until the process exits; a map whose lp_map_workspace_bytes()
 *     exceeds it is rejected with LP_ERR_INVALID (use lp_map instead);
 *   - the spectra must exist already (their creation builds the FFT plans),
 *     and pass timing must be off (it creates events); otherwise
 *     LP_ERR_INVALID;
 *   - the first call on a device looks the array's device address up
 *     (cudaGetSymbolAddress, with that device current) and caches it: make
 *     that first call before any stream capture;
 *   - all calls share the array: calls whose work overlaps on the GPU race
 *     and must be serialised by the caller.  Nothing needs clearing between
 *     calls (every scratch element read is first written by the same call).
 */
#define LP_NOALLOC_SCRATCH_BYTES (64ull << 20)

/*
 * CUDA graphs (no counterpart in the paper).  lp_map_noalloc, lp_map and
 * lp_map_tiled may be called on a stream that is being captured into a CUDA
 * graph (cudaStreamBeginCapture, any capture mode); the call then only
 * enqueues its kernels, so a loop of maps replays as one graph launch.
 * Conditions, each an LP_ERR_INVALID before anything is enqueued: every
 * spectrum's build has completed and been seen complete by an earlier
 * uncaptured map call (make one such call after lp_sync_status); pass
 * timing is off; lp_map and lp_map_tiled need their stream's workspace to
 * be large enough already (the same call once before capturing), since
 * growing it would allocate.  While capturing, the library neither frees
 * released spectra nor records their use, and it does not see the graph's
 * replays: keep L, out[] and the spectra alive while the graph may run.
 * lp_map_host cannot be captured (LP_ERR_INVALID).
 */
lp_status lp_map_noalloc(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                         const lp_spectrum* const* spectra, int n, float* const* out, int ldo,
                         lp_outmode mode, lp_precision prec, void* stream);

/* Size in bytes of the static scratch of lp_map_noalloc. */
size_t lp_map_noalloc_scratch_bytes(void);

/* Device bytes of workspace one lp_map call needs (0 if unsupported). */
size_t lp_map_workspace_bytes(int h, int w, int ny, int nx, int hk, int wk, int n,
                              lp_outmode mode);

/*
 * Wait (bounded by timeout_ms; < 0 = no limit) for `stream`, then read and
 * clear the context's sticky device status word.  LP_ERR_TIMEOUT if the
 * stream is still busy, LP_ERR_DEVICE if a kernel flagged an anomaly,
 * LP_ERR_CUDA for an asynchronous CUDA error.
 */
lp_status lp_sync_status(lp_ctx* ctx, void* stream, int timeout_ms);

/*
 * Test hooks (no counterpart in the paper; for the failure-detection tests).
 * LP_TEST_TC_NO_MMA: the split-precision column pass issues no tensor-core
 * instruction, so its first bounded MMA wait (100 ms of device time) runs
 * out; the kernel then sets bit 2 of the device status word, frees its
 * tensor memory and returns, and lp_sync_status reports LP_ERR_DEVICE.  The
 * context stays usable.  0 clears the hooks; unknown bits: LP_ERR_INVALID.
 */
#define LP_TEST_TC_NO_MMA 1
/* LP_TEST_FP_COLLIDE: every PSF gets the same cache fingerprint, so that
 * the value comparison that confirms a cache hit is what tells PSFs apart. */
#define LP_TEST_FP_COLLIDE 2
/* LP_TEST_SERVE_FAIL: the serving scheduler fails the next request it
 * admits as if its launch had failed (LP_ERR_CUDA, from the host: no kernel
 * runs), then clears the bit; the other requests are unaffected. */
#define LP_TEST_SERVE_FAIL 4
/* LP_TEST_BOUNDS: the map calls declare their intermediate buffer T one
 * column block shorter than it is.  In the debug build (LP_DEBUG=1, the
 * library paper_1907_02891_gb300/_build/debug/liblp.so, which checks every
 * work unit's extents in every buffer before touching global memory) the
 * units of the last columns then fail their checks: they are skipped and
 * set bit 3 of the device status word, so lp_sync_status reports
 * LP_ERR_DEVICE; no access leaves the real buffer.  The release build
 * compiles the checks away and ignores the hook. */
#define LP_TEST_BOUNDS 8
lp_status lp_set_test_hook(lp_ctx* ctx, int hook);

/*
 * Maps larger than the padded size (overlap-save tiling; Sec. 4 computes
 * extended regions band by band, here the pieces share one grid).  The SAME-mode result of
 * lp_map for an h x w map of any size, computed in tiles of
 * (Ny - hk + 1) x (Nx - wk + 1) output pixels, or in one tile along a
 * dimension where h <= Ny - (hk - 1) / 2 (w <= Nx - (wk - 1) / 2: the SAME
 * crop needs no more padding than that, less than lp_map's h + hk - 1):
 * each tile convolves the input
 * window that covers it plus the PSF's reach ((hk - 1) / 2 rows,
 * (wk - 1) / 2 columns, clipped to the map) in one P1 / P2 / P3 sequence,
 * which is exact for the tile's pixels (no wrap-around reaches them), and
 * writes its part of out[] in place.  The spectra need one PSF size and
 * any padded size Ny > hk - 1, Nx > wk - 1 (build them with an explicit
 * pad_ny / pad_nx; a larger pad gives fewer, larger tiles).  L, out[],
 * ldl, ldo, prec and stream as lp_map; the workspace holds one tile, and the
 * tiles run in stream order.  Errors as lp_map; LP_ERR_INVALID also for
 * spectra of different PSF sizes or a pad that leaves no tile.
 */
lp_status lp_map_tiled(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                       const lp_spectrum* const* spectra, int n, float* const* out, int ldo,
                       lp_precision prec, void* stream);

/*
 * Padded size for lp_map_tiled (host only, no device needed): per dimension
 * the supported length N >= hk (>= wk) that minimises the points transformed
 * over all tiles, tiles * N, with the tiles lp_map_tiled cuts (one where
 * h <= N - (hk - 1) / 2, else ceil(h / (N - hk + 1))); ties: fewer tiles.
 * For LP_PREC_SPLIT_BF16 the column length has the tensor-core pass.  A map
 * one transform holds usually gets one tile at the SAME crop's padding.
 * Errors: LP_ERR_INVALID (empty map, even or non-positive PSF sides, NULL
 * outputs), LP_ERR_UNSUPPORTED (precision, or no length holds the PSF);
 * the outputs are -1 on error.
 */
lp_status lp_tiled_pad(int h, int w, int hk, int wk, lp_precision prec, int* pad_ny, int* pad_nx);

/*
 * Serving: continuous batching of map requests.  lp_serve_start creates
 * n_slots CUDA streams (each with its own workspace) and a scheduler thread.
 * lp_serve_submit validates a request exactly like lp_map (LP_OUT_* mode;
 * the precision is the spectra's: LP_PREC_FP32, or LP_PREC_SPLIT_BF16 when
 * all of them were built in it) and queues it, holding a reference on each
 * spectrum until the request has finished; the scheduler starts queued requests in arrival order
 * as soon as a slot is free and the request's workspace fits, next to the
 * requests already running, into the serving capacity (the context's HBM
 * budget minus what it holds at start, or 90 % of the free device memory
 * when the context has no budget).  Requests admitted while others run
 * overlap with them on the device.  A request larger than the capacity is
 * refused at submission (LP_ERR_OOM); a full queue gives LP_ERR_BUSY.
 * The caller keeps L and out[] alive until the request is polled as
 * finished; the spectra may be released at any time after submission.
 *
 * lp_serve_poll waits up to timeout_ms (< 0: no limit) for a ticket:
 * LP_OK with the latency (submission to completion, milliseconds, host
 * clock), LP_ERR_TIMEOUT if still pending, or the request's failure status.
 * A finished ticket can be polled once.  lp_serve_stop drains the queue,
 * waits for running requests and releases the slots.
 */
lp_status lp_serve_start(lp_ctx* ctx, int n_slots);
lp_status lp_serve_submit(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                          const lp_spectrum* const* spectra, int n, float* const* out, int ldo,
                          lp_outmode mode, uint64_t* ticket);
lp_status lp_serve_poll(lp_ctx* ctx, uint64_t ticket, int timeout_ms, double* latency_ms);
lp_status lp_serve_stats(lp_ctx* ctx, uint64_t* completed, uint64_t* failed, int* queued,
                         int* running);
lp_status lp_serve_stop(lp_ctx* ctx);

/*
 * Cancel a queued request: LP_OK if it had not started (it never runs, its
 * spectrum references are dropped, and lp_serve_poll then returns
 * LP_ERR_CANCELLED for it), LP_ERR_BUSY if it is already running or
 * finished (work on the GPU is not interrupted), LP_ERR_INVALID for an
 * unknown ticket.
 */
lp_status lp_serve_cancel(lp_ctx* ctx, uint64_t ticket);

/*
 * Per-request log of the serving loop (metrics; no counterpart in the
 * paper).  While a log file is set, every finished request appends one JSON
 * line: ticket, status, h, w, n_psf, mode, precision, workspace_bytes,
 * output_mpix (h w n_psf / 1e6) and the host-clock times submit_ms,
 * start_ms (admitted and launched), end_ms (completion seen by the
 * scheduler's event poll, which runs every 20 us while requests are in
 * flight), all in ms from lp_serve_start, plus queue_ms = start - submit and
 * latency_ms = end - submit (the value lp_serve_poll returns).  path is
 * opened for appending (LP_ERR_INVALID if it cannot be); NULL or "" closes
 * the log.  lp_serve_stop closes it too.  LP_ERR_BUSY when serving has not
 * started.
 */
lp_status lp_serve_log(lp_ctx* ctx, const char* path);

/*
 * Pass timing (tracing).  While enabled, every map call records CUDA events
 * around each of its kernel passes on its own stream:
 *   pass 0 = row forward transform (P1), 1 = column transform with the
 *   spectrum product (P2), 2 = row inverse transform and crop (P3).
 * lp_get_pass_timing waits for the recorded work, returns the summed
 * milliseconds and launch counts per pass (arrays of 3) and clears them.
 */
lp_status lp_set_pass_timing(lp_ctx* ctx, int enable);
lp_status lp_get_pass_timing(lp_ctx* ctx, double* ms, int* launches);

#ifdef __cplusplus
}
#endif

#endif /* LP_H */
