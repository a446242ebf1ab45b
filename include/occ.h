/*
 * occ.h -- C ABI of the GB300 (sm_103a) fast edge-aware occlusion detection library.
 *
 * The library computes, for a fused center-view disparity map D and the baseline direction of each peripheral
 * camera, the center pixels that the peripheral camera does not see (Sippel, Seiler, Kaup, "Fast Edge-Aware
 * Occlusion Detection in the Context of Multispectral Camera Arrays", ICIP 2024, Section 3):
 *   Eq. 1   forward-difference edge maps E_x, E_y of D, the magnitude E and the angle A;
 *   Eq. 2   candidates C: E > gamma and the gradient pointing along the baseline angle alpha;
 *   Eq. 3   scan length L = ceil(2 (max D - min D));
 *   Eq. 4   a scan line of 2h+1 samples (h = ceil(L/2)) along alpha through every candidate, with depth values V;
 *           the warp W = G - V of each sample, and the sort of each scan line by (W, k);
 *   Eq. 5   the occlusion count of every sorted sample against its N nearest sorted neighbours
 *           (|W_p - W_q| < zeta and V_p + beta < V_q);
 *   Eq. 6   the occlusion sum O (every scan line's counts accumulated per pixel) and the mask M = (O > 0).
 *
 * Readings of the paper's silent or garbled passages, applied everywhere below:
 *   - alpha is the direction from the center camera to the peripheral camera, in degrees, measured from +x
 *     (columns) toward +y (rows, pointing down); content moves by -r D along alpha, so W = G - V.
 *   - The disparity test of Eq. 5 is V_p + beta < V_q (p is behind q by more than beta).
 *   - The angle test of Eq. 2 is the sign test E_x cos(alpha) + E_y sin(alpha) > 0 (equivalent to
 *     |wrap(atan2(E_y, E_x) - alpha)| < pi/2); cos and sin are rounded to binary32 after reducing alpha to
 *     [0, 45] degrees, so multiples of 90 degrees give exact 0 and +-1.
 *   - A peripheral camera with baseline ratio r (its baseline over the axial one) sees disparity r D: the whole
 *     method runs on D_r = fl(r D); E and A outputs are those of D itself (r = 1).
 *   - Scan line positions are rounded to the nearest pixel (ties away from zero); samples outside the image are
 *     dropped; the sort key is (W ascending, k ascending); overlapping scan lines add up in O.
 * All arithmetic that decides M and O is binary32, round-to-nearest, one operation at a time (no contraction),
 * so M and O are reproducible bit for bit.
 *
 * Memory and streams.  Every device pointer is a plain CUDA device address on the context's device (for example
 * torch.Tensor.data_ptr() of a CUDA tensor).  Calls are asynchronous on the given stream (a cudaStream_t passed as
 * void*, NULL = the legacy default stream); outputs are complete when the stream reaches that point.  One context
 * serves one host thread and one stream at a time.
 *
 * Errors.  Every entry point returns an int status.  Argument errors are detected on the host before any work is
 * queued (OCC_ERR_INVALID_ARG).  Conditions only the device can see (non-finite input, candidate list overflow,
 * a scan length above OCC_MAX_SCAN) set bits in a device status word that occ_get_status() reads; while that
 * status is not OCC_OK the outputs of that call are unspecified.  No call aborts, traps or throws.
 */
#ifndef OCC_H
#define OCC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define OCC_OK 0
#define OCC_ERR_INVALID_ARG 1     /* a host-checked argument is out of range */
#define OCC_ERR_NONFINITE_INPUT 2 /* D holds a NaN or an infinity (the method is defined for finite maps) */
#define OCC_ERR_CAPACITY 3        /* candidate list overflow, or the automatic L exceeds OCC_MAX_SCAN */
#define OCC_ERR_TIMEOUT 4         /* a bounded device wait gave up */
#define OCC_ERR_CUDA 5            /* a CUDA runtime call failed (allocation, launch, copy) */

/* Limits. */
#define OCC_MAX_VIEWS 64     /* views per call */
#define OCC_MAX_FRAMES 1024  /* frames per occ_detect_batched call */
#define OCC_MAX_SCAN 4094    /* largest scan length L (Eq. 3); 2h+1 <= 4095 samples per scan line */
#define OCC_MAX_SIDE 65535   /* largest H and W */
#define OCC_MAX_N 64         /* largest neighbour count N (Eq. 5) */

typedef struct occ_ctx occ_ctx; /* opaque; owns the device scratch of one device */

/* One peripheral view: baseline angle alpha in degrees (Eq. 2, Eq. 4) and baseline ratio r > 0. */
typedef struct {
    double alpha_deg;
    float ratio;
} occ_view;

/* Parameters of Section 3.  gamma: edge threshold (Eq. 2).  zeta: distance threshold and beta: disparity threshold
 * (Eq. 5).  L: scan length; L <= 0 computes it per view by Eq. 3 on the device.  N: neighbours compared per sorted
 * sample (Eq. 5), even, 2 <= N <= OCC_MAX_N.  The paper fits gamma = 1.0, zeta = 2.0, beta = 0.5 on SceneFlow
 * (Section 4.1) and gives no N; occ_default_params() returns those values with N = 8. */
typedef struct {
    float gamma;
    float zeta;
    float beta;
    int32_t L;
    int32_t N;
} occ_params;

/* Work counts of one view of the last occ_detect call: |C| (Eq. 2), scan line samples inside the image, (p, d)
 * neighbour pairs tested (Eq. 5), and the scan length used (Eq. 3). */
typedef struct {
    int64_t candidates;
    int64_t samples;
    int64_t pair_tests;
    int32_t L;
    int32_t reserved;
} occ_view_stats;

/* Fills *p with gamma 1.0, zeta 2.0, beta 0.5, L 0 (automatic), N 8. */
void occ_default_params(occ_params* p);

/* The binary32 cos and sin of alpha_deg used by Eq. 2 and Eq. 4 (reduction to [0, 45] degrees, evaluation in
 * double, one rounding).  Host only; never fails. */
void occ_direction(double alpha_deg, float* c, float* s);

/* Creates a context on CUDA device `device` and allocates its scratch: the candidate lists (max_candidates entries
 * per view; <= 0 means max_pixels, which never overflows), the status word and the per-view counters.  A view that
 * takes the strip kernel (see occ_tuning) lists only its scan lines of three or more macro-runs there.
 * max_pixels >= 1 bounds H*W of later calls; 1 <= max_views <= OCC_MAX_VIEWS.  On success *out receives the
 * context; on failure *out is NULL and the return is OCC_ERR_INVALID_ARG or OCC_ERR_CUDA. */
int occ_create(occ_ctx** out, int device, int64_t max_pixels, int32_t max_views, int64_t max_candidates);

/* Frees the context and all its device memory.  NULL is ignored.  The caller makes sure no queued work still
 * uses the context (synchronise its stream first). */
void occ_destroy(occ_ctx* ctx);

/*
 * The whole method of Section 3 (Eq. 1-6) for one frame and n_views views, queued on `stream`.
 *   D      device, binary32 [H][pitch] row-major (x = column, y = row pointing down), 4-byte aligned, read only;
 *          pitch (elements) >= W, or 0 for pitch = W.  1 <= H, W <= OCC_MAX_SIDE, H*W <= the context's max_pixels.
 *   views  host, n_views entries (1 <= n_views <= the context's max_views), copied during the call;
 *          alpha finite, ratio finite and > 0.
 *   p      host, copied during the call; NULL means occ_default_params().  zeta > 0, all thresholds finite.
 *   M      device, uint8 [n_views][H][W], required: 1 where O > 0, else 0 (Eq. 6).  Fully overwritten.
 *   O      device, int32 [n_views][H][W], 4-byte aligned, or NULL: the occlusion sum of Eq. 5/6 per pixel.  Fully
 *          overwritten.  When NULL the context uses scratch of its own, allocated on the first such call.
 *   E, A   device, binary32 [H][W], or NULL: the edge magnitude and angle maps of D (r = 1), A = atan2(E_y, E_x).
 * The caller owns D, M, O, E and A; none may overlap.  Returns OCC_OK once the work is queued, or
 * OCC_ERR_INVALID_ARG / OCC_ERR_CUDA without queueing anything.  Device-detected errors surface through
 * occ_get_status().  A call that allocates (see O above) must not run under stream capture.
 */
int occ_detect(occ_ctx* ctx, const float* D, int32_t H, int32_t W, int64_t pitch, const occ_view* views,
               int32_t n_views, const occ_params* p, uint8_t* M, int32_t* O, float* E, float* A, void* stream);

/*
 * occ_detect on host buffers: copies D (host, binary32 [H][W], pinned memory recommended) to the device, runs
 * occ_detect, copies M (and O when O_host is not NULL) back to host memory, and waits for the stream.
 * D_host, M_host [n_views][H][W] and O_host [n_views][H][W] are host pointers owned by the caller.  The device
 * staging buffers are owned by the context and allocated on the first call.  Returns the status of the whole
 * call, device-detected errors included (as occ_get_status() would).
 */
int occ_detect_host(occ_ctx* ctx, const float* D_host, int32_t H, int32_t W, const occ_view* views,
                    int32_t n_views, const occ_params* p, uint8_t* M_host, int32_t* O_host, void* stream);

/*
 * occ_detect_host without the wait: returns OCC_OK once the copy in, the detection and the copies out are queued on
 * `stream` (or OCC_ERR_INVALID_ARG / OCC_ERR_CUDA without queueing anything).  D_host must stay unchanged, and
 * M_host / O_host must not be read, until the stream reaches that point; occ_get_status(ctx, stream) then gives the
 * call's device-detected status.  The copies run asynchronously only on pinned host memory.  Frames on two contexts
 * and two streams overlap one frame's copies with the other's detection; calls on one context must not overlap on
 * the GPU (they share its staging buffers), so a context takes its next frame on the same stream.
 */
int occ_detect_host_async(occ_ctx* ctx, const float* D_host, int32_t H, int32_t W, const occ_view* views,
                          int32_t n_views, const occ_params* p, uint8_t* M_host, int32_t* O_host, void* stream);

/*
 * The method for n_frames frames of possibly different sizes and the same views, queued as one batch: a handful of
 * launches for the whole batch (the candidate pass over every frame, one plan, one persistent launch of each scan
 * kernel over every frame, view and candidate, one mask pass), with results identical to n_frames occ_detect calls.
 * No call allocates, so the batch can be captured into a CUDA graph and replayed.
 *   D[f]   device, binary32 [H[f]][W[f]] row-major (pitch = W[f]); H, W, D, M, O are host arrays of n_frames
 *          entries; 1 <= n_frames <= OCC_MAX_FRAMES; the sum of H[f] * W[f] must not exceed the context's max_pixels.
 *   M[f]   device, uint8 [n_views][H[f]][W[f]]; O[f] device, int32 [n_views][H[f]][W[f]]: both required.
 * Each frame's candidate lists get the context's per-pixel share of its capacity (all of a frame's pixels with the
 * default max_candidates, so they never overflow).  occ_get_status reports the OR of every frame's conditions;
 * occ_get_stats sums candidates, samples and pair tests over the frames and reports the largest L.  Returns OCC_OK
 * once queued, OCC_ERR_INVALID_ARG, OCC_ERR_CAPACITY (before any work is queued) when the frames' candidate lists
 * together hold more than 2^32 - 1 entries (n_views times each frame's share; split the batch or create the context
 * with a smaller max_candidates), or OCC_ERR_CUDA.
 */
int occ_detect_batched(occ_ctx* ctx, int32_t n_frames, const float* const* D, const int32_t* H, const int32_t* W,
                       const occ_view* views, int32_t n_views, const occ_params* p, uint8_t* const* M,
                       int32_t* const* O, void* stream);

/* Waits for `stream` and returns the device status of the last occ_detect call of this context: OCC_OK,
 * OCC_ERR_NONFINITE_INPUT, OCC_ERR_CAPACITY or OCC_ERR_TIMEOUT (in that priority), or OCC_ERR_CUDA if the wait
 * itself failed. */
int occ_get_status(occ_ctx* ctx, void* stream);

/* Copies the work counts of the first n_views views of the last occ_detect / occ_detect_batched call into out (host;
 * summed over the frames of a batch, L the largest).  Waits for the last stream used.  Returns OCC_ERR_INVALID_ARG if
 * n_views exceeds the views of that call. */
int occ_get_stats(occ_ctx* ctx, occ_view_stats* out, int32_t n_views);

/* How the scan work (Eq. 4-6) is mapped onto the GPU; every choice gives bit-identical results, only the speed
 * differs (paper_2408_14050_gb300/autotune.py picks one per device and workload).
 *   line_max_runs        scan lines handled one per thread: 0 none (one warp per line for all), 1 lines whose
 *                        sort needs only adjacent swaps, 2 also lines made of two such stretches (default 2).
 *                        Ignored (0) when N > 8.
 *   line_blocks_per_sm   resident 256-thread blocks per multiprocessor of the line-per-thread kernel, 1 .. the
 *                        occupancy limit (default: the limit).
 *   warp_lines_per_block lines in flight per block of the one-warp-per-line kernel for lines of <= 256 samples:
 *                        4 or 8 (default 8).
 *   strip_px             the strip kernel, for the views whose scan lines stay on one row, column or diagonal
 *                        (alpha a multiple of 45 degrees) when N = 8 and no side of a frame exceeds 4096 pixels:
 *                        one block owns a strip of adjacent such lines of about strip_px pixels, holds D_r and O of
 *                        it in shared memory and writes O and M once.  0 turns it off (every view takes the
 *                        candidate-list kernels above); otherwise 1024 .. OCC_STRIP_PX_MAX, a multiple of 64,
 *                        raised for a call to its longest row, column or diagonal (default 4096).
 *   fused                1: a call whose views all take the strip kernel and that asks for no E, A or tile hits
 *                        runs as one kernel launch (the min/max of Eq. 3, the plan, the strips and the lines of
 *                        three or more macro-runs, with bounded waits between them; see occ_set_wait_limit), when
 *                        the context's scratch has room for its work lists; 0 (default): the same work in separate
 *                        launches, which measure faster on GB300. */
#define OCC_STRIP_PX_MAX 16384
typedef struct {
    int32_t line_max_runs;
    int32_t line_blocks_per_sm;
    int32_t warp_lines_per_block;
    int32_t strip_px;
    int32_t fused;
} occ_tuning;

/* Sets the tuning of later calls (NULL: the defaults).  OCC_ERR_INVALID_ARG for out-of-range fields. */
int occ_set_tuning(occ_ctx* ctx, const occ_tuning* t);

/* The tuning in effect, with the occupancy limit of line_blocks_per_sm in *max_line_blocks_per_sm (may be NULL). */
int occ_get_tuning(occ_ctx* ctx, occ_tuning* t, int32_t* max_line_blocks_per_sm);

/* The bound of every wait of the fused launch (occ_tuning.fused) between its stages: wait_us microseconds (0: the
 * default of 2 s; at most 60 s).  A wait that reaches it makes every block of the launch stop and the call's status
 * OCC_ERR_TIMEOUT (occ_get_status), with O and M unspecified; the context stays usable.  hold != 0 is a test hook:
 * the fused launches of later calls never release the frames' plans, so that their strips' waits reach the bound.
 * OCC_ERR_INVALID_ARG for a negative or too large wait_us. */
int occ_set_wait_limit(occ_ctx* ctx, int64_t wait_us, int32_t hold);

/* Stages of one occ_detect call, in launch order: candidates (Eq. 1-2 and the min/max of Eq. 3), the
 * line-per-thread scan (Eq. 4-6 for the scan lines whose sort is a set of adjacent swaps, or two such stretches;
 * N <= 8), the warp scan kernels of the three scan-line size classes (2h+1 <= 256, <= 1024, <= 4096 samples; Eq. 4-6
 * for the remaining lines), and the mask (Eq. 6).  When the line-per-thread kernels run (line_max_runs >= 1), calls of
 * up to 64 Mi pixel-views run the warp scan kernels on a second stream of the context beside the end of the
 * line-per-thread stage: their stage times count from where they start, and the mask's from the later of the two. */
#define OCC_NUM_STAGES 6

/* enable != 0: later occ_detect calls record a CUDA event before and after each stage, so that
 * occ_get_timings() can report the device time of each stage.  Off by default.  Returns OCC_OK or
 * OCC_ERR_INVALID_ARG. */
int occ_set_profiling(occ_ctx* ctx, int enable);

/* Device milliseconds of the first n (<= OCC_NUM_STAGES) stages of the last occ_detect call made with profiling on
 * (0 for a stage that was not launched), written to ms (host).  Waits for that call's last event.  Returns
 * OCC_ERR_INVALID_ARG if no profiled call was made. */
int occ_get_timings(occ_ctx* ctx, float* ms, int32_t n);

/* Largest H * W * n_views that occ_detect_noalloc accepts: its fixed scratch holds one candidate entry per pixel and
 * view (4 bytes each), e.g. one 1920x1080 map with 8 views. */
#define OCC_NOALLOC_MAX_PIXEL_VIEWS 16777216

/*
 * occ_detect without a context and without any device allocation, for callers that cannot call cudaMalloc: code
 * running where the allocator must not be touched (inside a custom allocator or memory-pool callback, a
 * real-time loop that may not block on allocation or risk fragmentation, a host whose memory budget is fixed and
 * fully reserved up front, or a framework that hands out only the tensors it manages).  The paper has no counterpart;
 * this is a deployment variant of the same computation with the same results.
 *
 * Its scratch (headers, counters and plan, 4 KB, scan-line position tables, 1 MiB, a bit per pixel and view, the
 * candidate lists, 4 bytes per pixel and view, and the list of scan lines handed from the line kernel to the merge
 * kernel, 4 more) is one array of about 131 MiB built into the library: every GPU on which the library is used holds
 * it until the process exits.  The call itself allocates and frees nothing.  Every call on a device
 * shares that array and overwrites it, clearing first what must start at zero; two calls that may run at the same
 * time on the GPU (different streams, or different host threads) race on it and give wrong results, so serialise
 * them (one stream).  The first call on a device also looks up the array's device address and sets the kernels'
 * shared-memory limits for that device (under a lock, with that device current; a set-up that fails is tried again
 * by the next call): make that first call before any stream capture.
 *
 * Arguments are those of occ_detect on the current CUDA device (D, M, O device pointers, views and p host), except:
 * O is required; there are no E / A outputs; status (device int32, or NULL) receives, in stream order, 0 when the
 * device found nothing wrong, else a non-zero value (bit 0: non-finite input; bit 2: automatic L above OCC_MAX_SCAN),
 * in which case M and O are unspecified.  Every view gathers from D directly.  Returns OCC_OK once the work is
 * queued; OCC_ERR_INVALID_ARG for bad arguments; OCC_ERR_CAPACITY, before any work is queued, when H * W * n_views
 * exceeds OCC_NOALLOC_MAX_PIXEL_VIEWS; OCC_ERR_CUDA if a launch fails.
 */
int occ_detect_noalloc(const float* D, int32_t H, int32_t W, int64_t pitch, const occ_view* views, int32_t n_views,
                       const occ_params* p, uint8_t* M, int32_t* O, int32_t* status, void* stream);

/*
 * The fused center map D as the pixel-wise median of the n_maps stereo disparity maps that the peripheral cameras
 * give for the center view (Section 4.2: the maps are fused by a pixel-wise median before the detection runs).
 * maps: n_maps (1..64) device pointers, each a binary32 [H][pitch] map (pitch in elements, 0 = W), read only.
 * D: device binary32 [H][d_pitch] output (0 = W); it may be one of the maps only if d_pitch equals pitch.  For odd
 * n_maps the result is the middle value; for even n_maps fl(fl(a + b) * 0.5) of the two middle values; a zero of
 * either sign counts as +0.  Runs on the current CUDA device, asynchronously on `stream`; allocates nothing.
 * status (device int32, or NULL) receives, in stream order, 0, or OCC_ERR_NONFINITE_INPUT when some map holds a NaN
 * or an infinity (D is then unspecified).  Returns OCC_OK once queued, OCC_ERR_INVALID_ARG for bad arguments (NULL
 * or misaligned pointers, sizes out of range), OCC_ERR_CUDA if the launch fails.
 */
int occ_fuse_median(const float* const* maps, int32_t n_maps, int32_t H, int32_t W, int64_t pitch, float* D,
                    int64_t d_pitch, int32_t* status, void* stream);

/*
 * Backward warp of the peripheral images to the center view (Section 1: every view is warped to the center view;
 * Section 4.2: the pixels the detection marks are the ones left for reconstruction).  For view v (alpha, ratio r as
 * in occ_detect) the center pixel (x, y) takes the bilinear interpolation of images[v] at
 * (x - cos(alpha) fl(r D), y - sin(alpha) fl(r D)), evaluated as top = I00 + fx (I01 - I00), bottom = I10 + fx
 * (I11 - I10), top + fy (bottom - top) with one binary32 rounding per operation and the upper neighbours clamped to
 * the last row / column; pixels with M[v] != 0, positions outside [0, W-1] x [0, H-1] and non-finite D give 0.
 * D: device binary32 [H][pitch] (0 = W).  images: n_views (1..64) device pointers to binary32 [H][img_pitch]
 * (0 = W).  M: device uint8 [n_views][H][W] (the mask of occ_detect), or NULL for no mask.  out: device binary32
 * [n_views][H][W]; it must not overlap the inputs.  Runs on the current CUDA device, asynchronously on `stream`;
 * allocates nothing.  Returns OCC_OK once queued, OCC_ERR_INVALID_ARG for bad arguments (NULL or misaligned
 * pointers, a ratio that is not finite and positive, sizes out of range), OCC_ERR_CUDA if the launch fails.
 */
int occ_warp_views(const float* D, int32_t H, int32_t W, int64_t pitch, const occ_view* views, int32_t n_views,
                   const float* const* images, int64_t img_pitch, const uint8_t* M, float* out, void* stream);

/* Side of the square pixel tiles of occ_detect_batched_tiles (proposals and hit flags). */
#define OCC_TILE 32

/*
 * occ_detect_batched with per-tile control of the candidates, for the learned tile proposer (a concrete form of the
 * paper's closing remark that thinning the candidate list would cut the runtime further) and for its training labels.
 * The frame is cut into tiles of OCC_TILE x OCC_TILE pixels, tiles_x = ceil(W / OCC_TILE) by tiles_y =
 * ceil(H / OCC_TILE) (the last row and column of tiles may be partial); a candidate belongs to the tile of its own
 * pixel.
 *   proposal   n_frames pointers (or NULL for "every tile" in all frames; an individual NULL likewise), each to a
 *              device uint8 [n_views][tiles_y][tiles_x]: 0 = the scan lines of the candidates of that tile and view
 *              are not walked (Eq. 4-6 skip them), non-zero = they are.  With every entry non-zero the results equal
 *              occ_detect_batched's.  Otherwise M and O equal the method run on the candidate list restricted to the
 *              proposed tiles.
 *   tile_hits  n_frames pointers (or NULL), each to a device uint8 [n_views][tiles_y][tiles_x] that receives 1 where
 *              at least one scan line walked from a candidate of the tile added a non-zero count to O (Eq. 5-6), else
 *              0: the per-tile label "the tile's candidates find an occlusion" of the plain method.
 * Everything else is as for occ_detect_batched.
 */
int occ_detect_batched_tiles(occ_ctx* ctx, int32_t n_frames, const float* const* D, const int32_t* H,
                             const int32_t* W, const occ_view* views, int32_t n_views, const occ_params* p,
                             const uint8_t* const* proposal, uint8_t* const* M, int32_t* const* O,
                             uint8_t* const* tile_hits, void* stream);

/*
 * Learned tile proposer.  A small convolutional network scores, for every OCC_TILE x OCC_TILE tile of a center map D
 * and every view, whether the scan lines of the tile's candidates find an occlusion, so that occ_detect_batched_tiles
 * can skip the tiles it rules out (a concrete form of the paper's closing remark, Section 5, that thinning the
 * candidate list would cut the runtime further).  It is trained on the tile_hits labels of the plain method.
 *
 * Network (all tensors NHWC; bf16 = bfloat16 rounded to nearest even):
 *   x0       = bf16(fl(D / 32) - 1) in channel 0 of 8, channels 1..7 zero
 *   a_l      = bf16(relu(conv3x3(a_{l-1}, bf16(W_l)) + b_l)), l = 1..4, channels 8 -> 16 -> 16 -> 32 -> 16, zero
 *              padding ('same'), bf16 products summed in fp32 on the tensor cores
 *   g(v)     = We (cos alpha, sin alpha, r) + be                 (16 values; cos, sin as occ_direction gives them)
 *   z_v(p)   = sum_c a_4(p)[c] g_c(v) + b0
 *   s_v(t)   = log(mean over the tile's pixels of exp(z_v))       (the tile logit; partial tiles use their pixels)
 *   loss     = mean over frames, views and tiles of -(w y log sigmoid(s) + (1 - y) log(1 - sigmoid(s)))
 * Back-propagated gradients of the pre-activations are gated by a_l > 0 and stored as bf16, like the activations.
 *
 * Parameters: one fp32 vector of OCC_NET_PARAMS values: per layer W_l [c_out][9][c_in] (tap = (dy+1)*3 + (dx+1))
 * then b_l [c_out]; then We [16][3], be [16], b0.
 *
 * Frames: n maps of one size H x W, contiguous ([n][H][W] binary32 device memory).  Per-tile tables (logits,
 * labels, proposals) are [n][n_views][tiles_y][tiles_x] with tiles_y = ceil(H / OCC_TILE), tiles_x = ceil(W /
 * OCC_TILE).  All calls run asynchronously on `stream` (NULL: the legacy default stream) on the network's device,
 * except occ_net_set_params / occ_net_get_params, which wait.  Returns as for the detection: OCC_OK once queued,
 * OCC_ERR_INVALID_ARG, OCC_ERR_CAPACITY (n * H * W above the network's max_pixels), OCC_ERR_CUDA.
 */
#define OCC_NET_PARAMS 12817

typedef struct occ_net occ_net;

/* Network state on `device`: parameters, Adam moments, bf16 operand copies, activations for up to max_pixels pixels
 * (n * H * W) per call, up to max_views views.  Parameters start at zero: set them before use. */
int occ_net_create(occ_net** out, int device, int64_t max_pixels, int32_t max_views);
void occ_net_destroy(occ_net* net);

/* Copy the fp32 parameter vector in from / out to host memory (count must be OCC_NET_PARAMS).  Setting them also
 * clears the Adam moments.  Both wait for completion. */
int occ_net_set_params(occ_net* net, const float* params, int64_t count);
int occ_net_get_params(occ_net* net, float* params, int64_t count);

/* Tile logits s [n][n_views][tiles_y][tiles_x] (device fp32) of the maps D. */
int occ_net_forward(occ_net* net, const float* D, int32_t n, int32_t H, int32_t W, const occ_view* views,
                    int32_t n_views, float* logits, void* stream);

/* Forward and backward pass on labelled maps: labels [n][n_views][tiles_y][tiles_x] (device uint8, non-zero = the
 * tile's candidates find an occlusion), positive weight w > 0.  Writes the loss (device fp32 [1]), the gradient of the
 * loss with respect to the parameter vector (device fp32 [OCC_NET_PARAMS], overwritten) and, if logits is not NULL,
 * the tile logits. */
int occ_net_loss_grad(occ_net* net, const float* D, int32_t n, int32_t H, int32_t W, const occ_view* views,
                      int32_t n_views, const uint8_t* labels, float pos_weight, float* grads, float* loss,
                      float* logits, void* stream);

/* One Adam step (step = 1, 2, ... for the bias corrections) on the fp32 parameters with the device gradient `grads`,
 * then the bf16 operand copies are refreshed. */
int occ_net_adam(occ_net* net, const float* grads, float lr, float beta1, float beta2, float eps, int32_t step,
                 void* stream);

/* proposal[i] = logits[i] > threshold (device arrays of `count` entries): the proposal table of
 * occ_detect_batched_tiles. */
int occ_net_propose(const float* logits, int64_t count, float threshold, uint8_t* proposal, void* stream);

/* OCC_ERR_TIMEOUT if a bounded wait of a network kernel on the tensor cores expired (on the current device) since
 * the library was loaded, else OCC_OK.  Waits for `stream`. */
int occ_net_status(void* stream);

/* One 3x3 'same' convolution layer of the network on the tensor cores, for tests and custom pipelines.  X: device
 * bf16 [n][H][W][c_in]; Wb: device bf16 [c_out][K] with K = 9 * c_in rounded up to a multiple of 16, k = tap * c_in
 * + ci, zero beyond 9 * c_in; bias: device fp32 [c_out] or NULL; gate: device bf16 [n][H][W][c_out] or NULL (an output
 * whose gate value is not > 0 becomes 0); relu != 0 clamps at 0 after the bias; Y: device bf16 [n][H][W][c_out].
 * (c_in, c_out) is one of (8, 16), (16, 16), (16, 32), (32, 16).  X, Wb, gate, Y 16-byte aligned. */
int occ_net_conv3x3(const void* X, int32_t n, int32_t H, int32_t W, int32_t c_in, const void* Wb, const float* bias,
                    int32_t c_out, const void* gate, int32_t relu, void* Y, void* stream);

/* Weight gradient of that layer on the tensor cores: dWt[tap * c_in + ci][co] += sum over pixels p of
 * X[p + tap][ci] dY[p][co] (zero padding), and dWt[9 * c_in][co] += sum_p dY[p][co] (the bias gradient).  X, dY as
 * above (16-byte aligned); dWt: device fp32 [9 * c_in + 1][c_out], accumulated. */
int occ_net_conv3x3_wgrad(const void* X, const void* dY, int32_t n, int32_t H, int32_t W, int32_t c_in,
                          int32_t c_out, float* dWt, void* stream);

/* A static, human-readable name of a status code. */
const char* occ_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* OCC_H */
