// occ_internal.cuh -- launch arguments and per-frame records shared by the kernels (occ_kernels.cu) and the host side
// of the C ABI (occ_api.cu, occ_noalloc.cu).  Not part of the public interface.
//
// Every call runs a batch of frames (one for occ_detect): the host writes one FrameArg per frame into a device
// table, k_plan derives per (frame, view) the scan length, the size class of the scan lines and the prefix sums that
// number the scan work items, and every kernel finds its frame and view from those tables.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "occ.h"

namespace occ {

constexpr int kMaxViews = OCC_MAX_VIEWS;
constexpr int kMaxFrames = OCC_MAX_FRAMES;

// Words of the per-frame device header (uint32); the host clears the headers and statistics of a call with one
// memset, the kernels fill them in stream order.
enum : int {
    HDR_STATUS = 0,                  // status bits of the frame (ST_*)
    HDR_MAX = 1,                     // max D, order-preserving encoding (atomicMax)
    HDR_NEGMIN = 2,                  // min D, complemented encoding (atomicMax)
    HDR_MMDONE = 3,                  // fused launch: min/max tickets of the frame done
    HDR_READY = 4,                   // fused launch: the frame's plan is written (1)
    HDR_COUNT = 8,                   // [kMaxViews] candidates found per view (may exceed the list capacity)
    HDR_L = HDR_COUNT + kMaxViews,   // [kMaxViews] scan length used per view (Eq. 3)
    HDR_OVF = HDR_L + kMaxViews,     // [kMaxViews] strip views: lines of three or more macro-runs listed for k_scan
    HDR_WORDS = HDR_OVF + kMaxViews,
};

// Device status bits.
enum : uint32_t {
    ST_NONFINITE = 1u,       // D holds NaN or Inf
    ST_CAND_OVERFLOW = 2u,   // more candidates than the list holds
    ST_SCAN_TOO_LONG = 4u,   // automatic L above OCC_MAX_SCAN
    ST_TIMEOUT = 8u,         // a bounded wait gave up
    ST_INTERNAL = 16u,       // a self-check failed (never expected)
};

// Scan-length classes of the warp scan kernel, sized by the samples of one scan line (2h+1).
constexpr int kNumClasses = 3;
constexpr int kTile = OCC_TILE;     // side of the square tiles of proposals and hit flags
constexpr int kClassCap[kNumClasses] = {256, 1024, 4096};
// The line-per-thread scan kernel keeps N/2 sorted neighbours in registers; larger N use the warp kernel only.
constexpr int kLineMaxHalf = 4;
// Position tables: per view, for g = -kTabHalf .. kTabHalf, round(fl(cos a * g)) and round(fl(sin a * g)).
constexpr int kTabHalf = (OCC_MAX_SCAN + 1) / 2;
constexpr int kTabLen = 2 * kTabHalf + 1;
// The strip kernel's offsets round(fl(cc * g)) of sample g along its line, for g = -kTabHalf .. kTabHalf + 8 (the
// entries past kTabHalf keep reads a step or two ahead of a line's end in bounds): one table per value of cc, which
// for the strip directions is cos or sin of the view rounded to binary32, +-1 or +-fl(sqrt(1/2)) (kNumSTabs tables,
// written once when the scratch is set up).
constexpr int kSTabLen = kTabLen + 8;
constexpr int kNumSTabs = 4;   // cc = 1, -1, fl(sqrt(1/2)), -fl(sqrt(1/2))

struct ViewArg {
    float c, s, r;   // binary32 cos(alpha), sin(alpha), ratio
    int32_t ridx;    // index of r in Args::ratio
    int32_t fam;     // strip family of the view's scan lines (kFam*), or -1: the view takes the list path
    int32_t stab;    // strip views: which of the kNumSTabs offset tables (cc = sin for columns, else cos)
};

// Directions whose scan lines (Eq. 4) stay on one digital line of the frame: rows (alpha = 0, 180), columns (90, 270),
// diagonals x - y = const (45, 225: cos = sin) and anti-diagonals x + y = const (135, 315: cos = -sin).  Along such a
// line the sample of g lies t = round(fl(cc * g)) positions from the candidate, cc = sin(alpha) for columns and
// cos(alpha) otherwise; for the diagonal directions this equals Eq. 4's per-coordinate rounding whenever every
// coordinate is below kStripMaxSide (checked exhaustively for |g| <= 2047 by the tests).
enum : int { kFamRows = 0, kFamCols = 1, kFamDiag = 2, kFamAnti = 3 };
constexpr int kStripMaxSide = 4096;
constexpr int kStripMaxLines = 16;   // lines of one strip (4 bits of a queue entry; the position takes 12)
constexpr int kStripPxDefault = 4096;

__host__ __device__ __forceinline__ int fam_lines(int fam, int H, int W)
{
    return fam == kFamRows ? H : (fam == kFamCols ? W : W + H - 1);
}
__host__ __device__ __forceinline__ int fam_len(int fam, int H, int W)
{
    return fam == kFamRows ? W : (fam == kFamCols ? H : (W < H ? W : H));
}
// Lines per strip: as many as fit strip_px pixels (at least one, at most kStripMaxLines).
__host__ __device__ __forceinline__ int strip_lines(int fam, int H, int W, int strip_px)
{
    const int b = strip_px / fam_len(fam, H, W);
    return b < 1 ? 1 : (b > kStripMaxLines ? kStripMaxLines : b);
}
__host__ __device__ __forceinline__ int fam_strips(int fam, int H, int W, int strip_px)
{
    const int b = strip_lines(fam, H, W, strip_px);
    return (fam_lines(fam, H, W) + b - 1) / b;
}

// Number of (p, d) pairs with d in {-K..K}\{0} and 0 <= p+d < n, summed over p (Eq. 5's neighbour set).
__host__ __device__ __forceinline__ unsigned long long pair_count(int n, int K)
{
    const long long nn = n, kk = K;
    const long long one_side = (nn <= kk) ? nn * (nn - 1) / 2 : kk * (kk - 1) / 2 + (nn - kk) * kk;
    return (unsigned long long)(2 * one_side);
}

// One frame of a call.
struct FrameArg {
    const float* D;               // [H][pitch]
    int64_t pitch;
    int32_t H, W;
    int32_t wide;                 // (H - 1) * pitch + W does not fit in int32
    int32_t pad;
    int32_t* O;                   // [nv][H][W]
    uint8_t* M;                   // [nv][H][W]
    float* E;                     // [H][W] or null
    float* A;                     // [H][W] or null
    uint32_t* cand;               // [nv][cap] packed (y << 16) | x
    int64_t cap;
    uint32_t* fb;                 // [nv][fb_words] bit per candidate: line left to the warp kernel
    int64_t fb_words;
    uint32_t* hdr;                // HDR_WORDS
    unsigned long long* stats;    // [nv][2]: samples, pair tests
    const uint8_t* prop;          // [nv][tiles_y][tiles_x]: 0 = the tile's candidates are skipped; null = none skipped
    uint8_t* hits;                // [nv][tiles_y][tiles_x]: 1 = a scan line from the tile found an occlusion; or null
    int32_t tiles_x, tiles_y;     // ceil(W / kTile), ceil(H / kTile)
    uint32_t strip0;              // index of the frame's first strip (k_strip grid), strips of its views in order
    int32_t pad2;
};

// Views that share the strips of k_strip: the same strip family and ratio (hence the same D_r, candidates test
// inputs and scan length), at most two (a direction and its opposite, in a camera array).
struct StripGroup {
    int32_t fam;
    int32_t va, vb;   // vb = -1: one view
    int32_t pad;
};

// Per (frame, view), written by k_plan.
struct PlanEntry {
    int32_t h;       // half scan length h = ceil(L / 2); -1: view skipped (non-finite input or L too long)
    int32_t cls;     // size class of its scan lines
    uint32_t count;  // candidates, clamped to the list capacity
    uint32_t pad;
};

// Words of the call's status region (zero at the start of every call): the status word, the counters of the list
// kernels, then those of the fused launch (k_fused).
enum : int {
    CTR_LINE = 1,            // work counter of the line kernel
    CTR_BRK = 2,             // two words: entries / pairs of the merge kernel's lists
    CTR_MERGE = 4,           // batch counter of the merge kernel
    CTR_TICKET = 8,          // fused: next ticket
    CTR_STRIPS = 10,         // fused: strips done
    CTR_OVF_READY = 11,      // fused: prefix sums of the listed lines written (1)
    CTR_OVF_CURSOR = 12,     // fused: [kNumClasses] next listed line of each size class
    CTR_ABORT = 15,          // fused: a wait gave up; every block stops
    CTR_POOL = 16,           // fused: entries of the published-line pool reserved
    CTR_CLAIM = 17,          // fused: entries of the pool taken by the workers
    CTR_EXIT = 18,           // fused: blocks that have ended
    CTR_MINMAX = 19,         // k_minmax: blocks done (the last one writes the plan)
    CTR_WORDS = 20,
    CTR_EPOCH = 32,          // fused: launches so far (kept across calls): the tag of this launch's pool entries
};
constexpr size_t kStatusBytes = 256;   // bytes of the status region in every scratch layout
static_assert(CTR_WORDS <= CTR_EPOCH && (CTR_EPOCH + 1) * sizeof(uint32_t) <= kStatusBytes,
              "status region too small for the counters");

// The fused launch (occ_strip.cu): one kernel for a call whose views all take the strip kernel and that asks for no E,
// A or tile hits.  Blocks take tickets from one counter in this order: the min/max tiles of every frame (the last one
// of a frame writes its plan), the strips, then worker tickets that take the published lines of three or more
// macro-runs (and, once every strip is done, those in the views' lists).
constexpr int kFusedQuadsPerTicket = 2048;   // 4-pixel quads of D per min/max ticket (128 threads x 16)
constexpr int kFusedMaxFrames = 128;         // frame records in the launch parameters
struct FusedPlan {
    uint32_t mm_end;                         // tickets [0, mm_end): min/max tiles, frame after frame
    uint32_t strip_end;                      // [mm_end, strip_end): strips (strip index = ticket - mm_end)
    uint32_t end;                            // [strip_end, end): workers
    uint32_t hold;                           // test hook: never release the frames' plans
    uint64_t wait_ns;                        // bound of every wait
    uint4* pool;                             // published lines: (y << 16 | x, frame << 8 | view or kPoolSkip, tag, -)
    unsigned char* slots;                    // per block, a warp buffer of the largest size class (global memory)
    uint32_t pool_cap;
};
constexpr uint32_t kPoolSkip = 0xFFFFFFFFu;  // a pool entry without a line (its reservation ran past the pool)
template <int NF>
struct FusedFrames {
    uint32_t mm0[NF + 1];                    // first min/max ticket of each frame (mm0[nf] = mm_end)
    FrameArg f[NF];
};

struct Args {
    int32_t nf, nv, nr;           // frames, views, distinct ratios
    float gamma, zeta, beta;
    float e2min;                  // smallest s >= 0 with fl(sqrt(s)) > gamma: E > gamma exactly when E_x^2 + E_y^2 >= e2min
    int32_t Lover;                // > 0: fixed scan length; else Eq. 3 per frame and view
    int32_t N;
    int32_t use_fb;               // the line kernel runs first: the warp kernels take only the lines it flagged
    int32_t line_max_runs;        // the line kernel keeps lines of at most this many macro-runs (1 or 2)
    int32_t hits;                 // some frame asks for per-tile hit flags
    int32_t line_dyn;             // the line kernel takes its chunks from a counter (large calls)
    int32_t max_quads;            // max over frames of H * ceil(W / 4)
    int64_t max_px;               // max over frames of n_views * H * W
    ViewArg view[kMaxViews];
    float ratio[kMaxViews];
    const FrameArg* frames;       // [nf]
    PlanEntry* plan;              // [nf * nv]
    uint32_t* pref_all;           // [nf * nv + 1] prefix of the candidate counts of every (frame, view)
    uint32_t* pref_cls;           // [kNumClasses][nf * nv + 1] the same restricted to each size class
    int32_t* ptab;                // [nv][kTabLen] packed (dx & 0xFFFF) | (dy << 16), or kTabExact
    const int16_t* stab;          // [kNumSTabs][kSTabLen] strip offsets (see kSTabLen)
    uint32_t* status;             // OR of every frame's status bits
    uint32_t* line_ctr;           // work counter of the line kernel, zero at the start of a call
    uint32_t* brk;                // lists of the merge kernel: from the front, the work items of the lines of more than
                                  // one macro-run (replays); from the back, pairs (work item, ks) of the lines of two
                                  // (merges), in the room the call's candidates leave free
    unsigned long long* brk_count;  // entries at the front (low word), pairs at the back (high word; may exceed the
                                    // room); zero at the start of a call
    uint32_t* merge_ctr;          // batch counter of the merge kernel, zero at the start of a call
    uint32_t brk_cap;             // entries brk holds: at least the candidates a call can have
    int32_t any_list;             // some view takes the candidate-list path (k_edges lists its candidates)
    int32_t strip_px;             // pixels of one strip (k_strip); 0 when no view takes the strip path
    uint32_t strip_total;         // strips of the call
    int32_t ngroups;              // strip groups (each frame has the strips of every group, in group order)
    StripGroup group[kMaxViews];
    uint32_t* pref_ovf;           // [kNumClasses][nf * nv + 1] prefix of the strip views' listed lines per size class
    FusedPlan fz;                 // the fused launch (unused otherwise)
};

// At most kFramesPerChunk frame records travel in the parameters of one k_frames launch (under 4 KB).
constexpr int kFramesPerChunk = 24;
struct FrameChunk {
    FrameArg* dst;
    int32_t first, count;
    FrameArg f[kFramesPerChunk];
};

// Launchers (occ_kernels.cu).  Each returns the cudaGetLastError() of its launch.
cudaError_t launch_frames(const FrameChunk& c, cudaStream_t st);
cudaError_t launch_tables(const Args& a, cudaStream_t st);
cudaError_t launch_edges(const Args& a, cudaStream_t st);
// k_edges' min/max and non-finite check alone, then the plan (k_plan's work, by the last block): for calls with no
// candidate-list view and no E, A or tile hit outputs.  c: the call's frame records (at most kFramesPerChunk), which
// the kernel also writes to the frame table in place of k_frames; null when k_frames has written them.
cudaError_t launch_minmax(const Args& a, const FrameChunk* c, cudaStream_t st);
cudaError_t launch_plan(const Args& a, cudaStream_t st);
// The line-per-thread scan over every view; wide = true when some frame's offsets need 64 bits.
cudaError_t launch_scan_lines(const Args& a, int grid, bool wide, cudaStream_t st);
cudaError_t launch_merge_lines(const Args& a, int grid, bool wide, cudaStream_t st);
// cls = kNumClasses launches the class-0 kernel with 4-warp blocks.
cudaError_t launch_scan(const Args& a, int cls, int grid, cudaStream_t st);
cudaError_t launch_mask(const Args& a, cudaStream_t st);
// Strip kernel (occ_strip.cu): the views with a strip family, every strip of the call; its last block writes the prefix
// sums of the lines the strips listed for the warp kernels.
cudaError_t launch_strip(const Args& a, cudaStream_t st);
size_t strip_smem(int strip_px);
cudaError_t configure_strip();
// The fused launch of an all-strip call (a.fz filled in, the status region and frame headers cleared), on `grid`
// blocks: the nf <= kFusedMaxFrames frame records f travel in the launch parameters, with the first min/max ticket of
// each frame (mm0[0 .. nf], mm0[nf] = a.fz.mm_end).
cudaError_t launch_fused(const Args& a, const FrameArg* f, const uint32_t* mm0, int nf, int grid, cudaStream_t st);
// Resident blocks per SM of the fused kernel with strips of strip_px pixels.
int fused_blocks_per_sm(int strip_px);
// Bytes of one block's warp buffer of the largest size class (FusedPlan::slots).
size_t fused_slot_bytes();
// Per-SM resident blocks of the persistent scan kernels (kNumClasses + 1 warp variants); also sets the shared-memory
// opt-ins.
cudaError_t configure_kernels(int* lines_blocks_per_sm, int scan_blocks_per_sm[kNumClasses + 1]);

}  // namespace occ

namespace occ {

// Device buffers one call works in: a context's scratch, or the fixed array of occ_detect_noalloc.
struct Scratch {
    uint32_t* hdr;                 // [max_frames][HDR_WORDS]
    unsigned long long* stats;     // [max_frames][max_views][2]
    uint32_t* status;              // one word
    FrameArg* frames;              // [max_frames]
    PlanEntry* plan;               // [max_frames * max_views]
    uint32_t* pref;                // [(1 + kNumClasses) * (max_frames * max_views + 1)]
    int32_t* ptab;                 // [max_views][kTabLen]
    int16_t* stab;                 // [kNumSTabs][kSTabLen], written by write_strip_tables
    uint32_t* cand;                // candidate list pool
    int64_t cand_entries;
    uint32_t* fb;                  // line-flag pool (words)
    int64_t fb_entries;
    uint32_t* brk;                 // list of lines for the merge kernel (cand_entries entries)
    int64_t brk_entries;
    int32_t max_frames, max_views;
    int32_t sms;                   // multiprocessors of the device
    int32_t lines_bps_max;         // resident blocks per SM of the line kernel
    int32_t scan_bps[kNumClasses + 1];  // of the warp kernels (classes 0, 1, 2, then class 0 with 4-warp blocks)
    occ_tuning tuning;             // mapping and grid choices (occ_set_tuning)
    uint64_t wait_ns = 2000000000ull;  // bound of the fused launch's waits (occ_set_wait_limit)
    int32_t hold = 0;              // test hook: the fused launch never releases the frames' plans
};

// One frame of a call as the caller gives it.
struct FrameIn {
    const float* D;
    int64_t pitch;
    int32_t H, W;
    int32_t* O;
    uint8_t* M;
    float* E;
    float* A;
    int64_t cap;   // candidate list entries per view
    const uint8_t* prop = nullptr;   // tile proposal (see FrameArg), or null
    uint8_t* hits = nullptr;         // tile hit flags (see FrameArg), or null
};

// Checks the parameters and views and fills the view part of `a` (directions, ratios).  OCC_OK or
// OCC_ERR_INVALID_ARG.
int prepare_views(const occ_view* views, int32_t n_views, const occ_params* p, Args& a);

// A second stream and two events a context lends run_frames, so that the merge kernel and the warp kernels run side
// by side (both only add to O and the statistics; the warp kernels' lines are flagged before either starts).
struct SideStream {
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

// Queues the method (Eq. 1-6) for nf validated frames on st (and side, when given).  ev (profiled calls) is null or
// OCC_NUM_STAGES + 2 events: the stage boundaries and the point where the side stream starts; *forked tells whether
// the warp kernels ran on the side stream.  Returns OCC_OK once queued, or OCC_ERR_CUDA.
int run_frames(const Scratch& sc, const FrameIn* fr, int nf, Args& a, cudaStream_t st, cudaEvent_t* ev,
               const SideStream* side = nullptr, bool* forked = nullptr);

// Computes the kNumSTabs strip offset tables on the host and copies them to stab (synchronous).
cudaError_t write_strip_tables(int16_t* stab);

// Occupancy of the persistent scan kernels on the current device (also sets their shared-memory opt-ins) and the
// default tuning.
cudaError_t scratch_grids(Scratch& sc);

}  // namespace occ
