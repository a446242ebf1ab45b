// occ_api.cu -- host side of the C ABI declared in include/occ.h: argument validation, the binary32 direction of each
// view, the context and its scratch, the launch sequence shared by every entry point (run_frames), status and
// statistics.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "occ_internal.cuh"

using namespace occ;

struct occ_ctx {
    int device = 0;
    int64_t max_pixels = 0;
    int32_t max_views = 0;
    int64_t cand_cap = 0;                      // list entries per view for a frame of max_pixels pixels
    Scratch sc{};
    void* d_block = nullptr;                   // one allocation for headers, statistics, tables and plan
    uint32_t* d_cand = nullptr;
    uint32_t* d_fb = nullptr;
    uint32_t* d_brk = nullptr;
    int32_t* d_O_scratch = nullptr;            // [max_views][max_pixels], allocated on first use
    float* d_D_stage = nullptr;                // occ_detect_host staging, allocated on first use
    uint8_t* d_M_stage = nullptr;
    int32_t* d_O_stage = nullptr;
    int32_t last_nf = 0, last_nv = 0;
    cudaStream_t last_stream = nullptr;
    bool profiling = false;
    bool profiled_call = false;
    bool forked_call = false;                  // its warp kernels ran on the side stream
    cudaEvent_t ev[OCC_NUM_STAGES + 2] = {};   // stage boundaries, then the start of the side stream
    SideStream side{};
};

namespace {

// Makes `dev` current for the lifetime of the guard and restores the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool is_finite_f(float x) { return std::isfinite(x); }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace occ {

// The smallest binary32 s >= 0 whose correctly rounded square root exceeds gamma (+inf if none is finite).  The
// rounded square root is non-decreasing in s, so fl(sqrt(s)) > gamma holds exactly for s >= this value; the
// candidate test of Eq. 2 then needs no square root on the device.  Host sqrtf is the IEEE correctly rounded square
// root, like the device's __fsqrt_rn.
float sqrt_threshold(float gamma)
{
    if (gamma < 0.0f) return 0.0f;
    uint32_t lo = 0, hi = 0x7f800000u;   // bit patterns of 0 and +inf; order of patterns = order of values
    auto f = [](uint32_t b) {
        float x;
        std::memcpy(&x, &b, sizeof(x));
        return x;
    };
    if (!(std::sqrt(f(hi - 1)) > gamma)) return f(hi);
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (std::sqrt(f(mid)) > gamma) hi = mid;
        else lo = mid + 1;
    }
    return f(lo);
}

int prepare_views(const occ_view* views, int32_t n_views, const occ_params* p_in, Args& a)
{
    occ_params p;
    if (p_in) p = *p_in; else occ_default_params(&p);
    if (!views || n_views < 1 || n_views > OCC_MAX_VIEWS) return OCC_ERR_INVALID_ARG;
    if (p.N < 2 || p.N > OCC_MAX_N || (p.N & 1) || !is_finite_f(p.gamma) || !is_finite_f(p.beta) ||
        !is_finite_f(p.zeta) || !(p.zeta > 0.0f) || p.L > OCC_MAX_SCAN)
        return OCC_ERR_INVALID_ARG;
    a.nv = n_views;
    a.nr = 0;
    for (int v = 0; v < n_views; v++) {
        const double al = views[v].alpha_deg;
        const float r = views[v].ratio;
        if (!std::isfinite(al) || !is_finite_f(r) || !(r > 0.0f)) return OCC_ERR_INVALID_ARG;
        occ_direction(al, &a.view[v].c, &a.view[v].s);
        a.view[v].r = r;
        int u = 0;
        while (u < a.nr && a.ratio[u] != r) u++;
        if (u == a.nr) a.ratio[a.nr++] = r;
        a.view[v].ridx = u;
    }
    a.gamma = p.gamma;
    a.e2min = sqrt_threshold(p.gamma);
    a.zeta = p.zeta;
    a.beta = p.beta;
    a.Lover = p.L > 0 ? p.L : 0;
    a.N = p.N;
    return OCC_OK;
}

cudaError_t scratch_grids(Scratch& sc)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sc.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = configure_kernels(&sc.lines_bps_max, sc.scan_bps);
    if (e != cudaSuccess) return e;
    if (sc.lines_bps_max < 1) sc.lines_bps_max = 1;
    for (int c = 0; c <= kNumClasses; c++)
        if (sc.scan_bps[c] < 1) sc.scan_bps[c] = 1;
    if ((e = configure_strip()) != cudaSuccess) return e;
    sc.tuning.line_max_runs = 2;
    sc.tuning.line_blocks_per_sm = sc.lines_bps_max;
    sc.tuning.warp_lines_per_block = 8;
    sc.tuning.strip_px = kStripPxDefault;
    sc.tuning.fused = 0;
    return cudaSuccess;
}

cudaError_t write_strip_tables(int16_t* stab)
{
    // cc = 1, -1, fl(sqrt(1/2)), -fl(sqrt(1/2)): cos and sin of the strip directions as occ_direction rounds them.
    float q = 0.0f, qs = 0.0f;
    occ_direction(45.0, &q, &qs);
    const float cc[kNumSTabs] = {1.0f, -1.0f, q, -q};
    static int16_t host[kNumSTabs][kSTabLen];
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    for (int t = 0; t < kNumSTabs; t++)
        for (int j = 0; j < kSTabLen; j++) {
            const float prod = cc[t] * (float)(j - kTabHalf);   // one binary32 multiply, as fl(cc * g) on the device
            host[t][j] = (int16_t)(int)std::round(prod);        // nearest, halves away from zero (roundf)
        }
    return cudaMemcpy(stab, host, sizeof(host), cudaMemcpyHostToDevice);
}

// Which strip offset table a strip view uses (see kNumSTabs): cc = sin for columns, cos otherwise.
int strip_table(int fam, float c, float s)
{
    const float cc = fam == kFamCols ? s : c;
    return cc == 1.0f ? 0 : (cc == -1.0f ? 1 : (cc > 0.0f ? 2 : 3));
}

// Strip family of a direction (cos, sin as occ_direction rounds them), or -1.
int strip_family(float c, float s)
{
    const float q = (float)std::sqrt(0.5);
    if (s == 0.0f && std::fabs(c) == 1.0f) return kFamRows;
    if (c == 0.0f && std::fabs(s) == 1.0f) return kFamCols;
    if (std::fabs(c) == q && c == s) return kFamDiag;
    if (std::fabs(c) == q && c == -s) return kFamAnti;
    return -1;
}

// The fused launch of a call: its tickets, grid, and the published-line pool and per-block warp buffers it keeps in
// the merge kernel's list pool (which an all-strip call does not use).
struct FusedLayout {
    FusedPlan plan;
    int grid;
    uint32_t mm0[kFusedMaxFrames + 1];
    FrameArg frames[kFusedMaxFrames];
};

bool fused_layout(const Scratch& sc, const FrameIn* fr, int nf, const Args& a, FusedLayout& fl)
{
    if (nf > kFusedMaxFrames || a.strip_px <= 0) return false;
    const int bps = fused_blocks_per_sm(a.strip_px);
    if (bps < 1) return false;
    std::memset(&fl.plan, 0, sizeof(fl.plan));
    int64_t t = 0, strips = 0;
    for (int f = 0; f < nf; f++) {
        fl.mm0[f] = (uint32_t)t;
        const int64_t quads = (int64_t)fr[f].H * ((fr[f].W + 3) / 4);
        t += (quads + kFusedQuadsPerTicket - 1) / kFusedQuadsPerTicket;
        for (int g = 0; g < a.ngroups; g++) strips += fam_strips(a.group[g].fam, fr[f].H, fr[f].W, a.strip_px);
    }
    fl.mm0[nf] = (uint32_t)t;
    const int64_t work = t + strips;
    const int64_t grid = std::min<int64_t>((int64_t)sc.sms * bps, work);
    if (work + grid > (int64_t)INT32_MAX || strips < 1) return false;
    // Scratch: warp buffers (one per block), then the pool of published lines.
    const size_t slot = fused_slot_bytes();
    char* base = reinterpret_cast<char*>(sc.brk);
    const size_t bytes = (size_t)sc.brk_entries * sizeof(uint32_t);
    const size_t off_pool = align256((size_t)grid * slot);
    if (off_pool + sizeof(uint4) * 1024 > bytes) return false;
    fl.grid = (int)grid;
    FusedPlan& z = fl.plan;
    z.mm_end = (uint32_t)t;
    z.strip_end = (uint32_t)(t + strips);
    z.end = (uint32_t)(t + strips + grid);
    z.hold = (uint32_t)sc.hold;
    z.wait_ns = sc.wait_ns;
    z.slots = reinterpret_cast<unsigned char*>(base);
    z.pool = reinterpret_cast<uint4*>(base + off_pool);
    z.pool_cap = (uint32_t)std::min<size_t>((bytes - off_pool) / sizeof(uint4), UINT32_MAX);
    return true;
}

int run_frames(const Scratch& sc, const FrameIn* fr, int nf, Args& a, cudaStream_t st, cudaEvent_t* ev,
               const SideStream* side, bool* forked)
{
    const int nv = a.nv;
    // Views whose scan lines stay on one row, column or diagonal take the strip kernel (N = 8, frames of at most
    // kStripMaxSide a side); the others take the candidate lists.
    bool strip_ok = sc.tuning.strip_px > 0 && a.N == 8;
    for (int f = 0; f < nf; f++)
        if (fr[f].H > kStripMaxSide || fr[f].W > kStripMaxSide) strip_ok = false;
    int n_strip = 0;
    a.ngroups = 0;
    for (int v = 0; v < nv; v++) {
        const int fam = strip_ok ? strip_family(a.view[v].c, a.view[v].s) : -1;
        a.view[v].fam = fam;
        a.view[v].stab = fam >= 0 ? strip_table(fam, a.view[v].c, a.view[v].s) : 0;
        if (fam < 0) continue;
        n_strip++;
        // Pair the view with an earlier one of the same family and ratio that is still alone.
        int g = 0;
        while (g < a.ngroups && !(a.group[g].fam == fam && a.group[g].vb < 0 && a.view[a.group[g].va].r == a.view[v].r))
            g++;
        if (g < a.ngroups) {
            a.group[g].vb = v;
        } else {
            a.group[a.ngroups] = StripGroup{fam, v, -1, 0};
            a.ngroups++;
        }
    }
    const bool list_views = n_strip < nv;
    a.any_list = list_views ? 1 : 0;
    // Pixels per strip: the tuning's, raised to the longest line of the call's strip families (a strip holds at least
    // one whole line), rounded up to a multiple of 64.
    int strip_px = 0;
    if (n_strip) {
        strip_px = sc.tuning.strip_px;
        for (int f = 0; f < nf; f++)
            for (int g = 0; g < a.ngroups; g++) strip_px = std::max(strip_px, fam_len(a.group[g].fam, fr[f].H, fr[f].W));
        strip_px = (strip_px + 63) & ~63;
    }
    a.strip_px = strip_px;
    const bool lines = list_views && (a.N / 2) <= kLineMaxHalf && sc.tuning.line_max_runs > 0;
    a.nf = nf;
    a.use_fb = lines ? 1 : 0;
    a.line_max_runs = sc.tuning.line_max_runs;
    a.frames = sc.frames;
    a.plan = sc.plan;
    a.pref_all = sc.pref;
    a.pref_cls = sc.pref + (nf * nv + 1);
    a.pref_ovf = sc.pref + (1 + kNumClasses) * (nf * nv + 1);
    a.ptab = sc.ptab;
    a.stab = sc.stab;
    a.status = sc.status;
    a.line_ctr = sc.status + CTR_LINE;   // the status region has room for the counters
    a.brk = sc.brk;
    a.brk_count = reinterpret_cast<unsigned long long*>(sc.status + CTR_BRK);
    a.merge_ctr = sc.status + CTR_MERGE;
    a.brk_cap = (uint32_t)(sc.brk_entries < (int64_t)UINT32_MAX ? sc.brk_entries : (int64_t)UINT32_MAX);
    a.max_quads = 0;
    a.max_px = 0;
    a.hits = 0;

    // Every view on strips and no E, A or hit flags asked for: one read of D for Eq. 3 (with the tables in the same
    // launch) is all the candidate pass has to do; with room in the scratch, the whole call is one fused launch.
    bool extras = false;
    for (int f = 0; f < nf; f++) extras = extras || fr[f].E || fr[f].A || fr[f].hits;
    const bool minmax_only = !list_views && !extras;
    FusedLayout fl;
    const bool fused = minmax_only && sc.tuning.fused && fused_layout(sc, fr, nf, a, fl);
    FrameArg* fused_frames = fused ? fl.frames : nullptr;
    // All-strip calls of at most kFramesPerChunk frames: the frame records go to k_minmax's parameters, which also
    // writes the frame table.
    const bool param_frames = minmax_only && !fused && nf <= kFramesPerChunk;

    // Frame records: lists and flags laid out frame after frame in the pools.
    FrameChunk chunk;
    std::memset(&chunk, 0, sizeof(chunk));
    chunk.dst = sc.frames;
    int64_t cand_off = 0, fb_off = 0, px_views = 0, strips = 0;
    bool wide = false;
    for (int f = 0; f < nf; f++) {
        FrameArg& F = chunk.f[f % kFramesPerChunk];
        std::memset(&F, 0, sizeof(F));
        F.D = fr[f].D;
        F.pitch = fr[f].pitch;
        F.H = fr[f].H;
        F.W = fr[f].W;
        F.wide = (int64_t)(F.H - 1) * F.pitch + F.W > (int64_t)INT32_MAX;
        wide = wide || F.wide;
        F.O = fr[f].O;
        F.M = fr[f].M;
        F.E = fr[f].E;
        F.A = fr[f].A;
        F.cap = fr[f].cap;
        F.cand = sc.cand + cand_off;
        cand_off += F.cap * nv;
        F.fb_words = (F.cap + 31) / 32;
        F.fb = sc.fb + fb_off;
        fb_off += F.fb_words * nv;
        F.hdr = sc.hdr + (size_t)f * HDR_WORDS;
        F.stats = sc.stats + (size_t)f * sc.max_views * 2;
        F.prop = fr[f].prop;
        F.hits = fr[f].hits;
        if (F.hits) a.hits = 1;
        px_views += (int64_t)F.H * F.W * nv;
        F.tiles_x = (F.W + kTile - 1) / kTile;
        F.tiles_y = (F.H + kTile - 1) / kTile;
        F.strip0 = (uint32_t)strips;
        for (int g = 0; g < a.ngroups; g++) strips += fam_strips(a.group[g].fam, F.H, F.W, a.strip_px);
        const int quads = F.H * ((F.W + 3) / 4);
        if (quads > a.max_quads) a.max_quads = quads;
        const int64_t px = (int64_t)nv * F.H * F.W;
        if (px > a.max_px) a.max_px = px;
        if (fused_frames) {
            fused_frames[f] = F;
        } else if (param_frames) {
            if (f == nf - 1) {
                chunk.first = 0;
                chunk.count = nf;
            }
        } else if (f % kFramesPerChunk == kFramesPerChunk - 1 || f == nf - 1) {
            chunk.first = f - f % kFramesPerChunk;
            chunk.count = f % kFramesPerChunk + 1;
            if (launch_frames(chunk, st) != cudaSuccess) return OCC_ERR_CUDA;
        }
    }
    if (cand_off > sc.cand_entries || (lines && fb_off > sc.fb_entries)) return OCC_ERR_INVALID_ARG;
    // The scan kernels number the candidates of a call (every frame and view) with 32-bit work items.
    if (cand_off > (int64_t)UINT32_MAX || strips > (int64_t)INT32_MAX) return OCC_ERR_CAPACITY;
    a.strip_total = (uint32_t)strips;
    // Above about four 1920x1080 frames of 8 views, static chunks let warps drift over more data than L2 holds.
    a.line_dyn = px_views > (int64_t)64 * 1024 * 1024 ? 1 : 0;

    auto mark = [&](int i) { return !ev || cudaEventRecord(ev[i], st) == cudaSuccess; };
    if (fused) {
        // One launch: its stage times all fall in the line-per-thread stage's slot.
        if (forked) *forked = false;
        a.fz = fl.plan;
        if (cudaMemsetAsync(sc.hdr, 0, sizeof(uint32_t) * HDR_WORDS * nf, st) != cudaSuccess ||
            cudaMemsetAsync(sc.stats, 0, sizeof(unsigned long long) * 2 * sc.max_views * nf, st) != cudaSuccess ||
            cudaMemsetAsync(sc.status, 0, CTR_WORDS * sizeof(uint32_t), st) != cudaSuccess || !mark(0) || !mark(1) ||
            launch_fused(a, fl.frames, fl.mm0, nf, fl.grid, st) != cudaSuccess)
            return OCC_ERR_CUDA;
        for (int i = 2; i <= OCC_NUM_STAGES; i++)
            if (!mark(i)) return OCC_ERR_CUDA;
        return OCC_OK;
    }
    if (cudaMemsetAsync(sc.hdr, 0, sizeof(uint32_t) * HDR_WORDS * nf, st) != cudaSuccess ||
        cudaMemsetAsync(sc.stats, 0, sizeof(unsigned long long) * 2 * sc.max_views * nf, st) != cudaSuccess ||
        cudaMemsetAsync(sc.status, 0, CTR_WORDS * sizeof(uint32_t), st) != cudaSuccess ||
        (lines && cudaMemsetAsync(sc.fb, 0, sizeof(uint32_t) * fb_off, st) != cudaSuccess))
        return OCC_ERR_CUDA;
    // Size classes of the warp kernels that can receive work: with a fixed L only one.
    bool run_cls[kNumClasses] = {true, true, true};
    if (a.Lover > 0) {
        const int nk = 2 * ((a.Lover + 1) / 2) + 1;
        const int c = nk <= kClassCap[0] ? 0 : (nk <= kClassCap[1] ? 1 : 2);
        for (int k = 0; k < kNumClasses; k++) run_cls[k] = (k == c);
    }
    if (!mark(0)) return OCC_ERR_CUDA;
    if (minmax_only) {
        // min/max and the plan in one launch (and the frame table, for a call of one chunk).
        if (launch_minmax(a, param_frames ? &chunk : nullptr, st) != cudaSuccess) return OCC_ERR_CUDA;
    } else if ((lines && launch_tables(a, st) != cudaSuccess) || launch_edges(a, st) != cudaSuccess ||
               launch_plan(a, st) != cudaSuccess) {
        return OCC_ERR_CUDA;
    }
    if (!mark(1)) return OCC_ERR_CUDA;
    // The strip views: O and M written once per strip; the lines of three or more macro-runs are listed for the warp
    // kernels below, which add their counts to O and M (the last strip block writes their prefix sums).
    if (n_strip && launch_strip(a, st) != cudaSuccess) return OCC_ERR_CUDA;
    const int lgrid = sc.sms * sc.tuning.line_blocks_per_sm;
    if (lines && launch_scan_lines(a, lgrid, wide, st) != cudaSuccess) return OCC_ERR_CUDA;
    // k_scan_lines has flagged every line the warp kernels take, and the merge kernel and the warp kernels only add
    // to O and the statistics: in calls below the size where the line kernel takes its chunks from a counter, the
    // merge kernel's few batches per warp leave it latency-bound, and the warp kernels run beside it on the side
    // stream.  Larger calls keep every multiprocessor busy on their own.
    const bool fork = side && side->st && lines && !a.line_dyn;
    if (forked) *forked = fork;
    cudaStream_t wst = st;
    if (fork) {
        if (cudaEventRecord(side->fork, st) != cudaSuccess || cudaStreamWaitEvent(side->st, side->fork, 0) != cudaSuccess ||
            (ev && cudaEventRecord(ev[OCC_NUM_STAGES + 1], side->st) != cudaSuccess))
            return OCC_ERR_CUDA;
        wst = side->st;
    }
    if (lines && launch_merge_lines(a, lgrid, wide, st) != cudaSuccess) return OCC_ERR_CUDA;
    if (!mark(2)) return OCC_ERR_CUDA;
    for (int c = 0; c < kNumClasses; c++) {
        const int id = (c == 0 && sc.tuning.warp_lines_per_block == 4) ? kNumClasses : c;
        if (run_cls[c] && launch_scan(a, id, sc.sms * sc.scan_bps[id], wst) != cudaSuccess) return OCC_ERR_CUDA;
        if (ev && cudaEventRecord(ev[3 + c], wst) != cudaSuccess) return OCC_ERR_CUDA;
    }
    if (fork && (cudaEventRecord(side->join, side->st) != cudaSuccess || cudaStreamWaitEvent(st, side->join, 0) != cudaSuccess))
        return OCC_ERR_CUDA;
    if ((list_views && launch_mask(a, st) != cudaSuccess) || !mark(OCC_NUM_STAGES)) return OCC_ERR_CUDA;
    return OCC_OK;
}

}  // namespace occ

extern "C" {

void occ_default_params(occ_params* p)
{
    if (!p) return;
    p->gamma = 1.0f;
    p->zeta = 2.0f;
    p->beta = 0.5f;
    p->L = 0;
    p->N = 8;
}

// cos / sin of alpha rounded once to binary32.  alpha is reduced to a quadrant and folded to [0, 45] degrees, where
// the double-precision library functions are evaluated; the quadrant then permutes and negates the pair.  Folding
// makes multiples of 90 degrees exact (0, +-1) and 45 degrees give fl(sqrt(1/2)) for both components.
void occ_direction(double alpha_deg, float* c_out, float* s_out)
{
    double a = std::fmod(alpha_deg, 360.0);
    if (a < 0.0) a += 360.0;
    if (a >= 360.0) a -= 360.0;
    int quad = (int)(a / 90.0);
    if (quad > 3) quad = 3;
    const double t = a - 90.0 * quad;  // exact, in [0, 90)
    double ct, st;
    if (t == 45.0) {
        ct = st = std::sqrt(0.5);
    } else if (t < 45.0) {
        ct = std::cos(t * (M_PI / 180.0));
        st = std::sin(t * (M_PI / 180.0));
    } else {
        const double u = 90.0 - t;  // exact
        ct = std::sin(u * (M_PI / 180.0));
        st = std::cos(u * (M_PI / 180.0));
    }
    double c = ct, s = st;
    if (quad == 1) { c = -st; s = ct; }
    else if (quad == 2) { c = -ct; s = -st; }
    else if (quad == 3) { c = st; s = -ct; }
    if (c_out) *c_out = (float)c;
    if (s_out) *s_out = (float)s;
}

const char* occ_status_string(int status)
{
    switch (status) {
    case OCC_OK: return "ok";
    case OCC_ERR_INVALID_ARG: return "invalid argument";
    case OCC_ERR_NONFINITE_INPUT: return "non-finite disparity input";
    case OCC_ERR_CAPACITY: return "capacity exceeded (candidate list or scan length)";
    case OCC_ERR_TIMEOUT: return "device wait timed out";
    case OCC_ERR_CUDA: return "CUDA runtime error";
    default: return "unknown status";
    }
}

void occ_destroy(occ_ctx* ctx)
{
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        cudaFree(ctx->d_block);
        cudaFree(ctx->d_cand);
        cudaFree(ctx->d_fb);
        cudaFree(ctx->d_brk);
        cudaFree(ctx->d_O_scratch);
        cudaFree(ctx->d_D_stage);
        cudaFree(ctx->d_M_stage);
        cudaFree(ctx->d_O_stage);
        for (int i = 0; i <= OCC_NUM_STAGES + 1; i++)
            if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
        if (ctx->side.fork) cudaEventDestroy(ctx->side.fork);
        if (ctx->side.join) cudaEventDestroy(ctx->side.join);
        if (ctx->side.st) cudaStreamDestroy(ctx->side.st);
    }
    delete ctx;
}

int occ_create(occ_ctx** out, int device, int64_t max_pixels, int32_t max_views, int64_t max_candidates)
{
    if (!out) return OCC_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_pixels < 1 || max_pixels > (int64_t)OCC_MAX_SIDE * OCC_MAX_SIDE || max_views < 1 ||
        max_views > OCC_MAX_VIEWS)
        return OCC_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return OCC_ERR_CUDA;

    occ_ctx* ctx = new (std::nothrow) occ_ctx();
    if (!ctx) return OCC_ERR_CUDA;
    ctx->device = device;
    ctx->max_pixels = max_pixels;
    ctx->max_views = max_views;
    ctx->cand_cap = (max_candidates > 0 && max_candidates < max_pixels) ? max_candidates : max_pixels;

    DeviceGuard g(device);
    if (!g.ok) { delete ctx; return OCC_ERR_CUDA; }
    Scratch& sc = ctx->sc;
    sc.max_frames = kMaxFrames;
    sc.max_views = max_views;
    const size_t nfv = (size_t)kMaxFrames * max_views;
    const size_t sz_hdr = align256(sizeof(uint32_t) * HDR_WORDS * kMaxFrames);
    const size_t sz_stats = align256(sizeof(unsigned long long) * 2 * nfv);
    const size_t sz_status = kStatusBytes;
    const size_t sz_frames = align256(sizeof(FrameArg) * kMaxFrames);
    const size_t sz_plan = align256(sizeof(PlanEntry) * nfv);
    const size_t sz_pref = align256(sizeof(uint32_t) * (1 + 2 * kNumClasses) * (nfv + 1));
    const size_t sz_tab = align256(sizeof(int32_t) * kTabLen * max_views) + align256(sizeof(int16_t) * kSTabLen * kNumSTabs);
    const size_t total = sz_hdr + sz_stats + sz_status + sz_frames + sz_plan + sz_pref + sz_tab;
    sc.cand_entries = ctx->cand_cap * max_views;
    sc.fb_entries = (ctx->cand_cap / 32 + kMaxFrames + 1) * (int64_t)max_views;
    // One entry per candidate: the list of broken lines cannot fill up.
    sc.brk_entries = sc.cand_entries;
    bool ok = scratch_grids(sc) == cudaSuccess && cudaMalloc(&ctx->d_block, total) == cudaSuccess &&
              cudaMalloc(&ctx->d_cand, sizeof(uint32_t) * (size_t)sc.cand_entries) == cudaSuccess &&
              cudaMalloc(&ctx->d_fb, sizeof(uint32_t) * (size_t)sc.fb_entries) == cudaSuccess &&
              cudaMalloc(&ctx->d_brk, sizeof(uint32_t) * (size_t)sc.brk_entries) == cudaSuccess &&
              cudaMemset(ctx->d_block, 0, total) == cudaSuccess &&
              cudaStreamCreateWithFlags(&ctx->side.st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&ctx->side.fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&ctx->side.join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        occ_destroy(ctx);
        return OCC_ERR_CUDA;
    }
    char* p = static_cast<char*>(ctx->d_block);
    sc.hdr = reinterpret_cast<uint32_t*>(p); p += sz_hdr;
    sc.stats = reinterpret_cast<unsigned long long*>(p); p += sz_stats;
    sc.status = reinterpret_cast<uint32_t*>(p); p += sz_status;
    sc.frames = reinterpret_cast<FrameArg*>(p); p += sz_frames;
    sc.plan = reinterpret_cast<PlanEntry*>(p); p += sz_plan;
    sc.pref = reinterpret_cast<uint32_t*>(p); p += sz_pref;
    sc.ptab = reinterpret_cast<int32_t*>(p);
    sc.stab = reinterpret_cast<int16_t*>(p + align256(sizeof(int32_t) * kTabLen * max_views));
    sc.cand = ctx->d_cand;
    sc.fb = ctx->d_fb;
    sc.brk = ctx->d_brk;
    if (write_strip_tables(sc.stab) != cudaSuccess) {
        cudaGetLastError();
        occ_destroy(ctx);
        return OCC_ERR_CUDA;
    }
    *out = ctx;
    return OCC_OK;
}

namespace {

// Queues nf validated frames on the context and records the call for status, statistics and timings.
int ctx_run(occ_ctx* ctx, const FrameIn* fr, int nf, Args& a, void* stream)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ctx->last_nf = nf;
    ctx->last_nv = a.nv;
    ctx->last_stream = st;
    bool forked = false;
    const int rc = run_frames(ctx->sc, fr, nf, a, st, ctx->profiling ? ctx->ev : nullptr, &ctx->side, &forked);
    ctx->profiled_call = ctx->profiling && rc == OCC_OK;
    ctx->forked_call = forked;
    return rc;
}

bool frame_ok(const occ_ctx* ctx, const float* D, int32_t H, int32_t W, int64_t pitch)
{
    return D && H >= 1 && W >= 1 && H <= OCC_MAX_SIDE && W <= OCC_MAX_SIDE && pitch >= W &&
           (int64_t)H * W <= ctx->max_pixels && !(reinterpret_cast<uintptr_t>(D) & 3);
}

}  // namespace

int occ_detect(occ_ctx* ctx, const float* D, int32_t H, int32_t W, int64_t pitch, const occ_view* views,
               int32_t n_views, const occ_params* p, uint8_t* M, int32_t* O, float* E, float* A, void* stream)
{
    if (!ctx || !M) return OCC_ERR_INVALID_ARG;
    if (pitch == 0) pitch = W;
    if (!frame_ok(ctx, D, H, W, pitch) || n_views > ctx->max_views) return OCC_ERR_INVALID_ARG;
    if ((O && (reinterpret_cast<uintptr_t>(O) & 3)) || (E && (reinterpret_cast<uintptr_t>(E) & 3)) ||
        (A && (reinterpret_cast<uintptr_t>(A) & 3)))
        return OCC_ERR_INVALID_ARG;
    Args a;
    std::memset(&a, 0, sizeof(a));
    const int rc = prepare_views(views, n_views, p, a);
    if (rc != OCC_OK) return rc;

    DeviceGuard g(ctx->device);
    if (!g.ok) return OCC_ERR_CUDA;
    if (!O) {
        if (!ctx->d_O_scratch &&
            cudaMalloc(&ctx->d_O_scratch, sizeof(int32_t) * (size_t)ctx->max_pixels * ctx->max_views) != cudaSuccess) {
            cudaGetLastError();
            ctx->d_O_scratch = nullptr;
            return OCC_ERR_CUDA;
        }
        O = ctx->d_O_scratch;
    }
    FrameIn fr{D, pitch, H, W, O, M, E, A, ctx->cand_cap};
    return ctx_run(ctx, &fr, 1, a, stream);
}

int occ_detect_batched_tiles(occ_ctx* ctx, int32_t n_frames, const float* const* D, const int32_t* H,
                             const int32_t* W, const occ_view* views, int32_t n_views, const occ_params* p,
                             const uint8_t* const* proposal, uint8_t* const* M, int32_t* const* O,
                             uint8_t* const* tile_hits, void* stream)
{
    if (!ctx || !D || !H || !W || !M || !O || n_frames < 1 || n_frames > OCC_MAX_FRAMES ||
        n_views > ctx->max_views)
        return OCC_ERR_INVALID_ARG;
    Args a;
    std::memset(&a, 0, sizeof(a));
    int rc = prepare_views(views, n_views, p, a);
    if (rc != OCC_OK) return rc;
    FrameIn* fr = static_cast<FrameIn*>(std::malloc(sizeof(FrameIn) * (size_t)n_frames));
    if (!fr) return OCC_ERR_CUDA;
    int64_t pixels = 0;
    for (int f = 0; f < n_frames && rc == OCC_OK; f++) {
        if (!frame_ok(ctx, D[f], H[f], W[f], W[f]) || !M[f] || !O[f] || (reinterpret_cast<uintptr_t>(O[f]) & 3)) {
            rc = OCC_ERR_INVALID_ARG;
            break;
        }
        pixels += (int64_t)H[f] * W[f];
        // List capacity in proportion to the frame: the context's per-pixel share, at least one entry.
        int64_t cap = (int64_t)((double)H[f] * W[f] * (double)ctx->cand_cap / (double)ctx->max_pixels);
        if (cap < 1) cap = 1;
        fr[f] = FrameIn{D[f], W[f], H[f], W[f], O[f], M[f], nullptr, nullptr, cap};
        fr[f].prop = proposal ? proposal[f] : nullptr;
        fr[f].hits = tile_hits ? tile_hits[f] : nullptr;
    }
    if (rc == OCC_OK && pixels > ctx->max_pixels) rc = OCC_ERR_INVALID_ARG;
    if (rc == OCC_OK) {
        DeviceGuard g(ctx->device);
        rc = g.ok ? ctx_run(ctx, fr, n_frames, a, stream) : OCC_ERR_CUDA;
    }
    std::free(fr);
    return rc;
}

int occ_detect_batched(occ_ctx* ctx, int32_t n_frames, const float* const* D, const int32_t* H, const int32_t* W,
                       const occ_view* views, int32_t n_views, const occ_params* p, uint8_t* const* M,
                       int32_t* const* O, void* stream)
{
    return occ_detect_batched_tiles(ctx, n_frames, D, H, W, views, n_views, p, nullptr, M, O, nullptr, stream);
}

int occ_set_tuning(occ_ctx* ctx, const occ_tuning* t)
{
    if (!ctx) return OCC_ERR_INVALID_ARG;
    occ_tuning d{2, ctx->sc.lines_bps_max, 8, kStripPxDefault, 0};
    if (!t) t = &d;
    if (t->line_max_runs < 0 || t->line_max_runs > 2 || t->line_blocks_per_sm < 1 ||
        t->line_blocks_per_sm > ctx->sc.lines_bps_max || (t->warp_lines_per_block != 4 && t->warp_lines_per_block != 8) ||
        (t->strip_px != 0 && (t->strip_px < 1024 || t->strip_px > OCC_STRIP_PX_MAX || (t->strip_px & 63))) ||
        (t->fused != 0 && t->fused != 1))
        return OCC_ERR_INVALID_ARG;
    ctx->sc.tuning = *t;
    return OCC_OK;
}

int occ_set_wait_limit(occ_ctx* ctx, int64_t wait_us, int32_t hold)
{
    if (!ctx || wait_us < 0 || wait_us > 60000000) return OCC_ERR_INVALID_ARG;
    ctx->sc.wait_ns = wait_us ? (uint64_t)wait_us * 1000u : 2000000000ull;
    ctx->sc.hold = hold ? 1 : 0;
    return OCC_OK;
}

int occ_get_tuning(occ_ctx* ctx, occ_tuning* t, int32_t* max_line_blocks_per_sm)
{
    if (!ctx || !t) return OCC_ERR_INVALID_ARG;
    *t = ctx->sc.tuning;
    if (max_line_blocks_per_sm) *max_line_blocks_per_sm = ctx->sc.lines_bps_max;
    return OCC_OK;
}

int occ_set_profiling(occ_ctx* ctx, int enable)
{
    if (!ctx) return OCC_ERR_INVALID_ARG;
    if (enable && !ctx->ev[0]) {
        DeviceGuard g(ctx->device);
        if (!g.ok) return OCC_ERR_CUDA;
        for (int i = 0; i <= OCC_NUM_STAGES + 1; i++)
            if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess) {
                cudaGetLastError();
                return OCC_ERR_CUDA;
            }
    }
    ctx->profiling = enable != 0;
    return OCC_OK;
}

int occ_get_timings(occ_ctx* ctx, float* ms, int32_t n)
{
    if (!ctx || !ms || n < 0 || n > OCC_NUM_STAGES || !ctx->profiled_call) return OCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return OCC_ERR_CUDA;
    if (cudaEventSynchronize(ctx->ev[OCC_NUM_STAGES]) != cudaSuccess) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    // Times of every event from the first; stage i lasts from its start to its end event.  When the warp kernels ran
    // on the side stream, they start where the line kernel ended (the fork) and the mask starts at the later of
    // the two streams' ends.
    float t[OCC_NUM_STAGES + 2] = {};
    const int ne = ctx->forked_call ? OCC_NUM_STAGES + 2 : OCC_NUM_STAGES + 1;
    for (int i = 1; i < ne; i++)
        if (cudaEventElapsedTime(&t[i], ctx->ev[0], ctx->ev[i]) != cudaSuccess) {
            cudaGetLastError();
            return OCC_ERR_CUDA;
        }
    float start[OCC_NUM_STAGES];
    for (int i = 0; i < OCC_NUM_STAGES; i++) start[i] = t[i];
    if (ctx->forked_call) {
        start[2] = t[OCC_NUM_STAGES + 1];
        start[OCC_NUM_STAGES - 1] = fmaxf(t[2], t[OCC_NUM_STAGES - 1]);
    }
    for (int i = 0; i < n; i++) ms[i] = t[i + 1] - start[i];
    return OCC_OK;
}

int occ_get_status(occ_ctx* ctx, void* stream)
{
    if (!ctx) return OCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return OCC_ERR_CUDA;
    uint32_t word = 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&word, ctx->sc.status, sizeof(word), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    if (word & ST_NONFINITE) return OCC_ERR_NONFINITE_INPUT;
    if (word & (ST_CAND_OVERFLOW | ST_SCAN_TOO_LONG)) return OCC_ERR_CAPACITY;
    if (word & ST_TIMEOUT) return OCC_ERR_TIMEOUT;
    if (word & ST_INTERNAL) return OCC_ERR_CUDA;
    return OCC_OK;
}

int occ_get_stats(occ_ctx* ctx, occ_view_stats* out, int32_t n_views)
{
    if (!ctx || !out || n_views < 0 || n_views > ctx->last_nv) return OCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return OCC_ERR_CUDA;
    const int nf = ctx->last_nf;
    uint32_t* hdr = static_cast<uint32_t*>(std::malloc(sizeof(uint32_t) * HDR_WORDS * (size_t)nf));
    unsigned long long* st =
        static_cast<unsigned long long*>(std::malloc(sizeof(unsigned long long) * 2 * ctx->max_views * (size_t)nf));
    int rc = (hdr && st) ? OCC_OK : OCC_ERR_CUDA;
    if (rc == OCC_OK &&
        (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess ||
         cudaMemcpy(hdr, ctx->sc.hdr, sizeof(uint32_t) * HDR_WORDS * nf, cudaMemcpyDeviceToHost) != cudaSuccess ||
         cudaMemcpy(st, ctx->sc.stats, sizeof(unsigned long long) * 2 * ctx->max_views * nf,
                    cudaMemcpyDeviceToHost) != cudaSuccess)) {
        cudaGetLastError();
        rc = OCC_ERR_CUDA;
    }
    if (rc == OCC_OK) {
        for (int v = 0; v < n_views; v++) {
            occ_view_stats s{0, 0, 0, 0, 0};
            for (int f = 0; f < nf; f++) {
                const uint32_t* h = hdr + (size_t)f * HDR_WORDS;
                const unsigned long long* x = st + (size_t)f * ctx->max_views * 2;
                s.candidates += h[HDR_COUNT + v];
                s.samples += (int64_t)x[2 * v];
                s.pair_tests += (int64_t)x[2 * v + 1];
                if ((int32_t)h[HDR_L + v] > s.L) s.L = (int32_t)h[HDR_L + v];
            }
            out[v] = s;
        }
    }
    std::free(hdr);
    std::free(st);
    return rc;
}

int occ_detect_host_async(occ_ctx* ctx, const float* D_host, int32_t H, int32_t W, const occ_view* views,
                          int32_t n_views, const occ_params* p, uint8_t* M_host, int32_t* O_host, void* stream)
{
    if (!ctx || !D_host || !M_host || !views) return OCC_ERR_INVALID_ARG;
    if (H < 1 || W < 1 || (int64_t)H * W > ctx->max_pixels || n_views < 1 || n_views > ctx->max_views)
        return OCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return OCC_ERR_CUDA;
    const size_t npx = (size_t)ctx->max_pixels, nv = (size_t)ctx->max_views;
    if ((!ctx->d_D_stage && cudaMalloc(&ctx->d_D_stage, sizeof(float) * npx) != cudaSuccess) ||
        (!ctx->d_M_stage && cudaMalloc(&ctx->d_M_stage, npx * nv) != cudaSuccess) ||
        (!ctx->d_O_stage && cudaMalloc(&ctx->d_O_stage, sizeof(int32_t) * npx * nv) != cudaSuccess)) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t plane = (size_t)H * W;
    if (cudaMemcpyAsync(ctx->d_D_stage, D_host, sizeof(float) * plane, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return OCC_ERR_CUDA;
    int rc = occ_detect(ctx, ctx->d_D_stage, H, W, W, views, n_views, p, ctx->d_M_stage, ctx->d_O_stage, nullptr,
                        nullptr, stream);
    if (rc != OCC_OK) return rc;
    if (cudaMemcpyAsync(M_host, ctx->d_M_stage, plane * n_views, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return OCC_ERR_CUDA;
    if (O_host && cudaMemcpyAsync(O_host, ctx->d_O_stage, sizeof(int32_t) * plane * n_views,
                                  cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return OCC_ERR_CUDA;
    return OCC_OK;
}

int occ_detect_host(occ_ctx* ctx, const float* D_host, int32_t H, int32_t W, const occ_view* views,
                    int32_t n_views, const occ_params* p, uint8_t* M_host, int32_t* O_host, void* stream)
{
    const int rc = occ_detect_host_async(ctx, D_host, H, W, views, n_views, p, M_host, O_host, stream);
    return rc != OCC_OK ? rc : occ_get_status(ctx, stream);
}

}  // extern "C"
