// occ_api.cu -- host side of the C ABI declared in include/occ.h: context and scratch ownership, argument
// validation, the binary32 direction of each view, the launch sequence of one detect call, status and statistics.
#include <cmath>
#include <cstdlib>
#include <climits>
#include <cstring>
#include <new>

#include "occ_internal.cuh"

using namespace occ;

struct occ_ctx {
    int device = 0;
    int num_sms = 0;
    int64_t max_pixels = 0;
    int32_t max_views = 0;
    int64_t cand_cap = 0;
    uint32_t* d_hdr = nullptr;                 // HDR_WORDS words, followed by the per-view statistics
    unsigned long long* d_stats = nullptr;     // [max_views][2] (inside the d_hdr allocation)
    size_t hdr_bytes = 0;                      // header + statistics, cleared by one memset per call
    uint32_t* d_cand = nullptr;                // [max_views][cand_cap]
    int32_t* d_O_scratch = nullptr;            // [max_views][max_pixels], allocated on first use
    float* d_D_stage = nullptr;                // occ_detect_host staging, allocated on first use
    uint8_t* d_M_stage = nullptr;
    int32_t* d_O_stage = nullptr;
    int grid_edges = 0, grid_mask = 0;
    int grid_scan[kNumClasses] = {0, 0, 0};
    int grid_lines = 0;
    uint32_t* d_fb = nullptr;                  // [max_views][fb_words] lines left to the warp scan kernel
    int32_t* d_ptab = nullptr;                 // [max_views][kTabLen] scan-line position tables
    int64_t fb_words = 0;
    int32_t last_nv = 0;
    cudaStream_t last_stream = nullptr;
    bool profiling = false;
    bool profiled_call = false;
    cudaEvent_t ev[OCC_NUM_STAGES + 1] = {};
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

}  // namespace

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
        cudaFree(ctx->d_hdr);
        cudaFree(ctx->d_cand);
        cudaFree(ctx->d_O_scratch);
        cudaFree(ctx->d_D_stage);
        cudaFree(ctx->d_M_stage);
        cudaFree(ctx->d_O_stage);
        cudaFree(ctx->d_fb);
        cudaFree(ctx->d_ptab);
        for (int i = 0; i <= OCC_NUM_STAGES; i++)
            if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
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
    int bps_edges = 0, bps_lines = 0, bps_mask = 0, bps_scan[kNumClasses] = {0, 0, 0};
    ctx->fb_words = (ctx->cand_cap + 31) / 32;
    ctx->hdr_bytes = sizeof(uint32_t) * HDR_WORDS + sizeof(unsigned long long) * 2 * (size_t)max_views;
    bool ok = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess &&
              configure_kernels(&bps_edges, &bps_lines, bps_scan, &bps_mask) == cudaSuccess &&
              cudaMalloc(&ctx->d_hdr, ctx->hdr_bytes) == cudaSuccess &&
              cudaMalloc(&ctx->d_cand, sizeof(uint32_t) * (size_t)ctx->cand_cap * (size_t)max_views) == cudaSuccess &&
              cudaMalloc(&ctx->d_fb, sizeof(uint32_t) * (size_t)ctx->fb_words * (size_t)max_views) == cudaSuccess &&
              cudaMalloc(&ctx->d_ptab, sizeof(int32_t) * (size_t)kTabLen * (size_t)max_views) == cudaSuccess &&
              cudaMemset(ctx->d_hdr, 0, ctx->hdr_bytes) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        occ_destroy(ctx);
        return OCC_ERR_CUDA;
    }
    ctx->d_stats = reinterpret_cast<unsigned long long*>(ctx->d_hdr + HDR_WORDS);
    ctx->grid_edges = ctx->num_sms * (bps_edges > 0 ? bps_edges : 1);
    ctx->grid_mask = ctx->num_sms * (bps_mask > 0 ? bps_mask : 1);
    ctx->grid_lines = ctx->num_sms * (bps_lines > 0 ? bps_lines : 1);
    for (int c = 0; c < kNumClasses; c++) ctx->grid_scan[c] = ctx->num_sms * (bps_scan[c] > 0 ? bps_scan[c] : 1);
    *out = ctx;
    return OCC_OK;
}

int occ_detect(occ_ctx* ctx, const float* D, int32_t H, int32_t W, int64_t pitch, const occ_view* views,
               int32_t n_views, const occ_params* p_in, uint8_t* M, int32_t* O, float* E, float* A, void* stream)
{
    if (!ctx || !D || !views || !M) return OCC_ERR_INVALID_ARG;
    occ_params p;
    if (p_in) p = *p_in; else occ_default_params(&p);
    if (pitch == 0) pitch = W;
    if (H < 1 || W < 1 || H > OCC_MAX_SIDE || W > OCC_MAX_SIDE || (int64_t)H * W > ctx->max_pixels || pitch < W)
        return OCC_ERR_INVALID_ARG;
    if (n_views < 1 || n_views > ctx->max_views) return OCC_ERR_INVALID_ARG;
    if (p.N < 2 || p.N > OCC_MAX_N || (p.N & 1) || !is_finite_f(p.gamma) || !is_finite_f(p.beta) || !is_finite_f(p.zeta) ||
        !(p.zeta > 0.0f) || p.L > OCC_MAX_SCAN)
        return OCC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(D) & 3) || (O && (reinterpret_cast<uintptr_t>(O) & 3)) ||
        (E && (reinterpret_cast<uintptr_t>(E) & 3)) || (A && (reinterpret_cast<uintptr_t>(A) & 3)))
        return OCC_ERR_INVALID_ARG;

    Args a;
    std::memset(&a, 0, sizeof(a));
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

    a.D = D;
    a.pitch = pitch;
    a.H = H;
    a.W = W;
    a.gamma = p.gamma;
    a.zeta = p.zeta;
    a.beta = p.beta;
    a.Lover = p.L > 0 ? p.L : 0;
    a.N = p.N;
    a.cand = ctx->d_cand;
    a.cand_cap = ctx->cand_cap;
    a.hdr = ctx->d_hdr;
    a.stats = ctx->d_stats;
    a.O = O;
    a.M = M;
    a.E = E;
    a.A = A;

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ctx->last_nv = n_views;
    ctx->last_stream = st;

    // Classes of scan kernels that can receive work: with a fixed L only one; with Eq. 3 the device decides, and
    // the kernels of the other classes return at once.
    bool run_cls[kNumClasses] = {true, true, true};
    if (a.Lover > 0) {
        const int nk = 2 * ((a.Lover + 1) / 2) + 1;
        const int c = nk <= kClassCap[0] ? 0 : (nk <= kClassCap[1] ? 1 : 2);
        for (int k = 0; k < kNumClasses; k++) run_cls[k] = (k == c);
    }
    const int64_t quads = (int64_t)H * ((W + 3) / 4);
    const int64_t edge_blocks = (quads + 255) / 256;
    const int grid_edges = (int)(edge_blocks < ctx->grid_edges ? edge_blocks : ctx->grid_edges);

    // Lines go to the line-per-thread kernel first (N/2 <= kLineMaxHalf); the warp kernels then take the lines it
    // flagged.  Larger N: the warp kernels take every line.
    const bool lines = (p.N / 2) <= kLineMaxHalf;
    a.fb = lines ? ctx->d_fb : nullptr;
    a.ptab = ctx->d_ptab;
    a.fb_words = ctx->fb_words;
    const bool wide = (int64_t)(H - 1) * pitch + W > (int64_t)INT32_MAX;

    const bool prof = ctx->profiling;
    auto mark = [&](int i) { return !prof || cudaEventRecord(ctx->ev[i], st) == cudaSuccess; };
    if (cudaMemsetAsync(ctx->d_hdr, 0, ctx->hdr_bytes, st) != cudaSuccess) return OCC_ERR_CUDA;
    if (lines && cudaMemsetAsync(ctx->d_fb, 0, sizeof(uint32_t) * (size_t)ctx->fb_words * n_views, st) != cudaSuccess)
        return OCC_ERR_CUDA;
    if (!mark(0) || (lines && launch_tables(a, st) != cudaSuccess) || launch_edges(a, grid_edges, st) != cudaSuccess ||
        !mark(1))
        return OCC_ERR_CUDA;
    if (lines && launch_scan_lines(a, ctx->grid_lines, wide, st) != cudaSuccess) return OCC_ERR_CUDA;
    if (!mark(2)) return OCC_ERR_CUDA;
    for (int c = 0; c < kNumClasses; c++) {
        if (run_cls[c] && launch_scan(a, c, ctx->grid_scan[c], st) != cudaSuccess) return OCC_ERR_CUDA;
        if (!mark(3 + c)) return OCC_ERR_CUDA;
    }
    if (launch_mask(a, ctx->grid_mask, st) != cudaSuccess || !mark(OCC_NUM_STAGES)) return OCC_ERR_CUDA;
    ctx->profiled_call = prof;
    return OCC_OK;
}

int occ_set_profiling(occ_ctx* ctx, int enable)
{
    if (!ctx) return OCC_ERR_INVALID_ARG;
    if (enable && !ctx->ev[0]) {
        DeviceGuard g(ctx->device);
        if (!g.ok) return OCC_ERR_CUDA;
        for (int i = 0; i <= OCC_NUM_STAGES; i++)
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
    for (int i = 0; i < n; i++) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, ctx->ev[i], ctx->ev[i + 1]) != cudaSuccess) {
            cudaGetLastError();
            return OCC_ERR_CUDA;
        }
        ms[i] = t;
    }
    return OCC_OK;
}

int occ_get_status(occ_ctx* ctx, void* stream)
{
    if (!ctx) return OCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return OCC_ERR_CUDA;
    uint32_t word = 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&word, ctx->d_hdr + HDR_STATUS, sizeof(word), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
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
    uint32_t hdr[HDR_WORDS];
    unsigned long long st[2 * OCC_MAX_VIEWS];
    if (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess ||
        cudaMemcpy(hdr, ctx->d_hdr, sizeof(hdr), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(st, ctx->d_stats, sizeof(unsigned long long) * 2 * ctx->last_nv, cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    for (int v = 0; v < n_views; v++) {
        out[v].candidates = hdr[HDR_COUNT + v];
        out[v].samples = (int64_t)st[2 * v];
        out[v].pair_tests = (int64_t)st[2 * v + 1];
        out[v].L = (int32_t)hdr[HDR_L + v];
        out[v].reserved = 0;
    }
    return OCC_OK;
}

int occ_detect_host(occ_ctx* ctx, const float* D_host, int32_t H, int32_t W, const occ_view* views,
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
    return occ_get_status(ctx, stream);
}

}  // extern "C"
