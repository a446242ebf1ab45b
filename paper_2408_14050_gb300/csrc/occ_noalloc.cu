// occ_noalloc.cu -- occ_detect_noalloc: the detection of occ_detect for callers that must not allocate device
// memory (see include/occ.h).  Its scratch is one file-scope device array, sized once at build time; no call here
// allocates or frees anything.
#include <climits>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>

#include "occ_internal.cuh"

using namespace occ;

namespace {

// The scratch every call shares: the detection header (status word, min/max of D, per-view counts), the per-view
// statistics, the bit per candidate marking lines left to the warp kernels, the scan-line position tables, then the
// candidate lists, [n_views][H*W] entries of the current call.  One array per device that loads the library; it lives until the process exits.
constexpr size_t kHeaderWords = HDR_WORDS;
constexpr size_t kStatsWords = 2 * 2 * OCC_MAX_VIEWS;  // [views][2] unsigned long long, counted in uint32 words
constexpr size_t kFlagWords = OCC_NOALLOC_MAX_PIXEL_VIEWS / 32 + OCC_MAX_VIEWS;
constexpr size_t kTabWords = (size_t)kTabLen * OCC_MAX_VIEWS;
constexpr size_t kScratchWords =
    kHeaderWords + kStatsWords + kFlagWords + kTabWords + (size_t)OCC_NOALLOC_MAX_PIXEL_VIEWS;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    std::once_flag once;
    cudaError_t err = cudaErrorInitializationError;
    uint32_t* scratch = nullptr;   // device address of g_noalloc_scratch on this device
    int grid_edges = 0, grid_mask = 0;
    int grid_scan[kNumClasses] = {0, 0, 0};
    int grid_lines = 0;
};

DeviceSetup g_setup[kMaxDevices];

// Runs once per device, with that device current: the device address of the scratch array, the shared-memory opt-ins
// of the kernels, and their persistent grid sizes.
void setup_device(int dev, DeviceSetup& s)
{
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    int sms = 0, bps_edges = 0, bps_lines = 0, bps_mask = 0, bps_scan[kNumClasses] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = configure_kernels(&bps_edges, &bps_lines, bps_scan, &bps_mask);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s.err = e;
        return;
    }
    s.scratch = static_cast<uint32_t*>(ptr);
    s.grid_edges = sms * (bps_edges > 0 ? bps_edges : 1);
    s.grid_mask = sms * (bps_mask > 0 ? bps_mask : 1);
    s.grid_lines = sms * (bps_lines > 0 ? bps_lines : 1);
    for (int c = 0; c < kNumClasses; c++) s.grid_scan[c] = sms * (bps_scan[c] > 0 ? bps_scan[c] : 1);
    s.err = cudaSuccess;
}

}  // namespace

extern "C" int occ_detect_noalloc(const float* D, int32_t H, int32_t W, int64_t pitch, const occ_view* views,
                                  int32_t n_views, const occ_params* p_in, uint8_t* M, int32_t* O, int32_t* status,
                                  void* stream)
{
    if (!D || !views || !M || !O) return OCC_ERR_INVALID_ARG;
    occ_params p;
    if (p_in) p = *p_in; else occ_default_params(&p);
    if (pitch == 0) pitch = W;
    if (H < 1 || W < 1 || H > OCC_MAX_SIDE || W > OCC_MAX_SIDE || pitch < W || n_views < 1 ||
        n_views > OCC_MAX_VIEWS)
        return OCC_ERR_INVALID_ARG;
    if (p.N < 2 || p.N > OCC_MAX_N || (p.N & 1) || !std::isfinite(p.gamma) || !std::isfinite(p.beta) ||
        !std::isfinite(p.zeta) || !(p.zeta > 0.0f) || p.L > OCC_MAX_SCAN)
        return OCC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(D) & 3) || (reinterpret_cast<uintptr_t>(O) & 3) ||
        (status && (reinterpret_cast<uintptr_t>(status) & 3)))
        return OCC_ERR_INVALID_ARG;
    // The candidate lists must fit the fixed scratch: one entry per pixel and view.
    const int64_t plane = (int64_t)H * W;
    if (plane * n_views > (int64_t)OCC_NOALLOC_MAX_PIXEL_VIEWS) return OCC_ERR_CAPACITY;

    Args a;
    std::memset(&a, 0, sizeof(a));
    a.nv = n_views;
    for (int v = 0; v < n_views; v++) {
        const double al = views[v].alpha_deg;
        const float r = views[v].ratio;
        if (!std::isfinite(al) || !std::isfinite(r) || !(r > 0.0f)) return OCC_ERR_INVALID_ARG;
        occ_direction(al, &a.view[v].c, &a.view[v].s);
        a.view[v].r = r;
        int u = 0;
        while (u < a.nr && a.ratio[u] != r) u++;
        if (u == a.nr) a.ratio[a.nr++] = r;
        a.view[v].ridx = u;
    }

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    DeviceSetup& s = g_setup[dev];
    std::call_once(s.once, setup_device, dev, std::ref(s));
    if (s.err != cudaSuccess) return OCC_ERR_CUDA;

    uint32_t* hdr = s.scratch;
    a.D = D;
    a.pitch = pitch;
    a.H = H;
    a.W = W;
    a.gamma = p.gamma;
    a.zeta = p.zeta;
    a.beta = p.beta;
    a.Lover = p.L > 0 ? p.L : 0;
    a.N = p.N;
    a.hdr = hdr;
    a.stats = reinterpret_cast<unsigned long long*>(hdr + kHeaderWords);
    const bool lines = (p.N / 2) <= kLineMaxHalf;
    a.fb_words = (plane + 31) / 32;
    a.fb = lines ? hdr + kHeaderWords + kStatsWords : nullptr;
    a.ptab = reinterpret_cast<int32_t*>(hdr + kHeaderWords + kStatsWords + kFlagWords);
    a.cand = hdr + kHeaderWords + kStatsWords + kFlagWords + kTabWords;
    a.cand_cap = plane;
    a.O = O;
    a.M = M;
    const bool wide = (int64_t)(H - 1) * pitch + W > (int64_t)INT32_MAX;

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // The header, statistics and line flags keep the previous call's values: clear them (the lists need no clearing).
    const size_t clear_words = kHeaderWords + kStatsWords + (lines ? (size_t)(a.fb_words * n_views) : 0);
    if (cudaMemsetAsync(hdr, 0, sizeof(uint32_t) * clear_words, st) != cudaSuccess) return OCC_ERR_CUDA;
    const int64_t quads = (int64_t)H * ((W + 3) / 4);
    const int64_t edge_blocks = (quads + 255) / 256;
    const int grid_edges = (int)(edge_blocks < s.grid_edges ? edge_blocks : s.grid_edges);
    if (lines && launch_tables(a, st) != cudaSuccess) return OCC_ERR_CUDA;
    if (launch_edges(a, grid_edges, st) != cudaSuccess) return OCC_ERR_CUDA;
    if (lines && launch_scan_lines(a, s.grid_lines, wide, st) != cudaSuccess) return OCC_ERR_CUDA;
    bool run_cls[kNumClasses] = {true, true, true};
    if (a.Lover > 0) {
        const int nk = 2 * ((a.Lover + 1) / 2) + 1;
        const int c = nk <= kClassCap[0] ? 0 : (nk <= kClassCap[1] ? 1 : 2);
        for (int k = 0; k < kNumClasses; k++) run_cls[k] = (k == c);
    }
    for (int c = 0; c < kNumClasses; c++)
        if (run_cls[c] && launch_scan(a, c, s.grid_scan[c], st) != cudaSuccess) return OCC_ERR_CUDA;
    if (launch_mask(a, s.grid_mask, st) != cudaSuccess) return OCC_ERR_CUDA;
    if (status && cudaMemcpyAsync(status, hdr + HDR_STATUS, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
                      cudaSuccess)
        return OCC_ERR_CUDA;
    return OCC_OK;
}
