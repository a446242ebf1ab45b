// occ_noalloc.cu -- occ_detect_noalloc: the detection of occ_detect for callers that must not allocate device
// memory (see include/occ.h).  Its scratch is one file-scope device array, sized once at build time; no call here
// allocates or frees anything.
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "occ_internal.cuh"

using namespace occ;

namespace {

// The scratch every call shares, laid out as the one-frame scratch of a context: the frame header, the per-view
// statistics, the batch status word, the frame record, the plan and its prefix sums, the scan-line position tables,
// the bit per candidate marking lines left to the warp kernels, the list of lines for the merge kernel, then the
// candidate lists ([n_views][H*W] entries of the current call).  One array per device that loads the library; it
// lives until the process exits.
constexpr size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffHdr = 0;
constexpr size_t kOffStats = kOffHdr + align_up(sizeof(uint32_t) * HDR_WORDS);
constexpr size_t kOffStatus = kOffStats + align_up(sizeof(unsigned long long) * 2 * OCC_MAX_VIEWS);
constexpr size_t kOffFrames = kOffStatus + kStatusBytes;
constexpr size_t kOffPlan = kOffFrames + align_up(sizeof(FrameArg));
constexpr size_t kOffPref = kOffPlan + align_up(sizeof(PlanEntry) * OCC_MAX_VIEWS);
constexpr size_t kOffTab = kOffPref + align_up(sizeof(uint32_t) * (1 + 2 * kNumClasses) * (OCC_MAX_VIEWS + 1));
constexpr size_t kFlagWords = OCC_NOALLOC_MAX_PIXEL_VIEWS / 32 + OCC_MAX_VIEWS;
constexpr size_t kOffSTab = kOffTab + align_up(sizeof(int32_t) * kTabLen * OCC_MAX_VIEWS);
constexpr size_t kOffFlags = kOffSTab + align_up(sizeof(int16_t) * kSTabLen * kNumSTabs);
constexpr size_t kBrkEntries = OCC_NOALLOC_MAX_PIXEL_VIEWS;
constexpr size_t kOffBrk = kOffFlags + align_up(sizeof(uint32_t) * kFlagWords);
constexpr size_t kOffCand = kOffBrk + align_up(sizeof(uint32_t) * kBrkEntries);
constexpr size_t kScratchBytes = kOffCand + sizeof(uint32_t) * (size_t)OCC_NOALLOC_MAX_PIXEL_VIEWS;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    std::mutex mu;
    std::atomic<bool> done{false};   // set only after a set-up that succeeded; a failed one is tried again next call
    Scratch sc{};
};

DeviceSetup g_setup[kMaxDevices];

// Runs under the device's lock, with that device current, until it succeeds once: the device address of the
// scratch array, the shared-memory opt-ins of the kernels and their persistent grid sizes.
cudaError_t setup_device(DeviceSetup& s)
{
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e == cudaSuccess) e = scratch_grids(s.sc);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    unsigned char* p = static_cast<unsigned char*>(ptr);
    Scratch& sc = s.sc;
    sc.hdr = reinterpret_cast<uint32_t*>(p + kOffHdr);
    sc.stats = reinterpret_cast<unsigned long long*>(p + kOffStats);
    sc.status = reinterpret_cast<uint32_t*>(p + kOffStatus);
    sc.frames = reinterpret_cast<FrameArg*>(p + kOffFrames);
    sc.plan = reinterpret_cast<PlanEntry*>(p + kOffPlan);
    sc.pref = reinterpret_cast<uint32_t*>(p + kOffPref);
    sc.ptab = reinterpret_cast<int32_t*>(p + kOffTab);
    sc.stab = reinterpret_cast<int16_t*>(p + kOffSTab);
    sc.fb = reinterpret_cast<uint32_t*>(p + kOffFlags);
    sc.fb_entries = (int64_t)kFlagWords;
    sc.brk = reinterpret_cast<uint32_t*>(p + kOffBrk);
    sc.brk_entries = (int64_t)kBrkEntries;
    sc.cand = reinterpret_cast<uint32_t*>(p + kOffCand);
    sc.cand_entries = OCC_NOALLOC_MAX_PIXEL_VIEWS;
    sc.max_frames = 1;
    sc.max_views = OCC_MAX_VIEWS;
    if ((e = write_strip_tables(sc.stab)) != cudaSuccess) cudaGetLastError();
    return e;
}

}  // namespace

extern "C" int occ_detect_noalloc(const float* D, int32_t H, int32_t W, int64_t pitch, const occ_view* views,
                                  int32_t n_views, const occ_params* p, uint8_t* M, int32_t* O, int32_t* status,
                                  void* stream)
{
    if (!D || !views || !M || !O) return OCC_ERR_INVALID_ARG;
    if (pitch == 0) pitch = W;
    if (H < 1 || W < 1 || H > OCC_MAX_SIDE || W > OCC_MAX_SIDE || pitch < W || n_views < 1 ||
        n_views > OCC_MAX_VIEWS)
        return OCC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(D) & 3) || (reinterpret_cast<uintptr_t>(O) & 3) ||
        (status && (reinterpret_cast<uintptr_t>(status) & 3)))
        return OCC_ERR_INVALID_ARG;
    Args a;
    std::memset(&a, 0, sizeof(a));
    const int rc = prepare_views(views, n_views, p, a);
    if (rc != OCC_OK) return rc;
    // The candidate lists must fit the fixed scratch: one entry per pixel and view.
    const int64_t plane = (int64_t)H * W;
    if (plane * n_views > (int64_t)OCC_NOALLOC_MAX_PIXEL_VIEWS) return OCC_ERR_CAPACITY;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    DeviceSetup& s = g_setup[dev];
    if (!s.done.load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lock(s.mu);
        if (!s.done.load(std::memory_order_relaxed)) {
            if (setup_device(s) != cudaSuccess) return OCC_ERR_CUDA;
            s.done.store(true, std::memory_order_release);
        }
    }

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // run_frames clears the header, statistics, status and line flags this call uses; the lists need no clearing.
    FrameIn fr{D, pitch, H, W, O, M, nullptr, nullptr, plane};
    const int r = run_frames(s.sc, &fr, 1, a, st, nullptr);
    if (r != OCC_OK) return r;
    if (status && cudaMemcpyAsync(status, s.sc.status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return OCC_ERR_CUDA;
    return OCC_OK;
}
