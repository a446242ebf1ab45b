// occ_fusion.cu -- the two steps around the detection in the registration pipeline of a camera array:
//   k_median  the pixel-wise median of the stereo disparity maps of the peripheral cameras, which gives the fused
//             center map D the detection runs on (Section 4.2);
//   k_warp    the backward warp of every peripheral image to the center view along its baseline, bilinear, with
//             the occluded pixels (M of the detection) and the pixels that fall outside the peripheral image set to
//             0 (Section 1 and Section 4.2: the occluded pixels are the ones left for reconstruction).
// Both are one pass over their inputs, HBM-bound, one thread per pixel with the loads of a warp on consecutive
// columns; neither needs scratch memory.  Arithmetic is binary32, one rounding per operation, no contraction
// (explicit __fadd_rn / __fmul_rn / __fsub_rn, and the file is compiled with --fmad=false).
#include <cfloat>
#include <cstdint>

#include "occ.h"

namespace {

constexpr int kMaxMaps = 64;
constexpr int kFuseThreads = 256;
constexpr int kWarpThreads = 256;

__device__ int32_t g_status_sink;

struct MedianArgs {
    const float* maps[kMaxMaps];
    int n;
    int H, W;
    int64_t pitch;
    float* D;
    int64_t d_pitch;
    int32_t* status;
};

__device__ __forceinline__ bool finite_f(float x) { return fabsf(x) <= FLT_MAX; }

// Ascending bitonic sorting network over P values (P a power of two), fully unrolled into registers.
template <int P>
__device__ __forceinline__ void bitonic_sort(float (&v)[P])
{
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < P; i++) {
                const int l = i ^ j;
                if (l > i) {
                    const float a = v[i], b = v[l];
                    const float lo = fminf(a, b), hi = fmaxf(a, b);
                    const bool up = (i & k) == 0;
                    v[i] = up ? lo : hi;
                    v[l] = up ? hi : lo;
                }
            }
        }
    }
}

// Median of the n maps at each pixel: the n values (signed zeros entered as +0 by adding +0, so that equal values
// are equal bit patterns and the network's order of ties cannot show) padded to P with +inf, sorted; odd n gives
// the middle value, even n fl(fl(a + b) * 0.5) of the two middle values.  A non-finite value sets *status.
template <int P>
__device__ __forceinline__ float median_of(float (&v)[P], int n)
{
    bitonic_sort<P>(v);
    const int mid = n >> 1;
    float lo = 0.0f, hi = 0.0f;
#pragma unroll P
    for (int m = 0; m < P; m++) {
        if (m == mid - 1) lo = v[m];
        if (m == mid) hi = v[m];
    }
    return (n & 1) ? hi : __fmul_rn(__fadd_rn(lo, hi), 0.5f);
}

__device__ __forceinline__ float median_in(float d, bool& bad)
{
    bad |= !finite_f(d);
    return __fadd_rn(d, 0.0f);
}

// One pixel per thread and row step.
template <int P>
__global__ void __launch_bounds__(kFuseThreads) k_median(const __grid_constant__ MedianArgs a)
{
    const int x = blockIdx.x * kFuseThreads + threadIdx.x;
    if (x >= a.W) return;
    bool bad = false;
    for (int y = blockIdx.y; y < a.H; y += gridDim.y) {
        const int64_t off = (int64_t)y * a.pitch + x;
        float v[P];
#pragma unroll
        for (int m = 0; m < P; m++) v[m] = m < a.n ? median_in(__ldcs(a.maps[m] + off), bad) : __int_as_float(0x7f800000);
        a.D[(int64_t)y * a.d_pitch + x] = median_of<P>(v, a.n);
    }
    if (bad) *a.status = OCC_ERR_NONFINITE_INPUT;
}

// Batcher's odd-even merge sorting network for 8 values (19 compare-exchanges).
__device__ __forceinline__ void cex(float& a, float& b)
{
    const float lo = fminf(a, b), hi = fmaxf(a, b);
    a = lo;
    b = hi;
}

__device__ __forceinline__ void sort8(float (&v)[8])
{
    cex(v[0], v[1]); cex(v[2], v[3]); cex(v[4], v[5]); cex(v[6], v[7]);
    cex(v[0], v[2]); cex(v[1], v[3]); cex(v[4], v[6]); cex(v[5], v[7]);
    cex(v[1], v[2]); cex(v[5], v[6]);
    cex(v[0], v[4]); cex(v[1], v[5]); cex(v[2], v[6]); cex(v[3], v[7]);
    cex(v[2], v[4]); cex(v[3], v[5]);
    cex(v[1], v[2]); cex(v[3], v[4]); cex(v[5], v[6]);
}

// Median of exactly N <= 8 maps (N a compile-time constant): the unused slots are the constant +inf, so the
// compare-exchanges that involve them fold away, and the middle positions are known registers.
template <int N>
__global__ void __launch_bounds__(kFuseThreads) k_median_n(const __grid_constant__ MedianArgs a)
{
    static_assert(N >= 1 && N <= 8, "up to 8 maps");
    const int x = blockIdx.x * kFuseThreads + threadIdx.x;
    if (x >= a.W) return;
    bool bad = false;
    for (int y = blockIdx.y; y < a.H; y += gridDim.y) {
        const int64_t off = (int64_t)y * a.pitch + x;
        float v[8];
#pragma unroll
        for (int m = 0; m < 8; m++) v[m] = m < N ? median_in(__ldcs(a.maps[m] + off), bad) : __int_as_float(0x7f800000);
        sort8(v);
        const float med = (N & 1) ? v[N / 2] : __fmul_rn(__fadd_rn(v[N / 2 - 1], v[N / 2]), 0.5f);
        a.D[(int64_t)y * a.d_pitch + x] = med;
    }
    if (bad) *a.status = OCC_ERR_NONFINITE_INPUT;
}

struct WarpArgs {
    const float* D;
    int H, W;
    int64_t pitch;
    int nv;
    float c[kMaxMaps], s[kMaxMaps], r[kMaxMaps];
    const float* img[kMaxMaps];
    int64_t img_pitch;
    const uint8_t* M;
    float* out;
};

// The center pixel (x, y) with disparity d = fl(r D) was seen by the peripheral camera at (x - cos(a) d,
// y - sin(a) d): content moves by -r D along the baseline.  Its value there is the bilinear interpolation of the
// peripheral image, top = I00 + fx (I01 - I00), bottom = I10 + fx (I11 - I10), top + fy (bottom - top), with the
// upper neighbours clamped to the last row / column.  Positions outside [0, W-1] x [0, H-1] give 0.
__device__ __forceinline__ float warp_px(const WarpArgs& a, int v, int x, int y, float dc)
{
    const float d = __fmul_rn(a.r[v], dc);
    const float sx = __fsub_rn((float)x, __fmul_rn(a.c[v], d));
    const float sy = __fsub_rn((float)y, __fmul_rn(a.s[v], d));
    if (!(sx >= 0.0f && sx <= (float)(a.W - 1) && sy >= 0.0f && sy <= (float)(a.H - 1))) return 0.0f;
    const float fx0 = floorf(sx), fy0 = floorf(sy);
    const int x0 = (int)fx0, y0 = (int)fy0;
    const int x1 = x0 + 1 < a.W ? x0 + 1 : x0;
    const int y1 = y0 + 1 < a.H ? y0 + 1 : y0;
    const float fx = __fsub_rn(sx, fx0), fy = __fsub_rn(sy, fy0);
    const float* I = a.img[v];
    const float i00 = __ldg(I + (int64_t)y0 * a.img_pitch + x0);
    const float i01 = __ldg(I + (int64_t)y0 * a.img_pitch + x1);
    const float i10 = __ldg(I + (int64_t)y1 * a.img_pitch + x0);
    const float i11 = __ldg(I + (int64_t)y1 * a.img_pitch + x1);
    const float top = __fadd_rn(i00, __fmul_rn(fx, __fsub_rn(i01, i00)));
    const float bot = __fadd_rn(i10, __fmul_rn(fx, __fsub_rn(i11, i10)));
    return __fadd_rn(top, __fmul_rn(fy, __fsub_rn(bot, top)));
}

// One pixel per thread and row step; occluded pixels (M != 0) give 0.  D is read once for all views.
__global__ void __launch_bounds__(kWarpThreads) k_warp(const __grid_constant__ WarpArgs a)
{
    const int x = blockIdx.x * kWarpThreads + threadIdx.x;
    if (x >= a.W) return;
    const int64_t plane = (int64_t)a.H * a.W;
    for (int y = blockIdx.y; y < a.H; y += gridDim.y) {
        const float dc = __ldg(a.D + (int64_t)y * a.pitch + x);
        const int64_t o = (int64_t)y * a.W + x;
        for (int v = 0; v < a.nv; v++) {
            const bool occluded = a.M && __ldcs(a.M + (int64_t)v * plane + o) != 0;
            __stcs(a.out + (int64_t)v * plane + o, occluded ? 0.0f : warp_px(a, v, x, y, dc));
        }
    }
}

// Four consecutive pixels per thread: 16-byte loads of D and stores of the output, 4-byte loads of M.  The four
// pixels' positions are computed first and their sixteen gathers issued together (out-of-range or occluded pixels
// read a clamped, valid address and are zeroed afterwards), so that the gathers of a view overlap.
struct WarpTap {
    int o00, o01, o10, o11;   // element offsets (the host checks that H x img_pitch fits in 31 bits)
    float fx, fy;
    bool ok;
};

__device__ __forceinline__ WarpTap warp_tap(const WarpArgs& a, int v, int x, int y, float dc)
{
    WarpTap t;
    const float d = __fmul_rn(a.r[v], dc);
    const float sx = __fsub_rn((float)x, __fmul_rn(a.c[v], d));
    const float sy = __fsub_rn((float)y, __fmul_rn(a.s[v], d));
    t.ok = sx >= 0.0f && sx <= (float)(a.W - 1) && sy >= 0.0f && sy <= (float)(a.H - 1);
    const float fx0 = t.ok ? floorf(sx) : 0.0f, fy0 = t.ok ? floorf(sy) : 0.0f;
    const int x0 = (int)fx0, y0 = (int)fy0;
    const int x1 = x0 + 1 < a.W ? x0 + 1 : x0;
    const int y1 = y0 + 1 < a.H ? y0 + 1 : y0;
    t.fx = __fsub_rn(t.ok ? sx : 0.0f, fx0);
    t.fy = __fsub_rn(t.ok ? sy : 0.0f, fy0);
    const int ip = (int)a.img_pitch;
    t.o00 = y0 * ip + x0;
    t.o01 = y0 * ip + x1;
    t.o10 = y1 * ip + x0;
    t.o11 = y1 * ip + x1;
    return t;
}

__device__ __forceinline__ float bilinear(float fx, float fy, float i00, float i01, float i10, float i11)
{
    const float top = __fadd_rn(i00, __fmul_rn(fx, __fsub_rn(i01, i00)));
    const float bot = __fadd_rn(i10, __fmul_rn(fx, __fsub_rn(i11, i10)));
    return __fadd_rn(top, __fmul_rn(fy, __fsub_rn(bot, top)));
}

__global__ void __launch_bounds__(kWarpThreads, 5) k_warp4(const __grid_constant__ WarpArgs a)
{
    const int q = blockIdx.x * kWarpThreads + threadIdx.x;
    const int x = 4 * q;
    if (x >= a.W) return;
    const int64_t plane = (int64_t)a.H * a.W;
    for (int y = blockIdx.y; y < a.H; y += gridDim.y) {
        const float4 dc = __ldg(reinterpret_cast<const float4*>(a.D + (int64_t)y * a.pitch + x));
        const float dv[4] = {dc.x, dc.y, dc.z, dc.w};
        const int64_t o = (int64_t)y * a.W + x;
        for (int v = 0; v < a.nv; v++) {
            const uint32_t m = a.M ? __ldcs(reinterpret_cast<const unsigned int*>(a.M + (int64_t)v * plane + o)) : 0u;
            const float* I = a.img[v];
            WarpTap t[4];
            float g[4][4];
#pragma unroll
            for (int j = 0; j < 4; j++) t[j] = warp_tap(a, v, x + j, y, dv[j]);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                g[j][0] = __ldg(I + t[j].o00);
                g[j][1] = __ldg(I + t[j].o01);
                g[j][2] = __ldg(I + t[j].o10);
                g[j][3] = __ldg(I + t[j].o11);
            }
            float r[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const bool keep = t[j].ok && ((m >> (8 * j)) & 0xffu) == 0;
                r[j] = keep ? bilinear(t[j].fx, t[j].fy, g[j][0], g[j][1], g[j][2], g[j][3]) : 0.0f;
            }
            __stcs(reinterpret_cast<float4*>(a.out + (int64_t)v * plane + o), make_float4(r[0], r[1], r[2], r[3]));
        }
    }
}

bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; }
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Rows per grid column: enough blocks to fill the GPU several times over, at most 65535.
int row_blocks(int H, int col_blocks)
{
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    int64_t want = ((int64_t)sms * 16 + col_blocks - 1) / col_blocks;
    if (want < 1) want = 1;
    if (want > H) want = H;
    if (want > 65535) want = 65535;
    return (int)want;
}

}  // namespace

extern "C" int occ_fuse_median(const float* const* maps, int32_t n_maps, int32_t H, int32_t W, int64_t pitch,
                               float* D, int64_t d_pitch, int32_t* status, void* stream)
{
    if (!maps || !D || n_maps < 1 || n_maps > kMaxMaps || H < 1 || W < 1 || H > OCC_MAX_SIDE || W > OCC_MAX_SIDE)
        return OCC_ERR_INVALID_ARG;
    if (pitch == 0) pitch = W;
    if (d_pitch == 0) d_pitch = W;
    if (pitch < W || d_pitch < W || !aligned4(D) || (status && !aligned4(status))) return OCC_ERR_INVALID_ARG;
    MedianArgs a{};
    for (int m = 0; m < n_maps; m++) {
        if (!maps[m] || !aligned4(maps[m])) return OCC_ERR_INVALID_ARG;
        a.maps[m] = maps[m];
    }
    a.n = n_maps;
    a.H = H;
    a.W = W;
    a.pitch = pitch;
    a.D = D;
    a.d_pitch = d_pitch;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int32_t* flag = status;
    if (flag && cudaMemsetAsync(flag, 0, sizeof(int32_t), st) != cudaSuccess) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    if (!flag) {
        // No status word: the non-finite flag goes to a word of the library that nobody reads.
        void* sink = nullptr;
        if (cudaGetSymbolAddress(&sink, g_status_sink) != cudaSuccess) {
            cudaGetLastError();
            return OCC_ERR_CUDA;
        }
        flag = static_cast<int32_t*>(sink);
    }
    a.status = flag;
    const int cols = (W + kFuseThreads - 1) / kFuseThreads;
    const dim3 grid(cols, row_blocks(H, cols));
    // One pixel per thread (full occupancy, up to eight 4-byte loads in flight per thread) measured faster than four
    // pixels per thread (16-byte loads, a quarter of the occupancy).
    if (n_maps <= 8) {
        switch (n_maps) {
        case 1: k_median_n<1><<<grid, kFuseThreads, 0, st>>>(a); break;
        case 2: k_median_n<2><<<grid, kFuseThreads, 0, st>>>(a); break;
        case 3: k_median_n<3><<<grid, kFuseThreads, 0, st>>>(a); break;
        case 4: k_median_n<4><<<grid, kFuseThreads, 0, st>>>(a); break;
        case 5: k_median_n<5><<<grid, kFuseThreads, 0, st>>>(a); break;
        case 6: k_median_n<6><<<grid, kFuseThreads, 0, st>>>(a); break;
        case 7: k_median_n<7><<<grid, kFuseThreads, 0, st>>>(a); break;
        default: k_median_n<8><<<grid, kFuseThreads, 0, st>>>(a); break;
        }
    }
    else if (n_maps <= 16) k_median<16><<<grid, kFuseThreads, 0, st>>>(a);
    else if (n_maps <= 32) k_median<32><<<grid, kFuseThreads, 0, st>>>(a);
    else k_median<64><<<grid, kFuseThreads, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return OCC_ERR_CUDA;
    return OCC_OK;
}

extern "C" int occ_warp_views(const float* D, int32_t H, int32_t W, int64_t pitch, const occ_view* views,
                              int32_t n_views, const float* const* images, int64_t img_pitch, const uint8_t* M,
                              float* out, void* stream)
{
    if (!D || !views || !images || !out || n_views < 1 || n_views > kMaxMaps || H < 1 || W < 1 ||
        H > OCC_MAX_SIDE || W > OCC_MAX_SIDE)
        return OCC_ERR_INVALID_ARG;
    if (pitch == 0) pitch = W;
    if (img_pitch == 0) img_pitch = W;
    if (pitch < W || img_pitch < W || !aligned4(D) || !aligned4(out)) return OCC_ERR_INVALID_ARG;
    WarpArgs a{};
    for (int v = 0; v < n_views; v++) {
        const float r = views[v].ratio;
        if (!(r > 0.0f) || !(r <= FLT_MAX) || !images[v] || !aligned4(images[v])) return OCC_ERR_INVALID_ARG;
        occ_direction(views[v].alpha_deg, &a.c[v], &a.s[v]);
        a.r[v] = r;
        a.img[v] = images[v];
    }
    a.D = D;
    a.H = H;
    a.W = W;
    a.pitch = pitch;
    a.nv = n_views;
    a.img_pitch = img_pitch;
    a.M = M;
    a.out = out;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if ((W & 3) == 0 && (pitch & 3) == 0 && aligned16(D) && aligned16(out) &&
        (!M || (reinterpret_cast<uintptr_t>(M) & 3) == 0) && (int64_t)H * img_pitch < ((int64_t)1 << 31)) {
        const int qcols = (W / 4 + kWarpThreads - 1) / kWarpThreads;
        k_warp4<<<dim3(qcols, row_blocks(H, qcols)), kWarpThreads, 0, st>>>(a);
    } else {
        const int cols = (W + kWarpThreads - 1) / kWarpThreads;
        k_warp<<<dim3(cols, row_blocks(H, cols)), kWarpThreads, 0, st>>>(a);
    }
    if (cudaGetLastError() != cudaSuccess) return OCC_ERR_CUDA;
    return OCC_OK;
}
