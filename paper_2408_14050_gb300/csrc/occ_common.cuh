// occ_common.cuh -- device helpers of the candidate pass shared by the kernels of occ_kernels.cu and the fused launch
// of occ_strip.cu: the order-preserving float codes of the min/max reduction, the scan length of Eq. 3, the per-view
// position tables, and the min/max of one quad of D.
#pragma once

#include <cstdint>

#include "occ_internal.cuh"

namespace occ {
namespace {

// Order-preserving map of binary32 onto uint32 (larger float -> larger code) for atomicMax-based min/max.
__device__ __forceinline__ uint32_t f2ord(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

// Scan length L of a view of ratio r (Eq. 3) from the frame's min/max codes (HDR_MAX, HDR_NEGMIN), or the fixed L;
// -1 when the automatic L exceeds OCC_MAX_SCAN.  max D_r = fl(r max D) and min D_r = fl(r min D): rounding is
// monotone.
__device__ __forceinline__ int scan_length(const Args& a, uint32_t hmax, uint32_t hnegmin, float r)
{
    if (a.Lover > 0) return a.Lover;
    const float mx = ord2f(hmax);
    const float mn = ord2f(~hnegmin);
    const float dmx = (r == 1.0f) ? mx : __fmul_rn(r, mx);
    const float dmn = (r == 1.0f) ? mn : __fmul_rn(r, mn);
    const float t = __fmul_rn(__fsub_rn(dmx, dmn), 2.0f);
    return (t <= (float)OCC_MAX_SCAN) ? (int)ceilf(t) : -1;
}

// Marks a position-table entry whose nearest pixel must be computed exactly (see k_tables).
constexpr int32_t kTabExact = (int32_t)0x80008000;

// Entry i of the list kernels' position tables (view i / kTabLen, g = i % kTabLen - kTabHalf): the packed pixel
// offsets of Eq. 4 (see k_tables).
__device__ __forceinline__ void tables_entry(const Args& a, int64_t i)
{
    const int v = (int)(i / kTabLen);
    const int j = (int)(i - (int64_t)v * kTabLen);
    const float g = (float)(j - kTabHalf);
    const float tx = __fmul_rn(a.view[v].c, g), ty = __fmul_rn(a.view[v].s, g);
    const float fx = tx - floorf(tx), fy = ty - floorf(ty);
    const bool risky = fabsf(fx - 0.5f) <= 0.00390625f || fabsf(fy - 0.5f) <= 0.00390625f;
    const int dx = (int)roundf(tx), dy = (int)roundf(ty);
    a.ptab[(int64_t)v * kTabLen + j] = risky ? kTabExact : (int32_t)((uint32_t)(dx & 0xFFFF) | ((uint32_t)dy << 16));
}


// Min, max and the non-finite check over quad q (4 pixels of a row, QW quads per row) of a frame's D; vec: rows are
// 16-byte aligned, so a whole quad is one float4 load.
__device__ __forceinline__ void minmax_quad(const float* Dp, int64_t pitch, int W, int QW, bool vec, int64_t q,
                                            float& lo, float& hi, bool& bad)
{
    const int y = (int)(q / QW);
    const int x0 = (int)(q - (int64_t)y * QW) * 4;
    const float* row = Dp + (int64_t)y * pitch;
    float d[4];
    if (vec && x0 + 4 <= W) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(row + x0));
        d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) d[j] = (x0 + j < W) ? __ldg(row + x0 + j) : d[0];
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        lo = fminf(lo, d[j]);
        hi = fmaxf(hi, d[j]);
        bad |= !isfinite(d[j]);
    }
}

}  // namespace
}  // namespace occ
