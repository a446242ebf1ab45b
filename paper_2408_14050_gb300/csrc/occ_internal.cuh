// occ_internal.cuh -- layout of the context scratch and the launch arguments shared by the kernels
// (occ_kernels.cu) and the host side of the C ABI (occ_api.cu, occ_noalloc.cu).  Not part of the public interface.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "occ.h"

namespace occ {

constexpr int kMaxViews = OCC_MAX_VIEWS;

// Words of the per-call device header (uint32).  The host clears the header (and the statistics after it) with one
// memset at the start of every detect call; the kernels then fill it in stream order.
enum : int {
    HDR_STATUS = 0,                  // status bits (ST_*)
    HDR_MAX = 1,                     // max D, order-preserving encoding (atomicMax)
    HDR_NEGMIN = 2,                  // min D, complemented encoding (atomicMax)
    HDR_COUNT = 8,                   // [kMaxViews] candidates found per view (may exceed the list capacity)
    HDR_L = HDR_COUNT + kMaxViews,   // [kMaxViews] scan length used per view (Eq. 3)
    HDR_WORDS = HDR_L + kMaxViews,
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
constexpr int kClassCap[kNumClasses] = {256, 1024, 4096};
// The line-per-thread scan kernel keeps N/2 sorted neighbours in registers; larger N use the warp kernel only.
constexpr int kLineMaxHalf = 4;
// Position tables: per view, for g = -kTabHalf .. kTabHalf, round(fl(cos a * g)) and round(fl(sin a * g)).
constexpr int kTabHalf = (OCC_MAX_SCAN + 1) / 2;
constexpr int kTabLen = 2 * kTabHalf + 1;

struct ViewArg {
    float c, s, r;   // binary32 cos(alpha), sin(alpha), ratio
    int32_t ridx;    // index of r in Args::ratio
};

struct Args {
    const float* D;
    int64_t pitch;   // elements between rows of D
    int32_t H, W;
    int32_t nv, nr;  // views, distinct ratios
    float gamma, zeta, beta;
    int32_t Lover;   // > 0: fixed scan length; else Eq. 3 per view
    int32_t N;
    ViewArg view[kMaxViews];
    float ratio[kMaxViews];
    uint32_t* cand;               // [nv][cand_cap] packed (y << 16) | x
    int64_t cand_cap;
    int32_t* ptab;                // [nv][kTabLen] packed (dx & 0xFFFF) | (dy << 16), or kTabExact; null: no tables
    uint32_t* fb;                 // [nv][fb_words] bit per candidate: left to the warp kernel (null: all are)
    int64_t fb_words;
    uint32_t* hdr;                // HDR_WORDS
    unsigned long long* stats;    // [nv][2]: samples, pair tests
    int32_t* O;                   // [nv][H][W]
    uint8_t* M;                   // [nv][H][W]
    float* E;                     // [H][W] or null
    float* A;                     // [H][W] or null
};

// Launchers (occ_kernels.cu).  Each returns the cudaGetLastError() of its launch.
cudaError_t launch_edges(const Args& a, int grid, cudaStream_t st);
cudaError_t launch_tables(const Args& a, cudaStream_t st);
// The line-per-thread scan over every view; wide = true when H * pitch does not fit in int32.
cudaError_t launch_scan_lines(const Args& a, int grid, bool wide, cudaStream_t st);
cudaError_t launch_scan(const Args& a, int cls, int grid, cudaStream_t st);
cudaError_t launch_mask(const Args& a, int grid, cudaStream_t st);
// Per-SM resident blocks of each kernel (for persistent grids); also sets the shared-memory opt-ins.
cudaError_t configure_kernels(int* edges_blocks_per_sm, int* lines_blocks_per_sm,
                              int scan_blocks_per_sm[kNumClasses], int* mask_blocks_per_sm);

}  // namespace occ
