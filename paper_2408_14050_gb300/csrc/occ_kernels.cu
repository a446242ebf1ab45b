// occ_kernels.cu -- sm_103a kernels of the fast edge-aware occlusion detection (Sippel, Seiler, Kaup, ICIP 2024,
// Section 3).
//
//   k_frames      frame records of a batch, from launch parameters into device memory.
//   k_tables      per view, the scan-line pixel offsets round(fl(cos a * g)), round(fl(sin a * g)) for every g.
//   k_edges       one pass over D: Eq. 1 forward differences on D_r = fl(r D) for every distinct baseline ratio,
//                 the candidate predicate of Eq. 2 for every view (optionally restricted to proposed tiles), the
//                 compaction of the candidate lists, the min/max reduction Eq. 3 needs, the non-finite check, the
//                 optional E / A maps, the zeroing of O and of the tile hit flags.
//   k_plan        per frame and view: the scan length (Eq. 3), its size class, the candidate counts, and the prefix
//                 sums that number the scan work.
//   k_scan_lines  one thread per scan line, every line once as one stream through a one-slot buffer: Eq. 4
//                 positions and gathers, the warp W = G - V, the sort, the neighbour test of Eq. 5 and the
//                 accumulation into O (Eq. 6); a line that turns out to need more lists itself for k_merge_lines.
//   k_merge_lines one thread per list entry, two kinds of independent work items: the two-buffer merge of a line of
//                 two macro-runs, and the stream of a broken line again with negated counts (which takes its
//                 partial counts back); longer lines are flagged for k_scan by k_scan_lines.
//   k_scan        one warp per scan line (any line, any N): the same steps with the sort as a merge of the line's
//                 monotone runs or, for many runs, a counting sort by W bucket.
//   k_mask        M = (O > 0) (Eq. 6).
//
// Every floating-point operation that decides a candidate, a position, an order or a count is an explicit
// round-to-nearest binary32 intrinsic (__fmul_rn, __fadd_rn, __fsub_rn, __fsqrt_rn) and the file is compiled with
// --fmad=false, so the results are bit-identical to a plain one-operation-at-a-time binary32 evaluation.
#include <cstdint>
#include <cstring>

#include "occ_internal.cuh"
#include "occ_common.cuh"
#include "occ_scanline.cuh"

namespace occ {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// O[p] += o as a reduction (no return value) predicated on o != 0 inside the asm: the count of a sample leaving the
// window goes to O without a divergent branch around the atomic.
__device__ __forceinline__ void o_red(int32_t* addr, int o)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %1, 0;\n\t@q red.add.s32 [%0], %1;\n\t}" ::"l"(addr), "r"(o)
                 : "memory");
}

// ------------------------------------------------------------------------------------------------------------------
// k_edges: Eq. 1, Eq. 2 (predicate + compaction), Eq. 3 (min/max), E/A, O = 0.
//
// Each thread owns a quad of 4 consecutive pixels of one row; quads are numbered row-major, so a warp covers 128
// consecutive pixels and its loads of D (this row and the next) are fully coalesced float4 loads.  Candidates of
// view v are appended to list v: one ballot per pixel slot gives every lane its offset inside the warp, the block
// combines its 8 warp totals, and one atomicAdd per block and view reserves the block's range in the list.

constexpr int kEdgeThreads = 256;
constexpr int kEdgeWarps = kEdgeThreads / 32;

__device__ __forceinline__ void load_quad(const float* row, int x0, int W, bool vec, float out[5])
{
    if (vec && x0 + 4 <= W) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(row + x0));
        out[0] = t.x; out[1] = t.y; out[2] = t.z; out[3] = t.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) out[j] = (x0 + j < W) ? __ldg(row + x0 + j) : 0.0f;
    }
    out[4] = (x0 + 4 < W) ? __ldg(row + x0 + 4) : 0.0f;
}

__global__ void __launch_bounds__(kEdgeThreads) k_edges(const __grid_constant__ Args a)
{
    __shared__ uint32_t s_tot[kEdgeWarps][kMaxViews];
    __shared__ uint32_t s_base[kEdgeWarps][kMaxViews];
    __shared__ float s_lo[kEdgeWarps], s_hi[kEdgeWarps];
    __shared__ int s_bad;

    const FrameArg F = a.frames[blockIdx.y];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = F.W, H = F.H;
    const int QW = (W + 3) >> 2;
    const int64_t nq = (int64_t)H * QW;
    const int64_t plane = (int64_t)H * W;
    const bool vecD = ((F.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(F.D) & 15) == 0);
    const bool vecO = ((W & 3) == 0) && ((reinterpret_cast<uintptr_t>(F.O) & 15) == 0);
    const unsigned lt = (1u << lane) - 1u;

    if (threadIdx.x == 0) s_bad = 0;
    float lo = INFINITY, hi = -INFINITY;
    bool bad = false;

    for (int64_t q0 = (int64_t)blockIdx.x * kEdgeThreads; q0 < nq; q0 += (int64_t)gridDim.x * kEdgeThreads) {
        const int64_t q = q0 + threadIdx.x;
        const bool active = q < nq;
        int y = 0, x0 = 0;
        float d[5] = {0, 0, 0, 0, 0}, dn[5] = {0, 0, 0, 0, 0};
        bool valid[4] = {false, false, false, false};
        bool hasd = false;
        if (active) {
            y = (int)(q / QW);
            x0 = (int)(q - (int64_t)y * QW) * 4;
            load_quad(F.D + (int64_t)y * F.pitch, x0, W, vecD, d);
            hasd = (y + 1 < H);
            if (hasd) load_quad(F.D + (int64_t)(y + 1) * F.pitch, x0, W, vecD, dn);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                valid[j] = (x0 + j < W);
                if (valid[j]) {
                    lo = fminf(lo, d[j]);
                    hi = fmaxf(hi, d[j]);
                    bad |= !isfinite(d[j]);
                }
            }
        }

        // E and A of D itself (r = 1).
        if (active && (F.E || F.A)) {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (!valid[j]) continue;
                const float ex = (x0 + j + 1 < W) ? __fsub_rn(d[j + 1], d[j]) : 0.0f;
                const float ey = hasd ? __fsub_rn(dn[j], d[j]) : 0.0f;
                const int64_t o = (int64_t)y * W + x0 + j;
                if (F.E) F.E[o] = __fsqrt_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)));
                if (F.A) F.A[o] = atan2f(ey, ex);
            }
        }

        // Eq. 1 on D_r for every distinct ratio, Eq. 2 for every view of that ratio.
        uint64_t bits[4] = {0, 0, 0, 0};
        if (active && a.any_list) {
            for (int u = 0; u < a.nr; u++) {
                const float r = a.ratio[u];
                const bool one = (r == 1.0f);
                float ex[4], ey[4];
                bool pe[4];
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const float dr = one ? d[j] : __fmul_rn(r, d[j]);
                    const float rr = one ? d[j + 1] : __fmul_rn(r, d[j + 1]);
                    const float dd = one ? dn[j] : __fmul_rn(r, dn[j]);
                    ex[j] = (x0 + j + 1 < W) ? __fsub_rn(rr, dr) : 0.0f;
                    ey[j] = hasd ? __fsub_rn(dd, dr) : 0.0f;
                    // E > gamma (Eq. 2) without the square root: E_x^2 + E_y^2 >= e2min is the same test.
                    const float e2 = __fadd_rn(__fmul_rn(ex[j], ex[j]), __fmul_rn(ey[j], ey[j]));
                    pe[j] = valid[j] && (e2 >= a.e2min);
                }
                for (int v = 0; v < a.nv; v++) {
                    if (a.view[v].ridx != u || a.view[v].fam >= 0) continue;   // strip views: k_strip
                    const float c = a.view[v].c, s = a.view[v].s;
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const float dot = __fadd_rn(__fmul_rn(ex[j], c), __fmul_rn(ey[j], s));
                        if (pe[j] && dot > 0.0f) bits[j] |= (1ull << v);
                    }
                }
            }
        }

        // Tile proposals: candidates of tiles proposed empty are dropped from the lists (the 4 pixels of a quad lie in
        // one tile).  The top-left quad of each tile clears the tile's hit flags.
        if (active && (F.prop || F.hits)) {
            const int tpv = F.tiles_x * F.tiles_y;
            const int t = (y / kTile) * F.tiles_x + x0 / kTile;
            if (F.prop) {
                uint64_t keep = 0;
                for (int v = 0; v < a.nv; v++)
                    if (F.prop[(int64_t)v * tpv + t]) keep |= 1ull << v;
#pragma unroll
                for (int j = 0; j < 4; j++) bits[j] &= keep;
            }
            if (F.hits && (y % kTile) == 0 && (x0 % kTile) == 0)
                for (int v = 0; v < a.nv; v++) F.hits[(int64_t)v * tpv + t] = 0;
        }

        // Compaction: warp totals per view, then one reservation per block and view; candidates keep pixel order.
        if (a.nv <= 8) {
            // Up to 8 views: the thread's candidate counts (0..4) of all views packed in bytes of one 64-bit word,
            // so that one warp scan gives every view's prefix (a warp's total per view is at most 128).
            uint32_t vm[8];
            uint64_t packed = 0;
#pragma unroll
            for (int v = 0; v < 8; v++) {
                vm[v] = 0;
#pragma unroll
                for (int j = 0; j < 4; j++) vm[v] |= (uint32_t)((bits[j] >> v) & 1ull) << j;
                packed |= (uint64_t)__popc(vm[v]) << (8 * v);
            }
            uint64_t incl = packed;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            const uint64_t total = __shfl_sync(kFull, incl, 31);
            const uint64_t excl = incl - packed;
            if (lane == 0)
#pragma unroll
                for (int v = 0; v < 8; v++)
                    if (v < a.nv) s_tot[warp][v] = (uint32_t)((total >> (8 * v)) & 0xffu);
            __syncthreads();
            if (threadIdx.x < a.nv) {
                const int v = threadIdx.x;
                uint32_t sum = 0;
#pragma unroll
                for (int w = 0; w < kEdgeWarps; w++) sum += s_tot[w][v];
                uint32_t base = sum ? atomicAdd(&F.hdr[HDR_COUNT + v], sum) : 0u;
#pragma unroll
                for (int w = 0; w < kEdgeWarps; w++) {
                    s_base[w][v] = base;
                    base += s_tot[w][v];
                }
            }
            __syncthreads();
            if (packed) {
#pragma unroll
                for (int v = 0; v < 8; v++) {
                    uint32_t m = vm[v];
                    if (v >= a.nv || !m) continue;
                    uint32_t pos = s_base[warp][v] + (uint32_t)((excl >> (8 * v)) & 0xffu);
                    while (m) {
                        const int j = __ffs(m) - 1;
                        m &= m - 1;
                        if ((int64_t)pos < F.cap)
                            F.cand[(int64_t)v * F.cap + pos] = ((uint32_t)y << 16) | (uint32_t)(x0 + j);
                        else
                            atomicOr(&F.hdr[HDR_STATUS], ST_CAND_OVERFLOW);
                        pos++;
                    }
                }
            }
        } else {
            for (int v = 0; v < a.nv; v++) {
                uint32_t tot = 0;
#pragma unroll
                for (int j = 0; j < 4; j++) tot += __popc(__ballot_sync(kFull, (bits[j] >> v) & 1ull));
                if (lane == 0) s_tot[warp][v] = tot;
            }
            __syncthreads();
            if (threadIdx.x < a.nv) {
                const int v = threadIdx.x;
                uint32_t sum = 0;
#pragma unroll
                for (int w = 0; w < kEdgeWarps; w++) sum += s_tot[w][v];
                uint32_t base = sum ? atomicAdd(&F.hdr[HDR_COUNT + v], sum) : 0u;
#pragma unroll
                for (int w = 0; w < kEdgeWarps; w++) {
                    s_base[w][v] = base;
                    base += s_tot[w][v];
                }
            }
            __syncthreads();
            for (int v = 0; v < a.nv; v++) {
                unsigned bal[4];
                uint32_t pre = 0;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    bal[j] = __ballot_sync(kFull, (bits[j] >> v) & 1ull);
                    pre += __popc(bal[j] & lt);
                }
                uint32_t pos = s_base[warp][v] + pre;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    if ((bits[j] >> v) & 1ull) {
                        if ((int64_t)pos < F.cap)
                            F.cand[(int64_t)v * F.cap + pos] = ((uint32_t)y << 16) | (uint32_t)(x0 + j);
                        else
                            atomicOr(&F.hdr[HDR_STATUS], ST_CAND_OVERFLOW);
                        pos++;
                    }
                }
            }
        }

        // O = 0 for the quad in every list-path view (the scan kernels accumulate into it; k_strip writes O of the
        // strip views once).
        if (active && a.any_list) {
            const int64_t o = (int64_t)y * W + x0;
            for (int v = 0; v < a.nv; v++) {
                if (a.view[v].fam >= 0) continue;
                int32_t* Ov = F.O + (int64_t)v * plane + o;
                if (vecO && x0 + 4 <= W) {
                    *reinterpret_cast<int4*>(Ov) = make_int4(0, 0, 0, 0);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        if (valid[j]) Ov[j] = 0;
                }
            }
        }
    }

    // Block reduction of min / max and the non-finite flag; one atomic per block.
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(kFull, lo, off));
        hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, off));
    }
    if (__any_sync(kFull, bad) && lane == 0) s_bad = 1;
    if (lane == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float blo = INFINITY, bhi = -INFINITY;
        for (int w = 0; w < kEdgeWarps; w++) {
            blo = fminf(blo, s_lo[w]);
            bhi = fmaxf(bhi, s_hi[w]);
        }
        if (blo <= bhi) {
            atomicMax(&F.hdr[HDR_MAX], f2ord(bhi));
            atomicMax(&F.hdr[HDR_NEGMIN], ~f2ord(blo));
        }
        if (s_bad) atomicOr(&F.hdr[HDR_STATUS], ST_NONFINITE);
    }
}

constexpr int kMinMaxThreads = 256;   // k_minmax (below, after k_plan, whose work its last block does)


// ------------------------------------------------------------------------------------------------------------------
// k_frames: copies a chunk of frame records from the launch parameters into the device frame table.

__global__ void k_frames(const __grid_constant__ FrameChunk c)
{
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) c.dst[c.first + i] = c.f[i];
}

// ------------------------------------------------------------------------------------------------------------------
// k_plan: per (frame, view) the scan length (Eq. 3 on D_r unless L is fixed), the size class of the scan lines and
// the candidate count; then the prefix sums that number the scan work items of all (frame, view)s and of each size
// class.  One block.

constexpr int kPlanThreads = 1024;

// The plan (see k_plan) by one block of T threads; frames: the call's frame records.  The frame headers are read
// through L2 (they may have been written by other blocks of the same launch, ahead of a releasing count).
template <int T>
__device__ __forceinline__ void plan_block(const Args& a, const FrameArg* frames)
{
    __shared__ uint32_t s_carry[1 + kNumClasses];
    __shared__ uint32_t s_warp[T / 32][1 + kNumClasses];
    const int n = a.nf * a.nv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 1 + kNumClasses) s_carry[threadIdx.x] = 0;
    uint32_t st_all = 0;
    __syncthreads();
    for (int base = 0; base < n; base += T) {
        const int i = base + threadIdx.x;
        uint32_t cnt[1 + kNumClasses] = {0, 0, 0, 0};
        if (i < n) {
            const int f = i / a.nv, v = i - f * a.nv;
            const FrameArg& F = frames[f];
            const uint32_t st = __ldcg(&F.hdr[HDR_STATUS]);
            PlanEntry pe{-1, 0, 0u, 0u};
            if (!(st & ST_NONFINITE)) {
                const int L = scan_length(a, __ldcg(&F.hdr[HDR_MAX]), __ldcg(&F.hdr[HDR_NEGMIN]), a.view[v].r);
                if (L < 0) {
                    atomicOr(&F.hdr[HDR_STATUS], ST_SCAN_TOO_LONG);
                    st_all |= ST_SCAN_TOO_LONG;
                } else {
                    F.hdr[HDR_L + v] = (uint32_t)L;
                    pe.h = (L + 1) / 2;
                    const int nk = 2 * pe.h + 1;
                    pe.cls = nk <= 256 ? 0 : (nk <= 1024 ? 1 : 2);   // kClassCap
                    uint32_t c = __ldcg(&F.hdr[HDR_COUNT + v]);
                    if ((int64_t)c > F.cap) c = (uint32_t)F.cap;
                    pe.count = c;
                    cnt[0] = c;
                    cnt[1 + pe.cls] = c;
                }
            }
            st_all |= st;
            a.plan[i] = pe;
        }
        // Block-wide exclusive scans of the four count vectors.
        uint32_t incl[1 + kNumClasses];
#pragma unroll
        for (int c = 0; c <= kNumClasses; c++) {
            uint32_t x = cnt[c];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, x, off);
                if (lane >= off) x += y;
            }
            incl[c] = x;
            if (lane == 31) s_warp[warp][c] = x;
        }
        __syncthreads();
        if (threadIdx.x < 1 + kNumClasses) {
            const int c = threadIdx.x;
            uint32_t run = s_carry[c];
            for (int w = 0; w < T / 32; w++) {
                const uint32_t t = s_warp[w][c];
                s_warp[w][c] = run;
                run += t;
            }
            s_carry[c] = run;
        }
        __syncthreads();
        if (i < n) {
            const int stride = n + 1;
            a.pref_all[i] = s_warp[warp][0] + incl[0] - cnt[0];
#pragma unroll
            for (int c = 0; c < kNumClasses; c++) a.pref_cls[c * stride + i] = s_warp[warp][1 + c] + incl[1 + c] - cnt[1 + c];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int stride = n + 1;
        a.pref_all[n] = s_carry[0];
        for (int c = 0; c < kNumClasses; c++) a.pref_cls[c * stride + n] = s_carry[1 + c];
    }
    st_all = __reduce_or_sync(kFull, st_all);
    if (lane == 0 && st_all) atomicOr(a.status, st_all);
}

__global__ void __launch_bounds__(kPlanThreads) k_plan(const __grid_constant__ Args a)
{
    plan_block<kPlanThreads>(a, a.frames);
}

// k_minmax: the min/max of D (Eq. 3) and the non-finite check, one read of D, four pixels per thread and step, for
// calls with no candidate-list view and no E, A or tile hit outputs; the block that finishes last (a releasing count
// over the grid) writes the plan, as k_plan would.  kParam: the frame records come in the launch parameters (calls of
// at most kFramesPerChunk frames), and block (0, 0) also writes them to the frame table, as k_frames would.
template <bool kParam>
__global__ void __launch_bounds__(kMinMaxThreads) k_minmax(const __grid_constant__ Args a,
                                                           const __grid_constant__ FrameChunk c)
{
    __shared__ float s_lo[kMinMaxThreads / 32], s_hi[kMinMaxThreads / 32];
    __shared__ int s_bad, s_last;
    const FrameArg* frames = kParam ? c.f : a.frames;
    if (kParam && blockIdx.x == 0 && blockIdx.y == 0)
        for (int i = threadIdx.x; i < c.count; i += kMinMaxThreads) c.dst[c.first + i] = c.f[i];
    const FrameArg& F = frames[blockIdx.y];
    const int W = F.W, H = F.H;
    const float* const Dp = F.D;
    const int64_t pitch = F.pitch;
    const int QW = (W + 3) >> 2;
    const int64_t nq = (int64_t)H * QW;
    const bool vec = ((pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(Dp) & 15) == 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_bad = 0;
    float lo = INFINITY, hi = -INFINITY;
    bool bad = false;
    for (int64_t q = (int64_t)blockIdx.x * kMinMaxThreads + threadIdx.x; q < nq; q += (int64_t)gridDim.x * kMinMaxThreads)
        minmax_quad(Dp, pitch, W, QW, vec, q, lo, hi, bad);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(kFull, lo, off));
        hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, off));
    }
    __syncthreads();
    if (__any_sync(kFull, bad) && lane == 0) s_bad = 1;
    if (lane == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float blo = INFINITY, bhi = -INFINITY;
        for (int w = 0; w < kMinMaxThreads / 32; w++) {
            blo = fminf(blo, s_lo[w]);
            bhi = fmaxf(bhi, s_hi[w]);
        }
        if (blo <= bhi) {
            atomicMax(&F.hdr[HDR_MAX], f2ord(bhi));
            atomicMax(&F.hdr[HDR_NEGMIN], ~f2ord(blo));
        }
        if (s_bad) atomicOr(&F.hdr[HDR_STATUS], ST_NONFINITE);
        __threadfence();
        s_last = atomicAdd(a.status + CTR_MINMAX, 1u) + 1 == gridDim.x * gridDim.y;
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last) plan_block<kMinMaxThreads>(a, frames);
}

// The (frame, view) index of a scan work item: the last i with pref[i] <= item (pref non-decreasing, pref[0] = 0,
// item < pref[n]).
__device__ __forceinline__ int item_owner(const uint32_t* pref, int n, uint32_t item)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (__ldg(pref + m) <= item) lo = m; else hi = m - 1;
    }
    return lo;
}


// ------------------------------------------------------------------------------------------------------------------
// k_tables: per view and g = -kTabHalf .. kTabHalf, the offsets round(fl(cos a * g)) and round(fl(sin a * g)) of
// the scan line's pixel from the candidate.  For a candidate at integer x, round(fl(fl(cos a * g) + x)) equals
// x + round(fl(cos a * g)) unless fl(cos a * g) lies within half an ulp of x + fl(cos a * g) from a half-integer:
// that ulp is at most 2^-7 for the coordinates this library accepts (x < 2^16, |g| <= 2047), so entries whose
// fraction lies within 2^-8 of 0.5 are marked kTabExact and computed without the table.


__global__ void __launch_bounds__(256) k_tables(const __grid_constant__ Args a)
{
    const int64_t total = (int64_t)a.nv * kTabLen;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < total; i += (int64_t)gridDim.x * 256)
        tables_entry(a, i);
}

// ------------------------------------------------------------------------------------------------------------------
// k_scan_lines, k_merge_lines: Eq. 4 - Eq. 6 with one thread per candidate, for N <= 2 * kLineMaxHalf.
//
// A one-slot buffer that always emits the smaller of the buffered and the arriving sample turns a sequence into
// sorted order exactly when no sample has to move back by more than one place -- the usual effect of noise, which
// lowers a W just below its predecessor's.  A scan line that crosses an edge breaks into a few such stretches
// ("macro-runs"): where a whole run of foreground samples falls behind the background, the buffer's output would go
// backwards, and a new macro-run starts there.  About three lines in four are one macro-run.
//   k_scan_lines (every candidate of a batch): the k range inside the image by bisection, then one pass that takes
//     the line to be one macro-run: positions, gather of V, W = g - V (Eq. 4 and the warp), the one-slot buffer,
//     and for every emitted sample the test (Eq. 5) against the N/2 samples emitted just before it, kept in registers
//     with their running counts, each pair once for both of its ends; a sample whose N/2 successors have all been
//     emitted is final and its count goes to O (Eq. 6).  A line whose output would go backwards stops there and is
//     listed.
//     The lane then looks for a third macro-run in the rest of the line, without counting, in the steps it would
//     otherwise wait for the rest of its warp; lines of more than two macro-runs are flagged for the warp kernel.
//   k_merge_lines (listed lines): the same stream with negated counts up to the same point takes the partial counts
//     back; a line of two macro-runs also goes, as a separate work item, through two one-slot buffers merged by
//     (W, k).

constexpr int kLineThreads = 256;

struct LineSample {
    float w, v;
    int p, k;
};

struct LineJob {
    int x, y;       // candidate
    int f, v;       // frame, view
    int idx;        // index in the (frame, view) candidate list
    int h;          // half scan length
    int k0, k1;     // first / last k inside the image
    int ks;         // start of the second macro-run
};

// Sample k of a line; `bounded` = false when k is known to lie inside the image.
template <bool kWide>
__device__ __forceinline__ bool line_sample(const Args& a, const FrameArg& F, const ViewArg& va, const int32_t* tab, int cx, int cy,
                                            int h, int k, bool bounded, LineSample& out)
{
    const int t = tab[k - h + kTabHalf];
    int px, py;
    const float g = (float)(k - h);
    if (t != kTabExact) {
        px = cx + (int)(int16_t)(t & 0xFFFF);
        py = cy + (t >> 16);
    } else {
        const float rx = roundf(__fadd_rn(__fmul_rn(va.c, g), (float)cx));
        const float ry = roundf(__fadd_rn(__fmul_rn(va.s, g), (float)cy));
        if (bounded && !((rx >= 0.0f) && (rx < (float)F.W) && (ry >= 0.0f) && (ry < (float)F.H))) return false;
        px = (int)rx;
        py = (int)ry;
    }
    if (bounded && !((unsigned)px < (unsigned)F.W && (unsigned)py < (unsigned)F.H)) return false;
    const float dv = kWide ? __ldg(F.D + (int64_t)py * F.pitch + px) : __ldg(F.D + (py * (int)F.pitch + px));
    out.v = (va.r == 1.0f) ? dv : __fmul_rn(va.r, dv);
    out.w = __fsub_rn(g, out.v);
    out.p = py * F.W + px;
    out.k = k;
    return true;
}

// Pixel index and element offset in D of sample k (inside the image) from its table word t; Wd and pitch are the
// frame's width and row pitch, held by the caller (a field of the frame record in global memory would be read again
// after every atomic add to O, which might alias it).
template <bool kWide>
__device__ __forceinline__ void line_pos(int Wd, int64_t pitch, const ViewArg& va, int cx, int cy, int h, int t, int k,
                                         int& pix, int64_t& off)
{
    int px, py;
    if (t != kTabExact) {
        px = cx + (int)(int16_t)(t & 0xFFFF);
        py = cy + (t >> 16);
    } else {
        const float g = (float)(k - h);
        px = (int)roundf(__fadd_rn(__fmul_rn(va.c, g), (float)cx));
        py = (int)roundf(__fadd_rn(__fmul_rn(va.s, g), (float)cy));
    }
    pix = py * Wd + px;
    off = kWide ? (int64_t)py * pitch + px : (int64_t)(py * (int)pitch + px);
}

// The sort key is (W, k).  A sample read later along a line has the larger k, so it precedes an earlier one exactly
// when its W is smaller; a sample of the first macro-run has a smaller k than every sample of the second, so it
// precedes one of the second exactly when its W is not larger.
__device__ __forceinline__ bool later_before(const LineSample& later, const LineSample& earlier)
{
    return later.w < earlier.w;
}

__device__ __forceinline__ bool first_run_before(const LineSample& a, const LineSample& b)
{
    return a.w <= b.w;
}

// Eq. 5 / Eq. 6 over the emitted (sorted) stream: a window of the last N/2 samples, slot 0 the most recent.
struct LineWindow {
    float w0, w1, w2, w3, v0, v1, v2, v3, b0, b1, b2, b3;
    int p0, p1, p2, p3, o0, o1, o2, o3;
    int wn;
    int hit;   // a non-zero count went to O
};

__device__ __forceinline__ void window_init(LineWindow& W)
{
    W.w0 = W.w1 = W.w2 = W.w3 = 0.f;
    W.v0 = W.v1 = W.v2 = W.v3 = 0.f;
    W.b0 = W.b1 = W.b2 = W.b3 = 0.f;
    W.p0 = W.p1 = W.p2 = W.p3 = 0;
    W.o0 = W.o1 = W.o2 = W.o3 = 0;
    W.wn = 0;
    W.hit = 0;
}

template <bool kHits>
__device__ __forceinline__ void window_push(LineWindow& W, const LineSample& e, int half, float zeta, float beta,
                                            int32_t* Ov, int sgn = 1)
{
    const float eb = __fadd_rn(e.v, beta);
    int eo = 0;
#define OCC_PAIR(J)                                                                                 \
    if (J < half && W.wn > J) {                                                                     \
        const bool close = fabsf(__fsub_rn(e.w, W.w##J)) < zeta;                                    \
        eo += (close && eb < W.v##J) ? 1 : 0;                                                       \
        W.o##J += (close && W.b##J < e.v) ? 1 : 0;                                                  \
    }
    OCC_PAIR(0) OCC_PAIR(1) OCC_PAIR(2) OCC_PAIR(3)
#undef OCC_PAIR
    // The oldest sample leaves the window once N/2 samples follow it: its count is final.
    if (W.wn == half) {
        const int ol = half == 1 ? W.o0 : (half == 2 ? W.o1 : (half == 3 ? W.o2 : W.o3));
        const int pl = half == 1 ? W.p0 : (half == 2 ? W.p1 : (half == 3 ? W.p2 : W.p3));
        if (ol) {
            atomicAdd(Ov + pl, sgn * ol);
            if (kHits) W.hit = 1;
        }
    } else {
        W.wn++;
    }
    W.w3 = W.w2; W.v3 = W.v2; W.b3 = W.b2; W.p3 = W.p2; W.o3 = W.o2;
    W.w2 = W.w1; W.v2 = W.v1; W.b2 = W.b1; W.p2 = W.p1; W.o2 = W.o1;
    W.w1 = W.w0; W.v1 = W.v0; W.b1 = W.b0; W.p1 = W.p0; W.o1 = W.o0;
    W.w0 = e.w; W.v0 = e.v; W.b0 = eb; W.p0 = e.p; W.o0 = eo;
}

// Returns whether the line added any non-zero count to O.
__device__ __forceinline__ bool window_flush(const LineWindow& W, int32_t* Ov)
{
    const bool h0 = W.wn > 0 && W.o0, h1 = W.wn > 1 && W.o1, h2 = W.wn > 2 && W.o2, h3 = W.wn > 3 && W.o3;
    if (h0) atomicAdd(Ov + W.p0, W.o0);
    if (h1) atomicAdd(Ov + W.p1, W.o1);
    if (h2) atomicAdd(Ov + W.p2, W.o2);
    if (h3) atomicAdd(Ov + W.p3, W.o3);
    return (W.hit != 0) || h0 || h1 || h2 || h3;
}

// The same window for N = 8 without moving samples between slots: the stream's i-th sample goes to slot i mod 4,
// which held sample i - 4 (the oldest, whose count is final once tested against the new one).  Callers unroll their
// loops by 4 so that every slot index is a compile-time constant; empty slots hold W = +inf, which no sample is close
// to, so the first samples need no count of the window's fill.
struct RotWindow {
    float w[4], v[4], b[4];
    int p[4], o[4];
};

__device__ __forceinline__ void rot_init(RotWindow& R)
{
#pragma unroll
    for (int i = 0; i < 4; i++) {
        R.w[i] = __int_as_float(0x7f800000);
        R.v[i] = R.b[i] = 0.0f;
        R.p[i] = R.o[i] = 0;
    }
}

template <int J, bool kHits>
__device__ __forceinline__ void rot_push(RotWindow& R, const LineSample& e, float zeta, float beta, int32_t* Ov,
                                         int& hit, int sgn = 1)
{
    const float eb = __fadd_rn(e.v, beta);
    int eo = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const bool close = fabsf(__fsub_rn(e.w, R.w[i])) < zeta;
        eo += (close && eb < R.v[i]) ? 1 : 0;
        R.o[i] += (close && R.b[i] < e.v) ? 1 : 0;
    }
    o_red(Ov + R.p[J], sgn * R.o[J]);
    if (kHits) hit |= R.o[J];
    R.w[J] = e.w;
    R.v[J] = e.v;
    R.b[J] = eb;
    R.p[J] = e.p;
    R.o[J] = eo;
}

__device__ __forceinline__ bool rot_flush(const RotWindow& R, int32_t* Ov, int hit)
{
#pragma unroll
    for (int i = 0; i < 4; i++) {
        o_red(Ov + R.p[i], R.o[i]);
        hit |= R.o[i];
    }
    return hit != 0;
}

// A line of two macro-runs [k0, ks - 1] and [ks, k1], each read through its own one-slot buffer; the merge emits
// the smaller head, and the chosen run reads at most one sample per step.
template <bool kWide, bool kHits, bool kHalf4>
__device__ __forceinline__ bool line_counts2(const Args& a, const FrameArg& F, const ViewArg& va, const int32_t* tab, int32_t* Ov, int cx,
                                             int cy, int h, int half, int k0, int k1, int ks)
{
    LineWindow Wn;
    window_init(Wn);
    // Run A: next k, last k, buffer, head; run B likewise.
    int kna = k0 + 1, knb = ks + 1;
    const int ea = ks - 1, eb = k1;
    LineSample bufa, bufb, ha, hb, s;
    bool hba = true, hbb = true;
    line_sample<kWide>(a, F, va, tab, cx, cy, h, k0, false, bufa);
    line_sample<kWide>(a, F, va, tab, cx, cy, h, ks, false, bufb);
    bool has_a = true, has_b = true;
    // First heads.
    if (kna <= ea) {
        line_sample<kWide>(a, F, va, tab, cx, cy, h, kna++, false, s);
        if (later_before(s, bufa)) ha = s; else { ha = bufa; bufa = s; }
    } else {
        ha = bufa;
        hba = false;
    }
    if (knb <= eb) {
        line_sample<kWide>(a, F, va, tab, cx, cy, h, knb++, false, s);
        if (later_before(s, bufb)) hb = s; else { hb = bufb; bufb = s; }
    } else {
        hb = bufb;
        hbb = false;
    }
    // Each run's next sample (k = kn) is loaded ahead: its D value and pixel, used when the run next advances.
    const int* tk = tab + (kTabHalf - h);
    float da = 0.0f, db = 0.0f;
    int pa = 0, pb = 0;
    auto load = [&](int k, float& d, int& p) {
        int64_t off;
        line_pos<kWide>(F.W, F.pitch, va, cx, cy, h, tk[k], k, p, off);
        d = __ldg(F.D + off);
    };
    if (kna <= ea) load(kna, da, pa);
    if (knb <= eb) load(knb, db, pb);
    // One merge step: the smaller head is emitted, its run advances by one sample through its buffer.
#define OCC_MERGE_STEP(PUSH)                                                                   \
    {                                                                                          \
        const bool ta = has_a && (!has_b || first_run_before(ha, hb));                         \
        const LineSample e = ta ? ha : hb;                                                     \
        int kn = ta ? kna : knb;                                                               \
        const int ke = ta ? ea : eb;                                                           \
        bool hbuf = ta ? hba : hbb;                                                            \
        LineSample buf = ta ? bufa : bufb;                                                     \
        float d = ta ? da : db;                                                                \
        int p = ta ? pa : pb;                                                                  \
        LineSample head = buf;                                                                 \
        bool has = false;                                                                      \
        if (kn <= ke) {                                                                        \
            s.v = (va.r == 1.0f) ? d : __fmul_rn(va.r, d);                                     \
            s.w = __fsub_rn((float)(kn - h), s.v);                                             \
            s.p = p;                                                                           \
            s.k = kn;                                                                          \
            kn++;                                                                              \
            if (kn <= ke) load(kn, d, p);                                                      \
            const bool sb = later_before(s, buf);                                              \
            head = sb ? s : buf;                                                               \
            if (!sb) buf = s;                                                                  \
            has = true;                                                                        \
        } else if (hbuf) {                                                                     \
            hbuf = false;                                                                      \
            has = true;                                                                        \
        }                                                                                      \
        if (ta) { kna = kn; hba = hbuf; bufa = buf; ha = head; has_a = has; da = d; pa = p; }  \
        else { knb = kn; hbb = hbuf; bufb = buf; hb = head; has_b = has; db = d; pb = p; }     \
        PUSH;                                                                                  \
    }
    if constexpr (kHalf4) {
        RotWindow R;
        rot_init(R);
        int hit = 0;
        for (;;) {
            if (!(has_a || has_b)) break;
            OCC_MERGE_STEP((rot_push<0, kHits>(R, e, a.zeta, a.beta, Ov, hit)))
            if (!(has_a || has_b)) break;
            OCC_MERGE_STEP((rot_push<1, kHits>(R, e, a.zeta, a.beta, Ov, hit)))
            if (!(has_a || has_b)) break;
            OCC_MERGE_STEP((rot_push<2, kHits>(R, e, a.zeta, a.beta, Ov, hit)))
            if (!(has_a || has_b)) break;
            OCC_MERGE_STEP((rot_push<3, kHits>(R, e, a.zeta, a.beta, Ov, hit)))
        }
        return rot_flush(R, Ov, hit);
    } else {
        while (has_a || has_b) OCC_MERGE_STEP((window_push<kHits>(Wn, e, half, a.zeta, a.beta, Ov)))
        return window_flush(Wn, Ov);
    }
#undef OCC_MERGE_STEP
}

// First and last k of a scan line inside the image.  Each coordinate of a sample is a rounding of a monotone
// function of g, so the samples inside the image form one interval of k, which holds k = h (the candidate itself);
// its ends are found by bisection on both sides of h.
__device__ __forceinline__ void line_range(const FrameArg& F, const ViewArg& va, const int32_t* tab, int cx, int cy,
                                           int h, int& k0, int& k1)
{
    const int* tk = tab + (kTabHalf - h);
    auto inside = [&](int k) -> bool {
        const int t = tk[k];
        if (t == kTabExact) {
            const float g = (float)(k - h);
            const float rx = roundf(__fadd_rn(__fmul_rn(va.c, g), (float)cx));
            const float ry = roundf(__fadd_rn(__fmul_rn(va.s, g), (float)cy));
            return (rx >= 0.0f) && (rx < (float)F.W) && (ry >= 0.0f) && (ry < (float)F.H);
        }
        const int px = cx + (int)(int16_t)(t & 0xFFFF), py = cy + (t >> 16);
        return (unsigned)px < (unsigned)F.W && (unsigned)py < (unsigned)F.H;
    };
    int lo0 = 0, hi0 = h;           // k0 lies in [lo0, hi0]
    int lo1 = h, hi1 = 2 * h;       // k1 lies in [lo1, hi1]
    if (inside(0)) hi0 = 0;
    if (inside(2 * h)) lo1 = 2 * h;
    while (lo0 < hi0 || lo1 < hi1) {
        if (lo0 < hi0) {
            const int m = (lo0 + hi0) >> 1;
            if (inside(m)) hi0 = m; else lo0 = m + 1;
        }
        if (lo1 < hi1) {
            const int m = (lo1 + hi1 + 1) >> 1;
            if (inside(m)) lo1 = m; else hi1 = m - 1;
        }
    }
    k0 = lo0;
    k1 = lo1;
}


// One pass over a line that takes it to be a single macro-run: samples k0 .. k1 through the one-slot buffer, each
// emitted sample tested (Eq. 5) against the N/2 emitted before it, final counts to O (Eq. 6).  Every lane of the warp
// calls it (live = false: no line).  The emitted stream must not go backwards; where it would (the sample about to
// be emitted precedes the last one emitted), a second macro-run starts there, and the function returns that k with
// the line's counts so far still in O.  Until the rest of the warp is done the lane goes on through the remaining
// samples without counting (zeta < 0: no pair is close, Eq. 5) to see whether a third macro-run starts (more).
// Returns -1 when the line was one macro-run (hit: a non-zero count went to O).  With sgn = -1 every count is
// negated and the stream stops at the first break: the same pushes again take a broken line's counts back out of O.
//
// The stream is padded so that every lane pushes from its first step and loads one sample ahead from the start: the
// buffer starts with a sample of W = -inf and the first "current" sample is another (V = +inf); after k1 the
// current sample has W = +inf, which flushes the buffer.  Samples of infinite W are never close (Eq. 5) to any
// other, so they leave no count, and the n samples of the line take n + 2 pushes.
template <bool kWide, bool kHits, bool kHalf4>
__device__ __forceinline__ int line_stream(const Args& a, const FrameArg& F, const ViewArg& va, const int32_t* tab,
                                           int32_t* Ov, int cx, int cy, int h, int half, int k0, int k1, bool live,
                                           int sgn, bool& hit, bool& more)
{
    const float kInf = __int_as_float(0x7f800000);
    const int* tk = tab + (kTabHalf - h);
    const float* const Dp = F.D;
    const int64_t pitch = F.pitch;
    const int Wd = F.W;
    const float r = va.r;
    RotWindow R;
    LineWindow Wn;
    LineSample buf;
    float lastw, dn, gq;
    int pn, tnext = 0, kq, left = 0, ht = 0;
    int64_t on;
    bool go = live;
    // zeta of the pair test (Eq. 5).  At the first break it becomes -(ks + 1): no pair is close any more, and the
    // k where the second macro-run starts is kept without a register of its own.
    float zl = a.zeta;
    more = false;
    if (live) {
        if constexpr (kHalf4) rot_init(R); else window_init(Wn);
        buf.w = -kInf;
        buf.v = kInf;
        buf.p = 0;
        buf.k = 0;
        lastw = -kInf;
        pn = 0;
        dn = kInf;
        kq = k0 - 1;
        gq = (float)(k0 - 1 - h);
        tnext = tk[k0];
        left = k1 - k0 + 3;
    }
    // One step: the sample in flight becomes current, the next one is loaded; the smaller of current and buffer is
    // emitted unless that would go backwards.
#define OCC_STREAM_STEP(PUSH)                                                                  \
    if (go) {                                                                                  \
        const int p = pn;                                                                      \
        const float dv = dn;                                                                   \
        if (kq < k1) {                                                                         \
            const int t = tnext;                                                               \
            tnext = tk[min(kq + 2, k1)];                                                       \
            line_pos<kWide>(Wd, pitch, va, cx, cy, h, t, kq + 1, pn, on);                      \
            dn = __ldg(Dp + on);                                                               \
        } else {                                                                               \
            dn = -kInf;                                                                        \
        }                                                                                      \
        LineSample s;                                                                          \
        s.v = (r == 1.0f) ? dv : __fmul_rn(r, dv);                                             \
        s.w = __fsub_rn(gq, s.v);                                                              \
        s.p = p;                                                                               \
        s.k = 0;                                                                               \
        const bool sb = later_before(s, buf);                                                  \
        if (sb && s.w < lastw) {                                                               \
            if (zl < 0.0f) {                                                                   \
                go = false;                                                                    \
                more = true;                                                                   \
            } else {                                                                           \
                zl = -(float)(kq + 1);                                                         \
                if (sgn > 0) {                                                                 \
                    if constexpr (kHalf4) { R.o[0] = R.o[1] = R.o[2] = R.o[3] = 0; }           \
                    else { Wn.o0 = Wn.o1 = Wn.o2 = Wn.o3 = 0; }                                \
                    buf = s;                                                                   \
                    lastw = -kInf;                                                             \
                } else {                                                                       \
                    go = false;                                                                \
                }                                                                              \
            }                                                                                  \
        } else {                                                                               \
            const LineSample e = sb ? s : buf;                                                 \
            if (!sb) buf = s;                                                                  \
            PUSH;                                                                              \
            lastw = e.w;                                                                       \
            go = --left != 0;                                                                  \
        }                                                                                      \
        kq++;                                                                                  \
        gq += 1.0f;                                                                            \
    }
    for (;;) {
        if (!__any_sync(kFull, go)) break;
        if constexpr (kHalf4) {
            OCC_STREAM_STEP((rot_push<0, kHits>(R, e, zl, a.beta, Ov, ht, sgn)))
            OCC_STREAM_STEP((rot_push<1, kHits>(R, e, zl, a.beta, Ov, ht, sgn)))
            OCC_STREAM_STEP((rot_push<2, kHits>(R, e, zl, a.beta, Ov, ht, sgn)))
            OCC_STREAM_STEP((rot_push<3, kHits>(R, e, zl, a.beta, Ov, ht, sgn)))
        } else {
            OCC_STREAM_STEP((window_push<kHits>(Wn, e, half, zl, a.beta, Ov, sgn)))
            OCC_STREAM_STEP((window_push<kHits>(Wn, e, half, zl, a.beta, Ov, sgn)))
        }
    }
#undef OCC_STREAM_STEP
    if (!live) return -1;
    if (zl < 0.0f) return (int)(-zl) - 1;
    if constexpr (kHalf4) hit = rot_flush(R, Ov, ht);
    else hit = window_flush(Wn, Ov);
    return -1;
}

constexpr int kStatsSmem = 512;   // (frame, view) statistics accumulated in shared memory before going global

// Per-(frame, view) statistics of the lines a block completes: accumulated per thread while its lines stay in one
// (frame, view), then in shared memory, then once per block in global memory.
struct LineStats {
    unsigned long long* s_st;
    int cur = -1;
    unsigned long long acc_n = 0, acc_p = 0;

    __device__ void flush(const Args& a)
    {
        if (cur < 0) return;
        if (cur < kStatsSmem) {
            atomicAdd(&s_st[2 * cur], acc_n);
            atomicAdd(&s_st[2 * cur + 1], acc_p);
        } else {
            const int f = cur / a.nv, v = cur - f * a.nv;
            atomicAdd(&a.frames[f].stats[2 * v], acc_n);
            atomicAdd(&a.frames[f].stats[2 * v + 1], acc_p);
        }
    }
    __device__ void add(const Args& a, int i, int n, int half)
    {
        if (i != cur) {
            flush(a);
            cur = i;
            acc_n = acc_p = 0;
        }
        acc_n += (unsigned long long)n;
        acc_p += pair_count(n, half);
    }
};

__device__ __forceinline__ void stats_init(unsigned long long* s_st)
{
    for (int i = threadIdx.x; i < 2 * kStatsSmem; i += blockDim.x) s_st[i] = 0;
    __syncthreads();
}

__device__ __forceinline__ void stats_publish(const Args& a, const unsigned long long* s_st)
{
    __syncthreads();
    const int nfv = a.nf * a.nv;
    const int ns = nfv < kStatsSmem ? nfv : kStatsSmem;
    for (int i = threadIdx.x; i < 2 * ns; i += blockDim.x)
        if (s_st[i]) {
            const int fv = i >> 1, f = fv / a.nv, v = fv - f * a.nv;
            atomicAdd(&a.frames[f].stats[2 * v + (i & 1)], s_st[i]);
        }
}

// A line's candidate, half length and k range inside the image from its work item.
__device__ __forceinline__ LineJob line_job(const Args& a, uint32_t item)
{
    LineJob jb;
    const int nfv = a.nf * a.nv;
    const int i = item_owner(a.pref_all, nfv, item);
    const int f = i / a.nv, v = i - f * a.nv;
    const FrameArg& F = a.frames[f];
    const int64_t idx = (int64_t)(item - a.pref_all[i]);
    const uint32_t cw = F.cand[(int64_t)v * F.cap + idx];
    jb.x = (int)(cw & 0xFFFFu);
    jb.y = (int)(cw >> 16);
    jb.f = f;
    jb.v = v;
    jb.idx = (int)idx;
    jb.h = a.plan[i].h;
    jb.ks = -1;
    line_range(F, a.view[v], a.ptab + (int64_t)v * kTabLen, jb.x, jb.y, jb.h, jb.k0, jb.k1);
    return jb;
}

__device__ __forceinline__ uint32_t* line_flag_word(const Args& a, const LineJob& jb)
{
    const FrameArg& F = a.frames[jb.f];
    return &F.fb[(int64_t)jb.v * F.fb_words + (jb.idx >> 5)];
}

// kHits: some frame of the batch asks for per-tile hit flags.
__device__ __forceinline__ void line_mark_hit(const FrameArg& F, const LineJob& jb)
{
    if (F.hits) F.hits[(int64_t)jb.v * F.tiles_x * F.tiles_y + (jb.y / kTile) * F.tiles_x + jb.x / kTile] = 1;
}

// The replay of a broken line's stream with the counts negated (every lane calls it; live: this lane has a line): it
// takes what the line kernel added back out of O, and returns the k where the second macro-run starts.  Kept out of
// line: an inlined copy of the stream next to the merge costs the merge kernel registers.
template <bool kWide, bool kHits, bool kHalf4>
__device__ __noinline__ int line_undo(const Args& a, const LineJob& jb, bool live)
{
    const FrameArg& F = a.frames[jb.f];
    bool hit = false, more = false;
    return line_stream<kWide, kHits, kHalf4>(a, F, a.view[jb.v], a.ptab + (int64_t)jb.v * kTabLen,
                                             F.O + (int64_t)jb.v * F.H * F.W, jb.x, jb.y, jb.h, a.N >> 1, jb.k0, jb.k1,
                                             live, -1, hit, more);
}

// Next chunk of 32 work items of a warp.  Small calls: warp w takes chunks w, w + n_warps, ... (static).  Large calls
// (kDyn): after its first chunk a warp takes the next one from a counter, so that the lines in flight stay within a
// narrow window of the item order (one frame and view at a time) however far warps drift apart, and the D and O
// planes they touch stay in L2 for large frames and long batches.
template <bool kDyn>
__device__ __forceinline__ uint64_t next_chunk(uint64_t chunk, uint64_t nwarps, uint32_t* ctr, int lane)
{
    if constexpr (kDyn) {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(ctr, 1u);
        return nwarps + __shfl_sync(kFull, c, 0);
    } else {
        return chunk + nwarps;
    }
}

template <bool kWide, bool kHits, bool kHalf4, bool kDyn>
__global__ void __launch_bounds__(kLineThreads, 3) k_scan_lines(const __grid_constant__ Args a)
{
    constexpr int kWarps = kLineThreads / 32;
    __shared__ unsigned long long s_st[2 * kStatsSmem];
    stats_init(s_st);
    const uint32_t total = a.pref_all[a.nf * a.nv];
    const int half = a.N >> 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    LineStats stats{s_st};
    const uint64_t nwarps = (uint64_t)gridDim.x * kWarps;
    for (uint64_t chunk = (uint64_t)blockIdx.x * kWarps + warp;;) {
        const uint64_t b0 = chunk * 32;
        if (b0 >= total) break;
        // One line per lane.
        const uint64_t item = b0 + lane;
        const bool live = item < total;
        LineJob jb{0, 0, 0, 0, 0, 0, 0, 0, -1};
        if (live) jb = line_job(a, (uint32_t)item);
        const FrameArg& F = a.frames[jb.f];
        bool hit = false, more = false;
        const int ks = line_stream<kWide, kHits, kHalf4>(a, F, a.view[jb.v], a.ptab + (int64_t)jb.v * kTabLen,
                                                         F.O + (int64_t)jb.v * F.H * F.W, jb.x, jb.y, jb.h, half,
                                                         jb.k0, jb.k1, live, 1, hit, more);
        if (live && ks < 0) {
            stats.add(a, jb.f * a.nv + jb.v, jb.k1 - jb.k0 + 1, half);
            if (kHits && hit) line_mark_hit(F, jb);
        }
        // More than one macro-run: the line's counts so far are still in O, and it goes to the front of the merge
        // kernel's list, whose replay takes them back out; the list has an entry for every candidate the call can
        // hold, so the front cannot fill up (the check only guards the store).  A line of exactly two macro-runs
        // (when line_max_runs = 2) also takes a pair of entries (item, ks) from the back of the list, in the room the
        // call's candidates leave free, for the two-run merge; every other broken line, and a two-run line that
        // finds no room, is flagged for the warp kernel now.
        const bool broken = live && ks >= 0;
        bool two = broken && !more && a.line_max_runs >= 2;
        const unsigned mb = __ballot_sync(kFull, broken), m2 = __ballot_sync(kFull, two);
        if (mb) {
            // One atomic reserves both: front entries in the low word, pairs in the high one (the front count never
            // exceeds the candidates, so the low word cannot carry).
            unsigned long long base = 0;
            if (lane == 0)
                base = atomicAdd(a.brk_count, ((unsigned long long)__popc(m2) << 32) | (unsigned long long)__popc(mb));
            base = __shfl_sync(kFull, base, 0);
            if (two) {
                const uint32_t j = (uint32_t)(base >> 32) + (uint32_t)__popc(m2 & lt);
                if (j < (a.brk_cap - total) / 2) {
                    a.brk[a.brk_cap - 2 - 2 * j] = (uint32_t)item;
                    a.brk[a.brk_cap - 1 - 2 * j] = (uint32_t)ks;
                } else {
                    two = false;
                }
            }
            if (broken) {
                const uint32_t pos = (uint32_t)base + (uint32_t)__popc(mb & lt);
                if (pos < total) a.brk[pos] = (uint32_t)item;
                else atomicOr(a.status, ST_INTERNAL);
            }
        }
        if (broken && !two) atomicOr(line_flag_word(a, jb), 1u << (jb.idx & 31));
        chunk = next_chunk<kDyn>(chunk, nwarps, a.line_ctr, lane);
    }
    stats.flush(a);
    stats_publish(a, s_st);
}

// k_merge_lines: the lines k_scan_lines listed, one thread per list entry, 32 entries per warp; two kinds of work,
// independent of each other (both only add to O and the statistics), so a line's two jobs can run on different
// warps at the same time.  The pairs at the back of the list come first: the two-buffer merge of a line of exactly two
// macro-runs [k0, ks - 1] and [ks, k1] by (W, k), with Eq. 5 and Eq. 6 as in the stream.  Then the entries at the
// front: the stream of a broken line again with the counts negated, up to the point where it broke, which takes its
// partial counts back out of O.  A warp's first batch is fixed by its index, the next ones come from a counter, so
// that the longer merges do not pile up on the warps that drew two of them.
template <bool kWide, bool kHits, bool kHalf4>
__global__ void __launch_bounds__(kLineThreads, 3) k_merge_lines(const __grid_constant__ Args a)
{
    constexpr int kWarps = kLineThreads / 32;
    __shared__ unsigned long long s_st[2 * kStatsSmem];
    stats_init(s_st);
    const uint32_t total = a.pref_all[a.nf * a.nv];
    const unsigned long long cnt = *a.brk_count;
    const uint32_t nr = min((uint32_t)cnt, total), nm = min((uint32_t)(cnt >> 32), (a.brk_cap - total) / 2);
    const uint64_t nbm = (nm + 31u) / 32u, nb = nbm + (nr + 31u) / 32u;
    const int half = a.N >> 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    LineStats stats{s_st};
    const uint64_t nwarps = (uint64_t)gridDim.x * kWarps;
    for (uint64_t b = (uint64_t)blockIdx.x * kWarps + warp; b < nb; b = next_chunk<true>(b, nwarps, a.merge_ctr, lane)) {
        if (b < nbm) {
            const uint64_t e = b * 32 + lane;
            if (e < nm) {
                LineJob jb = line_job(a, a.brk[a.brk_cap - 2 - 2 * e]);
                jb.ks = (int)a.brk[a.brk_cap - 1 - 2 * e];
                const FrameArg& F = a.frames[jb.f];
                const bool hit = line_counts2<kWide, kHits, kHalf4>(a, F, a.view[jb.v], a.ptab + (int64_t)jb.v * kTabLen,
                                                                    F.O + (int64_t)jb.v * F.H * F.W, jb.x, jb.y, jb.h,
                                                                    half, jb.k0, jb.k1, jb.ks);
                if (kHits && hit) line_mark_hit(F, jb);
                stats.add(a, jb.f * a.nv + jb.v, jb.k1 - jb.k0 + 1, half);
            }
        } else {
            const uint64_t e = (b - nbm) * 32 + lane;
            const bool valid = e < nr;
            LineJob jb{0, 0, 0, 0, 0, 0, 0, 0, -1};
            if (valid) jb = line_job(a, a.brk[e]);
            line_undo<kWide, kHits, kHalf4>(a, jb, valid);
        }
        __syncwarp();
    }
    stats.flush(a);
    stats_publish(a, s_st);
}

// ------------------------------------------------------------------------------------------------------------------
// k_scan: Eq. 4 - Eq. 6 with one warp per candidate, for lines of up to CAP samples; any line, any N (the per-line
// steps are scan_line, occ_scanline.cuh).  When the line-per-thread kernel ran first, only the candidates it flagged
// are processed here.

template <int CAP, int WPB>
__global__ void __launch_bounds__(WPB * 32) k_scan(const __grid_constant__ Args a, int cls)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ScanSmem<CAP>& S = reinterpret_cast<ScanSmem<CAP>*>(smem_raw)[warp];
    const int nfv = a.nf * a.nv;
    // Work items: the candidates of the list-path views in this size class, then the lines k_strip listed for it.
    const uint32_t* pref = a.pref_cls + (int64_t)cls * (nfv + 1);
    const uint32_t* pref1 = a.pref_ovf + (int64_t)cls * (nfv + 1);
    const uint64_t total0 = pref[nfv];
    const uint64_t total = total0 + (a.strip_px ? pref1[nfv] : 0u);
    if (total == 0) return;
    int cur_v = -1;
    unsigned long long acc_n = 0, acc_p = 0;

    // Work distribution: warp w owns the lines w, w + nwarps, w + 2 nwarps, ... (so that lines the line kernel
    // left, which cluster along edges, spread over the warps).  It looks at 32 of them at once, one per lane, finds
    // with one ballot which are its to do (all, or the flagged ones), and walks those.
    const uint64_t gwarp = (uint64_t)blockIdx.x * WPB + warp, nwarps = (uint64_t)gridDim.x * WPB;
    for (uint64_t round = 0;; round++) {
        const uint64_t first = gwarp + round * 32 * nwarps;
        if (first >= total) break;
        const uint64_t mine = first + (uint64_t)lane * nwarps;
        bool want = mine < total;
        int my_i = 0;
        uint32_t my_idx = 0;
        if (want && mine >= total0) {
            const uint32_t m1 = (uint32_t)(mine - total0);
            my_i = item_owner(pref1, nfv, m1);
            my_idx = m1 - pref1[my_i];
        } else if (want) {
            my_i = item_owner(pref, nfv, (uint32_t)mine);
            my_idx = (uint32_t)(mine - pref[my_i]);
            if (a.use_fb) {
                const int mf = my_i / a.nv, mv = my_i - mf * a.nv;
                const FrameArg& MF = a.frames[mf];
                want = (MF.fb[(int64_t)mv * MF.fb_words + (my_idx >> 5)] >> (my_idx & 31)) & 1u;
            }
        }
        unsigned todo = __ballot_sync(kFull, want);
        while (todo) {
        const int jl = __ffs(todo) - 1;
        todo &= todo - 1;
        const int i = __shfl_sync(kFull, my_i, jl);
        const int64_t idx = (int64_t)__shfl_sync(kFull, my_idx, jl);
        const FrameArg& F = a.frames[i / a.nv];
        const uint32_t cw = F.cand[(int64_t)(i % a.nv) * F.cap + idx];
        scan_item<CAP>(a, a.frames, S, lane, i, cw, cur_v, acc_n, acc_p);
        }
    }
    flush_item_stats(a.frames, a.nv, lane, cur_v, acc_n, acc_p);
}

// ------------------------------------------------------------------------------------------------------------------
// k_mask: M = (O > 0), 16 pixels per thread and iteration when aligned.

constexpr int kMaskThreads = 256;

__global__ void __launch_bounds__(kMaskThreads) k_mask(const __grid_constant__ Args a)
{
    const FrameArg& F = a.frames[blockIdx.y];
    const int64_t n = (int64_t)a.nv * F.H * F.W;
    const int64_t stride = (int64_t)gridDim.x * kMaskThreads;
    const int64_t t0 = (int64_t)blockIdx.x * kMaskThreads + threadIdx.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(F.O) & 15) == 0) && ((reinterpret_cast<uintptr_t>(F.M) & 15) == 0);
    int64_t done = 0;
    if (vec) {
        const int64_t n16 = n >> 4;
        const int4* O4 = reinterpret_cast<const int4*>(F.O);
        uint4* M16 = reinterpret_cast<uint4*>(F.M);
        for (int64_t i = t0; i < n16; i += stride) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int4 o = __ldcs(O4 + 4 * i + j);
                w[j] = (uint32_t)(o.x > 0) | ((uint32_t)(o.y > 0) << 8) | ((uint32_t)(o.z > 0) << 16) |
                       ((uint32_t)(o.w > 0) << 24);
            }
            __stcs(M16 + i, make_uint4(w[0], w[1], w[2], w[3]));
        }
        done = n16 << 4;
    }
    for (int64_t i = done + t0; i < n; i += stride) F.M[i] = (uint8_t)(F.O[i] > 0);
}

template <int CAP, int WPB>
constexpr size_t scan_smem()
{
    return sizeof(ScanSmem<CAP>) * WPB;
}

constexpr int kWpb0 = 8, kWpb0s = 4, kWpb1 = 4, kWpb2 = 2;

}  // namespace

cudaError_t configure_kernels(int* lines_bps, int scan_bps[kNumClasses + 1])
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_scan<256, kWpb0s>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)scan_smem<256, kWpb0s>())) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&scan_bps[kNumClasses], k_scan<256, kWpb0s>, kWpb0s * 32,
                                                           scan_smem<256, kWpb0s>())) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_scan<256, kWpb0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)scan_smem<256, kWpb0>())) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_scan<1024, kWpb1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)scan_smem<1024, kWpb1>())) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_scan<4096, kWpb2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)scan_smem<4096, kWpb2>())) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(lines_bps, k_scan_lines<false, false, true, false>, kLineThreads, 0)) !=
        cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&scan_bps[0], k_scan<256, kWpb0>, kWpb0 * 32,
                                                           scan_smem<256, kWpb0>())) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&scan_bps[1], k_scan<1024, kWpb1>, kWpb1 * 32,
                                                           scan_smem<1024, kWpb1>())) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&scan_bps[2], k_scan<4096, kWpb2>, kWpb2 * 32,
                                                         scan_smem<4096, kWpb2>());
}

cudaError_t launch_frames(const FrameChunk& c, cudaStream_t st)
{
    k_frames<<<1, kFramesPerChunk, 0, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_tables(const Args& a, cudaStream_t st)
{
    const int64_t total = (int64_t)a.nv * kTabLen;
    k_tables<<<(int)((total + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_edges(const Args& a, cudaStream_t st)
{
    int bx = (a.max_quads + kEdgeThreads - 1) / kEdgeThreads;
    if (bx > 2048) bx = 2048;
    if (bx < 1) bx = 1;
    k_edges<<<dim3(bx, a.nf), kEdgeThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_minmax(const Args& a, const FrameChunk* c, cudaStream_t st)
{
    int bx = (a.max_quads + kMinMaxThreads - 1) / kMinMaxThreads;
    if (bx > 1024) bx = 1024;
    if (bx < 1) bx = 1;
    if (c) {
        k_minmax<true><<<dim3(bx, a.nf), kMinMaxThreads, 0, st>>>(a, *c);
    } else {
        FrameChunk none;
        std::memset(&none, 0, sizeof(none));
        k_minmax<false><<<dim3(bx, a.nf), kMinMaxThreads, 0, st>>>(a, none);
    }
    return cudaGetLastError();
}

cudaError_t launch_plan(const Args& a, cudaStream_t st)
{
    k_plan<<<1, kPlanThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan_lines(const Args& a, int grid, bool wide, cudaStream_t st)
{
    // N = 8 (the default) takes the rotating window; wide frames and hit flags are the rarer variants; large calls
    // take their chunks from a counter.
    const bool h4 = a.N == 8;
#define OCC_LINES(W, HI, DY)                                                                       \
    do {                                                                                           \
        if (h4) k_scan_lines<W, HI, true, DY><<<grid, kLineThreads, 0, st>>>(a);                   \
        else k_scan_lines<W, HI, false, DY><<<grid, kLineThreads, 0, st>>>(a);                     \
    } while (0)
    if (a.line_dyn) {
        if (!wide && !a.hits) OCC_LINES(false, false, true);
        else if (!wide) OCC_LINES(false, true, true);
        else if (!a.hits) OCC_LINES(true, false, true);
        else OCC_LINES(true, true, true);
    } else {
        if (!wide && !a.hits) OCC_LINES(false, false, false);
        else if (!wide) OCC_LINES(false, true, false);
        else if (!a.hits) OCC_LINES(true, false, false);
        else OCC_LINES(true, true, false);
    }
#undef OCC_LINES
    return cudaGetLastError();
}

cudaError_t launch_merge_lines(const Args& a, int grid, bool wide, cudaStream_t st)
{
    const bool h4 = a.N == 8;
#define OCC_MERGE(W, HI)                                                                           \
    do {                                                                                           \
        if (h4) k_merge_lines<W, HI, true><<<grid, kLineThreads, 0, st>>>(a);                      \
        else k_merge_lines<W, HI, false><<<grid, kLineThreads, 0, st>>>(a);                        \
    } while (0)
    if (!wide && !a.hits) OCC_MERGE(false, false);
    else if (!wide) OCC_MERGE(false, true);
    else if (!a.hits) OCC_MERGE(true, false);
    else OCC_MERGE(true, true);
#undef OCC_MERGE
    return cudaGetLastError();
}

cudaError_t launch_scan(const Args& a, int cls, int grid, cudaStream_t st)
{
    switch (cls) {
    case 0: k_scan<256, kWpb0><<<grid, kWpb0 * 32, scan_smem<256, kWpb0>(), st>>>(a, 0); break;
    case 1: k_scan<1024, kWpb1><<<grid, kWpb1 * 32, scan_smem<1024, kWpb1>(), st>>>(a, 1); break;
    case 2: k_scan<4096, kWpb2><<<grid, kWpb2 * 32, scan_smem<4096, kWpb2>(), st>>>(a, 2); break;
    default: k_scan<256, kWpb0s><<<grid, kWpb0s * 32, scan_smem<256, kWpb0s>(), st>>>(a, 0); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_mask(const Args& a, cudaStream_t st)
{
    int64_t bx = a.max_px / (4096 * 4);
    if (bx > 1024) bx = 1024;
    if (bx < 1) bx = 1;
    k_mask<<<dim3((unsigned)bx, a.nf), kMaskThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace occ
