// occ_scanline.cuh -- Eq. 4 - Eq. 6 for one scan line by one warp, with the sort as a merge of the line's monotone runs
// (or a counting sort for many runs); shared by the warp kernel k_scan (occ_kernels.cu), which takes the lines of the
// candidate lists, and by the strip kernel (occ_strip.cu), which takes its lines of three or more macro-runs.  Every
// floating-point operation that decides a position, an order or a count is an explicit round-to-nearest binary32
// intrinsic; the including files are compiled with --fmad=false.
#pragma once

#include <cstdint>

#include "occ_internal.cuh"

namespace occ {
namespace {

// Sort.  The valid samples split into maximal runs already ordered by (W, k) (a run ends where W drops).  A sample
// of run a precedes, in sorted order, exactly the samples of later runs with smaller W and of earlier runs with W
// not larger than its own; its rank is its index plus the first count minus the number of samples of earlier runs
// with larger W.  Runs whose W range does not straddle the sample's W contribute nothing or everything, so only
// straddling runs need a binary search, and a sample that no other run straddles keeps its index.  A line that is
// one run is already sorted; a line with more than kMaxRuns runs goes through a counting sort by W bucket and
// transposition passes within the buckets.
// Occlusion test (Eq. 5).  Every pair of sorted positions (q, q+d), d <= N/2, is tested once from its lower end:
// |fl(W_q - W_{q+d})| is symmetric, and |dW| grows with d in sorted order, so the pairs found this way are exactly
// the ones the walk of Eq. 5 reaches from either end.  q is hit when V_q + beta < V_{q+d}, and q+d when
// V_{q+d} + beta < V_q; hits on the upper end go to a shared counter.  Eq. 6: the counts are added to O.

constexpr int kMaxRuns = 16;

template <int CAP>
struct ScanSmem {
    float uw[CAP];      // W by k; after the sort, hit counters
    float uv[CAP];      // V by k; after the sort, hit counters
    float sw[CAP];      // sorted W (hit counters when the line is one run; bucket counts during the bucket sort)
    float sv[CAP];      // sorted V (hit counters when the line is one run)
    uint16_t sidx[CAP]; // sample index (k - k0) of each sorted position
    int32_t runs[kMaxRuns + 2];
    float run_lo[kMaxRuns + 1];   // first (smallest) W of each run
    float run_hi[kMaxRuns + 1];   // last (largest) W of each run
    float lo_after[kMaxRuns + 2]; // min of run_lo over the runs after run b
    float hi_before[kMaxRuns + 2];// max of run_hi over the runs before run b
};

// First index in [lo, hi) whose value is > x (upper) or >= x (lower); a[lo..hi) is non-decreasing.
__device__ __forceinline__ int upper_bound_f(const float* a, int lo, int hi, float x)
{
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (a[m] <= x) lo = m + 1; else hi = m;
    }
    return lo;
}
__device__ __forceinline__ int lower_bound_f(const float* a, int lo, int hi, float x)
{
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (a[m] < x) lo = m + 1; else hi = m;
    }
    return lo;
}

// One scan line (Eq. 4) through the candidate at (fcx, fcy) of a map D (row pitch `pitch`, W x H), direction (c, s),
// ratio r, half length h; the warp W = g - V, the sort by (W, k) and the test of Eq. 5 with N = 2 half neighbours.
// emit(k, o) is called once for every sample k (0 .. 2h) with o > 0 hits, by the lane that holds it; the caller adds
// o to O at the sample's pixel (Eq. 6).  Returns the number of samples inside the map, 0 for none, and -1 when they
// do not form one interval of k (a self-check; positions are monotone in g).  Uses the warp's ScanSmem; lines of at
// most CAP samples (2h + 1 <= CAP).
template <int CAP, class Emit>
__device__ __forceinline__ int scan_line(ScanSmem<CAP>& S, int lane, const float* D, int64_t pitch, int Wd, int Hd,
                                         float c, float s, float r, float fcx, float fcy, int h, int half, float beta,
                                         float zeta, Emit&& emit)
{
    constexpr unsigned kFull = 0xFFFFFFFFu;
    const unsigned lt = (1u << lane) - 1u;
    const bool one = (r == 1.0f);
    const int nk = 2 * h + 1;
    const float fW = (float)Wd, fH = (float)Hd;

    // Eq. 4: positions, bounds, V = D_r at the nearest pixel, W = g - V.
    int k0 = -1, kl = -1, n = 0;
    auto record = [&](int base, bool ok) {
        const unsigned b = __ballot_sync(kFull, ok);
        if (b) {
            if (k0 < 0) k0 = base + __ffs(b) - 1;
            kl = base + 31 - __clz(b);
            n += __popc(b);
        }
    };
    if constexpr (CAP <= 256) {
        // Every lane's gathers (at most CAP / 32) are issued before any is used.
        constexpr int kSl = CAP / 32;
        float dvs[kSl];
        bool oks[kSl];
#pragma unroll
        for (int i = 0; i < kSl; i++) {
            const int k = i * 32 + lane;
            oks[i] = false;
            dvs[i] = 0.0f;
            if (k < nk) {
                const float g = (float)(k - h);
                const float rx = roundf(__fadd_rn(__fmul_rn(c, g), fcx));
                const float ry = roundf(__fadd_rn(__fmul_rn(s, g), fcy));
                oks[i] = (rx >= 0.0f) && (rx < fW) && (ry >= 0.0f) && (ry < fH);
                if (oks[i]) dvs[i] = __ldg(D + (int64_t)(int)ry * pitch + (int)rx);
            }
        }
#pragma unroll
        for (int i = 0; i < kSl; i++) {
            const int base = i * 32;
            if (base >= nk) break;
            const int k = base + lane;
            if (oks[i]) {
                const float V = one ? dvs[i] : __fmul_rn(r, dvs[i]);
                S.uw[k] = __fsub_rn((float)(k - h), V);
                S.uv[k] = V;
            }
            record(base, oks[i]);
        }
    } else {
        for (int base = 0; base < nk; base += 32) {
            const int k = base + lane;
            bool ok = false;
            if (k < nk) {
                const float g = (float)(k - h);
                const float rx = roundf(__fadd_rn(__fmul_rn(c, g), fcx));
                const float ry = roundf(__fadd_rn(__fmul_rn(s, g), fcy));
                ok = (rx >= 0.0f) && (rx < fW) && (ry >= 0.0f) && (ry < fH);
                if (ok) {
                    const float dv = __ldg(D + (int64_t)(int)ry * pitch + (int)rx);
                    const float V = one ? dv : __fmul_rn(r, dv);
                    S.uw[k] = __fsub_rn(g, V);
                    S.uv[k] = V;
                }
            }
            record(base, ok);
        }
    }
    // The samples inside the image form one interval of k (positions are monotone in g).
    if (n == 0 || kl - k0 + 1 != n) {
        __syncwarp();
        return n == 0 ? 0 : -1;
    }
    __syncwarp();
    const float* uw = S.uw + k0;
    const float* uv = S.uv + k0;

    // Runs: a new run starts after every descent W[i+1] < W[i].
    int R = 1;
    for (int base = 0; base < n - 1; base += 32) {
        const int i = base + lane;
        const bool dsc = (i < n - 1) && (uw[i + 1] < uw[i]);
        const unsigned b = __ballot_sync(kFull, dsc);
        if (dsc) {
            const int slot = R + __popc(b & lt);
            if (slot <= kMaxRuns) S.runs[slot] = i + 1;
        }
        R += __popc(b);
    }

    const float* sw;
    const float* sv;
    int* cnt_own;
    int* cnt_up;
    if (R == 1) {
        sw = uw; sv = uv;
        cnt_own = reinterpret_cast<int*>(S.sv);
        cnt_up = reinterpret_cast<int*>(S.sw);
    } else {
        sw = S.sw; sv = S.sv;
        cnt_own = reinterpret_cast<int*>(S.uv);
        cnt_up = reinterpret_cast<int*>(S.uw);
        if (R <= kMaxRuns) {
            if (lane == 0) {
                S.runs[0] = 0;
                S.runs[R] = n;
            }
            __syncwarp();
            if (lane < R) {
                S.run_lo[lane] = uw[S.runs[lane]];
                S.run_hi[lane] = uw[S.runs[lane + 1] - 1];
            }
            __syncwarp();
            if (lane == 0) {
                float m = INFINITY;
                S.lo_after[R] = m;
                for (int b = R - 1; b >= 0; b--) {
                    S.lo_after[b] = m;            // min run_lo over runs b+1 .. R-1
                    m = fminf(m, S.run_lo[b]);
                }
                float x = -INFINITY;
                for (int b = 0; b < R; b++) {
                    S.hi_before[b] = x;           // max run_hi over runs 0 .. b-1
                    x = fmaxf(x, S.run_hi[b]);
                }
            }
            __syncwarp();
            for (int i = lane; i < n; i += 32) {
                const float wi = uw[i];
                int ra = 0;
                while (ra + 1 < R && S.runs[ra + 1] <= i) ra++;
                int rank = i;
                if (S.lo_after[ra] < wi) {        // some later run has smaller W
                    for (int b = ra + 1; b < R; b++) {
                        if (S.run_lo[b] >= wi) continue;
                        const int st = S.runs[b], en = S.runs[b + 1];
                        rank += (S.run_hi[b] < wi) ? en - st : lower_bound_f(uw, st, en, wi) - st;
                    }
                }
                if (S.hi_before[ra] > wi) {       // some earlier run has larger W
                    for (int b = 0; b < ra; b++) {
                        if (S.run_hi[b] <= wi) continue;
                        const int st = S.runs[b], en = S.runs[b + 1];
                        rank -= (S.run_lo[b] > wi) ? en - st : en - upper_bound_f(uw, st, en, wi);
                    }
                }
                S.sw[rank] = wi;
                S.sv[rank] = uv[i];
                S.sidx[rank] = (uint16_t)i;
            }
        } else {
            // Many runs: a counting sort by the bucket (int)(fl(W - W_min) * scale) -- a non-decreasing function of W,
            // so it orders the samples of different buckets -- then odd-even transposition passes by (W, index)
            // until none swaps, which orders the samples within a bucket.  Buckets are about one W unit wide, at
            // most CAP of them, so most hold a sample or two.
            float wlo = INFINITY, whi = -INFINITY;
            for (int i = lane; i < n; i += 32) {
                wlo = fminf(wlo, uw[i]);
                whi = fmaxf(whi, uw[i]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                wlo = fminf(wlo, __shfl_xor_sync(kFull, wlo, o));
                whi = fmaxf(whi, __shfl_xor_sync(kFull, whi, o));
            }
            const float span = __fsub_rn(whi, wlo);
            int B = CAP;
            float scale = 1.0f;
            if (span < (float)(CAP - 1)) B = (int)span + 1;
            else scale = (float)(CAP - 1) / span;
            auto bucket = [&](float w) { return min((int)(__fsub_rn(w, wlo) * scale), B - 1); };
            int* cnt = reinterpret_cast<int*>(S.sw);
            for (int b = lane; b < B; b += 32) cnt[b] = 0;
            __syncwarp();
            for (int i = lane; i < n; i += 32) atomicAdd(&cnt[bucket(uw[i])], 1);
            __syncwarp();
            // Exclusive prefix sums of the counts, 32 buckets at a time.
            int carry = 0;
            for (int b0 = 0; b0 < B; b0 += 32) {
                const int b = b0 + lane;
                const int c = b < B ? cnt[b] : 0;
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                if (b < B) cnt[b] = carry + incl - c;
                carry += __shfl_sync(kFull, incl, 31);
            }
            __syncwarp();
            for (int i = lane; i < n; i += 32) S.sidx[atomicAdd(&cnt[bucket(uw[i])], 1)] = (uint16_t)i;
            __syncwarp();
            for (;;) {
                bool swapped = false;
#pragma unroll
                for (int par = 0; par < 2; par++) {
                    for (int i = 2 * lane + par; i + 1 < n; i += 64) {
                        const int ia = S.sidx[i], ib = S.sidx[i + 1];
                        const float wa = uw[ia], wb = uw[ib];
                        if (wa > wb || (wa == wb && ia > ib)) {
                            S.sidx[i] = (uint16_t)ib;
                            S.sidx[i + 1] = (uint16_t)ia;
                            swapped = true;
                        }
                    }
                    __syncwarp();
                }
                if (!__any_sync(kFull, swapped)) break;
            }
            for (int q = lane; q < n; q += 32) {
                const int idx = S.sidx[q];
                S.sw[q] = uw[idx];
                S.sv[q] = uv[idx];
            }
        }
    }
    __syncwarp();

    // Eq. 5, every pair once from its lower sorted end.
    for (int q = lane; q < n; q += 32) cnt_up[q] = 0;
    __syncwarp();
    for (int q = lane; q < n; q += 32) {
        const float wq = sw[q];
        const float vq = sv[q];
        const float vbq = __fadd_rn(vq, beta);
        int o = 0;
        if (half <= 4) {
#pragma unroll
            for (int d = 1; d <= 4; d++) {
                if (d <= half && q + d < n) {
                    const float wd = sw[q + d];
                    const float vd = sv[q + d];
                    const bool close = fabsf(__fsub_rn(wq, wd)) < zeta;
                    o += (close && vbq < vd) ? 1 : 0;
                    if (close && __fadd_rn(vd, beta) < vq) atomicAdd(&cnt_up[q + d], 1);
                }
            }
        } else {
            for (int d = 1; d <= half && q + d < n; d++) {
                const float wd = sw[q + d];
                if (!(fabsf(__fsub_rn(wq, wd)) < zeta)) break;
                const float vd = sv[q + d];
                o += (vbq < vd) ? 1 : 0;
                if (__fadd_rn(vd, beta) < vq) atomicAdd(&cnt_up[q + d], 1);
            }
        }
        cnt_own[q] = o;
    }
    __syncwarp();
    __syncwarp();
    // Eq. 6 is the caller's: every sample's count, with its k.
    for (int q = lane; q < n; q += 32) {
        const int o = cnt_own[q] + cnt_up[q];
        if (o) emit(k0 + (R == 1 ? q : (int)S.sidx[q]), o);
    }
    return n;
}

// One work item of the warp kernels: the scan line of the candidate cw = (y << 16) | x of (frame, view) i = f * nv + v,
// its counts added
// to the frame's O (Eq. 6) with global atomics, M set for strip views (whose O is otherwise final), the tile hit flag
// of the candidate, and the samples and pair tests accumulated per (frame, view) in (cur_v, acc_n, acc_p), flushed
// to the frame's statistics when i changes.  frames: the call's frame records.
template <int CAP>
__device__ __forceinline__ void scan_item(const Args& a, const FrameArg* frames, ScanSmem<CAP>& S, int lane, int i,
                                          uint32_t cw, int& cur_v, unsigned long long& acc_n, unsigned long long& acc_p)
{
    constexpr unsigned kFull = 0xFFFFFFFFu;
    const int half = a.N >> 1;
    const float beta = a.beta, zeta = a.zeta;
    const int f = i / a.nv, v = i - f * a.nv;
    const FrameArg& F = frames[f];
    const ViewArg va = a.view[v];
    const float fcx = (float)(cw & 0xFFFFu), fcy = (float)(cw >> 16);
    const int h = a.plan[i].h;
    const int W = F.W;

    // Eq. 6: every sample's count goes to the occlusion sum of its pixel, found again from its k (Eq. 4).  A strip
    // view's O is final apart from these lines, and k_mask does not run for it: M is set here.
    int32_t* Ov = F.O + (int64_t)v * F.H * F.W;
    uint8_t* Mv = F.M + (int64_t)v * F.H * F.W;
    const bool strip_view = va.fam >= 0;
    bool hit = false;
    const int n = scan_line<CAP>(S, lane, F.D, F.pitch, F.W, F.H, va.c, va.s, va.r, fcx, fcy, h, half, beta, zeta,
                                 [&](int k, int o) {
                                     const float g = (float)(k - h);
                                     const int px = (int)roundf(__fadd_rn(__fmul_rn(va.c, g), fcx));
                                     const int py = (int)roundf(__fadd_rn(__fmul_rn(va.s, g), fcy));
                                     atomicAdd(Ov + py * W + px, o);
                                     if (strip_view) Mv[py * W + px] = 1;
                                     hit = true;
                                 });
    if (n <= 0) {
        if (lane == 0 && n < 0) atomicOr(a.status, ST_INTERNAL);
        __syncwarp();
        return;
    }
    if (__any_sync(kFull, hit) && lane == 0 && F.hits) {
        const int cx = (int)(cw & 0xFFFFu), cy = (int)(cw >> 16);
        F.hits[(int64_t)v * F.tiles_x * F.tiles_y + (cy / kTile) * F.tiles_x + cx / kTile] = 1;
    }

    if (lane == 0) {
        if (i != cur_v) {
            if (cur_v >= 0) {
                const int cf = cur_v / a.nv, cv = cur_v - cf * a.nv;
                atomicAdd(&frames[cf].stats[2 * cv], acc_n);
                atomicAdd(&frames[cf].stats[2 * cv + 1], acc_p);
            }
            cur_v = i;
            acc_n = acc_p = 0;
        }
        acc_n += (unsigned long long)n;
        acc_p += pair_count(n, half);
    }
    __syncwarp();
}

// The statistics a warp accumulated in scan_item, added to its last (frame, view).
__device__ __forceinline__ void flush_item_stats(const FrameArg* frames, int nv, int lane, int cur_v,
                                                 unsigned long long acc_n, unsigned long long acc_p)
{
    if (lane == 0 && cur_v >= 0) {
        const int cf = cur_v / nv, cv = cur_v - cf * nv;
        atomicAdd(&frames[cf].stats[2 * cv], acc_n);
        atomicAdd(&frames[cf].stats[2 * cv + 1], acc_p);
    }
}

}  // namespace
}  // namespace occ
