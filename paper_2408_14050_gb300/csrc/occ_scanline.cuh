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

// A warp's shared memory for one line: V by sample, the sorted order as sample indices, and 16 bits of counts per
// sorted position, 8 bytes per sample.  W is stored only for the 256-sample class, whose warps are limited by registers
// rather than shared memory; otherwise W = fl(g - V) is recomputed from the sample's index wherever it is compared,
// the same operation that defines it.
template <int CAP>
struct ScanSmem {
    static constexpr bool kKeepW = CAP <= 256;   // lines of the 256-sample class also keep W by k (1 KB per warp)
    float uw[kKeepW ? CAP : 1];   // W by k (kKeepW)
    float uv[CAP];        // V by k
    uint16_t sidx[CAP];   // sample index (k - k0) of each sorted position (unused when the line is one run)
    uint32_t cnt[CAP / 2];// per sorted position q, 16 bits at (q & 1) * 16 of word q / 2: hits of the sample itself
                          // (low byte, <= N/2) and from below it (high byte, <= N/2); during the bucket sort, 16-bit
                          // bucket counts and offsets (at most CAP)
    int32_t runs[kMaxRuns + 2];
    float run_lo[kMaxRuns + 1];   // first (smallest) W of each run
    float run_hi[kMaxRuns + 1];   // last (largest) W of each run
    float lo_after[kMaxRuns + 2]; // min of run_lo over the runs after run b
    float hi_before[kMaxRuns + 2];// max of run_hi over the runs before run b
};

// First index in [lo, hi) whose W is > x (upper) or >= x (lower); W(lo..hi-1) is non-decreasing.
template <class WF>
__device__ __forceinline__ int upper_bound_w(const WF& Wat, int lo, int hi, float x)
{
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (Wat(m) <= x) lo = m + 1; else hi = m;
    }
    return lo;
}
template <class WF>
__device__ __forceinline__ int lower_bound_w(const WF& Wat, int lo, int hi, float x)
{
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (Wat(m) < x) lo = m + 1; else hi = m;
    }
    return lo;
}

// One scan line (Eq. 4) through the candidate at (fcx, fcy) of a map D (row pitch `pitch`, W x H), direction (c, s),
// ratio r, half length h; the warp W = g - V, the sort by (W, k) and the test of Eq. 5 with N = 2 half neighbours.
// emit(k, o) is called once for every sample k (0 .. 2h) with o > 0 hits, by the lane that holds it; the caller adds
// o to O at the sample's pixel (Eq. 6).  Returns the number of samples inside the map, 0 for none, and -1 when they
// do not form one interval of k (a self-check; positions are monotone in g).  Uses the warp's ScanSmem; lines of at
// most CAP samples (2h + 1 <= CAP), N <= 64.
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

    // Eq. 4: positions, bounds, V = D_r at the nearest pixel.
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
                S.uv[k] = V;
                if constexpr (ScanSmem<CAP>::kKeepW) S.uw[k] = __fsub_rn((float)(k - h), V);
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
                    S.uv[k] = one ? dv : __fmul_rn(r, dv);
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
    const float* uv = S.uv + k0;
    const float* uw = S.uw + (ScanSmem<CAP>::kKeepW ? k0 : 0);
    // W of sample i (k = k0 + i): fl(g - V), g = k - h; kept by k for the 256-sample class, else recomputed.
    auto Wat = [&](int i) {
        if constexpr (ScanSmem<CAP>::kKeepW) return uw[i];
        else return __fsub_rn((float)(k0 + i - h), uv[i]);
    };

    // Runs: a new run starts after every descent W[i+1] < W[i].
    int R = 1;
    for (int base = 0; base < n - 1; base += 32) {
        const int i = base + lane;
        const bool dsc = (i < n - 1) && (Wat(i + 1) < Wat(i));
        const unsigned b = __ballot_sync(kFull, dsc);
        if (dsc) {
            const int slot = R + __popc(b & lt);
            if (slot <= kMaxRuns) S.runs[slot] = i + 1;
        }
        R += __popc(b);
    }

    if (R > 1 && R <= kMaxRuns) {
        if (lane == 0) {
            S.runs[0] = 0;
            S.runs[R] = n;
        }
        __syncwarp();
        if (lane < R) {
            S.run_lo[lane] = Wat(S.runs[lane]);
            S.run_hi[lane] = Wat(S.runs[lane + 1] - 1);
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
            const float wi = Wat(i);
            int ra = 0;
            while (ra + 1 < R && S.runs[ra + 1] <= i) ra++;
            int rank = i;
            if (S.lo_after[ra] < wi) {        // some later run has smaller W
                for (int b = ra + 1; b < R; b++) {
                    if (S.run_lo[b] >= wi) continue;
                    const int st = S.runs[b], en = S.runs[b + 1];
                    rank += (S.run_hi[b] < wi) ? en - st : lower_bound_w(Wat, st, en, wi) - st;
                }
            }
            if (S.hi_before[ra] > wi) {       // some earlier run has larger W
                for (int b = 0; b < ra; b++) {
                    if (S.run_hi[b] <= wi) continue;
                    const int st = S.runs[b], en = S.runs[b + 1];
                    rank -= (S.run_lo[b] > wi) ? en - st : en - upper_bound_w(Wat, st, en, wi);
                }
            }
            S.sidx[rank] = (uint16_t)i;
        }
    } else if (R > kMaxRuns) {
        // Many runs: a counting sort by the bucket (int)(fl(W - W_min) * scale) -- a non-decreasing function of W,
        // so it orders the samples of different buckets -- then odd-even transposition passes by (W, index) until
        // none swaps, which orders the samples within a bucket.  Buckets are about one W unit wide, at most CAP of
        // them, so most hold a sample or two; their counts and offsets are 16-bit halves of the count words.
        float wlo = INFINITY, whi = -INFINITY;
        for (int i = lane; i < n; i += 32) {
            const float w = Wat(i);
            wlo = fminf(wlo, w);
            whi = fmaxf(whi, w);
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
        for (int b = lane; b < (B + 1) / 2; b += 32) S.cnt[b] = 0u;
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            const int b = bucket(Wat(i));
            atomicAdd(&S.cnt[b >> 1], 1u << ((b & 1) * 16));
        }
        __syncwarp();
        // Exclusive prefix sums of the counts, 32 buckets (16 words) at a time.
        uint32_t carry = 0;
        for (int b0 = 0; b0 < B; b0 += 32) {
            const int b = b0 + lane;
            const uint32_t cb = b < B ? (S.cnt[b >> 1] >> ((b & 1) * 16)) & 0xFFFFu : 0u;
            uint32_t incl = cb;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t ex = carry + incl - cb;
            const uint32_t ex_next = __shfl_down_sync(kFull, ex, 1);
            __syncwarp();   // every lane has read its count before its pair's word is rewritten
            if (!(lane & 1) && b < B) S.cnt[b >> 1] = ex | (ex_next << 16);
            carry += __shfl_sync(kFull, incl, 31);
        }
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            const int b = bucket(Wat(i));
            const int sh = (b & 1) * 16;
            const uint32_t old = atomicAdd(&S.cnt[b >> 1], 1u << sh);
            S.sidx[(old >> sh) & 0xFFFFu] = (uint16_t)i;
        }
        __syncwarp();
        for (;;) {
            bool swapped = false;
#pragma unroll
            for (int par = 0; par < 2; par++) {
                for (int i = 2 * lane + par; i + 1 < n; i += 64) {
                    const int ia = S.sidx[i], ib = S.sidx[i + 1];
                    const float wa = Wat(ia), wb = Wat(ib);
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
    }
    __syncwarp();

    // Eq. 5.  Sorted positions (q, q + d), d <= N/2, are the pairs tested; |fl(W_q - W_{q+d})| is symmetric.
    const bool sorted = R == 1;
    auto at = [&](int q) { return sorted ? q : (int)S.sidx[q]; };
    if (half <= 4) {
        // N <= 8: chunks of 32 sorted positions, one per lane, each lane counting the hits of its own position from
        // both sides (q hit by q + d when V_q + beta < V_{q+d}, and by q - d when V_q + beta < V_{q-d}) with the
        // neighbours' W and V from the lanes d away, or from the previous or next chunk at the chunk's ends: every
        // pair is tested from both of its ends, with no shared counters.  W = +inf past either end (never close).
        const float kInf = __int_as_float(0x7f800000);
        auto load = [&](int q, int& i, float& w, float& v) {
            if (q < n) {
                i = at(q);
                v = uv[i];
                w = Wat(i);
            } else {
                i = 0;
                v = 0.0f;
                w = kInf;
            }
        };
        int ci;
        float cw, cv, pw = kInf, pv = 0.0f;
        load(lane, ci, cw, cv);
        for (int base = 0; base < n; base += 32) {
            int ni;
            float nw, nv;
            load(base + 32 + lane, ni, nw, nv);
            const float vbq = __fadd_rn(cv, beta);
            int o = 0;
#pragma unroll
            for (int d = 1; d <= 4; d++) {
                const int up = (lane + d) & 31, dn = (lane - d) & 31;
                const float aw_c = __shfl_sync(kFull, cw, up), av_c = __shfl_sync(kFull, cv, up);
                const float aw_n = __shfl_sync(kFull, nw, up), av_n = __shfl_sync(kFull, nv, up);
                const float bw_c = __shfl_sync(kFull, cw, dn), bv_c = __shfl_sync(kFull, cv, dn);
                const float bw_p = __shfl_sync(kFull, pw, dn), bv_p = __shfl_sync(kFull, pv, dn);
                if (d <= half) {
                    const bool wrap_up = lane + d >= 32, wrap_dn = lane < d;
                    const float aw = wrap_up ? aw_n : aw_c, av = wrap_up ? av_n : av_c;
                    const float bw = wrap_dn ? bw_p : bw_c, bv = wrap_dn ? bv_p : bv_c;
                    o += (fabsf(__fsub_rn(cw, aw)) < zeta && vbq < av) ? 1 : 0;
                    o += (fabsf(__fsub_rn(bw, cw)) < zeta && vbq < bv) ? 1 : 0;
                }
            }
            // Eq. 6 is the caller's: every sample's count, with its k.
            if (base + lane < n && o) emit(k0 + ci, o);
            pw = cw;
            pv = cv;
            ci = ni;
            cw = nw;
            cv = nv;
        }
        return n;
    }
    // N > 8: every pair once from its lower sorted end, up to the first that is not close; the counts of sorted
    // position q in its 16-bit half word.
    for (int w = lane; w < (n + 1) / 2; w += 32) S.cnt[w] = 0u;
    __syncwarp();
    for (int q = lane; q < n; q += 32) {
        const int iq = at(q);
        const float wq = Wat(iq);
        const float vq = uv[iq];
        const float vbq = __fadd_rn(vq, beta);
        int o = 0;
        for (int d = 1; d <= half && q + d < n; d++) {
            const int id = at(q + d);
            const float wd = Wat(id);
            if (!(fabsf(__fsub_rn(wq, wd)) < zeta)) break;
            const float vd = uv[id];
            o += (vbq < vd) ? 1 : 0;
            if (__fadd_rn(vd, beta) < vq) atomicAdd(&S.cnt[(q + d) >> 1], 1u << (((q + d) & 1) * 16 + 8));
        }
        if (o) atomicAdd(&S.cnt[q >> 1], (uint32_t)o << ((q & 1) * 16));
    }
    __syncwarp();
    // Eq. 6 is the caller's: every sample's count, with its k.
    for (int q = lane; q < n; q += 32) {
        const uint32_t w = S.cnt[q >> 1] >> ((q & 1) * 16);
        const int o = (int)(w & 0xFFu) + (int)((w >> 8) & 0xFFu);
        if (o) emit(k0 + at(q), o);
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
