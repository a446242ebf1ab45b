// occ_kernels.cu -- sm_103a kernels of the fast edge-aware occlusion detection (Sippel, Seiler, Kaup, ICIP 2024,
// Section 3).
//
//   k_edges  one pass over D: Eq. 1 forward differences on D_r = fl(r D) for every distinct baseline ratio, the
//            candidate predicate of Eq. 2 for every view, warp-ballot compaction of the candidate lists, the min/max
//            reduction Eq. 3 needs, the non-finite check, the optional E / A maps, and the zeroing of O.
//   k_scan   one warp per candidate: the scan line of Eq. 4 (positions, gather of V, warp W = G - V), the sort by
//            (W, k) as a merge of the line's monotone runs, the neighbour test of Eq. 5, and the accumulation of
//            the counts into O (Eq. 6, summed over all scan lines).
//   k_mask   M = (O > 0) (Eq. 6).
//
// Every floating-point operation that decides a candidate, a position, an order or a count is an explicit
// round-to-nearest binary32 intrinsic (__fmul_rn, __fadd_rn, __fsub_rn, __fsqrt_rn) and the file is compiled with
// --fmad=false, so the results are bit-identical to a plain one-operation-at-a-time binary32 evaluation.
#include <climits>
#include <cstdint>

#include "occ_internal.cuh"

namespace occ {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

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

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = a.W, H = a.H;
    const int QW = (W + 3) >> 2;
    const int64_t nq = (int64_t)H * QW;
    const int64_t plane = (int64_t)H * W;
    const bool vecD = ((a.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.D) & 15) == 0);
    const bool vecO = ((W & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.O) & 15) == 0);
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
            load_quad(a.D + (int64_t)y * a.pitch, x0, W, vecD, d);
            hasd = (y + 1 < H);
            if (hasd) load_quad(a.D + (int64_t)(y + 1) * a.pitch, x0, W, vecD, dn);
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
        if (active && (a.E || a.A)) {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (!valid[j]) continue;
                const float ex = (x0 + j + 1 < W) ? __fsub_rn(d[j + 1], d[j]) : 0.0f;
                const float ey = hasd ? __fsub_rn(dn[j], d[j]) : 0.0f;
                const int64_t o = (int64_t)y * W + x0 + j;
                if (a.E) a.E[o] = __fsqrt_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)));
                if (a.A) a.A[o] = atan2f(ey, ex);
            }
        }

        // Eq. 1 on D_r for every distinct ratio, Eq. 2 for every view of that ratio.
        uint64_t bits[4] = {0, 0, 0, 0};
        if (active) {
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
                    const float e = __fsqrt_rn(__fadd_rn(__fmul_rn(ex[j], ex[j]), __fmul_rn(ey[j], ey[j])));
                    pe[j] = valid[j] && (e > a.gamma);
                }
                for (int v = 0; v < a.nv; v++) {
                    if (a.view[v].ridx != u) continue;
                    const float c = a.view[v].c, s = a.view[v].s;
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const float dot = __fadd_rn(__fmul_rn(ex[j], c), __fmul_rn(ey[j], s));
                        if (pe[j] && dot > 0.0f) bits[j] |= (1ull << v);
                    }
                }
            }
        }

        // Compaction: warp totals per view, then one reservation per block and view.
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
            uint32_t base = sum ? atomicAdd(&a.hdr[HDR_COUNT + v], sum) : 0u;
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
                    if ((int64_t)pos < a.cand_cap)
                        a.cand[(int64_t)v * a.cand_cap + pos] = ((uint32_t)y << 16) | (uint32_t)(x0 + j);
                    else
                        atomicOr(&a.hdr[HDR_STATUS], ST_CAND_OVERFLOW);
                    pos++;
                }
            }
        }

        // O = 0 for the quad in every view (the scan kernel accumulates into it).
        if (active) {
            const int64_t o = (int64_t)y * W + x0;
            for (int v = 0; v < a.nv; v++) {
                int32_t* Ov = a.O + (int64_t)v * plane + o;
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
            atomicMax(&a.hdr[HDR_MAX], f2ord(bhi));
            atomicMax(&a.hdr[HDR_NEGMIN], ~f2ord(blo));
        }
        if (s_bad) atomicOr(&a.hdr[HDR_STATUS], ST_NONFINITE);
    }
}

// ------------------------------------------------------------------------------------------------------------------
// k_scan: Eq. 4, the warp, the sort and Eq. 5 / Eq. 6 for every candidate, one warp per candidate.
//
// Sort.  floor(W) is monotone in W, so ordering the samples by (floor(W), W, k) is ordering them by (W, k): the
// samples are counted into unit-width bins of W (shared-memory atomics), a warp prefix sum turns the counts into
// bin offsets, and each sample's rank is its bin offset plus the number of samples of its own bin that precede it
// in (W, k) order (bins hold one to a few samples).  Scan lines whose W span more bins than the buffer holds are
// sorted by a bitonic network instead.
//
// Occlusion test.  For sorted positions r < q = r + d (d <= N/2) with |W_q - W_r| < zeta, sample r is hit when
// V_r + beta < V_q and sample q when V_q + beta < V_r.  |fl(W_r - W_q)| = |fl(W_q - W_r)|, and because W is sorted
// the walk of Eq. 5 from either end reaches the pair exactly when the other does, so every pair is tested once,
// from its lower end; hits on the upper sample go to a shared-memory counter.

template <int CAP>
struct ScanSmem {
    static constexpr int kBins = 2 * CAP;
    float uw[CAP];            // W of sample k (scan line order), valid for k in [k0, k0 + n)
    float uv[CAP];            // V of sample k
    int32_t upix[CAP];        // y * W + x of sample k
    int32_t ubs[CAP];         // bin | (arrival slot << 16) of sample i = k - k0
    int32_t bins[kBins + 1];  // counts, then exclusive offsets (bins[nb] = n)
    float tw[CAP];            // W in (bin, arrival) order; later the forward-hit counts
    int32_t ti[CAP];          // sample index in (bin, arrival) order; later the backward-hit counts
    float sw[CAP];            // W in sorted order
    float sv[CAP];            // V in sorted order
    int32_t spix[CAP];        // pixel in sorted order (also the index buffer of the bitonic fallback)
};

// Number of (p, d) pairs with d in {-K..K}\{0} and 0 <= p+d < n, summed over p (Eq. 5's neighbour set).
__device__ __forceinline__ unsigned long long pair_count(int n, int K)
{
    const long long nn = n, kk = K;
    const long long one_side = (nn <= kk) ? nn * (nn - 1) / 2 : kk * (kk - 1) / 2 + (nn - kk) * kk;
    return (unsigned long long)(2 * one_side);
}

// Thread 0 of a scan block: the scan length of every view (Eq. 3 on D_r unless L is fixed), and the list and
// candidate-count prefix of the views whose scan lines (2h+1 samples) fall into size class `cls`.  Returns the number
// of such views.  A view whose automatic L exceeds OCC_MAX_SCAN sets ST_SCAN_TOO_LONG and is skipped.
__device__ int scan_views_of_class(const Args& a, int cls, int32_t* s_h, int32_t* s_vid, uint32_t* s_pref)
{
    const uint32_t st = a.hdr[HDR_STATUS];
    int ncls = 0;
    uint32_t pref = 0;
    s_pref[0] = 0;
    if (st & ST_NONFINITE) return 0;
    const float mx = ord2f(a.hdr[HDR_MAX]);
    const float mn = ord2f(~a.hdr[HDR_NEGMIN]);
    for (int v = 0; v < a.nv; v++) {
        int L;
        if (a.Lover > 0) {
            L = a.Lover;
        } else {
            // Eq. 3 on D_r: max D_r = fl(r max D) and min D_r = fl(r min D) (rounding is monotone).
            const float r = a.view[v].r;
            const float dmx = (r == 1.0f) ? mx : __fmul_rn(r, mx);
            const float dmn = (r == 1.0f) ? mn : __fmul_rn(r, mn);
            const float t = __fmul_rn(__fsub_rn(dmx, dmn), 2.0f);
            L = (t <= (float)OCC_MAX_SCAN) ? (int)ceilf(t) : -1;
        }
        if (L < 0) {
            atomicOr(&a.hdr[HDR_STATUS], ST_SCAN_TOO_LONG);
            continue;
        }
        const int h = (L + 1) / 2;
        s_h[v] = h;
        if (blockIdx.x == 0) a.hdr[HDR_L + v] = (uint32_t)L;
        const int nk = 2 * h + 1;
        const int c = nk <= kClassCap[0] ? 0 : (nk <= kClassCap[1] ? 1 : 2);
        if (c != cls) continue;
        uint32_t cnt = a.hdr[HDR_COUNT + v];
        if ((int64_t)cnt > a.cand_cap) cnt = (uint32_t)a.cand_cap;
        s_vid[ncls] = v;
        pref += cnt;
        s_pref[++ncls] = pref;
    }
    return ncls;
}

template <int CAP>
__device__ __forceinline__ void bitonic_sort_warp(ScanSmem<CAP>& S, const float* uw, const float* uv,
                                                  const int32_t* upix, int n, int lane)
{
    int P = 32;
    while (P < n) P <<= 1;
    for (int i = lane; i < P; i += 32) {
        S.sw[i] = (i < n) ? uw[i] : INFINITY;
        S.spix[i] = (i < n) ? i : INT_MAX;
    }
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < (P >> 1); t += 32) {
                const int i = 2 * t - (t & (stride - 1));
                const int j = i + stride;
                const float wi = S.sw[i], wj = S.sw[j];
                const int ii = S.spix[i], ij = S.spix[j];
                const bool gt = (wi > wj) || (wi == wj && ii > ij);
                if (gt == ((i & size) == 0)) {
                    S.sw[i] = wj; S.sw[j] = wi;
                    S.spix[i] = ij; S.spix[j] = ii;
                }
            }
            __syncwarp();
        }
    }
    for (int q = lane; q < n; q += 32) {
        const int idx = S.spix[q];
        S.sv[q] = uv[idx];
        S.spix[q] = upix[idx];
    }
}

template <int CAP, int WPB>
__global__ void __launch_bounds__(WPB * 32) k_scan(const __grid_constant__ Args a, int cls)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t s_h[kMaxViews];
    __shared__ int32_t s_vid[kMaxViews];
    __shared__ uint32_t s_pref[kMaxViews + 1];
    __shared__ int s_ncls;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ScanSmem<CAP>& S = reinterpret_cast<ScanSmem<CAP>*>(smem_raw)[warp];

    if (threadIdx.x == 0) s_ncls = scan_views_of_class(a, cls, s_h, s_vid, s_pref);
    __syncthreads();
    const int ncls = s_ncls;
    if (ncls == 0) return;
    const uint32_t total = s_pref[ncls];

    const int W = a.W, H = a.H;
    const int64_t plane = (int64_t)H * W;
    const int half = a.N >> 1;
    const float fW = (float)W, fH = (float)H;
    const float beta = a.beta, zeta = a.zeta;

    int cur_v = -1;
    unsigned long long acc_n = 0, acc_p = 0;

    for (uint64_t item = (uint64_t)blockIdx.x * WPB + warp; item < total; item += (uint64_t)gridDim.x * WPB) {
        int j = 0;
        while (item >= s_pref[j + 1]) j++;
        const int v = s_vid[j];
        const uint32_t cw = a.cand[(int64_t)v * a.cand_cap + (int64_t)(item - s_pref[j])];
        const float fcx = (float)(cw & 0xFFFFu), fcy = (float)(cw >> 16);
        const float c = a.view[v].c, s = a.view[v].s, r = a.view[v].r;
        const bool one = (r == 1.0f);
        const int h = s_h[v];
        const int nk = 2 * h + 1;

        // Eq. 4: positions, bounds, V = D_r at the nearest pixel, W = g - V.
        int k0 = -1, kl = -1, n = 0;
        float wmin = INFINITY, wmax = -INFINITY;
        for (int base = 0; base < nk; base += 32) {
            const int k = base + lane;
            bool ok = false;
            if (k < nk) {
                const float g = (float)(k - h);
                const float rx = roundf(__fadd_rn(__fmul_rn(c, g), fcx));
                const float ry = roundf(__fadd_rn(__fmul_rn(s, g), fcy));
                ok = (rx >= 0.0f) && (rx < fW) && (ry >= 0.0f) && (ry < fH);
                if (ok) {
                    const int px = (int)rx, py = (int)ry;
                    const float dv = __ldg(a.D + (int64_t)py * a.pitch + px);
                    const float V = one ? dv : __fmul_rn(r, dv);
                    const float Wk = __fsub_rn(g, V);
                    S.uw[k] = Wk;
                    S.uv[k] = V;
                    S.upix[k] = py * W + px;
                    wmin = fminf(wmin, Wk);
                    wmax = fmaxf(wmax, Wk);
                }
            }
            const unsigned b = __ballot_sync(kFull, ok);
            if (b) {
                if (k0 < 0) k0 = base + __ffs(b) - 1;
                kl = base + 31 - __clz(b);
                n += __popc(b);
            }
        }
        // The samples inside the image form one interval of k (positions are monotone in g).
        if (n == 0 || kl - k0 + 1 != n) {
            if (lane == 0 && n != 0) atomicOr(&a.hdr[HDR_STATUS], ST_INTERNAL);
            __syncwarp();
            continue;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            wmin = fminf(wmin, __shfl_xor_sync(kFull, wmin, off));
            wmax = fmaxf(wmax, __shfl_xor_sync(kFull, wmax, off));
        }
        __syncwarp();
        const float* uw = S.uw + k0;
        const float* uv = S.uv + k0;
        const int32_t* upix = S.upix + k0;

        const float fb0 = floorf(wmin);
        const float span = __fsub_rn(floorf(wmax), fb0);
        if (span < (float)ScanSmem<CAP>::kBins) {
            const int nb = (int)span + 1;
            for (int b = lane; b < nb; b += 32) S.bins[b] = 0;
            __syncwarp();
            // Count every sample into its bin; the returned count is its arrival slot inside the bin.
            for (int i = lane; i < n; i += 32) {
                const int b = (int)__fsub_rn(floorf(uw[i]), fb0);
                const int slot = atomicAdd(&S.bins[b], 1);
                S.ubs[i] = b | (slot << 16);
            }
            __syncwarp();
            // Exclusive prefix sum of the bin counts, 32 bins per step.
            int carry = 0;
            for (int b0 = 0; b0 < nb; b0 += 32) {
                const int b = b0 + lane;
                const int x = (b < nb) ? S.bins[b] : 0;
                int incl = x;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, off);
                    if (lane >= off) incl += y;
                }
                if (b < nb) S.bins[b] = carry + incl - x;
                carry += __shfl_sync(kFull, incl, 31);
            }
            if (lane == 0) S.bins[nb] = n;
            __syncwarp();
            for (int i = lane; i < n; i += 32) {
                const int bs = S.ubs[i];
                const int p = S.bins[bs & 0xFFFF] + (bs >> 16);
                S.tw[p] = uw[i];
                S.ti[p] = i;
            }
            __syncwarp();
            // Rank = bin offset + samples of the same bin before this one in (W, k) order (k order = i order).
            for (int i = lane; i < n; i += 32) {
                const int b = S.ubs[i] & 0xFFFF;
                const int st = S.bins[b], en = S.bins[b + 1];
                const float wi = uw[i];
                int rank = st;
                for (int p = st; p < en; p++) {
                    const float wp = S.tw[p];
                    rank += (wp < wi) || (wp == wi && S.ti[p] < i);
                }
                S.sw[rank] = wi;
                S.sv[rank] = uv[i];
                S.spix[rank] = upix[i];
            }
        } else {
            bitonic_sort_warp<CAP>(S, uw, uv, upix, n, lane);
        }
        __syncwarp();

        // Eq. 5, each pair once from its lower sorted end; forward hits in tw (as int), backward hits in ti.
        int* fwd = reinterpret_cast<int*>(S.tw);
        int* bwd = S.ti;
        for (int q = lane; q < n; q += 32) bwd[q] = 0;
        __syncwarp();
        for (int q = lane; q < n; q += 32) {
            const float wq = S.sw[q];
            const float vq = S.sv[q];
            const float vbq = __fadd_rn(vq, beta);
            int o = 0;
            const int dmax = min(half, n - 1 - q);
            for (int d = 1; d <= dmax; d++) {
                const float wd = S.sw[q + d];
                if (!(fabsf(__fsub_rn(wq, wd)) < zeta)) break;
                const float vd = S.sv[q + d];
                o += (vbq < vd);
                if (__fadd_rn(vd, beta) < vq) atomicAdd(&bwd[q + d], 1);
            }
            fwd[q] = o;
        }
        __syncwarp();
        // Eq. 6: add every sample's count to the occlusion sum of its pixel.
        int32_t* Ov = a.O + (int64_t)v * plane;
        for (int q = lane; q < n; q += 32) {
            const int o = fwd[q] + bwd[q];
            if (o) atomicAdd(Ov + S.spix[q], o);
        }

        if (lane == 0) {
            if (v != cur_v) {
                if (cur_v >= 0) {
                    atomicAdd(&a.stats[2 * cur_v], acc_n);
                    atomicAdd(&a.stats[2 * cur_v + 1], acc_p);
                }
                cur_v = v;
                acc_n = acc_p = 0;
            }
            acc_n += (unsigned long long)n;
            acc_p += pair_count(n, half);
        }
        __syncwarp();
    }
    if (lane == 0 && cur_v >= 0) {
        atomicAdd(&a.stats[2 * cur_v], acc_n);
        atomicAdd(&a.stats[2 * cur_v + 1], acc_p);
    }
}

// ------------------------------------------------------------------------------------------------------------------
// k_scan_fast: the scan kernel for scan lines of at most 256 samples and N <= 8 (the common case), one warp per
// candidate, with the line held in registers: lane l owns the M = ceil((2h+1)/32) consecutive samples
// k = l*M .. l*M+M-1.
//
// Sort.  The rank of sample i among the valid samples is rank_i = i + #{j > i : W_j < W_i} - #{j < i : W_j > W_i}
// (ties go to the smaller k).  A suffix minimum and a prefix maximum of W (register scans plus one warp scan) bound
// both counts: the right count is zero when min(W_{i+1..}) >= W_i and otherwise runs only while that minimum stays
// below W_i, and symmetrically on the left.  Nearly sorted lines therefore cost two compares per sample, and a
// line crossing an edge pays only for its actual inversions.
//
// Occlusion test.  After the scatter into sorted order each lane reloads M consecutive sorted samples plus the next
// N/2, and tests every pair (p, p+d), d <= N/2, once: |fl(W_p - W_q)| is symmetric, and in sorted order |dW| only
// grows with d, so testing every d <= N/2 without stopping counts exactly the neighbours Eq. 5's walk reaches.

struct FastSmem {
    float w[256];       // W by k
    float pmax[256];    // prefix max of W by k (-inf outside the valid samples)
    float smin[256];    // suffix min of W by k (+inf outside the valid samples)
    float sw[256];      // sorted W
    float sv[256];      // sorted V
    int32_t spix[256];  // sorted pixel
    int32_t ocnt[256];  // hits on a sorted sample from pairs tested by another lane
};

template <int M>
__device__ __forceinline__ void line_fast(const Args& a, FastSmem& S, int lane, int v, uint32_t cw, int h,
                                          int half, int& n_out)
{
    const float fcx = (float)(cw & 0xFFFFu), fcy = (float)(cw >> 16);
    const float c = a.view[v].c, s = a.view[v].s, r = a.view[v].r;
    const bool one = (r == 1.0f);
    const int nk = 2 * h + 1;
    const float fW = (float)a.W, fH = (float)a.H;
    const int W = a.W;

    float w[M], vv[M];
    int pix[M];
    bool ok[M];
    int nloc = 0;
#pragma unroll
    for (int t = 0; t < M; t++) {
        const int k = lane * M + t;
        ok[t] = false;
        w[t] = INFINITY;
        vv[t] = 0.0f;
        pix[t] = 0;
        if (k < nk) {
            const float g = (float)(k - h);
            const float rx = roundf(__fadd_rn(__fmul_rn(c, g), fcx));
            const float ry = roundf(__fadd_rn(__fmul_rn(s, g), fcy));
            if ((rx >= 0.0f) && (rx < fW) && (ry >= 0.0f) && (ry < fH)) {
                const int px = (int)rx, py = (int)ry;
                const float dv = __ldg(a.D + (int64_t)py * a.pitch + px);
                vv[t] = one ? dv : __fmul_rn(r, dv);
                w[t] = __fsub_rn(g, vv[t]);
                pix[t] = py * W + px;
                ok[t] = true;
                nloc++;
            }
        }
    }
    // Valid samples form one interval [k0, k0 + n) of k.
    int n = nloc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) n += __shfl_xor_sync(kFull, n, off);
    int k0;
    {
        // first valid k: lowest lane with a valid sample, and its first valid slot
        int myfirst = 1 << 30;
#pragma unroll
        for (int t = M - 1; t >= 0; t--)
            if (ok[t]) myfirst = lane * M + t;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) myfirst = min(myfirst, __shfl_xor_sync(kFull, myfirst, off));
        k0 = myfirst;
    }
    n_out = n;
    if (n == 0) return;

    // Prefix max (invalid = -inf) and suffix min (invalid = +inf) of W over k.
    float pm[M], sm[M];
    float run = -INFINITY;
#pragma unroll
    for (int t = 0; t < M; t++) {
        run = fmaxf(run, ok[t] ? w[t] : -INFINITY);
        pm[t] = run;
    }
    float incl = run;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl = fmaxf(incl, y);
    }
    float excl = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0) excl = -INFINITY;
#pragma unroll
    for (int t = 0; t < M; t++) pm[t] = fmaxf(pm[t], excl);
    run = INFINITY;
#pragma unroll
    for (int t = M - 1; t >= 0; t--) {
        run = fminf(run, ok[t] ? w[t] : INFINITY);
        sm[t] = run;
    }
    incl = run;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float y = __shfl_down_sync(kFull, incl, off);
        if (lane + off < 32) incl = fminf(incl, y);
    }
    excl = __shfl_down_sync(kFull, incl, 1);
    if (lane == 31) excl = INFINITY;
#pragma unroll
    for (int t = 0; t < M; t++) sm[t] = fminf(sm[t], excl);
#pragma unroll
    for (int t = 0; t < M; t++) {
        const int k = lane * M + t;
        S.w[k] = w[t];
        S.pmax[k] = pm[t];
        S.smin[k] = sm[t];
    }
    const float next_sm = __shfl_down_sync(kFull, sm[0], 1);   // smin at k = (lane+1)*M
    const float prev_pm = __shfl_up_sync(kFull, pm[M - 1], 1);  // pmax at k = lane*M - 1
    for (int i = lane; i < n; i += 32) S.ocnt[i] = 0;
    __syncwarp();

    // Rank and scatter into sorted order.
#pragma unroll
    for (int t = 0; t < M; t++) {
        if (!ok[t]) continue;
        const int k = lane * M + t;
        const float wi = w[t];
        int rank = k - k0;
        const float smn = (t + 1 < M) ? sm[(t + 1 < M) ? t + 1 : 0] : (lane == 31 ? INFINITY : next_sm);
        if (smn < wi) {
            for (int j = k + 1; j < 32 * M && S.smin[j] < wi; j++) rank += (S.w[j] < wi);
        }
        const float pmx = (t > 0) ? pm[(t > 0) ? t - 1 : 0] : (lane == 0 ? -INFINITY : prev_pm);
        if (pmx > wi) {
            for (int j = k - 1; j >= 0 && S.pmax[j] > wi; j--) rank -= (S.w[j] > wi);
        }
        S.sw[rank] = wi;
        S.sv[rank] = vv[t];
        S.spix[rank] = pix[t];
    }
    __syncwarp();

    // Eq. 5 on the sorted samples: lane l tests pairs whose lower end is one of its M positions.
    const float beta = a.beta, zeta = a.zeta;
    float w2[M + kFastMaxHalf], v2[M + kFastMaxHalf], vb2[M + kFastMaxHalf];
#pragma unroll
    for (int t = 0; t < M + kFastMaxHalf; t++) {
        const int q = lane * M + t;
        const bool in = q < n;
        w2[t] = in ? S.sw[q] : INFINITY;
        v2[t] = in ? S.sv[q] : 0.0f;
        vb2[t] = __fadd_rn(v2[t], beta);
    }
    int o[M];
#pragma unroll
    for (int t = 0; t < M; t++) o[t] = 0;
#pragma unroll
    for (int t = 0; t < M; t++) {
#pragma unroll
        for (int d = 1; d <= kFastMaxHalf; d++) {
            if (d > half) break;
            const bool close = fabsf(__fsub_rn(w2[t], w2[t + d])) < zeta;
            o[t] += (close && (vb2[t] < v2[t + d])) ? 1 : 0;
            const bool hitp = close && (vb2[t + d] < v2[t]);
            if (t + d < M) {
                o[(t + d < M) ? t + d : 0] += hitp ? 1 : 0;
            } else if (hitp) {
                atomicAdd(&S.ocnt[lane * M + t + d], 1);
            }
        }
    }
    __syncwarp();
    int32_t* Ov = a.O + (int64_t)v * ((int64_t)a.H * a.W);
#pragma unroll
    for (int t = 0; t < M; t++) {
        const int q = lane * M + t;
        if (q < n) {
            const int tot = o[t] + S.ocnt[q];
            if (tot) atomicAdd(Ov + S.spix[q], tot);
        }
    }
    __syncwarp();
}

template <int WPB>
__global__ void __launch_bounds__(WPB * 32) k_scan_fast(const __grid_constant__ Args a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t s_h[kMaxViews];
    __shared__ int32_t s_vid[kMaxViews];
    __shared__ uint32_t s_pref[kMaxViews + 1];
    __shared__ int s_ncls;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    FastSmem& S = reinterpret_cast<FastSmem*>(smem_raw)[warp];
    if (threadIdx.x == 0) s_ncls = scan_views_of_class(a, 0, s_h, s_vid, s_pref);
    __syncthreads();
    const int ncls = s_ncls;
    if (ncls == 0) return;
    const uint32_t total = s_pref[ncls];
    const int half = a.N >> 1;

    int cur_v = -1;
    unsigned long long acc_n = 0, acc_p = 0;
    for (uint64_t item = (uint64_t)blockIdx.x * WPB + warp; item < total; item += (uint64_t)gridDim.x * WPB) {
        int j = 0;
        while (item >= s_pref[j + 1]) j++;
        const int v = s_vid[j];
        const uint32_t cw = a.cand[(int64_t)v * a.cand_cap + (int64_t)(item - s_pref[j])];
        const int h = s_h[v];
        const int M = (2 * h + 1 + 31) >> 5;
        int n = 0;
        switch (M) {
        case 1: line_fast<1>(a, S, lane, v, cw, h, half, n); break;
        case 2: line_fast<2>(a, S, lane, v, cw, h, half, n); break;
        case 3: line_fast<3>(a, S, lane, v, cw, h, half, n); break;
        case 4: line_fast<4>(a, S, lane, v, cw, h, half, n); break;
        case 5: line_fast<5>(a, S, lane, v, cw, h, half, n); break;
        case 6: line_fast<6>(a, S, lane, v, cw, h, half, n); break;
        case 7: line_fast<7>(a, S, lane, v, cw, h, half, n); break;
        default: line_fast<8>(a, S, lane, v, cw, h, half, n); break;
        }
        if (lane == 0) {
            if (v != cur_v) {
                if (cur_v >= 0) {
                    atomicAdd(&a.stats[2 * cur_v], acc_n);
                    atomicAdd(&a.stats[2 * cur_v + 1], acc_p);
                }
                cur_v = v;
                acc_n = acc_p = 0;
            }
            acc_n += (unsigned long long)n;
            acc_p += pair_count(n, half);
        }
    }
    if (lane == 0 && cur_v >= 0) {
        atomicAdd(&a.stats[2 * cur_v], acc_n);
        atomicAdd(&a.stats[2 * cur_v + 1], acc_p);
    }
}

// ------------------------------------------------------------------------------------------------------------------
// k_mask: M = (O > 0), 16 pixels per thread and iteration when aligned.

constexpr int kMaskThreads = 256;

__global__ void __launch_bounds__(kMaskThreads) k_mask(const __grid_constant__ Args a)
{
    const int64_t n = (int64_t)a.nv * a.H * a.W;
    const int64_t stride = (int64_t)gridDim.x * kMaskThreads;
    const int64_t t0 = (int64_t)blockIdx.x * kMaskThreads + threadIdx.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(a.O) & 15) == 0) && ((reinterpret_cast<uintptr_t>(a.M) & 15) == 0);
    int64_t done = 0;
    if (vec) {
        const int64_t n16 = n >> 4;
        const int4* O4 = reinterpret_cast<const int4*>(a.O);
        uint4* M16 = reinterpret_cast<uint4*>(a.M);
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
    for (int64_t i = done + t0; i < n; i += stride) a.M[i] = (uint8_t)(a.O[i] > 0);
}

template <int CAP, int WPB>
constexpr size_t scan_smem()
{
    return sizeof(ScanSmem<CAP>) * WPB;
}

constexpr int kWpb0 = 8, kWpb1 = 4, kWpb2 = 1, kWpbFast = 8;

}  // namespace

cudaError_t configure_kernels(int* edges_bps, int scan_bps[kNumClasses], int* mask_bps)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_scan_fast<kWpbFast>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(FastSmem) * kWpbFast))) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_scan<256, kWpb0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)scan_smem<256, kWpb0>())) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_scan<1024, kWpb1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)scan_smem<1024, kWpb1>())) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_scan<4096, kWpb2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)scan_smem<4096, kWpb2>())) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(edges_bps, k_edges, kEdgeThreads, 0)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&scan_bps[0], k_scan<256, kWpb0>, kWpb0 * 32,
                                                           scan_smem<256, kWpb0>())) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&scan_bps[kNumClasses], k_scan_fast<kWpbFast>,
                                                           kWpbFast * 32, sizeof(FastSmem) * kWpbFast)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&scan_bps[1], k_scan<1024, kWpb1>, kWpb1 * 32,
                                                           scan_smem<1024, kWpb1>())) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&scan_bps[2], k_scan<4096, kWpb2>, kWpb2 * 32,
                                                           scan_smem<4096, kWpb2>())) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(mask_bps, k_mask, kMaskThreads, 0);
}

cudaError_t launch_edges(const Args& a, int grid, cudaStream_t st)
{
    k_edges<<<grid, kEdgeThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan(const Args& a, int cls, int grid, cudaStream_t st)
{
    switch (cls) {
    case kFastClass: k_scan_fast<kWpbFast><<<grid, kWpbFast * 32, sizeof(FastSmem) * kWpbFast, st>>>(a); break;
    case 0: k_scan<256, kWpb0><<<grid, kWpb0 * 32, scan_smem<256, kWpb0>(), st>>>(a, 0); break;
    case 1: k_scan<1024, kWpb1><<<grid, kWpb1 * 32, scan_smem<1024, kWpb1>(), st>>>(a, 1); break;
    default: k_scan<4096, kWpb2><<<grid, kWpb2 * 32, scan_smem<4096, kWpb2>(), st>>>(a, 2); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_mask(const Args& a, int grid, cudaStream_t st)
{
    k_mask<<<grid, kMaskThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace occ
