// occ_strip.cu -- k_strip: Eq. 1-6 for the views whose scan lines stay on one digital line of the frame (rows,
// columns, diagonals, anti-diagonals: the eight directions of a 3x3 camera array), with a strip of such lines owned by
// one CTA.
//
// A strip is B adjacent lines of one (frame, view).  Every scan line walked from a candidate of the strip stays on the
// candidate's own line (Eq. 4 with the view's direction), so the CTA holds all the data its scan lines touch:
//   1. it stages D_r = fl(r D) of its lines in shared memory (coalesced loads) and evaluates Eq. 1-2 for every pixel
//      of them, one bit per pixel;
//   2. it compacts the candidates (ballots, block prefix sums) into a queue, round by round;
//   3. per candidate, one pass over its scan line with the one-slot buffer finds its macro-runs (the stretches the
//      buffer sorts): lines of one macro-run go to one queue, lines of two to another, longer lines to a short list
//      of the strip (those that do not fit it, or have more than 255 samples, to the frame's list for the warp
//      kernel k_scan);
//   4. the lines of each queue are counted in batches of 32 per warp, every lane streaming one line: a plain stream
//      (one run) or the merge of two one-slot buffers (two runs), the sorted samples tested against the N/2 emitted
//      before them (Eq. 5), final counts added to the strip's occlusion sums O in shared memory (Eq. 6);
//   5. the lines of the strip's short list, one warp each, go through the warp sort of the list path (scan_line),
//      their counts added to the same shared sums;
//   6. it writes O and M = (O > 0) of its lines once, coalesced: no zero fill, no global atomics, no mask pass.
// O of one strip pixel fits 16 bits: at most 2h + 1 <= 4095 scan lines reach a pixel, each with at most two samples
// on it (|cos| or |sin| <= 1 moves a diagonal line by at most one pixel per step) and each sample counts at most
// N = 8 partners, so O <= 65520; two sums share a 32-bit word and are added with 32-bit shared atomics, which cannot
// carry from one half into the other.
//
// Every floating-point operation that decides a candidate, an order or a count is the same round-to-nearest binary32
// operation as in the list path (occ_kernels.cu) and the oracle, so the results are bit-identical.
#include <atomic>
#include <cstdint>
#include <cstring>

#include "occ_internal.cuh"
#include "occ_common.cuh"
#include "occ_scanline.cuh"

namespace occ {

namespace {

constexpr unsigned kFullMask = 0xFFFFFFFFu;
constexpr int kStripThreads = 128;
constexpr int kStripWarps = kStripThreads / 32;
constexpr int kStripQueue = 512;           // queue entries of one round
constexpr int kStripMany = 16;             // fused kernel: lines of three or more macro-runs a strip keeps to publish
constexpr int kStripManyMaxH = 127;        // ... when their 2h + 1 samples fit the 256-sample warp buffers

// Shared memory of a strip block: a 16-byte guard, D_r and the O words of strip_px pixels, two candidate bit maps, the
// line queue and the round's candidates.
__host__ __device__ __forceinline__ size_t strip_smem_bytes(int strip_px)
{
    return 16 + (size_t)strip_px * 4 + (size_t)strip_px * 4 + (size_t)strip_px / 4 + sizeof(uint2) * kStripQueue +
           sizeof(uint32_t) * kStripQueue;
}

// The fused launch's tag of its published-line entries: the count of earlier launches (CTR_EPOCH, raised by the last
// block to end, so constant while any block runs), top bit set so that it is never 0.
__device__ __forceinline__ uint32_t fused_tag(const Args& a)
{
    return (*reinterpret_cast<const volatile uint32_t*>(a.status + CTR_EPOCH) & 0x7FFFFFFFu) | 0x80000000u;
}

// First pixel (x0, y0), step (ax, ay) per position and length n of line l of a family.
__device__ __forceinline__ void line_geom(int fam, int H, int W, int l, int& x0, int& y0, int& ay, int& n)
{
    if (fam == kFamRows) {
        x0 = 0; y0 = l; ay = 0; n = W;
    } else if (fam == kFamCols) {
        x0 = l; y0 = 0; ay = 1; n = H;
    } else if (fam == kFamDiag) {            // x - y = l - (H - 1)
        const int d = l - (H - 1);
        x0 = d > 0 ? d : 0;
        y0 = x0 - d;
        ay = 1;
        n = min(W - x0, H - y0);
    } else {                                 // x + y = l
        x0 = l - (H - 1) > 0 ? l - (H - 1) : 0;
        y0 = l - x0;
        ay = -1;
        n = min(W - x0, y0 + 1);
    }
}

// Pixel of position t of a line: columns advance in y only, every other family in x by one per position.
__device__ __forceinline__ void line_pixel(int fam, int x0, int y0, int ay, int t, int& x, int& y)
{
    x = fam == kFamCols ? x0 : x0 + t;
    y = y0 + ay * t;
}

// O of a strip pixel: one 32-bit shared word per pixel holds the sums of the strip's two views, view A in the low
// and view B in the high 16 bits (sh = 0 or 16); added with a shared-memory reduction (no return value) predicated
// on o != 0 inside the asm, so that the count of a sample leaving the window goes to O without a branch.
__device__ __forceinline__ void o_add(uint32_t* sO, int p, int o, int sh)
{
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(sO + p);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q red.shared.add.u32 [%0], %1;\n\t}"
                 ::"r"(addr), "r"((uint32_t)o << sh), "r"((uint32_t)o) : "memory");
}
// Eq. 5 / Eq. 6 over an emitted (sorted) stream: the last N/2 = 4 samples, the i-th emitted sample in slot i mod 4,
// which held sample i - 4 (final once tested against the new one).  Empty slots hold W = +inf, close to nothing.
struct Win {
    float w[4], v[4], b[4];
    int p[4], o[4];
};

__device__ __forceinline__ void win_init(Win& R)
{
#pragma unroll
    for (int i = 0; i < 4; i++) {
        R.w[i] = __int_as_float(0x7f800000);
        R.v[i] = R.b[i] = 0.0f;
        R.p[i] = R.o[i] = 0;
    }
}

template <int J>
__device__ __forceinline__ void win_push(Win& R, float ew, float ev, int ep, float zeta, float beta, uint32_t* sO,
                                         int sh, int& hit)
{
    const float eb = __fadd_rn(ev, beta);
    int eo = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const bool close = fabsf(__fsub_rn(ew, R.w[i])) < zeta;
        eo += (close && eb < R.v[i]) ? 1 : 0;
        R.o[i] += (close && R.b[i] < ev) ? 1 : 0;
    }
    o_add(sO, R.p[J], R.o[J], sh);
    hit |= R.o[J];
    R.w[J] = ew;
    R.v[J] = ev;
    R.b[J] = eb;
    R.p[J] = ep;
    R.o[J] = eo;
}

__device__ __forceinline__ void win_flush(const Win& R, uint32_t* sO, int sh, int& hit)
{
#pragma unroll
    for (int i = 0; i < 4; i++) {
        o_add(sO, R.p[i], R.o[i], sh);
        hit |= R.o[i];
    }
}

// The samples of one scan line: k = 0 .. 2h at position tc + tab[k] of line row lb (its first shared index), its
// view's half of the O words (sh).
struct LineRef {
    const float* sV;
    const int16_t* tab;
    int base;   // lb + tc
    int h;
    int sh;
};

__device__ __forceinline__ void sample(const LineRef& L, int k, float& w, float& v, int& p)
{
    p = L.base + __ldg(L.tab + k);
    v = L.sV[p];
    w = __fsub_rn((float)(k - L.h), v);
}

// Macro-runs of samples k0 .. k1 under the one-slot buffer: returns 1, 2, or 3 for three or more; ks = the first k of
// the second run.  A run ends where the sample the buffer would emit precedes the last one emitted; the next run
// starts from that sample with an empty history (the buffered sample belongs to the run before).
__device__ __forceinline__ int detect_runs(const LineRef& L, int k0, int k1, int& ks)
{
    const float kNegInf = __int_as_float(0xff800000);
    float g = (float)(k0 - L.h);
    float bufw = __fsub_rn(g, L.sV[L.base + __ldg(L.tab + k0)]);
    float lastw = kNegInf;
    int runs = 1;
    ks = -1;
    int k = k0 + 1;
    int tn = __ldg(L.tab + k);   // k <= 2h + 1: the view's table runs past g = h (kSTabLen)
#define OCC_DSTEP                                                                    \
    {                                                                                \
        const float v = L.sV[L.base + tn];                                           \
        tn = __ldg(L.tab + k + 1);                                                   \
        g = __fadd_rn(g, 1.0f);                                                      \
        const float w = __fsub_rn(g, v);                                             \
        const bool sb = w < bufw;                                                    \
        if (sb && w < lastw) {                                                       \
            if (runs == 2) return 3;                                                 \
            runs = 2;                                                                \
            ks = k;                                                                  \
            bufw = w;                                                                \
            lastw = kNegInf;                                                         \
        } else {                                                                     \
            lastw = sb ? w : bufw;                                                   \
            bufw = sb ? bufw : w;                                                    \
        }                                                                            \
        k++;                                                                         \
    }
    for (; k + 3 <= k1;) {
        OCC_DSTEP OCC_DSTEP OCC_DSTEP OCC_DSTEP
    }
    for (; k <= k1;) OCC_DSTEP
#undef OCC_DSTEP
    return runs;
}

// One macro-run k0 .. k1 through the one-slot buffer: every emitted sample tested against the four before it.  The
// n - 1 samples after the first go in four at a time (the window slot of a step is its index mod 4), then the rest, then
// the buffered sample is emitted last.
__device__ __forceinline__ void count_stream(const LineRef& L, int k0, int k1, float zeta, float beta, uint32_t* sO,
                                             int& hit)
{
    Win R;
    win_init(R);
    float bw, bv;
    int bp;
    sample(L, k0, bw, bv, bp);
    float g = (float)(k0 - L.h);
    // The sample in flight (k) and the table offset of the one after it.
    int k = k0 + 1;
    int pn = L.base + __ldg(L.tab + k);   // k + 2 <= 2h + 2 below: the view's table runs past g = h (kSTabLen)
    float vn = L.sV[pn];
    int tn = __ldg(L.tab + k + 1);
    int rem = k1 - k0;
#define OCC_RSTEP(J)                                                                 \
    {                                                                                \
        g = __fadd_rn(g, 1.0f);                                                      \
        const float sv = vn;                                                         \
        const int sp = pn;                                                           \
        const float sw = __fsub_rn(g, sv);                                           \
        pn = L.base + tn;                                                            \
        vn = L.sV[pn];                                                               \
        tn = __ldg(L.tab + k + 2);                                                   \
        k++;                                                                         \
        const bool sb = sw < bw;                                                     \
        const float ew = sb ? sw : bw, ev = sb ? sv : bv;                            \
        const int ep = sb ? sp : bp;                                                 \
        if (!sb) {                                                                   \
            bw = sw;                                                                 \
            bv = sv;                                                                 \
            bp = sp;                                                                 \
        }                                                                            \
        win_push<J>(R, ew, ev, ep, zeta, beta, sO, L.sh, hit);                             \
    }
#define OCC_FSTEP(J) win_push<J>(R, bw, bv, bp, zeta, beta, sO, L.sh, hit);
    for (; rem >= 4; rem -= 4) {
        OCC_RSTEP(0)
        OCC_RSTEP(1)
        OCC_RSTEP(2)
        OCC_RSTEP(3)
    }
    switch (rem) {
    case 0: OCC_FSTEP(0) break;
    case 1: OCC_RSTEP(0) OCC_FSTEP(1) break;
    case 2: OCC_RSTEP(0) OCC_RSTEP(1) OCC_FSTEP(2) break;
    default: OCC_RSTEP(0) OCC_RSTEP(1) OCC_RSTEP(2) OCC_FSTEP(3) break;
    }
#undef OCC_RSTEP
#undef OCC_FSTEP
    win_flush(R, sO, L.sh, hit);
}

// Two macro-runs [k0, ks - 1] and [ks, k1], each through its own one-slot buffer, merged by (W, k): a head of the
// first run precedes one of the second exactly when its W is not larger.
__device__ __forceinline__ void count_merge2(const LineRef& L, int k0, int k1, int ks, float zeta, float beta,
                                             uint32_t* sO, int& hit)
{
    Win R;
    win_init(R);
    // Run state: next k, last k, buffered sample (its presence: hb*), head (present: has*).
    int kna = k0 + 1, knb = ks + 1;
    const int ea = ks - 1, eb = k1;
    float baw, bav, bbw, bbv, haw, hav, hbw, hbv, sw, sv;
    int bap, bbp, hap, hbp, sp;
    bool hba = true, hbb = true, has_a = true, has_b = true;
    sample(L, k0, baw, bav, bap);
    sample(L, ks, bbw, bbv, bbp);
    if (kna <= ea) {
        sample(L, kna++, sw, sv, sp);
        if (sw < baw) { haw = sw; hav = sv; hap = sp; }
        else { haw = baw; hav = bav; hap = bap; baw = sw; bav = sv; bap = sp; }
    } else {
        haw = baw; hav = bav; hap = bap;
        hba = false;
    }
    if (knb <= eb) {
        sample(L, knb++, sw, sv, sp);
        if (sw < bbw) { hbw = sw; hbv = sv; hbp = sp; }
        else { hbw = bbw; hbv = bbv; hbp = bbp; bbw = sw; bbv = sv; bbp = sp; }
    } else {
        hbw = bbw; hbv = bbv; hbp = bbp;
        hbb = false;
    }
#define OCC_MSTEP(J)                                                                 \
    {                                                                                \
        if (!(has_a || has_b)) break;                                                \
        const bool ta = has_a && (!has_b || haw <= hbw);                             \
        const float ew = ta ? haw : hbw, ev = ta ? hav : hbv;                        \
        const int ep = ta ? hap : hbp;                                               \
        int kn = ta ? kna : knb;                                                     \
        const int ke = ta ? ea : eb;                                                 \
        bool hbuf = ta ? hba : hbb;                                                  \
        float bw = ta ? baw : bbw, bv = ta ? bav : bbv;                              \
        int bp = ta ? bap : bbp;                                                     \
        float nw = bw, nv = bv;                                                      \
        int np = bp;                                                                 \
        bool has = false;                                                            \
        if (kn <= ke) {                                                              \
            sample(L, kn, sw, sv, sp);                                               \
            kn++;                                                                    \
            const bool sb = sw < bw;                                                 \
            if (sb) { nw = sw; nv = sv; np = sp; }                                   \
            else { bw = sw; bv = sv; bp = sp; }                                      \
            has = true;                                                              \
        } else if (hbuf) {                                                           \
            hbuf = false;                                                            \
            has = true;                                                              \
        }                                                                            \
        if (ta) {                                                                    \
            kna = kn; hba = hbuf; baw = bw; bav = bv; bap = bp;                      \
            haw = nw; hav = nv; hap = np; has_a = has;                               \
        } else {                                                                     \
            knb = kn; hbb = hbuf; bbw = bw; bbv = bv; bbp = bp;                      \
            hbw = nw; hbv = nv; hbp = np; has_b = has;                               \
        }                                                                            \
        win_push<J>(R, ew, ev, ep, zeta, beta, sO, L.sh, hit);                             \
    }
    for (;;) {
        OCC_MSTEP(0)
        OCC_MSTEP(1)
        OCC_MSTEP(2)
        OCC_MSTEP(3)
    }
#undef OCC_MSTEP
    win_flush(R, sO, L.sh, hit);
}

// First and last k of a scan line inside its digital line of n positions: tab is monotone, so the samples inside
// form one interval of k around k = h (the candidate itself).
__device__ __forceinline__ void strip_range(const int16_t* tab, int h, int tc, int n, int& k0, int& k1)
{
    auto inside = [&](int k) { return (unsigned)(tc + __ldg(tab + k)) < (unsigned)n; };
    int lo = 0, hi = h;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (inside(m)) hi = m; else lo = m + 1;
    }
    k0 = lo;
    lo = h;
    hi = 2 * h;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (inside(m)) lo = m; else hi = m - 1;
    }
    k1 = lo;
}

// The 16 bytes before D_r: a sample read ahead of a line's end (never used) may land there.
__device__ __forceinline__ void smem_guard_init(unsigned char* smem)
{
    reinterpret_cast<uint4*>(smem)[0] = make_uint4(0, 0, 0, 0);
}

// Block-wide inclusive scan of one value per thread (kStripThreads threads); *total gets the sum.
__device__ __forceinline__ uint32_t block_scan(uint32_t x, uint32_t* s_warp, uint32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFullMask, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kStripWarps; w++) {
        const uint32_t t = s_warp[w];
        if (w < warp) before += t;
        all += t;
    }
    __syncthreads();
    *total = all;
    return x + before;
}

// One strip (index sid over the call's strips) of the strip kernel, run by the whole block; frames: the call's frame
// records.  kFused (the fused kernel): the lines of three or more macro-runs are kept in shared memory and published
// after the strip's O is written, for the worker blocks; the rest go to the views' lists, as in k_strip.
template <bool kHits, bool kFused>
__device__ __forceinline__ void strip_run(const Args& a, const FrameArg* frames, uint32_t sid)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_warp[kStripWarps];
    __shared__ uint32_t s_n1, s_n2, s_b1, s_cand[2];
    __shared__ unsigned long long s_st[2][2];
    __shared__ uint2 s_many[kStripMany];
    __shared__ uint32_t s_n3;

    const int tid = threadIdx.x, lane = tid & 31;
    // The strip: frame (last with strip0 <= sid), then the groups' strips in group order.
    int f = 0;
    {
        int lo = 0, hi = a.nf - 1;
        while (lo < hi) {
            const int m = (lo + hi + 1) >> 1;
            if (frames[m].strip0 <= sid) lo = m; else hi = m - 1;
        }
        f = lo;
    }
    const FrameArg& F = frames[f];
    const int H = F.H, W = F.W;
    // Fields used in the pixel loops, held in registers (a global record might alias the stores as far as the
    // compiler can tell, and would be read again after each one).
    const float* const Dp = F.D;
    const int64_t pitch = F.pitch;
    const uint8_t* const prop = F.prop;
    const int tiles_x = F.tiles_x;
    uint32_t rem = sid - F.strip0;
    int gi = -1;
    for (int u = 0; u < a.ngroups; u++) {
        const uint32_t ns = (uint32_t)fam_strips(a.group[u].fam, H, W, a.strip_px);
        if (rem < ns) {
            gi = u;
            break;
        }
        rem -= ns;
    }
    if (gi < 0) return;
    const StripGroup grp = a.group[gi];
    const int fam = grp.fam;
    const int nvw = grp.vb >= 0 ? 2 : 1;               // views of the group (same family, same ratio)
    const int vw0 = grp.va, vw1 = grp.vb >= 0 ? grp.vb : grp.va;
    const int h = a.plan[f * a.nv + vw0].h;             // equal for both: same ratio, same L (Eq. 3)
    if (h < 0) return;   // the views were not run (non-finite input or L too long): M and O unspecified
    const ViewArg va = a.view[vw0], vb = a.view[vw1];
    const int len = fam_len(fam, H, W);
    const int B = strip_lines(fam, H, W, a.strip_px);
    const int l0 = (int)rem * B;
    const int nb = min(B, fam_lines(fam, H, W) - l0);
    const float r = va.r;
    const float zeta = a.zeta, beta = a.beta;
    const int64_t plane = (int64_t)H * W;

    // Shared memory: a guard word (a sample read one step ahead of a line's end may fall one position before its
    // first), D_r of the lines, the O words, the candidate bits of each view, the line queue and the round's
    // candidates.  Each view's sample offsets (k = 0 .. 2h + 4) come from its table in global memory (L1).
    float* sV = reinterpret_cast<float*>(smem + 16);                                        // [nb][len]
    uint32_t* sO = reinterpret_cast<uint32_t*>(smem + 16 + (size_t)a.strip_px * 4);         // [nb][len]
    uint32_t* sBits = sO + a.strip_px;                                                      // [2][strip_px / 32]
    uint2* sQ = reinterpret_cast<uint2*>(sBits + 2 * (a.strip_px / 32));                    // [kStripQueue]
    uint32_t* sRaw = reinterpret_cast<uint32_t*>(sQ + kStripQueue);                         // [kStripQueue]
    const int16_t* tabs[2] = {a.stab + (int64_t)va.stab * kSTabLen + (kTabHalf - h),
                              a.stab + (int64_t)vb.stab * kSTabLen + (kTabHalf - h)};

    const int npx = nb * len;   // shared positions of the strip (lines shorter than len leave some unused)
    const int nwords = (npx + 31) >> 5;
    for (int i = tid; i < npx; i += kStripThreads) sO[i] = 0;
    for (int i = tid; i < 2 * nwords; i += kStripThreads) sBits[(i < nwords ? 0 : a.strip_px / 32 - nwords) + i] = 0;
    if (tid < 2) {
        s_cand[tid] = 0;
        s_st[tid][0] = s_st[tid][1] = 0;
    }
    if (tid == 0) {
        smem_guard_init(smem);
        s_n3 = 0;
    }
    __syncthreads();

    // Thread layout of the two pixel passes (staging, output), without divisions per pixel: along rows every thread
    // walks x of each line in turn (coalesced); for the other families the nb lines of the strip lie side by side in
    // a row of the frame, so groups of nb neighbouring threads take one row each, the whole group walking y.
    const int tb = fam == kFamRows ? 0 : tid % nb;
    const int ty = fam == kFamRows ? tid : tid / nb;
    const int ystep = kStripThreads / nb;
    const bool in_grp = fam == kFamRows || ty < ystep;
    int bx0, by0, bay, bn;
    line_geom(fam, H, W, l0 + tb, bx0, by0, bay, bn);
    const int dl = fam == kFamDiag ? (l0 + tb) - (H - 1) : l0 + tb;   // x - y of a diagonal, x + y of an anti-diagonal

    // 1. Stage D_r and evaluate Eq. 1-2 (on D_r, shared by the group's views) for every pixel of the strip, four
    //    pixels of a thread at a time with their twelve loads (D, right and lower neighbours) issued first.
    const int tpv = F.tiles_x * F.tiles_y;
    uint32_t my_cand[2] = {0, 0};
    {
        const bool one = (r == 1.0f);
        auto stage4 = [&](const int (&bq)[4], const int (&xq)[4], const int (&yq)[4], const int (&tq)[4],
                          const bool (&ok)[4]) {
            float d[4], dx[4], dy[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                d[u] = dx[u] = dy[u] = 0.0f;
                if (ok[u]) {
                    const float* row = Dp + (int64_t)yq[u] * pitch + xq[u];
                    d[u] = __ldg(row);
                    if (xq[u] + 1 < W) dx[u] = __ldg(row + 1);
                    if (yq[u] + 1 < H) dy[u] = __ldg(row + pitch);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (!ok[u]) continue;
                const float dr = one ? d[u] : __fmul_rn(r, d[u]);
                const int q = bq[u] * len + tq[u];
                sV[q] = dr;
                const float ex = (xq[u] + 1 < W) ? __fsub_rn(one ? dx[u] : __fmul_rn(r, dx[u]), dr) : 0.0f;
                const float ey = (yq[u] + 1 < H) ? __fsub_rn(one ? dy[u] : __fmul_rn(r, dy[u]), dr) : 0.0f;
                const float e2 = __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey));
                if (!(e2 >= a.e2min)) continue;
                const int tile = (yq[u] / kTile) * tiles_x + xq[u] / kTile;
#pragma unroll
                for (int w = 0; w < 2; w++) {
                    if (w >= nvw) break;
                    const ViewArg& vv = w ? vb : va;
                    bool cand = __fadd_rn(__fmul_rn(ex, vv.c), __fmul_rn(ey, vv.s)) > 0.0f;
                    if (cand && prop) cand = prop[(int64_t)(w ? vw1 : vw0) * tpv + tile] != 0;
                    if (cand) {
                        atomicOr(sBits + w * (a.strip_px / 32) + (q >> 5), 1u << (q & 31));
                        my_cand[w]++;
                    }
                }
            }
        };
        int bq[4], xq[4], yq[4], tq[4];
        bool ok[4];
        if (fam == kFamRows) {
            for (int b = 0; b < nb; b++)
                for (int x0 = tid; x0 < W; x0 += 4 * kStripThreads) {
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        bq[u] = b;
                        xq[u] = x0 + u * kStripThreads;
                        yq[u] = l0 + b;
                        tq[u] = xq[u];
                        ok[u] = xq[u] < W;
                    }
                    stage4(bq, xq, yq, tq, ok);
                }
        } else if (in_grp) {
            for (int y0 = ty; y0 < H; y0 += 4 * ystep) {
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int y = y0 + u * ystep;
                    const int x = fam == kFamCols ? dl : (fam == kFamDiag ? y + dl : dl - y);
                    bq[u] = tb;
                    xq[u] = x;
                    yq[u] = y;
                    tq[u] = fam == kFamCols ? y : (fam == kFamDiag ? y - by0 : x - bx0);
                    ok[u] = y < H && (unsigned)x < (unsigned)W;
                }
                stage4(bq, xq, yq, tq, ok);
            }
        }
    }
    atomicAdd(&s_cand[0], my_cand[0]);
    if (nvw > 1) atomicAdd(&s_cand[1], my_cand[1]);
    __syncthreads();

    unsigned long long acc_n0 = 0, acc_p0 = 0, acc_n1 = 0, acc_p1 = 0;
    // 2-4. Rounds: up to kStripQueue candidates each, the first view's in pixel order, then the second view's.
    const int nw_all = nvw * nwords;
    for (int wc = 0; wc < nw_all;) {
        // Compaction: words wc, wc + 1, ... while the queue has room (a word that does not fit starts the next round).
        uint32_t nraw = 0;
        while (wc < nw_all) {
            const int wi = wc + tid;
            const int w = wi >= nwords ? 1 : 0;
            const int wl = wi - w * nwords;
            const uint32_t word = wi < nw_all ? sBits[w * (a.strip_px / 32) + wl] : 0u;
            const uint32_t c = __popc(word);
            uint32_t total;
            const uint32_t incl = block_scan(c, s_warp, &total);
            const bool fits = nraw + incl <= (uint32_t)kStripQueue;
            if (fits && word) {
                uint32_t pos = nraw + incl - c;
                uint32_t m = word;
                while (m) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1;
                    const int q = wl * 32 + j;
                    const int b = q / len;
                    sRaw[pos++] = ((uint32_t)w << 16) | ((uint32_t)b << 12) | (uint32_t)(q - b * len);
                }
            }
            // Words that fit: a prefix of the sweep (incl is non-decreasing).
            const uint32_t nfit = __syncthreads_count(fits && wi < nw_all);
            uint32_t added = 0;
            if (nfit > 0) {
                // The sum of c over the fitting words is the inclusive count of the last fitting thread.
                if (tid == (int)nfit - 1) s_warp[0] = incl;
                __syncthreads();
                added = s_warp[0];
                __syncthreads();
            }
            nraw += added;
            wc += (int)nfit;
            if (nfit < (uint32_t)kStripThreads) break;   // queue full, or every word taken
        }
        if (nraw == 0) break;

        // 3. Macro-runs of every candidate's scan line.
        if (tid == 0) s_n1 = s_n2 = s_b1 = 0;
        __syncthreads();
        for (uint32_t e = tid; e < nraw; e += kStripThreads) {
            const uint32_t ent = sRaw[e];
            const int w = (int)(ent >> 16), b = (int)((ent >> 12) & 15u), tc = (int)(ent & 4095u);
            int x0, y0, ay, n;
            line_geom(fam, H, W, l0 + b, x0, y0, ay, n);
            const int16_t* tab = w ? tabs[1] : tabs[0];
            int k0, k1, ks;
            strip_range(tab, h, tc, n, k0, k1);
            const LineRef L{sV, tab, b * len + tc, h, w << 4};
            const int runs = detect_runs(L, k0, k1, ks);
            const uint32_t w0 = (ent & 0xFFFFu) | ((uint32_t)k0 << 16) | ((uint32_t)w << 28);
            if (runs == 1) {
                sQ[atomicAdd(&s_n1, 1u)] = make_uint2(w0, (uint32_t)k1);
            } else if (runs == 2) {
                sQ[kStripQueue - 1 - atomicAdd(&s_n2, 1u)] = make_uint2(w0, (uint32_t)k1 | ((uint32_t)ks << 16));
            } else {
                // Three or more macro-runs: listed for the warp kernel k_scan, which adds its counts to O and M; in the
                // fused kernel first kept in the strip's short list (published after O is written), while it has room
                // and the line fits the warp buffers of the workers' shared memory.
                if (kFused && h <= kStripManyMaxH) {
                    const uint32_t i3 = atomicAdd(&s_n3, 1u);
                    if (i3 < (uint32_t)kStripMany) {
                        s_many[i3] = make_uint2(w0, (uint32_t)k1);
                        continue;
                    }
                }
                int x, y;
                line_pixel(fam, x0, y0, ay, tc, x, y);
                const int v = w ? vw1 : vw0;
                const uint32_t i = atomicAdd(&F.hdr[HDR_OVF + v], 1u);   // (rare)
                if ((int64_t)i < F.cap) {
                    F.cand[(int64_t)v * F.cap + i] = ((uint32_t)y << 16) | (uint32_t)x;
                } else {
                    // k_plan has already gathered the frames' status words into the call's: set both.
                    atomicOr(&F.hdr[HDR_STATUS], ST_CAND_OVERFLOW);
                    atomicOr(a.status, ST_CAND_OVERFLOW);
                }
            }
        }
        __syncthreads();

        // 4. Counts: batches of 32 lines per warp from one counter, the one-run lines' batches first, then the
        //    two-run lines'; every batch holds lines of one kind, so the lanes of a warp run the same loop.
        const uint32_t n1 = s_n1, n2 = s_n2;
        const uint32_t nb1 = (n1 + 31) / 32, nbt = nb1 + (n2 + 31) / 32;
        for (;;) {
            uint32_t bi = 0;
            if (lane == 0) bi = atomicAdd(&s_b1, 1u);
            bi = __shfl_sync(kFullMask, bi, 0);
            if (bi >= nbt) break;
            const int pass = bi < nb1 ? 0 : 1;
            const uint32_t e = (pass == 0 ? bi : bi - nb1) * 32 + lane;
            const uint32_t nq = pass == 0 ? n1 : n2;
            if (e < nq) {
                const uint2 q = pass == 0 ? sQ[e] : sQ[kStripQueue - 1 - e];
                const int w = (int)(q.x >> 28);
                const int b = (int)((q.x >> 12) & 15u), tc = (int)(q.x & 4095u);
                const int k0 = (int)((q.x >> 16) & 4095u), k1 = (int)(q.y & 0xFFFFu);
                const LineRef L{sV, w ? tabs[1] : tabs[0], b * len + tc, h, w << 4};
                int hit = 0;
                if (pass == 0) count_stream(L, k0, k1, zeta, beta, sO, hit);
                else count_merge2(L, k0, k1, (int)(q.y >> 16), zeta, beta, sO, hit);
                const int n = k1 - k0 + 1;
                const unsigned long long pc = pair_count(n, 4);
                if (w) {
                    acc_n1 += (unsigned long long)n;
                    acc_p1 += pc;
                } else {
                    acc_n0 += (unsigned long long)n;
                    acc_p0 += pc;
                }
                if (kHits && hit && F.hits) {
                    int x0, y0, ay, nl, x, y;
                    line_geom(fam, H, W, l0 + b, x0, y0, ay, nl);
                    line_pixel(fam, x0, y0, ay, tc, x, y);
                    F.hits[(int64_t)(w ? vw1 : vw0) * tpv + (y / kTile) * tiles_x + x / kTile] = 1;
                }
            }
        }
        __syncthreads();
    }

    // 5. O and M of the strip's views, once; statistics and the candidate counts of the views.
    int32_t* OA = F.O + (int64_t)vw0 * plane;
    uint8_t* MA = F.M + (int64_t)vw0 * plane;
    int32_t* OB = F.O + (int64_t)vw1 * plane;
    uint8_t* MB = F.M + (int64_t)vw1 * plane;
    auto out1 = [&](int b, int x, int y, int t) {
        const uint32_t o = sO[b * len + t];
        const int64_t g = (int64_t)y * W + x;
        OA[g] = (int32_t)(o & 0xFFFFu);
        MA[g] = (o & 0xFFFFu) ? 1 : 0;
        if (nvw > 1) {
            OB[g] = (int32_t)(o >> 16);
            MB[g] = (o >> 16) ? 1 : 0;
        }
    };
    if (fam == kFamRows) {
        for (int b = 0; b < nb; b++)
            for (int x = tid; x < W; x += kStripThreads) out1(b, x, l0 + b, x);
    } else if (in_grp) {
        for (int y = ty; y < H; y += ystep) {
            const int x = fam == kFamCols ? dl : (fam == kFamDiag ? y + dl : dl - y);
            if ((unsigned)x >= (unsigned)W) continue;
            out1(tb, x, y, fam == kFamCols ? y : (fam == kFamDiag ? y - by0 : x - bx0));
        }
    }
    atomicAdd(&s_st[0][0], acc_n0);
    atomicAdd(&s_st[0][1], acc_p0);
    if (nvw > 1) {
        atomicAdd(&s_st[1][0], acc_n1);
        atomicAdd(&s_st[1][1], acc_p1);
    }
    __syncthreads();
    if (tid < nvw) {
        const int v = tid ? vw1 : vw0;
        if (s_st[tid][0]) atomicAdd(&F.stats[2 * v], s_st[tid][0]);
        if (s_st[tid][1]) atomicAdd(&F.stats[2 * v + 1], s_st[tid][1]);
        if (s_cand[tid]) atomicAdd(&F.hdr[HDR_COUNT + v], s_cand[tid]);
    }
    if constexpr (kFused) {
        // 6. The kept lines, published for the workers now that O and M of the strip are written: each in an entry of
        //    the pool reserved for the strip, the launch's tag written last (after a fence).  Entries past the pool's
        //    end go to the views' lists instead, which the workers take once every strip is done.
        const uint32_t n3 = min(s_n3, (uint32_t)kStripMany);
        if (n3 > 0) {
            __shared__ uint32_t s_off;
            if (tid == 0) s_off = atomicAdd(&a.status[CTR_POOL], n3);
            __syncthreads();
            const uint32_t off = s_off;
            for (uint32_t e = tid; e < n3; e += kStripThreads) {
                const uint2 q = s_many[e];
                const int w = (int)(q.x >> 28);
                const int b = (int)((q.x >> 12) & 15u), tc = (int)(q.x & 4095u);
                int x0, y0, ay, nl, x, y;
                line_geom(fam, H, W, l0 + b, x0, y0, ay, nl);
                line_pixel(fam, x0, y0, ay, tc, x, y);
                const int v = w ? vw1 : vw0;
                const uint32_t cw = ((uint32_t)y << 16) | (uint32_t)x;
                const uint64_t j = (uint64_t)off + e;
                if (j < a.fz.pool_cap) {
                    uint4* ent = a.fz.pool + j;
                    ent->x = cw;
                    ent->y = ((uint32_t)f << 8) | (uint32_t)v;
                    __threadfence();
                    *reinterpret_cast<volatile uint32_t*>(&ent->z) = fused_tag(a);
                } else {
                    const uint32_t i = atomicAdd(&F.hdr[HDR_OVF + v], 1u);
                    if ((int64_t)i < F.cap) {
                        F.cand[(int64_t)v * F.cap + i] = cw;
                    } else {
                        atomicOr(&F.hdr[HDR_STATUS], ST_CAND_OVERFLOW);
                        atomicOr(a.status, ST_CAND_OVERFLOW);
                    }
                }
            }
        }
    }
}


// The prefix sums over (frame, view), per size class, of the lines the strips listed (clamped to the list capacity),
// for the warp kernels: one block of T threads, one (frame, view) per thread and iteration.
template <int T>
__device__ __forceinline__ void plan_ovf_block(const Args& a, const FrameArg* frames)
{
    __shared__ uint32_t s_carry[kNumClasses];
    __shared__ uint32_t s_warp[T / 32][kNumClasses];
    const int n = a.nf * a.nv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int stride = n + 1;
    if (threadIdx.x < kNumClasses) s_carry[threadIdx.x] = 0;
    __syncthreads();
    for (int base = 0; base < n; base += T) {
        const int i = base + threadIdx.x;
        uint32_t cnt[kNumClasses] = {0, 0, 0};
        if (i < n) {
            const int f = i / a.nv, v = i - f * a.nv;
            const FrameArg& F = frames[f];
            const PlanEntry pe = a.plan[i];
            if (a.view[v].fam >= 0 && pe.h >= 0) {
                uint32_t c = __ldcg(&F.hdr[HDR_OVF + v]);
                if ((int64_t)c > F.cap) c = (uint32_t)F.cap;
                cnt[pe.cls] = c;
            }
        }
        uint32_t incl[kNumClasses];
#pragma unroll
        for (int c = 0; c < kNumClasses; c++) {
            uint32_t x = cnt[c];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFullMask, x, o);
                if (lane >= o) x += y;
            }
            incl[c] = x;
            if (lane == 31) s_warp[warp][c] = x;
        }
        __syncthreads();
        if (threadIdx.x < kNumClasses) {
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
#pragma unroll
            for (int c = 0; c < kNumClasses; c++) a.pref_ovf[c * stride + i] = s_warp[warp][c] + incl[c] - cnt[c];
        }
        __syncthreads();
    }
    if (threadIdx.x < kNumClasses) a.pref_ovf[threadIdx.x * stride + n] = s_carry[threadIdx.x];
}

// plan_ovf_block for the last strip block, out of line (one block of a launch runs it).
__device__ __noinline__ void strip_plan_ovf(const Args& a)
{
    plan_ovf_block<kStripThreads>(a, a.frames);
}

// k_strip: one strip per block; the block that ends last (a releasing count over the grid) writes the prefix sums of
// the lines the strips listed, for the warp kernels.
template <bool kHits>
__global__ void __launch_bounds__(kStripThreads, 5) k_strip(const __grid_constant__ Args a)
{
    __shared__ int s_last;
    strip_run<kHits, false>(a, a.frames, blockIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(a.status + CTR_STRIPS, 1u) + 1 == gridDim.x;
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last) strip_plan_ovf(a);
}

// ------------------------------------------------------------------------------------------------------------------
// k_fused: the whole call in one launch, for calls whose views all take the strip kernel and that ask for no E, A or
// tile hits.  Blocks take tickets from one counter (CTR_TICKET), in this order:
//   min/max  kFusedQuadsPerTicket quads of one frame's D each (as k_minmax); the block that finishes a frame's last
//            one writes the frame's plan (Eq. 3: L and h per view) and releases it (HDR_READY);
//   strips   strip_run after the frame's plan; its kept lines of three or more macro-runs are published in
//            entries of a pool (the launch's tag written last) once its O and M are written; the block that
//            finishes the last strip writes the prefix sums of the lines in the views' lists (CTR_OVF_READY);
//   workers  one per block: the published lines, one warp each, claimed entry by entry in reservation order (the
//            sort of the warp kernels, counts added to O with global atomics, M set); then, once every strip is done,
//            the listed lines of every size class.
// A ticket waits only for tickets handed out before it, and every such ticket is held by a block that is running and
// waits only for earlier ones, so the launch needs no co-residency: the earliest unfinished ticket always progresses.
// Every wait is bounded (FusedPlan::wait_ns, from %globaltimer, and a spin count); one that gives up sets ST_TIMEOUT
// and CTR_ABORT, and every block then stops at its next wait or ticket.  Data written earlier in the launch is read
// with plain loads after an acquiring wait, never through the read-only cache.

constexpr uint32_t kFusedMaxSpins = 1u << 26;
constexpr int kFusedSmallFrames = 4;   // launch parameters of a call of at most this many frames

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One thread: gives up the launch (timeout) or sees another block's abort.  Returns true to go on waiting, after a
// sleep that grows with the spins (128 ns doubling to 8 us), so that waiting blocks leave the memory system to the
// blocks they wait for.
__device__ __forceinline__ bool fused_keep_waiting(const Args& a, uint64_t t0, uint32_t it)
{
    if (*reinterpret_cast<volatile uint32_t*>(a.status + CTR_ABORT)) return false;
    if ((it & 15u) == 15u && (global_ns() - t0 > a.fz.wait_ns || it > kFusedMaxSpins)) {
        atomicOr(a.status, ST_TIMEOUT);
        atomicExch(a.status + CTR_ABORT, 1u);
        return false;
    }
    __nanosleep(128u << min(it, 6u));
    return true;
}

// One thread: waits until *p >= target, then acquires (fence).  false: the launch gave up.
__device__ __forceinline__ bool fused_wait_geq(const Args& a, const uint32_t* p, uint32_t target)
{
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; it++) {
        if (*reinterpret_cast<const volatile uint32_t*>(p) >= target) {
            __threadfence();
            return true;
        }
        if (!fused_keep_waiting(a, t0, it)) return false;
    }
}

// One thread: marks a ticket done (release) and returns the count before it.
__device__ __forceinline__ uint32_t fused_done(uint32_t* ctr)
{
    __threadfence();
    return atomicAdd(ctr, 1u);
}

// The (frame, view) of a listed line: the last i with pref[i] <= item (plain loads: written in this launch).
__device__ __forceinline__ int fused_owner(const uint32_t* pref, int n, uint32_t item)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (pref[m] <= item) lo = m; else hi = m - 1;
    }
    return lo;
}

// The listed lines of size class CAP, one warp each, from the class's cursor.
template <int CAP>
__device__ __forceinline__ void fused_listed(const Args& a, const FrameArg* frames, ScanSmem<CAP>& S, int cls, int lane,
                                             int& cur_v, unsigned long long& acc_n, unsigned long long& acc_p)
{
    const int nfv = a.nf * a.nv;
    const uint32_t* pref = a.pref_ovf + (int64_t)cls * (nfv + 1);
    const uint32_t total = pref[nfv];
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(a.status + CTR_OVF_CURSOR + cls, 1u);
        item = __shfl_sync(kFullMask, item, 0);
        if (item >= total) break;
        const int i = fused_owner(pref, nfv, item);
        const FrameArg& F = frames[i / a.nv];
        const uint32_t cw = F.cand[(int64_t)(i % a.nv) * F.cap + (item - pref[i])];
        scan_item<CAP>(a, frames, S, lane, i, cw, cur_v, acc_n, acc_p);
    }
}

// One published line for a worker warp (lane 0 decides, the warp gets the result): the next pool entry from the
// claim counter, once it carries this launch's tag.  Returns 1 with the line in *line, 0 when every strip is done and
// no published entry is left, -1 when the launch gave up.
__device__ __forceinline__ int fused_next_published(const Args& a, uint2* line)
{
    const uint32_t epoch = fused_tag(a);
    int res = -1;
    uint2 q = make_uint2(0u, 0u);
    if ((threadIdx.x & 31) == 0) {
        const uint32_t j = atomicAdd(a.status + CTR_CLAIM, 1u);
        const uint64_t t0 = global_ns();
        for (uint32_t it = 0;; it++) {
            if (j < a.fz.pool_cap && *reinterpret_cast<const volatile uint32_t*>(&a.fz.pool[j].z) == epoch) {
                __threadfence();
                q = make_uint2(a.fz.pool[j].x, a.fz.pool[j].y);
                res = 1;
                break;
            }
            // Every strip done: every entry is reserved and written, and one past them (or past the pool) is none.
            if (*reinterpret_cast<const volatile uint32_t*>(a.status + CTR_STRIPS) >= a.strip_total) {
                __threadfence();
                if (j >= a.fz.pool_cap || j >= *reinterpret_cast<const volatile uint32_t*>(a.status + CTR_POOL)) {
                    res = 0;
                    break;
                }
            }
            if (!fused_keep_waiting(a, t0, it)) break;
        }
    }
    res = __shfl_sync(kFullMask, res, 0);
    line->x = __shfl_sync(kFullMask, q.x, 0);
    line->y = __shfl_sync(kFullMask, q.y, 0);
    return res;
}

// A worker block (see k_fused).  smem: the block's dynamic shared memory (bytes), slot: its global warp buffer.
__device__ __noinline__ void fused_worker(const Args& a, const FrameArg* frames, unsigned char* smem, size_t bytes,
                                          unsigned char* slot)
{
    __shared__ int s_got;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int cur_v = -1;
    unsigned long long acc_n = 0, acc_p = 0;
    const int slots0 = min(kStripWarps, (int)(bytes / sizeof(ScanSmem<256>)));
    ScanSmem<256>& S0 = reinterpret_cast<ScanSmem<256>*>(smem)[warp < slots0 ? warp : 0];

    // Published lines, every warp on its own (no block barrier until they are used up).
    bool gave_up = false;
    if (warp < slots0) {
        for (;;) {
            uint2 q;
            const int got = fused_next_published(a, &q);
            if (got <= 0) {
                gave_up = got < 0;
                break;
            }
            const int f = (int)(q.y >> 8), v = (int)(q.y & 255u);
            scan_item<256>(a, frames, S0, lane, f * a.nv + v, q.x, cur_v, acc_n, acc_p);
        }
    }
    if (__syncthreads_or(gave_up)) return;

    // The views' lists, once the last strip has written their prefix sums; size classes in turn.  A class's warps
    // use the shared memory while their buffers fit it, else warp 0 uses the block's global slot.
    if (tid == 0) s_got = fused_wait_geq(a, a.status + CTR_OVF_READY, 1u) ? 1 : 0;
    __syncthreads();
    if (s_got) {
        if (warp < slots0) fused_listed<256>(a, frames, S0, 0, lane, cur_v, acc_n, acc_p);
        __syncthreads();   // the next class's buffers overlap this one's
        const int slots1 = min(kStripWarps, (int)(bytes / sizeof(ScanSmem<1024>)));
        if (warp < slots1) {
            fused_listed<1024>(a, frames, reinterpret_cast<ScanSmem<1024>*>(smem)[warp], 1, lane, cur_v, acc_n, acc_p);
        } else if (slots1 == 0 && warp == 0) {
            fused_listed<1024>(a, frames, *reinterpret_cast<ScanSmem<1024>*>(slot), 1, lane, cur_v, acc_n, acc_p);
        }
        __syncthreads();
        const int slots2 = min(kStripWarps, (int)(bytes / sizeof(ScanSmem<4096>)));
        if (warp < slots2) {
            fused_listed<4096>(a, frames, reinterpret_cast<ScanSmem<4096>*>(smem)[warp], 2, lane, cur_v, acc_n, acc_p);
        } else if (slots2 == 0 && warp == 0) {
            fused_listed<4096>(a, frames, *reinterpret_cast<ScanSmem<4096>*>(slot), 2, lane, cur_v, acc_n, acc_p);
        }
    }
    flush_item_stats(frames, a.nv, lane, cur_v, acc_n, acc_p);
}

// A strip of the fused kernel.
__device__ __forceinline__ void fused_strip(const Args& a, const FrameArg* frames, uint32_t sid)
{
    strip_run<false, true>(a, frames, sid);
}

template <int NF>
__global__ void __launch_bounds__(kStripThreads, 5) k_fused(const __grid_constant__ Args a,
                                                             const __grid_constant__ FusedFrames<NF> fr)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_t;
    __shared__ int s_go;
    __shared__ float s_lo[kStripWarps], s_hi[kStripWarps];
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const FrameArg* frames = fr.f;
    for (;;) {
        if (tid == 0)
            s_t = *reinterpret_cast<volatile uint32_t*>(a.status + CTR_ABORT) ? 0xFFFFFFFFu
                                                                               : atomicAdd(a.status + CTR_TICKET, 1u);
        __syncthreads();
        const uint32_t t = s_t;
        __syncthreads();
        if (t >= a.fz.end) break;
        if (t < a.fz.mm_end) {
            int f = 0;
            {
                int lo = 0, hi = a.nf - 1;
                while (lo < hi) {
                    const int m = (lo + hi + 1) >> 1;
                    if (fr.mm0[m] <= t) lo = m; else hi = m - 1;
                }
                f = lo;
            }
            const FrameArg& F = frames[f];
            const int QW = (F.W + 3) >> 2;
            const int64_t nq = (int64_t)F.H * QW;
            const bool vec = ((F.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(F.D) & 15) == 0);
            const int64_t q0 = (int64_t)(t - fr.mm0[f]) * kFusedQuadsPerTicket;
            const int64_t q1 = min(nq, q0 + kFusedQuadsPerTicket);
            float lo = INFINITY, hi = -INFINITY;
            bool bad = false;
            for (int64_t q = q0 + tid; q < q1; q += kStripThreads) minmax_quad(F.D, F.pitch, F.W, QW, vec, q, lo, hi, bad);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                lo = fminf(lo, __shfl_xor_sync(kFullMask, lo, off));
                hi = fmaxf(hi, __shfl_xor_sync(kFullMask, hi, off));
            }
            if (tid == 0) s_bad = 0;
            __syncthreads();
            if (__any_sync(kFullMask, bad) && lane == 0) s_bad = 1;
            if (lane == 0) {
                s_lo[warp] = lo;
                s_hi[warp] = hi;
            }
            __syncthreads();
            if (tid == 0) {
                float blo = INFINITY, bhi = -INFINITY;
                for (int w = 0; w < kStripWarps; w++) {
                    blo = fminf(blo, s_lo[w]);
                    bhi = fmaxf(bhi, s_hi[w]);
                }
                if (blo <= bhi) {
                    atomicMax(&F.hdr[HDR_MAX], f2ord(bhi));
                    atomicMax(&F.hdr[HDR_NEGMIN], ~f2ord(blo));
                }
                if (s_bad) atomicOr(&F.hdr[HDR_STATUS], ST_NONFINITE);
                const uint32_t before = fused_done(&F.hdr[HDR_MMDONE]);
                s_go = before + 1 == fr.mm0[f + 1] - fr.mm0[f];
                if (s_go) __threadfence();
            }
            __syncthreads();
            if (s_go) {
                // The frame's plan (as k_plan): L and h per view (Eq. 3), the size class of its lines.
                const uint32_t st = *reinterpret_cast<volatile uint32_t*>(&F.hdr[HDR_STATUS]);
                const uint32_t hmax = *reinterpret_cast<volatile uint32_t*>(&F.hdr[HDR_MAX]);
                const uint32_t hneg = *reinterpret_cast<volatile uint32_t*>(&F.hdr[HDR_NEGMIN]);
                for (int v = tid; v < a.nv; v += kStripThreads) {
                    PlanEntry pe{-1, 0, 0u, 0u};
                    if (!(st & ST_NONFINITE)) {
                        const int L = scan_length(a, hmax, hneg, a.view[v].r);
                        if (L < 0) {
                            atomicOr(&F.hdr[HDR_STATUS], ST_SCAN_TOO_LONG);
                            atomicOr(a.status, ST_SCAN_TOO_LONG);
                        } else {
                            F.hdr[HDR_L + v] = (uint32_t)L;
                            pe.h = (L + 1) / 2;
                            const int nk = 2 * pe.h + 1;
                            pe.cls = nk <= 256 ? 0 : (nk <= 1024 ? 1 : 2);   // kClassCap
                        }
                    }
                    a.plan[f * a.nv + v] = pe;
                }
                if (tid == 0 && st) atomicOr(a.status, st);
                __syncthreads();
                if (tid == 0 && !a.fz.hold) {
                    __threadfence();
                    atomicExch(&F.hdr[HDR_READY], 1u);
                }
            }
        } else if (t < a.fz.strip_end) {
            const uint32_t sid = t - a.fz.mm_end;
            if (tid == 0) {
                int lo = 0, hi = a.nf - 1;
                while (lo < hi) {
                    const int m = (lo + hi + 1) >> 1;
                    if (frames[m].strip0 <= sid) lo = m; else hi = m - 1;
                }
                s_go = fused_wait_geq(a, &frames[lo].hdr[HDR_READY], 1u);
            }
            __syncthreads();
            if (!s_go) break;
            fused_strip(a, frames, sid);
            __syncthreads();
            if (tid == 0) {
                s_go = fused_done(a.status + CTR_STRIPS) + 1 == a.strip_total;
                if (s_go) __threadfence();
            }
            __syncthreads();
            if (s_go) {
                plan_ovf_block<kStripThreads>(a, frames);
                __syncthreads();
                if (tid == 0) {
                    __threadfence();
                    atomicExch(a.status + CTR_OVF_READY, 1u);
                }
            }
        } else {
            fused_worker(a, frames, smem, strip_smem_bytes(a.strip_px),
                         a.fz.slots + (size_t)blockIdx.x * sizeof(ScanSmem<4096>));
            break;
        }
    }
    __syncthreads();
    if (tid == 0 && atomicAdd(a.status + CTR_EXIT, 1u) == gridDim.x - 1) atomicAdd(a.status + CTR_EPOCH, 1u);
}

}  // namespace

size_t strip_smem(int strip_px)
{
    return strip_smem_bytes(strip_px);
}

cudaError_t configure_strip()
{
    const int mx = (int)strip_smem(OCC_STRIP_PX_MAX);
    cudaError_t e = cudaFuncSetAttribute(k_strip<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_strip<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fused<kFusedSmallFrames>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fused<kFusedMaxFrames>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return e;
}

size_t fused_slot_bytes()
{
    return sizeof(ScanSmem<4096>);
}

int fused_blocks_per_sm(int strip_px)
{
    // Per strip size (a multiple of 64 up to OCC_STRIP_PX_MAX), computed once: the occupancy does not change.
    static std::atomic<int> cache[OCC_STRIP_PX_MAX / 64 + 1];
    const int key = strip_px / 64;
    if (strip_px <= 0 || strip_px > OCC_STRIP_PX_MAX || strip_px % 64) return 0;
    int b = cache[key].load(std::memory_order_relaxed);
    if (b > 0) return b;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused<kFusedMaxFrames>, kStripThreads,
                                                      strip_smem(strip_px)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cache[key].store(b, std::memory_order_relaxed);
    return b;
}

namespace {
template <int NF>
cudaError_t launch_fused_n(const Args& a, const FrameArg* f, const uint32_t* mm0, int nf, int grid, cudaStream_t st)
{
    FusedFrames<NF> fr;
    std::memset(&fr, 0, sizeof(fr));
    for (int i = 0; i < nf; i++) {
        fr.f[i] = f[i];
        fr.mm0[i] = mm0[i];
    }
    fr.mm0[nf] = mm0[nf];
    k_fused<NF><<<grid, kStripThreads, strip_smem(a.strip_px), st>>>(a, fr);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_fused(const Args& a, const FrameArg* f, const uint32_t* mm0, int nf, int grid, cudaStream_t st)
{
    if (nf < 1 || nf > kFusedMaxFrames || grid < 1) return cudaErrorInvalidValue;
    if (nf <= kFusedSmallFrames) return launch_fused_n<kFusedSmallFrames>(a, f, mm0, nf, grid, st);
    return launch_fused_n<kFusedMaxFrames>(a, f, mm0, nf, grid, st);
}

cudaError_t launch_strip(const Args& a, cudaStream_t st)
{
    if (a.strip_total == 0) return cudaSuccess;
    const size_t sm = strip_smem(a.strip_px);
    if (a.hits) k_strip<true><<<a.strip_total, kStripThreads, sm, st>>>(a);
    else k_strip<false><<<a.strip_total, kStripThreads, sm, st>>>(a);
    return cudaGetLastError();
}


}  // namespace occ
