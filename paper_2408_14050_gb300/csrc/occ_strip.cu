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
//      buffer sorts): lines of one macro-run go to one queue, lines of two to another, longer lines to the frame's
//      list for the warp kernel k_scan;
//   4. the lines of each queue are counted in batches of 32 per warp, every lane streaming one line: a plain stream
//      (one run) or the merge of two one-slot buffers (two runs), the sorted samples tested against the N/2 emitted
//      before them (Eq. 5), final counts added to the strip's occlusion sums O in shared memory (Eq. 6);
//   5. it writes O and M = (O > 0) of its lines once, coalesced: no zero fill, no global atomics, no mask pass.
// O of one strip pixel fits 16 bits: at most 2h + 1 <= 4095 scan lines reach a pixel, each with at most two samples
// on it (|cos| or |sin| <= 1 moves a diagonal line by at most one pixel per step) and each sample counts at most
// N = 8 partners, so O <= 65520; two sums share a 32-bit word and are added with 32-bit shared atomics, which cannot
// carry from one half into the other.
//
// Every floating-point operation that decides a candidate, an order or a count is the same round-to-nearest binary32
// operation as in the list path (occ_kernels.cu) and the oracle, so the results are bit-identical.
#include <cstdint>

#include "occ_internal.cuh"

namespace occ {

namespace {

constexpr unsigned kFullMask = 0xFFFFFFFFu;
constexpr int kStripThreads = 128;
constexpr int kStripWarps = kStripThreads / 32;
constexpr int kStripQueue = 512;           // queue entries of one round

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

template <bool kHits>
__global__ void __launch_bounds__(kStripThreads, 5) k_strip(const __grid_constant__ Args a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_warp[kStripWarps];
    __shared__ uint32_t s_n1, s_n2, s_b1, s_cand[2];
    __shared__ unsigned long long s_st[2][2];

    const int tid = threadIdx.x, lane = tid & 31;
    // The strip of this CTA: frame (last with strip0 <= block), then the groups' strips in group order.
    const uint32_t sid = blockIdx.x;
    int f = 0;
    {
        int lo = 0, hi = a.nf - 1;
        while (lo < hi) {
            const int m = (lo + hi + 1) >> 1;
            if (a.frames[m].strip0 <= sid) lo = m; else hi = m - 1;
        }
        f = lo;
    }
    const FrameArg& F = a.frames[f];
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
    const int16_t* tabs[2] = {a.stab + (int64_t)vw0 * kSTabLen + (kTabHalf - h),
                              a.stab + (int64_t)vw1 * kSTabLen + (kTabHalf - h)};

    const int npx = nb * len;   // shared positions of the strip (lines shorter than len leave some unused)
    const int nwords = (npx + 31) >> 5;
    for (int i = tid; i < npx; i += kStripThreads) sO[i] = 0;
    for (int i = tid; i < 2 * nwords; i += kStripThreads) sBits[(i < nwords ? 0 : a.strip_px / 32 - nwords) + i] = 0;
    if (tid < 2) {
        s_cand[tid] = 0;
        s_st[tid][0] = s_st[tid][1] = 0;
    }
    if (tid == 0) smem_guard_init(smem);
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
                // Three or more macro-runs: listed for the warp kernel (k_scan), which adds its counts to O and M.
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
}

// k_plan_ovf: per size class, the prefix sums over (frame, view) of the lines k_strip listed (clamped to the list
// capacity), for k_scan.  One block, one (frame, view) per thread and iteration.
constexpr int kPlanOvfThreads = 1024;

__global__ void __launch_bounds__(kPlanOvfThreads) k_plan_ovf(const __grid_constant__ Args a)
{
    __shared__ uint32_t s_carry[kNumClasses];
    __shared__ uint32_t s_warp[kPlanOvfThreads / 32][kNumClasses];
    const int n = a.nf * a.nv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int stride = n + 1;
    if (threadIdx.x < kNumClasses) s_carry[threadIdx.x] = 0;
    __syncthreads();
    for (int base = 0; base < n; base += kPlanOvfThreads) {
        const int i = base + threadIdx.x;
        uint32_t cnt[kNumClasses] = {0, 0, 0};
        if (i < n) {
            const int f = i / a.nv, v = i - f * a.nv;
            const FrameArg& F = a.frames[f];
            const PlanEntry pe = a.plan[i];
            if (a.view[v].fam >= 0 && pe.h >= 0) {
                uint32_t c = F.hdr[HDR_OVF + v];
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
            for (int w = 0; w < kPlanOvfThreads / 32; w++) {
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

}  // namespace

size_t strip_smem(int strip_px)
{
    return 16 + (size_t)strip_px * 4 + (size_t)strip_px * 4 + (size_t)strip_px / 4 + sizeof(uint2) * kStripQueue +
           sizeof(uint32_t) * kStripQueue;
}

cudaError_t configure_strip()
{
    const int mx = (int)strip_smem(OCC_STRIP_PX_MAX);
    cudaError_t e = cudaFuncSetAttribute(k_strip<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_strip<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return e;
}

cudaError_t launch_strip(const Args& a, cudaStream_t st)
{
    if (a.strip_total == 0) return cudaSuccess;
    const size_t sm = strip_smem(a.strip_px);
    if (a.hits) k_strip<true><<<a.strip_total, kStripThreads, sm, st>>>(a);
    else k_strip<false><<<a.strip_total, kStripThreads, sm, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_plan_ovf(const Args& a, cudaStream_t st)
{
    k_plan_ovf<<<1, kPlanOvfThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace occ
