/*
 * occ_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the fast edge-aware occlusion detection of
 * Sippel, Seiler and Kaup (ICIP 2024), Section 3, written from the paper's equations.  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark call it; the CUDA library shares no code,
 * header, table or helper with it, and the library never calls it.
 *
 * Arithmetic is binary32, round-to-nearest-even, one operation at a time.  The build passes
 * -ffp-contract=off (no fused multiply-add) and no fast-math, so every `a op b` below is fl(a op b).
 * The paper fixes no precision; binary32 is the precision the GPU path decides its integer outputs in.
 *
 * Readings of the paper where its text is silent, ambiguous or garbled (the same list is kept in the
 * design notes):
 *   R1  W = G - V (Section 3, warp of the scan lines): alpha is the direction from the center camera to the
 *       peripheral camera, so center content moves by -r*D along alpha; the candidate rule of Eq. 2 is kept.
 *   R2  The disparity test of Eq. 5 is read as V_p + beta < V_q (p lies behind q by more than beta).
 *   R3  The angle test of Eq. 2, |A - alpha| < pi/2 with A = atan2(E_y, E_x), is evaluated as the sign of the
 *       dot product E_x*cos(alpha) + E_y*sin(alpha) > 0.
 *   R4  Eq. 1 is the forward difference D[x+1] - D[x]; it is 0 on the last column / row.
 *   R5  N (Eq. 5) is a parameter, even and >= 2; default 8.
 *   R6  G = {-h..h} with h = ceil(L/2) = (L+1)/2.
 *   R7  Scan line positions (Eq. 4) are rounded to the nearest pixel, ties away from zero.
 *   R8  Samples outside the image are dropped.
 *   R9  The sort (Section 3) orders by (W ascending, k ascending); -0 equals +0.
 *   R10 Eq. 5's neighbour index runs over sorted positions of the same scan line.
 *   R11 Eq. 6 is applied with OR semantics: O[pixel] accumulates every scan line's count, M = (O > 0).
 *   R12 A peripheral camera with baseline ratio r sees disparity r*D: the method runs on D_r = fl(r*D).
 *   R13 Eq. 3 is L = ceil(2*(max D_r - min D_r)).
 *   R14 x is the column, y the row (pointing down); alpha turns from +x toward +y.
 *   R15 The thresholds are strict, as printed.
 *   R16 Non-finite input is rejected.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_ERR_ARG 1
#define ORA_ERR_NONFINITE 2
#define ORA_ERR_NOMEM 3

typedef struct {
    float gamma; /* edge threshold (Eq. 2) */
    float zeta;  /* distance threshold (Eq. 5) */
    float beta;  /* disparity threshold (Eq. 5) */
    int32_t L;   /* scan length override; <= 0 means Eq. 3 */
    int32_t N;   /* neighbours compared per sorted sample (Eq. 5), even */
} ora_params;

typedef struct {
    int64_t candidates; /* |C| (Eq. 2) */
    int64_t samples;    /* scan line samples inside the image, summed over candidates */
    int64_t pair_tests; /* (p, d) pairs with 0 <= p+d < n, summed over candidates */
    int64_t hits;       /* sum of all O */
    int32_t L;          /* scan length used */
} ora_stats;

/* cos and sin of alpha (degrees) as binary32, evaluated in double after reducing alpha to [0, 45] degrees,
 * so that multiples of 90 degrees give exactly 0 and +-1 and 45 degrees gives fl(sqrt(1/2)) for both. */
void ora_direction(double alpha_deg, float* c_out, float* s_out)
{
    double a = fmod(alpha_deg, 360.0);
    if (a < 0.0) a += 360.0;
    if (a >= 360.0) a -= 360.0;
    int quadrant = (int)(a / 90.0);
    if (quadrant > 3) quadrant = 3;
    double t = a - 90.0 * quadrant; /* [0, 90) */
    double ct, st;
    if (t == 45.0) {
        ct = sqrt(0.5);
        st = ct;
    } else if (t < 45.0) {
        ct = cos(t * (M_PI / 180.0));
        st = sin(t * (M_PI / 180.0));
    } else {
        double u = 90.0 - t;
        ct = sin(u * (M_PI / 180.0));
        st = cos(u * (M_PI / 180.0));
    }
    double c, s;
    switch (quadrant) {
    case 0: c = ct; s = st; break;
    case 1: c = -st; s = ct; break;
    case 2: c = -ct; s = -st; break;
    default: c = st; s = -ct; break;
    }
    *c_out = (float)c;
    *s_out = (float)s;
}

/* D_r[y][x] = fl(r * D[y][x]) (reading R12). */
static float dr(const float* D, int64_t W, int64_t x, int64_t y, float r)
{
    float d = D[y * W + x];
    return r * d;
}

static int all_finite(const float* D, int64_t n)
{
    for (int64_t i = 0; i < n; i++)
        if (!isfinite(D[i])) return 0;
    return 1;
}

/* Eq. 1 and the maps E, A of Section 3 on D itself (r = 1). */
int ora_edges(const float* D, int32_t H, int32_t W, float* E, float* A)
{
    if (H < 1 || W < 1) return ORA_ERR_ARG;
    if (!all_finite(D, (int64_t)H * W)) return ORA_ERR_NONFINITE;
    for (int64_t y = 0; y < H; y++) {
        for (int64_t x = 0; x < W; x++) {
            float d = D[y * W + x];
            float ex = (x + 1 < W) ? D[y * W + x + 1] - d : 0.0f;
            float ey = (y + 1 < H) ? D[(y + 1) * W + x] - d : 0.0f;
            float e2 = ex * ex + ey * ey;
            if (E) E[y * W + x] = sqrtf(e2);
            if (A) A[y * W + x] = atan2f(ey, ex);
        }
    }
    return ORA_OK;
}

/* Eq. 3: L = ceil(2 * (max D_r - min D_r)). */
int32_t ora_scan_length(const float* D, int32_t H, int32_t W, float r)
{
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t y = 0; y < H; y++)
        for (int64_t x = 0; x < W; x++) {
            float v = dr(D, W, x, y, r);
            if (v < mn) mn = v;
            if (v > mx) mx = v;
        }
    float range = mx - mn;
    float twice = range * 2.0f;
    return (int32_t)ceilf(twice);
}

/* Eq. 2 with reading R3: is (x, y) a candidate for direction (c, s) on D_r? */
static int is_candidate(const float* D, int32_t H, int32_t W, int64_t x, int64_t y, float r, float c,
                        float s, float gamma)
{
    float d = dr(D, W, x, y, r);
    float ex = (x + 1 < W) ? dr(D, W, x + 1, y, r) - d : 0.0f;
    float ey = (y + 1 < H) ? dr(D, W, x, y + 1, r) - d : 0.0f;
    float e2 = ex * ex + ey * ey;
    float e = sqrtf(e2);
    float pcx = ex * c;
    float pcy = ey * s;
    float dot = pcx + pcy;
    return e > gamma && dot > 0.0f;
}

typedef struct {
    float w;     /* warped position W_k = g - V_k (reading R1) */
    float v;     /* depth value V_k (Section 3) */
    int32_t k;   /* index along the general scan line G */
    int64_t pix; /* y * W + x of the sample */
} ora_sample;

/* Reading R9: ascending W as a real number, then ascending k. */
static int cmp_sample(const void* pa, const void* pb)
{
    const ora_sample* a = (const ora_sample*)pa;
    const ora_sample* b = (const ora_sample*)pb;
    if (a->w < b->w) return -1;
    if (a->w > b->w) return 1;
    return (a->k > b->k) - (a->k < b->k);
}

/* Eq. 4 (with R6, R7, R8): the samples of the scan line through candidate (cx, cy).  Returns n. */
static int32_t scanline(const float* D, int32_t H, int32_t W, float r, float c, float s, int32_t h,
                        int64_t cx, int64_t cy, ora_sample* out)
{
    int32_t n = 0;
    for (int32_t k = 0; k <= 2 * h; k++) {
        float g = (float)(k - h);
        float tx = c * g;
        float ty = s * g;
        float fx = tx + (float)cx;
        float fy = ty + (float)cy;
        float rx = roundf(fx);
        float ry = roundf(fy);
        if (!(rx >= 0.0f && rx < (float)W && ry >= 0.0f && ry < (float)H)) continue;
        int64_t px = (int64_t)rx, py = (int64_t)ry;
        float v = dr(D, W, px, py, r);
        out[n].v = v;
        out[n].w = g - v;
        out[n].k = k;
        out[n].pix = py * (int64_t)W + px;
        n++;
    }
    return n;
}

/* Eq. 5 on the sorted samples of one scan line, accumulated into O (Eq. 6 with R11). */
static int64_t count_occlusions(const ora_sample* srt, int32_t n, const ora_params* p, int32_t* O,
                                int64_t* pair_tests)
{
    int64_t hits = 0;
    int32_t half = p->N / 2;
    for (int32_t i = 0; i < n; i++) {
        float vb = srt[i].v + p->beta;
        int32_t o = 0;
        for (int32_t d = -half; d <= half; d++) {
            if (d == 0) continue;
            int32_t j = i + d;
            if (j < 0 || j >= n) continue;
            (*pair_tests)++;
            float dw = srt[i].w - srt[j].w;
            if (fabsf(dw) < p->zeta && vb < srt[j].v) o++;
        }
        O[srt[i].pix] += o;
        hits += o;
    }
    return hits;
}

/*
 * The whole method of Section 3 for one view: Eq. 1 -> Eq. 2 -> Eq. 3 -> Eq. 4 -> sort -> Eq. 5 -> Eq. 6.
 * D: [H][W] binary32.  O: [H][W] int32 (overwritten).  M: [H][W] uint8 (overwritten, may be NULL).
 * Only candidates inside [cx0, cx1) x [cy0, cy1) and, when cand_mask is not NULL, with cand_mask[y*W+x] != 0 are
 * processed (pass 0, 0, W, H, NULL for the whole map).  The selection lets a test recompute a window of a large
 * map from the candidates whose scan lines can reach it; it changes no arithmetic.
 */
int ora_detect_view_masked(const float* D, int32_t H, int32_t W, double alpha_deg, float r,
                           const ora_params* p, int32_t cx0, int32_t cy0, int32_t cx1, int32_t cy1,
                           const uint8_t* cand_mask, int32_t* O, uint8_t* M, ora_stats* st)
{
    if (H < 1 || W < 1 || !p || !O) return ORA_ERR_ARG;
    if (p->N < 2 || (p->N % 2) != 0 || !(p->zeta > 0.0f) || !(r > 0.0f) || !isfinite(r)) return ORA_ERR_ARG;
    if (!all_finite(D, (int64_t)H * W)) return ORA_ERR_NONFINITE;

    float c, s;
    ora_direction(alpha_deg, &c, &s);
    int32_t L = p->L > 0 ? p->L : ora_scan_length(D, H, W, r);
    int32_t h = (L + 1) / 2;

    memset(O, 0, sizeof(int32_t) * (size_t)H * (size_t)W);
    ora_sample* buf = (ora_sample*)malloc(sizeof(ora_sample) * (size_t)(2 * (int64_t)h + 1));
    if (!buf) return ORA_ERR_NOMEM;

    ora_stats acc = {0, 0, 0, 0, L};
    if (cx0 < 0) cx0 = 0;
    if (cy0 < 0) cy0 = 0;
    if (cx1 > W) cx1 = W;
    if (cy1 > H) cy1 = H;
    for (int64_t y = cy0; y < cy1; y++) {
        for (int64_t x = cx0; x < cx1; x++) {
            if (cand_mask && !cand_mask[y * (int64_t)W + x]) continue;
            if (!is_candidate(D, H, W, x, y, r, c, s, p->gamma)) continue;
            acc.candidates++;
            int32_t n = scanline(D, H, W, r, c, s, h, x, y, buf);
            acc.samples += n;
            qsort(buf, (size_t)n, sizeof(ora_sample), cmp_sample);
            acc.hits += count_occlusions(buf, n, p, O, &acc.pair_tests);
        }
    }
    free(buf);
    if (M)
        for (int64_t i = 0; i < (int64_t)H * W; i++) M[i] = O[i] > 0 ? 1 : 0;
    if (st) *st = acc;
    return ORA_OK;
}

int ora_detect_view_region(const float* D, int32_t H, int32_t W, double alpha_deg, float r,
                           const ora_params* p, int32_t cx0, int32_t cy0, int32_t cx1, int32_t cy1,
                           int32_t* O, uint8_t* M, ora_stats* st)
{
    return ora_detect_view_masked(D, H, W, alpha_deg, r, p, cx0, cy0, cx1, cy1, NULL, O, M, st);
}

int ora_detect_view(const float* D, int32_t H, int32_t W, double alpha_deg, float r, const ora_params* p,
                    int32_t* O, uint8_t* M, ora_stats* st)
{
    return ora_detect_view_masked(D, H, W, alpha_deg, r, p, 0, 0, W, H, NULL, O, M, st);
}

/* The candidate list of Eq. 2 for one view, in row-major order, as y * W + x.  Returns the count, or -1 if
 * it exceeds cap (the list is then truncated). */
int64_t ora_candidates(const float* D, int32_t H, int32_t W, double alpha_deg, float r, float gamma,
                       int64_t* out, int64_t cap)
{
    float c, s;
    ora_direction(alpha_deg, &c, &s);
    int64_t n = 0;
    for (int64_t y = 0; y < H; y++)
        for (int64_t x = 0; x < W; x++)
            if (is_candidate(D, H, W, x, y, r, c, s, gamma)) {
                if (n < cap) out[n] = y * (int64_t)W + x;
                n++;
            }
    return n > cap ? -1 : n;
}

/* The sorted samples of one candidate's scan line, for tests of the sort and the scan line alone.
 * Writes up to cap entries of (w, v, k, pix) into the four arrays; returns n (or -1 if n > cap). */
int32_t ora_scanline_sorted(const float* D, int32_t H, int32_t W, double alpha_deg, float r, int32_t L,
                            int32_t cx, int32_t cy, float* w, float* v, int32_t* k, int64_t* pix, int32_t cap)
{
    float c, s;
    ora_direction(alpha_deg, &c, &s);
    int32_t h = (L + 1) / 2;
    ora_sample* buf = (ora_sample*)malloc(sizeof(ora_sample) * (size_t)(2 * (int64_t)h + 1));
    if (!buf) return -1;
    int32_t n = scanline(D, H, W, r, c, s, h, cx, cy, buf);
    qsort(buf, (size_t)n, sizeof(ora_sample), cmp_sample);
    if (n <= cap)
        for (int32_t i = 0; i < n; i++) {
            w[i] = buf[i].w;
            v[i] = buf[i].v;
            k[i] = buf[i].k;
            pix[i] = buf[i].pix;
        }
    free(buf);
    return n <= cap ? n : -1;
}

/*
 * Pixel-wise median of n disparity maps (Section 4.2: the stereo disparities of the peripheral cameras fused into
 * one center map).  maps: n pointers to [H][W].  Readings: for even n the median is the mean of the two middle
 * order statistics, fl(a + b) * 0.5 (the paper names a median and gives no rule for an even count); a zero of
 * either sign enters as +0 (fl(v + 0) maps -0 to +0), so the result does not depend on how equal keys are ordered;
 * non-finite input is rejected, as for the detection.
 */
static int cmp_float(const void* pa, const void* pb)
{
    float a = *(const float*)pa, b = *(const float*)pb;
    return (a > b) - (a < b);
}

int ora_median(const float* const* maps, int32_t n, int32_t H, int32_t W, float* out)
{
    if (n < 1 || n > 64 || H < 1 || W < 1) return ORA_ERR_ARG;
    float v[64];
    for (int64_t i = 0; i < (int64_t)H * W; i++) {
        for (int32_t m = 0; m < n; m++) {
            v[m] = maps[m][i] + 0.0f;
            if (!isfinite(v[m])) return ORA_ERR_NONFINITE;
        }
        qsort(v, (size_t)n, sizeof(float), cmp_float);
        if (n & 1) {
            out[i] = v[n / 2];
        } else {
            float s = v[n / 2 - 1] + v[n / 2];
            out[i] = s * 0.5f;
        }
    }
    return ORA_OK;
}

/*
 * Backward warp of one peripheral view into the center view (Section 1: the registration step whose occluded pixels
 * the mask marks).  The center pixel (x, y) of disparity d = fl(r D[y][x]) was seen by the peripheral camera at
 * (x - cos(alpha) d, y - sin(alpha) d) (reading R1: content moves by -r D along alpha); its value is the bilinear
 * interpolation of the peripheral image there, evaluated as
 *   top = I00 + fx (I01 - I00), bottom = I10 + fx (I11 - I10), value = top + fy (bottom - top)
 * with one binary32 rounding per operation.  Pixels marked in M (occluded) and positions outside
 * [0, W-1] x [0, H-1] get 0.  img: [H][W] binary32.  M: [H][W] uint8 or NULL.  out: [H][W].
 */
int ora_warp_view(const float* D, int32_t H, int32_t W, double alpha_deg, float r, const float* img,
                  const uint8_t* M, float* out)
{
    if (H < 1 || W < 1 || !(r > 0.0f)) return ORA_ERR_ARG;
    float c, s;
    ora_direction(alpha_deg, &c, &s);
    for (int64_t y = 0; y < H; y++) {
        for (int64_t x = 0; x < W; x++) {
            int64_t i = y * W + x;
            out[i] = 0.0f;
            if (M && M[i]) continue;
            float d = r * D[i];
            float dx = c * d;
            float dy = s * d;
            float sx = (float)x - dx;
            float sy = (float)y - dy;
            if (!(sx >= 0.0f && sx <= (float)(W - 1) && sy >= 0.0f && sy <= (float)(H - 1))) continue;
            float fx0 = floorf(sx), fy0 = floorf(sy);
            int64_t x0 = (int64_t)fx0, y0 = (int64_t)fy0;
            int64_t x1 = x0 + 1 < W ? x0 + 1 : x0;
            int64_t y1 = y0 + 1 < H ? y0 + 1 : y0;
            float fx = sx - fx0;
            float fy = sy - fy0;
            float i00 = img[y0 * W + x0], i01 = img[y0 * W + x1];
            float i10 = img[y1 * W + x0], i11 = img[y1 * W + x1];
            float top = i00 + fx * (i01 - i00);
            float bot = i10 + fx * (i11 - i10);
            out[i] = top + fy * (bot - top);
        }
    }
    return ORA_OK;
}
