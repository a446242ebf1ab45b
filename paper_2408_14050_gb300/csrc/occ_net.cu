// occ_net.cu -- the learned tile proposer: a four-layer 3x3 convolutional network (bf16 operands, fp32 accumulation)
// that scores, for every 32x32 tile of the center disparity map D and every peripheral view, whether the scan lines
// of the tile's candidates (Eq. 2, Eq. 4) find an occlusion (Eq. 5-6).  It is a concrete form of the paper's closing
// remark (Section 5) that thinning the candidate list would cut the runtime further; occ_detect_batched_tiles skips
// the tiles it rules out.  Network, loss and the rounding points of the stored tensors are stated in include/occ.h.
//
// Kernels:
//   k_prep     D -> x0 (NHWC bf16, 8 channels: fl(D / 32) - 1 in channel 0)
//   k_conv_tma 3x3 'same' convolution as an implicit GEMM on the 5th-generation tensor cores, for c_in >= 16: a CTA
//              computes a 16 x 8 block of output pixels (M = 128) for all output channels (N = 16 or 32).  TMA
//              (cp.async.bulk.tensor) brings the 18 x 10 pixel halo of the block into shared memory, one copy per
//              8 channels, laid out so that the 8 pixels of an output row form one canonical K-major core matrix:
//              every tap is then the same halo read at a shifted start address (SBO = one halo row), and one thread
//              issues 9 x c_in / 16 tcgen05.mma (kind::f16, bf16 x bf16 -> fp32, accumulator in tensor memory)
//              without any im2col copy.  The epilogue reads the accumulator with tcgen05.ld and applies bias, ReLU
//              or a ReLU gate before rounding to bf16.  The forward layers and the input-gradient (dgrad) pass both
//              use it: dgrad is the same convolution of the output gradient with the taps mirrored and the channel
//              roles swapped.
//   k_conv     the same convolution for the 8-channel input layer, gathering im2col rows into shared memory (a tap
//              is a single 8-channel chunk there, so taps cannot be addressed as shifted halo reads).
//   k_wgrad    weight gradient dW[co][tap][ci] = sum_p dY[p][co] X[p + tap][ci] (and the bias gradient, through a
//              row of ones) as a GEMM with M = (tap, ci), N = co, K = pixels on the tensor cores; the CTA transposes
//              8x8 blocks of the NHWC tensors into K-major core matrices, accumulates 128-pixel stages in tensor
//              memory, and adds its partial sums to the fp32 result with atomics (split over pixels).
//   k_head     per tile: the view code g(v) = We (cos a, sin a, r) + be, pixel scores z = a4 . g(v) + b0, the
//              log-sum-exp pooled tile logit; in training also the loss, dz, the gate of a4 and the head gradients.
//   k_pack / k_adam / k_weights   gradient layout, Adam update of the fp32 master parameters, bf16 operand copies.
//
// Every wait on the tensor cores is bounded (about two seconds of %globaltimer); on expiry the kernel records an
// error, waits once more (bounded) for the outstanding MMA, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <mutex>

#include "occ.h"

namespace {

constexpr int kTile = OCC_TILE;
constexpr int kNumLayers = 4;
__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? 8 : l == 1 ? 16 : l == 2 ? 16 : 32; }
__host__ __device__ constexpr int cout_of(int l) { return l == 0 ? 16 : l == 1 ? 16 : l == 2 ? 32 : 16; }
constexpr int kFeat = 16;
constexpr int kEnc = 3;
constexpr int kMaxViews = OCC_MAX_VIEWS;
constexpr int kHeadThreads = 256;
constexpr int kConvThreads = 128;
constexpr int kWgradStagesPerCta = 16;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kGuard = 0;       // shared memory past the operands (the descriptors read only inside them)

__host__ __device__ constexpr int kpad(int cin) { return ((9 * cin + 15) / 16) * 16; }

// Offsets of the parameter blocks in the flat vector (conv weights [co][9][ci], bias [co] per layer; We [16][3],
// be [16], b0).
struct ParamLayout {
    int w[kNumLayers], b[kNumLayers];
    int we, be, b0, total;
};

__host__ __device__ constexpr ParamLayout param_layout()
{
    ParamLayout L{};
    int off = 0;
    for (int l = 0; l < kNumLayers; l++) {
        L.w[l] = off;
        off += cout_of(l) * 9 * cin_of(l);
        L.b[l] = off;
        off += cout_of(l);
    }
    L.we = off;
    off += kFeat * kEnc;
    L.be = off;
    off += kFeat;
    L.b0 = off;
    off += 1;
    L.total = off;
    return L;
}

static_assert(param_layout().total == OCC_NET_PARAMS, "parameter count");

__device__ int g_net_error;   // 1: a bounded wait on the tensor cores expired

// ------------------------------------------------------------------------------------------------------------------
// PTX helpers: shared-memory addresses, mbarriers, tensor memory, tcgen05.

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete; false if about kWaitNs passed first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase)
{
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, phase))
        if (globaltimer() - t0 > kWaitNs) return false;
    return true;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Whole warp: allocate `cols` columns of tensor memory (power of two >= 32); the address lands in *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t addr, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(addr), "r"(cols) : "memory");
}

// Shared-memory matrix descriptor, canonical layout without swizzling: 8 rows x 16 bytes per core matrix (stored
// contiguously), `lbo` bytes between core matrices adjacent along K, `sbo` bytes between groups of 8 rows.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
    return d;                 // base offset 0, relative LBO, no swizzling
}

// Instruction descriptor of kind::f16: bf16 A and B (both K-major), fp32 accumulator, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4)                        // accumulator format: f32
           | (1u << 7)                      // A format: bf16
           | (1u << 10)                     // B format: bf16
           | ((uint32_t)(N >> 3) << 17)     // N / 8
           | ((uint32_t)(M >> 4) << 24);    // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// TMA: the 4-D box at (c, x, y, n) of the tensor map into shared memory; completion is counted on `bar`.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c, int x, int y, int n, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(x), "r"(y), "r"(n), "r"(smem_u32(bar))
        : "memory");
}

// 16 consecutive fp32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_val(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// 8x8 transpose of 16-bit values: in[j] holds row j (8 values), out[i] receives column i.
__device__ __forceinline__ void transpose8x8(const uint4 (&in)[8], uint4 (&out)[8])
{
    const uint32_t* w = reinterpret_cast<const uint32_t*>(in);   // w[j * 4 + q]: elements 2q, 2q+1 of row j
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int q = i >> 1;
        const uint32_t sel = (i & 1) ? 0x7632u : 0x5410u;
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; k++) o[k] = __byte_perm(w[(2 * k) * 4 + q], w[(2 * k + 1) * 4 + q], sel);
        out[i] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

// ------------------------------------------------------------------------------------------------------------------
// k_conv: implicit-GEMM 3x3 'same' convolution, NHWC bf16 in and out.

struct ConvArgs {
    const uint16_t* X;      // [P][CIN]
    const uint16_t* Wb;     // [COUT][kpad(CIN)]: k = tap * CIN + ci, zero beyond 9 * CIN
    const float* bias;      // [COUT] or null
    const uint16_t* gate;   // [P][COUT] or null: out = gate > 0 ? acc : 0
    uint16_t* Y;            // [P][COUT]
    int n, H, W;
    int relu;
};

template <int CIN, int COUT>
constexpr size_t conv_smem()
{
    // A (128 rows) + B (COUT rows), K = kpad(CIN), plus room for 1024-byte alignment and a guard band.
    return (size_t)kpad(CIN) / 8 * 2048 + (size_t)kpad(CIN) / 8 * COUT * 16 + 1024 + kGuard;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) k_conv(const __grid_constant__ ConvArgs a)
{
    constexpr int KP = kpad(CIN);
    constexpr int KC = KP / 8;            // 16-byte chunks along K
    constexpr uint32_t kLboA = 2048;      // 16 row groups x 128 bytes
    constexpr uint32_t kLboB = COUT * 16;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + KC * 2048;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t HW = (int64_t)a.H * a.W;
    const int64_t P = (int64_t)a.n * HW;
    const int64_t p = (int64_t)blockIdx.x * 128 + tid;   // this thread's output pixel (row of A and of D)

    if (warp == 0) tmem_alloc(&s_tmem, 32);
    if (tid == 0) mbar_init(&s_bar, 1);

    // A: the im2col row of pixel p, chunk kc = 8 channels of one tap.
    const bool pv = p < P;
    int img = 0, y = 0, x = 0;
    if (pv) {
        img = (int)(p / HW);
        const int64_t r = p - (int64_t)img * HW;
        y = (int)(r / a.W);
        x = (int)(r - (int64_t)y * a.W);
    }
#pragma unroll 4
    for (int kc = 0; kc < KC; kc++) {
        uint4 v = make_uint4(0, 0, 0, 0);
        const int k = kc * 8;
        const int tap = k / CIN, c0 = k - tap * CIN;
        if (pv && tap < 9) {
            const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
            if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
                v = __ldg(reinterpret_cast<const uint4*>(a.X + (((int64_t)img * a.H + yy) * a.W + xx) * CIN + c0));
        }
        *reinterpret_cast<uint4*>(sA + kc * 2048 + (tid >> 3) * 128 + (tid & 7) * 16) = v;
    }
    // B: the weights.
    for (int u = tid; u < COUT * KC; u += kConvThreads) {
        const int nrow = u % COUT, kc = u / COUT;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(a.Wb + (int64_t)nrow * KP + kc * 8));
        *reinterpret_cast<uint4*>(sB + kc * kLboB + (nrow >> 3) * 128 + (nrow & 7) * 16) = v;
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = s_tmem;

    if (tid == 0) {
        constexpr uint32_t idesc = idesc_bf16(128, COUT);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll 1
        for (int j = 0; j < KC / 2; j++)
            mma_bf16(tmem, smem_desc(a0 + j * 2 * kLboA, kLboA, 128), smem_desc(b0 + j * 2 * kLboB, kLboB, 128), idesc,
                     j > 0 ? 1u : 0u);
        mma_commit(&s_bar);
    }
    bool ok = mbar_wait_bounded(&s_bar, 0);
    if (!ok) mbar_wait_bounded(&s_bar, 0);   // once more for the outstanding MMA before its memory is freed
    ok = __syncthreads_and(ok);              // uniform across the CTA (tcgen05.ld is warp-collective)
    if (!ok && tid == 0) atomicExch(&g_net_error, 1);
    tc_after_sync();

    if (ok) {
        float acc[COUT];
#pragma unroll
        for (int c = 0; c < COUT; c += 16) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, acc + c);
        if (pv) {
            uint16_t gv[COUT];
            if (a.gate) {
#pragma unroll
                for (int c = 0; c < COUT; c += 8) {
                    const uint4 g = __ldg(reinterpret_cast<const uint4*>(a.gate + p * COUT + c));
                    const uint16_t* gh = reinterpret_cast<const uint16_t*>(&g);
#pragma unroll
                    for (int i = 0; i < 8; i++) gv[c + i] = gh[i];
                }
            }
            uint32_t outw[COUT / 2];
#pragma unroll
            for (int c = 0; c < COUT; c += 2) {
                float v0 = acc[c], v1 = acc[c + 1];
                if (a.bias) {
                    v0 = __fadd_rn(v0, __ldg(a.bias + c));
                    v1 = __fadd_rn(v1, __ldg(a.bias + c + 1));
                }
                if (a.relu) {
                    v0 = fmaxf(v0, 0.0f);
                    v1 = fmaxf(v1, 0.0f);
                }
                if (a.gate) {
                    // bf16 bit patterns of positive values are positive int16 values other than 0.
                    if ((int16_t)gv[c] <= 0) v0 = 0.0f;
                    if ((int16_t)gv[c + 1] <= 0) v1 = 0.0f;
                }
                outw[c / 2] = (uint32_t)bf16_bits(v0) | ((uint32_t)bf16_bits(v1) << 16);
            }
#pragma unroll
            for (int c = 0; c < COUT / 2; c += 4)
                *reinterpret_cast<uint4*>(a.Y + p * COUT + 2 * c) = make_uint4(outw[c], outw[c + 1], outw[c + 2],
                                                                               outw[c + 3]);
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, 32);
}

// ------------------------------------------------------------------------------------------------------------------
// k_conv_tma: the convolution for c_in in {16, 32} on a 16 x 8 output block with a TMA-loaded halo.

constexpr int kBlkH = 16, kBlkW = 8;                              // output block (M = 128 pixels, row-major)
constexpr int kHaloH = kBlkH + 2, kHaloW = kBlkW + 2;             // 18 x 10 input pixels
constexpr uint32_t kHaloBytes = kHaloH * kHaloW * 16;             // one 8-channel plane: 2880 bytes
constexpr uint32_t kPlane = (kHaloBytes + 127) / 128 * 128;       // plane stride (TMA destinations are 128-aligned)

template <int CIN, int COUT>
constexpr size_t conv_tma_smem()
{
    return 2 * (size_t)(CIN / 8) * kPlane + (size_t)kpad(CIN) / 8 * COUT * 16 + 1024 + kGuard;
}

// Persistent: a CTA loads the weights once and walks output blocks b = blockIdx.x, + gridDim.x, ...; the halo of
// the next block is loaded (TMA, second buffer) while the current block's MMAs and epilogue run.
template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) k_conv_tma(const __grid_constant__ CUtensorMap xmap,
                                                          const __grid_constant__ ConvArgs a)
{
    static_assert(CIN % 16 == 0, "two 8-channel planes per MMA");
    constexpr int KP = kpad(CIN);
    constexpr int KC = KP / 8;
    constexpr int NPL = CIN / 8;
    constexpr uint32_t kLboB = COUT * 16;
    constexpr uint32_t kHalo = NPL * kPlane;   // one halo buffer
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t s_bar[3];   // 0, 1: halo buffer loaded; 2: MMAs of the current block done
    __shared__ uint32_t s_tmem;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;                    // 2 x [NPL][18][10][16 B]
    uint8_t* sB = smem + 2 * kHalo;        // [KC][COUT][16 B]

    const int tid = threadIdx.x, warp = tid >> 5;
    const int bx_n = (a.W + kBlkW - 1) / kBlkW, by_n = (a.H + kBlkH - 1) / kBlkH;
    const int nblk = bx_n * by_n * a.n;
    auto block_xy = [&](int b, int& x0, int& y0, int& img) {
        img = b / (bx_n * by_n);
        const int r = b - img * bx_n * by_n;
        y0 = (r / bx_n) * kBlkH;
        x0 = (r - (r / bx_n) * bx_n) * kBlkW;
    };
    auto load_halo = [&](int b, int buf) {
        int x0, y0, img;
        block_xy(b, x0, y0, img);
        mbar_expect_tx(&s_bar[buf], NPL * kHaloBytes);
#pragma unroll
        for (int pl = 0; pl < NPL; pl++)
            tma_load_4d(sA + buf * kHalo + pl * kPlane, &xmap, pl * 8, x0 - 1, y0 - 1, img, &s_bar[buf]);
    };

    if (warp == 0) tmem_alloc(&s_tmem, 32);
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_init(&s_bar[2], 1);
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&xmap)) : "memory");
    }
    __syncthreads();
    // Halo loads issued into / waited for in each buffer (every thread keeps the same counts: the conditions are
    // uniform).  A buffer is loaded again only after its previous load was waited for, so at most one is in flight.
    int issued[2] = {0, 0}, consumed[2] = {0, 0};
    if ((int)blockIdx.x < nblk) {
        if (tid == 0) load_halo(blockIdx.x, 0);
        issued[0]++;
    }
    if ((int)(blockIdx.x + gridDim.x) < nblk) {
        if (tid == 0) load_halo(blockIdx.x + gridDim.x, 1);
        issued[1]++;
    }
    for (int u = tid; u < COUT * KC; u += kConvThreads) {
        const int nrow = u % COUT, kc = u / COUT;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(a.Wb + (int64_t)nrow * KP + kc * 8));
        *reinterpret_cast<uint4*>(sB + kc * kLboB + (nrow >> 3) * 128 + (nrow & 7) * 16) = v;
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = s_tmem;
    float bias[COUT];
#pragma unroll
    for (int c = 0; c < COUT; c++) bias[c] = a.bias ? __ldg(a.bias + c) : 0.0f;

    bool ok = true;
    int it = 0;
    for (int b = blockIdx.x; b < nblk; b += gridDim.x, it++) {
        const int buf = it & 1;
        ok = mbar_wait_bounded(&s_bar[buf], (uint32_t)((it >> 1) & 1));
        ok = __syncthreads_and(ok);
        if (!ok) break;
        consumed[buf]++;
        tc_after_sync();
        if (tid == 0) {
            constexpr uint32_t idesc = idesc_bf16(128, COUT);
            const uint32_t a0 = smem_u32(sA + buf * kHalo), b0 = smem_u32(sB);
#pragma unroll 1
            for (int tap = 0; tap < 9; tap++) {
                const uint32_t shift = (uint32_t)(((tap / 3) * kHaloW + tap % 3) * 16);
#pragma unroll
                for (int j = 0; j < CIN / 16; j++)
                    mma_bf16(tmem, smem_desc(a0 + 2 * j * kPlane + shift, kPlane, kHaloW * 16),
                             smem_desc(b0 + (tap * NPL + 2 * j) * kLboB, kLboB, 128), idesc,
                             (tap > 0 || j > 0) ? 1u : 0u);
            }
            mma_commit(&s_bar[2]);
        }
        ok = mbar_wait_bounded(&s_bar[2], (uint32_t)(it & 1));
        if (!ok) mbar_wait_bounded(&s_bar[2], (uint32_t)(it & 1));
        ok = __syncthreads_and(ok);
        tc_after_sync();
        if (!ok) break;
        // The halo buffer is free again: fetch the block after next into it.
        if (b + 2 * (int)gridDim.x < nblk) {
            if (tid == 0) load_halo(b + 2 * gridDim.x, buf);
            issued[buf]++;
        }

        float acc[COUT];
#pragma unroll
        for (int c = 0; c < COUT; c += 16) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, acc + c);
        int x0, y0, img;
        block_xy(b, x0, y0, img);
        const int y = y0 + (tid >> 3), x = x0 + (tid & 7);
        if (y < a.H && x < a.W) {
            const int64_t p = ((int64_t)img * a.H + y) * a.W + x;
            uint16_t gv[COUT];
            if (a.gate) {
#pragma unroll
                for (int c = 0; c < COUT; c += 8) {
                    const uint4 g = __ldg(reinterpret_cast<const uint4*>(a.gate + p * COUT + c));
                    const uint16_t* gh = reinterpret_cast<const uint16_t*>(&g);
#pragma unroll
                    for (int i = 0; i < 8; i++) gv[c + i] = gh[i];
                }
            }
            uint32_t outw[COUT / 2];
#pragma unroll
            for (int c = 0; c < COUT; c += 2) {
                float v0 = __fadd_rn(acc[c], bias[c]), v1 = __fadd_rn(acc[c + 1], bias[c + 1]);
                if (a.relu) {
                    v0 = fmaxf(v0, 0.0f);
                    v1 = fmaxf(v1, 0.0f);
                }
                if (a.gate) {
                    if ((int16_t)gv[c] <= 0) v0 = 0.0f;
                    if ((int16_t)gv[c + 1] <= 0) v1 = 0.0f;
                }
                outw[c / 2] = (uint32_t)bf16_bits(v0) | ((uint32_t)bf16_bits(v1) << 16);
            }
#pragma unroll
            for (int c = 0; c < COUT / 2; c += 4)
                *reinterpret_cast<uint4*>(a.Y + p * COUT + 2 * c) = make_uint4(outw[c], outw[c + 1], outw[c + 2],
                                                                               outw[c + 3]);
        }
        // Every warp has read the accumulator before the next block's MMAs overwrite it.
        tc_before_sync();
        __syncthreads();
    }
    if (!ok && tid == 0) {
        atomicExch(&g_net_error, 1);
        // Left early: wait (bounded) for the halo loads still in flight, so that no bulk copy writes into this
        // CTA's shared memory after it exits.  A load's completion is phase consumed[buf] of its barrier.
        for (int q = 0; q < 2; q++)
            if (issued[q] > consumed[q]) mbar_wait_bounded(&s_bar[q], (uint32_t)(consumed[q] & 1));
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, 32);
}

// ------------------------------------------------------------------------------------------------------------------
// k_wgrad: dWt[(tap, ci)][co] += sum over this CTA's pixels of X[p + tap][ci] dY[p][co]; row 9 * CIN is the bias
// gradient (a row of ones).  blockIdx.y: 128-row slice of (tap, ci); blockIdx.x: pixel range.

struct WgradArgs {
    const uint16_t* X;     // [P][CIN]
    const uint16_t* dY;    // [P][COUT]
    float* dWt;            // [9 * CIN + 1][COUT], accumulated
    int n, H, W;
    int stages;            // 128-pixel stages per CTA
};

template <int COUT>
constexpr size_t wgrad_smem()
{
    return 16 * 2048 + 16 * COUT * 16 + 1024 + kGuard;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) k_wgrad(const __grid_constant__ WgradArgs a)
{
    constexpr uint32_t kLboA = 2048;      // 16 row groups x 128 bytes per 8-pixel chunk
    constexpr uint32_t kLboB = COUT * 16;
    constexpr int kRows = 9 * CIN + 1;    // weight rows and the bias row
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + 16 * 2048;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t HW = (int64_t)a.H * a.W;
    const int64_t P = (int64_t)a.n * HW;
    const int row0 = blockIdx.y * 128;

    if (warp == 0) tmem_alloc(&s_tmem, 32);
    if (tid == 0) mbar_init(&s_bar, 1);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = s_tmem;

    auto pixel = [&](int64_t q, int& img, int& y, int& x) {
        img = (int)(q / HW);
        const int64_t r = q - (int64_t)img * HW;
        y = (int)(r / a.W);
        x = (int)(r - (int64_t)y * a.W);
    };

    bool ok = true;
    int issued = 0;
    for (int s = 0; s < a.stages; s++) {
        const int64_t p0 = ((int64_t)blockIdx.x * a.stages + s) * 128;
        if (p0 >= P) break;
        // A: core matrix (row group g, pixel chunk kc) = rows 8g..8g+7 of (tap, ci) x 8 pixels.
        for (int cm = tid; cm < 256; cm += kConvThreads) {
            const int g = cm & 15, kc = cm >> 4;
            const int rg = row0 + 8 * g;     // first (tap, ci) row of the group
            uint4 rows[8];
            if (rg < 9 * CIN) {
                const int tap = rg / CIN, c0 = rg - tap * CIN;
                const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                uint4 px[8];
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    px[j] = make_uint4(0, 0, 0, 0);
                    const int64_t q = p0 + kc * 8 + j;
                    if (q < P) {
                        int img, y, x;
                        pixel(q, img, y, x);
                        const int yy = y + dy, xx = x + dx;
                        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
                            px[j] = __ldg(reinterpret_cast<const uint4*>(
                                a.X + (((int64_t)img * a.H + yy) * a.W + xx) * CIN + c0));
                    }
                }
                transpose8x8(px, rows);
            } else {
#pragma unroll
                for (int i = 0; i < 8; i++) rows[i] = make_uint4(0, 0, 0, 0);
                if (rg == 9 * CIN) {   // the bias row: 1.0 (bf16 0x3F80) for every pixel of the image batch
                    uint32_t w[4];
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const int64_t q = p0 + kc * 8 + 2 * k;
                        w[k] = (q < P ? 0x3F80u : 0u) | (q + 1 < P ? 0x3F800000u : 0u);
                    }
                    rows[0] = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
#pragma unroll
            for (int i = 0; i < 8; i++) *reinterpret_cast<uint4*>(sA + kc * kLboA + g * 128 + i * 16) = rows[i];
        }
        // B: core matrix (channel group cg, pixel chunk kc) = 8 output channels x 8 pixels of dY.
        for (int cm = tid; cm < (COUT / 8) * 16; cm += kConvThreads) {
            const int cg = cm % (COUT / 8), kc = cm / (COUT / 8);
            uint4 px[8], rows[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int64_t q = p0 + kc * 8 + j;
                px[j] = q < P ? __ldg(reinterpret_cast<const uint4*>(a.dY + q * COUT + cg * 8)) : make_uint4(0, 0, 0, 0);
            }
            transpose8x8(px, rows);
#pragma unroll
            for (int i = 0; i < 8; i++) *reinterpret_cast<uint4*>(sB + kc * kLboB + cg * 128 + i * 16) = rows[i];
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
        if (tid == 0) {
            constexpr uint32_t idesc = idesc_bf16(128, COUT);
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll 1
            for (int j = 0; j < 8; j++)
                mma_bf16(tmem, smem_desc(a0 + j * 2 * kLboA, kLboA, 128), smem_desc(b0 + j * 2 * kLboB, kLboB, 128),
                         idesc, (issued > 0 || j > 0) ? 1u : 0u);
            mma_commit(&s_bar);
        }
        // The stage's shared memory is rewritten next: wait for its MMAs.
        ok = mbar_wait_bounded(&s_bar, (uint32_t)(issued & 1));
        if (!ok) mbar_wait_bounded(&s_bar, (uint32_t)(issued & 1));   // once more before giving up
        issued++;
        ok = __syncthreads_and(ok);   // uniform: every thread leaves the loop together
        tc_after_sync();
        if (!ok) {
            if (tid == 0) atomicExch(&g_net_error, 1);
            break;
        }
    }
    tc_after_sync();
    if (ok && issued > 0) {
        float acc[COUT];
#pragma unroll
        for (int c = 0; c < COUT; c += 16) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, acc + c);
        const int row = row0 + tid;
        if (row < kRows) {
#pragma unroll
            for (int c = 0; c < COUT; c++)
                if (acc[c] != 0.0f) atomicAdd(a.dWt + (int64_t)row * COUT + c, acc[c]);
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, 32);
}

// ------------------------------------------------------------------------------------------------------------------
// k_prep: x0 = bf16(fl(D * 1/32) - 1) in channel 0 of 8.

__global__ void k_prep(const float* D, int64_t n_px, uint16_t* x0)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_px; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = __fsub_rn(__fmul_rn(__ldg(D + i), 0.03125f), 1.0f);
        reinterpret_cast<uint4*>(x0)[i] = make_uint4(bf16_bits(v), 0, 0, 0);
    }
}

// ------------------------------------------------------------------------------------------------------------------
// k_head: tile logits (and, with labels, the loss, the head gradients and the gated gradient of a4).

struct HeadArgs {
    const uint16_t* f;         // a4 [n][H][W][16]
    int n, H, W, tx, ty, nv;
    const float* params;       // fp32 master parameters (We, be, b0)
    float enc[kMaxViews][kEnc];
    float* logits;             // [n][nv][ty][tx]
    const uint8_t* labels;     // [n][nv][ty][tx] or null (forward only)
    float pos_weight, inv_count;
    uint16_t* dpre4;           // [n][H][W][16] (training)
    float* grads;              // flat gradient (training): We, be, b0 blocks
    float* loss;               // (training)
};

__device__ __forceinline__ float block_reduce(float v, float* red, bool is_max)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmaxf(v, w) : v + w;
    }
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float r = red[0];
    for (int w = 1; w < kHeadThreads / 32; w++) r = is_max ? fmaxf(r, red[w]) : r + red[w];
    return r;
}

__global__ void __launch_bounds__(kHeadThreads) k_head(const __grid_constant__ HeadArgs a)
{
    constexpr ParamLayout L = param_layout();
    __shared__ float s_g[kMaxViews][kFeat];
    __shared__ float s_red[kHeadThreads / 32];
    __shared__ float s_dg[kMaxViews][kFeat];
    const int t = blockIdx.x, img = blockIdx.y;
    const int i = t / a.tx, j = t - i * a.tx;
    const int y0 = i * kTile, x0 = j * kTile;
    const int th = min(kTile, a.H - y0), tw = min(kTile, a.W - x0);
    const int npx = th * tw;
    const bool train = a.labels != nullptr;

    for (int u = threadIdx.x; u < a.nv * kFeat; u += kHeadThreads) {
        const int v = u / kFeat, c = u - v * kFeat;
        float g = a.params[L.be + c];
        for (int e = 0; e < kEnc; e++) g += a.params[L.we + c * kEnc + e] * a.enc[v][e];
        s_g[v][c] = g;
        s_dg[v][c] = 0.0f;
    }
    __syncthreads();
    const float b0 = a.params[L.b0];

    // This thread's pixels of the tile (up to 4) and their features.
    float f[4][kFeat];
    int64_t pix[4];
    int np = 0;
    for (int q = threadIdx.x; q < npx && np < 4; q += kHeadThreads, np++) {
        const int yy = y0 + q / tw, xx = x0 + q % tw;
        pix[np] = ((int64_t)img * a.H + yy) * a.W + xx;
        const uint4* src = reinterpret_cast<const uint4*>(a.f + pix[np] * kFeat);
        const uint4 u0 = __ldg(src), u1 = __ldg(src + 1);
        const uint16_t* h0 = reinterpret_cast<const uint16_t*>(&u0);
        const uint16_t* h1 = reinterpret_cast<const uint16_t*>(&u1);
#pragma unroll
        for (int c = 0; c < 8; c++) {
            f[np][c] = bf16_val(h0[c]);
            f[np][8 + c] = bf16_val(h1[c]);
        }
    }
    float df[4][kFeat];
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int c = 0; c < kFeat; c++) df[k][c] = 0.0f;
    float loss_acc = 0.0f, db0 = 0.0f;

    for (int v = 0; v < a.nv; v++) {
        float z[4];
        float m = -INFINITY;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            z[k] = -INFINITY;
            if (k < np) {
                float s = 0.0f;
#pragma unroll
                for (int c = 0; c < kFeat; c++) s += f[k][c] * s_g[v][c];
                z[k] = s + b0;
                m = fmaxf(m, z[k]);
            }
        }
        m = block_reduce(m, s_red, true);
        float e[4], se = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            e[k] = k < np ? expf(z[k] - m) : 0.0f;
            se += e[k];
        }
        se = block_reduce(se, s_red, false);
        const float logit = logf(se) + m - logf((float)npx);
        const int64_t li = (((int64_t)img * a.nv + v) * a.ty + i) * a.tx + j;
        if (!train) {
            if (threadIdx.x == 0) a.logits[li] = logit;
            continue;
        }
        if (threadIdx.x == 0 && a.logits) a.logits[li] = logit;
        const float yv = a.labels[li] ? 1.0f : 0.0f;
        const float sig = 1.0f / (1.0f + expf(-logit));
        // -(w y log sig(s) + (1 - y) log(1 - sig(s))) with log sig(s) = -softplus(-s), log(1 - sig(s)) = -softplus(s)
        const float sp_neg = fmaxf(-logit, 0.0f) + log1pf(expf(-fabsf(logit)));
        const float sp_pos = fmaxf(logit, 0.0f) + log1pf(expf(-fabsf(logit)));
        if (threadIdx.x == 0) loss_acc += (a.pos_weight * yv * sp_neg + (1.0f - yv) * sp_pos) * a.inv_count;
        const float ds = (a.pos_weight * yv * (sig - 1.0f) + (1.0f - yv) * sig) * a.inv_count;
        float dgl[kFeat];
#pragma unroll
        for (int c = 0; c < kFeat; c++) dgl[c] = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (k < np) {
                const float dz = ds * e[k] / se;
                db0 += dz;
#pragma unroll
                for (int c = 0; c < kFeat; c++) {
                    df[k][c] += dz * s_g[v][c];
                    dgl[c] += dz * f[k][c];
                }
            }
        }
#pragma unroll
        for (int c = 0; c < kFeat; c++) {
            float r = dgl[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(&s_dg[v][c], r);
        }
    }
    if (!train) return;
    // The gated gradient of a4 (bf16), the head gradients.
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (k < np) {
            uint32_t w[8];
#pragma unroll
            for (int c = 0; c < kFeat; c += 2) {
                const float g0 = f[k][c] > 0.0f ? df[k][c] : 0.0f;
                const float g1 = f[k][c + 1] > 0.0f ? df[k][c + 1] : 0.0f;
                w[c / 2] = (uint32_t)bf16_bits(g0) | ((uint32_t)bf16_bits(g1) << 16);
            }
            uint4* dst = reinterpret_cast<uint4*>(a.dpre4 + pix[k] * kFeat);
            dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
            dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
    }
    float r = db0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(a.grads + L.b0, r);
    if (threadIdx.x == 0) atomicAdd(a.loss, loss_acc);
    __syncthreads();
    for (int u = threadIdx.x; u < kFeat * (kEnc + 1); u += kHeadThreads) {
        const int c = u / (kEnc + 1), e = u - c * (kEnc + 1);
        float s = 0.0f;
        for (int v = 0; v < a.nv; v++) s += s_dg[v][c] * (e < kEnc ? a.enc[v][e] : 1.0f);
        atomicAdd(a.grads + (e < kEnc ? L.we + c * kEnc + e : L.be + c), s);
    }
}

// Inference only, up to kFwdViews views: the same tile logits as k_head with every view's pixel scores kept in
// registers and the max / sum reductions of all views done together (two block barriers in all).
constexpr int kFwdViews = 8;

__global__ void __launch_bounds__(kHeadThreads) k_head_fwd(const __grid_constant__ HeadArgs a)
{
    constexpr ParamLayout L = param_layout();
    constexpr int kWarps = kHeadThreads / 32;
    __shared__ float s_g[kFwdViews][kFeat];
    __shared__ float s_red[kWarps][kFwdViews];
    const int t = blockIdx.x, img = blockIdx.y;
    const int i = t / a.tx, j = t - i * a.tx;
    const int y0 = i * kTile, x0 = j * kTile;
    const int th = min(kTile, a.H - y0), tw = min(kTile, a.W - x0);
    const int npx = th * tw;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (int u = threadIdx.x; u < a.nv * kFeat; u += kHeadThreads) {
        const int v = u / kFeat, c = u - v * kFeat;
        float g = a.params[L.be + c];
        for (int e = 0; e < kEnc; e++) g += a.params[L.we + c * kEnc + e] * a.enc[v][e];
        s_g[v][c] = g;
    }
    __syncthreads();
    const float b0 = a.params[L.b0];

    float z[4][kFwdViews];
    float m[kFwdViews];
#pragma unroll
    for (int v = 0; v < kFwdViews; v++) m[v] = -INFINITY;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int q = threadIdx.x + k * kHeadThreads;
        float f[kFeat];
        const bool ok = q < npx;
        if (ok) {
            const int yy = y0 + q / tw, xx = x0 + q % tw;
            const uint4* src = reinterpret_cast<const uint4*>(a.f + (((int64_t)img * a.H + yy) * a.W + xx) * kFeat);
            const uint4 u0 = __ldg(src), u1 = __ldg(src + 1);
            const uint16_t* h0 = reinterpret_cast<const uint16_t*>(&u0);
            const uint16_t* h1 = reinterpret_cast<const uint16_t*>(&u1);
#pragma unroll
            for (int c = 0; c < 8; c++) {
                f[c] = bf16_val(h0[c]);
                f[8 + c] = bf16_val(h1[c]);
            }
        }
#pragma unroll
        for (int v = 0; v < kFwdViews; v++) {
            float sum = 0.0f;
            if (ok && v < a.nv) {
#pragma unroll
                for (int c = 0; c < kFeat; c++) sum += f[c] * s_g[v][c];
                sum += b0;
            } else {
                sum = -INFINITY;
            }
            z[k][v] = sum;
            m[v] = fmaxf(m[v], sum);
        }
    }
    // Block max of every view.
#pragma unroll
    for (int v = 0; v < kFwdViews; v++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m[v] = fmaxf(m[v], __shfl_xor_sync(0xffffffffu, m[v], o));
    }
    if (lane == 0)
#pragma unroll
        for (int v = 0; v < kFwdViews; v++) s_red[warp][v] = m[v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < kFwdViews; v++) {
        float r = s_red[0][v];
        for (int w = 1; w < kWarps; w++) r = fmaxf(r, s_red[w][v]);
        m[v] = r;
    }
    __syncthreads();
    // Block sum of exp(z - max) of every view.
    float se[kFwdViews];
#pragma unroll
    for (int v = 0; v < kFwdViews; v++) {
        float sv = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; k++) sv += (z[k][v] > -INFINITY) ? expf(z[k][v] - m[v]) : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
        se[v] = sv;
    }
    if (lane == 0)
#pragma unroll
        for (int v = 0; v < kFwdViews; v++) s_red[warp][v] = se[v];
    __syncthreads();
    if (threadIdx.x < a.nv) {
        const int v = threadIdx.x;
        float r = 0.0f;
        for (int w = 0; w < kWarps; w++) r += s_red[w][v];
        a.logits[(((int64_t)img * a.nv + v) * a.ty + i) * a.tx + j] = logf(r) + m[v] - logf((float)npx);
    }
}

// ------------------------------------------------------------------------------------------------------------------
// Parameter kernels.

struct WeightArgs {
    const float* params;
    uint16_t* fwd[kNumLayers];    // [cout][kpad(cin)]
    uint16_t* bwd[kNumLayers];    // [cin][kpad(cout)]: taps mirrored, channel roles swapped (layers 1..3)
};

// bf16 operand copies of the master weights for the forward and the dgrad convolutions.
__global__ void k_weights(const __grid_constant__ WeightArgs a)
{
    constexpr ParamLayout L = param_layout();
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
#pragma unroll
    for (int l = 0; l < kNumLayers; l++) {
        const int ci_n = cin_of(l), co_n = cout_of(l);
        const int kp = kpad(ci_n), kpb = kpad(co_n);
        for (int u = t0; u < co_n * kp; u += st) {
            const int co = u / kp, k = u - co * kp;
            float w = 0.0f;
            if (k < 9 * ci_n) {
                const int tap = k / ci_n, ci = k - tap * ci_n;
                w = a.params[L.w[l] + (co * 9 + tap) * ci_n + ci];
            }
            a.fwd[l][u] = bf16_bits(w);
        }
        if (l == 0) continue;
        for (int u = t0; u < ci_n * kpb; u += st) {
            const int ci = u / kpb, k = u - ci * kpb;
            float w = 0.0f;
            if (k < 9 * co_n) {
                const int tap = k / co_n, co = k - tap * co_n;
                w = a.params[L.w[l] + (co * 9 + (8 - tap)) * ci_n + ci];
            }
            a.bwd[l][u] = bf16_bits(w);
        }
    }
}

struct PackArgs {
    const float* dWt[kNumLayers];   // [9 cin + 1][cout]
    float* grads;
};

// dWt[(tap, ci)][co] -> the flat gradient's [co][tap][ci]; row 9 cin -> the bias block.
__global__ void k_pack(const __grid_constant__ PackArgs a)
{
    constexpr ParamLayout L = param_layout();
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
#pragma unroll
    for (int l = 0; l < kNumLayers; l++) {
        const int ci_n = cin_of(l), co_n = cout_of(l);
        for (int u = t0; u < (9 * ci_n + 1) * co_n; u += st) {
            const int row = u / co_n, co = u - row * co_n;
            const float g = a.dWt[l][u];
            if (row < 9 * ci_n) {
                const int tap = row / ci_n, ci = row - tap * ci_n;
                a.grads[L.w[l] + (co * 9 + tap) * ci_n + ci] = g;
            } else {
                a.grads[L.b[l] + co] = g;
            }
        }
    }
}

struct AdamArgs {
    float* params;
    float* m;
    float* v;
    const float* grads;
    float lr, b1, b2, eps, c1, c2;   // c1 = 1 - b1^t, c2 = 1 - b2^t
    int count;
};

__global__ void k_adam(const __grid_constant__ AdamArgs a)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.count; i += gridDim.x * blockDim.x) {
        const float g = a.grads[i];
        const float m = a.b1 * a.m[i] + (1.0f - a.b1) * g;
        const float v = a.b2 * a.v[i] + (1.0f - a.b2) * g * g;
        a.m[i] = m;
        a.v[i] = v;
        a.params[i] -= a.lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
    }
}

__global__ void k_propose(const float* logits, int64_t n, float threshold, uint8_t* out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = logits[i] > threshold ? 1 : 0;
}

// ------------------------------------------------------------------------------------------------------------------
// Host side.

template <int CIN, int COUT>
cudaError_t conv_attr()
{
    return cudaFuncSetAttribute(k_conv<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)conv_smem<CIN, COUT>());
}

template <int CIN, int COUT>
cudaError_t conv_tma_attr()
{
    return cudaFuncSetAttribute(k_conv_tma<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)conv_tma_smem<CIN, COUT>());
}

template <int CIN, int COUT>
cudaError_t wgrad_attr()
{
    return cudaFuncSetAttribute(k_wgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)wgrad_smem<COUT>());
}

// Once per process and device: the shared-memory opt-ins of the tensor-core kernels.
cudaError_t setup_device()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return e != cudaSuccess ? e : cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    if ((e = conv_attr<8, 16>()) != cudaSuccess || (e = conv_tma_attr<16, 16>()) != cudaSuccess ||
        (e = conv_tma_attr<16, 32>()) != cudaSuccess || (e = conv_tma_attr<32, 16>()) != cudaSuccess ||
        (e = wgrad_attr<8, 16>()) != cudaSuccess || (e = wgrad_attr<16, 16>()) != cudaSuccess ||
        (e = wgrad_attr<16, 32>()) != cudaSuccess || (e = wgrad_attr<32, 16>()) != cudaSuccess)
        return e;
    done[dev] = true;
    return cudaSuccess;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

// Tensor map of an NHWC bf16 tensor [n][H][W][C] with an 8-channel x 10 x 18 box (the halo of one output block);
// coordinates outside the tensor read as zero.
bool halo_map(CUtensorMap* map, const uint16_t* X, int n, int H, int W, int C)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || (reinterpret_cast<uintptr_t>(X) & 15)) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)kHaloW, (cuuint32_t)kHaloH, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t*>(X), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_conv(const ConvArgs& a, int cin, int cout, cudaStream_t st)
{
    const int64_t P = (int64_t)a.n * a.H * a.W;
    if (P == 0) return cudaSuccess;
    if (cin == 8) {
        if (cout != 16) return cudaErrorInvalidValue;
        k_conv<8, 16><<<(unsigned)((P + 127) / 128), kConvThreads, conv_smem<8, 16>(), st>>>(a);
        return cudaGetLastError();
    }
    CUtensorMap map;
    if (!halo_map(&map, a.X, a.n, a.H, a.W, cin)) return cudaErrorInvalidValue;
    // Persistent grid: a few CTAs per SM of the current device, each walking output blocks.
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms < 1)
        sms = 148;
    cudaGetLastError();
    const int64_t nblk = (int64_t)((a.W + kBlkW - 1) / kBlkW) * ((a.H + kBlkH - 1) / kBlkH) * a.n;
    const dim3 grid((unsigned)std::min<int64_t>(nblk, (int64_t)sms * 4));
    if (cin == 16 && cout == 16) k_conv_tma<16, 16><<<grid, kConvThreads, conv_tma_smem<16, 16>(), st>>>(map, a);
    else if (cin == 16 && cout == 32) k_conv_tma<16, 32><<<grid, kConvThreads, conv_tma_smem<16, 32>(), st>>>(map, a);
    else if (cin == 32 && cout == 16) k_conv_tma<32, 16><<<grid, kConvThreads, conv_tma_smem<32, 16>(), st>>>(map, a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_wgrad(WgradArgs a, int cin, int cout, cudaStream_t st)
{
    const int64_t P = (int64_t)a.n * a.H * a.W;
    const int64_t stages = (P + 127) / 128;
    if (stages == 0) return cudaSuccess;
    a.stages = kWgradStagesPerCta;
    const dim3 grid((unsigned)((stages + a.stages - 1) / a.stages), (unsigned)((9 * cin + 1 + 127) / 128));
    if (cin == 8 && cout == 16) k_wgrad<8, 16><<<grid, kConvThreads, wgrad_smem<16>(), st>>>(a);
    else if (cin == 16 && cout == 16) k_wgrad<16, 16><<<grid, kConvThreads, wgrad_smem<16>(), st>>>(a);
    else if (cin == 16 && cout == 32) k_wgrad<16, 32><<<grid, kConvThreads, wgrad_smem<32>(), st>>>(a);
    else if (cin == 32 && cout == 16) k_wgrad<32, 16><<<grid, kConvThreads, wgrad_smem<16>(), st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

bool supported_pair(int cin, int cout)
{
    return (cin == 8 && cout == 16) || (cin == 16 && cout == 16) || (cin == 16 && cout == 32) ||
           (cin == 32 && cout == 16);
}

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    return (int)g;
}

}  // namespace

struct occ_net {
    int device = 0;
    int64_t max_pixels = 0;
    int32_t max_views = 0;
    float* params = nullptr;     // fp32 master [OCC_NET_PARAMS]
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* grads = nullptr;      // scratch gradient
    float* dWt[kNumLayers] = {};
    uint16_t* wf[kNumLayers] = {};
    uint16_t* wb[kNumLayers] = {};
    uint16_t* act[kNumLayers + 1] = {};   // x0, a1..a4 for max_pixels
    uint16_t* dbuf[2] = {};               // pre-activation gradients, up to 32 channels
    void* block = nullptr;
};

namespace {

struct NetGuard {
    int prev = -1;
    bool ok = false;
    explicit NetGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~NetGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool encode_views(const occ_view* views, int32_t n_views, float (*enc)[kEnc])
{
    if (!views || n_views < 1 || n_views > kMaxViews) return false;
    for (int v = 0; v < n_views; v++) {
        const float r = views[v].ratio;
        if (!(r > 0.0f) || !(r <= FLT_MAX)) return false;
        occ_direction(views[v].alpha_deg, &enc[v][0], &enc[v][1]);
        enc[v][2] = r;
    }
    return true;
}

int forward_trunk(occ_net* net, const float* D, int32_t n, int32_t H, int32_t W, cudaStream_t st)
{
    const int64_t P = (int64_t)n * H * W;
    k_prep<<<grid_for(P, 256), 256, 0, st>>>(D, P, net->act[0]);
    if (cudaGetLastError() != cudaSuccess) return OCC_ERR_CUDA;
    constexpr ParamLayout L = param_layout();
    for (int l = 0; l < kNumLayers; l++) {
        ConvArgs a{net->act[l], net->wf[l], net->params + L.b[l], nullptr, net->act[l + 1], n, H, W, 1};
        if (launch_conv(a, cin_of(l), cout_of(l), st) != cudaSuccess) return OCC_ERR_CUDA;
    }
    return OCC_OK;
}

int check_frames(occ_net* net, const float* D, int32_t n, int32_t H, int32_t W)
{
    if (!net || !D || n < 1 || H < 1 || W < 1 || H > OCC_MAX_SIDE || W > OCC_MAX_SIDE) return OCC_ERR_INVALID_ARG;
    if ((int64_t)n * H * W > net->max_pixels) return OCC_ERR_CAPACITY;
    if (reinterpret_cast<uintptr_t>(D) & 3) return OCC_ERR_INVALID_ARG;
    return OCC_OK;
}

}  // namespace

extern "C" {

int occ_net_create(occ_net** out, int device, int64_t max_pixels, int32_t max_views)
{
    if (!out) return OCC_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_pixels < 1 || max_views < 1 || max_views > kMaxViews) return OCC_ERR_INVALID_ARG;
    NetGuard g(device);
    if (!g.ok || setup_device() != cudaSuccess) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    occ_net* net = new occ_net;
    net->device = device;
    net->max_pixels = max_pixels;
    net->max_views = max_views;
    // One allocation: parameters and Adam state, gradient scratch, bf16 weight copies, activations.
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t sz = 4 * al(sizeof(float) * OCC_NET_PARAMS);
    size_t wsz = 0;
    for (int l = 0; l < kNumLayers; l++) {
        sz += al(sizeof(float) * (9 * cin_of(l) + 1) * cout_of(l));
        wsz += al(2 * (size_t)cout_of(l) * kpad(cin_of(l))) + al(2 * (size_t)cin_of(l) * kpad(cout_of(l)));
    }
    sz += wsz;
    size_t asz = al(2 * (size_t)max_pixels * cin_of(0));
    for (int l = 0; l < kNumLayers; l++) asz += al(2 * (size_t)max_pixels * cout_of(l));
    asz += 2 * al(2 * (size_t)max_pixels * 32);
    sz += asz;
    if (cudaMalloc(&net->block, sz) != cudaSuccess) {
        cudaGetLastError();
        delete net;
        return OCC_ERR_CUDA;
    }
    uint8_t* p = static_cast<uint8_t*>(net->block);
    auto take = [&](size_t b) {
        uint8_t* r = p;
        p += al(b);
        return r;
    };
    net->params = reinterpret_cast<float*>(take(sizeof(float) * OCC_NET_PARAMS));
    net->adam_m = reinterpret_cast<float*>(take(sizeof(float) * OCC_NET_PARAMS));
    net->adam_v = reinterpret_cast<float*>(take(sizeof(float) * OCC_NET_PARAMS));
    net->grads = reinterpret_cast<float*>(take(sizeof(float) * OCC_NET_PARAMS));
    for (int l = 0; l < kNumLayers; l++) {
        net->dWt[l] = reinterpret_cast<float*>(take(sizeof(float) * (9 * cin_of(l) + 1) * cout_of(l)));
        net->wf[l] = reinterpret_cast<uint16_t*>(take(2 * (size_t)cout_of(l) * kpad(cin_of(l))));
        net->wb[l] = reinterpret_cast<uint16_t*>(take(2 * (size_t)cin_of(l) * kpad(cout_of(l))));
    }
    net->act[0] = reinterpret_cast<uint16_t*>(take(2 * (size_t)max_pixels * cin_of(0)));
    for (int l = 0; l < kNumLayers; l++) net->act[l + 1] = reinterpret_cast<uint16_t*>(take(2 * (size_t)max_pixels * cout_of(l)));
    net->dbuf[0] = reinterpret_cast<uint16_t*>(take(2 * (size_t)max_pixels * 32));
    net->dbuf[1] = reinterpret_cast<uint16_t*>(take(2 * (size_t)max_pixels * 32));
    if (cudaMemset(net->block, 0, 4 * al(sizeof(float) * OCC_NET_PARAMS)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(net->block);
        delete net;
        return OCC_ERR_CUDA;
    }
    *out = net;
    return OCC_OK;
}

void occ_net_destroy(occ_net* net)
{
    if (!net) return;
    {
        NetGuard g(net->device);
        if (g.ok) cudaFree(net->block);
    }
    delete net;
}

int occ_net_set_params(occ_net* net, const float* params, int64_t count)
{
    if (!net || !params || count != OCC_NET_PARAMS) return OCC_ERR_INVALID_ARG;
    NetGuard g(net->device);
    if (!g.ok) return OCC_ERR_CUDA;
    WeightArgs w{};
    w.params = net->params;
    for (int l = 0; l < kNumLayers; l++) {
        w.fwd[l] = net->wf[l];
        w.bwd[l] = net->wb[l];
    }
    if (cudaMemcpy(net->params, params, sizeof(float) * OCC_NET_PARAMS, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(net->adam_m, 0, sizeof(float) * OCC_NET_PARAMS) != cudaSuccess ||
        cudaMemset(net->adam_v, 0, sizeof(float) * OCC_NET_PARAMS) != cudaSuccess) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    k_weights<<<16, 256>>>(w);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return OCC_ERR_CUDA;
    return OCC_OK;
}

int occ_net_get_params(occ_net* net, float* params, int64_t count)
{
    if (!net || !params || count != OCC_NET_PARAMS) return OCC_ERR_INVALID_ARG;
    NetGuard g(net->device);
    if (!g.ok) return OCC_ERR_CUDA;
    if (cudaMemcpy(params, net->params, sizeof(float) * OCC_NET_PARAMS, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    return OCC_OK;
}

int occ_net_forward(occ_net* net, const float* D, int32_t n, int32_t H, int32_t W, const occ_view* views,
                    int32_t n_views, float* logits, void* stream)
{
    int rc = check_frames(net, D, n, H, W);
    if (rc != OCC_OK) return rc;
    HeadArgs h{};
    if (!logits || n_views > net->max_views || !encode_views(views, n_views, h.enc)) return OCC_ERR_INVALID_ARG;
    NetGuard g(net->device);
    if (!g.ok) return OCC_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if ((rc = forward_trunk(net, D, n, H, W, st)) != OCC_OK) return rc;
    h.f = net->act[kNumLayers];
    h.n = n;
    h.H = H;
    h.W = W;
    h.tx = (W + kTile - 1) / kTile;
    h.ty = (H + kTile - 1) / kTile;
    h.nv = n_views;
    h.params = net->params;
    h.logits = logits;
    if (n_views <= kFwdViews) k_head_fwd<<<dim3((unsigned)(h.tx * h.ty), (unsigned)n), kHeadThreads, 0, st>>>(h);
    else k_head<<<dim3((unsigned)(h.tx * h.ty), (unsigned)n), kHeadThreads, 0, st>>>(h);
    return cudaGetLastError() == cudaSuccess ? OCC_OK : OCC_ERR_CUDA;
}

int occ_net_loss_grad(occ_net* net, const float* D, int32_t n, int32_t H, int32_t W, const occ_view* views,
                      int32_t n_views, const uint8_t* labels, float pos_weight, float* grads, float* loss,
                      float* logits, void* stream)
{
    int rc = check_frames(net, D, n, H, W);
    if (rc != OCC_OK) return rc;
    HeadArgs h{};
    if (!labels || !grads || !loss || n_views > net->max_views || !encode_views(views, n_views, h.enc) ||
        !(pos_weight > 0.0f) || !(pos_weight <= FLT_MAX))
        return OCC_ERR_INVALID_ARG;
    NetGuard g(net->device);
    if (!g.ok) return OCC_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(grads, 0, sizeof(float) * OCC_NET_PARAMS, st) != cudaSuccess ||
        cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    for (int l = 0; l < kNumLayers; l++)
        if (cudaMemsetAsync(net->dWt[l], 0, sizeof(float) * (9 * cin_of(l) + 1) * cout_of(l), st) != cudaSuccess) {
            cudaGetLastError();
            return OCC_ERR_CUDA;
        }
    if ((rc = forward_trunk(net, D, n, H, W, st)) != OCC_OK) return rc;
    h.f = net->act[kNumLayers];
    h.n = n;
    h.H = H;
    h.W = W;
    h.tx = (W + kTile - 1) / kTile;
    h.ty = (H + kTile - 1) / kTile;
    h.nv = n_views;
    h.params = net->params;
    h.logits = logits;
    h.labels = labels;
    h.pos_weight = pos_weight;
    h.inv_count = 1.0f / (float)((int64_t)n * n_views * h.tx * h.ty);
    h.dpre4 = net->dbuf[0];
    h.grads = grads;
    h.loss = loss;
    k_head<<<dim3((unsigned)(h.tx * h.ty), (unsigned)n), kHeadThreads, 0, st>>>(h);
    if (cudaGetLastError() != cudaSuccess) return OCC_ERR_CUDA;
    // Layers 4..1: weight gradient, then (but for the first layer) the gated input gradient.
    int cur = 0;
    for (int l = kNumLayers - 1; l >= 0; l--) {
        WgradArgs w{net->act[l], net->dbuf[cur], net->dWt[l], n, H, W, 0};
        if (launch_wgrad(w, cin_of(l), cout_of(l), st) != cudaSuccess) return OCC_ERR_CUDA;
        if (l == 0) break;
        ConvArgs c{net->dbuf[cur], net->wb[l], nullptr, net->act[l], net->dbuf[cur ^ 1], n, H, W, 0};
        if (launch_conv(c, cout_of(l), cin_of(l), st) != cudaSuccess) return OCC_ERR_CUDA;
        cur ^= 1;
    }
    PackArgs pk{};
    for (int l = 0; l < kNumLayers; l++) pk.dWt[l] = net->dWt[l];
    pk.grads = grads;
    k_pack<<<16, 256, 0, st>>>(pk);
    return cudaGetLastError() == cudaSuccess ? OCC_OK : OCC_ERR_CUDA;
}

int occ_net_adam(occ_net* net, const float* grads, float lr, float beta1, float beta2, float eps, int32_t step,
                 void* stream)
{
    if (!net || !grads || step < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return OCC_ERR_INVALID_ARG;
    NetGuard g(net->device);
    if (!g.ok) return OCC_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    AdamArgs a{net->params, net->adam_m, net->adam_v, grads, lr, beta1, beta2, eps,
               (float)(1.0 - std::pow((double)beta1, step)), (float)(1.0 - std::pow((double)beta2, step)),
               OCC_NET_PARAMS};
    k_adam<<<grid_for(OCC_NET_PARAMS, 256), 256, 0, st>>>(a);
    WeightArgs w{};
    w.params = net->params;
    for (int l = 0; l < kNumLayers; l++) {
        w.fwd[l] = net->wf[l];
        w.bwd[l] = net->wb[l];
    }
    k_weights<<<16, 256, 0, st>>>(w);
    return cudaGetLastError() == cudaSuccess ? OCC_OK : OCC_ERR_CUDA;
}

int occ_net_propose(const float* logits, int64_t count, float threshold, uint8_t* proposal, void* stream)
{
    if (!logits || !proposal || count < 0) return OCC_ERR_INVALID_ARG;
    if (count == 0) return OCC_OK;
    k_propose<<<grid_for(count, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(logits, count, threshold,
                                                                                       proposal);
    return cudaGetLastError() == cudaSuccess ? OCC_OK : OCC_ERR_CUDA;
}

int occ_net_status(void* stream)
{
    int v = 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyFromSymbolAsync(&v, g_net_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    return v ? OCC_ERR_TIMEOUT : OCC_OK;
}

int occ_net_conv3x3(const void* X, int32_t n, int32_t H, int32_t W, int32_t c_in, const void* Wb, const float* bias,
                    int32_t c_out, const void* gate, int32_t relu, void* Y, void* stream)
{
    if (!X || !Wb || !Y || n < 1 || H < 1 || W < 1 || !supported_pair(c_in, c_out)) return OCC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Wb) | reinterpret_cast<uintptr_t>(Y) |
         reinterpret_cast<uintptr_t>(gate)) & 15)
        return OCC_ERR_INVALID_ARG;
    if (setup_device() != cudaSuccess) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    ConvArgs a{static_cast<const uint16_t*>(X), static_cast<const uint16_t*>(Wb), bias,
               static_cast<const uint16_t*>(gate), static_cast<uint16_t*>(Y), n, H, W, relu ? 1 : 0};
    return launch_conv(a, c_in, c_out, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? OCC_OK : OCC_ERR_CUDA;
}

int occ_net_conv3x3_wgrad(const void* X, const void* dY, int32_t n, int32_t H, int32_t W, int32_t c_in,
                          int32_t c_out, float* dWt, void* stream)
{
    if (!X || !dY || !dWt || n < 1 || H < 1 || W < 1 || !supported_pair(c_in, c_out)) return OCC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(dY)) & 15 ||
        (reinterpret_cast<uintptr_t>(dWt) & 3))
        return OCC_ERR_INVALID_ARG;
    if (setup_device() != cudaSuccess) {
        cudaGetLastError();
        return OCC_ERR_CUDA;
    }
    WgradArgs a{static_cast<const uint16_t*>(X), static_cast<const uint16_t*>(dY), dWt, n, H, W, 0};
    return launch_wgrad(a, c_in, c_out, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? OCC_OK
                                                                                               : OCC_ERR_CUDA;
}

}  // extern "C"
