// Learned proposal net (workload extension; the paper initialises offsets at zero):
// 3x3 convolutions as implicit GEMMs on the tcgen05 tensor cores, bf16 operands, f32
// accumulation in tensor memory.
//
// Activations are NHWC bf16 with 16 or 32 channels (the 4-channel input and 2-channel
// output are zero-padded). A conv tile is 128 consecutive output pixels of one image row
// (the MMA's M), all output channels (N = 16 or 32) and K = 9 taps x C_in. The three
// input rows the tile reads are staged once in shared memory as K-major 16-byte units
// [row][channel chunk][pixel]; the tap (dy, dx) is then just a descriptor start offset of
// dx units into row dy, so no im2col copy is made. Weights are staged once per block in
// the B layout [tap][channel chunk][c_out]. One thread issues the 9 x C_in/16 MMAs, a
// tcgen05.commit arrives on an mbarrier, and the four warps read their 32 accumulator
// rows back with tcgen05.ld for the epilogue (bias + ReLU + bf16; or the ReLU-masked
// input gradient; or the two f32 outputs).
//
// The weight gradient dW[t][i][o] = sum_p x[p + d_t][i] dy[p][o] is a GEMM with the
// pixels as K: its A rows are (tap, input channel) pairs, 4 or 8 taps per 128-row MMA,
// plus one row of ones whose product gives the bias gradient. A 64-pixel K block of the
// three input rows is staged pixel-major and transposed into the K-major layout with
// ldmatrix.trans / stmatrix (one copy per dx shift); the next K block's rows are fetched
// by cp.async into a second buffer meanwhile; the accumulators stay in tensor memory
// across all K blocks of the persistent block and are added to the output with one
// atomic per (row, column) at the end.
#include <cuda.h>
#include <cuda_bf16.h>

#include "sgad_net_device.cuh"
#include "tc5.cuh"

namespace sgad {
namespace net {

constexpr uint32_t kSpinLimit = 1u << 22;   // bounded mbarrier waits (each try_wait may suspend)
constexpr int kTileM = 128;                  // output pixels per conv tile
constexpr int kRowUnits = kTileM + 2;        // staged pixels per input row (1-pixel halo)
constexpr int kKBlock = 64;                  // pixels per weight-gradient K block

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t code)
{
    atomicCAS(status, 0u, code);
}

// ------------------------------------------------------------------ small kernels

// (N,3,H,W) colour + (N,H,W) depth (f32) -> NHWC bf16, 16 channels (R, G, B, D, 0 ...).
__global__ void k_pack_input(const float *__restrict__ rgb, const float *__restrict__ depth, uint4 *__restrict__ x0,
                             int n, int h, int w)
{
    const size_t hw = (size_t)h * w, total = (size_t)n * hw;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const size_t f = p / hw, q = p - f * hw;
        const float *c = rgb + f * 3 * hw + q;
        __nv_bfloat162 rg = __floats2bfloat162_rn(c[0], c[hw]);
        __nv_bfloat162 bd = __floats2bfloat162_rn(c[2 * hw], depth[p]);
        uint4 v0;
        v0.x = *reinterpret_cast<uint32_t *>(&rg);
        v0.y = *reinterpret_cast<uint32_t *>(&bd);
        v0.z = 0u;
        v0.w = 0u;
        x0[2 * p] = v0;
        x0[2 * p + 1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// f32 master weights W[9][ci_p][co_p] -> forward B units [9][ci_p/8][co_p] (unit = 8
// consecutive input channels of one output channel) and, when bwd != nullptr, the
// input-gradient B units [9][co_p/8][ci_p] of the flipped taps (unit = 8 consecutive
// output channels of one input channel).
__global__ void k_prep_weights(const float *__restrict__ w, uint4 *__restrict__ fwd, uint4 *__restrict__ bwd, int ci_p,
                               int co_p)
{
    const int nf = 9 * (ci_p / 8) * co_p, nb = 9 * (co_p / 8) * ci_p;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf) {
        const int co = i % co_p, kc = (i / co_p) % (ci_p / 8), t = i / (co_p * (ci_p / 8));
        uint32_t u[4];
        for (int j = 0; j < 4; ++j) {
            __nv_bfloat162 v = __floats2bfloat162_rn(w[((size_t)t * ci_p + 8 * kc + 2 * j) * co_p + co],
                                                     w[((size_t)t * ci_p + 8 * kc + 2 * j + 1) * co_p + co]);
            u[j] = *reinterpret_cast<uint32_t *>(&v);
        }
        fwd[i] = make_uint4(u[0], u[1], u[2], u[3]);
    }
    if (bwd && i < nb) {
        const int ci = i % ci_p, kc = (i / ci_p) % (co_p / 8), t = i / (ci_p * (co_p / 8));
        const int tf = 8 - t;     // (ky, kx) -> (2 - ky, 2 - kx)
        uint32_t u[4];
        for (int j = 0; j < 4; ++j) {
            __nv_bfloat162 v = __floats2bfloat162_rn(w[((size_t)tf * ci_p + ci) * co_p + 8 * kc + 2 * j],
                                                     w[((size_t)tf * ci_p + ci) * co_p + 8 * kc + 2 * j + 1]);
            u[j] = *reinterpret_cast<uint32_t *>(&v);
        }
        bwd[i] = make_uint4(u[0], u[1], u[2], u[3]);
    }
}

// Training loss mean_p (y0 - delta_t / 0.01)^2 + lw (y1 - logit_t)^2 and its gradient,
// written as the 16-channel bf16 output gradient (channels 0, 1; the rest zero).
__global__ void k_loss(const float2 *__restrict__ y4, const float *__restrict__ td, const float *__restrict__ tl,
                       float lw, uint4 *__restrict__ dy4, float *loss, size_t total)
{
    const float inv = 1.0f / (float)total;
    float acc = 0.f;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const float2 y = y4[p];
        const float e0 = y.x - td[p] * 100.0f, e1 = y.y - tl[p];
        acc += e0 * e0 + lw * e1 * e1;
        __nv_bfloat162 g = __floats2bfloat162_rn(2.0f * e0 * inv, 2.0f * lw * e1 * inv);
        uint4 v = make_uint4(*reinterpret_cast<uint32_t *>(&g), 0u, 0u, 0u);
        dy4[2 * p] = v;
        dy4[2 * p + 1] = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (loss && (threadIdx.x & 31) == 0) atomicAdd(loss, acc * inv);
}

// ------------------------------------------------------------------ conv (forward / input gradient)

template <int CI, int CO>
struct ConvSmem {
    static constexpr int kA = 3 * (CI / 8) * kRowUnits;   // uint4 units
    static constexpr int kB = 9 * (CI / 8) * CO;
    static constexpr size_t bytes = (size_t)(kA + kB) * 16;
};

__device__ __forceinline__ bool bf16_positive(uint32_t half_bits) { return (half_bits & 0x8000u) == 0 && (half_bits & 0x7FFFu) != 0; }

// Epilogue of one output pixel p from its accumulator row r (CO f32 values).
template <int CO, int MODE>
__device__ __forceinline__ void conv_epilogue(const ConvArgs &a, size_t p, const uint32_t (&r)[32])
{
    if (MODE == kModeOut) {
        const float y0 = __uint_as_float(r[0]) + a.bias[0], y1 = __uint_as_float(r[1]) + a.bias[1];
        a.y4[p] = make_float2(y0, y1);
        if (a.delta) a.delta[p] = 0.01f * y0;
        if (a.logit) a.logit[p] = y1;
    } else {
        uint32_t packed[CO / 2];
        if (MODE == kModeRelu) {
#pragma unroll
            for (int c = 0; c < CO; c += 2) {
                const float v0 = fmaxf(__uint_as_float(r[c]) + a.bias[c], 0.0f);
                const float v1 = fmaxf(__uint_as_float(r[c + 1]) + a.bias[c + 1], 0.0f);
                __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                packed[c / 2] = *reinterpret_cast<uint32_t *>(&h);
            }
        } else {     // kModeMask: input gradient times [activation > 0]
            const uint4 *mk = a.mask + p * (CO / 8);
#pragma unroll
            for (int u = 0; u < CO / 8; ++u) {
                const uint4 mm = __ldg(&mk[u]);
                const uint32_t mw[4] = {mm.x, mm.y, mm.z, mm.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = 8 * u + 2 * j;
                    const float v0 = bf16_positive(mw[j] & 0xFFFFu) ? __uint_as_float(r[c]) : 0.0f;
                    const float v1 = bf16_positive(mw[j] >> 16) ? __uint_as_float(r[c + 1]) : 0.0f;
                    __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                    packed[c / 2] = *reinterpret_cast<uint32_t *>(&h);
                }
            }
        }
        uint4 *dst = a.out + p * (CO / 8);
#pragma unroll
        for (int u = 0; u < CO / 8; ++u)
            dst[u] = make_uint4(packed[4 * u], packed[4 * u + 1], packed[4 * u + 2], packed[4 * u + 3]);
    }
}

template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(128) k_conv3x3(const ConvArgs a)
{
    static_assert(CI % 16 == 0 && (CO == 16 || CO == 32), "channel counts");
    extern __shared__ uint4 smem[];
    uint4 *sA = smem;
    uint4 *sB = smem + ConvSmem<CI, CO>::kA;
    __shared__ uint64_t bar;
    __shared__ uint32_t taddr_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int segs = (a.W + kTileM - 1) / kTileM;
    const long long n_tiles = (long long)a.N * a.H * segs;

    if (warp == 0) tc::tmem_alloc(&taddr_s, 32);
    if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
    for (int i = threadIdx.x; i < ConvSmem<CI, CO>::kB; i += blockDim.x) sB[i] = a.wB[i];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = taddr_s;
    constexpr uint32_t idesc = tc::idesc_bf16(kTileM, CO);
    const uint32_t a_base = tc::smem_u32(sA), b_base = tc::smem_u32(sB);
    uint32_t phase = 0;
    bool failed = false;

    for (long long tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        const int xs = (int)(tile % segs);
        const long long ry = tile / segs;
        const int y = (int)(ry % a.H), n = (int)(ry / a.H);
        const int x0 = xs * kTileM;
        // stage rows y-1, y, y+1, pixels x0-1 .. x0+128 (zero outside the image)
        constexpr int kc_n = CI / 8;
        for (int i = threadIdx.x; i < 3 * kRowUnits * kc_n; i += blockDim.x) {
            const int kc = i % kc_n, px = (i / kc_n) % kRowUnits, dy = i / (kc_n * kRowUnits);
            const int yy = y + dy - 1, xx = x0 + px - 1;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
                v = __ldg(&a.in[(((size_t)n * a.H + yy) * a.W + xx) * kc_n + kc]);
            sA[(dy * kc_n + kc) * kRowUnits + px] = v;
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int dy = t / 3, dx = t % 3;
#pragma unroll
                for (int s = 0; s < CI / 16; ++s) {
                    const uint32_t aa = a_base + (uint32_t)(((dy * kc_n + 2 * s) * kRowUnits + dx) * 16);
                    const uint32_t bb = b_base + (uint32_t)(((t * kc_n + 2 * s) * CO) * 16);
                    tc::mma_bf16(tmem, tc::sdesc(aa, kRowUnits * 16, 128), tc::sdesc(bb, CO * 16, 128), idesc,
                                 (t | s) != 0);
                }
            }
            tc::mma_commit(&bar);
        }
        const bool ok = tc::mbar_wait_bounded(&bar, phase, kSpinLimit);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) set_status(a.status, 1u);
            failed = true;
            // the MMAs may still be running: wait once more (bounded) before freeing TMEM
            tc::mbar_wait_bounded(&bar, phase ^ 1u, kSpinLimit);
            break;
        }
        tc::fence_after_sync();
        // epilogue: warp w owns accumulator rows (pixels) 32w .. 32w + 31
        const int m = warp * 32 + lane, x = x0 + m;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        uint32_t r[32];
        {
            uint32_t q[16];
            tc::tmem_ld16(trow, q);
#pragma unroll
            for (int c = 0; c < 16; ++c) r[c] = q[c];
            if (CO == 32) {
                tc::tmem_ld16(trow + 16, q);
#pragma unroll
                for (int c = 0; c < 16; ++c) r[16 + c] = q[c];
            }
        }
        tc::tmem_wait_ld();
        if (x < a.W) conv_epilogue<CO, MODE>(a, ((size_t)n * a.H + y) * a.W + x, r);
        tc::fence_before_sync();
        __syncthreads();     // all reads of this tile's accumulator and staged rows are done
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

// ------------------------------------------------------------------ conv, TMA-fed pipeline
//
// The same tiles, operands and epilogues as k_conv3x3, with the work split between warps
// so that loads, MMAs and epilogues of consecutive tiles overlap:
//   warp 0 (one lane)  TMA producer: the three input rows of a tile arrive as 3 x CI/8
//                      boxes (8 channels x 130 pixels, zero-filled outside the image)
//                      into one of kStages shared-memory stages; an mbarrier counts the
//                      bytes;
//   warp 1 (one lane)  MMA issuer: waits for a full stage and a free accumulator, issues
//                      the 9 x CI/16 MMAs into one of two TMEM accumulators, and commits
//                      to the stage's "empty" and the accumulator's "full" barriers;
//   warps 2-5          epilogue: wait for a full accumulator, read their 32 rows (warp
//                      w reads lanes 32 (w % 4) ...), release the accumulator, store.
// Every wait is bounded; a wait that gives up records a status and ends the block's loop.
constexpr int kStages = 2;
constexpr int kSlabUnits = 136;        // 16-byte units per staged (row, chunk) slab: 130 used, 128-byte aligned

template <int CI, int CO>
struct TmaConvSmem {
    static constexpr int kB = 9 * (CI / 8) * CO * 16;                 // weights (bytes)
    static constexpr int kStage = 3 * (CI / 8) * kSlabUnits * 16;     // one stage of input rows
    static constexpr int kStageTx = 3 * (CI / 8) * kRowUnits * 16;    // bytes the TMA boxes deliver
    static constexpr size_t bytes = (size_t)kB + (size_t)kStages * kStage + 1024;   // + alignment slack
};

template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(192) k_conv3x3_tma(const __grid_constant__ CUtensorMap tmap, const ConvArgs a)
{
    static_assert(CI % 16 == 0 && (CO == 16 || CO == 32), "channel counts");
    using S = TmaConvSmem<CI, CO>;
    constexpr int kcn = CI / 8;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint4 *sB = reinterpret_cast<uint4 *>(base);
    uint8_t *sA = base + S::kB;
    __shared__ uint64_t full[kStages], empty[kStages], tfull[2], tempty[2];
    __shared__ uint32_t taddr_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int segs = (a.W + kTileM - 1) / kTileM;
    const long long n_tiles = (long long)a.N * a.H * segs;

    if (warp == 0) tc::tmem_alloc(&taddr_s, 64);
    if (threadIdx.x == 32) {
        for (int i = 0; i < kStages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&tfull[i], 1);
            tc::mbar_init(&tempty[i], 4);
        }
    }
    for (int i = threadIdx.x; i < S::kB / 16; i += blockDim.x) sB[i] = a.wB[i];
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = taddr_s;
    constexpr uint32_t idesc = tc::idesc_bf16(kTileM, CO);

    if (warp == 0) {
        if (lane == 0) {                                       // TMA producer
            int k = 0;
            for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
                // (the stage's previous box landed before the MMA that freed it ran)
                const int st = k % kStages;
                if (!tc::mbar_wait_bounded(&empty[st], ((k / kStages) & 1) ^ 1, kSpinLimit)) {
                    set_status(a.status, 3u);
                    break;
                }
                const int xs = (int)(tile % segs);
                const long long ry = tile / segs;
                const int y = (int)(ry % a.H), n = (int)(ry / a.H);
                tc::mbar_arrive_expect_tx(&full[st], (uint32_t)S::kStageTx);
                const uint32_t dst0 = tc::smem_u32(sA + (size_t)st * S::kStage);
                for (int dy = 0; dy < 3; ++dy)
                    for (int kc = 0; kc < kcn; ++kc)
                        tc::tma_load_4d(dst0 + (uint32_t)((dy * kcn + kc) * kSlabUnits * 16), &tmap, 8 * kc,
                                        xs * kTileM - 1, y + dy - 1, n, &full[st]);
            }
            // drain: the last boxes have landed before the block may exit
            if (k > 0) tc::mbar_wait_bounded(&full[(k - 1) % kStages], ((k - 1) / kStages) & 1, kSpinLimit);
        }
    } else if (warp == 1) {
        if (lane == 0) {                                       // MMA issuer
            int k = 0;
            for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
                const int st = k % kStages, acc = k & 1;
                if (!tc::mbar_wait_bounded(&full[st], (k / kStages) & 1, kSpinLimit) ||
                    !tc::mbar_wait_bounded(&tempty[acc], ((k >> 1) & 1) ^ 1, kSpinLimit)) {
                    set_status(a.status, 3u);
                    break;
                }
                tc::fence_after_sync();
                const uint32_t a_base = tc::smem_u32(sA + (size_t)st * S::kStage), b_base = tc::smem_u32(sB);
                const uint32_t d = tmem + (uint32_t)(acc * 32);
#pragma unroll
                for (int t = 0; t < 9; ++t) {
                    const int dy = t / 3, dx = t % 3;
#pragma unroll
                    for (int sk = 0; sk < CI / 16; ++sk) {
                        const uint32_t aa = a_base + (uint32_t)(((dy * kcn + 2 * sk) * kSlabUnits + dx) * 16);
                        const uint32_t bb = b_base + (uint32_t)(((t * kcn + 2 * sk) * CO) * 16);
                        tc::mma_bf16(d, tc::sdesc(aa, kSlabUnits * 16, 128), tc::sdesc(bb, CO * 16, 128), idesc,
                                     (t | sk) != 0);
                    }
                }
                tc::mma_commit(&empty[st]);
                tc::mma_commit(&tfull[acc]);
            }
            // drain: the last committed MMAs finish before the accumulators are freed
            if (k > 0) tc::mbar_wait_bounded(&tfull[(k - 1) & 1], ((k - 1) >> 1) & 1, kSpinLimit);
        }
    } else {                                                   // epilogue warps 2..5
        const int quarter = warp & 3;
        int k = 0;
        for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
            const int acc = k & 1;
            if (!tc::mbar_wait_bounded(&tfull[acc], (k >> 1) & 1, kSpinLimit)) {
                if (lane == 0) set_status(a.status, 3u);
                break;
            }
            tc::fence_after_sync();
            const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * 32);
            uint32_t r[32];
            {
                uint32_t q[16];
                tc::tmem_ld16(trow, q);
#pragma unroll
                for (int c = 0; c < 16; ++c) r[c] = q[c];
                if (CO == 32) {
                    tc::tmem_ld16(trow + 16, q);
#pragma unroll
                    for (int c = 0; c < 16; ++c) r[16 + c] = q[c];
                }
            }
            tc::tmem_wait_ld();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[acc]);
            const int xs = (int)(tile % segs);
            const long long ry = tile / segs;
            const int y = (int)(ry % a.H), n = (int)(ry / a.H);
            const int x = xs * kTileM + quarter * 32 + lane;
            if (x < a.W) conv_epilogue<CO, MODE>(a, ((size_t)n * a.H + y) * a.W + x, r);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// ------------------------------------------------------------------ weight gradient

template <int CI, int CO>
struct WgradSmem {
    static constexpr int kRows = 9 * CI + 1;                       // (tap, channel) rows + the ones row
    static constexpr int kGroups = (kRows + 127) / 128;
    static constexpr int kRowsP = kGroups * 128;
    static constexpr int kXStride = CI / 8 + 1;                    // padded pixel stride (uint4)
    static constexpr int kYStride = CO / 8 + 1;
    static constexpr int kNatX = 3 * (kKBlock + 2) * kXStride;
    static constexpr int kNatY = kKBlock * kYStride;
    static constexpr int kA = (kKBlock / 8) * kRowsP;
    static constexpr int kB = (kKBlock / 8) * CO;
    // two natural-layout buffers: the next K block's rows arrive (cp.async) while the
    // current one is transposed and multiplied
    static constexpr size_t bytes = (size_t)(2 * (kNatX + kNatY) + kA + kB) * 16;
    static constexpr int kCols = kGroups * CO <= 32 ? 32 : (kGroups * CO <= 64 ? 64 : 128);
};

template <int CI, int CO>
__global__ void __launch_bounds__(128) k_conv3x3_wgrad(const WgradArgs a)
{
    using S = WgradSmem<CI, CO>;
    extern __shared__ uint4 smem[];
    uint4 *nat = smem;                                   // [2][kNatX + kNatY]
    uint4 *sA = nat + 2 * (S::kNatX + S::kNatY);
    uint4 *sB = sA + S::kA;
    __shared__ uint64_t bar;
    __shared__ uint32_t taddr_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int segs = (a.W + kKBlock - 1) / kKBlock;
    const long long n_blocks = (long long)a.N * a.H * segs;

    if (warp == 0) tc::tmem_alloc(&taddr_s, S::kCols);
    if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
    // rows past the (tap, channel) rows: zero, except the ones row (bias gradient)
    for (int i = threadIdx.x; i < (kKBlock / 8) * (S::kRowsP - 9 * CI); i += blockDim.x) {
        const int kc = i / (S::kRowsP - 9 * CI), r = 9 * CI + i % (S::kRowsP - 9 * CI);
        const uint32_t one2 = 0x3F803F80u;     // two bf16 ones
        sA[kc * S::kRowsP + r] = r == 9 * CI ? make_uint4(one2, one2, one2, one2) : make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = taddr_s;
    constexpr uint32_t idesc = tc::idesc_bf16(128, CO);
    const uint32_t a_base = tc::smem_u32(sA), b_base = tc::smem_u32(sB);
    uint32_t phase = 0;
    bool any = false, failed = false;
    constexpr int kcx = CI / 8, kcy = CO / 8;

    // natural-layout staging of K block kb into buffer `buf` by 16-byte cp.async (zero
    // fill outside the image): x rows y-1..y+1, pixels x0-1 .. x0+64; dy row y, x0 .. x0+63
    const auto stage = [&](long long kb, int buf) {
        const int xs = (int)(kb % segs);
        const long long ry = kb / segs;
        const int y = (int)(ry % a.H), n = (int)(ry / a.H);
        const int x0 = xs * kKBlock;
        uint4 *natx = nat + buf * (S::kNatX + S::kNatY), *naty = natx + S::kNatX;
        for (int i = threadIdx.x; i < 3 * (kKBlock + 2) * kcx; i += blockDim.x) {
            const int kc = i % kcx, px = (i / kcx) % (kKBlock + 2), dy = i / (kcx * (kKBlock + 2));
            const int yy = y + dy - 1, xx = x0 + px - 1;
            const bool in = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            const uint4 *src = in ? &a.x[(((size_t)n * a.H + yy) * a.W + xx) * kcx + kc] : a.x;
            tc::cp_async16(tc::smem_u32(&natx[(dy * (kKBlock + 2) + px) * S::kXStride + kc]), src, in ? 16u : 0u);
        }
        for (int i = threadIdx.x; i < kKBlock * kcy; i += blockDim.x) {
            const int kc = i % kcy, px = i / kcy, xx = x0 + px;
            const bool in = xx < a.W;
            const uint4 *src = in ? &a.dy[(((size_t)n * a.H + y) * a.W + xx) * kcy + kc] : a.dy;
            tc::cp_async16(tc::smem_u32(&naty[px * S::kYStride + kc]), src, in ? 16u : 0u);
        }
        tc::cp_async_commit();
    };

    int buf = 0;
    if (blockIdx.x < n_blocks) stage(blockIdx.x, 0);
    for (long long kb = blockIdx.x; kb < n_blocks; kb += gridDim.x, buf ^= 1) {
        const bool more = kb + gridDim.x < n_blocks;
        if (more) stage(kb + gridDim.x, buf ^ 1);       // the next block's loads in flight
        if (more)
            tc::cp_async_wait<1>();
        else
            tc::cp_async_wait<0>();
        __syncthreads();
        const uint32_t natx_base = tc::smem_u32(nat + buf * (S::kNatX + S::kNatY));
        const uint32_t naty_base = natx_base + (uint32_t)S::kNatX * 16u;
        // transposed copies: A[kp][(3 dy + dx) CI + 8 kcc + r] = x[y+dy-1][x0 + 8 kp + j + dx - 1][8 kcc + r], j = 0..7
        constexpr int kABlocks = 9 * kcx * (kKBlock / 8);
        constexpr int kBBlocks = kcy * (kKBlock / 8);
        for (int op = warp; op < (kABlocks + kBBlocks) / 4; op += 4) {
            const int blk = op * 4 + (lane >> 3), r = lane & 7;
            uint32_t src, dst;
            if (blk < kABlocks) {
                const int kp = blk % (kKBlock / 8), kcc = (blk / (kKBlock / 8)) % kcx, t = blk / ((kKBlock / 8) * kcx);
                const int dy = t / 3, dx = t % 3;
                src = natx_base + (uint32_t)(((dy * (kKBlock + 2) + kp * 8 + dx + r) * S::kXStride + kcc) * 16);
                dst = a_base + (uint32_t)((kp * S::kRowsP + t * CI + 8 * kcc + r) * 16);
            } else {
                const int b = blk - kABlocks, kp = b % (kKBlock / 8), kcc = b / (kKBlock / 8);
                src = naty_base + (uint32_t)(((kp * 8 + r) * S::kYStride + kcc) * 16);
                dst = b_base + (uint32_t)((kp * CO + 8 * kcc + r) * 16);
            }
            tc::transpose_copy_x4(src, dst);
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int s = 0; s < kKBlock / 16; ++s)
#pragma unroll
                for (int g = 0; g < S::kGroups; ++g) {
                    const uint32_t aa = a_base + (uint32_t)((2 * s * S::kRowsP + 128 * g) * 16);
                    const uint32_t bb = b_base + (uint32_t)(2 * s * CO * 16);
                    tc::mma_bf16(tmem + (uint32_t)(g * CO), tc::sdesc(aa, S::kRowsP * 16, 128),
                                 tc::sdesc(bb, CO * 16, 128), idesc, (any || s > 0) ? 1u : 0u);
                }
            tc::mma_commit(&bar);
        }
        any = true;
        const bool ok = tc::mbar_wait_bounded(&bar, phase, kSpinLimit);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) set_status(a.status, 2u);
            failed = true;
            tc::mbar_wait_bounded(&bar, phase ^ 1u, kSpinLimit);
            break;
        }
    }
    tc::cp_async_wait<0>();                               // no copy outlives the loop
    tc::fence_after_sync();
    if (any && !failed) {
        for (int g = 0; g < S::kGroups; ++g) {
            const int row = 128 * g + 32 * warp + lane;
            const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(g * CO);
#pragma unroll
            for (int c0 = 0; c0 < CO; c0 += 16) {
                uint32_t q[16];
                tc::tmem_ld16(trow + c0, q);
                tc::tmem_wait_ld();
                if (row < 9 * CI) {
                    float *dst = a.dw + (size_t)row * CO + c0;      // row = tap * CI + channel
#pragma unroll
                    for (int c = 0; c < 16; ++c) atomicAdd(dst + c, __uint_as_float(q[c]));
                } else if (row == 9 * CI) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) atomicAdd(a.db + c0 + c, __uint_as_float(q[c]));
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::kCols);
}

// ------------------------------------------------------------------ weight gradient, TMA-fed
//
// The same sums, with the operands read in the layout the TMA boxes land in, so that no
// shared-memory transpose is needed: a K block is 128 pixels of one output row; its three
// input rows (pixels x0 - 1 .. x0 + 128) arrive as 3 x CI/8 slabs [pixel][8 channels] of
// kSlabUnits units and the output-gradient row as CO/8 slabs of 128 units. Read with the
// pixels as K and the channels as M (x) or N (dy), a slab is the MN-major canonical
// layout: a core matrix is 8 pixels x 8 channels, 128 contiguous bytes; the next 8
// channels are one slab further, the next 8 pixels 128 bytes further. For a fixed dx the
// (dy, channel group) rows of the three input rows form one uniformly strided M
// dimension of 3 CI rows that starts dx pixels into the slabs, so one M = 128 MMA per
// (dx, 16-pixel K step) covers the three taps (dy, dx); the M rows after 3 CI read a slab
// of ones (row 3 CI: the bias gradient, taken from dx = 0) and zero slabs, whose products
// are not used. Accumulators: three TMEM blocks of CO columns (one per dx) for the whole
// persistent block, added to dW with one atomic per (row, column) at the end.
// One thread issues the TMA loads (two stages) and the MMAs; the four warps run the
// epilogue. Every wait is bounded.
constexpr int kWgPix = 128;                // pixels per K block
constexpr int kWgGroups = 16;              // M groups read by an M = 128 MMA

template <int CI, int CO>
struct WgradTmaSmem {
    static constexpr int kXBytes = kWgGroups * kSlabUnits * 16;       // slabs of x (+ ones, zeros)
    static constexpr int kYBytes = (CO / 8) * kWgPix * 16;            // slabs of dy
    static constexpr int kStage = kXBytes + kYBytes;
    static constexpr uint32_t kTx = (uint32_t)(3 * (CI / 8) * kRowUnits * 16 + (CO / 8) * kWgPix * 16);
    static constexpr size_t bytes = (size_t)2 * kStage + 1024;       // + alignment slack
    static constexpr int kCols = 3 * CO <= 32 ? 32 : (3 * CO <= 64 ? 64 : 128);
    static_assert(3 * (CI / 8) + 1 <= kWgGroups, "the three rows and the ones slab fit one M = 128 MMA");
};

// Instruction descriptor of kind::f16, bf16 A and B both MN-major (transposed), f32
// accumulator, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N)
{
    return tc::idesc_bf16(M, N) | (1u << 15) | (1u << 16);
}

// Descriptor of an MN-major operand without swizzle: the leading byte offset is the
// distance between core matrices adjacent in K (here 8 pixels, 128 bytes), the stride byte
// offset the distance between core matrices adjacent in M or N (8 channels, one slab).
// (The weight-gradient parity tests fail with the two offsets exchanged.)
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t mn_stride, uint32_t k_stride)
{
    return tc::sdesc(saddr, k_stride, mn_stride);
}

template <int CI, int CO>
__global__ void __launch_bounds__(128) k_conv3x3_wgrad_tma(const __grid_constant__ CUtensorMap xmap,
                                                           const __grid_constant__ CUtensorMap ymap,
                                                           const WgradArgs a)
{
    static_assert(CI % 16 == 0 && (CO == 16 || CO == 32), "channel counts");
    using S = WgradTmaSmem<CI, CO>;
    constexpr int kcx = CI / 8, kcy = CO / 8;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full[2], empty[2];
    __shared__ uint32_t taddr_s;
    __shared__ int failed_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int segs = (a.W + kWgPix - 1) / kWgPix;
    const long long n_kb = (long long)a.N * a.H * segs;

    if (warp == 0) tc::tmem_alloc(&taddr_s, S::kCols);
    if (threadIdx.x == 32) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        failed_s = 0;
    }
    // the slabs after the three input rows: ones (first element of each unit) then zeros
    for (int st = 0; st < 2; ++st) {
        uint4 *x = reinterpret_cast<uint4 *>(base + (size_t)st * S::kStage);
        for (int i = threadIdx.x; i < (kWgGroups - 3 * kcx) * kSlabUnits; i += blockDim.x) {
            const int g = 3 * kcx + i / kSlabUnits;
            x[g * kSlabUnits + i % kSlabUnits] = make_uint4(g == 3 * kcx ? 0x3F80u : 0u, 0u, 0u, 0u);
        }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = taddr_s;
    constexpr uint32_t idesc = idesc_bf16_mn(128, CO);
    long long issued = 0;                  // K blocks whose MMAs were issued

    if (threadIdx.x == 0) {
        const auto load = [&](long long kb, int st) {
            const int xs = (int)(kb % segs);
            const long long ry = kb / segs;
            const int y = (int)(ry % a.H), n = (int)(ry / a.H);
            const uint32_t xb = tc::smem_u32(base + (size_t)st * S::kStage), yb = xb + (uint32_t)S::kXBytes;
            tc::mbar_arrive_expect_tx(&full[st], S::kTx);
            for (int dy = 0; dy < 3; ++dy)
                for (int kc = 0; kc < kcx; ++kc)
                    tc::tma_load_4d(xb + (uint32_t)((dy * kcx + kc) * kSlabUnits * 16), &xmap, 8 * kc,
                                    xs * kWgPix - 1, y + dy - 1, n, &full[st]);
            for (int kc = 0; kc < kcy; ++kc)
                tc::tma_load_4d(yb + (uint32_t)(kc * kWgPix * 16), &ymap, 8 * kc, xs * kWgPix, y, n, &full[st]);
        };
        int loaded = 0;                    // K blocks whose loads were issued
        for (int i = 0; i < 2; ++i)
            if (blockIdx.x + (long long)i * gridDim.x < n_kb) {
                load(blockIdx.x + (long long)i * gridDim.x, i);
                ++loaded;
            }
        bool ok = true;
        for (long long j = 0;; ++j) {
            const long long kb = blockIdx.x + j * gridDim.x;
            if (kb >= n_kb) break;
            const int st = (int)(j & 1);
            if (!tc::mbar_wait_bounded(&full[st], (uint32_t)((j >> 1) & 1), kSpinLimit)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const uint32_t xb = tc::smem_u32(base + (size_t)st * S::kStage), yb = xb + (uint32_t)S::kXBytes;
#pragma unroll
            for (int s = 0; s < kWgPix / 16; ++s)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
                    tc::mma_bf16(tmem + (uint32_t)(dx * CO), sdesc_mn(xb + (uint32_t)(dx * 16 + s * 256), kSlabUnits * 16, 128),
                                 sdesc_mn(yb + (uint32_t)(s * 256), kWgPix * 16, 128), idesc, (j | s) != 0);
            tc::mma_commit(&empty[st]);
            issued = j + 1;
            const long long next = kb + 2 * (long long)gridDim.x;
            if (next < n_kb) {
                if (!tc::mbar_wait_bounded(&empty[st], (uint32_t)((j >> 1) & 1), kSpinLimit)) {
                    ok = false;
                    break;
                }
                load(next, st);
                ++loaded;
            }
        }
        // drain: the last MMAs have completed and no box is still landing
        if (issued > 0 && !tc::mbar_wait_bounded(&empty[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1), kSpinLimit))
            ok = false;
        for (long long u = issued; u < loaded; ++u)
            if (!tc::mbar_wait_bounded(&full[u & 1], (uint32_t)((u >> 1) & 1), kSpinLimit)) ok = false;
        if (!ok) {
            set_status(a.status, 2u);
            failed_s = 1;
        }
        if (issued == 0) failed_s = failed_s | 2;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (failed_s == 0) {
        const int row = 32 * warp + lane;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
#pragma unroll
            for (int c0 = 0; c0 < CO; c0 += 16) {
                uint32_t q[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(dx * CO + c0), q);
                tc::tmem_wait_ld();
                if (row < 3 * CI) {
                    const int tap = 3 * (row / CI) + dx, ci = row % CI;
                    float *dst = a.dw + ((size_t)tap * CI + ci) * CO + c0;
#pragma unroll
                    for (int c = 0; c < 16; ++c) atomicAdd(dst + c, __uint_as_float(q[c]));
                } else if (row == 3 * CI && dx == 0) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) atomicAdd(a.db + c0 + c, __uint_as_float(q[c]));
                }
            }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::kCols);
}

// ------------------------------------------------------------------ launchers

namespace {

// Blocks of a persistent grid: resident blocks per SM (from the kernel's registers and
// shared memory and the SM's limits) times SMs, at most `work`.
int resident_grid(const void *fn, size_t smem, long long work, int threads = 128)
{
    int dev = 0, sms = 1, smem_sm = 0, regs_sm = 65536, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncAttributes fa;
    int per_sm = 1;
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess) {
        const size_t block_smem = smem + fa.sharedSizeBytes + (size_t)reserved;
        const int by_smem = block_smem ? (int)((size_t)smem_sm / block_smem) : 16;
        const int regs = fa.numRegs > 0 ? fa.numRegs : 64;
        const int warps = (threads + 31) / 32;
        const int by_regs = regs_sm / (((regs * 32 + 255) / 256) * 256 * warps);
        per_sm = by_smem < by_regs ? by_smem : by_regs;
        if (per_sm > 2048 / (warps * 32)) per_sm = 2048 / (warps * 32);         // 2048 threads per SM
        if (per_sm < 1) per_sm = 1;
    }
    long long g = (long long)per_sm * sms;
    if (g > work) g = work;
    return (int)(g > 0 ? g : 1);
}

template <class F>
cudaError_t set_smem(F *fn, size_t bytes)
{
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

}  // namespace

// cuTensorMapEncodeTiled from the driver, fetched once through the runtime.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t encode_tiled(EncodeTiledFn *out)
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    *out = fn;
    return cudaSuccess;
}

// Tensor map of an NHWC bf16 activation with CI channels, as dims (CI, W, H, N), boxes of
// 8 channels x box_px pixels x 1 row x 1 frame, zero fill outside.
cudaError_t input_map(const void *base, int ci, int n, int h, int w, CUtensorMap *m, int box_px = kTileM + 2)
{
    EncodeTiledFn fn = nullptr;
    cudaError_t e = encode_tiled(&fn);
    if (e != cudaSuccess) return e;
    const cuuint64_t dims[4] = {(cuuint64_t)ci, (cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)n};
    const cuuint64_t strides[3] = {(cuuint64_t)ci * 2, (cuuint64_t)w * ci * 2, (cuuint64_t)h * w * ci * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)box_px, 1, 1};
    const cuuint32_t elem[4] = {1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, box, elem,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

#ifndef SGAD_NET_CONV_TMA
#define SGAD_NET_CONV_TMA 1
#endif

template <int CI, int CO, int MODE>
cudaError_t launch_conv(const ConvArgs &a, cudaStream_t st)
{
#if SGAD_NET_CONV_TMA
    {
        const size_t smem = TmaConvSmem<CI, CO>::bytes;
        cudaError_t e = set_smem(k_conv3x3_tma<CI, CO, MODE>, smem);
        if (e != cudaSuccess) return e;
        const long long tiles = (long long)a.N * a.H * ((a.W + kTileM - 1) / kTileM);
        if (tiles <= 0) return cudaSuccess;
        CUtensorMap m;
        e = input_map(a.in, CI, a.N, a.H, a.W, &m);
        if (e != cudaSuccess) return e;
        // TMEM: 64 columns per block, at most 8 blocks of 512 columns per SM
        const int grid = resident_grid((const void *)k_conv3x3_tma<CI, CO, MODE>, smem, tiles, 192);
        k_conv3x3_tma<CI, CO, MODE><<<grid, 192, smem, st>>>(m, a);
        return cudaGetLastError();
    }
#endif
    const size_t smem = ConvSmem<CI, CO>::bytes;
    cudaError_t e = set_smem(k_conv3x3<CI, CO, MODE>, smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)a.N * a.H * ((a.W + kTileM - 1) / kTileM);
    if (tiles <= 0) return cudaSuccess;
    const int grid = resident_grid((const void *)k_conv3x3<CI, CO, MODE>, smem, tiles);
    k_conv3x3<CI, CO, MODE><<<grid, 128, smem, st>>>(a);
    return cudaGetLastError();
}

#ifndef SGAD_NET_WGRAD_TMA
#define SGAD_NET_WGRAD_TMA 1
#endif

template <int CI, int CO>
cudaError_t launch_wgrad(const WgradArgs &a, cudaStream_t st)
{
#if SGAD_NET_WGRAD_TMA
    {
        using S = WgradTmaSmem<CI, CO>;
        cudaError_t e = set_smem(k_conv3x3_wgrad_tma<CI, CO>, S::bytes);
        if (e != cudaSuccess) return e;
        const long long blocks = (long long)a.N * a.H * ((a.W + kWgPix - 1) / kWgPix);
        if (blocks <= 0) return cudaSuccess;
        CUtensorMap xm, ym;
        e = input_map(a.x, CI, a.N, a.H, a.W, &xm);
        if (e == cudaSuccess) e = input_map(a.dy, CO, a.N, a.H, a.W, &ym, kWgPix);
        if (e != cudaSuccess) return e;
        int grid = resident_grid((const void *)k_conv3x3_wgrad_tma<CI, CO>, S::bytes, blocks);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long cap = (long long)sms * (512 / S::kCols);
        if (grid > cap) grid = (int)cap;
        k_conv3x3_wgrad_tma<CI, CO><<<grid, 128, S::bytes, st>>>(xm, ym, a);
        return cudaGetLastError();
    }
#endif
    const size_t smem = WgradSmem<CI, CO>::bytes;
    cudaError_t e = set_smem(k_conv3x3_wgrad<CI, CO>, smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)a.N * a.H * ((a.W + kKBlock - 1) / kKBlock);
    if (blocks <= 0) return cudaSuccess;
    // keep (resident blocks x TMEM columns) within the 512 columns of an SM
    int grid = resident_grid((const void *)k_conv3x3_wgrad<CI, CO>, smem, blocks);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long cap = (long long)sms * (512 / WgradSmem<CI, CO>::kCols);
    if (grid > cap) grid = (int)cap;
    k_conv3x3_wgrad<CI, CO><<<grid, 128, smem, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_conv<16, 32, kModeRelu>(const ConvArgs &, cudaStream_t);
template cudaError_t launch_conv<32, 32, kModeRelu>(const ConvArgs &, cudaStream_t);
template cudaError_t launch_conv<32, 16, kModeOut>(const ConvArgs &, cudaStream_t);
template cudaError_t launch_conv<16, 32, kModeMask>(const ConvArgs &, cudaStream_t);
template cudaError_t launch_conv<32, 32, kModeMask>(const ConvArgs &, cudaStream_t);
template cudaError_t launch_wgrad<16, 32>(const WgradArgs &, cudaStream_t);
template cudaError_t launch_wgrad<32, 32>(const WgradArgs &, cudaStream_t);
template cudaError_t launch_wgrad<32, 16>(const WgradArgs &, cudaStream_t);

cudaError_t launch_pack_input(const float *rgb, const float *depth, uint4 *x0, int n, int h, int w, cudaStream_t st)
{
    const size_t total = (size_t)n * h * w;
    if (!total) return cudaSuccess;
    const int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    k_pack_input<<<grid, 256, 0, st>>>(rgb, depth, x0, n, h, w);
    return cudaGetLastError();
}

cudaError_t launch_prep_weights(const float *w, uint4 *fwd, uint4 *bwd, int ci_p, int co_p, cudaStream_t st)
{
    const int n = 9 * ci_p * co_p / 8;
    k_prep_weights<<<(n + 127) / 128, 128, 0, st>>>(w, fwd, bwd, ci_p, co_p);
    return cudaGetLastError();
}

cudaError_t launch_loss(const float2 *y4, const float *td, const float *tl, float lw, uint4 *dy4, float *loss,
                        size_t total, cudaStream_t st)
{
    if (!total) return cudaSuccess;
    const int grid = (int)((total + 255) / 256 < 2048 ? (total + 255) / 256 : 2048);
    k_loss<<<grid, 256, 0, st>>>(y4, td, tl, lw, dy4, loss, total);
    return cudaGetLastError();
}

}  // namespace net
}  // namespace sgad
