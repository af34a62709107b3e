// Learned proposal net (workload extension; the paper initialises offsets at zero):
// 3x3 convolutions as implicit GEMMs on the tcgen05 tensor cores, bf16 operands, f32
// accumulation in tensor memory.
//
// Activations are bf16 with 16 or 32 channels (the 4-channel input and 2-channel output
// are zero-padded), stored chunk-planar: 16-byte units of 8 channels, [frame][row][channel
// chunk][pixel], so the units of one chunk of one image row are contiguous (a TMA box of a
// chunk over a row reads whole sectors).
//
// Forward and input gradient (k_conv3x3_tma): a tile is 128 consecutive output pixels of
// one image row (the MMA's M), all output channels (N = 16 or 32) and K = 9 taps x C_in.
// The three input rows arrive by TMA as one box per (row, chunk) of 130 pixels, which in
// shared memory is the K-major canonical layout; the tap (dy, dx) is a descriptor start
// offset of dx units into row dy, so no im2col copy is made. Weights are staged once per
// block in the B layout [tap][channel chunk][c_out]. A producer lane, an MMA lane and
// four epilogue warps overlap loads, MMAs (double TMEM accumulator) and the epilogue
// (bias + ReLU + bf16; or the ReLU-masked input gradient; or the two f32 outputs).
//
// Weight gradient (k_conv3x3_wgrad_tma): dW[t][i][o] = sum_p x[p + d_t][i] dy[p][o] is a
// GEMM with the pixels as K; the same TMA boxes, read with the channels as M (x) or N
// (dy), are the MN-major canonical layout, so three taps share one M = 128 MMA (below)
// and no shared-memory transpose is needed; the accumulators stay in tensor memory for
// the whole persistent block and are added to the output with one atomic per (row,
// column) at the end.
#include <cuda.h>
#include <cuda_bf16.h>

#include "sgad_net_device.cuh"
#include "tc5.cuh"

namespace sgad {
namespace net {

constexpr uint32_t kSpinLimit = 1u << 22;   // bounded mbarrier waits (each try_wait may suspend)
constexpr int kTileM = 128;                  // output pixels per conv tile
constexpr int kRowUnits = kTileM + 2;        // staged pixels per input row (1-pixel halo)

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t code)
{
    atomicCAS(status, 0u, code);
}

// Unit index of (pixel p = (frame * H + row) * W + x, channel chunk c) in a chunk-planar
// tensor with kc chunks per pixel.
__device__ __forceinline__ size_t planar_unit(size_t p, int c, int kc, int w)
{
    const size_t row = p / (size_t)w;
    return (row * kc + c) * (size_t)w + (p - row * (size_t)w);
}

// ------------------------------------------------------------------ small kernels

// (N,3,H,W) colour + (N,H,W) depth (f32) -> chunk-planar bf16, 16 channels (R, G, B, D, 0 ...).
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
        x0[planar_unit(p, 0, 2, w)] = v0;
        x0[planar_unit(p, 1, 2, w)] = make_uint4(0u, 0u, 0u, 0u);
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
                       float lw, uint4 *__restrict__ dy4, float *loss, size_t total, int w)
{
    const float inv = 1.0f / (float)total;
    float acc = 0.f;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const float2 y = y4[p];
        const float e0 = y.x - td[p] * 100.0f, e1 = y.y - tl[p];
        acc += e0 * e0 + lw * e1 * e1;
        __nv_bfloat162 g = __floats2bfloat162_rn(2.0f * e0 * inv, 2.0f * lw * e1 * inv);
        uint4 v = make_uint4(*reinterpret_cast<uint32_t *>(&g), 0u, 0u, 0u);
        dy4[planar_unit(p, 0, 2, w)] = v;
        dy4[planar_unit(p, 1, 2, w)] = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (loss && (threadIdx.x & 31) == 0) atomicAdd(loss, acc * inv);
}

// ------------------------------------------------------------------ conv (forward / input gradient)

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
#pragma unroll
            for (int u = 0; u < CO / 8; ++u) {
                const uint4 mm = __ldg(&a.mask[planar_unit(p, u, CO / 8, a.W)]);
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
#pragma unroll
        for (int u = 0; u < CO / 8; ++u)
            a.out[planar_unit(p, u, CO / 8, a.W)] = make_uint4(packed[4 * u], packed[4 * u + 1], packed[4 * u + 2],
                                                              packed[4 * u + 3]);
    }
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
constexpr int kStages = 3;
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
                        tc::tma_load_4d(dst0 + (uint32_t)((dy * kcn + kc) * kSlabUnits * 16), &tmap, 0,
                                        xs * kTileM - 1, (y + dy - 1) * kcn + kc, n, &full[st]);
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
// of ones (row 3 CI: the bias gradient, taken from dx = 0) and then whatever follows it
// in the stage, rows whose products are not used. Accumulators: three TMEM blocks of CO columns (one per dx) for the whole
// persistent block, added to dW with one atomic per (row, column) at the end.
// One thread of warp 0 issues the TMA loads into kWgStages stages, one thread of warp 1
// the MMAs (its descriptors precomputed: an offset adds to the address field); the four
// warps run the epilogue. Every wait is bounded.
constexpr int kWgPix = 128;                // pixels per K block
constexpr int kWgGroups = 16;              // M groups read by an M = 128 MMA
constexpr int kWgStages = 3;               // shared-memory stages of the load pipeline

template <int CI, int CO>
struct WgradTmaSmem {
    static constexpr int kXBytes = (3 * (CI / 8) + 1) * kSlabUnits * 16;   // slabs of x, then the ones slab
    static constexpr int kYBytes = (CO / 8) * kWgPix * 16;                 // slabs of dy
    // an M = 128 MMA reads kWgGroups slabs from the x base: past the ones slab it reads
    // the dy slabs (or padding), rows whose products are not used
    static constexpr int kStage = kXBytes + kYBytes > kWgGroups * kSlabUnits * 16 ? kXBytes + kYBytes
                                                                                 : kWgGroups * kSlabUnits * 16;
    static constexpr uint32_t kTx = (uint32_t)(3 * (CI / 8) * kRowUnits * 16 + (CO / 8) * kWgPix * 16);
    static constexpr size_t bytes = (size_t)kWgStages * kStage + 1024;   // + alignment slack
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
    __shared__ uint64_t full[kWgStages], empty[kWgStages];
    __shared__ uint32_t taddr_s;
    __shared__ int failed_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int segs = (a.W + kWgPix - 1) / kWgPix;
    const int n_kb = a.N * a.H * segs;          // < 2^31 (checked by the launcher)

    if (warp == 0) tc::tmem_alloc(&taddr_s, S::kCols);
    if (threadIdx.x == 32) {
        for (int i = 0; i < kWgStages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        failed_s = 0;
    }
    // the slab after the three input rows: ones (first element of each unit)
    for (int st = 0; st < kWgStages; ++st) {
        uint4 *x = reinterpret_cast<uint4 *>(base + (size_t)st * S::kStage) + 3 * kcx * kSlabUnits;
        for (int i = threadIdx.x; i < kSlabUnits; i += blockDim.x) x[i] = make_uint4(0x3F80u, 0u, 0u, 0u);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = taddr_s;
    constexpr uint32_t idesc = idesc_bf16_mn(128, CO);

    if (threadIdx.x == 0) {                                    // TMA producer
        int k = 0;
        bool ok = true;
        for (int kb = blockIdx.x; kb < n_kb; kb += gridDim.x, ++k) {
            const int st = k % kWgStages;
            if (!tc::mbar_wait_bounded(&empty[st], (uint32_t)(((k / kWgStages) & 1) ^ 1), kSpinLimit)) {
                ok = false;
                break;
            }
            const int xs = kb % segs, ry = kb / segs;
            const int y = ry % a.H, n = ry / a.H;
            const uint32_t xb = tc::smem_u32(base + (size_t)st * S::kStage), yb = xb + (uint32_t)S::kXBytes;
            tc::mbar_arrive_expect_tx(&full[st], S::kTx);
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int kc = 0; kc < kcx; ++kc)
                    tc::tma_load_4d(xb + (uint32_t)((dy * kcx + kc) * kSlabUnits * 16), &xmap, 0,
                                    xs * kWgPix - 1, (y + dy - 1) * kcx + kc, n, &full[st]);
#pragma unroll
            for (int kc = 0; kc < kcy; ++kc)
                tc::tma_load_4d(yb + (uint32_t)(kc * kWgPix * 16), &ymap, 0, xs * kWgPix, y * kcy + kc, n, &full[st]);
        }
        // drain: the last boxes have landed before the block may exit
        if (k > 0 && !tc::mbar_wait_bounded(&full[(k - 1) % kWgStages], (uint32_t)(((k - 1) / kWgStages) & 1), kSpinLimit))
            ok = false;
        if (!ok) {
            set_status(a.status, 3u);
            failed_s = 1;
        }
    } else if (threadIdx.x == 32) {                           // MMA issuer
        // descriptors of stage 0 at offset 0; an offset of o bytes adds o / 16
        const uint32_t x0 = tc::smem_u32(base), y0 = x0 + (uint32_t)S::kXBytes;
        const uint64_t ad0 = sdesc_mn(x0, kSlabUnits * 16, 128), bd0 = sdesc_mn(y0, kWgPix * 16, 128);
        int k = 0;
        bool ok = true;
        for (int kb = blockIdx.x; kb < n_kb; kb += gridDim.x, ++k) {
            const int st = k % kWgStages;
            if (!tc::mbar_wait_bounded(&full[st], (uint32_t)((k / kWgStages) & 1), kSpinLimit)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const uint64_t so = (uint64_t)(st * S::kStage / 16);
#pragma unroll
            for (int s = 0; s < kWgPix / 16; ++s)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
                    tc::mma_bf16(tmem + (uint32_t)(dx * CO), ad0 + so + (uint64_t)(dx + s * 16),
                                 bd0 + so + (uint64_t)(s * 16), idesc, (k | s) != 0);
            tc::mma_commit(&empty[st]);
        }
        // drain: the last MMAs have completed before the accumulators are read
        if (k > 0 && !tc::mbar_wait_bounded(&empty[(k - 1) % kWgStages], (uint32_t)(((k - 1) / kWgStages) & 1), kSpinLimit))
            ok = false;
        if (!ok) {
            set_status(a.status, 2u);
            failed_s = 1;
        }
        if (k == 0) failed_s = failed_s | 2;
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

// Tensor map of a chunk-planar bf16 activation with ci channels, as dims (8 channels, W,
// H x ci/8 (row, chunk), N), boxes of 8 channels x box_px pixels of one (row, chunk) of
// one frame, zero fill outside: the (row, chunk) coordinate of row y and chunk c is
// y ci/8 + c, so rows -1 and H fall outside the tensor.
cudaError_t input_map(const void *base, int ci, int n, int h, int w, CUtensorMap *m, int box_px = kTileM + 2)
{
    EncodeTiledFn fn = nullptr;
    cudaError_t e = encode_tiled(&fn);
    if (e != cudaSuccess) return e;
    const cuuint64_t kc = (cuuint64_t)(ci / 8);
    const cuuint64_t dims[4] = {8, (cuuint64_t)w, (cuuint64_t)h * kc, (cuuint64_t)n};
    const cuuint64_t strides[3] = {16, (cuuint64_t)w * 16, (cuuint64_t)h * kc * w * 16};
    const cuuint32_t box[4] = {8, (cuuint32_t)box_px, 1, 1};
    const cuuint32_t elem[4] = {1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, box, elem,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CI, int CO, int MODE>
cudaError_t launch_conv(const ConvArgs &a, cudaStream_t st)
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

template <int CI, int CO>
cudaError_t launch_wgrad(const WgradArgs &a, cudaStream_t st)
{
    using S = WgradTmaSmem<CI, CO>;
    cudaError_t e = set_smem(k_conv3x3_wgrad_tma<CI, CO>, S::bytes);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)a.N * a.H * ((a.W + kWgPix - 1) / kWgPix);
    if (blocks <= 0) return cudaSuccess;
    if (blocks >= (1ll << 31)) return cudaErrorInvalidValue;
    CUtensorMap xm, ym;
    e = input_map(a.x, CI, a.N, a.H, a.W, &xm);
    if (e == cudaSuccess) e = input_map(a.dy, CO, a.N, a.H, a.W, &ym, kWgPix);
    if (e != cudaSuccess) return e;
    // keep (resident blocks x TMEM columns) within the 512 columns of an SM
    int grid = resident_grid((const void *)k_conv3x3_wgrad_tma<CI, CO>, S::bytes, blocks);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long cap = (long long)sms * (512 / S::kCols);
    if (grid > cap) grid = (int)cap;
    k_conv3x3_wgrad_tma<CI, CO><<<grid, 128, S::bytes, st>>>(xm, ym, a);
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
                        size_t total, int w, cudaStream_t st)
{
    if (!total) return cudaSuccess;
    const int grid = (int)((total + 255) / 256 < 2048 ? (total + 255) / 256 : 2048);
    k_loss<<<grid, 256, 0, st>>>(y4, td, tl, lw, dy4, loss, total, w);
    return cudaGetLastError();
}

}  // namespace net
}  // namespace sgad
