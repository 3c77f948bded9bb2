// mlp.cu -- the control variate's network on the 5th-generation tensor
// cores (tcgen05.mma, accumulators in tensor memory): Fourier features (16
// frequencies 2^(k/3), sin and cos of 2 pi f y_d: 96 inputs) ->
// 4 x (64, SiLU) -> 1.  BF16 operands, FP32 accumulation; FP32 master weights
// (out x in layout, biases after each matrix) and Adam state in device
// memory.  Operands live in shared memory in the canonical K-major layout
// of tcgen05.cuh; every product is issued by one thread with M = 128 rows.
#include <atomic>
#include <cmath>

#include <cuda_bf16.h>

#include "tcgen05.cuh"
#include "wob_device.cuh"
#include "wob_host.h"

namespace wob {

constexpr int kFeat = 96;
constexpr int kWidth = 64;
constexpr int kParams = 96 * 64 + 64 + 3 * (64 * 64 + 64) + 64 + 1;  // 18753

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
// offsets (floats) of each layer's matrix and bias in the parameter vector
__host__ __device__ constexpr int w_off(int l) { return l == 0 ? 0 : 96 * 64 + 64 + (l - 1) * (64 * 64 + 64); }
__host__ __device__ constexpr int b_off(int l) { return w_off(l) + (l == 0 ? 96 * 64 : 64 * 64); }
constexpr int kW5 = 96 * 64 + 64 + 3 * (64 * 64 + 64);
constexpr int kB5 = kW5 + 64;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// SiLU and its derivative with the fast exponential and reciprocal (relative
// error ~1e-6, far below the BF16 rounding of the activations).
__device__ __forceinline__ float silu(float a) { return __fdividef(a, 1.0f + __expf(-a)); }
__device__ __forceinline__ float silu_grad(float a)
{
    const float s = __fdividef(1.0f, 1.0f + __expf(-a));
    return s * (1.0f + a * (1.0f - s));
}

// Fourier feature of column c at y: c = 32 d + 2 k + s
__device__ __forceinline__ float feature(const float y[3], int c)
{
    const int d = c >> 5, j = c & 31, k = j >> 1;
    const float f = exp2f((float)k * (1.0f / 3.0f));
    float sv, cv;
    sincospif(2.0f * f * y[d], &sv, &cv);
    return (j & 1) ? cv : sv;
}

__device__ __forceinline__ void load_point(const float* __restrict__ x, int64_t n, int64_t r,
                                           float y[3], int stride = 3)
{
    if (r < n) {
        y[0] = x[stride * r];
        y[1] = x[stride * r + 1];
        y[2] = x[stride * r + 2];
    } else {
        y[0] = y[1] = y[2] = 0.f;
    }
}

// ---------------------------------------------------------------------------
// Forward on the 5th-generation tensor cores (tcgen05).  A CTA of 512
// threads is four independent quarters of 128 threads; each quarter takes
// tiles of 128 points in turn (thread t of the quarter owns row t), so that
// one quarter's products run on the tensor cores while the others convert
// and activate (one CTA per SM: four tiles in flight).
// Per tile the features (BF16) go to the quarter's A buffer in the canonical
// K-major layout, one thread issues the layer's tcgen05.mma (M 128, N 64,
// K 16 per instruction) into the quarter's 64 FP32 columns of tensor memory,
// the commit arrives on the quarter's mbarrier, every thread loads its row of
// the accumulator (tcgen05.ld), adds the bias, applies SiLU and writes the
// BF16 activations back as the next layer's A operand.  The weights (B
// operand, W as stored: out x in = N x K, K-major) stay in shared memory for
// the whole launch.  The 64 -> 1 output layer runs in FP32 per thread on the
// BF16-rounded activations, as the tensor cores would see them.
// ---------------------------------------------------------------------------
constexpr int kTcRows = 128;
constexpr int kTcThreads = 4 * kTcRows;              // four quarters
constexpr int kTcCols = 256;                         // tensor-memory columns per CTA (64 per quarter)
constexpr int kTcOffW0 = 0;                          // 64 x 96 BF16, canonical K-major
constexpr int kTcOffW1 = kTcOffW0 + 64 * kFeat * 2;  // W1..W3: 64 x 64
constexpr int kTcOffA = kTcOffW1 + 3 * 64 * kWidth * 2;  // per quarter 128 x 96 BF16 (layers 1-3: 128 x 64)
constexpr int kTcABytes = kTcRows * kFeat * 2;
constexpr int kTcOffBias = kTcOffA + 4 * kTcABytes;       // 4 x 64 FP32
constexpr int kTcOffW5 = kTcOffBias + 4 * 64 * 4;         // 64 FP32, then b5
constexpr int kTcOffMisc = kTcOffW5 + 64 * 4 + 16;        // 4 mbarriers (8 B each), TMEM address
constexpr int kTcFwdSmem = kTcOffMisc + 48;
constexpr uint32_t kTcWaitLimit = 1u << 26;  // mbarrier polls before giving up (seconds)
// Polls of the first wait on each product (the wait that detects a failure);
// the drain of a product still in flight after a failure always takes
// kTcWaitLimit.  wob_debug_set_tc_wait_limit lowers it (0: every first wait
// gives up at once) so that tests can run the failure path.
std::atomic<uint32_t> g_tc_first_wait{kTcWaitLimit};
static_assert(kTcOffA % 1024 == 0 && kTcOffW1 % 1024 == 0 && kTcABytes % 1024 == 0,
              "operand alignment");

// One layer's matrix (64 x IN, row-major FP32 in params) into shared memory
// as BF16 in the canonical K-major layout (rows = outputs, K = inputs).
template <int IN>
__device__ __forceinline__ void load_layer_kmajor(const float* __restrict__ W, unsigned char* dst,
                                                  bool vec)
{
    constexpr int kChunks = 64 * IN / 8;  // 8 consecutive inputs of one output
    for (int c = threadIdx.x; c < kChunks; c += blockDim.x) {
        const int o = c / (IN / 8), k0 = (c % (IN / 8)) * 8;
        const float* src = W + o * IN + k0;
        float4 lo, hi;
        if (vec) {
            lo = __ldg(reinterpret_cast<const float4*>(src));
            hi = __ldg(reinterpret_cast<const float4*>(src) + 1);
        } else {
            lo = make_float4(__ldg(src), __ldg(src + 1), __ldg(src + 2), __ldg(src + 3));
            hi = make_float4(__ldg(src + 4), __ldg(src + 5), __ldg(src + 6), __ldg(src + 7));
        }
        const uint4 v = make_uint4(pack_bf16(lo.x, lo.y), pack_bf16(lo.z, lo.w),
                                   pack_bf16(hi.x, hi.y), pack_bf16(hi.z, hi.w));
        *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(o, k0, IN)) = v;
    }
}

__global__ void __launch_bounds__(kTcThreads) k_mlp_forward_tc(const float* __restrict__ params,
                                                              const float* __restrict__ x,
                                                              int stride, int64_t n,
                                                              float* __restrict__ out,
                                                              uint32_t first_wait)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int qtr = threadIdx.x >> 7, tid = threadIdx.x & 127, warp = threadIdx.x >> 5;
    float* bias = reinterpret_cast<float*>(smem + kTcOffBias);
    float* w5 = reinterpret_cast<float*>(smem + kTcOffW5);
    const uint32_t mbar = tc::smem_addr(smem + kTcOffMisc + 8 * qtr);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kTcOffMisc + 32);
    unsigned char* A = smem + kTcOffA + qtr * kTcABytes;

    // the network into shared memory, the accumulators into tensor memory
    const bool vec = (reinterpret_cast<uintptr_t>(params) & 15) == 0;
    load_layer_kmajor<kFeat>(params + w_off(0), smem + kTcOffW0, vec);
    for (int l = 1; l < 4; ++l)
        load_layer_kmajor<kWidth>(params + w_off(l), smem + kTcOffW1 + (l - 1) * 64 * kWidth * 2,
                                  vec);
    for (int i = threadIdx.x; i < 4 * 64; i += blockDim.x) bias[i] = params[b_off(i >> 6) + (i & 63)];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) w5[i] = params[kW5 + i];
    if (threadIdx.x == 0) w5[64] = params[kB5];
    if (tid == 0) tc::mbar_init(mbar, 1);
    __syncwarp();
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), kTcCols);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot + 64u * qtr;                 // this quarter's columns
    const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lanes
    constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kTcRows, 64);
    const uint32_t a_base = tc::smem_addr(A);
    const int bar = 1 + qtr;  // the quarter's named barrier
    uint32_t phase = 0;
    bool failed = false;

    const int64_t tiles = (n + kTcRows - 1) / kTcRows;
    for (int64_t tile = 4 * (int64_t)blockIdx.x + qtr; tile < tiles && !failed;
         tile += 4 * (int64_t)gridDim.x) {
        const int64_t r = tile * kTcRows + tid;
        float y[3];
        load_point(x, n, r, y, stride);
        // features of row tid: 12 chunks of 8 columns, one 16-byte store each
#pragma unroll 1
        for (int c = 0; c < kFeat / 8; ++c) {
            float f[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) f[j] = feature(y, 8 * c + j);
            *reinterpret_cast<uint4*>(A + tc::kmajor_offset(tid, 8 * c, kFeat)) =
                make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]),
                           pack_bf16(f[6], f[7]));
        }
        float o = 0.f;
        for (int l = 0; l < 4; ++l) {
            const int K = l == 0 ? kFeat : kWidth;
            tc::fence_proxy_async();
            tc::fence_before_sync();
            tc::bar_sync(bar, kTcRows);
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t b_base =
                    tc::smem_addr(smem + (l == 0 ? kTcOffW0 : kTcOffW1 + (l - 1) * 64 * kWidth * 2));
                for (int kb = 0; kb < K / 16; ++kb)
                    tc::mma_bf16(tmem, tc::smem_desc(a_base + 256 * kb, 128, K * 16),
                                 tc::smem_desc(b_base + 256 * kb, 128, K * 16), kIdesc, kb > 0);
                tc::commit(mbar);
            }
            const bool ok = tc::mbar_wait(mbar, phase, first_wait);
            if (tc::bar_sync_or(bar, kTcRows, !ok)) {  // the quarter stops together
                failed = true;
                if (!ok) tc::mbar_wait(mbar, phase, kTcWaitLimit);  // the product in flight, bounded
                break;
            }
            phase ^= 1u;
            tc::fence_after_sync();
            float h[64];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[16];
                tc::tmem_ld16(trow + 16 * q, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) h[16 * q + j] = v[j];
            }
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 64; ++j) h[j] = silu(h[j] + bias[64 * l + j]);
            if (l < 3) {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    *reinterpret_cast<uint4*>(A + tc::kmajor_offset(tid, 8 * c, kWidth)) =
                        make_uint4(pack_bf16(h[8 * c], h[8 * c + 1]), pack_bf16(h[8 * c + 2], h[8 * c + 3]),
                                   pack_bf16(h[8 * c + 4], h[8 * c + 5]),
                                   pack_bf16(h[8 * c + 6], h[8 * c + 7]));
            } else {
#pragma unroll
                for (int j = 0; j < 64; ++j)
                    o = fmaf(__bfloat162float(__float2bfloat16_rn(h[j])), w5[j], o);
                o += w5[64];
            }
        }
        if (r < n) out[r] = failed ? __int_as_float(0x7FC00000) : o;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(*tslot, kTcCols);
}

// ---------------------------------------------------------------------------
// Training step on the tensor cores: forward and backward of 128 rows per
// CTA, per-CTA partial gradients (summed in a fixed order by k_mlp_adam).
// 256 threads: thread (w, lane) owns row 32 (w % 4) + lane and the columns
// [32 (w / 4), 32 (w / 4) + 32) of every 64-wide layer.  Every product is a
// tcgen05.mma of M 128 with the accumulator in tensor memory:
//   forward   a_l = h_l W_l^T         A = h_l (K-major), B = W_l (K-major)
//   weights   dW_l^T = h_l^T da_l     A = h_l read MN-major, B = da_l read MN-major
//   inputs    dh_l = da_l W_l          A = da_l (K-major), B = W_l read MN-major
// so no operand is ever transposed: the MN-major reads see the same bytes.
// The pre-activations of the hidden layers stay in tensor memory (columns
// 64 l .. 64 l + 63) until the backward pass needs them; every h_l carries a
// column of ones after its K_l inputs, so row K_l of dW_l^T is the bias
// gradient.
// ---------------------------------------------------------------------------
constexpr int kTrainRows = 128;
constexpr int kTrThreads = 2 * kTrainRows;
constexpr int kH0Cols = kFeat + 8;   // 96 inputs, the ones column, padding
constexpr int kHCols = kWidth + 8;   // 64 inputs, the ones column, padding
constexpr int kTrOffW0 = 0;                                // W0: 64 x 96
constexpr int kTrOffW1 = kTrOffW0 + 64 * kFeat * 2;        // W1..W3: 64 x 64
constexpr int kTrOffH0 = kTrOffW1 + 3 * 64 * kWidth * 2;   // h0: 128 x 104
constexpr int kTrOffH1 = kTrOffH0 + 27 * 1024;             // h1..h3: 128 x 72 (18 KB each)
constexpr int kTrOffDA = kTrOffH1 + 3 * kTrainRows * kHCols * 2;  // da: 128 x 64
constexpr int kTrOffBias = kTrOffDA + kTrainRows * kWidth * 2;    // 4 x 64 FP32
constexpr int kTrOffW5 = kTrOffBias + 4 * 64 * 4;                 // 64 FP32 + b5
constexpr int kTrOffRed = kTrOffW5 + 64 * 4 + 16;                 // reductions across warps
constexpr int kTrRedFloats = 8 * 34 + 2 * 128;
constexpr int kTrOffMisc = kTrOffRed + kTrRedFloats * 4;          // mbarrier, TMEM address
// Slack after the last operand: the products read up to 128 MN-major rows
// of an h_l whose own buffer has fewer, and the slack keeps every operand
// read inside the block's shared memory.
constexpr int kTrainSmem = kTrOffMisc + 16 + 32 * 1024;
static_assert(kTrainRows * kH0Cols * 2 <= 27 * 1024, "h0 buffer");
static_assert(kTrainSmem <= 227 * 1024, "training tile exceeds shared memory");
static_assert(kTrOffH0 % 1024 == 0 && kTrOffH1 % 1024 == 0 && kTrOffDA % 1024 == 0,
              "operand alignment");
constexpr int kTrCols = 512;  // 4 x 64 pre-activations, 64 dh, 64 dW^T (+ unused)
constexpr uint32_t kColDX = 256, kColDW = 320;
constexpr int kSboH0 = kH0Cols * 16, kSboH = kHCols * 16, kSboDA = kWidth * 16;

// 32 FP32 columns [col, col + 32) of the calling thread's tensor-memory row.
__device__ __forceinline__ void tmem_row32(uint32_t taddr, float (&h)[32])
{
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        float v[16];
        tc::tmem_ld16(taddr + 16 * q, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) h[16 * q + j] = v[j];
    }
    tc::tmem_wait_ld();
}

// 32 values of row r, columns [c0, c0 + 32), into a K-major BF16 matrix with
// `cols` columns (four 16-byte stores).
__device__ __forceinline__ void store_row32(unsigned char* base, int r, int c0, int cols,
                                            const float (&v)[32])
{
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4*>(base + tc::kmajor_offset(r, c0 + 8 * c, cols)) =
            make_uint4(pack_bf16(v[8 * c], v[8 * c + 1]), pack_bf16(v[8 * c + 2], v[8 * c + 3]),
                       pack_bf16(v[8 * c + 4], v[8 * c + 5]), pack_bf16(v[8 * c + 6], v[8 * c + 7]));
}

__global__ void __launch_bounds__(kTrThreads, 1) k_mlp_train_tc(const float* __restrict__ params,
                                                               const float* __restrict__ x,
                                                               const float* __restrict__ target,
                                                               int64_t n,
                                                               float* __restrict__ partial,
                                                               float* __restrict__ loss_partial,
                                                               TrainCtl* __restrict__ ctl,
                                                               uint32_t first_wait)
{
    // graph-replayed steps: advance the step number (the previous step's
    // Adam update has completed; this step's reads it after this kernel)
    if (ctl && blockIdx.x == 0 && threadIdx.x == 0) ctl->step += 1;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = 32 * (warp & 3) + lane;  // the row this thread owns
    const int ch = warp >> 2;              // its half of the columns
    const int c0 = 32 * ch;
    float* bias = reinterpret_cast<float*>(smem + kTrOffBias);
    float* w5 = reinterpret_cast<float*>(smem + kTrOffW5);
    float* red = reinterpret_cast<float*>(smem + kTrOffRed);
    const uint32_t mbar = tc::smem_addr(smem + kTrOffMisc);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kTrOffMisc + 8);
    unsigned char* DA = smem + kTrOffDA;
    auto hb = [&](int l) { return smem + (l == 0 ? kTrOffH0 : kTrOffH1 + (l - 1) * kTrainRows * kHCols * 2); };
    auto wb = [&](int l) { return smem + (l == 0 ? kTrOffW0 : kTrOffW1 + (l - 1) * 64 * kWidth * 2); };

    const bool vec = (reinterpret_cast<uintptr_t>(params) & 15) == 0;
    load_layer_kmajor<kFeat>(params + w_off(0), wb(0), vec);
    for (int l = 1; l < 4; ++l) load_layer_kmajor<kWidth>(params + w_off(l), wb(l), vec);
    for (int i = threadIdx.x; i < 4 * 64; i += blockDim.x) bias[i] = params[b_off(i >> 6) + (i & 63)];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) w5[i] = params[kW5 + i];
    // the ones column (bias gradients) and the padding of every h_l
    if (ch == 0) {
        const uint4 ones = make_uint4(pack_bf16(1.f, 0.f), 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(hb(0) + tc::kmajor_offset(r, kFeat, kH0Cols)) = ones;
        for (int l = 1; l < 4; ++l)
            *reinterpret_cast<uint4*>(hb(l) + tc::kmajor_offset(r, kWidth, kHCols)) = ones;
    }
    if (threadIdx.x == 0) {
        w5[64] = params[kB5];
        tc::mbar_init(mbar, 1);
    }
    __syncwarp();
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), kTrCols);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
    constexpr uint32_t kIdFwd = tc::idesc_bf16_f32(kTrainRows, 64);
    constexpr uint32_t kIdDW = tc::idesc_bf16_f32(kTrainRows, 64, true, true);
    constexpr uint32_t kIdDX = tc::idesc_bf16_f32(kTrainRows, 64, false, true);
    uint32_t phase = 0;
    bool failed = false;

    // issue the products of one stage (thread 0), then every thread waits
    auto run = [&](auto issue) -> bool {
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            issue();
            tc::commit(mbar);
        }
        const bool ok = tc::mbar_wait(mbar, phase, first_wait);
        if (__syncthreads_or(!ok)) {
            if (!ok) tc::mbar_wait(mbar, phase, kTcWaitLimit);  // the products in flight, bounded
            return false;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        return true;
    };
    const int64_t row = (int64_t)blockIdx.x * kTrainRows + r;
    float y[3];
    load_point(x, n, row, y);
    // ---- forward: features -> h0 (this thread's 48 of the 96)
#pragma unroll 1
    for (int c = 6 * ch; c < 6 * ch + 6; ++c) {
        float f[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) f[j] = feature(y, 8 * c + j);
        *reinterpret_cast<uint4*>(hb(0) + tc::kmajor_offset(r, 8 * c, kH0Cols)) =
            make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]),
                       pack_bf16(f[6], f[7]));
    }
    float h[32];
    float out = 0.f;
    for (int l = 0; l < 4; ++l) {
        const int K = l == 0 ? kFeat : kWidth;
        const int sbo = l == 0 ? kSboH0 : kSboH;
        if (!run([&] {
                const uint32_t ab = tc::smem_addr(hb(l)), bb = tc::smem_addr(wb(l));
                for (int kb = 0; kb < K / 16; ++kb)
                    tc::mma_bf16(tmem + 64u * l, tc::smem_desc(ab + 256 * kb, 128, sbo),
                                 tc::smem_desc(bb + 256 * kb, 128, K * 16), kIdFwd, kb > 0);
            })) {
            failed = true;
            break;
        }
        tmem_row32(trow + 64u * l, h);
#pragma unroll
        for (int j = 0; j < 32; ++j) h[j] = silu(h[j] + bias[64 * l + c0 + j]);
        if (l < 3) {
            store_row32(hb(l + 1), r, c0, kHCols, h);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                h[j] = __bfloat162float(__float2bfloat16_rn(h[j]));  // h4 as the layers see it
                out = fmaf(h[j], w5[c0 + j], out);
            }
        }
    }
    float* gpart = partial + (int64_t)blockIdx.x * kParams;
    float* outs = red + 8 * 34;  // per row: the two column halves of the output
    if (!failed) {
        // ---- output layer: dout, dw5, db5, da3
        outs[ch * 128 + r] = out;
        __syncthreads();
        const float o = outs[r] + outs[128 + r] + w5[64];
        const float e = row < n ? o - target[row] : 0.f;
        const float dout = 2.f * e / (float)n;
#pragma unroll 1
        for (int j = 0; j < 32; ++j) {
            float v = dout * h[j];
            for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(kFull, v, s);
            if (lane == 0) red[warp * 34 + j] = v;
        }
        float dsum = dout, le = e * e;
        for (int s = 16; s > 0; s >>= 1) {
            dsum += __shfl_xor_sync(kFull, dsum, s);
            le += __shfl_xor_sync(kFull, le, s);
        }
        if (lane == 0) {
            red[warp * 34 + 32] = dsum;
            red[warp * 34 + 33] = le;
        }
        float a[32];
        tmem_row32(trow + 192u, a);
#pragma unroll
        for (int j = 0; j < 32; ++j) h[j] = dout * w5[c0 + j] * silu_grad(a[j] + bias[192 + c0 + j]);
        store_row32(DA, r, c0, kWidth, h);
        __syncthreads();
        if (threadIdx.x < 64) {  // w5 column j: warps 0-3 (j < 32) or 4-7
            const int j = threadIdx.x, w0 = (j >> 5) * 4, jj = j & 31;
            gpart[kW5 + j] = ((red[w0 * 34 + jj] + red[(w0 + 1) * 34 + jj]) +
                              red[(w0 + 2) * 34 + jj]) + red[(w0 + 3) * 34 + jj];
        } else if (threadIdx.x == 64) {
            gpart[kB5] = ((red[32] + red[34 + 32]) + red[68 + 32]) + red[102 + 32];
            loss_partial[blockIdx.x] = ((red[33] + red[34 + 33]) + red[68 + 33]) + red[102 + 33];
        }
        // ---- layers 3 .. 0: weight gradients, then the previous layer's da
        for (int l = 3; l >= 0; --l) {
            const int K = l == 0 ? kFeat : kWidth;
            const int sbo = l == 0 ? kSboH0 : kSboH;
            if (!run([&] {
                    const uint32_t hbase = tc::smem_addr(hb(l)), dbase = tc::smem_addr(DA);
                    for (int kb = 0; kb < kTrainRows / 16; ++kb)
                        tc::mma_bf16(tmem + kColDW, tc::smem_desc(hbase + 2 * sbo * kb, sbo, 128),
                                     tc::smem_desc(dbase + 2 * kSboDA * kb, kSboDA, 128), kIdDW,
                                     kb > 0);
                    if (l > 0) {
                        const uint32_t wbase = tc::smem_addr(wb(l));
                        for (int kb = 0; kb < kWidth / 16; ++kb)
                            tc::mma_bf16(tmem + kColDX, tc::smem_desc(dbase + 256 * kb, 128, kSboDA),
                                         tc::smem_desc(wbase + 2 * (kWidth * 16) * kb, kWidth * 16, 128),
                                         kIdDX, kb > 0);
                    }
                })) {
                failed = true;
                break;
            }
            float g[32];
            tmem_row32(trow + kColDW, g);  // row r of dW_l^T: input r, outputs c0 .. c0 + 31
            if (r < K) {
                for (int j = 0; j < 32; ++j) gpart[w_off(l) + (c0 + j) * K + r] = g[j];
            } else if (r == K) {
                for (int j = 0; j < 32; ++j) gpart[b_off(l) + c0 + j] = g[j];
            }
            if (l == 0) break;
            tmem_row32(trow + kColDX, g);
            tmem_row32(trow + 64u * (l - 1), a);
#pragma unroll
            for (int j = 0; j < 32; ++j) h[j] = g[j] * silu_grad(a[j] + bias[64 * (l - 1) + c0 + j]);
            store_row32(DA, r, c0, kWidth, h);
        }
    }
    if (failed) {  // a wait gave up: this block's gradients and loss are NaN
        __syncthreads();
        for (int i = threadIdx.x; i < kParams; i += blockDim.x) gpart[i] = __int_as_float(0x7FC00000);
        if (threadIdx.x == 0) loss_partial[blockIdx.x] = __int_as_float(0x7FC00000);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, kTrCols);
}

// Sum the per-block partial gradients in block order, then one Adam step
// (Kingma & Ba 2015, bias-corrected) on the FP32 master weights.
__global__ void k_mlp_adam(float* __restrict__ params, float* __restrict__ m,
                           float* __restrict__ v, const float* __restrict__ partial, int blocks,
                           float* __restrict__ grad_out, float lr, float b1, float b2, float eps,
                           int step, const TrainCtl* __restrict__ ctl,
                           const float* __restrict__ lp, float n, float* __restrict__ loss_out)
{
    if (ctl) {  // graph-replayed steps: step number and rate from device memory
        step = ctl->step;
        lr = ctl->lr;
    }
    if (loss_out && blockIdx.x == 0 && threadIdx.x < 32) {
        // loss = (sum of the blocks' squared errors, in block order) / n
        float ls = 0.f;
        for (int b = threadIdx.x; b < blocks; b += 32) ls += lp[b];
        for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(kFull, ls, o);
        if (threadIdx.x == 0) *loss_out = ls / n;
    }
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
        float gsum = 0.f;
#pragma unroll 8
        for (int b = 0; b < blocks; ++b) gsum += partial[(int64_t)b * kParams + i];
        if (grad_out) grad_out[i] = gsum;
        if (lr == 0.f) continue;
        const float mi = b1 * m[i] + (1.f - b1) * gsum;
        const float vi = b2 * v[i] + (1.f - b2) * gsum * gsum;
        m[i] = mi;
        v[i] = vi;
        params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_train_ctl(TrainCtl* ctl, int step, float lr, int set_step)
{
    if (set_step) ctl->step = step;
    ctl->lr = lr;
}

// He-uniform initial weights from the counter-based stream: parameter i
// (flat index) of a weight matrix with fan-in f is sqrt(6 / f) (2 u - 1),
// u = u24 of the first word of block (i, 0, 0 | init purpose, 0); biases 0.
__global__ void k_mlp_init(float* __restrict__ params, uint32_t key0, uint32_t key1)
{
    const StreamKey key{key0, key1};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
        int l = 0;
        while (l < 4 && i >= w_off(l + 1)) ++l;
        const int fan_in = l == 0 ? kFeat : kWidth;
        const int wend = l < 4 ? b_off(l) : kB5;
        if (i >= wend) {
            params[i] = 0.f;
            continue;
        }
        const u32x4 u = stream_block(key, (uint32_t)i, 0u, 0u, kPurposeInit, 0u, 0u);
        const float lim = sqrtf(6.0f / (float)fan_in);
        params[i] = lim * (2.0f * u24f(u.x) - 1.0f);
    }
}

// The kernels' dynamic shared memory above 48 KB must be allowed once per
// device (a function attribute of each device's context); one bit per
// device, set by whichever thread configures it first.
std::atomic<unsigned long long> g_fwd_configured{0}, g_train_configured{0};

int allow_smem(std::atomic<unsigned long long>& done, const void* kernel, int bytes)
{
    int dev = 0;
    WOB_CUDA_TRY(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return WOB_OK;
    WOB_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done.fetch_or(bit, std::memory_order_release);
    return WOB_OK;
}

}  // namespace

int mlp_forward(const float* params, const float* x, int64_t n, float* out, cudaStream_t s,
                int stride)
{
    if (n <= 0) return WOB_OK;
    WOB_TRY(allow_smem(g_fwd_configured, (const void*)k_mlp_forward_tc, kTcFwdSmem));
    const int64_t tiles = (n + kTcRows - 1) / kTcRows;
    const int grid = grid_for((const void*)k_mlp_forward_tc, kTcThreads, kTcFwdSmem,
                              (tiles + 3) / 4 * kTcThreads);
    k_mlp_forward_tc<<<grid, kTcThreads, kTcFwdSmem, s>>>(params, x, stride, n, out,
                                                          g_tc_first_wait.load());
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int64_t mlp_train_workspace(int64_t n)
{
    const int64_t blocks = (n + kTrainRows - 1) / kTrainRows;
    return blocks * (kParams + 1);
}

int mlp_train_step_ws(float* params, float* m, float* v, const float* x, const float* target,
                      int64_t n, float lr, int step, float* grad_out, float* loss_out, float* ws,
                      cudaStream_t s, TrainCtl* ctl)
{
    if (n <= 0) return WOB_OK;
    WOB_TRY(allow_smem(g_train_configured, (const void*)k_mlp_train_tc, kTrainSmem));
    const int blocks = (int)((n + kTrainRows - 1) / kTrainRows);
    float* partial = ws;
    float* lp = ws + (int64_t)blocks * kParams;
    k_mlp_train_tc<<<blocks, kTrThreads, kTrainSmem, s>>>(params, x, target, n, partial, lp, ctl,
                                                          g_tc_first_wait.load());
    WOB_CUDA_TRY(cudaGetLastError());
    k_mlp_adam<<<(kParams + 255) / 256, 256, 0, s>>>(params, m, v, partial, blocks, grad_out, lr,
                                                     0.9f, 0.999f, 1e-8f, step, ctl, lp, (float)n,
                                                     loss_out);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int train_ctl_set(TrainCtl* ctl, int step, float lr, bool set_step, cudaStream_t s)
{
    k_train_ctl<<<1, 1, 0, s>>>(ctl, step, lr, set_step ? 1 : 0);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int mlp_train_prepare()
{
    return allow_smem(g_train_configured, (const void*)k_mlp_train_tc, kTrainSmem);
}

int mlp_train_step(float* params, float* m, float* v, const float* x, const float* target,
                   int64_t n, float lr, int step, float* grad_out, float* loss_out,
                   cudaStream_t s)
{
    if (n <= 0) return WOB_OK;
    float* ws = nullptr;
    WOB_CUDA_TRY(cudaMallocAsync((void**)&ws, (size_t)mlp_train_workspace(n) * sizeof(float), s));
    const int rc = mlp_train_step_ws(params, m, v, x, target, n, lr, step, grad_out, loss_out, ws, s);
    cudaFreeAsync(ws, s);
    if (rc != WOB_OK) set_error("MLP training step failed");
    return rc;
}

}  // namespace wob

extern "C" {

int wob_mlp_num_params(void) { return wob::kParams; }

int wob_mlp_init(float* params, uint64_t seed, void* stream)
{
    wob::clear_error();
    if (!params) {
        wob::set_error("wob_mlp_init: NULL params");
        return WOB_ERR_INVALID_ARG;
    }
    wob::k_mlp_init<<<(wob::kParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        params, (uint32_t)seed, (uint32_t)(seed >> 32));
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int wob_debug_set_tc_wait_limit(uint32_t polls, uint32_t* previous)
{
    wob::clear_error();
    const uint32_t old = wob::g_tc_first_wait.exchange(polls);
    if (previous) *previous = old;
    return WOB_OK;
}

int wob_mlp_forward(const float* params, const float* x, int64_t n, float* out, void* stream)
{
    wob::clear_error();
    if (n < 0 || (n > 0 && (!params || !x || !out))) {
        wob::set_error("wob_mlp_forward: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    return wob::mlp_forward(params, x, n, out, (cudaStream_t)stream, 3);
}

int wob_mlp_train_step(float* params, float* adam_m, float* adam_v, const float* x,
                       const float* target, int64_t n, float lr, int32_t step, float* grad_out,
                       float* loss_out, void* stream)
{
    wob::clear_error();
    if (n < 0 || (n > 0 && (!params || !adam_m || !adam_v || !x || !target)) || step < 1 ||
        !(lr >= 0.f)) {
        wob::set_error("wob_mlp_train_step: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    return wob::mlp_train_step(params, adam_m, adam_v, x, target, n, lr, step, grad_out, loss_out,
                               (cudaStream_t)stream);
}

}  // extern "C"
