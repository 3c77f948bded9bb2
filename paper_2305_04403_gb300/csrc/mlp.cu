// mlp.cu -- the control variate's network on the tensor cores:
// Fourier features (16 frequencies 2^(k/3), sin and cos of 2 pi f y_d:
// 96 inputs) -> 4 x (64, SiLU) -> 1.  BF16 operands, FP32 accumulation,
// mma.sync.m16n8k16; FP32 master weights (out x in layout, biases after
// each matrix) and Adam state in device memory.
//
// Layouts (m16n8k16, g = lane / 4, t = lane % 4):
//   A (16 x 16, row-major): regs (row g, k 2t..2t+1), (row g+8, k 2t..),
//                           (row g, k 8+2t..), (row g+8, k 8+2t..)
//   B (16 x 8, "col"):      regs (k 2t.., n g), (k 8+2t.., n g)
//   C (16 x 8, f32):        (row g, n 2t), (row g, n 2t+1), (row g+8, n 2t), (row g+8, n 2t+1)
// so the C tiles 2j and 2j+1 of one layer are, after the activation, exactly
// the A fragment of k-block j of the next layer (kept in registers).
#include <atomic>
#include <cmath>

#include <cuda_bf16.h>

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

constexpr int kLd1 = kFeat + 8;   // smem row stride (bf16) of a 96-wide matrix
constexpr int kLd = kWidth + 8;   // of a 64-wide matrix

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t (&r)[4], const void* p)
{
    const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ float silu(float a) { return a / (1.0f + __expf(-a)); }
__device__ __forceinline__ float silu_grad(float a)
{
    const float s = 1.0f / (1.0f + __expf(-a));
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

// Weights into shared memory as BF16: Wt[l] = [out][in] (forward B operand)
// and optionally, for layers 1..3, W[l] = [in][out] (the B operand of the
// backward product da . W; layer 0's input gradient is never needed).
struct SmemNet {
    __nv_bfloat16* wt[4];
    __nv_bfloat16* w[4];
    float* bias;  // 4 x 64
    float* w5;    // 64
    float b5;
};

// One layer's matrix (64 x IN, row-major FP32) into shared memory as BF16.
// 128 threads; every thread issues all of its float4 loads before any
// store, so the loads are in flight together.
template <int IN>
__device__ __forceinline__ void load_layer(const float* __restrict__ W, __nv_bfloat16* wt,
                                           __nv_bfloat16* w, bool vec)
{
    constexpr int kLdIn = IN == kFeat ? kLd1 : kLd;
    constexpr int kPer = 64 * IN / 4 / 128;  // float4 per thread
    static_assert(64 * IN % (4 * 128) == 0, "layer size");
    float4 r[kPer];
    if (vec) {
        const float4* W4 = reinterpret_cast<const float4*>(W);
#pragma unroll
        for (int u = 0; u < kPer; ++u) r[u] = __ldg(W4 + threadIdx.x + 128 * u);
    } else {
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const float* p = W + 4 * (threadIdx.x + 128 * u);
            r[u] = make_float4(__ldg(p), __ldg(p + 1), __ldg(p + 2), __ldg(p + 3));
        }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = 4 * (threadIdx.x + 128 * u);
        const int o = i / IN, k = i - o * IN;  // 4 consecutive k of row o
        const __nv_bfloat16 b[4] = {__float2bfloat16_rn(r[u].x), __float2bfloat16_rn(r[u].y),
                                    __float2bfloat16_rn(r[u].z), __float2bfloat16_rn(r[u].w)};
        __nv_bfloat16* d = wt + o * kLdIn + k;
        *reinterpret_cast<uint2*>(d) =
            make_uint2((uint32_t)__bfloat16_as_ushort(b[0]) | ((uint32_t)__bfloat16_as_ushort(b[1]) << 16),
                       (uint32_t)__bfloat16_as_ushort(b[2]) | ((uint32_t)__bfloat16_as_ushort(b[3]) << 16));
        if (w)
            for (int c = 0; c < 4; ++c) w[(k + c) * kLd + o] = b[c];
    }
}

// The network into shared memory (launched with 128 threads).
__device__ void load_net(const float* __restrict__ params, SmemNet& n, bool with_transposed)
{
    const bool vec = (reinterpret_cast<uintptr_t>(params) & 15) == 0;
    load_layer<kFeat>(params + w_off(0), n.wt[0], nullptr, vec);
    for (int l = 1; l < 4; ++l)
        load_layer<kWidth>(params + w_off(l), n.wt[l], with_transposed ? n.w[l] : nullptr, vec);
    for (int i = threadIdx.x; i < 4 * 64; i += blockDim.x)
        n.bias[i] = params[b_off(i >> 6) + (i & 63)];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) n.w5[i] = params[kW5 + i];
    n.b5 = params[kB5];
    __syncthreads();
}

// Forward of one 16-row tile held by a warp.  Features at rows r0 = g and
// r1 = g + 8 of the tile (ya, yb); returns the outputs of those rows.
// Optionally stores pre-activations (FP32) and activations (BF16) of every
// layer for the backward pass (row stride kLd / kLd1 per layer buffer).
template <bool STORE>
__device__ __forceinline__ void forward_tile(const SmemNet& n, const float ya[3], const float yb[3],
                                             float& out_a, float& out_b, float* const* pre,
                                             __nv_bfloat16* const* act, int row0)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t A[6][4];
    for (int kb = 0; kb < 6; ++kb) {
        const int c = 16 * kb + 2 * t;
        A[kb][0] = pack_bf16(feature(ya, c), feature(ya, c + 1));
        A[kb][1] = pack_bf16(feature(yb, c), feature(yb, c + 1));
        A[kb][2] = pack_bf16(feature(ya, c + 8), feature(ya, c + 9));
        A[kb][3] = pack_bf16(feature(yb, c + 8), feature(yb, c + 9));
        if (STORE) {
            __nv_bfloat16* h0 = act[0];
            *reinterpret_cast<uint32_t*>(h0 + (row0 + g) * kLd1 + c) = A[kb][0];
            *reinterpret_cast<uint32_t*>(h0 + (row0 + g + 8) * kLd1 + c) = A[kb][1];
            *reinterpret_cast<uint32_t*>(h0 + (row0 + g) * kLd1 + c + 8) = A[kb][2];
            *reinterpret_cast<uint32_t*>(h0 + (row0 + g + 8) * kLd1 + c + 8) = A[kb][3];
        }
    }
    float H[8][4];
    int kblocks = 6;
    for (int l = 0; l < 4; ++l) {
        const int ld_in = l == 0 ? kLd1 : kLd;
        const __nv_bfloat16* wt = n.wt[l];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            const __nv_bfloat16* brow = wt + (nt * 8 + g) * ld_in + 2 * t;
            for (int kb = 0; kb < kblocks; ++kb) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(brow + 16 * kb);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(brow + 16 * kb + 8);
                mma_bf16(c, A[kb], b0, b1);
            }
            const float bias0 = n.bias[l * 64 + nt * 8 + 2 * t];
            const float bias1 = n.bias[l * 64 + nt * 8 + 2 * t + 1];
            H[nt][0] = c[0] + bias0;
            H[nt][1] = c[1] + bias1;
            H[nt][2] = c[2] + bias0;
            H[nt][3] = c[3] + bias1;
            if (STORE) {
                float* p = pre[l];
                const int col = nt * 8 + 2 * t;
                p[(row0 + g) * kLd + col] = H[nt][0];
                p[(row0 + g) * kLd + col + 1] = H[nt][1];
                p[(row0 + g + 8) * kLd + col] = H[nt][2];
                p[(row0 + g + 8) * kLd + col + 1] = H[nt][3];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) H[nt][i] = silu(H[nt][i]);
        }
        // activations -> A fragments of the next layer
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
            A[kb][0] = pack_bf16(H[2 * kb][0], H[2 * kb][1]);
            A[kb][1] = pack_bf16(H[2 * kb][2], H[2 * kb][3]);
            A[kb][2] = pack_bf16(H[2 * kb + 1][0], H[2 * kb + 1][1]);
            A[kb][3] = pack_bf16(H[2 * kb + 1][2], H[2 * kb + 1][3]);
            if (STORE) {
                __nv_bfloat16* h = act[l + 1];
                const int c = 16 * kb + 2 * t;
                *reinterpret_cast<uint32_t*>(h + (row0 + g) * kLd + c) = A[kb][0];
                *reinterpret_cast<uint32_t*>(h + (row0 + g + 8) * kLd + c) = A[kb][1];
                *reinterpret_cast<uint32_t*>(h + (row0 + g) * kLd + c + 8) = A[kb][2];
                *reinterpret_cast<uint32_t*>(h + (row0 + g + 8) * kLd + c + 8) = A[kb][3];
            }
        }
        kblocks = 4;
    }
    // output layer (64 -> 1) in FP32 on the last activations (rounded as
    // the next layer would see them), reduced over the 4 lanes of a row
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + 2 * t;
        const float w0 = n.w5[col], w1 = n.w5[col + 1];
        sa += __bfloat162float(__float2bfloat16_rn(H[nt][0])) * w0 +
              __bfloat162float(__float2bfloat16_rn(H[nt][1])) * w1;
        sb += __bfloat162float(__float2bfloat16_rn(H[nt][2])) * w0 +
              __bfloat162float(__float2bfloat16_rn(H[nt][3])) * w1;
    }
    sa += __shfl_xor_sync(kFull, sa, 1);
    sa += __shfl_xor_sync(kFull, sa, 2);
    sb += __shfl_xor_sync(kFull, sb, 1);
    sb += __shfl_xor_sync(kFull, sb, 2);
    out_a = sa + n.b5;
    out_b = sb + n.b5;
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

constexpr int kFwdSmem = 64 * kLd1 * 2 + 3 * 64 * kLd * 2 + 4 * 64 * 4 + 64 * 4;

__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ params,
                                                     const float* __restrict__ x, int stride,
                                                     int64_t n, float* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemNet net;
    unsigned char* p = smem;
    net.wt[0] = (__nv_bfloat16*)p;
    p += 64 * kLd1 * 2;
    for (int l = 1; l < 4; ++l) {
        net.wt[l] = (__nv_bfloat16*)p;
        p += 64 * kLd * 2;
    }
    net.bias = (float*)p;
    p += 4 * 64 * 4;
    net.w5 = (float*)p;
    load_net(params, net, false);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2;
    const int64_t tiles = (n + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < tiles; tile += (int64_t)gridDim.x * 4) {
        const int64_t ra = tile * 16 + g, rb = ra + 8;
        float ya[3], yb[3];
        load_point(x, n, ra, ya, stride);
        load_point(x, n, rb, yb, stride);
        float oa, ob;
        forward_tile<false>(net, ya, yb, oa, ob, nullptr, nullptr, 0);
        if ((lane & 3) == 0) {
            if (ra < n) out[ra] = oa;
            if (rb < n) out[rb] = ob;
        }
    }
}

// ---------------------------------------------------------------------------
// training step: forward + backward of 64 rows per block, per-block partial
// gradients (reduced in a fixed order by k_mlp_adam)
// ---------------------------------------------------------------------------
constexpr int kTrainRows = 64;
// shared-memory layout of the training kernel (byte offsets); the size the
// kernel is launched with is the end of the last region
constexpr int kOffWt = 0;                                   // Wt[0..3]
constexpr int kOffW = kOffWt + 64 * kLd1 * 2 + 3 * 64 * kLd * 2;  // W[1..3], [64][kLd]
constexpr int kOffBias = kOffW + 3 * 64 * kLd * 2;          // bias 4 x 64, w5 64
constexpr int kOffAct = kOffBias + 4 * 64 * 4 + 64 * 4;     // h0 [rows][kLd1], h1..h4 [rows][kLd]
constexpr int kOffPre = kOffAct + kTrainRows * kLd1 * 2 + 4 * kTrainRows * kLd * 2;  // a1..a4 FP32
constexpr int kOffDa = kOffPre + 4 * kTrainRows * kLd * 4;  // da (BF16, current layer)
constexpr int kOffDout = kOffDa + kTrainRows * kLd * 2;     // dL/dout per row
constexpr int kTrainSmem = kOffDout + kTrainRows * 4;
static_assert(kTrainSmem <= 227 * 1024, "training tile exceeds shared memory");
static_assert(kOffW % 16 == 0 && kOffAct % 16 == 0 && kOffPre % 16 == 0 && kOffDa % 16 == 0,
              "ldmatrix rows need 16-byte alignment");

__global__ void __launch_bounds__(128) k_mlp_train(const float* __restrict__ params,
                                                   const float* __restrict__ x,
                                                   const float* __restrict__ target, int64_t n,
                                                   float* __restrict__ partial,
                                                   float* __restrict__ loss_partial)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemNet net;
    net.wt[0] = (__nv_bfloat16*)(smem + kOffWt);
    for (int l = 1; l < 4; ++l)
        net.wt[l] = (__nv_bfloat16*)(smem + kOffWt + 64 * kLd1 * 2 + (l - 1) * 64 * kLd * 2);
    net.w[0] = nullptr;
    for (int l = 1; l < 4; ++l) net.w[l] = (__nv_bfloat16*)(smem + kOffW + (l - 1) * 64 * kLd * 2);
    net.bias = (float*)(smem + kOffBias);
    net.w5 = net.bias + 4 * 64;
    __nv_bfloat16* act[5];
    act[0] = (__nv_bfloat16*)(smem + kOffAct);
    for (int l = 1; l < 5; ++l)
        act[l] = (__nv_bfloat16*)(smem + kOffAct + kTrainRows * kLd1 * 2 + (l - 1) * kTrainRows * kLd * 2);
    float* pre[4];
    for (int l = 0; l < 4; ++l) pre[l] = (float*)(smem + kOffPre + l * kTrainRows * kLd * 4);
    __nv_bfloat16* da = (__nv_bfloat16*)(smem + kOffDa);
    float* dout = (float*)(smem + kOffDout);

    load_net(params, net, true);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int64_t row_base = (int64_t)blockIdx.x * kTrainRows;
    const int row0 = warp * 16;

    // forward, storing activations
    {
        const int64_t ra = row_base + row0 + g, rb = ra + 8;
        float ya[3], yb[3];
        load_point(x, n, ra, ya);
        load_point(x, n, rb, yb);
        float oa, ob;
        forward_tile<true>(net, ya, yb, oa, ob, pre, act, row0);
        // dL/dout of the mean squared error over the n samples
        if (t == 0) {
            const float ea = ra < n ? oa - target[ra] : 0.f;
            const float eb = rb < n ? ob - target[rb] : 0.f;
            dout[row0 + g] = 2.f * ea / (float)n;
            dout[row0 + g + 8] = 2.f * eb / (float)n;
            atomicAdd(loss_partial + blockIdx.x, ea * ea + eb * eb);
        }
    }
    __syncthreads();
    float* gpart = partial + (int64_t)blockIdx.x * kParams;

    // output layer: dw5[j] = sum_r dout[r] h4[r][j]; db5 = sum_r dout[r];
    // da4[r][j] = dout[r] w5[j] silu'(a4[r][j])
    for (int j = threadIdx.x; j < 64; j += blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < kTrainRows; ++r) s += dout[r] * __bfloat162float(act[4][r * kLd + j]);
        gpart[kW5 + j] = s;
    }
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int r = 0; r < kTrainRows; ++r) s += dout[r];
        gpart[kB5] = s;
    }
    for (int i = threadIdx.x; i < kTrainRows * 64; i += blockDim.x) {
        const int r = i >> 6, j = i & 63;
        const float v = dout[r] * net.w5[j] * silu_grad(pre[3][r * kLd + j]);
        da[r * kLd + j] = __float2bfloat16_rn(v);
    }
    __syncthreads();

    for (int l = 3; l >= 0; --l) {
        const int in = l == 0 ? kFeat : kWidth;
        const int ld_in = l == 0 ? kLd1 : kLd;
        const __nv_bfloat16* h_in = act[l];
        // bias gradient: column sums of da
        for (int j = threadIdx.x; j < 64; j += blockDim.x) {
            float s = 0.f;
            for (int r = 0; r < kTrainRows; ++r) s += __bfloat162float(da[r * kLd + j]);
            gpart[b_off(l) + j] = s;
        }
        // dW[o][i] = sum_r da[r][o] h[r][i]: warp w owns outputs 16w..16w+15
        {
            const int m0 = warp * 16;
            const int n_tiles = in / 8;
            float C[12][4];
            for (int nt = 0; nt < n_tiles; ++nt)
                for (int i = 0; i < 4; ++i) C[nt][i] = 0.f;
            for (int kb = 0; kb < kTrainRows / 16; ++kb) {
                uint32_t A[4];
                {
                    const int mat = lane >> 3, j = lane & 7;
                    const int k = kb * 16 + (mat >> 1) * 8 + j;
                    const int m = m0 + (mat & 1) * 8;
                    ldmatrix_x4_trans(A, da + k * kLd + m);
                }
                for (int nt = 0; nt < n_tiles; nt += 2) {
                    uint32_t B[4];
                    const int mat = lane >> 3, j = lane & 7;
                    const int k = kb * 16 + (mat & 1) * 8 + j;
                    const int ncol = (nt + (mat >> 1)) * 8;
                    ldmatrix_x4_trans(B, h_in + k * ld_in + ncol);
                    mma_bf16(C[nt], A, B[0], B[1]);
                    mma_bf16(C[nt + 1], A, B[2], B[3]);
                }
            }
            for (int nt = 0; nt < n_tiles; ++nt) {
                const int col = nt * 8 + 2 * t;
                gpart[w_off(l) + (m0 + g) * in + col] = C[nt][0];
                gpart[w_off(l) + (m0 + g) * in + col + 1] = C[nt][1];
                gpart[w_off(l) + (m0 + g + 8) * in + col] = C[nt][2];
                gpart[w_off(l) + (m0 + g + 8) * in + col + 1] = C[nt][3];
            }
        }
        if (l == 0) break;
        __syncthreads();
        // dh_{l-1}[r][i] = sum_o da[r][o] W[o][i]; da_{l-1} = dh * silu'(a_{l-1})
        {
            float C[8][4];
            for (int nt = 0; nt < 8; ++nt)
                for (int i = 0; i < 4; ++i) C[nt][i] = 0.f;
            for (int kb = 0; kb < 4; ++kb) {
                uint32_t A[4];
                const int c = 16 * kb + 2 * t;
                A[0] = *reinterpret_cast<const uint32_t*>(da + (row0 + g) * kLd + c);
                A[1] = *reinterpret_cast<const uint32_t*>(da + (row0 + g + 8) * kLd + c);
                A[2] = *reinterpret_cast<const uint32_t*>(da + (row0 + g) * kLd + c + 8);
                A[3] = *reinterpret_cast<const uint32_t*>(da + (row0 + g + 8) * kLd + c + 8);
                for (int nt = 0; nt < 8; ++nt) {
                    // B[k = o][n = i] = W[o][i]: stored transposed as w[i][o]
                    const __nv_bfloat16* brow = net.w[l] + (nt * 8 + g) * kLd + 16 * kb + 2 * t;
                    mma_bf16(C[nt], A, *reinterpret_cast<const uint32_t*>(brow),
                             *reinterpret_cast<const uint32_t*>(brow + 8));
                }
            }
            __syncthreads();  // every warp has read da
            for (int nt = 0; nt < 8; ++nt) {
                const int col = nt * 8 + 2 * t;
                const float* a = pre[l - 1];
                da[(row0 + g) * kLd + col] = __float2bfloat16_rn(C[nt][0] * silu_grad(a[(row0 + g) * kLd + col]));
                da[(row0 + g) * kLd + col + 1] = __float2bfloat16_rn(C[nt][1] * silu_grad(a[(row0 + g) * kLd + col + 1]));
                da[(row0 + g + 8) * kLd + col] = __float2bfloat16_rn(C[nt][2] * silu_grad(a[(row0 + g + 8) * kLd + col]));
                da[(row0 + g + 8) * kLd + col + 1] = __float2bfloat16_rn(C[nt][3] * silu_grad(a[(row0 + g + 8) * kLd + col + 1]));
            }
        }
        __syncthreads();
    }
}

// Sum the per-block partial gradients in block order, then one Adam step
// (Kingma & Ba 2015, bias-corrected) on the FP32 master weights.
__global__ void k_mlp_adam(float* __restrict__ params, float* __restrict__ m,
                           float* __restrict__ v, const float* __restrict__ partial, int blocks,
                           float* __restrict__ grad_out, float lr, float b1, float b2, float eps,
                           int step)
{
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

// loss = (sum of the blocks' squared errors, in block order) / n
__global__ void k_mlp_loss(const float* __restrict__ lp, int blocks, float n, float* out)
{
    float s = 0.f;
    for (int b = threadIdx.x; b < blocks; b += 32) s += lp[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (threadIdx.x == 0) *out = s / n;
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
    WOB_TRY(allow_smem(g_fwd_configured, (const void*)k_mlp_forward, kFwdSmem));
    const int64_t tiles = (n + 15) / 16;
    const int grid = grid_for((const void*)k_mlp_forward, 128, kFwdSmem, tiles * 32);
    k_mlp_forward<<<grid, 128, kFwdSmem, s>>>(params, x, stride, n, out);
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
                      cudaStream_t s)
{
    if (n <= 0) return WOB_OK;
    WOB_TRY(allow_smem(g_train_configured, (const void*)k_mlp_train, kTrainSmem));
    const int blocks = (int)((n + kTrainRows - 1) / kTrainRows);
    float* partial = ws;
    float* lp = ws + (int64_t)blocks * kParams;
    WOB_CUDA_TRY(cudaMemsetAsync(lp, 0, blocks * sizeof(float), s));
    k_mlp_train<<<blocks, 128, kTrainSmem, s>>>(params, x, target, n, partial, lp);
    WOB_CUDA_TRY(cudaGetLastError());
    k_mlp_adam<<<(kParams + 255) / 256, 256, 0, s>>>(params, m, v, partial, blocks, grad_out, lr,
                                                     0.9f, 0.999f, 1e-8f, step);
    WOB_CUDA_TRY(cudaGetLastError());
    if (loss_out) {
        k_mlp_loss<<<1, 32, 0, s>>>(lp, blocks, (float)n, loss_out);
        WOB_CUDA_TRY(cudaGetLastError());
    }
    return WOB_OK;
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
