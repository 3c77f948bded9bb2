// wob_device.cuh -- device-side building blocks shared by the library's
// kernels: the counter-based generator, line-axis sampling, the BVH node
// layout and the all-hits line traversal.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "wob_internal.h"

namespace wob {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Each round multiplies
// counter words 0 and 2 by the two round constants (full 64-bit products),
// xors the high halves with the other counter words and the round key, and
// the key is bumped by the two Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct u32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// Stream addressing: key (seed_lo ^ problem, seed_hi), counter
// (query, walk, step << 16 | purpose << 12 | attempt, extra).
struct StreamKey {
    uint32_t k0, k1;
};

__device__ __forceinline__ u32x4 stream_block(StreamKey key, uint32_t q, uint32_t walk,
                                              uint32_t step, uint32_t purpose,
                                              uint32_t attempt, uint32_t extra)
{
    return philox4x32_10(q, walk, (step << 16) | (purpose << 12) | attempt, extra, key.k0,
                         key.k1);
}

__device__ __forceinline__ double u24(uint32_t x) { return (double)(x >> 8) * 0x1p-24; }
__device__ __forceinline__ float u24f(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }
__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo)
{
    return (double)((((uint64_t)hi) << 21) | (uint64_t)(lo >> 11)) * 0x1p-53;
}

// Line axis uniform on the sphere (Marsaglia 1972): (a, b) uniform in the
// square [-1, 1]^2 on the odd multiples of 2^-24, accepted when
// a^2 + b^2 < 1 (an exact integer test), then
// d = (2 a sqrt(1 - s), 2 b sqrt(1 - s), 1 - 2 s).  Computed in double; the
// operations are exact except for the correctly rounded sqrt and one
// product, so the axis is bit-reproducible.
__device__ __forceinline__ double3 line_axis(StreamKey key, uint32_t q, uint32_t walk,
                                             uint32_t step)
{
    for (uint32_t call = 0; call < 256u; ++call) {
        const u32x4 x = stream_block(key, q, walk, step, kPurposeDir, call, 0u);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const uint32_t xa = a ? x.z : x.x;
            const uint32_t xb = a ? x.w : x.y;
            const int64_t A = 2 * (int64_t)(xa >> 8) - (int64_t(1) << 24) + 1;
            const int64_t B = 2 * (int64_t)(xb >> 8) - (int64_t(1) << 24) + 1;
            const int64_t S = A * A + B * B;
            if (S < (int64_t(1) << 48)) {
                const double av = (double)A * 0x1p-24;
                const double bv = (double)B * 0x1p-24;
                const double s = (double)S * 0x1p-48;
                const double root = __dsqrt_rn(1.0 - s);
                return make_double3(__dmul_rn(2.0 * av, root), __dmul_rn(2.0 * bv, root),
                                    1.0 - 2.0 * s);
            }
        }
    }
    return make_double3(0.0, 0.0, 1.0);
}

// ---------------------------------------------------------------------------
// BVH layout.  A node holds the boxes of both children (so one 64-byte fetch
// decides which children the line meets) and two child references:
//   ref >= 0 : interior node index
//   ref <  0 : leaf, ~ref = first << 3 | (count - 1), triangles
//              tv[3 * first .. 3 * (first + count) - 1] in leaf order.
//   n0 = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   n1 = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   n2 = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   n3 = (ref0, ref1, -, -) as int bits
// Triangle in leaf order: tv[3p] = (v0, original id bits), tv[3p+1] =
// (v1, |(v1-v0) x (v2-v0)|), tv[3p+2] = (v2, 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int leaf_first(int ref) { return (~ref) >> 3; }
__device__ __forceinline__ int leaf_count(int ref) { return ((~ref) & 7) + 1; }

struct LinePre {
    float ox, oy, oz;     // origin
    float ix, iy, iz;     // 1 / d (guarded)
    float oix, oiy, oiz;  // o / d
    // Woop-Benthin-Wald watertight shear
    int kx, ky, kz;
    float Sx, Sy, Sz;
    float dkz_abs;
};

__device__ __forceinline__ float guard_inv(float d)
{
    const float a = fabsf(d) < 1e-20f ? copysignf(1e-20f, d) : d;
    return 1.0f / a;
}

__device__ __forceinline__ float comp(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ LinePre line_pre(float3 o, float3 d)
{
    LinePre L;
    L.ox = o.x; L.oy = o.y; L.oz = o.z;
    L.ix = guard_inv(d.x); L.iy = guard_inv(d.y); L.iz = guard_inv(d.z);
    L.oix = o.x * L.ix; L.oiy = o.y * L.iy; L.oiz = o.z * L.iz;
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz + 1 == 3 ? 0 : kz + 1;
    int ky = kx + 1 == 3 ? 0 : kx + 1;
    const float dkz = comp(d, kz);
    if (dkz < 0.0f) { const int t = kx; kx = ky; ky = t; }
    L.kx = kx; L.ky = ky; L.kz = kz;
    L.Sx = comp(d, kx) / dkz;
    L.Sy = comp(d, ky) / dkz;
    L.Sz = 1.0f / dkz;
    L.dkz_abs = fabsf(dkz);
    return L;
}

// Does the line meet the box [lo, hi]?  No parameter range: a line.
__device__ __forceinline__ bool line_box(const LinePre& L, float lox, float hix, float loy,
                                         float hiy, float loz, float hiz)
{
    const float t0x = fmaf(lox, L.ix, -L.oix), t1x = fmaf(hix, L.ix, -L.oix);
    const float t0y = fmaf(loy, L.iy, -L.oiy), t1y = fmaf(hiy, L.iy, -L.oiy);
    const float t0z = fmaf(loz, L.iz, -L.oiz), t1z = fmaf(hiz, L.iz, -L.oiz);
    const float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fminf(t0z, t1z));
    const float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fmaxf(t0z, t1z));
    return tn <= tf;
}

// Result of one all-hits line query.
struct LineHits {
    int m;          // number of hits
    int pos;        // leaf-order index of the picked triangle (-1: none)
    int sum_s;      // sum over hits of sign(omega . n) (debug)
    int flag;       // near-degenerate
    uint64_t best;  // smallest key
};

struct TraverseCounters {
    uint32_t nodes, tris;
};

template <bool COUNT>
__device__ __forceinline__ LineHits trace_line(const float4* __restrict__ nodes,
                                               const float4* __restrict__ tv, int root,
                                               float3 o, float3 d, int exclude_pos,
                                               StreamKey key, uint32_t q, uint32_t walk,
                                               uint32_t step, float edge_thr_L, float tauL,
                                               float graze, bool want_sum_s,
                                               TraverseCounters& cnt, int& overflow,
                                               int iter_limit)
{
    const LinePre L = line_pre(o, d);
    // An edge closer than tau*L to the line has |U| < tau*L*max_edge/|d_kz|.
    const float Tthr = edge_thr_L / L.dkz_abs;
    LineHits h;
    h.m = 0; h.pos = -1; h.sum_s = 0; h.flag = 0; h.best = ~0ull;
    uint32_t best_prim = 0xFFFFFFFFu;
    int stack[kStackSize];
    int sp = 0;
    int ref = root;
    int iters = 0;  // a tree visits each node at most once: bounded loop
    while (true) {
        // interior nodes: descend until a leaf or nothing left
        while (ref >= 0) {
            if (++iters > iter_limit) {
                overflow |= 2;
                ref = kNoRef;
                sp = 0;
                break;
            }
            const float4 n0 = __ldg(nodes + 4 * ref + 0);
            const float4 n1 = __ldg(nodes + 4 * ref + 1);
            const float4 n2 = __ldg(nodes + 4 * ref + 2);
            const int4 n3 = __ldg(reinterpret_cast<const int4*>(nodes) + 4 * ref + 3);
            if (COUNT) cnt.nodes++;
            const bool h0 = line_box(L, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y);
            const bool h1 = line_box(L, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w);
            if (h0 && h1) {
                if (sp < kStackSize) {
                    stack[sp++] = n3.y;
                } else {
                    overflow |= 1;
                }
                ref = n3.x;
            } else if (h0) {
                ref = n3.x;
            } else if (h1) {
                ref = n3.y;
            } else {
                ref = sp > 0 ? stack[--sp] : kNoRef;
            }
        }
        if (ref == kNoRef) break;
        // leaf: test its triangles
        const int first = leaf_first(ref), count = leaf_count(ref);
        for (int p = first; p < first + count; ++p) {
            if (p == exclude_pos) continue;
            if (COUNT) cnt.tris++;
            const float4 a4 = __ldg(tv + 3 * p + 0);
            const float4 b4 = __ldg(tv + 3 * p + 1);
            const float4 c4 = __ldg(tv + 3 * p + 2);
            // vertices relative to the origin, then the shear that maps d to
            // the kz axis (Woop, Benthin, Wald, JCGT 2013)
            const float3 A = make_float3(a4.x - L.ox, a4.y - L.oy, a4.z - L.oz);
            const float3 B = make_float3(b4.x - L.ox, b4.y - L.oy, b4.z - L.oz);
            const float3 C = make_float3(c4.x - L.ox, c4.y - L.oy, c4.z - L.oz);
            const float Akz = comp(A, L.kz), Bkz = comp(B, L.kz), Ckz = comp(C, L.kz);
            const float Ax = fmaf(-L.Sx, Akz, comp(A, L.kx));
            const float Ay = fmaf(-L.Sy, Akz, comp(A, L.ky));
            const float Bx = fmaf(-L.Sx, Bkz, comp(B, L.kx));
            const float By = fmaf(-L.Sy, Bkz, comp(B, L.ky));
            const float Cx = fmaf(-L.Sx, Ckz, comp(C, L.kx));
            const float Cy = fmaf(-L.Sy, Ckz, comp(C, L.ky));
            const float U = Cx * By - Cy * Bx;
            const float V = Ax * Cy - Ay * Cx;
            const float W = Bx * Ay - By * Ax;
            const bool pos_side = (U > -Tthr) && (V > -Tthr) && (W > -Tthr);
            const bool neg_side = (U < Tthr) && (V < Tthr) && (W < Tthr);
            if (pos_side || neg_side) {
                const float det = U + V + W;
                const float mn = fminf(fminf(fabsf(U), fabsf(V)), fabsf(W));
                if (mn < Tthr || fabsf(det) * L.dkz_abs < graze * b4.w) h.flag = 1;
                const bool hit = (U > 0.f && V > 0.f && W > 0.f) || (U < 0.f && V < 0.f && W < 0.f);
                if (hit) {
                    const float T = fmaf(U, L.Sz * Akz, fmaf(V, L.Sz * Bkz, W * (L.Sz * Ckz)));
                    const float t = T / det;
                    if (fabsf(t) < tauL) h.flag = 1;
                    h.m++;
                    const uint32_t prim = __float_as_uint(a4.w);
                    const u32x4 k = stream_block(key, q, walk, step, kPurposeHit, 0u, prim);
                    const uint64_t kk = ((uint64_t)k.x << 32) | (uint64_t)k.y;
                    if (kk < h.best || (kk == h.best && prim < best_prim)) {
                        h.best = kk;
                        h.pos = p;
                        best_prim = prim;
                    }
                    if (want_sum_s) {
                        // s = sign(t) * sign(d . N)
                        const float e1x = b4.x - a4.x, e1y = b4.y - a4.y, e1z = b4.z - a4.z;
                        const float e2x = c4.x - a4.x, e2y = c4.y - a4.y, e2z = c4.z - a4.z;
                        const float nx = e1y * e2z - e1z * e2y;
                        const float ny = e1z * e2x - e1x * e2z;
                        const float nz = e1x * e2y - e1y * e2x;
                        const float dn = d.x * nx + d.y * ny + d.z * nz;
                        h.sum_s += ((t > 0.f) == (dn > 0.f)) ? 1 : -1;
                    }
                }
            }
        }
        ref = sp > 0 ? stack[--sp] : kNoRef;
        if (ref == kNoRef) break;
    }
    return h;
}

// FP64 refinement of the picked hit: intersection of the line x + t d with
// the triangle's plane, t = N.(v0 - x) / N.d, and s = sign(t) sign(d . N).
struct Refined {
    double3 y;
    int s;
};

__device__ __forceinline__ Refined refine_hit(const float4* __restrict__ tv, int pos, double3 x,
                                              double3 d)
{
    const float4 a4 = __ldg(tv + 3 * pos + 0);
    const float4 b4 = __ldg(tv + 3 * pos + 1);
    const float4 c4 = __ldg(tv + 3 * pos + 2);
    const double e1x = (double)b4.x - a4.x, e1y = (double)b4.y - a4.y, e1z = (double)b4.z - a4.z;
    const double e2x = (double)c4.x - a4.x, e2y = (double)c4.y - a4.y, e2z = (double)c4.z - a4.z;
    const double nx = e1y * e2z - e1z * e2y;
    const double ny = e1z * e2x - e1x * e2z;
    const double nz = e1x * e2y - e1y * e2x;
    const double dn = d.x * nx + d.y * ny + d.z * nz;
    const double num = nx * ((double)a4.x - x.x) + ny * ((double)a4.y - x.y) + nz * ((double)a4.z - x.z);
    const double t = num / dn;
    Refined r;
    r.y = make_double3(x.x + t * d.x, x.y + t * d.y, x.z + t * d.z);
    r.s = ((t > 0.0) == (dn > 0.0)) ? 1 : -1;
    return r;
}

}  // namespace wob
