// wob_device.cuh -- device-side building blocks shared by the library's
// kernels: the counter-based generator, line-axis sampling, the BVH node
// layout and the all-hits line traversal.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ff.cuh"
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

// 1 / sqrt(x), the approximate MUFU form (relative error below 2^-22), with
// subnormal inputs and results flushed to zero: for the squared distances it
// is used on (0, or far above the subnormal range) it is the same value as
// rsqrtf without the instructions that handle subnormal inputs.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
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
// product, so the axis is bit-reproducible.  The debug entry points
// (wob_line_axes, wob_trace_lines) use this form; the walk kernels use
// line_axis_ff below (the same axis to about 2^-44).
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

// The same axis in float-float: s = S 2^-48, 1 - s and 1 - 2 s are exact
// as float-float (48-bit integers), sqrt(1 - s) by one correction step.
__device__ __forceinline__ ff ff_of_int48(int64_t v)
{
    const float h = (float)v;
    return {h, (float)(v - (int64_t)h)};
}
__device__ __forceinline__ void line_axis_ff(StreamKey key, uint32_t q, uint32_t walk,
                                             uint32_t step, ff (&d)[3])
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
                const ff r = ff_of_int48((int64_t(1) << 48) - S);  // (1 - s) 2^48
                const float s0 = __fsqrt_rn(r.hi);                 // sqrt((1 - s)) 2^24
                const ff sq = two_prod(s0, s0);
                const float e = __fadd_rn(__fadd_rn(__fsub_rn(r.hi, sq.hi), -sq.lo), r.lo);
                ff root = s0 > 0.f ? fast_two_sum(s0, __fdiv_rn(e, __fmul_rn(2.f, s0))) : ff{0.f, 0.f};
                root.hi *= 0x1p-24f;
                root.lo *= 0x1p-24f;
                d[0] = ff_mul_f(root, (float)A * 0x1p-23f);
                d[1] = ff_mul_f(root, (float)B * 0x1p-23f);
                const ff z = ff_of_int48((int64_t(1) << 48) - 2 * S);
                d[2] = {z.hi * 0x1p-48f, z.lo * 0x1p-48f};
                return;
            }
        }
    }
    d[0] = {0.f, 0.f};
    d[1] = {0.f, 0.f};
    d[2] = {1.f, 0.f};
}

// ---------------------------------------------------------------------------
// BVH layout (built in bvh.cu): a binary LBVH collapsed into 8-wide nodes
// of 6 float4 (96 bytes), root = node 0:
//   f[0] = (origin x, y, z, bits: ex | ey << 8 | ez << 16 | nint << 24 | nchild << 28)
//   f[1..3] = per axis: quantised child lows (8 bytes) then highs (8 bytes);
//             child box = origin + q * 2^(e - 127), rounded outward
//   f[4..5] = refs[0..7]: refs[0] = first interior child when nint > 0
//             (interior children are slots 0 .. nint-1, stored at
//             refs[0] + slot); leaf slots hold ~(first << 3 | (count - 1)),
//             triangles tv[3 * first .. 3 * (first + count) - 1].
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
    float Sx, Sy, Sz;  // shear; |Sz| = 1 / |d_kz|
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

// ---------------------------------------------------------------------------
// All-hits traversal of one line.  Hits are recorded by leaf position; the
// selection keys are computed after the traversal (select_hit), and only when
// there is more than one hit.
// ---------------------------------------------------------------------------
constexpr int kMaxHits = 8;

struct Trav {
    int m;          // hits so far
    int flag;       // near-degenerate line
    int sum_s;      // sum of sign(omega . n) over hits (debug only)
    uint64_t best;  // smallest key among hits, once m > kMaxHits
    int bpos;       // its leaf position
};

__device__ __forceinline__ void trav_init(Trav& t)
{
    t.m = 0;
    t.flag = 0;
    t.sum_s = 0;
    t.best = ~0ull;
    t.bpos = -1;
}

__device__ __forceinline__ uint64_t hit_key(StreamKey key, uint32_t q, uint32_t walk,
                                            uint32_t step, uint32_t prim)
{
    const u32x4 k = stream_block(key, q, walk, step, kPurposeHit, 0u, prim);
    return ((uint64_t)k.x << 32) | (uint64_t)k.y;
}

__device__ __forceinline__ uint32_t prim_of(const float4* __restrict__ tv, int pos)
{
    return __float_as_uint(__ldg(tv + 3 * pos).w);
}

// Smallest key wins; equal keys: smaller triangle id.
__device__ __forceinline__ void keep_min(uint64_t k, uint32_t prim, int pos, uint64_t& best,
                                         uint32_t& best_prim, int& bpos)
{
    if (k < best || (k == best && prim < best_prim)) {
        best = k;
        best_prim = prim;
        bpos = pos;
    }
}

// Line-triangle test of the triangle (a4, b4, c4) in leaf layout, applied
// to a line (no parameter range): true on a hit (tl = its line parameter);
// flag = 1 on a near-degenerate configuration.
//
// The test works in the sheared frame of Woop, Benthin and Wald
// ("Watertight ray/triangle intersection", JCGT 2013), where the line is the
// kz axis and each directed edge P -> Q has the edge function
// f = cross2(Q', P') (twice the signed area of the origin and the projected
// edge).  A hit is f > 0 on all three edges or f < 0 on all three.
//
// Main path: the edge functions are formed from the sheared vertex A' and
// the sheared WORLD differences b - a and c - a (nearby vertices, so these
// differences are nearly exact): W = f(A->B) = cross2(eb', A'),
// V = f(C->A) = cross2(A', ec'), det = U + V + W = cross2(ec', eb') and
// U = det - V - W.  Their rounding error is of order 2^-24 |A'| |e'| -- a
// distance of order 2^-24 |A'| from the edge, not 2^-24 |A'|^2 / |e'| as
// when the edge functions are products of two sheared vertices.
//
// Near an edge (some |f| < Trare, a bound above both that rounding error and
// the flag distance) the three edge functions are recomputed by near_edges
// in a canonical form, so that two triangles sharing an edge obtain exactly
// opposite values for it (watertight), and the near-degenerate flag is
// decided from the true distances of the line to the edges.
// Sheared coordinates (kx, ky) of a point p relative to the line origin.
__device__ __forceinline__ float2 shear_rel(const float4& p, const LinePre& L)
{
    const float3 r = make_float3(p.x - L.ox, p.y - L.oy, p.z - L.oz);
    const float rz = comp(r, L.kz);
    return make_float2(fmaf(-L.Sx, rz, comp(r, L.kx)), fmaf(-L.Sy, rz, comp(r, L.ky)));
}

// Edge function of the directed edge P -> Q in the canonical form: the world
// difference e = Q - P sheared to e', then cross2(e', X') at the anchor X,
// the endpoint whose sheared (x, y) is lexicographically smaller.  Reversing
// the edge negates e' exactly and keeps the anchor, so the value is exactly
// negated: the two triangles of an edge agree on the side the line passes.
// len2 receives |d x e|^2 / d_kz^2, so that f^2 / len2 is the squared
// distance of the line to the edge's supporting line.
__device__ __forceinline__ float edge_fn(const float4& P, float2 Pp, const float4& Q, float2 Qp,
                                         const LinePre& L, float& len2)
{
    const float3 e = make_float3(Q.x - P.x, Q.y - P.y, Q.z - P.z);
    const float ez = comp(e, L.kz);
    const float ex = fmaf(-L.Sx, ez, comp(e, L.kx)), ey = fmaf(-L.Sy, ez, comp(e, L.ky));
    const bool anchor_p = Pp.x < Qp.x || (Pp.x == Qp.x && Pp.y < Qp.y);
    const float2 X = anchor_p ? Pp : Qp;
    const float c = fmaf(L.Sx, ey, -L.Sy * ex);
    len2 = fmaf(ex, ex, fmaf(ey, ey, c * c));
    return __fmaf_rn(ex, X.y, -__fmul_rn(ey, X.x));
}

// Canonical edge functions and the near-degenerate flag of a line that
// passes close to an edge of the triangle: (U, V, W, flag).  The flag
// follows the oracle's definition with the distance kFlagMargin tau L: the
// line lies within that distance of the triangle (the expanded projection
// contains it) and within it of an edge.  Not inlined: it runs on a small
// fraction of the triangle tests, and kept out of line it adds no register
// pressure to the traversal loop.
struct EdgeFns {
    float U, V, W;
    int flag;
};

static __device__ __noinline__ EdgeFns near_edges(float4 a4, float4 b4, float4 c4, LinePre L, float tauL)
{
    const float2 A = shear_rel(a4, L), B = shear_rel(b4, L), C = shear_rel(c4, L);
    float lu, lv, lw;
    EdgeFns r;
    r.W = edge_fn(a4, A, b4, B, L, lw);
    r.U = edge_fn(b4, B, c4, C, L, lu);
    r.V = edge_fn(c4, C, a4, A, L, lv);
    const float t = kFlagMargin * tauL;
    const float du = t * sqrtf(lu), dv = t * sqrtf(lv), dw = t * sqrtf(lw);
    const bool inside = (r.U > -du && r.V > -dv && r.W > -dw) || (r.U < du && r.V < dv && r.W < dw);
    r.flag = inside && (fabsf(r.U) < du || fabsf(r.V) < dv || fabsf(r.W) < dw);
    return r;
}

__device__ __forceinline__ bool line_tri(const float4& a4, const float4& b4, const float4& c4,
                                         const LinePre& L, float Trare, float tauL, float graze,
                                         int& flag, float& tl)
{
    const float3 A = make_float3(a4.x - L.ox, a4.y - L.oy, a4.z - L.oz);
    const float3 eb = make_float3(b4.x - a4.x, b4.y - a4.y, b4.z - a4.z);
    const float3 ec = make_float3(c4.x - a4.x, c4.y - a4.y, c4.z - a4.z);
    const float Akz = comp(A, L.kz), bkz = comp(eb, L.kz), ckz = comp(ec, L.kz);
    const float Ax = fmaf(-L.Sx, Akz, comp(A, L.kx));
    const float Ay = fmaf(-L.Sy, Akz, comp(A, L.ky));
    const float bx = fmaf(-L.Sx, bkz, comp(eb, L.kx));
    const float by = fmaf(-L.Sy, bkz, comp(eb, L.ky));
    const float cx = fmaf(-L.Sx, ckz, comp(ec, L.kx));
    const float cy = fmaf(-L.Sy, ckz, comp(ec, L.ky));
    float W = bx * Ay - by * Ax;  // edge A -> B
    float V = Ax * cy - Ay * cx;  // edge C -> A
    float det = cx * by - cy * bx;
    float U = det - V - W;        // edge B -> C
    const bool pos_side = (U > -Trare) && (V > -Trare) && (W > -Trare);
    const bool neg_side = (U < Trare) && (V < Trare) && (W < Trare);
    if (!(pos_side || neg_side)) return false;
    if (fminf(fminf(fabsf(U), fabsf(V)), fabsf(W)) < Trare) {
        const EdgeFns e = near_edges(a4, b4, c4, L, tauL);
        U = e.U;
        V = e.V;
        W = e.W;
        flag |= e.flag;
        det = U + V + W;
    }
    if (fabsf(det) < graze * b4.w * fabsf(L.Sz)) flag = 1;
    const bool hit = (U > 0.f && V > 0.f && W > 0.f) || (U < 0.f && V < 0.f && W < 0.f);
    if (!hit) return false;
    // kz of the hit relative to the origin: barycentric mix of A, B, C
    tl = L.Sz * (Akz + fmaf(V, bkz, W * ckz) / det);
    if (fabsf(tl) < kFlagMargin * tauL) flag = 1;
    return true;
}

// Test of leaf triangle p for the one-lane traversal: record a hit.
template <bool SUM_S>
__device__ __forceinline__ void test_tri(const float4* __restrict__ tv, const LinePre& L, float3 d,
                                         float Tthr, float tauL, float graze, int p, Trav& t,
                                         int* hits, StreamKey key, uint32_t q, uint32_t walk,
                                         uint32_t step)
{
    const float4 a4 = __ldg(tv + 3 * p + 0);
    const float4 b4 = __ldg(tv + 3 * p + 1);
    const float4 c4 = __ldg(tv + 3 * p + 2);
    float tl = 0.f;
    if (!line_tri(a4, b4, c4, L, Tthr, tauL, graze, t.flag, tl)) return;
    if (t.m < kMaxHits) {
        hits[t.m] = p;
    } else {
        // more hits than recorded: from here on keep a running minimum
        uint32_t bprim = t.bpos >= 0 ? prim_of(tv, t.bpos) : 0xFFFFFFFFu;
        if (t.m == kMaxHits)
            for (int i = 0; i < kMaxHits; ++i)
                keep_min(hit_key(key, q, walk, step, prim_of(tv, hits[i])), prim_of(tv, hits[i]),
                         hits[i], t.best, bprim, t.bpos);
        keep_min(hit_key(key, q, walk, step, __float_as_uint(a4.w)), __float_as_uint(a4.w), p,
                 t.best, bprim, t.bpos);
    }
    t.m++;
    if (SUM_S) {
        const float e1x = b4.x - a4.x, e1y = b4.y - a4.y, e1z = b4.z - a4.z;
        const float e2x = c4.x - a4.x, e2y = c4.y - a4.y, e2z = c4.z - a4.z;
        const float nx = e1y * e2z - e1z * e2y;
        const float ny = e1z * e2x - e1x * e2z;
        const float nz = e1x * e2y - e1y * e2x;
        const float dn = d.x * nx + d.y * ny + d.z * nz;
        t.sum_s += ((tl > 0.f) == (dn > 0.f)) ? 1 : -1;
    }
}

// ---------------------------------------------------------------------------
// 8-wide traversal (nodes collapsed from the binary tree; layout in bvh.cu).
// All hits are wanted, so the order of the children does not matter: a stack
// entry is a group (first interior child, mask of children still to visit),
// at most one per level.
// ---------------------------------------------------------------------------
// Byte q = b of w as the exact float 1 + q 2^-15 (one byte permute: q into
// the second mantissa byte under the exponent of 1.0).  A plane q of a node
// with quantisation step s lies at t = q s / d + b = (1 + q 2^-15) a + (b - a)
// with a = 2^15 s / d: one FMA per plane with a and b - a fixed per node.
// Rounding b - a costs up to s / 512 in position (1.53e-5 of the node's
// extent, below the boxes' padding of 2e-5 L), so the box test stays
// conservative.
__device__ __forceinline__ float dequant(uint32_t w, int b)
{
    return __uint_as_float(__byte_perm(w, 0x3F800000u, 0x7604u | ((uint32_t)b << 4)));
}

__device__ __forceinline__ int pick4(int4 v, int j)
{
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// Leaf triangles are not tested during the node visit that finds them: a
// lane queues them and keeps visiting nodes until every lane still
// traversing (the converged set) holds queued triangles or has run out of
// nodes, then the lanes test their queues together (Aila and Laine,
// "Understanding the efficiency of ray traversal on GPUs", HPG 2009:
// postponed leaves, speculative traversal).  A leaf that does not fit in
// the queue is tested on the spot.  The set of triangles tested is the
// same as with immediate tests.
// 15 entries: with the 8 KB of parked walk state a 128-thread block holds
// 15.5 KB of shared memory, so eight blocks (each with 1 KB reserved) fit
// the 132 KB shared-memory carveout and leave 124 KB of L1 per SM (16
// entries need the 164 KB carveout, 92 KB of L1, and run 3% slower).
constexpr int kLeafQ = 15;

// Where a lane keeps its queued leaf triangles: entry i at base[i * stride]
// (shared memory, structure of arrays, in the walk kernels; a local array
// elsewhere).
struct LeafQueue {
    int* base;
    int stride;
    __device__ __forceinline__ int& operator[](int i) const { return base[i * stride]; }
};

// HIT_MASK picks how the slots beyond a node's children are dropped: one
// mask per node (true) or a test per slot (false).  Both give the same hit
// set; which runs faster depends on the kernel's register allocation (on a
// GB300 the mask is 4% faster in the direct-BIE walk kernel, 3% in the
// batched one, 1% in the gradient walks and 1% slower in the plain
// double-layer walks).
template <bool COUNT, bool SUM_S, bool HIT_MASK = false>
__device__ __forceinline__ void trace_wide_q(const float4* __restrict__ wn,
                                             const float4* __restrict__ tv, const LinePre& L,
                                             float3 d, float Tthr, float tauL, float graze,
                                             int exclude_pos, Trav& t, int* hits, int* stack,
                                             StreamKey key, uint32_t q, uint32_t walk,
                                             uint32_t step, uint32_t& n_nodes, uint32_t& n_tris,
                                             int& err, int iter_limit, LeafQueue lq)
{
    int node = 0, sp = 0, iters = 0, nq = 0;
    bool done = false;
    while (true) {
        // nodes, until every converged lane holds queued triangles (or is done)
        while (true) {
            if (node < 0) {
                if (sp == 0) {
                    done = true;
                    break;
                }
                const uint32_t e = (uint32_t)stack[--sp];
                const int base = (int)(e & 0xFFFFFFu);
                uint32_t m = e >> 24;
                const int c = __ffs(m) - 1;
                m &= m - 1;
                if (m) stack[sp++] = base | (int)(m << 24);
                node = base + c;
            }
            if (++iters > iter_limit) {  // each node is visited at most once per line
                err |= 2;
                done = true;
                break;
            }
            if (COUNT) n_nodes++;
            const float4* nd = wn + 6 * node;
            const float4 h = __ldg(nd);
            const uint32_t hdr = __float_as_uint(h.w);
            const int nint = (hdr >> 24) & 15, nch = hdr >> 28;
            // slab parameter of a quantised plane: (origin + q s - o) / d
            // = (1 + q 2^-15) a + b with a = 2^15 s / d (see dequant)
            const float ax = __uint_as_float(((hdr & 255u) + 15u) << 23) * L.ix;
            const float ay = __uint_as_float((((hdr >> 8) & 255u) + 15u) << 23) * L.iy;
            const float az = __uint_as_float((((hdr >> 16) & 255u) + 15u) << 23) * L.iz;
            const float bx = fmaf(h.x, L.ix, -L.oix) - ax, by = fmaf(h.y, L.iy, -L.oiy) - ay,
                        bz = fmaf(h.z, L.iz, -L.oiz) - az;
            const uint4 qx = __ldg(reinterpret_cast<const uint4*>(nd + 1));
            const uint4 qy = __ldg(reinterpret_cast<const uint4*>(nd + 2));
            const uint4 qz = __ldg(reinterpret_cast<const uint4*>(nd + 3));
            // per axis the near plane is the low one when the axis component
            // is positive (t = q a + b is monotone in q): pick near / far
            // byte words once, so a slab test is max of 3 nears <= min of 3 fars
            const bool px_ = L.ix >= 0.f, py_ = L.iy >= 0.f, pz_ = L.iz >= 0.f;
            const uint32_t nx0 = px_ ? qx.x : qx.z, nx1 = px_ ? qx.y : qx.w;
            const uint32_t fx0 = px_ ? qx.z : qx.x, fx1 = px_ ? qx.w : qx.y;
            const uint32_t ny0 = py_ ? qy.x : qy.z, ny1 = py_ ? qy.y : qy.w;
            const uint32_t fy0 = py_ ? qy.z : qy.x, fy1 = py_ ? qy.w : qy.y;
            const uint32_t nz0 = pz_ ? qz.x : qz.z, nz1 = pz_ ? qz.y : qz.w;
            const uint32_t fz0 = pz_ ? qz.z : qz.x, fz1 = pz_ ? qz.w : qz.y;
            uint32_t hit = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float tnx = fmaf(dequant(j < 4 ? nx0 : nx1, j & 3), ax, bx);
                const float tfx = fmaf(dequant(j < 4 ? fx0 : fx1, j & 3), ax, bx);
                const float tny = fmaf(dequant(j < 4 ? ny0 : ny1, j & 3), ay, by);
                const float tfy = fmaf(dequant(j < 4 ? fy0 : fy1, j & 3), ay, by);
                const float tnz = fmaf(dequant(j < 4 ? nz0 : nz1, j & 3), az, bz);
                const float tfz = fmaf(dequant(j < 4 ? fz0 : fz1, j & 3), az, bz);
                const float tn = fmaxf(fmaxf(tnx, tny), tnz);
                const float tf = fminf(fminf(tfx, tfy), tfz);
                if (HIT_MASK) hit |= (tn <= tf ? 1u : 0u) << j;
                else if (j < nch && tn <= tf) hit |= 1u << j;
            }
            if (HIT_MASK) hit &= (1u << nch) - 1u;
            const int4 r0 = __ldg(reinterpret_cast<const int4*>(nd + 4));
            uint32_t lm = hit >> nint;  // leaf children: queue their triangles
            if (lm) {
                const int4 r1 = __ldg(reinterpret_cast<const int4*>(nd + 5));
                while (lm) {
                    const int j = nint + __ffs(lm) - 1;
                    lm &= lm - 1;
                    const int ref = j < 4 ? pick4(r0, j) : pick4(r1, j - 4);
                    const int first = leaf_first(ref), count = leaf_count(ref);
                    for (int p = first; p < first + count; ++p) {
                        if (p == exclude_pos) continue;
                        if (nq < kLeafQ) {
                            lq[nq++] = p;
                        } else {
                            if (COUNT) n_tris++;
                            test_tri<SUM_S>(tv, L, d, Tthr, tauL, graze, p, t, hits, key, q,
                                            walk, step);
                        }
                    }
                }
            }
            uint32_t im = hit & ((1u << nint) - 1u);  // interior children
            if (im) {
                const int c = __ffs(im) - 1;
                im &= im - 1;
                if (im) {
                    if (sp < kStackSize) stack[sp++] = r0.x | (int)(im << 24);
                    else err |= 1;
                }
                node = r0.x + c;
            } else {
                node = -1;
            }
            if (__all_sync(__activemask(), nq > 0)) break;
        }
        // the queued triangles, all lanes together
        for (int i = 0; i < nq; ++i) {
            if (COUNT) n_tris++;
            test_tri<SUM_S>(tv, L, d, Tthr, tauL, graze, lq[i], t, hits, key, q, walk, step);
        }
        nq = 0;
        if (done) break;
    }
}

template <bool COUNT, bool SUM_S>
__device__ __forceinline__ void trace_wide(const float4* __restrict__ wn,
                                           const float4* __restrict__ tv, const LinePre& L,
                                           float3 d, float Tthr, float tauL, float graze,
                                           int exclude_pos, Trav& t, int* hits, int* stack,
                                           StreamKey key, uint32_t q, uint32_t walk,
                                           uint32_t step, uint32_t& n_nodes, uint32_t& n_tris,
                                           int& err, int iter_limit)
{
    int lq[kLeafQ];
    trace_wide_q<COUNT, SUM_S>(wn, tv, L, d, Tthr, tauL, graze, exclude_pos, t, hits, stack, key,
                               q, walk, step, n_nodes, n_tris, err, iter_limit, LeafQueue{lq, 1});
}

// The picked hit (leaf position) after the traversal; -1 if m == 0.
__device__ __forceinline__ int select_hit(const float4* __restrict__ tv, const Trav& t,
                                          const int* hits, StreamKey key, uint32_t q,
                                          uint32_t walk, uint32_t step)
{
    if (t.m == 0) return -1;
    if (t.m == 1) return hits[0];
    if (t.m > kMaxHits) return t.bpos;
    uint64_t best = ~0ull;
    uint32_t bprim = 0xFFFFFFFFu;
    int bpos = -1;
    for (int i = 0; i < t.m; ++i) {
        const uint32_t prim = prim_of(tv, hits[i]);
        keep_min(hit_key(key, q, walk, step, prim), prim, hits[i], best, bprim, bpos);
    }
    return bpos;
}

// Whole traversal of one line (debug entry point).
template <bool SUM_S>
__device__ __forceinline__ int trace_line(const float4* __restrict__ nodes,
                                          const float4* __restrict__ tv, float3 o,
                                          float3 d, int exclude_pos, StreamKey key, uint32_t q,
                                          uint32_t walk, uint32_t step, float edge_thr_L,
                                          float tauL, float graze, Trav& t, int& err,
                                          int iter_limit)
{
    const LinePre L = line_pre(o, d);
    const float Tthr = edge_thr_L * fabsf(L.Sz);
    int stack[kStackSize];
    int hits[kMaxHits];
    uint32_t nn = 0, nt = 0;
    trav_init(t);
    trace_wide<false, SUM_S>(nodes, tv, L, d, Tthr, tauL, graze, exclude_pos, t, hits, stack, key,
                             q, walk, step, nn, nt, err, iter_limit);
    return select_hit(tv, t, hits, key, q, walk, step);
}

// FP64 refinement of the picked hit (the line-query debug entry point):
// intersection of the line x + t d with the triangle's plane,
// t = N.(v0 - x) / N.d, and s = sign(t) sign(d . N).
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

// The same refinement in float-float (the walk kernels): the edges b - a,
// c - a are exact (two-sum of FP32 vertices), the normal N, N.d and
// N.(a - x) are float-float products and sums, t = N.(a - x) / N.d takes one
// correction step, y = x + t d; relative error about 2^-44, so the hit
// point agrees with the FP64 refinement far below the walk tolerance.  x and
// d are float-float, the hit y is returned as float-float and the sign
// s = sign(t) sign(d . N) as the result.
__device__ __forceinline__ int refine_hit_ff(const float4* __restrict__ tv, int pos,
                                             const ff (&x)[3], const ff (&d)[3], ff (&y)[3])
{
    const float4 a4 = __ldg(tv + 3 * pos + 0);
    const float4 b4 = __ldg(tv + 3 * pos + 1);
    const float4 c4 = __ldg(tv + 3 * pos + 2);
    const ff e1[3] = {two_sum(b4.x, -a4.x), two_sum(b4.y, -a4.y), two_sum(b4.z, -a4.z)};
    const ff e2[3] = {two_sum(c4.x, -a4.x), two_sum(c4.y, -a4.y), two_sum(c4.z, -a4.z)};
    const ff n[3] = {ff_sub(ff_mul(e1[1], e2[2]), ff_mul(e1[2], e2[1])),
                     ff_sub(ff_mul(e1[2], e2[0]), ff_mul(e1[0], e2[2])),
                     ff_sub(ff_mul(e1[0], e2[1]), ff_mul(e1[1], e2[0]))};
    const ff w[3] = {ff_sub({a4.x, 0.f}, x[0]), ff_sub({a4.y, 0.f}, x[1]), ff_sub({a4.z, 0.f}, x[2])};
    ff dn = ff_mul(d[0], n[0]), num = ff_mul(n[0], w[0]);
    dn = ff_add(dn, ff_mul(d[1], n[1]));
    dn = ff_add(dn, ff_mul(d[2], n[2]));
    num = ff_add(num, ff_mul(n[1], w[1]));
    num = ff_add(num, ff_mul(n[2], w[2]));
    const float q1 = __fdiv_rn(num.hi, dn.hi);
    const ff r = ff_sub(num, ff_mul_f(dn, q1));
    const ff t = fast_two_sum(q1, __fdiv_rn(r.hi, dn.hi));
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = ff_add(x[c], ff_mul(t, d[c]));
    return ((t.hi > 0.f) == (dn.hi > 0.f)) ? 1 : -1;
}

// A double that holds a float-float value exactly (hi + lo, |lo| <= ulp(hi)
// / 2) and back.
__device__ __forceinline__ ff ff_split(double v)
{
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double ff_join(ff v) { return (double)v.hi + (double)v.lo; }

// Dirichlet data g at a boundary point y of the triangle in leaf order `pos`.
__device__ __forceinline__ float dl_data_f(const DataDev& D, const float4* __restrict__ tv, int pos,
                                           float3 y)
{
    if (D.mode == WOB_DATA_POLY) {
        const float* c = D.poly;
        return c[0] + c[1] * y.x + c[2] * y.y + c[3] * y.z + c[4] * y.x * y.x +
               c[5] * y.y * y.y + c[6] * y.z * y.z + c[7] * y.x * y.y + c[8] * y.y * y.z +
               c[9] * y.z * y.x;
    }
    if (D.mode == WOB_DATA_POINT) {
        const float dx = y.x - D.x0[0], dy = y.y - D.x0[1], dz = y.z - D.x0[2];
        return D.scale / sqrtf(dx * dx + dy * dy + dz * dz);
    }
    // linear interpolation of vertex values over the triangle
    const float4 a = __ldg(tv + 3 * pos), b = __ldg(tv + 3 * pos + 1), c = __ldg(tv + 3 * pos + 2);
    const float e1x = b.x - a.x, e1y = b.y - a.y, e1z = b.z - a.z;
    const float e2x = c.x - a.x, e2y = c.y - a.y, e2z = c.z - a.z;
    const float px = y.x - a.x, py = y.y - a.y, pz = y.z - a.z;
    const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    const float nn = nx * nx + ny * ny + nz * nz;
    const float b1 = ((py * e2z - pz * e2y) * nx + (pz * e2x - px * e2z) * ny +
                      (px * e2y - py * e2x) * nz) / nn;
    const float b2 = ((e1y * pz - e1z * py) * nx + (e1z * px - e1x * pz) * ny +
                      (e1x * py - e1y * px) * nz) / nn;
    const int prim = __float_as_int(a.w);
    const int32_t* t = D.tris + 3 * (int64_t)prim;
    return (1.f - b1 - b2) * __ldg(D.vdata + t[0]) + b1 * __ldg(D.vdata + t[1]) +
           b2 * __ldg(D.vdata + t[2]);
}

__device__ __forceinline__ float dl_data(const DataDev& D, const float4* __restrict__ tv, int pos,
                                         double3 yd)
{
    return dl_data_f(D, tv, pos, make_float3((float)yd.x, (float)yd.y, (float)yd.z));
}

// Geometry a double-layer walk needs.
struct DLGeom {
    const float4* nodes;  // 8-wide nodes, root = node 0
    const float4* tv;
    int iter_limit;
    float edge_thr_L;
    float tauL;
    float graze;
};

struct WalkCount {
    unsigned long long lines, nodes, tris, hits, flag;
};

// Where a walk keeps its state (point and axis as float-float pairs, S and
// P in FP64) while its lines are traversed: eight 8-byte slots per thread in
// shared memory, structure of arrays
// (field j of thread t at base[j * stride + t]) so that a warp's accesses
// are conflict-free.  The state is touched once per line; keeping it out of
// registers leaves the traversal loop its 64 registers.
// A float-float value in one double-sized slot (the two floats' bits, no
// arithmetic).
__device__ __forceinline__ double pack_ff(ff v)
{
    return __hiloint2double(__float_as_int(v.hi), __float_as_int(v.lo));
}
__device__ __forceinline__ ff unpack_ff(double v)
{
    return {__int_as_float(__double2hiint(v)), __int_as_float(__double2loint(v))};
}

struct WalkSlot {
    volatile double* base;  // &smem[threadIdx.x]
    int stride;             // threads per block
    __device__ __forceinline__ double get(int j) const { return base[j * stride]; }
    __device__ __forceinline__ void set(int j, double v) const { base[j * stride] = v; }
};

// Gradient weight of the first step (Sec. 4.1.3): the first line's weight
// -dG/dn_y / p = (m/2) s becomes -grad_x dG/dn_y / p, with
// grad_x dG/dn_y(x, y) = (n - 3 (w . n) w) / (4 pi r^3), w = (y - x) / r
// (App. A): (m/2) s times -(n - 3 (w . n) w) / (r (w . n)), the factor
// returned here (FP64, normal from the leaf triangle's vertices).
__device__ __forceinline__ double3 grad_factor(const float4* __restrict__ tv, int pos, double3 x,
                                               double3 y)
{
    const float4 a4 = __ldg(tv + 3 * pos + 0);
    const float4 b4 = __ldg(tv + 3 * pos + 1);
    const float4 c4 = __ldg(tv + 3 * pos + 2);
    const double e1x = (double)b4.x - a4.x, e1y = (double)b4.y - a4.y, e1z = (double)b4.z - a4.z;
    const double e2x = (double)c4.x - a4.x, e2y = (double)c4.y - a4.y, e2z = (double)c4.z - a4.z;
    double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    const double nl = sqrt(nx * nx + ny * ny + nz * nz);
    nx /= nl;
    ny /= nl;
    nz /= nl;
    double wx = y.x - x.x, wy = y.y - x.y, wz = y.z - x.z;
    const double r = sqrt(wx * wx + wy * wy + wz * wz);
    wx /= r;
    wy /= r;
    wz /= r;
    const double wn = wx * nx + wy * ny + wz * nz;
    const double k = -1.0 / (r * wn);
    return make_double3(k * (nx - 3.0 * wn * wx), k * (ny - 3.0 * wn * wy),
                        k * (nz - 3.0 * wn * wz));
}

// Per-line debug outputs of one walk (each pointer may be NULL): hit count
// (-1: line not traced), picked triangle (original id, -1: none) and the
// near-degenerate flag of every line k = 0 .. M-1.
struct LineOut {
    int32_t* m;
    int32_t* prim;
    uint8_t* flag;
    __device__ __forceinline__ void put(int k, int mk, int pk, int fk) const
    {
        if (m) m[k] = mk;
        if (prim) prim[k] = pk;
        if (flag) flag[k] = (uint8_t)fk;
    }
};

// One double-layer walk from x (Sec. 4.1.1-4.1.2, ray sampling of Sec.
// 4.4.1): per line, draw the axis, traverse (descend to a leaf, test it,
// repeat), pick the hit (keys only when m > 1), refine it in float-float
// and accumulate (weight product and sum in FP64).  Returns the walk value;
// `lo` (DEBUG only) receives the per-line outputs.  start_pos >= 0: x0 lies
// on that triangle (leaf position) and the walk estimates the density nu(x0)
// (Eq. indirect_double_boundary_reordered2): x0 is vertex 1 with weight 1
// and lines 1 .. M-1 follow.  HIT_MASK: the node-test form of trace_wide_q.
template <bool COUNT, bool DEBUG, bool GRAD = false, bool HIT_MASK = true>
__device__ __forceinline__ double dl_walk(const DLGeom& G, const DataDev& D, double phi, int M,
                                          StreamKey key, uint32_t q, uint32_t w, double3 x0,
                                          int start_pos, const WalkSlot& ws, int* stack,
                                          int* hits, int& err, int& wflag, const LineOut& lo,
                                          WalkCount& c, LeafQueue lq)
{
    enum { X0 = 0, X1, X2, D0, D1, D2, SS, PP, GX, GY, GZ };  // GX..GZ: GRAD only
    if (GRAD) {
        ws.set(GX, 0.0);
        ws.set(GY, 0.0);
        ws.set(GZ, 0.0);
    }
    ws.set(X0, pack_ff({(float)x0.x, 0.f}));
    ws.set(X1, pack_ff({(float)x0.y, 0.f}));
    ws.set(X2, pack_ff({(float)x0.z, 0.f}));
    ws.set(SS, 0.0);
    ws.set(PP, 1.0);
    int self = -1, k = 0;
    if (start_pos >= 0) {
        const double g = (double)dl_data(D, G.tv, start_pos, x0);
        ws.set(SS, ((M == 1) ? phi : 2.0 * phi) * g);
        self = start_pos;
        k = 1;
        if (DEBUG) lo.put(0, -1, -1, 0);
    }
    for (; k < M; ++k) {
        LinePre L;
        {
            ff d[3];
            line_axis_ff(key, q, w, (uint32_t)k, d);
            ws.set(D0, pack_ff(d[0]));
            ws.set(D1, pack_ff(d[1]));
            ws.set(D2, pack_ff(d[2]));
            L = line_pre(make_float3(unpack_ff(ws.get(X0)).hi, unpack_ff(ws.get(X1)).hi,
                                     unpack_ff(ws.get(X2)).hi),
                         make_float3(d[0].hi, d[1].hi, d[2].hi));
        }
        const float Tthr = G.edge_thr_L * fabsf(L.Sz);
        Trav t;
        trav_init(t);
        uint32_t nn = 0, nt = 0;
        trace_wide_q<COUNT, false, HIT_MASK>(G.nodes, G.tv, L, make_float3(0.f, 0.f, 0.f), Tthr,
                                             G.tauL, G.graze, self, t, hits, stack, key, q, w, (uint32_t)k, nn, nt,
                                   err, G.iter_limit, lq);
        if (COUNT) {
            c.lines++;
            c.nodes += nn;
            c.tris += nt;
            c.hits += t.m;
            c.flag += t.flag;
        }
        wflag |= t.flag;
        if (t.m == 0) {
            if (DEBUG) lo.put(k, 0, -1, t.flag);
            ++k;
            break;
        }
        const int pos = select_hit(G.tv, t, hits, key, q, w, (uint32_t)k);
        if (DEBUG) lo.put(k, t.m, (int)prim_of(G.tv, pos), t.flag);
        const ff x[3] = {unpack_ff(ws.get(X0)), unpack_ff(ws.get(X1)), unpack_ff(ws.get(X2))};
        const ff d[3] = {unpack_ff(ws.get(D0)), unpack_ff(ws.get(D1)), unpack_ff(ws.get(D2))};
        double S = ws.get(SS), P = ws.get(PP);
        ff y[3];
        const int sgn = refine_hit_ff(G.tv, pos, x, d, y);
        const double ms = (double)(t.m * sgn);
        P = (k == 0) ? 0.5 * ms : P * (-phi * ms);
        const double g = (double)dl_data_f(D, G.tv, pos, make_float3(y[0].hi, y[1].hi, y[2].hi));
        const double cc = (k == M - 1) ? phi : 2.0 * phi;
        S = fma(P * cc, g, S);
        if (GRAD && k == 0 && start_pos < 0) {
            const double3 gf = grad_factor(G.tv, pos, make_double3((double)x[0].hi + x[0].lo, (double)x[1].hi + x[1].lo, (double)x[2].hi + x[2].lo),
                                           make_double3((double)y[0].hi + y[0].lo, (double)y[1].hi + y[1].lo, (double)y[2].hi + y[2].lo));
            ws.set(GX, gf.x);
            ws.set(GY, gf.y);
            ws.set(GZ, gf.z);
        }
        ws.set(X0, pack_ff(y[0]));
        ws.set(X1, pack_ff(y[1]));
        ws.set(X2, pack_ff(y[2]));
        ws.set(SS, S);
        ws.set(PP, P);
        self = pos;
    }
    if (DEBUG)
        for (int k2 = k; k2 < M; ++k2) lo.put(k2, -1, -1, 0);
    return ws.get(SS);
}

// Per-query partial sums of the walk values.  Slot (query qi, block b of 32
// walks of the call) holds (sum, sum of squares) at part[2 s], part[2 s + 1],
// s = qi * tpq + b.  The 32 lanes of a warp hold 32 consecutive walks of the
// call (walk index qi * N + w, the group aligned to 32); the lanes of one
// slot sum their values in a fixed tree order (segmented scan) and the
// slot's last lane adds the result with an atomic.  A slot's walks span at
// most two aligned groups of 32, so it receives at most two adds onto zero,
// and two adds commute exactly: the sums do not depend on scheduling.  All
// 32 lanes call this together (live = false for lanes without a walk).
__device__ __forceinline__ void add_tile_partials(double v, bool live, int64_t qi, int64_t w,
                                                  int tpq, double* __restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const long long slot = live ? qi * tpq + (w >> 5) : -1ll;
    double s = live ? v : 0.0, ss = live ? v * v : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double s2 = __shfl_up_sync(0xFFFFFFFFu, s, o);
        const double ss2 = __shfl_up_sync(0xFFFFFFFFu, ss, o);
        const long long sl2 = __shfl_up_sync(0xFFFFFFFFu, slot, o);
        if (lane >= o && sl2 == slot) {
            s += s2;
            ss += ss2;
        }
    }
    const long long next = __shfl_down_sync(0xFFFFFFFFu, slot, 1);
    if (live && (lane == 31 || next != slot)) {
        atomicAdd(part + 2 * slot, s);
        atomicAdd(part + 2 * slot + 1, ss);
    }
}

}  // namespace wob
