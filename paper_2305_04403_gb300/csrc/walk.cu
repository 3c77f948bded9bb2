// walk.cu -- the walk-on-boundary kernels:
//   k_dl_walks   Dirichlet problems, double-layer formulation, ray (line)
//                sampling with all-hits queries (Sec. 4.1, 4.4.1)
//   k_sl_walks_ff / k_sl_walks
//                Neumann / Robin problems, single-layer formulation, area
//                sampling / resampled importance sampling (Sec. 4.3)
//   k_nd_walks   Neumann problems through the direct boundary integral
//                equation (Sec. 4.2)
//   k_reduce*    per-query FP64 mean and variance (Sec. 4.1.1)
// plus the debug kernels behind wob_trace_lines / wob_line_axes /
// wob_philox4x32_10.
//
// One thread owns one walk from start to end; the walk values of a warp's 32
// walks are summed per query in a fixed order into (sum, sum of squares)
// partials (add_tile_partials), which k_reduce_part combines per query in a
// fixed order, so results do not depend on scheduling.  Debug solves also
// write every walk's value.
#include <cmath>
#include <cstddef>
#include <cstdlib>

#include "bits.cuh"
#include "ff.cuh"
#include "wob_device.cuh"
#include "wob_host.h"

namespace wob {

namespace {

constexpr double kFourPi = 12.566370614359172953850573533118;

#ifndef WOB_DL_MIN_BLOCKS
#define WOB_DL_MIN_BLOCKS 8
#endif
// Single-layer walks with area sampling: 6 blocks of 128 threads per SM (71
// registers, no spills) hide the latency of the CDF search better than the
// unbounded 121 registers (4 blocks; 8% slower) or 8 blocks (64 registers,
// spills; 3% slower).
#ifndef WOB_SL_MIN_BLOCKS
#define WOB_SL_MIN_BLOCKS 6
#endif

// One thread owns one walk; warps take tiles of 32 consecutive walks from a
// global counter until none are left (dynamic balance; consecutive walks of
// a query start their first lines at the same point).  Per line:
// draw the axis, traverse (descend to a leaf, test it, repeat), then pick
// the hit (keys only when m > 1), refine it in float-float and add the
// data term (evaluated in FP32) to the FP64 walk sum.  The kernel is
// limited to 64 registers (8 blocks of 128 threads per SM): the traversal
// is latency-bound and occupancy pays more than the few values the
// compiler keeps in local memory.  Lanes that start their lines
// together share the fetches of the upper tree levels; variants that broke
// this (persistent lanes refilled from a global counter, or a wavefront of
// separate traversal and FP64-update kernels) measured 8-18% slower.
template <bool COUNT, bool DEBUG, bool GRAD = false>
__global__ void __launch_bounds__(128, WOB_DL_MIN_BLOCKS) k_dl_walks(WalkParams p)
{
    const StreamKey key{p.key0, p.key1};
    const int64_t total = p.Q * (int64_t)p.N;
    const DLGeom G{p.nodes, p.tv, p.iter_limit, p.edge_thr_L, p.tauL, p.graze};
    __shared__ double slots[(GRAD ? 11 : 8) * 128];
    __shared__ int leafq[kLeafQ * 128];
    const WalkSlot ws{slots + threadIdx.x, 128};
    const LeafQueue lq{leafq + threadIdx.x, 128};
    int err = 0;
    int stack[kStackSize];
    int hits[kMaxHits];
    WalkCount c{0, 0, 0, 0, 0};
    const int lane = threadIdx.x & 31;
    while (true) {
        // a warp takes the next 32 consecutive walks (one atomic per warp)
        unsigned long long tile = 0;
        if (lane == 0) tile = atomicAdd(p.tile_counter, 1ull);
        tile = __shfl_sync(0xFFFFFFFFu, tile, 0);
        if ((int64_t)tile * 32 >= total) break;
        const int64_t idx = (int64_t)tile * 32 + lane;
        const bool live = idx < total;
        const int64_t qi = live ? idx / p.N : 0;
        const int64_t wi = idx - qi * p.N;
        double v = 0.0;
        if (live) {
            const uint32_t q = p.q_base + (uint32_t)qi;
            const uint32_t w = (uint32_t)(p.walk_begin + wi);
            const double3 x =
                make_double3(p.queries[3 * qi], p.queries[3 * qi + 1], p.queries[3 * qi + 2]);
            int wflag = 0;
            int start = -1;
            if (p.query_prim) {  // density walks from boundary points
                const int32_t prim = p.query_prim[qi];
                start = (prim >= 0 && prim < p.T) ? p.inv_order[prim] : -1;
            }
            const int64_t lk = idx * p.M;
            const LineOut lo{DEBUG && p.line_m ? p.line_m + lk : nullptr,
                             DEBUG && p.line_prim ? p.line_prim + lk : nullptr,
                             DEBUG && p.line_flag ? p.line_flag + lk : nullptr};
            v = dl_walk<COUNT, DEBUG, GRAD, GRAD>(G, p.data, (double)p.phi, p.M, key, q, w, x,
                                                  start, ws, stack, hits, err, wflag, lo, c, lq);
            if (p.per_walk) p.per_walk[idx] = v;
            if (GRAD) {  // gradient of the same walk: first-step factor x walk value
                p.per_walk_grad[idx] = ws.get(8) * v;
                p.per_walk_grad[total + idx] = ws.get(9) * v;
                p.per_walk_grad[2 * total + idx] = ws.get(10) * v;
            }
            if (DEBUG && p.walk_flag) p.walk_flag[idx] = (uint8_t)wflag;
        }
        if (p.part) add_tile_partials(v, live, qi, wi, p.tpq, p.part);
    }
    if (err) atomicOr(p.error_word, err);
    if (COUNT) {
        atomicAdd(p.counters + 0, c.lines);
        atomicAdd(p.counters + 1, c.nodes);
        atomicAdd(p.counters + 2, c.tris);
        atomicAdd(p.counters + 3, c.hits);
        atomicAdd(p.counters + 4, c.flag);
    }
}

// Data of the single-layer problems at y on triangle j (original order):
// with condition bc (wob_bc) the field h (Dirichlet), its normal derivative
// dh/dn (Neumann) or dh/dn + alpha h (Robin); P1 mode: the vertex values.
__device__ __forceinline__ double sl_data(const WalkParams& p, int64_t j, double3 y, double b0,
                                          double b1, double b2, double3 n, int bc)
{
    const DataDev& D = p.data;
    if (D.mode == WOB_DATA_VERTEX_P1) {
        const int32_t* t = D.tris + 3 * j;
        return b0 * __ldg(D.vdata + t[0]) + b1 * __ldg(D.vdata + t[1]) + b2 * __ldg(D.vdata + t[2]);
    }
    double h, gx, gy, gz;
    if (D.mode == WOB_DATA_POLY) {
        const float* c = D.poly;
        h = c[0] + c[1] * y.x + c[2] * y.y + c[3] * y.z + c[4] * y.x * y.x + c[5] * y.y * y.y +
            c[6] * y.z * y.z + c[7] * y.x * y.y + c[8] * y.y * y.z + c[9] * y.z * y.x;
        gx = c[1] + 2.0 * c[4] * y.x + c[7] * y.y + c[9] * y.z;
        gy = c[2] + 2.0 * c[5] * y.y + c[7] * y.x + c[8] * y.z;
        gz = c[3] + 2.0 * c[6] * y.z + c[8] * y.y + c[9] * y.x;
    } else {
        const double rx = y.x - D.x0[0], ry = y.y - D.x0[1], rz = y.z - D.x0[2];
        const double rl = sqrt(rx * rx + ry * ry + rz * rz);
        h = D.scale / rl;
        const double f = -D.scale / (rl * rl * rl);
        gx = f * rx;
        gy = f * ry;
        gz = f * rz;
    }
    if (bc == WOB_BC_DIRICHLET) return h;
    const double dhdn = n.x * gx + n.y * gy + n.z * gz;
    return bc == WOB_BC_ROBIN ? dhdn + (double)p.alpha * h : dhdn;
}

// Index of the triangle whose area-CDF interval holds the 53-bit uniform
// U = (hi, lo) times the total area: the first j with cdf[j] > fl(U 2^-53
// |Gamma|), else T - 1 (inverse CDF).  The guide table brackets the answer
// by the top bits of U (about one triangle per bucket), and a binary search
// inside the bracket makes the same comparisons as one over the whole CDF.
// Non-negative doubles order as their bit patterns: the search compares
// 64-bit integers (the same decisions as double compares, off the FP64
// pipe, which issues at 1/64 of the FP32 rate on this GPU).  The target is
// one FP64 multiply, (U 2^-53) |Gamma|; U 2^-53 is exact and formed from its
// bit pattern in the integer pipes (u53_unit).
__device__ __forceinline__ int64_t area_pick(const WalkParams& p, uint32_t hi, uint32_t lo)
{
    const uint64_t U = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
    const long long target = __double_as_longlong(u53_unit(U) * p.area);
    const uint32_t b = hi >> (32 - p.guide_bits);  // top guide_bits bits of U
    int64_t a = __ldg(p.guide + b);
    int64_t e = __ldg(p.guide + b + 1);
    e = e < p.T - 1 ? e : p.T - 1;
    while (a < e) {
        const int64_t mid = a + ((e - a) >> 1);
        if (__double_as_longlong(__ldg(p.cdf + mid)) > target) e = mid; else a = mid + 1;
    }
    return a;
}

// Area-uniform boundary point of stream (q, w, step, attempt): triangle j (original
// order) by inverse CDF of the areas (area_pick), then a uniform point on it
// (square-root warp), barycentrics b0..b2; n = the triangle's unit normal.
struct AreaPoint {
    int64_t j;
    double3 y, n;
    double b0, b1, b2;
};

__device__ __forceinline__ AreaPoint area_point(const WalkParams& p, StreamKey key, uint32_t q,
                                                uint32_t w, uint32_t step, uint32_t attempt = 0u)
{
    AreaPoint a;
    const u32x4 u = stream_block(key, q, w, step, kPurposeArea, attempt, 0u);
    const int64_t lo = area_pick(p, u.x, u.y);
    const double su = sqrt(u24(u.z)), u2 = u24(u.w);
    a.b0 = 1.0 - su;
    a.b1 = su * (1.0 - u2);
    a.b2 = su * u2;
    const int32_t* t = p.tris + 3 * lo;
    const double* v0 = p.verts_d + 3 * (int64_t)__ldg(t);
    const double* v1 = p.verts_d + 3 * (int64_t)__ldg(t + 1);
    const double* v2 = p.verts_d + 3 * (int64_t)__ldg(t + 2);
    a.y = make_double3(a.b0 * __ldg(v0) + a.b1 * __ldg(v1) + a.b2 * __ldg(v2),
                       a.b0 * __ldg(v0 + 1) + a.b1 * __ldg(v1 + 1) + a.b2 * __ldg(v2 + 1),
                       a.b0 * __ldg(v0 + 2) + a.b1 * __ldg(v1 + 2) + a.b2 * __ldg(v2 + 2));
    const double2 nxy = __ldg(reinterpret_cast<const double2*>(p.tri_n + lo));
    const double nz = __ldg(reinterpret_cast<const double*>(p.tri_n + lo) + 2);
    a.n = make_double3(nxy.x, nxy.y, nz);
    a.j = lo;
    return a;
}

// Transition kernel of the single-layer recursion from x (condition bx,
// normal nx; bx < 0: the query) to y, without the 1/p of the sampling
// (Table 1; Sec. 4.3 for the Dirichlet parts of mixed problems): G (query),
// -2 phi dG/dn_x (Neumann), -2 phi (dG/dn_x + alpha G) (Robin), -(k/p_k) G
// (Dirichlet, moving branch); dG/dn_x = (y - x) . n_x / (4 pi r^3).  0 for
// r < rmin.
__device__ __forceinline__ double sl_kernel(const WalkParams& p, int bx, double3 x, double3 nx,
                                            double3 y, double rmin)
{
    const double rx = y.x - x.x, ry = y.y - x.y, rz = y.z - x.z;
    const double rl = sqrt(rx * rx + ry * ry + rz * rz);
    if (rl < rmin) return 0.0;
    const double G = 1.0 / (kFourPi * rl);
    if (bx < 0) return G;
    if (bx == WOB_BC_DIRICHLET) return -((double)p.kmix / (double)p.pk) * G;
    const double dgdn = (rx * nx.x + ry * nx.y + rz * nx.z) / (kFourPi * rl * rl * rl);
    const double phi = (double)p.phi;
    if (bx == WOB_BC_NEUMANN) return -2.0 * phi * dgdn;
    return -2.0 * phi * (dgdn + (double)p.alpha * G);
}

// sl_data with the point-source field in FP32 from an FP64 difference and
// the normal derivative n . grad h in FP64 (it cancels where the field runs
// along the surface); polynomial and P1 data as sl_data (a polynomial's
// monomials cancel, and its FP64 evaluation costs little).
__device__ __forceinline__ double sl_data32(const WalkParams& p, int64_t j, double3 y, double b0,
                                            double b1, double b2, double3 n, int bc)
{
    const DataDev& D = p.data;
    if (D.mode == WOB_DATA_VERTEX_P1) {
        const int32_t* t = D.tris + 3 * j;
        return b0 * __ldg(D.vdata + t[0]) + b1 * __ldg(D.vdata + t[1]) + b2 * __ldg(D.vdata + t[2]);
    }
    if (D.mode == WOB_DATA_POLY) return sl_data(p, j, y, b0, b1, b2, n, bc);
    const double dx = y.x - D.x0[0], dy = y.y - D.x0[1], dz = y.z - D.x0[2];
    const float ri = rsqrtf((float)(dx * dx + dy * dy + dz * dz));
    const float h = D.scale * ri;
    const float f = -h * ri * ri;
    const float gx = f * (float)dx, gy = f * (float)dy, gz = f * (float)dz;
    if (bc == WOB_BC_DIRICHLET) return (double)h;
    const double dhdn = n.x * (double)gx + n.y * (double)gy + n.z * (double)gz;
    return bc == WOB_BC_ROBIN ? dhdn + (double)p.alpha * (double)h : dhdn;
}

// Single-layer walks (Table 1, Sec. 4.3), one thread per walk:
// u(x0) = int G mu and mu(x) = int K(x, y) mu(y) + src(x), src = 2 phi q
// (Neumann), 2 phi (q + alpha h) (Robin), k u_D (Dirichlet parts of mixed
// problems, whose mu(x) = mu(x) - k S mu + k u_D is sampled by moving with
// probability p_k or staying at x with weight 1 / (1 - p_k)).  The last
// source is halved (Sec. 4.1.2).  This kernel (FP64 kernels) serves
// resampled importance sampling (Talbot et al. 2005): the next point is
// drawn from p.ris area-uniform candidates with target |K|, weight sign(K)
// |Gamma| (sum of |K| over the candidates) / ris.  Plain area sampling runs
// in k_sl_walks_ff.
template <bool DEBUG>
__global__ void __launch_bounds__(128) k_sl_walks(WalkParams p)
{
    const StreamKey key{p.key0, p.key1};
    const int64_t total = p.Q * (int64_t)p.N;
    const double phi = (double)p.phi;
    const double area = p.area;
    const double rmin = 1e-12 * p.L;
    const int uniform_bc = p.kind == WOB_ROBIN_SL ? WOB_BC_ROBIN : WOB_BC_NEUMANN;
    double wc[kMaxRis];
    const int lane = threadIdx.x & 31;
    // warp-uniform loop over groups of 32 consecutive walks
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < total;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = base + lane;
        const bool live = idx < total;
        const int64_t qi = live ? idx / p.N : 0;
        const int64_t wi = idx - qi * p.N;
        double value = 0.0;
        if (live) {
            const uint32_t q = p.q_base + (uint32_t)qi;
            const uint32_t w = (uint32_t)(p.walk_begin + wi);
            double3 x = make_double3(p.queries[3 * qi], p.queries[3 * qi + 1], p.queries[3 * qi + 2]);
            double3 nx = make_double3(0.0, 0.0, 0.0);
            int bx = -1;
            int64_t jx = -1;
            double S = 0.0, P = 1.0, W0 = 0.0;
            for (int k = 0; k < p.M; ++k) {
                bool stay = false;
                if (bx == WOB_BC_DIRICHLET) {
                    const u32x4 u = stream_block(key, q, w, (uint32_t)k, kPurposeBranch, 0u, 0u);
                    stay = u24(u.x) >= (double)p.pk;
                }
                AreaPoint a;
                double wfac;
                if (stay) {
                    a.j = jx;
                    a.y = x;
                    a.n = nx;
                    a.b0 = a.b1 = a.b2 = 0.0;  // mixed problems take analytic data
                    wfac = 1.0 / (1.0 - (double)p.pk);
                } else {
                    double sumw = 0.0;
                    for (int c = 0; c < p.ris; ++c) {
                        const AreaPoint ac = area_point(p, key, q, w, (uint32_t)k, (uint32_t)c);
                        wc[c] = fabs(sl_kernel(p, bx, x, nx, ac.y, rmin));
                        sumw += wc[c];
                    }
                    if (!(sumw > 0.0)) break;  // every candidate has a zero kernel
                    const u32x4 u = stream_block(key, q, w, (uint32_t)k, kPurposeRis, 0u, 0u);
                    const double target = u53(u.x, u.y) * sumw;
                    double acc = 0.0;
                    int pick = p.ris - 1;
                    for (int c = 0; c < p.ris; ++c) {
                        acc += wc[c];
                        if (acc > target) {
                            pick = c;
                            break;
                        }
                    }
                    a = area_point(p, key, q, w, (uint32_t)k, (uint32_t)pick);
                    const double K = sl_kernel(p, bx, x, nx, a.y, rmin);
                    wfac = (K > 0.0 ? 1.0 : -1.0) * area * sumw / (double)p.ris;
                }
                if (k == 0) W0 = wfac; else P *= wfac;
                const int by = p.bc_type ? (int)__ldg(p.bc_type + a.j) : uniform_bc;
                const double dat = sl_data32(p, a.j, a.y, a.b0, a.b1, a.b2, a.n, by);
                double src = by == WOB_BC_DIRICHLET ? (double)p.kmix * dat : 2.0 * phi * dat;
                if (k == p.M - 1) src *= 0.5;
                S = fma(P, src, S);
                x = a.y;
                nx = a.n;
                bx = by;
                jx = a.j;
            }
            value = W0 * S;
            if (p.per_walk) p.per_walk[idx] = value;
            if (DEBUG && p.walk_flag) p.walk_flag[idx] = 0;
        }
        if (p.part) add_tile_partials(value, live, qi, wi, p.tpq, p.part);
    }
}

// ---------------------------------------------------------------------------
// Single-layer walks with area sampling in compensated FP32.  Each sample
// point is kept as its triangle's first vertex v0 (FP32, exact) plus the
// offset p = b1 e1 + b2 e2 in float-float (hi + lo, about 44 bits); the
// difference of two points is (v0_y - v0_x) + (p_y - p_x), with the vertex
// difference exact (Knuth's two-sum), so it is accurate relative to its own
// length however close the points are.  r . n_x (which cancels to ~r^2 / 2
// near x on a smooth surface) and the Robin numerator alpha r^2 + r . n_x
// (whose terms can cancel) are float-float sums; 1 / r, G and dG/dn_x are
// FP32 with relative error ~1e-7.  The product of weights is an FP32
// significand renormalised every step with an integer exponent; FP64 holds
// only the sum of terms (one add per step, the term assembled exactly from
// its bits by scale2) and the CDF target (one multiply).
// ---------------------------------------------------------------------------

// A boundary point in the compensated representation.
struct FFPoint {
    float v0[3];  // the triangle's first vertex
    ff p[3];      // offset from v0
    ff n[3];      // unit normal of the triangle
};

// Area-uniform boundary point of stream (q, w, step) in the compensated
// form: triangle j by area_pick, then (frame_point_ff, uniforms uz, uw) the
// square-root warp b1 = sqrt(u1) (1 - u2), b2 = sqrt(u1) u2 with sqrt(u1) in
// float-float and the offset p = b1 e1 + b2 e2 in float-float from the
// triangle's frame (six 16-byte loads); b0..b2 in FP32 for P1 data.
__device__ __forceinline__ void frame_point_ff(const WalkParams& p, int64_t j, uint32_t uz,
                                               uint32_t uw, FFPoint& y, float& b0, float& b1f,
                                               float& b2f)
{
    float fr[24];
    const float4* F = reinterpret_cast<const float4*>(p.tri_f + j);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float4 t = __ldg(F + i);
        fr[4 * i] = t.x; fr[4 * i + 1] = t.y; fr[4 * i + 2] = t.z; fr[4 * i + 3] = t.w;
    }
    constexpr int o_e1h = offsetof(TriFrame, e1h) / 4, o_e1l = offsetof(TriFrame, e1l) / 4;
    constexpr int o_e2h = offsetof(TriFrame, e2h) / 4, o_e2l = offsetof(TriFrame, e2l) / 4;
    constexpr int o_nh = offsetof(TriFrame, nh) / 4, o_nl = offsetof(TriFrame, nl) / 4;
    const float u2 = u24f(uw);
    const ff su = ff_sqrt(u24f(uz));
    const ff b1 = ff_mul_f(su, 1.f - u2), b2 = ff_mul_f(su, u2);
    b0 = 1.f - su.hi;
    b1f = b1.hi;
    b2f = b2.hi;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        y.v0[c] = fr[c];
        const ff e1 = {fr[o_e1h + c], fr[o_e1l + c]}, e2 = {fr[o_e2h + c], fr[o_e2l + c]};
        y.n[c] = {fr[o_nh + c], fr[o_nl + c]};
        y.p[c] = ff_add(ff_mul(e1, b1), ff_mul(e2, b2));
    }
}

__device__ __forceinline__ int64_t area_sample_ff(const WalkParams& p, StreamKey key, uint32_t q,
                                                  uint32_t w, uint32_t step, FFPoint& y,
                                                  float& b0, float& b1f, float& b2f)
{
    const u32x4 u = stream_block(key, q, w, step, kPurposeArea, 0u, 0u);
    const int64_t j = area_pick(p, u.x, u.y);
    frame_point_ff(p, j, u.z, u.w, y, b0, b1f, b2f);
    return j;
}

// Data of the single-layer problems at the point (v0 + p, normal n, on
// triangle j with barycentrics b0..b2), as sl_data, rounded to FP32: P1
// values in FP32, the point-source field in FP32 with n . grad h by FMAs (its
// error ~1e-7 of |grad h|; with precise_dn the projection n . (y - x0) is a
// float-float dot product, so the error is ~1e-7 of n . grad h itself),
// polynomial data in FP64 at the FP64 position (its monomials cancel) and
// then rounded.
__device__ __forceinline__ float sl_data_ff(const WalkParams& p, int64_t j, const FFPoint& y,
                                            float b0, float b1, float b2, int bc,
                                            bool precise_dn = false)
{
    const DataDev& D = p.data;
    if (D.mode == WOB_DATA_VERTEX_P1) {
        const int32_t* t = D.tris + 3 * j;
        return __fmaf_rn(b0, __ldg(D.vdata + t[0]),
                         __fmaf_rn(b1, __ldg(D.vdata + t[1]), b2 * __ldg(D.vdata + t[2])));
    }
    if (D.mode == WOB_DATA_POLY) {
        double3 yd, nd;
        yd.x = (double)y.v0[0] + ((double)y.p[0].hi + (double)y.p[0].lo);
        yd.y = (double)y.v0[1] + ((double)y.p[1].hi + (double)y.p[1].lo);
        yd.z = (double)y.v0[2] + ((double)y.p[2].hi + (double)y.p[2].lo);
        nd = make_double3((double)y.n[0].hi + (double)y.n[0].lo, (double)y.n[1].hi + (double)y.n[1].lo,
                          (double)y.n[2].hi + (double)y.n[2].lo);
        return (float)sl_data(p, j, yd, (double)b0, (double)b1, (double)b2, nd, bc);
    }
    const float dx = (y.v0[0] - D.x0[0]) + y.p[0].hi;
    const float dy = (y.v0[1] - D.x0[1]) + y.p[1].hi;
    const float dz = (y.v0[2] - D.x0[2]) + y.p[2].hi;
    const float ri = rsqrt_ftz(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz)));
    const float h = D.scale * ri;
    if (bc == WOB_BC_DIRICHLET) return h;
    float dn = __fmaf_rn(y.n[0].hi, dx, __fmaf_rn(y.n[1].hi, dy, y.n[2].hi * dz));
    if (precise_dn) {  // n . (y - x0) as a float-float dot product (it cancels where
                       // the field runs along the surface)
        ff d[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) d[c] = ff_add(two_sum(y.v0[c], -D.x0[c]), y.p[c]);
        dn = ff_dot3(y.n, d).hi;
    }
    const float dhdn = -h * ri * ri * dn;
    return bc == WOB_BC_ROBIN ? __fmaf_rn(p.alpha, h, dhdn) : dhdn;
}

// The single-layer walks of k_sl_walks for area sampling (p.ris <= 1), in
// the compensated FP32 arithmetic above; the transition kernel and the
// sources are those of sl_kernel / sl_data (Table 1, Sec. 4.3).
template <bool DEBUG>
__global__ void __launch_bounds__(128, WOB_SL_MIN_BLOCKS) k_sl_walks_ff(WalkParams p)
{
    constexpr float kInv4Pi = 0.0795774715459476678f;
    const StreamKey key{p.key0, p.key1};
    const int64_t total = p.Q * (int64_t)p.N;
    const float two_phi = 2.f * (float)p.phi;
    const float rmin2 = (float)(1e-24 * p.L * p.L);
    const int uniform_bc = p.kind == WOB_ROBIN_SL ? WOB_BC_ROBIN : WOB_BC_NEUMANN;
    // weight factors: |Gamma| (query), -|Gamma| k / p_k (Dirichlet parts),
    // -2 phi |Gamma| (Neumann / Robin), rounded to FP32 once
    const float w_query = (float)p.area;
    const float w_dirichlet = (float)(-p.area * (double)(p.kmix / p.pk));
    const float w_layer = (float)(-2.0 * (double)p.phi * p.area);
    const float w_stay = (float)(1.0 / (1.0 - (double)p.pk));
    const int lane = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < total;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = base + lane;
        const bool live = idx < total;
        const int64_t qi = live ? idx / p.N : 0;
        const int64_t wi = idx - qi * p.N;
        double value = 0.0;
        if (live) {
            const uint32_t q = p.q_base + (uint32_t)qi;
            const uint32_t w = (uint32_t)(p.walk_begin + wi);
            // x: the query (v0 = its coordinates, p = 0) or the last sample
            FFPoint x;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                x.v0[c] = p.queries[3 * qi + c];
                x.p[c] = {0.f, 0.f};
                x.n[c] = {0.f, 0.f};
            }
            int bx = -1;
            int64_t jx = -1;
            // the weight product P = Pm 2^Pe (FP32 significand renormalised to
            // [1, 2) every step, integer exponent: no overflow over long walks)
            // and the sum of terms S in FP64
            double S = 0.0;
            float Pm = 1.f, W0 = 0.f;
            int Pe = 0;
            for (int k = 0; k < p.M; ++k) {
                bool stay = false;
                if (bx == WOB_BC_DIRICHLET) {
                    const u32x4 u = stream_block(key, q, w, (uint32_t)k, kPurposeBranch, 0u, 0u);
                    stay = u24f(u.x) >= p.pk;  // both exact in FP32
                }
                FFPoint y;
                int64_t j;
                float b0 = 0.f, b1f = 0.f, b2f = 0.f;  // mixed problems' stays take analytic data
                float wf;
                if (stay) {
                    y = x;
                    j = jx;
                    wf = w_stay;
                } else {
                    j = area_sample_ff(p, key, q, w, (uint32_t)k, y, b0, b1f, b2f);
                    ff r[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        r[c] = ff_add(two_sum(y.v0[c], -x.v0[c]), ff_sub(y.p[c], x.p[c]));
                    const float r2 =
                        __fmaf_rn(r[0].hi, r[0].hi, __fmaf_rn(r[1].hi, r[1].hi, r[2].hi * r[2].hi));
                    if (r2 < rmin2) break;  // empty sample
                    const float ri = rsqrt_ftz(r2);
                    const float G = kInv4Pi * ri;
                    if (bx < 0) {
                        wf = w_query * G;
                    } else if (bx == WOB_BC_DIRICHLET) {
                        wf = w_dirichlet * G;
                    } else {
                        ff num = ff_dot3(x.n, r);  // r . n_x
                        if (bx == WOB_BC_ROBIN) {
                            // alpha r^2 + r . n_x, r^2 as a float-float sum of squares
                            const ff rr = ff_dot3(r, r);
                            num = ff_add(num, ff_mul_f(rr, p.alpha));
                        }
                        wf = w_layer * (num.hi * (ri * ri) * G);
                    }
                }
                if (k == 0) {
                    W0 = wf;
                } else {
                    Pm *= wf;
                    const uint32_t pb = __float_as_uint(Pm);
                    const int pe = (int)((pb >> 23) & 0xFFu);
                    if (pe != 0 && pe != 255) {  // zero, subnormal, inf, NaN stay as they are
                        Pe += pe - 127;
                        Pm = __uint_as_float((pb & 0x807FFFFFu) | 0x3F800000u);
                    }
                }
                const int by = p.bc_type ? (int)__ldg(p.bc_type + j) : uniform_bc;
                const float dat = sl_data_ff(p, j, y, b0, b1f, b2f, by);
                float src = (by == WOB_BC_DIRICHLET ? p.kmix : two_phi) * dat;
                if (k == p.M - 1) src *= 0.5f;
                S += scale2(Pm * src, Pe);
                x = y;
                bx = by;
                jx = j;
            }
            value = (double)W0 * S;
            if (p.per_walk) p.per_walk[idx] = value;
            if (DEBUG && p.walk_flag) p.walk_flag[idx] = 0;
        }
        if (p.part) add_tile_partials(value, live, qi, wi, p.tpq, p.part);
    }
}

// Neumann walks through the direct boundary integral equation (Sec. 4.2):
// at a point x off the boundary u = phi (S q - int dG/dn_y u), on it
// u = 2 phi (S q - int dG/dn_y u).  Each vertex takes one area-uniform
// point x' for the source (|Gamma| G(x, x') q(x'), times c = phi off the
// boundary, 2 phi on it, halved at the last vertex x_M -- Sec. 4.1.2) and
// one line for the dG/dn_y term (weight phi (m/2) s from x0, phi m s from a
// boundary vertex, as the double-layer walks).  A query on triangle
// query_prim is boundary vertex 1 with weight 1.  One thread per walk.
template <bool DEBUG>
__global__ void __launch_bounds__(128, WOB_DL_MIN_BLOCKS) k_nd_walks(WalkParams p)
{
    const StreamKey key{p.key0, p.key1};
    const int64_t total = p.Q * (int64_t)p.N;
    const double phi = (double)p.phi;
    const float phi_f = (float)p.phi, area_f = (float)p.area;
    const float rmin2 = (float)(1e-24 * p.L * p.L);
    // walk state (point and axis as float-float pairs, S and P in FP64)
    // parked in shared memory during the traversal (as in k_dl_walks), which
    // leaves the postponed-leaf traversal its registers
    __shared__ double slots[8 * 128];
    __shared__ int leafq[kLeafQ * 128];
    const WalkSlot ws{slots + threadIdx.x, 128};
    const LeafQueue lq{leafq + threadIdx.x, 128};
    enum { X0 = 0, X1, X2, D0, D1, D2, SS, PP };
    int err = 0;
    int stack[kStackSize];
    int hits[kMaxHits];
    const int lane = threadIdx.x & 31;
    // warp-uniform loop over groups of 32 consecutive walks
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < total;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = base + lane;
        const bool live = idx < total;
        const int64_t qi = live ? idx / p.N : 0;
        const int64_t wi = idx - qi * p.N;
        double value = 0.0;
        if (live) {
            const uint32_t q = p.q_base + (uint32_t)qi;
            const uint32_t w = (uint32_t)(p.walk_begin + wi);
            ws.set(X0, pack_ff({p.queries[3 * qi], 0.f}));
            ws.set(X1, pack_ff({p.queries[3 * qi + 1], 0.f}));
            ws.set(X2, pack_ff({p.queries[3 * qi + 2], 0.f}));
            ws.set(SS, 0.0);
            ws.set(PP, 1.0);
            const LineOut lo{DEBUG && p.line_m ? p.line_m + idx * p.M : nullptr,
                             DEBUG && p.line_prim ? p.line_prim + idx * p.M : nullptr,
                             DEBUG && p.line_flag ? p.line_flag + idx * p.M : nullptr};
            if (DEBUG)
                for (int k = 0; k < p.M; ++k) lo.put(k, -1, -1, 0);
            int self = -1, k0 = 0, wflag = 0;
            if (p.query_prim) {
                const int32_t prim = p.query_prim[qi];
                if (prim >= 0 && prim < p.T) {
                    self = p.inv_order[prim];
                    k0 = 1;
                }
            }
            for (int k = k0; k <= p.M; ++k) {
                // source at vertex k
                {
                    FFPoint y;
                    float b0, b1, b2;
                    const int64_t j = area_sample_ff(p, key, q, w, (uint32_t)k, y, b0, b1, b2);
                    float r2 = 0.f;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const ff x = unpack_ff(ws.get(X0 + c));
                        const float rc = ff_add(ff_sub({y.v0[c], 0.f}, x), y.p[c]).hi;
                        r2 = __fmaf_rn(rc, rc, r2);
                    }
                    if (r2 >= rmin2) {
                        const float f = sl_data_ff(p, j, y, b0, b1, b2, WOB_BC_NEUMANN);
                        float c = (k == 0) ? phi_f : 2.f * phi_f;
                        if (k == p.M) c *= 0.5f;
                        const float G = 0.0795774715459476678f * rsqrt_ftz(r2);
                        ws.set(SS, fma(ws.get(PP), (double)(c * area_f * G * f), ws.get(SS)));
                    }
                }
                if (k == p.M) break;
                // line from vertex k to vertex k + 1
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
                const float Tthr = p.edge_thr_L * fabsf(L.Sz);
                Trav t;
                trav_init(t);
                uint32_t nn = 0, nt = 0;
                trace_wide_q<false, false, true>(p.nodes, p.tv, L, make_float3(0.f, 0.f, 0.f), Tthr, p.tauL,
                                           p.graze, self, t, hits, stack, key, q, w, (uint32_t)k, nn,
                                           nt, err, p.iter_limit, lq);
                wflag |= t.flag;
                if (t.m == 0) {
                    if (DEBUG) lo.put(k, 0, -1, t.flag);
                    break;
                }
                const int pos = select_hit(p.tv, t, hits, key, q, w, (uint32_t)k);
                if (DEBUG) lo.put(k, t.m, (int)prim_of(p.tv, pos), t.flag);
                const ff x[3] = {unpack_ff(ws.get(X0)), unpack_ff(ws.get(X1)), unpack_ff(ws.get(X2))};
                const ff d[3] = {unpack_ff(ws.get(D0)), unpack_ff(ws.get(D1)), unpack_ff(ws.get(D2))};
                ff y[3];
                const double ms = (double)(t.m * refine_hit_ff(p.tv, pos, x, d, y));
                ws.set(PP, ws.get(PP) * ((k == 0) ? 0.5 * phi * ms : phi * ms));
                ws.set(X0, pack_ff(y[0]));
                ws.set(X1, pack_ff(y[1]));
                ws.set(X2, pack_ff(y[2]));
                self = pos;
            }
            value = ws.get(SS);
            if (p.per_walk) p.per_walk[idx] = value;
            if (DEBUG && p.walk_flag) p.walk_flag[idx] = (uint8_t)wflag;
        }
        if (p.part) add_tile_partials(value, live, qi, wi, p.tpq, p.part);
    }
    if (err) atomicOr(p.error_word, err);
}

// ---------------------------------------------------------------------------
// Forward (adjoint) single-layer Neumann paths (Sec. 4.4.3).  With
// u(x) = int G(x, y) mu(y) dA, mu = T mu + f, T's kernel
// K(y, z) = -2 phi dG/dn_x(y, z) and f = 2 phi q, a path reads the truncated
// series sum_j c_j <G(x, .), T^j f> from its source end: z_0 ~ p on the
// boundary, a_0 = f(z_0) / p(z_0); from z_j a line (all hits, one picked,
// as the double-layer walks) gives z_{j+1} and K(z_{j+1}, z_j) / p = phi m s,
// so a_{j+1} = a_j phi m s; vertex j then contributes c_j a_j G(x, z_j) to
// every evaluation point x (c_j = 1, 1/2 for the last, Sec. 4.1.2).
// Streams: path p draws as query p, walk kForwardWalk.
// ---------------------------------------------------------------------------
constexpr uint32_t kForwardWalk = 0xFFFFFFFFu;

// Start weight of triangle j for boundary-value-weighted paths, first part:
// area x |q(centroid)|.
__global__ void k_fwd_qc(WalkParams p, double* __restrict__ aq)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < p.T;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t* t = p.tris + 3 * j;
        double c[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 3; ++d) c[d] += (double)__ldg(p.verts + 3 * (int64_t)__ldg(t + k) + d);
        const double3 y = make_double3(c[0] / 3.0, c[1] / 3.0, c[2] / 3.0);
        const NormalArea na = p.tri_n[j];
        const double3 n = make_double3(na.nx, na.ny, na.nz);
        const double q = sl_data(p, j, y, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, n, WOB_BC_NEUMANN);
        aq[j] = na.area * fabs(q);
    }
}

// ... second part: + beta mean|q| area (mean over the boundary, from the
// inclusive sums of the first part); inclusive sums of the result are the CDF.
__global__ void k_fwd_mix(WalkParams p, const double* __restrict__ aq_incl, double beta,
                          double* __restrict__ w)
{
    const double qbar = aq_incl[p.T - 1] / p.area;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < p.T;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double aq = aq_incl[j] - (j > 0 ? aq_incl[j - 1] : 0.0);
        w[j] = aq + beta * qbar * p.tri_n[j].area;
    }
}

__global__ void __launch_bounds__(128, WOB_DL_MIN_BLOCKS)
    k_fwd_paths(WalkParams p, int64_t n_paths, int start_mode, const double* __restrict__ wcdf,
                double* __restrict__ zpos, double* __restrict__ zw, uint8_t* __restrict__ flags)
{
    const StreamKey key{p.key0, p.key1};
    const double phi = (double)p.phi;
    const double* cdf = start_mode == 1 ? wcdf : p.cdf;
    const double tot = start_mode == 1 ? wcdf[p.T - 1] : p.area;
    int err = 0;
    int stack[kStackSize];
    int hits[kMaxHits];
    for (int64_t path = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; path < n_paths;
         path += (int64_t)gridDim.x * blockDim.x) {
        double* zp = zpos + path * p.M * 3;
        double* wp = zw + path * p.M;
        for (int j = 0; j < p.M; ++j) {
            zp[3 * j] = zp[3 * j + 1] = zp[3 * j + 2] = 0.0;
            wp[j] = 0.0;
        }
        const uint32_t q = (uint32_t)path;
        const u32x4 u = stream_block(key, q, kForwardWalk, 0u, kPurposeArea, 0u, 0u);
        const long long target = __double_as_longlong(u53(u.x, u.y) * tot);
        int64_t lo = 0, hi = p.T - 1;
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (__double_as_longlong(__ldg(cdf + mid)) > target) hi = mid; else lo = mid + 1;
        }
        FFPoint y;
        float b0, b1, b2;
        frame_point_ff(p, lo, u.z, u.w, y, b0, b1, b2);
        const double pdf = start_mode == 1
                               ? ((cdf[lo] - (lo > 0 ? cdf[lo - 1] : 0.0)) / p.tri_n[lo].area) / tot
                               : 1.0 / p.area;
        double a = 2.0 * phi * (double)sl_data_ff(p, lo, y, b0, b1, b2, WOB_BC_NEUMANN, true) / pdf;
        ff z[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) z[c] = ff_add({y.v0[c], 0.f}, y.p[c]);
        int self = p.inv_order[lo], flag = 0;
        for (int j = 0; j < p.M; ++j) {
            zp[3 * j] = ff_join(z[0]);
            zp[3 * j + 1] = ff_join(z[1]);
            zp[3 * j + 2] = ff_join(z[2]);
            wp[j] = (j == p.M - 1 ? 0.5 : 1.0) * a;
            if (j == p.M - 1) break;
            ff d[3];
            line_axis_ff(key, q, kForwardWalk, (uint32_t)j, d);
            const LinePre L = line_pre(make_float3(z[0].hi, z[1].hi, z[2].hi),
                                       make_float3(d[0].hi, d[1].hi, d[2].hi));
            const float Tthr = p.edge_thr_L * fabsf(L.Sz);
            Trav tr;
            trav_init(tr);
            uint32_t nn = 0, nt = 0;
            trace_wide<false, false>(p.nodes, p.tv, L, make_float3(0.f, 0.f, 0.f), Tthr, p.tauL,
                                     p.graze, self, tr, hits, stack, key, q, kForwardWalk,
                                     (uint32_t)j, nn, nt, err, p.iter_limit);
            flag |= tr.flag;
            if (tr.m == 0) break;
            const int pos = select_hit(p.tv, tr, hits, key, q, kForwardWalk, (uint32_t)j);
            ff yz[3];
            a *= phi * (double)(tr.m * refine_hit_ff(p.tv, pos, z, d, yz));
#pragma unroll
            for (int c = 0; c < 3; ++c) z[c] = yz[c];
            self = pos;
        }
        if (flags) flags[path] = (uint8_t)flag;
    }
    if (err) atomicOr(p.error_word, err);
}

// Explicit connection of every path vertex to every query (an N-body sum):
// per query, v_p = sum_j w_pj G(x, z_pj) for each path, est = mean of v_p,
// var = their unbiased variance.
//
// k_fwd_pack turns each path into M float4 records (position, w / 4 pi; a
// vertex of weight 0 -- after a missed line -- sits far away with weight 0,
// so the inner loop needs no branch) and one live byte (0: every record of
// the path is 0, the path adds nothing but still counts in the mean).
// k_fwd_connect: work items are (block of kFwdThreads x kFwdQ queries, split
// of the paths); a persistent grid takes them in turn.  Whole paths are
// staged in shared memory; each thread keeps kFwdQ queries in registers as
// pairs, so one broadcast shared load feeds kFwdQ pairs and the distances,
// squared distances and the sum of w G run as packed FP32x2 operations (two
// queries per instruction, each lane rounded as the scalar operation would
// be), which leaves the reciprocal square roots (one MUFU operation per
// pair) as the bound; distances, G and v_p in FP32.
// The sums over paths run in FP32 for kFwdFold paths and are then folded into
// FP64 sums kept in shared memory (FP64 issues at 1/64 of the FP32 rate on
// this GPU: one FP64 add per path and query would cost as much as the
// pairs).  k_fwd_finish adds the
// splits' FP64 partial sums in a fixed order.
constexpr int kFwdTile = 1024;     // vertex records per tile (max_len <= kFwdTile)
constexpr int kFwdThreads = 128;
constexpr int kFwdQ = 8;           // queries per thread
static_assert(kFwdQ % 2 == 0, "queries are processed in pairs");
constexpr int kFwdFold = 32;       // paths summed in FP32 before an FP64 fold
constexpr float kFwdFar = 1e18f;   // |r|^2 ~ 3e36 stays finite in FP32

__global__ void k_fwd_pack(const double* __restrict__ zpos, const double* __restrict__ zw,
                           int64_t n_paths, int M, float4* __restrict__ rec,
                           uint8_t* __restrict__ live)
{
    constexpr double kInv4Pi = 0.0795774715459476678844418816862571810;
    for (int64_t path = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; path < n_paths;
         path += (int64_t)gridDim.x * blockDim.x) {
        int any = 0;
        for (int j = 0; j < M; ++j) {
            const int64_t r = path * M + j;
            const float w = (float)(zw[r] * kInv4Pi);
            rec[r] = w != 0.f ? make_float4((float)zpos[3 * r], (float)zpos[3 * r + 1],
                                            (float)zpos[3 * r + 2], w)
                              : make_float4(kFwdFar, kFwdFar, kFwdFar, 0.f);
            any |= w != 0.f;
        }
        live[path] = (uint8_t)any;
    }
}

__global__ void __launch_bounds__(kFwdThreads)
    k_fwd_connect(const float* __restrict__ queries, int64_t Q, const float4* __restrict__ rec_g,
                  const uint8_t* __restrict__ live_g, int64_t n_paths, int M, int64_t q_blocks,
                  int splits, int64_t per_split, double* __restrict__ part)
{
    __shared__ float4 rec[kFwdTile];
    __shared__ uint8_t live[kFwdTile];
    __shared__ double fsum[kFwdQ][kFwdThreads], fsq[kFwdQ][kFwdThreads];  // FP64 folds
    const int ppt = kFwdTile / M;  // whole paths per tile
    const int64_t items = q_blocks * splits;
    const int t = threadIdx.x;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t qb = item % q_blocks;
        const int sp = (int)(item / q_blocks);
        const int64_t pb = (int64_t)sp * per_split;
        const int64_t pe = pb + per_split < n_paths ? pb + per_split : n_paths;
        // negated query coordinates, queries 2i and 2i + 1 in pair i: c - x
        // is computed as c + (-x), which rounds identically
        float2 nx[kFwdQ / 2], ny[kFwdQ / 2], nz[kFwdQ / 2];
        float s32[kFwdQ], ss32[kFwdQ];
#pragma unroll
        for (int k = 0; k < kFwdQ; ++k) {
            const int64_t qi = (qb * kFwdQ + k) * kFwdThreads + t;
            const bool ok = qi < Q;
            const float qx = ok ? -queries[3 * qi] : 0.f, qy = ok ? -queries[3 * qi + 1] : 0.f,
                        qz = ok ? -queries[3 * qi + 2] : 0.f;
            if (k & 1) {
                nx[k / 2].y = qx;
                ny[k / 2].y = qy;
                nz[k / 2].y = qz;
            } else {
                nx[k / 2].x = qx;
                ny[k / 2].x = qy;
                nz[k / 2].x = qz;
            }
            s32[k] = ss32[k] = 0.f;
            fsum[k][t] = fsq[k][t] = 0.0;
        }
        int cnt = 0;
        for (int64_t p0 = pb; p0 < pe; p0 += ppt) {
            const int np = (int)(pe - p0 < ppt ? pe - p0 : ppt);
            __syncthreads();
            for (int i = t; i < np * M; i += kFwdThreads) rec[i] = rec_g[p0 * M + i];
            for (int i = t; i < np; i += kFwdThreads) live[i] = live_g[p0 + i];
            __syncthreads();
            for (int pp = 0; pp < np; ++pp) {
                if (!live[pp]) continue;  // the same path for the whole block
                float2 v2[kFwdQ / 2];
#pragma unroll
                for (int k = 0; k < kFwdQ / 2; ++k) v2[k] = make_float2(0.f, 0.f);
                const float4* rp = rec + pp * M;
#pragma unroll 2
                for (int j = 0; j < M; ++j) {
                    const float4 c = rp[j];
                    const float2 cx = make_float2(c.x, c.x), cy = make_float2(c.y, c.y),
                                 cz = make_float2(c.z, c.z), cw = make_float2(c.w, c.w);
#pragma unroll
                    for (int k = 0; k < kFwdQ / 2; ++k) {
                        const float2 dx = __fadd2_rn(cx, nx[k]), dy = __fadd2_rn(cy, ny[k]),
                                     dz = __fadd2_rn(cz, nz[k]);
                        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                        v2[k] = __ffma2_rn(cw, make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y)), v2[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < kFwdQ; ++k) {
                    const float v = (k & 1) ? v2[k / 2].y : v2[k / 2].x;
                    s32[k] += v;
                    ss32[k] = fmaf(v, v, ss32[k]);
                }
                if (++cnt == kFwdFold) {
#pragma unroll
                    for (int k = 0; k < kFwdQ; ++k) {
                        fsum[k][t] += (double)s32[k];
                        fsq[k][t] += (double)ss32[k];
                        s32[k] = ss32[k] = 0.f;
                    }
                    cnt = 0;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kFwdQ; ++k) {
            const int64_t qi = (qb * kFwdQ + k) * kFwdThreads + t;
            if (qi < Q) {
                part[(2 * (int64_t)sp) * Q + qi] = fsum[k][t] + (double)s32[k];
                part[(2 * (int64_t)sp + 1) * Q + qi] = fsq[k][t] + (double)ss32[k];
            }
        }
    }
}

__global__ void k_fwd_finish(const double* __restrict__ part, int splits, int64_t Q,
                             int64_t n_paths, double* __restrict__ est, double* __restrict__ var,
                             const int* __restrict__ err)
{
    const bool bad = err && *err != 0;  // a path's line gave up
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Q;
         q += (int64_t)gridDim.x * blockDim.x) {
        double sum = 0.0, sumsq = 0.0;
        for (int sp = 0; sp < splits; ++sp) {
            sum += part[(2 * (int64_t)sp) * Q + q];
            sumsq += part[(2 * (int64_t)sp + 1) * Q + q];
        }
        const double mean = sum / (double)n_paths;
        est[q] = bad ? __longlong_as_double(0x7FF8000000000000ll) : mean;
        var[q] = bad ? __longlong_as_double(0x7FF8000000000000ll)
                     : (n_paths > 1 ? fmax(sumsq - sum * mean, 0.0) / (double)(n_paths - 1)
                                    : 0.0);
    }
}

// Splits of the paths for k_fwd_connect: enough work items to fill every
// resident block slot, and a count of items close to a whole number of
// rounds of the persistent grid (the last round is the idle tail).
static int fwd_splits(int64_t q_blocks, int64_t max_splits, int64_t slots)
{
    int best = 1;
    double best_eff = -1.0;
    for (int s = 1; s <= 64 && s <= max_splits; ++s) {
        const int64_t items = q_blocks * s;
        const int64_t rounds = (items + slots - 1) / slots;
        const double eff = (double)items / (double)(rounds * slots);
        if (eff > best_eff + 0.02) {
            best_eff = eff;
            best = s;
        }
        if (eff >= 0.95) break;
    }
    return best;
}

// One warp per query: mean and unbiased variance in a fixed order.
// err (may be NULL): the solve's device check word; when a traversal check
// fired during the solve, every estimate of the call is NaN (the walk
// kernels themselves carry no per-walk check: it would cost registers in
// the traversal loop).
__device__ __forceinline__ bool solve_failed(const int* err) { return err && *err != 0; }

__global__ void k_reduce(const double* __restrict__ per_walk, int64_t Q, int32_t N,
                         double* __restrict__ est, double* __restrict__ var,
                         const int* __restrict__ err)
{
    const bool bad = solve_failed(err);
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); q < Q;
         q += warps) {
        const double* v = per_walk + q * N;
        double s = 0.0;
        for (int i = lane; i < N; i += 32) s += v[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        const double mean = s / N;
        double ss = 0.0;
        for (int i = lane; i < N; i += 32) {
            const double e = v[i] - mean;
            ss = fma(e, e, ss);
        }
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
        if (lane == 0) {
            est[q] = bad ? __longlong_as_double(0x7FF8000000000000ll) : mean;
            var[q] = bad ? __longlong_as_double(0x7FF8000000000000ll)
                         : (N > 1 ? ss / (N - 1) : 0.0);
        }
    }
}

__global__ void k_reduce_accum(const double* __restrict__ per_walk, int64_t Q, int32_t N,
                               double* __restrict__ sum, double* __restrict__ sumsq,
                               const int* __restrict__ err)
{
    const double bad = solve_failed(err) ? __longlong_as_double(0x7FF8000000000000ll) : 0.0;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); q < Q;
         q += warps) {
        const double* v = per_walk + q * N;
        double s = 0.0, ss = 0.0;
        for (int i = lane; i < N; i += 32) {
            s += v[i];
            ss = fma(v[i], v[i], ss);
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
            ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
        }
        if (lane == 0) {
            sum[q] += s + bad;
            sumsq[q] += ss + bad;
        }
    }
}

// One warp per query from the (sum, sum of squares) partials of its tpq
// 32-walk blocks: mean and unbiased variance, blocks combined in a fixed
// order (lane i takes blocks i, i + 32, ..., then a fixed shuffle tree).
__global__ void k_reduce_part(const double* __restrict__ part, int64_t Q, int32_t N, int32_t tpq,
                              double* __restrict__ est, double* __restrict__ var,
                              double* __restrict__ sum, double* __restrict__ sumsq,
                              const int* __restrict__ err)
{
    const bool bad = solve_failed(err);
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); q < Q;
         q += warps) {
        const double2* pq = reinterpret_cast<const double2*>(part) + q * tpq;
        double s = 0.0, ss = 0.0;
        for (int i = lane; i < tpq; i += 32) {
            const double2 v = pq[i];
            s += v.x;
            ss += v.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
            ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
        }
        if (lane == 0) {
            const double nan = __longlong_as_double(0x7FF8000000000000ll);
            if (est) {
                const double mean = s / N;
                est[q] = bad ? nan : mean;
                var[q] = bad ? nan : (N > 1 ? fmax(ss - s * mean, 0.0) / (N - 1) : 0.0);
            }
            if (sum) {
                sum[q] += bad ? nan : s;
                sumsq[q] += bad ? nan : ss;
            }
        }
    }
}

__global__ void k_trace_lines(const float4* __restrict__ nodes, const float4* __restrict__ tv,
                              const int32_t* __restrict__ inv_order, int64_t n_tris,
                              int iter_limit, const double* __restrict__ o,
                              const double* __restrict__ d, const int32_t* __restrict__ exclude,
                              const uint32_t* __restrict__ keys, int64_t n, uint32_t key0,
                              uint32_t key1, float tauL, float edge_thr_L, int32_t* m,
                              int32_t* sum_s, int32_t* prim, int32_t* s_out, double* t_out,
                              double* y_out, uint8_t* flag, int* error_word)
{
    int err = 0;
    const StreamKey key{key0, key1};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double3 x = make_double3(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
        const double3 dd = make_double3(d[3 * i], d[3 * i + 1], d[3 * i + 2]);
        const int ex = exclude ? exclude[i] : -1;
        const int self = (ex >= 0 && ex < n_tris) ? inv_order[ex] : -1;
        Trav t;
        const int pos = trace_line<true>(
            nodes, tv, make_float3((float)x.x, (float)x.y, (float)x.z),
            make_float3((float)dd.x, (float)dd.y, (float)dd.z), self, key, keys[3 * i],
            keys[3 * i + 1], keys[3 * i + 2], edge_thr_L, tauL, kGraze, t, err, iter_limit);
        m[i] = t.m;
        if (sum_s) sum_s[i] = t.sum_s;
        if (flag) flag[i] = (uint8_t)t.flag;
        int pr = -1, sg = 0;
        double tt = 0.0;
        double3 yy = make_double3(0.0, 0.0, 0.0);
        if (pos >= 0) {
            const Refined r = refine_hit(tv, pos, x, dd);
            pr = (int)prim_of(tv, pos);
            sg = r.s;
            yy = r.y;
            tt = (r.y.x - x.x) * dd.x + (r.y.y - x.y) * dd.y + (r.y.z - x.z) * dd.z;
        }
        if (prim) prim[i] = pr;
        if (s_out) s_out[i] = sg;
        if (t_out) t_out[i] = tt;
        if (y_out) {
            y_out[3 * i] = yy.x;
            y_out[3 * i + 1] = yy.y;
            y_out[3 * i + 2] = yy.z;
        }
    }
    if (err) atomicOr(error_word, err);
}

__global__ void k_line_axes(uint32_t key0, uint32_t key1, const uint32_t* __restrict__ qws,
                            int64_t n, double* __restrict__ d)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double3 a = line_axis(StreamKey{key0, key1}, qws[3 * i], qws[3 * i + 1], qws[3 * i + 2]);
        d[3 * i] = a.x;
        d[3 * i + 1] = a.y;
        d[3 * i + 2] = a.z;
    }
}

__global__ void k_philox(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ keyv,
                         int64_t n, uint32_t* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const u32x4 r = philox4x32_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3],
                                      keyv[2 * i], keyv[2 * i + 1]);
        out[4 * i] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    }
}

}  // namespace

int launch_dl_walks(const WalkParams& p, bool counted, bool debug, cudaStream_t s)
{
    const int threads = 128;
    const int64_t work = p.Q * (int64_t)p.N;
    if (p.per_walk_grad) {
        k_dl_walks<false, false, true><<<grid_for((const void*)k_dl_walks<false, false, true>,
                                                  threads, 0, work), threads, 0, s>>>(p);
    } else if (counted) {
        k_dl_walks<true, true><<<grid_for((const void*)k_dl_walks<true, true>, threads, 0, work),
                                 threads, 0, s>>>(p);
    } else if (debug) {
        k_dl_walks<false, true><<<grid_for((const void*)k_dl_walks<false, true>, threads, 0, work),
                                  threads, 0, s>>>(p);
    } else {
        k_dl_walks<false, false><<<grid_for((const void*)k_dl_walks<false, false>, threads, 0, work),
                                   threads, 0, s>>>(p);
    }
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int launch_sl_walks(const WalkParams& p, bool debug, cudaStream_t s)
{
    const int threads = 128;
    const int64_t work = p.Q * (int64_t)p.N;
    if (p.ris > 1) {  // resampling: FP64 kernels (its pick compares running sums)
        if (debug)
            k_sl_walks<true><<<grid_for((const void*)k_sl_walks<true>, threads, 0, work), threads, 0, s>>>(p);
        else
            k_sl_walks<false><<<grid_for((const void*)k_sl_walks<false>, threads, 0, work), threads, 0, s>>>(p);
    } else if (debug) {
        k_sl_walks_ff<true><<<grid_for((const void*)k_sl_walks_ff<true>, threads, 0, work), threads, 0, s>>>(p);
    } else {
        k_sl_walks_ff<false><<<grid_for((const void*)k_sl_walks_ff<false>, threads, 0, work), threads, 0, s>>>(p);
    }
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int launch_nd_walks(const WalkParams& p, bool debug, cudaStream_t s)
{
    const int threads = 128;
    const int64_t work = p.Q * (int64_t)p.N;
    if (debug)
        k_nd_walks<true><<<grid_for((const void*)k_nd_walks<true>, threads, 0, work), threads, 0, s>>>(p);
    else
        k_nd_walks<false><<<grid_for((const void*)k_nd_walks<false>, threads, 0, work), threads, 0, s>>>(p);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int launch_forward(const WalkParams& p, int64_t n_paths, int start_mode, double beta,
                   const float* queries, int64_t Q, double* zpos, double* zw, uint8_t* flags,
                   double* est, double* var, cudaStream_t s)
{
    double* buf = nullptr;  // aq, its sums, start weights, their sums: 4 x T doubles
    if (start_mode == 1) {
        WOB_CUDA_TRY(cudaMallocAsync((void**)&buf, 4 * p.T * sizeof(double), s));
        const int g = grid_for((const void*)k_fwd_qc, 256, 0, p.T);
        k_fwd_qc<<<g, 256, 0, s>>>(p, buf);
        int rc = inclusive_scan<double>(buf, buf + p.T, p.T, s);
        if (rc == WOB_OK) {
            k_fwd_mix<<<g, 256, 0, s>>>(p, buf + p.T, beta, buf + 2 * p.T);
            rc = inclusive_scan<double>(buf + 2 * p.T, buf + 3 * p.T, p.T, s);
        }
        if (rc != WOB_OK) {
            cudaFreeAsync(buf, s);
            return rc;
        }
    }
    const int threads = 128;
    k_fwd_paths<<<grid_for((const void*)k_fwd_paths, threads, 0, n_paths), threads, 0, s>>>(
        p, n_paths, start_mode, buf ? buf + 3 * p.T : nullptr, zpos, zw, flags);
    int rc = cudaGetLastError() == cudaSuccess ? WOB_OK : WOB_ERR_CUDA;
    if (buf) cudaFreeAsync(buf, s);
    if (rc == WOB_OK && Q > 0) {
        // packed records and live bytes, then (sum, sum of squares) per split and query
        const int64_t R = n_paths * p.M;
        const int64_t q_blocks = (Q + kFwdThreads * kFwdQ - 1) / (kFwdThreads * kFwdQ);
        const int ppt = kFwdTile / p.M;
        int dev = 0, sms = 1, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fwd_connect, kFwdThreads,
                                                          0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        const int64_t slots = (int64_t)sms * per_sm;
        const int splits = fwd_splits(q_blocks, (n_paths + ppt - 1) / ppt, slots);
        const int64_t per_split = (n_paths + splits - 1) / splits;
        const size_t rec_bytes = ((size_t)R * sizeof(float4) + 255) & ~(size_t)255;
        const size_t live_bytes = ((size_t)n_paths + 255) & ~(size_t)255;
        char* cb = nullptr;
        WOB_CUDA_TRY(cudaMallocAsync((void**)&cb,
                                     rec_bytes + live_bytes + 2 * splits * Q * sizeof(double), s));
        float4* rec = (float4*)cb;
        uint8_t* live = (uint8_t*)(cb + rec_bytes);
        double* part = (double*)(cb + rec_bytes + live_bytes);
        k_fwd_pack<<<grid_for((const void*)k_fwd_pack, threads, 0, n_paths), threads, 0, s>>>(
            zpos, zw, n_paths, p.M, rec, live);
        const int64_t items = q_blocks * splits;
        k_fwd_connect<<<(int)(items < slots ? items : slots), kFwdThreads, 0, s>>>(
            queries, Q, rec, live, n_paths, p.M, q_blocks, splits, per_split, part);
        k_fwd_finish<<<grid_for((const void*)k_fwd_finish, 256, 0, Q), 256, 0, s>>>(
            part, splits, Q, n_paths, est, var, p.error_word);
        if (cudaGetLastError() != cudaSuccess) rc = WOB_ERR_CUDA;
        cudaFreeAsync(cb, s);
    }
    if (rc != WOB_OK) set_error("forward paths failed");
    return rc;
}

int launch_reduce(const double* per_walk, int64_t Q, int32_t N, double* est, double* var,
                  cudaStream_t s, const int* err)
{
    const int threads = 256;
    k_reduce<<<grid_for((const void*)k_reduce, threads, 0, Q * 32), threads, 0, s>>>(
        per_walk, Q, N, est, var, err);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int launch_reduce_part(const double* part, int64_t Q, int32_t N, int32_t tpq, double* est,
                       double* var, double* sum, double* sumsq, cudaStream_t s, const int* err)
{
    const int threads = 256;
    k_reduce_part<<<grid_for((const void*)k_reduce_part, threads, 0, Q * 32), threads, 0, s>>>(
        part, Q, N, tpq, est, var, sum, sumsq, err);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int launch_reduce_accum(const double* per_walk, int64_t Q, int32_t N, double* sum, double* sumsq,
                        cudaStream_t s, const int* err)
{
    const int threads = 256;
    k_reduce_accum<<<grid_for((const void*)k_reduce_accum, threads, 0, Q * 32), threads, 0, s>>>(
        per_walk, Q, N, sum, sumsq, err);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int launch_trace_lines(const BvhDev& b, const double* o, const double* d, const int32_t* exclude,
                       const uint32_t* keys, int64_t n, uint32_t key0, uint32_t key1, float tauL,
                       float edge_thr_L, int32_t* m, int32_t* sum_s, int32_t* prim,
                       int32_t* s_out, double* t, double* y, uint8_t* flag, int* error_word,
                       cudaStream_t s)
{
    const int threads = 128;
    k_trace_lines<<<grid_for((const void*)k_trace_lines, threads, 0, n), threads, 0, s>>>(
        b.wnodes, b.tv, b.inv_order, b.mesh->T, (int)(4 * b.n_wide + 64), o, d,
        exclude, keys, n, key0, key1, tauL,
        edge_thr_L, m, sum_s, prim, s_out, t, y, flag, error_word);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int launch_line_axes(uint32_t key0, uint32_t key1, const uint32_t* qws, int64_t n, double* d,
                     cudaStream_t s)
{
    const int threads = 256;
    k_line_axes<<<grid_for((const void*)k_line_axes, threads, 0, n), threads, 0, s>>>(key0, key1, qws, n, d);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

// Streaming read of n float4 (L1 bypassed), `passes` times; one atomic per
// warp keeps the loads.
__global__ void __launch_bounds__(256) k_probe_read(const float4* __restrict__ buf, int64_t n,
                                                    int passes, float* __restrict__ out)
{
    float acc = 0.f;
    for (int r = 0; r < passes; ++r)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const float4 v = __ldcg(buf + i);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

int launch_probe_read(const float4* buf, int64_t n, int passes, float* out, cudaStream_t s)
{
    WOB_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(float), s));
    const int grid = grid_for((const void*)k_probe_read, 256, 0, (int64_t)1 << 40);
    k_probe_read<<<grid, 256, 0, s>>>(buf, n, passes, out);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int launch_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out,
                  cudaStream_t s)
{
    const int threads = 256;
    k_philox<<<grid_for((const void*)k_philox, threads, 0, n), threads, 0, s>>>(ctr, key, n, out);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

}  // namespace wob
