// cv.cu -- the learned control variate: quadrature of its double-layer
// integrals and the residual walks.
//
// With nu = nu_t + rho (nu_t the network), rho solves rho = H rho + r with
//   r = 2 phi g - nu_t + H nu_t,   and   u(x0) = D nu_t(x0) + D rho(x0),
// where (H f)(x) = 2 phi int dG/dn_y f dA (Table 1, Dirichlet source density)
// and (D f)(x0) = -int dG/dn_y f dA (Eq. indirect_double_domain).  D nu_t and
// H nu_t are computed by quadrature (Radon's 7-point degree-5 rule on every
// triangle; triangles whose centroid lies closer than `near` times their
// longest edge to the target are split into 4^level sub-triangles with the
// same rule); H uses H[nu_t - nu_t(x)](x) - phi nu_t(x) (H[1] = -phi by
// Gauss) and skips the target's own flat triangle.  The walk is the
// double-layer recursion with r in place of 2 phi g.
//
// Residual walks run as a small wavefront per step: traverse + refine
// (one thread per walk), the network at every new vertex (batched on the
// tensor cores), then quadrature + accumulation (one thread per walk; the
// far-field loop over triangles is the same for every lane of a warp, so its
// node loads are broadcasts).
#include <array>
#include <climits>
#include <cmath>
#include <new>
#include <vector>

#include "wob_device.cuh"
#include "wob_host.h"

namespace wob {

namespace {

constexpr int kCoarse = 7;
constexpr int kMaxFine = 7 * 64;  // level <= 3
constexpr float kInvFourPi = 0.0795774715459476678f;

__constant__ float c_coarse_b[kCoarse * 3];
__constant__ float c_coarse_w[kCoarse];
__constant__ float c_fine_b[kMaxFine * 3];
__constant__ float c_fine_w[kMaxFine];

struct CvGeom {
    int T;
    int F;                       // fine nodes per triangle
    const float4* tri_c;         // centroid, near radius (near x longest edge)
    const float4* tri_p;         // unit normal n, plane offset n . y of the triangle
    const float* tri_a;          // area
    const float4* coarse_pk;     // T x 7: position, weight x node value (paired, k_cv_pack)
    const float4* fine_pk;       // T x F, the same layout
    const int* cand_off;         // per triangle: candidate near triangles
    const int* cand;
};

// Radon's rule (degree 5) in barycentric coordinates and its
// 4^level-subdivided version, computed once in double.
void rule_tables(int level, std::vector<float>& cb, std::vector<float>& cw,
                 std::vector<float>& fb, std::vector<float>& fw)
{
    const double s15 = std::sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, b1 = (9.0 + 2.0 * s15) / 21.0;
    const double a2 = (6.0 + s15) / 21.0, b2 = (9.0 - 2.0 * s15) / 21.0;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    const double P[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {b1, a1, a1}, {a1, b1, a1}, {a1, a1, b1},
                            {b2, a2, a2}, {a2, b2, a2}, {a2, a2, b2}};
    const double W[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
    cb.clear();
    cw.clear();
    for (int q = 0; q < 7; ++q) {
        for (int c = 0; c < 3; ++c) cb.push_back((float)P[q][c]);
        cw.push_back((float)W[q]);
    }
    // sub-triangles as barycentric corner triples
    std::vector<std::array<std::array<double, 3>, 3>> tris;
    tris.push_back({{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}});
    for (int l = 0; l < level; ++l) {
        std::vector<std::array<std::array<double, 3>, 3>> nxt;
        for (auto& T : tris) {
            std::array<double, 3> ab, bc, ca;
            for (int c = 0; c < 3; ++c) {
                ab[c] = 0.5 * (T[0][c] + T[1][c]);
                bc[c] = 0.5 * (T[1][c] + T[2][c]);
                ca[c] = 0.5 * (T[2][c] + T[0][c]);
            }
            nxt.push_back({{T[0], ab, ca}});
            nxt.push_back({{T[1], bc, ab}});
            nxt.push_back({{T[2], ca, bc}});
            nxt.push_back({{ab, bc, ca}});
        }
        tris = nxt;
    }
    fb.clear();
    fw.clear();
    for (auto& T : tris)
        for (int q = 0; q < 7; ++q) {
            for (int c = 0; c < 3; ++c)
                fb.push_back((float)(P[q][0] * T[0][c] + P[q][1] * T[1][c] + P[q][2] * T[2][c]));
            fw.push_back((float)(W[q] / tris.size()));
        }
}

__global__ void k_cv_nodes(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                           int T, int F, float near, float4* __restrict__ tri_c,
                           float4* __restrict__ tri_p, float* __restrict__ tri_R,
                           float* __restrict__ tri_a, float4* __restrict__ coarse,
                           float4* __restrict__ fine)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < T; j += gridDim.x * blockDim.x) {
        double v[3][3];
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < 3; ++c) v[k][c] = verts[3 * (int64_t)tris[3 * j + k] + c];
        double e1[3], e2[3], e3[3], cen[3];
        for (int c = 0; c < 3; ++c) {
            e1[c] = v[1][c] - v[0][c];
            e2[c] = v[2][c] - v[0][c];
            e3[c] = v[2][c] - v[1][c];
            cen[c] = (v[0][c] + v[1][c] + v[2][c]) / 3.0;
        }
        const double N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                             e1[0] * e2[1] - e1[1] * e2[0]};
        const double nl = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        const double area = 0.5 * nl;
        const double n[3] = {N[0] / nl, N[1] / nl, N[2] / nl};
        auto len = [](const double* e) { return sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]); };
        const double h = fmax(len(e1), fmax(len(e2), len(e3)));
        double R = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double d[3] = {v[k][0] - cen[0], v[k][1] - cen[1], v[k][2] - cen[2]};
            R = fmax(R, len(d));
        }
        tri_c[j] = make_float4((float)cen[0], (float)cen[1], (float)cen[2], (float)(near * h));
        tri_p[j] = make_float4((float)n[0], (float)n[1], (float)n[2],
                               (float)(n[0] * cen[0] + n[1] * cen[1] + n[2] * cen[2]));
        tri_R[j] = (float)R;
        tri_a[j] = (float)area;
        for (int q = 0; q < kCoarse; ++q) {
            double p[3];
            for (int c = 0; c < 3; ++c)
                p[c] = c_coarse_b[3 * q] * v[0][c] + c_coarse_b[3 * q + 1] * v[1][c] +
                       c_coarse_b[3 * q + 2] * v[2][c];
            coarse[kCoarse * j + q] = make_float4((float)p[0], (float)p[1], (float)p[2],
                                                  (float)(c_coarse_w[q] * area));
        }
        for (int q = 0; q < F; ++q) {
            double p[3];
            for (int c = 0; c < 3; ++c)
                p[c] = c_fine_b[3 * q] * v[0][c] + c_fine_b[3 * q + 1] * v[1][c] +
                       c_fine_b[3 * q + 2] * v[2][c];
            fine[(int64_t)F * j + q] = make_float4((float)p[0], (float)p[1], (float)p[2],
                                                   (float)(c_fine_w[q] * area));
        }
    }
}

// Packed nodes for the sums: position and weight x value, `per` nodes per
// triangle in the paired layout the sums read -- nodes 2i and 2i + 1 as
// (x, x', y, y'), (z, z', w, w'), an odd last node as (x, y, z, w) -- so
// that two nodes run as packed FP32x2 operations.
__global__ void k_cv_pack(const float4* __restrict__ nodes, const float* __restrict__ val,
                          int64_t n, int per, float4* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = nodes[i];
        const float w = a.w * val[i];
        const int64_t j = i / per;
        const int q = (int)(i - j * per);
        if (q < (per & ~1)) {
            float* e = reinterpret_cast<float*>(out + j * per) + 8 * (q >> 1) + (q & 1);
            e[0] = a.x;
            e[2] = a.y;
            e[4] = a.z;
            e[6] = w;
        } else {
            out[i] = make_float4(a.x, a.y, a.z, w);
        }
    }
}

// Candidates of triangle p: every j != p that can be near some point of p:
// |c_j - c_p| < near_j + R_p.  Pass 0 counts, pass 1 fills.
__global__ void k_cv_candidates(int T, const float4* __restrict__ tri_c,
                                const float* __restrict__ tri_R, const int* __restrict__ off,
                                int* __restrict__ count, int* __restrict__ cand, int pass)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < T; p += gridDim.x * blockDim.x) {
        const float4 cp = tri_c[p];
        const float Rp = tri_R[p];
        int n = 0;
        for (int j = 0; j < T; ++j) {
            if (j == p) continue;
            const float4 cj = tri_c[j];
            const float dx = cj.x - cp.x, dy = cj.y - cp.y, dz = cj.z - cp.z;
            const float lim = cj.w + Rp;
            if (dx * dx + dy * dy + dz * dz < lim * lim) {
                if (pass == 1) cand[(p == 0 ? 0 : off[p - 1]) + n] = j;
                ++n;
            }
        }
        if (pass == 0) count[p] = n;
    }
}

__device__ __forceinline__ bool is_near(float4 tc, float3 x)
{
    const float dx = tc.x - x.x, dy = tc.y - x.y, dz = tc.z - x.z;
    return dx * dx + dy * dy + dz * dz < tc.w * tc.w;
}

// One node: t = 1/r^3, r = |y - x|; s1 += (w f) t, s0 += omega t (omega: the
// rule weight without the triangle's area).
__device__ __forceinline__ void node_acc(float4 nd, float omega, float3 x, float& s1, float& s0)
{
    const float rx = nd.x - x.x, ry = nd.y - x.y, rz = nd.z - x.z;
    const float ri = rsqrt_ftz(fmaf(rx, rx, fmaf(ry, ry, rz * rz)));
    const float t = ri * ri * ri;
    s1 = fmaf(nd.w, t, s1);
    s0 = fmaf(omega, t, s0);
}

// node_acc for two nodes at once, stored as (x, x', y, y'), (z, z', w, w'):
// packed FP32x2 operations, every lane rounded as node_acc rounds it (r =
// node - x as node + (-x)).
static_assert(kCoarse % 2 == 1, "coarse nodes: pairs plus one");
struct NegPoint2 {
    float2 x, y, z;  // (-x, -x), ...
};

__device__ __forceinline__ void node_acc2(float4 a, float4 b, float2 omega, const NegPoint2& nx,
                                          float2& s1, float2& s0)
{
    const float2 rx = __fadd2_rn(make_float2(a.x, a.y), nx.x);
    const float2 ry = __fadd2_rn(make_float2(a.z, a.w), nx.y);
    const float2 rz = __fadd2_rn(make_float2(b.x, b.y), nx.z);
    const float2 r2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, __fmul2_rn(rz, rz)));
    const float2 ri = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
    const float2 t = __fmul2_rn(__fmul2_rn(ri, ri), ri);
    s1 = __ffma2_rn(make_float2(b.z, b.w), t, s1);
    s0 = __ffma2_rn(omega, t, s0);
}

// On the flat triangle j every node has the same r . n_j = d_j - x . n_j, so
//   sum_q w_q (r . n)/r^3 (f_q - fx) = (d_j - x . n_j) (S1 - fx area_j S0),
// S1 = sum_q (w_q f_q) / r_q^3, S0 = sum_q omega_q / r_q^3 (w_q = area_j omega_q).
__device__ __forceinline__ float tri_term(float4 tp, float area, float3 x, float fx, float s1,
                                          float s0)
{
    const float dot = tp.w - fmaf(x.x, tp.x, fmaf(x.y, tp.y, x.z * tp.z));
    return dot * fmaf(-fx * area, s0, s1);
}

// Far-field tile: kTileTris triangles (centroid + near radius, plane, area)
// and their packed coarse nodes (paired layout, see k_cv_pack), staged in
// shared memory by the whole block.
constexpr int kQuadThreads = 256;
constexpr int kTileTris = 64;
// Near-field stage: the fine nodes of up to kNearStage / F candidate
// triangles (at least one: F <= kMaxFine <= kNearStage).
constexpr int kNearStage = 512;
static_assert(kMaxFine <= kNearStage, "one triangle's fine nodes fit the stage");
struct FarTile {
    float4 tc[kTileTris];
    float4 tp[kTileTris];
    float ta[kTileTris];
    float4 node[kTileTris * kCoarse];
    float4 fine[kNearStage];
    int own0;
};

// Fine-node sum of triangle j (its 4^level sub-triangles) from its F nodes
// at nd: global memory (read-only path) or a block's shared-memory stage.
template <bool SHARED>
__device__ __forceinline__ float fine_sum(const CvGeom& c, const float4* nd, int j, float3 x,
                                          float fx)
{
    const NegPoint2 nx{make_float2(-x.x, -x.x), make_float2(-x.y, -x.y), make_float2(-x.z, -x.z)};
    float2 s1p = make_float2(0.f, 0.f), s0p = make_float2(0.f, 0.f);
    const int pairs = c.F >> 1;
#pragma unroll 4  // four pairs' loads in flight (the far loop unrolled too runs slower)
    for (int q = 0; q < pairs; ++q)
        node_acc2(SHARED ? nd[2 * q] : __ldg(nd + 2 * q), SHARED ? nd[2 * q + 1] : __ldg(nd + 2 * q + 1),
                  make_float2(c_fine_w[2 * q], c_fine_w[2 * q + 1]), nx, s1p, s0p);
    float s1 = s1p.x + s1p.y, s0 = s0p.x + s0p.y;
    if (c.F & 1) node_acc(SHARED ? nd[c.F - 1] : __ldg(nd + c.F - 1), c_fine_w[c.F - 1], x, s1, s0);
    return tri_term(__ldg(c.tri_p + j), __ldg(c.tri_a + j), x, fx, s1, s0);
}

__device__ __forceinline__ float fine_tri(const CvGeom& c, int j, float3 x, float fx)
{
    return fine_sum<false>(c, c.fine_pk + (int64_t)c.F * j, j, x, fx);
}

// sum over quadrature nodes of w (r . n)/(4 pi r^3) (f(y) - fx), r = y - x,
// i.e. -int dG/dn_y (f - fx) dA, skipping triangle `own` (-1: none).
// Called by EVERY thread of the block (the triangle tiles and the near
// field's fine nodes are loaded cooperatively); `own` must be negative for
// all threads of the block or for none.  The far field (coarse nodes of every triangle not near x) is an
// N-body sum over shared-memory tiles, FP32 within a tile and FP64 across
// tiles.  Near triangles (fine nodes): per lane from the candidate list of
// `own` when own >= 0; otherwise decided per triangle for the whole warp.
__device__ __forceinline__ float quad_sum(const CvGeom& c, FarTile& sm, float3 x, int own,
                                          float fx)
{
    double tot = 0.0;
    // the coarse weights of the node pairs and the negated query, in registers
    float2 om[(kCoarse - 1) / 2];
#pragma unroll
    for (int q = 0; q < (kCoarse - 1) / 2; ++q)
        om[q] = make_float2(c_coarse_w[2 * q], c_coarse_w[2 * q + 1]);
    const float om_last = c_coarse_w[kCoarse - 1];
    const NegPoint2 nx{make_float2(-x.x, -x.x), make_float2(-x.y, -x.y), make_float2(-x.z, -x.z)};
    for (int j0 = 0; j0 < c.T; j0 += kTileTris) {
        const int nt = min(kTileTris, c.T - j0);
        __syncthreads();  // the previous tile is no longer read
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            sm.tc[i] = __ldg(c.tri_c + j0 + i);
            sm.tp[i] = __ldg(c.tri_p + j0 + i);
            sm.ta[i] = __ldg(c.tri_a + j0 + i);
        }
        for (int i = threadIdx.x; i < nt * kCoarse; i += blockDim.x)
            sm.node[i] = __ldg(c.coarse_pk + (int64_t)kCoarse * j0 + i);
        __syncthreads();
        float part = 0.f;
        for (int jj = 0; jj < nt; ++jj) {
            const int j = j0 + jj;
            const bool near_me = is_near(sm.tc[jj], x);
            const float4* nb = sm.node + kCoarse * jj;
            float2 s1p = make_float2(0.f, 0.f), s0p = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < (kCoarse - 1) / 2; ++q)
                node_acc2(nb[2 * q], nb[2 * q + 1], om[q], nx, s1p, s0p);
            float s1 = s1p.x + s1p.y, s0 = s0p.x + s0p.y;
            node_acc(nb[kCoarse - 1], om_last, x, s1, s0);
            const float term = tri_term(sm.tp[jj], sm.ta[jj], x, fx, s1, s0);
            part += (j == own || near_me) ? 0.f : term;
            if (own < 0 && __any_sync(0xFFFFFFFFu, near_me)) {
                const float fterm = fine_tri(c, j, x, fx);
                part += near_me ? fterm : 0.f;
            }
        }
        tot += (double)part;
    }
    if (own >= 0) {
        float near_tot = 0.f;
        __syncthreads();  // the last far tile is no longer read
        if (threadIdx.x == 0) sm.own0 = own;
        __syncthreads();
        if (__syncthreads_and(own == sm.own0)) {
            // the whole block shares the triangle (the walks are bucketed by
            // it): its candidates' fine nodes are staged in shared memory,
            // chunk by chunk, and read by every lane as broadcasts; the
            // candidates are visited in the same order as below
            const int beg = own == 0 ? 0 : c.cand_off[own - 1], end = c.cand_off[own];
            const int per = kNearStage / c.F;
            for (int c0 = beg; c0 < end; c0 += per) {
                const int nt = min(per, end - c0);
                __syncthreads();  // the previous chunk is no longer read
                for (int i = threadIdx.x; i < nt * c.F; i += blockDim.x)
                    sm.fine[i] = __ldg(c.fine_pk + (int64_t)c.F * c.cand[c0 + i / c.F] + i % c.F);
                __syncthreads();
                for (int k = 0; k < nt; ++k) {
                    const int j = c.cand[c0 + k];
                    if (is_near(__ldg(c.tri_c + j), x))
                        near_tot += fine_sum<true>(c, sm.fine + k * c.F, j, x, fx);
                }
            }
        } else {
            for (int ci = own == 0 ? 0 : c.cand_off[own - 1]; ci < c.cand_off[own]; ++ci) {
                const int j = c.cand[ci];
                if (is_near(__ldg(c.tri_c + j), x)) near_tot += fine_tri(c, j, x, fx);
            }
        }
        tot += (double)near_tot;
    }
    return (float)(tot * (double)kInvFourPi);
}

// (D f)(x0) at points off the surface: -quad_sum(f) with f(x) = 0.
__global__ void __launch_bounds__(kQuadThreads, 4) k_cv_quad_D(CvGeom c, const float* __restrict__ x,
                                                           int64_t n, float* out)
{
    __shared__ FarTile sm;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < n;
        const float3 p = ok ? make_float3(x[3 * i], x[3 * i + 1], x[3 * i + 2])
                            : make_float3(0.f, 0.f, 0.f);
        const float v = quad_sum(c, sm, p, -1, 0.f);
        if (ok) out[i] = v;
    }
}

// (H f)(x) at points on triangles prims (original ids): 2 phi int dG/dn_y f
// = -2 phi quad_sum(f - f(x)) - phi f(x).
__global__ void __launch_bounds__(kQuadThreads) k_cv_quad_H(CvGeom c, int phi,
                                                           const float* __restrict__ x,
                                                           const int32_t* __restrict__ prims,
                                                           const float* __restrict__ fx,
                                                           int64_t n, float* out)
{
    __shared__ FarTile sm;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int own = i < n ? prims[i] : -1;
        const bool ok = i < n && own >= 0 && own < c.T;  // else: not a triangle of this mesh
        const float3 p = ok ? make_float3(x[3 * i], x[3 * i + 1], x[3 * i + 2])
                            : make_float3(0.f, 0.f, 0.f);
        const float f0 = ok ? fx[i] : 0.f;
        const float s = quad_sum(c, sm, p, ok ? own : 0, f0);
        if (i < n) out[i] = ok ? -2.f * (float)phi * s - (float)phi * f0 : __int_as_float(0x7FC00000);
    }
}

// ------------------------------------------------------------ residual walks
struct CvWalk {
    double* x;    // 3 x W
    double* S;    // walk sums = per-walk values
    double* P;
    int* self;    // leaf position of the current vertex (-1: off the surface)
    int* alive;   // 0 once a line missed
    float* vpos;  // 3 x W (contiguous per walk: x, y, z) for the network
    float* nut;   // network value at the current vertex
    int* own;     // triangle of the current vertex (original id; T once dead)
    int* perm;    // walks bucketed by `own` (the order k_cvw_accum visits them)
    int* count;   // T + 1 bucket sizes
    int* incl;    // their inclusive prefix sums
    int* cursor;  // scatter cursors
    int64_t W;
    int T;
};

__global__ void k_cvw_init(WalkParams p, CvWalk st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < st.W;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t qi = i / p.N;
        st.x[i] = p.queries[3 * qi];
        st.x[st.W + i] = p.queries[3 * qi + 1];
        st.x[2 * st.W + i] = p.queries[3 * qi + 2];
        st.S[i] = 0.0;
        st.P[i] = 1.0;
        st.self[i] = -1;
        st.alive[i] = 1;
        st.own[i] = st.T;
        st.vpos[3 * i] = p.queries[3 * qi];
        st.vpos[3 * i + 1] = p.queries[3 * qi + 1];
        st.vpos[3 * i + 2] = p.queries[3 * qi + 2];
    }
}

// Line of step k from the current vertex: traversal, pick, float-float
// refine (positions kept as doubles holding the float-float values) and the
// weight (first step (m/2)s, later -phi m s).
__global__ void __launch_bounds__(128, 4) k_cvw_trace(WalkParams p, CvWalk st, int k)
{
    const StreamKey key{p.key0, p.key1};
    int stack[kStackSize];
    int hits[kMaxHits];
    int err = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < st.W;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!st.alive[i]) continue;
        const int64_t qi = i / p.N;
        const uint32_t q = p.q_base + (uint32_t)qi;
        const uint32_t w = (uint32_t)(p.walk_begin + (i - qi * p.N));
        const ff x[3] = {ff_split(st.x[i]), ff_split(st.x[st.W + i]), ff_split(st.x[2 * st.W + i])};
        const int self = st.self[i];
        ff d[3];
        line_axis_ff(key, q, w, (uint32_t)k, d);
        const LinePre L = line_pre(make_float3(x[0].hi, x[1].hi, x[2].hi),
                                   make_float3(d[0].hi, d[1].hi, d[2].hi));
        const float Tthr = p.edge_thr_L * fabsf(L.Sz);
        Trav t;
        trav_init(t);
        uint32_t nn = 0, nt = 0;
        trace_wide<false, false>(p.nodes, p.tv, L, make_float3(0.f, 0.f, 0.f), Tthr, p.tauL,
                                 p.graze, self, t, hits, stack, key, q, w, (uint32_t)k, nn, nt,
                                 err, p.iter_limit);
        if (t.m == 0) {
            st.alive[i] = 0;
            st.own[i] = st.T;
            continue;
        }
        const int pos = select_hit(p.tv, t, hits, key, q, w, (uint32_t)k);
        ff y[3];
        const int sgn = refine_hit_ff(p.tv, pos, x, d, y);
        const double ms = (double)(t.m * sgn);
        st.P[i] = (k == 0) ? 0.5 * ms : st.P[i] * (-(double)p.phi * ms);
        st.x[i] = ff_join(y[0]);
        st.x[st.W + i] = ff_join(y[1]);
        st.x[2 * st.W + i] = ff_join(y[2]);
        st.vpos[3 * i] = y[0].hi;
        st.vpos[3 * i + 1] = y[1].hi;
        st.vpos[3 * i + 2] = y[2].hi;
        st.self[i] = pos;
        st.own[i] = (int)prim_of(p.tv, pos);
    }
    if (err) atomicOr(p.error_word, err);
}

// Bucket the walks by the triangle their vertex lies on (a counting sort;
// dead walks go to bucket T, last).  Walks of one bucket share the near-field
// candidate list, so a warp of them reads the same fine nodes.
__global__ void k_cvw_count(CvWalk st)
{
    // warp-uniform loop: every lane takes part in the match
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31;
         base < st.W; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + (threadIdx.x & 31);
        const int b = i < st.W ? st.own[i] : -1;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, b);
        if (b >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
            atomicAdd(st.count + b, __popc(peers));
    }
}

__global__ void k_cvw_cursor(CvWalk st)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= st.T; b += gridDim.x * blockDim.x)
        st.cursor[b] = st.incl[b] - st.count[b];
}

__global__ void k_cvw_scatter(CvWalk st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < st.W;
         i += (int64_t)gridDim.x * blockDim.x)
        st.perm[atomicAdd(st.cursor + st.own[i], 1)] = (int)i;
}

// Source r = 2 phi g - nu_t + H nu_t at the vertex reached at step k,
// halved on the last vertex (Sec. 4.1.2), times the weight product.
// 4 blocks of 256 per SM: 64 registers without spills (the compiler's own
// choice, 48 registers and 5 blocks, spilled and ran 2.4% slower).
__global__ void __launch_bounds__(kQuadThreads, 4) k_cvw_accum(WalkParams p, CvWalk st, CvGeom c,
                                                           int k)
{
    __shared__ FarTile sm;
    const double phi = (double)p.phi;
    const int64_t n_alive = st.T > 0 ? st.incl[st.T - 1] : 0;  // buckets 0..T-1
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n_alive;
         base += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = base + threadIdx.x < n_alive;
        const int64_t i = ok ? st.perm[base + threadIdx.x] : 0;
        const int pos = ok ? st.self[i] : 0;
        const float3 v = ok ? make_float3(st.vpos[3 * i], st.vpos[3 * i + 1], st.vpos[3 * i + 2])
                            : make_float3(0.f, 0.f, 0.f);
        const float fx = ok ? st.nut[i] : 0.f;
        const int own = ok ? (int)prim_of(p.tv, pos) : 0;
        const float h = -2.f * (float)p.phi * quad_sum(c, sm, v, own, fx) - (float)p.phi * fx;
        if (!ok) continue;
        const double3 y = make_double3(st.x[i], st.x[st.W + i], st.x[2 * st.W + i]);
        const double g = (double)dl_data(p.data, p.tv, pos, y);
        const double r = 2.0 * phi * g - (double)fx + (double)h;
        const double cw = (k == p.M - 1) ? 0.5 : 1.0;
        st.S[i] = fma(st.P[i] * cw, r, st.S[i]);
    }
}

// ------------------------------------------- Monte Carlo control variate
// D nu_t (x0) and H nu_t (x_i) as means of K one-line estimates (no
// quadrature: meshes of any size): K independent all-hits lines from the
// point, the pick y_j with the walk's own line weights -- (m/2) s from the
// query, -phi m s from a boundary vertex -- and nu_t(y_j) from the network.
// Extra line j of vertex v (0 = the query) draws from the stream
// (query, walk | 2^31, v K + j).
constexpr uint32_t kMcWalkBit = 0x80000000u;

struct CvMc {
    float* pos;  // W x K x 3: picks of the extra lines
    float* wgt;  // W x K: their weights (0: missed line, or the walk ended)
    float* nut;  // W x K: the network at the picks
    int K;
};

__global__ void __launch_bounds__(128, 4) k_cvmc_lines(WalkParams p, CvWalk st, CvMc mc, int v)
{
    const StreamKey key{p.key0, p.key1};
    int stack[kStackSize];
    int hits[kMaxHits];
    int err = 0;
    const int64_t n = st.W * mc.K;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / mc.K;
        const int j = (int)(t - i * mc.K);
        float* pp = mc.pos + 3 * t;
        if (!st.alive[i]) {
            mc.wgt[t] = 0.f;
            pp[0] = pp[1] = pp[2] = 0.f;
            continue;
        }
        const int64_t qi = i / p.N;
        const uint32_t q = p.q_base + (uint32_t)qi;
        const uint32_t w = (uint32_t)(p.walk_begin + (i - qi * p.N)) | kMcWalkBit;
        const uint32_t step = (uint32_t)(v * mc.K + j);
        const ff x[3] = {ff_split(st.x[i]), ff_split(st.x[st.W + i]), ff_split(st.x[2 * st.W + i])};
        ff d[3];
        line_axis_ff(key, q, w, step, d);
        const LinePre L = line_pre(make_float3(x[0].hi, x[1].hi, x[2].hi),
                                   make_float3(d[0].hi, d[1].hi, d[2].hi));
        const float Tthr = p.edge_thr_L * fabsf(L.Sz);
        Trav tr;
        trav_init(tr);
        uint32_t nn = 0, nt = 0;
        trace_wide<false, false>(p.nodes, p.tv, L, make_float3(0.f, 0.f, 0.f), Tthr, p.tauL,
                                 p.graze, st.self[i], tr, hits, stack, key, q, w, step, nn, nt,
                                 err, p.iter_limit);
        if (tr.m == 0) {
            mc.wgt[t] = 0.f;
            pp[0] = pp[1] = pp[2] = 0.f;
            continue;
        }
        const int pos = select_hit(p.tv, tr, hits, key, q, w, step);
        ff y[3];
        const float ms = (float)(tr.m * refine_hit_ff(p.tv, pos, x, d, y));
        mc.wgt[t] = v == 0 ? 0.5f * ms : -(float)p.phi * ms;
        pp[0] = y[0].hi;
        pp[1] = y[1].hi;
        pp[2] = y[2].hi;
    }
    if (err) atomicOr(p.error_word, err);
}

// k < 0: S = D^ nu_t (x0), the walk's start value.  k >= 0: the source
// r^ = 2 phi g - nu_t + H^ nu_t at the vertex reached at step k, halved on
// the last vertex (Sec. 4.1.2), times the weight product.
__global__ void k_cvmc_accum(WalkParams p, CvWalk st, CvMc mc, int k)
{
    const double phi = (double)p.phi;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < st.W;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (k >= 0 && !st.alive[i]) continue;
        double acc = 0.0;
        for (int j = 0; j < mc.K; ++j)
            acc += (double)mc.wgt[i * mc.K + j] * (double)mc.nut[i * mc.K + j];
        acc /= (double)mc.K;
        if (k < 0) {
            st.S[i] = acc;
            continue;
        }
        const double3 y = make_double3(st.x[i], st.x[st.W + i], st.x[2 * st.W + i]);
        const double g = (double)dl_data(p.data, p.tv, st.self[i], y);
        const double r = 2.0 * phi * g - (double)st.nut[i] + acc;
        const double cw = (k == p.M - 1) ? 0.5 : 1.0;
        st.S[i] = fma(st.P[i] * cw, r, st.S[i]);
    }
}

// Area-uniform boundary points: point i is the area sample of the stream
// (query i, walk 0, step 0) -- triangle by inverse CDF of the areas, then a
// square-root-warped uniform point on it -- the same draw the single-layer
// walks make at their vertices.
__global__ void k_sample_boundary(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                                  const double* __restrict__ cdf, int64_t T, double area,
                                  uint32_t key0, uint32_t key1, int64_t n, float* __restrict__ pts,
                                  int32_t* __restrict__ prims)
{
    const StreamKey key{key0, key1};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const u32x4 u = stream_block(key, (uint32_t)i, 0u, 0u, kPurposeArea, 0u, 0u);
        const double target = u53(u.x, u.y) * area;
        int64_t lo = 0, hi = T - 1;
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (__ldg(cdf + mid) > target) hi = mid; else lo = mid + 1;
        }
        const double su = sqrt(u24(u.z)), u2 = u24(u.w);
        const double b0 = 1.0 - su, b1 = su * (1.0 - u2), b2 = su * u2;
        const int32_t* t = tris + 3 * lo;
        const float* v0 = verts + 3 * (int64_t)__ldg(t);
        const float* v1 = verts + 3 * (int64_t)__ldg(t + 1);
        const float* v2 = verts + 3 * (int64_t)__ldg(t + 2);
        for (int c = 0; c < 3; ++c)
            pts[3 * i + c] = (float)(b0 * __ldg(v0 + c) + b1 * __ldg(v1 + c) + b2 * __ldg(v2 + c));
        prims[i] = (int32_t)lo;
    }
}

__global__ void k_to_float(const double* __restrict__ in, int64_t n, float* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

int sample_boundary(const MeshDev& m, int64_t n, uint64_t seed, uint32_t problem, float* pts,
                    int32_t* prims, cudaStream_t s)
{
    if (n <= 0) return WOB_OK;
    const int grid = grid_for((const void*)k_sample_boundary, 128, 0, n);
    k_sample_boundary<<<grid, 128, 0, s>>>(m.verts, m.tris, m.cdf, m.T, m.area,
                                            (uint32_t)seed ^ problem, (uint32_t)(seed >> 32), n,
                                            pts, prims);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

}  // namespace
}  // namespace wob

using namespace wob;

struct wob_cv_s {
    const MeshDev* mesh = nullptr;
    int T = 0, F = 0, level = 2;
    float near = 2.f;
    float4 *tri_c = nullptr, *tri_p = nullptr, *coarse = nullptr, *fine = nullptr;
    float4 *coarse_pk = nullptr, *fine_pk = nullptr;
    float *tri_R = nullptr, *tri_a = nullptr, *coarse_val = nullptr, *fine_val = nullptr;
    int *cand_off = nullptr, *cand = nullptr;
    int64_t n_cand = 0;
    CvGeom geom() const
    {
        return CvGeom{T, F, tri_c, tri_p, tri_a, coarse_pk, fine_pk, cand_off, cand};
    }
};

namespace {

void free_cv(wob_cv_s* c)
{
    for (void* p : {(void*)c->tri_c, (void*)c->tri_p, (void*)c->tri_R, (void*)c->tri_a,
                    (void*)c->coarse, (void*)c->fine, (void*)c->coarse_pk, (void*)c->fine_pk,
                    (void*)c->coarse_val, (void*)c->fine_val, (void*)c->cand_off, (void*)c->cand})
        if (p) cudaFree(p);
}

// Packed nodes from the current node values.
int pack_nodes(wob_cv_s* c, cudaStream_t s)
{
    const int64_t nc = (int64_t)c->T * kCoarse, nf = (int64_t)c->T * c->F;
    k_cv_pack<<<grid_for((const void*)k_cv_pack, 256, 0, nc), 256, 0, s>>>(
        c->coarse, c->coarse_val, nc, kCoarse, c->coarse_pk);
    k_cv_pack<<<grid_for((const void*)k_cv_pack, 256, 0, nf), 256, 0, s>>>(
        c->fine, c->fine_val, nf, c->F, c->fine_pk);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

}  // namespace

extern "C" {

int wob_cv_create(wob_mesh m, int32_t level, float near, void* stream, wob_cv* out)
{
    clear_error();
    if (!m || !out || level < 0 || level > 3 || !(near > 0.f)) {
        set_error("wob_cv_create: invalid arguments (level 0..3, near > 0)");
        return WOB_ERR_INVALID_ARG;
    }
    if (m->d.T > (1 << 20)) {
        set_error("wob_cv_create: the control variate's quadrature supports up to 2^20 triangles");
        return WOB_ERR_UNSUPPORTED;
    }
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    wob_cv_s* c = new (std::nothrow) wob_cv_s();
    if (!c) return WOB_ERR_OOM;
    c->mesh = &m->d;
    c->T = (int)m->d.T;
    c->level = level;
    c->near = near;
    c->F = 7 << (2 * level);
    std::vector<float> cb, cw, fb, fw;
    rule_tables(level, cb, cw, fb, fw);
    auto fail = [&](int code, const char* msg) {
        set_error("wob_cv_create: %s", msg);
        cudaStreamSynchronize(s);
        free_cv(c);
        delete c;
        return code;
    };
    if (cudaMemcpyToSymbolAsync(c_coarse_b, cb.data(), cb.size() * 4, 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_coarse_w, cw.data(), cw.size() * 4, 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_fine_b, fb.data(), fb.size() * 4, 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(c_fine_w, fw.data(), fw.size() * 4, 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(WOB_ERR_CUDA, "rule upload failed");
    const int T = c->T;
    if (cudaMalloc((void**)&c->tri_c, T * sizeof(float4)) != cudaSuccess ||
        cudaMalloc((void**)&c->tri_p, T * sizeof(float4)) != cudaSuccess ||
        cudaMalloc((void**)&c->tri_R, T * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&c->tri_a, T * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&c->coarse, (size_t)T * kCoarse * sizeof(float4)) != cudaSuccess ||
        cudaMalloc((void**)&c->fine, (size_t)T * c->F * sizeof(float4)) != cudaSuccess ||
        cudaMalloc((void**)&c->coarse_pk, (size_t)T * kCoarse * sizeof(float4)) != cudaSuccess ||
        cudaMalloc((void**)&c->fine_pk, (size_t)T * c->F * sizeof(float4)) != cudaSuccess ||
        cudaMalloc((void**)&c->coarse_val, (size_t)T * kCoarse * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&c->fine_val, (size_t)T * c->F * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&c->cand_off, T * sizeof(int)) != cudaSuccess)
        return fail(WOB_ERR_OOM, "device allocation failed");
    cudaMemsetAsync(c->coarse_val, 0, (size_t)T * kCoarse * sizeof(float), s);
    cudaMemsetAsync(c->fine_val, 0, (size_t)T * c->F * sizeof(float), s);
    const int threads = 128;
    const int grid = grid_for((const void*)k_cv_nodes, threads, 0, T);
    k_cv_nodes<<<grid, threads, 0, s>>>(m->d.verts, m->d.tris, T, c->F, near, c->tri_c, c->tri_p,
                                        c->tri_R, c->tri_a, c->coarse, c->fine);
    if (pack_nodes(c, s) != WOB_OK) return fail(WOB_ERR_CUDA, "node setup failed");
    int* count = nullptr;
    if (cudaMallocAsync((void**)&count, T * sizeof(int), s) != cudaSuccess)
        return fail(WOB_ERR_OOM, "device allocation failed");
    k_cv_candidates<<<grid, threads, 0, s>>>(T, c->tri_c, c->tri_R, nullptr, count, nullptr, 0);
    int rc = inclusive_scan<int>(count, c->cand_off, T, s);
    int total = 0;
    cudaMemcpyAsync(&total, c->cand_off + T - 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(count, s);
    if (rc != WOB_OK || cudaStreamSynchronize(s) != cudaSuccess) return fail(WOB_ERR_CUDA, "node setup failed");
    c->n_cand = total;
    if (cudaMalloc((void**)&c->cand, (size_t)(total > 0 ? total : 1) * sizeof(int)) != cudaSuccess)
        return fail(WOB_ERR_OOM, "device allocation failed");
    k_cv_candidates<<<grid, threads, 0, s>>>(T, c->tri_c, c->tri_R, c->cand_off, nullptr, c->cand, 1);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return fail(WOB_ERR_CUDA, "candidate lists failed");
    *out = c;
    return WOB_OK;
}

int wob_cv_set_network(wob_cv c, const float* params, void* stream)
{
    clear_error();
    if (!c || !params) {
        set_error("NULL argument");
        return WOB_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    WOB_TRY(mlp_forward(params, (const float*)c->coarse, (int64_t)c->T * kCoarse, c->coarse_val, s, 4));
    WOB_TRY(mlp_forward(params, (const float*)c->fine, (int64_t)c->T * c->F, c->fine_val, s, 4));
    return pack_nodes(c, s);
}

int wob_cv_set_node_values(wob_cv c, const float* coarse, const float* fine, void* stream)
{
    clear_error();
    if (!c || !coarse || !fine) {
        set_error("NULL argument");
        return WOB_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    WOB_CUDA_TRY(cudaMemcpyAsync(c->coarse_val, coarse, (size_t)c->T * kCoarse * 4, cudaMemcpyDeviceToDevice, s));
    WOB_CUDA_TRY(cudaMemcpyAsync(c->fine_val, fine, (size_t)c->T * c->F * 4, cudaMemcpyDeviceToDevice, s));
    return pack_nodes(c, s);
}

int wob_cv_get_nodes(wob_cv c, float* coarse_out, float* fine_out, void* stream)
{
    clear_error();
    if (!c || !coarse_out || !fine_out) {
        set_error("NULL argument");
        return WOB_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    WOB_CUDA_TRY(cudaMemcpyAsync(coarse_out, c->coarse, (size_t)c->T * kCoarse * sizeof(float4),
                                 cudaMemcpyDeviceToDevice, s));
    WOB_CUDA_TRY(cudaMemcpyAsync(fine_out, c->fine, (size_t)c->T * c->F * sizeof(float4),
                                 cudaMemcpyDeviceToDevice, s));
    return WOB_OK;
}

int wob_cv_quad_D(wob_cv c, const float* points, int64_t n, float* out, void* stream)
{
    clear_error();
    if (!c || n < 0 || (n > 0 && (!points || !out))) {
        set_error("wob_cv_quad_D: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    if (n == 0) return WOB_OK;
    const int grid = grid_for((const void*)k_cv_quad_D, kQuadThreads, 0, n);
    k_cv_quad_D<<<grid, kQuadThreads, 0, (cudaStream_t)stream>>>(c->geom(), points, n, out);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int wob_cv_quad_H(wob_cv c, int32_t phi, const float* points, const int32_t* prims,
                  const float* fx, int64_t n, float* out, void* stream)
{
    clear_error();
    if (!c || (phi != 1 && phi != -1) || n < 0 || (n > 0 && (!points || !prims || !fx || !out))) {
        set_error("wob_cv_quad_H: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    if (n == 0) return WOB_OK;
    const int grid = grid_for((const void*)k_cv_quad_H, kQuadThreads, 0, n);
    k_cv_quad_H<<<grid, kQuadThreads, 0, (cudaStream_t)stream>>>(c->geom(), phi, points, prims, fx, n, out);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

int wob_cv_solve(const wob_problem* prob, wob_cv c, const float* params, const float* queries,
                 int64_t Q, int64_t walk_begin, int32_t walks, int32_t max_len, uint64_t seed,
                 double* sum, double* sumsq, double* per_walk, float* dnt, void* stream)
{
    clear_error();
    if (!c || !params || (Q > 0 && (!queries || !sum || !sumsq))) {
        set_error("wob_cv_solve: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    WOB_TRY(check_problem(prob));
    WOB_TRY(check_sizes(Q, walk_begin, walks, max_len));
    if (prob->kind != WOB_DIRICHLET_DL || prob->bvh->d.mesh != c->mesh) {
        set_error("wob_cv_solve: needs WOB_DIRICHLET_DL on the control variate's mesh");
        return WOB_ERR_UNSUPPORTED;
    }
    if (Q == 0) return WOB_OK;
    if (Q * (int64_t)walks > INT32_MAX) {
        set_error("wob_cv_solve: Q x walks must be below 2^31 per call");
        return WOB_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    WalkParams p;
    fill_params(p, prob, queries, nullptr, Q, walk_begin, walks, max_len, seed);
    CvWalk st;
    st.W = Q * (int64_t)walks;
    st.T = c->T;
    const size_t W = (size_t)st.W;
    const size_t nb = (size_t)c->T + 1;
    char* buf = nullptr;
    const size_t bytes = W * (8 * 5 + 4 * 2 + 4 * 4 + 4 * 2) + nb * 12 + 256;
    WOB_CUDA_TRY(cudaMallocAsync((void**)&buf, bytes, s));
    st.x = (double*)buf;
    st.S = st.x + 3 * W;
    st.P = st.S + W;
    st.self = (int*)(st.P + W);
    st.alive = st.self + W;
    st.vpos = (float*)(st.alive + W);
    st.nut = st.vpos + 3 * W;
    st.own = (int*)(st.nut + W);
    st.perm = st.own + W;
    st.count = st.perm + W;
    st.incl = st.count + nb;
    st.cursor = st.incl + nb;
    int* err = st.cursor + nb;
    int rc = WOB_OK;
    cudaMemsetAsync(err, 0, sizeof(int), s);
    p.error_word = err;
    const CvGeom g = c->geom();
    const int threads = 128;
    k_cvw_init<<<grid_for((const void*)k_cvw_init, threads, 0, st.W), threads, 0, s>>>(p, st);
    const int g_trace = grid_for((const void*)k_cvw_trace, threads, 0, st.W);
    const int g_acc = grid_for((const void*)k_cvw_accum, kQuadThreads, 0, st.W);
    const int g_walk = grid_for((const void*)k_cvw_count, 256, 0, st.W);
    const int g_buck = grid_for((const void*)k_cvw_cursor, 256, 0, (int64_t)nb);
    for (int k = 0; k < max_len && rc == WOB_OK; ++k) {
        k_cvw_trace<<<g_trace, threads, 0, s>>>(p, st, k);
        rc = mlp_forward(params, st.vpos, st.W, st.nut, s, 3);
        if (rc != WOB_OK) break;
        cudaMemsetAsync(st.count, 0, nb * sizeof(int), s);
        k_cvw_count<<<g_walk, 256, 0, s>>>(st);
        rc = inclusive_scan<int>(st.count, st.incl, (int64_t)nb, s);
        if (rc != WOB_OK) break;
        k_cvw_cursor<<<g_buck, 256, 0, s>>>(st);
        k_cvw_scatter<<<g_walk, 256, 0, s>>>(st);
        k_cvw_accum<<<g_acc, kQuadThreads, 0, s>>>(p, st, g, k);
    }
    if (rc == WOB_OK && cudaGetLastError() != cudaSuccess) rc = WOB_ERR_CUDA;
    if (rc == WOB_OK) rc = launch_reduce_accum(st.S, Q, walks, sum, sumsq, s, err);
    if (rc == WOB_OK && per_walk)
        if (cudaMemcpyAsync(per_walk, st.S, W * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            rc = WOB_ERR_CUDA;
    if (rc == WOB_OK && dnt) {
        const int grid = grid_for((const void*)k_cv_quad_D, kQuadThreads, 0, Q);
        k_cv_quad_D<<<grid, kQuadThreads, 0, s>>>(g, queries, Q, dnt);
        if (cudaGetLastError() != cudaSuccess) rc = WOB_ERR_CUDA;
    }
    cudaFreeAsync(buf, s);
    if (rc != WOB_OK) set_error("wob_cv_solve failed");
    return rc;
}

int wob_cv_solve_mc(const wob_problem* prob, const float* params, const float* queries, int64_t Q,
                    int64_t walk_begin, int32_t walks, int32_t max_len, int32_t K, uint64_t seed,
                    double* sum, double* sumsq, double* per_walk, void* stream)
{
    clear_error();
    if (!params || (Q > 0 && (!queries || !sum || !sumsq))) {
        set_error("wob_cv_solve_mc: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    WOB_TRY(check_problem(prob));
    WOB_TRY(check_sizes(Q, walk_begin, walks, max_len));
    if (prob->kind != WOB_DIRICHLET_DL) {
        set_error("wob_cv_solve_mc: needs WOB_DIRICHLET_DL");
        return WOB_ERR_UNSUPPORTED;
    }
    if (K < 1 || K > 16 || max_len > 1024 || walk_begin + walks > (int64_t)kMcWalkBit) {
        set_error("wob_cv_solve_mc: 1 <= K <= 16, max_len <= 1024, walk indices below 2^31");
        return WOB_ERR_INVALID_ARG;
    }
    if (Q == 0) return WOB_OK;
    if (Q * (int64_t)walks * K > INT32_MAX) {
        set_error("wob_cv_solve_mc: Q x walks x K must be below 2^31 per call");
        return WOB_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    WalkParams p;
    fill_params(p, prob, queries, nullptr, Q, walk_begin, walks, max_len, seed);
    CvWalk st{};
    st.W = Q * (int64_t)walks;
    st.T = (int)p.T;
    const size_t W = (size_t)st.W, WK = W * (size_t)K;
    char* buf = nullptr;
    const size_t bytes = W * (8 * 5 + 4 * 2 + 4 * 4 + 4) + WK * 4 * 5 + 256;
    WOB_CUDA_TRY(cudaMallocAsync((void**)&buf, bytes, s));
    st.x = (double*)buf;
    st.S = st.x + 3 * W;
    st.P = st.S + W;
    st.self = (int*)(st.P + W);
    st.alive = st.self + W;
    st.vpos = (float*)(st.alive + W);
    st.nut = st.vpos + 3 * W;
    st.own = (int*)(st.nut + W);
    CvMc mc;
    mc.pos = (float*)(st.own + W);
    mc.wgt = mc.pos + 3 * WK;
    mc.nut = mc.wgt + WK;
    mc.K = K;
    int* err = (int*)(mc.nut + WK);
    int rc = WOB_OK;
    cudaMemsetAsync(err, 0, sizeof(int), s);
    p.error_word = err;
    const int threads = 128;
    k_cvw_init<<<grid_for((const void*)k_cvw_init, threads, 0, st.W), threads, 0, s>>>(p, st);
    const int g_trace = grid_for((const void*)k_cvw_trace, threads, 0, st.W);
    const int g_lines = grid_for((const void*)k_cvmc_lines, threads, 0, (int64_t)WK);
    const int g_acc = grid_for((const void*)k_cvmc_accum, threads, 0, st.W);
    // D^ nu_t at the queries
    k_cvmc_lines<<<g_lines, threads, 0, s>>>(p, st, mc, 0);
    rc = mlp_forward(params, mc.pos, (int64_t)WK, mc.nut, s, 3);
    if (rc == WOB_OK) k_cvmc_accum<<<g_acc, threads, 0, s>>>(p, st, mc, -1);
    for (int k = 0; k < max_len && rc == WOB_OK; ++k) {
        k_cvw_trace<<<g_trace, threads, 0, s>>>(p, st, k);
        rc = mlp_forward(params, st.vpos, st.W, st.nut, s, 3);
        if (rc != WOB_OK) break;
        k_cvmc_lines<<<g_lines, threads, 0, s>>>(p, st, mc, k + 1);
        rc = mlp_forward(params, mc.pos, (int64_t)WK, mc.nut, s, 3);
        if (rc != WOB_OK) break;
        k_cvmc_accum<<<g_acc, threads, 0, s>>>(p, st, mc, k);
    }
    if (rc == WOB_OK && cudaGetLastError() != cudaSuccess) rc = WOB_ERR_CUDA;
    if (rc == WOB_OK) rc = launch_reduce_accum(st.S, Q, walks, sum, sumsq, s, err);
    if (rc == WOB_OK && per_walk)
        if (cudaMemcpyAsync(per_walk, st.S, W * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            rc = WOB_ERR_CUDA;
    cudaFreeAsync(buf, s);
    if (rc != WOB_OK) set_error("wob_cv_solve_mc failed");
    return rc;
}

int wob_sample_boundary(wob_mesh m, int64_t n, uint64_t seed, uint32_t problem, float* points,
                        int32_t* prims, void* stream)
{
    clear_error();
    if (!m || n < 0 || n > INT32_MAX || (n > 0 && (!points || !prims))) {
        set_error("wob_sample_boundary: invalid arguments (0 <= n < 2^31)");
        return WOB_ERR_INVALID_ARG;
    }
    return sample_boundary(m->d, n, seed, problem, points, prims, (cudaStream_t)stream);
}

int wob_cv_train(const wob_problem* prob, wob_cv c, const wob_cv_train_params* tp,
                 float* params, float* adam_m, float* adam_v, float* loss_out, void* stream)
{
    clear_error();
    if (!c || !tp || !params || !adam_m || !adam_v || tp->points < 1 || tp->points > INT32_MAX ||
        tp->walks < 2 || tp->max_len < 1 || tp->max_len > kMaxLen || tp->epochs < 0 ||
        tp->batch < 1 || tp->batch > (1 << 22) || !(tp->lr >= 0.f) || !(tp->lr_end >= 0.f) ||
        tp->tail_epochs < 0 || tp->step0 < 0) {
        set_error("wob_cv_train: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    WOB_TRY(check_problem(prob));
    if (prob->kind != WOB_DIRICHLET_DL || prob->bvh->d.mesh != c->mesh) {
        set_error("wob_cv_train: needs WOB_DIRICHLET_DL on the control variate's mesh");
        return WOB_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = tp->points;
    const int64_t b = tp->batch < n ? tp->batch : n;
    const int64_t steps = (n + b - 1) / b;
    const int64_t ws_floats = mlp_train_workspace(b);
    // one allocation: points (3n f32), prims (n i32), est / var (2n f64), targets (n f32), ws,
    // the training control word and one epoch's losses
    const size_t bytes =
        (size_t)n * (12 + 4 + 16 + 4) + (size_t)(ws_floats + 2 + steps) * 4 + 256;
    char* buf = nullptr;
    WOB_CUDA_TRY(cudaMallocAsync((void**)&buf, bytes, s));
    double* est = (double*)buf;
    double* var = est + n;
    float* pts = (float*)(var + n);
    float* targets = pts + 3 * n;
    int32_t* prims = (int32_t*)(targets + n);
    float* ws = (float*)(prims + n);
    int rc = sample_boundary(*c->mesh, n, tp->point_seed, prob->problem, pts, prims, s);
    if (rc == WOB_OK)
        rc = wob_solve_density(prob, pts, prims, n, tp->walks, tp->max_len, tp->walk_seed, est, var,
                               stream);
    if (rc == WOB_OK) {
        k_to_float<<<grid_for((const void*)k_to_float, 256, 0, n), 256, 0, s>>>(est, n, targets);
        if (cudaGetLastError() != cudaSuccess) rc = WOB_ERR_CUDA;
    }
    // One epoch (every minibatch: training kernel, Adam, loss) is captured
    // once as a CUDA graph on a private stream and replayed per epoch on the
    // caller's stream: the step number and learning rate live in device
    // memory (TrainCtl: the training kernel advances the step, Adam reads
    // it), the epoch's losses in a scratch row copied out after each
    // replay.  The same kernels as unrolled launches.
    // step schedule: the last tail_epochs epochs run at lr_end
    auto epoch_lr = [&](int e) { return e >= tp->epochs - tp->tail_epochs ? tp->lr_end : tp->lr; };
    TrainCtl* ctl = reinterpret_cast<TrainCtl*>(ws + ws_floats);
    float* lrow = ws + ws_floats + 2;
    if (rc == WOB_OK && tp->epochs > 0) {
        rc = mlp_train_prepare();
        if (rc == WOB_OK) rc = train_ctl_set(ctl, tp->step0, epoch_lr(0), true, s);
    }
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (rc == WOB_OK && tp->epochs > 0) {
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) rc = WOB_ERR_CUDA;
        if (rc == WOB_OK &&
            cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            rc = WOB_ERR_CUDA;
        if (rc == WOB_OK) {
            for (int64_t j = 0; j < steps && rc == WOB_OK; ++j) {
                const int64_t r0 = j * b, nb = (r0 + b <= n) ? b : n - r0;
                rc = mlp_train_step_ws(params, adam_m, adam_v, pts + 3 * r0, targets + r0, nb, 0.f,
                                       0, nullptr, lrow + j, ws, cs, ctl);
            }
            const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
            if (rc == WOB_OK && (ce != cudaSuccess ||
                                 cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess))
                rc = WOB_ERR_CUDA;
        }
        for (int e = 0; e < tp->epochs && rc == WOB_OK; ++e) {
            if (e > 0 && epoch_lr(e) != epoch_lr(e - 1))
                rc = train_ctl_set(ctl, 0, epoch_lr(e), false, s);
            if (rc == WOB_OK && cudaGraphLaunch(exec, s) != cudaSuccess) rc = WOB_ERR_CUDA;
            if (rc == WOB_OK && loss_out &&
                cudaMemcpyAsync(loss_out + (int64_t)e * steps, lrow, steps * sizeof(float),
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                rc = WOB_ERR_CUDA;
        }
        if (rc == WOB_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = WOB_ERR_CUDA;
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        if (rc != WOB_OK && wob_last_error()[0] == 0)
            set_error("wob_cv_train: training graph failed (%s)", cudaGetErrorString(cudaGetLastError()));
    }
    if (rc == WOB_OK) rc = wob_cv_set_network(c, params, stream);
    cudaFreeAsync(buf, s);
    if (rc != WOB_OK && wob_last_error()[0] == 0) set_error("wob_cv_train failed");
    return rc;
}

int wob_cv_get_info(wob_cv c, int32_t* T, int32_t* F, int64_t* candidates)
{
    clear_error();
    if (!c) {
        set_error("NULL argument");
        return WOB_ERR_INVALID_ARG;
    }
    if (T) *T = c->T;
    if (F) *F = c->F;
    if (candidates) *candidates = c->n_cand;
    return WOB_OK;
}

void wob_cv_destroy(wob_cv c)
{
    if (!c) return;
    free_cv(c);
    delete c;
}

}  // extern "C"
