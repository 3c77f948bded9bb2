// wob_internal.h -- library-internal constants, handle layouts and the
// launch parameter blocks shared by the host code and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "wob.h"

namespace wob {

constexpr uint32_t kPurposeDir = 0;   // line axis draws
constexpr uint32_t kPurposeHit = 1;   // hit-selection keys
constexpr uint32_t kPurposeArea = 2;  // area-sampled boundary points
constexpr uint32_t kPurposeInit = 3;  // initial network weights
constexpr uint32_t kPurposeBranch = 4;  // move / stay on Dirichlet parts of mixed problems
constexpr uint32_t kPurposeRis = 5;     // resampled importance sampling pick
constexpr int kMaxRis = 64;             // candidates of one resampling
constexpr int kStackSize = 64;        // traversal stack entries per line
constexpr int kNoRef = INT32_MIN;     // empty traversal stack marker
constexpr int64_t kMaxTriangles = (int64_t(1) << 28) - 2;
constexpr float kDefaultTau = 2e-6f;
constexpr float kGraze = 1e-4f;
// The line-triangle test flags a line within kFlagMargin tau L of an edge,
// or with a hit at |t| < kFlagMargin tau L (the oracle flags within tau L;
// the margin covers the FP32 rounding of the line's origin and axis, so that
// every line the oracle flags is flagged),
// and recomputes the edge functions of a triangle in their canonical form
// when one is below kRareMargin times that distance (scaled by the longest
// edge): a bound above the main path's rounding error.
constexpr float kFlagMargin = 1.25f;
constexpr float kRareMargin = 1.5f;
constexpr int kMaxLen = 4096;
// Box padding in units of the mesh diagonal L: above the slab test's
// rounding (at most 1.53e-5 of a node's extent, see dequant).
constexpr double kBoxPad = 2e-5;

// Per-triangle unit normal and area, FP64 (32 bytes, read as two 16-byte loads).
struct alignas(32) NormalArea {
    double nx, ny, nz, area;
};

// Per-triangle frame for area samples in compensated FP32 (original order):
// vertex v0 and, as pairs hi + lo of FP32 values whose sum is the FP64
// value, the edges e1 = v1 - v0 and e2 = v2 - v0 (exact: differences of FP32
// coordinates) and the unit normal; 96 bytes, read as six float4.
struct alignas(16) TriFrame {
    float v0[3];
    float e1h[3], e1l[3];
    float e2h[3], e2l[3];
    float nh[3], nl[3];
    float pad[3];
};
static_assert(sizeof(TriFrame) == 96, "six float4");

struct MeshDev {
    float* verts = nullptr;   // V x 3
    double* verts_d = nullptr;  // V x 3, the same positions in FP64 (resampled area samples)
    int32_t* tris = nullptr;  // T x 3
    NormalArea* tri_n = nullptr;  // unit normal (FP64), area
    TriFrame* tri_f = nullptr;    // compensated FP32 frame of each triangle
    double* cdf = nullptr;    // inclusive prefix sums of areas
    int32_t* guide = nullptr; // guide table of the area CDF: 2^guide_bits + 1 entries
    int guide_bits = 0;
    int64_t V = 0, T = 0;
    double lo[3], hi[3];
    double L = 0, area = 0, volume = 0, max_edge = 0;
    int device = 0;
};

struct BvhDev {
    float4* nodes = nullptr;  // 4 float4 per interior node
    float4* wnodes = nullptr; // 8-wide nodes, 6 float4 each (collapsed from `nodes`)
    int64_t n_wide = 0;
    int wide_levels = 0;
    float4* tv = nullptr;     // 3 float4 per triangle, leaf order
    int32_t* order = nullptr; // leaf order -> original triangle id
    int32_t* inv_order = nullptr; // original triangle id -> leaf order
    int root = kNoRef;
    int64_t n_nodes_alloc = 0;
    int64_t nodes_reachable = 0, leaves = 0;
    int depth = 0;
    int leaf_size = 4;
    MeshDev* mesh = nullptr;
};

// Data term, evaluated at a boundary point.
struct DataDev {
    int mode;
    const float* vdata;
    const int32_t* tris;  // original triangles (P1 lookup)
    float poly[10];
    float x0[3];
    float scale;
};

struct WalkParams {
    // geometry
    const float4* nodes;  // 8-wide BVH nodes (root = node 0)
    const float4* tv;
    const int32_t* inv_order;
    int iter_limit;  // traversal loop bound (4 x wide nodes + 64)
    const float* verts;
    const double* verts_d;  // FP64 copy of verts (resampled area samples)
    const int32_t* tris;
    const NormalArea* tri_n;
    const TriFrame* tri_f;
    const double* cdf;
    const int32_t* guide;  // guide table of the area CDF (see area_pick)
    int guide_bits;
    int64_t T;
    double area;
    double L;
    // problem
    int kind;
    const uint8_t* bc_type;  // mixed problems: condition per triangle (original order)
    float kmix, pk;          // mixed problems: Dirichlet-part constant, move probability
    int ris;                 // > 1: resampled importance sampling candidates
    int phi;
    float alpha;
    DataDev data;
    uint32_t key0, key1;
    // queries and walks
    const float* queries;
    const int32_t* query_prim;
    int64_t Q;
    int32_t N;
    int32_t M;
    int64_t walk_begin;
    uint32_t q_base;
    // near-degenerate thresholds
    float tauL;
    float edge_thr_L;  // kRareMargin * kFlagMargin * tau * L * max_edge
    float graze;
    // outputs
    double* part;        // (sum, sum of squares) per (query, 32-walk block): Q x tpq x 2
    int32_t tpq;         // 32-walk blocks per query, ceil(N / 32)
    double* per_walk;    // Q x N (optional: debug and gradient solves)
    double* per_walk_grad;  // 3 x Q x N gradient estimates (gradient kernels only)
    uint8_t* walk_flag;  // Q x N (optional)
    int32_t* line_m;     // Q x N x M (optional)
    int32_t* line_prim;  // Q x N x M picked triangle (original id, -1: none) (optional)
    uint8_t* line_flag;  // Q x N x M near-degenerate line (optional)
    unsigned long long* counters;  // [lines, nodes, tris, hits, flagged] (optional)
    int* error_word;
    unsigned long long* tile_counter;  // next walk tile (zero before the launch)
};

}  // namespace wob

// Host-side handle types named in the public header.
struct wob_mesh_s {
    wob::MeshDev d;
};
struct wob_bvh_s {
    wob::BvhDev d;
};
