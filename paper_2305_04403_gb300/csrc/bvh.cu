// bvh.cu -- linear BVH over triangle centroids, built on the GPU:
//   1. 63-bit Morton codes of the centroids (21 bits per axis);
//   2. bitonic sort of (code, triangle id) pairs;
//   3. binary radix tree over the sorted codes (Karras, "Maximizing
//      Parallelism in the Construction of BVHs, Octrees, and k-d Trees",
//      HPG 2012): one thread per interior node finds its range and split;
//   4. bottom-up boxes: each leaf walks to the root, the second thread to
//      reach a node (atomic visit counter) merges its children's boxes;
//   5. subtrees of at most leaf_size triangles become leaves; the remaining
//      interior nodes are renumbered densely and written in the traversal
//      layout (both child boxes in one 64-byte node).
#include <cfloat>
#include <cmath>

#include "wob_host.h"

namespace wob {

namespace {

__device__ __forceinline__ uint64_t spread21(uint32_t v)
{
    uint64_t x = v & 0x1FFFFFu;
    x = (x | x << 32) & 0x1F00000000FFFFull;
    x = (x | x << 16) & 0x1F0000FF0000FFull;
    x = (x | x << 8) & 0x100F00F00F00F00Full;
    x = (x | x << 4) & 0x10C30C30C30C30C3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__global__ void k_morton(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                         int64_t T, int64_t n_pad, float3 lo, float3 scale,
                         uint64_t* __restrict__ keys, int32_t* __restrict__ vals)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_pad;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (j >= T) {
            keys[j] = ~0ull;
            vals[j] = INT32_MAX;
            continue;
        }
        float c[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int64_t v = tris[3 * j + k];
            c[0] += verts[3 * v];
            c[1] += verts[3 * v + 1];
            c[2] += verts[3 * v + 2];
        }
        const float m = (float)((1u << 21) - 1);
        const uint32_t ix = (uint32_t)fminf(fmaxf((c[0] / 3.f - lo.x) * scale.x, 0.f), m);
        const uint32_t iy = (uint32_t)fminf(fmaxf((c[1] / 3.f - lo.y) * scale.y, 0.f), m);
        const uint32_t iz = (uint32_t)fminf(fmaxf((c[2] / 3.f - lo.z) * scale.z, 0.f), m);
        keys[j] = (spread21(ix) << 2) | (spread21(iy) << 1) | spread21(iz);
        vals[j] = (int32_t)j;
    }
}

// one compare-exchange stage of a bitonic sort of (key, val) pairs
__global__ void k_bitonic(uint64_t* __restrict__ keys, int32_t* __restrict__ vals, int64_t n,
                          int64_t k, int64_t jj)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i ^ jj;
        if (p <= i) continue;
        const bool up = (i & k) == 0;
        const uint64_t ki = keys[i], kp = keys[p];
        const int32_t vi = vals[i], vp = vals[p];
        const bool gt = (ki > kp) || (ki == kp && vi > vp);
        if (gt == up) {
            keys[i] = kp;
            keys[p] = ki;
            vals[i] = vp;
            vals[p] = vi;
        }
    }
}

// length of the common prefix of sorted keys i and j (index tie-break)
__device__ __forceinline__ int delta(const uint64_t* __restrict__ keys, int64_t n, int64_t i,
                                     int64_t j)
{
    if (j < 0 || j >= n) return -1;
    const uint64_t a = keys[i], b = keys[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

// Interior node i of n - 1: child references (>= 0 interior, < 0 leaf = -1 - pos),
// covered range [first, last], parents.
__global__ void k_radix_tree(const uint64_t* __restrict__ keys, int64_t n,
                             int32_t* __restrict__ left, int32_t* __restrict__ right,
                             int32_t* __restrict__ first, int32_t* __restrict__ last,
                             int32_t* __restrict__ parent_node,
                             int32_t* __restrict__ parent_leaf)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n - 1;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
        const int dmin = delta(keys, n, i, i - d);
        int64_t lmax = 2;
        while (delta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
        int64_t l = 0;
        for (int64_t t = lmax / 2; t >= 1; t /= 2)
            if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
        const int64_t j = i + l * d;
        const int dnode = delta(keys, n, i, j);
        int64_t s = 0;
        int64_t div = 2;
        int64_t t = (l + div - 1) / div;
        while (true) {
            if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
            if (t == 1) break;
            div *= 2;
            t = (l + div - 1) / div;
        }
        const int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
        const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
        const int32_t lref = (lo == gamma) ? (int32_t)(-1 - gamma) : (int32_t)gamma;
        const int32_t rref = (hi == gamma + 1) ? (int32_t)(-1 - (gamma + 1)) : (int32_t)(gamma + 1);
        left[i] = lref;
        right[i] = rref;
        first[i] = (int32_t)lo;
        last[i] = (int32_t)hi;
        if (lref >= 0) parent_node[lref] = (int32_t)i; else parent_leaf[-1 - lref] = (int32_t)i;
        if (rref >= 0) parent_node[rref] = (int32_t)i; else parent_leaf[-1 - rref] = (int32_t)i;
        if (i == 0) parent_node[0] = -1;
    }
}

struct Box {
    float lo[3], hi[3];
};

__device__ __forceinline__ Box leaf_box(const float* __restrict__ verts,
                                        const int32_t* __restrict__ tris, int32_t prim, float pad)
{
    Box b;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        b.lo[c] = FLT_MAX;
        b.hi[c] = -FLT_MAX;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t v = tris[3 * (int64_t)prim + k];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float x = verts[3 * v + c];
            b.lo[c] = fminf(b.lo[c], x);
            b.hi[c] = fmaxf(b.hi[c], x);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        b.lo[c] -= pad;
        b.hi[c] += pad;
    }
    return b;
}

__device__ __forceinline__ Box load_box(const float* __restrict__ p)
{
    Box b;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        b.lo[c] = __ldcg(p + c);
        b.hi[c] = __ldcg(p + 3 + c);
    }
    return b;
}

__device__ __forceinline__ void store_box(float* p, const Box& b)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        __stcg(p + c, b.lo[c]);
        __stcg(p + 3 + c, b.hi[c]);
    }
}

// Boxes, bottom-up.  No thread waits: the first thread to reach a node
// stops, the second merges (the visit counter orders the two).
__global__ void k_refit(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                        const int32_t* __restrict__ order, int64_t n, float pad,
                        const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                        const int32_t* __restrict__ parent_node,
                        const int32_t* __restrict__ parent_leaf, float* __restrict__ leaf_boxes,
                        float* __restrict__ node_boxes, int* __restrict__ visits)
{
    for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < n;
         pos += (int64_t)gridDim.x * blockDim.x) {
        const Box lb = leaf_box(verts, tris, order[pos], pad);
        store_box(leaf_boxes + 6 * pos, lb);
        __threadfence();
        int32_t p = n > 1 ? parent_leaf[pos] : -1;
        for (int step = 0; p >= 0 && step < 4096; ++step) {
            if (atomicAdd(visits + p, 1) != 1) break;  // first arrival (or a malformed tree)
            __threadfence();
            const int32_t l = left[p], r = right[p];
            const Box a = l >= 0 ? load_box(node_boxes + 6 * (int64_t)l) : load_box(leaf_boxes + 6 * (int64_t)(-1 - l));
            const Box b = r >= 0 ? load_box(node_boxes + 6 * (int64_t)r) : load_box(leaf_boxes + 6 * (int64_t)(-1 - r));
            Box u;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                u.lo[c] = fminf(a.lo[c], b.lo[c]);
                u.hi[c] = fmaxf(a.hi[c], b.hi[c]);
            }
            store_box(node_boxes + 6 * (int64_t)p, u);
            __threadfence();
            p = parent_node[p];
        }
    }
}

// Depth of every leaf (walk to the root), reduced to the maximum.
__global__ void k_depth(const int32_t* __restrict__ parent_node,
                        const int32_t* __restrict__ parent_leaf, int64_t n, int* __restrict__ out)
{
    int dmax = 0;
    for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < n;
         pos += (int64_t)gridDim.x * blockDim.x) {
        int d = 0;
        int32_t p = n > 1 ? parent_leaf[pos] : -1;
        while (p >= 0 && d < 4096) {
            ++d;
            p = parent_node[p];
        }
        dmax = max(dmax, d);
    }
    atomicMax(out, dmax);
}

// keep[i] = 1 if interior node i stays interior (covers > leaf_size triangles)
__global__ void k_keep(const int32_t* __restrict__ first, const int32_t* __restrict__ last,
                       int64_t n_int, int leaf_size, int* __restrict__ keep)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_int;
         i += (int64_t)gridDim.x * blockDim.x)
        keep[i] = (last[i] - first[i] + 1) > leaf_size ? 1 : 0;
}

__device__ __forceinline__ int child_ref(int32_t raw, const int32_t* __restrict__ first,
                                         const int32_t* __restrict__ last,
                                         const int* __restrict__ keep_scan, int leaf_size)
{
    if (raw < 0) return ~((-1 - raw) << 3);  // one-triangle leaf
    const int cnt = last[raw] - first[raw] + 1;
    if (cnt <= leaf_size) return ~((first[raw] << 3) | (cnt - 1));
    return keep_scan[raw] - 1;  // dense index of a kept interior node
}

__global__ void k_emit_nodes(int64_t n_int, const int32_t* __restrict__ left,
                             const int32_t* __restrict__ right, const int32_t* __restrict__ first,
                             const int32_t* __restrict__ last, const int* __restrict__ keep_scan,
                             int leaf_size, const float* __restrict__ leaf_boxes,
                             const float* __restrict__ node_boxes, float4* __restrict__ nodes,
                             int* __restrict__ leaf_count)
{
    int leaves = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_int;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (last[i] - first[i] + 1 <= leaf_size) continue;
        const int dst = keep_scan[i] - 1;
        const int32_t l = left[i], r = right[i];
        const float* bl = l >= 0 ? node_boxes + 6 * (int64_t)l : leaf_boxes + 6 * (int64_t)(-1 - l);
        const float* br = r >= 0 ? node_boxes + 6 * (int64_t)r : leaf_boxes + 6 * (int64_t)(-1 - r);
        const int rl = child_ref(l, first, last, keep_scan, leaf_size);
        const int rr = child_ref(r, first, last, keep_scan, leaf_size);
        leaves += (rl < 0) + (rr < 0);
        nodes[4 * dst + 0] = make_float4(bl[0], bl[3], bl[1], bl[4]);
        nodes[4 * dst + 1] = make_float4(br[0], br[3], br[1], br[4]);
        nodes[4 * dst + 2] = make_float4(bl[2], bl[5], br[2], br[5]);
        nodes[4 * dst + 3] = make_float4(__int_as_float(rl), __int_as_float(rr), 0.f, 0.f);
    }
    for (int o = 16; o > 0; o >>= 1) leaves += __shfl_xor_sync(0xFFFFFFFFu, leaves, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(leaf_count, leaves);
}

__global__ void k_emit_tris(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                            const int32_t* __restrict__ order, int64_t n,
                            float4* __restrict__ tv, int32_t* __restrict__ inv_order)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t prim = order[p];
        inv_order[prim] = (int32_t)p;
        float v[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int64_t vi = tris[3 * (int64_t)prim + k];
#pragma unroll
            for (int c = 0; c < 3; ++c) v[k][c] = verts[3 * vi + c];
        }
        const float e1x = v[1][0] - v[0][0], e1y = v[1][1] - v[0][1], e1z = v[1][2] - v[0][2];
        const float e2x = v[2][0] - v[0][0], e2y = v[2][1] - v[0][1], e2z = v[2][2] - v[0][2];
        const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z,
                    nz = e1x * e2y - e1y * e2x;
        tv[3 * p + 0] = make_float4(v[0][0], v[0][1], v[0][2], __int_as_float(prim));
        tv[3 * p + 1] = make_float4(v[1][0], v[1][1], v[1][2], sqrtf(nx * nx + ny * ny + nz * nz));
        tv[3 * p + 2] = make_float4(v[2][0], v[2][1], v[2][2], 0.f);
    }
}

template <typename T>
int dev_alloc(T** p, int64_t count, cudaStream_t s)
{
    WOB_CUDA_TRY(cudaMallocAsync((void**)p, (count > 0 ? count : 1) * sizeof(T), s));
    return WOB_OK;
}

// ---------------------------------------------------------------------------
// 8-wide BVH, collapsed top-down from the binary tree: a wide node starts
// from a binary interior node's two children and repeatedly replaces the
// interior child of largest surface area by its two children, up to 8.
// Layout (6 float4 = 96 bytes):
//   f[0] = (origin x, y, z, bits: ex | ey << 8 | ez << 16 | nint << 24 | nchild << 28)
//   f[1..3] = per axis: 8 quantised lows (bytes, slots 0..7) then 8 highs
//   f[4..5] = refs[0..7]: refs[0] = first internal child (when nint > 0);
//             leaf slots s >= nint hold binary leaf refs ~(first << 3 | count - 1)
// Slots 0 .. nint-1 are interior children stored at first_child + slot;
// child box = origin + q * 2^(e - 127) per axis, rounded outward.
// ---------------------------------------------------------------------------
struct WEntry {
    int ref;
    float lo[3], hi[3];
};

__device__ __forceinline__ float box_area(const WEntry& e)
{
    const float dx = e.hi[0] - e.lo[0], dy = e.hi[1] - e.lo[1], dz = e.hi[2] - e.lo[2];
    return dx * dy + dy * dz + dz * dx;
}

// children of binary interior node i as two entries
__device__ __forceinline__ void binary_children(const float4* __restrict__ nodes, int i, WEntry& a,
                                                WEntry& b)
{
    const float4 n0 = nodes[4 * i + 0], n1 = nodes[4 * i + 1], n2 = nodes[4 * i + 2];
    const int4 n3 = reinterpret_cast<const int4*>(nodes)[4 * i + 3];
    a.ref = n3.x;
    a.lo[0] = n0.x; a.hi[0] = n0.y; a.lo[1] = n0.z; a.hi[1] = n0.w; a.lo[2] = n2.x; a.hi[2] = n2.y;
    b.ref = n3.y;
    b.lo[0] = n1.x; b.hi[0] = n1.y; b.lo[1] = n1.z; b.hi[1] = n1.w; b.lo[2] = n2.z; b.hi[2] = n2.w;
}

__global__ void k_wide_collapse(const float4* __restrict__ nodes, int root_ref, float3 root_lo,
                                float3 root_hi, int64_t w_begin, int64_t w_end,
                                int32_t* __restrict__ src, float4* __restrict__ wn,
                                int* __restrict__ counter)
{
    for (int64_t w = w_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < w_end;
         w += (int64_t)gridDim.x * blockDim.x) {
        WEntry e[8];
        int n;
        const int s0 = w == 0 ? root_ref : src[w];
        if (s0 >= 0) {
            binary_children(nodes, s0, e[0], e[1]);
            n = 2;
        } else {  // the whole mesh is one leaf
            e[0].ref = s0;
            e[0].lo[0] = root_lo.x; e[0].lo[1] = root_lo.y; e[0].lo[2] = root_lo.z;
            e[0].hi[0] = root_hi.x; e[0].hi[1] = root_hi.y; e[0].hi[2] = root_hi.z;
            n = 1;
        }
        while (n < 8) {
            int best = -1;
            float ba = -1.f;
            for (int j = 0; j < n; ++j)
                if (e[j].ref >= 0 && box_area(e[j]) > ba) {
                    ba = box_area(e[j]);
                    best = j;
                }
            if (best < 0) break;
            WEntry a, b;
            binary_children(nodes, e[best].ref, a, b);
            e[best] = a;
            e[n++] = b;
        }
        // interior children first
        WEntry o[8];
        int nint = 0;
        for (int j = 0; j < n; ++j)
            if (e[j].ref >= 0) o[nint++] = e[j];
        int k = nint;
        for (int j = 0; j < n; ++j)
            if (e[j].ref < 0) o[k++] = e[j];
        const int first_child = nint > 0 ? atomicAdd(counter, nint) : 0;
        for (int j = 0; j < nint; ++j) src[first_child + j] = o[j].ref;
        // node box and quantisation (FP64, outward)
        double lo[3], hi[3];
        for (int c = 0; c < 3; ++c) {
            lo[c] = o[0].lo[c];
            hi[c] = o[0].hi[c];
            for (int j = 1; j < n; ++j) {
                lo[c] = fmin(lo[c], (double)o[j].lo[c]);
                hi[c] = fmax(hi[c], (double)o[j].hi[c]);
            }
        }
        // origin rounded down; the scale covers [origin, hi] in 255 steps
        float org[3];
        for (int c = 0; c < 3; ++c) org[c] = __double2float_rd(lo[c]);
        uint32_t ebits[3];
        double scale[3];
        for (int c = 0; c < 3; ++c) {
            const double ext = hi[c] - (double)org[c];
            int ex = -126;
            if (ext > 0.0) {
                int e2;
                frexp(ext / 255.0, &e2);  // ext / 255 < 2^e2
                ex = e2 < -126 ? -126 : e2;
            }
            ebits[c] = (uint32_t)(ex + 127);
            scale[c] = ldexp(1.0, ex);
        }
        uint32_t q[3][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};  // [axis][lo0-3, lo4-7, hi0-3, hi4-7]
        for (int j = 0; j < n; ++j)
            for (int c = 0; c < 3; ++c) {
                const double ql = floor(((double)o[j].lo[c] - org[c]) / scale[c]);
                const double qh = ceil(((double)o[j].hi[c] - org[c]) / scale[c]);
                const uint32_t bl = (uint32_t)fmin(fmax(ql, 0.0), 255.0);
                const uint32_t bh = (uint32_t)fmin(fmax(qh, 0.0), 255.0);
                q[c][j >> 2] |= bl << (8 * (j & 3));
                q[c][2 + (j >> 2)] |= bh << (8 * (j & 3));
            }
        int refs[8];
        for (int j = 0; j < 8; ++j) refs[j] = (j < n && j >= nint) ? o[j].ref : 0;
        if (nint > 0) refs[0] = first_child;
        float4* d = wn + 6 * w;
        const uint32_t hdr = ebits[0] | (ebits[1] << 8) | (ebits[2] << 16) | ((uint32_t)nint << 24) |
                             ((uint32_t)n << 28);
        d[0] = make_float4(org[0], org[1], org[2], __uint_as_float(hdr));
        for (int c = 0; c < 3; ++c)
            d[1 + c] = make_float4(__uint_as_float(q[c][0]), __uint_as_float(q[c][1]),
                                   __uint_as_float(q[c][2]), __uint_as_float(q[c][3]));
        d[4] = make_float4(__int_as_float(refs[0]), __int_as_float(refs[1]),
                           __int_as_float(refs[2]), __int_as_float(refs[3]));
        d[5] = make_float4(__int_as_float(refs[4]), __int_as_float(refs[5]),
                           __int_as_float(refs[6]), __int_as_float(refs[7]));
    }
}

}  // namespace

// Collapse the binary tree into 8-wide nodes (level by level from the root).
int build_wide(BvhDev& b, const MeshDev& m, cudaStream_t s)
{
    const int64_t cap = b.n_nodes_alloc > 0 ? b.n_nodes_alloc : 1;
    WOB_CUDA_TRY(cudaMalloc((void**)&b.wnodes, 6 * cap * sizeof(float4)));
    int32_t* src = nullptr;
    int* counter = nullptr;
    WOB_CUDA_TRY(cudaMallocAsync((void**)&src, cap * sizeof(int32_t), s));
    WOB_CUDA_TRY(cudaMallocAsync((void**)&counter, sizeof(int), s));
    const int one = 1;
    WOB_CUDA_TRY(cudaMemcpyAsync(counter, &one, sizeof(int), cudaMemcpyHostToDevice, s));
    const float pad = (float)(kBoxPad * m.L);
    const float3 rlo = make_float3((float)m.lo[0] - pad, (float)m.lo[1] - pad, (float)m.lo[2] - pad);
    const float3 rhi = make_float3((float)m.hi[0] + pad, (float)m.hi[1] + pad, (float)m.hi[2] + pad);
    int64_t w_begin = 0, w_end = 1;
    int levels = 0, rc = WOB_OK;
    while (w_begin < w_end && levels < 1024) {
        const int grid = grid_for((const void*)k_wide_collapse, 128, 0, w_end - w_begin);
        k_wide_collapse<<<grid, 128, 0, s>>>(b.nodes, b.root, rlo, rhi, w_begin, w_end, src,
                                             b.wnodes, counter);
        int c = 0;
        if (cudaMemcpyAsync(&c, counter, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = WOB_ERR_CUDA;
            break;
        }
        w_begin = w_end;
        w_end = c;
        ++levels;
    }
    cudaFreeAsync(src, s);
    cudaFreeAsync(counter, s);
    if (rc != WOB_OK) {
        set_error("wide BVH collapse failed");
        return rc;
    }
    b.n_wide = w_end;
    b.wide_levels = levels;
    return WOB_OK;
}

void free_bvh(BvhDev& b)
{
    cudaFree(b.nodes);
    cudaFree(b.wnodes);
    b.wnodes = nullptr;
    cudaFree(b.tv);
    cudaFree(b.order);
    cudaFree(b.inv_order);
    b.nodes = nullptr;
    b.tv = nullptr;
    b.order = nullptr;
    b.inv_order = nullptr;
}

int build_bvh_impl(MeshDev& m, int leaf_size, cudaStream_t s, BvhDev& b)
{
    const int64_t n = m.T;
    if (n < 1 || n > kMaxTriangles) {
        set_error("BVH: triangle count %lld outside [1, %lld]", (long long)n,
                  (long long)kMaxTriangles);
        return WOB_ERR_INVALID_ARG;
    }
    b.mesh = &m;
    b.leaf_size = leaf_size;
    int64_t n_pad = 1;
    while (n_pad < n) n_pad <<= 1;
    const int threads = 256;

    uint64_t* keys = nullptr;
    int32_t* vals = nullptr;
    WOB_TRY(dev_alloc(&keys, n_pad, s));
    WOB_TRY(dev_alloc(&vals, n_pad, s));
    const float3 lo = make_float3((float)m.lo[0], (float)m.lo[1], (float)m.lo[2]);
    auto sc = [](double l, double h) {
        const double e = h - l;
        return (float)(e > 0 ? ((1u << 21) - 1) / e : 0.0);
    };
    const float3 scale = make_float3(sc(m.lo[0], m.hi[0]), sc(m.lo[1], m.hi[1]), sc(m.lo[2], m.hi[2]));
    k_morton<<<grid_for((const void*)k_morton, threads, 0, n_pad), threads, 0, s>>>(
        m.verts, m.tris, n, n_pad, lo, scale, keys, vals);
    WOB_CUDA_TRY(cudaGetLastError());
    const int gb = grid_for((const void*)k_bitonic, threads, 0, n_pad);
    for (int64_t k = 2; k <= n_pad; k <<= 1)
        for (int64_t jj = k >> 1; jj > 0; jj >>= 1)
            k_bitonic<<<gb, threads, 0, s>>>(keys, vals, n_pad, k, jj);
    WOB_CUDA_TRY(cudaGetLastError());

    const int64_t n_int = n - 1;
    int32_t *left, *right, *first, *last, *parent_node, *parent_leaf;
    int *visits, *keep, *counters;
    float *leaf_boxes, *node_boxes;
    WOB_TRY(dev_alloc(&left, n_int, s));
    WOB_TRY(dev_alloc(&right, n_int, s));
    WOB_TRY(dev_alloc(&first, n_int, s));
    WOB_TRY(dev_alloc(&last, n_int, s));
    WOB_TRY(dev_alloc(&parent_node, n_int, s));
    WOB_TRY(dev_alloc(&parent_leaf, n, s));
    WOB_TRY(dev_alloc(&visits, n_int, s));
    WOB_TRY(dev_alloc(&keep, n_int, s));
    WOB_TRY(dev_alloc(&counters, 2, s));
    WOB_TRY(dev_alloc(&leaf_boxes, 6 * n, s));
    WOB_TRY(dev_alloc(&node_boxes, 6 * (n_int > 0 ? n_int : 1), s));
    WOB_CUDA_TRY(cudaMemsetAsync(visits, 0, (n_int > 0 ? n_int : 1) * sizeof(int), s));
    WOB_CUDA_TRY(cudaMemsetAsync(counters, 0, 2 * sizeof(int), s));
    WOB_CUDA_TRY(cudaMalloc((void**)&b.order, n * sizeof(int32_t)));
    WOB_CUDA_TRY(cudaMemcpyAsync(b.order, vals, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (n_int > 0) {
        k_radix_tree<<<grid_for((const void*)k_radix_tree, threads, 0, n_int), threads, 0, s>>>(
            keys, n, left, right, first, last, parent_node, parent_leaf);
        WOB_CUDA_TRY(cudaGetLastError());
    }
    // pad boxes so that FP32 slab tests never cull a triangle the line meets
    const float pad = (float)(kBoxPad * m.L);
    k_refit<<<grid_for((const void*)k_refit, threads, 0, n), threads, 0, s>>>(
        m.verts, m.tris, b.order, n, pad, left, right, parent_node, parent_leaf, leaf_boxes,
        node_boxes, visits);
    WOB_CUDA_TRY(cudaGetLastError());
    k_depth<<<grid_for((const void*)k_depth, threads, 0, n), threads, 0, s>>>(
        parent_node, parent_leaf, n, counters);
    WOB_CUDA_TRY(cudaGetLastError());

    int kept = 0;
    int* keep_scan = nullptr;
    if (n_int > 0) {
        WOB_TRY(dev_alloc(&keep_scan, n_int, s));
        k_keep<<<grid_for((const void*)k_keep, threads, 0, n_int), threads, 0, s>>>(
            first, last, n_int, leaf_size, keep);
        WOB_CUDA_TRY(cudaGetLastError());
        WOB_TRY(inclusive_scan<int>(keep, keep_scan, n_int, s));
        WOB_CUDA_TRY(cudaMemcpyAsync(&kept, keep_scan + n_int - 1, sizeof(int),
                                     cudaMemcpyDeviceToHost, s));
        WOB_CUDA_TRY(cudaStreamSynchronize(s));
    }
    b.n_nodes_alloc = kept > 0 ? kept : 1;
    WOB_CUDA_TRY(cudaMalloc((void**)&b.nodes, 4 * b.n_nodes_alloc * sizeof(float4)));
    WOB_CUDA_TRY(cudaMalloc((void**)&b.tv, 3 * n * sizeof(float4)));
    WOB_CUDA_TRY(cudaMalloc((void**)&b.inv_order, n * sizeof(int32_t)));
    if (kept > 0) {
        k_emit_nodes<<<grid_for((const void*)k_emit_nodes, threads, 0, n_int), threads, 0, s>>>(
            n_int, left, right, first, last, keep_scan, leaf_size, leaf_boxes, node_boxes,
            b.nodes, counters + 1);
        WOB_CUDA_TRY(cudaGetLastError());
        b.root = 0;
    } else {
        // the whole mesh fits one leaf: the root reference is that leaf
        b.root = ~((0 << 3) | (int)(n - 1));
    }
    k_emit_tris<<<grid_for((const void*)k_emit_tris, threads, 0, n), threads, 0, s>>>(
        m.verts, m.tris, b.order, n, b.tv, b.inv_order);
    WOB_CUDA_TRY(cudaGetLastError());
    int hc[2];
    WOB_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
    for (void* p : {(void*)keys, (void*)vals, (void*)left, (void*)right, (void*)first,
                    (void*)last, (void*)parent_node, (void*)parent_leaf, (void*)visits,
                    (void*)keep, (void*)counters, (void*)leaf_boxes, (void*)node_boxes,
                    (void*)keep_scan})
        if (p) cudaFreeAsync(p, s);
    WOB_CUDA_TRY(cudaStreamSynchronize(s));
    b.depth = hc[0];
    b.nodes_reachable = kept > 0 ? kept : 1;
    b.leaves = kept > 0 ? hc[1] : 1;
    if (b.depth >= kStackSize) {
        set_error("BVH depth %d exceeds the traversal stack (%d)", b.depth, kStackSize);
        free_bvh(b);
        return WOB_ERR_UNSUPPORTED;
    }
    if (b.n_nodes_alloc >= (1 << 24)) {
        set_error("BVH: %lld interior nodes exceed the wide traversal's 2^24", (long long)b.n_nodes_alloc);
        free_bvh(b);
        return WOB_ERR_UNSUPPORTED;
    }
    const int wrc = build_wide(b, m, s);
    if (wrc != WOB_OK) {
        free_bvh(b);
        return wrc;
    }
    // the binary nodes were only the input of the collapse
    cudaFree(b.nodes);
    b.nodes = nullptr;
    return WOB_OK;
}

}  // namespace wob
