// mesh.cu -- mesh upload, validation and per-triangle precompute (unit
// normals, areas, area prefix sums for area sampling), plus the generic
// inclusive scan used here and by the BVH builder.
#include <cfloat>
#include <cmath>
#include <cstdio>

#include "wob_host.h"

namespace wob {

namespace {

constexpr int kErrIndex = 1;
constexpr int kErrNonFinite = 2;
constexpr int kErrZeroArea = 4;

__device__ __forceinline__ unsigned int float_to_ordered(float f)
{
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float ordered_to_float(unsigned int u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
#else
    unsigned int v = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
    float f;
    memcpy(&f, &v, 4);
    return f;
#endif
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// bbox of the vertices and a finiteness check
__global__ void k_vertex_bounds(const float* __restrict__ verts, int64_t V,
                                unsigned int* __restrict__ bounds, int* __restrict__ err)
{
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float x = verts[3 * i + c];
            if (!isfinite(x)) {
                atomicOr(err, kErrNonFinite);
                continue;
            }
            lo[c] = fminf(lo[c], x);
            hi[c] = fmaxf(hi[c], x);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xFFFFFFFFu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xFFFFFFFFu, hi[c], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicMin(bounds + c, float_to_ordered(lo[c]));
            atomicMax(bounds + 3 + c, float_to_ordered(hi[c]));
        }
    }
}

// Unit normal and area (FP64), signed-volume and
// longest-edge reductions, index and degeneracy checks.
__global__ void k_triangles(const float* __restrict__ verts, int64_t V,
                            const int32_t* __restrict__ tris, int64_t T,
                            NormalArea* __restrict__ tri_n, TriFrame* __restrict__ tri_f,
                            double* __restrict__ area,
                            double* __restrict__ volume, unsigned int* __restrict__ max_edge,
                            int* __restrict__ err)
{
    double vol = 0.0;
    float emax = 0.0f;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < T;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i0 = tris[3 * j], i1 = tris[3 * j + 1], i2 = tris[3 * j + 2];
        if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= V || i1 >= V || i2 >= V) {
            atomicOr(err, kErrIndex);
            tri_n[j] = NormalArea{0.0, 0.0, 0.0, 0.0};
            area[j] = 0.0;
            continue;
        }
        const double a[3] = {verts[3 * (int64_t)i0], verts[3 * (int64_t)i0 + 1], verts[3 * (int64_t)i0 + 2]};
        const double b[3] = {verts[3 * (int64_t)i1], verts[3 * (int64_t)i1 + 1], verts[3 * (int64_t)i1 + 2]};
        const double c[3] = {verts[3 * (int64_t)i2], verts[3 * (int64_t)i2 + 1], verts[3 * (int64_t)i2 + 2]};
        const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                             e1[0] * e2[1] - e1[1] * e2[0]};
        const double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nl > 0.0) || !isfinite(nl)) {
            atomicOr(err, kErrZeroArea);
            tri_n[j] = NormalArea{0.0, 0.0, 0.0, 0.0};
            area[j] = 0.0;
            continue;
        }
        tri_n[j] = NormalArea{n[0] / nl, n[1] / nl, n[2] / nl, 0.5 * nl};
        area[j] = 0.5 * nl;
        TriFrame fr;
        for (int c = 0; c < 3; ++c) {
            const double nc = n[c] / nl;
            fr.v0[c] = (float)a[c];
            fr.e1h[c] = (float)e1[c];
            fr.e1l[c] = (float)(e1[c] - (double)fr.e1h[c]);
            fr.e2h[c] = (float)e2[c];
            fr.e2l[c] = (float)(e2[c] - (double)fr.e2h[c]);
            fr.nh[c] = (float)nc;
            fr.nl[c] = (float)(nc - (double)fr.nh[c]);
            fr.pad[c] = 0.f;
        }
        tri_f[j] = fr;
        // signed volume: a . (b x c) / 6
        vol += (a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
                a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
        const double e3[3] = {c[0] - b[0], c[1] - b[1], c[2] - b[2]};
        const float l1 = (float)sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        const float l2 = (float)sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
        const float l3 = (float)sqrt(e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
        emax = fmaxf(emax, fmaxf(l1, fmaxf(l2, l3)));
    }
    vol = warp_sum(vol);
    for (int o = 16; o > 0; o >>= 1) emax = fmaxf(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, o));
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(volume, vol);
        atomicMax(max_edge, __float_as_uint(emax));
    }
}

// ---------------------------------------------------------------------------
// Inclusive scan: each block scans 4 * 256 elements, writes its total; the
// totals are scanned recursively and added back.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

template <typename T>
__global__ void k_scan_tile(const T* __restrict__ in, T* __restrict__ out, int64_t n,
                            T* __restrict__ block_sums)
{
    __shared__ T warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    T v[kScanPer];
    T run = T(0);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int64_t k = base + i;
        run += (k < n) ? in[k] : T(0);
        v[i] = run;
    }
    // inclusive scan of the per-thread totals within the warp
    T x = run;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kScanThreads / 32 ? warp_tot[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    const T offset = (x - run) + (warp > 0 ? warp_tot[warp - 1] : T(0));
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int64_t k = base + i;
        if (k < n) out[k] = v[i] + offset;
    }
    if (threadIdx.x == kScanThreads - 1 && block_sums) block_sums[blockIdx.x] = x + (warp > 0 ? warp_tot[warp - 1] : T(0));
}

template <typename T>
__global__ void k_scan_add(T* __restrict__ out, int64_t n, const T* __restrict__ scanned_sums)
{
    const int64_t b = blockIdx.x + 1;  // block 0 needs no offset
    const T off = scanned_sums[b - 1];
    for (int64_t k = b * kScanTile + threadIdx.x; k < n && k < (b + 1) * kScanTile;
         k += blockDim.x)
        out[k] += off;
}

}  // namespace

template <typename T>
int inclusive_scan(const T* in, T* out, int64_t n, cudaStream_t s)
{
    if (n <= 0) return WOB_OK;
    const int64_t blocks = (n + kScanTile - 1) / kScanTile;
    T* sums = nullptr;
    if (blocks > 1) WOB_CUDA_TRY(cudaMallocAsync((void**)&sums, blocks * sizeof(T), s));
    k_scan_tile<T><<<(unsigned)blocks, kScanThreads, 0, s>>>(in, out, n, sums);
    WOB_CUDA_TRY(cudaGetLastError());
    if (blocks > 1) {
        int rc = inclusive_scan<T>(sums, sums, blocks, s);
        if (rc == WOB_OK) {
            k_scan_add<T><<<(unsigned)(blocks - 1), kScanThreads, 0, s>>>(out, n, sums);
            if (cudaGetLastError() != cudaSuccess) rc = WOB_ERR_CUDA;
        }
        cudaFreeAsync(sums, s);
        if (rc != WOB_OK) {
            set_error("inclusive_scan failed");
            return rc;
        }
    }
    return WOB_OK;
}

template int inclusive_scan<double>(const double*, double*, int64_t, cudaStream_t);
template int inclusive_scan<int>(const int*, int*, int64_t, cudaStream_t);

// FP64 copy of the vertex positions: the resampled single-layer walks form
// their area samples in FP64 from it without a conversion per coordinate
// (exact: every float is a double).
__global__ void k_to_f64(const float* __restrict__ in, int64_t n, double* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// Guide table of the area CDF (indexed search, Chen and Asau 1974): the
// area sample of the 53-bit uniform U picks the first j with cdf[j] >
// fl(U 2^-53 |Gamma|) (else T - 1).  For every U whose top `bits` bits are
// b that pick lies in [guide[b], guide[b + 1]], where guide[b] is the pick of
// U = b 2^(53 - bits): the rounded product is monotone in U.  Each entry is
// a binary search with the same comparison (doubles' bit patterns).
static __global__ void k_area_guide(const double* __restrict__ cdf, int64_t T, double area, int bits,
                             int32_t* __restrict__ guide)
{
    const int64_t nb = ((int64_t)1 << bits) + 1;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb;
         b += (int64_t)gridDim.x * blockDim.x) {
        const long long t =
            __double_as_longlong((double)((uint64_t)b << (53 - bits)) * 0x1p-53 * area);
        int64_t lo = 0, hi = T - 1;
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (__double_as_longlong(cdf[mid]) > t) hi = mid; else lo = mid + 1;
        }
        guide[b] = (int32_t)lo;
    }
}

void free_mesh(MeshDev& m)
{
    cudaFree(m.verts);
    cudaFree(m.verts_d);
    cudaFree(m.tris);
    cudaFree(m.tri_n);
    cudaFree(m.tri_f);
    cudaFree(m.cdf);
    cudaFree(m.guide);
    m.verts = nullptr;
    m.verts_d = nullptr;
    m.tris = nullptr;
    m.tri_n = nullptr;
    m.tri_f = nullptr;
    m.cdf = nullptr;
    m.guide = nullptr;
}

int build_mesh_impl(const float* verts, int64_t V, const int32_t* tris, int64_t T,
                    bool on_device, cudaStream_t s, MeshDev& m)
{
    WOB_CUDA_TRY(cudaGetDevice(&m.device));
    m.V = V;
    m.T = T;
    WOB_CUDA_TRY(cudaMalloc((void**)&m.verts, V * 3 * sizeof(float)));
    WOB_CUDA_TRY(cudaMalloc((void**)&m.verts_d, V * 3 * sizeof(double)));
    WOB_CUDA_TRY(cudaMalloc((void**)&m.tris, T * 3 * sizeof(int32_t)));
    WOB_CUDA_TRY(cudaMalloc((void**)&m.tri_n, T * sizeof(NormalArea)));
    WOB_CUDA_TRY(cudaMalloc((void**)&m.tri_f, T * sizeof(TriFrame)));
    WOB_CUDA_TRY(cudaMalloc((void**)&m.cdf, T * sizeof(double)));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    WOB_CUDA_TRY(cudaMemcpyAsync(m.verts, verts, V * 3 * sizeof(float), kind, s));
    WOB_CUDA_TRY(cudaMemcpyAsync(m.tris, tris, T * 3 * sizeof(int32_t), kind, s));

    // scratch: [bounds 6 uint][max_edge uint][err int][volume double]
    struct Scratch {
        unsigned int bounds[6];
        unsigned int max_edge;
        int err;
        double volume;
    };
    Scratch* sc = nullptr;
    double* area = nullptr;
    WOB_CUDA_TRY(cudaMallocAsync((void**)&sc, sizeof(Scratch), s));
    WOB_CUDA_TRY(cudaMallocAsync((void**)&area, T * sizeof(double), s));
    Scratch init;
    for (int c = 0; c < 3; ++c) {
        init.bounds[c] = 0xFFFFFFFFu;
        init.bounds[3 + c] = 0u;
    }
    init.max_edge = 0u;
    init.err = 0;
    init.volume = 0.0;
    WOB_CUDA_TRY(cudaMemcpyAsync(sc, &init, sizeof(Scratch), cudaMemcpyHostToDevice, s));
    const int threads = 256;
    k_to_f64<<<grid_for((const void*)k_to_f64, threads, 0, 3 * V), threads, 0, s>>>(m.verts, 3 * V,
                                                                                  m.verts_d);
    WOB_CUDA_TRY(cudaGetLastError());
    k_vertex_bounds<<<grid_for((const void*)k_vertex_bounds, threads, 0, V), threads, 0, s>>>(
        m.verts, V, sc->bounds, &sc->err);
    WOB_CUDA_TRY(cudaGetLastError());
    k_triangles<<<grid_for((const void*)k_triangles, threads, 0, T), threads, 0, s>>>(
        m.verts, V, m.tris, T, m.tri_n, m.tri_f, area, &sc->volume, &sc->max_edge, &sc->err);
    WOB_CUDA_TRY(cudaGetLastError());
    int rc = inclusive_scan<double>(area, m.cdf, T, s);
    Scratch h;
    WOB_CUDA_TRY(cudaMemcpyAsync(&h, sc, sizeof(Scratch), cudaMemcpyDeviceToHost, s));
    double total = 0.0;
    if (T > 0) WOB_CUDA_TRY(cudaMemcpyAsync(&total, m.cdf + T - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(sc, s);
    cudaFreeAsync(area, s);
    WOB_CUDA_TRY(cudaStreamSynchronize(s));
    if (rc != WOB_OK) return rc;
    if (h.err & kErrIndex) {
        set_error("triangle vertex index outside [0, V)");
        return WOB_ERR_DEGENERATE_MESH;
    }
    if (h.err & kErrNonFinite) {
        set_error("non-finite vertex coordinate");
        return WOB_ERR_DEGENERATE_MESH;
    }
    if (h.err & kErrZeroArea) {
        set_error("zero-area triangle");
        return WOB_ERR_DEGENERATE_MESH;
    }
    for (int c = 0; c < 3; ++c) {
        m.lo[c] = ordered_to_float(h.bounds[c]);
        m.hi[c] = ordered_to_float(h.bounds[3 + c]);
    }
    const double dx = m.hi[0] - m.lo[0], dy = m.hi[1] - m.lo[1], dz = m.hi[2] - m.lo[2];
    m.L = std::sqrt(dx * dx + dy * dy + dz * dz);
    float me;
    memcpy(&me, &h.max_edge, 4);
    m.max_edge = me;
    m.volume = h.volume;
    m.area = total;
    if (!(m.volume > 0.0)) {
        set_error("signed volume %.6g <= 0: triangles must be counter-clockwise seen from "
                  "outside the interior domain", m.volume);
        return WOB_ERR_DEGENERATE_MESH;
    }
    // guide table: about one triangle per bucket, at most 2^24 buckets
    int bits = 1;
    while (bits < 24 && ((int64_t)1 << bits) < T) ++bits;
    const int64_t nb = ((int64_t)1 << bits) + 1;
    WOB_CUDA_TRY(cudaMalloc((void**)&m.guide, nb * sizeof(int32_t)));
    m.guide_bits = bits;
    k_area_guide<<<grid_for((const void*)k_area_guide, threads, 0, nb), threads, 0, s>>>(
        m.cdf, T, m.area, bits, m.guide);
    WOB_CUDA_TRY(cudaGetLastError());
    WOB_CUDA_TRY(cudaStreamSynchronize(s));
    return WOB_OK;
}

}  // namespace wob
