// noalloc.cu -- wob_solve_noalloc: the same solve as wob_solve, for callers
// that cannot allocate device memory.
//
// wob_solve keeps per-query partial sums of the walk values (a sum and a sum
// of squares per block of 32 walks of a query) in scratch memory that it
// allocates on the stream for every call.  Some callers cannot let a library
// do that: an application or framework that has already reserved the GPU's
// memory for its own allocator (a library cudaMalloc would fail, or eat into
// memory the caller has promised elsewhere), or a latency-critical loop in
// which a cudaMalloc / cudaFree and the synchronisation it may imply are not
// acceptable.  This entry point keeps the partial sums in a fixed-size array
// compiled into the library instead (kNoAllocScratch doubles, 8 MiB); it
// calls no cudaMalloc, cudaFree or other allocating routine.
//
// Costs and rules of that choice:
//  * every GPU on which the library's device code is loaded holds the 8 MiB
//    array until the process exits;
//  * all calls share the one array per device, so calls whose work overlaps
//    on the GPU (different streams, or different host threads) race: order
//    them on one stream or synchronise between them;
//  * Q * ceil(walks / 32) must not exceed kNoAllocScratch / 2 = 2^19 (two
//    doubles per query and block of 32 walks; checked, rejected with
//    WOB_ERR_INVALID_ARG before any GPU work);
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (a host-side name of a __device__ variable is not
//    a device pointer); make that first call before any stream capture.
//    The address is cached per device for the life of the process: a
//    cudaDeviceReset (or any other end of the device's primary context)
//    invalidates it, so do not call this entry point after one.
#include <mutex>

#include "wob_host.h"

namespace wob {

namespace {

constexpr int64_t kNoAllocScratch = int64_t(1) << 20;  // 8 MiB of doubles
constexpr int kMaxDevices = 64;

// Walk-value partial sums of the most recent call; check word and walk-tile counter.
static __device__ __align__(256) double g_walk_values[kNoAllocScratch];
static __device__ __align__(256) int g_check_word[64];

std::mutex g_setup_mutex;
double* g_values_dev[kMaxDevices] = {};
int* g_check_dev[kMaxDevices] = {};

// Once per device, with that device current: device addresses of the arrays.
int device_arrays(int dev, double** values, int** check)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_values_dev[dev]) {
        void* v = nullptr;
        void* c = nullptr;
        WOB_CUDA_TRY(cudaGetSymbolAddress(&v, g_walk_values));
        WOB_CUDA_TRY(cudaGetSymbolAddress(&c, g_check_word));
        g_values_dev[dev] = static_cast<double*>(v);
        g_check_dev[dev] = static_cast<int*>(c);
    }
    *values = g_values_dev[dev];
    *check = g_check_dev[dev];
    return WOB_OK;
}

}  // namespace
}  // namespace wob

using namespace wob;

extern "C" int wob_solve_noalloc(const wob_problem* prob, const float* queries,
                                 const int32_t* query_prim, int64_t Q, int32_t walks,
                                 int32_t max_len, uint64_t seed, double* est, double* var,
                                 void* stream)
{
    clear_error();
    if (walks < 2) {
        set_error("walks must be >= 2 for a sample variance");
        return WOB_ERR_INVALID_ARG;
    }
    WOB_TRY(check_problem(prob));
    WOB_TRY(check_sizes(Q, 0, walks, max_len));
    if (Q == 0) return WOB_OK;
    if (!queries || !est || !var) {
        set_error("queries/est/var is NULL");
        return WOB_ERR_INVALID_ARG;
    }
    const int64_t blocks = Q * (int64_t)((walks + 31) / 32);
    if (2 * blocks > kNoAllocScratch) {
        set_error("wob_solve_noalloc: Q * ceil(walks / 32) = %lld exceeds the fixed scratch of "
                  "%lld blocks of 32 walks; split the queries or use wob_solve",
                  (long long)blocks, (long long)(kNoAllocScratch / 2));
        return WOB_ERR_INVALID_ARG;
    }
    if (prob->kind == WOB_DIRICHLET_DL && query_prim) {
        set_error("query_prim must be NULL for WOB_DIRICHLET_DL");
        return WOB_ERR_UNSUPPORTED;
    }
    int dev = 0;
    WOB_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d beyond %d", dev, kMaxDevices);
        return WOB_ERR_UNSUPPORTED;
    }
    double* values = nullptr;
    int* check = nullptr;
    WOB_TRY(device_arrays(dev, &values, &check));
    cudaStream_t s = (cudaStream_t)stream;
    WalkParams p;
    fill_params(p, prob, queries, query_prim, Q, 0, walks, max_len, seed);
    p.part = values;  // the walk kernels add into it: cleared below
    p.error_word = check;                                                   // check[0]
    p.tile_counter = reinterpret_cast<unsigned long long*>(check + 2);      // check[2..3]
    WOB_CUDA_TRY(cudaMemsetAsync(check, 0, 4 * sizeof(int), s));  // both must start at zero
    WOB_CUDA_TRY(cudaMemsetAsync(values, 0, 2 * blocks * sizeof(double), s));
    if (p.kind == WOB_DIRICHLET_DL)
        WOB_TRY(launch_dl_walks(p, false, false, s));
    else if (p.kind == WOB_NEUMANN_DIRECT)
        WOB_TRY(launch_nd_walks(p, false, s));
    else
        WOB_TRY(launch_sl_walks(p, false, s));
    return launch_reduce_part(values, Q, walks, p.tpq, est, var, nullptr, nullptr, s, check);
}
