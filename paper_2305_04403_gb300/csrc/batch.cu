// batch.cu -- many independent double-layer problems in one persistent,
// graph-captured launch, with an autotuned tile schedule.
//
// Work decomposition: the walks of problem p (Q_p x N_p, walk index
// qi * N_p + w) are cut into tiles of 32 * tile_rounds consecutive walks.
// A warp takes one tile at a time from a global counter, so its 32 lanes
// always run walks of a single problem (same BVH, same path length) and the
// lanes of a warp start their lines together, as in the single-problem
// kernel.  Tile order is either problem after problem (neighbouring warps
// share a BVH in L2) or costliest problems first (shorter tail); the
// autotuner measures both for each tile size on the batch at hand.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include <sys/stat.h>
#include <unistd.h>

#include "wob_device.cuh"
#include "wob_host.h"

namespace wob {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

struct BatchProblem {
    const float4* nodes;  // 8-wide nodes
    const float4* tv;
    DataDev data;
    int iter_limit;
    int phi;
    int M;
    int N;
    uint32_t problem;
    float tauL;
    float edge_thr_L;
    float graze;
    int64_t query_base;  // first row of this problem in queries / est / var
    int64_t part_base;   // first (query, 32-walk block) slot of this problem's partials
    int64_t n_walks;     // Q_p * N_p
};

struct Tile {
    int32_t problem;
    int32_t pad;
    int64_t first;  // first walk (problem-local)
};

template <int ROUNDS>
__global__ void __launch_bounds__(128, 8)
    k_dl_batched(const BatchProblem* __restrict__ probs, const Tile* __restrict__ tiles,
                 int64_t n_tiles, const float* __restrict__ queries,
                 const uint64_t* __restrict__ seed_dev, unsigned long long* counter,
                 double* __restrict__ part, int* err_word)
{
    const int lane = threadIdx.x & 31;
    const uint64_t seed = *seed_dev;
    __shared__ double slots[8 * 128];
    __shared__ int leafq[kLeafQ * 128];
    const WalkSlot ws{slots + threadIdx.x, 128};
    const LeafQueue lq{leafq + threadIdx.x, 128};
    int stack[kStackSize];
    int hits[kMaxHits];
    int err = 0;
    WalkCount c{0, 0, 0, 0, 0};
    while (true) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(counter, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if (t >= (unsigned long long)n_tiles) break;
        const Tile tile = tiles[t];
        const BatchProblem& P = probs[tile.problem];
        const DLGeom G{P.nodes, P.tv, P.iter_limit, P.edge_thr_L, P.tauL, P.graze};
        const StreamKey key{(uint32_t)seed ^ P.problem, (uint32_t)(seed >> 32)};
#pragma unroll 1
        for (int r = 0; r < ROUNDS; ++r) {
            const int64_t local = tile.first + r * 32 + lane;
            const bool live = local < P.n_walks;
            const int64_t qi = live ? local / P.N : 0;
            const int64_t w = local - qi * P.N;
            double v = 0.0;
            if (live) {
                const float* qp = queries + 3 * (P.query_base + qi);
                const double3 x = make_double3(qp[0], qp[1], qp[2]);
                int wflag = 0;
                v = dl_walk<false, false>(G, P.data, (double)P.phi, P.M, key, (uint32_t)qi,
                                          (uint32_t)w, x, -1, ws, stack, hits, err, wflag,
                                          LineOut{nullptr, nullptr, nullptr}, c, lq);
            }
            add_tile_partials(v, live, qi, w, (P.N + 31) / 32, part + 2 * P.part_base);
        }
    }
    if (err) atomicOr(err_word, err);
}

// One warp per query: find the query's problem, then mean and variance from
// the partials of its 32-walk blocks in a fixed order.
__global__ void k_reduce_batched(const double* __restrict__ part,
                                 const int64_t* __restrict__ qoff,
                                 const int64_t* __restrict__ part_base,
                                 const int32_t* __restrict__ walks, int32_t P, int64_t Qt,
                                 double* __restrict__ est, double* __restrict__ var,
                                 const int* __restrict__ err)
{
    const bool bad = *err != 0;  // a traversal check fired in this replay
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t gq = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); gq < Qt;
         gq += warps) {
        int lo = 0, hi = P - 1;  // last problem with qoff[p] <= gq
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (qoff[mid] <= gq) lo = mid; else hi = mid - 1;
        }
        const int N = walks[lo];
        const int tpq = (N + 31) / 32;
        const double2* v =
            reinterpret_cast<const double2*>(part) + part_base[lo] + (gq - qoff[lo]) * tpq;
        double s = 0.0, ss = 0.0;
        for (int i = lane; i < tpq; i += 32) {
            const double2 x = v[i];
            s += x.x;
            ss += x.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(kFull, s, o);
            ss += __shfl_xor_sync(kFull, ss, o);
        }
        if (lane == 0) {
            const double mean = s / N;
            est[gq] = bad ? __longlong_as_double(0x7FF8000000000000ll) : mean;
            var[gq] = bad ? __longlong_as_double(0x7FF8000000000000ll)
                          : (N > 1 ? fmax(ss - s * mean, 0.0) / (N - 1) : 0.0);
        }
    }
}

__global__ void k_set_seed(uint64_t* seed_dev, uint64_t seed) { *seed_dev = seed; }

// ------------------------------------------------------------------ autotune
std::mutex g_cache_mutex;

std::string cache_path()
{
    if (const char* e = getenv("WOB_TUNE_CACHE")) return e;
    const char* home = getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/wob_autotune.json";
}

// The cache is a flat JSON object {"key": "rounds,order", ...}.
std::map<std::string, std::string> read_cache()
{
    std::map<std::string, std::string> m;
    std::ifstream f(cache_path());
    if (!f) return m;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    size_t i = 0;
    while (true) {
        const size_t k0 = s.find('"', i);
        if (k0 == std::string::npos) break;
        const size_t k1 = s.find('"', k0 + 1);
        const size_t v0 = s.find('"', k1 + 1);
        const size_t v1 = v0 == std::string::npos ? v0 : s.find('"', v0 + 1);
        if (k1 == std::string::npos || v1 == std::string::npos) break;
        m[s.substr(k0 + 1, k1 - k0 - 1)] = s.substr(v0 + 1, v1 - v0 - 1);
        i = v1 + 1;
    }
    return m;
}

void make_parent_dirs(const std::string& path)
{
    for (size_t i = 1; i < path.size(); ++i)
        if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);  // existing dirs: EEXIST
}

void write_cache(const std::map<std::string, std::string>& m)
{
    const std::string path = cache_path();
    make_parent_dirs(path);
    // a temporary file of this process, renamed over the cache: concurrent
    // writers never interleave, the last rename wins
    const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
    std::ofstream f(tmp);
    if (!f) return;
    f << "{\n";
    size_t n = 0;
    for (const auto& kv : m)
        f << "  \"" << kv.first << "\": \"" << kv.second << "\"" << (++n < m.size() ? "," : "") << "\n";
    f << "}\n";
    f.close();
    rename(tmp.c_str(), path.c_str());
}

int log2_bucket(double x) { return x <= 1 ? 0 : (int)std::floor(std::log2(x)); }

}  // namespace
}  // namespace wob

using namespace wob;

struct wob_batch_s {
    int32_t P = 0;
    int64_t Qt = 0, W = 0, max_lines = 0;
    int64_t n_slots = 0;  // (query, 32-walk block) slots of all problems
    std::vector<BatchProblem> host_probs;
    std::vector<int32_t> walks;
    std::vector<int64_t> qoff, part_base;
    BatchProblem* probs = nullptr;
    Tile* tiles = nullptr;
    int64_t n_tiles = 0;
    int64_t* qoff_dev = nullptr;
    int64_t* part_base_dev = nullptr;
    int32_t* walks_dev = nullptr;
    double* part = nullptr;  // (sum, sum of squares) per slot
    unsigned long long* counter = nullptr;
    uint64_t* seed_dev = nullptr;
    int* err = nullptr;
    const float* queries = nullptr;
    double* est = nullptr;
    double* var = nullptr;
    int rounds = 1, order = 0, from_cache = 0;
    double tune_ms[8] = {0};
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// Tiles of 32 * rounds walks; order 0: problems in input order, 1: by
// descending estimated cost per walk (path length x log2 triangles).
std::vector<Tile> make_tiles(const wob_batch_s& b, const std::vector<double>& cost, int rounds,
                             int order, const std::vector<int64_t>& n_walks)
{
    std::vector<int> idx(b.P);
    for (int p = 0; p < b.P; ++p) idx[p] = p;
    if (order == 1)
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    std::vector<Tile> t;
    const int64_t ts = 32 * (int64_t)rounds;
    for (int p : idx)
        for (int64_t f = 0; f < n_walks[p]; f += ts) t.push_back(Tile{p, 0, f});
    return t;
}

int batch_grid(int rounds, int64_t n_tiles)
{
    const void* kern = rounds == 4 ? (const void*)k_dl_batched<4>
                     : rounds == 2 ? (const void*)k_dl_batched<2> : (const void*)k_dl_batched<1>;
    return grid_for(kern, 128, 0, n_tiles * 32);
}

// Counter reset + walk kernel (no API call here may break stream capture).
int launch_batch_kernels(wob_batch_s& b, const BatchProblem* probs, const Tile* tiles,
                         int64_t n_tiles, int rounds, int grid, double* part, int64_t n_slots,
                         cudaStream_t s)
{
    WOB_CUDA_TRY(cudaMemsetAsync(b.counter, 0, sizeof(unsigned long long), s));
    WOB_CUDA_TRY(cudaMemsetAsync(b.err, 0, sizeof(int), s));  // this run's checks
    WOB_CUDA_TRY(cudaMemsetAsync(part, 0, n_slots * 2 * sizeof(double), s));  // added into
    const int threads = 128;
    if (rounds == 4)
        k_dl_batched<4><<<grid, threads, 0, s>>>(probs, tiles, n_tiles, b.queries, b.seed_dev, b.counter, part, b.err);
    else if (rounds == 2)
        k_dl_batched<2><<<grid, threads, 0, s>>>(probs, tiles, n_tiles, b.queries, b.seed_dev, b.counter, part, b.err);
    else
        k_dl_batched<1><<<grid, threads, 0, s>>>(probs, tiles, n_tiles, b.queries, b.seed_dev, b.counter, part, b.err);
    WOB_CUDA_TRY(cudaGetLastError());
    return WOB_OK;
}

void free_batch(wob_batch_s* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (void* p : {(void*)b->probs, (void*)b->tiles, (void*)b->qoff_dev, (void*)b->part_base_dev,
                    (void*)b->walks_dev, (void*)b->part, (void*)b->counter,
                    (void*)b->seed_dev, (void*)b->err})
        if (p) cudaFree(p);
}

// Time every (rounds, order) candidate once with the walk counts scaled
// down (every problem keeps at least 32 walks); pick the fastest.
int autotune(wob_batch_s& b, const std::vector<double>& cost, cudaStream_t s)
{
    std::vector<BatchProblem> small = b.host_probs;
    std::vector<int64_t> n_small(b.P);
    int64_t base = 0;
    for (int p = 0; p < b.P; ++p) {
        const int Ns = std::max(32, b.walks[p] / 8);
        small[p].N = std::min(Ns, b.walks[p]);
        small[p].n_walks = (b.qoff[p + 1] - b.qoff[p]) * (int64_t)small[p].N;
        small[p].part_base = base;  // fewer walks: at most the full batch's slots
        base += (b.qoff[p + 1] - b.qoff[p]) * (int64_t)((small[p].N + 31) / 32);
        n_small[p] = small[p].n_walks;
    }
    BatchProblem* dprobs = nullptr;
    WOB_CUDA_TRY(cudaMalloc((void**)&dprobs, b.P * sizeof(BatchProblem)));
    WOB_CUDA_TRY(cudaMemcpy(dprobs, small.data(), b.P * sizeof(BatchProblem), cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    const int rounds_c[3] = {1, 2, 4};
    int rc = WOB_OK;
    for (int ri = 0; ri < 3 && rc == WOB_OK; ++ri)
        for (int order = 0; order < 2 && rc == WOB_OK; ++order) {
            std::vector<Tile> t = make_tiles(b, cost, rounds_c[ri], order, n_small);
            Tile* dt = nullptr;
            if (cudaMalloc((void**)&dt, t.size() * sizeof(Tile)) != cudaSuccess) {
                rc = WOB_ERR_OOM;
                break;
            }
            cudaMemcpy(dt, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice);
            float ms = 0.f, best_rep = 1e30f;
            for (int rep = 0; rep < 2 && rc == WOB_OK; ++rep) {  // first run warms caches
                cudaEventRecord(e0, s);
                rc = launch_batch_kernels(b, dprobs, dt, (int64_t)t.size(), rounds_c[ri],
                                          batch_grid(rounds_c[ri], (int64_t)t.size()), b.part,
                                          base, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 1) best_rep = ms;
            }
            cudaFree(dt);
            b.tune_ms[ri * 2 + order] = best_rep;
            if (best_rep < best) {
                best = best_rep;
                b.rounds = rounds_c[ri];
                b.order = order;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dprobs);
    return rc;
}

}  // namespace

extern "C" {

int wob_batch_create(const wob_problem* problems, int32_t P, const int64_t* query_offsets,
                     const int32_t* walks, const int32_t* max_len, const float* queries,
                     double* est, double* var, const wob_batch_params* params, void* stream,
                     wob_batch* out)
{
    clear_error();
    if (!problems || P < 1 || !query_offsets || !walks || !max_len || !out) {
        set_error("wob_batch_create: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    wob_batch_s* b = new (std::nothrow) wob_batch_s();
    if (!b) {
        set_error("host allocation failed");
        return WOB_ERR_OOM;
    }
    b->P = P;
    b->queries = queries;
    b->est = est;
    b->var = var;
    b->walks.assign(walks, walks + P);
    b->qoff.assign(query_offsets, query_offsets + P + 1);
    b->part_base.resize(P + 1);
    b->host_probs.resize(P);
    std::vector<double> cost(P);
    std::vector<int64_t> n_walks(P);
    int rc = WOB_OK;
    double tris = 0.0;
    for (int p = 0; p < P && rc == WOB_OK; ++p) {
        const wob_problem* pr = problems + p;
        if ((rc = check_problem(pr)) != WOB_OK) break;
        if (pr->kind != WOB_DIRICHLET_DL) {
            set_error("problem %d: batched solves support WOB_DIRICHLET_DL only", p);
            rc = WOB_ERR_UNSUPPORTED;
            break;
        }
        const int64_t Qp = query_offsets[p + 1] - query_offsets[p];
        if (Qp < 0 || walks[p] < 2) {
            set_error("problem %d: negative query count or walks < 2", p);
            rc = WOB_ERR_INVALID_ARG;
            break;
        }
        if ((rc = check_sizes(Qp, 0, walks[p], max_len[p])) != WOB_OK) break;
        WalkParams wp;
        fill_params(wp, pr, nullptr, nullptr, Qp, 0, walks[p], max_len[p], 0);
        BatchProblem& bp = b->host_probs[p];
        bp.nodes = wp.nodes;
        bp.tv = wp.tv;
        bp.data = wp.data;
        bp.iter_limit = wp.iter_limit;
        bp.phi = wp.phi;
        bp.M = max_len[p];
        bp.N = walks[p];
        bp.problem = pr->problem;
        bp.tauL = wp.tauL;
        bp.edge_thr_L = wp.edge_thr_L;
        bp.graze = wp.graze;
        bp.query_base = query_offsets[p];
        bp.part_base = b->n_slots;
        bp.n_walks = Qp * walks[p];
        n_walks[p] = bp.n_walks;
        b->part_base[p] = b->n_slots;
        b->n_slots += Qp * (int64_t)((walks[p] + 31) / 32);
        b->W += bp.n_walks;
        b->max_lines += bp.n_walks * max_len[p];
        const double T = (double)pr->bvh->d.mesh->T;
        tris += T;
        cost[p] = max_len[p] * std::log2(T + 1.0);
    }
    b->part_base[P] = b->n_slots;
    b->Qt = query_offsets[P];
    if (rc == WOB_OK && b->Qt > 0 && (!queries || !est || !var)) {
        set_error("queries/est/var is NULL");
        rc = WOB_ERR_INVALID_ARG;
    }
    auto fail = [&](int code) {
        cudaStreamSynchronize(s);
        free_batch(b);
        delete b;
        return code;
    };
    if (rc != WOB_OK) return fail(rc);
    if (cudaMalloc((void**)&b->probs, P * sizeof(BatchProblem)) != cudaSuccess ||
        cudaMalloc((void**)&b->qoff_dev, (P + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc((void**)&b->part_base_dev, (P + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc((void**)&b->walks_dev, P * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc((void**)&b->part, std::max<int64_t>(b->n_slots, 1) * 2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&b->counter, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void**)&b->seed_dev, sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc((void**)&b->err, sizeof(int)) != cudaSuccess) {
        set_error("wob_batch_create: device allocation failed");
        return fail(WOB_ERR_OOM);
    }
    cudaMemcpy(b->probs, b->host_probs.data(), P * sizeof(BatchProblem), cudaMemcpyHostToDevice);
    cudaMemcpy(b->qoff_dev, b->qoff.data(), (P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(b->part_base_dev, b->part_base.data(), (P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(b->walks_dev, b->walks.data(), P * sizeof(int32_t), cudaMemcpyHostToDevice);
    cudaMemset(b->err, 0, sizeof(int));
    cudaMemset(b->seed_dev, 0, sizeof(uint64_t));

    // schedule: explicit, cached, or measured
    const bool tune = !params || params->autotune;
    if (!tune) {
        b->rounds = params->tile_rounds == 2 || params->tile_rounds == 4 ? params->tile_rounds : 1;
        b->order = params->order == 1 ? 1 : 0;
    } else {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceProp prop;
        cudaGetDeviceProperties(&prop, dev);
        double mean_M = 0.0;
        for (int p = 0; p < P; ++p) mean_M += max_len[p];
        mean_M /= P;
        char key[512];
        snprintf(key, sizeof(key), "dl_batched|%s|P%d|W%d|T%d|M%d", prop.name, log2_bucket(P),
                 log2_bucket((double)b->W), log2_bucket(tris), log2_bucket(mean_M));
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        auto cache = read_cache();
        auto it = cache.find(key);
        int r = 0, o = 0;
        if (it != cache.end() && sscanf(it->second.c_str(), "%d,%d", &r, &o) == 2 &&
            (r == 1 || r == 2 || r == 4) && (o == 0 || o == 1)) {
            b->rounds = r;
            b->order = o;
            b->from_cache = 1;
        } else {
            if ((rc = autotune(*b, cost, s)) != WOB_OK) return fail(rc);
            char val[32];
            snprintf(val, sizeof(val), "%d,%d", b->rounds, b->order);
            cache[key] = val;
            write_cache(cache);
        }
    }
    std::vector<Tile> t = make_tiles(*b, cost, b->rounds, b->order, n_walks);
    b->n_tiles = (int64_t)t.size();
    if (cudaMalloc((void**)&b->tiles, std::max<size_t>(t.size(), 1) * sizeof(Tile)) != cudaSuccess) {
        set_error("wob_batch_create: device allocation failed");
        return fail(WOB_ERR_OOM);
    }
    cudaMemcpy(b->tiles, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice);

    // capture counter reset + walk kernel + reduction into one graph
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("wob_batch_create: stream creation failed");
        return fail(WOB_ERR_CUDA);
    }
    const int g_walk = batch_grid(b->rounds, b->n_tiles);
    const int g_red = grid_for((const void*)k_reduce_batched, 256, 0, b->Qt * 32);
    cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    rc = launch_batch_kernels(*b, b->probs, b->tiles, b->n_tiles, b->rounds, g_walk, b->part,
                              b->n_slots, b->cap_stream);
    if (rc == WOB_OK && b->Qt > 0)
        k_reduce_batched<<<g_red, 256, 0, b->cap_stream>>>(b->part, b->qoff_dev,
                                                           b->part_base_dev, b->walks_dev, P,
                                                           b->Qt, est, var, b->err);
    const cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &b->graph);
    if (rc != WOB_OK || ce != cudaSuccess ||
        cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
        set_error("wob_batch_create: graph capture failed (%s)", cudaGetErrorString(ce));
        return fail(WOB_ERR_CUDA);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        set_error("wob_batch_create: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(WOB_ERR_CUDA);
    }
    *out = b;
    return WOB_OK;
}

int wob_solve_batched(const wob_problem* problems, int32_t P, const int64_t* query_offsets,
                      const float* queries, const int32_t* walks, const int32_t* max_len,
                      uint64_t seed, double* est, double* var, void* stream)
{
    wob_batch b = nullptr;
    int rc = wob_batch_create(problems, P, query_offsets, walks, max_len, queries, est, var,
                              nullptr, stream, &b);
    if (rc != WOB_OK) {  // report under this entry point's name
        const std::string inner = wob_last_error();
        set_error("wob_solve_batched (creating the batch): %s", inner.c_str());
        return rc;
    }
    rc = wob_batch_run(b, seed, stream);
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    wob_batch_destroy(b);
    if (rc == WOB_OK && e != cudaSuccess) {
        set_error("wob_solve_batched: %s", cudaGetErrorString(e));
        rc = WOB_ERR_CUDA;
    }
    return rc;
}

int wob_batch_run(wob_batch b, uint64_t seed, void* stream)
{
    clear_error();
    if (!b) {
        set_error("NULL batch");
        return WOB_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    k_set_seed<<<1, 1, 0, s>>>(b->seed_dev, seed);
    WOB_CUDA_TRY(cudaGetLastError());
    WOB_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    return WOB_OK;
}

int wob_batch_get_info(wob_batch b, wob_batch_info* out)
{
    clear_error();
    if (!b || !out) {
        set_error("NULL argument");
        return WOB_ERR_INVALID_ARG;
    }
    memset(out, 0, sizeof(*out));
    out->P = b->P;
    out->tile_rounds = b->rounds;
    out->order = b->order;
    out->from_cache = b->from_cache;
    out->queries = b->Qt;
    out->walks = b->W;
    out->max_lines = b->max_lines;
    out->tiles = b->n_tiles;
    for (int i = 0; i < 8; ++i) out->tune_ms[i] = b->tune_ms[i];
    return WOB_OK;
}

void wob_batch_destroy(wob_batch b)
{
    if (!b) return;
    free_batch(b);
    delete b;
}

}  // extern "C"
