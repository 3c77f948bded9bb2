// api.cu -- the extern "C" entry points declared in include/wob.h:
// argument validation, handle management, scratch allocation and launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include <climits>

#include "wob_host.h"

namespace wob {

namespace {
thread_local std::string g_error;
thread_local wob_stats g_last_stats = {0, 0, 0, 0, 0};  // of the last counted solve
}

void set_error(const char* fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_error = buf;
}

void clear_error() { g_error.clear(); }

int grid_for(const void* kernel, int threads, size_t smem, int64_t work_items)
{
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t full = (int64_t)sms * per_sm;
    int64_t need = (work_items + threads - 1) / threads;
    if (need < 1) need = 1;
    return (int)(need < full ? need : full);
}

int check_problem(const wob_problem* prob)
{
    if (!prob || !prob->bvh) {
        set_error("problem or problem->bvh is NULL");
        return WOB_ERR_INVALID_ARG;
    }
    if (prob->kind < WOB_DIRICHLET_DL || prob->kind > WOB_MIXED_SL) {
        set_error("unknown kind %d", prob->kind);
        return WOB_ERR_INVALID_ARG;
    }
    if (prob->iter_limit < 0) {
        set_error("iter_limit = %d is negative", prob->iter_limit);
        return WOB_ERR_INVALID_ARG;
    }
    if (prob->kind == WOB_MIXED_SL &&
        (!prob->bc_type || !(prob->k_mix > 0.0f) || !(prob->p_k > 0.0f && prob->p_k < 1.0f) ||
         prob->data_mode == WOB_DATA_VERTEX_P1)) {
        set_error("WOB_MIXED_SL needs bc_type, k_mix > 0, 0 < p_k < 1 and POLY or POINT data");
        return WOB_ERR_INVALID_ARG;
    }
    if (prob->ris < 0 || prob->ris > kMaxRis) {
        set_error("ris must be in [0, %d]", kMaxRis);
        return WOB_ERR_INVALID_ARG;
    }
    if (prob->side != 1 && prob->side != -1) {
        set_error("side must be +1 (interior) or -1 (exterior), got %d", prob->side);
        return WOB_ERR_INVALID_ARG;
    }
    if (prob->data_mode < WOB_DATA_VERTEX_P1 || prob->data_mode > WOB_DATA_POINT) {
        set_error("unknown data mode %d", prob->data_mode);
        return WOB_ERR_INVALID_ARG;
    }
    if (prob->data_mode == WOB_DATA_VERTEX_P1 && !prob->vertex_data) {
        set_error("vertex_data is NULL in WOB_DATA_VERTEX_P1 mode");
        return WOB_ERR_INVALID_ARG;
    }
    if (!std::isfinite(prob->alpha) || !(prob->tau >= 0.0f)) {
        set_error("alpha must be finite and tau >= 0");
        return WOB_ERR_INVALID_ARG;
    }
    return WOB_OK;
}

int check_sizes(int64_t Q, int64_t walk_begin, int32_t walks, int32_t max_len)
{
    if (Q < 0 || Q > (int64_t)UINT32_MAX) {
        set_error("Q = %lld outside [0, 2^32)", (long long)Q);
        return WOB_ERR_INVALID_ARG;
    }
    if (walks < 1 || walk_begin < 0 || walk_begin + walks > (int64_t)UINT32_MAX + 1) {
        set_error("walk range [%lld, %lld) invalid", (long long)walk_begin,
                  (long long)(walk_begin + walks));
        return WOB_ERR_INVALID_ARG;
    }
    if (max_len < 1 || max_len > kMaxLen) {
        set_error("max_len = %d outside [1, %d]", max_len, kMaxLen);
        return WOB_ERR_INVALID_ARG;
    }
    return WOB_OK;
}

void fill_params(WalkParams& p, const wob_problem* prob, const float* queries,
                 const int32_t* query_prim, int64_t Q, int64_t walk_begin, int32_t walks,
                 int32_t max_len, uint64_t seed)
{
    memset(&p, 0, sizeof(p));
    const BvhDev& b = prob->bvh->d;
    const MeshDev& m = *b.mesh;
    p.nodes = b.wnodes;
    p.tv = b.tv;
    p.inv_order = b.inv_order;
    p.iter_limit = prob->iter_limit > 0 ? prob->iter_limit : (int)(4 * b.n_wide + 64);
    p.verts = m.verts;
    p.verts_d = m.verts_d;
    p.tris = m.tris;
    p.tri_n = m.tri_n;
    p.tri_f = m.tri_f;
    p.cdf = m.cdf;
    p.guide = m.guide;
    p.guide_bits = m.guide_bits;
    p.T = m.T;
    p.area = m.area;
    p.L = m.L;
    p.kind = prob->kind;
    p.bc_type = prob->kind == WOB_MIXED_SL ? prob->bc_type : nullptr;
    p.kmix = prob->k_mix;
    p.pk = prob->p_k;
    p.ris = prob->ris;
    p.phi = prob->side;
    p.alpha = prob->alpha;
    p.data.mode = prob->data_mode;
    p.data.vdata = prob->vertex_data;
    p.data.tris = m.tris;
    for (int i = 0; i < 10; ++i) p.data.poly[i] = prob->poly[i];
    for (int i = 0; i < 3; ++i) p.data.x0[i] = prob->x0[i];
    p.data.scale = prob->scale;
    p.key0 = (uint32_t)seed ^ prob->problem;
    p.key1 = (uint32_t)(seed >> 32);
    p.queries = queries;
    p.query_prim = query_prim;
    p.Q = Q;
    p.N = walks;
    p.M = max_len;
    p.tpq = (walks + 31) / 32;
    p.walk_begin = walk_begin;
    p.q_base = 0;
    const float tau = prob->tau > 0.0f ? prob->tau : kDefaultTau;
    p.tauL = (float)(tau * m.L);
    p.edge_thr_L = (float)((double)kRareMargin * kFlagMargin * tau * m.L * m.max_edge);
    p.graze = kGraze;
}

namespace {

// Run the walks of one problem into the partials p.part (and p.per_walk, if set).
int run_walks(WalkParams& p, const wob_debug_out* dbg, bool counted, cudaStream_t s,
              int* err_dev)
{
    p.error_word = err_dev;
    if (dbg) {
        p.walk_flag = dbg->walk_flag;
        p.line_m = dbg->line_m;
        p.line_prim = dbg->line_prim;
        p.line_flag = dbg->line_flag;
    }
    if (p.kind == WOB_DIRICHLET_DL) return launch_dl_walks(p, counted, dbg != nullptr, s);
    if (p.kind == WOB_NEUMANN_DIRECT) return launch_nd_walks(p, dbg != nullptr, s);
    return launch_sl_walks(p, dbg != nullptr, s);
}

// Launch control words: traversal check word and the walk-tile counter.
struct Control {
    int err;
    int pad;
    unsigned long long next_tile;
};

struct Scratch {
    double* per_walk = nullptr;  // per-walk values or (sum, sum of squares) partials
    Control* err = nullptr;
    unsigned long long* counters = nullptr;
    cudaStream_t s = nullptr;
    ~Scratch()
    {
        if (per_walk) cudaFreeAsync(per_walk, s);
        if (err) cudaFreeAsync(err, s);
        if (counters) cudaFreeAsync(counters, s);
    }
};

int solve_common(const wob_problem* prob, const float* queries, const int32_t* query_prim,
                 int64_t Q, int64_t walk_begin, int32_t walks, int32_t max_len, uint64_t seed,
                 double* est, double* var, double* sum, double* sumsq,
                 const wob_debug_out* dbg, wob_stats* stats, cudaStream_t s,
                 bool density = false)
{
    WOB_TRY(check_problem(prob));
    WOB_TRY(check_sizes(Q, walk_begin, walks, max_len));
    if (Q == 0) return WOB_OK;
    if (!queries) {
        set_error("queries is NULL");
        return WOB_ERR_INVALID_ARG;
    }
    if (density && (prob->kind != WOB_DIRICHLET_DL || !query_prim)) {
        set_error("density walks need WOB_DIRICHLET_DL and query_prim");
        return WOB_ERR_INVALID_ARG;
    }
    if (!density && prob->kind == WOB_DIRICHLET_DL && query_prim) {
        set_error("query_prim must be NULL for WOB_DIRICHLET_DL (the solution on the "
                  "boundary is the Dirichlet data)");
        return WOB_ERR_UNSUPPORTED;
    }
    WalkParams p;
    fill_params(p, prob, queries, query_prim, Q, walk_begin, walks, max_len, seed);
    Scratch sc;
    sc.s = s;
    // (sum, sum of squares) per query and block of 32 walks
    const size_t part_bytes = (size_t)Q * p.tpq * 2 * sizeof(double);
    WOB_CUDA_TRY(cudaMallocAsync((void**)&sc.per_walk, part_bytes, s));
    WOB_CUDA_TRY(cudaMemsetAsync(sc.per_walk, 0, part_bytes, s));
    p.part = sc.per_walk;
    p.per_walk = dbg ? dbg->per_walk : nullptr;
    WOB_CUDA_TRY(cudaMallocAsync((void**)&sc.err, sizeof(Control), s));
    WOB_CUDA_TRY(cudaMemsetAsync(sc.err, 0, sizeof(Control), s));
    p.tile_counter = &sc.err->next_tile;
    if (stats) {
        WOB_CUDA_TRY(cudaMallocAsync((void**)&sc.counters, 5 * sizeof(unsigned long long), s));
        WOB_CUDA_TRY(cudaMemsetAsync(sc.counters, 0, 5 * sizeof(unsigned long long), s));
        p.counters = sc.counters;
    }
    WOB_TRY(run_walks(p, dbg, stats != nullptr, s, &sc.err->err));
    WOB_TRY(launch_reduce_part(p.part, Q, walks, p.tpq, est, var, sum, sumsq, s, &sc.err->err));
    if (stats) {
        unsigned long long h[5];
        int herr = 0;
        WOB_CUDA_TRY(cudaMemcpyAsync(h, sc.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
        WOB_CUDA_TRY(cudaMemcpyAsync(&herr, &sc.err->err, sizeof(int), cudaMemcpyDeviceToHost, s));
        WOB_CUDA_TRY(cudaStreamSynchronize(s));
        stats->lines = (int64_t)h[0];
        stats->node_visits = (int64_t)h[1];
        stats->tri_tests = (int64_t)h[2];
        stats->hits = (int64_t)h[3];
        stats->flagged = (int64_t)h[4];
        if (herr) {
            set_error("traversal check failed (%s)", herr & 2 ? "iteration bound" : "stack overflow");
            return WOB_ERR_DEVICE_CHECK;
        }
    }
    return WOB_OK;
}

}  // namespace
}  // namespace wob

using namespace wob;

extern "C" {

int wob_version(void) { return 100; }

const char* wob_last_error(void) { return wob::g_error.c_str(); }

int wob_build_mesh(const float* verts, int64_t V, const int32_t* tris, int64_t T,
                   int on_device, void* stream, wob_mesh* out)
{
    clear_error();
    if (!verts || !tris || !out || V < 3 || T < 1 || T > kMaxTriangles ||
        V > (int64_t)INT32_MAX) {
        set_error("wob_build_mesh: invalid arguments (V=%lld, T=%lld)", (long long)V,
                  (long long)T);
        return WOB_ERR_INVALID_ARG;
    }
    *out = nullptr;
    wob_mesh m = new (std::nothrow) wob_mesh_s();
    if (!m) {
        set_error("host allocation failed");
        return WOB_ERR_OOM;
    }
    const int rc = build_mesh_impl(verts, V, tris, T, on_device != 0, (cudaStream_t)stream, m->d);
    if (rc != WOB_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        free_mesh(m->d);
        delete m;
        return rc;
    }
    *out = m;
    return WOB_OK;
}

int wob_mesh_get_info(wob_mesh m, wob_mesh_info* out)
{
    clear_error();
    if (!m || !out) {
        set_error("NULL argument");
        return WOB_ERR_INVALID_ARG;
    }
    out->V = m->d.V;
    out->T = m->d.T;
    for (int c = 0; c < 3; ++c) {
        out->bbox_lo[c] = m->d.lo[c];
        out->bbox_hi[c] = m->d.hi[c];
    }
    out->L = m->d.L;
    out->area = m->d.area;
    out->volume = m->d.volume;
    out->max_edge = m->d.max_edge;
    return WOB_OK;
}

void wob_destroy_mesh(wob_mesh m)
{
    if (!m) return;
    free_mesh(m->d);
    delete m;
}

int wob_build_bvh(wob_mesh m, const wob_bvh_params* p, void* stream, wob_bvh* out)
{
    clear_error();
    if (!m || !out) {
        set_error("NULL argument");
        return WOB_ERR_INVALID_ARG;
    }
    int leaf = p && p->leaf_size ? p->leaf_size : 1;
    if (leaf < 1 || leaf > 8) {
        set_error("leaf_size %d outside [1, 8]", leaf);
        return WOB_ERR_INVALID_ARG;
    }
    *out = nullptr;
    wob_bvh b = new (std::nothrow) wob_bvh_s();
    if (!b) {
        set_error("host allocation failed");
        return WOB_ERR_OOM;
    }
    const int rc = build_bvh_impl(m->d, leaf, (cudaStream_t)stream, b->d);
    if (rc != WOB_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        free_bvh(b->d);
        delete b;
        return rc;
    }
    *out = b;
    return WOB_OK;
}

int wob_bvh_get_info(wob_bvh b, wob_bvh_info* out)
{
    clear_error();
    if (!b || !out) {
        set_error("NULL argument");
        return WOB_ERR_INVALID_ARG;
    }
    out->nodes = b->d.n_wide;
    out->leaves = b->d.leaves;
    out->depth = b->d.wide_levels - 1;
    out->leaf_size = b->d.leaf_size;
    out->bytes = b->d.n_wide * 96 + b->d.mesh->T * 48;
    return WOB_OK;
}

void wob_destroy_bvh(wob_bvh b)
{
    if (!b) return;
    free_bvh(b->d);
    delete b;
}

int wob_solve(const wob_problem* prob, const float* queries, const int32_t* query_prim,
              int64_t Q, int32_t walks, int32_t max_len, uint64_t seed, double* est,
              double* var, void* stream)
{
    clear_error();
    if (walks < 2) {
        set_error("walks must be >= 2 for a sample variance");
        return WOB_ERR_INVALID_ARG;
    }
    if (Q > 0 && (!est || !var)) {
        set_error("est/var is NULL");
        return WOB_ERR_INVALID_ARG;
    }
    return solve_common(prob, queries, query_prim, Q, 0, walks, max_len, seed, est, var,
                        nullptr, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}

int wob_solve_density(const wob_problem* prob, const float* points, const int32_t* prims,
                      int64_t Q, int32_t walks, int32_t max_len, uint64_t seed, double* est,
                      double* var, void* stream)
{
    clear_error();
    if (walks < 2 || (Q > 0 && (!est || !var || !prims))) {
        set_error("wob_solve_density: walks < 2 or NULL est/var/prims");
        return WOB_ERR_INVALID_ARG;
    }
    return solve_common(prob, points, prims, Q, 0, walks, max_len, seed, est, var, nullptr,
                        nullptr, nullptr, nullptr, (cudaStream_t)stream, true);
}

int wob_solve_range(const wob_problem* prob, const float* queries, const int32_t* query_prim,
                    int64_t Q, int64_t walk_begin, int32_t walks, int32_t max_len,
                    uint64_t seed, double* sum, double* sumsq, void* stream)
{
    clear_error();
    if (Q > 0 && (!sum || !sumsq)) {
        set_error("sum/sumsq is NULL");
        return WOB_ERR_INVALID_ARG;
    }
    return solve_common(prob, queries, query_prim, Q, walk_begin, walks, max_len, seed,
                        nullptr, nullptr, sum, sumsq, nullptr, nullptr, (cudaStream_t)stream);
}

int wob_solve_debug(const wob_problem* prob, const float* queries, const int32_t* query_prim,
                    int64_t Q, int32_t walks, int32_t max_len, uint64_t seed, double* est,
                    double* var, const wob_debug_out* dbg, void* stream)
{
    clear_error();
    if (!dbg) {
        set_error("dbg is NULL");
        return WOB_ERR_INVALID_ARG;
    }
    if (walks < 2 || (Q > 0 && (!est || !var))) {
        set_error("walks < 2 or est/var NULL");
        return WOB_ERR_INVALID_ARG;
    }
    const bool density = prob && prob->kind == WOB_DIRICHLET_DL && query_prim;
    return solve_common(prob, queries, query_prim, Q, 0, walks, max_len, seed, est, var,
                        nullptr, nullptr, dbg, nullptr, (cudaStream_t)stream, density);
}

int wob_solve_grad(const wob_problem* prob, const float* queries, int64_t Q, int32_t walks,
                   int32_t max_len, uint64_t seed, double* est, double* var, double* grad_est,
                   double* grad_var, double* per_walk_grad, void* stream)
{
    clear_error();
    WOB_TRY(check_problem(prob));
    WOB_TRY(check_sizes(Q, 0, walks, max_len));
    if (prob->kind != WOB_DIRICHLET_DL) {
        set_error("wob_solve_grad: gradients are implemented for WOB_DIRICHLET_DL");
        return WOB_ERR_UNSUPPORTED;
    }
    if (walks < 2 || (Q > 0 && (!queries || !est || !var || !grad_est || !grad_var))) {
        set_error("wob_solve_grad: walks < 2 or a NULL output");
        return WOB_ERR_INVALID_ARG;
    }
    if (Q == 0) return WOB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    WalkParams p;
    fill_params(p, prob, queries, nullptr, Q, 0, walks, max_len, seed);
    Scratch sc;
    sc.s = s;
    const int64_t W = Q * (int64_t)walks;
    WOB_CUDA_TRY(cudaMallocAsync((void**)&sc.per_walk, W * sizeof(double), s));
    double* g = per_walk_grad;
    double* g_owned = nullptr;
    if (!g) {
        WOB_CUDA_TRY(cudaMallocAsync((void**)&g_owned, 3 * W * sizeof(double), s));
        g = g_owned;
    }
    WOB_CUDA_TRY(cudaMallocAsync((void**)&sc.err, sizeof(Control), s));
    WOB_CUDA_TRY(cudaMemsetAsync(sc.err, 0, sizeof(Control), s));
    p.tile_counter = &sc.err->next_tile;
    p.per_walk = sc.per_walk;
    p.per_walk_grad = g;
    int rc = run_walks(p, nullptr, false, s, &sc.err->err);
    if (rc == WOB_OK) rc = launch_reduce(sc.per_walk, Q, walks, est, var, s, &sc.err->err);
    for (int c = 0; c < 3 && rc == WOB_OK; ++c)
        rc = launch_reduce(g + c * W, Q, walks, grad_est + c * Q, grad_var + c * Q, s,
                           &sc.err->err);
    if (g_owned) cudaFreeAsync(g_owned, s);
    return rc;
}

int wob_solve_forward(const wob_problem* prob, const float* queries, int64_t Q, int32_t paths,
                      int32_t max_len, uint64_t seed, int32_t start_mode, float beta,
                      double* est, double* var, double* zpos, double* zw, uint8_t* path_flag,
                      void* stream)
{
    clear_error();
    WOB_TRY(check_problem(prob));
    if (prob->kind != WOB_NEUMANN_SL) {
        set_error("wob_solve_forward: forward paths are implemented for WOB_NEUMANN_SL");
        return WOB_ERR_UNSUPPORTED;
    }
    if (paths < 2 || max_len < 1 || max_len > 1024 || (start_mode != 0 && start_mode != 1) ||
        !(beta > 0.0f) || Q < 0 || (Q > 0 && (!queries || !est || !var)) ||
        (int64_t)paths * max_len > INT32_MAX) {
        set_error("wob_solve_forward: invalid arguments (paths >= 2, 1 <= max_len <= 1024, "
                  "start_mode 0 or 1, beta > 0)");
        return WOB_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    WalkParams p;
    fill_params(p, prob, queries, nullptr, Q, 0, paths, max_len, seed);
    Scratch sc;
    sc.s = s;
    const int64_t R = (int64_t)paths * max_len;
    WOB_CUDA_TRY(cudaMallocAsync((void**)&sc.err, sizeof(Control), s));  // freed by sc
    WOB_CUDA_TRY(cudaMemsetAsync(sc.err, 0, sizeof(Control), s));
    p.error_word = &sc.err->err;
    double* zp = zpos;
    double* w = zw;
    double* own = nullptr;
    if (!zp || !w) {
        WOB_CUDA_TRY(cudaMallocAsync((void**)&own, 4 * R * sizeof(double), s));
        if (!zp) zp = own;
        if (!w) w = own + 3 * R;
    }
    int rc = launch_forward(p, paths, start_mode, (double)beta, queries, Q, zp, w, path_flag, est,
                            var, s);
    if (own) cudaFreeAsync(own, s);
    return rc;
}

int wob_solve_counted(const wob_problem* prob, const float* queries, const int32_t* query_prim,
                      int64_t Q, int32_t walks, int32_t max_len, uint64_t seed, double* est,
                      double* var, wob_stats* stats, void* stream)
{
    clear_error();
    if (!stats || walks < 2 || (Q > 0 && (!est || !var))) {
        set_error("stats NULL, walks < 2 or est/var NULL");
        return WOB_ERR_INVALID_ARG;
    }
    memset(stats, 0, sizeof(*stats));
    const int rc = solve_common(prob, queries, query_prim, Q, 0, walks, max_len, seed, est, var,
                                nullptr, nullptr, nullptr, stats, (cudaStream_t)stream);
    if (rc == WOB_OK) wob::g_last_stats = *stats;
    return rc;
}

int wob_get_stats(wob_stats* out)
{
    clear_error();
    if (!out) {
        set_error("wob_get_stats: out is NULL");
        return WOB_ERR_INVALID_ARG;
    }
    *out = wob::g_last_stats;
    return WOB_OK;
}

int wob_solve_host(const wob_problem* prob, const float* queries_host,
                   const int32_t* query_prim_host, int64_t Q, int32_t walks, int32_t max_len,
                   uint64_t seed, double* est_host, double* var_host, void* stream)
{
    clear_error();
    if (walks < 2 || Q < 0 || (Q > 0 && (!queries_host || !est_host || !var_host))) {
        set_error("wob_solve_host: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    if (Q == 0) return WOB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // one device block: queries | query_prim | est | var
    const size_t qb = (size_t)Q * 3 * sizeof(float);
    const size_t pb = query_prim_host ? (size_t)Q * sizeof(int32_t) : 0;
    const size_t ob = (size_t)Q * sizeof(double);
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t total = align(qb) + align(pb) + 2 * align(ob);
    char* buf = nullptr;
    WOB_CUDA_TRY(cudaMallocAsync((void**)&buf, total, s));
    float* dq = (float*)buf;
    int32_t* dp = query_prim_host ? (int32_t*)(buf + align(qb)) : nullptr;
    double* de = (double*)(buf + align(qb) + align(pb));
    double* dv = (double*)(buf + align(qb) + align(pb) + align(ob));
    int rc = WOB_OK;
    if (cudaMemcpyAsync(dq, queries_host, qb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (dp && cudaMemcpyAsync(dp, query_prim_host, pb, cudaMemcpyHostToDevice, s) != cudaSuccess)) {
        set_error("host-to-device copy failed");
        rc = WOB_ERR_CUDA;
    }
    if (rc == WOB_OK)
        rc = solve_common(prob, dq, dp, Q, 0, walks, max_len, seed, de, dv, nullptr, nullptr,
                          nullptr, nullptr, s);
    if (rc == WOB_OK &&
        (cudaMemcpyAsync(est_host, de, ob, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaMemcpyAsync(var_host, dv, ob, cudaMemcpyDeviceToHost, s) != cudaSuccess)) {
        set_error("device-to-host copy failed");
        rc = WOB_ERR_CUDA;
    }
    cudaFreeAsync(buf, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (rc == WOB_OK && e != cudaSuccess) {
        set_error("wob_solve_host: %s", cudaGetErrorString(e));
        rc = WOB_ERR_CUDA;
    }
    return rc;
}

int wob_trace_lines(wob_bvh b, const double* origins, const double* dirs,
                    const int32_t* exclude, const uint32_t* keys, int64_t n, uint64_t seed,
                    uint32_t problem, float tau, int32_t* m, int32_t* sum_s, int32_t* prim,
                    int32_t* s, double* t, double* y, uint8_t* flag, void* stream)
{
    clear_error();
    if (!b || n < 0 || (n > 0 && (!origins || !dirs || !keys || !m))) {
        set_error("wob_trace_lines: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    if (n == 0) return WOB_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const MeshDev& md = *b->d.mesh;
    const float tu = tau > 0.0f ? tau : kDefaultTau;
    int* err = nullptr;
    WOB_CUDA_TRY(cudaMallocAsync((void**)&err, sizeof(int), st));
    WOB_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    int rc = launch_trace_lines(b->d, origins, dirs, exclude, keys, n, (uint32_t)seed ^ problem,
                                (uint32_t)(seed >> 32), (float)(tu * md.L),
                                (float)((double)kRareMargin * kFlagMargin * tu * md.L * md.max_edge),
                                m, sum_s, prim, s, t, y, flag, err, st);
    int herr = 0;
    cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(err, st);
    WOB_CUDA_TRY(cudaStreamSynchronize(st));
    if (rc == WOB_OK && herr) {
        set_error("traversal stack overflow");
        rc = WOB_ERR_DEVICE_CHECK;
    }
    return rc;
}

int wob_line_axes(uint64_t seed, uint32_t problem, const uint32_t* qws, int64_t n, double* d,
                  void* stream)
{
    clear_error();
    if (n < 0 || (n > 0 && (!qws || !d))) {
        set_error("wob_line_axes: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    if (n == 0) return WOB_OK;
    return launch_line_axes((uint32_t)seed ^ problem, (uint32_t)(seed >> 32), qws, n, d,
                            (cudaStream_t)stream);
}

int wob_probe_l2_read(const void* buf, int64_t bytes, int32_t passes, float* out, void* stream)
{
    clear_error();
    if (!buf || !out || bytes < 16 || bytes % 16 != 0 || ((uintptr_t)buf & 15) != 0 ||
        passes < 1) {
        set_error("wob_probe_l2_read: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    return launch_probe_read((const float4*)buf, bytes / 16, passes, out, (cudaStream_t)stream);
}

int wob_philox4x32_10(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out,
                      void* stream)
{
    clear_error();
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) {
        set_error("wob_philox4x32_10: invalid arguments");
        return WOB_ERR_INVALID_ARG;
    }
    if (n == 0) return WOB_OK;
    return launch_philox(ctr, key, n, out, (cudaStream_t)stream);
}

}  // extern "C"
