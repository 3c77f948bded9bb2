// wob_host.h -- host-side helpers: error reporting, CUDA checks and the
// internal entry points implemented by the library's .cu files.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <cuda_runtime.h>

#include "wob_internal.h"

namespace wob {

void set_error(const char* fmt, ...);
void clear_error();

#define WOB_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess) {                                                        \
            ::wob::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e),    \
                             __FILE__, __LINE__);                                       \
            return _e == cudaErrorMemoryAllocation ? WOB_ERR_OOM : WOB_ERR_CUDA;        \
        }                                                                               \
    } while (0)

#define WOB_TRY(expr)                 \
    do {                              \
        int _rc = (expr);             \
        if (_rc != WOB_OK) return _rc; \
    } while (0)

// api.cu: argument checks and the launch parameter block of one solve.
int check_problem(const wob_problem* prob);
int check_sizes(int64_t Q, int64_t walk_begin, int32_t walks, int32_t max_len);
void fill_params(WalkParams& p, const wob_problem* prob, const float* queries,
                 const int32_t* query_prim, int64_t Q, int64_t walk_begin, int32_t walks,
                 int32_t max_len, uint64_t seed);

// Persistent-grid size: SM count x resident blocks of `kernel` at `threads`.
int grid_for(const void* kernel, int threads, size_t smem, int64_t work_items);

// mesh.cu
int build_mesh_impl(const float* verts, int64_t V, const int32_t* tris, int64_t T,
                    bool on_device, cudaStream_t s, MeshDev& m);
void free_mesh(MeshDev& m);
template <typename T>
int inclusive_scan(const T* in, T* out, int64_t n, cudaStream_t s);

// bvh.cu
int build_bvh_impl(MeshDev& m, int leaf_size, cudaStream_t s, BvhDev& b);
void free_bvh(BvhDev& b);

// walk.cu
int launch_dl_walks(const WalkParams& p, bool counted, bool debug, cudaStream_t s);
int launch_sl_walks(const WalkParams& p, bool debug, cudaStream_t s);
int launch_nd_walks(const WalkParams& p, bool debug, cudaStream_t s);
// forward single-layer Neumann paths and their connection to the queries
// streaming read probe (wob_probe_l2_read)
int launch_probe_read(const float4* buf, int64_t n, int passes, float* out, cudaStream_t s);
int launch_forward(const WalkParams& p, int64_t n_paths, int start_mode, double beta,
                   const float* queries, int64_t Q, double* zpos, double* zw, uint8_t* flags,
                   double* est, double* var, cudaStream_t s);
// err: the solve's device check word (NULL: none); when set, the outputs are NaN
int launch_reduce(const double* per_walk, int64_t Q, int32_t N, double* est, double* var,
                  cudaStream_t s, const int* err);
// From the (sum, sum of squares) partials of the walk kernels (Q x tpq x 2):
// est / var (may be NULL) and, accumulated, sum / sumsq (may be NULL).
int launch_reduce_part(const double* part, int64_t Q, int32_t N, int32_t tpq, double* est,
                       double* var, double* sum, double* sumsq, cudaStream_t s, const int* err);
int launch_reduce_accum(const double* per_walk, int64_t Q, int32_t N, double* sum,
                        double* sumsq, cudaStream_t s, const int* err);
int launch_trace_lines(const BvhDev& b, const double* o, const double* d, const int32_t* exclude,
                       const uint32_t* keys, int64_t n, uint32_t key0, uint32_t key1,
                       float tauL, float edge_thr_L, int32_t* m, int32_t* sum_s, int32_t* prim,
                       int32_t* s_out, double* t, double* y, uint8_t* flag, int* error_word,
                       cudaStream_t s);
int launch_line_axes(uint32_t key0, uint32_t key1, const uint32_t* qws, int64_t n, double* d,
                     cudaStream_t s);
int launch_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out,
                  cudaStream_t s);

// mlp.cu: the control variate's network
int mlp_forward(const float* params, const float* x, int64_t n, float* out, cudaStream_t s,
                int stride);  // point r at x[stride * r .. + 2]
int mlp_train_step(float* params, float* m, float* v, const float* x, const float* target,
                   int64_t n, float lr, int step, float* grad_out, float* loss_out,
                   cudaStream_t s);
// floats of workspace a training step on n samples needs
int64_t mlp_train_workspace(int64_t n);
// Step number and learning rate of graph-replayed training steps, in device
// memory: the training kernel advances the step, Adam reads both.
struct TrainCtl {
    int step;
    float lr;
};
int mlp_train_step_ws(float* params, float* m, float* v, const float* x, const float* target,
                      int64_t n, float lr, int step, float* grad_out, float* loss_out, float* ws,
                      cudaStream_t s, TrainCtl* ctl = nullptr);
int train_ctl_set(TrainCtl* ctl, int step, float lr, bool set_step, cudaStream_t s);
int mlp_train_prepare();

}  // namespace wob
