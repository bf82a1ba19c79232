// C ABI entry points (declared in include/gofd.h).  Argument checks, the
// handle's life cycle, and translation of internal errors into gofd_status.
#include <chrono>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "gofd_internal.cuh"

namespace {

thread_local std::string g_build_error;

gofd_status record(gofd_problem* p, const gofd::Error& e) {
    if (p) p->last_error = e.msg;
    else g_build_error = e.msg;
    return e.code;
}

#define GOFD_API_BODY(handle, ...)                                                        \
    try {                                                                                 \
        __VA_ARGS__;                                                                      \
        return GOFD_OK;                                                                   \
    } catch (const gofd::Error& e) {                                                      \
        return record(handle, e);                                                         \
    } catch (const std::bad_alloc&) {                                                     \
        return record(handle, gofd::Error{GOFD_E_NOMEM, "host allocation failed"});      \
    } catch (...) {                                                                       \
        return record(handle, gofd::Error{GOFD_E_CUDA, "unexpected internal error"});    \
    }

int64_t default_filon_M(int d, int n, int levels) {
    int64_t M = (d == 3) ? (1 << 11) : (1 << 14);
    while ((M >> (levels - 1)) < n) M *= 2;
    return M;
}

int circulant_length(int n) {
    int P = 1;
    while (P < 2 * n - 2) P *= 2;
    return P < 32 ? 32 : P;
}

}  // namespace

namespace {

void release_all(gofd_problem* p) {
    gofd::free_batch(p);
    gofd::free_adjoint(p);
    gofd::free_workspace(p);
    gofd::free_precond(p);
    if (p->setup_stream) cudaStreamDestroy(p->setup_stream);
    p->setup_stream = nullptr;
}

}  // namespace

extern "C" {

gofd_status gofd_build(int d, const double* vertices, int64_t n_v, const int32_t* simplices, int64_t n_e,
                       double alpha, double h, const double* box_lo, const double* box_hi,
                       const gofd_options* opt, gofd_problem** out) {
    if (out) *out = nullptr;
    gofd_problem* p = nullptr;
    try {
        auto t0 = std::chrono::steady_clock::now();
        using gofd::fail;
        if (!out) fail(GOFD_E_ARG, "out is NULL");
        if (d < 1 || d > 3) fail(GOFD_E_ARG, "d must be 1, 2 or 3");
        if (!vertices || !simplices || !box_lo || !box_hi) fail(GOFD_E_ARG, "NULL input array");
        if (n_v < d + 1 || n_e < 1) fail(GOFD_E_ARG, "need at least one simplex and d+1 vertices");
        if (n_v >= (int64_t)INT32_MAX || n_e >= (int64_t)INT32_MAX) fail(GOFD_E_ARG, "mesh too large");
        if (d == 3 && n_v >= (int64_t)1 << 21) fail(GOFD_E_ARG, "3D meshes are limited to 2^21 vertices");
        if (!(alpha > 0.0 && alpha <= 2.0)) fail(GOFD_E_ARG, "alpha must be in (0, 2]");
        if (!(h > 0.0) || !std::isfinite(h)) fail(GOFD_E_ARG, "h must be positive and finite");
        int n[3] = {1, 1, 1};
        for (int i = 0; i < d; ++i) {
            if (!(box_hi[i] > box_lo[i])) fail(GOFD_E_GRID, "box_hi must exceed box_lo");
            const double q = (box_hi[i] - box_lo[i]) / h;
            const double r = std::nearbyint(q);
            if (std::fabs(q - r) > 1e-9 * std::fmax(1.0, q) || r < 1 || r > 65535)
                fail(GOFD_E_GRID, "(hi-lo)/h must be an integer in [1, 65535] on every axis");
            n[i] = (int)r + 1;
        }
        for (int i = 1; i < d; ++i)
            if (n[i] != n[0]) fail(GOFD_E_GRID, "the grid must have the same node count on every axis");
        if (n[0] > 4097) fail(GOFD_E_GRID, "at most 4097 grid nodes per axis (circulant length <= 8192)");
        if (d == 3 && n[0] > 513) fail(GOFD_E_GRID, "3D: at most 513 grid nodes per axis (circulant length <= 1024)");
        int64_t ngrid = 1;
        for (int i = 0; i < d; ++i) ngrid *= n[i];
        if (ngrid > (int64_t)INT32_MAX) fail(GOFD_E_GRID, "more than 2^31-1 grid nodes");
        for (int64_t v = 0; v < n_v; ++v)
            for (int i = 0; i < d; ++i) {
                const double x = vertices[v * d + i];
                if (!(x >= box_lo[i] && x <= box_hi[i])) fail(GOFD_E_OUTSIDE_BOX, "a mesh vertex lies outside the box");
            }
        for (int64_t e = 0; e < n_e * (d + 1); ++e)
            if (simplices[e] < 0 || simplices[e] >= n_v) fail(GOFD_E_ARG, "simplex vertex index out of range");
        if (ngrid < n_v) fail(GOFD_E_TOO_FEW_GRID_NODES, "fewer grid nodes than mesh vertices (Remark 3.2)");

        int dev = 0;
        GOFD_CUDA_TRY(cudaGetDevice(&dev));
        cudaDeviceProp prop;
        GOFD_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
        if (!(prop.major == 10 && prop.minor == 3))
            fail(GOFD_E_CUDA, "this library is built for compute capability 10.3 (sm_103a) only");

        p = new gofd_problem();
        p->device = dev;
        GOFD_CUDA_TRY(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev));
        p->d = d;
        p->nv = n_v;
        p->ne = n_e;
        p->alpha = alpha;
        p->s = alpha / 2.0;
        p->h = h;
        for (int i = 0; i < 3; ++i) {
            p->lo[i] = i < d ? box_lo[i] : 0.0;
            p->hi[i] = i < d ? box_hi[i] : 0.0;
            p->n[i] = n[i];
        }
        p->ngrid = ngrid;
        p->nlines = ngrid / n[0];
        if (opt) p->opt = *opt;
        p->rich_levels = p->opt.richardson_levels > 0 ? p->opt.richardson_levels : 4;
        if (p->rich_levels > 8) fail(GOFD_E_ARG, "richardson_levels must be at most 8");
        if (p->opt.filon_M > 0) {
            const int64_t M = p->opt.filon_M;
            if ((M & (M - 1)) != 0 || (M >> p->rich_levels) < 1 || (M >> (p->rich_levels - 1)) < n[0])
                fail(GOFD_E_ARG, "filon_M must be a power of two with M/2^(levels-1) >= n");
            p->filon_M = M;
        } else {
            p->filon_M = default_filon_M(d, n[0], p->rich_levels);
        }
        p->P = circulant_length(n[0]);
        GOFD_CUDA_TRY(cudaStreamCreateWithFlags(&p->setup_stream, cudaStreamNonBlocking));

        gofd::setup_mesh(p, vertices, simplices);
        gofd::setup_coefficients(p);
        gofd::setup_apply(p);
        gofd::setup_precond(p);
        GOFD_CUDA_TRY(cudaStreamSynchronize(p->setup_stream));
        auto t1 = std::chrono::steady_clock::now();
        p->t_setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        *out = p;
        return GOFD_OK;
    } catch (const gofd::Error& e) {
        g_build_error = e.msg;
        if (p) {
            release_all(p);
            delete p;
        }
        return e.code;
    } catch (const std::bad_alloc&) {
        g_build_error = "host allocation failed";
        if (p) {
            release_all(p);
            delete p;
        }
        return GOFD_E_NOMEM;
    }
}

void gofd_destroy(gofd_problem* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    release_all(p);
    delete p;
}

const char* gofd_last_error(const gofd_problem* p) {
    if (p) return p->last_error.c_str();
    return g_build_error.c_str();
}

gofd_status gofd_apply_interior(gofd_problem* p, gofd_precision prec, const void* x_dev, void* y_dev,
                                void* stream) {
    if (!p) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        if (!x_dev || !y_dev) gofd::fail(GOFD_E_ARG, "NULL vector");
        if (prec != GOFD_FP64 && prec != GOFD_FP32 && prec != GOFD_FP64_DF) gofd::fail(GOFD_E_ARG, "bad precision");
        if (prec == GOFD_FP64_DF) {
            if (p->d < 2) gofd::fail(GOFD_E_ARG, "GOFD_FP64_DF is supported in 2D and 3D");
            gofd::apply_interior_df(p, (const double*)x_dev, (double*)y_dev, (cudaStream_t)stream);
        } else {
            gofd::apply_interior(p, prec == GOFD_FP64, x_dev, y_dev, (cudaStream_t)stream);
        }
    })
}

gofd_status gofd_precond_apply(gofd_problem* p, gofd_precision prec, const void* r_dev, void* z_dev, void* stream) {
    if (!p) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        if (!r_dev || !z_dev) gofd::fail(GOFD_E_ARG, "NULL vector");
        if (prec != GOFD_FP64 && prec != GOFD_FP32) gofd::fail(GOFD_E_ARG, "bad precision");
        if (r_dev == z_dev) gofd::fail(GOFD_E_ARG, "r and z must not alias");
        const size_t b = prec == GOFD_FP64 ? 8 : 4;
        gofd::precond_apply(p, prec == GOFD_FP64, r_dev, z_dev, (cudaStream_t)stream);
        GOFD_CUDA_TRY(cudaMemsetAsync(static_cast<char*>(z_dev) + b * p->nint, 0, b, (cudaStream_t)stream));
        gofd::precond_check(p, (cudaStream_t)stream);
    })
}

gofd_status gofd_apply_interior_batch(gofd_problem* p, gofd_precision prec, int nb, const void* x_dev, int64_t ld,
                                      void* y_dev, void* stream) {
    if (!p) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        if (!x_dev || !y_dev) gofd::fail(GOFD_E_ARG, "NULL vector");
        if (prec != GOFD_FP64 && prec != GOFD_FP32) gofd::fail(GOFD_E_ARG, "bad precision");
        if (nb < 1 || nb > 4096) gofd::fail(GOFD_E_ARG, "nb must be in [1, 4096]");
        if (ld < p->nint + 1) gofd::fail(GOFD_E_ARG, "ld must be >= n_interior + 1");
        gofd::apply_batch(p, prec == GOFD_FP64, x_dev, y_dev, nb, ld, (cudaStream_t)stream);
    })
}

gofd_status gofd_apply_interior_profiled(gofd_problem* p, gofd_precision prec, const void* x_dev, void* y_dev,
                                         void* stream, float* stage_ms, const char** stage_names, int cap,
                                         int* n_stages) {
    if (!p || !stage_ms || !n_stages) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        if (!x_dev || !y_dev) gofd::fail(GOFD_E_ARG, "NULL vector");
        *n_stages = gofd::apply_interior_profiled(p, prec == GOFD_FP64, x_dev, y_dev, (cudaStream_t)stream,
                                                  stage_ms, stage_names, cap);
    })
}

gofd_status gofd_apply(gofd_problem* p, gofd_op op, gofd_precision prec, const void* u_dev, void* y_dev,
                       void* stream) {
    if (!p) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        if (!u_dev || !y_dev) gofd::fail(GOFD_E_ARG, "NULL vector");
        if (prec != GOFD_FP64 && prec != GOFD_FP32) gofd::fail(GOFD_E_ARG, "bad precision");
        if (op != GOFD_OP_STIFFNESS && op != GOFD_OP_FRACLAP) gofd::fail(GOFD_E_ARG, "bad operator");
        cudaStream_t st = (cudaStream_t)stream;
        const bool f64 = prec == GOFD_FP64;
        gofd::compact_vertex(p, f64, u_dev, p->xin.ptr, st);
        gofd::apply_interior(p, f64, p->xin.ptr, p->yout.ptr, st);
        const double sc = (op == GOFD_OP_FRACLAP) ? std::pow(p->h, -2.0 * p->s) : 0.0;
        gofd::expand_interior(p, f64, p->yout.ptr, y_dev, sc, st);
    })
}

gofd_status gofd_apply_host(gofd_problem* p, gofd_op op, gofd_precision prec, const void* u_host, void* y_host,
                            void* stream) {
    if (!p) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        if (!u_host || !y_host) gofd::fail(GOFD_E_ARG, "NULL vector");
        cudaStream_t st = (cudaStream_t)stream;
        const size_t bytes = (prec == GOFD_FP64 ? 8 : 4) * (size_t)p->nv;
        // pinned host buffers are mapped into the device's address space: the
        // compaction kernel reads u and the expansion kernel writes y there
        // directly (over the CPU-GPU link), with no staging copies
        cudaPointerAttributes au{}, ay{};
        const bool mapped = cudaPointerGetAttributes(&au, u_host) == cudaSuccess && au.type == cudaMemoryTypeHost &&
                            au.devicePointer && cudaPointerGetAttributes(&ay, y_host) == cudaSuccess &&
                            ay.type == cudaMemoryTypeHost && ay.devicePointer;
        cudaGetLastError();   // a pageable pointer is not an error here
        if (mapped) {
            gofd_status s = gofd_apply(p, op, prec, au.devicePointer, ay.devicePointer, stream);
            if (s != GOFD_OK) throw gofd::Error{s, p->last_error};
            GOFD_CUDA_TRY(cudaStreamSynchronize(st));
            return GOFD_OK;
        }
        // otherwise staging buffers, allocated on the first such call and kept by the handle
        if (p->stage_u.bytes < bytes) p->stage_u.alloc(bytes);
        if (p->stage_y.bytes < bytes) p->stage_y.alloc(bytes);
        gofd::DevBuf& u = p->stage_u;
        gofd::DevBuf& y = p->stage_y;
        GOFD_CUDA_TRY(cudaMemcpyAsync(u.ptr, u_host, bytes, cudaMemcpyHostToDevice, st));
        gofd_status s = gofd_apply(p, op, prec, u.ptr, y.ptr, stream);
        if (s != GOFD_OK) throw gofd::Error{s, p->last_error};
        GOFD_CUDA_TRY(cudaMemcpyAsync(y_host, y.ptr, bytes, cudaMemcpyDeviceToHost, st));
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    })
}

gofd_status gofd_solve(gofd_problem* p, gofd_solve_mode mode, gofd_rhs rhs, const double* f_dev, double tol,
                       int maxit, int init_zero, double* u_dev, gofd_solve_info* info, void* stream) {
    if (!p) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        if (!f_dev || !u_dev) gofd::fail(GOFD_E_ARG, "NULL vector");
        if (mode != GOFD_SOLVE_FP64 && mode != GOFD_SOLVE_MIXED) gofd::fail(GOFD_E_ARG, "bad mode");
        if (rhs != GOFD_RHS_GRID && rhs != GOFD_RHS_VERTEX) gofd::fail(GOFD_E_ARG, "bad rhs kind");
        if (!(tol > 0.0) || maxit < 1) gofd::fail(GOFD_E_ARG, "tol must be > 0 and maxit >= 1");
        gofd::solve(p, mode, rhs, f_dev, tol, maxit, init_zero != 0, u_dev, info, (cudaStream_t)stream);
    })
}

gofd_status gofd_adjoint(gofd_problem* p, gofd_solve_mode mode, const double* f_dev, const double* u_dev,
                         const double* g_dev, double tol, int maxit, double* grad_f_dev, double* grad_x_dev,
                         gofd_solve_info* info, void* stream) {
    if (!p) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        if (!f_dev || !u_dev || !g_dev || !grad_f_dev || !grad_x_dev) gofd::fail(GOFD_E_ARG, "NULL vector");
        if (mode != GOFD_SOLVE_FP64 && mode != GOFD_SOLVE_MIXED) gofd::fail(GOFD_E_ARG, "bad mode");
        if (!(tol > 0.0) || maxit < 1) gofd::fail(GOFD_E_ARG, "tol must be > 0 and maxit >= 1");
        gofd::adjoint(p, mode, f_dev, u_dev, g_dev, tol, maxit, grad_f_dev, grad_x_dev, info, (cudaStream_t)stream);
    })
}

gofd_status gofd_solve_batch(gofd_problem* p, gofd_solve_mode mode, gofd_rhs rhs, int nb, const double* f_dev,
                             int64_t ldf, double tol, int maxit, double* u_dev, gofd_solve_info* infos,
                             void* stream) {
    if (!p) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        if (nb < 1 || nb > 4096) gofd::fail(GOFD_E_ARG, "nb must be in [1, 4096]");
        if (!f_dev || !u_dev) gofd::fail(GOFD_E_ARG, "NULL vector");
        if (mode != GOFD_SOLVE_FP64 && mode != GOFD_SOLVE_MIXED) gofd::fail(GOFD_E_ARG, "bad mode");
        if (rhs != GOFD_RHS_GRID && rhs != GOFD_RHS_VERTEX) gofd::fail(GOFD_E_ARG, "bad rhs kind");
        if (ldf < (rhs == GOFD_RHS_GRID ? p->ngrid : p->nv)) gofd::fail(GOFD_E_ARG, "ldf smaller than a column");
        if (!(tol > 0.0) || maxit < 1) gofd::fail(GOFD_E_ARG, "tol must be > 0 and maxit >= 1");
        gofd::solve_batch(p, mode, rhs, nb, f_dev, ldf, tol, maxit, u_dev, infos, (cudaStream_t)stream);
    })
}

struct gofd_group {
    gofd::Group* impl = nullptr;
};

gofd_status gofd_group_create(int np, gofd_problem* const* problems, int nb, gofd_group** out) {
    if (out) *out = nullptr;
    GOFD_API_BODY(nullptr, {
        if (!out || !problems || np < 1 || nb < 1 || (int64_t)np * nb > 65535)
            gofd::fail(GOFD_E_ARG, "need problems, 1 <= np, 1 <= nb and np*nb <= 65535");
        auto* g = new gofd_group();
        try {
            g->impl = gofd::group_create(np, problems, nb);
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
    })
}

gofd_status gofd_group_autotune(gofd_group* g, void* stream, double* best_ms) {
    if (!g) return GOFD_E_ARG;
    GOFD_API_BODY(nullptr, {
        const double ms = gofd::group_autotune(g->impl, (cudaStream_t)stream);
        if (best_ms) *best_ms = ms;
    })
}

gofd_status gofd_group_solve(gofd_group* g, gofd_solve_mode mode, gofd_rhs rhs, const double* const* f_dev,
                             const int64_t* ldf, double tol, int maxit, double* const* u_dev,
                             gofd_solve_info* infos, void* stream) {
    if (!g) return GOFD_E_ARG;
    GOFD_API_BODY(nullptr, {
        if (!f_dev || !ldf || !u_dev) gofd::fail(GOFD_E_ARG, "NULL argument");
        if (mode != GOFD_SOLVE_FP64 && mode != GOFD_SOLVE_MIXED) gofd::fail(GOFD_E_ARG, "bad mode");
        if (rhs != GOFD_RHS_GRID && rhs != GOFD_RHS_VERTEX) gofd::fail(GOFD_E_ARG, "bad rhs kind");
        if (!(tol > 0.0) || maxit < 1) gofd::fail(GOFD_E_ARG, "tol must be > 0 and maxit >= 1");
        gofd::group_solve(g->impl, mode, rhs, f_dev, ldf, tol, maxit, u_dev, infos, (cudaStream_t)stream);
    })
}

void gofd_group_destroy(gofd_group* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    gofd::group_destroy(g->impl);
    delete g;
}

gofd_status gofd_autotune(gofd_problem* p, int nb, void* stream, double* best_ms) {
    if (!p) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        if (nb < 1 || nb > 4096) gofd::fail(GOFD_E_ARG, "nb must be in [1, 4096]");
        const double ms = gofd::autotune(p, nb, (cudaStream_t)stream);
        if (best_ms) *best_ms = ms;
    })
}

gofd_status gofd_set_launch_shapes(gofd_problem* p, int lines_per_cta, int cols_per_cta, int scatter_lanes,
                                   int col_elems, int row_elems, int batch_chunk) {
    if (!p) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        auto in = [](int v, std::initializer_list<int> ok) {
            if (v == 0) return true;
            for (int o : ok)
                if (v == o) return true;
            return false;
        };
        if (!in(lines_per_cta, {1, 2, 4}) || !in(cols_per_cta, {1, 2, 4}) || !in(scatter_lanes, {4, 8, 16, 32}) ||
            !in(col_elems, {8, 16, 32}) || !in(row_elems, {8, 16}) || batch_chunk < 0)
            gofd::fail(GOFD_E_ARG, "launch shape out of range");
        gofd::invalidate_graphs(p);
        p->tune_lpc = lines_per_cta;
        p->tune_cols = cols_per_cta;
        p->tune_tpr = scatter_lanes;
        p->tune_cole = col_elems;
        p->tune_rowe = row_elems;
        p->tune_bchunk = batch_chunk;
    })
}

gofd_status gofd_get_info(const gofd_problem* p, gofd_info* info) {
    if (!p || !info) return GOFD_E_ARG;
    std::memset(info, 0, sizeof(*info));
    info->d = p->d;
    for (int i = 0; i < 3; ++i) info->n[i] = p->n[i];
    info->P = p->P;
    info->n_v = p->nv;
    info->n_e = p->ne;
    info->n_interior = p->nint;
    info->n_grid = p->ngrid;
    info->n_loc = p->nloc;
    info->nnz_t = p->nnz_t;
    info->n_runs = p->nruns;
    info->filon_M = p->filon_M;
    info->richardson_levels = p->rich_levels;
    info->alpha = p->alpha;
    info->s = p->s;
    info->h = p->h;
    info->a_h = p->a_h;
    info->min_colsum = p->min_colsum;
    info->precond_nnz = gofd::precond_nnz(p);
    info->precond_levels = gofd::precond_levels(p);
    info->ic_shift = gofd::precond_shift(p);
    info->t_setup_ms = p->t_setup_ms;
    info->tune_lines_per_cta = p->tune_lpc;
    info->tune_cols_per_cta = p->tune_cols;
    info->tune_scatter_lanes = p->tune_tpr;
    info->tune_col_elems = p->tune_cole;
    info->tune_batch_chunk = p->tune_bchunk;
    info->tune_row_elems = p->tune_rowe;
    info->warp_fft_path = gofd::afd_2d_warp_eligible(p) ? 1 : 0;
    return GOFD_OK;
}

gofd_status gofd_export_transfer(const gofd_problem* p, int32_t* owner, int32_t* ell_idx, double* ell_w) {
    if (!p) return GOFD_E_ARG;
    gofd_problem* q = const_cast<gofd_problem*>(p);
    GOFD_API_BODY(q, {
        const size_t dp1 = p->d + 1;
        if (owner) GOFD_CUDA_TRY(cudaMemcpy(owner, p->owner.ptr, 4 * p->ngrid, cudaMemcpyDeviceToHost));
        if (ell_idx && p->nloc)
            GOFD_CUDA_TRY(cudaMemcpy(ell_idx, p->ell_vidx.ptr, 4 * dp1 * p->nloc, cudaMemcpyDeviceToHost));
        if (ell_w && p->nloc)
            GOFD_CUDA_TRY(cudaMemcpy(ell_w, p->ell_w64.ptr, 8 * dp1 * p->nloc, cudaMemcpyDeviceToHost));
    })
}

gofd_status gofd_export_vertex_data(const gofd_problem* p, int32_t* interior_index, double* colsum) {
    if (!p) return GOFD_E_ARG;
    gofd_problem* q = const_cast<gofd_problem*>(p);
    GOFD_API_BODY(q, {
        std::vector<int32_t> v2i(p->nv);
        GOFD_CUDA_TRY(cudaMemcpy(v2i.data(), p->vert2int.ptr, 4 * p->nv, cudaMemcpyDeviceToHost));
        if (interior_index) std::memcpy(interior_index, v2i.data(), 4 * p->nv);
        if (colsum) {
            std::vector<double> cs(p->nint);
            GOFD_CUDA_TRY(cudaMemcpy(cs.data(), p->colsum.ptr, 8 * p->nint, cudaMemcpyDeviceToHost));
            for (int64_t v = 0; v < p->nv; ++v) colsum[v] = v2i[v] >= 0 ? cs[v2i[v]] : 0.0;
        }
    })
}

gofd_status gofd_export_precond(const gofd_problem* p, int32_t* perm, int32_t* lptr, int32_t* lcol, double* lval) {
    if (!p) return GOFD_E_ARG;
    gofd_problem* q = const_cast<gofd_problem*>(p);
    GOFD_API_BODY(q, { gofd::precond_export(p, perm, lptr, lcol, lval); })
}

gofd_status gofd_export_diagonal(const gofd_problem* p, double* diag) {
    if (!p || !diag) return GOFD_E_ARG;
    GOFD_API_BODY(const_cast<gofd_problem*>(p), { gofd::precond_diagonal(p, diag); })
}

gofd_status gofd_get_coefficients(const gofd_problem* p, double* T) {
    if (!p || !T) return GOFD_E_ARG;
    gofd_problem* q = const_cast<gofd_problem*>(p);
    GOFD_API_BODY(q, { GOFD_CUDA_TRY(cudaMemcpy(T, p->T.ptr, 8 * p->ngrid, cudaMemcpyDeviceToHost)); })
}

gofd_status gofd_get_symbol(const gofd_problem* p, double* lambda) {
    if (!p || !lambda) return GOFD_E_ARG;
    gofd_problem* q = const_cast<gofd_problem*>(p);
    GOFD_API_BODY(q, {
        int64_t nh = 1;
        double sc = 1.0;
        for (int i = 0; i < p->d; ++i) {
            nh *= p->P / 2 + 1;
            sc *= p->P;
        }
        GOFD_CUDA_TRY(cudaMemcpy(lambda, p->lam64.ptr, 8 * nh, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < nh; ++i) lambda[i] *= sc;
    })
}

gofd_status gofd_afd_apply(gofd_problem* p, gofd_precision prec, const void* v_dev, void* w_dev, void* stream) {
    if (!p) return GOFD_E_ARG;
    GOFD_API_BODY(p, {
        if (!v_dev || !w_dev) gofd::fail(GOFD_E_ARG, "NULL vector");
        gofd::afd_apply_grid(p, prec == GOFD_FP64, v_dev, w_dev, (cudaStream_t)stream);
    })
}

gofd_status gofd_afd_apply_noalloc(int d, int n, const float* lambda_dev, const float* v_dev, float* w_dev,
                                   void* stream) {
    GOFD_API_BODY(nullptr, { gofd::afd_apply_noalloc(d, n, lambda_dev, v_dev, w_dev, (cudaStream_t)stream); })
}

}  // extern "C"
