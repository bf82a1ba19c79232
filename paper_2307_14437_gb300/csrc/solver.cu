// Preconditioned conjugate gradients on the interior block of (GoFD-2)
// (Section 3.2), in two modes:
//   FP64   : FP64 operator, vectors, scalars;
//   MIXED  : outer FP64 iterative refinement r = b - S x, inner PCG with the
//            FP32 operator and FP32 vectors, FP64 inner products and scalars.
// The right-hand side follows (GoFD-2) for grid data or (GoFD-3) for vertex data.
// Inner products are reduced in a fixed order (per-block partial sums, then the
// last block to finish adds the partials in block order), so results do not
// depend on scheduling.  Scalars stay on the device; the host reads the
// residual only every `check_every` iterations.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "gofd_internal.cuh"

namespace gofd {

void scatter_grid_f64(gofd_problem* p, const double* f, double* y, double scale, cudaStream_t st);

constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs
constexpr int RED_THREADS = 256;

struct Scal {
    double rz;      // (r, z)
    double rz_new;
    double pq;      // (p, q)
    double alpha;
    double beta;
    double rr;      // (r, r)
    double aux;
    int bad;        // breakdown flag
    int it;         // iterations done by the device-side loop
    double stop_rr; // the device-side loop stops once rr <= stop_rr
    int maxit;      // ... or when another `check` iterations would pass maxit
    int pad;
};

// Device-side loop control: arm before the loop, decide after every `check`
// iterations whether the conditional (while) node of the graph runs again.
__global__ void loop_arm_kernel(Scal* s, double stop_rr, int maxit) {
    s->it = 0;
    s->stop_rr = stop_rr;
    s->maxit = maxit;
}

__global__ void loop_continue_kernel(cudaGraphConditionalHandle h, Scal* s, int check) {
    s->it += check;
    const bool more = !s->bad && s->rr > s->stop_rr && s->it + check <= s->maxit;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

struct Workspace {
    DevBuf x64, r64, b64, p64, q64, z64, d64;
    DevBuf d32, r32, p32, q32, z32;
    DevBuf partial, counter, scal;
    Scal* host = nullptr;   // pinned
    // the solver runs on its own stream, ordered after / before the caller's
    // stream by events, so that `check` PCG iterations can be captured once as
    // a CUDA graph and replayed (one graph per precision)
    cudaStream_t gs = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool no_graph = false;   // building the loop graph failed once: host-driven loop
    ~Workspace() {
        for (auto& g : graph)
            if (g) cudaGraphExecDestroy(g);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (gs) cudaStreamDestroy(gs);
        if (host) cudaFreeHost(host);
    }
};

// The captured iterations depend on the launch shapes; a new choice of shapes
// (the autotuner) drops them.
void invalidate_graphs(gofd_problem* p) {
    if (!p->ws) return;
    for (auto& g : p->ws->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// ---------------------------------------------------------------------------
// fixed-order block reduction helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0;
    if (warp == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// the last block to arrive adds the partials in block order; returns true there
__device__ __forceinline__ bool finish_reduction(double mine, double* partial, unsigned* counter,
                                                 double* total) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = mine;
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __shared__ double sh[32];
    double v = 0;
    // fixed order: thread t sums partials t, t+blockDim, ... ; then a fixed tree
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += ((volatile double*)partial)[i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) {
        *total = v;
        *counter = 0;
    }
    return true;
}

// pq = (p, q); alpha = rz / pq
template <class V>
__global__ void dot_pq_kernel(const V* __restrict__ p, const V* __restrict__ q, int64_t n, double* partial,
                              unsigned* counter, Scal* s) {
    pdl_enter();
    __shared__ double sh[32];
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)p[i] * (double)q[i];
    acc = block_sum(acc, sh);
    double tot;
    if (finish_reduction(acc, partial, counter, &tot) && threadIdx.x == 0) {
        s->pq = tot;
        if (!(tot > 0.0) || !isfinite(tot)) s->bad = 1;
        s->alpha = (tot > 0.0) ? s->rz / tot : 0.0;
    }
}

// x += alpha p ; r -= alpha q ; rr = (r, r) ; (if no preconditioner: rz_new = rr, beta)
template <class V>
__global__ void update_xr_kernel(V* __restrict__ x, V* __restrict__ r, const V* __restrict__ p,
                                 const V* __restrict__ q, int64_t n, double* partial, unsigned* counter, Scal* s,
                                 int has_precond) {
    pdl_enter();
    __shared__ double sh[32];
    const double a = s->alpha;
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        V xi = x[i], ri = r[i];
        xi = (V)((double)xi + a * (double)p[i]);
        ri = (V)((double)ri - a * (double)q[i]);
        x[i] = xi;
        r[i] = ri;
        acc += (double)ri * (double)ri;
    }
    acc = block_sum(acc, sh);
    double tot;
    if (finish_reduction(acc, partial, counter, &tot) && threadIdx.x == 0) {
        s->rr = tot;
        if (!has_precond) {
            s->beta = tot / s->rz;
            s->rz = tot;
        }
    }
}

// rz_new = (r, z); beta = rz_new / rz
template <class V>
__global__ void dot_rz_kernel(const V* __restrict__ r, const V* __restrict__ z, int64_t n, double* partial,
                              unsigned* counter, Scal* s, int init) {
    pdl_enter();
    __shared__ double sh[32];
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)r[i] * (double)z[i];
    acc = block_sum(acc, sh);
    double tot;
    if (finish_reduction(acc, partial, counter, &tot) && threadIdx.x == 0) {
        if (init) {
            s->rz = tot;
            s->beta = 0.0;
        } else {
            s->beta = tot / s->rz;
            s->rz = tot;
        }
    }
}

// rr = (r, r) only
template <class V>
__global__ void dot_rr_kernel(const V* __restrict__ r, int64_t n, double* partial, unsigned* counter,
                              double* out) {
    __shared__ double sh[32];
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)r[i] * (double)r[i];
    acc = block_sum(acc, sh);
    double tot;
    if (finish_reduction(acc, partial, counter, &tot) && threadIdx.x == 0) *out = tot;
}

// p = z + beta p
template <class V>
__global__ void update_p_kernel(V* __restrict__ p, const V* __restrict__ z, int64_t n, const Scal* s) {
    pdl_enter();
    const double b = s->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (V)((double)z[i] + b * (double)p[i]);
}

// r = b - y  (FP64)
__global__ void residual_kernel(const double* __restrict__ b, const double* __restrict__ y, double* __restrict__ r,
                                int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = b[i] - y[i];
}

// out32 = (float)(in64 * scale)
__global__ void to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, double scale, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)(in[i] * scale);
}

// x64 += scale * d32
__global__ void accumulate_kernel(double* __restrict__ x, const float* __restrict__ d, double scale, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += scale * (double)d[i];
}

// x += d  (FP64)
__global__ void add_kernel(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += d[i];
}

template <class V>
__global__ void copy_kernel(const V* __restrict__ a, V* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

// b_i = scale * colsum_i * f[vertex(i)]   (GoFD-3 multiplied through by h^{2s} D_h)
__global__ void rhs_vertex_kernel(const double* __restrict__ f, const int32_t* __restrict__ i2v,
                                  const double* __restrict__ colsum, double scale, int64_t nint,
                                  double* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nint; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = scale * colsum[i] * f[i2v[i]];
}

// ---------------------------------------------------------------------------
static Workspace* ensure_ws(gofd_problem* p) {
    if (p->ws) return p->ws;
    Workspace* w = new Workspace();
    const int64_t n1 = p->nint + 1;
    w->x64.alloc(8 * n1); w->r64.alloc(8 * n1); w->b64.alloc(8 * n1);
    w->p64.alloc(8 * n1); w->q64.alloc(8 * n1); w->z64.alloc(8 * n1); w->d64.alloc(8 * n1);
    w->d32.alloc(4 * n1); w->r32.alloc(4 * n1); w->p32.alloc(4 * n1);
    w->q32.alloc(4 * n1); w->z32.alloc(4 * n1);
    w->partial.alloc(sizeof(double) * RED_BLOCKS);
    w->counter.alloc(sizeof(unsigned) * 4);
    w->scal.alloc(sizeof(Scal));
    GOFD_CUDA_TRY(cudaMemset(w->counter.ptr, 0, sizeof(unsigned) * 4));
    GOFD_CUDA_TRY(cudaMemset(w->p64.ptr, 0, 8 * n1));
    GOFD_CUDA_TRY(cudaMemset(w->p32.ptr, 0, 4 * n1));
    GOFD_CUDA_TRY(cudaMallocHost((void**)&w->host, sizeof(Scal)));
    GOFD_CUDA_TRY(cudaStreamCreateWithFlags(&w->gs, cudaStreamNonBlocking));
    GOFD_CUDA_TRY(cudaEventCreateWithFlags(&w->ev_in, cudaEventDisableTiming));
    GOFD_CUDA_TRY(cudaEventCreateWithFlags(&w->ev_out, cudaEventDisableTiming));
    p->ws = w;
    return w;
}

void free_workspace(gofd_problem* p) {
    delete p->ws;
    p->ws = nullptr;
}

static void read_scal(Workspace* w, cudaStream_t st) {
    GOFD_CUDA_TRY(cudaMemcpyAsync(w->host, w->scal.ptr, sizeof(Scal), cudaMemcpyDeviceToHost, st));
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
}

static double norm64(gofd_problem* p, Workspace* w, const double* v, cudaStream_t st) {
    Scal* s = w->scal.as<Scal>();
    dot_rr_kernel<double><<<RED_BLOCKS, RED_THREADS, 0, st>>>(v, p->nint, w->partial.as<double>(),
                                                              w->counter.as<unsigned>(), &s->aux);
    GOFD_CHECK_LAUNCH();
    read_scal(w, st);
    return std::sqrt(w->host->aux);
}

// PCG on S d = r (precision V) from d = 0; r is overwritten.  Returns iterations;
// stops when ||r_k|| <= rtol * ||r_0|| or after maxit iterations.
template <class V>
static int pcg(gofd_problem* p, Workspace* w, V* d, V* r, V* pv, V* q, V* z, double rtol, int maxit,
               cudaStream_t st, double* final_rel) {
    const bool fp64 = sizeof(V) == 8;
    const int64_t n = p->nint;
    Scal* s = w->scal.as<Scal>();
    double* part = w->partial.as<double>();
    unsigned* cnt = w->counter.as<unsigned>();
    const int nb = grid_blocks(n, 256);
    const bool pc = p->pc != nullptr;
    const int check = p->opt.check_every > 0 ? p->opt.check_every : 8;
    GOFD_CUDA_TRY(cudaMemsetAsync(s, 0, sizeof(Scal), st));
    GOFD_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(V) * n, st));
    V* zz = r;
    if (pc) {
        precond_apply(p, fp64, r, z, st);
        zz = z;
    }
    dot_rz_kernel<V><<<RED_BLOCKS, RED_THREADS, 0, st>>>(r, zz, n, part, cnt, s, 1);
    dot_rr_kernel<V><<<RED_BLOCKS, RED_THREADS, 0, st>>>(r, n, part, cnt, &s->rr);
    copy_kernel<V><<<nb, 256, 0, st>>>(zz, pv, n);
    GOFD_CHECK_LAUNCH();
    read_scal(w, st);
    const double r0 = std::sqrt(w->host->rr);
    if (r0 == 0.0) {
        *final_rel = 0.0;
        return 0;
    }
    int it = 0;
    double rel = 1.0;
    auto iteration = [&]() {
        apply_interior(p, fp64, pv, q, st);
        launch_pdl(dot_pq_kernel<V>, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, st, (const V*)pv, (const V*)q, n,
                   part, cnt, s);
        launch_pdl(update_xr_kernel<V>, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, st, d, r, (const V*)pv,
                   (const V*)q, n, part, cnt, s, pc ? 1 : 0);
        if (pc) {
            precond_apply(p, fp64, r, z, st);
            launch_pdl(dot_rz_kernel<V>, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, st, (const V*)r, (const V*)z, n,
                       part, cnt, s, 0);
        }
        launch_pdl(update_p_kernel<V>, dim3(nb), dim3(256), 0, st, pv, (const V*)zz, n, (const Scal*)s);
        GOFD_CHECK_LAUNCH();
    };
    // The iterations run as one CUDA graph: a conditional while node whose
    // body is `check` iterations and a kernel that decides on the device
    // whether to go on (converged, breakdown or maxit reached), so the host
    // does not wait between checks.  The vectors of a precision are always
    // the workspace's, so the graph is built once per handle.
    cudaGraphExec_t& graph = w->graph[fp64 ? 1 : 0];
    if (!graph && !w->no_graph && st == w->gs && maxit >= check) {
        try {
            build_loop_graph(st, check, iteration, [&](cudaGraphConditionalHandle h) {
                loop_continue_kernel<<<1, 1, 0, st>>>(h, s, check);
            }, &graph);
        } catch (const Error&) {   // no device-side loop here: iterate from the host
            graph = nullptr;
            w->no_graph = true;
            cudaGetLastError();
        }
    }
    bool done = false;
    if (graph && st == w->gs && maxit >= check) {
        loop_arm_kernel<<<1, 1, 0, st>>>(s, rtol * rtol * r0 * r0, maxit);
        GOFD_CHECK_LAUNCH();
        GOFD_CUDA_TRY(cudaGraphLaunch(graph, st));
        read_scal(w, st);
        it = w->host->it;
        rel = std::sqrt(w->host->rr) / r0;
        done = w->host->bad || rel <= rtol;
    }
    // without the graph, or for the last iterations before maxit: one by one
    while (!done && it < maxit) {
        iteration();
        ++it;
        if (it % check == 0 || it == maxit) {
            read_scal(w, st);
            if (w->host->bad) break;
            rel = std::sqrt(w->host->rr) / r0;
            if (rel <= rtol) break;
        }
    }
    read_scal(w, st);
    rel = std::sqrt(w->host->rr) / r0;
    *final_rel = rel;
    return it;
}

// Solve S x = b on the interior unknowns (b, x: device, n_int (+1) FP64 each,
// x[n_int] = 0 on exit).  x holds the initial guess unless init_zero.
void solve_core(gofd_problem* p, gofd_solve_mode mode, const double* b, double tol, int maxit, bool init_zero,
                double* x, gofd_solve_info* info, cudaStream_t caller) {
    auto t0 = std::chrono::steady_clock::now();
    Workspace* w = ensure_ws(p);
    // run on the workspace's stream, after the caller's pending work; the
    // caller's stream waits for the solve on every exit path
    const cudaStream_t st = w->gs;
    GOFD_CUDA_TRY(cudaEventRecord(w->ev_in, caller));
    GOFD_CUDA_TRY(cudaStreamWaitEvent(st, w->ev_in, 0));
    struct Join {
        Workspace* w;
        cudaStream_t caller;
        ~Join() {
            cudaEventRecord(w->ev_out, w->gs);
            cudaStreamWaitEvent(caller, w->ev_out, 0);
        }
    } join{w, caller};
    const int64_t n = p->nint;
    const int nb = grid_blocks(n, 256);
    double* r = w->r64.as<double>();
    if (init_zero) GOFD_CUDA_TRY(cudaMemsetAsync(x, 0, 8 * (n + 1), st));
    else GOFD_CUDA_TRY(cudaMemsetAsync(x + n, 0, 8, st));
    const double bn = norm64(p, w, b, st);
    if (!std::isfinite(bn)) fail(GOFD_E_ARG, "the right-hand side has a non-finite entry");
    int outer = 0, inner = 0;
    double rel = 0.0;
    bool converged = false;
    if (bn == 0.0) {
        GOFD_CUDA_TRY(cudaMemsetAsync(x, 0, 8 * (n + 1), st));
        converged = true;
    }
    const int max_outer = 200;
    // estimate of the relative residual the next refinement round measures
    // (last measured residual times the reduction its inner solve was asked for)
    double expected = 1.0;
    while (!converged && outer < max_outer && inner < maxit) {
        // true residual with the FP64 operator
        if (outer == 0 && init_zero) {
            copy_kernel<double><<<nb, 256, 0, st>>>(b, r, n);
        } else {
            // FP64 residual; in mixed mode its convolution in double-float
            // while the residual expected is at least residual_df_floor (below
            // it b - S x cancels enough that the double-float product's error,
            // about 1e-15 of ||S x||, could matter)
            if (mode == GOFD_SOLVE_MIXED && expected >= residual_df_floor)
                apply_interior_residual(p, x, w->q64.as<double>(), st);
            else apply_interior(p, true, x, w->q64.ptr, st);
            residual_kernel<<<nb, 256, 0, st>>>(b, w->q64.as<double>(), r, n);
        }
        GOFD_CHECK_LAUNCH();
        const double rn = norm64(p, w, r, st);
        if (!std::isfinite(rn)) {
            if (outer == 0) fail(GOFD_E_ARG, "the initial guess has a non-finite entry");
            precond_check(p, st);
            fail(GOFD_E_NOT_CONVERGED, "the residual became non-finite");
        }
        rel = rn / bn;
        if (rel <= tol) {
            converged = true;
            break;
        }
        ++outer;
        double inner_rel = 0;
        if (mode == GOFD_SOLVE_FP64) {
            // FP64 PCG on S d = r down to the full tolerance, then x += d
            double* d = w->d64.as<double>();
            int its = pcg<double>(p, w, d, r, w->p64.as<double>(), w->q64.as<double>(), w->z64.as<double>(),
                                  0.5 * tol * bn / rn, maxit - inner, st, &inner_rel);
            inner += its;
            add_kernel<<<nb, 256, 0, st>>>(x, d, n);
            GOFD_CHECK_LAUNCH();
            if (its == 0) break;
        } else {
            // inner FP32 PCG on S d = r / ||r||
            to_f32_kernel<<<nb, 256, 0, st>>>(r, w->r32.as<float>(), 1.0 / rn, n);
            GOFD_CHECK_LAUNCH();
            // the inner reduction a round needs: 1e-4 (the FP32 solve's
            // reach), or less when the residual is already near tol (half of
            // the remaining factor, so that the round's FP32 error still fits)
            const double itol0 = p->opt.inner_tol > 0 ? p->opt.inner_tol : 1e-4;
            const double itol = std::max(itol0, 0.5 * tol * bn / rn);
            int its = pcg<float>(p, w, w->d32.as<float>(), w->r32.as<float>(), w->p32.as<float>(),
                                 w->q32.as<float>(), w->z32.as<float>(), itol, maxit - inner, st, &inner_rel);
            inner += its;
            accumulate_kernel<<<nb, 256, 0, st>>>(x, w->d32.as<float>(), rn, n);
            GOFD_CHECK_LAUNCH();
            expected = rel * itol;
            if (its == 0) break;
        }
    }
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    precond_check(p, st);
    auto t1 = std::chrono::steady_clock::now();
    if (info) {
        info->outer_iters = outer;
        info->inner_iters = inner;
        info->rel_res_fp64 = rel;
        info->a_h = p->a_h;
        info->min_colsum = p->min_colsum;
        info->ic_shift = precond_shift(p);
        const double dd = p->d;
        info->h_within_strict_bound = p->h <= p->a_h / ((dd + 1) * std::sqrt(dd));
        info->h_within_practical_bound = p->h <= p->a_h;
        info->t_setup_ms = p->t_setup_ms;
        info->t_solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        info->device_loop = !w->no_graph && (w->graph[0] || w->graph[1]);
    }
    if (!converged) fail(GOFD_E_NOT_CONVERGED, "solver reached maxit before tol");
}

// b = h^{2s} I^T f (grid data) or h^{2s} D_h f (vertex data) on the interior
void assemble_rhs(gofd_problem* p, gofd_rhs rhs, const double* f, double* b, cudaStream_t st) {
    const int64_t n = p->nint;
    const double h2s = std::pow(p->h, 2.0 * p->s);
    if (rhs == GOFD_RHS_GRID) {
        scatter_grid_f64(p, f, b, h2s, st);
    } else {
        rhs_vertex_kernel<<<grid_blocks(n, 256), 256, 0, st>>>(f, p->int2vert.as<int32_t>(), p->colsum.as<double>(),
                                                             h2s, n, b);
        GOFD_CHECK_LAUNCH();
    }
}

void solve(gofd_problem* p, gofd_solve_mode mode, gofd_rhs rhs, const double* f, double tol, int maxit,
           bool init_zero, double* u, gofd_solve_info* info, cudaStream_t st) {
    Workspace* w = ensure_ws(p);
    double* b = w->b64.as<double>();
    double* x = w->x64.as<double>();
    assemble_rhs(p, rhs, f, b, st);
    if (!init_zero) compact_vertex(p, true, u, x, st);
    try {
        solve_core(p, mode, b, tol, maxit, init_zero, x, info, st);
    } catch (const Error& e) {
        expand_interior(p, true, x, u, 0.0, st);   // the last iterate
        throw;
    }
    expand_interior(p, true, x, u, 0.0, st);
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace gofd
