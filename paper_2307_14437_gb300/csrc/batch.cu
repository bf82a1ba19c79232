// Many right-hand sides on one problem: lock-step block PCG.
//
// nb right-hand sides advance together: every iteration applies S to all nb
// search directions in one batched launch sequence (2D: the product kernels
// run over a batch index; other dimensions: one product per column), and the
// inner products are reduced per column in a fixed order.  Each column keeps
// its own scalars and stops (alpha = 0 from then on) when its residual meets
// its tolerance.  Mixed mode refines every column in FP64 around FP32 inner
// solves, as the single-vector solver does.  The autotuner times the launch
// shapes of the product (lines / columns per CTA, lanes per scatter row) on
// the batch and keeps the fastest.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <memory>
#include <vector>

#include "gofd_internal.cuh"

namespace gofd {

constexpr int BRED_BLOCKS = 96;
constexpr int BRED_THREADS = 256;

struct BScal {
    double rz, pq, alpha, beta, rr, r0, rtol, aux;
    int done, pad;
};

struct BatchWork {
    int cap = 0;
    int64_t ld = 0;
    DevBuf b64, x64, r64, p64, q64, z64, d64;
    DevBuf r32, p32, q32, z32, d32;
    DevBuf grid, spec, partial, counters;
    DevBuf red, cnt, scal, colv, ctl;
    std::vector<BScal> host;
    // own stream (joined to the caller's by events) so that `check` block-PCG
    // iterations are captured once as a CUDA graph per precision and batch size
    cudaStream_t gs = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_nb[2] = {0, 0};
    bool no_graph = false;
    ~BatchWork() {
        for (auto& g : graph)
            if (g) cudaGraphExecDestroy(g);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (gs) cudaStreamDestroy(gs);
    }
};

// ---------------------------------------------------------------------------
// per-column fixed-order reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double bblock_sum(double v, double* sh) {
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
    return t;
}

// adds the block partials of column blockIdx.y in block order in the last block
__device__ __forceinline__ bool bfinish(double mine, double* red, unsigned* cnt, double* total) {
    __shared__ bool last;
    double* part = red + (int64_t)blockIdx.y * gridDim.x;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = mine;
        __threadfence();
        last = atomicAdd(&cnt[blockIdx.y], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __shared__ double sh[32];
    double v = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += ((volatile double*)part)[i];
    v = bblock_sum(v, sh);
    if (threadIdx.x == 0) {
        *total = v;
        cnt[blockIdx.y] = 0;
    }
    return true;
}

template <class V>
__device__ __forceinline__ double bdot_local(const V* a, const V* b, int64_t n) {
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    return acc;
}

// mode 0: rz = (r,z) init; 1: rz_new = (r,z) -> beta; 2: pq -> alpha; 3: aux = (a,a)
template <class V>
__global__ void bdot_kernel(const V* __restrict__ A, const V* __restrict__ B, int64_t n, int64_t ld, double* red,
                            unsigned* cnt, BScal* s, int mode) {
    pdl_enter();
    __shared__ double sh[32];
    const V* a = A + blockIdx.y * ld;
    const V* b = B + blockIdx.y * ld;
    double acc = bblock_sum(bdot_local(a, b, n), sh);
    double tot;
    if (bfinish(acc, red, cnt, &tot) && threadIdx.x == 0) {
        BScal& c = s[blockIdx.y];
        if (mode == 0) {
            c.rz = tot;
            c.beta = 0.0;
        } else if (mode == 1) {
            c.beta = c.done ? 0.0 : tot / c.rz;
            c.rz = tot;
        } else if (mode == 2) {
            c.pq = tot;
            c.alpha = (c.done || !(tot > 0.0)) ? 0.0 : c.rz / tot;
            if (!(tot > 0.0)) c.done = 1;
        } else {
            c.aux = tot;
        }
    }
}

// x += alpha p; r -= alpha q; rr = (r,r); (no preconditioner: rz = rr, beta); done test
template <class V>
__global__ void bupdate_kernel(V* __restrict__ X, V* __restrict__ R, const V* __restrict__ Pp,
                               const V* __restrict__ Q, int64_t n, int64_t ld, double* red, unsigned* cnt, BScal* s,
                               int has_pc) {
    pdl_enter();
    __shared__ double sh[32];
    const double a = s[blockIdx.y].alpha;
    V* x = X + blockIdx.y * ld;
    V* r = R + blockIdx.y * ld;
    const V* p = Pp + blockIdx.y * ld;
    const V* q = Q + blockIdx.y * ld;
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        V ri = r[i];
        if (a != 0.0) {   // alpha = 0 (a converged column): q was not computed, x and r stay
            ri = (V)((double)ri - a * (double)q[i]);
            x[i] = (V)((double)x[i] + a * (double)p[i]);
            r[i] = ri;
        }
        acc += (double)ri * (double)ri;
    }
    acc = bblock_sum(acc, sh);
    double tot;
    if (bfinish(acc, red, cnt, &tot) && threadIdx.x == 0) {
        BScal& c = s[blockIdx.y];
        c.rr = tot;
        if (!has_pc) {
            c.beta = c.done ? 0.0 : tot / c.rz;
            c.rz = tot;
        }
        if (sqrt(tot) <= c.rtol * c.r0) c.done = 1;
    }
}

template <class V>
__global__ void bupdate_p_kernel(V* __restrict__ Pp, const V* __restrict__ Z, int64_t n, int64_t ld,
                                 const BScal* s) {
    pdl_enter();
    const double b = s[blockIdx.y].beta;
    V* p = Pp + blockIdx.y * ld;
    const V* z = Z + blockIdx.y * ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (V)((double)z[i] + b * (double)p[i]);
}

// device-side loop control of the block PCG: ctl = {iterations done, maxit}
__global__ void bloop_arm_kernel(int* ctl, int maxit) {
    ctl[0] = 0;
    ctl[1] = maxit;
}

__global__ void bloop_continue_kernel(cudaGraphConditionalHandle h, const BScal* s, int nb, int* ctl, int check) {
    int all = 1;
    for (int c = threadIdx.x; c < nb; c += blockDim.x) all &= s[c].done != 0;
    all = __syncthreads_and(all);
    if (threadIdx.x == 0) {
        ctl[0] += check;
        const bool more = !all && ctl[0] + check <= ctl[1];
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

__global__ void bset_start_kernel(BScal* s, const double* __restrict__ rtol, int nb) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nb; c += gridDim.x * blockDim.x) {
        BScal& x = s[c];
        x.r0 = sqrt(x.aux);
        x.rr = x.aux;
        x.rtol = rtol[c];
        x.done = x.r0 == 0.0;
        x.alpha = x.beta = 0.0;
    }
}

template <class V>
__global__ void bcopy_kernel(const V* __restrict__ a, V* __restrict__ b, int64_t n, int64_t ld) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[blockIdx.y * ld + i] = a[blockIdx.y * ld + i];
}

__global__ void bresidual_kernel(const double* __restrict__ B, const double* __restrict__ Y, double* __restrict__ R,
                                 int64_t n, int64_t ld) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        R[blockIdx.y * ld + i] = B[blockIdx.y * ld + i] - Y[blockIdx.y * ld + i];
}

// R *= inv (per column, in place)
__global__ void bscale_kernel(double* __restrict__ R, const double* __restrict__ inv, int64_t n, int64_t ld) {
    const double s = inv[blockIdx.y];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        R[blockIdx.y * ld + i] *= s;
}

__global__ void baccumulate64_kernel(double* __restrict__ X, const double* __restrict__ D,
                                     const double* __restrict__ sc, int64_t n, int64_t ld) {
    const double s = sc[blockIdx.y];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        X[blockIdx.y * ld + i] += s * D[blockIdx.y * ld + i];
}

// r32 = r / ||r|| (columns already converged get 0)
__global__ void bscale_to_f32_kernel(const double* __restrict__ R, float* __restrict__ R32,
                                     const double* __restrict__ inv, int64_t n, int64_t ld) {
    const double s = inv[blockIdx.y];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        R32[blockIdx.y * ld + i] = (float)(R[blockIdx.y * ld + i] * s);
}

__global__ void baccumulate_kernel(double* __restrict__ X, const float* __restrict__ D32, const double* __restrict__ sc,
                                   int64_t n, int64_t ld) {
    const double s = sc[blockIdx.y];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        X[blockIdx.y * ld + i] += s * (double)D32[blockIdx.y * ld + i];
}

// ---------------------------------------------------------------------------
// workspace of nb columns of length ld on problem p's grid; long-row partial
// sums and counters: nchunks / nrows per column (for a group: the totals)
static void alloc_batch(BatchWork* w, const gofd_problem* p, int nb, int64_t ld, int64_t part_total,
                        int64_t cnt_total) {
    w->cap = nb;
    w->ld = ld;
    const int64_t m = w->ld * nb;
    // every vector starts at zero: in a group, entries past a column's n_int
    // are never written and must stay zero (the products write only the
    // interior rows of their instance)
    for (DevBuf* b : {&w->b64, &w->x64, &w->r64, &w->p64, &w->q64, &w->z64, &w->d64}) {
        b->alloc(8 * m);
        GOFD_CUDA_TRY(cudaMemset(b->ptr, 0, 8 * m));
    }
    for (DevBuf* b : {&w->r32, &w->p32, &w->q32, &w->z32, &w->d32}) {
        b->alloc(4 * m);
        GOFD_CUDA_TRY(cudaMemset(b->ptr, 0, 4 * m));
    }
    w->grid.alloc(8 * p->ngrid * nb);
    if (p->d == 2) w->spec.alloc(sizeof(double2) * (size_t)(p->P / 2 + 1) * p->ldT * nb);
    w->partial.alloc(8 * (part_total + 1));
    w->counters.alloc(4 * (cnt_total + 1));
    GOFD_CUDA_TRY(cudaMemset(w->counters.ptr, 0, 4 * (cnt_total + 1)));
    w->red.alloc(8 * BRED_BLOCKS * nb);
    w->cnt.alloc(sizeof(unsigned) * nb);
    GOFD_CUDA_TRY(cudaMemset(w->cnt.ptr, 0, sizeof(unsigned) * nb));
    w->scal.alloc(sizeof(BScal) * nb);
    w->colv.alloc(8 * 3 * nb);
    w->ctl.alloc(sizeof(int) * 2);
    GOFD_CUDA_TRY(cudaStreamCreateWithFlags(&w->gs, cudaStreamNonBlocking));
    GOFD_CUDA_TRY(cudaEventCreateWithFlags(&w->ev_in, cudaEventDisableTiming));
    GOFD_CUDA_TRY(cudaEventCreateWithFlags(&w->ev_out, cudaEventDisableTiming));
    w->host.resize(nb);
}

static BatchWork* ensure_batch(gofd_problem* p, int nb) {
    BatchWork* w = p->batch;
    if (w && w->cap >= nb) return w;
    delete w;
    w = new BatchWork();
    p->batch = w;
    alloc_batch(w, p, nb, p->nint + 1, (p->n_long_chunks + 1) * nb, (p->n_long_rows + 1) * nb);
    return w;
}

// The operator of a block solve: one problem's S on every column, or a group
// (column c belongs to instance c / nbper, all on rp's grid).  n is the
// vector length (a group: the largest n_int; shorter columns are zero past
// their n_int and every block-PCG step keeps them so).
struct BOp {
    gofd_problem* p = nullptr;
    const std::vector<gofd_problem*>* members = nullptr;
    int nbper = 1;
    GroupArg ga;
    int64_t n = 0;
    gofd_problem* member(int c) const { return members ? (*members)[c / nbper] : p; }
    // skip: per-column flags (device; column c at skip[c * skip_stride]);
    // a column whose flag is set is not computed (block PCG: converged)
    // df: an FP64 product with its convolution in double-float (2D)
    void apply(bool f64, const void* X, void* Y, int nb, int64_t ld, BatchWork* w, cudaStream_t st,
               const int* skip = nullptr, int skip_stride = 0, bool df = false) const {
        if (members) {
            GroupArg g = ga;
            g.skip = skip;
            g.skip_stride = skip_stride;
            apply_interior_group(p, f64, X, Y, nb, ld, w->grid.ptr, w->spec.ptr, w->partial.ptr, w->counters.ptr, g,
                                 st, df);
        } else {
            apply_interior_batch(p, f64, X, Y, nb, ld, w->grid.ptr, w->spec.ptr, w->partial.ptr, w->counters.ptr, st,
                                 skip, skip_stride, df);
        }
    }
};

void free_batch(gofd_problem* p) {
    delete p->batch;
    p->batch = nullptr;
}

static void read_bscal(BatchWork* w, int nb, cudaStream_t st) {
    GOFD_CUDA_TRY(cudaMemcpyAsync(w->host.data(), w->scal.ptr, sizeof(BScal) * nb, cudaMemcpyDeviceToHost, st));
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
}

// column norms^2 of A (FP64) into host vector
static void bnorms(const BOp& op, BatchWork* w, const double* A, int nb, std::vector<double>& out, cudaStream_t st) {
    bdot_kernel<double><<<dim3(BRED_BLOCKS, nb), BRED_THREADS, 0, st>>>(A, A, op.n, w->ld, w->red.as<double>(),
                                                                       w->cnt.as<unsigned>(), w->scal.as<BScal>(), 3);
    GOFD_CHECK_LAUNCH();
    read_bscal(w, nb, st);
    out.resize(nb);
    for (int c = 0; c < nb; ++c) out[c] = w->host[c].aux;
}

// block PCG on S D = R (all columns, precision V) from D = 0; column c stops at
// ||r_c|| <= rtol[c] ||r_c(0)|| (rtol: device, nb entries)
template <class V>
static int bpcg(const BOp& op, BatchWork* w, int nb, V* D, V* R, V* Pd, V* Q, V* Z, const double* rtol, int maxit,
                cudaStream_t st) {
    gofd_problem* p = op.p;
    const bool f64 = sizeof(V) == 8;
    const int64_t n = op.n, ld = w->ld;
    BScal* s = w->scal.as<BScal>();
    double* red = w->red.as<double>();
    unsigned* cnt = w->cnt.as<unsigned>();
    const dim3 vg(grid_blocks(n, 256, 512), nb);
    const dim3 rg(BRED_BLOCKS, nb);
    const bool pc = op.member(0)->pc != nullptr;
    const int check = p->opt.check_every > 0 ? p->opt.check_every : 8;
    GOFD_CUDA_TRY(cudaMemsetAsync(D, 0, sizeof(V) * ld * nb, st));
    V* ZZ = R;
    if (pc) {
        for (int c = 0; c < nb; ++c) precond_apply(op.member(c), f64, R + c * ld, Z + c * ld, st);
        ZZ = Z;
    }
    // r0 and tolerances
    {
        bdot_kernel<V><<<rg, BRED_THREADS, 0, st>>>(R, R, n, ld, red, cnt, s, 3);
        bset_start_kernel<<<1, 128, 0, st>>>(s, rtol, nb);
        bdot_kernel<V><<<rg, BRED_THREADS, 0, st>>>(R, ZZ, n, ld, red, cnt, s, 0);
        bcopy_kernel<V><<<vg, 256, 0, st>>>(ZZ, Pd, n, ld);
        GOFD_CHECK_LAUNCH();
    }
    int it = 0;
    // converged columns (BScal::done) are skipped by the product kernels:
    // their alpha is 0 from then on, so their q is never used
    static_assert(sizeof(BScal) % sizeof(int) == 0, "flag stride");
    const int* done_flags = reinterpret_cast<const int*>(reinterpret_cast<const char*>(s) + offsetof(BScal, done));
    const int done_stride = (int)(sizeof(BScal) / sizeof(int));
    auto iteration = [&]() {
        op.apply(f64, Pd, Q, nb, ld, w, st, done_flags, done_stride);
        launch_pdl(bdot_kernel<V>, rg, dim3(BRED_THREADS), 0, st, Pd, Q, n, ld, red, cnt, s, 2);
        launch_pdl(bupdate_kernel<V>, rg, dim3(BRED_THREADS), 0, st, D, R, Pd, Q, n, ld, red, cnt, s, pc ? 1 : 0);
        if (pc) {
            for (int c = 0; c < nb; ++c) precond_apply(op.member(c), f64, R + c * ld, Z + c * ld, st);
            launch_pdl(bdot_kernel<V>, rg, dim3(BRED_THREADS), 0, st, R, Z, n, ld, red, cnt, s, 1);
        }
        launch_pdl(bupdate_p_kernel<V>, vg, dim3(256), 0, st, Pd, ZZ, n, ld, s);
        GOFD_CHECK_LAUNCH();
    };
    const int gi = f64 ? 1 : 0;
    if (w->graph[gi] && w->graph_nb[gi] != nb) {
        cudaGraphExecDestroy(w->graph[gi]);
        w->graph[gi] = nullptr;
    }
    if (!w->graph[gi] && !w->no_graph && st == w->gs && maxit >= check) {
        try {
            build_loop_graph(st, check, iteration, [&](cudaGraphConditionalHandle h) {
                bloop_continue_kernel<<<1, 128, 0, st>>>(h, s, nb, w->ctl.as<int>(), check);
            }, &w->graph[gi]);
            w->graph_nb[gi] = nb;
        } catch (const Error&) {   // no device-side loop here: iterate from the host
            w->graph[gi] = nullptr;
            w->no_graph = true;
            cudaGetLastError();
        }
    }
    bool done = false;
    if (w->graph[gi] && st == w->gs && maxit >= check) {
        bloop_arm_kernel<<<1, 1, 0, st>>>(w->ctl.as<int>(), maxit);
        GOFD_CHECK_LAUNCH();
        GOFD_CUDA_TRY(cudaGraphLaunch(w->graph[gi], st));
        int hc[2] = {0, 0};
        GOFD_CUDA_TRY(cudaMemcpyAsync(hc, w->ctl.ptr, sizeof hc, cudaMemcpyDeviceToHost, st));
        read_bscal(w, nb, st);
        it = hc[0];
        done = true;
        for (int c = 0; c < nb; ++c) done &= w->host[c].done != 0;
    }
    while (!done && it < maxit) {
        iteration();
        ++it;
        if (it % check == 0 || it == maxit) {
            read_bscal(w, nb, st);
            bool all = true;
            for (int c = 0; c < nb; ++c) all &= w->host[c].done != 0;
            if (all) break;
        }
    }
    return it;
}

// Columns of a block solve: column c reads its right-hand side at Fc(c) and
// writes its solution (N_v of its problem) at Uc(c).
struct Cols {
    const double* const* F;   // per instance
    const int64_t* ldf;       // per instance
    double* const* U;         // per instance
    int nbper;
    const double* fcol(int c) const { return F[c / nbper] + (c % nbper) * ldf[c / nbper]; }
};

static void solve_cols(const BOp& op, BatchWork* w, const Cols& cols, gofd_solve_mode mode, gofd_rhs rhs, int nb,
                       double tol, int maxit, gofd_solve_info* infos, cudaStream_t caller) {
    auto t0 = std::chrono::steady_clock::now();
    gofd_problem* p = op.p;
    const cudaStream_t st = w->gs;
    GOFD_CUDA_TRY(cudaEventRecord(w->ev_in, caller));
    GOFD_CUDA_TRY(cudaStreamWaitEvent(st, w->ev_in, 0));
    struct Join {
        BatchWork* w;
        cudaStream_t caller;
        ~Join() {
            cudaEventRecord(w->ev_out, w->gs);
            cudaStreamWaitEvent(caller, w->ev_out, 0);
        }
    } join{w, caller};
    const int64_t n = op.n, ld = w->ld;
    double* B = w->b64.as<double>();
    double* X = w->x64.as<double>();
    double* R = w->r64.as<double>();
    const dim3 vg(grid_blocks(n, 256, 512), nb);
    if (op.members) GOFD_CUDA_TRY(cudaMemsetAsync(B, 0, 8 * ld * nb, st));   // zero past each n_int
    for (int c = 0; c < nb; ++c) assemble_rhs(op.member(c), rhs, cols.fcol(c), B + c * ld, st);
    GOFD_CUDA_TRY(cudaMemsetAsync(X, 0, 8 * ld * nb, st));
    std::vector<double> bn, rn;
    bnorms(op, w, B, nb, bn, st);
    for (double& v : bn) {
        v = std::sqrt(v);
        if (!std::isfinite(v)) fail(GOFD_E_ARG, "a right-hand side has a non-finite entry");
    }
    std::vector<int> outer(nb, 0), inner(nb, 0);
    std::vector<double> rel(nb, 0.0);
    // smallest relative residual the next round expects over the columns
    // still being refined (their last residual times their inner reduction)
    double expected = 1.0;
    int total_inner = 0, rounds = 0;
    bool all_done = false;
    // a timed-out wait of the persistent IC solves ends the solve with GOFD_E_TIMEOUT
    auto check_precond = [&]() {
        for (int c = 0; c < nb; ++c)
            if (c == 0 || op.member(c) != op.member(c - 1)) precond_check(op.member(c), st);
    };
    while (rounds < 200 && total_inner < maxit) {
        if (rounds == 0) {
            bcopy_kernel<double><<<vg, 256, 0, st>>>(B, R, n, ld);
        } else {
            // FP64 residual; in mixed mode its convolution in double-float (2D,
            // 3D) while every refined column expects at least residual_df_floor
            const bool df = mode == GOFD_SOLVE_MIXED && p->d >= 2 && p->opt.fp64_residual == 0 &&
                            expected >= residual_df_floor;
            op.apply(true, X, w->q64.ptr, nb, ld, w, st, nullptr, 0, df);
            bresidual_kernel<<<vg, 256, 0, st>>>(B, w->q64.as<double>(), R, n, ld);
        }
        GOFD_CHECK_LAUNCH();
        bnorms(op, w, R, nb, rn, st);
        all_done = true;
        std::vector<double> inv(nb), scale(nb);
        for (int c = 0; c < nb; ++c) {
            const double r = std::sqrt(rn[c]);
            if (!std::isfinite(r)) {
                check_precond();
                fail(GOFD_E_NOT_CONVERGED, "a residual became non-finite");
            }
            rel[c] = bn[c] > 0 ? r / bn[c] : 0.0;
            const bool act = rel[c] > tol;
            all_done &= !act;
            inv[c] = act ? 1.0 / r : 0.0;
            scale[c] = act ? r : 0.0;
            if (act) ++outer[c];
        }
        if (all_done) break;
        ++rounds;
        const double itol = p->opt.inner_tol > 0 ? p->opt.inner_tol : 1e-4;
        std::vector<double> colv(3 * nb);
        for (int c = 0; c < nb; ++c) {
            colv[c] = inv[c];
            colv[nb + c] = scale[c];
            // FP64: each column straight to its own tolerance; mixed: the inner FP32 tolerance
            // mixed: 1e-4, or the smaller reduction a column near tol still needs
            const double need = scale[c] > 0 ? 0.5 * tol * bn[c] / scale[c] : 1.0;
            colv[2 * nb + c] = mode == GOFD_SOLVE_FP64 ? need : std::max(itol, need);
        }
        expected = 1.0;
        for (int c = 0; c < nb; ++c)
            if (scale[c] > 0) expected = std::min(expected, rel[c] * colv[2 * nb + c]);
        GOFD_CUDA_TRY(cudaMemcpyAsync(w->colv.ptr, colv.data(), 8 * 3 * nb, cudaMemcpyHostToDevice, st));
        const double* dinv = w->colv.as<double>();
        const double* dscale = dinv + nb;
        const double* drtol = dinv + 2 * nb;
        int its;
        if (mode == GOFD_SOLVE_FP64) {
            // columns normalised to unit residual; converged columns are all zero and stay put
            bscale_kernel<<<vg, 256, 0, st>>>(R, dinv, n, ld);
            its = bpcg<double>(op, w, nb, w->d64.as<double>(), R, w->p64.as<double>(), w->q64.as<double>(),
                               w->z64.as<double>(), drtol, maxit - total_inner, st);
            baccumulate64_kernel<<<vg, 256, 0, st>>>(X, w->d64.as<double>(), dscale, n, ld);
        } else {
            bscale_to_f32_kernel<<<vg, 256, 0, st>>>(R, w->r32.as<float>(), dinv, n, ld);
            its = bpcg<float>(op, w, nb, w->d32.as<float>(), w->r32.as<float>(), w->p32.as<float>(),
                              w->q32.as<float>(), w->z32.as<float>(), drtol, maxit - total_inner, st);
            baccumulate_kernel<<<vg, 256, 0, st>>>(X, w->d32.as<float>(), dscale, n, ld);
        }
        GOFD_CHECK_LAUNCH();
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
        total_inner += its;
        for (int c = 0; c < nb; ++c)
            if (scale[c] > 0) inner[c] += its;
        if (its == 0) break;
    }
    for (int c = 0; c < nb; ++c)
        expand_interior(op.member(c), true, X + c * ld, cols.U[c / cols.nbper] + (int64_t)(c % cols.nbper) * op.member(c)->nv,
                        0.0, st);
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    check_precond();
    auto t1 = std::chrono::steady_clock::now();
    if (infos)
        for (int c = 0; c < nb; ++c) {
            gofd_solve_info& info = infos[c];
            const gofd_problem* q = op.member(c);
            info.outer_iters = outer[c];
            info.inner_iters = inner[c];
            info.rel_res_fp64 = rel[c];
            info.a_h = q->a_h;
            info.min_colsum = q->min_colsum;
            info.ic_shift = precond_shift(q);
            const double dd = q->d;
            info.h_within_strict_bound = q->h <= q->a_h / ((dd + 1) * std::sqrt(dd));
            info.h_within_practical_bound = q->h <= q->a_h;
            info.t_setup_ms = q->t_setup_ms;
            info.t_solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
            info.device_loop = !w->no_graph && (w->graph[0] || w->graph[1]);
        }
    if (!all_done) fail(GOFD_E_NOT_CONVERGED, "batched solver reached maxit before tol");
}

void solve_batch(gofd_problem* p, gofd_solve_mode mode, gofd_rhs rhs, int nb, const double* F, int64_t ldf,
                 double tol, int maxit, double* U, gofd_solve_info* infos, cudaStream_t caller) {
    BatchWork* w = ensure_batch(p, nb);
    BOp op;
    op.p = p;
    op.n = p->nint;
    Cols cols{&F, &ldf, &U, nb};
    solve_cols(op, w, cols, mode, rhs, nb, tol, maxit, infos, caller);
}

void apply_batch(gofd_problem* p, bool fp64, const void* x, void* y, int nb, int64_t ld, cudaStream_t st) {
    BatchWork* w = ensure_batch(p, nb);
    apply_interior_batch(p, fp64, x, y, nb, ld, w->grid.ptr, w->spec.ptr, w->partial.ptr, w->counters.ptr, st);
}

// ---------------------------------------------------------------------------
// autotuner: time the batched FP32 product for each launch shape
// ---------------------------------------------------------------------------
static double tune_op(const BOp& op, BatchWork* w, int nb, cudaStream_t st);

double autotune(gofd_problem* p, int nb, cudaStream_t st) {
    BatchWork* w = ensure_batch(p, nb);
    invalidate_graphs(p);
    BOp op;
    op.p = p;
    op.n = p->nint;
    return tune_op(op, w, nb, st);
}

static double tune_op(const BOp& op, BatchWork* w, int nb, cudaStream_t st) {
    gofd_problem* p = op.p;
    for (auto& g : w->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    const int64_t ld = w->ld;
    GOFD_CUDA_TRY(cudaMemsetAsync(w->p32.ptr, 0, 4 * ld * nb, st));
    cudaEvent_t a, b;
    GOFD_CUDA_TRY(cudaEventCreate(&a));
    GOFD_CUDA_TRY(cudaEventCreate(&b));
    // coordinate descent over the choices (each swept with the others at
    // their current best): column elements per thread, row elements per
    // thread (2D), lines per CTA of the row transforms, columns per CTA,
    // scatter lanes per row, sub-batch size (2D batches)
    auto time_current = [&]() {
        op.apply(false, w->p32.ptr, w->q32.ptr, nb, ld, w, st);   // warm
        constexpr int reps = 10;
        GOFD_CUDA_TRY(cudaEventRecord(a, st));
        for (int r = 0; r < reps; ++r) op.apply(false, w->p32.ptr, w->q32.ptr, nb, ld, w, st);
        GOFD_CUDA_TRY(cudaEventRecord(b, st));
        GOFD_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0;
        GOFD_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        return ms / reps;
    };
    const std::vector<int> shapes = p->d == 2 ? std::vector<int>{1, 2, 4} : std::vector<int>{0};
    const std::vector<int> elems = p->d == 1 ? std::vector<int>{0} : std::vector<int>{8, 16, 32};
    // a group always takes the packed scatter: no lane widths to sweep
    const std::vector<int> lanes = op.members ? std::vector<int>{} : std::vector<int>{4, 8, 16, 32};
    const std::vector<int> rowe = p->d >= 2 ? std::vector<int>{8, 16} : std::vector<int>{0};
    p->tune_cole = p->tune_lpc = p->tune_cols = p->tune_tpr = p->tune_bchunk = p->tune_rowe = 0;
    double best = time_current();
    int be = 0, bl = 0, bc = 0, bt = 0, bk = 0, br = 0;
    auto sweep = [&](int* field, const std::vector<int>& vals, int* keep) {
        for (int v : vals) {
            *field = v;
            const double t = time_current();
            if (t < best) {
                best = t;
                *keep = v;
            }
        }
        *field = *keep;
    };
    sweep(&p->tune_cole, elems, &be);
    sweep(&p->tune_rowe, rowe, &br);
    sweep(&p->tune_lpc, shapes, &bl);
    sweep(&p->tune_cols, shapes, &bc);
    sweep(&p->tune_tpr, lanes, &bt);
    if (p->d == 2 && nb > 1 && !op.members) {
        std::vector<int> chunks;
        for (int k : {1, 2, 4})
            if (k < nb) chunks.push_back(k);
        sweep(&p->tune_bchunk, chunks, &bk);
    }
    p->tune_bchunk = bk;
    p->tune_cole = be;
    p->tune_lpc = bl;
    p->tune_cols = bc;
    p->tune_tpr = bt;
    p->tune_rowe = br;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// ---------------------------------------------------------------------------
// groups: problems on one grid solved together (the batched workload)
// ---------------------------------------------------------------------------
struct Group {
    std::vector<gofd_problem*> members;
    int nbper = 0;
    int64_t n = 0;
    BatchWork work;
    DevBuf views;
    GroupArg ga;
    BOp op() {
        BOp o;
        o.p = members[0];
        o.members = &members;
        o.nbper = nbper;
        o.ga = ga;
        o.n = n;
        return o;
    }
};

Group* group_create(int np, gofd_problem* const* probs, int nb) {
    const gofd_problem* r = probs[0];
    for (int i = 0; i < np; ++i) {
        const gofd_problem* q = probs[i];
        if (!q) fail(GOFD_E_ARG, "NULL problem in the group");
        if (q->d != 2) fail(GOFD_E_ARG, "groups are 2D");
        if (q->n[0] != r->n[0] || q->n[1] != r->n[1] || q->P != r->P || q->h != r->h || q->lo[0] != r->lo[0] ||
            q->lo[1] != r->lo[1] || q->device != r->device)
            fail(GOFD_E_ARG, "the problems of a group must share one grid (box, h) and one device");
    }
    auto g = std::make_unique<Group>();
    g->members.assign(probs, probs + np);
    g->nbper = nb;
    std::vector<InstView> v(np);
    int64_t part = 0, cnt = 0;
    for (int i = 0; i < np; ++i) {
        const gofd_problem* q = probs[i];
        v[i] = inst_view(q);
        v[i].part_off = part;
        v[i].cnt_off = cnt;
        part += (int64_t)nb * q->n_long_chunks;
        cnt += (int64_t)nb * q->n_long_rows;
        g->n = std::max<int64_t>(g->n, q->nint);
        g->ga.max_nloc = std::max<int64_t>(g->ga.max_nloc, q->nloc);
        g->ga.max_scatter = std::max<int64_t>(g->ga.max_scatter, q->n_pack + q->n_long_chunks);
        // one symbol per (alpha, Filon M, Richardson levels) on this grid
        for (int j = 0; j < i; ++j) {
            const gofd_problem* o = probs[j];
            if (o->alpha == q->alpha && o->filon_M == q->filon_M && o->rich_levels == q->rich_levels) {
                v[i].lamT32 = v[j].lamT32;
                v[i].lamT64 = v[j].lamT64;
                break;
            }
        }
    }
    g->views.alloc(sizeof(InstView) * np);
    GOFD_CUDA_TRY(cudaMemcpy(g->views.ptr, v.data(), sizeof(InstView) * np, cudaMemcpyHostToDevice));
    g->ga.iv = g->views.as<InstView>();
    g->ga.nbper = nb;
    alloc_batch(&g->work, r, np * nb, g->n + 1, part, cnt);
    return g.release();
}

void group_destroy(Group* g) { delete g; }

double group_autotune(Group* g, cudaStream_t st) {
    BatchWork* w = &g->work;
    for (auto& gr : w->graph)
        if (gr) {
            cudaGraphExecDestroy(gr);
            gr = nullptr;
        }
    invalidate_graphs(g->members[0]);
    const int nb = (int)g->members.size() * g->nbper;
    GOFD_CUDA_TRY(cudaMemsetAsync(w->p32.ptr, 0, 4 * w->ld * nb, st));
    return tune_op(g->op(), w, nb, st);
}

void group_solve(Group* g, gofd_solve_mode mode, gofd_rhs rhs, const double* const* F, const int64_t* ldf, double tol,
                 int maxit, double* const* U, gofd_solve_info* infos, cudaStream_t st) {
    const int np = (int)g->members.size();
    for (int i = 0; i < np; ++i) {
        if (!F[i] || !U[i]) fail(GOFD_E_ARG, "NULL vector");
        if (ldf[i] < (rhs == GOFD_RHS_GRID ? g->members[i]->ngrid : g->members[i]->nv))
            fail(GOFD_E_ARG, "ldf smaller than a column");
    }
    Cols cols{F, ldf, U, g->nbper};
    solve_cols(g->op(), &g->work, cols, mode, rhs, np * g->nbper, tol, maxit, infos, st);
}

}  // namespace gofd
