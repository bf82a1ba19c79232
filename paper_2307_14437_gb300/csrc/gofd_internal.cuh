// Internal declarations shared by the GoFD CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gofd.h"

namespace gofd {

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
struct Error {
    gofd_status code;
    std::string msg;
};

#define GOFD_CUDA_TRY(expr)                                                        \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess)                                                     \
            throw ::gofd::Error{GOFD_E_CUDA, std::string(#expr) + ": " +           \
                                             cudaGetErrorString(_e)};              \
    } while (0)

#define GOFD_CHECK_LAUNCH() GOFD_CUDA_TRY(cudaGetLastError())

[[noreturn]] inline void fail(gofd_status c, const std::string& m) { throw Error{c, m}; }

// ---------------------------------------------------------------------------
// programmatic dependent launch
//
// The kernels of the product are launched with programmatic stream
// serialization: a kernel's CTAs may be scheduled while the previous kernel in
// the stream is still running.  Each such kernel first lets its own successor
// be scheduled (launch_dependents) and then waits until its predecessor has
// completed and its memory is visible (griddepcontrol.wait, a no-op for an
// ordinary launch).  Before that wait a kernel only reads data that no kernel
// of the product writes (set-up tables: runs, CSR structure and weights) and
// writes nothing.  Every CTA waits, so a kernel completes only after its
// predecessor has, and the ordering is transitive.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_trigger() {
#if defined(__CUDA_ARCH__)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__)
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_enter() {
    pdl_trigger();
    pdl_wait();
}

template <class... KArgs, class... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    GOFD_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
}

// ---------------------------------------------------------------------------
// device-side solver loops: a CUDA graph whose conditional while node runs
// `check` iterations (body, captured from stream st) followed by a control
// kernel (control(handle), which calls cudaGraphSetConditional) as long as the
// control kernel asks for more.  *exec receives the instantiated graph.
// ---------------------------------------------------------------------------
template <class Body, class Control>
void build_loop_graph(cudaStream_t st, int check, Body& body, Control control, cudaGraphExec_t* exec) {
    cudaGraph_t g = nullptr;
    GOFD_CUDA_TRY(cudaGraphCreate(&g, 0));
    struct Guard {
        cudaGraph_t g;
        ~Guard() { cudaGraphDestroy(g); }
    } guard{g};
    cudaGraphConditionalHandle h;
    GOFD_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    GOFD_CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    GOFD_CUDA_TRY(cudaStreamBeginCaptureToGraph(st, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
        for (int k = 0; k < check; ++k) body();
        control(h);
        GOFD_CUDA_TRY(cudaGetLastError());
    } catch (...) {
        cudaGraph_t tmp = nullptr;
        cudaStreamEndCapture(st, &tmp);
        throw;
    }
    cudaGraph_t out = nullptr;
    GOFD_CUDA_TRY(cudaStreamEndCapture(st, &out));
    const cudaError_t e = cudaGraphInstantiate(exec, g, 0);
    if (e != cudaSuccess) {
        *exec = nullptr;
        fail(GOFD_E_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
    }
}

// ---------------------------------------------------------------------------
// device buffers owned by the handle
// ---------------------------------------------------------------------------
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void alloc(size_t b) {
        release();
        if (b == 0) b = 16;
        cudaError_t e = cudaMalloc(&ptr, b);
        if (e != cudaSuccess) {
            ptr = nullptr;
            throw Error{GOFD_E_NOMEM, "cudaMalloc of " + std::to_string(b) + " bytes: " +
                                          cudaGetErrorString(e)};
        }
        bytes = b;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// ---------------------------------------------------------------------------
// FFT plans (per line length)
// ---------------------------------------------------------------------------
struct LinePlan {
    int N = 0;               // complex line length (power of two)
    int nthr = 0;            // threads per line = N / 16 (or N if N < 16)
    int npass = 0;
    int radix[8] = {0};
};
LinePlan make_line_plan(int N);

// ---------------------------------------------------------------------------
// the problem handle
// ---------------------------------------------------------------------------
// A group of 2D problems on the same grid, solved together: the batched
// product kernels take the instance of column blockIdx.y (instance
// blockIdx.y / nbper) from a device table of these views.
struct InstView {
    const int32_t* ell_iidx;
    const float* ell_w32;
    const double* ell_w64;
    const int32_t* ell_node;
    int64_t nloc;
    const int32_t *run_ptr, *run_k0, *run_len, *run_e0;
    const int4* wdesc_line;
    const int32_t* ell4_node;   // 2D warp-FFT path: the ELL with its slot stride padded to ell4_ld
    const int32_t* ell4_iidx;
    const float* ell4_w32;
    int64_t ell4_ld;
    const float* lamT32;
    const double* lamT64;
    const int32_t *csr_ptr, *csr_col;
    const float* csr_val32;
    const double* csr_val64;
    const int4* pack_desc;
    int64_t n_pack;
    const int32_t *cbeg, *cend, *crow, *lrows, *cptr;   // long rows of I^T and their chunks
    int64_t nchunks, nrows;
    int64_t part_off, cnt_off;   // this instance's long-row partial sums / counters in the group workspace
};
struct GroupArg {
    const InstView* iv = nullptr;   // nullptr: one problem (the kernel's own arguments)
    int nbper = 1;                  // columns per instance
    int64_t max_nloc = 0;           // host side: largest n_loc / scatter grid over the instances
    int64_t max_scatter = 0;
    // block PCG: column c of the launch (blockIdx.y) is left untouched when
    // skip[(col0 + c) * skip_stride] != 0 (the column has converged; its
    // output is not read).  nullptr: every column is computed.
    const int* skip = nullptr;
    int skip_stride = 0;
    int col0 = 0;
    // symbol in the column kernels' layout (lamT32 / lamT64) used instead of
    // the problem's: the circulant preconditioner's 1/lambda (nullptr: lambda)
    const float* lam32 = nullptr;
    const double* lam64 = nullptr;
};

// True when this CTA's column is to be left alone.  Call it after pdl_wait():
// the flags are written by an earlier kernel of the same stream, and only
// after the wait is that kernel known to be complete.  The flag is the same
// for every CTA of a column, so a whole column returns or none of it.
__device__ __forceinline__ bool column_skipped(const GroupArg& ga) {
    return ga.skip && *(const volatile int*)(ga.skip + (int64_t)(ga.col0 + (int)blockIdx.y) * ga.skip_stride) != 0;
}

struct Precond;   // defined in precond.cu

struct Workspace;  // solver vectors, defined in solver.cu

struct Adjoint;    // adjoint buffers, defined in adjoint.cu
struct BatchWork;  // many-right-hand-side solver vectors, defined in batch.cu

}  // namespace gofd

struct gofd_problem {
    // inputs
    int d = 0;
    int64_t nv = 0, ne = 0;
    double alpha = 0, s = 0, h = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int n[3] = {1, 1, 1};
    int64_t ngrid = 0;
    int64_t nlines = 0;        // n_1*n_2 (lines along axis 0)
    int P = 0;                 // circulant length per axis
    int64_t filon_M = 0;
    int rich_levels = 4;
    gofd_options opt{};
    cudaStream_t setup_stream = nullptr;
    int sm_count = 152;   // multiprocessors of the device (set at build)
    int device = 0;

    // mesh on the device
    gofd::DevBuf verts, simp;

    // point location / transfer
    gofd::DevBuf owner;        // int32 [ngrid]
    int64_t nloc = 0;
    gofd::DevBuf ell_node;     // int32 [nloc]      grid index of each ELL row
    gofd::DevBuf ell_vidx;     // int32 [(d+1)*nloc] vertex numbering (canonical)
    gofd::DevBuf ell_w64;      // double[(d+1)*nloc]
    gofd::DevBuf ell_w32;      // float [(d+1)*nloc]
    gofd::DevBuf ell_iidx;     // int32 [(d+1)*nloc] interior numbering, boundary -> nint (zero slot)
    gofd::DevBuf wdesc_line;   // 2D warp-FFT path: per-line run descriptors (2 int4 per line)
    // 2D warp-FFT path: node, interior index and FP32 weight of the ELL with
    // the slot stride ell4_ld = n_loc rounded up to 4 (every slot 16-byte
    // aligned; padding rows: node -1, index 0, weight 0), read four rows at a time
    gofd::DevBuf ell4_node, ell4_iidx, ell4_w32;
    int64_t ell4_ld = 0;
    int64_t nruns = 0;
    gofd::DevBuf line_run_ptr; // int32 [nlines+1]
    gofd::DevBuf run_k0;       // int32 [nruns]   first k0 of the run
    gofd::DevBuf run_len;      // int32 [nruns]
    gofd::DevBuf run_e0;       // int32 [nruns]   ELL row of the first node

    // vertices
    int64_t nint = 0;
    gofd::DevBuf vert2int;     // int32 [nv], -1 on the boundary
    gofd::DevBuf int2vert;     // int32 [nint]
    gofd::DevBuf csr_ptr;      // int32 [nint+1]
    gofd::DevBuf csr_col;      // int32 [nnz]   grid index
    gofd::DevBuf csr_val64;    // double[nnz]
    gofd::DevBuf csr_val32;    // float [nnz]
    int64_t nnz_t = 0;
    gofd::DevBuf colsum;       // double[nint]  D_h over interior vertices
    gofd::DevBuf long_rows;    // int32 [n_long_rows] rows of I^T with more than 1024 entries
    gofd::DevBuf long_chunk_ptr, chunk_beg, chunk_end, chunk_row;  // chunks of the long rows
    gofd::DevBuf long_cnt;     // unsigned [n_long_rows] chunk counters (zero between products)
    gofd::DevBuf long_partial; // chunk partial sums (largest precision)
    int64_t n_long_rows = 0, n_long_chunks = 0;
    gofd::DevBuf pack_desc;    // int4 [n_pack] packed runs of short rows {r0, r1, e0, e1} (default scatter)
    int64_t n_pack = 0;
    double a_h = 0, min_colsum = 0;

    // coefficients and symbol
    gofd::DevBuf T;            // double[n^d]
    gofd::DevBuf lam64;        // double[(P/2+1)^d], scaled by 1/P^d
    gofd::DevBuf lam32;        // float [(P/2+1)^d], scaled by 1/P^d
    gofd::DevBuf tw64, tw32;   // twiddle tables e^{-2 pi i m / L} for L = P and P/2 (concatenated)
    gofd::DevBuf twdf;         // the P-point table in double-float (float4: re hi, re lo, im hi, im lo)
    gofd::DevBuf twp32;        // 2D warp-FFT path: W_1024^{i j} at [i*32 + j] (float2)

    // FFT convolution work buffers
    int pitch0 = 0;            // complex entries per spectrum row along axis 0 (>= P/2+1)
    gofd::DevBuf specA;        // complex, n_{d-1}..n_1 rows x pitch0 (largest precision)
    gofd::DevBuf specB;        // 3D only: n x P x pitch0 complex
    gofd::DevBuf specT;        // 2D/3D: transposed half spectrum, (P/2+1) x ldT complex
    int ldT = 0;               // leading dimension of specT (n^(d-1) rounded up to 16)
    gofd::DevBuf specM;        // 3D: middle-stage buffer for midK planes, midK x P x n complex
    int midK = 0;              // 3D: planes k_x0 per chunk of the middle stage
    int tune_lpc = 0, tune_cols = 0, tune_tpr = 0;  // launch shapes picked by the autotuner (0 = default)
    int tune_cole = 0;         // elements per thread of the column transforms (0 = default)
    int tune_rowe = 0;         // elements per thread of the 2D row transforms (0 = default)
    int tune_bchunk = 0;       // 2D batched product: columns per sub-batch (0 = all)
    gofd::DevBuf lamT64, lamT32;  // 2D/3D: scaled symbol with the axis order reversed
    gofd::DevBuf gridw;        // real [ngrid] (largest precision): A_FD v on the grid
    gofd::DevBuf xin;          // real [nint+1] compacted input (largest precision)
    gofd::DevBuf yout;         // real [nint]
    gofd::DevBuf stage_u, stage_y;  // host-call staging (allocated on first use)

    // solver / preconditioner
    gofd::Workspace* ws = nullptr;
    gofd::Precond* pc = nullptr;
    gofd::Adjoint* adj = nullptr;
    gofd::BatchWork* batch = nullptr;

    double t_setup_ms = 0;
    std::string last_error;
};

namespace gofd {

// set-up stages (setup_mesh.cu)
void setup_mesh(gofd_problem* p, const double* verts_h, const int32_t* simp_h);

// coefficients and symbol (coeff.cu)
void setup_coefficients(gofd_problem* p);

// FFT-convolution apply (apply.cu)
void setup_apply(gofd_problem* p);
void setup_apply_2d(gofd_problem* p);
void setup_apply_3d(gofd_problem* p);
void afd_3d_f32(gofd_problem* p, const float* x, const float* vgrid, float* wgrid, cudaStream_t st);
void afd_3d_f64(gofd_problem* p, const double* x, const double* vgrid, double* wgrid, cudaStream_t st);
void afd_3d_df(gofd_problem* p, const double* x, const double* vgrid, double* wgrid, cudaStream_t st);
void afd_3d_attrs_df(int limit, int P, size_t* need);
// nb right-hand sides: inputs at x + b*xs (or vgrid + b*xs), outputs at wgrid + b*ws;
// spec = batch spectrum buffer (nb x (P/2+1) x ldT complex) or NULL for one vector
void afd_2d_f32(gofd_problem* p, const float* x, const float* vgrid, float* wgrid, int nb, int64_t xs, int64_t ws,
                void* spec, cudaStream_t st, GroupArg ga = GroupArg{});
void afd_2d_f64(gofd_problem* p, const double* x, const double* vgrid, double* wgrid, int nb, int64_t xs,
                int64_t ws, void* spec, cudaStream_t st, GroupArg ga = GroupArg{});
// the same with FP64 inputs and outputs and the transforms in double-float
// arithmetic (apply2d_df.cu): FP64-accurate (about 1e-13) at FP32 rates
void afd_2d_df(gofd_problem* p, const double* x, const double* vgrid, double* wgrid, int nb, int64_t xs,
               int64_t ws, void* spec, cudaStream_t st, GroupArg ga = GroupArg{});
void afd_2d_attrs_df(int limit, int P, size_t* need);
// 2D FP32 product for a 2048-point circulant, one warp per 1024-point FFT
// (apply2d_warp.cu); used by afd_2d_f32 when eligible (default launch shapes)
void setup_apply_2d_warp(gofd_problem* p);
bool afd_2d_warp_eligible(const gofd_problem* p);
void afd_2d_warp_f32(gofd_problem* p, const float* x, float* wgrid, int nb, int64_t xs, int64_t ws, void* spec,
                     cudaStream_t st, GroupArg ga = GroupArg{});

void apply_interior(gofd_problem* p, bool fp64, const void* x, void* y, cudaStream_t st);
// y = S x in FP64 with the FFT convolution in double-float arithmetic (2D, 3D)
void apply_interior_df(gofd_problem* p, const double* x, double* y, cudaStream_t st);
// the mixed solver's FP64 residual product: apply_interior_df in 2D and 3D unless
// opt.fp64_residual asks for plain FP64, else the FP64 product
void apply_interior_residual(gofd_problem* p, const double* x, double* y, cudaStream_t st);
// the mixed solvers use apply_interior_residual for a refinement step's
// residual while its expected relative size is at least this, plain FP64 below
constexpr double residual_df_floor = 1e-9;
void afd_apply_grid(gofd_problem* p, bool fp64, const void* v, void* w, cudaStream_t st);
void afd_apply_noalloc(int d, int n, const float* lam, const float* v, float* w, cudaStream_t st);
int apply_interior_profiled(gofd_problem* p, bool fp64, const void* x, void* y, cudaStream_t st, float* ms,
                            const char** names, int cap);
void compact_vertex(gofd_problem* p, bool fp64, const void* u, void* x, cudaStream_t st);
void expand_interior(gofd_problem* p, bool fp64, const void* y, void* u, double scale_by_inv_colsum,
                     cudaStream_t st);

// solver (solver.cu)
void solve(gofd_problem* p, gofd_solve_mode mode, gofd_rhs rhs, const double* f, double tol,
           int maxit, bool init_zero, double* u, gofd_solve_info* info, cudaStream_t st);
void free_workspace(gofd_problem* p);
void invalidate_graphs(gofd_problem* p);   // drop captured solver iterations
void solve_core(gofd_problem* p, gofd_solve_mode mode, const double* b, double tol, int maxit, bool init_zero,
                double* x, gofd_solve_info* info, cudaStream_t st);
void assemble_rhs(gofd_problem* p, gofd_rhs rhs, const double* f, double* b, cudaStream_t st);

// preconditioner (precond.cu)
void setup_precond(gofd_problem* p);
void free_precond(gofd_problem* p);
int64_t precond_nnz(const gofd_problem* p);
double precond_shift(const gofd_problem* p);
int precond_levels(const gofd_problem* p);
void precond_export(const gofd_problem* p, int32_t* perm, int32_t* lptr, int32_t* lcol, double* lval);
void precond_diagonal(const gofd_problem* p, double* diag);
// z = M^{-1} r on interior vectors (length nint); fp64 selects the precision
void precond_apply(gofd_problem* p, bool fp64, const void* r, void* z, cudaStream_t st);
// GOFD_E_TIMEOUT if a wait of the persistent IC solves ran out (synchronises st)
void precond_check(gofd_problem* p, cudaStream_t st);

// utilities (setup_mesh.cu)
int64_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st);
int grid_blocks(int64_t work, int threads, int cap = 152 * 16);
void sort_packed_rows(const int32_t* ptr, int64_t nrows, int64_t* packed, int64_t nnz, cudaStream_t st);
// partial_ws: nb x n_long_chunks reals (8 bytes each), counter_ws: nb x n_long_rows
// unsigned, zero on entry and on exit
// skip (2D): column c is left untouched when skip[c * skip_stride] != 0
// (device flags, read by the kernels; nullptr: every column is computed)
// df (2D, fp64): the FFT convolution in double-float arithmetic
void apply_interior_batch(gofd_problem* p, bool fp64, const void* x, void* y, int nb, int64_t ld, void* grid_ws,
                          void* spec_ws, void* partial_ws, void* counter_ws, cudaStream_t st,
                          const int* skip = nullptr, int skip_stride = 0, bool df = false);
// a group of 2D problems on one grid (apply.cu): the view of one problem, and
// Y[c] = S_{c / nbper} X[c] for all columns of the group in one launch sequence
InstView inst_view(const gofd_problem* p);
void apply_interior_group(gofd_problem* rp, bool fp64, const void* x, void* y, int nbtot, int64_t ld, void* grid_ws,
                          void* spec_ws, void* partial_ws, void* counter_ws, GroupArg ga, cudaStream_t st,
                          bool df = false);
// y = I^T C I x (2D, interior-compacted vectors) with the column kernels'
// symbol replaced by lamT (FP32 or FP64 as the precision, layout of lamT32)
void apply_interior_symbol(gofd_problem* p, bool fp64, const void* x, void* y, const void* lamT, cudaStream_t st);
// w = A_FD I x on the grid for an interior-compacted x (n_int + 1 entries)
void afd_of_interior(gofd_problem* p, bool fp64, const void* x, void* wgrid, cudaStream_t st);
// adjoint (adjoint.cu)
void adjoint(gofd_problem* p, gofd_solve_mode mode, const double* f, const double* u, const double* g, double tol,
             int maxit, double* grad_f, double* grad_x, gofd_solve_info* info, cudaStream_t st);
void free_adjoint(gofd_problem* p);
// many right-hand sides (batch.cu): F column c at F + c*ldf, U column c at U + c*nv
void solve_batch(gofd_problem* p, gofd_solve_mode mode, gofd_rhs rhs, int nb, const double* F, int64_t ldf,
                 double tol, int maxit, double* U, gofd_solve_info* infos, cudaStream_t st);
double autotune(gofd_problem* p, int nb, cudaStream_t st);
void apply_batch(gofd_problem* p, bool fp64, const void* x, void* y, int nb, int64_t ld, cudaStream_t st);
void free_batch(gofd_problem* p);
// groups of 2D problems on one grid (batch.cu)
struct Group;
Group* group_create(int np, gofd_problem* const* probs, int nb);
void group_destroy(Group* g);
double group_autotune(Group* g, cudaStream_t st);
void group_solve(Group* g, gofd_solve_mode mode, gofd_rhs rhs, const double* const* F, const int64_t* ldf, double tol,
                 int maxit, double* const* U, gofd_solve_info* infos, cudaStream_t st);

}  // namespace gofd
