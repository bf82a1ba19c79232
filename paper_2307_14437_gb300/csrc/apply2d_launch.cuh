// Host launchers of the transposed-spectrum 2D product, one precision per
// translation unit (REAL is float or double).
#include "apply2d.cuh"

namespace gofd {

void mark_stage(cudaStream_t st, const char* name);

namespace {

using Real = REAL;
using C = Cplx<Real>::T;

// elements per thread (largest radix) of the row and column transforms
constexpr int ct_elems_row(int N) { return N >= 4096 ? 16 : 8; }
constexpr int ct_elems_col(int N) { return N >= 4096 ? 16 : 8; }
int lines_per_cta(int nthr) { return std::max(1, std::min(4, 512 / nthr)); }
int cols_per_cta(int nthr) { return std::max(1, std::min(4, 256 / nthr)); }
size_t row_smem(int N, int lpc) { return sizeof(C) * std::max<size_t>((size_t)spad_len(N) * lpc, (size_t)(N + 1) * lpc); }
size_t col_smem(int N, int G) { return sizeof(C) * (size_t)spad_len(N) * G; }

template <int N>
void set_attrs(int limit) {
    constexpr int ER = ct_elems_row(N / 2), EC = ct_elems_col(N);
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_fwd_t_kernel<Real, 3, N / 2, ER>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_inv_t_kernel<Real, N / 2, ER>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(col_conv_t_kernel<Real, N, EC>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
}

// P = circulant length (column lines), rows use P/2
template <int P>
void run(gofd_problem* p, const Real* x, const Real* vgrid, Real* wgrid, cudaStream_t st) {
    constexpr int NR = P / 2, NC = P;
    constexpr int ER = ct_elems_row(NR), EC = ct_elems_col(NC);
    constexpr int tr = NR / ER, tc = NC / EC;
    const int lpc = lines_per_cta(tr), G = cols_per_cta(tc);
    const int n = p->n[0], H = P / 2 + 1, nlines = (int)p->nlines;
    const C* tw = reinterpret_cast<const C*>(sizeof(Real) == 4 ? p->tw32.ptr : p->tw64.ptr);
    const Real* lamT = reinterpret_cast<const Real*>(sizeof(Real) == 4 ? p->lamT32.ptr : p->lamT64.ptr);
    const Real* w = reinterpret_cast<const Real*>(sizeof(Real) == 4 ? p->ell_w32.ptr : p->ell_w64.ptr);
    C* S = p->specT.as<C>();
    const unsigned rblocks = (unsigned)((nlines + lpc - 1) / lpc);
    row_fwd_t_kernel<Real, 3, NR, ER><<<rblocks, lpc * tr, row_smem(NR, lpc), st>>>(
        x, p->ell_iidx.as<int32_t>(), w, p->nloc, p->line_run_ptr.as<int32_t>(), p->run_k0.as<int32_t>(),
        p->run_len.as<int32_t>(), p->run_e0.as<int32_t>(), vgrid, nlines, n, tw, S, p->ldT, lpc);
    GOFD_CHECK_LAUNCH();
    mark_stage(st, "gather_row_fft");
    col_conv_t_kernel<Real, NC, EC><<<(unsigned)((H + G - 1) / G), G * tc, col_smem(NC, G), st>>>(S, p->ldT, n, H, tw, lamT);
    GOFD_CHECK_LAUNCH();
    mark_stage(st, "col_fft_conv");
    row_inv_t_kernel<Real, NR, ER><<<rblocks, lpc * tr, row_smem(NR, lpc), st>>>(S, p->ldT, nlines, n, tw, wgrid, lpc);
    GOFD_CHECK_LAUNCH();
    mark_stage(st, "row_ifft");
}

}  // namespace

void AFD2D_FN(gofd_problem* p, const Real* x, const Real* vgrid, Real* wgrid, cudaStream_t st) {
    switch (p->P) {
        case 32: run<32>(p, x, vgrid, wgrid, st); break;
        case 64: run<64>(p, x, vgrid, wgrid, st); break;
        case 128: run<128>(p, x, vgrid, wgrid, st); break;
        case 256: run<256>(p, x, vgrid, wgrid, st); break;
        case 512: run<512>(p, x, vgrid, wgrid, st); break;
        case 1024: run<1024>(p, x, vgrid, wgrid, st); break;
        case 2048: run<2048>(p, x, vgrid, wgrid, st); break;
        case 4096: run<4096>(p, x, vgrid, wgrid, st); break;
        case 8192: run<8192>(p, x, vgrid, wgrid, st); break;
        default: fail(GOFD_E_GRID, "unsupported circulant length");
    }
}

void AFD2D_ATTR_FN(int limit, int P, size_t* need) {
    switch (P) {
#define ATTR(PP) case PP: set_attrs<PP>(limit); break;
        ATTR(32) ATTR(64) ATTR(128) ATTR(256) ATTR(512) ATTR(1024) ATTR(2048) ATTR(4096) ATTR(8192)
#undef ATTR
        default: fail(GOFD_E_GRID, "unsupported circulant length");
    }
    const int tr = P / 2 / ct_elems_row(P / 2), tc = P / ct_elems_col(P);
    *need = std::max(row_smem(P / 2, lines_per_cta(tr)), col_smem(P, cols_per_cta(tc)));
}

}  // namespace gofd
