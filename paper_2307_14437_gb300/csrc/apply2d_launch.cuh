// Host launchers of the transposed-spectrum 2D product, one precision per
// translation unit (REAL is float, double, or dfl: double-float arithmetic
// on FP64 inputs, weights, symbol and outputs).
#include <type_traits>

#include "apply2d.cuh"

namespace gofd {

void mark_stage(cudaStream_t st, const char* name);

namespace {

using Real = REAL;
using C = Cplx<Real>::T;
using S = Sto<Real>::T;   // inputs, weights, symbol and outputs

const C* twiddles(const gofd_problem* p) {
    if constexpr (std::is_same<Real, float>::value) return reinterpret_cast<const C*>(p->tw32.ptr);
    else if constexpr (std::is_same<Real, double>::value) return reinterpret_cast<const C*>(p->tw64.ptr);
    else return reinterpret_cast<const C*>(p->twdf.ptr);
}

// elements per thread (largest radix) of the row and column transforms
constexpr int ct_elems_row(int N) { return N >= 4096 ? 16 : 8; }
constexpr int ct_elems_col(int N) { return N >= 4096 ? 16 : 8; }
// column transform: 8, 16 or 32 elements per thread (32 only in FP32 and for
// lines of at least 1024: one warp or more per column); tuned > 0 selects one,
// 0 the default (32 for FP32 lines >= 2048, else the table above)
// launch bounds of the column kernel: at most max(N/E, 256) threads; with 32
// elements per thread the registers are capped for two CTAs per SM
constexpr int col_maxt(int N, int E) { return N / E > 256 ? N / E : 256; }
constexpr int col_minb(int E) { return E == 32 ? 2 : 1; }
template <int N, int E>
constexpr auto col_kernel() { return col_conv_t_kernel<Real, N, E, col_maxt(N, E), col_minb(E)>; }

int col_elems(int N, int tuned) {
    const bool fp32 = sizeof(Real) == 4;
    auto ok = [&](int e) { return e == 8 || (e == 16 && N >= 512) || (e == 32 && fp32 && N >= 1024); };
    if (tuned > 0 && ok(tuned)) return tuned;
    if (fp32 && N >= 2048) return 32;
    return ct_elems_col(N);
}
// row transforms: 8 or 16 elements per thread; tuned > 0 selects the other
// one for FP32 lines of 512 to 2048 complex points
constexpr bool row_alt(int NR) { return NR >= 512 && NR <= 2048; }
constexpr int row_alt_elems(int NR) { return ct_elems_row(NR) == 8 ? 16 : 8; }
int row_elems(int NR, int tuned) {
    if (sizeof(Real) == 4 && row_alt(NR) && tuned == row_alt_elems(NR)) return tuned;
    return ct_elems_row(NR);
}
int lines_per_cta(int nthr, int tuned) {
    if (tuned > 0 && (tuned & (tuned - 1)) == 0 && tuned * nthr <= 512 && tuned <= 4) return tuned;
    return std::max(1, std::min(4, 512 / nthr));
}
// the column kernel is compiled for at most max(N/E, 256) threads per CTA;
// by default a CTA takes one column (two or four when a column has fewer
// than 64 threads): with about a thousand columns this spreads them evenly
// over the SMs (at 2048 x 1025, four columns per CTA leave 257 CTAs for 152
// SMs and cost 5 us of a 61 us product)
int cols_per_cta(int nthr, int tuned) {
    if (tuned > 0 && (tuned & (tuned - 1)) == 0 && tuned * nthr <= std::max(nthr, 256) && tuned <= 4) return tuned;
    return std::max(1, std::min(4, 64 / nthr));
}
size_t row_smem(int N, int lpc) {
    return sizeof(C) * std::max<size_t>((size_t)spad_len(N) * lpc, (size_t)tile_ld(N + 1, lpc) * lpc);
}
size_t col_smem(int N, int G) { return sizeof(C) * (size_t)spad_len(N) * G; }

template <int N>
void set_attrs(int limit) {
    constexpr int ER = ct_elems_row(N / 2);
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_fwd_t_kernel<Real, 3, N / 2, ER>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_inv_t_kernel<Real, N / 2, ER>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    if constexpr (sizeof(Real) == 4 && row_alt(N / 2)) {
        constexpr int EA = row_alt_elems(N / 2);
        GOFD_CUDA_TRY(cudaFuncSetAttribute(row_fwd_t_kernel<Real, 3, N / 2, EA>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
        GOFD_CUDA_TRY(cudaFuncSetAttribute(row_inv_t_kernel<Real, N / 2, EA>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    }
    GOFD_CUDA_TRY(cudaFuncSetAttribute(col_kernel<N, 8>(), cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    if constexpr (N >= 512)
        GOFD_CUDA_TRY(cudaFuncSetAttribute(col_kernel<N, 16>(), cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    if constexpr (N >= 1024 && sizeof(Real) == 4)
        GOFD_CUDA_TRY(cudaFuncSetAttribute(col_kernel<N, 32>(), cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
}

// P = circulant length (column lines), rows use P/2; nb right-hand sides with
// strides xs (input), ws (output grid) and the batch spectrum buffer
template <int P, int EC, int ER>
void run_e(gofd_problem* p, const S* x, const S* vgrid, S* wgrid, int nb, int64_t xs, int64_t ws, C* Sp,
           cudaStream_t st, GroupArg ga) {
    constexpr int NR = P / 2, NC = P;
    constexpr int tr = NR / ER, tc = NC / EC;
    const int lpc = lines_per_cta(tr, p->tune_lpc), G = cols_per_cta(tc, p->tune_cols);
    const int n = p->n[0], H = P / 2 + 1, nlines = (int)p->nlines;
    const C* tw = twiddles(p);
    const S* lamT = reinterpret_cast<const S*>(sizeof(Real) == 4 ? p->lamT32.ptr : p->lamT64.ptr);
    const S* w = reinterpret_cast<const S*>(sizeof(Real) == 4 ? p->ell_w32.ptr : p->ell_w64.ptr);
    const int64_t ss = (int64_t)H * p->ldT;
    const unsigned rblocks = (unsigned)((nlines + lpc - 1) / lpc);
    const int64_t sb = nb > 1 ? ss : 0;
    launch_pdl(row_fwd_t_kernel<Real, 3, NR, ER>, dim3(rblocks, nb), dim3(lpc * tr), row_smem(NR, lpc), st, x,
               p->ell_iidx.as<int32_t>(), w, p->nloc, p->line_run_ptr.as<int32_t>(), p->run_k0.as<int32_t>(),
               p->run_len.as<int32_t>(), p->run_e0.as<int32_t>(), vgrid, nlines, n, tw, Sp, p->ldT, lpc, xs, sb, ga);
    mark_stage(st, "gather_row_fft");
    launch_pdl(col_kernel<NC, EC>(), dim3((unsigned)((H + G - 1) / G), nb), dim3(G * tc), col_smem(NC, G), st, Sp,
               p->ldT, n, H, H, tw, lamT, sb, 0, (int64_t)0, ga);
    mark_stage(st, "col_fft_conv");
    launch_pdl(row_inv_t_kernel<Real, NR, ER>, dim3(rblocks, nb), dim3(lpc * tr), row_smem(NR, lpc), st, Sp, p->ldT,
               nlines, n, tw, wgrid, lpc, sb, ws, ga);
    mark_stage(st, "row_ifft");
}

template <int P, int EC>
void run_r(gofd_problem* p, const S* x, const S* vgrid, S* wgrid, int nb, int64_t xs, int64_t ws, C* Sp,
           cudaStream_t st, GroupArg ga) {
    constexpr int ER = ct_elems_row(P / 2);
    if constexpr (sizeof(Real) == 4 && row_alt(P / 2))
        if (row_elems(P / 2, p->tune_rowe) != ER)
            return run_e<P, EC, row_alt_elems(P / 2)>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga);
    run_e<P, EC, ER>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga);
}

template <int P>
void run(gofd_problem* p, const S* x, const S* vgrid, S* wgrid, int nb, int64_t xs, int64_t ws, C* Sp,
         cudaStream_t st, GroupArg ga) {
    const int e = col_elems(P, p->tune_cole);
    if constexpr (P >= 1024 && sizeof(Real) == 4)
        if (e == 32) return run_r<P, 32>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga);
    if constexpr (P >= 512)
        if (e == 16) return run_r<P, 16>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga);
    run_r<P, 8>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga);
}

}  // namespace

void AFD2D_FN(gofd_problem* p, const S* x, const S* vgrid, S* wgrid, int nb, int64_t xs, int64_t ws,
              void* spec, cudaStream_t st, GroupArg ga) {
    if constexpr (sizeof(Real) == 4)
        if (!vgrid && afd_2d_warp_eligible(p)) {
            afd_2d_warp_f32(p, reinterpret_cast<const float*>(x), reinterpret_cast<float*>(wgrid), nb, xs, ws, spec,
                            st, ga);
            return;
        }
    C* Sp = spec ? static_cast<C*>(spec) : p->specT.as<C>();
    switch (p->P) {
        case 32: run<32>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga); break;
        case 64: run<64>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga); break;
        case 128: run<128>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga); break;
        case 256: run<256>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga); break;
        case 512: run<512>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga); break;
        case 1024: run<1024>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga); break;
        case 2048: run<2048>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga); break;
        case 4096: run<4096>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga); break;
        case 8192: run<8192>(p, x, vgrid, wgrid, nb, xs, ws, Sp, st, ga); break;
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
    const int tr = P / 2 / ct_elems_row(P / 2);
    size_t nd = 0;
    for (int k = 1; k <= 4; ++k) {   // every shape the autotuner may pick
        if (k * tr <= 512) nd = std::max(nd, row_smem(P / 2, k));
        for (int e : {8, 16, 32}) {
            const int tc = P / e;
            if (tc >= 1 && k * tc <= std::max(tc, 256)) nd = std::max(nd, col_smem(P, k));
        }
    }
    *need = nd;
}

}  // namespace gofd
