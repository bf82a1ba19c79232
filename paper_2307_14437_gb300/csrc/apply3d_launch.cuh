// Host launchers of the 3D product, one precision per translation unit
// (REAL is float, double, or dfl: double-float arithmetic on FP64 inputs,
// weights, symbol and outputs): axis-0 row kernels over the n^2 grid lines,
// then per k_x0 plane the (axis 1, axis 2) convolution of apply3d.cuh.
#include <type_traits>

#include "apply3d.cuh"

namespace gofd {

void mark_stage(cudaStream_t st, const char* name);

namespace {

using Real = REAL;
using C = Cplx<Real>::T;
using S = Sto<Real>::T;   // inputs, weights, symbol and outputs

const C* twiddles3(const gofd_problem* p) {
    if constexpr (std::is_same<Real, float>::value) return reinterpret_cast<const C*>(p->tw32.ptr);
    else if constexpr (std::is_same<Real, double>::value) return reinterpret_cast<const C*>(p->tw64.ptr);
    else return reinterpret_cast<const C*>(p->twdf.ptr);
}

constexpr int ct3_elems(int N) { return N >= 4096 ? 16 : 8; }
// elements per thread of the axis-2 column transform: 8, 16 or 32 (32 in FP32
// only; tuned > 0 selects, 0 the default 8); the 32-element kernel caps its
// registers for two CTAs of 256 threads per SM, as in 2D
constexpr bool col3_alt(int N) { return N >= 512 && N <= 1024; }
int col3_elems(int N, int tuned) {
    if (!col3_alt(N)) return ct3_elems(N);
    if (tuned == 16 || (tuned == 32 && sizeof(Real) == 4)) return tuned;
    return 8;
}
template <int N, int E>
constexpr auto col3_kernel() { return col_conv_t_kernel<Real, N, E, (N / E > 256 ? N / E : 256), E == 32 ? 2 : 1>; }
// elements per thread of the axis-1 (plane) transforms: 8 or 16 for FP32
// lines of 512 and 1024 (tuned row elements select)
int plane3_elems(int N, int tuned) {
    return (sizeof(Real) == 4 && col3_alt(N) && tuned == 16) ? 16 : ct3_elems(N);
}
int rows_per_cta(int nthr) { return std::max(1, std::min(4, 512 / nthr)); }
int groups_per_cta(int nthr) { return std::max(1, std::min(4, 256 / nthr)); }
size_t row_smem3(int N, int lpc) {
    return sizeof(C) * std::max<size_t>((size_t)spad_len(N) * lpc, (size_t)tile_ld(N + 1, lpc) * lpc);
}
size_t mid_smem3(int N, int G) { return sizeof(C) * std::max<size_t>((size_t)spad_len(N) * G, (size_t)tile_ld(N, G) * G); }

template <int P>
void set_attrs3(int limit) {
    constexpr int NR = P / 2, NC = P, ER = ct3_elems(NR), EC = ct3_elems(NC);
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_fwd_t_kernel<Real, 4, NR, ER>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_inv_t_kernel<Real, NR, ER>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(plane_fwd_t_kernel<Real, NC, EC>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(plane_inv_t_kernel<Real, NC, EC>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(col3_kernel<NC, EC>(), cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    if constexpr (col3_alt(NC)) {
        GOFD_CUDA_TRY(cudaFuncSetAttribute(col3_kernel<NC, 16>(), cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
        if constexpr (sizeof(Real) == 4) {
            GOFD_CUDA_TRY(cudaFuncSetAttribute(col3_kernel<NC, 32>(), cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
            GOFD_CUDA_TRY(cudaFuncSetAttribute(plane_fwd_t_kernel<Real, NC, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
            GOFD_CUDA_TRY(cudaFuncSetAttribute(plane_inv_t_kernel<Real, NC, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
        }
    }
}

template <int P, int ECC, int EC>
void run3_e(gofd_problem* p, const S* x, const S* vgrid, S* wgrid, cudaStream_t st) {
    constexpr int NR = P / 2, NC = P, ER = ct3_elems(NR);
    constexpr int tr = NR / ER, tc = NC / EC, tcc = NC / ECC;
    const int lpc = rows_per_cta(tr), G = groups_per_cta(tc), GC = groups_per_cta(tcc);
    const int n = p->n[0], H = P / 2 + 1, nlines = (int)p->nlines;
    const C* tw = twiddles3(p);
    const S* lamT = reinterpret_cast<const S*>(sizeof(Real) == 4 ? p->lamT32.ptr : p->lamT64.ptr);
    const S* w = reinterpret_cast<const S*>(sizeof(Real) == 4 ? p->ell_w32.ptr : p->ell_w64.ptr);
    C* Sp = p->specT.as<C>();
    C* M = p->specM.as<C>();
    const int64_t ld = p->ldT;
    const unsigned rblocks = (unsigned)((nlines + lpc - 1) / lpc);
    launch_pdl(row_fwd_t_kernel<Real, 4, NR, ER>, dim3(rblocks), dim3(lpc * tr), row_smem3(NR, lpc), st, x,
               p->ell_iidx.as<int32_t>(), w, p->nloc, p->line_run_ptr.as<int32_t>(), p->run_k0.as<int32_t>(),
               p->run_len.as<int32_t>(), p->run_e0.as<int32_t>(), vgrid, nlines, n, tw, Sp, (int)ld, lpc,
               (int64_t)0, (int64_t)0, GroupArg{});
    mark_stage(st, "gather_row_fft");
    const int ngroups = (n + G - 1) / G;
    // planes k_x0 in chunks of p->midK so that the chunk's middle buffer
    // stays in L2 from the axis-1 FFT through the inverse
    for (int k0 = 0; k0 < H; k0 += p->midK) {
        const int kc = std::min(p->midK, H - k0);
        launch_pdl(plane_fwd_t_kernel<Real, NC, EC>, dim3((unsigned)(kc * ngroups)), dim3(G * tc), mid_smem3(NC, G),
                   st, (const C*)Sp, ld, M, n, ngroups, k0, tw);
        launch_pdl(col3_kernel<NC, ECC>(), dim3((unsigned)(((int64_t)kc * P + GC - 1) / GC)),
                   dim3(GC * tcc), mid_smem3(NC, GC), st, M, n, n, (int)((int64_t)kc * P), H, tw, lamT, (int64_t)0,
                   P, (int64_t)k0 * P, GroupArg{});
        launch_pdl(plane_inv_t_kernel<Real, NC, EC>, dim3((unsigned)(kc * ngroups)), dim3(G * tc), mid_smem3(NC, G),
                   st, (const C*)M, n, ngroups, k0, Sp, ld, tw);
    }
    mark_stage(st, "axis12_conv");
    launch_pdl(row_inv_t_kernel<Real, NR, ER>, dim3(rblocks), dim3(lpc * tr), row_smem3(NR, lpc), st, (const C*)Sp,
               (int)ld, nlines, n, tw, wgrid, lpc, (int64_t)0, (int64_t)0, GroupArg{});
    mark_stage(st, "row_ifft");
}

template <int P, int ECC>
void run3_p(gofd_problem* p, const S* x, const S* vgrid, S* wgrid, cudaStream_t st) {
    if constexpr (sizeof(Real) == 4 && col3_alt(P))
        if (plane3_elems(P, p->tune_rowe) == 16) return run3_e<P, ECC, 16>(p, x, vgrid, wgrid, st);
    run3_e<P, ECC, ct3_elems(P)>(p, x, vgrid, wgrid, st);
}

template <int P>
void run3(gofd_problem* p, const S* x, const S* vgrid, S* wgrid, cudaStream_t st) {
    if constexpr (col3_alt(P)) {
        const int e = col3_elems(P, p->tune_cole);
        if constexpr (sizeof(Real) == 4)
            if (e == 32) return run3_p<P, 32>(p, x, vgrid, wgrid, st);
        if (e == 16) return run3_p<P, 16>(p, x, vgrid, wgrid, st);
    }
    run3_p<P, ct3_elems(P)>(p, x, vgrid, wgrid, st);
}

}  // namespace

void AFD3D_FN(gofd_problem* p, const S* x, const S* vgrid, S* wgrid, cudaStream_t st) {
    switch (p->P) {
        case 32: run3<32>(p, x, vgrid, wgrid, st); break;
        case 64: run3<64>(p, x, vgrid, wgrid, st); break;
        case 128: run3<128>(p, x, vgrid, wgrid, st); break;
        case 256: run3<256>(p, x, vgrid, wgrid, st); break;
        case 512: run3<512>(p, x, vgrid, wgrid, st); break;
        case 1024: run3<1024>(p, x, vgrid, wgrid, st); break;
        default: fail(GOFD_E_GRID, "3D circulant length beyond 1024 (n > 513) is not supported");
    }
}

void AFD3D_ATTR_FN(int limit, int P, size_t* need) {
    switch (P) {
#define ATTR(PP) case PP: set_attrs3<PP>(limit); break;
        ATTR(32) ATTR(64) ATTR(128) ATTR(256) ATTR(512) ATTR(1024)
#undef ATTR
        default: fail(GOFD_E_GRID, "3D circulant length beyond 1024 (n > 513) is not supported");
    }
    const int tr = P / 2 / ct3_elems(P / 2);
    size_t nd = row_smem3(P / 2, rows_per_cta(tr));
    for (int e : {8, 16, 32})   // every middle-stage shape the tuner may pick
        if (P / e >= 1) nd = std::max(nd, mid_smem3(P, groups_per_cta(P / e)));
    *need = nd;
}

}  // namespace gofd
