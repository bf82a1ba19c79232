// 3D stiffness product: kernels of the middle (axis 1, axis 2) stage.
//
// The axis-0 stages are the 2D row kernels over the n^2 grid lines: the
// half spectrum is stored spec_T[k_x0][line] with line = k_1 + n k_2, so each
// k_x0 plane is an n x n complex array (k_1 fastest).  Per plane the middle
// stage is a 2D zero-padded FFT convolution:
//
//   plane_fwd_t   lines along k_1 (contiguous), forward FFT of length P over
//                 the n nonzero entries, output stored transposed through a
//                 shared-memory tile: M[k_x0 - k0][k_x1'][k_2] (k_2 fastest)
//
// The planes are taken in chunks [k0, k0 + K) that bound the size of M.
//   col_conv_t    (shared with 2D) lines along k_2, contiguous in M: forward
//                 FFT, times the symbol row (k_x0, k_x1'), inverse FFT, n kept
//   plane_inv_t   transposed tile load of G lines along k_x1', inverse FFT of
//                 length P, the n kept entries written back to spec_T
//
// G lines per CTA (at most 4: one named barrier id per line; at most
// max(N/E, 256) threads per CTA).
#pragma once

#include "apply2d.cuh"

namespace gofd {

template <class Real, int N, int E>
__global__ void __launch_bounds__(N / E > 256 ? N / E : 256) plane_fwd_t_kernel(
    const typename Cplx<Real>::T* __restrict__ specT, int64_t ld, typename Cplx<Real>::T* __restrict__ M, int n,
    int ngroups, int kx0, const typename Cplx<Real>::T* __restrict__ tw) {
    pdl_enter();
    using C = typename Cplx<Real>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    constexpr int nthr = N / E;
    const int G = blockDim.x / nthr, msk = G - 1, gsh = __ffs(G) - 1;   // G is a power of two
    const int kl = blockIdx.x / ngroups, kx = kx0 + kl, k20 = (blockIdx.x % ngroups) * G;
    const int g = threadIdx.x / nthr, t = threadIdx.x % nthr;
    const int k2 = k20 + g;
    const bool active = k2 < n;
    const C* line = specT + (int64_t)kx * ld + (int64_t)(active ? k2 : 0) * n;
    C v[E];
    each_elem_r<ct_radix_o(N, E, false, 0), E>(t, nthr, N, [&](int i, int pos) {
        v[i] = (active && pos < n) ? line[pos] : cmk<C>(0.0, 0.0);
    });
    fft_ct<false, N, E, false>(v, sm + g * spad_len(N), t, g, tw, 1);
    __syncthreads();   // the tile reuses the line buffers
    const int LS = tile_ld(N, G);   // tile: (pos, line l) at l*LS + pos
    each_elem_r<ct_last<N, E, false>(), E>(t, nthr, N, [&](int i, int pos) { sm[g * LS + pos] = v[i]; });
    __syncthreads();
    C* out = M + (int64_t)kl * N * n;   // plane kl of the chunk
    for (int i = threadIdx.x; i < N * G; i += blockDim.x) {
        const int pos = i >> gsh, l = i & msk;
        if (k20 + l < n) out[(int64_t)pos * n + k20 + l] = sm[l * LS + pos];
    }
}

template <class Real, int N, int E>
__global__ void __launch_bounds__(N / E > 256 ? N / E : 256) plane_inv_t_kernel(
    const typename Cplx<Real>::T* __restrict__ M, int n, int ngroups, int kx0,
    typename Cplx<Real>::T* __restrict__ specT, int64_t ld, const typename Cplx<Real>::T* __restrict__ tw) {
    pdl_enter();
    using C = typename Cplx<Real>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    constexpr int nthr = N / E;
    const int G = blockDim.x / nthr, msk = G - 1, gsh = __ffs(G) - 1;   // G is a power of two
    const int kl = blockIdx.x / ngroups, kx = kx0 + kl, k20 = (blockIdx.x % ngroups) * G;
    const C* in = M + (int64_t)kl * N * n;
    const int LS = tile_ld(N, G);   // tile: (pos, line l) at l*LS + pos
    for (int i = threadIdx.x; i < N * G; i += blockDim.x) {
        const int pos = i >> gsh, l = i & msk;
        sm[l * LS + pos] = (k20 + l < n) ? in[(int64_t)pos * n + k20 + l] : cmk<C>(0.0, 0.0);
    }
    __syncthreads();
    const int g = threadIdx.x / nthr, t = threadIdx.x % nthr;
    const int k2 = k20 + g;
    C v[E];
    each_elem_r<ct_radix_o(N, E, false, 0), E>(t, nthr, N, [&](int i, int pos) { v[i] = sm[g * LS + pos]; });
    __syncthreads();   // the line buffers reuse the tile
    fft_ct<true, N, E, false>(v, sm + g * spad_len(N), t, g, tw, 1);
    if (k2 >= n) return;
    C* line = specT + (int64_t)kx * ld + (int64_t)k2 * n;
    each_elem_r<ct_last<N, E, false>(), E>(t, nthr, N, [&](int i, int pos) {
        if (pos < n) line[pos] = v[i];
    });
}

}  // namespace gofd
