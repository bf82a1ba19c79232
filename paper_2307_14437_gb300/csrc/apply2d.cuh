// 2D stiffness product with the half spectrum stored transposed (kernels).
//
//   row_fwd_t    gather v = I x straight into the registers of the first FFT
//                pass of each grid line (no padded grid vector in memory), real
//                FFT of the line, half spectrum written transposed through a
//                shared-memory tile: spec_T[k_x0][line]
//   col_conv_t   one spectrum column per thread group, contiguous in memory:
//                loads go straight into registers, forward FFT over the n
//                nonzero rows, the real even symbol multiplied in registers,
//                inverse FFT starting from the same registers, n rows stored
//   row_inv_t    transposed tile load, inverse real FFT of each line, the n
//                kept samples written to the grid vector
//
// Line lengths are compile-time constants (powers of two), so every pass has
// a constant radix and stride.  Passes exchange data through padded shared
// memory with per-line named barriers, so lines of one CTA do not wait for
// each other.
#pragma once

#include <algorithm>

#include "gofd_internal.cuh"
#include "fft_common.cuh"

namespace gofd {

// Per-group barrier.  The ids are spelled out so that the compiler reserves
// only ids 1..4 (dynamic ids make it reserve all 16 and halve residency).
__device__ __forceinline__ void group_sync(int g, int nthr) {
    if (nthr < 32) {
        __syncthreads();
        return;
    }
    if (nthr == 32) {   // one warp per line
        __syncwarp();
        return;
    }
    switch (g) {
        case 0: asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory"); break;
        case 1: asm volatile("bar.sync 2, %0;" ::"r"(nthr) : "memory"); break;
        case 2: asm volatile("bar.sync 3, %0;" ::"r"(nthr) : "memory"); break;
        default: asm volatile("bar.sync 4, %0;" ::"r"(nthr) : "memory"); break;
    }
}

template <int R, bool INV, int E, class C>
__device__ __forceinline__ void reg_pass(C (&v)[E], int t, int nthr, int N, int Ns, const C* __restrict__ tw,
                                         int twstride) {
    constexpr int Q = E / R;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = t + q * nthr;
        const int k = b % Ns;
        if (k != 0) {
            const int step = (N / (Ns * R)) * twstride;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = cld(&tw[k * r * step]);
                if (INV) w.y = -w.y;
                v[q * R + r] = cmul(v[q * R + r], w);
            }
        }
        dft_reg<R, INV>(v + q * R);
    }
}

template <int R, int E, class C>
__device__ __forceinline__ void reg_store(C* buf, const C (&v)[E], int t, int nthr, int Ns) {
    constexpr int Q = E / R;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = t + q * nthr;
        const int base = (b / Ns) * Ns * R + b % Ns;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[spad(base + r * Ns)] = v[q * R + r];
    }
}

template <int R, int E, class C>
__device__ __forceinline__ void reg_load(const C* buf, C (&v)[E], int t, int nthr, int N) {
    constexpr int Q = E / R;
    const int S = N / R;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = t + q * nthr;
#pragma unroll
        for (int r = 0; r < R; ++r) v[q * R + r] = buf[spad(b + r * S)];
    }
}

// Visit the thread's elements of a pass of radix R: f(i, pos) with i the
// register index (a compile-time constant after unrolling) and pos = b + r N/R
// the line position.  Dispatching on R keeps v[] in registers.
template <int R, int E, class F>
__device__ __forceinline__ void each_elem_r(int t, int nthr, int N, F&& f) {
    constexpr int Q = E / R;
    const int S = N / R;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = t + q * nthr;
#pragma unroll
        for (int r = 0; r < R; ++r) f(q * R + r, b + r * S);
    }
}
// ---------------------------------------------------------------------------
// compile-time pass plans: radix 16 passes first, then the remainder
// ---------------------------------------------------------------------------
// E = elements per thread = the largest radix; passes of radix E first, then
// the remainder.
__host__ __device__ constexpr int ct_full(int N, int E) { int f = 0; while (N >= E) { N /= E; ++f; } return f; }
__host__ __device__ constexpr int ct_rem(int N, int E) { while (N >= E) N /= E; return N; }
__host__ __device__ constexpr int ct_npass(int N, int E) { return ct_full(N, E) + (ct_rem(N, E) > 1 ? 1 : 0); }
__host__ __device__ constexpr int ct_radix(int N, int E, int i) { return i < ct_full(N, E) ? E : ct_rem(N, E); }
// REV: the same radices in reverse order (the inverse column transform starts
// with the forward transform's last radix so the data stays in registers)
__host__ __device__ constexpr int ct_radix_o(int N, int E, bool rev, int i) {
    return rev ? ct_radix(N, E, ct_npass(N, E) - 1 - i) : ct_radix(N, E, i);
}
template <int N, int E, bool REV>
__host__ __device__ constexpr int ct_last() { return ct_radix_o(N, E, REV, ct_npass(N, E) - 1); }

template <bool INV, int N, int E, bool REV, int PS = 0, int NS = 1, class C>
__device__ __forceinline__ void fft_ct(C (&v)[E], C* buf, int t, int g, const C* __restrict__ tw, int tws) {
    if constexpr (PS < ct_npass(N, E)) {
        constexpr int R = ct_radix_o(N, E, REV, PS);
        constexpr int NTHR = N / E;
        if constexpr (PS > 0) {
            constexpr int RP = ct_radix_o(N, E, REV, PS - 1);
            reg_store<RP>(buf, v, t, NTHR, NS / RP);
            group_sync(g, NTHR);
            reg_load<R>(buf, v, t, NTHR, N);
            group_sync(g, NTHR);
        }
        reg_pass<R, INV>(v, t, NTHR, N, NS, tw, tws);
        fft_ct<INV, N, E, REV, PS + 1, NS * R>(v, buf, t, g, tw, tws);
    }
}

// ---------------------------------------------------------------------------
// gather of one grid sample: sum over the owner simplex's slots (ELL row e)
// ---------------------------------------------------------------------------
template <class Real, int DP1>
__device__ __forceinline__ Real ell_value(const typename Sto<Real>::T* __restrict__ x, const int32_t* __restrict__ iidx,
                                          const typename Sto<Real>::T* __restrict__ w, int64_t nloc, int64_t e) {
    typename Sto<Real>::T acc = 0;   // in the storage precision (FP64 for double-float)
#pragma unroll
    for (int s = 0; s < DP1; ++s) acc += __ldg(&w[s * nloc + e]) * __ldg(&x[__ldg(&iidx[s * nloc + e])]);
    return from_sto<Real>(acc);
}

struct Runs {
    int n;          // runs on this line
    int k0[2], len[2], e0[2];
    int rb;         // first run index (for lines with more than two runs)
};

template <class Real, int DP1>
__device__ __forceinline__ Real sample(int k, const Runs& rs, const int32_t* __restrict__ run_k0,
                                       const int32_t* __restrict__ run_len, const int32_t* __restrict__ run_e0,
                                       const typename Sto<Real>::T* __restrict__ x, const int32_t* __restrict__ iidx,
                                       const typename Sto<Real>::T* __restrict__ w, int64_t nloc) {
    if (rs.n <= 2) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (r < rs.n && k >= rs.k0[r] && k < rs.k0[r] + rs.len[r])
                return ell_value<Real, DP1>(x, iidx, w, nloc, rs.e0[r] + (k - rs.k0[r]));
        return real_zero<Real>();
    }
    for (int r = rs.rb; r < rs.rb + rs.n; ++r) {
        const int a = __ldg(&run_k0[r]);
        if (k >= a && k < a + __ldg(&run_len[r])) return ell_value<Real, DP1>(x, iidx, w, nloc, __ldg(&run_e0[r]) + (k - a));
    }
    return real_zero<Real>();
}

// ---------------------------------------------------------------------------
// kernel 1: gather + real FFT per grid line, transposed half spectrum out
// ---------------------------------------------------------------------------
// MAXT / MINB: launch bounds (threads per CTA, CTAs per SM) the register
// allocation is compiled for
template <class Real, int DP1, int N, int E, int MAXT = 512, int MINB = 1>
__global__ void __launch_bounds__(MAXT, MINB) row_fwd_t_kernel(
    const typename Sto<Real>::T* __restrict__ x, const int32_t* __restrict__ iidx,
    const typename Sto<Real>::T* __restrict__ w, int64_t nloc, const int32_t* __restrict__ run_ptr,
    const int32_t* __restrict__ run_k0, const int32_t* __restrict__ run_len, const int32_t* __restrict__ run_e0,
    const typename Sto<Real>::T* __restrict__ vgrid, int nlines, int n,
    const typename Cplx<Real>::T* __restrict__ tw, typename Cplx<Real>::T* __restrict__ specT, int ld, int lpc,
    int64_t xstride, int64_t sstride, GroupArg ga) {
    pdl_trigger();
    if (ga.iv) {   // a group: this column's instance
        const InstView& I = ga.iv[blockIdx.y / ga.nbper];
        iidx = I.ell_iidx;
        w = sizeof(Real) == 4 ? reinterpret_cast<const typename Sto<Real>::T*>(I.ell_w32)
                              : reinterpret_cast<const typename Sto<Real>::T*>(I.ell_w64);
        nloc = I.nloc;
        run_ptr = I.run_ptr;
        run_k0 = I.run_k0;
        run_len = I.run_len;
        run_e0 = I.run_e0;
    }
    using C = typename Cplx<Real>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    constexpr int nthr = N / E;
    // batch of right-hand sides along gridDim.y (strides 0 for one vector)
    x += blockIdx.y * xstride;
    if (vgrid) vgrid += blockIdx.y * xstride;
    specT += blockIdx.y * sstride;
    const int g = threadIdx.x / nthr, t = threadIdx.x % nthr;
    const int line = blockIdx.x * lpc + g;
    const bool active = line < nlines;
    C* buf = sm + g * spad_len(N);

    Runs rs;
    rs.n = 0;
    rs.rb = 0;
    if (active && !vgrid) {   // set-up tables: read before the predecessor completes
        rs.rb = __ldg(&run_ptr[line]);
        rs.n = __ldg(&run_ptr[line + 1]) - rs.rb;
        for (int r = 0; r < 2; ++r)
            if (r < rs.n) {
                rs.k0[r] = __ldg(&run_k0[rs.rb + r]);
                rs.len[r] = __ldg(&run_len[rs.rb + r]);
                rs.e0[r] = __ldg(&run_e0[rs.rb + r]);
            }
    }
    pdl_wait();
    if (column_skipped(ga)) return;
    // pass-0 inputs z[m] = (v[2m], v[2m+1]) gathered straight into registers
    C v[E];
    if (vgrid || rs.n > 2) {
        each_elem_r<ct_radix_o(N, E, false, 0), E>(t, nthr, N, [&](int i, int m) {
            const int k = 2 * m;
            Real a0 = real_zero<Real>(), a1 = real_zero<Real>();
            if (active && k < n) {
                if (vgrid) {
                    a0 = from_sto<Real>(vgrid[(int64_t)line * n + k]);
                    if (k + 1 < n) a1 = from_sto<Real>(vgrid[(int64_t)line * n + k + 1]);
                } else {
                    a0 = sample<Real, DP1>(k, rs, run_k0, run_len, run_e0, x, iidx, w, nloc);
                    if (k + 1 < n) a1 = sample<Real, DP1>(k + 1, rs, run_k0, run_len, run_e0, x, iidx, w, nloc);
                }
            }
            v[i].x = a0;
            v[i].y = a1;
        });
    } else if (rs.n > 0) {
        // at most two runs on this line: ELL rows by selects, every load
        // issued without branches so that many are in flight at once
        each_elem_r<ct_radix_o(N, E, false, 0), E>(t, nthr, N, [&](int i, int m) {
            const int k = 2 * m;
            if (k >= n) {
                v[i].x = real_zero<Real>();
                v[i].y = real_zero<Real>();
                return;
            }
            int ea = -1, eb = -1;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (r < rs.n) {
                    const int lo = rs.k0[r], hi = rs.k0[r] + rs.len[r];
                    ea = (k >= lo && k < hi) ? rs.e0[r] + (k - lo) : ea;
                    eb = (k + 1 >= lo && k + 1 < hi) ? rs.e0[r] + (k + 1 - lo) : eb;
                }
            }
            const int64_t ca = ea >= 0 ? ea : 0, cb = eb >= 0 ? eb : 0;
            typename Sto<Real>::T a0 = 0, a1 = 0;   // the gather in the storage precision
#pragma unroll
            for (int s = 0; s < DP1; ++s) {
                a0 += __ldg(&w[s * nloc + ca]) * __ldg(&x[__ldg(&iidx[s * nloc + ca])]);
                a1 += __ldg(&w[s * nloc + cb]) * __ldg(&x[__ldg(&iidx[s * nloc + cb])]);
            }
            v[i].x = from_sto<Real>(ea >= 0 ? a0 : 0);
            v[i].y = from_sto<Real>(eb >= 0 ? a1 : 0);
        });
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = cmk<C>(0.0, 0.0);
    }
    fft_ct<false, N, E, false>(v, buf, t, g, tw, 2);
    {
        constexpr int RL = ct_last<N, E, false>();
        reg_store<RL>(buf, v, t, nthr, N / RL);
    }
    __syncthreads();
    // X[k] = (Z_k + conj Z_{N-k})/2 - i/2 W_P^k (Z_k - conj Z_{N-k}),  k = 0..N
    constexpr int JMAX = E + 1;
    C X[JMAX];
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        const int k = t + j * nthr;
        if (k <= N) {
            const C zk = buf[spad(k & (N - 1))];
            const C zc = cconj(buf[spad((N - k) & (N - 1))]);
            const C e = cadd(zk, zc), o = csub(zk, zc);
            C mo;
            mo.x = o.y;
            mo.y = -o.x;
            C r = cadd(e, cmul(cld(&tw[k]), mo));
            r.x *= real_half<Real>();
            r.y *= real_half<Real>();
            X[j] = r;
        }
    }
    __syncthreads();
    // transposed tile: element (k, line g) at g*LS + k, LS = tile_ld(N+1, lpc)
    const int msk = lpc - 1, lsh = __ffs(lpc) - 1;   // lpc is a power of two
    const int LS = tile_ld(N + 1, lpc);
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        const int k = t + j * nthr;
        if (k <= N) sm[g * LS + k] = X[j];
    }
    __syncthreads();
    const int total = (N + 1) * lpc;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int k = i >> lsh, l = i & msk;
        const int ln = blockIdx.x * lpc + l;
        if (ln < nlines) specT[(int64_t)k * ld + ln] = sm[l * LS + k];
    }
}

// ---------------------------------------------------------------------------
// kernel 2: per spectrum column: FFT (n nonzero rows), symbol, inverse FFT
// (ncols columns of stride ld; H = P/2+1 is the symbol's extent per axis)
// ---------------------------------------------------------------------------
template <class Real, int N, int E, int MAXT = (N / E > 256 ? N / E : 256), int MINB = 1>
__global__ void __launch_bounds__(MAXT, MINB) col_conv_t_kernel(typename Cplx<Real>::T* __restrict__ specT, int ld, int n,
                                                       int ncols, int H, const typename Cplx<Real>::T* __restrict__ tw,
                                                       const typename Sto<Real>::T* __restrict__ lamT, int64_t sstride, int pm,
                                                       int64_t col0, GroupArg ga) {
    pdl_enter();
    if (column_skipped(ga)) return;
    if (ga.iv) {
        const InstView& I = ga.iv[blockIdx.y / ga.nbper];
        lamT = sizeof(Real) == 4 ? reinterpret_cast<const typename Sto<Real>::T*>(I.lamT32)
                                 : reinterpret_cast<const typename Sto<Real>::T*>(I.lamT64);
    } else if (sizeof(Real) == 4 ? ga.lam32 != nullptr : ga.lam64 != nullptr) {
        lamT = sizeof(Real) == 4 ? reinterpret_cast<const typename Sto<Real>::T*>(ga.lam32)
                                 : reinterpret_cast<const typename Sto<Real>::T*>(ga.lam64);
    }
    using C = typename Cplx<Real>::T;
    specT += blockIdx.y * sstride;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    constexpr int nthr = N / E;
    const int G = blockDim.x / nthr;
    const int g = threadIdx.x / nthr, t = threadIdx.x % nthr;
    const int col = blockIdx.x * G + g;
    const bool active = col < ncols;
    C* buf = sm + g * spad_len(N);
    C* column = specT + (int64_t)(active ? col : 0) * ld;
    C v[E];
    each_elem_r<ct_radix_o(N, E, false, 0), E>(t, nthr, N, [&](int i, int row) {
        v[i] = (active && row < n) ? column[row] : cmk<C>(0.0, 0.0);
    });
    fft_ct<false, N, E, false>(v, buf, t, g, tw, 1);
    {
        // multiply by the (pre-scaled) symbol: row k_x1 folded to [0, N/2].
        // 2D (pm = 0): column = k_x0.  3D (pm = P): column col0 + col =
        // k_x0 * P + k_x1' with k_x1' folded too; the symbol row is
        // (k_x0, fold(k_x1')).
        const int64_t cc = (active ? col : 0) + col0;
        int64_t lrow = cc;
        if (pm) {
            const int64_t a = cc / pm;
            const int b = (int)(cc % pm);
            lrow = a * H + (b <= pm / 2 ? b : pm - b);
        }
        const typename Sto<Real>::T* lc = lamT + lrow * H;
        each_elem_r<ct_last<N, E, false>(), E>(t, nthr, N, [&](int i, int row) {
            const int fr = row <= N / 2 ? row : N - row;
            const Real l = from_sto<Real>(__ldg(&lc[fr]));
            v[i].x *= l;
            v[i].y *= l;
        });
    }
    fft_ct<true, N, E, true>(v, buf, t, g, tw, 1);
    each_elem_r<ct_last<N, E, true>(), E>(t, nthr, N, [&](int i, int row) {
        if (active && row < n) column[row] = v[i];
    });
}

// ---------------------------------------------------------------------------
// kernel 3: transposed tile in, inverse real FFT per line, n samples out
// ---------------------------------------------------------------------------
template <class Real, int N, int E, int MAXT = 512, int MINB = 1>
__global__ void __launch_bounds__(MAXT, MINB) row_inv_t_kernel(const typename Cplx<Real>::T* __restrict__ specT, int ld,
                                                      int nlines, int n, const typename Cplx<Real>::T* __restrict__ tw,
                                                      typename Sto<Real>::T* __restrict__ wgrid, int lpc, int64_t sstride,
                                                      int64_t wstride, GroupArg ga) {
    pdl_enter();
    if (column_skipped(ga)) return;
    using C = typename Cplx<Real>::T;
    specT += blockIdx.y * sstride;
    wgrid += blockIdx.y * wstride;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    constexpr int nthr = N / E;
    const int msk = lpc - 1, lsh = __ffs(lpc) - 1;   // lpc is a power of two
    const int LS = tile_ld(N + 1, lpc);                // tile: (k, line l) at l*LS + k
    const int total = (N + 1) * lpc;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int k = i >> lsh, l = i & msk;
        const int ln = blockIdx.x * lpc + l;
        sm[l * LS + k] = (ln < nlines) ? specT[(int64_t)k * ld + ln] : cmk<C>(0.0, 0.0);
    }
    __syncthreads();
    const int g = threadIdx.x / nthr, t = threadIdx.x % nthr;
    const int line = blockIdx.x * lpc + g;
    const bool active = line < nlines;
    C v[E];
    // Z'_k = (X_k + conj X_{N-k}) + i W_P^{-k} (X_k - conj X_{N-k})
    each_elem_r<ct_radix_o(N, E, false, 0), E>(t, nthr, N, [&](int i, int k) {
        const int kc = N - k;
        const C xk = sm[g * LS + k];
        const C xc = cconj(sm[g * LS + kc]);
        const C e = cadd(xk, xc);
        const C o = cmulc(csub(xk, xc), cld(&tw[k]));
        C z;
        z.x = e.x - o.y;
        z.y = e.y + o.x;
        v[i] = z;
    });
    __syncthreads();
    C* buf = sm + g * spad_len(N);
    fft_ct<true, N, E, false>(v, buf, t, g, tw, 2);
    if (!active) return;
    typename Sto<Real>::T* wl = wgrid + (int64_t)line * n;
    each_elem_r<ct_last<N, E, false>(), E>(t, nthr, N, [&](int i, int m) {
        const int k = 2 * m;
        if (k < n) wl[k] = to_sto<Real>(v[i].x);
        if (k + 1 < n) wl[k + 1] = to_sto<Real>(v[i].y);
    });
}

}  // namespace gofd
