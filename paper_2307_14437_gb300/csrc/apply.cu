// The stiffness product y = I^T A_FD I x (GoFD-2) on interior-compacted vectors.
//
//   gather   v = I x on the grid, fused into the first FFT pass (ELL runs per line)
//   A_FD v   zero-padded circulant convolution (Section 2.2, (AU-1)):
//            real FFT along axis 0 (only the n nonzero lines), complex FFTs along
//            the other axes (only n nonzero inputs; outputs kept on the needed
//            range), multiplication by the real even symbol, inverse transforms
//            that keep the n^d corner
//   scatter  y = I^T w through the interior-vertex CSR, fixed summation order
//
// The FFTs are Stockham passes of radix 16 (and one of radix 2/4/8) computed in
// registers, with the exchange between passes through padded shared memory.
// Every transform is unnormalised; the symbol carries the 1/P^d factor.
#include <algorithm>
#include <mutex>
#include <vector>

#include "gofd_internal.cuh"
#include "fft_common.cuh"

namespace gofd {

LinePlan make_line_plan(int N) {
    LinePlan p;
    p.N = N;
    p.nthr = N / FFT_E;
    int rem = N;
    while (rem >= 16) {
        p.radix[p.npass++] = 16;
        rem /= 16;
    }
    if (rem > 1) p.radix[p.npass++] = rem;
    return p;
}

// ---------------------------------------------------------------------------
// kernel 1: gather + real FFT along axis 0
// ---------------------------------------------------------------------------
template <class Real, int DP1>
__global__ void __launch_bounds__(512) row_forward_kernel(const Real* __restrict__ x, const int32_t* __restrict__ iidx,
                                   const Real* __restrict__ w, int64_t nloc,
                                   const int32_t* __restrict__ run_ptr, const int32_t* __restrict__ run_k0,
                                   const int32_t* __restrict__ run_len, const int32_t* __restrict__ run_e0,
                                   int64_t nlines, LinePlan plan, const typename Cplx<Real>::T* __restrict__ tw,
                                   typename Cplx<Real>::T* __restrict__ spec, int pitch, int gather_from_grid,
                                   const Real* __restrict__ vgrid, int n0) {
    using C = typename Cplx<Real>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int N = plan.N;  // P/2
    const int nthr = plan.nthr;
    const int g = threadIdx.x / nthr, t = threadIdx.x % nthr;
    const int64_t line = (int64_t)blockIdx.x * (blockDim.x / nthr) + g;
    const bool active = line < nlines;
    C* buf = sm + g * spad_len(N);
    for (int i = t; i < spad_len(N); i += nthr) buf[i] = cmk<C>(0.0, 0.0);
    __syncthreads();
    if (active) {
        Real* re = reinterpret_cast<Real*>(buf);
        if (gather_from_grid) {
            for (int k = t; k < n0; k += nthr) re[2 * spad(k >> 1) + (k & 1)] = vgrid[line * n0 + k];
        } else {
            const int r1 = run_ptr[line + 1];
            for (int r = run_ptr[line]; r < r1; ++r) {
                const int k0 = run_k0[r], len = run_len[r], e0 = run_e0[r];
                for (int q = t; q < len; q += nthr) {
                    const int64_t e = e0 + q;
                    Real acc = 0;
#pragma unroll
                    for (int s = 0; s < DP1; ++s) acc += w[s * nloc + e] * x[iidx[s * nloc + e]];
                    const int k = k0 + q;
                    re[2 * spad(k >> 1) + (k & 1)] = acc;
                }
            }
        }
    }
    __syncthreads();
    line_fft<false>(buf, plan, t, tw, 2);
    if (!active) return;
    // X[k] = (Z_k + conj Z_{N-k})/2 - i/2 W_P^k (Z_k - conj Z_{N-k}),  k = 0..N
    C* out = spec + line * pitch;
    for (int k = t; k <= N; k += nthr) {
        C zk = buf[spad(k & (N - 1))];
        C zc = cconj(buf[spad((N - k) & (N - 1))]);
        C e = cadd(zk, zc), o = csub(zk, zc);
        // -i * o
        C mo;
        mo.x = o.y;
        mo.y = -o.x;
        C wk = __ldg(&tw[k]);
        C r = cadd(e, cmul(wk, mo));
        r.x *= (Real)0.5;
        r.y *= (Real)0.5;
        out[k] = r;
    }
}

// ---------------------------------------------------------------------------
// kernel 2: complex FFTs along a strided axis for TC adjacent columns
//   MODE 0: forward, rows_in nonzero rows -> P rows out
//   MODE 1: forward, multiply by the symbol, inverse; rows_out rows kept
//   MODE 2: inverse, P rows in -> rows_out rows out
// ---------------------------------------------------------------------------
struct ColDesc {
    int64_t in_slab, in_row, out_slab, out_row;
    int rows_in, rows_out, ncols, TC;
    int64_t lam_slab, lam_row;  // symbol strides (MODE 1), folded indices
    int P;
};

// in and out may be the same array (in-place columns): every column is read
// into shared memory before any of it is stored, and neither pointer is
// declared __restrict__.
template <class Real, int MODE>
__global__ void __launch_bounds__(512) col_fft_kernel(const typename Cplx<Real>::T* in, typename Cplx<Real>::T* out,
                               ColDesc cd, LinePlan plan, const typename Cplx<Real>::T* __restrict__ tw,
                               const Real* __restrict__ lam) {
    using C = typename Cplx<Real>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int N = plan.N;  // P
    const int TC = cd.TC;
    const int g = threadIdx.x % TC, t = threadIdx.x / TC;
    const int c0 = blockIdx.x * TC;
    const int64_t slab = blockIdx.y;
    C* buf = sm + g * spad_len(N);
    const C* src = in + slab * cd.in_slab + c0;
    // load rows_in rows of TC columns (consecutive threads -> consecutive columns)
    for (int i = threadIdx.x; i < N * TC; i += blockDim.x) {
        const int row = i / TC, cc = i % TC;
        C v = cmk<C>(0.0, 0.0);
        if (row < cd.rows_in && c0 + cc < cd.ncols) v = src[row * cd.in_row + cc];
        sm[cc * spad_len(N) + spad(row)] = v;
    }
    __syncthreads();
    if (MODE == 2) {
        line_fft<true>(buf, plan, t, tw, 1);
    } else {
        line_fft<false>(buf, plan, t, tw, 1);
    }
    if (MODE == 1) {
        const int H = cd.P / 2;
        const int64_t sl = slab <= H ? slab : cd.P - slab;
        const Real* lp = lam + sl * cd.lam_slab + c0;
        for (int i = threadIdx.x; i < N * TC; i += blockDim.x) {
            const int row = i / TC, cc = i % TC;
            if (c0 + cc >= cd.ncols) continue;
            const int fr = row <= H ? row : N - row;
            const Real l = lp[fr * cd.lam_row + cc];
            C& v = sm[cc * spad_len(N) + spad(row)];
            v.x *= l;
            v.y *= l;
        }
        __syncthreads();
        line_fft<true>(buf, plan, t, tw, 1);
    }
    C* dst = out + slab * cd.out_slab + c0;
    const int rows = (MODE == 0) ? N : cd.rows_out;
    for (int i = threadIdx.x; i < rows * TC; i += blockDim.x) {
        const int row = i / TC, cc = i % TC;
        if (c0 + cc < cd.ncols) dst[row * cd.out_row + cc] = sm[cc * spad_len(N) + spad(row)];
    }
}

// 1D: multiply the half spectrum by the symbol
template <class Real>
__global__ void spec_scale_kernel(typename Cplx<Real>::T* __restrict__ spec, const Real* __restrict__ lam, int H) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < H; k += gridDim.x * blockDim.x) {
        spec[k].x *= lam[k];
        spec[k].y *= lam[k];
    }
}

// ---------------------------------------------------------------------------
// kernel 3: inverse real FFT along axis 0, keeps k0 < n0
// ---------------------------------------------------------------------------
template <class Real>
__global__ void __launch_bounds__(512) row_inverse_kernel(const typename Cplx<Real>::T* __restrict__ spec, int pitch, int64_t nlines,
                                   LinePlan plan, const typename Cplx<Real>::T* __restrict__ tw,
                                   Real* __restrict__ wgrid, int n0) {
    using C = typename Cplx<Real>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int N = plan.N;
    const int nthr = plan.nthr;
    const int g = threadIdx.x / nthr, t = threadIdx.x % nthr;
    const int64_t line = (int64_t)blockIdx.x * (blockDim.x / nthr) + g;
    const bool active = line < nlines;
    C* buf = sm + g * spad_len(N);
    if (active) {
        const C* X = spec + line * pitch;
        // Z'_k = (X_k + conj X_{N-k}) + i W_P^{-k} (X_k - conj X_{N-k}),  k < N
        for (int k = t; k < N; k += nthr) {
            C xk = X[k], xc = cconj(X[N - k]);
            C e = cadd(xk, xc);
            C o = cmulc(csub(xk, xc), __ldg(&tw[k]));
            C z;
            z.x = e.x - o.y;
            z.y = e.y + o.x;
            buf[spad(k)] = z;
        }
    }
    __syncthreads();
    line_fft<true>(buf, plan, t, tw, 2);
    if (!active) return;
    Real* wl = wgrid + line * n0;
    const Real* re = reinterpret_cast<const Real*>(buf);
    for (int k = t; k < n0; k += nthr) wl[k] = re[2 * spad(k >> 1) + (k & 1)];
}

// ---------------------------------------------------------------------------
// kernel 4: y = I^T w, TPR lanes per interior vertex, fixed order
// ---------------------------------------------------------------------------
// rows longer than SCATTER_LONG entries (patches of large elements on a fine
// grid) are left to scatter_long_kernel, one CTA per row
constexpr int SCATTER_LONG = 1024;

// Long rows are cut into chunks of SCATTER_CHUNK entries; one CTA sums a
// chunk (fixed-order tree), then one thread per long row adds its chunks in
// order, so the result does not depend on scheduling.
constexpr int SCATTER_CHUNK = 2048;

// Sum of one chunk of a long row by one CTA of 256 threads (fixed order:
// strided lane sums, then a shared-memory tree); every thread returns it.
template <class Real>
__device__ __forceinline__ Real chunk_sum(const int32_t* __restrict__ col, const Real* __restrict__ val,
                                          const Real* __restrict__ w, int32_t b, int32_t e, Real* part) {
    Real a0 = 0, a1 = 0;
    int a = b + threadIdx.x;
    for (; a + 256 < e; a += 512) {
        const int c0 = __ldg(&col[a]), c1 = __ldg(&col[a + 256]);
        a0 += __ldg(&val[a]) * __ldg(&w[c0]);
        a1 += __ldg(&val[a + 256]) * __ldg(&w[c1]);
    }
    for (; a < e; a += 256) a0 += __ldg(&val[a]) * __ldg(&w[__ldg(&col[a])]);
    part[threadIdx.x] = a0 + a1;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    return part[0];
}

// Long-row bookkeeping of the scatter (rows of I^T with more than
// SCATTER_LONG entries, cut into chunks of SCATTER_CHUNK entries).
struct LongRows {
    const int32_t* cbeg;    // [nchunks] first entry of each chunk
    const int32_t* cend;    // [nchunks] one past its last entry
    const int32_t* crow;    // [nchunks] long-row index of each chunk
    const int32_t* rows;    // [nrows] interior row of each long row
    const int32_t* cptr;    // [nrows+1] chunks of each long row
    int64_t nchunks, nrows;
};

// y_i = scale * sum_k val_k w[col_k] over row i of I^T, for nb right-hand sides
// (grid y).  Blocks [0, nshort) take the rows of at most SCATTER_LONG entries,
// TPR lanes per row; each further block takes one chunk of a long row, writes
// its partial sum, and the last chunk of a row to finish (counted with an
// atomic counter) adds the row's partials in chunk order.  Every sum has a
// fixed order, so results are bitwise reproducible.
template <class Real, int TPR>
__global__ void __launch_bounds__(256) scatter_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                                      const Real* __restrict__ val, const Real* __restrict__ w,
                                                      int64_t nint, Real* __restrict__ y, Real scale, int64_t ws,
                                                      int64_t ys, unsigned nshort, LongRows lr, Real* partial,
                                                      unsigned* counters, GroupArg ga) {
    pdl_trigger();
    w += blockIdx.y * ws;
    y += blockIdx.y * ys;
    if (blockIdx.x >= nshort) {
        pdl_wait();
        if (column_skipped(ga)) return;
        __shared__ Real part[256];
        __shared__ bool last;
        const int64_t c = blockIdx.x - nshort;
        Real* pp = partial + (int64_t)blockIdx.y * lr.nchunks;
        unsigned* cnt = counters + (int64_t)blockIdx.y * lr.nrows;
        const Real sum = chunk_sum<Real>(col, val, w, __ldg(&lr.cbeg[c]), __ldg(&lr.cend[c]), part);
        const int r = __ldg(&lr.crow[c]);
        const int c0 = __ldg(&lr.cptr[r]), c1 = __ldg(&lr.cptr[r + 1]);
        if (threadIdx.x == 0) {
            pp[c] = sum;
            __threadfence();
            last = atomicAdd(&cnt[r], 1u) == (unsigned)(c1 - c0 - 1);
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            Real acc = 0;
            for (int k = c0; k < c1; ++k) acc += ((volatile Real*)pp)[k];
            y[__ldg(&lr.rows[r])] = acc * scale;
            cnt[r] = 0;   // ready for the next product
        }
        return;
    }
    // Short rows: TPR lanes per row; lane l accumulates the entries
    // b + l + (4k + u) TPR of its row in partial sum u (u < 4), then the sums
    // are combined as (s0 + s1) + (s2 + s3) and across the lanes by shuffles.
    // The loop is uniform across each warp so that every lane reaches the
    // shuffles.  The first row group's bounds and first entries are set-up
    // data, loaded before waiting for the kernel that writes w.
    const int64_t nthreads = (int64_t)nshort * blockDim.x;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x % TPR;
    int64_t t0 = gid - (threadIdx.x & 31);
    int b, e, c4[4];
    bool mine;   // a row of at most SCATTER_LONG entries (written here)
    Real v4[4];
    auto bounds = [&](int64_t tt) {
        const int64_t i = (tt + (threadIdx.x & 31)) / TPR;
        b = e = 0;
        mine = false;
        if (i < nint) {
            b = __ldg(&ptr[i]);
            e = __ldg(&ptr[i + 1]);
            mine = e - b <= SCATTER_LONG;
            if (!mine) e = b;   // a long row: the chunk blocks take it
        }
    };
    auto first4 = [&]() {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int a = b + lane + u * TPR;
            c4[u] = a < e ? __ldg(&col[a]) : -1;
            v4[u] = a < e ? __ldg(&val[a]) : (Real)0;
        }
    };
    bounds(t0);
    first4();
    pdl_wait();
    if (column_skipped(ga)) return;
    for (; t0 < nint * TPR; t0 += nthreads) {
        if (t0 != gid - (threadIdx.x & 31)) {
            bounds(t0);
            first4();
        }
        Real acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = c4[u] >= 0 ? v4[u] * __ldg(&w[c4[u]]) : (Real)0;
        for (int a = b + lane + 4 * TPR; a < e; a += 4 * TPR) {
            int cc[4];
            Real vv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = a + u * TPR < e;
                cc[u] = ok ? __ldg(&col[a + u * TPR]) : -1;
                vv[u] = ok ? __ldg(&val[a + u * TPR]) : (Real)0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (cc[u] >= 0) acc[u] += vv[u] * __ldg(&w[cc[u]]);
        }
        Real sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, TPR);
        const int64_t i = (t0 + (threadIdx.x & 31)) / TPR;
        if (lane == 0 && mine) y[i] = sum * scale;
    }
}

// Packed scatter (the default): block c < npack takes a run of consecutive
// rows of at most SCATTER_LONG entries each, at most SCATTER_PACK entries in
// all (descriptor {first row, end row, first entry, end entry} from set-up).
// Every thread loads its entries' columns and weights (set-up data) before
// the launch dependency is resolved, then multiplies by w into shared
// memory; one thread per row adds its products in ascending entry order.
// Blocks from npack on take the chunks of the long rows exactly as
// scatter_kernel does (fixed-order tree per chunk, chunks added in order).
constexpr int SCATTER_PACK = 2048;
constexpr int PACK_THREADS = 256;
template <class Real>
__global__ void __launch_bounds__(PACK_THREADS) scatter_packed_kernel(
    const int32_t* __restrict__ ptr, const int32_t* __restrict__ col, const Real* __restrict__ val,
    const Real* __restrict__ w, Real* __restrict__ y, Real scale, int64_t ws, int64_t ys,
    const int4* __restrict__ pdesc, unsigned npack, LongRows lr, Real* partial, unsigned* counters, GroupArg ga) {
    w += blockIdx.y * ws;
    y += blockIdx.y * ys;
    int64_t part_off = (int64_t)blockIdx.y * lr.nchunks, cnt_off = (int64_t)blockIdx.y * lr.nrows;
    if (ga.iv) {   // a group: this column's instance (the grid covers the largest one)
        const InstView& I = ga.iv[blockIdx.y / ga.nbper];
        ptr = I.csr_ptr;
        col = I.csr_col;
        val = sizeof(Real) == 4 ? reinterpret_cast<const Real*>(I.csr_val32) : reinterpret_cast<const Real*>(I.csr_val64);
        pdesc = I.pack_desc;
        npack = (unsigned)I.n_pack;
        lr = LongRows{I.cbeg, I.cend, I.crow, I.lrows, I.cptr, I.nchunks, I.nrows};
        const int64_t c = blockIdx.y % ga.nbper;
        part_off = I.part_off + c * I.nchunks;
        cnt_off = I.cnt_off + c * I.nrows;
        if (blockIdx.x >= npack + lr.nchunks) {
            pdl_trigger();
            return;
        }
    }
    if (blockIdx.x >= npack) {
        pdl_trigger();
        pdl_wait();
        if (column_skipped(ga)) return;
        __shared__ Real part[256];
        __shared__ bool last;
        const int64_t c = blockIdx.x - npack;
        Real* pp = partial + part_off;
        unsigned* cnt = counters + cnt_off;
        const Real sum = chunk_sum<Real>(col, val, w, __ldg(&lr.cbeg[c]), __ldg(&lr.cend[c]), part);
        const int r = __ldg(&lr.crow[c]);
        const int c0 = __ldg(&lr.cptr[r]), c1 = __ldg(&lr.cptr[r + 1]);
        if (threadIdx.x == 0) {
            pp[c] = sum;
            __threadfence();
            last = atomicAdd(&cnt[r], 1u) == (unsigned)(c1 - c0 - 1);
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            Real acc = 0;
            for (int k = c0; k < c1; ++k) acc += ((volatile Real*)pp)[k];
            y[__ldg(&lr.rows[r])] = acc * scale;
            cnt[r] = 0;   // ready for the next product
        }
        return;
    }
    __shared__ Real pr[SCATTER_PACK];
    __shared__ int rp[SCATTER_PACK + 1];
    constexpr int PER = SCATTER_PACK / PACK_THREADS;
    const int4 d = __ldg(&pdesc[blockIdx.x]);   // r0, r1, e0, e1
    const int nr = d.y - d.x;
    for (int r = threadIdx.x; r <= nr; r += PACK_THREADS) rp[r] = __ldg(&ptr[d.x + r]) - d.z;
    int cc[PER];
    Real vv[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int e = d.z + threadIdx.x + PACK_THREADS * j;
        cc[j] = e < d.w ? __ldg(&col[e]) : -1;
        vv[j] = e < d.w ? __ldg(&val[e]) : (Real)0;
    }
    pdl_trigger();
    pdl_wait();
    if (column_skipped(ga)) return;
#pragma unroll
    for (int j = 0; j < PER; ++j)
        if (cc[j] >= 0) pr[threadIdx.x + PACK_THREADS * j] = vv[j] * __ldg(&w[cc[j]]);
    __syncthreads();
    for (int r = threadIdx.x; r < nr; r += PACK_THREADS) {
        Real s = 0;
        for (int k = rp[r]; k < rp[r + 1]; ++k) s += pr[k];
        y[d.x + r] = s * scale;
    }
}

// x[v2i[v]] = u[v] for the interior vertices, x[n_int] = 0: u is read in vertex
// order (coalesced also when it lives in mapped host memory)
template <class Real>
__global__ void compact_kernel(const Real* __restrict__ u, const int32_t* __restrict__ v2i, int64_t nv,
                               int64_t nint, Real* __restrict__ x) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = v2i[v];
        if (i >= 0) x[i] = u[v];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) x[nint] = (Real)0;
}

template <class Real>
__global__ void expand_kernel(const Real* __restrict__ y, const int32_t* __restrict__ v2i, int64_t nv,
                              const double* __restrict__ colsum, double scale, Real* __restrict__ u) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = v2i[v];
        Real r = 0;
        if (i >= 0) {
            r = y[i];
            if (colsum) r = (Real)((double)r * scale / colsum[i]);
        }
        u[v] = r;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct ApplyCfg {
    LinePlan row, col;
    int lpc;          // lines per CTA in the row kernels
    int tc32, tc64;   // columns per CTA in the column kernels
};

static ApplyCfg cfg_for(const gofd_problem* p) {
    ApplyCfg c;
    c.row = make_line_plan(p->P / 2);
    c.col = make_line_plan(p->P);
    c.lpc = std::max(1, 256 / c.row.nthr);
    c.tc32 = std::max(1, std::min(16, 8192 / p->P));
    c.tc64 = std::max(1, std::min(16, 4096 / p->P));
    return c;
}

template <class Real> static size_t row_smem(const ApplyCfg& c) {
    return sizeof(typename Cplx<Real>::T) * spad_len(c.row.N) * c.lpc;
}
template <class Real> static size_t col_smem(const ApplyCfg& c, int tc) {
    return sizeof(typename Cplx<Real>::T) * spad_len(c.col.N) * tc;
}

// The dynamic shared-memory limit is a per-kernel attribute shared by every
// handle, so it is raised once to the device's opt-in maximum; each launch
// still requests only what its line length needs.
template <class Real> static void set_smem_attrs(int limit) {
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_forward_kernel<Real, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_forward_kernel<Real, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_forward_kernel<Real, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_inverse_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(col_fft_kernel<Real, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(col_fft_kernel<Real, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(col_fft_kernel<Real, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
}

void setup_apply(gofd_problem* p) {
    ApplyCfg c = cfg_for(p);
    const int P = p->P, d = p->d;
    p->pitch0 = ((P / 2 + 1) + 15) / 16 * 16;
    const int64_t n = p->n[0];
    int64_t rowsA = p->nlines;
    size_t cbytes = sizeof(double2);
    if (d == 1) p->specA.alloc(cbytes * rowsA * p->pitch0);   // 2D and 3D use their own layouts
    (void)n;
    p->gridw.alloc(sizeof(double) * p->ngrid);
    p->xin.alloc(sizeof(double) * (p->nint + 1));
    p->yout.alloc(sizeof(double) * (p->nint + 1));
    {
        // long rows of I^T and their chunks (set-up bookkeeping on the host)
        std::vector<int32_t> ptr(p->nint + 1), rows, cptr(1, 0), cb, ce, cr;
        GOFD_CUDA_TRY(cudaMemcpy(ptr.data(), p->csr_ptr.ptr, 4 * (p->nint + 1), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < p->nint; ++i)
            if (ptr[i + 1] - ptr[i] > SCATTER_LONG) {
                rows.push_back((int32_t)i);
                for (int32_t a = ptr[i]; a < ptr[i + 1]; a += SCATTER_CHUNK) {
                    cb.push_back(a);
                    ce.push_back(std::min(a + SCATTER_CHUNK, ptr[i + 1]));
                    cr.push_back((int32_t)rows.size() - 1);
                }
                cptr.push_back((int32_t)cb.size());
            }
        // packed runs of short rows for scatter_packed_kernel: {r0, r1, e0, e1}
        std::vector<int4> pd;
        for (int64_t i = 0; i < p->nint;) {
            if (ptr[i + 1] - ptr[i] > SCATTER_LONG) { ++i; continue; }
            const int64_t r0 = i;
            while (i < p->nint && i - r0 < SCATTER_PACK && ptr[i + 1] - ptr[i] <= SCATTER_LONG &&
                   ptr[i + 1] - ptr[r0] <= SCATTER_PACK)
                ++i;
            pd.push_back(make_int4((int)r0, (int)i, ptr[r0], ptr[i]));
        }
        p->n_pack = (int64_t)pd.size();
        p->pack_desc.alloc(sizeof(int4) * (pd.size() + 1));
        if (!pd.empty())
            GOFD_CUDA_TRY(cudaMemcpy(p->pack_desc.ptr, pd.data(), sizeof(int4) * pd.size(), cudaMemcpyHostToDevice));
        p->n_long_rows = (int64_t)rows.size();
        p->n_long_chunks = (int64_t)cb.size();
        p->long_rows.alloc(4 * (rows.size() + 1));
        p->long_chunk_ptr.alloc(4 * cptr.size());
        p->chunk_beg.alloc(4 * (cb.size() + 1));
        p->chunk_end.alloc(4 * (ce.size() + 1));
        p->chunk_row.alloc(4 * (cr.size() + 1));
        p->long_partial.alloc(8 * (cb.size() + 1));
        p->long_cnt.alloc(4 * (rows.size() + 1));
        GOFD_CUDA_TRY(cudaMemset(p->long_cnt.ptr, 0, 4 * (rows.size() + 1)));
        if (!rows.empty()) {
            GOFD_CUDA_TRY(cudaMemcpy(p->chunk_row.ptr, cr.data(), 4 * cr.size(), cudaMemcpyHostToDevice));
            GOFD_CUDA_TRY(cudaMemcpy(p->long_rows.ptr, rows.data(), 4 * rows.size(), cudaMemcpyHostToDevice));
            GOFD_CUDA_TRY(cudaMemcpy(p->long_chunk_ptr.ptr, cptr.data(), 4 * cptr.size(), cudaMemcpyHostToDevice));
            GOFD_CUDA_TRY(cudaMemcpy(p->chunk_beg.ptr, cb.data(), 4 * cb.size(), cudaMemcpyHostToDevice));
            GOFD_CUDA_TRY(cudaMemcpy(p->chunk_end.ptr, ce.data(), 4 * ce.size(), cudaMemcpyHostToDevice));
        }
    }
    int limit = 0;
    GOFD_CUDA_TRY(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    const size_t need = std::max({row_smem<double>(c), col_smem<float>(c, c.tc32), col_smem<double>(c, c.tc64)});
    if (need > (size_t)limit) fail(GOFD_E_GRID, "FFT line does not fit in shared memory");
    set_smem_attrs<float>(limit);
    set_smem_attrs<double>(limit);
    if (d == 2) setup_apply_2d(p);
    if (d == 3) setup_apply_3d(p);
}

// Optional stage markers: when non-null, an event is recorded on the stream
// after every launch of the product (used by gofd_apply_interior_profiled).
struct StageEvents {
    static constexpr int kMax = 32;
    cudaEvent_t ev[kMax];
    const char* name[kMax];
    int n = 0;
};
static thread_local StageEvents* g_marks = nullptr;

void mark_stage(cudaStream_t st, const char* name) {
    if (!g_marks || g_marks->n >= StageEvents::kMax) return;
    GOFD_CUDA_TRY(cudaEventRecord(g_marks->ev[g_marks->n], st));
    g_marks->name[g_marks->n++] = name;
}

template <class Real>
static void afd_core(gofd_problem* p, const ApplyCfg& c, const Real* x, const Real* vgrid, Real* wgrid,
                     cudaStream_t st) {
    using C = typename Cplx<Real>::T;
    if (p->d == 2) {
        if (sizeof(Real) == 4) afd_2d_f32(p, (const float*)x, (const float*)vgrid, (float*)wgrid, 1, 0, 0, nullptr, st);
        else afd_2d_f64(p, (const double*)x, (const double*)vgrid, (double*)wgrid, 1, 0, 0, nullptr, st);
        return;
    }
    if (p->d == 3) {
        if (sizeof(Real) == 4) afd_3d_f32(p, (const float*)x, (const float*)vgrid, (float*)wgrid, st);
        else afd_3d_f64(p, (const double*)x, (const double*)vgrid, (double*)wgrid, st);
        return;
    }
    // 1D: gather + real FFT, symbol, inverse real FFT
    const int P = p->P, H = P / 2 + 1;
    const int64_t n = p->n[0];
    const C* tw = reinterpret_cast<const C*>(sizeof(Real) == 4 ? p->tw32.ptr : p->tw64.ptr);
    const Real* lam = reinterpret_cast<const Real*>(sizeof(Real) == 4 ? p->lam32.ptr : p->lam64.ptr);
    const Real* w = reinterpret_cast<const Real*>(sizeof(Real) == 4 ? p->ell_w32.ptr : p->ell_w64.ptr);
    C* A = p->specA.as<C>();

    // 1. gather + forward real FFT along axis 0
    {
        const int threads = c.lpc * c.row.nthr;
        const unsigned blocks = (unsigned)((p->nlines + c.lpc - 1) / c.lpc);
        const size_t sm = row_smem<Real>(c);
        const int gfg = vgrid != nullptr;
#define ROWF(DP1)                                                                                      \
    row_forward_kernel<Real, DP1><<<blocks, threads, sm, st>>>(                                        \
        x, p->ell_iidx.as<int32_t>(), w, p->nloc, p->line_run_ptr.as<int32_t>(), p->run_k0.as<int32_t>(), \
        p->run_len.as<int32_t>(), p->run_e0.as<int32_t>(), p->nlines, c.row, tw, A, p->pitch0, gfg, vgrid, \
        (int)n)
        ROWF(2);
#undef ROWF
        GOFD_CHECK_LAUNCH();
        mark_stage(st, "gather_row_fft");
    }
    // 2. 1D: the symbol multiply (2D and 3D take their own paths above)
    spec_scale_kernel<Real><<<grid_blocks(H, 256), 256, 0, st>>>(A, lam, H);
    GOFD_CHECK_LAUNCH();
    mark_stage(st, "symbol_mul");
    // 3. inverse real FFT along axis 0
    {
        const int threads = c.lpc * c.row.nthr;
        const unsigned blocks = (unsigned)((p->nlines + c.lpc - 1) / c.lpc);
        row_inverse_kernel<Real><<<blocks, threads, row_smem<Real>(c), st>>>(A, p->pitch0, p->nlines, c.row, tw,
                                                                           wgrid, (int)n);
        GOFD_CHECK_LAUNCH();
        mark_stage(st, "row_ifft");
    }
}

// y_b = scale * I^T w_b for nb right-hand sides (w_b = wgrid + b ws, y_b = y + b ys);
// partial / counters: nb x n_long_chunks reals and nb x n_long_rows zeroed
// counters for the long rows (NULL: the handle's, nb = 1).  One launch.
template <class Real>
static void scatter_b(gofd_problem* p, const Real* wgrid, Real* y, Real scale, int nb, int64_t ws, int64_t ys,
                      Real* partial, unsigned* counters, cudaStream_t st, GroupArg ga = GroupArg{}) {
    const Real* val = reinterpret_cast<const Real*>(sizeof(Real) == 4 ? p->csr_val32.ptr : p->csr_val64.ptr);
    const double avg = p->nint ? (double)p->nnz_t / p->nint : 0;
    const int threads = 256;
    int tpr = avg > 96 ? 32 : (avg > 24 ? 8 : 4);
    if (p->tune_tpr == 4 || p->tune_tpr == 8 || p->tune_tpr == 16 || p->tune_tpr == 32) tpr = p->tune_tpr;
    LongRows lr{p->chunk_beg.as<int32_t>(), p->chunk_end.as<int32_t>(), p->chunk_row.as<int32_t>(),
                p->long_rows.as<int32_t>(), p->long_chunk_ptr.as<int32_t>(), p->n_long_chunks, p->n_long_rows};
    Real* part = partial ? partial : reinterpret_cast<Real*>(p->long_partial.ptr);
    unsigned* cnt = counters ? counters : p->long_cnt.as<unsigned>();
    if (p->tune_tpr == 0 || ga.iv) {   // default, and every group: the packed kernel
        const dim3 grid((unsigned)(ga.iv ? ga.max_scatter : p->n_pack + p->n_long_chunks), nb);
        if (grid.x == 0) return;
        launch_pdl(scatter_packed_kernel<Real>, grid, dim3(PACK_THREADS), 0, st, p->csr_ptr.as<int32_t>(),
                   p->csr_col.as<int32_t>(), val, wgrid, y, scale, ws, ys, p->pack_desc.as<int4>(),
                   (unsigned)p->n_pack, lr, part, cnt, ga);
        GOFD_CHECK_LAUNCH();
        mark_stage(st, "scatter");
        return;
    }
    // at most one wave of CTAs (the short-row loop is grid-stride): a second
    // wave cannot load its first entries while the previous kernel finishes
    const unsigned nshort = (unsigned)grid_blocks(p->nint * tpr, threads, p->sm_count * (2048 / threads));
    const dim3 grid(nshort + (unsigned)p->n_long_chunks, nb);
#define SCAT(TPR)                                                                                              \
    launch_pdl(scatter_kernel<Real, TPR>, grid, dim3(threads), 0, st, p->csr_ptr.as<int32_t>(),                   \
               p->csr_col.as<int32_t>(), val, wgrid, p->nint, y, scale, ws, ys, nshort, lr, part, cnt, ga)
    if (tpr == 32) SCAT(32);
    else if (tpr == 16) SCAT(16);
    else if (tpr == 8) SCAT(8);
    else SCAT(4);
#undef SCAT
    GOFD_CHECK_LAUNCH();
    mark_stage(st, "scatter");
}

template <class Real>
static void scatter(gofd_problem* p, const Real* wgrid, Real* y, Real scale, cudaStream_t st) {
    scatter_b<Real>(p, wgrid, y, scale, 1, 0, 0, nullptr, nullptr, st);
}

template <class Real>
static void apply_t(gofd_problem* p, const Real* x, Real* y, cudaStream_t st) {
    ApplyCfg c = cfg_for(p);
    Real* wg = p->gridw.as<Real>();
    afd_core<Real>(p, c, x, nullptr, wg, st);
    scatter<Real>(p, wg, y, (Real)1, st);
}

void apply_interior(gofd_problem* p, bool fp64, const void* x, void* y, cudaStream_t st) {
    if (fp64) apply_t<double>(p, (const double*)x, (double*)y, st);
    else apply_t<float>(p, (const float*)x, (float*)y, st);
}

void apply_interior_df(gofd_problem* p, const double* x, double* y, cudaStream_t st) {
    if (p->d != 2 && p->d != 3) fail(GOFD_E_ARG, "the double-float product is 2D and 3D");
    double* wg = p->gridw.as<double>();
    if (p->d == 2) afd_2d_df(p, x, nullptr, wg, 1, 0, 0, nullptr, st);
    else afd_3d_df(p, x, nullptr, wg, st);
    scatter<double>(p, wg, y, 1.0, st);
}

void apply_interior_residual(gofd_problem* p, const double* x, double* y, cudaStream_t st) {
    if (p->d >= 2 && p->opt.fp64_residual == 0) apply_interior_df(p, x, y, st);
    else apply_interior(p, true, x, y, st);
}

void apply_interior_symbol(gofd_problem* p, bool fp64, const void* x, void* y, const void* lamT, cudaStream_t st) {
    if (p->d != 2) fail(GOFD_E_ARG, "a replaced symbol is supported in 2D only");
    GroupArg ga;
    if (fp64) {
        ga.lam64 = static_cast<const double*>(lamT);
        double* wg = p->gridw.as<double>();
        afd_2d_f64(p, (const double*)x, nullptr, wg, 1, 0, 0, nullptr, st, ga);
        scatter<double>(p, wg, (double*)y, 1.0, st);
    } else {
        ga.lam32 = static_cast<const float*>(lamT);
        float* wg = p->gridw.as<float>();
        afd_2d_f32(p, (const float*)x, nullptr, wg, 1, 0, 0, nullptr, st, ga);
        scatter<float>(p, wg, (float*)y, 1.0f, st);
    }
}

int apply_interior_profiled(gofd_problem* p, bool fp64, const void* x, void* y, cudaStream_t st, float* ms,
                            const char** names, int cap) {
    StageEvents se;
    for (int i = 0; i < StageEvents::kMax; ++i) GOFD_CUDA_TRY(cudaEventCreate(&se.ev[i]));
    cudaEvent_t start;
    GOFD_CUDA_TRY(cudaEventCreate(&start));
    GOFD_CUDA_TRY(cudaEventRecord(start, st));
    g_marks = &se;
    try {
        apply_interior(p, fp64, x, y, st);
    } catch (...) {
        g_marks = nullptr;
        throw;
    }
    g_marks = nullptr;
    GOFD_CUDA_TRY(cudaEventSynchronize(se.ev[se.n - 1]));
    int n = se.n < cap ? se.n : cap;
    cudaEvent_t prev = start;
    for (int i = 0; i < n; ++i) {
        GOFD_CUDA_TRY(cudaEventElapsedTime(&ms[i], prev, se.ev[i]));
        if (names) names[i] = se.name[i];
        prev = se.ev[i];
    }
    for (int i = 0; i < StageEvents::kMax; ++i) cudaEventDestroy(se.ev[i]);
    cudaEventDestroy(start);
    return n;
}

// Y[b] = S X[b] for nb interior vectors: X[b] = x + b ld (ld >= n_int + 1, pad
// slot zero), Y[b] = y + b ld.  2D: one launch sequence over the batch with
// the scratch of the batch workspace; otherwise one product per vector.
void apply_interior_batch(gofd_problem* p, bool fp64, const void* x, void* y, int nb, int64_t ld, void* grid_ws,
                          void* spec_ws, void* partial_ws, void* counter_ws, cudaStream_t st, const int* skip,
                          int skip_stride, bool df) {
    if (p->d == 2) {
        // columns in sub-batches of p->tune_bchunk (0: all at once); each
        // sub-batch reuses the first workspace slots, so a small one keeps its
        // spectra in L2
        const int64_t ws = p->ngrid;
        const int cs = (p->tune_bchunk > 0 && p->tune_bchunk < nb) ? p->tune_bchunk : nb;
        const size_t b = fp64 ? 8 : 4;
        for (int c0 = 0; c0 < nb; c0 += cs) {
            const int k = std::min(cs, nb - c0);
            const char* xc = (const char*)x + (int64_t)c0 * ld * b;
            char* yc = (char*)y + (int64_t)c0 * ld * b;
            GroupArg ga;
            ga.skip = skip;
            ga.skip_stride = skip_stride;
            ga.col0 = c0;
            if (fp64) {
                if (df) afd_2d_df(p, (const double*)xc, nullptr, (double*)grid_ws, k, ld, ws, spec_ws, st, ga);
                else afd_2d_f64(p, (const double*)xc, nullptr, (double*)grid_ws, k, ld, ws, spec_ws, st, ga);
                scatter_b<double>(p, (const double*)grid_ws, (double*)yc, 1.0, k, ws, ld, (double*)partial_ws,
                                  (unsigned*)counter_ws, st, ga);
            } else {
                afd_2d_f32(p, (const float*)xc, nullptr, (float*)grid_ws, k, ld, ws, spec_ws, st, ga);
                scatter_b<float>(p, (const float*)grid_ws, (float*)yc, 1.0f, k, ws, ld, (float*)partial_ws,
                                 (unsigned*)counter_ws, st, ga);
            }
        }
        return;
    }
    const size_t b = fp64 ? 8 : 4;
    for (int k = 0; k < nb; ++k) {
        const char* xk = (const char*)x + k * ld * b;
        char* yk = (char*)y + k * ld * b;
        if (fp64 && df && p->d == 3) apply_interior_df(p, (const double*)xk, (double*)yk, st);
        else apply_interior(p, fp64, xk, yk, st);
    }
}

// Y[c] = S_i X[c] for the columns of a group of 2D problems on one grid
// (instance i = c / ga.nbper, views in ga.iv): one launch sequence for all
// columns.  Columns have length ld; entries past an instance's n_int are zero
// and stay zero.  rp supplies the grid, the twiddles and the launch shapes.
void apply_interior_group(gofd_problem* rp, bool fp64, const void* x, void* y, int nbtot, int64_t ld, void* grid_ws,
                          void* spec_ws, void* partial_ws, void* counter_ws, GroupArg ga, cudaStream_t st,
                          bool df) {
    const int64_t ws = rp->ngrid;
    if (fp64) {
        if (df) afd_2d_df(rp, (const double*)x, nullptr, (double*)grid_ws, nbtot, ld, ws, spec_ws, st, ga);
        else afd_2d_f64(rp, (const double*)x, nullptr, (double*)grid_ws, nbtot, ld, ws, spec_ws, st, ga);
        scatter_b<double>(rp, (const double*)grid_ws, (double*)y, 1.0, nbtot, ws, ld, (double*)partial_ws,
                          (unsigned*)counter_ws, st, ga);
    } else {
        afd_2d_f32(rp, (const float*)x, nullptr, (float*)grid_ws, nbtot, ld, ws, spec_ws, st, ga);
        scatter_b<float>(rp, (const float*)grid_ws, (float*)y, 1.0f, nbtot, ws, ld, (float*)partial_ws,
                         (unsigned*)counter_ws, st, ga);
    }
}

InstView inst_view(const gofd_problem* p) {
    InstView v;
    v.ell_iidx = p->ell_iidx.as<int32_t>();
    v.ell_w32 = p->ell_w32.as<float>();
    v.ell_w64 = p->ell_w64.as<double>();
    v.ell_node = p->ell_node.as<int32_t>();
    v.nloc = p->nloc;
    v.run_ptr = p->line_run_ptr.as<int32_t>();
    v.run_k0 = p->run_k0.as<int32_t>();
    v.run_len = p->run_len.as<int32_t>();
    v.run_e0 = p->run_e0.as<int32_t>();
    v.wdesc_line = p->wdesc_line.as<int4>();
    v.ell4_node = p->ell4_node.as<int32_t>();
    v.ell4_iidx = p->ell4_iidx.as<int32_t>();
    v.ell4_w32 = p->ell4_w32.as<float>();
    v.ell4_ld = p->ell4_ld;
    v.lamT32 = p->lamT32.as<float>();
    v.lamT64 = p->lamT64.as<double>();
    v.csr_ptr = p->csr_ptr.as<int32_t>();
    v.csr_col = p->csr_col.as<int32_t>();
    v.csr_val32 = p->csr_val32.as<float>();
    v.csr_val64 = p->csr_val64.as<double>();
    v.pack_desc = p->pack_desc.as<int4>();
    v.n_pack = p->n_pack;
    v.cbeg = p->chunk_beg.as<int32_t>();
    v.cend = p->chunk_end.as<int32_t>();
    v.crow = p->chunk_row.as<int32_t>();
    v.lrows = p->long_rows.as<int32_t>();
    v.cptr = p->long_chunk_ptr.as<int32_t>();
    v.nchunks = p->n_long_chunks;
    v.nrows = p->n_long_rows;
    v.part_off = v.cnt_off = 0;
    return v;
}

void afd_of_interior(gofd_problem* p, bool fp64, const void* x, void* wgrid, cudaStream_t st) {
    ApplyCfg c = cfg_for(p);
    if (fp64) afd_core<double>(p, c, (const double*)x, nullptr, (double*)wgrid, st);
    else afd_core<float>(p, c, (const float*)x, nullptr, (float*)wgrid, st);
}

void afd_apply_grid(gofd_problem* p, bool fp64, const void* v, void* w, cudaStream_t st) {
    ApplyCfg c = cfg_for(p);
    if (fp64) afd_core<double>(p, c, nullptr, (const double*)v, (double*)w, st);
    else afd_core<float>(p, c, nullptr, (const float*)v, (float*)w, st);
}

void compact_vertex(gofd_problem* p, bool fp64, const void* u, void* x, cudaStream_t st) {
    if (fp64)
        compact_kernel<double><<<grid_blocks(p->nv, 256), 256, 0, st>>>(
            (const double*)u, p->vert2int.as<int32_t>(), p->nv, p->nint, (double*)x);
    else
        compact_kernel<float><<<grid_blocks(p->nv, 256), 256, 0, st>>>(
            (const float*)u, p->vert2int.as<int32_t>(), p->nv, p->nint, (float*)x);
    GOFD_CHECK_LAUNCH();
}

void expand_interior(gofd_problem* p, bool fp64, const void* y, void* u, double scale_by_inv_colsum,
                     cudaStream_t st) {
    const double* cs = scale_by_inv_colsum != 0.0 ? p->colsum.as<double>() : nullptr;
    if (fp64)
        expand_kernel<double><<<grid_blocks(p->nv, 256), 256, 0, st>>>(
            (const double*)y, p->vert2int.as<int32_t>(), p->nv, cs, scale_by_inv_colsum, (double*)u);
    else
        expand_kernel<float><<<grid_blocks(p->nv, 256), 256, 0, st>>>(
            (const float*)y, p->vert2int.as<int32_t>(), p->nv, cs, scale_by_inv_colsum, (float*)u);
    GOFD_CHECK_LAUNCH();
}

// y = scale * I^T f for a grid vector f (FP64): the RHS of (GoFD-2)
void scatter_grid_f64(gofd_problem* p, const double* f, double* y, double scale, cudaStream_t st) {
    scatter<double>(p, f, y, scale, st);
}

}  // namespace gofd

// ===========================================================================
// Allocation-free grid convolution w = A_FD v (FP32).
//
// Some callers cannot call cudaMalloc when they need this product: plug-ins
// living inside a host framework whose device memory is entirely owned by
// that framework's own allocator (an allocation behind its back can fail or
// break its accounting), real-time loops that must not risk an allocation
// failure or its latency, and code whose device memory is fixed up front.  This variant takes the symbol,
// the input and the output from the caller and keeps its spectrum scratch in
// a fixed file-scope device array instead of any allocation.  Every GPU that
// loads the library holds that array (8.1 MiB plus 32 KiB of twiddle tables)
// until the process exits.  It launches the generic line-FFT kernels of this
// file (gather-free row FFTs, column FFTs, inverse row FFTs).
// ===========================================================================
namespace gofd {

constexpr int64_t NOALLOC_MAX_COMPLEX = 1064960;  // 1024 rows x 1040: a 2D grid with n <= 1024
constexpr int NOALLOC_MIN_P = 32, NOALLOC_MAX_P = 2048;
// twiddle tables e^{-2 pi i m / P}, m < P, one per power of two P from 32 to
// 2048, stored one after another: the table of P starts at entry P - 32
constexpr int NOALLOC_TW_ENTRIES = 2 * NOALLOC_MAX_P - NOALLOC_MIN_P;
static __device__ __align__(256) float2 g_noalloc_spec[NOALLOC_MAX_COMPLEX];
static __device__ __align__(256) float2 g_noalloc_tw[NOALLOC_TW_ENTRIES];

struct NoallocDevice {
    bool ready = false;
    float2* spec = nullptr;  // device address of g_noalloc_spec on this device
    float2* tw = nullptr;    // device address of g_noalloc_tw on this device
};
static std::mutex g_noalloc_mu;
static NoallocDevice g_noalloc_devices[128];

// every table at once: entry i belongs to the table of P = the largest power
// of two <= i + 32, at position m = i - (P - 32)
__global__ void noalloc_twiddle_kernel(float2* __restrict__ tw) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NOALLOC_TW_ENTRIES; i += gridDim.x * blockDim.x) {
        int P = NOALLOC_MIN_P;
        while (2 * P <= i + NOALLOC_MIN_P) P *= 2;
        const int m = i - (P - NOALLOC_MIN_P);
        double sn, cs;
        sincospi(2.0 * (double)m / (double)P, &sn, &cs);
        tw[i] = make_float2((float)cs, (float)-sn);
    }
}

// Set-up once per device, with that device current: look up the arrays'
// device addresses (a host-side symbol is not a device address), raise the
// kernels' dynamic shared-memory limit and fill the twiddle tables (one
// launch on the caller's stream, waited for, so that later calls on any
// stream see the tables).
static NoallocDevice noalloc_device(cudaStream_t st) {
    int dev = 0;
    GOFD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) fail(GOFD_E_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice& d = g_noalloc_devices[dev];
    if (!d.ready) {
        void* spec = nullptr;
        void* tw = nullptr;
        GOFD_CUDA_TRY(cudaGetSymbolAddress(&spec, g_noalloc_spec));
        GOFD_CUDA_TRY(cudaGetSymbolAddress(&tw, g_noalloc_tw));
        int limit = 0;
        GOFD_CUDA_TRY(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        set_smem_attrs<float>(limit);
        noalloc_twiddle_kernel<<<grid_blocks(NOALLOC_TW_ENTRIES, 256), 256, 0, st>>>(static_cast<float2*>(tw));
        GOFD_CHECK_LAUNCH();
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
        d.spec = static_cast<float2*>(spec);
        d.tw = static_cast<float2*>(tw);
        d.ready = true;
    }
    return d;
}

void afd_apply_noalloc(int d, int n, const float* lam, const float* v, float* w, cudaStream_t st) {
    if (d < 1 || d > 3) fail(GOFD_E_ARG, "d must be 1, 2 or 3");
    if (n < 2) fail(GOFD_E_ARG, "n must be at least 2");
    if (!lam || !v || !w) fail(GOFD_E_ARG, "NULL vector");
    int P = 1;
    while (P < 2 * n - 2) P *= 2;
    if (P < 32) P = 32;
    const int H = P / 2 + 1;
    const int pitch = (H + 15) / 16 * 16;
    int64_t nlines = 1;
    for (int i = 1; i < d; ++i) nlines *= n;
    const int64_t needA = nlines * pitch;
    const int64_t needB = (d == 3) ? (int64_t)n * P * pitch : 0;
    if (P > NOALLOC_MAX_P || needA + needB > NOALLOC_MAX_COMPLEX)
        fail(GOFD_E_ARG, "grid too large for the static scratch of 1064960 complex values "
                         "(a 2D grid needs n*pitch, a 3D grid n^2*pitch + n*P*pitch, pitch = P/2+1 rounded up to 16)");
    const NoallocDevice dv = noalloc_device(st);
    float2* A = dv.spec;
    float2* B = dv.spec + needA;
    const float2* tw = dv.tw + (P - NOALLOC_MIN_P);
    const LinePlan row = make_line_plan(P / 2), col = make_line_plan(P);
    const int lpc = std::max(1, 256 / row.nthr);
    const int tc = std::max(1, std::min(16, 8192 / P));
    const size_t rsm = sizeof(float2) * spad_len(row.N) * lpc;
    const size_t csm = sizeof(float2) * spad_len(col.N) * tc;
    const unsigned rblocks = (unsigned)((nlines + lpc - 1) / lpc);
    // forward real FFT along axis 0 of the caller's grid vector
    if (d == 1)
        row_forward_kernel<float, 2><<<rblocks, lpc * row.nthr, rsm, st>>>(
            nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, nlines, row, tw, A, pitch, 1, v, n);
    else if (d == 2)
        row_forward_kernel<float, 3><<<rblocks, lpc * row.nthr, rsm, st>>>(
            nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, nlines, row, tw, A, pitch, 1, v, n);
    else
        row_forward_kernel<float, 4><<<rblocks, lpc * row.nthr, rsm, st>>>(
            nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, nlines, row, tw, A, pitch, 1, v, n);
    GOFD_CHECK_LAUNCH();
    const unsigned cblocks = (unsigned)((H + tc - 1) / tc);
    const int threads_c = tc * col.nthr;
    if (d == 1) {
        spec_scale_kernel<float><<<grid_blocks(H, 256), 256, 0, st>>>(A, lam, H);
    } else if (d == 2) {
        ColDesc cd{0, pitch, 0, pitch, n, n, H, tc, 0, H, P};
        col_fft_kernel<float, 1><<<dim3(cblocks, 1), threads_c, csm, st>>>(A, A, cd, col, tw, lam);
    } else {
        const int64_t pt = pitch;
        ColDesc f{(int64_t)n * pt, pt, (int64_t)P * pt, pt, n, P, H, tc, 0, 0, P};
        col_fft_kernel<float, 0><<<dim3(cblocks, (unsigned)n), threads_c, csm, st>>>(A, B, f, col, tw, lam);
        GOFD_CHECK_LAUNCH();
        ColDesc m{pt, (int64_t)P * pt, pt, (int64_t)P * pt, n, n, H, tc, (int64_t)H, (int64_t)H * H, P};
        col_fft_kernel<float, 1><<<dim3(cblocks, (unsigned)P), threads_c, csm, st>>>(B, B, m, col, tw, lam);
        GOFD_CHECK_LAUNCH();
        ColDesc iv{(int64_t)P * pt, pt, (int64_t)n * pt, pt, P, n, H, tc, 0, 0, P};
        col_fft_kernel<float, 2><<<dim3(cblocks, (unsigned)n), threads_c, csm, st>>>(B, A, iv, col, tw, lam);
    }
    GOFD_CHECK_LAUNCH();
    row_inverse_kernel<float><<<rblocks, lpc * row.nthr, rsm, st>>>(A, pitch, nlines, row, tw, w, n);
    GOFD_CHECK_LAUNCH();
}

}  // namespace gofd
