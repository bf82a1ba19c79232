// 2D stiffness-product convolution w = A_FD I x in FP32 for a circulant of
// length 2048 (grids of 514 to 1024 nodes per axis), one warp per 1024-point
// FFT (Section 2.2, (AU-1); gather of (IhFD-1) in front).
//
//   gather_w    v = I x at the located grid nodes, linear over the ELL rows
//               (four consecutive rows per thread, one 16-byte load per ELL
//               array from a copy whose slot stride is padded to four rows;
//               the ELL is set-up data and is loaded before the launch
//               dependency is resolved).  v goes into the output grid buffer, which the
//               inverse row kernel overwrites with w only after the forward
//               row kernel has read v.
//   row_fwd_w   per grid line, one warp: z[m] = v[2m] + i v[2m+1] (zero off the
//               mesh, from the line's runs), a 1024-point FFT in registers
//               (two radix-32 passes, one warp-synchronous transpose), the
//               real-input spectrum
//               unpacked with shuffles into a shared tile of four lines, stored
//               transposed: specT[k_x0][line]
//   col_conv_w  one spectrum column (fixed k_x0, n <= 1024 nonzero rows) per
//               CTA of two warps.  Its 2048-point transform splits into the
//               even bins (the 1024-point FFT of the column) and the odd bins
//               (the 1024-point FFT of the column times W_2048^m); each warp
//               multiplies its bins by the real even symbol, transforms back,
//               and the halves are combined, y[m] = a[m] + W_2048^{-m} b[m],
//               for the n kept rows
//   row_inv_w   the transposed tile of four lines is loaded, each warp packs
//               the real-output inverse, runs the inverse 1024-point FFT and
//               writes the n kept samples
//
// Twiddles come from registers: each lane loads W_1024^{c L} for ten
// multipliers c once (lane L) and forms the other inter-pass twiddles
// W_1024^{k L} = W_1024^{4aL} W_1024^{bL} (k = 4a + b) with one product; every
// W_2048^{L + 32 r} is W_2048^L times the compile-time constant W_64^r.
// While the row kernel works, the symbol and the scatter's CSR are prefetched
// into L2 by bulk prefetches (HBM is otherwise idle then).
#include <algorithm>
#include <cmath>
#include <vector>

#include "gofd_internal.cuh"
#include "fft_common.cuh"
#include "async_copy.cuh"

namespace gofd {

void mark_stage(cudaStream_t st, const char* name);

namespace {

constexpr int WN = 1024;               // FFT length per warp
constexpr int WP = 2048;               // circulant length
constexpr int WH = WP / 2 + 1;         // bins of the real-input transform along axis 0
constexpr int LINES = 4;               // grid lines (warps) per CTA of the row kernels
constexpr int TLD = LINES + 1;         // tile row stride (complex), padded against bank conflicts
constexpr int XB = 33;                 // transpose buffer row stride (complex)
constexpr int XBUF = 32 * XB;          // transpose buffer per warp (complex)
constexpr unsigned FULL = 0xffffffffu;

constexpr size_t ROW_SMEM = (size_t)(LINES * XBUF + WH * TLD) * 8;

// cos(2 pi r / 64), r taken modulo 64
__host__ __device__ constexpr double cos64(int r) {
    constexpr double q[17] = {1.0,
                              0.99518472667219688624,
                              0.98078528040323044913,
                              0.95694033573220886494,
                              0.92387953251128675613,
                              0.88192126434835502971,
                              0.83146961230254523708,
                              0.77301045336273696081,
                              0.70710678118654752440,
                              0.63439328416364549822,
                              0.55557023301960222474,
                              0.47139673682599764856,
                              0.38268343236508977173,
                              0.29028467725446236764,
                              0.19509032201612826785,
                              0.09801714032956060199,
                              0.0};
    r &= 63;
    if (r <= 16) return q[r];
    if (r <= 32) return -q[32 - r];
    if (r <= 48) return -q[r - 32];
    return q[64 - r];
}
// W_64^r = exp(-2 pi i r / 64)
__device__ __forceinline__ float2 w64c(int r) {
    return make_float2((float)cos64(r), (float)-cos64(r - 16));
}

// Per-lane twiddles: b[0..2] = W_1024^{cL} (c = 1, 2, 3), a[0..6] = W_1024^{4cL}
// (c = 1..7), w2 = W_2048^L.
struct LaneTw {
    float2 b[3], a[7], w2;
};
__device__ __forceinline__ LaneTw lane_twiddles(const float2* __restrict__ twp, const float2* __restrict__ tw,
                                                int lane) {
    LaneTw t;
#pragma unroll
    for (int c = 0; c < 3; ++c) t.b[c] = __ldg(&twp[(c + 1) * 32 + lane]);
#pragma unroll
    for (int c = 0; c < 7; ++c) t.a[c] = __ldg(&twp[4 * (c + 1) * 32 + lane]);
    t.w2 = __ldg(&tw[lane]);
    return t;
}
// v * W_1024^{k L} (INV: times the conjugate), k a compile-time constant in 1..31
template <bool INV>
__device__ __forceinline__ float2 tw1024(float2 v, const LaneTw& t, int k) {
    const int a = k >> 2, b = k & 3;
    if (a) v = INV ? cmulc(v, t.a[a - 1]) : cmul(v, t.a[a - 1]);
    if (b) v = INV ? cmulc(v, t.b[b - 1]) : cmul(v, t.b[b - 1]);
    return v;
}
// W_2048^{L + 32 r}
__device__ __forceinline__ float2 tw2048(const LaneTw& t, int r) { return r ? cmul(t.w2, w64c(r)) : t.w2; }

// Forward 32-point DFT of the 32 registers (natural order in and out;
// radix-2 decimation in frequency with constant twiddles).
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int span = 16 >> st;
#pragma unroll
        for (int blk = 0; blk < 32; blk += 2 * span)
#pragma unroll
            for (int j = 0; j < span; ++j) {
                const float2 a = v[blk + j], b = v[blk + j + span];
                v[blk + j] = cadd(a, b);
                v[blk + j + span] = twc32<false>(csub(a, b), j * (32 / (2 * span)));
            }
    }
    float2 t[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) t[k] = v[bitrev(k, 5)];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = t[k];
}

// lane l, register i  <->  lane i, register l, through the warp's buffer
__device__ __forceinline__ void xpose(float2 (&v)[32], float2* buf, int lane) {
#pragma unroll
    for (int i = 0; i < 32; ++i) buf[i * XB + lane] = v[i];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = buf[lane * XB + i];
    __syncwarp();
}

// forward: lane t, register r = x[t + 32 r]  ->  lane k1, register k2 = X[k1 + 32 k2]
// (X[k1 + 32 k2] = sum_t W_32^{t k2} W_1024^{t k1} sum_r W_32^{r k1} x[t + 32 r]).
// The two radix-32 passes run in a loop that is not unrolled, so the kernel
// holds one copy of the 32-point DFT (the instruction cache is small).
__device__ __forceinline__ void wfft_fwd(float2 (&v)[32], float2* buf, int lane, const LaneTw& t) {
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        dft32(v);
        if (h == 1) break;
#pragma unroll
        for (int k1 = 1; k1 < 32; ++k1) v[k1] = tw1024<false>(v[k1], t, k1);
        xpose(v, buf, lane);
    }
}

__device__ __forceinline__ void conj32(float2 (&v)[32]) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i].y = -v[i].y;
}

// inverse, unnormalised: lane k1, register k2 = X[k1 + 32 k2]  ->  lane a, register b = y[a + 32 b].
// The transposed distribution of X is the natural input distribution of the
// forward transform, and sum_k X_k W^{-mk} = conj(sum_k conj(X_k) W^{mk}).
__device__ __forceinline__ void wfft_inv(float2 (&v)[32], float2* buf, int lane, const LaneTw& t) {
    conj32(v);
    wfft_fwd(v, buf, lane, t);
    conj32(v);
}

// one bulk L2 prefetch of this CTA's share of [base, base + bytes) (base
// 16-byte aligned; the shares are multiples of 16 bytes)
__device__ __forceinline__ void prefetch_share(const void* base, int64_t bytes, unsigned cta, unsigned ncta) {
    if (threadIdx.x != 0 || bytes <= 0) return;
    const int64_t share = ((bytes + ncta - 1) / ncta + 15) & ~(int64_t)15;
    const int64_t b0 = (int64_t)cta * share;
    const int64_t b1 = std::min<int64_t>(b0 + share, bytes & ~(int64_t)15);
    if (b1 > b0) bulk_prefetch_l2(static_cast<const char*>(base) + b0, (uint32_t)(b1 - b0));
}

// ---------------------------------------------------------------------------
// kernel 0: gather v = I x at the located grid nodes
// ---------------------------------------------------------------------------
constexpr int GTH = 128;   // threads of the gather kernel
__global__ void __launch_bounds__(GTH, 12) gather_w_kernel(const float* __restrict__ x,
                                                          const int32_t* __restrict__ iidx,
                                                          const float* __restrict__ w,
                                                          const int32_t* __restrict__ node, int64_t ld4,
                                                          float* __restrict__ vgrid, int64_t xstride,
                                                          int64_t vstride, GroupArg ga) {
    if (ga.iv) {   // a group: this column's instance
        const InstView& I = ga.iv[blockIdx.y / ga.nbper];
        iidx = I.ell4_iidx;
        w = I.ell4_w32;
        node = I.ell4_node;
        ld4 = I.ell4_ld;
    }
    x += blockIdx.y * xstride;
    vgrid += blockIdx.y * vstride;
    // rows 4e .. 4e + 3: one 16-byte load per slot array (set-up data, loaded
    // before the predecessor completes); a warp reads 512 contiguous bytes of each
    const int64_t e = (int64_t)blockIdx.x * GTH + threadIdx.x;
    const bool in = 4 * e < ld4;
    int4 nd = make_int4(-1, -1, -1, -1), ii[3];
    float4 ww[3];
    if (in) nd = __ldg(reinterpret_cast<const int4*>(node) + e);
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
        ii[sl] = in ? __ldg(reinterpret_cast<const int4*>(iidx + sl * ld4) + e) : make_int4(0, 0, 0, 0);
        ww[sl] = in ? __ldg(reinterpret_cast<const float4*>(w + sl * ld4) + e) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    pdl_trigger();
    pdl_wait();
    if (column_skipped(ga)) return;
    const int n4[4] = {nd.x, nd.y, nd.z, nd.w};
    float acc[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[r] = 0.f;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
        const int i4[4] = {ii[sl].x, ii[sl].y, ii[sl].z, ii[sl].w};
        const float w4[4] = {ww[sl].x, ww[sl].y, ww[sl].z, ww[sl].w};
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] = fmaf(w4[r], n4[r] >= 0 ? __ldg(&x[i4[r]]) : 0.f, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
        if (n4[r] >= 0) vgrid[n4[r]] = acc[r];
}

// ---------------------------------------------------------------------------
// kernel 1: forward real FFT of four lines of v, transposed store
// ---------------------------------------------------------------------------
// Line descriptors made at set-up: {runs, first run index, k0, len} and
// {0, k0, len, 0} of the line's first two runs; v is read only on the runs.
// pf*: arrays of later kernels (symbol, CSR of I^T) prefetched into L2.
__device__ __forceinline__ bool on_mesh(int k, const int4& d0, const int4& d1, const int32_t* __restrict__ run_k0,
                                        const int32_t* __restrict__ run_len) {
    if (d0.x <= 2) return (k >= d0.z && k < d0.z + d0.w) || (k >= d1.y && k < d1.y + d1.z);
    for (int j = d0.y; j < d0.y + d0.x; ++j) {
        const int a = __ldg(&run_k0[j]);
        if (k >= a && k < a + __ldg(&run_len[j])) return true;
    }
    return false;
}

__global__ void __launch_bounds__(128, 3) row_fwd_w_kernel(
    const float* __restrict__ vgrid, const int4* __restrict__ ldesc, const int32_t* __restrict__ run_k0,
    const int32_t* __restrict__ run_len, int nlines, int n, const float2* __restrict__ tw,
    const float2* __restrict__ twp, const void* pf0, int64_t pb0, const void* pf1, int64_t pb1, const void* pf2,
    int64_t pb2, const void* pf3, int64_t pb3, float2* __restrict__ specT, int ld, int64_t vstride,
    int64_t sstride, GroupArg ga) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int l0 = blockIdx.x * LINES, line = l0 + g;
    if (ga.iv) {
        const InstView& I = ga.iv[blockIdx.y / ga.nbper];
        ldesc = I.wdesc_line;
        run_k0 = I.run_k0;
        run_len = I.run_len;
    }
    vgrid += blockIdx.y * vstride;
    specT += blockIdx.y * sstride;
    const LaneTw t = lane_twiddles(twp, tw, lane);
    int4 d0 = make_int4(0, 0, 0, 0), d1 = make_int4(0, 0, 0, 0);
    if (line < nlines) {
        d0 = __ldg(&ldesc[2 * line]);
        d1 = __ldg(&ldesc[2 * line + 1]);
    }
    pdl_wait();
    if (blockIdx.y == 0 && !ga.iv) {
        prefetch_share(pf0, pb0, blockIdx.x, gridDim.x);
        prefetch_share(pf1, pb1, blockIdx.x, gridDim.x);
        prefetch_share(pf2, pb2, blockIdx.x, gridDim.x);
        prefetch_share(pf3, pb3, blockIdx.x, gridDim.x);
    }
    if (column_skipped(ga)) return;
    // z[t + 32 r] = (v[2t + 64 r], v[2t + 64 r + 1]); z[m] = 0 for m >= 512 (n <= 1024)
    float2 z[32];
    const float* vl = vgrid + (int64_t)line * n;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int k = 2 * lane + 64 * r;
        const bool a = line < nlines && k < n && on_mesh(k, d0, d1, run_k0, run_len);
        const bool b = line < nlines && k + 1 < n && on_mesh(k + 1, d0, d1, run_k0, run_len);
        z[r].x = a ? __ldcg(&vl[k]) : 0.f;
        z[r].y = b ? __ldcg(&vl[k + 1]) : 0.f;
    }
#pragma unroll
    for (int r = 16; r < 32; ++r) z[r] = make_float2(0.f, 0.f);
    float2* xbuf = reinterpret_cast<float2*>(smem_raw) + g * XBUF;
    float2* tile = reinterpret_cast<float2*>(smem_raw) + LINES * XBUF;   // [WH][TLD]
    wfft_fwd(z, xbuf, lane, t);
    pdl_trigger();   // the column kernel may be scheduled now (it waits for this grid's completion)
    // X[k] = (Z_k + conj Z_{N-k})/2 - i/2 W_2048^k (Z_k - conj Z_{N-k}), k = k1 + 32 k2;
    // Z_{N-k} is register 31 - k2 of lane 32 - k1 (lane 0: its own register 32 - k2)
    const int pl = (32 - lane) & 31;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
        float2 s;
        s.x = __shfl_sync(FULL, z[31 - k2].x, pl);
        s.y = __shfl_sync(FULL, z[31 - k2].y, pl);
        float2 zc = lane == 0 ? z[(32 - k2) & 31] : s;
        zc.y = -zc.y;
        const float2 e = cadd(z[k2], zc), o = csub(z[k2], zc);
        float2 mo;
        mo.x = o.y;
        mo.y = -o.x;
        float2 r = cadd(e, cmul(tw2048(t, k2), mo));
        r.x *= 0.5f;
        r.y *= 0.5f;
        tile[(lane + 32 * k2) * TLD + g] = r;
    }
    if (lane == 0) {   // X[N] from Z_N = Z_0, W_2048^N = -1
        tile[WN * TLD + g] = make_float2(z[0].x - z[0].y, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (WH * LINES + 127) / 128; ++q) {
        const int i = threadIdx.x + 128 * q;
        const int k = i >> 2, gg = i & 3;
        if (i < WH * LINES && l0 + gg < nlines) specT[(int64_t)k * ld + l0 + gg] = tile[k * TLD + gg];
    }
}

// ---------------------------------------------------------------------------
// kernel 2: one spectrum column per CTA: even and odd bins, symbol, inverse
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64, 7) col_conv_w_kernel(float2* __restrict__ specT, int ld, int n,
                                                        const float2* __restrict__ tw,
                                                        const float2* __restrict__ twp,
                                                        const float* __restrict__ lamT, int64_t sstride,
                                                        GroupArg ga) {
    if (ga.iv) lamT = ga.iv[blockIdx.y / ga.nbper].lamT32;
    else if (ga.lam32) lamT = ga.lam32;
    __shared__ __align__(16) float2 xb[2][XBUF];
    __shared__ __align__(16) float2 cb[WN];
    __shared__ __align__(16) float lb[WH + 3];
    const int lane = threadIdx.x & 31, par = threadIdx.x >> 5;   // par 0: even bins, 1: odd bins
    const int col = blockIdx.x;
    float2* column = specT + blockIdx.y * sstride + (int64_t)col * ld;
    const LaneTw t = lane_twiddles(twp, tw, lane);
    // the symbol row (set-up data) before the predecessor completes
    const float* lc = lamT + (int64_t)col * WH;
    for (int i = threadIdx.x; i < WH; i += 64) lb[i] = __ldcg(&lc[i]);
    pdl_wait();
    if (column_skipped(ga)) return;
#pragma unroll
    for (int i = 0; i < WN / 64; ++i) {
        const int m = threadIdx.x + 64 * i;
        cb[m] = m < n ? __ldcg(&column[m]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = cb[lane + 32 * r];
    if (par) {
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = cmul(v[r], tw2048(t, r));   // W_2048^m, m = L + 32 r
    }
    // forward transform (lane k1, register k2: bin 2(k1 + 32 k2) + par), the
    // symbol, then the inverse as conj(forward(conj)): one copy of the FFT code
#pragma unroll 1
    for (int ph = 0; ph < 2; ++ph) {
        wfft_fwd(v, xb[par], lane, t);
        if (ph == 1) break;
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
            const int q = 2 * (lane + 32 * k2) + par;
            const float l = lb[q <= WP / 2 ? q : WP - q];
            v[k2].x *= l;
            v[k2].y = -v[k2].y * l;
        }
    }
    conj32(v);   // lane a, register b: the half's row m = a + 32 b
    pdl_trigger();
    if (par) {
#pragma unroll
        for (int b = 0; b < 32; ++b) v[b] = cmulc(v[b], tw2048(t, b));   // W_2048^{-m}
    }
#pragma unroll
    for (int b = 0; b < 32; ++b) xb[par][lane + 32 * b] = v[b];
    __syncthreads();
#pragma unroll
    for (int b = 16 * par; b < 16 * par + 16; ++b) {
        const int m = lane + 32 * b;
        if (m < n) column[m] = cadd(xb[0][m], xb[1][m]);
    }
}

// ---------------------------------------------------------------------------
// kernel 3: transposed tile in, inverse real FFT per line, n samples out
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 3) row_inv_w_kernel(const float2* __restrict__ specT, int ld, int nlines,
                                                           int n, const float2* __restrict__ tw,
                                                           const float2* __restrict__ twp,
                                                           float* __restrict__ wgrid, int64_t sstride,
                                                           int64_t wstride, GroupArg ga) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* tile = reinterpret_cast<float2*>(smem_raw);   // [WH][TLD]
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int l0 = blockIdx.x * LINES, line = l0 + g;
    specT += blockIdx.y * sstride;
    wgrid += blockIdx.y * wstride;
    const LaneTw t = lane_twiddles(twp, tw, lane);
    pdl_wait();
    if (column_skipped(ga)) return;
#pragma unroll
    for (int q = 0; q < (WH * LINES + 127) / 128; ++q) {
        const int i = threadIdx.x + 128 * q;
        const int k = i >> 2, gg = i & 3;
        if (i < WH * LINES)
            tile[k * TLD + gg] = (l0 + gg < nlines) ? __ldcg(&specT[(int64_t)k * ld + l0 + gg]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    // Z'_k = (X_k + conj X_{N-k}) + i W_2048^{-k} (X_k - conj X_{N-k}), k = k1 + 32 k2
    float2 z[32];
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
        const int k = lane + 32 * k2;
        const float2 xk = tile[k * TLD + g];
        float2 xc = tile[(WN - k) * TLD + g];
        xc.y = -xc.y;
        const float2 e = cadd(xk, xc);
        const float2 o = cmulc(csub(xk, xc), tw2048(t, k2));
        z[k2].x = e.x - o.y;
        z[k2].y = e.y + o.x;
    }
    float2* xbuf = tile + WH * TLD + g * XBUF;
    wfft_inv(z, xbuf, lane, t);   // lane a, register b = z[a + 32 b]: samples 2m, 2m + 1
    pdl_trigger();
    if (line >= nlines) return;
    float* wl = wgrid + (int64_t)line * n;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
        const int k = 2 * (lane + 32 * b);
        if (k < n) wl[k] = z[b].x;
        if (k + 1 < n) wl[k + 1] = z[b].y;
    }
}

}  // namespace

bool afd_2d_warp_eligible(const gofd_problem* p) {
    return p->d == 2 && p->P == WP && p->n[0] <= WN && p->wdesc_line.ptr != nullptr && p->tune_rowe == 0 &&
           p->tune_cole == 0 && p->tune_lpc == 0 && p->tune_cols == 0;
}

// Set-up of the warp-FFT path: the line descriptors, the [register][lane]
// table W_1024^{ij}, the kernels' shared-memory limits.
void setup_apply_2d_warp(gofd_problem* p) {
    if (p->d != 2 || p->P != WP || p->n[0] > WN) return;
    int limit = 0;
    GOFD_CUDA_TRY(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    if ((size_t)limit < ROW_SMEM) return;
    std::vector<float2> t(32 * 32);
    for (int i = 0; i < 32; ++i)
        for (int j = 0; j < 32; ++j) {
            const double a = -2.0 * 3.14159265358979323846 * (double)((i * j) % WN) / WN;
            t[i * 32 + j] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    // line descriptors: {runs, first run, k0, len} {0, k0, len, 0} of the first two runs
    const int64_t nl = p->nlines, nr = p->nruns;
    std::vector<int32_t> rptr(nl + 1), rk0(nr), rlen(nr);
    GOFD_CUDA_TRY(cudaMemcpy(rptr.data(), p->line_run_ptr.ptr, 4 * (nl + 1), cudaMemcpyDeviceToHost));
    if (nr) {
        GOFD_CUDA_TRY(cudaMemcpy(rk0.data(), p->run_k0.ptr, 4 * nr, cudaMemcpyDeviceToHost));
        GOFD_CUDA_TRY(cudaMemcpy(rlen.data(), p->run_len.ptr, 4 * nr, cudaMemcpyDeviceToHost));
    }
    std::vector<int4> ldesc(2 * nl);
    for (int64_t l = 0; l < nl; ++l) {
        const int q = rptr[l], k = rptr[l + 1] - q;
        int4 d0 = make_int4(k, q, 0, 0), d1 = make_int4(0, 0, 0, 0);
        if (k > 0) { d0.z = rk0[q]; d0.w = rlen[q]; }
        if (k > 1) { d1.y = rk0[q + 1]; d1.z = rlen[q + 1]; }
        ldesc[2 * l] = d0;
        ldesc[2 * l + 1] = d1;
    }
    p->twp32.alloc(sizeof(float2) * t.size());
    GOFD_CUDA_TRY(cudaMemcpy(p->twp32.ptr, t.data(), sizeof(float2) * t.size(), cudaMemcpyHostToDevice));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_fwd_w_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ROW_SMEM));
    GOFD_CUDA_TRY(cudaFuncSetAttribute(row_inv_w_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ROW_SMEM));
    // the largest shared-memory carveout, so that every CTA of a kernel is
    // resident at once (three row CTAs or seven column CTAs per SM)
    for (const void* k : {(const void*)row_fwd_w_kernel, (const void*)row_inv_w_kernel, (const void*)col_conv_w_kernel,
                          (const void*)gather_w_kernel})
        GOFD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                           (int)cudaSharedmemCarveoutMaxShared));
    // the ELL with its slot stride rounded up to four rows (gather_w_kernel
    // reads four rows with one 16-byte load per array)
    const int64_t nloc = p->nloc, ld4 = (nloc + 3) / 4 * 4;
    p->ell4_node.alloc(sizeof(int32_t) * std::max<int64_t>(ld4, 4));
    p->ell4_iidx.alloc(sizeof(int32_t) * 3 * std::max<int64_t>(ld4, 4));
    p->ell4_w32.alloc(sizeof(float) * 3 * std::max<int64_t>(ld4, 4));
    const cudaStream_t ss = p->setup_stream;   // after the ELL's own set-up kernels
    GOFD_CUDA_TRY(cudaMemsetAsync(p->ell4_node.ptr, 0xff, p->ell4_node.bytes, ss));   // node -1
    GOFD_CUDA_TRY(cudaMemsetAsync(p->ell4_iidx.ptr, 0, p->ell4_iidx.bytes, ss));
    GOFD_CUDA_TRY(cudaMemsetAsync(p->ell4_w32.ptr, 0, p->ell4_w32.bytes, ss));
    if (nloc > 0) {
        GOFD_CUDA_TRY(cudaMemcpyAsync(p->ell4_node.ptr, p->ell_node.ptr, 4 * nloc, cudaMemcpyDeviceToDevice, ss));
        GOFD_CUDA_TRY(cudaMemcpy2DAsync(p->ell4_iidx.ptr, 4 * ld4, p->ell_iidx.ptr, 4 * nloc, 4 * nloc, 3,
                                        cudaMemcpyDeviceToDevice, ss));
        GOFD_CUDA_TRY(cudaMemcpy2DAsync(p->ell4_w32.ptr, 4 * ld4, p->ell_w32.ptr, 4 * nloc, 4 * nloc, 3,
                                        cudaMemcpyDeviceToDevice, ss));
    }
    p->ell4_ld = ld4;
    p->wdesc_line.alloc(sizeof(int4) * 2 * nl);
    GOFD_CUDA_TRY(cudaMemcpy(p->wdesc_line.ptr, ldesc.data(), sizeof(int4) * 2 * nl, cudaMemcpyHostToDevice));
}

// w_b = A_FD I x_b on the grid for nb interior vectors x_b = x + b xs
// (outputs wgrid + b ws), spectra in spec (nb x (P/2+1) x ldT complex) or the
// handle's buffer for nb = 1.  v = I x_b is formed in wgrid + b ws first.
void afd_2d_warp_f32(gofd_problem* p, const float* x, float* wgrid, int nb, int64_t xs, int64_t ws, void* spec,
                     cudaStream_t st, GroupArg ga) {
    float2* S = spec ? static_cast<float2*>(spec) : p->specT.as<float2>();
    const int n = p->n[0], nlines = (int)p->nlines;
    const int64_t ss = (int64_t)WH * p->ldT;
    const int64_t sb = nb > 1 ? ss : 0;
    const float2* tw = p->tw32.as<float2>();
    const float2* twp = p->twp32.as<float2>();
    const unsigned rblocks = (unsigned)((nlines + LINES - 1) / LINES);
    const float* lam = p->lamT32.as<float>();
    const int64_t nloc_max = ga.iv ? ga.max_nloc : p->nloc;
    const unsigned gblocks = (unsigned)std::max<int64_t>(1, (nloc_max + 4 * GTH - 1) / (4 * GTH));
    launch_pdl(gather_w_kernel, dim3(gblocks, nb), dim3(GTH), 0, st, x, p->ell4_iidx.as<int32_t>(),
               p->ell4_w32.as<float>(), p->ell4_node.as<int32_t>(), p->ell4_ld, wgrid, xs, ws, ga);
    mark_stage(st, "gather");
    launch_pdl(row_fwd_w_kernel, dim3(rblocks, nb), dim3(128), ROW_SMEM, st, (const float*)wgrid,
               p->wdesc_line.as<int4>(), p->run_k0.as<int32_t>(), p->run_len.as<int32_t>(), nlines, n, tw, twp,
               (const void*)lam, (int64_t)4 * WH * WH, (const void*)p->csr_col.ptr, (int64_t)4 * p->nnz_t,
               (const void*)p->csr_val32.ptr, (int64_t)4 * p->nnz_t, (const void*)p->csr_ptr.ptr,
               (int64_t)4 * (p->nint + 1), S, p->ldT, ws, sb, ga);
    mark_stage(st, "row_fft");
    launch_pdl(col_conv_w_kernel, dim3(WH, nb), dim3(64), 0, st, S, p->ldT, n, tw, twp, lam, sb, ga);
    mark_stage(st, "col_fft_conv");
    launch_pdl(row_inv_w_kernel, dim3(rblocks, nb), dim3(128), ROW_SMEM, st, (const float2*)S, p->ldT, nlines, n,
               tw, twp, wgrid, sb, ws, ga);
    mark_stage(st, "row_ifft");
}

}  // namespace gofd
