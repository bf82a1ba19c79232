// FD coefficients T (Section 2.3) and the circulant symbol (Section 2.2), FP64.
//
// T^{(M)}_p = prod_i [(-1)^{p_i} sinc^2(p_i/M) / M] * sum_{j in [0,M)^d} psi~(j/M) prod_i cos(2 pi p_i j_i / M)
// is the Filon-linear quadrature of (T-0): (Tp-1D-2) rewritten with the second
// difference moved onto the exponential, and the tensor product of the 1D
// factors in d dimensions.  psi~ (psi-2) is even about 1/2 in each variable,
// so the sum folds onto j_i in [0, M/2] with weights 1, 2, ..., 2, 1.  Levels
// M, M/2, ... are combined by Richardson extrapolation with the exponents of
// the error expansion (2, 4, ... from the Filon factor; d+2s, d+2s+2, ...
// from the |xi|^{2s} singularity), taken in ascending order.
//
// Every transform is a restricted cosine transform along one axis,
//   out[b][p][i] = scale[p] * sum_j wt[j] cos(2 pi (p j mod L) / L) in[b][j][i],
// evaluated as a tiled FP64 GEMM whose left factor is generated from a table.
// The symbol lambda = DFT_P(c) of the even embedding of T uses the same kernel
// with L = P.
#include <algorithm>
#include <cmath>
#include <set>

#include "gofd_internal.cuh"

namespace gofd {

constexpr int CT_TM = 64, CT_TN = 64, CT_TK = 16, CT_THREADS = 256;

// out[z][m][n] = scale[m] * sum_k wt[k] C[(m k) mod L] in[z][k][n]
__global__ void __launch_bounds__(CT_THREADS)
cos_transform_kernel(const double* __restrict__ in, double* __restrict__ out, int Mout, int K, int N,
                     int64_t in_zstride, int64_t out_zstride, const double* __restrict__ ctab, int L,
                     const double* __restrict__ wt, const double* __restrict__ scale) {
    __shared__ double As[CT_TK][CT_TM + 1];
    __shared__ double Bs[CT_TK][CT_TN];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * CT_TM, n0 = blockIdx.x * CT_TN;
    const double* inz = in + (int64_t)blockIdx.z * in_zstride;
    double* outz = out + (int64_t)blockIdx.z * out_zstride;
    const int tm = (tid / 16) * 4, tn = (tid % 16) * 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += CT_TK) {
        // A tile: cos(2 pi m k / L) * wt[k]
        for (int t = tid; t < CT_TK * CT_TM; t += CT_THREADS) {
            int kk = t / CT_TM, mm = t % CT_TM;
            int m = m0 + mm, k = k0 + kk;
            double v = 0.0;
            if (m < Mout && k < K) {
                int64_t idx = ((int64_t)m * k) % L;
                v = __ldg(&ctab[idx]) * __ldg(&wt[k]);
            }
            As[kk][mm] = v;
        }
        for (int t = tid; t < CT_TK * CT_TN; t += CT_THREADS) {
            int kk = t / CT_TN, nn = t % CT_TN;
            int k = k0 + kk, n = n0 + nn;
            Bs[kk][nn] = (k < K && n < N) ? inz[(int64_t)k * N + n] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < CT_TK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tm + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tn + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + tm + i;
        if (m >= Mout) continue;
        double sc = scale ? scale[m] : 1.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + tn + j;
            if (n < N) outz[(int64_t)m * N + n] = acc[i][j] * sc;
        }
    }
}

// out[c][r] = in[r][c] for an (R x C) row-major matrix
__global__ void transpose_f64_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t R,
                                     int64_t C) {
    __shared__ double tile[32][33];
    int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[i][threadIdx.x] = in[r * C + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) out[c * R + r] = tile[threadIdx.x][i];
    }
}

__global__ void cos_table_kernel(double* __restrict__ t, int L) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x)
        t[m] = cospi(2.0 * (double)m / (double)L);
}

// psi~(j/M) = (sum_i 4 cos^2(pi j_i / M))^s on the folded range [0, M/2]^d
__global__ void psi_samples_kernel(double* __restrict__ out, int d, int J, int M, double s) {
    int64_t total = 1;
    for (int i = 0; i < d; ++i) total *= J;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = t;
        double sum = 0.0;
        for (int i = 0; i < d; ++i) {
            int j = (int)(r % J);
            r /= J;
            double c = cospi((double)j / (double)M);
            sum += 4.0 * c * c;
        }
        out[t] = pow(sum, s);
    }
}

__global__ void axpy_f64_kernel(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

__global__ void symbol_finish_kernel(const double* __restrict__ lam, double* __restrict__ l64,
                                     float* __restrict__ l32, double inv, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = lam[i] * inv;
        l64[i] = v;
        l32[i] = (float)v;
    }
}

// e^{-2 pi i m / P} in FP64, FP32 and double-float (hi, lo of the real part,
// then of the imaginary part)
__global__ void twiddle_kernel(double2* __restrict__ t64, float2* __restrict__ t32, float4* __restrict__ tdf, int P) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P; m += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)m / (double)P, &sn, &cs);
        t64[m] = make_double2(cs, -sn);
        t32[m] = make_float2((float)cs, (float)-sn);
        const float ch = (float)cs, sh = (float)-sn;
        tdf[m] = make_float4(ch, (float)(cs - (double)ch), sh, (float)(-sn - (double)sh));
    }
}

// Apply the restricted cosine transform along every axis of a d-dimensional
// array with all extents J (axis 0 fastest), producing extents Pout.
static void transform_all_axes(const double* src, DevBuf& result, int d, int J, int Pout,
                               const double* ctab, int L, const double* wt, const double* scale,
                               cudaStream_t st) {
    // current array shape: ext[d-1] ... ext[0]; we transform the slowest axis
    // first, then the next, ...; axis 0 is transposed to the slow position.
    int64_t ext[3] = {J, J, J};
    DevBuf a, b;
    const double* cur = src;
    for (int ax = d - 1; ax >= 1; --ax) {
        int64_t Bz = 1, I = 1;
        for (int q = ax + 1; q < d; ++q) Bz *= ext[q];
        for (int q = 0; q < ax; ++q) I *= ext[q];
        DevBuf& dst = (cur == a.as<double>()) ? b : a;
        dst.alloc(sizeof(double) * Bz * Pout * I);
        dim3 grid((unsigned)((I + CT_TN - 1) / CT_TN), (unsigned)((Pout + CT_TM - 1) / CT_TM), (unsigned)Bz);
        cos_transform_kernel<<<grid, CT_THREADS, 0, st>>>(cur, dst.as<double>(), Pout, (int)ext[ax], (int)I,
                                                          ext[ax] * I, (int64_t)Pout * I, ctab, L, wt, scale);
        GOFD_CHECK_LAUNCH();
        ext[ax] = Pout;
        cur = dst.as<double>();
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
        if (&dst == &a) b.release();
        else a.release();
    }
    // axis 0: view as (R x J) with R = product of the other extents; transpose,
    // transform as (1 x J x R), transpose back
    int64_t R = 1;
    for (int q = 1; q < d; ++q) R *= ext[q];
    DevBuf t1, t2;
    t1.alloc(sizeof(double) * R * ext[0]);
    dim3 tb(32, 8);
    transpose_f64_kernel<<<dim3((unsigned)((ext[0] + 31) / 32), (unsigned)((R + 31) / 32)), tb, 0, st>>>(
        cur, t1.as<double>(), R, ext[0]);
    GOFD_CHECK_LAUNCH();
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    a.release();
    b.release();
    t2.alloc(sizeof(double) * R * Pout);
    dim3 grid((unsigned)((R + CT_TN - 1) / CT_TN), (unsigned)((Pout + CT_TM - 1) / CT_TM), 1);
    cos_transform_kernel<<<grid, CT_THREADS, 0, st>>>(t1.as<double>(), t2.as<double>(), Pout, (int)ext[0],
                                                      (int)R, 0, 0, ctab, L, wt, scale);
    GOFD_CHECK_LAUNCH();
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    t1.release();
    result.alloc(sizeof(double) * R * Pout);
    transpose_f64_kernel<<<dim3((unsigned)((R + 31) / 32), (unsigned)((Pout + 31) / 32)), tb, 0, st>>>(
        t2.as<double>(), result.as<double>(), Pout, R);
    GOFD_CHECK_LAUNCH();
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
}

// Exponents eliminated by the Richardson tableau (ascending, distinct).
static std::vector<double> richardson_exponents(int d, double s, int levels) {
    std::set<long long> seen;
    std::vector<double> c;
    for (int m = 1; m <= levels; ++m) {
        double e1 = 2.0 * m, e2 = d + 2.0 * s + 2.0 * (m - 1);
        for (double e : {e1, e2}) {
            long long key = llround(e * 1e12);
            if (!seen.count(key)) {
                seen.insert(key);
                c.push_back(e);
            }
        }
    }
    std::sort(c.begin(), c.end());
    c.resize(levels - 1);
    return c;
}

// Weights c_l of T = sum_l c_l T^{(M/2^l)} produced by the Richardson tableau
// R_{l,k} = (2^{e_k} R_{l,k-1} - R_{l+1,k-1}) / (2^{e_k} - 1).
static std::vector<double> richardson_weights(int d, double s, int levels) {
    std::vector<std::vector<double>> R(levels, std::vector<double>(levels, 0.0));
    for (int l = 0; l < levels; ++l) R[l][l] = 1.0;
    for (double e : richardson_exponents(d, s, levels)) {
        double r = std::pow(2.0, e);
        std::vector<std::vector<double>> Rn;
        for (size_t l = 0; l + 1 < R.size(); ++l) {
            std::vector<double> v(levels);
            for (int q = 0; q < levels; ++q) v[q] = (r * R[l][q] - R[l + 1][q]) / (r - 1.0);
            Rn.push_back(v);
        }
        R = Rn;
    }
    return R[0];
}

void setup_coefficients(gofd_problem* p) {
    cudaStream_t st = p->setup_stream;
    const int d = p->d, n = p->n[0], levels = p->rich_levels;
    const int64_t nd = p->ngrid;
    p->T.alloc(sizeof(double) * nd);
    GOFD_CUDA_TRY(cudaMemsetAsync(p->T.ptr, 0, sizeof(double) * nd, st));
    std::vector<double> cw = richardson_weights(d, p->s, levels);
    for (int l = 0; l < levels; ++l) {
        const int M = (int)(p->filon_M >> l);
        const int J = M / 2 + 1;
        DevBuf ctab, wt, scale, samples, Tl;
        ctab.alloc(sizeof(double) * M);
        wt.alloc(sizeof(double) * J);
        scale.alloc(sizeof(double) * n);
        cos_table_kernel<<<grid_blocks(M, 256), 256, 0, st>>>(ctab.as<double>(), M);
        std::vector<double> hw(J, 2.0), hs(n);
        hw[0] = 1.0;
        hw[J - 1] = 1.0;
        for (int q = 0; q < n; ++q) {
            double x = (double)q / M;
            double sc = (q == 0) ? 1.0 : std::sin(M_PI * x) / (M_PI * x);
            hs[q] = ((q & 1) ? -1.0 : 1.0) * sc * sc / (double)M;
        }
        GOFD_CUDA_TRY(cudaMemcpyAsync(wt.ptr, hw.data(), sizeof(double) * J, cudaMemcpyHostToDevice, st));
        GOFD_CUDA_TRY(cudaMemcpyAsync(scale.ptr, hs.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
        int64_t tot = 1;
        for (int i = 0; i < d; ++i) tot *= J;
        samples.alloc(sizeof(double) * tot);
        psi_samples_kernel<<<grid_blocks(tot, 256), 256, 0, st>>>(samples.as<double>(), d, J, M, p->s);
        GOFD_CHECK_LAUNCH();
        transform_all_axes(samples.as<double>(), Tl, d, J, n, ctab.as<double>(), M, wt.as<double>(),
                           scale.as<double>(), st);
        samples.release();
        axpy_f64_kernel<<<grid_blocks(nd, 256), 256, 0, st>>>(cw[l], Tl.as<double>(), p->T.as<double>(), nd);
        GOFD_CHECK_LAUNCH();
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    }

    // symbol: lambda_k = sum over the P circulant slots of c_m cos(2 pi k m / P),
    // slot m (and P-m) holding T_m for m < n
    const int P = p->P, H = P / 2 + 1;
    DevBuf ctab, wt, lam;
    ctab.alloc(sizeof(double) * P);
    wt.alloc(sizeof(double) * n);
    cos_table_kernel<<<grid_blocks(P, 256), 256, 0, st>>>(ctab.as<double>(), P);
    std::vector<double> hw(n, 2.0);
    hw[0] = 1.0;
    if (n - 1 == P / 2) hw[n - 1] = 1.0;
    GOFD_CUDA_TRY(cudaMemcpyAsync(wt.ptr, hw.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    transform_all_axes(p->T.as<double>(), lam, d, n, H, ctab.as<double>(), P, wt.as<double>(), nullptr, st);
    int64_t nh = 1;
    for (int i = 0; i < d; ++i) nh *= H;
    p->lam64.alloc(sizeof(double) * nh);
    p->lam32.alloc(sizeof(float) * nh);
    double inv = 1.0;
    for (int i = 0; i < d; ++i) inv /= (double)P;
    symbol_finish_kernel<<<grid_blocks(nh, 256), 256, 0, st>>>(lam.as<double>(), p->lam64.as<double>(),
                                                               p->lam32.as<float>(), inv, nh);
    GOFD_CHECK_LAUNCH();
    p->tw64.alloc(sizeof(double2) * P);
    p->tw32.alloc(sizeof(float2) * P);
    p->twdf.alloc(sizeof(float4) * P);
    twiddle_kernel<<<grid_blocks(P, 256), 256, 0, st>>>(p->tw64.as<double2>(), p->tw32.as<float2>(),
                                                        p->twdf.as<float4>(), P);
    GOFD_CHECK_LAUNCH();
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace gofd
