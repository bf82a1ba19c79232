// Set-up of the transposed-spectrum 2D product: the transposed scaled symbol,
// the transposed spectrum buffer and the kernels' shared-memory limits.
#include <algorithm>

#include "gofd_internal.cuh"

namespace gofd {

void afd_2d_attrs_f32(int limit, int P, size_t* need);
void afd_2d_attrs_f64(int limit, int P, size_t* need);
void afd_3d_attrs_f32(int limit, int P, size_t* need);
void afd_3d_attrs_f64(int limit, int P, size_t* need);

__global__ void transpose_sym_kernel(const double* __restrict__ l64, double* __restrict__ t64,
                                     float* __restrict__ t32, int H) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)H * H;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / H, c = i % H;   // t[r][c] = l[c][r]
        const double v = l64[c * H + r];
        t64[i] = v;
        t32[i] = (float)v;
    }
}

// 3D: t[(a H + b) H + c] = l[(c H + b) H + a] (axis order reversed, so the
// symbol row of (k_x0, k_x1) is contiguous along k_x2)
__global__ void reverse_sym3_kernel(const double* __restrict__ l64, double* __restrict__ t64,
                                    float* __restrict__ t32, int H) {
    const int64_t HH = (int64_t)H * H;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < HH * H;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = i / HH, b = (i / H) % H, c = i % H;
        const double v = l64[(c * H + b) * H + a];
        t64[i] = v;
        t32[i] = (float)v;
    }
}

// 3D set-up: spectrum spec_T (H x round16(n^2) complex), middle buffer
// M (midK x P x n complex), reversed symbol, shared-memory limits
void setup_apply_3d(gofd_problem* p) {
    const int H = p->P / 2 + 1, n = p->n[0];
    p->ldT = (int)(((int64_t)n * n + 15) / 16 * 16);
    p->specT.alloc(sizeof(double2) * (size_t)H * p->ldT);
    // middle buffer for a chunk of planes, at most 1 GiB (FP64 size).  Chunks
    // small enough for L2 (64 MB) were measured slower at 256^3 (9 chunks: 649
    // against 602 us for the middle stage; the extra launches and their tails
    // cost more than the HBM traffic saved), so the chunks only bound memory.
    const size_t plane = sizeof(double2) * (size_t)p->P * n;
    p->midK = (int)std::max<size_t>(1, std::min<size_t>((size_t)H, ((size_t)1 << 30) / plane));
    if (p->opt.chunk_planes > 0) p->midK = std::min(p->opt.chunk_planes, H);
    p->specM.alloc(plane * p->midK);
    const size_t h3 = (size_t)H * H * H;
    p->lamT64.alloc(sizeof(double) * h3);
    p->lamT32.alloc(sizeof(float) * h3);
    reverse_sym3_kernel<<<grid_blocks((int64_t)h3, 256), 256, 0, p->setup_stream>>>(
        p->lam64.as<double>(), p->lamT64.as<double>(), p->lamT32.as<float>(), H);
    GOFD_CHECK_LAUNCH();
    int limit = 0;
    GOFD_CUDA_TRY(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    size_t n32 = 0, n64 = 0, ndf = 0;
    afd_3d_attrs_f32(limit, p->P, &n32);
    afd_3d_attrs_f64(limit, p->P, &n64);
    afd_3d_attrs_df(limit, p->P, &ndf);
    if (std::max({n32, n64, ndf}) > (size_t)limit) fail(GOFD_E_GRID, "FFT line does not fit in shared memory");
}

void setup_apply_2d(gofd_problem* p) {
    const int H = p->P / 2 + 1;
    p->ldT = (p->n[0] + 15) / 16 * 16;
    p->specT.alloc(sizeof(double2) * (size_t)H * p->ldT);
    p->lamT64.alloc(sizeof(double) * (size_t)H * H);
    p->lamT32.alloc(sizeof(float) * (size_t)H * H);
    transpose_sym_kernel<<<grid_blocks((int64_t)H * H, 256), 256, 0, p->setup_stream>>>(
        p->lam64.as<double>(), p->lamT64.as<double>(), p->lamT32.as<float>(), H);
    GOFD_CHECK_LAUNCH();
    int limit = 0;
    GOFD_CUDA_TRY(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    size_t n32 = 0, n64 = 0, ndf = 0;
    afd_2d_attrs_f32(limit, p->P, &n32);
    afd_2d_attrs_f64(limit, p->P, &n64);
    afd_2d_attrs_df(limit, p->P, &ndf);
    if (std::max({n32, n64, ndf}) > (size_t)limit) fail(GOFD_E_GRID, "FFT line does not fit in shared memory");
    setup_apply_2d_warp(p);
}

}  // namespace gofd
