// Diagonal (Jacobi) preconditioner of the stiffness matrix S = I^T A_FD I.
//
// The paper's Section 3.3 preconditions with incomplete factors of sparse
// stencil matrices; on graded meshes the diagonal of S itself varies by two
// orders of magnitude (it scales with the support of each hat function), and
// scaling by it is an elementwise operation.  Not in the paper.
//
//   S_jj = sum_{a, b in row j of I^T} w_a w_b T(|k_a - k_b|)
//
// with T(p) the FD coefficient at the per-axis distances of grid nodes k_a,
// k_b.  Row j is split into blocks of 256 "a" entries; each thread sums over
// all b of its row (FP32 products, FP64 sums of 64-term FP32 partial sums),
// blocks reduce in a fixed order and the partials of a row are added in block
// order, so the diagonal is reproducible run to run.
#include <algorithm>
#include <vector>

#include "gofd_internal.cuh"

namespace gofd {

constexpr int JAC_THREADS = 256;

__global__ void t_to_f32_kernel(const double* __restrict__ T, float* __restrict__ T32, int64_t nd) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd; i += (int64_t)gridDim.x * blockDim.x)
        T32[i] = (float)T[i];
}

__device__ __forceinline__ void grid_coords(int k, int n, int d, int& x, int& y, int& z) {
    x = k % n;
    y = d > 1 ? (k / n) % n : 0;
    z = d > 2 ? k / (n * n) : 0;
}

__global__ void __launch_bounds__(JAC_THREADS) jacobi_pairs_kernel(
    const int32_t* __restrict__ ptr, const int32_t* __restrict__ col, const float* __restrict__ val,
    const float* __restrict__ T32, int d, int n, const int32_t* __restrict__ blk_row,
    const int32_t* __restrict__ blk_a0, double* __restrict__ partial) {
    __shared__ double sh[JAC_THREADS / 32];
    const int j = blk_row[blockIdx.x];
    const int b0 = ptr[j], L = ptr[j + 1] - b0;
    const int a = blk_a0[blockIdx.x] + threadIdx.x;
    double acc = 0;
    if (a < L) {
        int xa, ya, za;
        grid_coords(col[b0 + a], n, d, xa, ya, za);
        const float wa = val[b0 + a];
        float part = 0;
        int cnt = 0;
        for (int t = 0; t < L; ++t) {
            int xb, yb, zb;
            grid_coords(__ldg(&col[b0 + t]), n, d, xb, yb, zb);
            const int64_t idx = ((int64_t)abs(zb - za) * n + abs(yb - ya)) * n + abs(xb - xa);
            part += __ldg(&val[b0 + t]) * __ldg(&T32[idx]);
            if (++cnt == 64) {
                acc += (double)part;
                part = 0;
                cnt = 0;
            }
        }
        acc = (acc + (double)part) * (double)wa;
    }
    // fixed-order block reduction
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < JAC_THREADS / 32; ++w) s += sh[w];
        partial[blockIdx.x] = s;
    }
}

// diag_j = sum of row j's block partials in block order; dinv = 1 / diag
__global__ void jacobi_finish_kernel(const int32_t* __restrict__ row_blk, const double* __restrict__ partial,
                                     int64_t n, double* __restrict__ diag, double* __restrict__ dinv64,
                                     float* __restrict__ dinv32) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double s = 0;
        for (int b = row_blk[j]; b < row_blk[j + 1]; ++b) s += partial[b];
        diag[j] = s;
        dinv64[j] = 1.0 / s;
        dinv32[j] = (float)(1.0 / s);
    }
}

template <class V>
__global__ void jacobi_apply_kernel(const V* __restrict__ r, V* __restrict__ z, const V* __restrict__ dinv,
                                    int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = r[i] * dinv[i];
}

void setup_jacobi(gofd_problem* p, DevBuf& diag, DevBuf& dinv64, DevBuf& dinv32) {
    cudaStream_t st = p->setup_stream;
    const int64_t n = p->nint;
    // blocks per row: ceil(L_j / 256), laid out row after row
    std::vector<int32_t> hptr(n + 1), row_blk(n + 1, 0), blk_row, blk_a0;
    GOFD_CUDA_TRY(cudaMemcpy(hptr.data(), p->csr_ptr.ptr, 4 * (n + 1), cudaMemcpyDeviceToHost));
    for (int64_t j = 0; j < n; ++j) {
        const int L = hptr[j + 1] - hptr[j];
        row_blk[j] = (int32_t)blk_row.size();
        for (int a0 = 0; a0 < L; a0 += JAC_THREADS) {
            blk_row.push_back((int32_t)j);
            blk_a0.push_back(a0);
        }
    }
    row_blk[n] = (int32_t)blk_row.size();
    const int64_t nblk = (int64_t)blk_row.size();
    DevBuf d_blk_row, d_blk_a0, d_row_blk, partial, T32;
    d_blk_row.alloc(4 * (nblk + 1));
    d_blk_a0.alloc(4 * (nblk + 1));
    d_row_blk.alloc(4 * (n + 1));
    partial.alloc(8 * (nblk + 1));
    T32.alloc(4 * p->ngrid);
    if (nblk > 0) {
        GOFD_CUDA_TRY(cudaMemcpyAsync(d_blk_row.ptr, blk_row.data(), 4 * nblk, cudaMemcpyHostToDevice, st));
        GOFD_CUDA_TRY(cudaMemcpyAsync(d_blk_a0.ptr, blk_a0.data(), 4 * nblk, cudaMemcpyHostToDevice, st));
    }
    GOFD_CUDA_TRY(cudaMemcpyAsync(d_row_blk.ptr, row_blk.data(), 4 * (n + 1), cudaMemcpyHostToDevice, st));
    t_to_f32_kernel<<<grid_blocks(p->ngrid, 256), 256, 0, st>>>(p->T.as<double>(), T32.as<float>(), p->ngrid);
    if (nblk > 0)
        jacobi_pairs_kernel<<<(unsigned)nblk, JAC_THREADS, 0, st>>>(
            p->csr_ptr.as<int32_t>(), p->csr_col.as<int32_t>(), p->csr_val32.as<float>(), T32.as<float>(), p->d,
            p->n[0], d_blk_row.as<int32_t>(), d_blk_a0.as<int32_t>(), partial.as<double>());
    diag.alloc(8 * (n + 1));
    dinv64.alloc(8 * (n + 1));
    dinv32.alloc(4 * (n + 1));
    jacobi_finish_kernel<<<grid_blocks(n, 256), 256, 0, st>>>(d_row_blk.as<int32_t>(), partial.as<double>(), n,
                                                              diag.as<double>(), dinv64.as<double>(),
                                                              dinv32.as<float>());
    GOFD_CHECK_LAUNCH();
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
}

void jacobi_apply(const gofd_problem* p, bool fp64, const void* dinv, const void* r, void* z, cudaStream_t st) {
    const int64_t n = p->nint;
    if (fp64)
        jacobi_apply_kernel<double><<<grid_blocks(n, 256), 256, 0, st>>>((const double*)r, (double*)z,
                                                                         (const double*)dinv, n);
    else
        jacobi_apply_kernel<float><<<grid_blocks(n, 256), 256, 0, st>>>((const float*)r, (float*)z,
                                                                        (const float*)dinv, n);
    GOFD_CHECK_LAUNCH();
}

}  // namespace gofd
