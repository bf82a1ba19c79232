// Adjoint of the solve with vertex data (GoFD-3): u = S(X)^{-1} b(f, X),
// b = h^{2s} D_h(X) f on the interior vertices.  For a loss L(u) with
// g = dL/du, the adjoint state solves the symmetric system S lambda = g, and
//
//   dL/df_i      = h^{2s} D_h,i lambda_i                     (interior i)
//   dL/dX_{j,c}  = sum_k phi_j(x_k) [ d_c(I_h lambda)|_K w_u,k
//                                   + d_c(I_h u)|_K w_lambda,k
//                                   - h^{2s} d_c(I_h(lambda f))|_K ]
//
// with w_u = A_FD I u, w_lambda = A_FD I lambda on the grid, K the owner
// simplex of grid node x_k and d_c the x_c-derivative of the P1 interpolant on
// K.  This follows from dL = lambda^T (db - dS u), S = I^T A_FD I, and the
// derivative of barycentric coordinates with respect to a vertex,
// d phi_a / d X_{j,c} = -phi_j d phi_a / d x_c (the owner map is held fixed).
// No CG iterate is stored: the adjoint state is one more solve.  The vertex
// sums run over a full vertex-major transpose of the ELL in grid order, so
// the gradients are deterministic.
#include <cmath>

#include "gofd_internal.cuh"

namespace gofd {

struct Adjoint {
    DevBuf fptr, fpacked;     // all vertices x (ELL row, slot), rows ascending
    int64_t nnz = 0;
    DevBuf g_int, lam_int, u_int, u_v, lam_v, lamf_v, wu, wl, C;
};

__global__ void full_count_kernel(const int32_t* __restrict__ vidx, int64_t total, int32_t* __restrict__ cnt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[vidx[t]], 1);
}

__global__ void full_fill_kernel(const int32_t* __restrict__ vidx, int64_t nloc, int dp1,
                                 const int32_t* __restrict__ ptr, int32_t* __restrict__ cursor,
                                 int64_t* __restrict__ packed) {
    const int64_t total = nloc * dp1;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = vidx[t];
        const int64_t s = t / nloc, e = t % nloc;
        packed[ptr[v] + atomicAdd(&cursor[v], 1)] = e * 4 + s;
    }
}

__global__ void hadamard_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c,
                                int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c[i] = a[i] * b[i];
}

// per located node (ELL row e): the d components of
// d(I_h lambda) w_u + d(I_h u) w_lambda - h2s d(I_h(lambda f)) on the owner simplex
template <int D>
__global__ void adj_node_kernel(const double* __restrict__ V, const int32_t* __restrict__ S,
                                const int32_t* __restrict__ owner, const int32_t* __restrict__ ell_node, int64_t nloc,
                                const double* __restrict__ u_v, const double* __restrict__ lam_v,
                                const double* __restrict__ lamf_v, const double* __restrict__ wu,
                                const double* __restrict__ wl, double h2s, double* __restrict__ C) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nloc; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = ell_node[e];
        const int32_t K = owner[k];
        double X[D + 1][D];
        int vv[D + 1];
        for (int a = 0; a <= D; ++a) {
            vv[a] = S[(int64_t)K * (D + 1) + a];
            for (int c = 0; c < D; ++c) X[a][c] = V[(int64_t)vv[a] * D + c];
        }
        // J = [X_1 - X_0, ..., X_D - X_0] (columns); grad phi_a = row a-1 of J^{-1}
        double J[D][D], Ji[D][D];
        for (int r = 0; r < D; ++r)
            for (int c = 0; c < D; ++c) J[r][c] = X[c + 1][r] - X[0][r];
        if constexpr (D == 1) {
            Ji[0][0] = 1.0 / J[0][0];
        } else if constexpr (D == 2) {
            const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            Ji[0][0] = J[1][1] / det;
            Ji[0][1] = -J[0][1] / det;
            Ji[1][0] = -J[1][0] / det;
            Ji[1][1] = J[0][0] / det;
        } else {
            const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
            Ji[0][0] = c00 / det;
            Ji[1][0] = c01 / det;
            Ji[2][0] = c02 / det;
            Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
            Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
            Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
            Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
            Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
            Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        }
        double grad[D + 1][D];
        for (int c = 0; c < D; ++c) {
            double s0 = 0.0;
            for (int a = 1; a <= D; ++a) {
                grad[a][c] = Ji[a - 1][c];
                s0 += Ji[a - 1][c];
            }
            grad[0][c] = -s0;
        }
        const double wuk = wu[k], wlk = wl[k];
        for (int c = 0; c < D; ++c) {
            double gl = 0.0, gu = 0.0, glf = 0.0;
            for (int a = 0; a <= D; ++a) {
                gl += lam_v[vv[a]] * grad[a][c];
                gu += u_v[vv[a]] * grad[a][c];
                glf += lamf_v[vv[a]] * grad[a][c];
            }
            C[c * nloc + e] = gl * wuk + gu * wlk - h2s * glf;
        }
    }
}

// grad_X[j][c] = sum over the grid nodes of vertex j (ascending) of phi_j(x_k) C[c][k]
__global__ void adj_gradx_kernel(const int32_t* __restrict__ ptr, const int64_t* __restrict__ packed,
                                 const double* __restrict__ w64, int64_t nloc, int d, int64_t nv,
                                 const double* __restrict__ C, double* __restrict__ gx) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nv; j += (int64_t)gridDim.x * blockDim.x) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int32_t a = ptr[j]; a < ptr[j + 1]; ++a) {
            const int64_t e = packed[a] >> 2, s = packed[a] & 3;
            const double phi = w64[s * nloc + e];
            for (int c = 0; c < d; ++c) acc[c] += phi * C[c * nloc + e];
        }
        for (int c = 0; c < d; ++c) gx[j * d + c] = acc[c];
    }
}

__global__ void adj_gradf_kernel(const int32_t* __restrict__ v2i, const double* __restrict__ colsum,
                                 const double* __restrict__ lam_int, double h2s, int64_t nv, double* __restrict__ gf) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = v2i[v];
        gf[v] = i >= 0 ? h2s * colsum[i] * lam_int[i] : 0.0;
    }
}

static Adjoint* ensure_adjoint(gofd_problem* p, cudaStream_t st) {
    if (p->adj) return p->adj;
    Adjoint* a = new Adjoint();
    p->adj = a;
    const int dp1 = p->d + 1;
    const int64_t total = p->nloc * dp1;
    DevBuf cnt, cur;
    cnt.alloc(4 * (p->nv + 1));
    cur.alloc(4 * (p->nv + 1));
    GOFD_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, 4 * (p->nv + 1), st));
    GOFD_CUDA_TRY(cudaMemsetAsync(cur.ptr, 0, 4 * (p->nv + 1), st));
    if (total > 0)
        full_count_kernel<<<grid_blocks(total, 256), 256, 0, st>>>(p->ell_vidx.as<int32_t>(), total, cnt.as<int32_t>());
    GOFD_CHECK_LAUNCH();
    a->fptr.alloc(4 * (p->nv + 1));
    a->nnz = exclusive_scan_i32(cnt.as<int32_t>(), a->fptr.as<int32_t>(), p->nv + 1, st);
    a->fpacked.alloc(8 * a->nnz);
    if (total > 0)
        full_fill_kernel<<<grid_blocks(total, 256), 256, 0, st>>>(p->ell_vidx.as<int32_t>(), p->nloc, dp1,
                                                                 a->fptr.as<int32_t>(), cur.as<int32_t>(),
                                                                 a->fpacked.as<int64_t>());
    GOFD_CHECK_LAUNCH();
    sort_packed_rows(a->fptr.as<int32_t>(), p->nv, a->fpacked.as<int64_t>(), a->nnz, st);
    const int64_t n1 = p->nint + 1;
    a->g_int.alloc(8 * n1);
    a->lam_int.alloc(8 * n1);
    a->u_int.alloc(8 * n1);
    a->lam_v.alloc(8 * p->nv);
    a->u_v.alloc(8 * p->nv);
    a->lamf_v.alloc(8 * p->nv);
    a->wu.alloc(8 * p->ngrid);
    a->wl.alloc(8 * p->ngrid);
    a->C.alloc(8 * (p->nloc * p->d + 1));
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    return a;
}

void free_adjoint(gofd_problem* p) {
    delete p->adj;
    p->adj = nullptr;
}

void adjoint(gofd_problem* p, gofd_solve_mode mode, const double* f, const double* u, const double* g, double tol,
             int maxit, double* grad_f, double* grad_x, gofd_solve_info* info, cudaStream_t st) {
    Adjoint* a = ensure_adjoint(p, st);
    const double h2s = std::pow(p->h, 2.0 * p->s);
    // adjoint state: S lambda = g on the interior (S is symmetric)
    compact_vertex(p, true, g, a->g_int.ptr, st);
    solve_core(p, mode, a->g_int.as<double>(), tol, maxit, true, a->lam_int.as<double>(), info, st);
    expand_interior(p, true, a->lam_int.ptr, a->lam_v.ptr, 0.0, st);
    compact_vertex(p, true, u, a->u_int.ptr, st);
    expand_interior(p, true, a->u_int.ptr, a->u_v.ptr, 0.0, st);   // u with its Dirichlet zeros
    // grid fields w_u = A_FD I u, w_lambda = A_FD I lambda (FP64)
    afd_of_interior(p, true, a->u_int.ptr, a->wu.ptr, st);
    afd_of_interior(p, true, a->lam_int.ptr, a->wl.ptr, st);
    hadamard_kernel<<<grid_blocks(p->nv, 256), 256, 0, st>>>(a->lam_v.as<double>(), f, a->lamf_v.as<double>(), p->nv);
    GOFD_CHECK_LAUNCH();
    if (p->nloc > 0) {
#define NODE(D)                                                                                                  \
    adj_node_kernel<D><<<grid_blocks(p->nloc, 128), 128, 0, st>>>(                                                 \
        p->verts.as<double>(), p->simp.as<int32_t>(), p->owner.as<int32_t>(), p->ell_node.as<int32_t>(), p->nloc, \
        a->u_v.as<double>(), a->lam_v.as<double>(), a->lamf_v.as<double>(), a->wu.as<double>(),                \
        a->wl.as<double>(), h2s,                                                                                   \
        a->C.as<double>())
        if (p->d == 1) NODE(1);
        else if (p->d == 2) NODE(2);
        else NODE(3);
#undef NODE
        GOFD_CHECK_LAUNCH();
    }
    adj_gradx_kernel<<<grid_blocks(p->nv, 128), 128, 0, st>>>(a->fptr.as<int32_t>(), a->fpacked.as<int64_t>(),
                                                              p->ell_w64.as<double>(), p->nloc, p->d, p->nv,
                                                              a->C.as<double>(), grad_x);
    adj_gradf_kernel<<<grid_blocks(p->nv, 256), 256, 0, st>>>(p->vert2int.as<int32_t>(), p->colsum.as<double>(),
                                                              a->lam_int.as<double>(), h2s, p->nv, grad_f);
    GOFD_CHECK_LAUNCH();
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace gofd
