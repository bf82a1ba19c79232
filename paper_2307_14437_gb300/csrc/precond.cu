// Sparse preconditioner of Section 3.3: incomplete Cholesky with level-1 fill
// of A_h^(k) = (I_h^FD)^T A_FD^(k) I_h^FD on the interior vertices ((Ah-4)),
// where A_FD^(k) keeps the entries T_delta of A_FD on a stencil: 5 or 9 points
// in 2D, 7 or 27 in 3D, 3 in 1D.
//
//   assembly   one thread per row; contributions w_ik T_delta w_lb summed into a
//              per-thread hash table in a fixed loop order (deterministic); the
//              pattern is structural: an entry exists iff some product of
//              nonzero factors reaches it, whatever the sum
//   ordering   natural vertex order, or a multicolour order (Jones-Plassmann
//              with hashed priorities on the graph of A_h^(k)) that shortens
//              the dependency chains of the triangular factor
//   symbolic   level-of-fill 1: row i keeps A_ij (j <= i) and j < i reached
//              through one pivot k < j with A_ik and A_kj nonzero
//   levels     longest dependency chain of each row, by relaxation sweeps
//   numeric    L_ij = (A_ij - sum_k L_ik L_jk) / L_jj, L_ii = sqrt(A_ii (1+sigma)
//              - sum_k L_ik^2), one launch per level; on a non-positive pivot
//              the factorisation restarts with sigma = 1e-3, 2e-3, 4e-3, ...
//   apply      z = L^{-T} L^{-1} r by level-scheduled forward and backward solves
#include <algorithm>
#include <cmath>
#include <vector>

#include "gofd_internal.cuh"

namespace gofd {

struct Precond {
    int pattern = 0;
    int ordering = 0;
    double shift = 0;
    int64_t n = 0;               // unknowns (interior vertices)
    int64_t nnz_a = 0, nnz = 0;  // entries of A_h^(k) and of L
    int nlevels = 0;
    DevBuf perm, iperm;          // new -> old, old -> new (ordering 1)
    DevBuf lptr, lcol, lval64, lval32;   // L, CSR, columns ascending (diagonal last)
    DevBuf uptr, ucol, uval64, uval32;   // U = L^T, CSR, columns ascending (diagonal first)
    DevBuf level_ptr, level_rows;        // rows grouped by level
    std::vector<int> hlevel_ptr;         // host copy
    int solve = 0;                       // 0: one persistent launch per triangular solve, 1: one per level
    DevBuf tile_pos;                     // persistent solves: tiles of at most 8 rows of one level
    int32_t ntiles = 0;                  //   (start positions in level_rows, ntiles + 1 entries)
    DevBuf ctl;                          //   TriCtl: claim counters and the sticky wait status
    int solve_blocks[4] = {0, 0, 0, 0};  //   resident CTAs of the four solve kernels (FP32/FP64 x fwd/bwd)
    unsigned long long budget = 0;       //   bound on one wait, clock64 cycles
    DevBuf tmp64a, tmp64b, tmp32a, tmp32b;   // apply work vectors
    DevBuf diag, dinv64, dinv32;         // pattern 1 (diagonal of S): the diagonal and its inverse;
                                         // pattern 2: 1 / D_h
    DevBuf lami64, lami32;               // pattern 2: the circulant's inverse symbol, lamT layout
};

// pattern 2: 1/lambda in the column kernels' symbol layout (lamT holds
// lambda / P^d; the inverse convolution needs (1/lambda) / P^d), and 1/D_h
__global__ void circulant_inverse_symbol_kernel(const double* __restrict__ lamT, double* __restrict__ i64,
                                                float* __restrict__ i32, double p2d, int64_t m) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = 1.0 / (lamT[i] * p2d);
        i64[i] = v;
        i32[i] = (float)v;
    }
}
__global__ void inverse_colsum_kernel(const double* __restrict__ colsum, double* __restrict__ i64,
                                      float* __restrict__ i32, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = 1.0 / colsum[i];
        i64[i] = v;
        i32[i] = (float)v;
    }
}

void setup_jacobi(gofd_problem* p, DevBuf& diag, DevBuf& dinv64, DevBuf& dinv32);
void jacobi_apply(const gofd_problem* p, bool fp64, const void* dinv, const void* r, void* z, cudaStream_t st);

// ---------------------------------------------------------------------------
// per-thread open-addressing accumulator (keys = column, values = sum)
// ---------------------------------------------------------------------------
template <int CAP>
struct RowAcc {
    int key[CAP];
    double val[CAP];
    int count;
    __device__ void clear() {
        for (int i = 0; i < CAP; ++i) key[i] = -1;
        count = 0;
    }
    // returns false on overflow
    __device__ bool add(int j, double v) {
        unsigned h = ((unsigned)j * 2654435761u) & (CAP - 1);
        for (int probe = 0; probe < CAP; ++probe) {
            const int k = key[h];
            if (k == j) {
                val[h] += v;
                return true;
            }
            if (k < 0) {
                key[h] = j;
                val[h] = v;
                ++count;
                return count < CAP / 2 + CAP / 4;
            }
            h = (h + 1) & (CAP - 1);
        }
        return false;
    }
};

struct StencilDesc {
    int d, n[3];
    int count;
    int off[27][3];
    double T[27];
};

// contributions of row i of A_h^(k) (old numbering), in a fixed order
template <int CAP>
__device__ bool assemble_row(int64_t i, RowAcc<CAP>& acc, const StencilDesc& sd, const int32_t* __restrict__ csr_ptr,
                             const int32_t* __restrict__ csr_col, const double* __restrict__ csr_val,
                             const int32_t* __restrict__ node_row, const int32_t* __restrict__ iidx,
                             const double* __restrict__ w64, int64_t nloc, int32_t nint) {
    for (int a = csr_ptr[i]; a < csr_ptr[i + 1]; ++a) {
        const int k = csr_col[a];
        const double wik = csr_val[a];
        int kc[3] = {k % sd.n[0], (k / sd.n[0]) % sd.n[1], k / (sd.n[0] * sd.n[1])};
        for (int q = 0; q < sd.count; ++q) {
            int lc[3];
            bool in = true;
            for (int c = 0; c < 3; ++c) {
                lc[c] = kc[c] + sd.off[q][c];
                in &= lc[c] >= 0 && lc[c] < sd.n[c];
            }
            if (!in) continue;
            const int l = lc[0] + sd.n[0] * (lc[1] + sd.n[1] * lc[2]);
            const int e = node_row[l];
            if (e < 0) continue;
            const double base = wik * sd.T[q];
            if (base == 0.0) continue;
            for (int s = 0; s <= sd.d; ++s) {
                const int j = iidx[s * nloc + e];
                const double c = base * w64[s * nloc + e];
                if (j >= nint || c == 0.0) continue;   // a zero factor contributes nothing
                if (!acc.add(j, c)) return false;
            }
        }
    }
    return true;
}

__device__ __forceinline__ void sort_pairs(int* k, double* v, int m) {
    for (int a = 1; a < m; ++a) {
        const int kk = k[a];
        const double vv = v[a];
        int b = a - 1;
        while (b >= 0 && k[b] > kk) {
            k[b + 1] = k[b];
            v[b + 1] = v[b];
            --b;
        }
        k[b + 1] = kk;
        v[b + 1] = vv;
    }
}

// pass 0: count; pass 1: write sorted row
template <int CAP>
__global__ void __launch_bounds__(64) assemble_kernel(int pass, StencilDesc sd, const int32_t* __restrict__ csr_ptr,
                                                      const int32_t* __restrict__ csr_col,
                                                      const double* __restrict__ csr_val,
                                                      const int32_t* __restrict__ node_row,
                                                      const int32_t* __restrict__ iidx, const double* __restrict__ w64,
                                                      int64_t nloc, int32_t nint, int32_t* __restrict__ cnt,
                                                      const int32_t* __restrict__ aptr, int32_t* __restrict__ acol,
                                                      double* __restrict__ aval, int* __restrict__ err) {
    RowAcc<CAP> acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nint; i += (int64_t)gridDim.x * blockDim.x) {
        acc.clear();
        if (!assemble_row<CAP>(i, acc, sd, csr_ptr, csr_col, csr_val, node_row, iidx, w64, nloc, nint)) {
            atomicOr(err, 1);
            continue;
        }
        if (pass == 0) {
            cnt[i] = acc.count;
            continue;
        }
        int m = 0;
        int* ok = acol + aptr[i];
        double* ov = aval + aptr[i];
        for (int h = 0; h < CAP; ++h)
            if (acc.key[h] >= 0) {
                ok[m] = acc.key[h];
                ov[m] = acc.val[h];
                ++m;
            }
        sort_pairs(ok, ov, m);
    }
}

// ---------------------------------------------------------------------------
// multicolour ordering (Jones-Plassmann, hashed priorities)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t prio(uint32_t i) {
    uint32_t x = i * 0x9E3779B1u;
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    return x;
}

__global__ void color_round_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col, int32_t n,
                                   int32_t* __restrict__ color, int c, int* __restrict__ remaining) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (color[i] >= 0) continue;
        const uint64_t pi = ((uint64_t)prio((uint32_t)i) << 32) | (uint32_t)i;
        bool best = true;
        for (int a = ptr[i]; a < ptr[i + 1]; ++a) {
            const int j = col[a];
            if (j == i) continue;
            const int cj = color[j];
            if (cj >= 0 && cj < c) continue;   // coloured in an earlier round
            const uint64_t pj = ((uint64_t)prio((uint32_t)j) << 32) | (uint32_t)j;
            if (pj > pi) {
                best = false;
                break;
            }
        }
        // colour c goes to local maxima among the vertices still uncoloured
        // before this colouring pass (colours of this pass are written to a
        // shadow value c + (1 << 20) and committed by the next kernel)
        if (best) color[i] = c + (1 << 20);
        else atomicAdd(remaining, 1);
    }
}

__global__ void color_commit_kernel(int32_t* __restrict__ color, int32_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (color[i] >= (1 << 20)) color[i] -= (1 << 20);
}

// perm[new] = old ordered by (colour, old index): counting per colour, then a
// stable fill by one thread per colour
__global__ void color_perm_kernel(const int32_t* __restrict__ color, int32_t n, int ncolors,
                                  const int32_t* __restrict__ cstart, int32_t* __restrict__ perm,
                                  int32_t* __restrict__ iperm) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncolors; c += gridDim.x * blockDim.x) {
        int at = cstart[c];
        for (int32_t i = 0; i < n; ++i)
            if (color[i] == c) {
                perm[at] = i;
                iperm[i] = at;
                ++at;
            }
    }
}

__global__ void color_count_kernel(const int32_t* __restrict__ color, int32_t n, int32_t* __restrict__ cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[color[i]], 1);
}

// B = P A P^T: row r of B is row perm[r] of A with columns mapped and sorted
__global__ void permute_count_kernel(const int32_t* __restrict__ aptr, const int32_t* __restrict__ perm, int32_t n,
                                     int32_t* __restrict__ cnt) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int i = perm[r];
        cnt[r] = aptr[i + 1] - aptr[i];
    }
}

__global__ void permute_fill_kernel(const int32_t* __restrict__ aptr, const int32_t* __restrict__ acol,
                                    const double* __restrict__ aval, const int32_t* __restrict__ perm,
                                    const int32_t* __restrict__ iperm, int32_t n, const int32_t* __restrict__ bptr,
                                    int32_t* __restrict__ bcol, double* __restrict__ bval) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int i = perm[r];
        int m = 0;
        for (int a = aptr[i]; a < aptr[i + 1]; ++a, ++m) {
            bcol[bptr[r] + m] = iperm[acol[a]];
            bval[bptr[r] + m] = aval[a];
        }
        sort_pairs(bcol + bptr[r], bval + bptr[r], m);
    }
}

// ---------------------------------------------------------------------------
// symbolic IC(1): lower pattern of row i (columns ascending, diagonal last)
// ---------------------------------------------------------------------------
template <int CAP>
__global__ void __launch_bounds__(64) ic_symbolic_kernel(int pass, const int32_t* __restrict__ aptr,
                                                         const int32_t* __restrict__ acol, int32_t n,
                                                         int32_t* __restrict__ cnt, const int32_t* __restrict__ lptr,
                                                         int32_t* __restrict__ lcol, int* __restrict__ err) {
    int keys[CAP];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int h = 0; h < CAP; ++h) keys[h] = -1;
        int count = 0;
        bool overflow = false;
        auto add = [&](int j) {
            unsigned h = ((unsigned)j * 2654435761u) & (CAP - 1);
            for (int probe = 0; probe < CAP; ++probe) {
                if (keys[h] == j) return;
                if (keys[h] < 0) {
                    keys[h] = j;
                    if (++count >= CAP / 2 + CAP / 4) overflow = true;
                    return;
                }
                h = (h + 1) & (CAP - 1);
            }
            overflow = true;
        };
        for (int a = aptr[i]; a < aptr[i + 1]; ++a) {
            const int k = acol[a];
            if (k > i) break;
            add(k);                                   // level 0
            if (k == i) break;
            for (int b = aptr[k]; b < aptr[k + 1]; ++b) {   // level 1 through pivot k < j < i
                const int j = acol[b];
                if (j <= k) continue;
                if (j >= i) break;
                add(j);
            }
        }
        if (overflow) {
            atomicOr(err, 2);
            continue;
        }
        if (pass == 0) {
            cnt[i] = count;
            continue;
        }
        int m = 0;
        int* out = lcol + lptr[i];
        for (int h = 0; h < CAP; ++h)
            if (keys[h] >= 0) out[m++] = keys[h];
        for (int a = 1; a < m; ++a) {   // ascending; the diagonal i is the largest
            const int kk = out[a];
            int b = a - 1;
            while (b >= 0 && out[b] > kk) {
                out[b + 1] = out[b];
                --b;
            }
            out[b + 1] = kk;
        }
    }
}

// ---------------------------------------------------------------------------
// levels by relaxation: lev[i] = 1 + max_{j in L row i, j < i} lev[j]
// ---------------------------------------------------------------------------
__global__ void level_sweep_kernel(const int32_t* __restrict__ lptr, const int32_t* __restrict__ lcol, int32_t n,
                                   int32_t* __restrict__ lev, int* __restrict__ changed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int m = 0;
        for (int a = lptr[i]; a < lptr[i + 1] - 1; ++a) m = max(m, lev[lcol[a]] + 1);
        if (m != lev[i]) {
            lev[i] = m;
            *changed = 1;
        }
    }
}

__global__ void level_count_kernel(const int32_t* __restrict__ lev, int32_t n, int32_t* __restrict__ cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[lev[i]], 1);
}

__global__ void level_fill_kernel(const int32_t* __restrict__ lev, int32_t n, const int32_t* __restrict__ lstart,
                                  int32_t* __restrict__ cursor, int32_t* __restrict__ rows) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        rows[lstart[lev[i]] + atomicAdd(&cursor[lev[i]], 1)] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// numeric factorisation of the rows of one level
// ---------------------------------------------------------------------------
__global__ void ic_numeric_level_kernel(const int32_t* __restrict__ rows, int32_t nrows,
                                        const int32_t* __restrict__ aptr, const int32_t* __restrict__ acol,
                                        const double* __restrict__ aval, const int32_t* __restrict__ lptr,
                                        const int32_t* __restrict__ lcol, double* __restrict__ lval, double shift,
                                        int* __restrict__ err) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nrows; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = rows[t];
        const int b = lptr[i], e = lptr[i + 1];   // columns ascending, last is i
        int ap = aptr[i];
        const int ae = aptr[i + 1];
        double diag = 0.0;
        for (int a = b; a < e; ++a) {
            const int j = lcol[a];
            // A_ij (0 where the pattern has fill)
            while (ap < ae && acol[ap] < j) ++ap;
            const double aij = (ap < ae && acol[ap] == j) ? aval[ap] : 0.0;
            if (j == i) {
                double s = aij * (1.0 + shift);
                for (int c = b; c < a; ++c) s -= lval[c] * lval[c];
                if (!(s > 0.0)) {
                    atomicOr(err, 4);
                    lval[a] = 1.0;
                } else {
                    lval[a] = sqrt(s);
                }
                diag = lval[a];
                continue;
            }
            // sum over k < j in both row i and row j (two-pointer merge)
            double s = aij;
            int p = b, q = lptr[j];
            const int qe = lptr[j + 1] - 1;   // row j without its diagonal
            while (p < a && q < qe) {
                const int cp = lcol[p], cq = lcol[q];
                if (cp == cq) {
                    s -= lval[p] * lval[q];
                    ++p;
                    ++q;
                } else if (cp < cq) {
                    ++p;
                } else {
                    ++q;
                }
            }
            lval[a] = s / lval[qe];
        }
        (void)diag;
    }
}

// U = L^T: count, then one thread per row of L scatters; rows of U are sorted after
__global__ void transpose_count_kernel(const int32_t* __restrict__ lptr, const int32_t* __restrict__ lcol, int32_t n,
                                       int32_t* __restrict__ cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = lptr[i]; a < lptr[i + 1]; ++a) atomicAdd(&cnt[lcol[a]], 1);
}

__global__ void transpose_fill_kernel(const int32_t* __restrict__ lptr, const int32_t* __restrict__ lcol,
                                      const double* __restrict__ lval, int32_t n, const int32_t* __restrict__ uptr,
                                      int32_t* __restrict__ cursor, int32_t* __restrict__ ucol,
                                      double* __restrict__ uval) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = lptr[i]; a < lptr[i + 1]; ++a) {
            const int j = lcol[a];
            const int at = uptr[j] + atomicAdd(&cursor[j], 1);
            ucol[at] = (int32_t)i;
            uval[at] = lval[a];
        }
}

__global__ void sort_rows_kernel(const int32_t* __restrict__ ptr, int32_t n, int32_t* __restrict__ col,
                                 double* __restrict__ val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        sort_pairs(col + ptr[i], val + ptr[i], ptr[i + 1] - ptr[i]);
}

__global__ void to_f32_copy_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

__global__ void node_row_kernel(const int32_t* __restrict__ owner, const int32_t* __restrict__ pos, int64_t ng,
                                int32_t* __restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ng; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = owner[k] >= 0 ? pos[k] : -1;
}

__global__ void located_flag_kernel(const int32_t* __restrict__ owner, int64_t ng, int32_t* __restrict__ flag) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ng; k += (int64_t)gridDim.x * blockDim.x)
        flag[k] = owner[k] >= 0;
}

// ---------------------------------------------------------------------------
// apply: forward (L y = r) and backward (L^T z = y) solves, one level per launch
// ---------------------------------------------------------------------------
template <class V>
__global__ void lower_solve_level_kernel(const int32_t* __restrict__ rows, int32_t nrows,
                                         const int32_t* __restrict__ lptr, const int32_t* __restrict__ lcol,
                                         const V* __restrict__ lval, const V* __restrict__ r, V* __restrict__ y) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nrows; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = rows[t];
        const int b = lptr[i], e = lptr[i + 1] - 1;
        V s = r[i];
        for (int a = b; a < e; ++a) s -= lval[a] * y[lcol[a]];
        y[i] = s / lval[e];
    }
}

template <class V>
__global__ void upper_solve_level_kernel(const int32_t* __restrict__ rows, int32_t nrows,
                                         const int32_t* __restrict__ uptr, const int32_t* __restrict__ ucol,
                                         const V* __restrict__ uval, const V* __restrict__ y, V* __restrict__ z) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nrows; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = rows[t];
        const int b = uptr[i], e = uptr[i + 1];   // first entry is the diagonal
        V s = y[i];
        for (int a = b + 1; a < e; ++a) s -= uval[a] * z[ucol[a]];
        z[i] = s / uval[b];
    }
}

// ---------------------------------------------------------------------------
// apply, persistent form: one launch per triangular solve.  The rows come in
// tiles of at most 32 rows of one level, in level order; a warp claims the
// next tile through an atomic counter and solves one row per lane.  The rows a
// row depends on lie in earlier levels, so in tiles that running warps have
// already claimed: the earliest unfinished claimed tile can always proceed,
// whatever the number of resident CTAs.  A solved value publishes itself: the
// output vector starts filled with a signalling-NaN word that arithmetic never
// produces, and a lane that reads that word polls it (bounded by the wait
// budget) until the owner's store lands.  A wait that runs out sets the
// sticky status word; the waits still running see it and give up, the
// remaining rows are left unsolved, and the host reports GOFD_E_TIMEOUT.
// ---------------------------------------------------------------------------
struct TriCtl {
    unsigned claim[2];   // tiles claimed by the forward / backward solve
    int status;          // 1 once a wait has run out (cleared by the host when it reports it)
    int pad;
};

template <class V>
struct Word;
template <>
struct Word<double> {
    using T = unsigned long long;
    static constexpr T pending = 0xFFF5A5A5A5A5A5A5ull;   // signalling NaN (quiet bit clear)
    static constexpr T qnan = 0x7FFFFFFFFFFFFFFFull;
};
template <>
struct Word<float> {
    using T = unsigned;
    static constexpr T pending = 0xFFA5A5A5u;
    static constexpr T qnan = 0x7FFFFFFFu;
};

__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_word(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_word(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_word(unsigned* p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_status(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ double word_value(unsigned long long w) { return __longlong_as_double((long long)w); }
__device__ __forceinline__ float word_value(unsigned w) { return __uint_as_float(w); }
__device__ __forceinline__ unsigned long long value_word(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ unsigned value_word(float v) { return __float_as_uint(v); }

template <int U, class W>
__device__ __forceinline__ bool any_pending(const W (&y)[U], int m, W pending) {
    bool p = false;
#pragma unroll
    for (int k = 0; k < U; ++k) p |= k < m && y[k] == pending;
    return p;
}

// waits until none of the entries y[k] = o[c[k]] (k < m) holds `pending`.
// Each round probes the first pending entry only, and once that one has
// arrived reloads all pending ones together (their loads in flight at once):
// a warp far ahead of the solved rows then costs one load per round, not one
// per dependency.  The pause between rounds doubles from 32 to 256 ns, and
// starts again from 32 ns after a round that saw progress.  False
// (and the status set) once `budget` cycles have passed; false too if another
// wait has run out (the shared status word is read every 16th round only:
// every waiting warp reading it every round makes one hot L2 line)
template <int U, class W>
__device__ bool wait_words(const W* o, const int32_t (&c)[U], W (&y)[U], int m, W pending,
                           unsigned long long budget, int* status) {
    const long long t0 = clock64();
    unsigned ns = 32;
    for (unsigned round = 1;; ++round) {
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        int32_t cf = 0;
#pragma unroll
        for (int k = U - 1; k >= 0; --k)
            if (k < m && y[k] == pending) cf = c[k];
        if (ld_word(o + cf) != pending) {
#pragma unroll
            for (int k = 0; k < U; ++k)
                if (k < m && y[k] == pending) y[k] = ld_word(o + c[k]);
            if (!any_pending<U>(y, m, pending)) return true;
            ns = 32;   // progress: the next dependency is likely close behind
        }
        if ((unsigned long long)(clock64() - t0) > budget) {
            atomicExch(status, 1);
            return false;
        }
        if ((round & 15) == 0 && ld_status(status)) return false;
    }
}

// FWD: L y = rhs, L in CSR with the diagonal last; BWD: L^T z = rhs, L^T in
// CSR with the diagonal first, tiles taken in reverse.  A tile holds at most
// kTriRows rows of one level; kTriLanes lanes share a row, lane q taking the
// off-diagonal entries q, q + kTriLanes, ... so that a row's (up to
// kTriLanes * U) dependencies are loaded and polled in one round; the lanes'
// partial sums are added by shuffles (fixed order).  `out` must hold the
// pending word in every row on entry.  FWD also stores the pending word into
// clear[i] once row i's right-hand side has been read (clear may be rhs
// itself): that primes the backward solve's output without another pass.
constexpr int kTriLanes = 4;
constexpr int kTriRows = 32 / kTriLanes;

template <class V, bool FWD>
__global__ void __launch_bounds__(256) tri_solve_kernel(const int32_t* __restrict__ tile_pos, int32_t ntiles,
                                                        const int32_t* __restrict__ rows,
                                                        const int32_t* __restrict__ ptr,
                                                        const int32_t* __restrict__ col, const V* __restrict__ val,
                                                        const V* rhs, V* out, V* clear, TriCtl* ctl,
                                                        unsigned long long budget) {
    using W = typename Word<V>::T;
    constexpr W pending = Word<V>::pending;
    constexpr int U = 8;   // entries per lane whose values are loaded together
    W* o = reinterpret_cast<W*>(out);
    const int lane = threadIdx.x & 31, q = lane % kTriLanes;
    for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(&ctl->claim[FWD ? 0 : 1], 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned)ntiles) return;
        const int32_t tt = FWD ? (int32_t)t : ntiles - 1 - (int32_t)t;
        const int32_t pos = tile_pos[tt] + lane / kTriLanes;
        const bool active = pos < tile_pos[tt + 1];
        int32_t i = 0;
        V part = V(0), r0 = V(0), dg = V(1);
        int bad = 0;
        if (active) {
            i = rows[pos];
            const int32_t b = ptr[i], e = ptr[i + 1];
            const int32_t a0 = FWD ? b : b + 1, a1 = FWD ? e - 1 : e;
            if (q == 0) {
                r0 = rhs[i];
                dg = val[FWD ? e - 1 : b];
            }
            for (int32_t a = a0 + q; a < a1; a += kTriLanes * U) {
                const int m = (a1 - a + kTriLanes - 1) / kTriLanes;   // entries of this lane in the chunk (may exceed U)
                int32_t c[U];
                V w[U];
                W y[U];
#pragma unroll
                for (int k = 0; k < U; ++k)
                    if (k < m) {
                        c[k] = col[a + k * kTriLanes];
                        w[k] = val[a + k * kTriLanes];
                    }
#pragma unroll
                for (int k = 0; k < U; ++k)
                    if (k < m) y[k] = ld_word(o + c[k]);
                if (!bad && any_pending<U>(y, m, pending))
                    bad = !wait_words<U>(o, c, y, m, pending, budget, &ctl->status);
#pragma unroll
                for (int k = 0; k < U; ++k)
                    if (k < m) part += w[k] * word_value(y[k]);
            }
        }
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        bad |= __shfl_xor_sync(0xffffffffu, bad, 1);
        bad |= __shfl_xor_sync(0xffffffffu, bad, 2);
        if (active && q == 0) {
            if (FWD && clear) reinterpret_cast<W*>(clear)[i] = pending;
            if (!bad) {
                W r = value_word((r0 - part) / dg);
                if (r == pending) r = Word<V>::qnan;   // not produced by arithmetic; kept for the invariant
                st_word(o + i, r);
            }
        }
    }
}

// out[i] = pending for i < n; with perm, g[i] = r[perm[i]]; resets the claims
template <class V>
__global__ void tri_prepare_kernel(V* __restrict__ out, const V* __restrict__ r, const int32_t* __restrict__ perm,
                                   V* __restrict__ g, int64_t n, TriCtl* ctl) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->claim[0] = 0;
        ctl->claim[1] = 0;
    }
    using W = typename Word<V>::T;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        reinterpret_cast<W*>(out)[i] = Word<V>::pending;
        if (perm) g[i] = r[perm[i]];
    }
}

template <class V>
__global__ void gather_perm_kernel(const V* __restrict__ in, const int32_t* __restrict__ perm, int64_t n,
                                   V* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static StencilDesc stencil_desc(gofd_problem* p, int pattern) {
    StencilDesc sd{};
    sd.d = p->d;
    for (int c = 0; c < 3; ++c) sd.n[c] = p->n[c];
    std::vector<double> T(p->ngrid);
    GOFD_CUDA_TRY(cudaMemcpy(T.data(), p->T.ptr, 8 * p->ngrid, cudaMemcpyDeviceToHost));
    const int d = p->d;
    const bool full = (pattern == 9 || pattern == 27 || pattern == 3);
    int cnt = 0;
    for (int dz = (d > 2 ? -1 : 0); dz <= (d > 2 ? 1 : 0); ++dz)
        for (int dy = (d > 1 ? -1 : 0); dy <= (d > 1 ? 1 : 0); ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int l1 = std::abs(dx) + std::abs(dy) + std::abs(dz);
                if (!full && l1 > 1) continue;
                sd.off[cnt][0] = dx;
                sd.off[cnt][1] = dy;
                sd.off[cnt][2] = dz;
                const int64_t tix = std::abs(dx) + (int64_t)p->n[0] * (std::abs(dy) + (int64_t)p->n[1] * std::abs(dz));
                sd.T[cnt] = T[tix];
                ++cnt;
            }
    sd.count = cnt;
    return sd;
}

static int64_t sum_counts(DevBuf& cnt, DevBuf& ptr, int64_t n, cudaStream_t st) {
    ptr.alloc(sizeof(int32_t) * (n + 1));
    return exclusive_scan_i32(cnt.as<int32_t>(), ptr.as<int32_t>(), n + 1, st);
}

void setup_precond(gofd_problem* p) {
    const int pattern = p->opt.precond;
    if (pattern == 0) return;
    if (pattern == 1) {   // the diagonal of S (jacobi.cu)
        Precond* pc = new Precond();
        p->pc = pc;
        pc->pattern = 1;
        pc->n = p->nint;
        pc->nnz = p->nint;
        setup_jacobi(p, pc->diag, pc->dinv64, pc->dinv32);
        return;
    }
    if (pattern == 2) {   // the circulant alternative of Section 3.3: D_h^{-1} I^T C^{-1} I D_h^{-1}
        if (p->d != 2) fail(GOFD_E_ARG, "the circulant preconditioner (precond = 2) is 2D");
        cudaStream_t st = p->setup_stream;
        Precond* pc = new Precond();
        p->pc = pc;
        pc->pattern = 2;
        pc->n = p->nint;
        const int64_t H = p->P / 2 + 1, m = H * H, n1 = p->nint + 1;
        double p2d = 1.0;
        for (int i = 0; i < 2 * p->d; ++i) p2d *= (double)p->P;
        pc->lami64.alloc(8 * m);
        pc->lami32.alloc(4 * m);
        circulant_inverse_symbol_kernel<<<grid_blocks(m, 256), 256, 0, st>>>(
            p->lamT64.as<double>(), pc->lami64.as<double>(), pc->lami32.as<float>(), p2d, m);
        pc->dinv64.alloc(8 * n1);
        pc->dinv32.alloc(4 * n1);
        GOFD_CUDA_TRY(cudaMemsetAsync(pc->dinv64.ptr, 0, 8 * n1, st));
        GOFD_CUDA_TRY(cudaMemsetAsync(pc->dinv32.ptr, 0, 4 * n1, st));
        inverse_colsum_kernel<<<grid_blocks(p->nint, 256), 256, 0, st>>>(
            p->colsum.as<double>(), pc->dinv64.as<double>(), pc->dinv32.as<float>(), p->nint);
        GOFD_CHECK_LAUNCH();
        // work vectors; entry n_int is the zero pad the gather reads for boundary slots
        for (DevBuf* b : {&pc->tmp64a, &pc->tmp64b}) {
            b->alloc(8 * n1);
            GOFD_CUDA_TRY(cudaMemsetAsync(b->ptr, 0, 8 * n1, st));
        }
        for (DevBuf* b : {&pc->tmp32a, &pc->tmp32b}) {
            b->alloc(4 * n1);
            GOFD_CUDA_TRY(cudaMemsetAsync(b->ptr, 0, 4 * n1, st));
        }
        return;
    }
    const int d = p->d;
    const bool ok = (d == 1 && pattern == 3) || (d == 2 && (pattern == 5 || pattern == 9)) ||
                    (d == 3 && (pattern == 7 || pattern == 27));
    if (!ok)
        fail(GOFD_E_ARG,
             "preconditioner must be 1 (diagonal), 2 (circulant, 2D), or IC on 3 (1D), 5 or 9 (2D), 7 or 27 (3D)");
    if (p->opt.ic_level != 0 && p->opt.ic_level != 1) fail(GOFD_E_ARG, "only ic_level 1 is supported");
    cudaStream_t st = p->setup_stream;
    const int T = 256;
    const int32_t n = (int32_t)p->nint;
    Precond* pc = new Precond();
    p->pc = pc;
    pc->pattern = pattern;
    pc->ordering = p->opt.ordering;
    pc->n = n;

    DevBuf err;
    err.alloc(sizeof(int));
    GOFD_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, sizeof(int), st));
    // grid node -> ELL row
    DevBuf flag, pos, node_row;
    flag.alloc(4 * p->ngrid);
    pos.alloc(4 * p->ngrid);
    node_row.alloc(4 * p->ngrid);
    located_flag_kernel<<<grid_blocks(p->ngrid, T), T, 0, st>>>(p->owner.as<int32_t>(), p->ngrid, flag.as<int32_t>());
    exclusive_scan_i32(flag.as<int32_t>(), pos.as<int32_t>(), p->ngrid, st);
    node_row_kernel<<<grid_blocks(p->ngrid, T), T, 0, st>>>(p->owner.as<int32_t>(), pos.as<int32_t>(), p->ngrid,
                                                           node_row.as<int32_t>());
    GOFD_CHECK_LAUNCH();
    flag.release();
    pos.release();

    // A_h^(k) on the interior vertices
    const StencilDesc sd = stencil_desc(p, pattern);
    DevBuf cnt, aptr, acol, aval;
    cnt.alloc(4 * (n + 1));
    GOFD_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, 4 * (n + 1), st));
    const int ab = grid_blocks(n, 64, 1 << 20);
#define ASSEMBLE(CAP, PASS)                                                                                      \
    assemble_kernel<CAP><<<ab, 64, 0, st>>>(PASS, sd, p->csr_ptr.as<int32_t>(), p->csr_col.as<int32_t>(),          \
                                            p->csr_val64.as<double>(), node_row.as<int32_t>(),                    \
                                            p->ell_iidx.as<int32_t>(), p->ell_w64.as<double>(), p->nloc, n,        \
                                            cnt.as<int32_t>(), aptr.as<int32_t>(), acol.as<int32_t>(),             \
                                            aval.as<double>(), err.as<int>())
    if (d <= 2) ASSEMBLE(256, 0);
    else ASSEMBLE(1024, 0);
    GOFD_CHECK_LAUNCH();
    pc->nnz_a = sum_counts(cnt, aptr, n, st);
    acol.alloc(4 * pc->nnz_a);
    aval.alloc(8 * pc->nnz_a);
    if (d <= 2) ASSEMBLE(256, 1);
    else ASSEMBLE(1024, 1);
#undef ASSEMBLE
    GOFD_CHECK_LAUNCH();
    node_row.release();
    int herr = 0;
    GOFD_CUDA_TRY(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr & 1) fail(GOFD_E_PRECOND, "a row of the stencil Galerkin matrix is too dense");

    // ordering
    if (pc->ordering == 1) {
        DevBuf color, rem, ccnt, cstart;
        color.alloc(4 * n);
        rem.alloc(sizeof(int));
        std::vector<int32_t> minus(n, -1);
        GOFD_CUDA_TRY(cudaMemcpyAsync(color.ptr, minus.data(), 4 * n, cudaMemcpyHostToDevice, st));
        int c = 0, hrem = n;
        while (hrem > 0) {
            if (c > 4096) fail(GOFD_E_PRECOND, "colouring did not finish");
            GOFD_CUDA_TRY(cudaMemsetAsync(rem.ptr, 0, sizeof(int), st));
            color_round_kernel<<<grid_blocks(n, T), T, 0, st>>>(aptr.as<int32_t>(), acol.as<int32_t>(), n,
                                                               color.as<int32_t>(), c, rem.as<int>());
            color_commit_kernel<<<grid_blocks(n, T), T, 0, st>>>(color.as<int32_t>(), n);
            GOFD_CHECK_LAUNCH();
            GOFD_CUDA_TRY(cudaMemcpyAsync(&hrem, rem.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
            GOFD_CUDA_TRY(cudaStreamSynchronize(st));
            ++c;
        }
        const int ncolors = c;
        ccnt.alloc(4 * (ncolors + 1));
        GOFD_CUDA_TRY(cudaMemsetAsync(ccnt.ptr, 0, 4 * (ncolors + 1), st));
        color_count_kernel<<<grid_blocks(n, T), T, 0, st>>>(color.as<int32_t>(), n, ccnt.as<int32_t>());
        cstart.alloc(4 * (ncolors + 1));
        exclusive_scan_i32(ccnt.as<int32_t>(), cstart.as<int32_t>(), ncolors + 1, st);
        pc->perm.alloc(4 * n);
        pc->iperm.alloc(4 * n);
        color_perm_kernel<<<grid_blocks(ncolors, 64), 64, 0, st>>>(color.as<int32_t>(), n, ncolors,
                                                                   cstart.as<int32_t>(), pc->perm.as<int32_t>(),
                                                                   pc->iperm.as<int32_t>());
        GOFD_CHECK_LAUNCH();
        DevBuf bcnt, bptr, bcol, bval;
        bcnt.alloc(4 * (n + 1));
        GOFD_CUDA_TRY(cudaMemsetAsync(bcnt.ptr, 0, 4 * (n + 1), st));
        permute_count_kernel<<<grid_blocks(n, T), T, 0, st>>>(aptr.as<int32_t>(), pc->perm.as<int32_t>(), n,
                                                             bcnt.as<int32_t>());
        sum_counts(bcnt, bptr, n, st);
        bcol.alloc(4 * pc->nnz_a);
        bval.alloc(8 * pc->nnz_a);
        permute_fill_kernel<<<grid_blocks(n, 64), 64, 0, st>>>(aptr.as<int32_t>(), acol.as<int32_t>(),
                                                               aval.as<double>(), pc->perm.as<int32_t>(),
                                                               pc->iperm.as<int32_t>(), n, bptr.as<int32_t>(),
                                                               bcol.as<int32_t>(), bval.as<double>());
        GOFD_CHECK_LAUNCH();
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
        std::swap(aptr.ptr, bptr.ptr);
        std::swap(aptr.bytes, bptr.bytes);
        std::swap(acol.ptr, bcol.ptr);
        std::swap(acol.bytes, bcol.bytes);
        std::swap(aval.ptr, bval.ptr);
        std::swap(aval.bytes, bval.bytes);
    } else if (pc->ordering != 0) {
        fail(GOFD_E_ARG, "ordering must be 0 (natural) or 1 (multicolour)");
    }

    // symbolic IC(1)
    DevBuf lcnt;
    lcnt.alloc(4 * (n + 1));
    GOFD_CUDA_TRY(cudaMemsetAsync(lcnt.ptr, 0, 4 * (n + 1), st));
#define SYMB(CAP, PASS)                                                                                      \
    ic_symbolic_kernel<CAP><<<ab, 64, 0, st>>>(PASS, aptr.as<int32_t>(), acol.as<int32_t>(), n, lcnt.as<int32_t>(), \
                                               pc->lptr.as<int32_t>(), pc->lcol.as<int32_t>(), err.as<int>())
    if (d <= 2) SYMB(512, 0);
    else SYMB(4096, 0);
    GOFD_CHECK_LAUNCH();
    pc->nnz = sum_counts(lcnt, pc->lptr, n, st);
    pc->lcol.alloc(4 * pc->nnz);
    if (d <= 2) SYMB(512, 1);
    else SYMB(4096, 1);
#undef SYMB
    GOFD_CHECK_LAUNCH();
    GOFD_CUDA_TRY(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr & 2) fail(GOFD_E_PRECOND, "a row of the IC(1) pattern is too dense");

    // levels
    DevBuf lev, changed;
    lev.alloc(4 * n);
    changed.alloc(sizeof(int));
    GOFD_CUDA_TRY(cudaMemsetAsync(lev.ptr, 0, 4 * n, st));
    for (int sweep = 0;; sweep += 8) {
        if (sweep > 4 * n + 16) fail(GOFD_E_PRECOND, "level schedule did not converge");
        GOFD_CUDA_TRY(cudaMemsetAsync(changed.ptr, 0, sizeof(int), st));
        for (int r = 0; r < 8; ++r)
            level_sweep_kernel<<<grid_blocks(n, T), T, 0, st>>>(pc->lptr.as<int32_t>(), pc->lcol.as<int32_t>(), n,
                                                               lev.as<int32_t>(), changed.as<int>());
        GOFD_CHECK_LAUNCH();
        int hc = 0;
        GOFD_CUDA_TRY(cudaMemcpyAsync(&hc, changed.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
        if (!hc) break;
    }
    std::vector<int32_t> hlev(n);
    GOFD_CUDA_TRY(cudaMemcpy(hlev.data(), lev.ptr, 4 * n, cudaMemcpyDeviceToHost));
    int nlev = 0;
    for (int32_t v : hlev) nlev = std::max(nlev, v + 1);
    pc->nlevels = nlev;
    {
        DevBuf lc, cur;
        lc.alloc(4 * (nlev + 1));
        cur.alloc(4 * (nlev + 1));
        GOFD_CUDA_TRY(cudaMemsetAsync(lc.ptr, 0, 4 * (nlev + 1), st));
        GOFD_CUDA_TRY(cudaMemsetAsync(cur.ptr, 0, 4 * (nlev + 1), st));
        level_count_kernel<<<grid_blocks(n, T), T, 0, st>>>(lev.as<int32_t>(), n, lc.as<int32_t>());
        pc->level_ptr.alloc(4 * (nlev + 1));
        exclusive_scan_i32(lc.as<int32_t>(), pc->level_ptr.as<int32_t>(), nlev + 1, st);
        pc->level_rows.alloc(4 * n);
        level_fill_kernel<<<grid_blocks(n, T), T, 0, st>>>(lev.as<int32_t>(), n, pc->level_ptr.as<int32_t>(),
                                                          cur.as<int32_t>(), pc->level_rows.as<int32_t>());
        GOFD_CHECK_LAUNCH();
        pc->hlevel_ptr.resize(nlev + 1);
        GOFD_CUDA_TRY(cudaMemcpyAsync(pc->hlevel_ptr.data(), pc->level_ptr.ptr, 4 * (nlev + 1),
                                      cudaMemcpyDeviceToHost, st));
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    }

    // numeric, with a diagonal shift on breakdown
    pc->lval64.alloc(8 * pc->nnz);
    double shift = 0.0;
    for (int attempt = 0;; ++attempt) {
        if (attempt > 24) fail(GOFD_E_PRECOND, "incomplete Cholesky broke down for every shift tried");
        GOFD_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, sizeof(int), st));
        for (int l = 0; l < nlev; ++l) {
            const int32_t nr = pc->hlevel_ptr[l + 1] - pc->hlevel_ptr[l];
            ic_numeric_level_kernel<<<grid_blocks(nr, 128), 128, 0, st>>>(
                pc->level_rows.as<int32_t>() + pc->hlevel_ptr[l], nr, aptr.as<int32_t>(), acol.as<int32_t>(),
                aval.as<double>(), pc->lptr.as<int32_t>(), pc->lcol.as<int32_t>(), pc->lval64.as<double>(), shift,
                err.as<int>());
        }
        GOFD_CHECK_LAUNCH();
        GOFD_CUDA_TRY(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
        if (!(herr & 4)) break;
        shift = 1e-3 * std::pow(2.0, attempt);
    }
    pc->shift = shift;

    // U = L^T for the backward solve, and FP32 copies
    {
        DevBuf ucnt, cur;
        ucnt.alloc(4 * (n + 1));
        cur.alloc(4 * (n + 1));
        GOFD_CUDA_TRY(cudaMemsetAsync(ucnt.ptr, 0, 4 * (n + 1), st));
        GOFD_CUDA_TRY(cudaMemsetAsync(cur.ptr, 0, 4 * (n + 1), st));
        transpose_count_kernel<<<grid_blocks(n, T), T, 0, st>>>(pc->lptr.as<int32_t>(), pc->lcol.as<int32_t>(), n,
                                                               ucnt.as<int32_t>());
        sum_counts(ucnt, pc->uptr, n, st);
        pc->ucol.alloc(4 * pc->nnz);
        pc->uval64.alloc(8 * pc->nnz);
        transpose_fill_kernel<<<grid_blocks(n, T), T, 0, st>>>(pc->lptr.as<int32_t>(), pc->lcol.as<int32_t>(),
                                                              pc->lval64.as<double>(), n, pc->uptr.as<int32_t>(),
                                                              cur.as<int32_t>(), pc->ucol.as<int32_t>(),
                                                              pc->uval64.as<double>());
        sort_rows_kernel<<<grid_blocks(n, 64), 64, 0, st>>>(pc->uptr.as<int32_t>(), n, pc->ucol.as<int32_t>(),
                                                           pc->uval64.as<double>());
        GOFD_CHECK_LAUNCH();
        pc->lval32.alloc(4 * pc->nnz);
        pc->uval32.alloc(4 * pc->nnz);
        to_f32_copy_kernel<<<grid_blocks(pc->nnz, T), T, 0, st>>>(pc->lval64.as<double>(), pc->lval32.as<float>(),
                                                                 pc->nnz);
        to_f32_copy_kernel<<<grid_blocks(pc->nnz, T), T, 0, st>>>(pc->uval64.as<double>(), pc->uval32.as<float>(),
                                                                 pc->nnz);
        GOFD_CHECK_LAUNCH();
    }
    // tiles of the persistent solves: at most kTriRows rows, never across a level
    {
        std::vector<int32_t> tp;
        for (int l = 0; l < nlev; ++l)
            for (int32_t b = pc->hlevel_ptr[l]; b < pc->hlevel_ptr[l + 1]; b += kTriRows) tp.push_back(b);
        tp.push_back(pc->hlevel_ptr[nlev]);
        pc->ntiles = (int32_t)tp.size() - 1;
        pc->tile_pos.alloc(4 * tp.size());
        GOFD_CUDA_TRY(cudaMemcpy(pc->tile_pos.ptr, tp.data(), 4 * tp.size(), cudaMemcpyHostToDevice));
        pc->ctl.alloc(sizeof(TriCtl));
        GOFD_CUDA_TRY(cudaMemset(pc->ctl.ptr, 0, sizeof(TriCtl)));
        pc->solve = p->opt.ic_solve;
        pc->budget = p->opt.wait_budget_cycles ? p->opt.wait_budget_cycles : 2000000000ull;
        const void* fns[4] = {(const void*)tri_solve_kernel<float, true>, (const void*)tri_solve_kernel<float, false>,
                              (const void*)tri_solve_kernel<double, true>,
                              (const void*)tri_solve_kernel<double, false>};
        // one CTA (eight warps, each holding one tile at a time) per SM: more
        // resident warps only add polling traffic on the rows being solved
        // (measured on the L-shape 1024^2 IC(1) factor: 0.55 ms per FP32
        // apply with one CTA per SM, 0.57 with two, 0.61 with three)
        const int need = (pc->ntiles + 7) / 8;
        for (int k = 0; k < 4; ++k) {
            int per_sm = 0;
            GOFD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[k], 256, 0));
            if (per_sm < 1) fail(GOFD_E_CUDA, "the triangular-solve kernel does not fit on an SM");
            pc->solve_blocks[k] = std::max(1, std::min(need, p->sm_count));
        }
    }
    pc->tmp64a.alloc(8 * (n + 1));
    pc->tmp64b.alloc(8 * (n + 1));
    pc->tmp32a.alloc(4 * (n + 1));
    pc->tmp32b.alloc(4 * (n + 1));
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
}

void free_precond(gofd_problem* p) {
    delete p->pc;
    p->pc = nullptr;
}

int64_t precond_nnz(const gofd_problem* p) { return p->pc ? p->pc->nnz : 0; }
double precond_shift(const gofd_problem* p) { return p->pc ? p->pc->shift : 0.0; }
int precond_levels(const gofd_problem* p) { return p->pc ? p->pc->nlevels : 0; }

template <class V>
static void apply_t(gofd_problem* p, const V* r, V* z, V* t1, V* t2, cudaStream_t st) {
    Precond* pc = p->pc;
    const int32_t n = (int32_t)pc->n;
    const bool f64 = sizeof(V) == 8;
    const V* lv = reinterpret_cast<const V*>(f64 ? pc->lval64.ptr : pc->lval32.ptr);
    const V* uv = reinterpret_cast<const V*>(f64 ? pc->uval64.ptr : pc->uval32.ptr);
    const V* rin = r;
    V* y = t1;
    V* zo = z;
    if (pc->solve == 0) {   // one persistent launch per solve
        const int32_t* perm = pc->ordering == 1 ? pc->perm.as<int32_t>() : nullptr;
        if (perm) {
            rin = t2;
            zo = t2;   // the backward solve's output overwrites the permuted r once the forward solve read it
        }
        TriCtl* ctl = pc->ctl.as<TriCtl>();
        tri_prepare_kernel<V><<<grid_blocks(n, 256), 256, 0, st>>>(y, r, perm, t2, n, ctl);
        const int k = f64 ? 2 : 0;
        tri_solve_kernel<V, true><<<pc->solve_blocks[k], 256, 0, st>>>(
            pc->tile_pos.as<int32_t>(), pc->ntiles, pc->level_rows.as<int32_t>(), pc->lptr.as<int32_t>(),
            pc->lcol.as<int32_t>(), lv, rin, y, zo, ctl, pc->budget);
        tri_solve_kernel<V, false><<<pc->solve_blocks[k + 1], 256, 0, st>>>(
            pc->tile_pos.as<int32_t>(), pc->ntiles, pc->level_rows.as<int32_t>(), pc->uptr.as<int32_t>(),
            pc->ucol.as<int32_t>(), uv, y, zo, nullptr, ctl, pc->budget);
        if (perm) gather_perm_kernel<V><<<grid_blocks(n, 256), 256, 0, st>>>(t2, pc->iperm.as<int32_t>(), n, z);
        GOFD_CHECK_LAUNCH();
        return;
    }
    if (pc->ordering == 1) {
        gather_perm_kernel<V><<<grid_blocks(n, 256), 256, 0, st>>>(r, pc->perm.as<int32_t>(), n, t2);
        rin = t2;
        zo = t2;   // the permuted z overwrites the permuted r (not read by the backward solve)
    }
    for (int l = 0; l < pc->nlevels; ++l) {
        const int32_t nr = pc->hlevel_ptr[l + 1] - pc->hlevel_ptr[l];
        lower_solve_level_kernel<V><<<grid_blocks(nr, 128), 128, 0, st>>>(
            pc->level_rows.as<int32_t>() + pc->hlevel_ptr[l], nr, pc->lptr.as<int32_t>(), pc->lcol.as<int32_t>(), lv,
            rin, y);
    }
    for (int l = pc->nlevels - 1; l >= 0; --l) {
        const int32_t nr = pc->hlevel_ptr[l + 1] - pc->hlevel_ptr[l];
        upper_solve_level_kernel<V><<<grid_blocks(nr, 128), 128, 0, st>>>(
            pc->level_rows.as<int32_t>() + pc->hlevel_ptr[l], nr, pc->uptr.as<int32_t>(), pc->ucol.as<int32_t>(), uv,
            y, zo);
    }
    if (pc->ordering == 1)
        gather_perm_kernel<V><<<grid_blocks(n, 256), 256, 0, st>>>(t2, pc->iperm.as<int32_t>(), n, z);
    GOFD_CHECK_LAUNCH();
}

void precond_apply(gofd_problem* p, bool fp64, const void* r, void* z, cudaStream_t st) {
    Precond* pc = p->pc;
    if (!pc) fail(GOFD_E_ARG, "no preconditioner");
    if (pc->pattern == 1) {
        jacobi_apply(p, fp64, fp64 ? pc->dinv64.ptr : pc->dinv32.ptr, r, z, st);
        return;
    }
    if (pc->pattern == 2) {   // z = D_h^{-1} I^T C^{-1} I D_h^{-1} r
        const void* dinv = fp64 ? pc->dinv64.ptr : pc->dinv32.ptr;
        void* a = fp64 ? pc->tmp64a.ptr : pc->tmp32a.ptr;
        void* b = fp64 ? pc->tmp64b.ptr : pc->tmp32b.ptr;
        jacobi_apply(p, fp64, dinv, r, a, st);
        apply_interior_symbol(p, fp64, a, b, fp64 ? pc->lami64.ptr : pc->lami32.ptr, st);
        jacobi_apply(p, fp64, dinv, b, z, st);
        return;
    }
    if (fp64) {
        apply_t<double>(p, (const double*)r, (double*)z, pc->tmp64a.as<double>(), pc->tmp64b.as<double>(), st);
    } else {
        apply_t<float>(p, (const float*)r, (float*)z, pc->tmp32a.as<float>(), pc->tmp32b.as<float>(), st);
    }
}

// GOFD_E_TIMEOUT if a wait of the persistent triangular solves has run out
// since the last check (synchronises the stream; clears the status)
void precond_check(gofd_problem* p, cudaStream_t st) {
    Precond* pc = p->pc;
    if (!pc || !pc->ctl.ptr || pc->solve != 0) return;
    TriCtl h{};
    GOFD_CUDA_TRY(cudaMemcpyAsync(&h, pc->ctl.ptr, sizeof(TriCtl), cudaMemcpyDeviceToHost, st));
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (h.status) {
        GOFD_CUDA_TRY(cudaMemsetAsync(&pc->ctl.as<TriCtl>()->status, 0, sizeof(int), st));
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
        fail(GOFD_E_TIMEOUT, "a wait of the IC triangular solves ran out (wait_budget_cycles)");
    }
}

// export of the factor for parity checks
void precond_export(const gofd_problem* p, int32_t* perm, int32_t* lptr, int32_t* lcol, double* lval) {
    const Precond* pc = p->pc;
    if (!pc) fail(GOFD_E_ARG, "no preconditioner");
    if (pc->pattern == 1) fail(GOFD_E_ARG, "the diagonal preconditioner has no factor (gofd_export_diagonal)");
    if (pc->pattern == 2) fail(GOFD_E_ARG, "the circulant preconditioner has no factor");
    const int32_t n = (int32_t)pc->n;
    if (perm) {
        if (pc->ordering == 1) GOFD_CUDA_TRY(cudaMemcpy(perm, pc->perm.ptr, 4 * n, cudaMemcpyDeviceToHost));
        else
            for (int32_t i = 0; i < n; ++i) perm[i] = i;
    }
    if (lptr) GOFD_CUDA_TRY(cudaMemcpy(lptr, pc->lptr.ptr, 4 * (n + 1), cudaMemcpyDeviceToHost));
    if (lcol) GOFD_CUDA_TRY(cudaMemcpy(lcol, pc->lcol.ptr, 4 * pc->nnz, cudaMemcpyDeviceToHost));
    if (lval) GOFD_CUDA_TRY(cudaMemcpy(lval, pc->lval64.ptr, 8 * pc->nnz, cudaMemcpyDeviceToHost));
}

// the diagonal of S (pattern 1) copied to host, n_interior doubles
void precond_diagonal(const gofd_problem* p, double* diag) {
    const Precond* pc = p->pc;
    if (!pc || pc->pattern != 1) fail(GOFD_E_ARG, "the problem was not built with the diagonal preconditioner");
    GOFD_CUDA_TRY(cudaMemcpy(diag, pc->diag.ptr, 8 * pc->n, cudaMemcpyDeviceToHost));
}

}  // namespace gofd
