// Mesh-side set-up on the device (Section 3.1 of the paper):
//   exact point location of every overlay node -> owner simplex (or -1),
//   the ELL form of I_h^FD (IhFD-1) with P1 barycentric weights,
//   runs of located nodes along axis 0 (used by the fused gather),
//   boundary vertices (facets with one adjacent simplex) and interior numbering,
//   the transpose I^T as interior-vertex-major CSR sorted by grid index,
//   column sums D_h (Lemma 3.1 (iv)) and the minimum element height a_h.
#include <climits>
#include <cmath>

#include "gofd_internal.cuh"
#include "predicates.cuh"

namespace gofd {

int grid_blocks(int64_t work, int threads, int cap) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// ---------------------------------------------------------------------------
// exclusive scan of int32 (three phases, recursive on block totals)
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void scan_tile_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                 int32_t* __restrict__ tile_sums, int64_t n) {
    __shared__ int32_t warp_tot[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t local = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t j = base + i;
        v[i] = (j < n) ? in[j] : 0;
        local += v[i];
    }
    // inclusive warp scan of thread totals
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t w = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    int32_t excl = incl - local + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t j = base + i;
        if (j < n) out[j] = excl;
        excl += v[i];
    }
    if (threadIdx.x == SCAN_THREADS - 1) tile_sums[blockIdx.x] = excl;
}

__global__ void scan_add_kernel(int32_t* __restrict__ out, const int32_t* __restrict__ offs, int64_t n) {
    int64_t j = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
    int32_t add = offs[blockIdx.x];
    for (int i = 0; i < SCAN_ITEMS; ++i, j += SCAN_THREADS)
        if (j < n) out[j] += add;
}

static void scan_rec(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    DevBuf sums, sums_scan;
    sums.alloc(sizeof(int32_t) * (tiles + 1));
    sums_scan.alloc(sizeof(int32_t) * (tiles + 1));
    scan_tile_kernel<<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, out, sums.as<int32_t>(), n);
    GOFD_CHECK_LAUNCH();
    if (tiles > 1) {
        scan_rec(sums.as<int32_t>(), sums_scan.as<int32_t>(), tiles, st);
        scan_add_kernel<<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(out, sums_scan.as<int32_t>(), n);
        GOFD_CHECK_LAUNCH();
    }
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
}

int64_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
    if (n == 0) return 0;
    scan_rec(in, out, n, st);
    int32_t last_in = 0, last_out = 0;
    GOFD_CUDA_TRY(cudaMemcpyAsync(&last_in, in + n - 1, 4, cudaMemcpyDeviceToHost, st));
    GOFD_CUDA_TRY(cudaMemcpyAsync(&last_out, out + n - 1, 4, cudaMemcpyDeviceToHost, st));
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    return (int64_t)last_in + (int64_t)last_out;
}

// ---------------------------------------------------------------------------
// geometry helpers
// ---------------------------------------------------------------------------
struct GridDesc {
    double lo[3];
    double h;
    int n[3];
};

__device__ __forceinline__ double grid_coord(const GridDesc& g, int ax, int k) {
    return __dadd_rn(g.lo[ax], __dmul_rn((double)k, g.h));
}

// Orientation sign and minimum height of every simplex.
template <int D>
__global__ void element_kernel(const double* __restrict__ V, const int32_t* __restrict__ S,
                               int64_t ne, int8_t* __restrict__ esign,
                               unsigned long long* __restrict__ ah_bits, int* __restrict__ err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        double pts[D + 1][D];
        const double* pp[D + 1];
        for (int a = 0; a <= D; ++a) {
            int v = S[e * (D + 1) + a];
            for (int c = 0; c < D; ++c) pts[a][c] = V[(int64_t)v * D + c];
            pp[a] = pts[a];
        }
        int o = orient_sign<D>(pp);
        esign[e] = (int8_t)o;
        if (o == 0) {
            atomicOr(err, 1);
            continue;
        }
        // a_j = D |K| / |S_j| (Section 3.1, heights before Lemma 3.3)
        double vol = fabs(orient_value<D>(pp));  // D! |K|
        double aK = INFINITY;
        for (int j = 0; j <= D; ++j) {
            double area;  // (D-1)! |S_j|
            if constexpr (D == 1) {
                area = 1.0;
            } else if constexpr (D == 2) {
                const double* p = pts[(j + 1) % 3];
                const double* q = pts[(j + 2) % 3];
                area = hypot(p[0] - q[0], p[1] - q[1]);
            } else {
                int f[3], m = 0;
                for (int a = 0; a < 4; ++a)
                    if (a != j) f[m++] = a;
                double u[3], w[3];
                for (int c = 0; c < 3; ++c) {
                    u[c] = pts[f[1]][c] - pts[f[0]][c];
                    w[c] = pts[f[2]][c] - pts[f[0]][c];
                }
                double cx = u[1] * w[2] - u[2] * w[1];
                double cy = u[2] * w[0] - u[0] * w[2];
                double cz = u[0] * w[1] - u[1] * w[0];
                area = sqrt(cx * cx + cy * cy + cz * cz);
            }
            // |K| = vol / D!, |S_j| = area / (D-1)!  ->  a_j = D |K| / |S_j| = vol / area
            double aj = vol / area;
            aK = fmin(aK, aj);
        }
        atomicMin(ah_bits, (unsigned long long)__double_as_longlong(aK));
    }
}

// Element-parallel point location: each simplex tests the grid nodes of its
// bounding box with exact orientation signs; the lowest containing element
// index wins (atomicMin on integers, independent of the order of updates).
template <int D>
__global__ void locate_kernel(const double* __restrict__ V, const int32_t* __restrict__ S,
                              const int8_t* __restrict__ esign, int64_t ne, GridDesc g,
                              int32_t* __restrict__ owner) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        double pts[D + 1][D];
        double bmin[3] = {0, 0, 0}, bmax[3] = {0, 0, 0};
        for (int a = 0; a <= D; ++a) {
            int v = S[e * (D + 1) + a];
            for (int c = 0; c < D; ++c) {
                double x = V[(int64_t)v * D + c];
                pts[a][c] = x;
                if (a == 0 || x < bmin[c]) bmin[c] = x;
                if (a == 0 || x > bmax[c]) bmax[c] = x;
            }
        }
        int o = esign[e];
        int klo[3] = {0, 0, 0}, khi[3] = {0, 0, 0};
        for (int c = 0; c < D; ++c) {
            double a = floor((bmin[c] - g.lo[c]) / g.h) - 1.0;
            double b = ceil((bmax[c] - g.lo[c]) / g.h) + 1.0;
            klo[c] = (int)fmax(0.0, a);
            khi[c] = (int)fmin((double)(g.n[c] - 1), b);
        }
        for (int k2 = klo[2]; k2 <= khi[2]; ++k2)
            for (int k1 = klo[1]; k1 <= khi[1]; ++k1)
                for (int k0 = klo[0]; k0 <= khi[0]; ++k0) {
                    int kk[3] = {k0, k1, k2};
                    double x[3];
                    bool inbox = true;
                    for (int c = 0; c < D; ++c) {
                        x[c] = grid_coord(g, c, kk[c]);
                        inbox &= (x[c] >= bmin[c]) && (x[c] <= bmax[c]);
                    }
                    if (!inbox) continue;
                    bool inside = true;
                    for (int i = 0; i <= D && inside; ++i) {
                        const double* pp[D + 1];
                        for (int a = 0; a <= D; ++a) pp[a] = (a == i) ? x : pts[a];
                        int si = orient_sign<D>(pp);
                        if (si != 0 && si != o) inside = false;
                    }
                    if (inside) {
                        int64_t lin = (int64_t)k0 + (int64_t)g.n[0] * ((int64_t)k1 + (int64_t)g.n[1] * k2);
                        atomicMin(&owner[lin], (int32_t)e);
                    }
                }
    }
}

__global__ void owner_finalize_kernel(int32_t* __restrict__ owner, int32_t* __restrict__ flag,
                                      int64_t ng) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ng;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t o = owner[k];
        if (o == INT_MAX) o = -1;
        owner[k] = o;
        flag[k] = o >= 0;
    }
}

// ELL rows in increasing grid index: node, vertex index and barycentric weight
// per slot, phi_i = D_i / D_K (Lemma 3.4), clamped to [0,1].
template <int D>
__global__ void ell_fill_kernel(const double* __restrict__ V, const int32_t* __restrict__ S,
                                const int32_t* __restrict__ owner, const int32_t* __restrict__ pos,
                                int64_t ng, int64_t nloc, GridDesc g, int32_t* __restrict__ ell_node,
                                int32_t* __restrict__ vidx, double* __restrict__ w64,
                                float* __restrict__ w32) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ng;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t o = owner[k];
        if (o < 0) continue;
        int64_t e = pos[k];
        ell_node[e] = (int32_t)k;
        double pts[D + 1][D];
        int vv[D + 1];
        for (int a = 0; a <= D; ++a) {
            vv[a] = S[(int64_t)o * (D + 1) + a];
            for (int c = 0; c < D; ++c) pts[a][c] = V[(int64_t)vv[a] * D + c];
        }
        int kk[3] = {(int)(k % g.n[0]), (int)((k / g.n[0]) % g.n[1]), (int)(k / ((int64_t)g.n[0] * g.n[1]))};
        double x[3];
        for (int c = 0; c < D; ++c) x[c] = grid_coord(g, c, kk[c]);
        const double* pk[D + 1];
        for (int a = 0; a <= D; ++a) pk[a] = pts[a];
        double DK = orient_value<D>(pk);
        for (int i = 0; i <= D; ++i) {
            const double* pp[D + 1];
            for (int a = 0; a <= D; ++a) pp[a] = (a == i) ? x : pts[a];
            // exactly 0 on the facet opposite vertex i (exact sign), else D_i / D_K
            double wi = orient_sign<D>(pp) == 0 ? 0.0 : orient_value<D>(pp) / DK;
            wi = fmin(1.0, fmax(0.0, wi));
            vidx[(int64_t)i * nloc + e] = vv[i];
            w64[(int64_t)i * nloc + e] = wi;
            w32[(int64_t)i * nloc + e] = (float)wi;
        }
    }
}

// Runs of consecutive located nodes along axis 0, one thread per grid line.
__global__ void run_count_kernel(const int32_t* __restrict__ flag, int64_t nlines, int n0,
                                 int32_t* __restrict__ cnt) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nlines;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int32_t* f = flag + l * n0;
        int c = 0, prev = 0;
        for (int k = 0; k < n0; ++k) {
            int cur = f[k];
            c += (cur && !prev);
            prev = cur;
        }
        cnt[l] = c;
    }
}

__global__ void run_fill_kernel(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                const int32_t* __restrict__ rptr, int64_t nlines, int n0,
                                int32_t* __restrict__ rk0, int32_t* __restrict__ rlen,
                                int32_t* __restrict__ re0) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nlines;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int32_t* f = flag + l * n0;
        int r = rptr[l];
        int k = 0;
        while (k < n0) {
            if (!f[k]) {
                ++k;
                continue;
            }
            int s = k;
            while (k < n0 && f[k]) ++k;
            rk0[r] = s;
            rlen[r] = k - s;
            re0[r] = pos[l * n0 + s];
            ++r;
        }
    }
}

// ---------------------------------------------------------------------------
// boundary facets by an open-addressing hash table of facet keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

constexpr unsigned long long EMPTY_KEY = 0xffffffffffffffffULL;

template <int D>
__device__ __forceinline__ uint64_t facet_key(const int32_t* s, int omit) {
    int f[3], m = 0;
    for (int a = 0; a <= D; ++a)
        if (a != omit) f[m++] = s[a];
    // sort the D vertex ids
    for (int i = 0; i < D; ++i)
        for (int j = i + 1; j < D; ++j)
            if (f[j] < f[i]) {
                int t = f[i];
                f[i] = f[j];
                f[j] = t;
            }
    if constexpr (D == 1) return (uint64_t)f[0];
    else if constexpr (D == 2) return ((uint64_t)f[0] << 32) | (uint64_t)f[1];
    else return ((uint64_t)f[0] << 42) | ((uint64_t)f[1] << 21) | (uint64_t)f[2];
}

template <int D>
__global__ void facet_insert_kernel(const int32_t* __restrict__ S, int64_t ne,
                                    unsigned long long* __restrict__ keys, int32_t* __restrict__ cnt,
                                    uint64_t mask, int* __restrict__ err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t* s = S + e * (D + 1);
        for (int j = 0; j <= D; ++j) {
            unsigned long long key = facet_key<D>(s, j);
            uint64_t slot = mix64(key) & mask;
            bool done = false;
            for (uint64_t probe = 0; probe <= mask; ++probe) {
                unsigned long long prev = atomicCAS(&keys[slot], EMPTY_KEY, key);
                if (prev == EMPTY_KEY || prev == key) {
                    atomicAdd(&cnt[slot], 1);
                    done = true;
                    break;
                }
                slot = (slot + 1) & mask;
            }
            if (!done) atomicOr(err, 2);
        }
    }
}

template <int D>
__global__ void facet_mark_kernel(const unsigned long long* __restrict__ keys,
                                  const int32_t* __restrict__ cnt, uint64_t cap,
                                  int32_t* __restrict__ bnd) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)cap;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long k = keys[i];
        if (k == EMPTY_KEY || cnt[i] != 1) continue;
        if constexpr (D == 1) {
            bnd[k] = 1;
        } else if constexpr (D == 2) {
            bnd[k >> 32] = 1;
            bnd[k & 0xffffffffULL] = 1;
        } else {
            bnd[k >> 42] = 1;
            bnd[(k >> 21) & 0x1fffffULL] = 1;
            bnd[k & 0x1fffffULL] = 1;
        }
    }
}

__global__ void interior_flag_kernel(const int32_t* __restrict__ bnd, int32_t* __restrict__ flag,
                                     int64_t nv) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        flag[v] = bnd[v] ? 0 : 1;
}

__global__ void interior_number_kernel(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                       int64_t nv, int32_t* __restrict__ v2i, int32_t* __restrict__ i2v) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (flag[v]) {
            v2i[v] = pos[v];
            i2v[pos[v]] = (int32_t)v;
        } else {
            v2i[v] = -1;
        }
    }
}

// ---------------------------------------------------------------------------
// transpose I^T over interior vertices
// ---------------------------------------------------------------------------
__global__ void ell_interior_kernel(const int32_t* __restrict__ vidx, const int32_t* __restrict__ v2i,
                                    int64_t total, int32_t nint, int32_t* __restrict__ iidx,
                                    int32_t* __restrict__ cnt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = v2i[vidx[t]];
        if (i >= 0) {
            iidx[t] = i;
            atomicAdd(&cnt[i], 1);
        } else {
            iidx[t] = nint;
        }
    }
}

__global__ void csr_scatter_kernel(const int32_t* __restrict__ iidx, int64_t nloc, int dp1,
                                   int32_t nint, const int32_t* __restrict__ ptr,
                                   int32_t* __restrict__ cursor, int64_t* __restrict__ packed) {
    int64_t total = nloc * dp1;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = iidx[t];
        if (i >= nint) continue;
        int64_t slot = t / nloc, e = t % nloc;
        int32_t at = ptr[i] + atomicAdd(&cursor[i], 1);
        packed[at] = e * 4 + slot;
    }
}

// Sort each row by ELL row (= by grid index).  Rows up to SHORT_ROW entries:
// insertion sort by one thread; longer rows (patches of large elements on a
// fine grid): one CTA per row, bottom-up merge sort where every element finds
// its place in the merged run by binary search in the partner run (keys are
// unique: a vertex appears once per grid node).
constexpr int SHORT_ROW = 256;

__global__ void csr_sort_short_kernel(const int32_t* __restrict__ ptr, int32_t nint, int64_t* __restrict__ packed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nint;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t b = ptr[i], e = ptr[i + 1];
        if (e - b > SHORT_ROW) continue;
        for (int32_t a = b + 1; a < e; ++a) {
            int64_t key = packed[a];
            int32_t c = a - 1;
            while (c >= b && packed[c] > key) {
                packed[c + 1] = packed[c];
                --c;
            }
            packed[c + 1] = key;
        }
    }
}

__global__ void csr_sort_long_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ rows,
                                     int64_t* __restrict__ packed, int64_t* __restrict__ tmp) {
    const int32_t i = rows[blockIdx.x];
    const int32_t b = ptr[i], L = ptr[i + 1] - b;
    int64_t* src = packed + b;
    int64_t* dst = tmp + b;
    for (int32_t run = 1; run < L; run *= 2) {
        for (int32_t p = threadIdx.x; p < L; p += blockDim.x) {
            const int32_t q = p / run;
            const int32_t own0 = q * run;
            const int32_t oth0 = (q ^ 1) * run;
            const int64_t key = src[p];
            int32_t pos = p;
            if (oth0 < L) {
                const int32_t oth1 = min(oth0 + run, L);
                int32_t lo = oth0, hi = oth1;   // number of partner keys below key
                while (lo < hi) {
                    const int32_t mid = (lo + hi) >> 1;
                    if (src[mid] < key) lo = mid + 1;
                    else hi = mid;
                }
                pos = min(own0, oth0) + (p - own0) + (lo - oth0);
            }
            dst[pos] = key;
        }
        __syncthreads();
        int64_t* t = src;
        src = dst;
        dst = t;
    }
    if (src != packed + b)
        for (int32_t p = threadIdx.x; p < L; p += blockDim.x) packed[b + p] = src[p];
}

__global__ void csr_long_rows_kernel(const int32_t* __restrict__ ptr, int32_t nint, int32_t* __restrict__ count,
                                     int32_t* __restrict__ rows) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nint;
         i += (int64_t)gridDim.x * blockDim.x)
        if (ptr[i + 1] - ptr[i] > SHORT_ROW) rows[atomicAdd(count, 1)] = (int32_t)i;
}

// Sort every row of a row-pointer array of unique packed keys ascending.
void sort_packed_rows(const int32_t* ptr, int64_t nrows, int64_t* packed, int64_t nnz, cudaStream_t st) {
    csr_sort_short_kernel<<<grid_blocks(nrows, 128), 128, 0, st>>>(ptr, (int32_t)nrows, packed);
    GOFD_CHECK_LAUNCH();
    DevBuf nlong, rows;
    nlong.alloc(sizeof(int32_t));
    rows.alloc(sizeof(int32_t) * (nrows + 1));
    GOFD_CUDA_TRY(cudaMemsetAsync(nlong.ptr, 0, sizeof(int32_t), st));
    csr_long_rows_kernel<<<grid_blocks(nrows, 256), 256, 0, st>>>(ptr, (int32_t)nrows, nlong.as<int32_t>(),
                                                                   rows.as<int32_t>());
    GOFD_CHECK_LAUNCH();
    int32_t hl = 0;
    GOFD_CUDA_TRY(cudaMemcpyAsync(&hl, nlong.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (hl > 0) {
        DevBuf tmp;
        tmp.alloc(sizeof(int64_t) * nnz);
        csr_sort_long_kernel<<<hl, 512, 0, st>>>(ptr, rows.as<int32_t>(), packed, tmp.as<int64_t>());
        GOFD_CHECK_LAUNCH();
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    }
}

// Emit columns, values and the column sum D_h in the sorted order.
__global__ void csr_finalize_kernel(const int32_t* __restrict__ ptr, int32_t nint,
                                    const int64_t* __restrict__ packed, const int32_t* __restrict__ ell_node,
                                    const double* __restrict__ w64, int64_t nloc,
                                    int32_t* __restrict__ col, double* __restrict__ v64,
                                    float* __restrict__ v32, double* __restrict__ colsum) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nint;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t b = ptr[i], e = ptr[i + 1];
        double sum = 0.0;
        for (int32_t a = b; a < e; ++a) {
            int64_t r = packed[a] >> 2, s = packed[a] & 3;
            double w = w64[s * nloc + r];
            col[a] = ell_node[r];
            v64[a] = w;
            v32[a] = (float)w;
            sum += w;
        }
        colsum[i] = sum;
    }
}

__global__ void min_positive_kernel(const double* __restrict__ x, int64_t n,
                                    unsigned long long* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicMin(out, (unsigned long long)__double_as_longlong(fmax(x[i], 0.0)));
}

__global__ void fill_i32_kernel(int32_t* p, int32_t v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void fill_u64_kernel(unsigned long long* p, unsigned long long v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ---------------------------------------------------------------------------
// host-side sequence of the set-up
// ---------------------------------------------------------------------------
template <int D>
static void setup_mesh_d(gofd_problem* p) {
    cudaStream_t st = p->setup_stream;
    const int T = 256;
    GridDesc g;
    for (int c = 0; c < 3; ++c) {
        g.lo[c] = p->lo[c];
        g.n[c] = p->n[c];
    }
    g.h = p->h;

    DevBuf err, esign, ahb;
    err.alloc(sizeof(int));
    esign.alloc(p->ne);
    ahb.alloc(sizeof(unsigned long long));
    GOFD_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, sizeof(int), st));
    fill_u64_kernel<<<1, 1, 0, st>>>(ahb.as<unsigned long long>(), 0x7ff0000000000000ULL, 1);
    element_kernel<D><<<grid_blocks(p->ne, T), T, 0, st>>>(
        p->verts.as<double>(), p->simp.as<int32_t>(), p->ne, esign.as<int8_t>(),
        ahb.as<unsigned long long>(), err.as<int>());
    GOFD_CHECK_LAUNCH();
    int herr = 0;
    unsigned long long ah = 0;
    GOFD_CUDA_TRY(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    GOFD_CUDA_TRY(cudaMemcpyAsync(&ah, ahb.ptr, sizeof(ah), cudaMemcpyDeviceToHost, st));
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr & 1) fail(GOFD_E_DEGENERATE_SIMPLEX, "a simplex has zero volume");
    double ahd;
    memcpy(&ahd, &ah, sizeof(double));
    p->a_h = ahd;

    // point location
    p->owner.alloc(sizeof(int32_t) * p->ngrid);
    DevBuf flag, pos;
    flag.alloc(sizeof(int32_t) * p->ngrid);
    pos.alloc(sizeof(int32_t) * p->ngrid);
    fill_i32_kernel<<<grid_blocks(p->ngrid, T), T, 0, st>>>(p->owner.as<int32_t>(), INT_MAX, p->ngrid);
    locate_kernel<D><<<grid_blocks(p->ne, 128, 1 << 20), 128, 0, st>>>(
        p->verts.as<double>(), p->simp.as<int32_t>(), esign.as<int8_t>(), p->ne, g,
        p->owner.as<int32_t>());
    GOFD_CHECK_LAUNCH();
    owner_finalize_kernel<<<grid_blocks(p->ngrid, T), T, 0, st>>>(p->owner.as<int32_t>(),
                                                                 flag.as<int32_t>(), p->ngrid);
    GOFD_CHECK_LAUNCH();
    p->nloc = exclusive_scan_i32(flag.as<int32_t>(), pos.as<int32_t>(), p->ngrid, st);
    const int64_t nloc = p->nloc;
    const int dp1 = D + 1;
    p->ell_node.alloc(sizeof(int32_t) * nloc);
    p->ell_vidx.alloc(sizeof(int32_t) * nloc * dp1);
    p->ell_w64.alloc(sizeof(double) * nloc * dp1);
    p->ell_w32.alloc(sizeof(float) * nloc * dp1);
    p->ell_iidx.alloc(sizeof(int32_t) * nloc * dp1);
    if (nloc > 0) {
        ell_fill_kernel<D><<<grid_blocks(p->ngrid, T), T, 0, st>>>(
            p->verts.as<double>(), p->simp.as<int32_t>(), p->owner.as<int32_t>(), pos.as<int32_t>(),
            p->ngrid, nloc, g, p->ell_node.as<int32_t>(), p->ell_vidx.as<int32_t>(),
            p->ell_w64.as<double>(), p->ell_w32.as<float>());
        GOFD_CHECK_LAUNCH();
    }

    // runs along axis 0
    {
        DevBuf cnt;
        cnt.alloc(sizeof(int32_t) * (p->nlines + 1));
        p->line_run_ptr.alloc(sizeof(int32_t) * (p->nlines + 1));
        GOFD_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, sizeof(int32_t) * (p->nlines + 1), st));
        run_count_kernel<<<grid_blocks(p->nlines, T), T, 0, st>>>(flag.as<int32_t>(), p->nlines,
                                                                   p->n[0], cnt.as<int32_t>());
        GOFD_CHECK_LAUNCH();
        p->nruns = exclusive_scan_i32(cnt.as<int32_t>(), p->line_run_ptr.as<int32_t>(), p->nlines + 1, st);
        p->run_k0.alloc(sizeof(int32_t) * p->nruns);
        p->run_len.alloc(sizeof(int32_t) * p->nruns);
        p->run_e0.alloc(sizeof(int32_t) * p->nruns);
        run_fill_kernel<<<grid_blocks(p->nlines, T), T, 0, st>>>(
            flag.as<int32_t>(), pos.as<int32_t>(), p->line_run_ptr.as<int32_t>(), p->nlines, p->n[0],
            p->run_k0.as<int32_t>(), p->run_len.as<int32_t>(), p->run_e0.as<int32_t>());
        GOFD_CHECK_LAUNCH();
    }

    // boundary vertices and interior numbering
    {
        int64_t nf = p->ne * dp1;
        uint64_t cap = 1;
        while (cap < (uint64_t)(2 * nf)) cap <<= 1;
        DevBuf keys, cnt, bnd, iflag, ipos;
        keys.alloc(sizeof(unsigned long long) * cap);
        cnt.alloc(sizeof(int32_t) * cap);
        bnd.alloc(sizeof(int32_t) * p->nv);
        iflag.alloc(sizeof(int32_t) * p->nv);
        ipos.alloc(sizeof(int32_t) * p->nv);
        fill_u64_kernel<<<grid_blocks(cap, T), T, 0, st>>>(keys.as<unsigned long long>(), EMPTY_KEY, cap);
        GOFD_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, sizeof(int32_t) * cap, st));
        GOFD_CUDA_TRY(cudaMemsetAsync(bnd.ptr, 0, sizeof(int32_t) * p->nv, st));
        facet_insert_kernel<D><<<grid_blocks(p->ne, T), T, 0, st>>>(
            p->simp.as<int32_t>(), p->ne, keys.as<unsigned long long>(), cnt.as<int32_t>(), cap - 1,
            err.as<int>());
        GOFD_CHECK_LAUNCH();
        facet_mark_kernel<D><<<grid_blocks(cap, T), T, 0, st>>>(keys.as<unsigned long long>(),
                                                                cnt.as<int32_t>(), cap, bnd.as<int32_t>());
        interior_flag_kernel<<<grid_blocks(p->nv, T), T, 0, st>>>(bnd.as<int32_t>(), iflag.as<int32_t>(), p->nv);
        GOFD_CHECK_LAUNCH();
        p->nint = exclusive_scan_i32(iflag.as<int32_t>(), ipos.as<int32_t>(), p->nv, st);
        p->vert2int.alloc(sizeof(int32_t) * p->nv);
        p->int2vert.alloc(sizeof(int32_t) * (p->nint + 1));
        interior_number_kernel<<<grid_blocks(p->nv, T), T, 0, st>>>(
            iflag.as<int32_t>(), ipos.as<int32_t>(), p->nv, p->vert2int.as<int32_t>(), p->int2vert.as<int32_t>());
        GOFD_CHECK_LAUNCH();
    }
    GOFD_CUDA_TRY(cudaMemcpyAsync(&herr, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    GOFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr & 2) fail(GOFD_E_CUDA, "facet hash table overflow");
    if (p->nint == 0) fail(GOFD_E_ARG, "the mesh has no interior vertex");

    // transpose over interior vertices
    {
        const int32_t nint = (int32_t)p->nint;
        DevBuf cnt, cursor, packed;
        cnt.alloc(sizeof(int32_t) * (p->nint + 1));
        cursor.alloc(sizeof(int32_t) * (p->nint + 1));
        GOFD_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, sizeof(int32_t) * (p->nint + 1), st));
        GOFD_CUDA_TRY(cudaMemsetAsync(cursor.ptr, 0, sizeof(int32_t) * (p->nint + 1), st));
        if (nloc > 0) {
            ell_interior_kernel<<<grid_blocks(nloc * dp1, T), T, 0, st>>>(
                p->ell_vidx.as<int32_t>(), p->vert2int.as<int32_t>(), nloc * dp1, nint,
                p->ell_iidx.as<int32_t>(), cnt.as<int32_t>());
            GOFD_CHECK_LAUNCH();
        }
        p->csr_ptr.alloc(sizeof(int32_t) * (p->nint + 1));
        p->nnz_t = exclusive_scan_i32(cnt.as<int32_t>(), p->csr_ptr.as<int32_t>(), p->nint + 1, st);
        packed.alloc(sizeof(int64_t) * p->nnz_t);
        p->csr_col.alloc(sizeof(int32_t) * p->nnz_t);
        p->csr_val64.alloc(sizeof(double) * p->nnz_t);
        p->csr_val32.alloc(sizeof(float) * p->nnz_t);
        p->colsum.alloc(sizeof(double) * p->nint);
        if (nloc > 0) {
            csr_scatter_kernel<<<grid_blocks(nloc * dp1, T), T, 0, st>>>(
                p->ell_iidx.as<int32_t>(), nloc, dp1, nint, p->csr_ptr.as<int32_t>(),
                cursor.as<int32_t>(), packed.as<int64_t>());
            GOFD_CHECK_LAUNCH();
        }
        sort_packed_rows(p->csr_ptr.as<int32_t>(), p->nint, packed.as<int64_t>(), p->nnz_t, st);
        csr_finalize_kernel<<<grid_blocks(p->nint, 128), 128, 0, st>>>(
            p->csr_ptr.as<int32_t>(), nint, packed.as<int64_t>(), p->ell_node.as<int32_t>(),
            p->ell_w64.as<double>(), nloc, p->csr_col.as<int32_t>(), p->csr_val64.as<double>(),
            p->csr_val32.as<float>(), p->colsum.as<double>());
        GOFD_CHECK_LAUNCH();
        fill_u64_kernel<<<1, 1, 0, st>>>(ahb.as<unsigned long long>(), 0x7ff0000000000000ULL, 1);
        min_positive_kernel<<<grid_blocks(p->nint, T), T, 0, st>>>(p->colsum.as<double>(), p->nint,
                                                                   ahb.as<unsigned long long>());
        GOFD_CHECK_LAUNCH();
        GOFD_CUDA_TRY(cudaMemcpyAsync(&ah, ahb.ptr, sizeof(ah), cudaMemcpyDeviceToHost, st));
        GOFD_CUDA_TRY(cudaStreamSynchronize(st));
        memcpy(&ahd, &ah, sizeof(double));
        p->min_colsum = ahd;
    }
    if (!(p->min_colsum > 0.0))
        fail(GOFD_E_ZERO_COLSUM,
             "an interior vertex has a zero column sum D_h (no grid node in its patch); use a smaller h");
}

void setup_mesh(gofd_problem* p, const double* verts_h, const int32_t* simp_h) {
    cudaStream_t st = p->setup_stream;
    p->verts.alloc(sizeof(double) * p->nv * p->d);
    p->simp.alloc(sizeof(int32_t) * p->ne * (p->d + 1));
    GOFD_CUDA_TRY(cudaMemcpyAsync(p->verts.ptr, verts_h, sizeof(double) * p->nv * p->d,
                                  cudaMemcpyHostToDevice, st));
    GOFD_CUDA_TRY(cudaMemcpyAsync(p->simp.ptr, simp_h, sizeof(int32_t) * p->ne * (p->d + 1),
                                  cudaMemcpyHostToDevice, st));
    if (p->d == 1) setup_mesh_d<1>(p);
    else if (p->d == 2) setup_mesh_d<2>(p);
    else setup_mesh_d<3>(p);
}

}  // namespace gofd
