// Exact orientation signs for point location.
//
// A float evaluation decides when |det| exceeds a forward error bound; the
// rest is evaluated exactly with floating-point expansion arithmetic
// (error-free two-sum and FMA-based two-product, summed by grow-expansion;
// Priest 1991, Shewchuk 1997).  All arithmetic uses explicit round-to-nearest
// intrinsics so that no contraction into FMA changes the error analysis.
// Valid for coordinates whose differences and products neither overflow nor
// underflow (|x| < 1e100 and no differences below 1e-100).
#pragma once

#include <cuda_runtime.h>

namespace gofd {

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

__device__ __forceinline__ void two_diff(double a, double b, double& s, double& e) {
    two_sum(a, -b, s, e);
}

__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
    p = __dmul_rn(a, b);
    e = __fma_rn(a, b, -p);
}

// h <- e + b, in place on e (length *len, capacity >= *len + 1), zero components dropped.
__device__ __forceinline__ void grow_expansion(double* e, int* len, double b) {
    double q = b;
    int out = 0;
    for (int i = 0; i < *len; ++i) {
        double s, err;
        two_sum(q, e[i], s, err);
        q = s;
        if (err != 0.0) e[out++] = err;
    }
    if (q != 0.0 || out == 0) e[out++] = q;
    *len = out;
}

__device__ __forceinline__ int expansion_sign(const double* e, int len) {
    for (int i = len - 1; i >= 0; --i) {
        if (e[i] > 0.0) return 1;
        if (e[i] < 0.0) return -1;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// 1D: sign(b - a) is exact in IEEE arithmetic
// ---------------------------------------------------------------------------
__device__ __forceinline__ int orient1_sign(double a, double b) {
    double d = __dsub_rn(b, a);
    return (d > 0.0) - (d < 0.0);
}

// ---------------------------------------------------------------------------
// 2D: det[a - c; b - c]
// ---------------------------------------------------------------------------
__device__ __noinline__ int orient2_exact(const double* a, const double* b, const double* c) {
    double acx, acxt, bcy, bcyt, acy, acyt, bcx, bcxt;
    two_diff(a[0], c[0], acx, acxt);
    two_diff(b[1], c[1], bcy, bcyt);
    two_diff(a[1], c[1], acy, acyt);
    two_diff(b[0], c[0], bcx, bcxt);
    double l[2] = {acx, acxt}, r[2] = {bcy, bcyt};
    double l2[2] = {acy, acyt}, r2[2] = {bcx, bcxt};
    double e[20];
    int len = 0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double p, q;
            two_prod(l[i], r[j], p, q);
            grow_expansion(e, &len, q);
            grow_expansion(e, &len, p);
            two_prod(l2[i], r2[j], p, q);
            grow_expansion(e, &len, -q);
            grow_expansion(e, &len, -p);
        }
    return expansion_sign(e, len);
}

__device__ __forceinline__ double orient2_value(const double* a, const double* b, const double* c,
                                                double* perm) {
    double acx = __dsub_rn(a[0], c[0]), bcy = __dsub_rn(b[1], c[1]);
    double acy = __dsub_rn(a[1], c[1]), bcx = __dsub_rn(b[0], c[0]);
    double l = __dmul_rn(acx, bcy), r = __dmul_rn(acy, bcx);
    *perm = __dadd_rn(fabs(l), fabs(r));
    return __dsub_rn(l, r);
}

__device__ __forceinline__ int orient2_sign(const double* a, const double* b, const double* c) {
    double perm;
    double det = orient2_value(a, b, c, &perm);
    const double bound = 8.0 * 1.1102230246251565e-16;  // 8 * 2^-53
    if (det > bound * perm) return 1;
    if (-det > bound * perm) return -1;
    return orient2_exact(a, b, c);
}

// ---------------------------------------------------------------------------
// 3D: det[a - d; b - d; c - d]
// ---------------------------------------------------------------------------
__device__ __noinline__ int orient3_exact(const double* a, const double* b, const double* c,
                                          const double* d) {
    double m[3][3][2];
    const double* rows[3] = {a, b, c};
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) two_diff(rows[i][k], d[k], m[i][k][0], m[i][k][1]);
    const int perms[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
    const double sgn[6] = {1, 1, 1, -1, -1, -1};
    double e[200];
    int len = 0;
    for (int t = 0; t < 6; ++t) {
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v)
                for (int w = 0; w < 2; ++w) {
                    double x = m[0][perms[t][0]][u], y = m[1][perms[t][1]][v],
                           z = m[2][perms[t][2]][w];
                    double p, pe, q0, q1, r0, r1;
                    two_prod(x, y, p, pe);
                    two_prod(p, z, q0, q1);
                    two_prod(pe, z, r0, r1);
                    grow_expansion(e, &len, sgn[t] * r1);
                    grow_expansion(e, &len, sgn[t] * q1);
                    grow_expansion(e, &len, sgn[t] * r0);
                    grow_expansion(e, &len, sgn[t] * q0);
                }
    }
    return expansion_sign(e, len);
}

__device__ __forceinline__ double orient3_value(const double* a, const double* b, const double* c,
                                                const double* d, double* perm) {
    double adx = __dsub_rn(a[0], d[0]), ady = __dsub_rn(a[1], d[1]), adz = __dsub_rn(a[2], d[2]);
    double bdx = __dsub_rn(b[0], d[0]), bdy = __dsub_rn(b[1], d[1]), bdz = __dsub_rn(b[2], d[2]);
    double cdx = __dsub_rn(c[0], d[0]), cdy = __dsub_rn(c[1], d[1]), cdz = __dsub_rn(c[2], d[2]);
    double t1 = __dmul_rn(bdy, cdz), t2 = __dmul_rn(bdz, cdy);
    double t3 = __dmul_rn(cdy, adz), t4 = __dmul_rn(cdz, ady);
    double t5 = __dmul_rn(ady, bdz), t6 = __dmul_rn(adz, bdy);
    double det = __dadd_rn(__dadd_rn(__dmul_rn(adx, __dsub_rn(t1, t2)),
                                     __dmul_rn(bdx, __dsub_rn(t3, t4))),
                           __dmul_rn(cdx, __dsub_rn(t5, t6)));
    *perm = __dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(fabs(t1), fabs(t2)), fabs(adx)),
                                __dmul_rn(__dadd_rn(fabs(t3), fabs(t4)), fabs(bdx))),
                      __dmul_rn(__dadd_rn(fabs(t5), fabs(t6)), fabs(cdx)));
    return det;
}

__device__ __forceinline__ int orient3_sign(const double* a, const double* b, const double* c,
                                            const double* d) {
    double perm;
    double det = orient3_value(a, b, c, d, &perm);
    const double bound = 16.0 * 1.1102230246251565e-16;  // 16 * 2^-53
    if (det > bound * perm) return 1;
    if (-det > bound * perm) return -1;
    return orient3_exact(a, b, c, d);
}

// ---------------------------------------------------------------------------
// orientation of d+1 points p[0..d] (each p[i] points at d doubles)
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ int orient_sign(const double* const* p) {
    if constexpr (D == 1) return orient1_sign(p[0][0], p[1][0]);
    else if constexpr (D == 2) return orient2_sign(p[0], p[1], p[2]);
    else return orient3_sign(p[0], p[1], p[2], p[3]);
}

template <int D>
__device__ __forceinline__ double orient_value(const double* const* p) {
    double perm;
    if constexpr (D == 1) return __dsub_rn(p[1][0], p[0][0]);
    else if constexpr (D == 2) return orient2_value(p[0], p[1], p[2], &perm);
    else return orient3_value(p[0], p[1], p[2], p[3], &perm);
}

}  // namespace gofd
