// Device helpers shared by the FFT-convolution kernels: complex arithmetic,
// in-register radix-2/4/8/16 DFTs and the shared-memory Stockham pass.
#pragma once

#include "gofd_internal.cuh"

namespace gofd {

// ---------------------------------------------------------------------------
// complex arithmetic
// ---------------------------------------------------------------------------
template <class R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

// ---------------------------------------------------------------------------
// double-float: a real number held as the unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi)/2, about 48 significant bits), for FFTs with FP64
// accuracy at FP32 arithmetic rates.  Sums and products use the error-free
// transformations of Knuth (two-sum: a + b = s + e exactly, six additions)
// and Dekker / FMA (two-product: a b = p + e exactly, p = fl(a b),
// e = fma(a, b, -p)); the result is renormalised with a fast two-sum.  Every
// step is a rounding intrinsic, so that the compiler cannot contract a
// product and a sum into one FMA and lose the exactness the method relies on.
// The sum below adds the two low parts in FP32 ("sloppy" double-float add):
// its error is bounded by about 2^-44 (|x| + |y|), the norm-wise bound an FFT
// needs.
// ---------------------------------------------------------------------------
struct dfl {
    float hi, lo;
};
__host__ __device__ __forceinline__ dfl dfl_from(double d) {
    dfl r;
    r.hi = (float)d;
    r.lo = (float)(d - (double)r.hi);
    return r;
}
__host__ __device__ __forceinline__ double dfl_to(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfl dfl_fast2sum(float s, float e) {   // |s| >= |e|
    dfl r;
    r.hi = __fadd_rn(s, e);
    r.lo = __fadd_rn(e, -__fadd_rn(r.hi, -s));
    return r;
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fadd_rn(s, -a.hi);
    const float e = __fadd_rn(__fadd_rn(a.hi, -__fadd_rn(s, -bb)), __fadd_rn(b.hi, -bb));
    return dfl_fast2sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl{-a.hi, -a.lo}; }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dfl_fast2sum(p, e);
}
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { return a = a * b; }
struct dfc {
    dfl x, y;
};
template <> struct Cplx<dfl> { using T = dfc; };

// storage type of the inputs, weights, symbol and outputs of a transform
// computed in Real: FP64 for double-float, else Real itself
template <class R> struct Sto { using T = R; };
template <> struct Sto<dfl> { using T = double; };
template <class R> __device__ __forceinline__ R from_sto(typename Sto<R>::T v) { return v; }
template <> __device__ __forceinline__ dfl from_sto<dfl>(double v) { return dfl_from(v); }
template <class R> __device__ __forceinline__ typename Sto<R>::T to_sto(R v) { return v; }
template <> __device__ __forceinline__ double to_sto<dfl>(dfl v) { return dfl_to(v); }
template <class R> __device__ __forceinline__ R real_zero() { return R(0); }
template <> __device__ __forceinline__ dfl real_zero<dfl>() { return dfl{0.f, 0.f}; }
template <class R> __device__ __forceinline__ R real_half() { return R(0.5); }
template <> __device__ __forceinline__ dfl real_half<dfl>() { return dfl{0.5f, 0.f}; }

// read-only load of a complex value (a double-float complex as one 16-byte load)
template <class C> __device__ __forceinline__ C cld(const C* p) { return __ldg(p); }
template <> __device__ __forceinline__ dfc cld<dfc>(const dfc* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return dfc{dfl{v.x, v.y}, dfl{v.z, v.w}};
}

template <class C> __device__ __forceinline__ C cmk(double x, double y);
template <> __device__ __forceinline__ float2 cmk<float2>(double x, double y) { return make_float2((float)x, (float)y); }
template <> __device__ __forceinline__ double2 cmk<double2>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ dfc cmk<dfc>(double x, double y) { return dfc{dfl_from(x), dfl_from(y)}; }

template <class C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * conj(b)
template <class C> __device__ __forceinline__ C cmulc(C a, C b) {
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
template <class C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

// shared-memory index with one pad slot per 16 complex entries (bank spread)
__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int spad_len(int n) { return n + (n >> 4) + 1; }

// Row stride of a shared-memory tile holding G lines (G = 1, 2, 4) of len
// complex entries, line after line: len rounded up to 16/G modulo 16.  Then
// both ways the tile is accessed are free of bank conflicts for 8-byte
// entries: one line's consecutive entries, and the tile order in which
// consecutive threads take the G lines' entries of consecutive positions
// (16 threads cover 16/G positions x G lines = 16 distinct slots mod 16).
__host__ __device__ constexpr int tile_ld(int len, int G) { return len + ((((16 / G) & 15) - (len & 15)) & 15); }

// cos / sin of 2 pi k / 16
__host__ __device__ constexpr double cos16(int k) {
    switch (k & 15) {
        case 0: return 1.0;
        case 1: return 0.92387953251128675613;
        case 2: return 0.70710678118654752440;
        case 3: return 0.38268343236508977173;
        case 4: return 0.0;
        case 5: return -0.38268343236508977173;
        case 6: return -0.70710678118654752440;
        case 7: return -0.92387953251128675613;
        case 8: return -1.0;
        case 9: return -0.92387953251128675613;
        case 10: return -0.70710678118654752440;
        case 11: return -0.38268343236508977173;
        case 12: return 0.0;
        case 13: return 0.38268343236508977173;
        case 14: return 0.70710678118654752440;
        default: return 0.92387953251128675613;
    }
}
__host__ __device__ constexpr double sin16(int k) { return cos16(k - 4); }

// multiply by exp(-+ 2 pi i j / 16) (sign by INV); j is a compile-time constant after unrolling
template <bool INV, class C> __device__ __forceinline__ C twc16(C a, int j) {
    j &= 15;
    if (j == 0) return a;
    if (j == 4) {  // -i (forward) or +i (inverse)
        C r;
        if (!INV) { r.x = a.y; r.y = -a.x; } else { r.x = -a.y; r.y = a.x; }
        return r;
    }
    if (j == 8) { a.x = -a.x; a.y = -a.y; return a; }
    if (j == 12) {
        C r;
        if (!INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
        return r;
    }
    double c = cos16(j), s = INV ? sin16(j) : -sin16(j);
    return cmul(a, cmk<C>(c, s));
}

// cos of 2 pi k / 32 for odd k (even k: cos16(k/2))
__host__ __device__ constexpr double cos32_odd(int k) {
    switch (k & 31) {
        case 1: case 31: return 0.98078528040323044913;
        case 3: case 29: return 0.83146961230254523708;
        case 5: case 27: return 0.55557023301960222474;
        case 7: case 25: return 0.19509032201612826785;
        case 9: case 23: return -0.19509032201612826785;
        case 11: case 21: return -0.55557023301960222474;
        case 13: case 19: return -0.83146961230254523708;
        default: return -0.98078528040323044913;   // 15, 17
    }
}

// multiply by exp(-+ 2 pi i j / 32); even j take the 16-point path unchanged
template <bool INV, class C> __device__ __forceinline__ C twc32(C a, int j) {
    j &= 31;
    if ((j & 1) == 0) return twc16<INV>(a, j >> 1);
    const double c = cos32_odd(j), sn = cos32_odd(j - 8);   // sin(2 pi j/32) = cos(2 pi (j-8)/32)
    return cmul(a, cmk<C>(c, INV ? sn : -sn));
}

__host__ __device__ constexpr int bitrev(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

// In-register DFT of length R (power of two <= 32), natural order in and out:
// v[k] <- sum_r v[r] exp(-+2 pi i r k / R).  Radix-2 decimation in frequency,
// then a compile-time bit-reversal permutation.
template <int R, bool INV, class C> __device__ __forceinline__ void dft_reg(C* v) {
    constexpr int LOG = (R == 2) ? 1 : (R == 4) ? 2 : (R == 8) ? 3 : (R == 16) ? 4 : 5;
#pragma unroll
    for (int st = 0; st < LOG; ++st) {
        const int span = R >> (st + 1);
#pragma unroll
        for (int blk = 0; blk < R; blk += 2 * span) {
#pragma unroll
            for (int j = 0; j < span; ++j) {
                C a = v[blk + j], b = v[blk + j + span];
                v[blk + j] = cadd(a, b);
                // twiddle exp(-2 pi i j / (2 span)) = index j * 32 / (2 span) of the 32-table
                v[blk + j + span] = twc32<INV>(csub(a, b), j * (32 / (2 * span)));
            }
        }
    }
    C t[R];
#pragma unroll
    for (int k = 0; k < R; ++k) t[k] = v[bitrev(k, LOG)];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = t[k];
}

// ---------------------------------------------------------------------------
// one line FFT of length N (power of two >= 16) in padded shared memory,
// computed by nthr = N/16 threads (thread index t of the line's group).
// Stockham autosort: pass with radix R reads x[b + r N/R], applies twiddles
// exp(-+2 pi i (b mod Ns) r / (Ns R)), a radix-R DFT, and writes
// y[(b/Ns) Ns R + b mod Ns + r Ns].  The twiddle table holds exp(-2 pi i m / P)
// for m < P; line length N = P / twstride.
// ---------------------------------------------------------------------------
constexpr int FFT_E = 16;

template <int R, bool INV, class C>
__device__ __forceinline__ void stockham_pass(C* buf, int N, int Ns, int t, int nthr, const C* __restrict__ tw,
                                              int twstride, C (&v)[FFT_E]) {
    constexpr int Q = FFT_E / R;
    const int stride_in = N / R;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = t + q * nthr;
#pragma unroll
        for (int r = 0; r < R; ++r) v[q * R + r] = buf[spad(b + r * stride_in)];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = t + q * nthr;
        const int k = b % Ns;
        const int step = (N / (Ns * R)) * twstride;
#pragma unroll
        for (int r = 1; r < R; ++r) {
            if (k != 0) {
                C w = cld(&tw[k * r * step]);
                if (INV) w.y = -w.y;
                v[q * R + r] = cmul(v[q * R + r], w);
            }
        }
        dft_reg<R, INV>(v + q * R);
        const int base = (b / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[spad(base + r * Ns)] = v[q * R + r];
    }
    __syncthreads();
}

template <bool INV, class C>
__device__ __forceinline__ void line_fft(C* buf, const LinePlan& plan, int t, const C* __restrict__ tw,
                                         int twstride) {
    C v[FFT_E];
    int Ns = 1;
    for (int ps = 0; ps < plan.npass; ++ps) {
        const int R = plan.radix[ps];
        if (R == 16) stockham_pass<16, INV>(buf, plan.N, Ns, t, plan.nthr, tw, twstride, v);
        else if (R == 8) stockham_pass<8, INV>(buf, plan.N, Ns, t, plan.nthr, tw, twstride, v);
        else if (R == 4) stockham_pass<4, INV>(buf, plan.N, Ns, t, plan.nthr, tw, twstride, v);
        else stockham_pass<2, INV>(buf, plan.N, Ns, t, plan.nthr, tw, twstride, v);
        Ns *= R;
    }
}


}  // namespace gofd
