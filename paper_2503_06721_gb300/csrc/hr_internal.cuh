// hr_internal.cuh -- shared device/host building blocks of libhr (sm_103a).
//
// Data layout in HBM (private to the library):
//   links   per output parity p, "duplicated" so that every output site finds
//           its 8 hop matrices in one contiguous record:
//             slot k = 0..3 : U_R(x, mu=k)            (forward hop)
//             slot k = 4..7 : U_R(x - mu, mu)^dag     (backward hop, mu = k-4)
//           stored as AoSoA tiles of 32 sites:  [tile][slot][component][lane]
//           (component = complex entry r*D+c, or real entry for the real
//           representations: ADJ and the real-basis SU(4) 2AS).  One warp streams one tile with fully coalesced
//           loads; each link is stored twice (once per endpoint parity), which
//           HBM capacity allows and which turns every link read into a
//           contiguous stream.
//   spinors site-major [site][spin][colour] complex, exactly the ABI layout,
//           read with 16-byte vector loads.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include "hr.h"

#define HR_MAX_N 8
#define HR_TILE 32
#define HR_NPREC 5   // F64, F32, F16, BF16, DF64

namespace hr {

// ---------------------------------------------------------------------------
// complex arithmetic
// ---------------------------------------------------------------------------
template <class R>
struct cx {
    R re, im;
};

template <class R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <class R>
__host__ __device__ __forceinline__ cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
// a += b * c
template <class R>
__host__ __device__ __forceinline__ void cmac(cx<R> &a, cx<R> b, cx<R> c)
{
    a.re = fma(b.re, c.re, a.re);
    a.re = fma(-b.im, c.im, a.re);
    a.im = fma(b.re, c.im, a.im);
    a.im = fma(b.im, c.re, a.im);
}
// a += conj(b) * c
template <class R>
__host__ __device__ __forceinline__ void cmac_cj(cx<R> &a, cx<R> b, cx<R> c)
{
    a.re = fma(b.re, c.re, a.re);
    a.re = fma(b.im, c.im, a.re);
    a.im = fma(b.re, c.im, a.im);
    a.im = fma(-b.im, c.re, a.im);
}
// a += s * c (s real)
template <class R>
__host__ __device__ __forceinline__ void rmac(cx<R> &a, R s, cx<R> c)
{
    a.re = fma(s, c.re, a.re);
    a.im = fma(s, c.im, a.im);
}
// the epilogue forms, each with one fixed rounding sequence so that every
// kernel variant produces the same bits:
//   s*x + t*y  = fma(s, x, t*y) per part;   n2 += |v|^2 as two fmas
template <class R>
__host__ __device__ __forceinline__ cx<R> axpby(R s, cx<R> x, R t, cx<R> y)
{
    cx<R> r = {t * y.re, t * y.im};
    rmac(r, s, x);
    return r;
}
template <class R>
__host__ __device__ __forceinline__ void norm_acc(R &n2, cx<R> v)
{
    n2 = fma(v.re, v.re, n2);
    n2 = fma(v.im, v.im, n2);
}
// s * v with each part rounded once and never fused into a following add:
// the dequantisation of per-site scaled (F16/BF16) values.  Left as a plain
// product, the compiler may contract it into the next addition in one kernel
// variant and not in another; written this way every variant rounds it alike.
__device__ __forceinline__ cx<float> scale_rn(float s, cx<float> v) { return {__fmul_rn(s, v.re), __fmul_rn(s, v.im)}; }

// acc += s * v as two fmas (s real): the hop of a per-site scaled
// (F16/BF16) field projects and multiplies the stored codes and applies the
// neighbour's scale once, here, instead of to every component it loaded
template <class R>
__host__ __device__ __forceinline__ void acc_scaled(cx<R> &acc, R s, cx<R> v)
{
    acc.re = fma(s, v.re, acc.re);
    acc.im = fma(s, v.im, acc.im);
}

// multiply by i^k, k known at compile time after unrolling
template <class R>
__host__ __device__ __forceinline__ cx<R> ipow(int k, cx<R> a)
{
    switch (k & 3) {
    case 0: return a;
    case 1: return {-a.im, a.re};
    case 2: return {-a.re, -a.im};
    default: return {a.im, -a.re};
    }
}

// ---------------------------------------------------------------------------
// float-float ("df64") numbers: value = hi + lo with |lo| <= ulp(hi)/2, about
// 48 significant bits.  Sums use Knuth's TwoSum, products the FMA-based exact
// product (Dekker's TwoProduct with a fused multiply-add), then a fast
// renormalisation.  GB300 executes FP32 FMAs at many times its FP64 rate, so
// FP64-class accuracy for the operator costs far less in float-float.
// ---------------------------------------------------------------------------
// the float-float overloads below join the standard ones instead of hiding them
using ::fma;
using ::isfinite;

// ---------------------------------------------------------------------------
// FP64 <-> FP32 conversions from the IEEE 754 bit patterns.  GB300 executes
// F2F conversions to and from 64-bit types at its FP64 rate (measured: about
// 1.8 per clock per SM, like a DFMA, against 109 FP32 FMAs), so the hot paths
// convert with integer and FP32 operations instead.  Each function returns
// exactly what the hardware conversion returns -- binary64 -> binary32 with
// round to nearest, ties to even; binary32 -> binary64 exactly -- handling
// zeros by their bits and handing the cases it does not treat (subnormal
// inputs or results, overflow, Inf, NaN) to the hardware conversion.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ unsigned long long bits_of(double v)
{
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(v);
#else
    unsigned long long u;
    memcpy(&u, &v, 8);
    return u;
#endif
}
__host__ __device__ __forceinline__ double double_of(unsigned long long u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double v;
    memcpy(&v, &u, 8);
    return v;
#endif
}
__host__ __device__ __forceinline__ float float_of(unsigned u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
__host__ __device__ __forceinline__ unsigned fbits_of(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    unsigned u;
    memcpy(&u, &f, 4);
    return u;
#endif
}

// binary64 -> binary32, round to nearest even.  The 52-bit significand keeps
// its top 23 bits; the 29 dropped bits decide the rounding (above half, or
// exactly half with an odd last kept bit, rounds up, and the carry runs into
// the exponent field, up to Inf).  Biased exponents e = 897 .. 1150 give
// normal results; every other e goes to the hardware.
__host__ __device__ __forceinline__ float f32_rn(double v)
{
    const unsigned long long u = bits_of(v);
    const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
    const unsigned e = (hw >> 20) & 0x7FFu;
    if (e - 897u > 253u) {
        if ((u << 1) == 0) return float_of(hw & 0x80000000u);   // +-0
        return (float)v;
    }
    const unsigned m = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    const unsigned rest = lw & 0x1FFFFFFFu;
    const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return float_of((hw & 0x80000000u) | (((e - 896u) << 23) + m + up));
}

// binary32 -> binary64 (exact): rebias the exponent, shift the significand
__host__ __device__ __forceinline__ double f64_of(float f)
{
    const unsigned u = fbits_of(f);
    const unsigned e = (u >> 23) & 0xFFu;
    if (e - 1u > 253u) {
        if ((u << 1) == 0) return double_of((unsigned long long)(u & 0x80000000u) << 32);   // +-0
        return (double)f;
    }
    const unsigned hw = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return double_of(((unsigned long long)hw << 32) | (unsigned long long)(u << 29));
}

struct df;
__host__ __device__ df df_split(double v);

struct df {
    float hi, lo;
    __host__ __device__ df() : hi(0.f), lo(0.f) {}
    __host__ __device__ df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ df(int v) : hi((float)v), lo(0.f) {}
    // hi = fl32(v), lo = fl32(v - hi) (df_split)
    __host__ __device__ df(double v);
    // hi + lo, exact in FP64 (|lo| <= ulp(hi) / 2): one FP64 addition
    __host__ __device__ explicit operator double() const { return f64_of(hi) + f64_of(lo); }
};

// the split of a double into hi = fl32(v) and lo = fl32(v - hi), without
// FP64 arithmetic: with hi from f32_rn, v - hi = rem 2^(E-52) exactly, where
// rem (|rem| <= 2^28) is the dropped 29-bit remainder, less 2^29 when hi was
// rounded up; rem = a 2^13 + b in two exactly representable floats, one fma
// rounds it once, and the power of two 2^(E-52) scales it exactly.  Biased
// exponents e = 949 .. 1149 (|v| about 2^-74 .. 2^127) take this path.
__host__ __device__ __forceinline__ df df_split(double v)
{
    const unsigned long long u = bits_of(v);
    const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
    const unsigned e = (hw >> 20) & 0x7FFu;
    if (e - 949u > 200u) {
        if ((u << 1) == 0) return df(float_of(hw & 0x80000000u), 0.f);   // +-0
        const float h = (float)v;
        return df(h, (float)(v - (double)h));
    }
    const unsigned m = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    const unsigned rest = lw & 0x1FFFFFFFu;
    const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    const unsigned sign = hw & 0x80000000u;
    const float hi = float_of(sign | (((e - 896u) << 23) + m + up));
    const int rem = (int)rest - (int)(up << 29);
    const int a = rem >> 13;                 // |a| <= 2^15
    const unsigned b = (unsigned)rem & 0x1FFFu;
    const float af = float_of(0x4B400000u + (unsigned)a) - 12582912.0f;   // 1.5 * 2^23 + a, exact
    const float bf = float_of(0x4B000000u | b) - 8388608.0f;              // 2^23 + b, exact
    const float lo = fmaf(af, 8192.0f, bf) * float_of((e - 948u) << 23);
    // v - hi carries the sign of v, but an exact zero difference is +0
    return df(hi, rem ? float_of(fbits_of(lo) ^ sign) : 0.f);
}
__host__ __device__ inline df::df(double v)
{
    const df t = df_split(v);
    hi = t.hi;
    lo = t.lo;
}
__host__ __device__ __forceinline__ df df_qts(float a, float b)   // |a| >= |b|
{
    const float s = a + b;
    return df(s, b - (s - a));
}
__host__ __device__ __forceinline__ df df_ts(float a, float b, float &err)
{
    const float s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
    return df(s, 0.f);
}
__host__ __device__ __forceinline__ df operator+(df a, df b)
{
    float e;
    const df s = df_ts(a.hi, b.hi, e);
    return df_qts(s.hi, e + a.lo + b.lo);
}
__host__ __device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__host__ __device__ __forceinline__ df operator*(df a, df b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_qts(p, e);
}
// a * b + c with one renormalisation
__host__ __device__ __forceinline__ df fma(df a, df b, df c)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float t;
    const df s = df_ts(p, c.hi, t);
    return df_qts(s.hi, t + c.lo + e);
}
__host__ __device__ __forceinline__ bool isfinite(df a) { return isfinite(a.hi); }

// a double in real type R (float: rounded to nearest even; df: split) and back
template <class R>
__host__ __device__ __forceinline__ R from_f64(double v);
template <>
__host__ __device__ __forceinline__ double from_f64<double>(double v) { return v; }
template <>
__host__ __device__ __forceinline__ float from_f64<float>(double v) { return f32_rn(v); }
template <>
__host__ __device__ __forceinline__ df from_f64<df>(double v) { return df_split(v); }
__host__ __device__ __forceinline__ double to_f64(double v) { return v; }
__host__ __device__ __forceinline__ double to_f64(float v) { return f64_of(v); }
__host__ __device__ __forceinline__ double to_f64(df v) { return (double)v; }

// ---------------------------------------------------------------------------
// representations (Table 1) -- compile-time structure
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int rep_dim(int N, int rep)
{
    return rep == HR_FUND ? N : rep == HR_ADJ ? N * N - 1 : rep == HR_SYM ? N * (N + 1) / 2 : N * (N - 1) / 2;
}
// (N, representation) pairs whose hop runs on the colour-parallel kernel:
// the fundamental for N >= 5, the SU(4) adjoint (D_R = 15) and symmetric
// (D_R = 10) representations
__host__ __device__ constexpr bool colour_pair(int N, int rep)
{
    return N >= 5 || (N == 4 && (rep == HR_ADJ || rep == HR_SYM));
}
// representations whose links are real in the library's basis (stored as reals)
__host__ __device__ constexpr bool rep_real(int rep) { return rep == HR_ADJ || rep == HR_ASYM_REAL; }

// the p-th pair (j,k), j<k, in lexicographic order
__host__ __device__ constexpr int pair_j(int N, int p)
{
    int j = 0;
    while (p >= N - 1 - j) { p -= N - 1 - j; j++; }
    return j;
}
__host__ __device__ constexpr int pair_k(int N, int p)
{
    int j = 0;
    while (p >= N - 1 - j) { p -= N - 1 - j; j++; }
    return j + 1 + p;
}
// the n-th pair (i,j), i<=j (SYM) or i<j (ASYM), in lexicographic order
__host__ __device__ constexpr int sympair_i(int N, int n, bool strict)
{
    int i = 0;
    while (true) {
        int cnt = strict ? N - 1 - i : N - i;
        if (n < cnt) return i;
        n -= cnt;
        i++;
    }
}
__host__ __device__ constexpr int sympair_j(int N, int n, bool strict)
{
    int i = 0;
    while (true) {
        int cnt = strict ? N - 1 - i : N - i;
        if (n < cnt) return i + (strict ? 1 : 0) + n;
        n -= cnt;
        i++;
    }
}

// ---------------------------------------------------------------------------
// gamma basis of Sec. 2.2: gamma_mu = [[0, e_mu], [e_mu^dag, 0]],
// e_0 = -1, e_i = -i sigma_i.  Each e_mu has one nonzero per row:
//   (e_mu)_{r, eperm(mu,r)} = i^{ephase(mu,r)}.
// A projector (1 + s gamma_mu) acting on psi = (up, dn) gives
//   h = up + s e dn,   lower = s e^dag h,
// so only the two "upper" spin components h_0, h_1 are multiplied by the
// colour matrix (the half-spinor of Sec. 3.5).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int eperm(int mu, int r) { return (mu == 1 || mu == 2) ? 1 - r : r; }
__host__ __device__ constexpr int ephase(int mu, int r)
{
    // e_0: -1,-1   e_1: -i,-i   e_2: -1,+1   e_3: -i,+i   (as powers of i)
    return mu == 0 ? 2 : mu == 1 ? 3 : mu == 2 ? (r == 0 ? 2 : 0) : (r == 0 ? 3 : 1);
}

// ---------------------------------------------------------------------------
// storage traits
// ---------------------------------------------------------------------------
template <int P>
struct St;
template <>
struct St<HR_F64> {
    using R = double;       // compute type
    using C = double2;      // stored complex
    using Rs = double;      // stored real
    static constexpr bool scaled = false;
    __device__ __forceinline__ static cx<R> ld(C v) { return {v.x, v.y}; }
    __device__ __forceinline__ static C st(cx<R> v) { return make_double2(v.re, v.im); }
    __device__ __forceinline__ static R ldr(Rs v) { return v; }
    __host__ __device__ __forceinline__ static Rs str(double v) { return v; }
};
template <>
struct St<HR_F32> {
    using R = float;
    using C = float2;
    using Rs = float;
    static constexpr bool scaled = false;
    __device__ __forceinline__ static cx<R> ld(C v) { return {v.x, v.y}; }
    __device__ __forceinline__ static C st(cx<R> v) { return make_float2(v.re, v.im); }
    __device__ __forceinline__ static R ldr(Rs v) { return v; }
    __host__ __device__ __forceinline__ static Rs str(double v) { return f32_rn(v); }
};
template <>
struct St<HR_F16> {
    using R = float;
    using C = __half2;
    using Rs = __half;
    static constexpr bool scaled = true;
    __device__ __forceinline__ static cx<R> ld(C v)
    {
        float2 f = __half22float2(v);
        return {f.x, f.y};
    }
    __device__ __forceinline__ static C st(cx<R> v) { return __floats2half2_rn(v.re, v.im); }
    __device__ __forceinline__ static R ldr(Rs v) { return __half2float(v); }
    __device__ __forceinline__ static Rs str(double v) { return __double2half(v); }
};
template <>
struct St<HR_BF16> {
    using R = float;
    using C = __nv_bfloat162;
    using Rs = __nv_bfloat16;
    static constexpr bool scaled = true;
    __device__ __forceinline__ static cx<R> ld(C v)
    {
        float2 f = __bfloat1622float2(v);
        return {f.x, f.y};
    }
    __device__ __forceinline__ static C st(cx<R> v) { return __floats2bfloat162_rn(v.re, v.im); }
    __device__ __forceinline__ static R ldr(Rs v) { return __bfloat162float(v); }
    __device__ __forceinline__ static Rs str(double v) { return __double2bfloat16(v); }
};

template <>
struct St<HR_DF64> {
    using R = df;
    using C = float4;   // (re.hi, re.lo, im.hi, im.lo)
    using Rs = float2;  // (hi, lo)
    static constexpr bool scaled = false;
    __device__ __forceinline__ static cx<R> ld(C v) { return {df(v.x, v.y), df(v.z, v.w)}; }
    __device__ __forceinline__ static C st(cx<R> v) { return make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo); }
    __device__ __forceinline__ static R ldr(Rs v) { return df(v.x, v.y); }
    __host__ __device__ __forceinline__ static Rs str(double v)
    {
        const df d(v);
        return make_float2(d.hi, d.lo);
    }
};

__host__ __device__ constexpr size_t prec_cbytes(int P) { return (P == HR_F64 || P == HR_DF64) ? 16 : P == HR_F32 ? 8 : 4; }
__host__ __device__ constexpr size_t prec_rbytes(int P) { return (P == HR_F64 || P == HR_DF64) ? 8 : P == HR_F32 ? 4 : 2; }

static inline size_t align_up(size_t n, size_t a) { return (n + a - 1) / a * a; }

// byte size of one right-hand side of a spinor field of nsites sites
static inline size_t field_rhs_bytes(long nsites, int D, int P)
{
    size_t data = (size_t)nsites * 4 * D * prec_cbytes(P);
    if (P == HR_F16 || P == HR_BF16) return align_up(data, 256) + align_up((size_t)nsites * 4, 256);
    return data;
}
static inline size_t field_scale_offset(long nsites, int D, int P)
{
    return align_up((size_t)nsites * 4 * D * prec_cbytes(P), 256);
}

// ---------------------------------------------------------------------------
// lattice geometry on the device
// ---------------------------------------------------------------------------
struct Geom {
    int T, X, Y, Z, hz;   // hz = Z/2
    long vh;              // sites per parity
    long ntiles;          // ceil(vh / 32)
    int bc[4];
};

struct Site {
    int c[4];     // t, x, y, z
    long row;     // (t*X + x)*Y + y
};

__device__ __forceinline__ Site site_of(const Geom &g, long i, int parity)
{
    Site s;
    int zh = (int)(i % g.hz);
    long r = i / g.hz;
    s.row = r;
    s.c[2] = (int)(r % g.Y);
    r /= g.Y;
    s.c[1] = (int)(r % g.X);
    s.c[0] = (int)(r / g.X);
    int rp = (s.c[0] + s.c[1] + s.c[2]) & 1;
    s.c[3] = 2 * zh + (parity ^ rp);
    return s;
}

// half index (inside the opposite parity) of the neighbour x + dir*mu
__device__ __forceinline__ long neighbour(const Geom &g, const Site &s, int mu, int dir)
{
    int t = s.c[0], x = s.c[1], y = s.c[2], z = s.c[3];
    if (mu == 3) {
        z += dir;
        z = z < 0 ? z + g.Z : (z >= g.Z ? z - g.Z : z);
        return s.row * g.hz + (z >> 1);
    }
    if (mu == 0) { t += dir; t = t < 0 ? t + g.T : (t >= g.T ? t - g.T : t); }
    if (mu == 1) { x += dir; x = x < 0 ? x + g.X : (x >= g.X ? x - g.X : x); }
    if (mu == 2) { y += dir; y = y < 0 ? y + g.Y : (y >= g.Y ? y - g.Y : y); }
    return (((long)t * g.X + x) * g.Y + y) * g.hz + (z >> 1);
}

// lexicographic index of a site
__device__ __forceinline__ long lex_of(const Geom &g, const Site &s)
{
    return s.row * g.Z + s.c[3];
}

// ---------------------------------------------------------------------------
// reductions: warp / block tree in double, grid level in double-double
// (compensated, Sec. 4.1.1); the last block to finish combines the per-block
// partials in a fixed order, so results are deterministic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV])
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < NV; k++) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
}

// Block-reduces v (all threads must call), stores the block's partial, and
// returns true in thread 0 of the last block to finish, with the grid total
// (double-double combined over blocks) in tot.  partials: [nblocks][NV],
// counter: one unsigned, reset to 0 by the last block.  blockDim.x <= 256.
template <int NV>
__device__ bool grid_reduce(double (&v)[NV], double *partials, unsigned *counter, int nblocks,
                            int block, double (&tot)[NV])
{
    __shared__ double sm[32][NV];
    __shared__ bool last;
    warp_sum<NV>(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) sm[wid][k] = v[k];
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (threadIdx.x == 0) {
        double s[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) s[k] = 0;
        for (int w = 0; w < nw; w++)
#pragma unroll
            for (int k = 0; k < NV; k++) s[k] += sm[w][k];
#pragma unroll
        for (int k = 0; k < NV; k++) partials[(size_t)block * NV + k] = s[k];
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == (unsigned)nblocks - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // last block: thread t sums blocks t, t+bd, ... in double-double
    double hi[NV], lo[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) { hi[k] = 0; lo[k] = 0; }
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double s, e;
            two_sum(hi[k], __ldcg(&partials[(size_t)b * NV + k]), s, e);
            hi[k] = s;
            lo[k] += e;
        }
    __shared__ double shi[256][NV];
    __shared__ double slo[256][NV];
#pragma unroll
    for (int k = 0; k < NV; k++) { shi[threadIdx.x][k] = hi[k]; slo[threadIdx.x][k] = lo[k]; }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double h = 0, l = 0;
            for (int t = 0; t < (int)blockDim.x; t++) {
                double s, e;
                two_sum(h, shi[t][k], s, e);
                h = s;
                l += e + slo[t][k];
            }
            tot[k] = h + l;
        }
        *counter = 0;
    }
    return threadIdx.x == 0;
}

// ---------------------------------------------------------------------------
// solver state kept on the device (one per right-hand side)
// ---------------------------------------------------------------------------
struct CgState {
    double rr;        // |r|^2
    double pAp;       // |Dhat p|^2 = <p, A p>
    double alpha, beta;
    double stop2;     // converge when rr <= stop2
    double b2;        // |b|^2
    int converged;
    int nonfinite;
    int iter;         // iterations done in the current (inner) solve
    int cap;          // iteration cap of the current (inner) solve
};

// a right-hand side takes no further iteration once it converged or hit its cap
__host__ __device__ __forceinline__ bool cg_idle(const CgState &s) { return s.converged || s.iter >= s.cap; }

// ---------------------------------------------------------------------------
// host-side helpers
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
hr_status cuda_fail(cudaError_t e, const char *what);
void count_launch(long long n = 1);

#define HR_CUDA_CHECK(call)                                        \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::hr::cuda_fail(_e, #call); \
    } while (0)

#define HR_LAUNCH_CHECK(what)                                      \
    do {                                                           \
        ::hr::count_launch();                                      \
        cudaError_t _e = cudaGetLastError();                       \
        if (_e != cudaSuccess) return ::hr::cuda_fail(_e, what);   \
    } while (0)

}  // namespace hr
