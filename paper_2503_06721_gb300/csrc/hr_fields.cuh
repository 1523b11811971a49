// hr_fields.cuh -- device access to spinor fields and link records.
#pragma once

#include "hr_internal.cuh"

namespace hr {

// One parity (or full) spinor field: data [nrhs][nsites][4][D] in precision
// P, and for F16/BF16 a float scale per site.  rhs_stride is in bytes and
// applies to both data and scale (each right-hand side is one block).
struct FieldView {
    char *data;
    char *scale;   // byte pointer to the first float scale (F16/BF16 only)
    size_t rhs_stride;
};

template <int P, int D>
struct SpinorIO {
    using S = St<P>;
    using R = typename S::R;
    static constexpr int NC = 4 * D;                    // complex components per site
    static constexpr int BYTES = NC * (int)prec_cbytes(P);
    static constexpr int NV = BYTES / 16;               // 16-byte vectors per site
    static_assert(BYTES % 16 == 0, "spinor record must be a multiple of 16 bytes");

    __device__ __forceinline__ static const uint4 *site_ptr(const FieldView &f, int rhs, long i)
    {
        return reinterpret_cast<const uint4 *>(f.data + (size_t)rhs * f.rhs_stride + (size_t)i * BYTES);
    }
    __device__ __forceinline__ static float ld_scale(const FieldView &f, int rhs, long i)
    {
        if constexpr (S::scaled)
            return __ldg(reinterpret_cast<const float *>(f.scale + (size_t)rhs * f.rhs_stride) + i);
        else
            return 1.0f;
    }

    // component n of a site from its raw 16-byte vectors
    __device__ __forceinline__ static cx<R> comp(const uint4 (&raw)[NV], int n)
    {
        if constexpr (P == HR_F64) {
            const uint4 &v = raw[n];
            return {__hiloint2double((int)v.y, (int)v.x), __hiloint2double((int)v.w, (int)v.z)};
        } else if constexpr (P == HR_DF64) {
            const uint4 &v = raw[n];
            return {df(__uint_as_float(v.x), __uint_as_float(v.y)), df(__uint_as_float(v.z), __uint_as_float(v.w))};
        } else if constexpr (P == HR_F32) {
            const uint4 &v = raw[n >> 1];
            return (n & 1) ? cx<R>{__uint_as_float(v.z), __uint_as_float(v.w)}
                           : cx<R>{__uint_as_float(v.x), __uint_as_float(v.y)};
        } else {
            const uint4 &v = raw[n >> 2];
            unsigned w = (n & 3) == 0 ? v.x : (n & 3) == 1 ? v.y : (n & 3) == 2 ? v.z : v.w;
            typename S::C h;
            static_assert(sizeof(h) == 4, "packed pair");
            memcpy(&h, &w, 4);
            return S::ld(h);
        }
    }

    __device__ __forceinline__ static void load(const FieldView &f, int rhs, long i, cx<R> (&psi)[4][D])
    {
        const uint4 *p = site_ptr(f, rhs, i);
        uint4 raw[NV];
#pragma unroll
        for (int j = 0; j < NV; j++) raw[j] = __ldg(p + j);
        R sc = (R)ld_scale(f, rhs, i);
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) {
                cx<R> v = comp(raw, s * D + c);
                if constexpr (S::scaled) v = scale_rn(sc, v);
                psi[s][c] = v;
            }
    }

    // the stored values without the site scale (the codes of F16/BF16 fields)
    __device__ __forceinline__ static void load_codes(const FieldView &f, int rhs, long i, cx<R> (&psi)[4][D])
    {
        const uint4 *p = site_ptr(f, rhs, i);
        uint4 raw[NV];
#pragma unroll
        for (int j = 0; j < NV; j++) raw[j] = __ldg(p + j);
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) psi[s][c] = comp(raw, s * D + c);
    }

    // plain (non-caching-hint) load for fields this kernel may also write
    __device__ __forceinline__ static void load_rw(const FieldView &f, int rhs, long i, cx<R> (&psi)[4][D])
    {
        const uint4 *p = site_ptr(f, rhs, i);
        uint4 raw[NV];
#pragma unroll
        for (int j = 0; j < NV; j++) raw[j] = p[j];
        R sc = (R)ld_scale(f, rhs, i);
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) {
                cx<R> v = comp(raw, s * D + c);
                if constexpr (S::scaled) v = scale_rn(sc, v);
                psi[s][c] = v;
            }
    }

    // one spin component (D complex numbers) of a site; sc = the site's scale
    // for F16/BF16 (ignored otherwise)
    __device__ __forceinline__ static void load_spin(const FieldView &f, int rhs, long i, int s, R sc,
                                                     cx<R> (&v)[D])
    {
        const char *b = f.data + (size_t)rhs * f.rhs_stride + (size_t)i * BYTES + (size_t)s * D * prec_cbytes(P);
#pragma unroll
        for (int c = 0; c < D; c++) {
            if constexpr (P == HR_F64) {
                const double2 d = *reinterpret_cast<const double2 *>(b + 16 * c);
                v[c] = {d.x, d.y};
            } else if constexpr (P == HR_DF64) {
                v[c] = S::ld(*reinterpret_cast<const float4 *>(b + 16 * c));
            } else if constexpr (P == HR_F32) {
                const float2 d = *reinterpret_cast<const float2 *>(b + 8 * c);
                v[c] = {d.x, d.y};
            } else {
                v[c] = scale_rn(sc, S::ld(*reinterpret_cast<const typename S::C *>(b + 4 * c)));
            }
        }
    }
    // one spin component of an unscaled (F64 / F32) site
    __device__ __forceinline__ static void store_spin(const FieldView &f, int rhs, long i, int s, const cx<R> (&v)[D])
    {
        static_assert(!S::scaled, "per-spin stores need an unscaled precision");
        char *b = f.data + (size_t)rhs * f.rhs_stride + (size_t)i * BYTES + (size_t)s * D * prec_cbytes(P);
#pragma unroll
        for (int c = 0; c < D; c++) {
            if constexpr (P == HR_F64)
                *reinterpret_cast<double2 *>(b + 16 * c) = make_double2(v[c].re, v[c].im);
            else if constexpr (P == HR_DF64)
                *reinterpret_cast<float4 *>(b + 16 * c) = S::st(v[c]);
            else
                *reinterpret_cast<float2 *>(b + 8 * c) = make_float2(v[c].re, v[c].im);
        }
    }

    __device__ __forceinline__ static void store(const FieldView &f, int rhs, long i, const cx<R> (&psi)[4][D])
    {
        uint4 raw[NV];
        R inv = 1;
        if constexpr (S::scaled) {
            R m = 0;
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < D; c++) m = fmaxf(m, fmaxf(fabsf(psi[s][c].re), fabsf(psi[s][c].im)));
            *(reinterpret_cast<float *>(f.scale + (size_t)rhs * f.rhs_stride) + i) = m;
            inv = m > 0 ? (R)1 / m : (R)0;
        }
#pragma unroll
        for (int n = 0; n < NC; n++) {
            cx<R> v = psi[n / D][n % D];
            if constexpr (P == HR_F64) {
                raw[n].x = (unsigned)__double2loint(v.re);
                raw[n].y = (unsigned)__double2hiint(v.re);
                raw[n].z = (unsigned)__double2loint(v.im);
                raw[n].w = (unsigned)__double2hiint(v.im);
            } else if constexpr (P == HR_DF64) {
                raw[n] = make_uint4(__float_as_uint(v.re.hi), __float_as_uint(v.re.lo), __float_as_uint(v.im.hi),
                                    __float_as_uint(v.im.lo));
            } else if constexpr (P == HR_F32) {
                if (n & 1) {
                    raw[n >> 1].z = __float_as_uint(v.re);
                    raw[n >> 1].w = __float_as_uint(v.im);
                } else {
                    raw[n >> 1].x = __float_as_uint(v.re);
                    raw[n >> 1].y = __float_as_uint(v.im);
                }
            } else {
                typename S::C h = S::st(inv * v);
                unsigned w;
                memcpy(&w, &h, 4);
                if ((n & 3) == 0) raw[n >> 2].x = w;
                if ((n & 3) == 1) raw[n >> 2].y = w;
                if ((n & 3) == 2) raw[n >> 2].z = w;
                if ((n & 3) == 3) raw[n >> 2].w = w;
            }
        }
        uint4 *p = const_cast<uint4 *>(site_ptr(f, rhs, i));
#pragma unroll
        for (int j = 0; j < NV; j++) p[j] = raw[j];
    }
};

// Link records: AoSoA [tile][slot 0..7][chunk][lane 0..31] of 16-byte chunks.
// Chunk j of a lane holds the slot's components j*VPC .. j*VPC+VPC-1 (VPC =
// 16 bytes / component bytes; the last chunk is zero-padded), so a warp reads
// 512 contiguous bytes per load instruction whatever the precision.
__host__ __device__ constexpr int link_elem_bytes(int P, bool real) { return real ? (int)prec_rbytes(P) : (int)prec_cbytes(P); }
__host__ __device__ constexpr int link_vpc(int P, bool real) { return 16 / link_elem_bytes(P, real); }
__host__ __device__ constexpr int link_nchunk(int P, bool real, int ncomp)
{
    return (ncomp + link_vpc(P, real) - 1) / link_vpc(P, real);
}
// Row stride (in components) of the stored D_R x D_R links: D_R, except for
// the pairs run by the colour-parallel kernel, where each thread reads one
// row: there the rows are padded to whole 16-byte chunks, so that a row
// never straddles a chunk boundary and each thread loads exactly its row
// (D_R = 5 complex FP32 rows take 3 chunks instead of up to 4, the real
// D_R = 15 adjoint rows of SU(4) 4 instead of up to 5).  Component (a, b) of
// a link is stored at a * stride + b; the padding is never read.
__host__ __device__ constexpr int link_row_stride(int N, int rep, int P)
{
    return colour_pair(N, rep) ? (rep_dim(N, rep) + link_vpc(P, rep_real(rep)) - 1) / link_vpc(P, rep_real(rep)) *
                                     link_vpc(P, rep_real(rep))
                               : rep_dim(N, rep);
}

// byte offset of component c of (tile, slot, lane) in a record of ncomp components
__host__ __device__ inline size_t link_offset(int P, bool real, int ncomp, long tile, int slot, int lane, int c)
{
    const int vpc = link_vpc(P, real), nch = link_nchunk(P, real, ncomp);
    return ((((size_t)tile * 8 + slot) * nch + c / vpc) * HR_TILE + lane) * 16 + (size_t)(c % vpc) * link_elem_bytes(P, real);
}

template <int P, bool REAL, int NCOMP>
struct LinkIO {
    using S = St<P>;
    using R = typename S::R;
    static constexpr int VPC = link_vpc(P, REAL);
    static constexpr int NCHUNK = link_nchunk(P, REAL, NCOMP);
    static constexpr size_t SLOT_CHUNKS = (size_t)NCHUNK * HR_TILE;

    __device__ __forceinline__ static const uint4 *slot_ptr(const void *base, long tile, int slot, int lane)
    {
        return reinterpret_cast<const uint4 *>(base) + ((size_t)tile * 8 + slot) * SLOT_CHUNKS + lane;
    }
    __device__ __forceinline__ static unsigned word(const uint4 &v, int k)
    {
        return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
    }
    // complex component k of a chunk
    __device__ __forceinline__ static cx<R> cunpack(const uint4 &v, int k)
    {
        if constexpr (P == HR_F64) {
            return {__hiloint2double((int)v.y, (int)v.x), __hiloint2double((int)v.w, (int)v.z)};
        } else if constexpr (P == HR_DF64) {
            return {df(__uint_as_float(v.x), __uint_as_float(v.y)), df(__uint_as_float(v.z), __uint_as_float(v.w))};
        } else if constexpr (P == HR_F32) {
            return {__uint_as_float(word(v, 2 * k)), __uint_as_float(word(v, 2 * k + 1))};
        } else {
            const unsigned w = word(v, k);
            typename S::C h;
            memcpy(&h, &w, 4);
            return S::ld(h);
        }
    }
    // real component k of a chunk
    __device__ __forceinline__ static R runpack(const uint4 &v, int k)
    {
        if constexpr (P == HR_F64) {
            return k == 0 ? __hiloint2double((int)v.y, (int)v.x) : __hiloint2double((int)v.w, (int)v.z);
        } else if constexpr (P == HR_DF64) {
            return k == 0 ? df(__uint_as_float(v.x), __uint_as_float(v.y)) : df(__uint_as_float(v.z), __uint_as_float(v.w));
        } else if constexpr (P == HR_F32) {
            return __uint_as_float(word(v, k));
        } else {
            const unsigned w = word(v, k >> 1);
            const unsigned short hbits = (k & 1) ? (unsigned short)(w >> 16) : (unsigned short)(w & 0xFFFF);
            typename S::Rs h;
            memcpy(&h, &hbits, 2);
            return S::ldr(h);
        }
    }
    // the whole slot, streamed with evict-first loads (each link is read once
    // per operator application)
    // keep = true: normal caching (the links will be read again soon)
    __device__ __forceinline__ static uint4 ld(const uint4 *p, bool keep) { return keep ? __ldcg(p) : __ldcs(p); }
    __device__ __forceinline__ static void load(const uint4 *p, cx<R> (&W)[NCOMP], bool keep = false)
    {
#pragma unroll
        for (int j = 0; j < NCHUNK; j++) {
            const uint4 v = ld(p + (size_t)j * HR_TILE, keep);
#pragma unroll
            for (int k = 0; k < VPC; k++)
                if (j * VPC + k < NCOMP) W[j * VPC + k] = cunpack(v, k);
        }
    }
    // the real components 2w, 2w+1 of a chunk of a 16-bit (F16/BF16) record:
    // one paired conversion of the 32-bit word w (exact, like two single ones)
    __device__ __forceinline__ static void runpack_pair(const uint4 &v, int w, R &lo, R &hi)
    {
        const unsigned u = word(v, w);
        typename S::C h;
        memcpy(&h, &u, 4);
        const cx<R> f = S::ld(h);
        lo = f.re;
        hi = f.im;
    }
    __device__ __forceinline__ static void unpack_real(const uint4 &v, int j, R (&W)[NCOMP])
    {
        if constexpr (S::scaled) {
#pragma unroll
            for (int w = 0; w < 4; w++) {
                const int e = j * VPC + 2 * w;
                if (e < NCOMP) {
                    R lo, hi;
                    runpack_pair(v, w, lo, hi);
                    W[e] = lo;
                    if (e + 1 < NCOMP) W[e + 1] = hi;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < VPC; k++)
                if (j * VPC + k < NCOMP) W[j * VPC + k] = runpack(v, k);
        }
    }
    __device__ __forceinline__ static void load(const uint4 *p, R (&W)[NCOMP], bool keep = false)
    {
#pragma unroll
        for (int j = 0; j < NCHUNK; j++) unpack_real(ld(p + (size_t)j * HR_TILE, keep), j, W);
    }
    // the same from a copy of the warp's slot records in shared memory
    // (chunk j of lane l at p[j * 32], p = base + l)
    __device__ __forceinline__ static void load_shared(const uint4 *p, cx<R> (&W)[NCOMP])
    {
#pragma unroll
        for (int j = 0; j < NCHUNK; j++) {
            const uint4 v = p[j * HR_TILE];
#pragma unroll
            for (int k = 0; k < VPC; k++)
                if (j * VPC + k < NCOMP) W[j * VPC + k] = cunpack(v, k);
        }
    }
    __device__ __forceinline__ static void load_shared(const uint4 *p, R (&W)[NCOMP])
    {
#pragma unroll
        for (int j = 0; j < NCHUNK; j++) unpack_real(p[j * HR_TILE], j, W);
    }
};

}  // namespace hr
