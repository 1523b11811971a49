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
                if constexpr (S::scaled) v = sc * v;
                psi[s][c] = v;
            }
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
                if constexpr (S::scaled) v = sc * v;
                psi[s][c] = v;
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

// Link records: AoSoA [tile][slot 0..7][component][lane 0..31].
template <int P, bool REAL, int NCOMP>
struct LinkIO {
    using S = St<P>;
    using R = typename S::R;
    using E = typename std::conditional<REAL, typename S::Rs, typename S::C>::type;
    static constexpr size_t SLOT_ELEMS = (size_t)NCOMP * HR_TILE;
    static constexpr size_t TILE_ELEMS = 8 * SLOT_ELEMS;

    __device__ __forceinline__ static const E *slot_ptr(const void *base, long tile, int slot, int lane)
    {
        return reinterpret_cast<const E *>(base) + (size_t)tile * TILE_ELEMS + (size_t)slot * SLOT_ELEMS + lane;
    }
    // streaming load (each link is read exactly once per operator application)
    __device__ __forceinline__ static cx<R> ldc(const E *p, int comp)
    {
        E v = __ldcs(p + (size_t)comp * HR_TILE);
        if constexpr (REAL)
            return {S::ldr(v), (R)0};
        else
            return S::ld(v);
    }
    __device__ __forceinline__ static R ldr(const E *p, int comp)
    {
        if constexpr (REAL)
            return S::ldr(__ldcs(p + (size_t)comp * HR_TILE));
        else
            return (R)0;
    }
};

}  // namespace hr
