// hr_blas.cuh -- fused site-parallel linear algebra for the solver
// (Sec. 3.2 "Linear Combinations" and "Reductions"): each kernel reads and
// writes every vector once and folds its reductions into the same pass.
#pragma once

#include "hr_fields.cuh"

namespace hr {

struct BlasParams {
    long nsites;
    int nrhs;
    FieldView a, b, c, d;     // meaning depends on the kernel
    double s;                 // scalar argument
    const double *sv;         // per-rhs scalars (device) or nullptr
    double *partials;         // [nrhs][nblocks][NV]
    unsigned *counters;       // [nrhs]
    double *red_out;          // [nrhs][NV]
    CgState *state;           // [nrhs]
    double tol2;              // squared relative tolerance for state init
    int cap;                  // iteration cap written into the state by init kernels
};

// Word copies and fills done by a kernel instead of the copy engines, so
// that the solver's small host round trips (through host-mapped pinned
// memory) and its device-side copies never queue behind bulk transfers that
// the caller runs on other streams.  Sizes are in bytes, multiples of 4;
// pointers 4-byte aligned (16-byte aligned for the bulk form).
hr_status kernel_copy(void *dst, const void *src, size_t bytes, cudaStream_t st);
hr_status kernel_zero(void *dst, size_t bytes, cudaStream_t st);

// a <- convert(b) * (sv ? sv[rhs] : s)            (any precisions)
hr_status blas_convert(int D, int Pdst, int Psrc, const BlasParams &bp, cudaStream_t st);
// a(F64) <- b(F64) - c(F64);  reduce |a|^2, |b|^2 into state (rr, b2, stop2 = tol2*b2)
// and red_out[rhs][0..1]
hr_status blas_residual_init(int D, const BlasParams &bp, cudaStream_t st);
// p(c, Pp) <- r(a, compute type of Pp) + beta p   (beta = state[rhs].beta), skips converged
hr_status blas_xpay_beta(int D, int Pp, const BlasParams &bp, cudaStream_t st);
// inner start of defect correction with f = sv[rhs]:
//   a (F32 r_in) <- f * b (F64 r);  c (F32 x_in) <- 0;  d (Pp p) <- a;
//   reduce |r_in|^2 into state: rr, b2, stop2 = tol2 * rr, converged, iter = 0
hr_status blas_inner_init(int D, int Pp, const BlasParams &bp, cudaStream_t st);
// a (F64 x) += sv[rhs] * b (F32 x_in)
hr_status blas_outer_update(int D, const BlasParams &bp, cudaStream_t st);
// red_out[rhs][0..1] <- <a, b> (re, im), both in precision P
hr_status blas_dot(int D, int P, const BlasParams &bp, cudaStream_t st);
// a(F64) <- x-update for plain CG initial state without guess: a = b, c = 0, reduce |b|^2
hr_status blas_start_zero(int D, const BlasParams &bp, cudaStream_t st);

constexpr int BLAS_THREADS = 256;

// runtime dispatch on the representation dimension D and on a precision: BODY
// is compiled once per case with the constant DD (and PN) set
#define HR_FOR_D(D_, BODY)                     \
    switch (D_) {                              \
    case 2: { constexpr int DD = 2; BODY; } break; \
    case 3: { constexpr int DD = 3; BODY; } break; \
    case 4: { constexpr int DD = 4; BODY; } break; \
    case 5: { constexpr int DD = 5; BODY; } break; \
    case 6: { constexpr int DD = 6; BODY; } break; \
    case 8: { constexpr int DD = 8; BODY; } break; \
    default: set_error("representation dimension %d not compiled", D_); return HR_ERR_UNSUPPORTED; \
    }

#define HR_FOR_P(P_, PN, BODY)                              \
    switch (P_) {                                           \
    case HR_F64: { constexpr int PN = HR_F64; BODY; } break; \
    case HR_F32: { constexpr int PN = HR_F32; BODY; } break; \
    case HR_F16: { constexpr int PN = HR_F16; BODY; } break; \
    case HR_BF16: { constexpr int PN = HR_BF16; BODY; } break; \
    default: set_error("bad precision %d", P_); return HR_ERR_INVALID; \
    }

// the same with the float-float storage (conversions and dot products only)
#define HR_FOR_PX(P_, PN, BODY)                              \
    switch (P_) {                                           \
    case HR_F64: { constexpr int PN = HR_F64; BODY; } break; \
    case HR_F32: { constexpr int PN = HR_F32; BODY; } break; \
    case HR_F16: { constexpr int PN = HR_F16; BODY; } break; \
    case HR_BF16: { constexpr int PN = HR_BF16; BODY; } break; \
    case HR_DF64: { constexpr int PN = HR_DF64; BODY; } break; \
    default: set_error("bad precision %d", P_); return HR_ERR_INVALID; \
    }

}  // namespace hr
