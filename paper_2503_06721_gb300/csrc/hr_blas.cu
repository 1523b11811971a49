// hr_blas.cu -- solver linear algebra kernels (see hr_blas.cuh).
#include <algorithm>
#include <cstdint>

#include "hr_blas.cuh"

namespace hr {

template <int P>
using Cplx = typename St<P>::R;

// compute-type precision that holds r and x of a solve whose operator
// fields are stored in P: F64 for P = F64, F32 otherwise
__host__ __device__ constexpr int work_prec(int P) { return P == HR_F64 ? HR_F64 : HR_F32; }

__global__ void __launch_bounds__(BLAS_THREADS) k_copy_words(unsigned *__restrict__ dst,
                                                             const unsigned *__restrict__ src, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
__global__ void __launch_bounds__(BLAS_THREADS) k_copy_vec(uint4 *__restrict__ dst, const uint4 *__restrict__ src,
                                                           size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
__global__ void __launch_bounds__(BLAS_THREADS) k_zero_vec(uint4 *__restrict__ dst, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = make_uint4(0, 0, 0, 0);
}
__global__ void __launch_bounds__(BLAS_THREADS) k_zero_words(unsigned *__restrict__ dst, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = 0;
}

static unsigned copy_grid(size_t n)
{
    const size_t b = (n + BLAS_THREADS - 1) / BLAS_THREADS;
    return (unsigned)std::min<size_t>(b, 152 * 8);
}

hr_status kernel_copy(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) return HR_OK;
    const bool vec = bytes % 16 == 0 && (reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) % 16 == 0;
    if (vec) {
        const size_t n = bytes / 16;
        k_copy_vec<<<copy_grid(n), BLAS_THREADS, 0, st>>>(static_cast<uint4 *>(dst), static_cast<const uint4 *>(src), n);
    } else {
        const size_t n = bytes / 4;
        k_copy_words<<<copy_grid(n), BLAS_THREADS, 0, st>>>(static_cast<unsigned *>(dst),
                                                             static_cast<const unsigned *>(src), n);
    }
    HR_LAUNCH_CHECK("kernel_copy");
    return HR_OK;
}

hr_status kernel_zero(void *dst, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) return HR_OK;
    if (bytes % 16 == 0 && reinterpret_cast<uintptr_t>(dst) % 16 == 0) {
        const size_t n = bytes / 16;
        k_zero_vec<<<copy_grid(n), BLAS_THREADS, 0, st>>>(static_cast<uint4 *>(dst), n);
    } else {
        const size_t n = bytes / 4;
        k_zero_words<<<copy_grid(n), BLAS_THREADS, 0, st>>>(static_cast<unsigned *>(dst), n);
    }
    HR_LAUNCH_CHECK("kernel_zero");
    return HR_OK;
}

template <int D, int PD, int PS>
__global__ void __launch_bounds__(BLAS_THREADS) k_convert(const BlasParams bp)
{
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bp.nsites) return;
    using RS = typename St<PS>::R;
    using RD = typename St<PD>::R;
    cx<RS> v[4][D];
    SpinorIO<PS, D>::load_rw(bp.b, rhs, i, v);
    const double f = bp.sv ? bp.sv[rhs] : bp.s;
    cx<RD> w[4][D];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < D; c++) {
            const double re = to_f64(v[s][c].re), im = to_f64(v[s][c].im);
            w[s][c] = f == 1.0 ? cx<RD>{from_f64<RD>(re), from_f64<RD>(im)}
                               : cx<RD>{from_f64<RD>(f * re), from_f64<RD>(f * im)};
        }
    SpinorIO<PD, D>::store(bp.a, rhs, i, w);
}

template <int D>
__global__ void __launch_bounds__(BLAS_THREADS) k_residual_init(const BlasParams bp)
{
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0, 0};
    if (i < bp.nsites) {
        cx<double> b[4][D], ax[4][D];
        SpinorIO<HR_F64, D>::load_rw(bp.b, rhs, i, b);
        if (bp.c.data) {
            SpinorIO<HR_F64, D>::load_rw(bp.c, rhs, i, ax);
        } else {   // x = 0: r = b
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < D; c++) ax[s][c] = {0.0, 0.0};
        }
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) {
                ax[s][c] = b[s][c] - ax[s][c];
                v[0] += ax[s][c].re * ax[s][c].re + ax[s][c].im * ax[s][c].im;
                v[1] += b[s][c].re * b[s][c].re + b[s][c].im * b[s][c].im;
            }
        SpinorIO<HR_F64, D>::store(bp.a, rhs, i, ax);
    }
    double tot[2];
    if (grid_reduce<2>(v, bp.partials + (size_t)rhs * gridDim.x * 2, bp.counters + rhs, gridDim.x, blockIdx.x, tot)) {
        if (bp.red_out) {
            bp.red_out[rhs * 2 + 0] = tot[0];
            bp.red_out[rhs * 2 + 1] = tot[1];
        }
        if (bp.state) {
            CgState &cs = bp.state[rhs];
            cs.rr = tot[0];
            cs.b2 = tot[1];
            cs.stop2 = bp.tol2 * tot[1];
            cs.iter = 0;
            cs.nonfinite = !(isfinite(tot[0]) && isfinite(tot[1]));
            cs.converged = (tot[0] <= cs.stop2) || cs.nonfinite;
            cs.alpha = cs.beta = 0;
            cs.cap = bp.cap;
        }
    }
}

template <int D>
__global__ void __launch_bounds__(BLAS_THREADS) k_start_zero(const BlasParams bp)
{
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0, 0};
    if (i < bp.nsites) {
        cx<double> b[4][D], z[4][D];
        SpinorIO<HR_F64, D>::load_rw(bp.b, rhs, i, b);
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) {
                z[s][c] = {0, 0};
                v[0] += b[s][c].re * b[s][c].re + b[s][c].im * b[s][c].im;
            }
        v[1] = v[0];
        SpinorIO<HR_F64, D>::store(bp.a, rhs, i, b);
        SpinorIO<HR_F64, D>::store(bp.c, rhs, i, z);
    }
    double tot[2];
    if (grid_reduce<2>(v, bp.partials + (size_t)rhs * gridDim.x * 2, bp.counters + rhs, gridDim.x, blockIdx.x, tot)) {
        if (bp.red_out) {
            bp.red_out[rhs * 2 + 0] = tot[0];
            bp.red_out[rhs * 2 + 1] = tot[1];
        }
        if (bp.state) {
            CgState &cs = bp.state[rhs];
            cs.rr = tot[0];
            cs.b2 = tot[1];
            cs.stop2 = bp.tol2 * tot[1];
            cs.iter = 0;
            cs.nonfinite = !isfinite(tot[0]);
            cs.converged = (tot[0] <= cs.stop2) || cs.nonfinite;
            cs.alpha = cs.beta = 0;
            cs.cap = bp.cap;
        }
    }
}

template <int D, int PP>
__global__ void __launch_bounds__(BLAS_THREADS) k_xpay_beta(const BlasParams bp)
{
    const int rhs = blockIdx.y;
    if (cg_idle(bp.state[rhs])) return;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bp.nsites) return;
    constexpr int PW = work_prec(PP);
    using R = typename St<PP>::R;
    const R beta = (R)bp.state[rhs].beta;
    cx<R> r[4][D], p[4][D];
    SpinorIO<PW, D>::load_rw(bp.a, rhs, i, r);
    SpinorIO<PP, D>::load_rw(bp.c, rhs, i, p);
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < D; c++) p[s][c] = r[s][c] + beta * p[s][c];
    SpinorIO<PP, D>::store(bp.c, rhs, i, p);
}

template <int D, int PP>
__global__ void __launch_bounds__(BLAS_THREADS) k_inner_init(const BlasParams bp)
{
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0};
    if (i < bp.nsites) {
        const double f = bp.sv[rhs];
        cx<double> r[4][D];
        SpinorIO<HR_F64, D>::load_rw(bp.b, rhs, i, r);
        cx<float> ri[4][D], z[4][D];
        float n2 = 0;
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) {
                ri[s][c] = {f32_rn(f * r[s][c].re), f32_rn(f * r[s][c].im)};
                z[s][c] = {0.f, 0.f};
                n2 += ri[s][c].re * ri[s][c].re + ri[s][c].im * ri[s][c].im;
            }
        v[0] = n2;
        SpinorIO<HR_F32, D>::store(bp.a, rhs, i, ri);
        SpinorIO<HR_F32, D>::store(bp.c, rhs, i, z);
        using RP = typename St<PP>::R;
        cx<RP> pv[4][D];
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) pv[s][c] = {(RP)ri[s][c].re, (RP)ri[s][c].im};
        SpinorIO<PP, D>::store(bp.d, rhs, i, pv);
    }
    double tot[1];
    if (grid_reduce<1>(v, bp.partials + (size_t)rhs * gridDim.x, bp.counters + rhs, gridDim.x, blockIdx.x, tot)) {
        CgState &cs = bp.state[rhs];
        cs.rr = tot[0];
        cs.b2 = tot[0];
        cs.stop2 = bp.tol2 * tot[0];
        cs.iter = 0;
        cs.nonfinite = !isfinite(tot[0]);
        cs.converged = (tot[0] <= cs.stop2) || cs.nonfinite || bp.sv[rhs] == 0.0;
        cs.alpha = cs.beta = 0;
        cs.cap = bp.cap;
    }
}

template <int D>
__global__ void __launch_bounds__(BLAS_THREADS) k_outer_update(const BlasParams bp)
{
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= bp.nsites) return;
    const double f = bp.sv[rhs];
    if (f == 0.0) return;
    cx<double> x[4][D];
    cx<float> e[4][D];
    SpinorIO<HR_F64, D>::load_rw(bp.a, rhs, i, x);
    SpinorIO<HR_F32, D>::load_rw(bp.b, rhs, i, e);
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < D; c++) {
            x[s][c].re = fma(f, f64_of(e[s][c].re), x[s][c].re);
            x[s][c].im = fma(f, f64_of(e[s][c].im), x[s][c].im);
        }
    SpinorIO<HR_F64, D>::store(bp.a, rhs, i, x);
}

template <int D, int P>
__global__ void __launch_bounds__(BLAS_THREADS) k_dot(const BlasParams bp)
{
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0, 0};
    if (i < bp.nsites) {
        using R = typename St<P>::R;
        cx<R> a[4][D], b[4][D];
        SpinorIO<P, D>::load_rw(bp.a, rhs, i, a);
        SpinorIO<P, D>::load_rw(bp.b, rhs, i, b);
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) {
                const double ar = to_f64(a[s][c].re), ai = to_f64(a[s][c].im);
                const double br = to_f64(b[s][c].re), bi = to_f64(b[s][c].im);
                v[0] += ar * br + ai * bi;
                v[1] += ar * bi - ai * br;
            }
    }
    double tot[2];
    if (grid_reduce<2>(v, bp.partials + (size_t)rhs * gridDim.x * 2, bp.counters + rhs, gridDim.x, blockIdx.x, tot)) {
        bp.red_out[rhs * 2 + 0] = tot[0];
        bp.red_out[rhs * 2 + 1] = tot[1];
    }
}

// ---------------------------------------------------------------------------
// host launchers with runtime dispatch on D and the precisions
// ---------------------------------------------------------------------------
static inline dim3 grid_of(const BlasParams &bp)
{
    return dim3((unsigned)((bp.nsites + BLAS_THREADS - 1) / BLAS_THREADS), (unsigned)bp.nrhs);
}

hr_status blas_convert(int D, int Pdst, int Psrc, const BlasParams &bp, cudaStream_t st)
{
    HR_FOR_D(D, HR_FOR_PX(Pdst, PD, HR_FOR_PX(Psrc, PS, (k_convert<DD, PD, PS><<<grid_of(bp), BLAS_THREADS, 0, st>>>(bp)))));
    HR_LAUNCH_CHECK("k_convert");
    return HR_OK;
}

hr_status blas_residual_init(int D, const BlasParams &bp, cudaStream_t st)
{
    HR_FOR_D(D, (k_residual_init<DD><<<grid_of(bp), BLAS_THREADS, 0, st>>>(bp)));
    HR_LAUNCH_CHECK("k_residual_init");
    return HR_OK;
}

hr_status blas_start_zero(int D, const BlasParams &bp, cudaStream_t st)
{
    HR_FOR_D(D, (k_start_zero<DD><<<grid_of(bp), BLAS_THREADS, 0, st>>>(bp)));
    HR_LAUNCH_CHECK("k_start_zero");
    return HR_OK;
}

hr_status blas_xpay_beta(int D, int Pp, const BlasParams &bp, cudaStream_t st)
{
    HR_FOR_D(D, HR_FOR_P(Pp, PP, (k_xpay_beta<DD, PP><<<grid_of(bp), BLAS_THREADS, 0, st>>>(bp))));
    HR_LAUNCH_CHECK("k_xpay_beta");
    return HR_OK;
}

hr_status blas_inner_init(int D, int Pp, const BlasParams &bp, cudaStream_t st)
{
    HR_FOR_D(D, HR_FOR_P(Pp, PP, (k_inner_init<DD, PP><<<grid_of(bp), BLAS_THREADS, 0, st>>>(bp))));
    HR_LAUNCH_CHECK("k_inner_init");
    return HR_OK;
}

hr_status blas_outer_update(int D, const BlasParams &bp, cudaStream_t st)
{
    HR_FOR_D(D, (k_outer_update<DD><<<grid_of(bp), BLAS_THREADS, 0, st>>>(bp)));
    HR_LAUNCH_CHECK("k_outer_update");
    return HR_OK;
}

hr_status blas_dot(int D, int P, const BlasParams &bp, cudaStream_t st)
{
    HR_FOR_D(D, HR_FOR_PX(P, PN, (k_dot<DD, PN><<<grid_of(bp), BLAS_THREADS, 0, st>>>(bp))));
    HR_LAUNCH_CHECK("k_dot");
    return HR_OK;
}

}  // namespace hr
