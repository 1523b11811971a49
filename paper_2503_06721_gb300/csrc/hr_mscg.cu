// hr_mscg.cu -- multi-shift CG: (A + sigma_k) x_k = b for every shift
// sigma_k >= 0 at the cost of one Krylov space.  Sec. 4.1.2 lists the
// multi-shift CG among the supported inverters; Sec. 4.3.2 needs it for the
// poles beta_k of the RHMC's rational approximation, (Q^2 + beta_k)^-1 phi.
//
// The shifted systems share the Krylov space of the base system (the
// smallest shift sigma_0): their residuals stay collinear with the base
// residual, r_k = zeta_k r, and zeta_k, alpha_k, beta_k follow from the base
// CG's alpha and beta by a three-term recurrence (the shifted-system
// identities of Krylov methods, e.g. Jegerlehner 1996).  An iteration costs
// one application of A (4 hops on the even/odd system) for all shifts and
// one vector pass that moves x_k and p_k of every shift still above its
// tolerance.
//
// Per iteration (system j of nsys; every scalar stays on the device):
//   w = A p,  |Dhat p|^2                          4 hops, one with a fused norm
//   alpha = rr / (|Dhat p|^2 + sigma_0 |p|^2)
//   r -= alpha (w + sigma_0 p),  |r|^2            k_ms_update_r; its last block
//                                                 advances zeta_k, alpha_k,
//                                                 beta_k and retires the shifts
//                                                 that met the tolerance
//   x_k += alpha_k p_k,  p_k = zeta_k r + beta_k p_k     k_ms_update_px
// (p_k of the base shift is p itself).  The iterations run as a CUDA graph:
// a WHILE conditional node whose body holds a few iterations and a
// one-thread check kernel.
//
// Precisions: plain FP64, or FP32 iterations followed by FP64 defect
// correction of each shift: the FP64 true residual of every shift, then
// single-shift FP32 solves of all unconverged shifts together (a batch of
// right-hand sides, each with its own shift, sharing every loaded link),
// until each shift meets the tolerance in FP64.
//
// The vector kernels here are element-wise over the complex numbers of a
// field (16-byte loads: one FP64 or two FP32 complex numbers), since none of
// them needs the site structure.
#include <cmath>
#include <cstring>

#include "hr_api.cuh"

namespace hr {

namespace {

constexpr int MS_MAX_SHIFTS = 64;
constexpr int MS_MAX_SYSTEMS = 4096;   // nrhs * nshift
constexpr int MS_BODY_ITERS = 4;
constexpr int MS_THREADS = 256;
constexpr int MS_BODIES_SLOT = 4;      // loop-body counter: counters[4 * reserved systems]

struct MsSys {
    double pp;            // |p|^2
    double alpha_old, beta_old;
    double sigma0;        // base shift
    int base;             // index of the base shift (its p_k is p)
    int upd;              // 1: the last k_ms_update_r advanced the system
};

struct MsShift {
    double delta;         // sigma_k - sigma_0 >= 0
    double zeta, zeta_old, zeta_new;
    double alpha, beta;   // alpha_k, beta_k of the running iteration
    int active;           // still above its tolerance
    int step;             // x_k moves in the running iteration
    int iters;            // iteration that met the tolerance (0: not met)
    int bad;              // the recurrence broke down for this shift
};

struct MsArgs {
    long n;               // complex numbers per system vector
    int nsys, S;
    size_t stride;        // bytes between systems of one vector
    // W-precision vectors: r, p, w [nsys]; x, ps [S][nsys] (ps[base] unused)
    char *r, *p, *w, *x, *ps;
    // FP64 vectors of the init, residual and outer-update kernels
    const char *b;        // source, system j reads source j % bmod
    size_t bstride;
    int bmod;
    char *x64, *ax64, *r64;
    size_t stride64;
    const double *tab;    // [nsys][S] absolute shifts
    const double *sv;     // [nsys] scale (init: of the source; outer: of the correction)
    const double *tol2v;  // [nsys] squared relative tolerance, or nullptr (then tol2)
    const double *qa, *qb;// |Dhat p|^2, or |D p|^2 of the even and odd halves
    double *partials;
    unsigned *counters;
    double *red;          // [nsys][2]
    CgState *state;
    MsSys *sys;
    MsShift *sh;
    double tol2;
    int cap;
};

__device__ __forceinline__ void ld16(const char *p, double (&v)[2])
{
    const double2 t = *reinterpret_cast<const double2 *>(p);
    v[0] = t.x;
    v[1] = t.y;
}
__device__ __forceinline__ void ld16(const char *p, float (&v)[4])
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
__device__ __forceinline__ void st16(char *p, const double (&v)[2])
{
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}
__device__ __forceinline__ void st16(char *p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// 16-byte vectors of one system vector in precision R
template <typename R>
__host__ __device__ __forceinline__ long nvec(long n) { return n * (long)sizeof(R) / 8; }

#define MS_LOOP(v, nv) \
    for (long v = (long)blockIdx.x * blockDim.x + threadIdx.x; v < (nv); v += (long)gridDim.x * blockDim.x)

// r = p = f b;  x_k = 0;  p_k = r;  |r|^2 starts the system's state
template <typename R>
__global__ void __launch_bounds__(MS_THREADS) k_ms_init(const MsArgs a)
{
    constexpr int K = 16 / sizeof(R);
    const int j = blockIdx.y;
    const double f = a.sv[j];
    const double *tab = a.tab + (size_t)j * a.S;
    int base = 0;
    for (int k = 1; k < a.S; k++)
        if (tab[k] < tab[base]) base = k;
    double acc = 0;
    if (f != 0.0) {
        const char *bj = a.b + (size_t)(j % a.bmod) * a.bstride;
        const long nv = nvec<R>(a.n);
        MS_LOOP(v, nv)
        {
            const size_t off = (size_t)v * 16;
            R val[K], z[K];
#pragma unroll
            for (int e = 0; e < K; e += 2) {
                double t[2];
                ld16(bj + (size_t)(v * K + e) * sizeof(double), t);
                val[e] = (R)(f * t[0]);
                val[e + 1] = (R)(f * t[1]);
                z[e] = z[e + 1] = (R)0;
            }
#pragma unroll
            for (int e = 0; e < K; e++) acc += (double)val[e] * (double)val[e];
            st16(a.r + (size_t)j * a.stride + off, val);
            st16(a.p + (size_t)j * a.stride + off, val);
            for (int k = 0; k < a.S; k++) {
                const size_t sk = ((size_t)k * a.nsys + j) * a.stride + off;
                st16(a.x + sk, z);
                if (k != base) st16(a.ps + sk, val);
            }
        }
    }
    double vv[1] = {acc}, tot[1];
    if (grid_reduce<1>(vv, a.partials + (size_t)j * gridDim.x, a.counters + j, gridDim.x, blockIdx.x, tot)) {
        const double tol2 = a.tol2v ? a.tol2v[j] : a.tol2;
        CgState &cs = a.state[j];
        cs.rr = tot[0];
        cs.b2 = tot[0];
        cs.stop2 = tol2 * tot[0];
        cs.pAp = cs.alpha = cs.beta = 0;
        cs.iter = 0;
        cs.cap = a.cap;
        cs.nonfinite = !isfinite(tot[0]);
        cs.converged = cs.nonfinite || f == 0.0 || !(tot[0] > 0.0);
        MsSys &ms = a.sys[j];
        ms.pp = tot[0];
        ms.alpha_old = 1.0;
        ms.beta_old = 0.0;
        ms.sigma0 = tab[base];
        ms.base = base;
        ms.upd = 0;
        for (int k = 0; k < a.S; k++) {
            MsShift &h = a.sh[(size_t)j * a.S + k];
            h.delta = tab[k] - tab[base];
            h.zeta = h.zeta_old = h.zeta_new = 1.0;
            h.alpha = h.beta = 0;
            h.active = !cs.converged;
            h.step = 0;
            h.iters = 0;
            h.bad = 0;
        }
    }
}

// r -= alpha (w + sigma_0 p) with alpha = rr / (|Dhat p|^2 + sigma_0 |p|^2);
// the last block advances the shifted-system scalars
template <typename R>
__global__ void __launch_bounds__(MS_THREADS) k_ms_update_r(const MsArgs a)
{
    constexpr int K = 16 / sizeof(R);
    const int j = blockIdx.y;
    CgState &cs = a.state[j];
    MsSys &ms = a.sys[j];
    if (cg_idle(cs)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ms.upd = 0;
        return;
    }
    const double sigma0 = ms.sigma0;
    const double pAp = a.qa[j] + (a.qb ? a.qb[j] : 0.0) + sigma0 * ms.pp;
    const double alpha = cs.rr / pAp;
    if (!(pAp > 0.0) || !isfinite(alpha)) {
        // breakdown (every block sees it): stop the system, the host reports it
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            cs.nonfinite = 1;
            cs.converged = 1;
            ms.upd = 0;
        }
        return;
    }
    const R al = (R)alpha, sg = (R)sigma0;
    char *rj = a.r + (size_t)j * a.stride;
    const char *wj = a.w + (size_t)j * a.stride;
    const char *pj = a.p + (size_t)j * a.stride;
    double acc = 0;
    const long nv = nvec<R>(a.n);
    MS_LOOP(v, nv)
    {
        const size_t off = (size_t)v * 16;
        R r[K], w[K], p[K];
        ld16(rj + off, r);
        ld16(wj + off, w);
        ld16(pj + off, p);
#pragma unroll
        for (int e = 0; e < K; e++) {
            r[e] = fma(-al, fma(sg, p[e], w[e]), r[e]);
            acc += (double)r[e] * (double)r[e];
        }
        st16(rj + off, r);
    }
    double vv[1] = {acc}, tot[1];
    if (!grid_reduce<1>(vv, a.partials + (size_t)j * gridDim.x, a.counters + j, gridDim.x, blockIdx.x, tot)) return;
    const double rr_new = tot[0];
    cs.pAp = pAp;
    cs.alpha = alpha;
    cs.iter += 1;
    if (!isfinite(rr_new)) {
        cs.nonfinite = 1;
        cs.converged = 1;
        ms.upd = 0;
        return;
    }
    const double beta = rr_new / cs.rr;
    bool any = false;
    for (int k = 0; k < a.S; k++) {
        MsShift &h = a.sh[(size_t)j * a.S + k];
        h.step = h.active;
        if (!h.active) continue;
        double zn = 1.0;
        if (k != ms.base) {
            const double den = alpha * ms.beta_old * (h.zeta_old - h.zeta) +
                               h.zeta_old * ms.alpha_old * (1.0 + h.delta * alpha);
            zn = h.zeta * h.zeta_old * ms.alpha_old / den;
        }
        if (!isfinite(zn) || zn < 0.0) {
            h.bad = 1;
            h.step = 0;
            h.active = 0;
            continue;
        }
        const double ratio = zn / h.zeta;
        h.alpha = alpha * ratio;
        h.beta = beta * ratio * ratio;
        h.zeta_new = zn;
        h.zeta_old = h.zeta;
        h.zeta = zn;
        if (zn * zn * rr_new <= cs.stop2) {
            h.active = 0;
            h.iters = cs.iter;
        }
        any |= h.active != 0;
    }
    ms.alpha_old = alpha;
    ms.beta_old = beta;
    cs.beta = beta;
    cs.rr = rr_new;
    if (!any) cs.converged = 1;
    ms.upd = 1;
}

// x_k += alpha_k p_k for the shifts that moved, then p_k = zeta_k r + beta_k p_k
// for those still iterating (p of the base shift while the system runs), |p|^2
template <typename R>
__global__ void __launch_bounds__(MS_THREADS) k_ms_update_px(const MsArgs a)
{
    constexpr int K = 16 / sizeof(R);
    const int j = blockIdx.y;
    const MsSys &ms = a.sys[j];
    if (!ms.upd) return;
    const bool cont = !cg_idle(a.state[j]);
    const int base = ms.base;
    __shared__ R s_al[MS_MAX_SHIFTS], s_be[MS_MAX_SHIFTS], s_ze[MS_MAX_SHIFTS];
    __shared__ int s_mode[MS_MAX_SHIFTS];
    for (int k = threadIdx.x; k < a.S; k += blockDim.x) {
        const MsShift &h = a.sh[(size_t)j * a.S + k];
        s_al[k] = (R)h.alpha;
        s_be[k] = (R)h.beta;
        s_ze[k] = (R)h.zeta_new;
        const bool pmove = cont && (k == base || h.active);
        s_mode[k] = (h.step ? 1 : 0) | (pmove ? 2 : 0);
    }
    __syncthreads();
    const char *rj = a.r + (size_t)j * a.stride;
    double acc = 0;
    const long nv = nvec<R>(a.n);
    MS_LOOP(v, nv)
    {
        const size_t off = (size_t)v * 16;
        R r[K];
        ld16(rj + off, r);
        for (int k = 0; k < a.S; k++) {
            const int mode = s_mode[k];
            if (!mode) continue;
            const size_t sk = ((size_t)k * a.nsys + j) * a.stride + off;
            char *pk = k == base ? a.p + (size_t)j * a.stride + off : a.ps + sk;
            R p[K];
            ld16(pk, p);
            if (mode & 1) {
                R x[K];
                ld16(a.x + sk, x);
#pragma unroll
                for (int e = 0; e < K; e++) x[e] = fma(s_al[k], p[e], x[e]);
                st16(a.x + sk, x);
            }
            if (mode & 2) {
#pragma unroll
                for (int e = 0; e < K; e++) p[e] = fma(s_be[k], p[e], s_ze[k] * r[e]);
                st16(pk, p);
                if (k == base)
#pragma unroll
                    for (int e = 0; e < K; e++) acc += (double)p[e] * (double)p[e];
            }
        }
    }
    double vv[1] = {acc}, tot[1];
    if (grid_reduce<1>(vv, a.partials + (size_t)j * gridDim.x, a.counters + j, gridDim.x, blockIdx.x, tot))
        a.sys[j].pp = tot[0];
}

__global__ void k_ms_check(cudaGraphConditionalHandle h, const CgState *st, int n, unsigned *bodies)
{
    if (threadIdx.x != 0) return;
    bool any = false;
    for (int i = 0; i < n; i++) any |= !cg_idle(st[i]);
    *bodies += 1;
    cudaGraphSetConditional(h, any ? 1u : 0u);
}

// |b_j|^2 (FP64) into red[2 j + 1]
__global__ void __launch_bounds__(MS_THREADS) k_ms_norm(const MsArgs a)
{
    const int j = blockIdx.y;
    const char *bj = a.b + (size_t)j * a.bstride;
    double acc = 0;
    MS_LOOP(v, a.n)
    {
        double t[2];
        ld16(bj + (size_t)v * 16, t);
        acc = fma(t[0], t[0], fma(t[1], t[1], acc));
    }
    double vv[1] = {acc}, tot[1];
    if (grid_reduce<1>(vv, a.partials + (size_t)j * gridDim.x, a.counters + j, gridDim.x, blockIdx.x, tot))
        a.red[2 * j + 1] = tot[0];
}

// system m = k * bmod + j:  r64_m = b_j - (A x_m) - sigma_m x_m  (FP64),
// |r64_m|^2 and |b_j|^2 into red[2m], red[2m + 1]
__global__ void __launch_bounds__(MS_THREADS) k_ms_residual(const MsArgs a)
{
    const int m = blockIdx.y;
    const double sg = a.tab[m];
    const char *bj = a.b + (size_t)(m % a.bmod) * a.bstride;
    const char *xm = a.x64 + (size_t)m * a.stride64;
    const char *am = a.ax64 + (size_t)m * a.stride64;
    char *rm = a.r64 + (size_t)m * a.stride64;
    double acc[2] = {0, 0};
    MS_LOOP(v, a.n)
    {
        const size_t off = (size_t)v * 16;
        double b[2], x[2], ax[2], r[2];
        ld16(bj + off, b);
        ld16(xm + off, x);
        ld16(am + off, ax);
#pragma unroll
        for (int e = 0; e < 2; e++) {
            r[e] = b[e] - fma(sg, x[e], ax[e]);
            acc[0] = fma(r[e], r[e], acc[0]);
            acc[1] = fma(b[e], b[e], acc[1]);
        }
        st16(rm + off, r);
    }
    double tot[2];
    if (grid_reduce<2>(acc, a.partials + (size_t)m * gridDim.x * 2, a.counters + m, gridDim.x, blockIdx.x, tot)) {
        a.red[2 * m] = tot[0];
        a.red[2 * m + 1] = tot[1];
    }
}

// x64_m += sv_m * x_m (x in precision R, systems with sv_m != 0)
template <typename R>
__global__ void __launch_bounds__(MS_THREADS) k_ms_outer(const MsArgs a)
{
    constexpr int K = 16 / sizeof(R);
    const int m = blockIdx.y;
    const double f = a.sv[m];
    if (f == 0.0) return;
    const char *xm = a.x + (size_t)m * a.stride;
    char *ym = a.x64 + (size_t)m * a.stride64;
    const long nv = nvec<R>(a.n);
    MS_LOOP(v, nv)
    {
        R e[K];
        ld16(xm + (size_t)v * 16, e);
#pragma unroll
        for (int q = 0; q < K; q += 2) {
            double y[2];
            char *yp = ym + (size_t)(v * K + q) * sizeof(double);
            ld16(yp, y);
            y[0] = fma(f, (double)e[q], y[0]);
            y[1] = fma(f, (double)e[q + 1], y[1]);
            st16(yp, y);
        }
    }
}

// y = a0 b + sum_k a_k x_k (FP64; x_k of right-hand side j at (k nrhs + j))
struct LincombArgs {
    long n;               // complex numbers per field
    int nterms, nrhs;
    size_t stride;
    const char *b, *x;
    char *y;
    double a0;
    double a[MS_MAX_SHIFTS];
};

__global__ void __launch_bounds__(MS_THREADS) k_lincomb(const LincombArgs a)
{
    const int j = blockIdx.y;
    const char *bj = a.b + (size_t)j * a.stride;
    char *yj = a.y + (size_t)j * a.stride;
    MS_LOOP(v, a.n)
    {
        const size_t off = (size_t)v * 16;
        double b[2], y[2];
        ld16(bj + off, b);
        y[0] = a.a0 * b[0];
        y[1] = a.a0 * b[1];
        for (int k = 0; k < a.nterms; k++) {
            double x[2];
            ld16(a.x + ((size_t)k * a.nrhs + j) * a.stride + off, x);
            y[0] = fma(a.a[k], x[0], y[0]);
            y[1] = fma(a.a[k], x[1], y[1]);
        }
        st16(yj + off, y);
    }
}

// ------------------------------- host side --------------------------------

struct MsCtx {
    const hr_gauge *g;
    hr_parity sys;
    cudaStream_t s;
    long vh, ns;
    int D;
    double m4;
    Scratch sc;       // with the systems' states (iteration launches skip finished systems)
    Scratch sc_ns;    // same buffers, no state
    unsigned grid_cap;
};

// the vectors one Krylov run iterates on (precision P for all of them)
struct MsVecs {
    int P, nsys, S;
    FieldView r, p, w, q, t;   // [nsys]
    char *x, *ps;              // [S][nsys], same stride as r
};

cudaStream_t ms_capture_stream()
{
    static cudaStream_t s = nullptr;
    if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
    return s;
}

dim3 ms_grid(const MsCtx &c, long nv, int nsys)
{
    long b = (nv + MS_THREADS - 1) / MS_THREADS;
    b = std::max(1L, std::min(b, (long)c.grid_cap));
    return dim3((unsigned)b, (unsigned)nsys);
}

// w = A v for nsys systems in precision P; with qa, |Dhat v|^2 (or the two
// halves of |D v|^2 into qa, qb)
hr_status ms_apply(const MsCtx &c, int P, int nsys, const FieldView &v, const FieldView &w, const FieldView &q,
                   const FieldView &t, const Scratch *sc, double *qa, double *qb)
{
    hr_status st;
    const int D = c.D;
    const int epi_n = qa ? EPI_STORE_NORM : EPI_STORE;
    if (c.g->clover_mode) {
        // the site-dependent diagonal C (Hermitian): D = C + hops,
        // Dhat = C_ee - D_eo C_oo^-1 D_oe, each diagonal product written first
        // and taken up by the hop as its diagonal term
        if (c.sys == HR_EO_PRECOND) {
            for (int dag = 0; dag < 2; dag++) {
                const FieldView &src = dag ? q : v;
                const FieldView &dst = dag ? w : q;
                st = hop(c.g, P, 1, dag, src, t, nullptr, -0.5, 0.0, nsys, c.s, EPI_STORE, sc);
                if (st == HR_OK) st = clover_apply(c.g, P, 1, 1, t, t, nsys, c.s);
                if (st == HR_OK) st = clover_apply(c.g, P, 0, 0, src, dst, nsys, c.s);
                if (st == HR_OK)
                    st = hop(c.g, P, 0, dag, t, dst, &dst, 0.5, 1.0, nsys, c.s, dag ? EPI_STORE : epi_n, sc,
                             FIN_WRITE, nullptr, dag ? nullptr : qa);
                if (st != HR_OK) return st;
            }
            return HR_OK;
        }
        for (int dag = 0; dag < 2; dag++) {
            const FieldView &src = dag ? q : v;
            const FieldView &dst = dag ? w : q;
            for (int par = 0; par < 2; par++) {
                FieldView in = half_view(src, 1 - par, c.vh, D, P), dg = half_view(src, par, c.vh, D, P);
                FieldView o = half_view(dst, par, c.vh, D, P);
                st = clover_apply(c.g, P, par, 0, dg, o, nsys, c.s);
                if (st == HR_OK)
                    st = hop(c.g, P, par, dag, in, o, &o, -0.5, 1.0, nsys, c.s, dag ? EPI_STORE : epi_n, sc, FIN_WRITE,
                             nullptr, dag ? nullptr : (par == 0 ? qa : qb));
                if (st != HR_OK) return st;
            }
        }
        return HR_OK;
    }
    if (c.sys == HR_EO_PRECOND) {
        st = hop(c.g, P, 1, 0, v, t, nullptr, -0.5, 0.0, nsys, c.s, EPI_STORE, sc);
        if (st == HR_OK) st = hop(c.g, P, 0, 0, t, q, &v, 0.5, c.m4 * c.m4, nsys, c.s, epi_n, sc, FIN_WRITE, nullptr, qa);
        if (st == HR_OK) st = hop(c.g, P, 1, 1, q, t, nullptr, -0.5, 0.0, nsys, c.s, EPI_STORE, sc);
        if (st == HR_OK) st = hop(c.g, P, 0, 1, t, w, &q, 0.5, c.m4 * c.m4, nsys, c.s, EPI_STORE, sc);
        return st;
    }
    for (int par = 0; par < 2; par++) {
        FieldView in = half_view(v, 1 - par, c.vh, D, P), dg = half_view(v, par, c.vh, D, P);
        FieldView o = half_view(q, par, c.vh, D, P);
        st = hop(c.g, P, par, 0, in, o, &dg, -0.5, c.m4, nsys, c.s, epi_n, sc, FIN_WRITE, nullptr,
                 par == 0 ? qa : qb);
        if (st != HR_OK) return st;
    }
    for (int par = 0; par < 2; par++) {
        FieldView in = half_view(q, 1 - par, c.vh, D, P), dg = half_view(q, par, c.vh, D, P);
        FieldView o = half_view(w, par, c.vh, D, P);
        st = hop(c.g, P, par, 1, in, o, &dg, -0.5, c.m4, nsys, c.s, EPI_STORE, sc);
        if (st != HR_OK) return st;
    }
    return HR_OK;
}

MsArgs ms_args(const MsCtx &c, const MsVecs &v, MsSys *sys, MsShift *sh)
{
    MsArgs a;
    memset(&a, 0, sizeof a);
    a.n = c.ns * 4 * c.D;
    a.nsys = v.nsys;
    a.S = v.S;
    a.stride = v.r.rhs_stride;
    a.r = v.r.data;
    a.p = v.p.data;
    a.w = v.w.data;
    a.x = v.x;
    a.ps = v.ps;
    a.partials = c.sc.partials;
    a.counters = c.sc.counters;
    a.red = c.sc.red;
    a.state = c.sc.state;
    a.sys = sys;
    a.sh = sh;
    return a;
}

template <typename R>
hr_status launch_pair(const MsCtx &c, const MsArgs &a)
{
    const dim3 gr = ms_grid(c, nvec<R>(a.n), a.nsys);
    k_ms_update_r<R><<<gr, MS_THREADS, 0, c.s>>>(a);
    HR_LAUNCH_CHECK("k_ms_update_r");
    k_ms_update_px<R><<<gr, MS_THREADS, 0, c.s>>>(a);
    HR_LAUNCH_CHECK("k_ms_update_px");
    return HR_OK;
}

hr_status ms_iteration(const MsCtx &c, const MsVecs &v, MsArgs a)
{
    a.qa = c.sc.red;
    a.qb = c.sys == HR_FULL ? c.sc.carry : nullptr;
    hr_status st = ms_apply(c, v.P, v.nsys, v.p, v.w, v.q, v.t, &c.sc, c.sc.red, c.sys == HR_FULL ? c.sc.carry : nullptr);
    if (st != HR_OK) return st;
    return v.P == HR_F64 ? launch_pair<double>(c, a) : launch_pair<float>(c, a);
}

hr_status ms_init(const MsCtx &c, const MsVecs &v, MsArgs a)
{
    if (v.P == HR_F64) {
        k_ms_init<double><<<ms_grid(c, nvec<double>(a.n), a.nsys), MS_THREADS, 0, c.s>>>(a);
    } else {
        k_ms_init<float><<<ms_grid(c, nvec<float>(a.n), a.nsys), MS_THREADS, 0, c.s>>>(a);
    }
    HR_LAUNCH_CHECK("k_ms_init");
    return HR_OK;
}

struct MsGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned *bodies = nullptr;
    unsigned *bodies_host = nullptr, *bodies_dev = nullptr;
    long long per_body = 0;
    ~MsGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }

    hr_status build(const MsCtx &c0, const MsVecs &v, const MsArgs &a)
    {
        HR_CUDA_CHECK(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle h;
        HR_CUDA_CHECK(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        HR_CUDA_CHECK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
        cudaGraph_t body = np.conditional.phGraph_out[0];
        MsCtx c = c0;
        c.s = ms_capture_stream();
        if (!c.s) {
            set_error("cudaStreamCreate failed");
            return HR_ERR_CUDA;
        }
        HR_CUDA_CHECK(cudaStreamBeginCaptureToGraph(c.s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        const long long before = launch_counter();
        hr_status st = HR_OK;
        for (int k = 0; k < MS_BODY_ITERS && st == HR_OK; k++) st = ms_iteration(c, v, a);
        if (st == HR_OK) {
            k_ms_check<<<1, 32, 0, c.s>>>(h, c.sc.state, v.nsys, bodies);
            count_launch();
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_fail(e, "k_ms_check");
        }
        cudaGraph_t out = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c.s, &out);
        per_body = launch_counter() - before;
        count_launch(-per_body);   // counted when the graph runs
        if (st != HR_OK) return st;
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        HR_CUDA_CHECK(cudaGraphInstantiate(&exec, graph, 0));
        return HR_OK;
    }

    hr_status run(cudaStream_t s)
    {
        hr_status st = kernel_zero(bodies, sizeof(unsigned), s);
        if (st != HR_OK) return st;
        HR_CUDA_CHECK(cudaGraphLaunch(exec, s));
        // the counter slot is a reduction ticket of other launches: back to zero
        st = kernel_copy(bodies_dev, bodies, sizeof(unsigned), s);
        return st == HR_OK ? kernel_zero(bodies, sizeof(unsigned), s) : st;
    }
    void account() { count_launch((long long)*bodies_host * per_body); }
};

// host-mapped mailbox layout for M = nrhs * nshift systems
struct MsMailbox {
    char *h, *d;   // host and device addresses of the same bytes
    size_t tab, sv, sv2, tol2, state, shift, red, bodies, bytes;
    explicit MsMailbox(int M)
    {
        size_t o = 0;
        auto take = [&](size_t b) { size_t r = o; o += align_up(b, 64); return r; };
        tab = take(sizeof(double) * M);
        sv = take(sizeof(double) * M);
        sv2 = take(sizeof(double) * M);
        tol2 = take(sizeof(double) * M);
        state = take(sizeof(CgState) * M);
        shift = take(sizeof(MsShift) * M);
        red = take(sizeof(double) * 2 * M);
        bodies = take(64);
        bytes = o;
        h = d = nullptr;
    }
};

hr_status ensure_tuned(const hr_gauge *cg, int P, int nsys, cudaStream_t s)
{
    hr_gauge *g = const_cast<hr_gauge *>(cg);
    const int rb = rebuild_for(g, P) ? 1 : 0;
    const bool untuned = (g->mode == HR_LINKS_AUTO && g->auto_mode[P] < 0) ||
                         (hop_variants_of(g, P) != 0x1u && g->tuned[P][rb][EPI_STORE][nsys > 1 ? 1 : 0] < 0);
    if (g->autotune && g->force_variant < 0 && untuned) return tune_hops(g, P, nsys, s);
    return HR_OK;
}

}  // namespace

}  // namespace hr

using namespace hr;

extern "C" hr_status hr_cg_solve_multishift(const hr_gauge *g, hr_parity sys, const void *b, void *x, int nrhs,
                                            const double *shifts, int nshift, const hr_cg_params *prm,
                                            hr_cg_result *res, void *stream)
{
    if (!g || !b || !x || !shifts || !prm || !res || nrhs < 1 || nshift < 1 || nshift > MS_MAX_SHIFTS ||
        (long)nrhs * nshift > MS_MAX_SYSTEMS) {
        set_error("hr_cg_solve_multishift: NULL argument, nrhs < 1, nshift outside [1, %d] or nrhs * nshift > %d",
                  MS_MAX_SHIFTS, MS_MAX_SYSTEMS);
        return HR_ERR_INVALID;
    }
    if (sys != HR_FULL && sys != HR_EO_PRECOND) {
        set_error("hr_cg_solve_multishift: sys must be HR_FULL or HR_EO_PRECOND");
        return HR_ERR_INVALID;
    }
    for (int k = 0; k < nshift; k++)
        if (!std::isfinite(shifts[k]) || shifts[k] < 0.0) {
            set_error("hr_cg_solve_multishift: shift %d is negative or not finite", k);
            return HR_ERR_INVALID;
        }
    if (!(prm->tol_rel > 0) || prm->max_iter < 1 || prm->use_initial_guess || prm->residual != HR_F64 ||
        (prm->inner != HR_F64 && prm->inner != HR_F32) ||
        (prm->inner == HR_F32 && !(prm->inner_tol > 0 && prm->inner_tol < 1))) {
        set_error("hr_cg_solve_multishift: needs tol_rel > 0, max_iter >= 1, use_initial_guess = 0, "
                  "residual = HR_F64, inner = HR_F64 or HR_F32 (then 0 < inner_tol < 1)");
        return HR_ERR_INVALID;
    }
    const int P = prm->inner;
    if (!(g->prec_mask & (1u << HR_F64)) || !(g->prec_mask & (1u << P))) {
        set_error("hr_cg_solve_multishift: the gauge handle must hold FP64 links and those of the inner precision");
        return HR_ERR_INVALID;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int M = nrhs * nshift;
    MsCtx c;
    c.g = g;
    c.sys = sys;
    c.s = s;
    c.vh = g->geom.vh;
    c.ns = sys == HR_FULL ? 2 * c.vh : c.vh;
    c.D = g->D;
    c.m4 = 4.0 + g->lat.m0;
    c.grid_cap = (unsigned)std::min<long>(152 * 8, max_blocks_for(g) - 1);
    const int D = c.D;
    const size_t fW = field_rhs_bytes(c.ns, D, P), tW = field_rhs_bytes(c.vh, D, P);
    const size_t f64 = field_rhs_bytes(c.ns, D, HR_F64), t64 = field_rhs_bytes(c.vh, D, HR_F64);
    if (x == b || (static_cast<const char *>(b) < static_cast<char *>(x) + f64 * M &&
                   static_cast<char *>(x) < static_cast<const char *>(b) + f64 * nrhs)) {
        set_error("hr_cg_solve_multishift: b and x must not overlap");
        return HR_ERR_INVALID;
    }
    // workspace: small device arrays, then phase 1 and phase 2 vectors over the same bytes
    const size_t small = align_up(sizeof(double) * M, 256) * 4 + align_up(sizeof(MsSys) * M, 256) +
                         align_up(sizeof(MsShift) * M, 256);
    const size_t ph1 = 4 * nrhs * fW + nrhs * tW + (P == HR_F64 ? 0 : M * fW) + M * fW + 8 * 256;
    const size_t ph2 = 3 * M * f64 + M * t64 + 5 * M * fW + M * tW + 12 * 256;
    hr_status st = ws_reserve(g, small + std::max(ph1, ph2), s);
    if (st != HR_OK) return st;
    st = scratch_reserve(g, M, s, &c.sc);
    if (st != HR_OK) return st;
    c.sc_ns = c.sc;
    c.sc_ns.state = nullptr;
    MsMailbox mb(M);
    st = pinned_reserve(g, mb.bytes, s, &mb.h, &mb.d);
    if (st != HR_OK) return st;
    char *q0 = g->ws;
    auto take = [&](char *&q, size_t bytes) { char *r = q; q += align_up(bytes, 256); return r; };
    double *d_tab = reinterpret_cast<double *>(take(q0, sizeof(double) * M));
    double *d_sv = reinterpret_cast<double *>(take(q0, sizeof(double) * M));
    double *d_sv2 = reinterpret_cast<double *>(take(q0, sizeof(double) * M));
    double *d_tol2 = reinterpret_cast<double *>(take(q0, sizeof(double) * M));
    MsSys *d_sys = reinterpret_cast<MsSys *>(take(q0, sizeof(MsSys) * M));
    MsShift *d_sh = reinterpret_cast<MsShift *>(take(q0, sizeof(MsShift) * M));
    auto put = [&](size_t off, void *dst, const void *src, size_t bytes) -> hr_status {
        memcpy(mb.h + off, src, bytes);
        return kernel_copy(dst, mb.d + off, bytes, s);
    };

    for (int i = 0; i < M; i++) {
        res[i].iters = 0;
        res[i].outer_iters = 0;
        res[i].true_rel_residual = NAN;
        res[i].status = HR_ERR_NOT_CONVERGED;
    }
    const FieldView vb = make_view(const_cast<void *>(b), c.ns, D, HR_F64);
    const FieldView vx = make_view(x, c.ns, D, HR_F64);
    std::vector<CgState> stt(M);
    std::vector<MsShift> shh(M);
    std::vector<double> hv(2 * M);
    std::vector<int> iters(M, 0), outer(M, 0);
    bool breakdown = false;

    // ---- phase 1: all shifts of every right-hand side in one Krylov space ----
    st = ensure_tuned(g, P, nrhs, s);
    if (st == HR_OK && M > nrhs) st = ensure_tuned(g, P, M, s);
    if (st != HR_OK) return st;
    {
        char *q = q0;
        MsVecs v;
        v.P = P;
        v.nsys = nrhs;
        v.S = nshift;
        v.r = make_view(take(q, nrhs * fW), c.ns, D, P);
        v.p = make_view(take(q, nrhs * fW), c.ns, D, P);
        v.w = make_view(take(q, nrhs * fW), c.ns, D, P);
        v.q = make_view(take(q, nrhs * fW), c.ns, D, P);
        v.t = make_view(take(q, nrhs * tW), c.vh, D, P);
        v.x = P == HR_F64 ? vx.data : take(q, M * fW);
        v.ps = take(q, M * fW);
        MsArgs a = ms_args(c, v, d_sys, d_sh);
        a.b = vb.data;
        a.bstride = vb.rhs_stride;
        a.bmod = nrhs;
        a.tab = d_tab;
        a.sv = d_sv;
        a.tol2 = P == HR_F64 ? prm->tol_rel * prm->tol_rel
                             : std::pow(std::max(prm->inner_tol, prm->tol_rel), 2.0);
        a.cap = prm->max_iter;
        std::vector<double> tab(M), sv(nrhs, 1.0);
        for (int j = 0; j < nrhs; j++)
            for (int k = 0; k < nshift; k++) tab[(size_t)j * nshift + k] = shifts[k];
        if ((st = put(mb.tab, d_tab, tab.data(), sizeof(double) * M)) != HR_OK) return st;
        std::vector<double> bnorm(nrhs, 1.0);
        if (P != HR_F64) {
            // the FP32 iterations run on b / |b|
            k_ms_norm<<<ms_grid(c, a.n, nrhs), MS_THREADS, 0, s>>>(a);
            HR_LAUNCH_CHECK("k_ms_norm");
            if ((st = kernel_copy(mb.d + mb.red, c.sc.red, sizeof(double) * 2 * nrhs, s)) != HR_OK) return st;
            HR_CUDA_CHECK(cudaStreamSynchronize(s));
            memcpy(hv.data(), mb.h + mb.red, sizeof(double) * 2 * nrhs);
            for (int j = 0; j < nrhs; j++) {
                bnorm[j] = std::sqrt(hv[2 * j + 1]);
                sv[j] = bnorm[j] > 0 && std::isfinite(bnorm[j]) ? 1.0 / bnorm[j] : 0.0;
            }
        }
        if ((st = put(mb.sv, d_sv, sv.data(), sizeof(double) * nrhs)) != HR_OK) return st;
        if ((st = ms_init(c, v, a)) != HR_OK) return st;
        MsGraph gr;
        gr.bodies = c.sc.counters + MS_BODIES_SLOT * M;
        gr.bodies_host = reinterpret_cast<unsigned *>(mb.h + mb.bodies);
        gr.bodies_dev = reinterpret_cast<unsigned *>(mb.d + mb.bodies);
        if ((st = gr.build(c, v, a)) != HR_OK) return st;
        if ((st = gr.run(s)) != HR_OK) return st;
        if ((st = kernel_copy(mb.d + mb.state, c.sc.state, sizeof(CgState) * nrhs, s)) != HR_OK) return st;
        if ((st = kernel_copy(mb.d + mb.shift, d_sh, sizeof(MsShift) * M, s)) != HR_OK) return st;
        HR_CUDA_CHECK(cudaStreamSynchronize(s));
        gr.account();
        memcpy(stt.data(), mb.h + mb.state, sizeof(CgState) * nrhs);
        memcpy(shh.data(), mb.h + mb.shift, sizeof(MsShift) * M);
        for (int j = 0; j < nrhs; j++)
            for (int k = 0; k < nshift; k++) {
                const MsShift &h = shh[(size_t)j * nshift + k];
                iters[(size_t)k * nrhs + j] = h.iters > 0 ? h.iters : stt[j].iter;
                if (h.bad || stt[j].nonfinite) breakdown = true;
            }
        if (P != HR_F64) {
            // x_k = |b| x32_k
            if ((st = kernel_zero(vx.data, vx.rhs_stride * M, s)) != HR_OK) return st;
            std::vector<double> sv2(M);
            for (int k = 0; k < nshift; k++)
                for (int j = 0; j < nrhs; j++) sv2[(size_t)k * nrhs + j] = sv[j] == 0.0 ? 0.0 : bnorm[j];
            if ((st = put(mb.sv2, d_sv2, sv2.data(), sizeof(double) * M)) != HR_OK) return st;
            MsArgs o = a;
            o.nsys = M;
            o.x64 = vx.data;
            o.stride64 = vx.rhs_stride;
            o.sv = d_sv2;
            k_ms_outer<float><<<ms_grid(c, nvec<float>(a.n), M), MS_THREADS, 0, s>>>(o);
            HR_LAUNCH_CHECK("k_ms_outer");
        }
    }

    // ---- phase 2: FP64 true residual of every shift, single-shift corrections ----
    char *q = q0;
    const FieldView r64 = make_view(take(q, M * f64), c.ns, D, HR_F64);
    const FieldView ax64 = make_view(take(q, M * f64), c.ns, D, HR_F64);
    const FieldView qq64 = make_view(take(q, M * f64), c.ns, D, HR_F64);
    const FieldView tt64 = make_view(take(q, M * t64), c.vh, D, HR_F64);
    MsVecs v2;
    v2.P = P;
    v2.nsys = M;
    v2.S = 1;
    v2.r = make_view(take(q, M * fW), c.ns, D, P);
    v2.p = make_view(take(q, M * fW), c.ns, D, P);
    v2.w = make_view(take(q, M * fW), c.ns, D, P);
    v2.q = make_view(take(q, M * fW), c.ns, D, P);
    v2.t = make_view(take(q, M * tW), c.vh, D, P);
    v2.x = take(q, M * fW);
    v2.ps = v2.x;   // single shift: p_k is p, never read
    MsArgs a2 = ms_args(c, v2, d_sys, d_sh);
    a2.b = vb.data;
    a2.bstride = vb.rhs_stride;
    a2.bmod = nrhs;
    a2.x64 = vx.data;
    a2.ax64 = ax64.data;
    a2.r64 = r64.data;
    a2.stride64 = f64;
    a2.tab = d_tab;
    a2.sv = d_sv;
    a2.tol2v = d_tol2;
    {
        std::vector<double> tab(M);
        for (int m = 0; m < M; m++) tab[m] = shifts[m / nrhs];
        // phase 1 has finished reading the table (the stream was synchronised)
        if ((st = put(mb.tab, d_tab, tab.data(), sizeof(double) * M)) != HR_OK) return st;
    }
    MsGraph gr2;
    gr2.bodies = c.sc.counters + MS_BODIES_SLOT * M;
    gr2.bodies_host = reinterpret_cast<unsigned *>(mb.h + mb.bodies);
    gr2.bodies_dev = reinterpret_cast<unsigned *>(mb.d + mb.bodies);
    const double tol = prm->tol_rel;
    std::vector<double> rel(M, NAN);
    int refined = 0;
    for (int round = 0; round < 10000; round++) {
        st = ms_apply(c, HR_F64, M, vx, ax64, qq64, tt64, &c.sc_ns, nullptr, nullptr);
        if (st != HR_OK) return st;
        MsArgs ra = a2;
        ra.red = c.sc.red;
        k_ms_residual<<<ms_grid(c, a2.n, M), MS_THREADS, 0, s>>>(ra);
        HR_LAUNCH_CHECK("k_ms_residual");
        if ((st = kernel_copy(mb.d + mb.red, c.sc.red, sizeof(double) * 2 * M, s)) != HR_OK) return st;
        HR_CUDA_CHECK(cudaStreamSynchronize(s));
        memcpy(hv.data(), mb.h + mb.red, sizeof(double) * 2 * M);
        bool all_ok = true, bad = false;
        std::vector<double> sv(M, 0.0), sv2(M, 0.0), tol2(M, 0.0);
        for (int m = 0; m < M; m++) {
            const double rr = hv[2 * m], b2 = hv[2 * m + 1];
            rel[m] = (!std::isfinite(rr) || !std::isfinite(b2)) ? NAN : (b2 > 0 ? std::sqrt(rr / b2) : 0.0);
            if (!std::isfinite(rel[m])) bad = true;
            if (rel[m] <= tol) continue;
            all_ok = false;
            sv[m] = rr > 0 ? 1.0 / std::sqrt(rr) : 0.0;
            sv2[m] = std::sqrt(rr);
            const double it = std::max(P == HR_F64 ? 0.5 * tol / rel[m] : prm->inner_tol, 0.5 * tol / rel[m]);
            tol2[m] = std::min(it, 0.5) * std::min(it, 0.5);
        }
        // every system has its FP64 true residual; a breakdown or a non-finite
        // residual ends the corrections
        if (all_ok || bad || breakdown || refined >= prm->max_iter) break;
        for (int m = 0; m < M; m++)
            if (sv[m] != 0.0) outer[m] += 1;
        if ((st = put(mb.sv, d_sv, sv.data(), sizeof(double) * M)) != HR_OK) return st;
        if ((st = put(mb.sv2, d_sv2, sv2.data(), sizeof(double) * M)) != HR_OK) return st;
        if ((st = put(mb.tol2, d_tol2, tol2.data(), sizeof(double) * M)) != HR_OK) return st;
        MsArgs ia = a2;
        ia.b = r64.data;
        ia.bstride = r64.rhs_stride;
        ia.bmod = M;
        ia.cap = prm->max_iter - refined;
        if ((st = ms_init(c, v2, ia)) != HR_OK) return st;
        if (!gr2.exec && (st = gr2.build(c, v2, a2)) != HR_OK) return st;
        if ((st = gr2.run(s)) != HR_OK) return st;
        if ((st = kernel_copy(mb.d + mb.state, c.sc.state, sizeof(CgState) * M, s)) != HR_OK) return st;
        MsArgs oa = a2;
        oa.sv = d_sv2;
        if (P == HR_F64) {
            k_ms_outer<double><<<ms_grid(c, nvec<double>(a2.n), M), MS_THREADS, 0, s>>>(oa);
        } else {
            k_ms_outer<float><<<ms_grid(c, nvec<float>(a2.n), M), MS_THREADS, 0, s>>>(oa);
        }
        HR_LAUNCH_CHECK("k_ms_outer");
        HR_CUDA_CHECK(cudaStreamSynchronize(s));
        gr2.account();
        memcpy(stt.data(), mb.h + mb.state, sizeof(CgState) * M);
        int ran = 0;
        for (int m = 0; m < M; m++) {
            if (sv[m] == 0.0) continue;
            iters[m] += stt[m].iter;
            ran = std::max(ran, stt[m].iter);
            if (stt[m].nonfinite) breakdown = true;
        }
        refined += std::max(ran, 1);
    }
    hr_status overall = HR_OK;
    for (int m = 0; m < M; m++) {
        res[m].iters = iters[m];
        res[m].outer_iters = outer[m];
        res[m].true_rel_residual = rel[m];
        res[m].status = !std::isfinite(rel[m]) ? HR_ERR_NONFINITE : (rel[m] <= tol ? HR_OK : HR_ERR_NOT_CONVERGED);
        if (res[m].status != HR_OK && overall == HR_OK) overall = res[m].status;
    }
    if (breakdown && overall == HR_OK) overall = HR_ERR_NONFINITE;
    if (overall == HR_ERR_NOT_CONVERGED) set_error("multi-shift CG stopped above tolerance");
    if (overall == HR_ERR_NONFINITE) set_error("multi-shift CG met a non-finite or non-positive reduction");
    return overall;
}

extern "C" hr_status hr_field_lincomb(const hr_lattice_desc *lat, hr_parity par, double a0, const void *b,
                                      int nterms, const double *a, const void *x, void *y, int nrhs, void *stream)
{
    hr_status st = check_lattice(lat);
    if (st != HR_OK) return st;
    if (!b || !y || nrhs < 1 || nterms < 0 || nterms > MS_MAX_SHIFTS || (nterms > 0 && (!a || !x)) ||
        (par != HR_EVEN && par != HR_ODD && par != HR_FULL)) {
        set_error("hr_field_lincomb: bad arguments (0 <= nterms <= %d, nrhs >= 1)", MS_MAX_SHIFTS);
        return HR_ERR_INVALID;
    }
    const long V = lat_volume(*lat);
    const long ns = par == HR_FULL ? V : V / 2;
    const int D = rep_dim(lat->N, lat->rep);
    const size_t stride = field_rhs_bytes(ns, D, HR_F64);
    if (nterms > 0 && static_cast<char *>(y) < static_cast<const char *>(x) + stride * nterms * nrhs &&
        static_cast<const char *>(x) < static_cast<char *>(y) + stride * nrhs) {
        set_error("hr_field_lincomb: y must not overlap x");
        return HR_ERR_INVALID;
    }
    LincombArgs la;
    memset(&la, 0, sizeof la);
    la.n = ns * 4 * D;
    la.nterms = nterms;
    la.nrhs = nrhs;
    la.stride = stride;
    la.b = static_cast<const char *>(b);
    la.x = static_cast<const char *>(x);
    la.y = static_cast<char *>(y);
    la.a0 = a0;
    for (int k = 0; k < nterms; k++) la.a[k] = a[k];
    const long blocks = std::max(1L, std::min((la.n + MS_THREADS - 1) / MS_THREADS, 152L * 8));
    k_lincomb<<<dim3((unsigned)blocks, (unsigned)nrhs), MS_THREADS, 0, reinterpret_cast<cudaStream_t>(stream)>>>(la);
    HR_LAUNCH_CHECK("k_lincomb");
    return HR_OK;
}
