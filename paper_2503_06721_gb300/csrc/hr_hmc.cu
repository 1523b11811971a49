// hr_hmc.cu -- the HMC building blocks around the fermion force (Sec. 2.4,
// Sec. 2.5, Sec. 4.2): the Wilson plaquette action and its force, the link
// update U <- exp(i eps pi^a T^a) U, the momenta's kinetic energy, and a
// molecular-dynamics trajectory (leapfrog or 2nd-order Omelyan) that drives
// them together with the fused fermion solve + force.
//
// Conventions (Sec. 2.5): H = H_pi + S_g + S_f with H_pi = T_F/2 sum pi^2,
// dU/dtau = pi U with pi = i pi^a T^a, dpi^a/dtau = F^a = -(1/T_F) dS/de^a,
// where dS/de^a is the Lie derivative along exp(i e T^a) U (the quantity
// hr_dirac_force and hr_gauge_force accumulate).  A momentum step
// pi += h F is therefore a force call with coeff = -h / T_F that accumulates
// straight into pi.
//
// The gauge field U_F is FP64 [V][4][N][N], lexicographic, periodic in every
// direction (the fermions' boundary signs live in the represented links).
// Every kernel is FP64 and one thread per site or link: the staple sums and
// matrix exponentials are FP64 arithmetic, a small part of a trajectory
// next to the fermion solves.
#include <cmath>
#include <cstring>

#include "hr_api.cuh"
#include "hr_rep.cuh"

namespace hr {

namespace {

constexpr int HMC_THREADS = 128;
constexpr double T_FUND = 0.5;

struct GaugeGeom {
    int d[4];     // T, X, Y, Z
    long V;
};

__device__ __forceinline__ void coords_of(const GaugeGeom &g, long x, int (&c)[4])
{
    c[3] = (int)(x % g.d[3]);
    x /= g.d[3];
    c[2] = (int)(x % g.d[2]);
    x /= g.d[2];
    c[1] = (int)(x % g.d[1]);
    c[0] = (int)(x / g.d[1]);
}
__device__ __forceinline__ long lex_of(const GaugeGeom &g, const int (&c)[4])
{
    return (((long)c[0] * g.d[1] + c[1]) * g.d[2] + c[2]) * g.d[3] + c[3];
}
// the site x + s mu (s = +1 / -1), periodic
__device__ __forceinline__ long shift(const GaugeGeom &g, const int (&c)[4], int mu, int s)
{
    int e[4] = {c[0], c[1], c[2], c[3]};
    e[mu] += s;
    if (e[mu] == g.d[mu]) e[mu] = 0;
    if (e[mu] < 0) e[mu] = g.d[mu] - 1;
    return lex_of(g, e);
}

template <int N>
struct Mat {
    cx<double> m[N][N];
};

template <int N>
__device__ __forceinline__ Mat<N> load_link(const cx<double> *U, long x, int mu)
{
    Mat<N> a;
    const cx<double> *p = U + ((size_t)x * 4 + mu) * N * N;
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) a.m[i][j] = p[i * N + j];
    return a;
}

// C = A B, A^dag B, A B^dag
template <int N>
__device__ __forceinline__ Mat<N> mul(const Mat<N> &A, const Mat<N> &B)
{
    Mat<N> C;
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) {
            cx<double> s = {0, 0};
#pragma unroll
            for (int k = 0; k < N; k++) cmac(s, A.m[i][k], B.m[k][j]);
            C.m[i][j] = s;
        }
    return C;
}
template <int N>
__device__ __forceinline__ Mat<N> mul_dn(const Mat<N> &A, const Mat<N> &B)   // A^dag B
{
    Mat<N> C;
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) {
            cx<double> s = {0, 0};
#pragma unroll
            for (int k = 0; k < N; k++) cmac(s, conj(A.m[k][i]), B.m[k][j]);
            C.m[i][j] = s;
        }
    return C;
}
template <int N>
__device__ __forceinline__ Mat<N> mul_nd(const Mat<N> &A, const Mat<N> &B)   // A B^dag
{
    Mat<N> C;
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) {
            cx<double> s = {0, 0};
#pragma unroll
            for (int k = 0; k < N; k++) cmac(s, A.m[i][k], conj(B.m[j][k]));
            C.m[i][j] = s;
        }
    return C;
}

// sum_{mu<nu} (1 - Re tr P_mu nu(x) / N) per site, summed over the lattice
template <int N>
__global__ void __launch_bounds__(HMC_THREADS) k_plaquette(const GaugeGeom g, const cx<double> *__restrict__ U,
                                                          double *partials, unsigned *counter, double *out)
{
    const long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0};
    if (x < g.V) {
        int c[4];
        coords_of(g, x, c);
        for (int mu = 0; mu < 4; mu++) {
            const long xm = shift(g, c, mu, +1);
            const Mat<N> Umu = load_link<N>(U, x, mu);
            for (int nu = mu + 1; nu < 4; nu++) {
                const long xn = shift(g, c, nu, +1);
                // P = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
                const Mat<N> a = mul<N>(Umu, load_link<N>(U, xm, nu));
                const Mat<N> b = mul_nd<N>(a, load_link<N>(U, xn, mu));
                const Mat<N> P = mul_nd<N>(b, load_link<N>(U, x, nu));
                double tr = 0;
#pragma unroll
                for (int i = 0; i < N; i++) tr += P.m[i][i].re;
                v[0] += 1.0 - tr / N;
            }
        }
    }
    double tot[1];
    if (grid_reduce<1>(v, partials, counter, gridDim.x, blockIdx.x, tot)) *out = tot[0];
}

// F[x][mu][a] += coeff * (-(beta/N) Re tr(i T^a U_mu(x) W_mu(x))), W the staple sum
template <int N>
__global__ void __launch_bounds__(HMC_THREADS) k_gauge_force(const GaugeGeom g, const cx<double> *__restrict__ U,
                                                            double *__restrict__ F, double scale)
{
    const long l = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4 * g.V) return;
    const long x = l >> 2;
    const int mu = (int)(l & 3);
    int c[4];
    coords_of(g, x, c);
    const long xm = shift(g, c, mu, +1);
    Mat<N> W;
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) W.m[i][j] = {0, 0};
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        const long xn = shift(g, c, nu, +1);
        const long xdn = shift(g, c, nu, -1);
        int cm[4] = {c[0], c[1], c[2], c[3]};
        cm[mu] = (cm[mu] + 1) % g.d[mu];
        const long xmdn = shift(g, cm, nu, -1);
        // upper: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
        const Mat<N> up = mul_nd<N>(mul_nd<N>(load_link<N>(U, xm, nu), load_link<N>(U, xn, mu)), load_link<N>(U, x, nu));
        // lower: U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
        //     = (U_mu(x-nu) U_nu(x+mu-nu))^dag U_nu(x-nu)
        const Mat<N> ba = mul<N>(load_link<N>(U, xdn, mu), load_link<N>(U, xmdn, nu));
        const Mat<N> low = mul_dn<N>(ba, load_link<N>(U, xdn, nu));
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int j = 0; j < N; j++) W.m[i][j] = W.m[i][j] + up.m[i][j] + low.m[i][j];
    }
    const Mat<N> M = mul<N>(load_link<N>(U, x, mu), W);
    // Re tr(i T^a M) = -Im tr(T^a M), tr(T^a M) = sum_e T^a_{rc} M_{cr}
    double *Fl = F + (size_t)l * (N * N - 1);
#pragma unroll
    for (int a = 0; a < N * N - 1; a++) {
        double im = 0;
#pragma unroll
        for (int e = 0; e < gen_nent(N, a); e++) {
            const cx<double> t = gen_val<double>(N, a, e);
            const cx<double> m = M.m[gen_col(N, a, e)][gen_row(N, a, e)];
            im += t.re * m.im + t.im * m.re;
        }
        Fl[a] = fma(scale, im, Fl[a]);   // scale = coeff * beta / N:  -(beta/N)(-im)
    }
}

// U_mu(x) <- exp(i eps pi^a T^a) U_mu(x): the exponential of Y = i eps X (X
// Hermitian) by scaling and squaring around a Taylor polynomial (Moler and
// Van Loan, "Nineteen dubious ways", 2003): Y / 2^s with |Y / 2^s|_F <= 1/2,
// terms to order 16 (remainder below 2^-17 / 17! ~ 6e-20), then s squarings.
template <int N>
__global__ void __launch_bounds__(HMC_THREADS) k_link_update(const GaugeGeom g, cx<double> *__restrict__ U,
                                                            const double *__restrict__ pi, double eps)
{
    const long l = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4 * g.V) return;
    const double *p = pi + (size_t)l * (N * N - 1);
    Mat<N> Y;
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) Y.m[i][j] = {0, 0};
#pragma unroll
    for (int a = 0; a < N * N - 1; a++) {
        const double w = eps * p[a];
#pragma unroll
        for (int e = 0; e < gen_nent(N, a); e++) {
            const cx<double> t = gen_val<double>(N, a, e);
            // i * w * T_rc
            cx<double> &y = Y.m[gen_row(N, a, e)][gen_col(N, a, e)];
            y = y + cx<double>{-w * t.im, w * t.re};
        }
    }
    double nf = 0;
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) nf += Y.m[i][j].re * Y.m[i][j].re + Y.m[i][j].im * Y.m[i][j].im;
    nf = sqrt(nf);
    int s = 0;
    while (nf > 0.5 && s < 60) {
        nf *= 0.5;
        s++;
    }
    const double sc = ldexp(1.0, -s);
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) Y.m[i][j] = sc * Y.m[i][j];
    // Horner: E = I + Y (I + Y/2 (I + Y/3 ( ... (I + Y/16))))
    Mat<N> E;
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) E.m[i][j] = {i == j ? 1.0 : 0.0, 0.0};
#pragma unroll 1
    for (int k = 16; k >= 1; k--) {
        Mat<N> T = mul<N>(Y, E);
        const double r = 1.0 / k;
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int j = 0; j < N; j++) E.m[i][j] = (i == j ? cx<double>{1.0, 0.0} : cx<double>{0.0, 0.0}) + r * T.m[i][j];
    }
    for (int q = 0; q < s; q++) E = mul<N>(E, E);
    const long x = l >> 2;
    const int mu = (int)(l & 3);
    const Mat<N> Un = mul<N>(E, load_link<N>(U, x, mu));
    cx<double> *o = U + (size_t)l * N * N;
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) o[i * N + j] = Un.m[i][j];
    (void)g;
}

// sum of squares of n doubles
__global__ void __launch_bounds__(HMC_THREADS) k_sumsq(const double *__restrict__ v, long n, double *partials,
                                                      unsigned *counter, double *out)
{
    double acc[1] = {0};
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        acc[0] = fma(v[i], v[i], acc[0]);
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, gridDim.x, blockIdx.x, tot)) *out = tot[0];
}

GaugeGeom gauge_geom(const hr_lattice_desc &l)
{
    GaugeGeom g;
    for (int i = 0; i < 4; i++) g.d[i] = l.dims[i];
    g.V = lat_volume(l);
    return g;
}

#define HR_FOR_N(N_, BODY)                                 \
    switch (N_) {                                          \
    case 2: { constexpr int NN = 2; BODY; } break;         \
    case 3: { constexpr int NN = 3; BODY; } break;         \
    case 4: { constexpr int NN = 4; BODY; } break;         \
    default: set_error("SU(%d) gauge kernels are not compiled", N_); return HR_ERR_UNSUPPORTED; \
    }

hr_status check_gauge_lat(const hr_lattice_desc *lat)
{
    if (!lat || lat->N < 2 || lat->N > 4) {
        set_error("gauge kernels: NULL lattice or N outside 2..4");
        return HR_ERR_INVALID;
    }
    for (int i = 0; i < 4; i++)
        if (lat->dims[i] < 1) {
            set_error("gauge kernels: bad lattice extents");
            return HR_ERR_INVALID;
        }
    return HR_OK;
}

// device reduction scratch for one grid-wide sum: [blocks] partials, a
// ticket, the result (stream-ordered allocation)
struct SumScratch {
    char *buf = nullptr;
    cudaStream_t s = nullptr;
    double *partials = nullptr, *out = nullptr;
    unsigned *counter = nullptr;
    hr_status alloc(long blocks, cudaStream_t st)
    {
        s = st;
        const size_t bytes = align_up(sizeof(double) * blocks, 256) + 256 + 256;
        HR_CUDA_CHECK(cudaMallocAsync((void **)&buf, bytes, s));
        HR_CUDA_CHECK(cudaMemsetAsync(buf, 0, bytes, s));
        partials = reinterpret_cast<double *>(buf);
        counter = reinterpret_cast<unsigned *>(buf + align_up(sizeof(double) * blocks, 256));
        out = reinterpret_cast<double *>(buf + align_up(sizeof(double) * blocks, 256) + 256);
        return HR_OK;
    }
    ~SumScratch()
    {
        if (buf) cudaFreeAsync(buf, s);
    }
};

hr_status read_sum(SumScratch &ss, double *host)
{
    HR_CUDA_CHECK(cudaMemcpyAsync(host, ss.out, sizeof(double), cudaMemcpyDeviceToHost, ss.s));
    HR_CUDA_CHECK(cudaStreamSynchronize(ss.s));
    return HR_OK;
}

hr_status gauge_force_launch(const hr_lattice_desc &lat, const void *U, double beta, double coeff, double *F,
                             cudaStream_t s)
{
    const GaugeGeom g = gauge_geom(lat);
    const unsigned blocks = (unsigned)((4 * g.V + HMC_THREADS - 1) / HMC_THREADS);
    const double scale = coeff * beta / lat.N;
    HR_FOR_N(lat.N, (k_gauge_force<NN><<<blocks, HMC_THREADS, 0, s>>>(g, static_cast<const cx<double> *>(U), F, scale)));
    HR_LAUNCH_CHECK("k_gauge_force");
    return HR_OK;
}

hr_status link_update_launch(const hr_lattice_desc &lat, void *U, const double *pi, double eps, cudaStream_t s)
{
    const GaugeGeom g = gauge_geom(lat);
    const unsigned blocks = (unsigned)((4 * g.V + HMC_THREADS - 1) / HMC_THREADS);
    HR_FOR_N(lat.N, (k_link_update<NN><<<blocks, HMC_THREADS, 0, s>>>(g, static_cast<cx<double> *>(U), pi, eps)));
    HR_LAUNCH_CHECK("k_link_update");
    return HR_OK;
}

}  // namespace

}  // namespace hr

using namespace hr;

extern "C" {

hr_status hr_gauge_action(const hr_lattice_desc *lat, const void *U_fund, double beta, double *S, void *stream)
{
    hr_status st = check_gauge_lat(lat);
    if (st != HR_OK) return st;
    if (!U_fund || !S) {
        set_error("hr_gauge_action: NULL argument");
        return HR_ERR_INVALID;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const GaugeGeom g = gauge_geom(*lat);
    const long blocks = (g.V + HMC_THREADS - 1) / HMC_THREADS;
    SumScratch ss;
    if ((st = ss.alloc(blocks, s)) != HR_OK) return st;
    HR_FOR_N(lat->N, (k_plaquette<NN><<<(unsigned)blocks, HMC_THREADS, 0, s>>>(
                          g, static_cast<const cx<double> *>(U_fund), ss.partials, ss.counter, ss.out)));
    HR_LAUNCH_CHECK("k_plaquette");
    double sum = 0;
    if ((st = read_sum(ss, &sum)) != HR_OK) return st;
    *S = beta * sum;
    return HR_OK;
}

hr_status hr_gauge_force(const hr_lattice_desc *lat, const void *U_fund, double beta, double coeff, double *F,
                         void *stream)
{
    hr_status st = check_gauge_lat(lat);
    if (st != HR_OK) return st;
    if (!U_fund || !F) {
        set_error("hr_gauge_force: NULL argument");
        return HR_ERR_INVALID;
    }
    return gauge_force_launch(*lat, U_fund, beta, coeff, F, reinterpret_cast<cudaStream_t>(stream));
}

hr_status hr_link_update(const hr_lattice_desc *lat, void *U_fund, const double *pi, double eps, void *stream)
{
    hr_status st = check_gauge_lat(lat);
    if (st != HR_OK) return st;
    if (!U_fund || !pi || !std::isfinite(eps)) {
        set_error("hr_link_update: NULL argument or non-finite step");
        return HR_ERR_INVALID;
    }
    return link_update_launch(*lat, U_fund, pi, eps, reinterpret_cast<cudaStream_t>(stream));
}

hr_status hr_momenta_energy(const hr_lattice_desc *lat, const double *pi, double *H, void *stream)
{
    hr_status st = check_gauge_lat(lat);
    if (st != HR_OK) return st;
    if (!pi || !H) {
        set_error("hr_momenta_energy: NULL argument");
        return HR_ERR_INVALID;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long n = lat_volume(*lat) * 4 * (lat->N * lat->N - 1);
    const long blocks = std::max(1L, std::min((n + HMC_THREADS - 1) / HMC_THREADS, 152L * 16));
    SumScratch ss;
    if ((st = ss.alloc(blocks, s)) != HR_OK) return st;
    k_sumsq<<<(unsigned)blocks, HMC_THREADS, 0, s>>>(pi, n, ss.partials, ss.counter, ss.out);
    HR_LAUNCH_CHECK("k_sumsq");
    double sum = 0;
    if ((st = read_sum(ss, &sum)) != HR_OK) return st;
    *H = 0.5 * T_FUND * sum;
    return HR_OK;
}

hr_status hr_md_trajectory(hr_gauge *g, void *U_fund, double *pi, const void *phi, const hr_md_params *p,
                           hr_md_stats *stats, void *stream)
{
    if (!g || !U_fund || !pi || !p || !stats || !(p->tau > 0) || p->nsteps < 1 ||
        (p->integrator != HR_MD_LEAPFROG && p->integrator != HR_MD_OMELYAN2) ||
        (phi && p->sys != HR_EO_PRECOND && p->sys != HR_FULL)) {
        set_error("hr_md_trajectory: bad arguments");
        return HR_ERR_INVALID;
    }
    hr_status st = check_gauge_lat(&g->lat);
    if (st != HR_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    memset(stats, 0, sizeof *stats);
    stats->status = HR_OK;
    const hr_lattice_desc &lat = g->lat;
    const long V = lat_volume(lat);
    const long ns = p->sys == HR_FULL ? V : V / 2;
    void *x = nullptr;
    if (phi) {
        // the solution of each force solve; zero, so that a chronological
        // initial guess (cg.use_initial_guess) starts the first solve from 0
        const size_t xb = field_rhs_bytes(ns, g->D, HR_F64);
        HR_CUDA_CHECK(cudaMallocAsync(&x, xb, s));
        HR_CUDA_CHECK(cudaMemsetAsync(x, 0, xb, s));
    }
    struct Free {
        void *p;
        cudaStream_t s;
        ~Free()
        {
            if (p) cudaFreeAsync(p, s);
        }
    } fx{x, s};
    // P(h): pi += h F = pi - (h / T_F) dS/de
    auto P = [&](double h) -> hr_status {
        const double coeff = -h / T_FUND;
        hr_status r = gauge_force_launch(lat, U_fund, p->beta, coeff, pi, s);
        if (r != HR_OK || !phi) return r;
        hr_cg_result res;
        r = hr_cg_solve_force(g, p->sys, phi, x, &p->cg, &res, nullptr, coeff, pi, stream);
        stats->cg_iters += res.iters;
        stats->max_true_rel_residual = std::max(stats->max_true_rel_residual, res.true_rel_residual);
        stats->force_evals += 1;
        return r;
    };
    // Q(h): U <- exp(i h pi) U, then the represented links follow
    auto Q = [&](double h) -> hr_status {
        hr_status r = link_update_launch(lat, U_fund, pi, h, s);
        if (r == HR_OK && phi) r = hr_gauge_update(g, U_fund, stream);
        return r;
    };
    const double h = p->tau / p->nsteps;
    const double lam = 0.1931833275037836;   // minimum-norm 2nd-order (Omelyan) parameter
    // the last momentum step of a step and the first of the next act on the
    // same links, so they are taken as one
    double carry = p->integrator == HR_MD_LEAPFROG ? 0.5 * h : lam * h;
    for (int k = 0; k < p->nsteps; k++) {
        if ((st = P(carry)) != HR_OK) break;
        if (p->integrator == HR_MD_LEAPFROG) {
            if ((st = Q(h)) != HR_OK) break;
            carry = k + 1 < p->nsteps ? h : 0.5 * h;
        } else {
            if ((st = Q(0.5 * h)) != HR_OK) break;
            if ((st = P((1.0 - 2.0 * lam) * h)) != HR_OK) break;
            if ((st = Q(0.5 * h)) != HR_OK) break;
            carry = k + 1 < p->nsteps ? 2.0 * lam * h : lam * h;
        }
    }
    if (st == HR_OK) st = P(carry);
    // the represented links match U_F at the end of the trajectory
    if (st == HR_OK && !phi) st = hr_gauge_update(g, U_fund, stream);
    stats->status = st;
    return st;
}

// H = (H_pi, S_g, S_f) for the links g represents (= U_fund); S_f =
// phi^dag A^-1 phi by one solve (to min(tol, 1e-11)) and one dot product
static hr_status hamiltonian(hr_gauge *g, const void *U_fund, const double *pi, const void *phi, void *x,
                             const hr_md_params *p, double H[3], void *stream)
{
    hr_status st = hr_momenta_energy(&g->lat, pi, &H[0], stream);
    if (st == HR_OK) st = hr_gauge_action(&g->lat, U_fund, p->beta, &H[1], stream);
    H[2] = 0;
    if (st != HR_OK || !phi) return st;
    hr_cg_params cg = p->cg;
    cg.tol_rel = std::min(cg.tol_rel, 1e-11);
    cg.use_initial_guess = 0;
    hr_cg_result r;
    st = hr_cg_solve(g, p->sys, phi, x, 1, &cg, &r, stream);
    if (st != HR_OK) return st;
    double d[2];
    st = hr_field_dot(&g->lat, p->sys == HR_FULL ? HR_FULL : HR_EVEN, HR_F64, phi, x, 1, d, stream);
    H[2] = d[0];
    return st;
}

hr_status hr_hmc_update(hr_gauge *g, void *U_fund, double *pi, const void *eta, double u_accept,
                        const hr_md_params *p, hr_hmc_result *res, void *stream)
{
    if (!g || !U_fund || !pi || !p || !res || !(u_accept >= 0.0) || !std::isfinite(u_accept) ||
        (eta && p->sys != HR_EO_PRECOND && p->sys != HR_FULL)) {
        set_error("hr_hmc_update: bad arguments");
        return HR_ERR_INVALID;
    }
    hr_status st = check_gauge_lat(&g->lat);
    if (st != HR_OK) return st;
    memset(res, 0, sizeof *res);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const hr_lattice_desc &lat = g->lat;
    const long V = lat_volume(lat);
    const long ns = p->sys == HR_FULL ? V : V / 2;
    const size_t fb = eta ? field_rhs_bytes(ns, g->D, HR_F64) : 0;
    const size_t ub = (size_t)V * 4 * lat.N * lat.N * 16;
    // [U_fund before the trajectory][phi][x]
    char *buf = nullptr;
    HR_CUDA_CHECK(cudaMallocAsync((void **)&buf, ub + 2 * fb, s));
    struct Free {
        char *p;
        cudaStream_t s;
        ~Free()
        {
            if (p) cudaFreeAsync(p, s);
        }
    } fbuf{buf, s};
    void *U0 = buf, *phi = eta ? buf + ub : nullptr, *x = eta ? buf + ub + fb : nullptr;
    if ((st = kernel_copy(U0, U_fund, ub, s)) != HR_OK) return st;
    // pseudofermion heat bath: phi = Dhat^dag eta (D^dag eta), so that
    // phi^dag (Dhat^dag Dhat)^-1 phi = eta^dag eta
    if (eta && (st = hr_dirac_dagger(g, p->sys, HR_F64, eta, phi, 1, stream)) != HR_OK) return st;
    if ((st = hamiltonian(g, U_fund, pi, phi, x, p, res->H0, stream)) != HR_OK) return st;
    if ((st = hr_md_trajectory(g, U_fund, pi, phi, p, &res->md, stream)) != HR_OK) return st;
    if ((st = hamiltonian(g, U_fund, pi, phi, x, p, res->H1, stream)) != HR_OK) return st;
    res->dH = (res->H1[0] + res->H1[1] + res->H1[2]) - (res->H0[0] + res->H0[1] + res->H0[2]);
    // Metropolis: accept with probability min(1, exp(-dH))
    res->accepted = std::isfinite(res->dH) && u_accept < std::exp(-res->dH);
    if (!res->accepted) {
        if ((st = kernel_copy(U_fund, U0, ub, s)) != HR_OK) return st;
        if ((st = hr_gauge_update(g, U_fund, stream)) != HR_OK) return st;
    }
    HR_CUDA_CHECK(cudaStreamSynchronize(s));
    return HR_OK;
}

}  // extern "C"
