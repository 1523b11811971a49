// hr_clover.cu -- the clover (Sec. 5.1.2) and exponential-clover (Sec. 5.1.3)
// diagonal.
//
//   D_ee + D_oo = (4+m) + c_sw (i/4) sum_{mu,nu} sigma_mu_nu F_mu_nu      (plain)
//               = (4+m) exp(c_sw/(4+m) (i/4) sum sigma F)                   (exponential)
//
// F_mu_nu(x) = (Q_mu_nu(x) - Q_mu_nu(x)^dag) / 8 with Q the four plaquettes of
// the (mu, nu) plane that have x as a corner, each as the closed loop through
// x (Eq. clover-term), taken in the fermion representation: since R is a
// homomorphism, R(leaf) of the fundamental loop (the antiperiodic signs cancel
// around a closed loop).  sigma_mu_nu = (i/2)[gamma_mu, gamma_nu] is block
// diagonal in the chiral basis of Sec. 2.2 (gamma5 = diag(1,1,-1,-1)), so the
// clover term is two Hermitian 2D x 2D blocks per site (spins 0,1 and 2,3).
//
// Build (once per gauge field, FP64): one thread block per site forms the 24
// represented leaves, the six F_mu_nu, both chiral blocks, the exponential
// when asked (Taylor series with scaling and squaring) and the inverse
// (Gauss-Jordan with partial pivoting), all in shared memory, and writes C
// and C^-1 in FP64 and FP32.  Records are AoSoA like the links: [kind
// C / C^-1][parity][32-site tile][block][entry][lane], so that a warp's load
// of one entry is one 512-byte (FP64) or 256-byte (FP32) line.
//
// Apply: one thread per site multiplies its spinor's two chiral halves by
// its blocks (C or C^-1).
#include <cmath>
#include <cstring>

#include "hr_api.cuh"
#include "hr_rep.cuh"

namespace hr {

namespace {

constexpr int CL_BUILD_THREADS = 128;
constexpr int CL_APPLY_THREADS = 128;

// the chiral blocks of sigma_mu_nu for the planes 01 02 03 12 13 23:
// upper (spins 0,1) (i/2)(e_mu e_nu^dag - e_nu e_mu^dag),
// lower (spins 2,3) (i/2)(e_mu^dag e_nu - e_nu^dag e_mu)
struct SigmaTab {
    double re[6][2][2][2], im[6][2][2][2];   // [plane][block][s][t]
};

SigmaTab sigma_table()
{
    // e_0 = -1, e_k = -i sigma_k  (Sec. 2.2)
    cx<double> e[4][2][2];
    const cx<double> z = {0, 0}, one = {1, 0}, mi = {0, -1}, pi = {0, 1};
    const cx<double> m1 = {-1, 0};
    cx<double> E0[2][2] = {{m1, z}, {z, m1}};
    cx<double> E1[2][2] = {{z, mi}, {mi, z}};          // -i sigma_1
    cx<double> E2[2][2] = {{z, m1}, {one, z}};         // -i sigma_2
    cx<double> E3[2][2] = {{mi, z}, {z, pi}};          // -i sigma_3
    memcpy(e[0], E0, sizeof E0);
    memcpy(e[1], E1, sizeof E1);
    memcpy(e[2], E2, sizeof E2);
    memcpy(e[3], E3, sizeof E3);
    auto mul = [](const cx<double> (&a)[2][2], const cx<double> (&b)[2][2], bool da, bool db, cx<double> (&c)[2][2]) {
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) {
                cx<double> s = {0, 0};
                for (int k = 0; k < 2; k++) {
                    const cx<double> x = da ? conj(a[k][i]) : a[i][k];
                    const cx<double> y = db ? conj(b[j][k]) : b[k][j];
                    s = s + x * y;
                }
                c[i][j] = s;
            }
    };
    SigmaTab t;
    int pl = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++, pl++) {
            cx<double> a[2][2], b[2][2];
            for (int blk = 0; blk < 2; blk++) {
                if (blk == 0) {
                    mul(e[mu], e[nu], false, true, a);
                    mul(e[nu], e[mu], false, true, b);
                } else {
                    mul(e[mu], e[nu], true, false, a);
                    mul(e[nu], e[mu], true, false, b);
                }
                for (int s = 0; s < 2; s++)
                    for (int u = 0; u < 2; u++) {
                        const cx<double> d = a[s][u] - b[s][u];
                        // (i/2) d
                        t.re[pl][blk][s][u] = -0.5 * d.im;
                        t.im[pl][blk][s][u] = 0.5 * d.re;
                    }
            }
        }
    return t;
}

struct CloverBuildParams {
    int d[4];
    long V;
    long ntiles;
    double m4, csw;
    int expo;
    const cx<double> *U;      // [V][4][N][N]
    char *rec64, *rec32;      // AoSoA records (rec32 may be null)
    int *err;                 // singular-block counter
    SigmaTab sig;
};

__device__ __forceinline__ size_t cl_index(long ntiles, int E, int kind, int parity, long tile, int blk, int e,
                                           int lane)
{
    return (((((size_t)kind * 2 + parity) * ntiles + tile) * 2 + blk) * E + e) * HR_TILE + lane;
}

// one thread block per site x
template <int N, int REP>
__global__ void __launch_bounds__(CL_BUILD_THREADS) k_clover_build(const CloverBuildParams p)
{
    constexpr int D = rep_dim(N, REP);
    constexpr int n = 2 * D;      // chiral block dimension
    constexpr int E = n * n;
    __shared__ cx<double> leaf[24][D][D];   // reused below as the augmented matrix
    __shared__ cx<double> F[6][D][D];
    __shared__ cx<double> Cm[n][n];
    __shared__ cx<double> Tm[n][n];
    __shared__ int s_piv;
    __shared__ cx<double> s_inv;
    __shared__ int s_bad;
    static_assert(sizeof(leaf) >= sizeof(cx<double>) * n * 2 * n, "augmented matrix must fit in the leaf buffer");
    cx<double>(*A)[2 * n] = reinterpret_cast<cx<double>(*)[2 * n]>(&leaf[0][0][0]);

    const long x = blockIdx.x;
    const int tid = threadIdx.x;
    int c[4];
    {
        long r = x;
        c[3] = (int)(r % p.d[3]);
        r /= p.d[3];
        c[2] = (int)(r % p.d[2]);
        r /= p.d[2];
        c[1] = (int)(r % p.d[1]);
        c[0] = (int)(r / p.d[1]);
    }
    auto lex = [&](const int (&q)[4]) {
        return (((long)q[0] * p.d[1] + q[1]) * p.d[2] + q[2]) * p.d[3] + q[3];
    };
    // ---- the 24 leaves, represented ----
    if (tid < 24) {
        int pl = tid / 4, k = tid % 4;
        const int planes[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
        const int mu = planes[pl][0], nu = planes[pl][1];
        // corner offsets of leaf k: the loop starts at x and runs
        //   k = 0: +mu +nu -mu -nu     k = 1: +nu -mu -nu +mu
        //   k = 2: -mu -nu +mu +nu     k = 3: -nu +mu +nu -mu
        const int dirs[4][4] = {{mu, nu, mu, nu}, {nu, mu, nu, mu}, {mu, nu, mu, nu}, {nu, mu, nu, mu}};
        const int sgn[4][4] = {{1, 1, -1, -1}, {1, -1, -1, 1}, {-1, -1, 1, 1}, {-1, 1, 1, -1}};
        int q[4] = {c[0], c[1], c[2], c[3]};
        cx<double> P[N][N];
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int j = 0; j < N; j++) P[i][j] = {i == j ? 1.0 : 0.0, 0.0};
        for (int st = 0; st < 4; st++) {
            const int dd = dirs[k][st], s = sgn[k][st];
            // a forward step uses U_dd(q); a backward step U_dd(q - dd)^dag
            int from[4] = {q[0], q[1], q[2], q[3]};
            if (s < 0) from[dd] = (from[dd] - 1 + p.d[dd]) % p.d[dd];
            const cx<double> *u = p.U + ((size_t)lex(from) * 4 + dd) * N * N;
            cx<double> T[N][N];
#pragma unroll
            for (int i = 0; i < N; i++)
#pragma unroll
                for (int j = 0; j < N; j++) {
                    cx<double> acc = {0, 0};
#pragma unroll
                    for (int l = 0; l < N; l++) {
                        const cx<double> m = s > 0 ? u[l * N + j] : conj(u[j * N + l]);
                        cmac(acc, P[i][l], m);
                    }
                    T[i][j] = acc;
                }
#pragma unroll
            for (int i = 0; i < N; i++)
#pragma unroll
                for (int j = 0; j < N; j++) P[i][j] = T[i][j];
            q[dd] = s > 0 ? (q[dd] + 1) % p.d[dd] : from[dd];
        }
        // R(leaf) entry by entry with the folded sums (compile-time indices)
        static_for<0, D>([&](auto AA) {
            static_for<0, D>([&](auto BB) {
                leaf[tid][decltype(AA)::value][decltype(BB)::value] =
                    rep_entry<N, REP, decltype(AA)::value, decltype(BB)::value>(P);
            });
        });
    }
    __syncthreads();
    // ---- F_mu_nu = (Q - Q^dag) / 8 ----
    for (int t = tid; t < 6 * D * D; t += blockDim.x) {
        const int pl = t / (D * D), a = (t / D) % D, b = t % D;
        cx<double> s = {0, 0};
        for (int k = 0; k < 4; k++) s = s + leaf[pl * 4 + k][a][b] - conj(leaf[pl * 4 + k][b][a]);
        F[pl][a][b] = 0.125 * s;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    const int parity = (c[0] + c[1] + c[2] + c[3]) & 1;
    const long ih = x / 2;
    const long tile = ih / HR_TILE;
    const int lane = (int)(ih % HR_TILE);
    for (int blk = 0; blk < 2; blk++) {
        // X = (i/2) sum_{mu<nu} s_blk(mu,nu) (x) F_mu_nu, Hermitian n x n
        for (int t = tid; t < E; t += blockDim.x) {
            const int r = t / n, cc = t % n;
            const int s = r / D, a = r % D, u = cc / D, b = cc % D;
            cx<double> acc = {0, 0};
            for (int pl = 0; pl < 6; pl++) {
                const cx<double> sg = {p.sig.re[pl][blk][s][u], p.sig.im[pl][blk][s][u]};
                acc = acc + sg * F[pl][a][b];
            }
            const cx<double> X = {-0.5 * acc.im, 0.5 * acc.re};   // (i/2) acc
            if (!p.expo) {
                Cm[r][cc] = p.csw * X + cx<double>{r == cc ? p.m4 : 0.0, 0.0};
            } else {
                Cm[r][cc] = (p.csw / p.m4) * X;   // Y, exponentiated below
            }
        }
        __syncthreads();
        if (p.expo) {
            // E = exp(Y): Y / 2^s with |Y / 2^s|_F <= 1/2, Taylor to order 16, s squarings
            __shared__ double s_nrm;
            __shared__ int s_sq;
            if (tid == 0) {
                double nf = 0;
                for (int r = 0; r < n; r++)
                    for (int cc = 0; cc < n; cc++) nf += Cm[r][cc].re * Cm[r][cc].re + Cm[r][cc].im * Cm[r][cc].im;
                nf = sqrt(nf);
                int sq = 0;
                while (nf > 0.5 && sq < 60) {
                    nf *= 0.5;
                    sq++;
                }
                s_sq = sq;
                s_nrm = ldexp(1.0, -sq);
            }
            __syncthreads();
            for (int t = tid; t < E; t += blockDim.x) {
                const int r = t / n, cc = t % n;
                Cm[r][cc] = s_nrm * Cm[r][cc];                                     // Y
                A[r][cc] = cx<double>{r == cc ? 1.0 : 0.0, 0.0} + (1.0 / 16) * Cm[r][cc];   // E_16
            }
            __syncthreads();
            for (int k = 15; k >= 1; k--) {
                for (int t = tid; t < E; t += blockDim.x) {
                    const int r = t / n, cc = t % n;
                    cx<double> acc = {0, 0};
                    for (int l = 0; l < n; l++) cmac(acc, Cm[r][l], A[l][cc]);
                    Tm[r][cc] = acc;
                }
                __syncthreads();
                for (int t = tid; t < E; t += blockDim.x) {
                    const int r = t / n, cc = t % n;
                    A[r][cc] = cx<double>{r == cc ? 1.0 : 0.0, 0.0} + (1.0 / k) * Tm[r][cc];
                }
                __syncthreads();
            }
            for (int q = 0; q < s_sq; q++) {
                for (int t = tid; t < E; t += blockDim.x) {
                    const int r = t / n, cc = t % n;
                    cx<double> acc = {0, 0};
                    for (int l = 0; l < n; l++) cmac(acc, A[r][l], A[l][cc]);
                    Tm[r][cc] = acc;
                }
                __syncthreads();
                for (int t = tid; t < E; t += blockDim.x) A[t / n][t % n] = Tm[t / n][t % n];
                __syncthreads();
            }
            for (int t = tid; t < E; t += blockDim.x) Cm[t / n][t % n] = p.m4 * A[t / n][t % n];
            __syncthreads();
        }
        // ---- store C, then invert by Gauss-Jordan on [C | 1] ----
        for (int t = tid; t < E; t += blockDim.x) {
            const int r = t / n, cc = t % n;
            const cx<double> v = Cm[r][cc];
            const size_t at = cl_index(p.ntiles, E, 0, parity, tile, blk, t, lane);
            reinterpret_cast<double2 *>(p.rec64)[at] = make_double2(v.re, v.im);
            if (p.rec32) reinterpret_cast<float2 *>(p.rec32)[at] = make_float2((float)v.re, (float)v.im);
            A[r][cc] = v;
            A[r][n + cc] = {r == cc ? 1.0 : 0.0, 0.0};
        }
        __syncthreads();
        for (int k = 0; k < n; k++) {
            if (tid == 0) {
                int piv = k;
                double best = -1;
                for (int i = k; i < n; i++) {
                    const double a = A[i][k].re * A[i][k].re + A[i][k].im * A[i][k].im;
                    if (a > best) {
                        best = a;
                        piv = i;
                    }
                }
                if (!(best > 0) || !isfinite(best)) s_bad = 1;
                s_piv = piv;
                // the pivot's reciprocal, one division per pivot
                const cx<double> pv = A[piv][k];
                const double in2 = 1.0 / (pv.re * pv.re + pv.im * pv.im);
                s_inv = {pv.re * in2, -pv.im * in2};
            }
            __syncthreads();
            const int piv = s_piv;
            if (piv != k)
                for (int j = tid; j < 2 * n; j += blockDim.x) {
                    const cx<double> t = A[k][j];
                    A[k][j] = A[piv][j];
                    A[piv][j] = t;
                }
            __syncthreads();
            // the columns j < k of the left half are already unit columns, so
            // row k is zero there: only the columns k .. 2n-1 change
            const cx<double> inv = s_inv;
            const int w = 2 * n - k;
            for (int j = k + tid; j < 2 * n; j += blockDim.x) A[k][j] = A[k][j] * inv;
            __syncthreads();
            // factors of the other rows, taken before their column k changes
            for (int i = tid; i < n; i += blockDim.x) Tm[0][i] = i == k ? cx<double>{0, 0} : A[i][k];
            __syncthreads();
            for (int t = tid; t < n * w; t += blockDim.x) {
                const int i = t / w, j = k + t % w;
                if (i == k) continue;
                const cx<double> f = Tm[0][i];
                A[i][j] = A[i][j] - f * A[k][j];
            }
            __syncthreads();
        }
        for (int t = tid; t < E; t += blockDim.x) {
            const int r = t / n, cc = t % n;
            const cx<double> v = A[r][n + cc];
            const size_t at = cl_index(p.ntiles, E, 1, parity, tile, blk, t, lane);
            reinterpret_cast<double2 *>(p.rec64)[at] = make_double2(v.re, v.im);
            if (p.rec32) reinterpret_cast<float2 *>(p.rec32)[at] = make_float2((float)v.re, (float)v.im);
        }
        __syncthreads();
    }
    if (tid == 0 && s_bad) atomicAdd(p.err, 1);
}

struct CloverApplyParams {
    long vh, ntiles;
    int parity, kind, nrhs;
    const char *rec;
    FieldView in, out;
};

// out = C_blk in per chiral half (C or C^-1 of the site's parity)
template <int P, int D>
__global__ void __launch_bounds__(CL_APPLY_THREADS) k_clover_apply(const CloverApplyParams a)
{
    using R = typename St<P>::R;
    using V2 = typename std::conditional<P == HR_F64, double2, float2>::type;
    constexpr int n = 2 * D, E = n * n;
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.vh) return;
    const long tile = i / HR_TILE;
    const int lane = (int)(i % HR_TILE);
    cx<R> psi[4][D], out[4][D];
    SpinorIO<P, D>::load_rw(a.in, rhs, i, psi);
    const V2 *rec = reinterpret_cast<const V2 *>(a.rec);
#pragma unroll
    for (int blk = 0; blk < 2; blk++)
#pragma unroll
        for (int r = 0; r < n; r++) {
            cx<R> acc = {0, 0};
#pragma unroll
            for (int cc = 0; cc < n; cc++) {
                const V2 m = __ldg(&rec[cl_index(a.ntiles, E, a.kind, a.parity, tile, blk, r * n + cc, lane)]);
                cmac(acc, cx<R>{(R)m.x, (R)m.y}, psi[2 * blk + cc / D][cc % D]);
            }
            out[2 * blk + r / D][r % D] = acc;
        }
    SpinorIO<P, D>::store(a.out, rhs, i, out);
}

#define HR_CL_PAIRS(X) X(2, HR_FUND) X(2, HR_ADJ) X(2, HR_SYM) X(3, HR_FUND) X(3, HR_ADJ) X(3, HR_SYM) \
    X(3, HR_ASYM) X(4, HR_FUND) X(4, HR_ASYM) X(4, HR_ASYM_REAL)

}  // namespace

size_t clover_record_bytes(const hr_gauge *g, int P)
{
    const int n = 2 * g->D;
    return (size_t)2 * 2 * g->geom.ntiles * 2 * n * n * HR_TILE * (P == HR_F64 ? 16 : 8);
}

hr_status clover_build(hr_gauge *g, const void *U_fund, cudaStream_t s)
{
    const bool want32 = (g->prec_mask >> HR_F32) & 1u;
    for (int P : {(int)HR_F64, (int)HR_F32}) {
        if (P == HR_F32 && !want32) continue;
        if (!g->cl[P]) {
            const size_t b = clover_record_bytes(g, P);
            cudaError_t e = cudaMalloc(&g->cl[P], b);
            if (e != cudaSuccess) {
                g->cl[P] = nullptr;
                cudaGetLastError();
                set_error("clover: cannot allocate %zu bytes", b);
                return HR_ERR_NOMEM;
            }
            // the padding lanes of the last tile hold zeros, never NaNs
            HR_CUDA_CHECK(cudaMemsetAsync(g->cl[P], 0, b, s));
        }
    }
    CloverBuildParams p;
    memset(&p, 0, sizeof p);
    for (int i = 0; i < 4; i++) p.d[i] = g->lat.dims[i];
    p.V = lat_volume(g->lat);
    p.ntiles = g->geom.ntiles;
    p.m4 = 4.0 + g->lat.m0;
    p.csw = g->csw;
    p.expo = g->clover_mode == HR_CLOVER_EXP;
    p.U = static_cast<const cx<double> *>(U_fund);
    p.rec64 = static_cast<char *>(g->cl[HR_F64]);
    p.rec32 = want32 ? static_cast<char *>(g->cl[HR_F32]) : nullptr;
    p.err = g->err;
    p.sig = sigma_table();
    HR_CUDA_CHECK(cudaMemsetAsync(g->err, 0, sizeof(int), s));
    bool done = false;
#define HR_CLB(N_, R_)                                                                           \
    if (!done && g->lat.N == N_ && g->lat.rep == R_) {                                          \
        k_clover_build<N_, R_><<<(unsigned)p.V, CL_BUILD_THREADS, 0, s>>>(p);                  \
        done = true;                                                                             \
    }
    HR_CL_PAIRS(HR_CLB)
#undef HR_CLB
    if (!done) {
        set_error("clover: SU(%d) representation %d not compiled", g->lat.N, (int)g->lat.rep);
        return HR_ERR_UNSUPPORTED;
    }
    HR_LAUNCH_CHECK("k_clover_build");
    int bad = 0;
    HR_CUDA_CHECK(cudaMemcpyAsync(&bad, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    HR_CUDA_CHECK(cudaStreamSynchronize(s));
    if (bad) {
        set_error("clover: %d singular or non-finite clover blocks", bad);
        return HR_ERR_NONFINITE;
    }
    return HR_OK;
}

hr_status clover_apply(const hr_gauge *g, int P, int parity, int kind, const FieldView &in, const FieldView &out,
                       int nrhs, cudaStream_t s)
{
    if ((P != HR_F64 && P != HR_F32) || !g->cl[P]) {
        set_error("clover: precision %d has no clover records (FP64 and FP32 only)", P);
        return HR_ERR_UNSUPPORTED;
    }
    CloverApplyParams a;
    a.vh = g->geom.vh;
    a.ntiles = g->geom.ntiles;
    a.parity = parity;
    a.kind = kind;
    a.nrhs = nrhs;
    a.rec = static_cast<const char *>(g->cl[P]);
    a.in = in;
    a.out = out;
    const dim3 grid((unsigned)((a.vh + CL_APPLY_THREADS - 1) / CL_APPLY_THREADS), (unsigned)nrhs);
#define HR_CLA(D_)                                                                                    \
    case D_:                                                                                          \
        if (P == HR_F64)                                                                              \
            k_clover_apply<HR_F64, D_><<<grid, CL_APPLY_THREADS, 0, s>>>(a);                          \
        else                                                                                          \
            k_clover_apply<HR_F32, D_><<<grid, CL_APPLY_THREADS, 0, s>>>(a);                          \
        break;
    switch (g->D) {
        HR_CLA(2) HR_CLA(3) HR_CLA(4) HR_CLA(6) HR_CLA(8)
    default:
        set_error("clover: representation dimension %d not compiled", g->D);
        return HR_ERR_UNSUPPORTED;
    }
#undef HR_CLA
    HR_LAUNCH_CHECK("k_clover_apply");
    return HR_OK;
}

}  // namespace hr

using namespace hr;

extern "C" hr_status hr_gauge_set_clover(hr_gauge *g, const void *U_fund, double csw, hr_clover_mode mode,
                                         void *stream)
{
    if (!g || (mode != HR_CLOVER_NONE && (!U_fund || !std::isfinite(csw))) ||
        (mode != HR_CLOVER_NONE && mode != HR_CLOVER_PLAIN && mode != HR_CLOVER_EXP)) {
        set_error("hr_gauge_set_clover: bad arguments");
        return HR_ERR_INVALID;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (mode == HR_CLOVER_NONE) {
        HR_CUDA_CHECK(cudaStreamSynchronize(s));
        for (int P = 0; P < HR_NPREC; P++)
            if (g->cl[P]) {
                cudaFree(g->cl[P]);
                g->cl[P] = nullptr;
            }
        g->clover_mode = HR_CLOVER_NONE;
        g->csw = 0;
        return HR_OK;
    }
    if (!(g->prec_mask & (1u << HR_F64))) {
        set_error("hr_gauge_set_clover: the handle must hold FP64 links");
        return HR_ERR_INVALID;
    }
    g->clover_mode = mode;
    g->csw = csw;
    hr_status st = clover_build(g, U_fund, s);
    if (st != HR_OK) {
        g->clover_mode = HR_CLOVER_NONE;
        g->csw = 0;
    }
    return st;
}
