// Host-side checks of library building blocks that are __host__ __device__
// (compiled as plain host code by tests/test_host_checks_cpu.py):
//   1. f32_rn / f64_of / df_split return exactly what the IEEE conversions of
//      the host return (round to nearest even) on random bit patterns of every
//      exponent, on exact ties, on roundings that carry into the exponent and
//      on special values;
//   2. rep_entry (one entry of R(U), folded sums) and rep_row (a row with a
//      run-time index) agree with represent() (the plain sums over the basis
//      elements) to rounding, for every compiled (N, representation) that the
//      represent kernel forms entry by entry, on random complex matrices.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "hr_rep.cuh"

using namespace hr;

static uint64_t bd(double v) { uint64_t u; memcpy(&u, &v, 8); return u; }
static uint32_t bf(float v) { uint32_t u; memcpy(&u, &v, 4); return u; }
static bool same(float a, float b) { return bf(a) == bf(b) || (std::isnan(a) && std::isnan(b)); }
static bool same(double a, double b) { return bd(a) == bd(b) || (std::isnan(a) && std::isnan(b)); }

static long check_conversions()
{
    std::mt19937_64 rng(20250306721ull);
    long bad = 0;
    auto check = [&](double v) {
        const float want = (float)v;
        if (!same(f32_rn(v), want)) bad++;
        if (!(std::isnan(v) || std::isinf(v))) {
            const df s = df_split(v);
            if (!same(s.hi, want) || !same(s.lo, (float)(v - (double)want))) bad++;
        }
        if (!same(f64_of(want), (double)want)) bad++;
    };
    for (long i = 0; i < 2000000; i++) {
        uint64_t u = rng();
        double v;
        memcpy(&v, &u, 8);
        check(v);
        uint64_t w = (rng() & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(900 + rng() % 300) << 52);
        memcpy(&v, &w, 8);
        check(v);
        w = (w & ~0x1FFFFFFFull) | 0x10000000ull;   // exact tie at the last kept bit
        memcpy(&v, &w, 8);
        check(v);
        w = (w & 0xFFF0000000000000ull) | 0x000FFFFFF0000001ull;   // carry into the exponent
        memcpy(&v, &w, 8);
        check(v);
    }
    const double sp[] = {0.0, -0.0, 1.0, -1.0, 1e-30, -1e-30, 1e-45, 3e38, 3.4028235e38, 3.4028235677973366e38,
                         INFINITY, -INFINITY, NAN, 1.0 + 0x1p-24, 1.0 + 0x1p-23 + 0x1p-24, 0x1p-74, 0x1p-75,
                         0x1.fffffffffffffp-75, 0x1p127, 0x1.ffffffp127, 0x1p-126, 0x1p-149};
    for (double v : sp) check(v);
    return bad;
}

template <int N, int REP>
static double check_rep(unsigned seed)
{
    constexpr int D = rep_dim(N, REP);
    std::mt19937 rng(seed);
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    cx<double> U[N][N];
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) U[i][j] = {u(rng), u(rng)};
    cx<double> R[D][D];
    represent<N, REP>(U, R);
    double err = 0, mx = 0;
    for (int a = 0; a < D; a++)
        for (int b = 0; b < D; b++) mx = std::fmax(mx, std::hypot(R[a][b].re, R[a][b].im));
    auto cmp = [&](cx<double> got, cx<double> want) {
        err = std::fmax(err, std::fabs(got.re - want.re));
        if (!rep_real(REP)) err = std::fmax(err, std::fabs(got.im - want.im));
    };
    static_for<0, D>([&](auto AA) {
        static_for<0, D>([&](auto BB) {
            constexpr int a = decltype(AA)::value, b = decltype(BB)::value;
            cmp(rep_entry<N, REP, a, b>(U), R[a][b]);
        });
    });
    auto ld = [&](int i, int k) { return U[i][k]; };
    const int nrow = REP == HR_ADJ ? noff(N) : D;
    for (int r = 0; r < nrow; r++) {
        cx<double> e[D];
        rep_row<N, REP>(r, ld, e);
        for (int q = 0; q < D; q++) cmp(e[q], R[r][q]);
    }
    return err / mx;
}

int main()
{
    const long bad = check_conversions();
    double e = 0;
    for (unsigned s = 1; s <= 20; s++) {
        e = std::fmax(e, check_rep<2, HR_FUND>(s));
        e = std::fmax(e, check_rep<2, HR_ADJ>(s));
        e = std::fmax(e, check_rep<2, HR_SYM>(s));
        e = std::fmax(e, check_rep<3, HR_FUND>(s));
        e = std::fmax(e, check_rep<3, HR_ADJ>(s));
        e = std::fmax(e, check_rep<3, HR_SYM>(s));
        e = std::fmax(e, check_rep<3, HR_ASYM>(s));
        e = std::fmax(e, check_rep<4, HR_FUND>(s));
        e = std::fmax(e, check_rep<4, HR_ADJ>(s));
        e = std::fmax(e, check_rep<4, HR_SYM>(s));
        e = std::fmax(e, check_rep<4, HR_ASYM>(s));
        e = std::fmax(e, check_rep<4, HR_ASYM_REAL>(s));
        e = std::fmax(e, check_rep<8, HR_FUND>(s));
    }
    printf("conversion mismatches %ld\nrepresentation max relative difference %.3e\n", bad, e);
    return (bad == 0 && e < 4e-15) ? 0 : 1;
}
