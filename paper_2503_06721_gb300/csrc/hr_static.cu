// hr_static.cu -- hr_field_dot_static: the field dot product <a, b> of
// hr_field_dot, for callers that must not allocate device memory.  It
// accepts every (representation dimension, precision) that hr_field_dot
// accepts and returns the same value up to rounding: both sum in FP64 and
// combine the per-block partials in double-double, but this kernel runs a
// fixed number of blocks, so each thread first accumulates several sites
// (compensated with TwoSum) and the summation order differs.
//
// Who needs it: code that runs where a device allocation is not allowed or
// not acceptable -- for example a caller whose device memory is entirely
// owned by another allocator (a framework's caching pool), a latency-critical
// loop that cannot afford the implicit device synchronisation of
// cudaMalloc/cudaFree, or host code inside a region that must not touch the
// allocator at all.  hr_field_dot takes its reduction scratch from
// cudaMallocAsync; this entry point takes it from a fixed array compiled into
// the library instead, and calls no allocating routine.
//
// The array (hr_dot_scratch) lives in device global memory for as long as
// the library is loaded, on every GPU that loads it.  Every call shares it and
// it keeps the previous call's contents: each call clears the tickets it uses
// before launching.  Calls that overlap on the GPU (different streams, or
// different host threads without ordering) race on the array.
#include <mutex>

#include "hr_api.cuh"

namespace hr {

// limits of the fixed scratch: right-hand sides per call and reduction blocks
constexpr int STATIC_DOT_MAX_RHS = 16;
// fixed upper bound on the blocks of one launch: it sizes the partials array;
// lattices with more sites than blocks x threads are covered by each thread
// taking several sites (grid-stride loop)
constexpr int STATIC_DOT_BLOCKS = 1216;
constexpr int STATIC_DOT_THREADS = 256;

// [tickets: MAX_RHS unsigned (padded to 256 B)] [results: MAX_RHS x 2 doubles]
// [partials: MAX_RHS x BLOCKS x 2 doubles]  -- about 311 KB
constexpr size_t STATIC_DOT_TICKETS = 256;
constexpr size_t STATIC_DOT_RESULTS = 256;
constexpr size_t STATIC_DOT_BYTES =
    STATIC_DOT_TICKETS + STATIC_DOT_RESULTS + sizeof(double) * 2 * STATIC_DOT_MAX_RHS * STATIC_DOT_BLOCKS;

static __device__ __align__(256) unsigned char hr_dot_scratch[STATIC_DOT_BYTES];

// grid-stride variant of the dot kernel: a fixed number of blocks, so the
// per-block partials fit the fixed array for any lattice size
template <int D, int P>
__global__ void __launch_bounds__(STATIC_DOT_THREADS) k_dot_static(long nsites, FieldView a, FieldView b,
                                                                 unsigned char *scr)
{
    const int rhs = blockIdx.y;
    unsigned *tickets = reinterpret_cast<unsigned *>(scr);
    double *results = reinterpret_cast<double *>(scr + STATIC_DOT_TICKETS);
    double *partials = reinterpret_cast<double *>(scr + STATIC_DOT_TICKETS + STATIC_DOT_RESULTS);
    using R = typename St<P>::R;
    // per-thread running sums kept as (hi, lo) pairs: TwoSum moves each
    // addition's rounding error into lo, so a thread that takes many sites
    // loses no more than one that takes one
    double hi[2] = {0, 0}, lo[2] = {0, 0};
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nsites; i += (long)gridDim.x * blockDim.x) {
        cx<R> x[4][D], y[4][D];
        SpinorIO<P, D>::load_rw(a, rhs, i, x);
        SpinorIO<P, D>::load_rw(b, rhs, i, y);
        double s0 = 0, s1 = 0;
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) {
                const double xr = to_f64(x[s][c].re), xi = to_f64(x[s][c].im);
                const double yr = to_f64(y[s][c].re), yi = to_f64(y[s][c].im);
                s0 += xr * yr + xi * yi;
                s1 += xr * yi - xi * yr;
            }
        double t, e;
        two_sum(hi[0], s0, t, e);
        hi[0] = t;
        lo[0] += e;
        two_sum(hi[1], s1, t, e);
        hi[1] = t;
        lo[1] += e;
    }
    double v[2] = {hi[0] + lo[0], hi[1] + lo[1]};
    double tot[2];
    if (grid_reduce<2>(v, partials + (size_t)rhs * gridDim.x * 2, tickets + rhs, gridDim.x, blockIdx.x, tot)) {
        results[rhs * 2 + 0] = tot[0];
        results[rhs * 2 + 1] = tot[1];
    }
}

// device address of hr_dot_scratch, looked up once per device with that
// device current (the host-side name is only a stand-in for it)
static unsigned char *static_scratch_for_current_device()
{
    static std::mutex mu;
    static unsigned char *addr[64] = {nullptr};
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cuda_fail(e, "cudaGetDevice");
        return nullptr;
    }
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d out of range", dev);
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, hr_dot_scratch);
        if (e != cudaSuccess) {
            cuda_fail(e, "cudaGetSymbolAddress(hr_dot_scratch)");
            return nullptr;
        }
        addr[dev] = reinterpret_cast<unsigned char *>(p);
    }
    return addr[dev];
}

}  // namespace hr

using namespace hr;

extern "C" hr_status hr_field_dot_static(const hr_lattice_desc *lat, hr_parity par, hr_prec prec, const void *a,
                                         const void *b, int nrhs, double *out, void *stream)
{
    hr_status st = check_lattice(lat);
    if (st != HR_OK) return st;
    if (!a || !b || !out || prec < HR_F64 || prec > HR_DF64 || par < HR_EVEN || par > HR_EO_PRECOND) {
        set_error("hr_field_dot_static: bad arguments");
        return HR_ERR_INVALID;
    }
    if (nrhs < 1 || nrhs > STATIC_DOT_MAX_RHS) {
        set_error("hr_field_dot_static: nrhs = %d outside 1..%d (the size of its fixed scratch)", nrhs,
                  STATIC_DOT_MAX_RHS);
        return HR_ERR_INVALID;
    }
    unsigned char *scr = static_scratch_for_current_device();
    if (!scr) return HR_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long V = lat_volume(*lat);
    const long ns = par == HR_FULL ? V : V / 2;
    const int D = rep_dim(lat->N, lat->rep);
    // tickets must start at zero; results and partials are overwritten
    HR_CUDA_CHECK(cudaMemsetAsync(scr, 0, STATIC_DOT_TICKETS, s));
    FieldView va = make_view(const_cast<void *>(a), ns, D, prec), vb = make_view(const_cast<void *>(b), ns, D, prec);
    long blocks = (ns + STATIC_DOT_THREADS - 1) / STATIC_DOT_THREADS;
    if (blocks > STATIC_DOT_BLOCKS) blocks = STATIC_DOT_BLOCKS;
    const dim3 grid((unsigned)blocks, (unsigned)nrhs);
    HR_FOR_D(D, HR_FOR_PX(prec, PN, (k_dot_static<DD, PN><<<grid, STATIC_DOT_THREADS, 0, s>>>(ns, va, vb, scr))));
    HR_LAUNCH_CHECK("k_dot_static");
    HR_CUDA_CHECK(cudaMemcpyAsync(out, scr + STATIC_DOT_TICKETS, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, s));
    HR_CUDA_CHECK(cudaStreamSynchronize(s));
    return HR_OK;
}
