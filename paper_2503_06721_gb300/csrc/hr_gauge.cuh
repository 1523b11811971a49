// hr_gauge.cuh -- the gauge handle and the per-(N, representation) entry
// points that the C ABI dispatches to.
#pragma once

#include <vector>

#include "hr_dslash.cuh"

struct hr_gauge {
    hr_lattice_desc lat;
    hr::Geom geom;
    int D;
    bool real;            // ADJ: represented links stored as reals
    unsigned prec_mask;
    unsigned link_modes;
    hr_link_mode mode;
    // link records per [precision][output parity]
    void *rep[HR_NPREC][2];
    void *fund[HR_NPREC][2];
    size_t rep_bytes[HR_NPREC], fund_bytes[HR_NPREC];
    // T_R^a tables for the force, [(N*N-1)][D][D] complex double
    double *TR;
    // field workspace (operator/force temporaries, solver vectors; grown on demand)
    char *ws;
    size_t ws_bytes;
    // reduction tickets, partial sums and solver state -- kept apart from ws so
    // that no field temporary ever overwrites the zeroed tickets
    char *scr;
    size_t scr_bytes;
    int *err;             // device counter of failures found by kernels (singular clover blocks)
    void *pinned;         // host-mapped pinned mailbox for the solver's small host transfers
    size_t pinned_bytes;
    int device;
    // hopping-kernel variant per [precision][rebuilt links][epilogue][nrhs > 1]
    // chosen by the autotuner; -1 = not tuned (a fixed default applies)
    signed char tuned[HR_NPREC][2][3][2];
    int force_variant;    // >= 0: every launch uses this variant (testing)
    signed char auto_mode[HR_NPREC];   // HR_LINKS_AUTO: the tuned mode per precision, -1 = not tuned
    int autotune;         // 1: the solver tunes its inner precision before iterating
    // clover diagonal (Sec. 5.1.2-5.1.3): mode, coefficient and the C / C^-1 records
    // per precision (FP64 and FP32 only), AoSoA [kind][parity][tile][block][entry][lane]
    int clover_mode;
    double csw;
    void *cl[HR_NPREC];
};

namespace hr {

struct RepOut {
    void *rep[HR_NPREC];    // record base for this parity per precision (nullptr = skip)
    void *fund[HR_NPREC];
};

// per-(N, REP) instantiated operations (hr_gauge_inst.cu)
template <int N, int REP>
hr_status represent_launch(const hr_gauge &g, const double2 *UF, cudaStream_t stream);

struct ForceParams {
    Geom g;
    int parity;             // sites of this parity own the links processed
    int arith;              // HR_F64: FP64 arithmetic, HR_DF64: float-float
    const void *links;      // stored records of this parity (U_R with signs), FP64 or DF64 as arith
    FieldView X_here, Y_here;   // FULL-field views of X, Y at sites of `parity`
    FieldView X_nb, Y_nb;       // views of the opposite parity
    const double *TR;
    double coeff;
    double *F;              // [V][4][N*N-1] lexicographic
};
template <int N, int REP>
hr_status force_launch(const ForceParams &fp, cudaStream_t stream);

// the colour-parallel hopping kernel of the large pairs (hr_dslash_colour.cuh)
template <int N, int REP, int P>
hr_status launch_colour(const HopParams &prm, int epi, cudaStream_t stream);

// precision dispatch of the hop kernel for a runtime (N, rep)
hr_status hop_dispatch(int N, int rep, int P, const HopParams &prm, bool rebuild, int epi, int variant,
                       cudaStream_t stream);
hr_status represent_dispatch(const hr_gauge &g, const double2 *UF, cudaStream_t stream);
hr_status force_dispatch(const hr_gauge &g, const ForceParams &fp, cudaStream_t stream);

// link record bytes of one parity: ntiles x 8 slots x chunks x 32 lanes x 16 B
inline size_t link_record_bytes(const Geom &g, int P, bool real, int ncomp)
{
    return (size_t)g.ntiles * 8 * link_nchunk(P, real, ncomp) * HR_TILE * 16;
}

}  // namespace hr
