// ep_refine.cuh -- the decisions of the refinement loop, shared by every
// kernel that ends a right-hand-side or residual pass (structured-stencil and
// Q2 paths).
#pragma once

#include "ep_dev.cuh"

namespace epk {

// Totals of a right-hand-side or residual pass (t: (ns b)^2, (ns r)^2,
// r32 . z32, r32 . r32): convergence, the inner solver's starting scalars and
// stop, the loop decisions.  Run by one thread after the grid's reduction.
__device__ __forceinline__ void rhs_finish(Dev& D, const double* t, bool FIRST, int graph, float ns) {
    // ||b||^2 as this pass summed it, so that r and b of the ratio come from
    // the same pass
    D.bb = t[0];
    const double rr = t[1], bb = D.bb;
    const bool nan = !(rr == rr);
    const bool conv = !nan && (rr <= D.tol * D.tol * bb);
    D.relres = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
    if (nan && D.status == EP_OK) D.status = EP_ENAN;
    D.it = 0;
    D.beta = 0.0;
    D.rz = t[2];
    D.rr0 = t[3];
    {
        const double ns2 = (double)ns * (double)ns;
        const double target = 0.81 * D.tol * D.tol * (D.bb / ns2);
        const double floor2 = D.inner_tol * D.inner_tol * t[3];
        D.inner_stop = target > floor2 ? target : floor2;
    }
    D.rr = t[3];
    if (FIRST) {
        D.fin_pending = 0;  // the ionic kernel before this pass has done it
        D.sweeps = 0;
        D.it_total = 0;
        // the persistent solver's barrier counter starts the step at 0
        *reinterpret_cast<unsigned long long*>(D.counter + CNT_BAR) = 0ull;
    } else {
        D.sweeps += 1;
        if (!conv && D.sweeps >= D.max_sweeps && D.status == EP_OK) D.status = EP_ENOCONV;
    }
    const bool more = !conv && !nan && D.sweeps < D.max_sweeps;
    set_cond(graph ? D.h_outer : 0ull, &D.f_outer, more ? 1u : 0u);
    if (FIRST && !more && D.u_hi && D.hist >= bdf_order(D) && bdf_order(D) >= 2) {
        // the step ends at its first pass with A u_EXT extrapolated from the
        // history: that value, not an operator apply, becomes its A u.  Later
        // extrapolations would weigh its rounding by up to 3 per step (BDF3)
        // and compound it, so no window uses it: the history restarts after
        // this step (end_of_step takes the count from -1 to 0).  BDF1 needs no
        // restart: its u_EXT is u_n, so the stored value is step n's A u.
        D.hist = -1;
    }
    // the step's refinement is over: rotate the time levels now (the
    // finishing kernel then works on the rotated levels)
    if (!more) end_of_step(D);
    // the next inner loop starts enabled (with the per-iteration inner
    // loop its handle belongs to the refinement body, where this runs)
    if (FIRST) D.f_inner = 1;
    else set_cond(graph ? D.h_inner : 0ull, &D.f_inner, 1u);
}

}  // namespace epk
