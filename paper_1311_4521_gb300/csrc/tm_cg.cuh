// tm_cg.cuh -- device-side state of the conjugate-gradient solvers
// (single system and batched): the scalars each system keeps in device
// memory, the operations that finish a reduction, and the gates that let
// iteration kernels skip finished or not-yet-due work inside a CUDA graph.
#pragma once

#include "tm_device.cuh"
#include "tmhop.h"

namespace twm {

struct CgScalars {
    double rr;       // |r|^2 of the residual the current direction was built from
    double rr_new;   // |r|^2 after the latest update
    double pAp;      // <p, Q^dag Q p> = |Q p|^2
    double alpha;
    double bb;       // |b|^2
    double tol2;     // tol^2
    double stop_rr;  // recursive-residual threshold tol^2 |b|^2 that ends a segment early
    double rr_true;  // |b - Q^dag Q x|^2 from the latest FP64 recomputation
    double rr_max;   // largest recursive |r|^2 since the latest reliable update
    double delta2;   // reliable update when |r|^2 < delta^2 rr_max
    int done;        // set: the remaining iterations of the segment are skipped
    int pending;     // set when the iteration should end after its p update
    int status;      // TM_OK or TM_ERR_NONFINITE
    int iters;       // inner iterations performed
    int maxiter;
    int reliable;    // mixed precision: an FP64 reliable update closes this iteration
    int since;       // iterations since the latest reliable update
    int every;       // reliable update at the latest after this many iterations
    int mixed;       // 1: reduced-precision inner solver with reliable updates
    int nreliable;   // FP64 residual recomputations so far
    unsigned ticket; // last-block-done counter of the current reduction
};

// Gates of the iteration kernels: 0 always run, 1 skip once the solve is
// done, 2 run only when a reliable update is due.
__device__ __forceinline__ bool gated(const CgScalars *s, int gate)
{
    return gate == 1 ? s->done != 0 : gate == 2 ? s->reliable == 0 : false;
}

enum Fin { FIN_PAP, FIN_RR_UPDATE, FIN_RR_TRUE, FIN_RR_CHECK, FIN_BB, FIN_ROLL };

__device__ __forceinline__ void cg_finish(int op, double total, CgScalars *s)
{
    bool bad = !isfinite(total);
    switch (op) {
    case FIN_PAP:
        s->pAp = total;
        if (bad || !(total > 0.0)) {
            s->alpha = 0.0;
            s->done = 1;
        } else {
            s->alpha = s->rr / total;
        }
        break;
    case FIN_RR_UPDATE: {
        s->rr_new = total;
        s->iters += 1;
        s->since += 1;
        bool stop = total <= s->stop_rr || s->iters >= s->maxiter;
        if (s->mixed) {
            // the recursive residual of the reduced-precision iteration drifts from the
            // true one once it has dropped by about the storage precision: recompute it
            // in FP64 whenever it has fallen by delta since the last recomputation
            s->rr_max = fmax(s->rr_max, total);
            if (stop || total < s->delta2 * s->rr_max || s->since >= s->every) s->reliable = 1;
        } else if (stop) {
            s->pending = 1;
        }
        break;
    }
    case FIN_RR_TRUE:
        s->rr_new = total;
        s->rr_true = total;
        s->rr_max = total;
        s->since = 0;
        s->reliable = 0;
        s->nreliable += 1;
        if (total <= s->stop_rr || s->iters >= s->maxiter) s->pending = 1;
        break;
    case FIN_RR_CHECK:
        s->rr_true = total;
        s->nreliable += 1;
        break;
    case FIN_BB:
        s->bb = total;
        s->stop_rr = s->tol2 * total;
        break;
    case FIN_ROLL:
        s->rr = s->rr_new;
        if (s->pending) {
            s->done = 1;
            s->pending = 0;
        }
        break;
    }
    if (bad && op != FIN_ROLL) {
        s->status = TM_ERR_NONFINITE;
        s->done = 1;
    }
}

template <typename R> __device__ __forceinline__ double norm2(const Spinor<R> &a)
{
    R n = R(0);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) n += a[sp][c].re * a[sp][c].re + a[sp][c].im * a[sp][c].im;
    return double(n);
}


}  // namespace twm
