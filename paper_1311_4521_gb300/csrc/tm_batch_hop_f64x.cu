// tm_batch_hop_f64x.cu -- the batched hop for F64X-18 storage (one
// translation unit per storage format so that they compile in parallel).
#include "tm_batch.cuh"

namespace twm {

cudaError_t batch_hop_f64x(const HopTable &t, const BSys *sys, int parity, int rin, int rout, int rx, const Coef &k,
                        int mode, int gate, cudaStream_t st)
{
    // no batched solver runs its inner iteration in this format: no fused norm
    return hop_pr<F64X, 18, false>(t, sys, parity, rin, rout, rx, k, mode, gate, st);
}

}  // namespace twm
