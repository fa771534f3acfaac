// tm_batch_hop_f32_12.cu -- the batched hop for F32-12 storage (one
// translation unit per storage format so that they compile in parallel).
#include "tm_stage.cuh"

namespace twm {

cudaError_t batch_hop_f32_12(const HopTable &t, const BSys *sys, int parity, int rin, int rout, int rx, const Coef &k,
                        int mode, int gate, cudaStream_t st)
{
    if (t.nrb == STAGE_CODE) return stage_hop<F32, 12>(t, sys, parity, rin, rout, rx, k, mode, gate, st);
    return hop_pr<F32, 12>(t, sys, parity, rin, rout, rx, k, mode, gate, st);
}

}  // namespace twm
