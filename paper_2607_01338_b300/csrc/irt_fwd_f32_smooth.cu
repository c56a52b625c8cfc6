// Float-arithmetic forward kernels, smooth integration.
#include "irt_forward_impl.cuh"

namespace irt {

int dispatch_fwd_f32_smooth(int store, int ni, const JobTable& jobs, int njobs,
                           const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                           cudaStream_t s) {
#define IRT_CASE(NI_, ST_)                                                                  \
  if (ni == NI_ && store == ST_)                                                            \
    return (L.flags & IRT_FLAG_SAVE_CHECKPOINTS)                                        \
               ? launch_fwd_inst<float, NI_, ST_, M_SMOOTH, true>(jobs, njobs, P, PF, L, s) \
               : launch_fwd_inst<float, NI_, ST_, M_SMOOTH, false>(jobs, njobs, P, PF, L, s);
  IRT_CASE(9, ST_F32) IRT_CASE(17, ST_F32) IRT_CASE(33, ST_F32)
  IRT_CASE(9, ST_H16) IRT_CASE(17, ST_H16) IRT_CASE(33, ST_H16)
  IRT_CASE(9, ST_F64) IRT_CASE(17, ST_F64) IRT_CASE(33, ST_F64)
#undef IRT_CASE
  return (int)cudaErrorInvalidValue;
}

}  // namespace irt
