// Forward kernels rendering several lines of one job in one launch (the
// rays' field samples shared by the lines), Kahan-compensated formal integration, float arithmetic.
#include "irt_forward_impl.cuh"

namespace irt {

int dispatch_fwd_ml_kahan(int store, int ni, const JobTable& jobs, int njobs,
                       const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                       cudaStream_t s) {
#define IRT_CASE(NI_, ST_)                                                                 \
  if (ni == NI_ && store == ST_)                                                           \
    return launch_fwd_inst<float, NI_, ST_, M_FORMAL_KAHAN, false, false, true>(jobs, njobs, P, PF, L, s);
  IRT_CASE(9, ST_F32) IRT_CASE(17, ST_F32) IRT_CASE(33, ST_F32)
  IRT_CASE(9, ST_H16) IRT_CASE(17, ST_H16) IRT_CASE(33, ST_H16)
#undef IRT_CASE
  return (int)cudaErrorInvalidValue;
}

}  // namespace irt
