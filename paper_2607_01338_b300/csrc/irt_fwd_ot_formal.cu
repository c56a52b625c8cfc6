// Forward kernels with optically thin level-balance line coefficients,
// formal integration (float arithmetic, and the double instance).
#include "irt_forward_impl.cuh"

namespace irt {

int dispatch_fwd_ot_formal(int precision, int store, int ni, const JobTable& jobs, int njobs,
                       const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                       cudaStream_t s) {
  if (precision == IRT_PREC_F64) {
    if (store != ST_F64 || ni != 17) return (int)cudaErrorInvalidValue;
    return launch_fwd_inst<double, 17, ST_F64, M_FORMAL, false, true>(jobs, njobs, P, PF, L, s);
  }
#define IRT_CASE(NI_, ST_)                                                                 \
  if (ni == NI_ && store == ST_)                                                           \
    return launch_fwd_inst<float, NI_, ST_, M_FORMAL, false, true>(jobs, njobs, P, PF, L, s);
  IRT_CASE(9, ST_F32) IRT_CASE(17, ST_F32) IRT_CASE(33, ST_F32)
  IRT_CASE(9, ST_H16) IRT_CASE(17, ST_H16) IRT_CASE(33, ST_H16)
  IRT_CASE(9, ST_F64) IRT_CASE(17, ST_F64) IRT_CASE(33, ST_F64)
#undef IRT_CASE
  return (int)cudaErrorInvalidValue;
}

}  // namespace irt
