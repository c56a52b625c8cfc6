// Double-arithmetic forward kernels (every channel explicit, exact Planck
// per velocity); used where the float path is checked against the oracle.
#include "irt_forward_impl.cuh"

namespace irt {

int dispatch_fwd_f64(int mode, int store, int ni, const JobTable& jobs, int njobs,
                     const PhysParams& P, const PhysF& PF, const FwdLaunch& L,
                     cudaStream_t s) {
  if (store != ST_F64 || ni != 17) return (int)cudaErrorInvalidValue;
  if (mode == M_SMOOTH)
    return launch_fwd_inst<double, 17, ST_F64, M_SMOOTH>(jobs, njobs, P, PF, L, s);
  if (mode == M_FORMAL)
    return launch_fwd_inst<double, 17, ST_F64, M_FORMAL>(jobs, njobs, P, PF, L, s);
  return launch_fwd_inst<double, 17, ST_F64, M_FORMAL_KAHAN>(jobs, njobs, P, PF, L, s);
}

}  // namespace irt
