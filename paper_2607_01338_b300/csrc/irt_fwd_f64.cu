// Double-arithmetic forward kernels (every channel explicit, exact Planck
// per velocity); used where the float path is checked against the oracle.
#include "irt_forward_impl.cuh"

namespace irt {

int dispatch_fwd_f64(int mode, int store, int ni, const JobTable& jobs, int njobs,
                     const PhysParams& P, const PhysF& PF, long long total, unsigned long long* queue,
                     int grid_blocks, int kmax, int fwmax, int cwmax, unsigned flags,
                     unsigned long long* stats, cudaStream_t s) {
  if (store != ST_F64 || ni != 17) return (int)cudaErrorInvalidValue;
  if (mode == M_SMOOTH)
    return launch_fwd_inst<double, 17, ST_F64, M_SMOOTH>(jobs, njobs, P, PF, total, queue,
                                                         grid_blocks, kmax, fwmax, cwmax, flags, stats, s);
  if (mode == M_FORMAL)
    return launch_fwd_inst<double, 17, ST_F64, M_FORMAL>(jobs, njobs, P, PF, total, queue,
                                                         grid_blocks, kmax, fwmax, cwmax, flags, stats, s);
  return launch_fwd_inst<double, 17, ST_F64, M_FORMAL_KAHAN>(jobs, njobs, P, PF, total, queue,
                                                             grid_blocks, kmax, fwmax, cwmax,
                                                             flags, stats, s);
}

}  // namespace irt
