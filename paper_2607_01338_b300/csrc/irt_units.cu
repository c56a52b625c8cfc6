// Conversion of rendered cubes to Planck brightness temperature with the
// continuum subtracted in that space (Sec. 4.9, 4.10): the thick render
// writes [T], [C], [B] as Rayleigh-Jeans temperatures at each channel's
// centre; this pass turns them into T_B in place and rewrites [L] = T_B([T])
// - T_B([C]) and [D] = T_B([C]) - T_B([B]).  Elementwise, HBM bound.
#include <cuda_runtime.h>

#include <algorithm>

#include "irt_internal.h"
#include "irt_units.cuh"

namespace irt {
namespace dev {

template <typename R>
__global__ void __launch_bounds__(256)
tb_convert_kernel(R* T, R* C, R* B, R* L, R* D, long long plane, int nchan, double v0, double dv,
                  double T0, double inv_c_kms) {
  const long long n = plane * nchan;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / plane);
    const double ucd = v0 + ((double)c + 0.5) * dv;
    const R uc = (R)ucd;
    const R y = (R)1 - uc * (R)inv_c_kms;
    const R y2 = y * y;   // T_RJ at the channel centre = I_K / y^2
    const R tT = brightness_k((R)T0, (R)inv_c_kms, uc, T[i] * y2);
    const R tC = brightness_k((R)T0, (R)inv_c_kms, uc, C[i] * y2);
    const R tB = brightness_k((R)T0, (R)inv_c_kms, uc, B[i] * y2);
    T[i] = tT;
    C[i] = tC;
    B[i] = tB;
    if (L) L[i] = tT - tC;
    if (D) D[i] = tC - tB;
  }
}

}  // namespace dev

// Launcher: one job's cubes (T, C, B required), precision 0 float / 1 double.
int launch_tb_convert(int precision, void* T, void* C, void* B, void* L, void* D,
                      long long plane, int nchan, double v0, double dv, double T0,
                      double inv_c_kms, cudaStream_t s) {
  int dev_id = 0, sms = 148;
  cudaGetDevice(&dev_id);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
  const long long n = plane * nchan;
  const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)sms * 8);
  if (precision)
    dev::tb_convert_kernel<double><<<blocks, 256, 0, s>>>(
        (double*)T, (double*)C, (double*)B, (double*)L, (double*)D, plane, nchan, v0, dv, T0,
        inv_c_kms);
  else
    dev::tb_convert_kernel<float><<<blocks, 256, 0, s>>>(
        (float*)T, (float*)C, (float*)B, (float*)L, (float*)D, plane, nchan, v0, dv, T0,
        inv_c_kms);
  return (int)cudaGetLastError();
}

}  // namespace irt
