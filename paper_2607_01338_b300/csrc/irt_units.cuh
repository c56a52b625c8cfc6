// Planck brightness temperature (Sec. 4.9) in the kernels' K units.  Kept out
// of the thick render's translation unit: that kernel's compiled code is
// sensitive to what its unit holds, and it converts to T_B in a separate
// pass (irt_units.cu).
#pragma once

namespace irt {
namespace dev {

// Brightness temperature [K] of an intensity I in K units (I c^2 / (2 k
// nu_ul^2)) at velocity u: Planck's law in K units solved for T, T0 y /
// ln(1 + T0 y^3 / I) with y = nu(u) / nu_ul; 0 for a non-positive intensity.
__device__ __forceinline__ float brightness_k(float T0, float inv_c_kms, float u, float I) {
  if (!(I > 0.0f)) return 0.0f;
  const float y = 1.0f - u * inv_c_kms;
  const float t0y = T0 * y;
  return t0y / log1pf(t0y * y * y / I);
}
__device__ __forceinline__ double brightness_k(double T0, double inv_c_kms, double u, double I) {
  if (!(I > 0.0)) return 0.0;
  const double y = 1.0 - u * inv_c_kms;
  const double t0y = T0 * y;
  return t0y / log1p(t0y * y * y / I);
}

}  // namespace dev
}  // namespace irt
