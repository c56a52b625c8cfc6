// Gaussian beam convolution of a PPV cube (Sec. 4.11): every channel image
// convolved with a separable Gaussian of the given FWHM in pixels (sigma =
// FWHM / (2 sqrt(2 ln 2)), taps out to ceil(4 sigma), normalised to unit sum),
// the sky outside the image taken as zero.  Two passes, along x into the
// caller's scratch cube and along y into the output: each reads and writes
// the cube once (HBM bound; the taps' neighbouring reads hit L1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "irt_internal.h"

namespace irt {
namespace dev {

constexpr int kBeamMaxR = 64;   // most taps on one side

struct BeamTaps {
  int R;
  float wf[2 * kBeamMaxR + 1];
  double wd[2 * kBeamMaxR + 1];
};

// One block per image row (row = channel * npy + y), threads over x.
template <typename T, bool ALONG_X>
__global__ void __launch_bounds__(256)
beam_pass(const T* __restrict__ in, T* __restrict__ out, int npy, int npx,
          const __grid_constant__ BeamTaps taps) {
  const long long row = blockIdx.x;
  const int y = (int)(row % npy);
  const int R = taps.R;
  const T* rin = in + row * npx;
  T* rout = out + row * npx;
  for (int x = threadIdx.x; x < npx; x += blockDim.x) {
    T acc = (T)0;
    if constexpr (ALONG_X) {
      const int lo = max(-R, -x), hi = min(R, npx - 1 - x);
      for (int d = lo; d <= hi; ++d)
        acc += (sizeof(T) == 4 ? (T)taps.wf[d + R] : (T)taps.wd[d + R]) * rin[x + d];
    } else {
      const int lo = max(-R, -y), hi = min(R, npy - 1 - y);
      for (int d = lo; d <= hi; ++d)
        acc += (sizeof(T) == 4 ? (T)taps.wf[d + R] : (T)taps.wd[d + R]) *
               rin[(long long)d * npx + x];
    }
    rout[x] = acc;
  }
}

}  // namespace dev

// Launcher (arguments validated by irt_beam_convolve): returns a cudaError_t,
// or cudaErrorInvalidValue when the beam needs more than kBeamMaxR taps a side
// (or the cube has more than 2^31 rows).
int launch_beam(const void* in, int dtype, long long nchan, int npy, int npx, double fwhm_px,
                void* scratch, void* out, cudaStream_t s) {
  dev::BeamTaps t;
  const double sigma = fwhm_px / (2.0 * std::sqrt(2.0 * std::log(2.0)));
  t.R = (int)std::ceil(4.0 * sigma);
  if (t.R > dev::kBeamMaxR) return (int)cudaErrorInvalidValue;
  double sum = 0.0;
  for (int d = -t.R; d <= t.R; ++d) {
    t.wd[d + t.R] = std::exp(-(double)d * d / (2.0 * sigma * sigma));
    sum += t.wd[d + t.R];
  }
  for (int k = 0; k <= 2 * t.R; ++k) {
    t.wd[k] /= sum;
    t.wf[k] = (float)t.wd[k];
  }
  const long long rows = nchan * npy;
  if (rows > 2147483647LL) return (int)cudaErrorInvalidValue;
  const int blocks = (int)rows;
  const int threads = npx >= 256 ? 256 : ((npx + 31) / 32) * 32;
  if (dtype == IRT_F32) {
    dev::beam_pass<float, true><<<blocks, threads, 0, s>>>(static_cast<const float*>(in),
        static_cast<float*>(scratch), npy, npx, t);
    dev::beam_pass<float, false><<<blocks, threads, 0, s>>>(static_cast<const float*>(scratch),
        static_cast<float*>(out), npy, npx, t);
  } else {
    dev::beam_pass<double, true><<<blocks, threads, 0, s>>>(static_cast<const double*>(in),
        static_cast<double*>(scratch), npy, npx, t);
    dev::beam_pass<double, false><<<blocks, threads, 0, s>>>(static_cast<const double*>(scratch),
        static_cast<double*>(out), npy, npx, t);
  }
  return (int)cudaGetLastError();
}

}  // namespace irt
