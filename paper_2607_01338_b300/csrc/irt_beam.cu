// Gaussian beam convolution of a PPV cube (Sec. 4.11): every channel image
// convolved with a separable Gaussian of the given FWHM in pixels (sigma =
// FWHM / (2 sqrt(2 ln 2)), taps out to ceil(4 sigma), normalised to unit sum),
// the sky outside the image taken as zero.  Two passes, along x into the
// caller's scratch cube and along y into the output: each reads and writes
// the cube once (HBM bound).  Both passes stage a tile with its halo in
// shared memory (zero outside the image): the x pass 8 rows by 256 columns
// plus 2R, the y pass 32 rows plus 2R by 128 columns, so each input element
// is read (tile + 2R) / tile times from the memory system instead of 2R + 1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "irt_internal.h"

namespace irt {
namespace dev {

constexpr int kBeamMaxR = 64;   // most taps on one side

struct BeamTaps {
  int R;
  float wf[2 * kBeamMaxR + 1];
  double wd[2 * kBeamMaxR + 1];
};

constexpr int kBeamXW = 256;   // output columns of an x-pass tile
constexpr int kBeamXH = 8;     // rows of an x-pass tile

// x pass, tiled: blockIdx.x = column tile, blockIdx.y = row tile, blockIdx.z
// = channel.
// Weight of tap k (k = d + R).
template <typename T>
__device__ __forceinline__ T tap(const BeamTaps& t, int k) {
  if constexpr (sizeof(T) == 4)
    return t.wf[k];
  else
    return t.wd[k];
}

// RC > 0: the tap count a side fixed at compile time (the loop unrolls);
// RC = 0: taken from taps.R at run time.
template <typename T, int RC>
__global__ void __launch_bounds__(256)
beam_pass_x_tiled(const T* __restrict__ in, T* __restrict__ out, int npy, int npx,
                  const __grid_constant__ BeamTaps taps) {
  extern __shared__ __align__(16) unsigned char beam_smem_x[];
  T* tile = reinterpret_cast<T*>(beam_smem_x);
  const int R = RC > 0 ? RC : taps.R;
  const int W = kBeamXW + 2 * R;
  const int x0 = blockIdx.x * kBeamXW, y0 = blockIdx.y * kBeamXH;
  const long long img = (long long)blockIdx.z * npy * npx;
  for (int i = threadIdx.x; i < kBeamXH * W; i += blockDim.x) {
    const int r = i / W, cx = i - r * W;
    const int y = y0 + r, x = x0 - R + cx;
    tile[i] = (y < npy && x >= 0 && x < npx) ? in[img + (long long)y * npx + x] : (T)0;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < kBeamXH * kBeamXW; o += blockDim.x) {
    const int ty = o / kBeamXW, cx = o - ty * kBeamXW;
    const int y = y0 + ty, x = x0 + cx;
    if (y < npy && x < npx) {
      T acc = (T)0;
      const T* row = tile + ty * W + cx;
      if constexpr (RC > 0) {
#pragma unroll
        for (int k = 0; k <= 2 * RC; ++k) acc += tap<T>(taps, k) * row[k];
      } else {
        for (int k = 0; k <= 2 * R; ++k) acc += tap<T>(taps, k) * row[k];
      }
      out[img + (long long)y * npx + x] = acc;
    }
  }
}

constexpr int kBeamTX = 128;   // columns of a y-pass tile
constexpr int kBeamTY = 32;    // output rows of a y-pass tile

// y pass, tiled: blockIdx.x = column tile, blockIdx.y = row tile, blockIdx.z
// = channel.
template <typename T, int RC>
__global__ void __launch_bounds__(256)
beam_pass_y_tiled(const T* __restrict__ in, T* __restrict__ out, int npy, int npx,
                  const __grid_constant__ BeamTaps taps) {
  extern __shared__ __align__(16) unsigned char beam_smem[];
  T* tile = reinterpret_cast<T*>(beam_smem);
  const int R = RC > 0 ? RC : taps.R;
  const int x0 = blockIdx.x * kBeamTX, y0 = blockIdx.y * kBeamTY;
  const long long img = (long long)blockIdx.z * npy * npx;
  const int rows = kBeamTY + 2 * R;
  for (int i = threadIdx.x; i < rows * kBeamTX; i += blockDim.x) {
    const int r = i / kBeamTX, cx = i - r * kBeamTX;
    const int y = y0 - R + r, x = x0 + cx;
    tile[i] = (y >= 0 && y < npy && x < npx) ? in[img + (long long)y * npx + x] : (T)0;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < kBeamTY * kBeamTX; o += blockDim.x) {
    const int ty = o / kBeamTX, cx = o - ty * kBeamTX;
    const int y = y0 + ty, x = x0 + cx;
    if (y < npy && x < npx) {
      T acc = (T)0;
      const T* col = tile + ty * kBeamTX + cx;
      if constexpr (RC > 0) {
#pragma unroll
        for (int k = 0; k <= 2 * RC; ++k) acc += tap<T>(taps, k) * col[k * kBeamTX];
      } else {
        for (int k = 0; k <= 2 * R; ++k) acc += tap<T>(taps, k) * col[k * kBeamTX];
      }
      out[img + (long long)y * npx + x] = acc;
    }
  }
}

}  // namespace dev

// Launcher (arguments validated by irt_beam_convolve): returns a cudaError_t,
// or cudaErrorInvalidValue when the beam needs more than kBeamMaxR taps a side
// (or the cube has more than 65535 channels).
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
  if (nchan > 65535) return (int)cudaErrorInvalidValue;
  const dim3 tgrid((unsigned)((npx + dev::kBeamTX - 1) / dev::kBeamTX),
                   (unsigned)((npy + dev::kBeamTY - 1) / dev::kBeamTY), (unsigned)nchan);
  const size_t es = dtype == IRT_F32 ? 4 : 8;
  const size_t smem = (size_t)(dev::kBeamTY + 2 * t.R) * dev::kBeamTX * es;
  const dim3 xgrid((unsigned)((npx + dev::kBeamXW - 1) / dev::kBeamXW),
                   (unsigned)((npy + dev::kBeamXH - 1) / dev::kBeamXH), (unsigned)nchan);
  const size_t xsmem = (size_t)dev::kBeamXH * (dev::kBeamXW + 2 * t.R) * es;
  auto run = [&](auto tag, auto rc) -> int {
    using T = decltype(tag);
    constexpr int RC = decltype(rc)::value;
    cudaError_t e = cudaFuncSetAttribute(dev::beam_pass_y_tiled<T, RC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    dev::beam_pass_x_tiled<T, RC><<<xgrid, 256, xsmem, s>>>(static_cast<const T*>(in),
        static_cast<T*>(scratch), npy, npx, t);
    dev::beam_pass_y_tiled<T, RC><<<tgrid, 256, smem, s>>>(static_cast<const T*>(scratch),
        static_cast<T*>(out), npy, npx, t);
    return 0;
  };
  auto by_r = [&](auto tag) -> int {
    switch (t.R) {
#define IRT_BEAM_R(N) \
      case N: return run(tag, std::integral_constant<int, N>{});
      IRT_BEAM_R(1) IRT_BEAM_R(2) IRT_BEAM_R(3) IRT_BEAM_R(4) IRT_BEAM_R(5) IRT_BEAM_R(6)
      IRT_BEAM_R(7) IRT_BEAM_R(8) IRT_BEAM_R(9) IRT_BEAM_R(10) IRT_BEAM_R(11) IRT_BEAM_R(12)
      IRT_BEAM_R(13) IRT_BEAM_R(14) IRT_BEAM_R(15) IRT_BEAM_R(16)
#undef IRT_BEAM_R
      default: return run(tag, std::integral_constant<int, 0>{});
    }
  };
  const int e = dtype == IRT_F32 ? by_r(float{}) : by_r(double{});
  if (e) return e;
  return (int)cudaGetLastError();
}

}  // namespace irt
