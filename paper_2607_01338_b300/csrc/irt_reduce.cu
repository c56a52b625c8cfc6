// Latitude-mean reductions of Sec. 6.1: the l-v image u(s)(l, v) = mean over
// b of a PPV cube s(l, b, v), and the top-down density map t(p)(r, l) = mean
// over b of the density field.  Both are out[a][c] = mean_b in[a][b][c] over
// the middle axis of a C-order [A][B][C] array (cube [nchan][npy][npx] with
// b = y; field [nz][ny][nx] with b = y).
//
// HBM bound: every input element is read once.  A block covers 128
// consecutive c (32 lanes x float4 when the row is 16-byte aligned) of one
// a; its 8 warps split the b axis and keep 8 independent row loads in
// flight each; the 8 partial sums meet in shared memory.  The sums accumulate in
// double for double input and in float (8 x B/8 partial sums) for float.
#include <cuda_runtime.h>

#include <algorithm>

#include "irt_internal.h"

namespace irt {
namespace dev {

constexpr int kRedWarps = 8;

template <typename T>
__global__ void __launch_bounds__(kRedWarps * 32)
mean_axis1_kernel(const T* __restrict__ in, long long A, long long B, long long C,
                  T* __restrict__ out, int vec) {
  __shared__ T part[kRedWarps][128];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const long long a = blockIdx.y;
  const long long c0 = (long long)blockIdx.x * 128;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  const T* base = in + a * B * C;
  if (vec) {
    // 16-byte loads: C is a multiple of the vector width and the rows aligned
    const long long c = c0 + 4 * lane;
    constexpr int U = 8;   // rows in flight per warp
    auto add = [&](const T* p) {
      if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        acc[0] += v.x; acc[1] += v.y; acc[2] += v.z; acc[3] += v.w;
      } else {
        const double2 v0 = __ldg(reinterpret_cast<const double2*>(p));
        const double2 v1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
        acc[0] += v0.x; acc[1] += v0.y; acc[2] += v1.x; acc[3] += v1.y;
      }
    };
    if (c < C) {
      long long b = warp;
      for (; b + (U - 1) * kRedWarps < B; b += U * kRedWarps) {
        const T* p = base + b * C + c;
        if constexpr (sizeof(T) == 4) {
          float4 v[U];
#pragma unroll
          for (int u = 0; u < U; ++u)
            v[u] = __ldg(reinterpret_cast<const float4*>(p + (long long)u * kRedWarps * C));
#pragma unroll
          for (int u = 0; u < U; ++u) {
            acc[0] += v[u].x; acc[1] += v[u].y; acc[2] += v[u].z; acc[3] += v[u].w;
          }
        } else {
#pragma unroll
          for (int u = 0; u < U; ++u) add(p + (long long)u * kRedWarps * C);
        }
      }
      for (; b < B; b += kRedWarps) add(base + b * C + c);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) part[warp][4 * lane + q] = acc[q];
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long c = c0 + 32 * q + lane;
      if (c < C)
        for (long long b = warp; b < B; b += kRedWarps) acc[q] += __ldg(base + b * C + c);
      part[warp][32 * q + lane] = acc[q];
    }
  }
  __syncthreads();
  if (threadIdx.x < 128) {
    const long long c = c0 + threadIdx.x;
    if (c < C) {
      T s = (T)0;
#pragma unroll
      for (int w = 0; w < kRedWarps; ++w) s += part[w][threadIdx.x];
      out[a * C + c] = s / (T)B;
    }
  }
}

}  // namespace dev
}  // namespace irt

namespace irt {

// Launcher (arguments validated by irt_mean_axis1): returns a cudaError_t.
int launch_mean_axis1(const void* in, int dtype, long long A, long long B, long long C,
                      void* out, cudaStream_t s) {
  const dim3 grid((unsigned)((C + 127) / 128), (unsigned)A);
  const long long es = dtype == IRT_F32 ? 4 : 8;
  const int vec = (C % 4 == 0) && ((reinterpret_cast<unsigned long long>(in) % 16) == 0) &&
                  ((C * es) % 16 == 0);
  if (dtype == IRT_F32)
    dev::mean_axis1_kernel<float><<<grid, dev::kRedWarps * 32, 0, s>>>(
        static_cast<const float*>(in), A, B, C, static_cast<float*>(out), vec);
  else
    dev::mean_axis1_kernel<double><<<grid, dev::kRedWarps * 32, 0, s>>>(
        static_cast<const double*>(in), A, B, C, static_cast<double*>(out), vec);
  return (int)cudaGetLastError();
}

}  // namespace irt
