// Packing of the caller's five field arrays into the grid's interleaved cells.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "irt_internal.h"

namespace irt {
namespace {

__device__ __forceinline__ double load_as_double(const void* p, int dtype, long long i) {
  switch (dtype) {
    case IRT_F32: return (double)reinterpret_cast<const float*>(p)[i];
    case IRT_F16: return (double)__half2float(reinterpret_cast<const __half*>(p)[i]);
    case IRT_BF16: return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[i]);
    default: return reinterpret_cast<const double*>(p)[i];
  }
}

struct Src {
  const void* p[5];
  int dt[5];
  double scale[5];
};

__global__ void pack_f32(Src s, CellF32* cells, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    CellF32 c;
#pragma unroll
    for (int q = 0; q < 5; ++q) c.v[q] = (float)(load_as_double(s.p[q], s.dt[q], i) * s.scale[q]);
    c.pad[0] = 0.5f;   // H2 abundance default: fully molecular
    c.pad[1] = c.pad[2] = 0.0f;
    cells[i] = c;
  }
}

__global__ void pack_f64(Src s, CellF64* cells, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    CellF64 c;
#pragma unroll
    for (int q = 0; q < 5; ++q) c.v[q] = load_as_double(s.p[q], s.dt[q], i) * s.scale[q];
    c.pad[0] = 0.5;
    c.pad[1] = c.pad[2] = 0.0;
    cells[i] = c;
  }
}

// 16-bit fields are copied bit for bit
__global__ void pack_h16(Src s, CellH16* cells, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    CellH16 c;
#pragma unroll
    for (int q = 0; q < 5; ++q) c.v[q] = reinterpret_cast<const uint16_t*>(s.p[q])[i];
    c.pad[0] = 0x3800u;   // fp16 0.5
    c.pad[1] = c.pad[2] = 0;
    cells[i] = c;
  }
}

// The H2 abundance of each cell into its spare slot (float, fp16 or double
// after the cell's storage).
__global__ void set_chi_kernel(int store, const void* chi, int dtype, void* cells, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double c = load_as_double(chi, dtype, i);
    if (store == ST_F32) reinterpret_cast<CellF32*>(cells)[i].pad[0] = (float)c;
    else if (store == ST_F64) reinterpret_cast<CellF64*>(cells)[i].pad[0] = c;
    else reinterpret_cast<CellH16*>(cells)[i].pad[0] = __half_as_ushort(__float2half_rn((float)c));
  }
}

}  // namespace

int launch_set_chi(int store, const void* chi, int dtype, void* cells, long long ncell,
                   void* stream) {
  const int threads = 256;
  long long blocks = (ncell + threads - 1) / threads;
  if (blocks > 148 * 32) blocks = 148 * 32;
  if (blocks < 1) blocks = 1;
  set_chi_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(store, chi, dtype, cells,
                                                                          ncell);
  return (int)cudaGetLastError();
}

int launch_pack(int store, const void* const* src, const int* dtypes, const double* scale,
                void* cells, long long ncell, void* stream) {
  Src s;
  for (int q = 0; q < 5; ++q) {
    s.p[q] = src[q];
    s.dt[q] = dtypes[q];
    s.scale[q] = scale[q];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256;
  long long blocks = (ncell + threads - 1) / threads;
  if (blocks > 148 * 32) blocks = 148 * 32;
  if (blocks < 1) blocks = 1;
  if (store == ST_F32) pack_f32<<<(unsigned)blocks, threads, 0, st>>>(s, (CellF32*)cells, ncell);
  else if (store == ST_F64) pack_f64<<<(unsigned)blocks, threads, 0, st>>>(s, (CellF64*)cells, ncell);
  else pack_h16<<<(unsigned)blocks, threads, 0, st>>>(s, (CellH16*)cells, ncell);
  return (int)cudaGetLastError();
}

}  // namespace irt
