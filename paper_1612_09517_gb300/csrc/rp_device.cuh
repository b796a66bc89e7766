// Device-side helpers shared by the kernel translation units: complex pairs,
// the singlet-slice layout of the tensor-core time integral, shared-memory
// addresses for PTX, and a block-wide FP64 sum.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <atomic>

namespace rp {
namespace {

template <typename T>
struct Cx {
  T re, im;
};

// Singlet slices in the tensor-core Gram layout (xblk != 0): per row, chunks of
// kXChunk configurations; in a chunk, real rows 2n (Re x_n) and 2n + 1 (Im x_n)
// padded to xrows_pad(n_c) rows, stored as 8-row x 4-configuration core
// matrices (128 contiguous bytes, rows 16 B apart), the 4 core matrices of an
// 8-row group along the configurations 128 B apart, and the row groups 512 B
// apart.  A chunk is then one contiguous block that a single bulk copy brings
// into shared memory in the K-major no-swizzle operand layout of tcgen05.mma.
constexpr int kXChunk = 16;
__host__ __device__ __forceinline__ int xrows_pad(int n_c) { return (2 * n_c + 15) & ~15; }
__host__ __device__ __forceinline__ size_t xblk_row_floats(long long Zs, int n_c) {
  return (size_t)((Zs + kXChunk - 1) / kXChunk) * xrows_pad(n_c) * kXChunk;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// Sum of v over the NT threads of the block (NT a power of two); sh holds NT
// doubles.  Every thread gets the sum.
template <int NT>
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) for `func` once per
// device (the attribute belongs to the current device); `done` is the call
// site's bit mask of devices already set.  Repeating the call from several
// host threads is harmless.
inline cudaError_t smem_attr_once(const void* func, int bytes,
                                  std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

}  // namespace
}  // namespace rp
