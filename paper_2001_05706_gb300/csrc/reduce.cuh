// Deterministic grid reductions without floating-point atomics.
//
// Each block reduces its threads' values with a fixed shuffle tree (FP64 for
// FP64 kernels, double-float for the others) and writes one FP64 partial per
// reduced quantity.  The partials are summed in a fixed order either by a
// separate launch (block_partials + finish_reduce, the solver path) or by the
// block that finishes last, found with an integer atomic counter that it
// resets (grid_reduce, for small one-off reductions).  Same grid, same
// inputs: bitwise-identical result, independent of block scheduling, and a
// launch sequence can be replayed or captured in a CUDA graph.
#pragma once
#include "common.cuh"

namespace lqcd {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The per-thread value a kernel reduces: FP64 kernels reduce doubles; kernels
// computing in FP32 (FP32, FP16/BF16 storage) or in double-float reduce
// double-float pairs.  GB300 adds doubles at 1/64 of its FP32 rate, so the
// five FP64 shuffle-adds per site and quantity of a double tree cost more than
// the streaming of an FP16 field (a three-quantity dot product ran at 37 % of
// HBM bandwidth); a double-float add is ~11 FP32 operations, exact up to
// 2^-44 of the operands, and the tree order is unchanged (deterministic).
template <typename T> struct RedVal { using type = df; };
template <> struct RedVal<double> { using type = double; };

__device__ __forceinline__ df warp_sum(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df w(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
    v = v + w;
  }
  return v;
}

// Reduce NV values per thread over the blocks of one grid row.  Block
// (x, y) contributes to quantities kbase .. kbase+NV-1 (callers use
// kbase = y * NV, so the rows of a 2-D grid hold different quantities);
// partials must hold nk_total * gridDim.x doubles and result[k] receives the
// sum of quantity k (at result[k * rstride]) for k < nk_total.  All threads of the block must call
// this (no early return before it).
template <int NV>
__device__ __forceinline__ void grid_reduce(const double (&v)[NV], double *partials, unsigned int *counter,
                                            double *result, int kbase, int nk_total, int rstride = 1) {
  __shared__ double sh[NV][32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
  const unsigned nblk_x = gridDim.x;
#pragma unroll
  for (int k = 0; k < NV; k++) {
    double s = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) {
      double s = lane < nwarp ? sh[k][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) partials[(long)(kbase + k) * nblk_x + blockIdx.x] = s;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned total = gridDim.x * gridDim.y;
    unsigned done = atomicAdd(counter, 1u);
    last = (done == total - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    // warp w sums quantities k = w, w + nwarp, ...; lane-strided then tree
    for (int k = warp; k < nk_total; k += nwarp) {
      double s = 0.0;
      for (unsigned b = lane; b < nblk_x; b += 32) s += __ldcg(partials + (long)k * nblk_x + b);
      s = warp_sum(s);
      if (lane == 0) result[(long)k * rstride] = s;
    }
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// The block-level half of a reduction for kernels whose grid has thousands of
// blocks: each block adds its threads' NV values with the fixed shuffle tree
// and writes one partial per quantity (same layout as grid_reduce); the sums
// over blocks are left to finish_reduce, a separate launch that spreads them
// over a whole block per quantity.  The last-block scheme of grid_reduce sums
// thousands of partials with one warp, a latency-bound tail of tens of
// microseconds per reduction.  All threads must call this.
template <int NV>
__device__ __forceinline__ void block_partials(const double (&v)[NV], double *partials, int kbase) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
    double s = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) {
      double s = lane < nwarp ? sh[k][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) partials[(long)(kbase + k) * gridDim.x + blockIdx.x] = s;
    }
  }
}

// The same with double-float values: both tree levels in double-float, one
// double per block and quantity written
template <int NV>
__device__ __forceinline__ void block_partials(const df (&v)[NV], double *partials, int kbase) {
  __shared__ float2 shf[NV][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
    const df s = warp_sum(v[k]);
    if (lane == 0) shf[k][warp] = make_float2(s.hi, s.lo);
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) {
      df s = lane < nwarp ? df(shf[k][lane].x, shf[k][lane].y) : df(0.0f, 0.0f);
      s = warp_sum(s);
      if (lane == 0) partials[(long)(kbase + k) * gridDim.x + blockIdx.x] = (double)s.hi + (double)s.lo;
    }
  }
}

// result[k * rstride] = sum over b < nblk of partials[k * nblk + b], k < nk, in
// a fixed order (blas.cu); stream-ordered after the kernel that wrote them
cudaError_t finish_reduce(const double *partials, int nblk, int nk, double *result, int rstride, cudaStream_t st);

}  // namespace lqcd
