// Device-side reduction helpers shared by the kernels that fuse a vector
// sweep with its inner products.
//
// Determinism: every block reduces its own elements in a fixed tree order
// (warp shuffles, then warps in order) and writes one partial per value; the
// last block to finish (found with a ticket counter) adds the partials in
// block order and runs the scalar epilogue.  The result does not depend on
// block scheduling.
#pragma once

#include "adr_common.cuh"

namespace adr {

__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Sums K complex values over the block; result valid in thread 0 (out[k]).
// sh must hold 32 * K double2.
template <int K>
__device__ __forceinline__ void block_sum_k(double2 (&v)[K], double2* sh, double2 (&out)[K]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum2(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[wid * K + k] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double2 s = lane < nw ? sh[lane * K + k] : make_double2(0.0, 0.0);
      out[k] = warp_sum2(s);
    }
  }
}

// As block_sum_k, but the per-thread values are complex of T: the warp
// stage runs in T (cheap for float), each warp's sum is widened to double.
template <typename T, int K>
__device__ __forceinline__ void block_sum_t(C<T> (&v)[K], double2* sh, double2 (&out)[K]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v[k].x += __shfl_down_sync(0xffffffffu, v[k].x, o);
      v[k].y += __shfl_down_sync(0xffffffffu, v[k].y, o);
    }
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[wid * K + k] = make_double2((double)v[k].x, (double)v[k].y);
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double2 s = lane < nw ? sh[lane * K + k] : make_double2(0.0, 0.0);
      out[k] = warp_sum2(s);
    }
  }
}

// Called by all threads of every block after thread 0 holds the block's K
// sums in `mine`.  Writes them to partial[blockIdx * K + k]; the last block
// to arrive returns true with total[k] (valid in thread 0) = sum over blocks
// in block order, and resets the ticket for the next launch.
template <int K>
__device__ __forceinline__ bool last_block_total(const double2 (&mine)[K], double2* partial, unsigned* ticket,
                                                 double2 (&total)[K], double2* sh) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partial[(size_t)blockIdx.x * K + k] = mine[k];
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double2 acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = make_double2(0.0, 0.0);
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const double2 p = __ldcg(&partial[(size_t)b * K + k]);
      acc[k].x += p.x;
      acc[k].y += p.y;
    }
  }
  block_sum_k<K>(acc, sh, total);
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// Thread 0 holds the block's k sums in blk[0..k); writes them as this block's
// partials; the last block of the problem to arrive reduces them in block
// order into out[0..k) and resets the ticket.  Returns true in that block.
__device__ __forceinline__ bool last_block_rt(int k, const double2* blk, double2* partial, unsigned* ticket, double2* out,
                                              double2* sh) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    for (int i = 0; i < k; ++i) partial[(size_t)blockIdx.x * k + i] = blk[i];
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  // one warp per value: lanes stride over the blocks' partials, then a fixed
  // shuffle tree (no block-wide step per value)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < k; i += nw) {
    double2 acc = make_double2(0.0, 0.0);
    for (unsigned b = lane; b < gridDim.x; b += 32) {
      const double2 p = __ldcg(&partial[(size_t)b * k + i]);
      acc.x += p.x;
      acc.y += p.y;
    }
    acc = warp_sum2(acc);
    if (lane == 0) out[i] = acc;
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __syncthreads();
  return true;
}

}  // namespace adr
