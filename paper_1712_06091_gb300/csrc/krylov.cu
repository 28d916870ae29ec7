// Krylov building blocks: fused Gram-Schmidt passes with deterministic
// last-block reductions (warp shuffles, then a fixed-order pass over
// per-block partials), scaling, the combination x += Z y, and the
// single-thread pieces that keep the Arnoldi Hessenberg matrix, its Givens
// rotations and the least-squares right-hand side on the device.
//
// They serve the outer flexible GMRES, the inner FGMRES of the K-cycle
// (Alg. Kcycle), the fixed-count Jacobi-preconditioned GMRES of the coarsest
// grid and the minimal-residual Jacobi relaxation (Sec. 3.1).  Every kernel
// handles a batch of problems with grid.y = problems (see krylov.cuh).
#include "krylov.cuh"
#include "reduce.cuh"
#include "krylov_dev.cuh"

namespace adr {

static inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Blocks of a reduction over n entries with `values` sums per block: one per
// 1024 entries (four grid-stride steps per thread), at most kMaxReduceBlocks.
// Spreading small coarse-level vectors over more blocks (one per 256 entries)
// measured slower: 699 against 606 us per coarsest solve.
int reduction_blocks(int64_t n, int values) {
  int64_t b = (n + 1023) / 1024;
  if (b < 1) b = 1;
  if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
  const int64_t cap = kPartialStride / (values > 0 ? values : 1);
  if (b > cap) b = cap;
  return (int)b;
}

// ---------------------------------------------------------------------------
// Elementwise
// ---------------------------------------------------------------------------
// A per-problem float64 scalar as complex T for every thread of the block,
// converted once by thread 0 through shared memory: a float64 conversion in
// every thread of a finest-grid launch costs tens of microseconds at the
// float64 pipe's rate.  Call once per kernel, from every thread.
template <typename T> __device__ __forceinline__ C<T> block_scalar(const double2* p) {
  __shared__ C<T> s;
  if (threadIdx.x == 0) {
    const double2 v = *p;
    s = mk<T>((T)v.x, (T)v.y);
  }
  __syncthreads();
  return s;
}

// out = w / |w| with the reciprocal norm precomputed in nrm2->y by the kernel
// that reduced nrm2->x (zero if the norm vanishes): no per-thread float64
// square root or division.
template <typename T>
__global__ void k_scale_inv_norm(const C<T>* w, C<T>* out, const double2* __restrict__ nrm2, Dims g) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  const T inv = block_scalar<T>(nrm2 + blockIdx.y).y;   // the reciprocal norm
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  shift_nodes(g, w, out);
  out[e] = cscale(w[e], inv);
}
template <typename T>
void launch_scale_inv_norm(const C<T>* w, C<T>* out, const double2* nrm2, const Dims& g, cudaStream_t st) {
  count_launches(1), k_scale_inv_norm<T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(w, out, nrm2, g);
}

// out = w / |w| and z = dinv .* out (the next Jacobi-preconditioned direction)
template <typename T>
__global__ void k_scale_dinv(const C<T>* w, C<T>* out, const C<T>* __restrict__ dinv, C<T>* z,
                             const double2* __restrict__ nrm2, Dims g) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  const T inv = block_scalar<T>(nrm2 + blockIdx.y).y;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  shift_nodes(g, w, out, dinv, z);
  const C<T> v = cscale(w[e], inv);
  out[e] = v;
  z[e] = cmul(dinv[e], v);
}
template <typename T>
void launch_scale_dinv(const C<T>* w, C<T>* out, const C<T>* dinv, C<T>* z, const double2* nrm2, const Dims& g,
                       cudaStream_t st) {
  count_launches(1), k_scale_dinv<T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(w, out, dinv, z, nrm2, g);
}

template <typename T>
__global__ void k_copy(const C<T>* __restrict__ a, C<T>* __restrict__ b, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) b[e] = a[e];
}
template <typename T> void launch_copy(const C<T>* a, C<T>* b, int64_t n, cudaStream_t st) {
  count_launches(1), k_copy<T><<<blocks_for(n, 256), 256, 0, st>>>(a, b, n);
}

template <typename T>
__global__ void k_zero(C<T>* __restrict__ a, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) a[e] = czero<T>();
}
template <typename T> void launch_zero(C<T>* a, int64_t n, cudaStream_t st) {
  count_launches(1), k_zero<T><<<blocks_for(n, 256), 256, 0, st>>>(a, n);
}

template <typename Ts, typename Td>
__global__ void k_ccast(const C<Ts>* __restrict__ a, C<Td>* __restrict__ b, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) b[e] = mk<Td>((Td)a[e].x, (Td)a[e].y);
}
template <typename Ts, typename Td> void launch_ccast(const C<Ts>* src, C<Td>* dst, int64_t n, cudaStream_t st) {
  count_launches(1), k_ccast<Ts, Td><<<blocks_for(n, 256), 256, 0, st>>>(src, dst, n);
}

template <typename T>
__global__ void k_cmul_vec(const C<T>* __restrict__ a, const C<T>* __restrict__ b, C<T>* __restrict__ out, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) out[e] = cmul(a[e], b[e]);
}
template <typename T> void launch_cmul_vec(const C<T>* a, const C<T>* b, C<T>* out, int64_t n, cudaStream_t st) {
  count_launches(1), k_cmul_vec<T><<<blocks_for(n, 256), 256, 0, st>>>(a, b, out, n);
}

// ---------------------------------------------------------------------------
// Single-thread Arnoldi pieces (one block per problem)
// ---------------------------------------------------------------------------
__global__ void k_backsolve(ArnoldiState st, int k) {
  if (threadIdx.x != 0) return;
  backsolve_dev(arnoldi_at(st, blockIdx.y), k);
}
void launch_backsolve(const ArnoldiState& s, int k, cudaStream_t st, int B) {
  count_launches(1), k_backsolve<<<dim3(1, B), 32, 0, st>>>(s, k);
}

__global__ void k_set_target(ArnoldiState st, const double2* nrm2, double tol) {
  if (threadIdx.x != 0) return;
  const ArnoldiState s = arnoldi_at(st, blockIdx.y);
  s.scal[kScalTarget] = tol * sqrt(nrm2[blockIdx.y].x);
}
void launch_set_target(const ArnoldiState& s, const double2* nrm2, double tol, cudaStream_t st, int B) {
  count_launches(1), k_set_target<<<dim3(1, B), 32, 0, st>>>(s, nrm2, tol);
}

// ===========================================================================
// Fused Arnoldi / Krylov kernels (one launch per pass, deterministic
// last-block reductions; see reduce.cuh)
// ===========================================================================

// Per-thread sums of conj(V_i[e]) * w[e] for i < k over a grid-stride range,
// reduced over the block into blk[i].
template <typename T>
__device__ __forceinline__ void block_dots(const C<T>* __restrict__ V, int64_t ld, int k, const C<T>* w, int64_t n,
                                           double2* blk, double2* sh) {
  for (int c = 0; c < k; c += 4) {
    C<T> acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = czero<T>();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
      const C<T> we = w[e];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c + q < k) acc[q] = cfma_conj(V[(int64_t)(c + q) * ld + e], we, acc[q]);
    }
    double2 o[4];
    block_sum_t<T, 4>(acc, sh, o);
    if (threadIdx.x == 0)
      for (int q = 0; q < 4 && c + q < k; ++q) blk[c + q] = o[q];
    __syncthreads();
  }
}

// w -= V c ; |w|^2 reduced over the problem's blocks.  Returns true in the
// last block (total in nrm2->x, valid in thread 0).
template <typename T>
__device__ __forceinline__ bool update_norm(const C<T>* __restrict__ V, int64_t ld, int k, C<T>* w, int64_t n,
                                            const double2* c, double2* partial, unsigned* ticket, double2* nrm2) {
  __shared__ double2 sh[32 * 4];
  __shared__ double2 blk[1];
  __shared__ C<T> coef[kMaxKrylov + 1];
  for (int i = threadIdx.x; i < k; i += blockDim.x) coef[i] = mk<T>((T)(-c[i].x), (T)(-c[i].y));
  __syncthreads();
  C<T> s2[1] = {czero<T>()};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    C<T> acc = w[e];
    for (int i = 0; i < k; ++i) acc = cfma(V[(int64_t)i * ld + e], coef[i], acc);
    w[e] = acc;
    s2[0] = cfma_conj(acc, acc, s2[0]);
  }
  double2 o[1];
  block_sum_t<T, 1>(s2, sh, o);
  if (threadIdx.x == 0) blk[0] = o[0];
  __syncthreads();
  return last_block_rt(1, blk, partial, ticket, nrm2, sh);
}

// pass 1: ha = V^H w
template <typename T>
__global__ void __launch_bounds__(256) k_cgs_pass1(const C<T>* __restrict__ V, int64_t ld, int k, const C<T>* w, Dims g,
                                                   KrylovScratch s) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  __shared__ double2 sh[32 * 4];
  __shared__ double2 blk[kMaxKrylov + 1];
  shift_nodes(g, V, w);
  s = scratch_at(s, blockIdx.y);
  block_dots<T>(V, ld, k, w, n, blk, sh);
  last_block_rt(k, blk, s.partial, s.ticket, s.ha, sh);
}

// pass 2: w -= V ha ; hb = V^H w
template <typename T>
__global__ void __launch_bounds__(256) k_cgs_pass2(const C<T>* __restrict__ V, int64_t ld, int k, C<T>* w, Dims g,
                                                   KrylovScratch s) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  __shared__ double2 sh[32 * 4];
  __shared__ double2 blk[kMaxKrylov + 1];
  __shared__ C<T> coef[kMaxKrylov + 1];
  shift_nodes(g, V, w);
  s = scratch_at(s, blockIdx.y);
  for (int i = threadIdx.x; i < k; i += blockDim.x) coef[i] = mk<T>((T)(-s.ha[i].x), (T)(-s.ha[i].y));
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    C<T> acc = w[e];
    for (int i = 0; i < k; ++i) acc = cfma(V[(int64_t)i * ld + e], coef[i], acc);
    w[e] = acc;
  }
  block_dots<T>(V, ld, k, w, n, blk, sh);   // each thread re-reads only its own elements of w
  last_block_rt(k, blk, s.partial, s.ticket, s.hb, sh);
}

// pass 3: w -= V hb ; |w|^2 ; Arnoldi column j and Givens rotation (last block)
template <typename T>
__global__ void __launch_bounds__(256) k_cgs_pass3(const C<T>* __restrict__ V, int64_t ld, int k, C<T>* w, Dims g,
                                                   KrylovScratch s, ArnoldiState st, int j) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  shift_nodes(g, V, w);
  s = scratch_at(s, blockIdx.y);
  if (update_norm<T>(V, ld, k, w, n, s.hb, s.partial, s.ticket, s.nrm2) && threadIdx.x == 0) {
    const double s2t = s.nrm2->x;
    s.nrm2->y = s2t > 0.0 ? rsqrt(s2t) : 0.0;
    if (st.m > 0) arnoldi_column_dev(arnoldi_at(st, blockIdx.y), j, s.ha, s.hb, s2t);
  }
}

// Coarsest-grid step with the selective second pass (see coarse_select_dev).
// First pass (when the apply does not fuse it): ha = V^H w and |w|^2, then
// the decision in the last block.
template <typename T>
__global__ void __launch_bounds__(256) k_cgs_dots_sel(const C<T>* __restrict__ V, int64_t ld, int k, const C<T>* w,
                                                      Dims g, KrylovScratch s, ArnoldiState st, int j, int finish,
                                                      double eta2) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  __shared__ double2 sh[32 * 5];
  __shared__ double2 blk[kMaxKrylov + 2];
  shift_nodes(g, V, w);
  s = scratch_at(s, blockIdx.y);
  for (int c = 0; c < k; c += 4) {
    C<T> acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = czero<T>();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
      const C<T> we = w[e];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c + q < k) acc[q] = cfma_conj(V[(int64_t)(c + q) * ld + e], we, acc[q]);
      if (c == 0) acc[4] = cfma_conj(we, we, acc[4]);
    }
    double2 o[5];
    block_sum_t<T, 5>(acc, sh, o);
    if (threadIdx.x == 0) {
      for (int q = 0; q < 4 && c + q < k; ++q) blk[c + q] = o[q];
      if (c == 0) blk[k] = o[4];
    }
    __syncthreads();
  }
  if (last_block_rt(k + 1, blk, s.partial, s.ticket, s.ha, sh) && threadIdx.x == 0)
    coarse_select_dev(s.ha, s.hb, k, eta2, arnoldi_at(st, blockIdx.y), j, finish, s.nrm2);
}

// Second pass, only where the first one cancelled (ha[k].y set; the blocks of
// a problem agree, so the whole problem returns at once otherwise):
// w -= V ha ; hb = V^H w and |w|^2 ; the column from ha + hb.
template <typename T>
__global__ void __launch_bounds__(256) k_cgs_reorth(const C<T>* __restrict__ V, int64_t ld, int k, C<T>* w, Dims g,
                                                    KrylovScratch s, ArnoldiState st, int j, int finish) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  s = scratch_at(s, blockIdx.y);
  if (s.ha[k].y == 0.0) return;
  __shared__ double2 sh[32 * 5];
  __shared__ double2 blk[kMaxKrylov + 2];
  __shared__ C<T> coef[kMaxKrylov + 1];
  shift_nodes(g, V, w);
  for (int i = threadIdx.x; i < k; i += blockDim.x) coef[i] = mk<T>((T)(-s.ha[i].x), (T)(-s.ha[i].y));
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    C<T> acc = w[e];
    for (int i = 0; i < k; ++i) acc = cfma(V[(int64_t)i * ld + e], coef[i], acc);
    w[e] = acc;
  }
  for (int c = 0; c < k; c += 4) {
    C<T> acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = czero<T>();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
      const C<T> we = w[e];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c + q < k) acc[q] = cfma_conj(V[(int64_t)(c + q) * ld + e], we, acc[q]);
      if (c == 0) acc[4] = cfma_conj(we, we, acc[4]);
    }
    double2 o[5];
    block_sum_t<T, 5>(acc, sh, o);
    if (threadIdx.x == 0) {
      for (int q = 0; q < 4 && c + q < k; ++q) blk[c + q] = o[q];
      if (c == 0) blk[k] = o[4];
    }
    __syncthreads();
  }
  if (last_block_rt(k + 1, blk, s.partial, s.ticket, s.hb, sh) && threadIdx.x == 0)
    coarse_reorth_dev(s.ha, s.hb, k, arnoldi_at(st, blockIdx.y), j, finish, s.nrm2);
}

// V_next = (w - V c) / h_{j+1,j} and z = dinv .* V_next (elementwise), c = ha
// after a single pass (w still A z), hb after the second pass (w already
// updated by ha).
template <typename T>
__global__ void k_cgs_next(const C<T>* __restrict__ V, int64_t ld, int k, const C<T>* __restrict__ w, Dims g,
                           KrylovScratch s, C<T>* __restrict__ Vnext, const C<T>* __restrict__ dinv, C<T>* __restrict__ z) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  __shared__ C<T> coef[kMaxKrylov + 1];
  __shared__ T s_inv;
  s = scratch_at(s, blockIdx.y);
  const double2* c = s.ha[k].y != 0.0 ? s.hb : s.ha;
  for (int i = threadIdx.x; i < k; i += blockDim.x) coef[i] = mk<T>((T)(-c[i].x), (T)(-c[i].y));
  if (threadIdx.x == 0) s_inv = (T)s.nrm2->y;
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  shift_nodes(g, V, w, Vnext, dinv, z);
  C<T> acc = w[e];
  for (int i = 0; i < k; ++i) acc = cfma(V[(int64_t)i * ld + e], coef[i], acc);
  const C<T> v = cscale(acc, s_inv);
  Vnext[e] = v;
  z[e] = cmul(dinv[e], v);
}

// x = dinv .* sum_{i<k} V_i y_i
template <typename T>
__global__ void k_combine_dinv(C<T>* x, const C<T>* __restrict__ V, int64_t ld, int k, ArnoldiState st,
                               const C<T>* __restrict__ dinv, Dims g) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  __shared__ C<T> coef[kMaxKrylov];
  const ArnoldiState a = arnoldi_at(st, blockIdx.y);
  for (int i = threadIdx.x; i < k; i += blockDim.x) coef[i] = mk<T>((T)a.y[i].x, (T)a.y[i].y);
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  shift_nodes(g, x, V, dinv);
  C<T> acc = czero<T>();
  for (int i = 0; i < k; ++i) acc = cfma(V[(int64_t)i * ld + e], coef[i], acc);
  x[e] = cmul(dinv[e], acc);
}

// ---------------------------------------------------------------------------
// Gram-Schmidt with a conditional second pass (selective re-orthogonalisation):
//   A: ha = V^H w and |w|^2 (kept in ha[k].x)
//   B: w -= V ha, t = |w'|^2; if t >= eta^2 |w|^2 the column is final
//      (hb = 0, Arnoldi column), else ha[k].y = 1 requests the second pass
//   C: (only if requested) hb = V^H w'
//   D: (only if requested) w' -= V hb, |w''|^2, Arnoldi column from ha + hb
// C and D exit at once when the flag is clear, so the launch sequence is
// fixed (graph-capturable) while the second pass costs nothing when skipped.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_sgs_dots_norm(const C<T>* __restrict__ V, int64_t ld, int k, const C<T>* w,
                                                       Dims g, KrylovScratch s) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  __shared__ double2 sh[32 * 5];
  __shared__ double2 blk[kMaxKrylov + 2];
  shift_nodes(g, V, w);
  s = scratch_at(s, blockIdx.y);
  for (int c = 0; c < k; c += 4) {
    C<T> acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = czero<T>();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
      const C<T> we = w[e];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c + q < k) acc[q] = cfma_conj(V[(int64_t)(c + q) * ld + e], we, acc[q]);
      if (c == 0) acc[4] = cfma_conj(we, we, acc[4]);
    }
    double2 o[5];
    block_sum_t<T, 5>(acc, sh, o);
    if (threadIdx.x == 0) {
      for (int q = 0; q < 4 && c + q < k; ++q) blk[c + q] = o[q];
      if (c == 0) blk[k] = o[4];
    }
    __syncthreads();
  }
  last_block_rt(k + 1, blk, s.partial, s.ticket, s.ha, sh);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sgs_update_test(const C<T>* __restrict__ V, int64_t ld, int k, C<T>* w, Dims g,
                                                         KrylovScratch s, ArnoldiState st, int j, double eta2) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  shift_nodes(g, V, w);
  s = scratch_at(s, blockIdx.y);
  if (update_norm<T>(V, ld, k, w, n, s.ha, s.partial, s.ticket, s.nrm2) && threadIdx.x == 0) {
    const double t = s.nrm2->x;
    if (t >= eta2 * s.ha[k].x) {
      s.ha[k].y = 0.0;
      for (int i = 0; i < k; ++i) s.hb[i] = make_double2(0.0, 0.0);
      s.nrm2->y = t > 0.0 ? rsqrt(t) : 0.0;
      if (st.m > 0) arnoldi_column_dev(arnoldi_at(st, blockIdx.y), j, s.ha, s.hb, t);
    } else {
      s.ha[k].y = 1.0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sgs_reorth_dots(const C<T>* __restrict__ V, int64_t ld, int k, const C<T>* w,
                                                         Dims g, KrylovScratch s) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  s = scratch_at(s, blockIdx.y);
  if (s.ha[k].y == 0.0) return;   // uniform over the problem's blocks
  __shared__ double2 sh[32 * 4];
  __shared__ double2 blk[kMaxKrylov + 1];
  shift_nodes(g, V, w);
  block_dots<T>(V, ld, k, w, n, blk, sh);
  last_block_rt(k, blk, s.partial, s.ticket, s.hb, sh);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sgs_reorth_update(const C<T>* __restrict__ V, int64_t ld, int k, C<T>* w, Dims g,
                                                           KrylovScratch s, ArnoldiState st, int j) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  s = scratch_at(s, blockIdx.y);
  if (s.ha[k].y == 0.0) return;   // uniform over the problem's blocks
  shift_nodes(g, V, w);
  if (update_norm<T>(V, ld, k, w, n, s.hb, s.partial, s.ticket, s.nrm2) && threadIdx.x == 0) {
    const double s2t = s.nrm2->x;
    s.nrm2->y = s2t > 0.0 ? rsqrt(s2t) : 0.0;
    if (st.m > 0) arnoldi_column_dev(arnoldi_at(st, blockIdx.y), j, s.ha, s.hb, s2t);
  }
}

// |b|^2 and (optionally) the start of an Arnoldi cycle with beta = |b|.
template <typename T>
__global__ void __launch_bounds__(256) k_norm_start(const C<T>* b, Dims g, KrylovScratch s, ArnoldiState st, int start,
                                                    double rel_target) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  __shared__ double2 sh[32 * 4];
  __shared__ double2 blk[1];
  shift_nodes(g, b);
  s = scratch_at(s, blockIdx.y);
  C<T> s2[1] = {czero<T>()};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s2[0] = cfma_conj(b[e], b[e], s2[0]);
  double2 o[1];
  block_sum_t<T, 1>(s2, sh, o);
  if (threadIdx.x == 0) blk[0] = o[0];
  __syncthreads();
  if (last_block_rt(1, blk, s.partial, s.ticket, s.nrm2, sh) && threadIdx.x == 0) {
    double beta, ibeta;
    sqrt_pair(s.nrm2->x, beta, ibeta);
    s.nrm2->y = ibeta;
    if (!start) return;
    const ArnoldiState a = arnoldi_at(st, blockIdx.y);
    for (int i = 0; i <= a.m; ++i) a.g[i] = make_double2(0.0, 0.0);
    a.g[0] = make_double2(beta, 0.0);
    a.scal[kScalBeta] = beta;
    a.scal[kScalEst] = beta;
    a.iscal[kIScalStop] = beta > 0.0 ? -1 : 0;
    if (rel_target >= 0.0) {   // a relative target is only tested after a step
      a.scal[kScalTarget] = rel_target * beta;
      a.iscal[kIScalConv] = beta > 0.0 ? -1 : 0;
    } else {
      a.iscal[kIScalConv] = beta <= a.scal[kScalTarget] ? 0 : -1;
    }
  }
}

// x = (assign ? 0 : x) + sum_i Z_i y_i  (y from the state, i < k)
template <typename T>
__global__ void k_combine(C<T>* x, const C<T>* __restrict__ Z, int64_t ld, int k, ArnoldiState st, int assign, Dims g) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  __shared__ C<T> coef[kMaxKrylov];
  const ArnoldiState a = arnoldi_at(st, blockIdx.y);
  for (int i = threadIdx.x; i < k; i += blockDim.x) coef[i] = mk<T>((T)a.y[i].x, (T)a.y[i].y);
  __syncthreads();
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  shift_nodes(g, x, Z);
  C<T> acc = assign ? czero<T>() : x[e];
  for (int i = 0; i < k; ++i) acc = cfma(Z[(int64_t)i * ld + e], coef[i], acc);
  x[e] = acc;
}

// x = (x_zero ? 0 : x) + alpha z ; r_dst = r_src - alpha w ; znext = dinv .* r_dst
template <typename T>
__global__ void k_mr_update2(C<T>* x, const C<T>* z, const C<T>* r_src, C<T>* r_dst,
                             const C<T>* __restrict__ w, const double2* __restrict__ alpha, const C<T>* __restrict__ dinv,
                             C<T>* znext, int x_zero, Dims g) {
  if (resolve(g)) return;
  const int64_t n = g.N;
  const C<T> al = block_scalar<T>(alpha + blockIdx.y);
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  shift_nodes(g, x, z, r_src, r_dst, w, dinv);
  shift_nodes_opt(g, znext);
  x[e] = cfma(al, z[e], x_zero ? czero<T>() : x[e]);
  const C<T> rn = csub(r_src[e], cmul(al, w[e]));
  r_dst[e] = rn;
  if (znext) znext[e] = cmul(dinv[e], rn);
}

template <typename T>
void launch_cgs2(const C<T>* V, int64_t ld, int k, C<T>* w, const Dims& g, const KrylovScratch& s, const ArnoldiState& st, int j,
                 cudaStream_t stream) {
  const dim3 grid(reduction_blocks(g.N, k + 2), g.B);
  count_launches(1), k_cgs_pass1<T><<<grid, 256, 0, stream>>>(V, ld, k, w, g, s);
  count_launches(1), k_cgs_pass2<T><<<grid, 256, 0, stream>>>(V, ld, k, w, g, s);
  count_launches(1), k_cgs_pass3<T><<<grid, 256, 0, stream>>>(V, ld, k, w, g, s, st, j);
}
template <typename T>
void launch_cgs_dots_sel(const C<T>* V, int64_t ld, int k, const C<T>* w, const Dims& g, const KrylovScratch& s,
                         const ArnoldiState& st, int j, int finish, double eta, cudaStream_t stream) {
  const dim3 grid(reduction_blocks(g.N, k + 2), g.B);
  count_launches(1), k_cgs_dots_sel<T><<<grid, 256, 0, stream>>>(V, ld, k, w, g, s, st, j, finish, eta * eta);
}
template <typename T>
void launch_cgs_reorth(const C<T>* V, int64_t ld, int k, C<T>* w, const Dims& g, const KrylovScratch& s,
                       const ArnoldiState& st, int j, int finish, cudaStream_t stream) {
  const dim3 grid(reduction_blocks(g.N, k + 2), g.B);
  count_launches(1), k_cgs_reorth<T><<<grid, 256, 0, stream>>>(V, ld, k, w, g, s, st, j, finish);
}
template <typename T>
void launch_cgs_next(const C<T>* V, int64_t ld, int k, const C<T>* w, const Dims& g, const KrylovScratch& s, C<T>* Vnext,
                     const C<T>* dinv, C<T>* z, cudaStream_t stream) {
  count_launches(1), k_cgs_next<T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, stream>>>(V, ld, k, w, g, s, Vnext, dinv, z);
}
template <typename T>
void launch_combine_dinv(C<T>* x, const C<T>* V, int64_t ld, int k, const ArnoldiState& st, const C<T>* dinv, const Dims& g,
                         cudaStream_t stream) {
  count_launches(1), k_combine_dinv<T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, stream>>>(x, V, ld, k, st, dinv, g);
}
template <typename T>
void launch_cgs_selective(const C<T>* V, int64_t ld, int k, C<T>* w, const Dims& g, const KrylovScratch& s,
                          const ArnoldiState& st, int j, double eta, cudaStream_t stream) {
  if (!(eta < 1.0)) {
    launch_cgs2<T>(V, ld, k, w, g, s, st, j, stream);
    return;
  }
  const dim3 grid(reduction_blocks(g.N, k + 2), g.B);
  count_launches(1), k_sgs_dots_norm<T><<<grid, 256, 0, stream>>>(V, ld, k, w, g, s);
  count_launches(1), k_sgs_update_test<T><<<grid, 256, 0, stream>>>(V, ld, k, w, g, s, st, j, eta * eta);
  count_launches(1), k_sgs_reorth_dots<T><<<grid, 256, 0, stream>>>(V, ld, k, w, g, s);
  count_launches(1), k_sgs_reorth_update<T><<<grid, 256, 0, stream>>>(V, ld, k, w, g, s, st, j);
}
template <typename T>
void launch_norm_start(const C<T>* b, const Dims& g, const KrylovScratch& s, const ArnoldiState* st, cudaStream_t stream,
                       double rel_target) {
  ArnoldiState dummy{};
  count_launches(1), k_norm_start<T><<<dim3(reduction_blocks(g.N, 1), g.B), 256, 0, stream>>>(b, g, s, st ? *st : dummy,
                                                                                        st ? 1 : 0, rel_target);
}
template <typename T>
void launch_combine(C<T>* x, const C<T>* Z, int64_t ld, int k, const ArnoldiState& st, bool assign, const Dims& g,
                    cudaStream_t stream) {
  count_launches(1), k_combine<T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, stream>>>(x, Z, ld, k, st, assign ? 1 : 0, g);
}
template <typename T>
void launch_mr_update2(C<T>* x, const C<T>* z, const C<T>* r_src, C<T>* r_dst, const C<T>* w, const double2* alpha,
                       const C<T>* dinv, C<T>* znext, bool x_zero, const Dims& g, cudaStream_t stream) {
  count_launches(1), k_mr_update2<T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, stream>>>(x, z, r_src, r_dst, w, alpha, dinv,
                                                                                       znext, x_zero ? 1 : 0, g);
}

#define ADR_INSTANTIATE_KRYLOV(T)                                                                                        \
  template void launch_scale_inv_norm<T>(const C<T>*, C<T>*, const double2*, const Dims&, cudaStream_t);               \
  template void launch_scale_dinv<T>(const C<T>*, C<T>*, const C<T>*, C<T>*, const double2*, const Dims&, cudaStream_t); \
  template void launch_copy<T>(const C<T>*, C<T>*, int64_t, cudaStream_t);                                               \
  template void launch_zero<T>(C<T>*, int64_t, cudaStream_t);                                                            \
  template void launch_cmul_vec<T>(const C<T>*, const C<T>*, C<T>*, int64_t, cudaStream_t);                              \
  template void launch_cgs2<T>(const C<T>*, int64_t, int, C<T>*, const Dims&, const KrylovScratch&, const ArnoldiState&, int, \
                               cudaStream_t);                                                                       \
  template void launch_cgs_selective<T>(const C<T>*, int64_t, int, C<T>*, const Dims&, const KrylovScratch&,                 \
                                        const ArnoldiState&, int, double, cudaStream_t);                            \
  template void launch_norm_start<T>(const C<T>*, const Dims&, const KrylovScratch&, const ArnoldiState*, cudaStream_t,   \
                                     double);                                                                            \
  template void launch_cgs_dots_sel<T>(const C<T>*, int64_t, int, const C<T>*, const Dims&, const KrylovScratch&,           \
                                       const ArnoldiState&, int, int, double, cudaStream_t);                        \
  template void launch_cgs_reorth<T>(const C<T>*, int64_t, int, C<T>*, const Dims&, const KrylovScratch&, const ArnoldiState&, \
                                     int, int, cudaStream_t);                                                       \
  template void launch_cgs_next<T>(const C<T>*, int64_t, int, const C<T>*, const Dims&, const KrylovScratch&, C<T>*,         \
                                   const C<T>*, C<T>*, cudaStream_t);                                               \
  template void launch_combine_dinv<T>(C<T>*, const C<T>*, int64_t, int, const ArnoldiState&, const C<T>*, const Dims&, \
                                       cudaStream_t);                                                               \
  template void launch_combine<T>(C<T>*, const C<T>*, int64_t, int, const ArnoldiState&, bool, const Dims&, cudaStream_t); \
  template void launch_mr_update2<T>(C<T>*, const C<T>*, const C<T>*, C<T>*, const C<T>*, const double2*, const C<T>*,    \
                                     C<T>*, bool, const Dims&, cudaStream_t);
ADR_INSTANTIATE_KRYLOV(double)
ADR_INSTANTIATE_KRYLOV(float)
template void launch_ccast<double, float>(const C<double>*, C<float>*, int64_t, cudaStream_t);
template void launch_ccast<float, double>(const C<float>*, C<double>*, int64_t, cudaStream_t);

}  // namespace adr
