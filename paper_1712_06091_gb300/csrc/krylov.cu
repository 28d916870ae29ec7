// Krylov building blocks: deterministic multi-dot reductions (warp shuffles,
// then a fixed-order pass over per-block partials), multi-AXPY, scaling, and
// the small single-thread kernels that keep the Arnoldi Hessenberg matrix,
// its Givens rotations and the least-squares right-hand side on the device.
//
// These serve the outer flexible GMRES, the inner FGMRES of the K-cycle
// (Alg. Kcycle), the fixed-count Jacobi-preconditioned GMRES of the coarsest
// grid and the minimal-residual Jacobi relaxation (Sec. 3.1).
#include "krylov.cuh"
#include "reduce.cuh"
#include "krylov_dev.cuh"

namespace adr {

static inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

int reduction_blocks(int64_t n) {
  int64_t b = (n + 1023) / 1024;
  if (b < 1) b = 1;
  if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
  return (int)b;
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Block-wide sum in a fixed order; result valid in thread 0.
__device__ __forceinline__ double2 block_sum(double2 v, double2* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    v = lane < nw ? sh[lane] : make_double2(0.0, 0.0);
    v = warp_sum(v);
  }
  return v;
}

constexpr int kDotChunk = 4;

// partial[b * k + i] = sum over this block's elements of conj(V_i) w
template <typename T>
__global__ void __launch_bounds__(256) k_dots_partial(const C<T>* __restrict__ V, int64_t ld, int k,
                                                      const C<T>* __restrict__ w, int64_t n, double2* __restrict__ partial) {
  __shared__ double2 sh[32];
  for (int c = 0; c < k; c += kDotChunk) {
    C<T> acc[kDotChunk];
#pragma unroll
    for (int q = 0; q < kDotChunk; ++q) acc[q] = czero<T>();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
      const C<T> we = w[e];
#pragma unroll
      for (int q = 0; q < kDotChunk; ++q)
        if (c + q < k) acc[q] = cfma_conj(V[(int64_t)(c + q) * ld + e], we, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kDotChunk; ++q) {
      if (c + q >= k) break;
      const double2 s = block_sum(make_double2((double)acc[q].x, (double)acc[q].y), sh);
      if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * k + c + q] = s;
    }
  }
}

// out[i] = sum_b partial[b * k + i]  (one block, fixed order)
__global__ void __launch_bounds__(256) k_dots_final(const double2* __restrict__ partial, int nb, int k,
                                                    double2* __restrict__ out, int accumulate) {
  __shared__ double2 sh[32];
  for (int i = 0; i < k; ++i) {
    double2 v = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      v.x += partial[(int64_t)b * k + i].x;
      v.y += partial[(int64_t)b * k + i].y;
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0) {
      if (accumulate) { out[i].x += v.x; out[i].y += v.y; }
      else out[i] = v;
    }
  }
}

template <typename T>
void launch_dots(const C<T>* V, int64_t ld, int k, const C<T>* w, int64_t n, double2* partial, double2* out,
                 cudaStream_t st, bool accumulate) {
  const int nb = reduction_blocks(n);
  count_launches(1), k_dots_partial<T><<<nb, 256, 0, st>>>(V, ld, k, w, n, partial);
  count_launches(1), k_dots_final<<<1, 256, 0, st>>>(partial, nb, k, out, accumulate ? 1 : 0);
}

// w += sign * sum_i V_i coef[i]
template <typename T>
__global__ void k_axpy_multi(C<T>* __restrict__ w, const C<T>* __restrict__ V, int64_t ld, int k,
                             const double2* __restrict__ coef, double sign, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  C<T> acc = w[e];
  for (int i = 0; i < k; ++i) {
    const double2 cd = coef[i];
    const C<T> c = mk<T>((T)(sign * cd.x), (T)(sign * cd.y));
    acc = cfma(V[(int64_t)i * ld + e], c, acc);
  }
  w[e] = acc;
}
template <typename T>
void launch_axpy_multi(C<T>* w, const C<T>* V, int64_t ld, int k, const double2* coef, double sign, int64_t n,
                       cudaStream_t st) {
  if (k <= 0) return;
  count_launches(1), k_axpy_multi<T><<<blocks_for(n, 256), 256, 0, st>>>(w, V, ld, k, coef, sign, n);
}

// out = w / |w| with the reciprocal norm precomputed in nrm2->y by the kernel
// that reduced nrm2->x (zero if the norm vanishes): no per-thread float64
// square root or division.
template <typename T>
__global__ void k_scale_inv_norm(const C<T>* w, C<T>* out, const double2* __restrict__ nrm2, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const T inv = (T)nrm2->y;
  out[e] = cscale(w[e], inv);
}
template <typename T>
void launch_scale_inv_norm(const C<T>* w, C<T>* out, const double2* nrm2, int64_t n, cudaStream_t st) {
  count_launches(1), k_scale_inv_norm<T><<<blocks_for(n, 256), 256, 0, st>>>(w, out, nrm2, n);
}

template <typename T>
__global__ void k_copy(const C<T>* __restrict__ a, C<T>* __restrict__ b, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) b[e] = a[e];
}
template <typename T> void launch_copy(const C<T>* a, C<T>* b, int64_t n, cudaStream_t st) {
  count_launches(1), k_copy<T><<<blocks_for(n, 256), 256, 0, st>>>(a, b, n);
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
// Small device-side Arnoldi state (one thread)
// ---------------------------------------------------------------------------
__global__ void k_cycle_start(ArnoldiState st, const double2* nrm2) {
  if (threadIdx.x != 0) return;
  const double beta = sqrt(nrm2->x);
  for (int i = 0; i <= st.m; ++i) st.g[i] = make_double2(0.0, 0.0);
  st.g[0] = make_double2(beta, 0.0);
  st.scal[kScalBeta] = beta;
  st.scal[kScalEst] = beta;
  st.iscal[kIScalStop] = beta > 0.0 ? -1 : 0;  // k at exact breakdown, -1 while none
}

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes and the
// squared norm of the orthogonalised vector; rotations and g updated.
__global__ void k_arnoldi_column(ArnoldiState st, int j, const double2* ha, const double2* hb, const double2* nrm2) {
  if (threadIdx.x != 0) return;
  arnoldi_column_dev(st, j, ha, hb, nrm2->x);
}

// y = R^{-1} g for the leading k x k block (k = breakdown index if any).
__global__ void k_backsolve(ArnoldiState st, int k) {
  if (threadIdx.x != 0) return;
  backsolve_dev(st, k);
}

// alpha = (w^H r) / (w^H w) from d[0] = w^H r, d[1] = w^H w (0 if w = 0).
__global__ void k_mr_alpha(const double2* d, double2* alpha) {
  if (threadIdx.x != 0) return;
  const double den = d[1].x;
  *alpha = den > 0.0 ? make_double2(d[0].x / den, d[0].y / den) : make_double2(0.0, 0.0);
}

void launch_cycle_start(const ArnoldiState& s, const double2* nrm2, cudaStream_t st) { count_launches(1), k_cycle_start<<<1, 32, 0, st>>>(s, nrm2); }
void launch_arnoldi_column(const ArnoldiState& s, int j, const double2* ha, const double2* hb, const double2* nrm2, cudaStream_t st) {
  count_launches(1), k_arnoldi_column<<<1, 32, 0, st>>>(s, j, ha, hb, nrm2);
}
void launch_backsolve(const ArnoldiState& s, int k, cudaStream_t st) { count_launches(1), k_backsolve<<<1, 32, 0, st>>>(s, k); }
void launch_mr_alpha(const double2* d, double2* alpha, cudaStream_t st) { count_launches(1), k_mr_alpha<<<1, 32, 0, st>>>(d, alpha); }

// Two dots against one vector a: d[0] = a^H b, d[1] = a^H c.
template <typename T>
__global__ void __launch_bounds__(256) k_dot2_partial(const C<T>* __restrict__ a, const C<T>* __restrict__ b,
                                                      const C<T>* __restrict__ c, int64_t n, double2* __restrict__ partial) {
  __shared__ double2 sh[32];
  C<T> s0 = czero<T>(), s1 = czero<T>();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const C<T> ae = a[e];
    s0 = cfma_conj(ae, b[e], s0);
    s1 = cfma_conj(ae, c[e], s1);
  }
  double2 v0 = block_sum(make_double2((double)s0.x, (double)s0.y), sh);
  if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * 2 + 0] = v0;
  double2 v1 = block_sum(make_double2((double)s1.x, (double)s1.y), sh);
  if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * 2 + 1] = v1;
}
template <typename T>
void launch_dot2(const C<T>* a, const C<T>* b, const C<T>* c, int64_t n, double2* partial, double2* out, cudaStream_t st) {
  const int nb = reduction_blocks(n);
  count_launches(1), k_dot2_partial<T><<<nb, 256, 0, st>>>(a, b, c, n, partial);
  count_launches(1), k_dots_final<<<1, 256, 0, st>>>(partial, nb, 2, out, 0);
}

// x += alpha z ; r -= alpha w ; (optional) znext = dinv .* r
template <typename T>
__global__ void k_mr_update(C<T>* __restrict__ x, const C<T>* __restrict__ z, C<T>* __restrict__ r,
                            const C<T>* __restrict__ w, const double2* __restrict__ alpha, const C<T>* __restrict__ dinv,
                            C<T>* __restrict__ znext, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const C<T> al = mk<T>((T)alpha->x, (T)alpha->y);
  x[e] = cfma(al, z[e], x[e]);
  const C<T> rn = csub(r[e], cmul(al, w[e]));
  r[e] = rn;
  if (znext) znext[e] = cmul(dinv[e], rn);
}
template <typename T>
void launch_mr_update(C<T>* x, const C<T>* z, C<T>* r, const C<T>* w, const double2* alpha, const C<T>* dinv, C<T>* znext,
                      int64_t n, cudaStream_t st) {
  count_launches(1), k_mr_update<T><<<blocks_for(n, 256), 256, 0, st>>>(x, z, r, w, alpha, dinv, znext, n);
}

template <typename T>
__global__ void k_zero(C<T>* __restrict__ a, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) a[e] = czero<T>();
}
template <typename T> void launch_zero(C<T>* a, int64_t n, cudaStream_t st) {
  count_launches(1), k_zero<T><<<blocks_for(n, 256), 256, 0, st>>>(a, n);
}

#define ADR_INSTANTIATE_KRYLOV(T)                                                                                    \
  template void launch_dots<T>(const C<T>*, int64_t, int, const C<T>*, int64_t, double2*, double2*, cudaStream_t, bool); \
  template void launch_axpy_multi<T>(C<T>*, const C<T>*, int64_t, int, const double2*, double, int64_t, cudaStream_t); \
  template void launch_scale_inv_norm<T>(const C<T>*, C<T>*, const double2*, int64_t, cudaStream_t);                  \
  template void launch_copy<T>(const C<T>*, C<T>*, int64_t, cudaStream_t);                                            \
  template void launch_cmul_vec<T>(const C<T>*, const C<T>*, C<T>*, int64_t, cudaStream_t);                           \
  template void launch_dot2<T>(const C<T>*, const C<T>*, const C<T>*, int64_t, double2*, double2*, cudaStream_t);     \
  template void launch_mr_update<T>(C<T>*, const C<T>*, C<T>*, const C<T>*, const double2*, const C<T>*, C<T>*, int64_t, cudaStream_t); \
  template void launch_zero<T>(C<T>*, int64_t, cudaStream_t);
ADR_INSTANTIATE_KRYLOV(double)
ADR_INSTANTIATE_KRYLOV(float)
template void launch_ccast<double, float>(const C<double>*, C<float>*, int64_t, cudaStream_t);
template void launch_ccast<float, double>(const C<float>*, C<double>*, int64_t, cudaStream_t);

// ===========================================================================
// Fused Arnoldi / Krylov kernels (one launch per pass, deterministic
// last-block reductions; see reduce.cuh)
// ===========================================================================

// Block sums of k values held per thread in chunks; the block's k totals are
// left in blk[0..k) (shared memory).  acc_fn(i) returns thread's value i.
// Then the last block reduces partials over blocks into out[0..k).
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
  for (int i = 0; i < k; ++i) {
    double2 acc = make_double2(0.0, 0.0);
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
      const double2 p = __ldcg(&partial[(size_t)b * k + i]);
      acc.x += p.x;
      acc.y += p.y;
    }
    double2 v[1] = {acc}, o[1];
    block_sum_k<1>(v, sh, o);
    if (threadIdx.x == 0) out[i] = o[0];
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __syncthreads();
  return true;
}

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

// pass 1: ha = V^H w
template <typename T>
__global__ void __launch_bounds__(256) k_cgs_pass1(const C<T>* __restrict__ V, int64_t ld, int k, const C<T>* w, int64_t n,
                                                   double2* partial, unsigned* ticket, double2* ha) {
  __shared__ double2 sh[32 * 4];
  __shared__ double2 blk[kMaxKrylov + 1];
  block_dots<T>(V, ld, k, w, n, blk, sh);
  last_block_rt(k, blk, partial, ticket, ha, sh);
}

// pass 2: w -= V ha ; hb = V^H w
template <typename T>
__global__ void __launch_bounds__(256) k_cgs_pass2(const C<T>* __restrict__ V, int64_t ld, int k, C<T>* w, int64_t n,
                                                   const double2* __restrict__ ha, double2* partial, unsigned* ticket,
                                                   double2* hb) {
  __shared__ double2 sh[32 * 4];
  __shared__ double2 blk[kMaxKrylov + 1];
  __shared__ C<T> coef[kMaxKrylov + 1];
  for (int i = threadIdx.x; i < k; i += blockDim.x) coef[i] = mk<T>((T)(-ha[i].x), (T)(-ha[i].y));
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    C<T> acc = w[e];
    for (int i = 0; i < k; ++i) acc = cfma(V[(int64_t)i * ld + e], coef[i], acc);
    w[e] = acc;
  }
  block_dots<T>(V, ld, k, w, n, blk, sh);   // each thread re-reads only its own elements of w
  last_block_rt(k, blk, partial, ticket, hb, sh);
}

// w -= V c ; |w|^2 reduced over the grid.  Returns true in the last block
// (total in nrm2->x, valid in thread 0).
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

// pass 3: w -= V hb ; |w|^2 ; Arnoldi column j and Givens rotation (last block)
template <typename T>
__global__ void __launch_bounds__(256) k_cgs_pass3(const C<T>* __restrict__ V, int64_t ld, int k, C<T>* w, int64_t n,
                                                   const double2* __restrict__ ha, const double2* __restrict__ hb,
                                                   double2* partial, unsigned* ticket, double2* nrm2, ArnoldiState st, int j) {
  if (update_norm<T>(V, ld, k, w, n, hb, partial, ticket, nrm2) && threadIdx.x == 0) {
    const double s2t = nrm2->x;
    nrm2->y = s2t > 0.0 ? 1.0 / sqrt(s2t) : 0.0;
    if (st.m > 0) arnoldi_column_dev(st, j, ha, hb, s2t);
  }
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
                                                       int64_t n, double2* partial, unsigned* ticket, double2* ha) {
  __shared__ double2 sh[32 * 5];
  __shared__ double2 blk[kMaxKrylov + 2];
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
  last_block_rt(k + 1, blk, partial, ticket, ha, sh);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sgs_update_test(const C<T>* __restrict__ V, int64_t ld, int k, C<T>* w, int64_t n,
                                                         double2* ha, double2* hb, double2* partial, unsigned* ticket,
                                                         double2* nrm2, ArnoldiState st, int j, double eta2) {
  if (update_norm<T>(V, ld, k, w, n, ha, partial, ticket, nrm2) && threadIdx.x == 0) {
    const double t = nrm2->x;
    if (t >= eta2 * ha[k].x) {
      ha[k].y = 0.0;
      for (int i = 0; i < k; ++i) hb[i] = make_double2(0.0, 0.0);
      nrm2->y = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
      if (st.m > 0) arnoldi_column_dev(st, j, ha, hb, t);
    } else {
      ha[k].y = 1.0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sgs_reorth_dots(const C<T>* __restrict__ V, int64_t ld, int k, const C<T>* w,
                                                         int64_t n, const double2* ha, double2* partial, unsigned* ticket,
                                                         double2* hb) {
  if (ha[k].y == 0.0) return;   // uniform over the grid
  __shared__ double2 sh[32 * 4];
  __shared__ double2 blk[kMaxKrylov + 1];
  block_dots<T>(V, ld, k, w, n, blk, sh);
  last_block_rt(k, blk, partial, ticket, hb, sh);
}

template <typename T>
__global__ void __launch_bounds__(256) k_sgs_reorth_update(const C<T>* __restrict__ V, int64_t ld, int k, C<T>* w, int64_t n,
                                                           const double2* ha, const double2* hb, double2* partial,
                                                           unsigned* ticket, double2* nrm2, ArnoldiState st, int j) {
  if (ha[k].y == 0.0) return;   // uniform over the grid
  if (update_norm<T>(V, ld, k, w, n, hb, partial, ticket, nrm2) && threadIdx.x == 0) {
    const double s2t = nrm2->x;
    nrm2->y = s2t > 0.0 ? 1.0 / sqrt(s2t) : 0.0;
    if (st.m > 0) arnoldi_column_dev(st, j, ha, hb, s2t);
  }
}

// |b|^2 and (optionally) the start of an Arnoldi cycle with beta = |b|.
template <typename T>
__global__ void __launch_bounds__(256) k_norm_start(const C<T>* b, int64_t n, double2* partial, unsigned* ticket,
                                                    double2* nrm2, ArnoldiState st, int start) {
  __shared__ double2 sh[32 * 4];
  __shared__ double2 blk[1];
  C<T> s2[1] = {czero<T>()};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s2[0] = cfma_conj(b[e], b[e], s2[0]);
  double2 o[1];
  block_sum_t<T, 1>(s2, sh, o);
  if (threadIdx.x == 0) blk[0] = o[0];
  __syncthreads();
  if (last_block_rt(1, blk, partial, ticket, nrm2, sh) && threadIdx.x == 0) {
    const double beta = sqrt(nrm2->x);
    nrm2->y = beta > 0.0 ? 1.0 / beta : 0.0;
    if (!start) return;
    for (int i = 0; i <= st.m; ++i) st.g[i] = make_double2(0.0, 0.0);
    st.g[0] = make_double2(beta, 0.0);
    st.scal[kScalBeta] = beta;
    st.scal[kScalEst] = beta;
    st.iscal[kIScalStop] = beta > 0.0 ? -1 : 0;
  }
}

// x = (assign ? 0 : x) + sum_i Z_i y_i  (y from the state, i < k)
template <typename T>
__global__ void k_combine(C<T>* x, const C<T>* __restrict__ Z, int64_t ld, int k, ArnoldiState st, int assign, int64_t n) {
  __shared__ C<T> coef[kMaxKrylov];
  for (int i = threadIdx.x; i < k; i += blockDim.x) coef[i] = mk<T>((T)st.y[i].x, (T)st.y[i].y);
  __syncthreads();
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  C<T> acc = assign ? czero<T>() : x[e];
  for (int i = 0; i < k; ++i) acc = cfma(Z[(int64_t)i * ld + e], coef[i], acc);
  x[e] = acc;
}

// x = (x_zero ? 0 : x) + alpha z ; r_dst = r_src - alpha w ; znext = dinv .* r_dst
template <typename T>
__global__ void k_mr_update2(C<T>* x, const C<T>* z, const C<T>* r_src, C<T>* r_dst,
                             const C<T>* __restrict__ w, const double2* __restrict__ alpha, const C<T>* __restrict__ dinv,
                             C<T>* znext, int x_zero, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const C<T> al = mk<T>((T)alpha->x, (T)alpha->y);
  x[e] = cfma(al, z[e], x_zero ? czero<T>() : x[e]);
  const C<T> rn = csub(r_src[e], cmul(al, w[e]));
  r_dst[e] = rn;
  if (znext) znext[e] = cmul(dinv[e], rn);
}

template <typename T>
void launch_cgs2(const C<T>* V, int64_t ld, int k, C<T>* w, int64_t n, const KrylovScratch& s, const ArnoldiState& st, int j,
                 cudaStream_t stream) {
  const int nb = reduction_blocks(n);
  count_launches(1), k_cgs_pass1<T><<<nb, 256, 0, stream>>>(V, ld, k, w, n, s.partial, s.ticket, s.ha);
  count_launches(1), k_cgs_pass2<T><<<nb, 256, 0, stream>>>(V, ld, k, w, n, s.ha, s.partial, s.ticket, s.hb);
  count_launches(1), k_cgs_pass3<T><<<nb, 256, 0, stream>>>(V, ld, k, w, n, s.ha, s.hb, s.partial, s.ticket, s.nrm2, st, j);
}
template <typename T>
void launch_cgs_selective(const C<T>* V, int64_t ld, int k, C<T>* w, int64_t n, const KrylovScratch& s,
                          const ArnoldiState& st, int j, double eta, cudaStream_t stream) {
  if (!(eta < 1.0)) {
    launch_cgs2<T>(V, ld, k, w, n, s, st, j, stream);
    return;
  }
  const int nb = reduction_blocks(n);
  count_launches(1), k_sgs_dots_norm<T><<<nb, 256, 0, stream>>>(V, ld, k, w, n, s.partial, s.ticket, s.ha);
  count_launches(1), k_sgs_update_test<T><<<nb, 256, 0, stream>>>(V, ld, k, w, n, s.ha, s.hb, s.partial, s.ticket, s.nrm2,
                                                                    st, j, eta * eta);
  count_launches(1), k_sgs_reorth_dots<T><<<nb, 256, 0, stream>>>(V, ld, k, w, n, s.ha, s.partial, s.ticket, s.hb);
  count_launches(1), k_sgs_reorth_update<T><<<nb, 256, 0, stream>>>(V, ld, k, w, n, s.ha, s.hb, s.partial, s.ticket,
                                                                      s.nrm2, st, j);
}
template <typename T>
void launch_norm_start(const C<T>* b, int64_t n, const KrylovScratch& s, const ArnoldiState* st, cudaStream_t stream) {
  const int nb = reduction_blocks(n);
  ArnoldiState dummy{};
  count_launches(1), k_norm_start<T><<<nb, 256, 0, stream>>>(b, n, s.partial, s.ticket, s.nrm2, st ? *st : dummy, st ? 1 : 0);
}
template <typename T>
void launch_combine(C<T>* x, const C<T>* Z, int64_t ld, int k, const ArnoldiState& st, bool assign, int64_t n, cudaStream_t stream) {
  count_launches(1), k_combine<T><<<blocks_for(n, 256), 256, 0, stream>>>(x, Z, ld, k, st, assign ? 1 : 0, n);
}
template <typename T>
void launch_mr_update2(C<T>* x, const C<T>* z, const C<T>* r_src, C<T>* r_dst, const C<T>* w, const double2* alpha,
                       const C<T>* dinv, C<T>* znext, bool x_zero, int64_t n, cudaStream_t stream) {
  count_launches(1), k_mr_update2<T><<<blocks_for(n, 256), 256, 0, stream>>>(x, z, r_src, r_dst, w, alpha, dinv, znext,
                                                                               x_zero ? 1 : 0, n);
}

#define ADR_INSTANTIATE_FUSED(T)                                                                                           \
  template void launch_cgs2<T>(const C<T>*, int64_t, int, C<T>*, int64_t, const KrylovScratch&, const ArnoldiState&, int, cudaStream_t); \
  template void launch_cgs_selective<T>(const C<T>*, int64_t, int, C<T>*, int64_t, const KrylovScratch&, const ArnoldiState&, int, \
                                        double, cudaStream_t);                                                              \
  template void launch_norm_start<T>(const C<T>*, int64_t, const KrylovScratch&, const ArnoldiState*, cudaStream_t);        \
  template void launch_combine<T>(C<T>*, const C<T>*, int64_t, int, const ArnoldiState&, bool, int64_t, cudaStream_t);     \
  template void launch_mr_update2<T>(C<T>*, const C<T>*, const C<T>*, C<T>*, const C<T>*, const double2*, const C<T>*, C<T>*, bool, int64_t, cudaStream_t);
ADR_INSTANTIATE_FUSED(double)
ADR_INSTANTIATE_FUSED(float)

}  // namespace adr
