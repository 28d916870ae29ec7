// Krylov building blocks: deterministic multi-dot reductions (warp shuffles,
// then a fixed-order pass over per-block partials), multi-AXPY, scaling, and
// the small single-thread kernels that keep the Arnoldi Hessenberg matrix,
// its Givens rotations and the least-squares right-hand side on the device.
//
// These serve the outer flexible GMRES, the inner FGMRES of the K-cycle
// (Alg. Kcycle), the fixed-count Jacobi-preconditioned GMRES of the coarsest
// grid and the minimal-residual Jacobi relaxation (Sec. 3.1).
#include "krylov.cuh"

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

// out = w / sqrt(nrm2->x), or zero if the norm vanishes.
template <typename T>
__global__ void k_scale_inv_norm(const C<T>* w, C<T>* out, const double2* __restrict__ nrm2, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double s = sqrt(nrm2->x);
  const T inv = s > 0.0 ? (T)(1.0 / s) : T(0);
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
// Complex Givens rotation with real cosine: [c s; -conj(s) c] [a; b] = [r; 0].
__device__ void givens(double2 a, double2 b, double& c, double2& s, double2& r) {
  const double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
  if (bb == 0.0) { c = 1.0; s = make_double2(0.0, 0.0); r = a; return; }
  if (aa == 0.0) { c = 0.0; s = make_double2(1.0, 0.0); r = b; return; }
  const double nu = sqrt(aa * aa + bb * bb);
  c = aa / nu;
  const double2 ph = make_double2(a.x / aa, a.y / aa);
  const double2 cb = make_double2(b.x / nu, -b.y / nu);
  s = cmul(ph, cb);
  r = make_double2(ph.x * nu, ph.y * nu);
}

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
  const int m1 = st.m + 1;
  double2* H = st.H + (int64_t)j * m1;
  if (st.iscal[kIScalStop] >= 0) {  // already broken down: leave the column empty
    for (int i = 0; i <= j + 1; ++i) H[i] = make_double2(0.0, 0.0);
    st.scal[kScalHn] = 0.0;
    return;
  }
  for (int i = 0; i <= j; ++i) H[i] = make_double2(ha[i].x + (hb ? hb[i].x : 0.0), ha[i].y + (hb ? hb[i].y : 0.0));
  const double hn = sqrt(nrm2->x);
  H[j + 1] = make_double2(hn, 0.0);
  for (int i = 0; i < j; ++i) {
    const double2 a = H[i], b = H[i + 1];
    const double c = st.cs[i];
    const double2 s = st.sn[i];
    const double2 cs_ = make_double2(s.x, -s.y);  // conj(s)
    H[i] = cadd(make_double2(c * a.x, c * a.y), cmul(s, b));
    H[i + 1] = csub(make_double2(c * b.x, c * b.y), cmul(cs_, a));
  }
  double c;
  double2 s, r;
  givens(H[j], H[j + 1], c, s, r);
  st.cs[j] = c;
  st.sn[j] = s;
  H[j] = r;
  H[j + 1] = make_double2(0.0, 0.0);
  const double2 gj = st.g[j];
  st.g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));  // -conj(s) g_j
  st.g[j] = make_double2(c * gj.x, c * gj.y);
  st.scal[kScalEst] = hypot(st.g[j + 1].x, st.g[j + 1].y);
  st.scal[kScalHn] = hn;
  if (hn == 0.0) st.iscal[kIScalStop] = j + 1;
}

// y = R^{-1} g for the leading k x k block (k = breakdown index if any).
__global__ void k_backsolve(ArnoldiState st, int k) {
  if (threadIdx.x != 0) return;
  const int m1 = st.m + 1;
  const int stop = st.iscal[kIScalStop];
  if (stop >= 0 && stop < k) k = stop;
  for (int i = 0; i < st.m; ++i) st.y[i] = make_double2(0.0, 0.0);
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = st.g[i];
    for (int q = i + 1; q < k; ++q) acc = csub(acc, cmul(st.H[(int64_t)q * m1 + i], st.y[q]));
    const double2 rii = st.H[(int64_t)i * m1 + i];
    st.y[i] = cmul(acc, cinv(rii));
  }
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

}  // namespace adr
