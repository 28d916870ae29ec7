// Coarse-level kernels: operators stored as Galerkin stencils
// (Eq. coarseGridMatrix, A_c = P^T A P), bilinear / trilinear transfers
// (P and its transpose, Sec. 3.1), relaxation and residuals on those levels.
#include "adr_common.cuh"
#include "coarse_stencil.cuh"
#include "krylov_dev.cuh"
#include "reduce.cuh"

namespace adr {

static inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }


// BT: batched launch (grid.y = problems).  The single-problem instantiation
// carries no per-problem pointer arithmetic, which keeps these
// register-capped kernels' spills at their unbatched level.
template <int DIM, typename T, bool BT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_stencil_apply(Dims g, const C<T>* __restrict__ A, const C<T>* __restrict__ x, C<T>* __restrict__ y) {
  if (BT && resolve(g)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  if (BT) {
    shift_stencil(g, A);
    shift_nodes(g, x, y);
  }
  int i0, i1, i2;
  unravel(g, j, i0, i1, i2);
  y[j] = stencil_dot<DIM, T>(g, A, x, j, i0, i1, i2);
}

template <int DIM, typename T>
__global__ void k_stencil_residual(Dims g, const C<T>* __restrict__ A, const C<T>* __restrict__ b,
                                   const C<T>* __restrict__ x, C<T>* __restrict__ r) {
  if (resolve(g)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  shift_stencil(g, A);
  shift_nodes(g, b, x, r);
  int i0, i1, i2;
  unravel(g, j, i0, i1, i2);
  r[j] = csub(b[j], stencil_dot<DIM, T>(g, A, x, j, i0, i1, i2));
}

template <int DIM, typename T>
__global__ void k_stencil_jacobi(Dims g, const C<T>* __restrict__ A, const C<T>* __restrict__ dinv,
                                 const C<T>* __restrict__ b, const C<T>* __restrict__ xin, C<T>* __restrict__ xout, T w) {
  if (resolve(g)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  shift_stencil(g, A);
  shift_nodes(g, dinv, b, xout);
  shift_nodes_opt(g, xin);
  if (xin == nullptr) {
    xout[j] = cscale(cmul(dinv[j], b[j]), w);
    return;
  }
  int i0, i1, i2;
  unravel(g, j, i0, i1, i2);
  const C<T> r = csub(b[j], stencil_dot<DIM, T>(g, A, xin, j, i0, i1, i2));
  xout[j] = cadd(xin[j], cscale(cmul(dinv[j], r), w));
}

// Galerkin product of a stored stencil (level l) into level l+1.
template <int DIM, typename T>
__global__ void k_galerkin_stored(Dims gf, Dims gc, const C<T>* __restrict__ Af, C<T>* __restrict__ out,
                                  C<T>* __restrict__ dinv) {
  if (resolve(gf)) return;
  resolve(gc);
  constexpr int S = PatternSize<DIM>::value;
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= gc.N) return;
  shift_stencil(gf, Af);
  shift_stencil(gc, out);
  shift_nodes(gc, dinv);
  int Ii[3];
  unravel(gc, I, Ii[0], Ii[1], Ii[2]);
  C<T> acc[S];
  for (int p = 0; p < S; ++p) acc[p] = czero<T>();
  const int lo2 = DIM > 2 ? -1 : 0, hi2 = DIM > 2 ? 1 : 0;
  for (int e2 = lo2; e2 <= hi2; ++e2)
    for (int e1 = -1; e1 <= 1; ++e1)
      for (int e0 = -1; e0 <= 1; ++e0) {
        const int fi[3] = {2 * Ii[0] + e0, 2 * Ii[1] + e1, DIM > 2 ? 2 * Ii[2] + e2 : 0};
        bool ok = true;
        for (int d = 0; d < DIM; ++d) ok = ok && fi[d] >= 0 && fi[d] < gf.n[d];
        if (!ok) continue;
        const T wi = (e0 ? T(0.5) : T(1)) * (e1 ? T(0.5) : T(1)) * (e2 ? T(0.5) : T(1));
        const int64_t fj = fi[0] + gf.s1 * fi[1] + gf.s2 * fi[2];
        for (int p = 0; p < S; ++p) {
          const int8_t* o = pattern_offset<DIM>(p);
          const int k[3] = {fi[0] + o[0], fi[1] + o[1], fi[2] + o[2]};
          bool in = true;
          for (int d = 0; d < DIM; ++d) in = in && k[d] >= 0 && k[d] < gf.n[d];
          if (!in) continue;
          const C<T> wa = cscale(stencil_get<DIM, T>(Af, p, fj), wi);
          int pj[3][2];
          T pw[3][2];
          int pc[3];
          for (int d = 0; d < 3; ++d) {
            if (d >= DIM) { pj[d][0] = 0; pw[d][0] = T(1); pc[d] = 1; continue; }
            if ((k[d] & 1) == 0) { pj[d][0] = k[d] >> 1; pw[d][0] = T(1); pc[d] = 1; }
            else { pj[d][0] = (k[d] - 1) >> 1; pj[d][1] = (k[d] + 1) >> 1; pw[d][0] = pw[d][1] = T(0.5); pc[d] = 2; }
          }
          for (int q2 = 0; q2 < pc[2]; ++q2)
            for (int q1 = 0; q1 < pc[1]; ++q1)
              for (int q0 = 0; q0 < pc[0]; ++q0) {
                const int s = pattern_slot<DIM>(pj[0][q0] - Ii[0], pj[1][q1] - Ii[1], DIM > 2 ? pj[2][q2] - Ii[2] : 0);
                acc[s] = cadd(acc[s], cscale(wa, pw[0][q0] * pw[1][q1] * pw[2][q2]));
              }
        }
      }
  for (int p = 0; p < S; ++p) stencil_put<DIM, T>(out, p, I, acc[p]);
  dinv[I] = cinv(acc[(S - 1) / 2]);
}

// r_c = P^T r_f : weights 1 on the coincident node, 1/2 per axis offset by one.
template <int DIM, typename T>
__global__ void k_restrict(Dims gf, Dims gc, const C<T>* __restrict__ rf, C<T>* __restrict__ rc) {
  if (resolve(gf)) return;
  resolve(gc);
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= gc.N) return;
  shift_nodes(gf, rf);
  shift_nodes(gc, rc);
  int Ii[3];
  unravel(gc, I, Ii[0], Ii[1], Ii[2]);
  C<T> acc = czero<T>();
  const int lo2 = DIM > 2 ? -1 : 0, hi2 = DIM > 2 ? 1 : 0;
  for (int e2 = lo2; e2 <= hi2; ++e2) {
    const int f2 = DIM > 2 ? 2 * Ii[2] + e2 : 0;
    if (DIM > 2 && (f2 < 0 || f2 >= gf.n[2])) continue;
    for (int e1 = -1; e1 <= 1; ++e1) {
      const int f1 = 2 * Ii[1] + e1;
      if (f1 < 0 || f1 >= gf.n[1]) continue;
      for (int e0 = -1; e0 <= 1; ++e0) {
        const int f0 = 2 * Ii[0] + e0;
        if (f0 < 0 || f0 >= gf.n[0]) continue;
        const T w = (e0 ? T(0.5) : T(1)) * (e1 ? T(0.5) : T(1)) * (e2 ? T(0.5) : T(1));
        acc = cadd(acc, cscale(rf[f0 + gf.s1 * f1 + gf.s2 * f2], w));
      }
    }
  }
  rc[I] = acc;
}

// x_f += P e_c
template <int DIM, typename T>
__global__ void k_prolong_add(Dims gf, Dims gc, const C<T>* __restrict__ ec, C<T>* __restrict__ xf) {
  if (resolve(gf)) return;
  resolve(gc);
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= gf.N) return;
  shift_nodes(gc, ec);
  shift_nodes(gf, xf);
  int ii[3];
  unravel(gf, j, ii[0], ii[1], ii[2]);
  int pj[3][2];
  T pw[3][2];
  int pc[3];
  for (int d = 0; d < 3; ++d) {
    if (d >= DIM) { pj[d][0] = 0; pw[d][0] = T(1); pc[d] = 1; continue; }
    if ((ii[d] & 1) == 0) { pj[d][0] = ii[d] >> 1; pw[d][0] = T(1); pc[d] = 1; }
    else { pj[d][0] = (ii[d] - 1) >> 1; pj[d][1] = (ii[d] + 1) >> 1; pw[d][0] = pw[d][1] = T(0.5); pc[d] = 2; }
  }
  C<T> acc = czero<T>();
  for (int q2 = 0; q2 < pc[2]; ++q2)
    for (int q1 = 0; q1 < pc[1]; ++q1)
      for (int q0 = 0; q0 < pc[0]; ++q0)
        acc = cadd(acc, cscale(ec[pj[0][q0] + gc.s1 * pj[1][q1] + gc.s2 * pj[2][q2]], pw[0][q0] * pw[1][q1] * pw[2][q2]));
  xf[j] = cadd(xf[j], acc);
}

// Point-major copy (entry p of node j at p * N + j) of a tiled stencil.
template <typename T>
__global__ void k_stencil_export(Dims g, const C<T>* __restrict__ A, C<T>* __restrict__ out, int S) {
  if (resolve(g)) return;
  const int64_t N = g.N;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N * S) return;
  shift_stencil(g, A);
  shift_scaled(g, S, out);
  const int p = (int)(e / N);
  const int64_t j = e - (int64_t)p * N;
  out[e] = S == kPattern2 ? stencil_get<2, T>(A, p, j) : stencil_get<3, T>(A, p, j);
}
template <typename T> void launch_stencil_export(const Dims& g, const C<T>* A, C<T>* out, int S, cudaStream_t st) {
  count_launches(1), k_stencil_export<T><<<dim3(blocks_for(g.N * S, 256), g.B), 256, 0, st>>>(g, A, out, S);
}
template void launch_stencil_export<double>(const Dims&, const double2*, double2*, int, cudaStream_t);
template void launch_stencil_export<float>(const Dims&, const float2*, float2*, int, cudaStream_t);

template <typename T> void launch_stencil_apply(const Dims& g, const C<T>* A, const C<T>* x, C<T>* y, cudaStream_t st) {
  const int th = 256;
  const dim3 grid(blocks_for(g.N, th), g.B);
  if (g.dim == 2) count_launches(1), (g.B > 1 ? k_stencil_apply<2, T, true> : k_stencil_apply<2, T, false>)<<<grid, th, 0, st>>>(g, A, x, y);
  else count_launches(1), (g.B > 1 ? k_stencil_apply<3, T, true> : k_stencil_apply<3, T, false>)<<<grid, th, 0, st>>>(g, A, x, y);
}
template <typename T> void launch_stencil_residual(const Dims& g, const C<T>* A, const C<T>* b, const C<T>* x, C<T>* r, cudaStream_t st) {
  const int th = 256;
  if (g.dim == 2) count_launches(1), k_stencil_residual<2, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, A, b, x, r);
  else count_launches(1), k_stencil_residual<3, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, A, b, x, r);
}
template <typename T> void launch_stencil_jacobi(const Dims& g, const C<T>* A, const C<T>* dinv, const C<T>* b, const C<T>* xin, C<T>* xout, T w, cudaStream_t st) {
  const int th = 256;
  if (g.dim == 2) count_launches(1), k_stencil_jacobi<2, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, A, dinv, b, xin, xout, w);
  else count_launches(1), k_stencil_jacobi<3, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, A, dinv, b, xin, xout, w);
}
template <typename T> void launch_galerkin_stored(const Dims& gf, const Dims& gc, const C<T>* Af, C<T>* Ac, C<T>* dinv, cudaStream_t st) {
  const int th = 64;
  if (gf.dim == 2) count_launches(1), k_galerkin_stored<2, T><<<dim3(blocks_for(gc.N, th), gf.B), th, 0, st>>>(gf, gc, Af, Ac, dinv);
  else count_launches(1), k_galerkin_stored<3, T><<<dim3(blocks_for(gc.N, th), gf.B), th, 0, st>>>(gf, gc, Af, Ac, dinv);
}
template <typename T> void launch_restrict(const Dims& gf, const Dims& gc, const C<T>* rf, C<T>* rc, cudaStream_t st) {
  const int th = 256;
  if (gf.dim == 2) count_launches(1), k_restrict<2, T><<<dim3(blocks_for(gc.N, th), gf.B), th, 0, st>>>(gf, gc, rf, rc);
  else count_launches(1), k_restrict<3, T><<<dim3(blocks_for(gc.N, th), gf.B), th, 0, st>>>(gf, gc, rf, rc);
}
template <typename T> void launch_prolong_add(const Dims& gf, const Dims& gc, const C<T>* ec, C<T>* xf, cudaStream_t st) {
  const int th = 256;
  if (gf.dim == 2) count_launches(1), k_prolong_add<2, T><<<dim3(blocks_for(gf.N, th), gf.B), th, 0, st>>>(gf, gc, ec, xf);
  else count_launches(1), k_prolong_add<3, T><<<dim3(blocks_for(gf.N, th), gf.B), th, 0, st>>>(gf, gc, ec, xf);
}

#define ADR_INSTANTIATE_COARSE(T)                                                                                          \
  template void launch_stencil_apply<T>(const Dims&, const C<T>*, const C<T>*, C<T>*, cudaStream_t);                          \
  template void launch_stencil_residual<T>(const Dims&, const C<T>*, const C<T>*, const C<T>*, C<T>*, cudaStream_t);          \
  template void launch_stencil_jacobi<T>(const Dims&, const C<T>*, const C<T>*, const C<T>*, const C<T>*, C<T>*, T, cudaStream_t); \
  template void launch_galerkin_stored<T>(const Dims&, const Dims&, const C<T>*, C<T>*, C<T>*, cudaStream_t);                 \
  template void launch_restrict<T>(const Dims&, const Dims&, const C<T>*, C<T>*, cudaStream_t);                               \
  template void launch_prolong_add<T>(const Dims&, const Dims&, const C<T>*, C<T>*, cudaStream_t);
ADR_INSTANTIATE_COARSE(double)
ADR_INSTANTIATE_COARSE(float)

}  // namespace adr

// ===========================================================================
// Fused relaxation kernels on stored-stencil levels and the one-block
// coarsest-grid GMRES
// ===========================================================================
namespace adr {

template <int DIM, typename T, bool BT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_stencil_mr_apply(Dims g, const C<T>* __restrict__ A, const C<T>* __restrict__ z,
                                                          const C<T>* __restrict__ r, C<T>* __restrict__ w,
                                                          double2* partial, unsigned* ticket, double2* alpha) {
  __shared__ double2 sh[32 * 2];
  if (BT) {
    if (resolve(g)) return;
    shift_stencil(g, A);
    shift_nodes(g, z, r, w);
    batch_shift(kPartialStride, partial);
    batch_shift(1, ticket, alpha);
  }
  C<T> s[2] = {czero<T>(), czero<T>()};
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < g.N; j += (int64_t)gridDim.x * blockDim.x) {
    int i0, i1, i2;
    unravel(g, j, i0, i1, i2);
    const C<T> wj = stencil_dot<DIM, T>(g, A, z, j, i0, i1, i2);
    w[j] = wj;
    s[0] = cfma_conj(wj, r[j], s[0]);
    s[1] = cfma_conj(wj, wj, s[1]);
  }
  double2 mine[2], tot[2];
  block_sum_t<T, 2>(s, sh, mine);
  if (last_block_total<2>(mine, partial, ticket, tot, sh) && threadIdx.x == 0) {
    const double den = tot[1].x;
    *alpha = den > 0.0 ? make_double2(tot[0].x / den, tot[0].y / den) : make_double2(0.0, 0.0);
  }
}

template <int DIM, typename T, bool BT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_stencil_residual_dinv(Dims g, const C<T>* __restrict__ A, const C<T>* __restrict__ b,
                                        const C<T>* __restrict__ x, const C<T>* __restrict__ dinv, C<T>* __restrict__ r,
                                        C<T>* __restrict__ z) {
  if (BT && resolve(g)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  if (BT) {
    shift_stencil(g, A);
    shift_nodes(g, b, x, dinv, r, z);
  }
  int i0, i1, i2;
  unravel(g, j, i0, i1, i2);
  const C<T> rj = csub(b[j], stencil_dot<DIM, T>(g, A, x, j, i0, i1, i2));
  r[j] = rj;
  z[j] = cmul(dinv[j], rj);
}

// Sums conj(V_i) w over the block for i < k into hh[i] (all threads see it after return).
template <typename T>
__device__ __forceinline__ void cta_dots(const C<T>* V, int64_t ld, int64_t n, int k, const C<T>* w, double2* hh,
                                         double2* sh) {
  for (int c = 0; c < k; c += 4) {
    C<T> acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = czero<T>();
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      const C<T> we = w[e];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c + q < k) acc[q] = cfma_conj(V[(int64_t)(c + q) * ld + e], we, acc[q]);
    }
    double2 o[4];
    block_sum_t<T, 4>(acc, sh, o);
    if (threadIdx.x == 0)
      for (int q = 0; q < 4 && c + q < k; ++q) hh[c + q] = o[q];
    __syncthreads();
  }
}

// The whole fixed-count Jacobi-preconditioned GMRES of a small coarsest grid
// in one block: x = D^{-1} V y with V the Arnoldi basis of A D^{-1} and b.
// V holds (k+1) * n entries of scratch, z n entries.
template <int DIM, typename T>
__global__ void __launch_bounds__(1024) k_coarse_gmres_cta(Dims g, const C<T>* __restrict__ A, const C<T>* __restrict__ dinv,
                                                           const C<T>* b, C<T>* x, C<T>* V, C<T>* z, int k, ArnoldiState st) {
  __shared__ double2 sh[32 * 4];
  __shared__ double2 ha[kMaxKrylov + 1];
  __shared__ double2 hb[kMaxKrylov + 1];
  __shared__ C<T> cv[kMaxKrylov + 1];
  __shared__ double s_scale;
  if (resolve(g)) return;
  const int64_t n = g.N;
  const int64_t ld = g.total;   // basis stride
  shift_stencil(g, A);
  shift_nodes(g, dinv, b, x, V, z);
  st = arnoldi_at(st, blockIdx.y);
  // beta = |b|, V_0 = b / beta
  {
    C<T> s[1] = {czero<T>()};
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s[0] = cfma_conj(b[e], b[e], s[0]);
    double2 o[1];
    block_sum_t<T, 1>(s, sh, o);
    if (threadIdx.x == 0) {
      const double beta = sqrt(o[0].x);
      for (int i = 0; i <= st.m; ++i) st.g[i] = make_double2(0.0, 0.0);
      st.g[0] = make_double2(beta, 0.0);
      st.scal[kScalBeta] = beta;
      st.scal[kScalEst] = beta;
      st.iscal[kIScalStop] = beta > 0.0 ? -1 : 0;
      st.iscal[kIScalConv] = beta > 0.0 ? -1 : 0;
      s_scale = beta > 0.0 ? 1.0 / beta : 0.0;
    }
    __syncthreads();
    const T inv = (T)s_scale;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) V[e] = cscale(b[e], inv);
    __syncthreads();
  }
  for (int j = 0; j < k; ++j) {
    const C<T>* vj = V + (int64_t)j * ld;
    C<T>* w = V + (int64_t)(j + 1) * ld;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) z[e] = cmul(dinv[e], vj[e]);
    __syncthreads();
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      int i0, i1, i2;
      unravel(g, e, i0, i1, i2);
      w[e] = stencil_dot<DIM, T, true>(g, A, z, e, i0, i1, i2);   // z was written in this launch
    }
    __syncthreads();
    cta_dots<T>(V, ld, n, j + 1, w, ha, sh);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) cv[i] = mk<T>((T)(-ha[i].x), (T)(-ha[i].y));
    __syncthreads();
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      C<T> acc = w[e];
      for (int i = 0; i <= j; ++i) acc = cfma(V[(int64_t)i * ld + e], cv[i], acc);
      w[e] = acc;
    }
    __syncthreads();
    cta_dots<T>(V, ld, n, j + 1, w, hb, sh);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) cv[i] = mk<T>((T)(-hb[i].x), (T)(-hb[i].y));
    __syncthreads();
    C<T> s[1] = {czero<T>()};
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      C<T> acc = w[e];
      for (int i = 0; i <= j; ++i) acc = cfma(V[(int64_t)i * ld + e], cv[i], acc);
      w[e] = acc;
      s[0] = cfma_conj(acc, acc, s[0]);
    }
    double2 o[1];
    block_sum_t<T, 1>(s, sh, o);
    if (threadIdx.x == 0) {
      arnoldi_column_dev(st, j, ha, hb, o[0].x);
      const double hn = st.scal[kScalHn];
      s_scale = hn > 0.0 ? 1.0 / hn : 0.0;
    }
    __syncthreads();
    if (j + 1 < k) {
      const T inv = (T)s_scale;
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x) w[e] = cscale(w[e], inv);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) backsolve_dev(st, k);
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) cv[i] = mk<T>((T)st.y[i].x, (T)st.y[i].y);
  __syncthreads();
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    C<T> acc = czero<T>();
    for (int i = 0; i < k; ++i) acc = cfma(V[(int64_t)i * ld + e], cv[i], acc);
    x[e] = cmul(dinv[e], acc);
  }
}

static inline unsigned mr_blocks_c(const Dims& g) {
  const int64_t cap = g.mrcap > 0 ? g.mrcap : kMaxMrBlocks;
  const int64_t b = (g.N + 255) / 256;
  return (unsigned)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <typename T>
void launch_stencil_mr_apply(const Dims& g, const C<T>* A, const C<T>* z, const C<T>* r, C<T>* w, double2* partial,
                             unsigned* ticket, double2* alpha, cudaStream_t st) {
  const unsigned nb = mr_blocks_c(g);
  const dim3 grid(nb, g.B);
  if (g.dim == 2)
    count_launches(1), (g.B > 1 ? k_stencil_mr_apply<2, T, true> : k_stencil_mr_apply<2, T, false>)<<<grid, 256, 0, st>>>(
                           g, A, z, r, w, partial, ticket, alpha);
  else
    count_launches(1), (g.B > 1 ? k_stencil_mr_apply<3, T, true> : k_stencil_mr_apply<3, T, false>)<<<grid, 256, 0, st>>>(
                           g, A, z, r, w, partial, ticket, alpha);
}
template <typename T>
void launch_stencil_residual_dinv(const Dims& g, const C<T>* A, const C<T>* b, const C<T>* x, const C<T>* dinv, C<T>* r,
                                  C<T>* z, cudaStream_t st) {
  const dim3 grid(blocks_for(g.N, 256), g.B);
  if (g.dim == 2)
    count_launches(1), (g.B > 1 ? k_stencil_residual_dinv<2, T, true> : k_stencil_residual_dinv<2, T, false>)<<<grid, 256, 0, st>>>(
                           g, A, b, x, dinv, r, z);
  else
    count_launches(1), (g.B > 1 ? k_stencil_residual_dinv<3, T, true> : k_stencil_residual_dinv<3, T, false>)<<<grid, 256, 0, st>>>(
                           g, A, b, x, dinv, r, z);
}
template <typename T>
void launch_coarse_gmres_cta(const Dims& g, const C<T>* A, const C<T>* dinv, const C<T>* b, C<T>* x, C<T>* V, C<T>* z, int k,
                             const ArnoldiState& s, cudaStream_t st) {
  if (g.dim == 2) count_launches(1), k_coarse_gmres_cta<2, T><<<dim3(1, g.B), 1024, 0, st>>>(g, A, dinv, b, x, V, z, k, s);
  else count_launches(1), k_coarse_gmres_cta<3, T><<<dim3(1, g.B), 1024, 0, st>>>(g, A, dinv, b, x, V, z, k, s);
}

#define ADR_INSTANTIATE_COARSE2(T)                                                                                          \
  template void launch_stencil_mr_apply<T>(const Dims&, const C<T>*, const C<T>*, const C<T>*, C<T>*, double2*, unsigned*, double2*, cudaStream_t); \
  template void launch_stencil_residual_dinv<T>(const Dims&, const C<T>*, const C<T>*, const C<T>*, const C<T>*, C<T>*, C<T>*, cudaStream_t); \
  template void launch_coarse_gmres_cta<T>(const Dims&, const C<T>*, const C<T>*, const C<T>*, C<T>*, C<T>*, C<T>*, int, const ArnoldiState&, cudaStream_t);
ADR_INSTANTIATE_COARSE2(double)
ADR_INSTANTIATE_COARSE2(float)

}  // namespace adr
