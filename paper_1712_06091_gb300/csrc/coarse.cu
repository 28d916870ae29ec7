// Coarse-level kernels: operators stored as Galerkin stencils
// (Eq. coarseGridMatrix, A_c = P^T A P), bilinear / trilinear transfers
// (P and its transpose, Sec. 3.1), relaxation and residuals on those levels.
#include "adr_common.cuh"

namespace adr {

static inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// sum_p A[p][j] x[j + o_p] over the pattern points whose neighbour is inside.
template <int DIM, typename T>
__device__ __forceinline__ C<T> stencil_dot(const Dims& g, const C<T>* __restrict__ A, const C<T>* __restrict__ x,
                                            int64_t j, int i0, int i1, int i2) {
  constexpr int S = PatternSize<DIM>::value;
  C<T> acc = czero<T>();
#pragma unroll 9
  for (int p = 0; p < S; ++p) {
    const int8_t* o = pattern_offset<DIM>(p);
    const int k0 = i0 + o[0], k1 = i1 + o[1], k2 = i2 + o[2];
    const bool in = (unsigned)k0 < (unsigned)g.n[0] && (unsigned)k1 < (unsigned)g.n[1] &&
                    (DIM < 3 || (unsigned)k2 < (unsigned)g.n[2]);
    if (in) acc = cfma(A[(int64_t)p * g.N + j], x[j + o[0] + g.s1 * o[1] + g.s2 * o[2]], acc);
  }
  return acc;
}

template <int DIM, typename T>
__global__ void k_stencil_apply(Dims g, const C<T>* __restrict__ A, const C<T>* __restrict__ x, C<T>* __restrict__ y) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  int i0, i1, i2;
  unravel(g, j, i0, i1, i2);
  y[j] = stencil_dot<DIM, T>(g, A, x, j, i0, i1, i2);
}

template <int DIM, typename T>
__global__ void k_stencil_residual(Dims g, const C<T>* __restrict__ A, const C<T>* __restrict__ b,
                                   const C<T>* __restrict__ x, C<T>* __restrict__ r) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  int i0, i1, i2;
  unravel(g, j, i0, i1, i2);
  r[j] = csub(b[j], stencil_dot<DIM, T>(g, A, x, j, i0, i1, i2));
}

template <int DIM, typename T>
__global__ void k_stencil_jacobi(Dims g, const C<T>* __restrict__ A, const C<T>* __restrict__ dinv,
                                 const C<T>* __restrict__ b, const C<T>* __restrict__ xin, C<T>* __restrict__ xout, T w) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
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
  constexpr int S = PatternSize<DIM>::value;
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= gc.N) return;
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
          const C<T> wa = cscale(Af[(int64_t)p * gf.N + fj], wi);
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
  for (int p = 0; p < S; ++p) out[(int64_t)p * gc.N + I] = acc[p];
  dinv[I] = cinv(acc[(S - 1) / 2]);
}

// r_c = P^T r_f : weights 1 on the coincident node, 1/2 per axis offset by one.
template <int DIM, typename T>
__global__ void k_restrict(Dims gf, Dims gc, const C<T>* __restrict__ rf, C<T>* __restrict__ rc) {
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= gc.N) return;
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
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= gf.N) return;
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

template <typename T> void launch_stencil_apply(const Dims& g, const C<T>* A, const C<T>* x, C<T>* y, cudaStream_t st) {
  const int th = 256;
  if (g.dim == 2) count_launches(1), k_stencil_apply<2, T><<<blocks_for(g.N, th), th, 0, st>>>(g, A, x, y);
  else count_launches(1), k_stencil_apply<3, T><<<blocks_for(g.N, th), th, 0, st>>>(g, A, x, y);
}
template <typename T> void launch_stencil_residual(const Dims& g, const C<T>* A, const C<T>* b, const C<T>* x, C<T>* r, cudaStream_t st) {
  const int th = 256;
  if (g.dim == 2) count_launches(1), k_stencil_residual<2, T><<<blocks_for(g.N, th), th, 0, st>>>(g, A, b, x, r);
  else count_launches(1), k_stencil_residual<3, T><<<blocks_for(g.N, th), th, 0, st>>>(g, A, b, x, r);
}
template <typename T> void launch_stencil_jacobi(const Dims& g, const C<T>* A, const C<T>* dinv, const C<T>* b, const C<T>* xin, C<T>* xout, T w, cudaStream_t st) {
  const int th = 256;
  if (g.dim == 2) count_launches(1), k_stencil_jacobi<2, T><<<blocks_for(g.N, th), th, 0, st>>>(g, A, dinv, b, xin, xout, w);
  else count_launches(1), k_stencil_jacobi<3, T><<<blocks_for(g.N, th), th, 0, st>>>(g, A, dinv, b, xin, xout, w);
}
template <typename T> void launch_galerkin_stored(const Dims& gf, const Dims& gc, const C<T>* Af, C<T>* Ac, C<T>* dinv, cudaStream_t st) {
  const int th = 64;
  if (gf.dim == 2) count_launches(1), k_galerkin_stored<2, T><<<blocks_for(gc.N, th), th, 0, st>>>(gf, gc, Af, Ac, dinv);
  else count_launches(1), k_galerkin_stored<3, T><<<blocks_for(gc.N, th), th, 0, st>>>(gf, gc, Af, Ac, dinv);
}
template <typename T> void launch_restrict(const Dims& gf, const Dims& gc, const C<T>* rf, C<T>* rc, cudaStream_t st) {
  const int th = 256;
  if (gf.dim == 2) count_launches(1), k_restrict<2, T><<<blocks_for(gc.N, th), th, 0, st>>>(gf, gc, rf, rc);
  else count_launches(1), k_restrict<3, T><<<blocks_for(gc.N, th), th, 0, st>>>(gf, gc, rf, rc);
}
template <typename T> void launch_prolong_add(const Dims& gf, const Dims& gc, const C<T>* ec, C<T>* xf, cudaStream_t st) {
  const int th = 256;
  if (gf.dim == 2) count_launches(1), k_prolong_add<2, T><<<blocks_for(gf.N, th), th, 0, st>>>(gf, gc, ec, xf);
  else count_launches(1), k_prolong_add<3, T><<<blocks_for(gf.N, th), th, 0, st>>>(gf, gc, ec, xf);
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
