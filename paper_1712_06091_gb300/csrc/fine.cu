// Fine-level (matrix-free) kernels of the ADR amplitude operator.
//
// Coefficients: Eq. travel_time_coeff with tau = tau0 tau1, tau0 = |x - x0|
// (analytic derivatives), d tau1 by central differences (first-order
// one-sided on the boundary), d^2 tau1 by central differences (second-order
// one-sided on the boundary).  A plain tau (no factor tau0) takes the same
// differences of tau itself.  Rows: Eq. ADR with the Laplacian, the
// advection of Eqs. londDiff / londUpwindDiff / 1up, the averaging mass of
// Sec. 2.3 for the Delta-tau term, central advection next to the source
// (Sec. 2.2), the Neumann condition of Eq. BCADR (n.grad a = i w (n.grad tau) a)
// by ghost elimination, and the row of M^{-1} H M at the source (Eq. helmADR2).
#include "adr_common.cuh"
#include "coarse_stencil.cuh"
#include "reduce.cuh"
#include "df.cuh"

namespace adr {

static inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// ---------------------------------------------------------------------------
// Coefficients
// ---------------------------------------------------------------------------
__device__ __forceinline__ double tau1_at(const Dims& g, const double* tau1, int64_t j, int d, int k_from, int k_to) {
  const int64_t stride = d == 0 ? 1 : (d == 1 ? g.s1 : g.s2);
  return tau1[j + (int64_t)(k_to - k_from) * stride];
}

__global__ void k_coefficients(Dims g, FineInputs in, double* g0, double* g1, double* g2, double* t0, double* t1,
                               double* t2, double2* rho, double* tau) {
  if (resolve(g)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  double dx[3], r2 = 0.0;
  for (int d = 0; d < g.dim; ++d) {
    dx[d] = (ii[d] - in.src[d]) * in.h[d];
    r2 += dx[d] * dx[d];
  }
  const double r = sqrt(r2);
  const double ir = r > 0.0 ? 1.0 / r : 0.0;
  const double T1 = in.tau1[j];
  double* gout[3] = {g0, g1, g2};
  double* tout[3] = {t0, t1, t2};
  double grad2 = 0.0;
  for (int d = 0; d < g.dim; ++d) {
    const int k = ii[d], n = g.n[d];
    const double ih = in.ih[d], ih2 = ih * ih;   // reciprocals precomputed: no float64 division per node
    double d1, dd1;
    if (k == 0) {
      d1 = (tau1_at(g, in.tau1, j, d, k, 1) - tau1_at(g, in.tau1, j, d, k, 0)) * ih;
      dd1 = (2.0 * tau1_at(g, in.tau1, j, d, k, 0) - 5.0 * tau1_at(g, in.tau1, j, d, k, 1) +
             4.0 * tau1_at(g, in.tau1, j, d, k, 2) - tau1_at(g, in.tau1, j, d, k, 3)) * ih2;
    } else if (k == n - 1) {
      d1 = (tau1_at(g, in.tau1, j, d, k, n - 1) - tau1_at(g, in.tau1, j, d, k, n - 2)) * ih;
      dd1 = (2.0 * tau1_at(g, in.tau1, j, d, k, n - 1) - 5.0 * tau1_at(g, in.tau1, j, d, k, n - 2) +
             4.0 * tau1_at(g, in.tau1, j, d, k, n - 3) - tau1_at(g, in.tau1, j, d, k, n - 4)) * ih2;
    } else {
      d1 = (tau1_at(g, in.tau1, j, d, k, k + 1) - tau1_at(g, in.tau1, j, d, k, k - 1)) * (0.5 * ih);
      dd1 = (tau1_at(g, in.tau1, j, d, k, k + 1) - 2.0 * T1 + tau1_at(g, in.tau1, j, d, k, k - 1)) * ih2;
    }
    double d0 = 0.0, dd0 = 0.0;
    if (r > 0.0) {
      d0 = dx[d] * ir;
      dd0 = (1.0 - d0 * d0) * ir;
    }
    const double gd = in.plain ? d1 : __dadd_rn(__dmul_rn(r, d1), __dmul_rn(T1, d0));
    const double td = in.plain ? dd1 : T1 * dd0 + 2.0 * d0 * d1 + r * dd1;
    gout[d][j] = gd;
    tout[d][j] = td;
    grad2 += gd * gd;
  }
  const double k2 = in.kappa[j] * in.kappa[j];
  rho[j] = make_double2(in.omega * in.omega * (k2 - grad2), -in.omega * in.gamma[j] * k2);
  tau[j] = in.plain ? T1 : r * T1;
}

// Row of M^{-1} H M at the source (one thread).  H has its own Neumann ghost
// u_{b+s} = u_{b-s}, so an off-grid neighbour folds onto its mirror.
__global__ void k_source_row(Dims g, FineInputs in, const double* tau, double2* row) {
  if (resolve(g)) return;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = 0; k < kCross3; ++k) row[k] = make_double2(0.0, 0.0);
  const int64_t js = in.src[0] + g.s1 * in.src[1] + g.s2 * in.src[2];
  const double ts = tau[js];   // 0 for the factored travel time
  double cre = 0.0;
  for (int d = 0; d < g.dim; ++d) {
    const int64_t stride = d == 0 ? 1 : (d == 1 ? g.s1 : g.s2);
    const double ih2 = 1.0 / (in.h[d] * in.h[d]);
    for (int s = -1; s <= 1; s += 2) {
      int k = in.src[d] + s;
      int slot_s = s;  // slot that receives the coefficient
      if (k < 0 || k >= g.n[d]) { k = in.src[d] - s; slot_s = -s; }
      const double tn = tau[js + (int64_t)(k - in.src[d]) * stride];
      double sn, cs;
      sincos(in.omega * (ts - tn), &sn, &cs);
      const int slot = 1 + 4 * d + (slot_s < 0 ? 0 : 1);
      row[slot].x += cs * ih2;
      row[slot].y += sn * ih2;
      cre -= ih2;
    }
  }
  const double k2 = in.kappa[js] * in.kappa[js];
  row[0] = make_double2(cre + in.omega * in.omega * k2, -in.omega * in.gamma[js] * k2);
}

void launch_coefficients(const Dims& g, const FineInputs& in, double* const gd[3], double* const td[3], double2* rho,
                         double* tau, double2* src_row, cudaStream_t st) {
  const int th = 256;
  count_launches(1), k_coefficients<<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, in, gd[0], gd[1], gd[2], td[0], td[1], td[2], rho, tau);
  count_launches(1), k_source_row<<<1, 32, 0, st>>>(g, in, tau, src_row);
}

// Eq. shift: the mass term -i alpha w^2 kappa^2 joins the reaction coefficient
// (the diagonal of every row) and the diagonal of the source row.
__global__ void k_shift(Dims g, FineInputs in, double alpha, const double2* rho, const double2* srow, double2* rho_s,
                        double2* srow_s) {
  if (resolve(g)) return;
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  const double m = alpha * in.omega * in.omega;
  const double2 r = rho[j];
  rho_s[j] = make_double2(r.x, r.y - m * (in.kappa[j] * in.kappa[j]));
  if (j < kCross3) {
    double2 e = srow[j];
    if (j == 0) {
      const int64_t js = in.src[0] + g.s1 * in.src[1] + g.s2 * in.src[2];
      e.y -= m * (in.kappa[js] * in.kappa[js]);
    }
    srow_s[j] = e;
  }
}
void launch_shift(const Dims& g, const FineInputs& in, double alpha, const double2* rho, const double2* src_row,
                  double2* rho_s, double2* src_row_s, cudaStream_t st) {
  count_launches(1), k_shift<<<blocks_for(g.N, 256), 256, 0, st>>>(g, in, alpha, rho, src_row, rho_s, src_row_s);
}

__global__ void k_to_f32(const double* s, float* d, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) d[i] = (float)s[i];
}
void launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t st) {
  count_launches(1), k_to_f32<<<blocks_for(n, 256), 256, 0, st>>>(src, dst, n);
}

// ---------------------------------------------------------------------------
// The fine row
// ---------------------------------------------------------------------------
// Writes the row of node j (coordinates ii) in cross form into c[1 + 4*DIM].
template <int DIM, typename T>
__device__ __forceinline__ void fine_row(const Dims& g, const FineOp<T>& f, int64_t j, const int ii[3], C<T>* c) {
  // Problem blockIdx.y of a batch (g resolved): its coefficients start g.off
  // entries in, its FineDyn and source row are entry pb of theirs.
  const int pb = blockIdx.y;
  const int64_t jo = j + g.off;
  if (f.rows) {
    const C<T>* rows = f.rows + (int64_t)(1 + 4 * DIM) * g.off;
#pragma unroll
    for (int q = 0; q < 1 + 4 * DIM; ++q) c[q] = __ldg(rows + (int64_t)q * g.N + j);
    return;
  }
  const FineDyn* dyn = f.dyn + pb;
  if (j == dyn->src_index) {
    const C<T>* srow = f.src_row + (int64_t)pb * kCross3;
    c[0] = srow[0];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
#pragma unroll
      for (int q = 0; q < 4; ++q) c[1 + 4 * d + q] = srow[1 + 4 * d + q];
    }
    return;
  }
  if (f.packed) {
    // Packed row: entry 0/1 = centre (re, im); 2 + 4 d + q = imaginary part
    // of neighbour slot q of axis d.  The real parts of the neighbour entries
    // are the Laplacian's 1/h^2, doubled onto the inner neighbour on a face
    // (ghost elimination) and zero at the eliminated ghost and at +-2, the
    // same values the computed row holds.
    const T* pk = f.packed + (int64_t)(2 + 4 * DIM) * g.off + j;
    c[0] = mk<T>(__ldg(pk), __ldg(pk + g.N));
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const T ih2 = f.ih2[d];
      const int k = ii[d], n = g.n[d];
      const T re_m1 = k == 0 ? T(0) : (k == n - 1 ? ih2 + ih2 : ih2);
      const T re_p1 = k == n - 1 ? T(0) : (k == 0 ? ih2 + ih2 : ih2);
      c[1 + 4 * d + 0] = mk<T>(re_m1, __ldg(pk + (int64_t)(2 + 4 * d + 0) * g.N));
      c[1 + 4 * d + 1] = mk<T>(re_p1, __ldg(pk + (int64_t)(2 + 4 * d + 1) * g.N));
      c[1 + 4 * d + 2] = mk<T>(T(0), __ldg(pk + (int64_t)(2 + 4 * d + 2) * g.N));
      c[1 + 4 * d + 3] = mk<T>(T(0), __ldg(pk + (int64_t)(2 + 4 * d + 3) * g.N));
    }
    return;
  }
  bool near = true;
#pragma unroll
  for (int d = 0; d < DIM; ++d) near = near && (abs(ii[d] - dyn->src[d]) <= f.near);
  const C<T> rho = f.rho[jo];
  const T omega = (T)dyn->omega;
  T cre = rho.x, cim = rho.y;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const T gd = f.g[d][jo];
    const T td = f.t[d][jo];
    const T h = f.h[d];
    const T ih2 = f.ih2[d];
    const int k = ii[d], n = g.n[d];
    T re_m1 = ih2, re_p1 = ih2;
    T im_m1 = T(-0.5) * omega * td, im_p1 = im_m1;
    cre -= T(2) * ih2;
    // advection difference weights at offsets -2..+2
    T wm2 = 0, wm1 = 0, w0 = 0, wp1 = 0, wp2 = 0;
    const T half_ih = f.hih[d];
    if (near || gd == T(0) || (f.central && k > 0 && k < n - 1)) {
      wp1 = half_ih; wm1 = -half_ih;
    } else {
      const T a2 = f.central ? T(1) : f.w2;
      const T a1 = f.central ? T(0) : f.w1;
      if (a2 != T(0)) {
        if (gd > T(0)) {
          if (k >= 2) { w0 += a2 * T(3) * half_ih; wm1 -= a2 * T(4) * half_ih; wm2 += a2 * half_ih; }
          else { wp1 += a2 * half_ih; wm1 -= a2 * half_ih; }
        } else {
          if (k <= n - 3) { w0 -= a2 * T(3) * half_ih; wp1 += a2 * T(4) * half_ih; wp2 -= a2 * half_ih; }
          else { wp1 += a2 * half_ih; wm1 -= a2 * half_ih; }
        }
      }
      if (a1 != T(0)) {
        const T ih = f.ih[d];
        if (gd > T(0)) {
          if (k >= 1) { w0 += a1 * ih; wm1 -= a1 * ih; }
          else { wp1 += a1 * half_ih; wm1 -= a1 * half_ih; }
        } else {
          if (k <= n - 2) { w0 -= a1 * ih; wp1 += a1 * ih; }
          else { wp1 += a1 * half_ih; wm1 -= a1 * half_ih; }
        }
      }
    }
    const T adv = T(-2) * omega * gd;  // -2 i w (d_d tau) D_d: imaginary factor
    im_m1 += adv * wm1;
    im_p1 += adv * wp1;
    cim += adv * w0;
    const T im_m2 = adv * wm2, im_p2 = adv * wp2;
    // Neumann ghost (Eq. BCADR read with the factor a): a_{b+s} = a_{b-s} + s 2 h i w g a_b
    if (k == 0) {
      const T fac = T(-2) * h * omega * gd;  // ghost adds (i fac) a_b per unit coefficient
      re_p1 += re_m1; im_p1 += im_m1;
      cre -= im_m1 * fac; cim += re_m1 * fac;
      re_m1 = 0; im_m1 = 0;
    }
    if (k == n - 1) {
      const T fac = T(2) * h * omega * gd;
      re_m1 += re_p1; im_m1 += im_p1;
      cre -= im_p1 * fac; cim += re_p1 * fac;
      re_p1 = 0; im_p1 = 0;
    }
    c[1 + 4 * d + 0] = mk<T>(re_m1, im_m1);
    c[1 + 4 * d + 1] = mk<T>(re_p1, im_p1);
    c[1 + 4 * d + 2] = mk<T>(T(0), im_m2);
    c[1 + 4 * d + 3] = mk<T>(T(0), im_p2);
  }
  c[0] = mk<T>(cre, cim);
}

template <int DIM> __device__ __forceinline__ int64_t axis_stride(const Dims& g, int d) {
  return d == 0 ? 1 : (d == 1 ? g.s1 : g.s2);
}

// sum_k c_k x_{j + o_k} over the cross entries.  Entries whose neighbour is
// off the grid are exactly zero (ghosts are eliminated into the row), so the
// load is redirected to node j instead of branching; all loads issue together.
template <int DIM, typename T>
__device__ __forceinline__ C<T> cross_dot(const Dims& g, const C<T>* c, const int ii[3], int64_t j, const C<T>* x) {
  C<T> acc0 = cmul(c[0], __ldg(x + j)), acc1 = czero<T>();
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int64_t s = axis_stride<DIM>(g, d);
    const int k = ii[d], n = g.n[d];
    const int64_t jm1 = k >= 1 ? j - s : j, jp1 = k <= n - 2 ? j + s : j;
    const int64_t jm2 = k >= 2 ? j - 2 * s : j, jp2 = k <= n - 3 ? j + 2 * s : j;
    acc1 = cfma(c[1 + 4 * d + 0], __ldg(x + jm1), acc1);
    acc0 = cfma(c[1 + 4 * d + 1], __ldg(x + jp1), acc0);
    acc1 = cfma(c[1 + 4 * d + 2], __ldg(x + jm2), acc1);
    acc0 = cfma(c[1 + 4 * d + 3], __ldg(x + jp2), acc0);
  }
  return cadd(acc0, acc1);
}

template <int DIM, typename T>
__global__ void k_fine_apply(Dims g, FineOp<T> f, const C<T>* __restrict__ x, C<T>* __restrict__ y) {
  if (resolve(g, f)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  shift_nodes(g, x, y);
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  C<T> c[1 + 4 * DIM];
  fine_row<DIM, T>(g, f, j, ii, c);
  y[j] = cross_dot<DIM, T>(g, c, ii, j, x);
}

template <int DIM, typename T>
__global__ void k_fine_residual(Dims g, FineOp<T> f, const C<T>* __restrict__ b, const C<T>* __restrict__ x,
                                C<T>* __restrict__ r) {
  if (resolve(g, f)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  shift_nodes(g, b, x, r);
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  C<T> c[1 + 4 * DIM];
  fine_row<DIM, T>(g, f, j, ii, c);
  r[j] = csub(b[j], cross_dot<DIM, T>(g, c, ii, j, x));
}

template <int DIM, typename T>
__global__ void k_fine_jacobi(Dims g, FineOp<T> f, const C<T>* __restrict__ b, const C<T>* __restrict__ xin,
                              C<T>* __restrict__ xout, T w) {
  if (resolve(g, f)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  shift_nodes(g, b, xout);
  shift_nodes_opt(g, xin);
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  C<T> c[1 + 4 * DIM];
  fine_row<DIM, T>(g, f, j, ii, c);
  const C<T> dinv = cinv(c[0]);
  if (xin == nullptr) {
    xout[j] = cscale(cmul(dinv, b[j]), w);
  } else {
    const C<T> r = csub(b[j], cross_dot<DIM, T>(g, c, ii, j, xin));
    xout[j] = cadd(xin[j], cscale(cmul(dinv, r), w));
  }
}

template <int DIM, typename T>
__global__ void k_fine_dinv(Dims g, FineOp<T> f, const C<T>* __restrict__ v, C<T>* __restrict__ z) {
  if (resolve(g, f)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  shift_nodes(g, z);
  shift_nodes_opt(g, v);
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  C<T> c[1 + 4 * DIM];
  fine_row<DIM, T>(g, f, j, ii, c);
  const C<T> dinv = cinv(c[0]);
  z[j] = v ? cmul(dinv, v[j]) : dinv;
}

// ---------------------------------------------------------------------------
// Galerkin product P^T A P from the fine operator (Eq. coarseGridMatrix).
// One thread per coarse node I accumulates the point-major stencil row
//   A_c[I, J] = sum_i sum_k P[i, I] A[i, k] P[k, J]
// over the fine nodes i next to 2I and the entries k of their rows.
// ---------------------------------------------------------------------------
template <int DIM, typename T, typename RowFn>
__device__ __forceinline__ void galerkin_accumulate(const Dims& gf, const Dims& gc, int64_t I, const int Ii[3],
                                                    RowFn row_of, C<T>* acc) {
  constexpr int S = PatternSize<DIM>::value;
  for (int p = 0; p < S; ++p) acc[p] = czero<T>();
  const int dlo2 = DIM > 2 ? -1 : 0, dhi2 = DIM > 2 ? 1 : 0;
  for (int e2 = dlo2; e2 <= dhi2; ++e2)
    for (int e1 = -1; e1 <= 1; ++e1)
      for (int e0 = -1; e0 <= 1; ++e0) {
        int fi[3] = {2 * Ii[0] + e0, 2 * Ii[1] + e1, DIM > 2 ? 2 * Ii[2] + e2 : 0};
        bool ok = true;
        for (int d = 0; d < DIM; ++d) ok = ok && fi[d] >= 0 && fi[d] < gf.n[d];
        if (!ok) continue;
        const T wi = (e0 ? T(0.5) : T(1)) * (e1 ? T(0.5) : T(1)) * (e2 ? T(0.5) : T(1));
        const int64_t fj = fi[0] + gf.s1 * fi[1] + gf.s2 * fi[2];
        row_of(fj, fi, [&](int o0, int o1, int o2, C<T> a) {
          const int k[3] = {fi[0] + o0, fi[1] + o1, fi[2] + o2};
          const C<T> wa = cscale(a, wi);
          // parents of k along each axis
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
                const T pwt = pw[0][q0] * pw[1][q1] * pw[2][q2];
                acc[s] = cadd(acc[s], cscale(wa, pwt));
              }
        });
      }
}

template <int DIM, typename T>
__global__ void k_galerkin_fine(Dims gf, Dims gc, FineOp<T> f, C<T>* __restrict__ out, C<T>* __restrict__ dinv) {
  if (resolve(gf, f)) return;
  resolve(gc);
  constexpr int S = PatternSize<DIM>::value;
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= gc.N) return;
  shift_stencil(gc, out);
  shift_nodes(gc, dinv);
  int Ii[3];
  unravel(gc, I, Ii[0], Ii[1], Ii[2]);
  C<T> acc[S];
  auto row_of = [&](int64_t fj, const int fi[3], auto emit) {
    C<T> c[1 + 4 * DIM];
    fine_row<DIM, T>(gf, f, fj, fi, c);
    emit(0, 0, 0, c[0]);
    for (int d = 0; d < DIM; ++d) {
      const int k = fi[d], n = gf.n[d];
      int o[3] = {0, 0, 0};
      if (k >= 1) { o[d] = -1; emit(o[0], o[1], o[2], c[1 + 4 * d + 0]); }
      if (k <= n - 2) { o[d] = 1; emit(o[0], o[1], o[2], c[1 + 4 * d + 1]); }
      if (k >= 2) { o[d] = -2; emit(o[0], o[1], o[2], c[1 + 4 * d + 2]); }
      if (k <= n - 3) { o[d] = 2; emit(o[0], o[1], o[2], c[1 + 4 * d + 3]); }
    }
  };
  galerkin_accumulate<DIM, T>(gf, gc, I, Ii, row_of, acc);
  for (int p = 0; p < S; ++p) stencil_put<DIM, T>(out, p, I, acc[p]);
  dinv[I] = cinv(acc[(S - 1) / 2]);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename T> void launch_fine_apply(const Dims& g, const FineOp<T>& f, const C<T>* x, C<T>* y, cudaStream_t st) {
  const int th = 256;
  if (g.dim == 2) count_launches(1), k_fine_apply<2, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, f, x, y);
  else count_launches(1), k_fine_apply<3, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, f, x, y);
}
template <typename T> void launch_fine_residual(const Dims& g, const FineOp<T>& f, const C<T>* b, const C<T>* x, C<T>* r, cudaStream_t st) {
  const int th = 256;
  if (g.dim == 2) count_launches(1), k_fine_residual<2, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, f, b, x, r);
  else count_launches(1), k_fine_residual<3, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, f, b, x, r);
}
template <typename T> void launch_fine_jacobi(const Dims& g, const FineOp<T>& f, const C<T>* b, const C<T>* xin, C<T>* xout, T w, cudaStream_t st) {
  const int th = 256;
  if (g.dim == 2) count_launches(1), k_fine_jacobi<2, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, f, b, xin, xout, w);
  else count_launches(1), k_fine_jacobi<3, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, f, b, xin, xout, w);
}
template <typename T> void launch_fine_dinv(const Dims& g, const FineOp<T>& f, const C<T>* v, C<T>* z, cudaStream_t st) {
  const int th = 256;
  if (g.dim == 2) count_launches(1), k_fine_dinv<2, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, f, v, z);
  else count_launches(1), k_fine_dinv<3, T><<<dim3(blocks_for(g.N, th), g.B), th, 0, st>>>(g, f, v, z);
}
template <typename T> void launch_galerkin_fine(const Dims& gf, const Dims& gc, const FineOp<T>& f, C<T>* stencil, C<T>* dinv, cudaStream_t st) {
  const int th = 64;
  if (gf.dim == 2) count_launches(1), k_galerkin_fine<2, T><<<dim3(blocks_for(gc.N, th), gf.B), th, 0, st>>>(gf, gc, f, stencil, dinv);
  else count_launches(1), k_galerkin_fine<3, T><<<dim3(blocks_for(gc.N, th), gf.B), th, 0, st>>>(gf, gc, f, stencil, dinv);
}

#define ADR_INSTANTIATE_FINE(T)                                                                                     \
  template void launch_fine_apply<T>(const Dims&, const FineOp<T>&, const C<T>*, C<T>*, cudaStream_t);               \
  template void launch_fine_residual<T>(const Dims&, const FineOp<T>&, const C<T>*, const C<T>*, C<T>*, cudaStream_t); \
  template void launch_fine_jacobi<T>(const Dims&, const FineOp<T>&, const C<T>*, const C<T>*, C<T>*, T, cudaStream_t); \
  template void launch_fine_dinv<T>(const Dims&, const FineOp<T>&, const C<T>*, C<T>*, cudaStream_t);                \
  template void launch_galerkin_fine<T>(const Dims&, const Dims&, const FineOp<T>&, C<T>*, C<T>*, cudaStream_t);
ADR_INSTANTIATE_FINE(double)
ADR_INSTANTIATE_FINE(float)

// ---------------------------------------------------------------------------
// Point source, reconstruction, coefficient export
// ---------------------------------------------------------------------------
// value = 1 / prod(h) (per-problem grids: from the problem's own spacing)
__global__ void k_rhs_point(Dims g, double2* q, const FineDyn* dyn, double value) {
  if (resolve(g)) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  shift_nodes(g, q);
  if (g.pd) {
    double vol = 1.0;
    for (int d = 0; d < g.dim; ++d) vol *= g.pd[blockIdx.y].h[d];
    value = 1.0 / vol;
  }
  q[i] = make_double2(i == dyn[blockIdx.y].src_index ? value : 0.0, 0.0);
}
void launch_rhs_point(const Dims& g, double2* q, const FineDyn* dyn, double value, cudaStream_t st) {
  count_launches(1), k_rhs_point<<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, q, dyn, value);
}

__global__ void k_reconstruct(Dims g, const double2* a, const double* tau, const FineDyn* dyn, double2* u) {
  if (resolve(g)) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  shift_nodes(g, a, tau, u);
  double s, c;
  sincos(-dyn[blockIdx.y].omega * tau[i], &s, &c);
  u[i] = cmul(a[i], make_double2(c, s));
}
void launch_reconstruct(const Dims& g, const double2* a, const double* tau, const FineDyn* dyn, double2* u, cudaStream_t st) {
  count_launches(1), k_reconstruct<<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, a, tau, dyn, u);
}

__global__ void k_phase(Dims g, const double* tau, const FineDyn* dyn, double2* phase) {
  if (resolve(g)) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  shift_nodes(g, tau, phase);
  double s, c;
  sincos(-dyn[blockIdx.y].omega * tau[i], &s, &c);
  phase[i] = make_double2(c, s);
}
void launch_phase(const Dims& g, const double* tau, const FineDyn* dyn, double2* phase, cudaStream_t st) {
  count_launches(1), k_phase<<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, tau, dyn, phase);
}

template <typename Ts, typename Td>
__global__ void k_phase_cast(const C<Ts>* __restrict__ src, const double2* __restrict__ phase, bool conj,
                             C<Td>* __restrict__ dst, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const C<Ts> v = src[i];
  double2 m = phase[i];
  if (conj) m.y = -m.y;
  const double2 r = cmul(make_double2((double)v.x, (double)v.y), m);
  dst[i] = mk<Td>((Td)r.x, (Td)r.y);
}
template <typename Ts, typename Td>
void launch_phase_cast(const C<Ts>* src, const double2* phase, bool conj, C<Td>* dst, int64_t n, cudaStream_t st) {
  count_launches(1), k_phase_cast<Ts, Td><<<blocks_for(n, 256), 256, 0, st>>>(src, phase, conj, dst, n);
}
template void launch_phase_cast<double, double>(const double2*, const double2*, bool, double2*, int64_t, cudaStream_t);
template void launch_phase_cast<double, float>(const double2*, const double2*, bool, float2*, int64_t, cudaStream_t);
template void launch_phase_cast<float, double>(const float2*, const double2*, bool, double2*, int64_t, cudaStream_t);

__global__ void k_pack(Dims g, const double* g0, const double* g1, const double* g2, const double* t0, const double* t1,
                       const double* t2, const double2* rho, const double* tau, double* out) {
  if (resolve(g)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  shift_nodes(g, g0, t0, rho, tau);
  shift_nodes_opt(g, g1, g2, t1, t2);
  shift_scaled(g, 2 * g.dim + 3, out);
  const double* gs[3] = {g0, g1, g2};
  const double* ts[3] = {t0, t1, t2};
  int k = 0;
  for (int d = 0; d < g.dim; ++d) out[(k++) * g.N + j] = gs[d][j];
  for (int d = 0; d < g.dim; ++d) out[(k++) * g.N + j] = ts[d][j];
  out[(k++) * g.N + j] = rho[j].x;
  out[(k++) * g.N + j] = rho[j].y;
  out[(k++) * g.N + j] = tau[j];
}
void launch_pack_coefficients(const Dims& g, const double* const gd[3], const double* const td[3], const double2* rho,
                              const double* tau, double* out, cudaStream_t st) {
  count_launches(1), k_pack<<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, gd[0], gd[1], gd[2], td[0], td[1], td[2], rho, tau, out);
}

}  // namespace adr

// ===========================================================================
// Fused relaxation kernels on the fine level
// ===========================================================================
namespace adr {

// w = A z and, over all nodes, alpha = (w^H r) / (w^H w) (the one-step
// minimal-residual weight), computed by the last block to finish.
// BT: 0 one problem (no per-problem resolution: its offsets are zero), 1 a
// batch on one grid, 2 a batch of per-problem grids (the spacing is the
// problem's own); the narrower instantiations keep this register-capped
// kernel's spills at their level.
template <int DIM, typename T, int BT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) k_fine_mr_apply(Dims g, FineOp<T> f, const C<T>* __restrict__ z,
                                                       const C<T>* __restrict__ r, C<T>* __restrict__ w,
                                                       double2* partial, unsigned* ticket, double2* alpha) {
  if (BT == 1 && resolve_uniform(g)) return;
  if (BT == 2 && resolve(g, f)) return;
  __shared__ double2 sh[32 * 2];
  if (BT) shift_nodes(g, z, r, w);
  C<T> s[2] = {czero<T>(), czero<T>()};
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < g.N; j += (int64_t)gridDim.x * blockDim.x) {
    int ii[3];
    unravel(g, j, ii[0], ii[1], ii[2]);
    C<T> c[1 + 4 * DIM];
    fine_row<DIM, T>(g, f, j, ii, c);
    const C<T> wj = cross_dot<DIM, T>(g, c, ii, j, z);
    w[j] = wj;
    s[0] = cfma_conj(wj, r[j], s[0]);
    s[1] = cfma_conj(wj, wj, s[1]);
  }
  batch_shift(kPartialStride, partial);
  batch_shift(1, ticket, alpha);
  double2 mine[2], tot[2];
  block_sum_t<T, 2>(s, sh, mine);
  if (last_block_total<2>(mine, partial, ticket, tot, sh) && threadIdx.x == 0) {
    const double den = tot[1].x;
    *alpha = den > 0.0 ? make_double2(tot[0].x / den, tot[0].y / den) : make_double2(0.0, 0.0);
  }
}

// r = b - A x ; z = D^{-1} r
template <int DIM, typename T, int BT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) k_fine_residual_dinv(Dims g, FineOp<T> f, const C<T>* __restrict__ b, const C<T>* __restrict__ x,
                                     const C<T>* __restrict__ dinv, C<T>* __restrict__ r, C<T>* __restrict__ z) {
  if (BT == 1 && resolve_uniform(g)) return;
  if (BT == 2 && resolve(g, f)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  if (BT) shift_nodes(g, b, x, dinv, r, z);
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  C<T> c[1 + 4 * DIM];
  fine_row<DIM, T>(g, f, j, ii, c);
  const C<T> rj = csub(b[j], cross_dot<DIM, T>(g, c, ii, j, x));
  r[j] = rj;
  z[j] = cmul(dinv[j], rj);
}

__global__ void k_set_dyn(FineDyn* d, FineDyn v) {
  if (threadIdx.x == 0) *d = v;
}
void launch_set_dyn(FineDyn* d, const FineDyn& v, cudaStream_t st) { count_launches(1), k_set_dyn<<<1, 32, 0, st>>>(d, v); }

static inline unsigned mr_blocks(const Dims& g) {
  const int64_t cap = g.mrcap > 0 ? g.mrcap : kMaxMrBlocks;
  const int64_t b = (g.N + 255) / 256;
  return (unsigned)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <typename T>
void launch_fine_mr_apply(const Dims& g, const FineOp<T>& f, const C<T>* z, const C<T>* r, C<T>* w, double2* partial,
                          unsigned* ticket, double2* alpha, cudaStream_t st) {
  const unsigned nb = mr_blocks(g);
  const int bt = g.pd ? 2 : (g.B > 1 ? 1 : 0);
  auto kern = g.dim == 2 ? (bt == 2 ? k_fine_mr_apply<2, T, 2> : bt ? k_fine_mr_apply<2, T, 1> : k_fine_mr_apply<2, T, 0>)
                         : (bt == 2 ? k_fine_mr_apply<3, T, 2> : bt ? k_fine_mr_apply<3, T, 1> : k_fine_mr_apply<3, T, 0>);
  count_launches(1), kern<<<dim3(nb, g.B), 256, 0, st>>>(g, f, z, r, w, partial, ticket, alpha);
}
template <typename T>
void launch_fine_residual_dinv(const Dims& g, const FineOp<T>& f, const C<T>* b, const C<T>* x, const C<T>* dinv, C<T>* r,
                               C<T>* z, cudaStream_t st) {
  const int bt = g.pd ? 2 : (g.B > 1 ? 1 : 0);
  auto kern = g.dim == 2 ? (bt == 2 ? k_fine_residual_dinv<2, T, 2> : bt ? k_fine_residual_dinv<2, T, 1>
                                                                          : k_fine_residual_dinv<2, T, 0>)
                         : (bt == 2 ? k_fine_residual_dinv<3, T, 2> : bt ? k_fine_residual_dinv<3, T, 1>
                                                                          : k_fine_residual_dinv<3, T, 0>);
  count_launches(1), kern<<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, f, b, x, dinv, r, z);
}
template void launch_fine_mr_apply<double>(const Dims&, const FineOp<double>&, const double2*, const double2*, double2*,
                                           double2*, unsigned*, double2*, cudaStream_t);
template void launch_fine_mr_apply<float>(const Dims&, const FineOp<float>&, const float2*, const float2*, float2*,
                                          double2*, unsigned*, double2*, cudaStream_t);
template void launch_fine_residual_dinv<double>(const Dims&, const FineOp<double>&, const double2*, const double2*,
                                                const double2*, double2*, double2*, cudaStream_t);
template void launch_fine_residual_dinv<float>(const Dims&, const FineOp<float>&, const float2*, const float2*,
                                               const float2*, float2*, float2*, cudaStream_t);

}  // namespace adr

// ===========================================================================
// Stored rows of a finest-grid operator, written once per setup: full complex
// cross rows (the adjoint operators' rows and their conjugate transpose, the
// rescaled cycle operator M A M^{-1}) and the packed rows (the cycle's
// operator and the float64 outer operator), so that no apply rebuilds a row.
// ===========================================================================
namespace adr {

template <int DIM, typename T>
__global__ void k_fine_store_rows(Dims g, FineOp<T> f, C<T>* __restrict__ rows) {
  if (resolve(g, f)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  shift_scaled(g, 1 + 4 * DIM, rows);
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  C<T> c[1 + 4 * DIM];
  fine_row<DIM, T>(g, f, j, ii, c);
#pragma unroll
  for (int q = 0; q < 1 + 4 * DIM; ++q) rows[(int64_t)q * g.N + j] = c[q];
}

// The packed form of the rows (see fine_row), built from the computed rows.
template <int DIM, typename T>
__global__ void k_fine_pack(Dims g, FineOp<T> f, T* __restrict__ packed) {
  if (resolve(g, f)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  f.packed = nullptr;
  shift_scaled(g, 2 + 4 * DIM, packed);
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  C<T> c[1 + 4 * DIM];
  fine_row<DIM, T>(g, f, j, ii, c);
  packed[j] = c[0].x;
  packed[g.N + j] = c[0].y;
#pragma unroll
  for (int q = 0; q < 4 * DIM; ++q) packed[(int64_t)(2 + q) * g.N + j] = c[1 + q].y;
}
template <typename T> void launch_fine_pack(const Dims& g, const FineOp<T>& f, T* packed, cudaStream_t st) {
  if (g.dim == 2) count_launches(1), k_fine_pack<2, T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, f, packed);
  else count_launches(1), k_fine_pack<3, T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, f, packed);
}
template void launch_fine_pack<double>(const Dims&, const FineOp<double>&, double*, cudaStream_t);
template void launch_fine_pack<float>(const Dims&, const FineOp<float>&, float*, cudaStream_t);

template <int DIM, typename T>
__device__ __forceinline__ C<T> rows_dot(const Dims& g, const C<T>* __restrict__ rows, int64_t j, const C<T>* __restrict__ x) {
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  C<T> c[1 + 4 * DIM];
#pragma unroll
  for (int q = 0; q < 1 + 4 * DIM; ++q) c[q] = __ldg(rows + (int64_t)q * g.N + j);
  return cross_dot<DIM, T>(g, c, ii, j, x);
}

template <int DIM, typename T>
__global__ void k_rows_apply(Dims g, const C<T>* __restrict__ rows, const C<T>* __restrict__ x, C<T>* __restrict__ y) {
  if (resolve(g)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  shift_scaled(g, 1 + 4 * DIM, rows);
  shift_nodes(g, x, y);
  y[j] = rows_dot<DIM, T>(g, rows, j, x);
}

template <int DIM, typename T>
__global__ void k_rows_residual(Dims g, const C<T>* __restrict__ rows, const C<T>* __restrict__ b,
                                const C<T>* __restrict__ x, C<T>* __restrict__ r) {
  if (resolve(g)) return;
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  shift_scaled(g, 1 + 4 * DIM, rows);
  shift_nodes(g, b, x, r);
  r[j] = csub(b[j], rows_dot<DIM, T>(g, rows, j, x));
}

// The outer iteration's float64 operator from packed rows (k_fine_pack: the
// centre and the imaginary parts of the neighbour entries, 14 reals per node
// in 3D).  The real parts of the neighbour entries are the Laplacian's 1/h^2
// (doubled on a face, zero at +-2), rebuilt from the node's position, so each
// neighbour costs a real scaling plus an imaginary one instead of a full
// complex product: 42 float64 operations per node in 3D against 54 for stored
// complex rows, and 112 bytes of row data against 208.  The float64 rate
// bounds this kernel, not memory.  The source node keeps its full row.
template <int DIM>
__device__ __forceinline__ double2 packed_dot(const Dims& g, const FineOp<double>& f, int64_t j,
                                              const double2* __restrict__ x) {
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  if (j == f.dyn[blockIdx.y].src_index) {
    double2 c[1 + 4 * DIM];
    fine_row<DIM, double>(g, f, j, ii, c);   // the source row (Eq. helmADR2)
    return cross_dot<DIM, double>(g, c, ii, j, x);
  }
  const double* pk = f.packed + (int64_t)(2 + 4 * DIM) * g.off + j;
  const double2 xj = __ldg(x + j);
  const double cr = __ldg(pk), ci = __ldg(pk + g.N);
  double ar = cr * xj.x, ai = cr * xj.y;
  ar = fma(-ci, xj.y, ar);
  ai = fma(ci, xj.x, ai);
  double br = 0.0, bi = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int64_t s = axis_stride<DIM>(g, d);
    const int k = ii[d], n = g.n[d];
    const int64_t jm1 = k >= 1 ? j - s : j, jp1 = k <= n - 2 ? j + s : j;
    const int64_t jm2 = k >= 2 ? j - 2 * s : j, jp2 = k <= n - 3 ? j + 2 * s : j;
    const double ih2 = f.ih2[d];
    const double re_m1 = k == 0 ? 0.0 : (k == n - 1 ? ih2 + ih2 : ih2);
    const double re_p1 = k == n - 1 ? 0.0 : (k == 0 ? ih2 + ih2 : ih2);
    const double2 xm1 = __ldg(x + jm1), xp1 = __ldg(x + jp1), xm2 = __ldg(x + jm2), xp2 = __ldg(x + jp2);
    const double bm1 = __ldg(pk + (int64_t)(2 + 4 * d + 0) * g.N), bp1 = __ldg(pk + (int64_t)(2 + 4 * d + 1) * g.N);
    const double bm2 = __ldg(pk + (int64_t)(2 + 4 * d + 2) * g.N), bp2 = __ldg(pk + (int64_t)(2 + 4 * d + 3) * g.N);
    ar = fma(re_m1, xm1.x, ar);
    ai = fma(re_m1, xm1.y, ai);
    br = fma(re_p1, xp1.x, br);
    bi = fma(re_p1, xp1.y, bi);
    ar = fma(-bm1, xm1.y, ar);
    ai = fma(bm1, xm1.x, ai);
    br = fma(-bp1, xp1.y, br);
    bi = fma(bp1, xp1.x, bi);
    ar = fma(-bm2, xm2.y, ar);
    ai = fma(bm2, xm2.x, ai);
    br = fma(-bp2, xp2.y, br);
    bi = fma(bp2, xp2.x, bi);
  }
  return make_double2(ar + br, ai + bi);
}

// BT as for k_fine_mr_apply: 0 one problem, 1 one grid, 2 per-problem grids.
template <int DIM, int BT>
__global__ void __launch_bounds__(256) k_packed_apply(Dims g, FineOp<double> f, const double2* __restrict__ x,
                                                      double2* __restrict__ y) {
  if (BT == 1 && resolve_uniform(g)) return;
  if (BT == 2 && resolve(g, f)) return;
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  if (BT) shift_nodes(g, x, y);
  y[j] = packed_dot<DIM>(g, f, j, x);
}

template <int DIM, int BT>
__global__ void __launch_bounds__(256) k_packed_residual(Dims g, FineOp<double> f, const double2* __restrict__ b,
                                                         const double2* __restrict__ x, double2* __restrict__ r) {
  if (BT == 1 && resolve_uniform(g)) return;
  if (BT == 2 && resolve(g, f)) return;
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  if (BT) shift_nodes(g, b, x, r);
  r[j] = csub(b[j], packed_dot<DIM>(g, f, j, x));
}

void launch_packed_apply(const Dims& g, const FineOp<double>& f, const double2* x, double2* y, cudaStream_t st) {
  const int bt = g.pd ? 2 : (g.B > 1 ? 1 : 0);
  auto kern = g.dim == 2 ? (bt == 2 ? k_packed_apply<2, 2> : bt ? k_packed_apply<2, 1> : k_packed_apply<2, 0>)
                         : (bt == 2 ? k_packed_apply<3, 2> : bt ? k_packed_apply<3, 1> : k_packed_apply<3, 0>);
  count_launches(1), kern<<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, f, x, y);
}
void launch_packed_residual(const Dims& g, const FineOp<double>& f, const double2* b, const double2* x, double2* r,
                            cudaStream_t st) {
  const int bt = g.pd ? 2 : (g.B > 1 ? 1 : 0);
  auto kern = g.dim == 2 ? (bt == 2 ? k_packed_residual<2, 2> : bt ? k_packed_residual<2, 1> : k_packed_residual<2, 0>)
                         : (bt == 2 ? k_packed_residual<3, 2> : bt ? k_packed_residual<3, 1> : k_packed_residual<3, 0>);
  count_launches(1), kern<<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, f, b, x, r);
}

// ---------------------------------------------------------------------------
// The outer float64 operator applied to a vector whose entries are float32
// values (the float32 cycle's output z_j), in double-float arithmetic.
//
// The float64 pipe of this GPU is far slower than the float32 one, and every
// product of a float64 coefficient c with a float32 x is recovered exactly by
// float32 error-free transformations: c = c_hi + c_lo (float32 pair, split at
// setup, |c - c_hi - c_lo| <= 2^-48 |c|), c_hi x = p + e exactly (the FMA
// two-product: p = fl(c_hi x), e = fma(c_hi, x, -p)), and the sums of the p
// are kept exactly as (s, t) by Knuth's two-sum while the small terms
// e + c_lo x gather in a float32 tail.  The row sum is then good to about
// 2^-46 of its largest term (float64: 2^-53), within rounding of the float64
// kernel for the outer Krylov iteration, which recomputes its residual
// explicitly in float64 at every restart.  The row sums are stored as
// normalised double-float planes (the next basis vector of the double-float
// outer iteration, krylov_df.cu), and x is copied out as z_j on the way.
// ---------------------------------------------------------------------------
template <int DIM, int BT>
__global__ void __launch_bounds__(256) k_packed_apply_df(Dims g, FineOp<double> f, const float2* __restrict__ pk2,
                                                         DfLaplacian lap, const float2* __restrict__ x,
                                                         float2* __restrict__ y, int64_t ylo, float2* __restrict__ zcopy) {
  if (BT == 1 && resolve_uniform(g)) return;
  if (BT == 2 && resolve(g, f)) return;
  if (BT == 2)   // the problem's own spacing
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      lap.hi[d] = (float)f.ih2[d];
      lap.lo[d] = (float)(f.ih2[d] - (double)lap.hi[d]);
    }
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  if (BT) {
    shift_nodes(g, x, y);
    shift_nodes_opt(g, zcopy);
  }
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  if (j == f.dyn[blockIdx.y].src_index) {        // the source row (Eq. helmADR2), in float64
    double2 c[1 + 4 * DIM];
    fine_row<DIM, double>(g, f, j, ii, c);
    const float2 x0 = __ldg(x + j);
    double2 acc = cmul(c[0], make_double2(x0.x, x0.y));
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int64_t st = axis_stride<DIM>(g, d);
      const int k = ii[d], n = g.n[d];
      const int64_t nb[4] = {k >= 1 ? j - st : j, k <= n - 2 ? j + st : j, k >= 2 ? j - 2 * st : j,
                             k <= n - 3 ? j + 2 * st : j};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 xv = __ldg(x + nb[q]);
        acc = cfma(c[1 + 4 * d + q], make_double2(xv.x, xv.y), acc);
      }
    }
    const float2 r = df_split(acc.x), m = df_split(acc.y);
    y[j] = make_float2(r.x, m.x);
    y[j + ylo] = make_float2(r.y, m.y);
    if (zcopy) zcopy[j] = x0;
    return;
  }
  const float2* pk = pk2 + (int64_t)(2 + 4 * DIM) * g.off + j;
  const float2 xj = __ldg(x + j);
  const float2 cr = __ldg(pk), ci = __ldg(pk + g.N);
  DfSum ar{0.f, 0.f}, ai{0.f, 0.f}, br{0.f, 0.f}, bi{0.f, 0.f};
  df_add_prod(ar, cr.x, cr.y, xj.x);
  df_add_prod(ar, -ci.x, -ci.y, xj.y);
  df_add_prod(ai, cr.x, cr.y, xj.y);
  df_add_prod(ai, ci.x, ci.y, xj.x);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int64_t s = axis_stride<DIM>(g, d);
    const int k = ii[d], n = g.n[d];
    const int64_t jm1 = k >= 1 ? j - s : j, jp1 = k <= n - 2 ? j + s : j;
    const int64_t jm2 = k >= 2 ? j - 2 * s : j, jp2 = k <= n - 3 ? j + 2 * s : j;
    // real parts of the +-1 entries: the Laplacian's 1/h^2, doubled on a face, zero off the grid
    const float mh = k == 0 ? 0.f : (k == n - 1 ? 2.f * lap.hi[d] : lap.hi[d]);
    const float ml = k == 0 ? 0.f : (k == n - 1 ? 2.f * lap.lo[d] : lap.lo[d]);
    const float ph = k == n - 1 ? 0.f : (k == 0 ? 2.f * lap.hi[d] : lap.hi[d]);
    const float pl = k == n - 1 ? 0.f : (k == 0 ? 2.f * lap.lo[d] : lap.lo[d]);
    const float2 xm1 = __ldg(x + jm1), xp1 = __ldg(x + jp1), xm2 = __ldg(x + jm2), xp2 = __ldg(x + jp2);
    const float2 bm1 = __ldg(pk + (int64_t)(2 + 4 * d + 0) * g.N), bp1 = __ldg(pk + (int64_t)(2 + 4 * d + 1) * g.N);
    const float2 bm2 = __ldg(pk + (int64_t)(2 + 4 * d + 2) * g.N), bp2 = __ldg(pk + (int64_t)(2 + 4 * d + 3) * g.N);
    df_add_prod(ar, mh, ml, xm1.x);
    df_add_prod(ai, mh, ml, xm1.y);
    df_add_prod(br, ph, pl, xp1.x);
    df_add_prod(bi, ph, pl, xp1.y);
    df_add_prod(ar, -bm1.x, -bm1.y, xm1.y);
    df_add_prod(ai, bm1.x, bm1.y, xm1.x);
    df_add_prod(br, -bp1.x, -bp1.y, xp1.y);
    df_add_prod(bi, bp1.x, bp1.y, xp1.x);
    df_add_prod(ar, -bm2.x, -bm2.y, xm2.y);
    df_add_prod(ai, bm2.x, bm2.y, xm2.x);
    df_add_prod(br, -bp2.x, -bp2.y, xp2.y);
    df_add_prod(bi, bp2.x, bp2.y, xp2.x);
  }
  df_add(ar, br);
  df_add(ai, bi);
  const float2 r = df_pair(ar), m = df_pair(ai);
  y[j] = make_float2(r.x, m.x);
  y[j + ylo] = make_float2(r.y, m.y);
  if (zcopy) zcopy[j] = xj;
}

// Split of the float64 packed rows into float32 (hi, lo) pairs.
__global__ void k_split_df(const double* __restrict__ src, float2* __restrict__ dst, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = src[i];
  const float hi = __double2float_rn(v);
  dst[i] = make_float2(hi, __double2float_rn(v - (double)hi));
}

DfLaplacian df_laplacian(const FineOp<double>& f) {
  DfLaplacian l{};
  for (int d = 0; d < 3; ++d) {
    const double v = f.ih2[d];
    l.hi[d] = (float)v;
    l.lo[d] = (float)(v - (double)l.hi[d]);
  }
  return l;
}
void launch_split_df(const double* src, float2* dst, int64_t n, cudaStream_t st) {
  count_launches(1), k_split_df<<<blocks_for(n, 256), 256, 0, st>>>(src, dst, n);
}
void launch_packed_apply_df(const Dims& g, const FineOp<double>& f, const float2* pk2, const float2* x, float2* y,
                            int64_t ylo, float2* zcopy, cudaStream_t st) {
  const DfLaplacian lap = df_laplacian(f);
  const int bt = g.pd ? 2 : (g.B > 1 ? 1 : 0);
  auto kern = g.dim == 2 ? (bt == 2 ? k_packed_apply_df<2, 2> : bt ? k_packed_apply_df<2, 1> : k_packed_apply_df<2, 0>)
                         : (bt == 2 ? k_packed_apply_df<3, 2> : bt ? k_packed_apply_df<3, 1> : k_packed_apply_df<3, 0>);
  count_launches(1), kern<<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, f, pk2, lap, x, y, ylo, zcopy);
}

void launch_fine_store_rows(const Dims& g, const FineOp<double>& f, double2* rows, cudaStream_t st) {
  if (g.dim == 2) count_launches(1), k_fine_store_rows<2, double><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, f, rows);
  else count_launches(1), k_fine_store_rows<3, double><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, f, rows);
}
void launch_fine_store_rows(const Dims& g, const FineOp<float>& f, float2* rows, cudaStream_t st) {
  if (g.dim == 2) count_launches(1), k_fine_store_rows<2, float><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, f, rows);
  else count_launches(1), k_fine_store_rows<3, float><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, f, rows);
}

// Conjugate transpose of stored cross rows: row i of A^H holds, at the slot
// of offset o, conj(A[i + o][i]), the entry of row i + o at offset -o (zero
// when i + o is off the grid, where A has no row).
template <int DIM, typename T>
__global__ void k_rows_adjoint(Dims g, const C<T>* __restrict__ rows, C<T>* __restrict__ rowsT) {
  if (resolve(g)) return;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  shift_scaled(g, 1 + 4 * DIM, rows, rowsT);
  int ii[3];
  unravel(g, i, ii[0], ii[1], ii[2]);
  const C<T> c0 = rows[i];
  rowsT[i] = mk<T>(c0.x, -c0.y);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int64_t stride = d == 0 ? 1 : (d == 1 ? g.s1 : g.s2);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int o = (s & 2) ? ((s & 1) ? 2 : -2) : ((s & 1) ? 1 : -1);   // slots -1, +1, -2, +2
      const int q = 1 + 4 * d + s, qbar = 1 + 4 * d + (s ^ 1);
      C<T> v = czero<T>();
      const int k = ii[d] + o;
      if (k >= 0 && k < g.n[d]) {
        const C<T> a = rows[(int64_t)qbar * g.N + i + o * stride];
        v = mk<T>(a.x, -a.y);
      }
      rowsT[(int64_t)q * g.N + i] = v;
    }
  }
}
template <typename T>
void launch_rows_adjoint(const Dims& g, const C<T>* rows, C<T>* rowsT, cudaStream_t st) {
  if (g.dim == 2) count_launches(1), k_rows_adjoint<2, T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, rows, rowsT);
  else count_launches(1), k_rows_adjoint<3, T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, rows, rowsT);
}
template void launch_rows_adjoint<double>(const Dims&, const double2*, double2*, cudaStream_t);

// M A M^{-1} for stored cross rows: the entry of row i at offset o is scaled
// by m_i conj(m_{i+o}) = exp(-i w (tau_i - tau_{i+o})) (|m| = 1); the centre
// and the zero slots of off-grid neighbours are unchanged.
template <int DIM, typename T>
__global__ void k_rows_rescale(Dims g, C<T>* __restrict__ rows, const double2* __restrict__ phase) {
  if (resolve(g)) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  shift_scaled(g, 1 + 4 * DIM, rows);
  shift_nodes(g, phase);
  int ii[3];
  unravel(g, i, ii[0], ii[1], ii[2]);
  const double2 mi = phase[i];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int64_t stride = d == 0 ? 1 : (d == 1 ? g.s1 : g.s2);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int o = (s & 2) ? ((s & 1) ? 2 : -2) : ((s & 1) ? 1 : -1);   // slots -1, +1, -2, +2
      const int k = ii[d] + o;
      if (k < 0 || k >= g.n[d]) continue;
      double2 mn = phase[i + o * stride];
      mn.y = -mn.y;
      const double2 f = cmul(mi, mn);
      C<T>& e = rows[(int64_t)(1 + 4 * d + s) * g.N + i];
      const double2 r = cmul(make_double2((double)e.x, (double)e.y), f);
      e = mk<T>((T)r.x, (T)r.y);
    }
  }
}
template <typename T> void launch_rows_rescale(const Dims& g, C<T>* rows, const double2* phase, cudaStream_t st) {
  if (g.dim == 2) count_launches(1), k_rows_rescale<2, T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, rows, phase);
  else count_launches(1), k_rows_rescale<3, T><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, rows, phase);
}
template void launch_rows_rescale<double>(const Dims&, double2*, const double2*, cudaStream_t);
template void launch_rows_rescale<float>(const Dims&, float2*, const double2*, cudaStream_t);
template void launch_rows_adjoint<float>(const Dims&, const float2*, float2*, cudaStream_t);
void launch_rows_apply(const Dims& g, const double2* rows, const double2* x, double2* y, cudaStream_t st) {
  if (g.dim == 2) count_launches(1), k_rows_apply<2, double><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, rows, x, y);
  else count_launches(1), k_rows_apply<3, double><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, rows, x, y);
}
void launch_rows_residual(const Dims& g, const double2* rows, const double2* b, const double2* x, double2* r, cudaStream_t st) {
  if (g.dim == 2) count_launches(1), k_rows_residual<2, double><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, rows, b, x, r);
  else count_launches(1), k_rows_residual<3, double><<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(g, rows, b, x, r);
}

}  // namespace adr
