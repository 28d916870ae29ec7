// Scalar (single-thread) parts of the Arnoldi process kept on the device:
// complex Givens rotations, the update of Hessenberg column j, and the
// back substitution for the least-squares coefficients.
#pragma once

#include <cmath>

#include "krylov.cuh"

namespace adr {

// 1/sqrt(v): the device's reciprocal square root, or 1/sqrt on the host
// (where these helpers are compiled for the host-side checks).
__host__ __device__ __forceinline__ double arnoldi_rsqrt(double v) {
#ifdef __CUDA_ARCH__
  return rsqrt(v);
#else
  return 1.0 / std::sqrt(v);
#endif
}

// These run on one thread, so their cost is the latency of a float64
// dependency chain.  Measured on GB300 (one thread, clock64): a dependent
// float64 FMA or add takes about 64 cycles (float32: 4.5), a square root
// about 600, a division or a reciprocal square root about 350, hypot about
// 1100.  Hence reciprocal square roots and products in place of hypot, sqrt
// and divisions, and short chains for sums.  The entries are far from the
// float64 overflow and underflow thresholds, so squared magnitudes need no
// scaling.

// Complex Givens rotation with real cosine: [c s; -conj(s) c] [a; b] = [r; 0].
__host__ __device__ __forceinline__ void givens(double2 a, double2 b, double& c, double2& s, double2& r) {
  const double a2 = a.x * a.x + a.y * a.y, b2 = b.x * b.x + b.y * b.y;
  if (b2 == 0.0) { c = 1.0; s = make_double2(0.0, 0.0); r = a; return; }
  if (a2 == 0.0) { c = 0.0; s = make_double2(1.0, 0.0); r = b; return; }
  const double n2 = a2 + b2;
  const double ia = arnoldi_rsqrt(a2), inu = arnoldi_rsqrt(n2);   // 1/|a|, 1/nu
  c = (a2 * ia) * inu;
  const double2 ph = make_double2(a.x * ia, a.y * ia);
  const double2 cb = make_double2(b.x * inu, -b.y * inu);
  s = cmul(ph, cb);
  const double nu = n2 * inu;
  r = make_double2(ph.x * nu, ph.y * nu);
}

// sqrt(v) and 1/sqrt(v) for v >= 0 (both 0 at 0; a NaN stays NaN in the first).
__host__ __device__ __forceinline__ void sqrt_pair(double v, double& root, double& inv) {
  inv = v > 0.0 ? arnoldi_rsqrt(v) : 0.0;
  root = v * inv;
}

// |h|^2 - sum_{i<k} |c_i|^2 with two interleaved partial sums (half the chain).
__host__ __device__ __forceinline__ double pythagoras_remainder(double s2, const double2* c, int k) {
  double t0 = 0.0, t1 = 0.0;
  int i = 0;
  for (; i + 1 < k; i += 2) {
    t0 = fma(c[i].x, c[i].x, fma(c[i].y, c[i].y, t0));
    t1 = fma(c[i + 1].x, c[i + 1].x, fma(c[i + 1].y, c[i + 1].y, t1));
  }
  if (i < k) t0 = fma(c[i].x, c[i].x, fma(c[i].y, c[i].y, t0));
  return s2 - (t0 + t1);
}

// Arnoldi column j from ha + hb and |w|^2, Givens update (one thread).
__host__ __device__ __forceinline__ void arnoldi_column_dev(ArnoldiState st, int j, const double2* ha, const double2* hb, double nrm2) {
  const int m1 = st.m + 1;
  double2* H = st.H + (int64_t)j * m1;
  if (st.iscal[kIScalStop] >= 0) {
    for (int i = 0; i <= j + 1; ++i) H[i] = make_double2(0.0, 0.0);
    st.scal[kScalHn] = 0.0;
    return;
  }
  for (int i = 0; i <= j; ++i) H[i] = make_double2(ha[i].x + hb[i].x, ha[i].y + hb[i].y);
  double hn, ihn;
  sqrt_pair(nrm2, hn, ihn);
  H[j + 1] = make_double2(hn, 0.0);
  for (int i = 0; i < j; ++i) {
    const double2 a = H[i], b = H[i + 1];
    const double c = st.cs[i];
    const double2 s = st.sn[i];
    const double2 cs_ = make_double2(s.x, -s.y);
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
  st.g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
  st.g[j] = make_double2(c * gj.x, c * gj.y);
  const double2 gn = st.g[j + 1];
  const double est = sqrt(gn.x * gn.x + gn.y * gn.y);
  st.scal[kScalEst] = est;
  st.scal[kScalHn] = hn;
  st.scal[kScalNrm2] = nrm2;
  if (hn == 0.0) st.iscal[kIScalStop] = j + 1;
  if (st.iscal[kIScalConv] < 0 && est <= st.scal[kScalTarget]) st.iscal[kIScalConv] = j + 1;
}

// y = R^{-1} g for the leading k x k block of the rotated Hessenberg matrix
// (k is cut to the breakdown or the convergence column if there was one).
__host__ __device__ __forceinline__ void backsolve_dev(ArnoldiState st, int k) {
  const int m1 = st.m + 1;
  const int stop = st.iscal[kIScalStop];
  if (stop >= 0 && stop < k) k = stop;
  const int conv = st.iscal[kIScalConv];
  if (conv >= 0 && conv < k) k = conv;
  for (int i = 0; i < st.m; ++i) st.y[i] = make_double2(0.0, 0.0);
  // the diagonal's inverses first: independent of each other, so their
  // divisions overlap instead of lengthening the substitution's chain
  for (int i = 0; i < k; ++i) st.y[i] = cinv(st.H[(int64_t)i * m1 + i]);
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = st.g[i];
    for (int q = i + 1; q < k; ++q) acc = csub(acc, cmul(st.H[(int64_t)q * m1 + i], st.y[q]));
    st.y[i] = cmul(acc, st.y[i]);
  }
}

// Epilogues of the coarsest-grid Arnoldi step with the selective second
// Gram-Schmidt pass (one thread, after the totals are in place).
//
// After the first pass: ha[0..k) = V^H w, ha[k].x = |w|^2.  The remainder
// |w - V ha|^2 = |w|^2 - |ha|^2 (V orthonormal) decides: at least eta2 |w|^2
// keeps the single pass (hb = 0, Arnoldi column j, reciprocal norm in nrm2,
// ha[k].y = 0, and on the last step the back substitution over `finish`
// columns); below it, ha[k].y = 1 requests the second pass.
__host__ __device__ __forceinline__ void coarse_select_dev(double2* ha, double2* hb, int k, double eta2, ArnoldiState st, int j,
                                                  int finish, double2* nrm2) {
  const double s2 = ha[k].x;
  double t = pythagoras_remainder(s2, ha, k);
  if (!(t > 0.0)) t = t == t ? 0.0 : t;   // clamp rounding below zero; keep a NaN
  if (t >= eta2 * s2) {
    ha[k].y = 0.0;
    for (int i = 0; i < k; ++i) hb[i] = make_double2(0.0, 0.0);
    double root, inv;
    sqrt_pair(t, root, inv);
    nrm2->x = t;
    nrm2->y = inv;
    arnoldi_column_dev(st, j, ha, hb, t);
    if (finish > 0) backsolve_dev(st, finish);
  } else {
    ha[k].y = 1.0;
  }
}
// After the second pass: hb[0..k) = V^H w', hb[k].x = |w'|^2 with w' = w - V ha;
// |w' - V hb|^2 = |w'|^2 - |hb|^2 (hb is at rounding level, no cancellation).
__host__ __device__ __forceinline__ void coarse_reorth_dev(const double2* ha, const double2* hb, int k, ArnoldiState st, int j,
                                                  int finish, double2* nrm2) {
  double t = pythagoras_remainder(hb[k].x, hb, k);
  if (!(t > 0.0)) t = t == t ? 0.0 : t;
  double root, inv;
  sqrt_pair(t, root, inv);
  nrm2->x = t;
  nrm2->y = inv;
  arnoldi_column_dev(st, j, ha, hb, t);
  if (finish > 0) backsolve_dev(st, finish);
}

// coarse_select_dev run by a whole block on a shared-memory copy.
//
// The single-thread epilogue walks the Arnoldi state in global memory, one
// dependent load after another (Givens rotations over the column, the
// rotation's cs and sn, g, the back substitution's columns): about 11 us per
// coarsest-grid step on GB300, a third of the step.  Here every thread of the
// block first loads the state's entries in one round into sm, thread 0 runs
// coarse_select_dev on the copy (the same arithmetic, so the same bits), and
// the block writes the copy back.  sm holds arnoldi_stage_words(m, k)
// double2; every thread of the block calls this.
__host__ __device__ constexpr int arnoldi_stage_words(int m, int k) {
  return (m + 1) * m + 4 * m + 1 + kNumScal + kNumIScal + 2 * (k + 1) + 1;
}
__device__ __forceinline__ void coarse_select_block(double2* ha, double2* hb, int k, double eta2, ArnoldiState st, int j,
                                                    int finish, double2* nrm2, double2* sm) {
  const int m = st.m, m1 = m + 1;
  double2* sH = sm;
  double* scs = reinterpret_cast<double*>(sH + (size_t)m1 * m);
  double2* ssn = sH + (size_t)m1 * m + m;
  double2* sg = ssn + m;
  double2* sy = sg + m1;
  double* sscal = reinterpret_cast<double*>(sy + m);
  int* siscal = reinterpret_cast<int*>(sy + m + kNumScal);
  double2* sha = sy + m + kNumScal + kNumIScal;
  double2* shb = sha + k + 1;
  double2* snrm = shb + k + 1;
  const int ncol = j + 1;   // columns 0..j (the back substitution reads them; column j is rewritten)
  for (int e = threadIdx.x; e < ncol * m1; e += blockDim.x) sH[e] = st.H[e];
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    scs[e] = st.cs[e];
    ssn[e] = st.sn[e];
    sy[e] = st.y[e];
  }
  for (int e = threadIdx.x; e < m1; e += blockDim.x) sg[e] = st.g[e];
  for (int e = threadIdx.x; e < kNumScal; e += blockDim.x) sscal[e] = st.scal[e];
  for (int e = threadIdx.x; e < kNumIScal; e += blockDim.x) siscal[e] = st.iscal[e];
  for (int e = threadIdx.x; e <= k; e += blockDim.x) {
    sha[e] = ha[e];
    shb[e] = hb[e];
  }
  if (threadIdx.x == 0) *snrm = *nrm2;
  __syncthreads();
  if (threadIdx.x == 0) {
    ArnoldiState sst{m, sH, scs, ssn, sg, sy, sscal, siscal};
    coarse_select_dev(sha, shb, k, eta2, sst, j, finish, snrm);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ncol * m1; e += blockDim.x) st.H[e] = sH[e];
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    st.cs[e] = scs[e];
    st.sn[e] = ssn[e];
    st.y[e] = sy[e];
  }
  for (int e = threadIdx.x; e < m1; e += blockDim.x) st.g[e] = sg[e];
  for (int e = threadIdx.x; e < kNumScal; e += blockDim.x) st.scal[e] = sscal[e];
  for (int e = threadIdx.x; e < kNumIScal; e += blockDim.x) st.iscal[e] = siscal[e];
  for (int e = threadIdx.x; e <= k; e += blockDim.x) {
    ha[e] = sha[e];
    hb[e] = shb[e];
  }
  if (threadIdx.x == 0) *nrm2 = *snrm;
}

}  // namespace adr
