// Scalar (single-thread) parts of the Arnoldi process kept on the device:
// complex Givens rotations, the update of Hessenberg column j, and the
// back substitution for the least-squares coefficients.
#pragma once

#include "krylov.cuh"

namespace adr {

// Complex Givens rotation with real cosine: [c s; -conj(s) c] [a; b] = [r; 0].
__device__ __forceinline__ void givens(double2 a, double2 b, double& c, double2& s, double2& r) {
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

// Arnoldi column j from ha + hb and |w|^2, Givens update (one thread).
__device__ __forceinline__ void arnoldi_column_dev(ArnoldiState st, int j, const double2* ha, const double2* hb, double nrm2) {
  const int m1 = st.m + 1;
  double2* H = st.H + (int64_t)j * m1;
  if (st.iscal[kIScalStop] >= 0) {
    for (int i = 0; i <= j + 1; ++i) H[i] = make_double2(0.0, 0.0);
    st.scal[kScalHn] = 0.0;
    return;
  }
  for (int i = 0; i <= j; ++i) H[i] = make_double2(ha[i].x + hb[i].x, ha[i].y + hb[i].y);
  const double hn = sqrt(nrm2);
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
  const double est = hypot(st.g[j + 1].x, st.g[j + 1].y);
  st.scal[kScalEst] = est;
  st.scal[kScalHn] = hn;
  st.scal[kScalNrm2] = nrm2;
  if (hn == 0.0) st.iscal[kIScalStop] = j + 1;
  if (st.iscal[kIScalConv] < 0 && est <= st.scal[kScalTarget]) st.iscal[kIScalConv] = j + 1;
}

// y = R^{-1} g for the leading k x k block of the rotated Hessenberg matrix
// (k is cut to the breakdown or the convergence column if there was one).
__device__ __forceinline__ void backsolve_dev(ArnoldiState st, int k) {
  const int m1 = st.m + 1;
  const int stop = st.iscal[kIScalStop];
  if (stop >= 0 && stop < k) k = stop;
  const int conv = st.iscal[kIScalConv];
  if (conv >= 0 && conv < k) k = conv;
  for (int i = 0; i < st.m; ++i) st.y[i] = make_double2(0.0, 0.0);
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = st.g[i];
    for (int q = i + 1; q < k; ++q) acc = csub(acc, cmul(st.H[(int64_t)q * m1 + i], st.y[q]));
    const double2 rii = st.H[(int64_t)i * m1 + i];
    st.y[i] = cmul(acc, cinv(rii));
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
__device__ __forceinline__ void coarse_select_dev(double2* ha, double2* hb, int k, double eta2, ArnoldiState st, int j,
                                                  int finish, double2* nrm2) {
  const double s2 = ha[k].x;
  double t = s2;
  for (int i = 0; i < k; ++i) t -= ha[i].x * ha[i].x + ha[i].y * ha[i].y;
  if (!(t > 0.0)) t = t == t ? 0.0 : t;   // clamp rounding below zero; keep a NaN
  if (t >= eta2 * s2) {
    ha[k].y = 0.0;
    for (int i = 0; i < k; ++i) hb[i] = make_double2(0.0, 0.0);
    nrm2->x = t;
    nrm2->y = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
    arnoldi_column_dev(st, j, ha, hb, t);
    if (finish > 0) backsolve_dev(st, finish);
  } else {
    ha[k].y = 1.0;
  }
}
// After the second pass: hb[0..k) = V^H w', hb[k].x = |w'|^2 with w' = w - V ha;
// |w' - V hb|^2 = |w'|^2 - |hb|^2 (hb is at rounding level, no cancellation).
__device__ __forceinline__ void coarse_reorth_dev(const double2* ha, const double2* hb, int k, ArnoldiState st, int j,
                                                  int finish, double2* nrm2) {
  double t = hb[k].x;
  for (int i = 0; i < k; ++i) t -= hb[i].x * hb[i].x + hb[i].y * hb[i].y;
  if (!(t > 0.0)) t = t == t ? 0.0 : t;
  nrm2->x = t;
  nrm2->y = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
  arnoldi_column_dev(st, j, ha, hb, t);
  if (finish > 0) backsolve_dev(st, finish);
}

}  // namespace adr
