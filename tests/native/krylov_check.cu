// Host check of the scalar Arnoldi helpers of the GMRES iterations
// (paper_1712_06091_gb300/csrc/krylov_dev.cuh, compiled here for the host):
//   givens: [c s; -conj(s) c] [a; b] = [r; 0] with c^2 + |s|^2 = 1;
//   arnoldi_column_dev over the columns of a random upper Hessenberg matrix
//   (real positive subdiagonal, as the Arnoldi process makes it), then
//   backsolve_dev: y minimises |beta e1 - H y| and the running estimate of
//   every step equals that step's least-squares residual, both against a
//   modified Gram-Schmidt QR of H in long double (no rotations);
//   a zero subdiagonal entry (breakdown) stops the columns there and y then
//   solves the square leading system;
//   coarse_select_dev: the selective decision from Pythagoras and, when the
//   single pass holds, the same column and reciprocal norm as
//   arnoldi_column_dev with the remainder's norm.
// Prints "ok" or the first failure.
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>
#include <vector>

#include "../../paper_1712_06091_gb300/csrc/krylov_dev.cuh"

using adr::ArnoldiState;
using cld = std::complex<long double>;

static int fail(const char* what, double a, double b) {
  std::printf("%s: %.17g %.17g\n", what, a, b);
  return 1;
}

struct Host {
  int m;
  std::vector<double2> H, sn, g, y;
  std::vector<double> cs, scal;
  std::vector<int> iscal;
  explicit Host(int m_) : m(m_), H((m_ + 1) * m_), sn(m_), g(m_ + 1), y(m_), cs(m_), scal(adr::kNumScal), iscal(adr::kNumIScal) {}
  ArnoldiState state() {
    ArnoldiState s;
    s.m = m; s.H = H.data(); s.cs = cs.data(); s.sn = sn.data(); s.g = g.data(); s.y = y.data();
    s.scal = scal.data(); s.iscal = iscal.data();
    return s;
  }
  void start(double beta) {
    for (auto& v : g) v = make_double2(0.0, 0.0);
    g[0] = make_double2(beta, 0.0);
    iscal[adr::kIScalStop] = -1;
    iscal[adr::kIScalConv] = -1;
    scal[adr::kScalTarget] = 0.0;
  }
};

// Least squares min |beta e1 - A y| for the (rows x cols) leading block of A
// (column-major, leading dimension ld) by modified Gram-Schmidt in long double:
// returns y and the norm of beta e1 - A y.
static void mgs_lsq(const std::vector<cld>& A, int ld, int rows, int cols, long double beta, std::vector<cld>& y,
                    long double& res) {
  std::vector<cld> Q(A.begin(), A.end()), R(cols * cols, cld(0));
  for (int j = 0; j < cols; ++j) {
    for (int i = 0; i < j; ++i) {
      cld d = 0;
      for (int r = 0; r < rows; ++r) d += std::conj(Q[i * ld + r]) * Q[j * ld + r];
      R[j * cols + i] = d;
      for (int r = 0; r < rows; ++r) Q[j * ld + r] -= d * Q[i * ld + r];
    }
    long double nn = 0;
    for (int r = 0; r < rows; ++r) nn += std::norm(Q[j * ld + r]);
    const long double n = std::sqrt(nn);
    R[j * cols + j] = n;
    for (int r = 0; r < rows; ++r) Q[j * ld + r] /= n;
  }
  std::vector<cld> qb(cols);
  for (int j = 0; j < cols; ++j) qb[j] = std::conj(Q[j * ld + 0]) * beta;
  y.assign(cols, cld(0));
  for (int i = cols - 1; i >= 0; --i) {
    cld acc = qb[i];
    for (int q = i + 1; q < cols; ++q) acc -= R[q * cols + i] * y[q];
    y[i] = acc / R[i * cols + i];
  }
  // the residual norm from the residual itself (beta^2 - |Q^H b|^2 cancels when it is small)
  long double rr = 0;
  for (int r = 0; r < rows; ++r) {
    cld v = r == 0 ? cld(beta) : cld(0);
    for (int q = 0; q < cols; ++q) v -= A[q * ld + r] * y[q];
    rr += std::norm(v);
  }
  res = std::sqrt(rr);
}

int main() {
  std::mt19937_64 rng(2024);
  std::normal_distribution<double> nd(0.0, 1.0);

  // Givens rotations
  for (int it = 0; it < 20000; ++it) {
    const double2 a = make_double2(nd(rng), nd(rng)), b = make_double2(nd(rng), nd(rng));
    double c;
    double2 s, r;
    adr::givens(a, b, c, s, r);
    if (std::fabs(c * c + s.x * s.x + s.y * s.y - 1.0) > 1e-14) return fail("givens c^2+|s|^2", c, s.x);
    const std::complex<double> A(a.x, a.y), B(b.x, b.y), S(s.x, s.y), R(r.x, r.y);
    const std::complex<double> top = c * A + S * B, bot = -std::conj(S) * A + c * B;
    const double sc = std::abs(A) + std::abs(B);
    if (std::abs(top - R) > 1e-14 * sc) return fail("givens r", std::abs(top - R), sc);
    if (std::abs(bot) > 1e-14 * sc) return fail("givens zero", std::abs(bot), sc);
  }

  // Hessenberg columns, estimates and the back substitution
  for (int trial = 0; trial < 200; ++trial) {
    const int m = 1 + trial % 12;
    Host h(m);
    const double beta = 0.5 + std::fabs(nd(rng));
    h.start(beta);
    ArnoldiState st = h.state();
    std::vector<cld> A((m + 1) * m, cld(0));
    std::vector<double2> ha(m + 1), hb(m + 1, make_double2(0.0, 0.0));
    for (int j = 0; j < m; ++j) {
      for (int i = 0; i <= j; ++i) {
        ha[i] = make_double2(nd(rng) + (i == j ? 3.0 : 0.0), nd(rng));
        A[j * (m + 1) + i] = cld(ha[i].x, ha[i].y);
      }
      const double sub = 0.2 + std::fabs(nd(rng));
      A[j * (m + 1) + j + 1] = sub;
      adr::arnoldi_column_dev(st, j, ha.data(), hb.data(), sub * sub);
      std::vector<cld> yj;
      long double res;
      mgs_lsq(A, m + 1, j + 2, j + 1, beta, yj, res);
      const double est = h.scal[adr::kScalEst];
      if (std::fabs(est - (double)res) > 1e-13 * beta) return fail("estimate", est, (double)res);
      if (std::fabs(h.scal[adr::kScalHn] - sub) > 1e-15 * sub) return fail("h_{j+1,j}", h.scal[adr::kScalHn], sub);
    }
    adr::backsolve_dev(st, m);
    std::vector<cld> yref;
    long double res;
    mgs_lsq(A, m + 1, m + 1, m, beta, yref, res);
    long double ny = 0;
    for (int i = 0; i < m; ++i) ny += std::norm(yref[i]);
    for (int i = 0; i < m; ++i) {
      const long double d = std::abs(cld(h.y[i].x, h.y[i].y) - yref[i]);
      if (d > 1e-11L * std::sqrt(ny)) return fail("back substitution", (double)d, (double)std::sqrt(ny));
    }
  }

  // breakdown: h_{b+1,b} = 0 stops the columns at b + 1; y solves the square system
  for (int trial = 0; trial < 100; ++trial) {
    const int m = 4 + trial % 6, bk = trial % m;
    Host h(m);
    const double beta = 1.0 + std::fabs(nd(rng));
    h.start(beta);
    ArnoldiState st = h.state();
    std::vector<cld> A((m + 1) * m, cld(0));
    std::vector<double2> ha(m + 1), hb(m + 1, make_double2(0.0, 0.0));
    for (int j = 0; j < m; ++j) {
      for (int i = 0; i <= j; ++i) {
        ha[i] = make_double2(nd(rng) + (i == j ? 3.0 : 0.0), nd(rng));
        A[j * (m + 1) + i] = cld(ha[i].x, ha[i].y);
      }
      const double sub = j == bk ? 0.0 : 0.2 + std::fabs(nd(rng));
      A[j * (m + 1) + j + 1] = sub;
      adr::arnoldi_column_dev(st, j, ha.data(), hb.data(), sub * sub);
    }
    if (h.iscal[adr::kIScalStop] != bk + 1) return fail("breakdown column", h.iscal[adr::kIScalStop], bk + 1);
    adr::backsolve_dev(st, m);
    const int k = bk + 1;
    for (int i = 0; i < k; ++i) {   // (H y)_i = beta e1 on the square leading block
      cld acc = 0;
      for (int q = 0; q < k; ++q) acc += A[q * (m + 1) + i] * cld(h.y[q].x, h.y[q].y);
      const cld want = i == 0 ? cld(beta) : cld(0);
      if (std::abs(acc - want) > 1e-12L * beta) return fail("breakdown solve", (double)std::abs(acc - want), beta);
    }
    for (int i = k; i < m; ++i)
      if (h.y[i].x != 0.0 || h.y[i].y != 0.0) return fail("breakdown tail", h.y[i].x, h.y[i].y);
  }

  // selective decision from Pythagoras
  for (int trial = 0; trial < 2000; ++trial) {
    const int k = 1 + trial % 9;
    const double eta = 0.1;
    std::vector<double2> ha(k + 1), hb(k + 1, make_double2(0.0, 0.0)), ha0;
    double h2 = 0.0;
    for (int i = 0; i < k; ++i) {
      ha[i] = make_double2(nd(rng), nd(rng));
      h2 += ha[i].x * ha[i].x + ha[i].y * ha[i].y;
    }
    // |w|^2 = |h|^2 + remainder, the remainder's share spread across the threshold
    const double share = std::ldexp(1.0, -(1 + trial % 20));   // remainder / |w|^2, 2^-1 .. 2^-20
    const double s2 = h2 / (1.0 - share);
    ha[k] = make_double2(s2, 0.0);
    ha0 = ha;
    Host h(10), ref(10);
    h.start(1.0);
    ref.start(1.0);
    double2 nrm2 = make_double2(0.0, 0.0);
    const int j = k - 1;
    for (int c = 0; c < j; ++c) {   // earlier columns, the same in both states
      std::vector<double2> col(c + 1);
      for (int i = 0; i <= c; ++i) col[i] = make_double2(nd(rng) + (i == c ? 3.0 : 0.0), nd(rng));
      const double sub = 0.5 + std::fabs(nd(rng));
      adr::arnoldi_column_dev(h.state(), c, col.data(), hb.data(), sub * sub);
      adr::arnoldi_column_dev(ref.state(), c, col.data(), hb.data(), sub * sub);
    }
    adr::coarse_select_dev(ha.data(), hb.data(), k, eta * eta, h.state(), j, 0, &nrm2);
    const double t = s2 - h2;
    const bool single = share >= eta * eta * (1.0 + 1e-9);
    const bool second = share <= eta * eta * (1.0 - 1e-9);
    if (single && ha[k].y != 0.0) return fail("selective: second pass where the single pass holds", share, eta);
    if (second && ha[k].y != 1.0) return fail("selective: no second pass after cancellation", share, eta);
    if (ha[k].y == 0.0) {
      if (std::fabs(nrm2.x - t) > 1e-12 * s2) return fail("remainder", nrm2.x, t);
      if (std::fabs(nrm2.y * std::sqrt(t) - 1.0) > 1e-14) return fail("reciprocal norm", nrm2.y, t);
      adr::arnoldi_column_dev(ref.state(), j, ha0.data(), hb.data(), nrm2.x);
      for (int i = 0; i < (j + 2) * 1; ++i) {
        const double2 a = h.H[j * 11 + i], b = ref.H[j * 11 + i];
        if (a.x != b.x || a.y != b.y) return fail("selective column", a.x, b.x);
      }
      if (h.scal[adr::kScalEst] != ref.scal[adr::kScalEst]) return fail("selective estimate", h.scal[adr::kScalEst], ref.scal[adr::kScalEst]);
    }
  }
  std::printf("ok\n");
  return 0;
}
