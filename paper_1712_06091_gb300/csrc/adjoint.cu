// Receiver sampling and the slowness gradient of a receiver misfit.
//
// With u = M a (M = diag(exp(-i w tau)), Eq. new_u) sampled at receiver nodes
// R and data d, the misfit J = 1/2 |R u - d|^2 depends on the slowness only
// through the reaction term of the ADR operator, w^2 kappa^2 - i w gamma
// kappa^2 on the diagonal (Eq. ADR; the travel time is held fixed).  With the
// adjoint state lambda solving H^H lambda = M^H R^T (R u - d),
//   dJ/dkappa_j = -Re( conj(lambda_j) (2 w^2 kappa_j - 2 i w gamma_j kappa_j) a_j ).
#include "adr_common.cuh"
#include "reduce.cuh"

namespace adr {

static inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// res_k = u[rec_k] - d_k ; rhs[rec_k] += exp(+i w tau) res_k ; sums of |res|^2
// and of out-of-grid receiver indices into out->x / out->y (one block).
__global__ void k_receivers(int64_t N, int nrec, const int64_t* __restrict__ rec, const double2* __restrict__ d,
                            const double2* __restrict__ u, const double* __restrict__ tau, double omega,
                            double2* __restrict__ res, double2* rhs, double2* out) {
  __shared__ double2 sh[32];
  double2 acc = make_double2(0.0, 0.0);
  for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
    const int64_t j = rec[k];
    if (j < 0 || j >= N) {
      acc.y += 1.0;
      if (res) res[k] = make_double2(0.0, 0.0);
      continue;
    }
    const double2 r = make_double2(u[j].x - d[k].x, u[j].y - d[k].y);
    if (res) res[k] = r;
    acc.x += r.x * r.x + r.y * r.y;
    if (rhs) {
      double s, c;
      sincos(omega * tau[j], &s, &c);
      atomicAdd(&rhs[j].x, c * r.x - s * r.y);
      atomicAdd(&rhs[j].y, s * r.x + c * r.y);
    }
  }
  double2 v[1] = {acc}, tot[1];
  block_sum_k<1>(v, sh, tot);
  if (threadIdx.x == 0) *out = tot[0];
}

void launch_receivers(int64_t N, int nrec, const int64_t* rec, const double2* d, const double2* u, const double* tau,
                      double omega, double2* res, double2* rhs, double2* out, cudaStream_t st) {
  count_launches(1), k_receivers<<<1, 256, 0, st>>>(N, nrec, rec, d, u, tau, omega, res, rhs, out);
}

__global__ void k_kappa_gradient(int64_t N, double omega, const double* __restrict__ kappa,
                                 const double* __restrict__ gamma, const double2* __restrict__ a,
                                 const double2* __restrict__ lam, double* grad) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  const double k = kappa[j];
  const double cr = 2.0 * omega * omega * k, ci = -2.0 * omega * gamma[j] * k;
  const double2 aj = a[j], lj = lam[j];
  const double pr = cr * aj.x - ci * aj.y, pi = cr * aj.y + ci * aj.x;
  grad[j] -= lj.x * pr + lj.y * pi;
}

void launch_kappa_gradient(int64_t N, double omega, const double* kappa, const double* gamma, const double2* a,
                           const double2* lambda, double* grad, cudaStream_t st) {
  count_launches(1), k_kappa_gradient<<<blocks_for(N, 256), 256, 0, st>>>(N, omega, kappa, gamma, a, lambda, grad);
}

}  // namespace adr
