// Travel-time factor tau1 on the device: the first-order upwind (Godunov)
// discretisation of the factored eikonal equation
//   |tau0 grad(tau1) + tau1 grad(tau0)|^2 = kappa^2   (Eq. factoredEikonal),
// tau0 = |x - x0| with analytic gradient, relaxed in place to its fixed point.
// Every node repeatedly solves its local quadratic from the current values
// of its face neighbours and keeps the smaller of the old and new value, so
// the iterate decreases monotonically from +inf and stops changing once the
// discrete system is satisfied (the same fixed point a fast-marching ordering
// reaches, without the sequential heap).  Axes whose neighbours are not
// smaller contribute nothing (Godunov); a root that would be smaller than a
// neighbour it used drops that axis.
#include <cmath>
#include <string>

#include "adr_common.cuh"

namespace adr {

static inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

struct EikParams {
  int src[3];
  double h[3];
  int64_t js;
};

__global__ void k_eik_init(double* tau1, int64_t N, int64_t js, const double* kappa) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) tau1[i] = i == js ? kappa[js] : INFINITY;
}

template <int DIM>
__global__ void k_eik_sweep(Dims g, EikParams P, const double* __restrict__ kappa, double* tau1, int* changed) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N || j == P.js) return;
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  double dx[3], r2 = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    dx[d] = (ii[d] - P.src[d]) * P.h[d];
    r2 += dx[d] * dx[d];
  }
  const double r = sqrt(r2);
  // best (smallest tau) neighbour per axis
  double tnb[3], t1nb[3];
  int side[3], ax[3];
  int na = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int64_t stride = d == 0 ? 1 : (d == 1 ? g.s1 : g.s2);
    double best = INFINITY, best1 = INFINITY;
    int bs = 0;
    for (int s = -1; s <= 1; s += 2) {
      const int k = ii[d] + s;
      if (k < 0 || k >= g.n[d]) continue;
      const double t1 = tau1[j + s * stride];
      if (!(t1 < INFINITY)) continue;
      double rr = 0.0;
#pragma unroll
      for (int e = 0; e < DIM; ++e) {
        const double de = (e == d) ? dx[e] + s * P.h[e] : dx[e];
        rr += de * de;
      }
      const double t = sqrt(rr) * t1;
      if (t < best) { best = t; best1 = t1; bs = s; }
    }
    if (bs != 0) { tnb[na] = best; t1nb[na] = best1; side[na] = bs; ax[na] = d; ++na; }
  }
  if (na == 0) return;
  // sort the used axes by neighbour tau (insertion sort, <= 3 entries)
  for (int a = 1; a < na; ++a)
    for (int b = a; b > 0 && tnb[b] < tnb[b - 1]; --b) {
      double t = tnb[b]; tnb[b] = tnb[b - 1]; tnb[b - 1] = t;
      t = t1nb[b]; t1nb[b] = t1nb[b - 1]; t1nb[b - 1] = t;
      int q = side[b]; side[b] = side[b - 1]; side[b - 1] = q;
      q = ax[b]; ax[b] = ax[b - 1]; ax[b - 1] = q;
    }
  const double kj = kappa[j];
  double cand = INFINITY;
  for (int use = na; use >= 1; --use) {
    double a2 = 0.0, a1 = 0.0, a0 = -kj * kj;
    for (int a = 0; a < use; ++a) {
      const int d = ax[a];
      const double d0 = dx[d] / r;
      const double A = -side[a] * r / P.h[d] + d0;
      const double B = side[a] * r * t1nb[a] / P.h[d];
      a2 += A * A;
      a1 += 2.0 * A * B;
      a0 += B * B;
    }
    double disc = a1 * a1 - 4.0 * a2 * a0;
    if (disc < 0.0 && use == 1) disc = 0.0;
    if (disc < 0.0) continue;
    const double t = (-a1 + sqrt(disc)) / (2.0 * a2);
    bool causal = true;
    for (int a = 0; a < use; ++a) causal = causal && (r * t >= tnb[a]);
    if (causal || use == 1) { cand = t; break; }
  }
  if (cand < tau1[j]) {
    tau1[j] = cand;
    *changed = 1;
  }
}

// Second-order phase.  One Jacobi sweep of the second-order update, read from
// tin, written to tout (deterministic): along each axis the one-sided
// difference points to the face neighbour nb with the smaller tau, and uses
// (3 t_j - 4 t_nb + t_nb2) / 2h when the node nb2 two steps out on that side
// exists with tau(nb2) <= tau(nb), except at Chebyshev distance 1 from the
// source (first order there, where tau has its kink).  The quadratic's
// larger root is taken; a root below a used neighbour's tau drops the axis
// with the largest neighbour tau; failing that with the second-order
// differences, the first-order ones are tried the same way (a negative
// discriminant with one axis left clamps to zero).  changed is raised when a
// node moves by more than rtol of its value.
template <int DIM>
__global__ void k_eik_sweep2(Dims g, EikParams P, const double* __restrict__ kappa, const double* __restrict__ tin,
                             double* __restrict__ tout, int* changed, double rtol) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  const double old = tin[j];
  if (j == P.js) { tout[j] = old; return; }
  int ii[3];
  unravel(g, j, ii[0], ii[1], ii[2]);
  double dx[3], r2 = 0.0;
  int cheb = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    dx[d] = (ii[d] - P.src[d]) * P.h[d];
    r2 += dx[d] * dx[d];
    const int a = ii[d] > P.src[d] ? ii[d] - P.src[d] : P.src[d] - ii[d];
    cheb = a > cheb ? a : cheb;
  }
  const double r = sqrt(r2);
  const bool near = cheb <= 1;
  auto tau_of = [&](int64_t k, int d, int off) {   // tau at node k = j + off along axis d
    double rr = 0.0;
#pragma unroll
    for (int e = 0; e < DIM; ++e) {
      const double de = (e == d) ? dx[e] + off * P.h[e] : dx[e];
      rr += de * de;
    }
    return sqrt(rr) * tin[k];
  };
  double tnb[3], t1nb[3], t1nb2[3];
  int side[3], ax[3];
  bool two[3];
  int na = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int64_t stride = d == 0 ? 1 : (d == 1 ? g.s1 : g.s2);
    double best = INFINITY;
    int bs = 0;
    for (int sg = -1; sg <= 1; sg += 2) {
      const int k = ii[d] + sg;
      if (k < 0 || k >= g.n[d]) continue;
      const double t = tau_of(j + sg * stride, d, sg);
      if (t < best) { best = t; bs = sg; }
    }
    if (bs == 0 || !(best < INFINITY)) continue;
    tnb[na] = best;
    t1nb[na] = tin[j + bs * stride];
    side[na] = bs;
    ax[na] = d;
    two[na] = false;
    const int k2 = ii[d] + 2 * bs;
    if (!near && k2 >= 0 && k2 < g.n[d]) {
      const double t2 = tau_of(j + 2 * bs * stride, d, 2 * bs);
      if (t2 <= best) { two[na] = true; t1nb2[na] = tin[j + 2 * bs * stride]; }
    }
    ++na;
  }
  double cand = old;
  if (na > 0) {
    for (int a = 1; a < na; ++a)
      for (int b = a; b > 0 && tnb[b] < tnb[b - 1]; --b) {
        double t = tnb[b]; tnb[b] = tnb[b - 1]; tnb[b - 1] = t;
        t = t1nb[b]; t1nb[b] = t1nb[b - 1]; t1nb[b - 1] = t;
        t = t1nb2[b]; t1nb2[b] = t1nb2[b - 1]; t1nb2[b - 1] = t;
        int q = side[b]; side[b] = side[b - 1]; side[b - 1] = q;
        q = ax[b]; ax[b] = ax[b - 1]; ax[b - 1] = q;
        const bool w = two[b]; two[b] = two[b - 1]; two[b - 1] = w;
      }
    const double kj = kappa[j];
    bool found = false;
    for (int pass = 0; pass < 2 && !found; ++pass) {
      const bool second = pass == 0;
      for (int use = na; use >= 1; --use) {
        double a2 = 0.0, a1 = 0.0, a0 = -kj * kj;
        for (int a = 0; a < use; ++a) {
          const int d = ax[a];
          const double d0 = dx[d] / r;
          double A, B;
          if (second && two[a]) {
            A = -side[a] * 1.5 * r / P.h[d] + d0;
            B = side[a] * r * (4.0 * t1nb[a] - t1nb2[a]) / (2.0 * P.h[d]);
          } else {
            A = -side[a] * r / P.h[d] + d0;
            B = side[a] * r * t1nb[a] / P.h[d];
          }
          a2 += A * A;
          a1 += 2.0 * A * B;
          a0 += B * B;
        }
        double disc = a1 * a1 - 4.0 * a2 * a0;
        if (disc < 0.0 && use == 1 && !second) disc = 0.0;
        if (disc < 0.0) continue;
        const double t = (-a1 + sqrt(disc)) / (2.0 * a2);
        bool causal = true;
        for (int a = 0; a < use; ++a) causal = causal && (r * t >= tnb[a]);
        if (causal || (use == 1 && !second)) { cand = t; found = true; break; }
      }
    }
  }
  tout[j] = cand;
  if (fabs(cand - old) > rtol * fabs(old)) *changed = 1;
}

}  // namespace adr

using namespace adr;

// First-order relaxation to its fixed point; with order 2 it then iterates
// the second-order update from there (ping-pong between tau1 and a scratch
// array) until no node moves by more than a relative 1e-12.
static int traveltime_impl(int dim, const int* n, const double* h, const int* src, const double* kappa, double* tau1,
                           int order, int max_sweeps, void* stream, int* sweeps_done) {
  if ((dim != 2 && dim != 3) || !n || !h || !src || !kappa || !tau1 || max_sweeps < 1)
    return set_last_error(ADR_ERR_ARG, "invalid argument");
  for (int d = 0; d < dim; ++d)
    if (n[d] < 2 || !(h[d] > 0.0) || src[d] < 0 || src[d] >= n[d]) return set_last_error(ADR_ERR_ARG, "invalid grid or source");
  cudaStream_t st = (cudaStream_t)stream;
  Dims g = make_dims(dim, n);
  EikParams P{};
  for (int d = 0; d < 3; ++d) {
    P.src[d] = d < dim ? src[d] : 0;
    P.h[d] = d < dim ? h[d] : 1.0;
  }
  P.js = P.src[0] + g.s1 * P.src[1] + g.s2 * P.src[2];
  int* flag = nullptr;
  int* host_flag = nullptr;
  double* scratch = nullptr;
  cudaError_t e = cudaMalloc(&flag, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_last_error(ADR_ERR_OOM, (std::string("cudaMalloc of the sweep flag: ") + cudaGetErrorString(e)).c_str());
  }
  e = cudaMallocHost(&host_flag, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(flag);
    return set_last_error(ADR_ERR_OOM, (std::string("cudaMallocHost of the sweep flag: ") + cudaGetErrorString(e)).c_str());
  }
  count_launches(1), k_eik_init<<<blocks_for(g.N, 256), 256, 0, st>>>(tau1, g.N, P.js, kappa);
  int done = 0;
  const int check_every = 16;
  e = cudaGetLastError();
  while (e == cudaSuccess && done < max_sweeps) {
    e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    for (int k = 0; e == cudaSuccess && k < check_every && done < max_sweeps; ++k, ++done) {
      if (dim == 2) count_launches(1), k_eik_sweep<2><<<blocks_for(g.N, 256), 256, 0, st>>>(g, P, kappa, tau1, flag);
      else count_launches(1), k_eik_sweep<3><<<blocks_for(g.N, 256), 256, 0, st>>>(g, P, kappa, tau1, flag);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && *host_flag == 0) break;
  }
  bool converged = e == cudaSuccess && done < max_sweeps;
  if (converged && order == 2) {
    e = cudaMalloc(&scratch, sizeof(double) * (size_t)g.N);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(flag);
      cudaFreeHost(host_flag);
      if (sweeps_done) *sweeps_done = done;
      return set_last_error(ADR_ERR_OOM, (std::string("cudaMalloc of the second-order scratch: ") + cudaGetErrorString(e)).c_str());
    }
    double* cur = tau1;
    double* nxt = scratch;
    int done2 = 0;
    converged = false;
    while (e == cudaSuccess && done2 < max_sweeps) {
      e = cudaMemsetAsync(flag, 0, sizeof(int), st);
      for (int k = 0; e == cudaSuccess && k < check_every && done2 < max_sweeps; ++k, ++done2) {
        if (dim == 2) count_launches(1), k_eik_sweep2<2><<<blocks_for(g.N, 256), 256, 0, st>>>(g, P, kappa, cur, nxt, flag, 1e-12);
        else count_launches(1), k_eik_sweep2<3><<<blocks_for(g.N, 256), 256, 0, st>>>(g, P, kappa, cur, nxt, flag, 1e-12);
        double* tmp = cur; cur = nxt; nxt = tmp;
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaMemcpyAsync(host_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e == cudaSuccess && *host_flag == 0) { converged = true; break; }
    }
    if (e == cudaSuccess && cur != tau1) e = cudaMemcpyAsync(tau1, cur, sizeof(double) * (size_t)g.N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    done += done2;
  }
  cudaFree(scratch);
  cudaFree(flag);
  cudaFreeHost(host_flag);
  if (sweeps_done) *sweeps_done = done;
  if (e != cudaSuccess) return set_last_error(ADR_ERR_CUDA, (std::string("travel-time sweeps: ") + cudaGetErrorString(e)).c_str());
  if (!converged) return set_last_error(ADR_ERR_NOT_CONVERGED, "max_sweeps reached while tau1 still changed");
  return ADR_OK;
}

extern "C" int adr_traveltime(int dim, const int* n, const double* h, const int* src, const double* kappa, double* tau1,
                              int max_sweeps, void* stream, int* sweeps_done) {
  return traveltime_impl(dim, n, h, src, kappa, tau1, 1, max_sweeps, stream, sweeps_done);
}

extern "C" int adr_traveltime_order(int dim, const int* n, const double* h, const int* src, const double* kappa,
                                    double* tau1, int order, int max_sweeps, void* stream, int* sweeps_done) {
  if (order != 1 && order != 2) return set_last_error(ADR_ERR_ARG, "order must be 1 or 2");
  return traveltime_impl(dim, n, h, src, kappa, tau1, order, max_sweeps, stream, sweeps_done);
}

// ---------------------------------------------------------------------------
// adr_traveltime_static: the same relaxation without any allocation.
//
// Callers that cannot allocate: a process whose device memory is held by a
// caching allocator (a cudaMalloc can then fail although the caller's pool has
// room), and callers keeping other streams busy, because cudaFree waits for
// the whole device and cudaMallocHost pins pages at a cost comparable to the
// solve of a small grid.  Here the convergence flags live in a fixed device
// array, one int per sweep: sweep k of a call sets flag k when it lowers any
// node.  The call zeroes the flags it will use before the first sweep, so
// the array may hold anything from an earlier call.  Every call on a device
// uses the same array: calls that overlap in time on one device (other
// threads, other streams) race on it and must be serialised by the caller.
// ---------------------------------------------------------------------------
#include <mutex>

namespace adr {

constexpr int kStaticMaxSweeps = 8192;   // 32 KiB of flags; ADR_TRAVELTIME_STATIC_MAX_SWEEPS
static __device__ __align__(256) int g_sweep_flags[kStaticMaxSweeps];

constexpr int kStaticMaxDevices = 64;
static std::mutex g_sweep_flags_mu;
static int* g_sweep_flags_ptr[kStaticMaxDevices] = {};

// Device address of g_sweep_flags on the current device, looked up once per
// device (the lookup may load the module on that device, so the first call
// on a device must not happen inside a stream capture).
static int sweep_flags_on_current_device(int** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_last_error(ADR_ERR_CUDA, (std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
  if (dev < 0 || dev >= kStaticMaxDevices) return set_last_error(ADR_ERR_ARG, "device index above 63");
  std::lock_guard<std::mutex> lock(g_sweep_flags_mu);
  if (!g_sweep_flags_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sweep_flags);
    if (e != cudaSuccess || !p)
      return set_last_error(ADR_ERR_CUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
    g_sweep_flags_ptr[dev] = static_cast<int*>(p);
  }
  *out = g_sweep_flags_ptr[dev];
  return ADR_OK;
}

}  // namespace adr

extern "C" int adr_traveltime_static(int dim, const int* n, const double* h, const int* src, const double* kappa,
                                     double* tau1, int max_sweeps, void* stream, int* sweeps_done) {
  if ((dim != 2 && dim != 3) || !n || !h || !src || !kappa || !tau1 || max_sweeps < 1)
    return set_last_error(ADR_ERR_ARG, "invalid argument");
  if (max_sweeps > kStaticMaxSweeps)
    return set_last_error(ADR_ERR_ARG, "max_sweeps exceeds the static flag array (8192 sweeps)");
  for (int d = 0; d < dim; ++d)
    if (n[d] < 2 || !(h[d] > 0.0) || src[d] < 0 || src[d] >= n[d]) return set_last_error(ADR_ERR_ARG, "invalid grid or source");
  int* flags = nullptr;
  const int rc0 = sweep_flags_on_current_device(&flags);
  if (rc0 != ADR_OK) return rc0;
  cudaStream_t st = (cudaStream_t)stream;
  Dims g = make_dims(dim, n);
  EikParams P{};
  for (int d = 0; d < 3; ++d) {
    P.src[d] = d < dim ? src[d] : 0;
    P.h[d] = d < dim ? h[d] : 1.0;
  }
  P.js = P.src[0] + g.s1 * P.src[1] + g.s2 * P.src[2];
  if (cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)max_sweeps, st) != cudaSuccess)
    return set_last_error(ADR_ERR_CUDA, "cudaMemsetAsync of the sweep flags failed");
  count_launches(1), k_eik_init<<<blocks_for(g.N, 256), 256, 0, st>>>(tau1, g.N, P.js, kappa);
  constexpr int check_every = 16;
  int host_flags[check_every];   // pageable stack memory: no pinned allocation
  int done = 0;
  while (done < max_sweeps) {
    const int first = done;
    for (int k = 0; k < check_every && done < max_sweeps; ++k, ++done) {
      if (dim == 2) count_launches(1), k_eik_sweep<2><<<blocks_for(g.N, 256), 256, 0, st>>>(g, P, kappa, tau1, flags + done);
      else count_launches(1), k_eik_sweep<3><<<blocks_for(g.N, 256), 256, 0, st>>>(g, P, kappa, tau1, flags + done);
    }
    const int batch = done - first;
    if (cudaMemcpyAsync(host_flags, flags + first, sizeof(int) * (size_t)batch, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      if (sweeps_done) *sweeps_done = done;
      return set_last_error(ADR_ERR_CUDA, "reading the sweep flags failed");
    }
    int any = 0;
    for (int k = 0; k < batch; ++k) any |= host_flags[k];
    if (!any) break;
  }
  if (sweeps_done) *sweeps_done = done;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_last_error(ADR_ERR_CUDA, cudaGetErrorString(e));
  if (done >= max_sweeps) return set_last_error(ADR_ERR_NOT_CONVERGED, "max_sweeps reached while tau1 still changed");
  return ADR_OK;
}
