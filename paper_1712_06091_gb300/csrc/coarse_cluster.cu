// Coarsest-grid solve on one thread-block cluster.
//
// The fixed-count Jacobi-preconditioned GMRES of the coarsest level (Sec. 3.1;
// ten iterations in place of a factorisation, Sec. 4.2) is a chain of small
// dependent steps: a stencil apply, three Gram-Schmidt reductions and a few
// vector updates per iteration.  Here every CTA of one cluster (up to 16 SMs)
// owns a contiguous slice of the nodes; vectors live in global memory (L2
// resident at these sizes) and the CTAs meet at hardware cluster barriers,
// whose release/acquire ordering makes each slice's writes visible to the
// other CTAs.  Reductions: each CTA sums its slice in a fixed order into its
// shared memory; after the barrier every CTA reads all CTAs' sums through
// distributed shared memory in rank order, so every CTA holds the same,
// deterministic totals.  Two reduction buffers alternate, so one barrier per
// reduction suffices.  The Hessenberg / Givens state is kept by CTA 0 only.
#include <cooperative_groups.h>

#include "coarse_stencil.cuh"
#include "krylov_dev.cuh"
#include "reduce.cuh"

namespace cg = cooperative_groups;

namespace adr {

constexpr int kClusterThreads = 256;
constexpr int kClusterMaxK = 32;   // Krylov dimension limit of this kernel

// Slice sums of conj(V_i) w for i < k into red[i] (valid in all threads after the call).
template <typename T>
__device__ __forceinline__ void slice_dots(const C<T>* V, int64_t ld, int64_t lo, int64_t hi, int k, const C<T>* w,
                                           double2* red, double2* sh) {
  for (int c = 0; c < k; c += 4) {
    C<T> acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = czero<T>();
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      const C<T> we = w[e];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c + q < k) acc[q] = cfma_conj(V[(int64_t)(c + q) * ld + e], we, acc[q]);
    }
    double2 o[4];
    block_sum_t<T, 4>(acc, sh, o);
    if (threadIdx.x == 0)
      for (int q = 0; q < 4 && c + q < k; ++q) red[c + q] = o[q];
    __syncthreads();
  }
}

// Totals over the cluster, in rank order, of the k values each CTA left in red.
__device__ __forceinline__ void cluster_totals(cg::cluster_group& cl, double2* red, int k, double2* out) {
  const int nb = (int)cl.num_blocks();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int r = 0; r < nb; ++r) {
      const double2* rr = cl.map_shared_rank(red, r);
      s.x += rr[i].x;
      s.y += rr[i].y;
    }
    out[i] = s;
  }
  __syncthreads();
}

template <int DIM, typename T>
__global__ void __launch_bounds__(kClusterThreads) k_coarse_gmres_cluster(Dims g, const C<T>* __restrict__ A,
                                                                         const C<T>* __restrict__ dinv, const C<T>* b,
                                                                         C<T>* x, C<T>* V, C<T>* z, int k, ArnoldiState st) {
  cg::cluster_group cl = cg::this_cluster();
  const int nb = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  if (resolve(g)) return;
  const int64_t n = g.N;
  const int64_t ld = g.total;   // basis stride (problem = blockIdx.y)
  shift_stencil(g, A);
  shift_nodes(g, dinv, b, x, V, z);
  st = arnoldi_at(st, blockIdx.y);
  const int64_t chunk = (n + nb - 1) / nb;
  const int64_t lo = rank * chunk < n ? rank * chunk : n;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;

  __shared__ double2 red[2][kClusterMaxK + 1];
  __shared__ double2 sh[32 * 4];
  __shared__ double2 ha[kClusterMaxK + 1];
  __shared__ double2 hb[kClusterMaxK + 1];
  __shared__ C<T> cv[kClusterMaxK + 1];
  __shared__ double s_val;
  int buf = 0;

  // beta = |b| ; V_0 = b / beta
  {
    C<T> s[1] = {czero<T>()};
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) s[0] = cfma_conj(b[e], b[e], s[0]);
    double2 o[1];
    block_sum_t<T, 1>(s, sh, o);
    if (threadIdx.x == 0) red[buf][0] = o[0];
    cl.sync();
    cluster_totals(cl, red[buf], 1, ha);
    buf ^= 1;
    const double beta = sqrt(ha[0].x);
    if (rank == 0 && threadIdx.x == 0) {
      for (int i = 0; i <= st.m; ++i) st.g[i] = make_double2(0.0, 0.0);
      st.g[0] = make_double2(beta, 0.0);
      st.scal[kScalBeta] = beta;
      st.scal[kScalEst] = beta;
      st.iscal[kIScalStop] = beta > 0.0 ? -1 : 0;
      st.iscal[kIScalConv] = beta > 0.0 ? -1 : 0;
    }
    const T inv = beta > 0.0 ? (T)(1.0 / beta) : T(0);
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) V[e] = cscale(b[e], inv);
  }
  for (int j = 0; j < k; ++j) {
    const C<T>* vj = V + (int64_t)j * ld;
    C<T>* w = V + (int64_t)(j + 1) * ld;
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) z[e] = cmul(dinv[e], vj[e]);
    cl.sync();  // z complete on every slice
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      int i0, i1, i2;
      unravel(g, e, i0, i1, i2);
      w[e] = stencil_dot<DIM, T, true>(g, A, z, e, i0, i1, i2);   // z was written in this launch
    }
    __syncthreads();
    // first Gram-Schmidt pass
    slice_dots<T>(V, ld, lo, hi, j + 1, w, red[buf], sh);
    cl.sync();
    cluster_totals(cl, red[buf], j + 1, ha);
    buf ^= 1;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) cv[i] = mk<T>((T)(-ha[i].x), (T)(-ha[i].y));
    __syncthreads();
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      C<T> acc = w[e];
      for (int i = 0; i <= j; ++i) acc = cfma(V[(int64_t)i * ld + e], cv[i], acc);
      w[e] = acc;
    }
    __syncthreads();
    // second pass
    slice_dots<T>(V, ld, lo, hi, j + 1, w, red[buf], sh);
    cl.sync();
    cluster_totals(cl, red[buf], j + 1, hb);
    buf ^= 1;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) cv[i] = mk<T>((T)(-hb[i].x), (T)(-hb[i].y));
    __syncthreads();
    C<T> s[1] = {czero<T>()};
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      C<T> acc = w[e];
      for (int i = 0; i <= j; ++i) acc = cfma(V[(int64_t)i * ld + e], cv[i], acc);
      w[e] = acc;
      s[0] = cfma_conj(acc, acc, s[0]);
    }
    double2 o[1];
    block_sum_t<T, 1>(s, sh, o);
    if (threadIdx.x == 0) red[buf][0] = o[0];
    cl.sync();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int r = 0; r < nb; ++r) t += cl.map_shared_rank(red[buf], r)[0].x;
      s_val = t;
      if (rank == 0) arnoldi_column_dev(st, j, ha, hb, t);
    }
    buf ^= 1;
    __syncthreads();
    const double hn = sqrt(s_val);
    if (j + 1 < k) {
      const T inv = hn > 0.0 ? (T)(1.0 / hn) : T(0);
      for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) w[e] = cscale(w[e], inv);
    }
  }
  cl.sync();  // CTA 0 holds the final rotations
  if (rank == 0 && threadIdx.x == 0) backsolve_dev(st, k);
  cl.sync();  // y visible to every CTA
  for (int i = threadIdx.x; i < k; i += blockDim.x) cv[i] = mk<T>((T)st.y[i].x, (T)st.y[i].y);
  __syncthreads();
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    C<T> acc = czero<T>();
    for (int i = 0; i < k; ++i) acc = cfma(V[(int64_t)i * ld + e], cv[i], acc);
    x[e] = cmul(dinv[e], acc);
  }
}

template <int DIM, typename T> static int set_cluster_attr() {
  return (int)cudaFuncSetAttribute(k_coarse_gmres_cluster<DIM, T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

// Picks the largest cluster size (16, else 8, else 0 = unavailable) that the
// device can schedule for this kernel.  Called once at operator creation,
// outside any stream capture.
int prepare_coarse_cluster(int dim, bool f32) {
  auto kernel = dim == 2 ? (f32 ? (const void*)k_coarse_gmres_cluster<2, float> : (const void*)k_coarse_gmres_cluster<2, double>)
                         : (f32 ? (const void*)k_coarse_gmres_cluster<3, float> : (const void*)k_coarse_gmres_cluster<3, double>);
  if (dim == 2) { if (f32) set_cluster_attr<2, float>(); else set_cluster_attr<2, double>(); }
  else { if (f32) set_cluster_attr<3, float>(); else set_cluster_attr<3, double>(); }
  cudaGetLastError();
  for (int size : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(size, 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) == cudaSuccess && clusters > 0) return size;
    cudaGetLastError();
  }
  return 0;
}

template <typename T>
void launch_coarse_gmres_cluster(const Dims& g, const C<T>* A, const C<T>* dinv, const C<T>* b, C<T>* x, C<T>* V, C<T>* z,
                                 int k, const ArnoldiState& s, int cluster, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, g.B, 1);   // one cluster per problem
  cfg.blockDim = dim3(kClusterThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launches(1);
  if (g.dim == 2) cudaLaunchKernelEx(&cfg, k_coarse_gmres_cluster<2, T>, g, A, dinv, b, x, V, z, k, s);
  else cudaLaunchKernelEx(&cfg, k_coarse_gmres_cluster<3, T>, g, A, dinv, b, x, V, z, k, s);
}

template void launch_coarse_gmres_cluster<double>(const Dims&, const double2*, const double2*, const double2*, double2*,
                                                  double2*, double2*, int, const ArnoldiState&, int, cudaStream_t);
template void launch_coarse_gmres_cluster<float>(const Dims&, const float2*, const float2*, const float2*, float2*,
                                                 float2*, float2*, int, const ArnoldiState&, int, cudaStream_t);

}  // namespace adr
