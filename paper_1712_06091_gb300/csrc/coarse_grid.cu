// Coarsest-grid solve as one persistent cooperative launch over all SMs.
//
// The fixed-count Jacobi-preconditioned GMRES of the coarsest level (Sec. 3.1;
// ten iterations in place of a factorisation, Sec. 4.2) on grids too large for
// one thread-block cluster: the problem's blocks (all co-resident, guaranteed
// by the cooperative launch) each own a contiguous slice of the nodes and meet
// at grid barriers.  Per GMRES step two or three barriers:
//   1. w = A z on the slice, the first Gram-Schmidt pass's slice sums V^H w
//      and |w|^2; the remainder |w - V ha|^2 = |w|^2 - |ha|^2 (V orthonormal)
//      decides whether the second pass runs (the selective test with
//      eta2 = reorth_eta^2; eta2 >= 1 always runs it);
//   2. only then: w -= V ha, the second pass's slice sums V^H w and |w|^2,
//      the column's norm again from Pythagoras (hb is at rounding level);
//   3. V_{j+1} = (w - V c) / h, z = D^{-1} V_{j+1} on the slice, visible to
//      every block before the next apply reads its neighbours.
//
// Reductions are deterministic: every block writes its slice sums to its row
// of a partial array; after the barrier every block adds all rows, one warp
// per value, lanes striding over the blocks and a fixed shuffle tree, so all
// blocks hold identical totals.  Two partial arrays alternate, so one barrier
// per reduction suffices (a block writes an array again only after every
// block has passed the barrier that follows its reads of it).  The Hessenberg
// matrix, rotations and least-squares solution are small and kept by every
// block in shared memory, updated redundantly from identical totals.
//
// Barriers spin on a generation counter with an iteration limit; a block that
// gives up raises the problem's error word, every block then leaves, and the
// solution is set to NaN so that the outer iteration reports the failure.
#include "coarse_stencil.cuh"
#include "krylov_dev.cuh"
#include "reduce.cuh"

namespace adr {

constexpr int kGridThreads = 512;
constexpr unsigned kBarrierSpins = 1u << 21;       // x (32 ns sleep + an L2 read): about a second
constexpr int kGridStride = kGridMaxK + 1;           // values per block row of a partial array

// Arrival counter bar[0] and generation bar[1] of one problem's blocks.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblk, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g0 = *gen;
    int ok = 1;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblk - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned spins = 0;
      while (*gen == g0) {
        if (++spins > kBarrierSpins || *(volatile int*)err) { ok = 0; break; }
        __nanosleep(32);
      }
      if (!ok) atomicExch(err, 1);
    }
    __threadfence();
    s_ok = ok && !*(volatile int*)err;
  }
  __syncthreads();
  return s_ok;
}

// Thread 0 holds the block's K slice sums in mine[0..K) (K <= kGridStride):
// row blockIdx.x of part.  The last block to arrive adds the rows in block
// order (one warp per value, lanes over the blocks, fixed shuffle tree) into
// tot_g and only then releases the others; every block copies the K totals
// into tot (shared).  One pass over the partials per reduction, by one block.
__device__ __forceinline__ bool grid_totals(const double2* mine, int K, double2* part, double2* tot_g, unsigned* bar,
                                            unsigned nblk, int* err, double2* tot) {
  __shared__ int s_last, s_ok;
  __shared__ unsigned s_gen;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < K; ++i) part[(size_t)blockIdx.x * kGridStride + i] = mine[i];
    s_gen = *(volatile unsigned*)(bar + 1);   // before arriving: the release comes after every arrival
    __threadfence();
    s_last = atomicAdd(bar, 1u) == nblk - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = wid; i < K; i += nw) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll 4
      for (unsigned b = lane; b < nblk; b += 32) {
        const double2 p = __ldcg(&part[(size_t)b * kGridStride + i]);
        acc.x += p.x;
        acc.y += p.y;
      }
      acc = warp_sum2(acc);
      if (lane == 0) {
        tot_g[i] = acc;
        __threadfence();
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
      s_ok = !*(volatile int*)err;
    }
  } else if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    int ok = 1;
    unsigned spins = 0;
    while (*gen == s_gen) {
      if (++spins > kBarrierSpins || *(volatile int*)err) { ok = 0; break; }
      __nanosleep(32);
    }
    if (!ok) atomicExch(err, 1);
    __threadfence();
    s_ok = ok && !*(volatile int*)err;
  }
  __syncthreads();
  if (!s_ok) return false;
  for (int i = threadIdx.x; i < K; i += blockDim.x) tot[i] = __ldcg(&tot_g[i]);
  __syncthreads();
  return true;
}

// Slice sums of conj(V_i) w for i < k, and (with norm) |w|^2 as value k, into
// blk (thread 0; shared).
template <typename T>
__device__ __forceinline__ void slice_dots_g(const C<T>* V, int64_t ld, int64_t lo, int64_t hi, int k, const C<T>* w,
                                             bool norm, double2* blk, double2* sh) {
  for (int c = 0; c < k || (norm && c == 0); c += 4) {
    C<T> acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = czero<T>();
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      const C<T> we = w[e];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c + q < k) acc[q] = cfma_conj(V[(int64_t)(c + q) * ld + e], we, acc[q]);
      if (norm && c == 0) acc[4] = cfma_conj(we, we, acc[4]);
    }
    double2 o[5];
    block_sum_t<T, 5>(acc, sh, o);
    if (threadIdx.x == 0) {
      for (int q = 0; q < 4 && c + q < k; ++q) blk[c + q] = o[q];
      if (norm && c == 0) blk[k] = o[4];
    }
    __syncthreads();
  }
}

template <int DIM, typename T>
__global__ void __launch_bounds__(kGridThreads) k_coarse_gmres_grid(Dims g, const C<T>* __restrict__ A,
                                                                    const C<T>* __restrict__ dinv, const C<T>* b, C<T>* x,
                                                                    C<T>* V, C<T>* z, int k, GridScratch gs,
                                                                    double eta2) {
  if (resolve(g)) return;
  const int pb = blockIdx.y;
  const unsigned nblk = gridDim.x;
  const int64_t n = g.N;
  const int64_t ld = g.total;
  shift_stencil(g, A);
  shift_nodes(g, dinv, b, x, V, z);
  double2* part0 = gs.part + (size_t)pb * 2 * gs.nblk * kGridStride;
  double2* part1 = part0 + (size_t)gs.nblk * kGridStride;
  double2* tot_g = gs.tot + (size_t)pb * kGridStride;
  unsigned* bar = gs.bar + 2 * pb;
  int* err = gs.err + pb;
  const int64_t chunk = (n + nblk - 1) / nblk;
  const int64_t lo = blockIdx.x * chunk < n ? blockIdx.x * chunk : n;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;

  __shared__ double2 sh[32 * 5];
  __shared__ double2 blk[kGridStride];
  __shared__ double2 ha[kGridStride];
  __shared__ double2 hb[kGridStride];
  __shared__ C<T> cv[kGridMaxK + 1];
  __shared__ double2 H[(kGridMaxK + 1) * kGridMaxK];
  __shared__ double cs[kGridMaxK];
  __shared__ double2 sn[kGridMaxK];
  __shared__ double2 gg[kGridMaxK + 1];
  __shared__ double2 y[kGridMaxK];
  __shared__ T s_inv;
  __shared__ int s_stop, s_two;
  int buf = 0;
  bool ok = true;
  auto part = [&]() { double2* p = buf ? part1 : part0; buf ^= 1; return p; };

  // beta = |b| ; V_0 = b / beta ; z = D^{-1} V_0
  {
    C<T> s[1] = {czero<T>()};
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) s[0] = cfma_conj(b[e], b[e], s[0]);
    double2 o[1];
    block_sum_t<T, 1>(s, sh, o);
    if (threadIdx.x == 0) blk[0] = o[0];
    ok = grid_totals(blk, 1, part(), tot_g, bar, nblk, err, ha);
    if (threadIdx.x == 0) {   // float64 square root and division once per block
      const double beta = sqrt(ha[0].x);
      for (int i = 0; i <= kGridMaxK; ++i) gg[i] = make_double2(0.0, 0.0);
      gg[0] = make_double2(beta, 0.0);
      s_stop = beta > 0.0 ? k : 0;
      s_inv = beta > 0.0 ? (T)(1.0 / beta) : T(0);
    }
    __syncthreads();
    const T inv = s_inv;
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      const C<T> v = cscale(b[e], inv);
      V[e] = v;
      z[e] = cmul(dinv[e], v);
    }
    ok = ok && grid_barrier(bar, nblk, err);
  }
  for (int j = 0; ok && j < k; ++j) {
    C<T>* w = V + (int64_t)(j + 1) * ld;
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
      int i0, i1, i2;
      unravel(g, e, i0, i1, i2);
      w[e] = stencil_dot<DIM, T, true>(g, A, z, e, i0, i1, i2);   // z of every block, written before the barrier
    }
    __syncthreads();
    // first Gram-Schmidt pass: ha = V^H w and |w|^2; the selective decision
    slice_dots_g<T>(V, ld, lo, hi, j + 1, w, true, blk, sh);
    if (!(ok = grid_totals(blk, j + 2, part(), tot_g, bar, nblk, err, ha))) break;
    if (threadIdx.x == 0) {
      double t = ha[j + 1].x;
      for (int i = 0; i <= j; ++i) t -= ha[i].x * ha[i].x + ha[i].y * ha[i].y;
      s_two = !(t >= eta2 * ha[j + 1].x);
      if (!s_two) {   // one pass: hb = 0, |w - V ha|^2 = t
        for (int i = 0; i <= j; ++i) hb[i] = make_double2(0.0, 0.0);
        hb[j + 1] = make_double2(t, 0.0);
      }
    }
    __syncthreads();
    if (s_two) {
      for (int i = threadIdx.x; i <= j; i += blockDim.x) cv[i] = mk<T>((T)(-ha[i].x), (T)(-ha[i].y));
      __syncthreads();
      for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        C<T> acc = w[e];
        for (int i = 0; i <= j; ++i) acc = cfma(V[(int64_t)i * ld + e], cv[i], acc);
        w[e] = acc;
      }
      __syncthreads();
      // second pass: hb = V^H w and |w|^2 in one reduction
      slice_dots_g<T>(V, ld, lo, hi, j + 1, w, true, blk, sh);
      if (!(ok = grid_totals(blk, j + 2, part(), tot_g, bar, nblk, err, hb))) break;
    }
    if (threadIdx.x == 0) {
      // Hessenberg column j, earlier rotations, new rotation (same in every block)
      double t = hb[j + 1].x;
      if (s_two)
        for (int i = 0; i <= j; ++i) t -= hb[i].x * hb[i].x + hb[i].y * hb[i].y;
      const double hn = t > 0.0 ? sqrt(t) : (t == t ? 0.0 : t);
      double2* Hj = H + j * (kGridMaxK + 1);
      for (int i = 0; i <= j; ++i) Hj[i] = make_double2(ha[i].x + hb[i].x, ha[i].y + hb[i].y);
      Hj[j + 1] = make_double2(hn, 0.0);
      for (int i = 0; i < j; ++i) {
        const double2 a0 = Hj[i], b0 = Hj[i + 1];
        const double2 cs_ = make_double2(sn[i].x, -sn[i].y);
        Hj[i] = cadd(make_double2(cs[i] * a0.x, cs[i] * a0.y), cmul(sn[i], b0));
        Hj[i + 1] = csub(make_double2(cs[i] * b0.x, cs[i] * b0.y), cmul(cs_, a0));
      }
      double c;
      double2 sv, r;
      givens(Hj[j], Hj[j + 1], c, sv, r);
      cs[j] = c;
      sn[j] = sv;
      Hj[j] = r;
      Hj[j + 1] = make_double2(0.0, 0.0);
      const double2 gj = gg[j];
      gg[j + 1] = make_double2(-(sv.x * gj.x + sv.y * gj.y), -(sv.x * gj.y - sv.y * gj.x));
      gg[j] = make_double2(c * gj.x, c * gj.y);
      if (!(hn > 0.0) && s_stop > j + 1) s_stop = j + 1;
      s_inv = hn > 0.0 ? (T)(1.0 / hn) : T(0);
    }
    __syncthreads();
    // V_{j+1} = (w - V c) / h with c = hb after the second pass (w already
    // updated), ha after a single pass ; z = D^{-1} V_{j+1}
    if (j + 1 < k) {
      const double2* c = s_two ? hb : ha;
      for (int i = threadIdx.x; i <= j; i += blockDim.x) cv[i] = mk<T>((T)(-c[i].x), (T)(-c[i].y));
      __syncthreads();
      const T inv = s_inv;
      for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        C<T> acc = w[e];
        for (int i = 0; i <= j; ++i) acc = cfma(V[(int64_t)i * ld + e], cv[i], acc);
        const C<T> v = cscale(acc, inv);
        w[e] = v;
        z[e] = cmul(dinv[e], v);
      }
      if (!(ok = grid_barrier(bar, nblk, err))) break;
    }
  }
  if (!ok) {
    const C<T> nan = mk<T>((T)NAN, (T)NAN);
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) x[e] = nan;
    return;
  }
  // y = R^{-1} g on the leading s_stop columns, x = D^{-1} V y
  if (threadIdx.x == 0) {
    const int kk = s_stop < k ? s_stop : k;
    for (int i = 0; i < kGridMaxK; ++i) y[i] = make_double2(0.0, 0.0);
    for (int i = kk - 1; i >= 0; --i) {
      double2 acc = gg[i];
      for (int q = i + 1; q < kk; ++q) acc = csub(acc, cmul(H[q * (kGridMaxK + 1) + i], y[q]));
      y[i] = cmul(acc, cinv(H[i * (kGridMaxK + 1) + i]));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) cv[i] = mk<T>((T)y[i].x, (T)y[i].y);
  __syncthreads();
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    C<T> acc = czero<T>();
    for (int i = 0; i < k; ++i) acc = cfma(V[(int64_t)i * ld + e], cv[i], acc);
    x[e] = cmul(dinv[e], acc);
  }
}

// Blocks of the persistent solve that can be co-resident on the device (0 if
// the cooperative launch is unavailable).  Called outside any stream capture.
int prepare_coarse_grid(int dim, bool f32) {
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 0; }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  const void* kernel = dim == 2 ? (f32 ? (const void*)k_coarse_gmres_grid<2, float> : (const void*)k_coarse_gmres_grid<2, double>)
                                : (f32 ? (const void*)k_coarse_gmres_grid<3, float> : (const void*)k_coarse_gmres_grid<3, double>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kGridThreads, 0) != cudaSuccess) per_sm = 0;
  cudaGetLastError();
  return coop ? per_sm * sms : 0;
}

template <typename T>
void launch_coarse_gmres_grid(const Dims& g, const C<T>* A, const C<T>* dinv, const C<T>* b, C<T>* x, C<T>* V, C<T>* z,
                              int k, const GridScratch& gs, double eta, cudaStream_t st) {
  const double eta2 = eta * eta;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(gs.nblk, g.B, 1);
  cfg.blockDim = dim3(kGridThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // A barrier that timed out in an earlier solve may have left its arrival
  // count part-filled and raised the error word: every solve starts from zero
  // (memset nodes when captured).
  cudaMemsetAsync(gs.bar, 0, sizeof(unsigned) * 2 * (size_t)g.B, st);
  cudaMemsetAsync(gs.err, 0, sizeof(int) * (size_t)g.B, st);
  count_launches(1);
  if (g.dim == 2) cudaLaunchKernelEx(&cfg, k_coarse_gmres_grid<2, T>, g, A, dinv, b, x, V, z, k, gs, eta2);
  else cudaLaunchKernelEx(&cfg, k_coarse_gmres_grid<3, T>, g, A, dinv, b, x, V, z, k, gs, eta2);
}

template void launch_coarse_gmres_grid<double>(const Dims&, const double2*, const double2*, const double2*, double2*,
                                               double2*, double2*, int, const GridScratch&, double, cudaStream_t);
template void launch_coarse_gmres_grid<float>(const Dims&, const float2*, const float2*, const float2*, float2*,
                                              float2*, float2*, int, const GridScratch&, double, cudaStream_t);

}  // namespace adr
