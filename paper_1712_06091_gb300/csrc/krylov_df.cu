// The outer flexible GMRES of the float32-cycle solve in double-float
// arithmetic (df.cuh): the selective Gram-Schmidt passes, the normalisation
// of the new basis vector and the combination x += Z y.
//
// A double-float basis vector is two float32 planes of complex values, the
// high parts at v and the low parts at v + lo (float2 units); vector i of a
// basis starts at V + i ld.  The passes compute exactly what the float64
// kernels of krylov.cu compute (Sec. 3.1, readings K1-K4), to about 2^-46
// instead of 2^-53 relative per operation; their inner products are reduced
// in double-float within a warp and in float64 across warps and blocks,
// deterministically (reduce.cuh).
#include "krylov.cuh"
#include "krylov_df.cuh"
#include "reduce.cuh"
#include "krylov_dev.cuh"
#include "df.cuh"

#include <math.h>

namespace adr {

static inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Blocks of the Gram-Schmidt passes: these stream the basis from memory, so
// they want more resident warps than the short reductions of the coarse
// levels (reduction_blocks): one resident wave of `per_sm` 256-thread blocks
// on each of the 152 SMs, one per 1024 entries, within the partial-sum
// stride for `values` sums.
static int df_blocks(int64_t n, int values, int per_sm) {
  int64_t b = (n + 1023) / 1024;
  if (b > 152 * per_sm) b = 152 * per_sm;
  const int64_t cap = kPartialStride / values;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// Block sum of K complex double-float values per thread, in double-float up
// to the block's total (float32 shuffles and two-sums: on this GPU a float64
// instruction costs the float64 pipe's rate even with one active lane), then
// widened to float64 once per value.  Result valid in thread 0; sh must hold
// 32 K float4.
template <int K>
__device__ __forceinline__ void block_sum_df(DfSum (&re)[K], DfSum (&im)[K], float4* sh, double2 (&out)[K]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      df_add(re[k], df_shfl_down(re[k], o));
      df_add(im[k], df_shfl_down(im[k], o));
    }
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[wid * K + k] = make_float4(re[k].s, re[k].t, im[k].s, im[k].t);
  }
  __syncthreads();
  __shared__ double2 s_tot[K];
  if (wid == 0) {
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      const float4 v = lane < nw ? sh[lane * K + k] : make_float4(0.f, 0.f, 0.f, 0.f);
      DfSum a{v.x, v.y}, b{v.z, v.w};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {   // the total lands in lane 0
        df_add(a, df_shfl_down(a, o));
        df_add(b, df_shfl_down(b, o));
      }
      if (lane == 0) s_tot[k] = make_double2(df_double(a), df_double(b));
    }
    __syncwarp();
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) out[k] = s_tot[k];
    }
  }
}

// Block partials of conj(V_i)^T w for i < k into blk[0..k) and, when norm,
// |w|^2 into blk[k].  Four basis vectors per sweep over w (eight measured
// slower: 231 against 188 us on the 257x257x129 grid, fewer resident warps).
constexpr int kDfChunk = 4;
__device__ __forceinline__ void df_block_dots(const float2* __restrict__ V, int64_t ld, int64_t lo, int k,
                                              const float2* w, int64_t n, bool norm, double2* blk, float4* sh) {
  for (int c = 0; c < k; c += kDfChunk) {
    DfSum re[kDfChunk + 1], im[kDfChunk + 1];
#pragma unroll
    for (int q = 0; q <= kDfChunk; ++q) re[q] = im[q] = DfSum{0.f, 0.f};
    const bool nq = norm && c == 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
      const float2 wh = w[e], wl = w[e + lo];
#pragma unroll
      for (int q = 0; q < kDfChunk; ++q) {
        if (c + q < k) {
          const float2* v = V + (int64_t)(c + q) * ld + e;
          const float2 vh = __ldg(v), vl = __ldg(v + lo);
          // conj(v) w = (vr wr + vi wi) + i (vr wi - vi wr)
          df_add_prod2(re[q], vh.x, vl.x, wh.x, wl.x);
          df_add_prod2(re[q], vh.y, vl.y, wh.y, wl.y);
          df_add_prod2(im[q], vh.x, vl.x, wh.y, wl.y);
          df_add_prod2(im[q], -vh.y, -vl.y, wh.x, wl.x);
        }
      }
      if (nq) {
        df_add_prod2(re[kDfChunk], wh.x, wl.x, wh.x, wl.x);
        df_add_prod2(re[kDfChunk], wh.y, wl.y, wh.y, wl.y);
      }
    }
    double2 o[kDfChunk + 1];
    block_sum_df<kDfChunk + 1>(re, im, sh, o);
    if (threadIdx.x == 0) {
      for (int q = 0; q < kDfChunk && c + q < k; ++q) blk[c + q] = o[q];
      if (nq) blk[k] = o[kDfChunk];
    }
    __syncthreads();
  }
}

// w -= V c with the coefficients c (float64, split into float32 pairs), w
// normalised back into its two planes; |w|^2 reduced over the problem's
// blocks.  Returns true in the last block (total in nrm2->x, thread 0).
__device__ __forceinline__ bool df_update_norm(const float2* __restrict__ V, int64_t ld, int64_t lo, int k, float2* w,
                                               int64_t n, const double2* c, double2* partial, unsigned* ticket,
                                               double2* nrm2) {
  __shared__ double2 sh[32];
  __shared__ double2 blk[1];
  __shared__ float4 coef[kMaxKrylov + 1];   // -c_i: (re hi, re lo, im hi, im lo)
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const float2 r = df_split(-c[i].x), m = df_split(-c[i].y);
    coef[i] = make_float4(r.x, r.y, m.x, m.y);
  }
  __syncthreads();
  DfSum s2[1] = {DfSum{0.f, 0.f}}, zero[1] = {DfSum{0.f, 0.f}};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float2 wh = w[e], wl = w[e + lo];
    DfSum ar{wh.x, wl.x}, ai{wh.y, wl.y};
#pragma unroll 4
    for (int i = 0; i < k; ++i) {
      const float4 cc = coef[i];
      const float2* v = V + (int64_t)i * ld + e;
      const float2 vh = __ldg(v), vl = __ldg(v + lo);
      // v c = (vr cr - vi ci) + i (vr ci + vi cr)
      df_add_prod2(ar, vh.x, vl.x, cc.x, cc.y);
      df_add_prod2(ar, -vh.y, -vl.y, cc.z, cc.w);
      df_add_prod2(ai, vh.x, vl.x, cc.z, cc.w);
      df_add_prod2(ai, vh.y, vl.y, cc.x, cc.y);
    }
    const float2 r = df_pair(ar), m = df_pair(ai);
    w[e] = make_float2(r.x, m.x);
    w[e + lo] = make_float2(r.y, m.y);
    df_add_prod2(s2[0], r.x, r.y, r.x, r.y);
    df_add_prod2(s2[0], m.x, m.y, m.x, m.y);
  }
  double2 o[1];
  block_sum_df<1>(s2, zero, reinterpret_cast<float4*>(sh), o);
  if (threadIdx.x == 0) blk[0] = o[0];
  __syncthreads();
  return last_block_rt(1, blk, partial, ticket, nrm2, sh);
}

// The selective Gram-Schmidt step in four passes:
//   A: ha = V^H w, ha[k] = |w|^2; the last block takes the selective
//      decision from Pythagoras, |w - V ha|^2 = |w|^2 - |ha|^2 (V
//      orthonormal; reading M2's test, as on the coarsest grid): a single
//      pass keeps the column, writes the Arnoldi column and 1/|w'|;
//   B: w' = w - V ha, normalised on the way when the single pass holds (the
//      normalisation pass disappears), its high plane into the cycle's input;
//   C: (only if flagged) hb = V^H w'
//   D: (only if flagged) w' -= V hb, |w''|^2, the Arnoldi column from ha + hb;
//      k_df_scale then normalises (it returns at once after a single pass).
__global__ void __launch_bounds__(256, 4) k_df_dots_norm(const float2* __restrict__ V, int64_t ld, int64_t lo, int k,
                                                      const float2* w, Dims g, KrylovScratch s, ArnoldiState st, int j,
                                                      double eta2) {
  if (resolve(g)) return;
  __shared__ double2 sh[32 * (kDfChunk + 1)];
  __shared__ double2 blk[kMaxKrylov + 2];
  shift_nodes(g, V, w);
  s = scratch_at(s, blockIdx.y);
  df_block_dots(V, ld, lo, k, w, g.N, true, blk, reinterpret_cast<float4*>(sh));
  if (last_block_rt(k + 1, blk, s.partial, s.ticket, s.ha, sh) && threadIdx.x == 0)
    coarse_select_dev(s.ha, s.hb, k, eta2, arnoldi_at(st, blockIdx.y), j, 0, s.nrm2);
}

// w' = w - V ha; after a single pass also w' / |w'| and its high plane into
// cyc (when not null).
__global__ void __launch_bounds__(256, 6) k_df_update(const float2* __restrict__ V, int64_t ld, int64_t lo, int k, float2* w,
                                                   float2* cyc, Dims g, KrylovScratch s) {
  if (resolve(g)) return;
  shift_nodes(g, V, w);
  shift_nodes_opt(g, cyc);
  s = scratch_at(s, blockIdx.y);
  __shared__ float4 coef[kMaxKrylov + 1];   // -ha_i: (re hi, re lo, im hi, im lo)
  __shared__ float2 s_inv;
  __shared__ int s_norm;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const float2 r = df_split(-s.ha[i].x), m = df_split(-s.ha[i].y);
    coef[i] = make_float4(r.x, r.y, m.x, m.y);
  }
  if (threadIdx.x == 0) {
    s_norm = s.ha[k].y == 0.0;
    s_inv = df_split(s.nrm2->y);
  }
  __syncthreads();
  const bool norm = s_norm;
  const float2 inv = s_inv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.N; e += (int64_t)gridDim.x * blockDim.x) {
    const float2 wh = w[e], wl = w[e + lo];
    DfSum ar{wh.x, wl.x}, ai{wh.y, wl.y};
#pragma unroll 4
    for (int i = 0; i < k; ++i) {
      const float4 cc = coef[i];
      const float2* v = V + (int64_t)i * ld + e;
      const float2 vh = __ldg(v), vl = __ldg(v + lo);
      df_add_prod2(ar, vh.x, vl.x, cc.x, cc.y);
      df_add_prod2(ar, -vh.y, -vl.y, cc.z, cc.w);
      df_add_prod2(ai, vh.x, vl.x, cc.z, cc.w);
      df_add_prod2(ai, vh.y, vl.y, cc.x, cc.y);
    }
    float2 r = df_pair(ar), m = df_pair(ai);
    if (norm) {
      DfSum a{0.f, 0.f}, b{0.f, 0.f};
      df_add_prod2(a, r.x, r.y, inv.x, inv.y);
      df_add_prod2(b, m.x, m.y, inv.x, inv.y);
      r = df_pair(a);
      m = df_pair(b);
      if (cyc) cyc[e] = make_float2(r.x, m.x);
    }
    w[e] = make_float2(r.x, m.x);
    w[e + lo] = make_float2(r.y, m.y);
  }
}

__global__ void __launch_bounds__(256, 4) k_df_reorth_dots(const float2* __restrict__ V, int64_t ld, int64_t lo, int k,
                                                        const float2* w, Dims g, KrylovScratch s) {
  if (resolve(g)) return;
  s = scratch_at(s, blockIdx.y);
  if (s.ha[k].y == 0.0) return;   // uniform over the problem's blocks
  __shared__ double2 sh[32 * (kDfChunk + 1)];
  __shared__ double2 blk[kMaxKrylov + 2];
  shift_nodes(g, V, w);
  df_block_dots(V, ld, lo, k, w, g.N, false, blk, reinterpret_cast<float4*>(sh));
  last_block_rt(k, blk, s.partial, s.ticket, s.hb, sh);
}

__global__ void __launch_bounds__(256) k_df_reorth_update(const float2* __restrict__ V, int64_t ld, int64_t lo, int k,
                                                          float2* w, Dims g, KrylovScratch s, ArnoldiState st, int j) {
  if (resolve(g)) return;
  s = scratch_at(s, blockIdx.y);
  if (s.ha[k].y == 0.0) return;   // uniform over the problem's blocks
  shift_nodes(g, V, w);
  if (df_update_norm(V, ld, lo, k, w, g.N, s.hb, s.partial, s.ticket, s.nrm2) && threadIdx.x == 0) {
    const double s2t = s.nrm2->x;
    s.nrm2->y = s2t > 0.0 ? rsqrt(s2t) : 0.0;
    if (st.m > 0) arnoldi_column_dev(arnoldi_at(st, blockIdx.y), j, s.ha, s.hb, s2t);
  }
}

// After a second Gram-Schmidt pass: w = w / |w| (reciprocal norm from
// nrm2->y) and its high plane into cyc when cyc is not null.  After a single
// pass (ha[k].y == 0) k_df_update has normalised already: nothing to do.
__global__ void k_df_scale(float2* w, int64_t lo, const double2* __restrict__ nrm2, float2* cyc, Dims g,
                           KrylovScratch s, int k) {
  if (resolve(g)) return;
  if (scratch_at(s, blockIdx.y).ha[k].y == 0.0) return;   // uniform over the problem's blocks
  __shared__ float2 inv;
  if (threadIdx.x == 0) inv = df_split(nrm2[blockIdx.y].y);
  __syncthreads();
  shift_nodes(g, w);
  shift_nodes_opt(g, cyc);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.N; e += (int64_t)gridDim.x * blockDim.x) {
    const float2 wh = w[e], wl = w[e + lo];
    DfSum a{0.f, 0.f}, b{0.f, 0.f};
    df_add_prod2(a, wh.x, wl.x, inv.x, inv.y);
    df_add_prod2(b, wh.y, wl.y, inv.x, inv.y);
    const float2 r = df_pair(a), m = df_pair(b);
    w[e] = make_float2(r.x, m.x);
    w[e + lo] = make_float2(r.y, m.y);
    if (cyc) cyc[e] = make_float2(r.x, m.x);
  }
}

// out = r / |r| for a float64 r, as double-float planes (high plane also into
// cyc when not null): the first basis vector of a restart cycle.
__global__ void k_df_from_double(const double2* __restrict__ r, float2* out, int64_t lo, const double2* __restrict__ nrm2,
                                 float2* cyc, Dims g) {
  if (resolve(g)) return;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  shift_nodes(g, r, out);
  shift_nodes_opt(g, cyc);
  const double inv = nrm2[blockIdx.y].y;
  const double2 v = r[e];
  const float2 a = df_split(v.x * inv), b = df_split(v.y * inv);
  out[e] = make_float2(a.x, b.x);
  out[e + lo] = make_float2(a.y, b.y);
  if (cyc) cyc[e] = make_float2(a.x, b.x);
}

// x += sum_{i<k} Z_i y_i with float32 vectors Z_i (the float32 cycle's
// outputs, exact), y from st; the sum in double-float, added to the float64 x.
__global__ void k_df_combine(double2* x, const float2* __restrict__ Z, int64_t ld, int k, ArnoldiState st, Dims g) {
  if (resolve(g)) return;
  __shared__ float4 coef[kMaxKrylov];   // y_i: (re hi, re lo, im hi, im lo)
  const ArnoldiState a = arnoldi_at(st, blockIdx.y);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const float2 r = df_split(a.y[i].x), m = df_split(a.y[i].y);
    coef[i] = make_float4(r.x, r.y, m.x, m.y);
  }
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  shift_nodes(g, x, Z);
  DfSum ar{0.f, 0.f}, ai{0.f, 0.f};
  for (int i = 0; i < k; ++i) {
    const float2 z = __ldg(Z + (int64_t)i * ld + e);
    const float4 c = coef[i];
    // z y = (zr yr - zi yi) + i (zr yi + zi yr)
    df_add_prod(ar, c.x, c.y, z.x);
    df_add_prod(ar, -c.z, -c.w, z.y);
    df_add_prod(ai, c.z, c.w, z.x);
    df_add_prod(ai, c.x, c.y, z.y);
  }
  double2 v = x[e];
  v.x += df_double(ar);
  v.y += df_double(ai);
  x[e] = v;
}

void launch_df_selective(const float2* V, int64_t ld, int64_t lo, int k, float2* w, float2* cyc, const Dims& g,
                         const KrylovScratch& s, const ArnoldiState& st, int j, double eta, cudaStream_t stream) {
  // eta >= 1: the second pass always runs (as launch_cgs2)
  const double eta2 = eta < 1.0 ? eta * eta : INFINITY;
  const dim3 gdots(df_blocks(g.N, k + 2, 4), g.B), gupd(df_blocks(g.N, k + 2, 4), g.B);
  // the update holds 40 registers, so six blocks fit on an SM where the dots'
  // 64 allow four: a grid of four per SM left it at half occupancy, waiting on
  // its loads (long-scoreboard stalls; elementwise, so the grid does not
  // change its result)
  const dim3 gew(df_blocks(g.N, k + 2, 6), g.B);
  count_launches(1), k_df_dots_norm<<<gdots, 256, 0, stream>>>(V, ld, lo, k, w, g, s, st, j, eta2);
  count_launches(1), k_df_update<<<gew, 256, 0, stream>>>(V, ld, lo, k, w, cyc, g, s);
  count_launches(1), k_df_reorth_dots<<<gdots, 256, 0, stream>>>(V, ld, lo, k, w, g, s);
  count_launches(1), k_df_reorth_update<<<gupd, 256, 0, stream>>>(V, ld, lo, k, w, g, s, st, j);
  // grid-stride over one resident wave: after a single pass every block returns at once
  count_launches(1), k_df_scale<<<gupd, 256, 0, stream>>>(w, lo, s.nrm2, cyc, g, s, k);
}

void launch_df_from_double(const double2* r, float2* out, int64_t lo, const double2* nrm2, float2* cyc, const Dims& g,
                           cudaStream_t st) {
  count_launches(1), k_df_from_double<<<dim3(blocks_for(g.N, 256), g.B), 256, 0, st>>>(r, out, lo, nrm2, cyc, g);
}

void launch_df_combine(double2* x, const float2* Z, int64_t ld, int k, const ArnoldiState& st, const Dims& g,
                       cudaStream_t stream) {
  count_launches(1), k_df_combine<<<dim3(blocks_for(g.N, 256), g.B), 256, 0, stream>>>(x, Z, ld, k, st, g);
}

}  // namespace adr
