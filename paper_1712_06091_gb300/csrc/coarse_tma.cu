// Relaxation apply of the stored-stencil levels with the coefficient stream
// moved by the bulk-copy (TMA) engine.
//
// The level-1 minimal-residual apply reads ~456 B of stencil per node and
// little else; in the plain kernel each thread issues those loads itself, so
// the bytes in flight per SM are bounded by its registers (64 per thread at 4
// blocks per SM) and the kernel waits on DRAM latency.  Here every warp owns a
// stream of 32-node tiles (a tile's coefficients are one contiguous block of
// the stored layout, 13.8 KB in 3D float) and keeps two of them in shared
// memory: while it computes on one, the copy engine fills the other
// (cp.async.bulk global -> shared, completion counted on an mbarrier).  One
// block of sixteen warps per SM, one tile buffer per warp (a warp's copy is
// overlapped by the other warps' work; a two-buffer variant with eight warps
// is also built): up to sixteen tiles (221 KB) in flight per SM, independent
// of registers.  The neighbour values z still come through the read-only
// cache; each node's arithmetic is the plain kernel's (the weight's block
// sums follow this kernel's grid).
//
// Every mbarrier wait is bounded.  A warp whose wait runs out raises the
// launch's error word, waits (bounded) for its other copy, and stops; the last
// block then publishes a NaN weight, which the relaxation and the Krylov
// iteration above report as a failure.
#include <cstdint>

#include "coarse_stencil.cuh"
#include "krylov_dev.cuh"
#include "reduce.cuh"

namespace adr {

constexpr unsigned kTmaWaitSpins = 1u << 22;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on phase `parity` of an mbarrier; false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, unsigned parity) {
  for (unsigned spins = 0; spins < kTmaWaitSpins; ++spins)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}
// One bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on mbar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(mbar))
      : "memory");
}

// One point's term with the coefficients in shared memory (tile layout as in
// global memory: box entries complex, two-points imaginary only).
template <int DIM, typename T, int P>
__device__ __forceinline__ void stencil_term_smem(const C<T>* tb, const T* tr, const C<T>* __restrict__ x, int64_t j,
                                                  int64_t s1, int64_t s2, unsigned m0, unsigned m1, unsigned m2, C<T>& acc) {
  const bool in = ((m0 >> (Off<DIM, P>::o0 + 2)) & (m1 >> (Off<DIM, P>::o1 + 2)) & (m2 >> (Off<DIM, P>::o2 + 2))) & 1u;
  const C<T> xv = __ldg(x + (in ? j + Off<DIM, P>::o0 + Off<DIM, P>::o1 * s1 + Off<DIM, P>::o2 * s2 : j));
  if constexpr (PointKind<DIM, P>::two) {
    const T a = tr[PointKind<DIM, P>::part * 32];
    acc.x = fma(-a, xv.y, acc.x);
    acc.y = fma(a, xv.x, acc.y);
  } else {
    acc = cfma(tb[PointKind<DIM, P>::part * 32], xv, acc);
  }
}

// One node's stencil row from a tile in shared memory (box entries complex,
// two-points imaginary only), times the neighbour values of x.
template <int DIM, typename T, int... P>
__device__ __forceinline__ C<T> tile_dot_seq(const C<T>* __restrict__ tb, const T* __restrict__ tr, const C<T>* __restrict__ x,
                                             int64_t j, int64_t s1, int64_t s2, unsigned m0, unsigned m1, unsigned m2,
                                             std::integer_sequence<int, P...>) {
  C<T> acc[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
  (stencil_term_smem<DIM, T, P>(tb, tr, x, j, s1, s2, m0, m1, m2, acc[P & 3]), ...);
  return cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
}

// A tile refilled in segments: NSEG = 2 splits it into the box entries and
// the two-point entries; NSEG = 4 splits each of those in two (slot ranges of
// the split layout, every boundary a multiple of 256 bytes).  seg_slot(q) is
// the first complex-word slot of segment q (seg_slot(NSEG) = W).
template <int DIM, int NSEG> struct Segs {
  static constexpr int NB = Split<DIM>::NB, NT2 = Split<DIM>::NT / 2, W = Split<DIM>::W;
  static constexpr int SB = NSEG == 4 ? (NB + 1) / 2 : NB;     // box slots in the first box segment
  static constexpr int ST = NSEG == 4 ? (NT2 + 1) / 2 : NT2;   // two-point slots in the first two-point segment
  __host__ __device__ static constexpr int slot(int q) {
    return NSEG == 2 ? (q == 0 ? 0 : q == 1 ? NB : W)
                     : (q == 0 ? 0 : q == 1 ? SB : q == 2 ? NB : q == 3 ? NB + ST : W);
  }
  // the segment that holds point P's coefficient
  template <int P> __host__ __device__ static constexpr int of() {
    return !PointKind<DIM, P>::two ? (NSEG == 4 && PointKind<DIM, P>::part >= SB ? 1 : 0)
                                   : (NSEG == 2 ? 1 : (PointKind<DIM, P>::part >= 2 * ST ? 3 : 2));
  }
};

// A node's terms whose coefficients lie in segment Q.
template <int DIM, typename T, int NSEG, int Q, int P>
__device__ __forceinline__ void stencil_term_seg(const C<T>* tb, const T* tr, const C<T>* __restrict__ x, int64_t j,
                                                 int64_t s1, int64_t s2, unsigned m0, unsigned m1, unsigned m2,
                                                 C<T>& acc) {
  if constexpr (Segs<DIM, NSEG>::template of<P>() == Q) stencil_term_smem<DIM, T, P>(tb, tr, x, j, s1, s2, m0, m1, m2, acc);
}
template <int DIM, typename T, int NSEG, int Q, int... P>
__device__ __forceinline__ C<T> tile_dot_seg(const C<T>* __restrict__ tb, const T* __restrict__ tr,
                                             const C<T>* __restrict__ x, int64_t j, int64_t s1, int64_t s2, unsigned m0,
                                             unsigned m1, unsigned m2, std::integer_sequence<int, P...>) {
  C<T> acc[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
  (stencil_term_seg<DIM, T, NSEG, Q, P>(tb, tr, x, j, s1, s2, m0, m1, m2, acc[P & 3]), ...);
  return cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
}

// Tile buffers per warp for STAGES: 1 and 2 whole tiles; kHalves and
// kQuarters one tile refilled in 2 or 4 segments (each segment reissued for
// the warp's next tile as soon as it has been consumed).
constexpr int kHalves = 3;
constexpr int kQuarters = 4;
__host__ __device__ constexpr int tile_buffers(int stages) { return stages == 2 ? 2 : 1; }
__host__ __device__ constexpr int tile_segments(int stages) {
  return stages == kHalves ? 2 : (stages == kQuarters ? 4 : 0);
}

// Modes of the streamed stencil kernel.
enum { kTmaMr = 0, kTmaApply = 1, kTmaResid = 2, kTmaArnoldi = 3 };

// What the kTmaArnoldi mode's last block needs for the Arnoldi column.
struct ArnoldiTail {
  ArnoldiState st;
  double2* hb;
  double2* nrm2;
  int j, finish;
  double eta2;
};

// All lanes receive the warp's sum of v (butterfly; float for a float cycle).
template <typename T> __device__ __forceinline__ C<T> warp_allsum(C<T> v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// One pass over the level with the coefficient tiles streamed into shared
// memory.  WARPS warps per block, each with STAGES tile buffers (1: the other
// warps of the SM overlap its copy; 2: it overlaps its own; kHalves: one
// buffer whose halves are refilled separately, so the box half of the next
// tile arrives while the two-point half of this one is consumed).
//   kTmaMr:    out = A x and the partial sums of out^H aux, out^H out; the last
//              block writes the minimal-residual weight to alpha
//   kTmaApply: out = A x
//   kTmaResid: out = aux - A x, out2 = dinv .* out
//   kTmaArnoldi: out = A x and the first Gram-Schmidt pass of an Arnoldi step,
//              ha[i] = sum_e conj(V_i[e]) out[e] for i < kd and ha[kd] =
//              |out|^2 (kd <= 63): each tile's products are summed over the
//              warp, lane i (and i - 32) keeps value i's running sum over the
//              warp's tiles (float32: a coarsest level gives a warp a few
//              tiles), the warps add theirs in float64 in warp order, the last block
//              adds the blocks' in block order (deterministic for a given
//              grid) and takes the selective decision (coarse_select_block)
template <int DIM, typename T, bool BT, int WARPS, int STAGES, int MODE>
__global__ void __launch_bounds__(WARPS * 32, 1)
    k_stencil_tma(Dims g, const C<T>* __restrict__ A, const C<T>* __restrict__ x, const C<T>* __restrict__ aux,
                  C<T>* __restrict__ out, const C<T>* __restrict__ dinv, C<T>* __restrict__ out2, double2* partial,
                  unsigned* ticket, double2* alpha, int* err, const C<T>* __restrict__ V, int64_t ld, int kd,
                  ArnoldiTail tail) {
  constexpr int W = Split<DIM>::W, NB = Split<DIM>::NB, S = PatternSize<DIM>::value;
  constexpr unsigned kTileBytes = W * 32 * sizeof(C<T>);
  extern __shared__ __align__(128) unsigned char tma_smem[];
  __shared__ __align__(8) uint64_t mbar[WARPS][4];
  __shared__ double2 sh[32 * 2];
  __shared__ int s_fail;
  if (BT) {
    if (resolve(g)) return;
    shift_stencil(g, A);
    shift_nodes(g, x, aux, out);
    shift_nodes_opt(g, dinv, out2, V);
    batch_shift_opt(kPartialStride, partial);
    batch_shift_opt(1, ticket);
    batch_shift_opt(MODE == kTmaArnoldi ? kMaxArnoldiDots : 1, alpha);
    if constexpr (MODE == kTmaArnoldi) {
      tail.hb += (int64_t)blockIdx.y * kMaxArnoldiDots;
      tail.nrm2 += blockIdx.y;
    }
    batch_shift(1, err);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NSEG = tile_segments(STAGES);   // 0: whole-tile copies
  using SG = Segs<DIM, NSEG == 0 ? 2 : NSEG>;
  C<T>* const buf0 = reinterpret_cast<C<T>*>(tma_smem) + (size_t)warp * tile_buffers(STAGES) * W * 32;
  C<T>* const buf1 = buf0 + (STAGES == 2 ? W * 32 : 0);
  if (threadIdx.x == 0) s_fail = 0;
  if (lane == 0) {
    for (int q = 0; q < (NSEG ? NSEG : STAGES); ++q) mbar_init(&mbar[warp][q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int64_t ntiles = (g.N + 31) >> 5;
  const int64_t stride = (int64_t)gridDim.x * WARPS;
  const int64_t t0 = (int64_t)blockIdx.x * WARPS + warp;
  unsigned pending = 0u;   // bit s: stage s has a copy issued and not yet consumed (warp-uniform)
  auto issue = [&](int64_t t, int s) {
    if (t < ntiles) {
      if (lane == 0) {
        mbar_expect_tx(&mbar[warp][s], kTileBytes);
        bulk_load(s ? buf1 : buf0, A + t * (int64_t)W * 32, kTileBytes, &mbar[warp][s]);
      }
      pending |= 1u << s;
    }
  };
  // segment q of tile t into its place in buf0, on mbar[warp][q]
  auto issue_seg = [&](int64_t t, int q) {
    if (t < ntiles) {
      if (lane == 0) {
        const size_t off = (size_t)SG::slot(q) * 32;
        const unsigned bytes = (unsigned)((SG::slot(q + 1) - SG::slot(q)) * 32 * sizeof(C<T>));
        mbar_expect_tx(&mbar[warp][q], bytes);
        bulk_load(buf0 + off, A + t * (int64_t)W * 32 + off, bytes, &mbar[warp][q]);
      }
      pending |= 1u << q;
    }
  };
  if constexpr (NSEG > 0) {
    for (int q = 0; q < NSEG; ++q) issue_seg(t0, q);
  } else {
    issue(t0, 0);
    if (STAGES > 1) issue(t0 + stride, 1);
  }
  unsigned phase = 0u;   // bit s: parity of stage s's next completion
  bool fail = false;
  C<T> sacc[2] = {czero<T>(), czero<T>()};
  C<T> facc0 = czero<T>(), facc1 = czero<T>();   // kTmaArnoldi: running sums of values lane, lane + 32
  int s = 0;
  int64_t t = t0;
  for (; t < ntiles; t += stride, s = STAGES == 2 ? s ^ 1 : 0) {
    const int64_t j = t * 32 + lane;
    C<T> axw = czero<T>();
    if constexpr (NSEG > 0) {
      // each segment: wait, add its terms, reissue it for the warp's next tile
      int i0 = 0, i1 = 0, i2 = 0;
      unsigned m0 = 0u, m1 = 0u, m2 = 0u;
      if (j < g.N) {
        unravel(g, j, i0, i1, i2);
        m0 = axis_mask(i0, g.n[0]);
        m1 = axis_mask(i1, g.n[1]);
        m2 = DIM > 2 ? axis_mask(i2, g.n[2]) : 4u;
      }
      const C<T>* tb = buf0 + lane;
      const T* tr = reinterpret_cast<const T*>(buf0 + NB * 32) + lane;
      auto segment = [&](auto qc) -> bool {
        constexpr int q = decltype(qc)::value;
        if (!mbar_wait(&mbar[warp][q], (phase >> q) & 1u)) fail = true;
        fail = __any_sync(0xffffffffu, fail);
        if (fail) return false;
        phase ^= 1u << q;
        pending &= ~(1u << q);
        if (j < g.N)
          axw = cadd(axw, tile_dot_seg<DIM, T, NSEG == 0 ? 2 : NSEG, q>(tb, tr, x, j, g.s1, g.s2, m0, m1, m2,
                                                                        std::make_integer_sequence<int, S>{}));
        __syncwarp();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_seg(t + stride, q);
        return true;
      };
      bool ok = segment(std::integral_constant<int, 0>{}) && segment(std::integral_constant<int, 1>{});
      if constexpr (NSEG == 4)
        ok = ok && segment(std::integral_constant<int, 2>{}) && segment(std::integral_constant<int, 3>{});
      if (!ok) break;
    } else {
      if (!mbar_wait(&mbar[warp][s], (phase >> s) & 1u)) fail = true;
      fail = __any_sync(0xffffffffu, fail);
      if (fail) break;
      phase ^= 1u << s;
      pending &= ~(1u << s);
      if (j < g.N) {
        int i0, i1, i2;
        unravel(g, j, i0, i1, i2);
        const unsigned m0 = axis_mask(i0, g.n[0]), m1 = axis_mask(i1, g.n[1]), m2 = DIM > 2 ? axis_mask(i2, g.n[2]) : 4u;
        const C<T>* bs = s ? buf1 : buf0;
        const C<T>* tb = bs + lane;
        const T* tr = reinterpret_cast<const T*>(bs + NB * 32) + lane;
        axw = tile_dot_seq<DIM, T>(tb, tr, x, j, g.s1, g.s2, m0, m1, m2, std::make_integer_sequence<int, S>{});
      }
    }
    if (j < g.N) {
      const C<T> ax = axw;
      if constexpr (MODE == kTmaArnoldi) {
        out[j] = ax;
      } else if constexpr (MODE == kTmaMr) {
        out[j] = ax;
        sacc[0] = cfma_conj(ax, aux[j], sacc[0]);
        sacc[1] = cfma_conj(ax, ax, sacc[1]);
      } else if constexpr (MODE == kTmaApply) {
        out[j] = ax;
      } else {
        const C<T> rj = csub(aux[j], ax);
        out[j] = rj;
        out2[j] = cmul(dinv[j], rj);
      }
    }
    if constexpr (MODE == kTmaArnoldi) {
      // Value i < kd: conj(V_i) . Ax over the tile; value kd: |Ax|^2.  Eight
      // values per round: their basis entries are all loaded before any
      // reduction, and their eight butterflies interleave.
      for (int i0 = 0; i0 <= kd; i0 += 8) {
        C<T> p[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 + q;
          C<T> vi = czero<T>();
          if (i < kd) {
            if (j < g.N) vi = V[(int64_t)i * ld + j];
          } else if (i == kd) {
            vi = axw;
          }
          p[q] = cfma_conj(vi, axw, czero<T>());
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            p[q].x += __shfl_xor_sync(0xffffffffu, p[q].x, o);
            p[q].y += __shfl_xor_sync(0xffffffffu, p[q].y, o);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 + q;
          if (i <= kd && lane == (i & 31)) {
            C<T>& d = i < 32 ? facc0 : facc1;
            d.x += p[q].x;
            d.y += p[q].y;
          }
        }
      }
    }
    if constexpr (NSEG == 0) {
      __syncwarp();
      // the generic-proxy reads of the buffer are done before the copy engine refills it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + STAGES * stride, s);
    }
  }
  if (fail) {
    // wait (bounded) for this warp's copies still in flight (only stages with
    // an issued, unconsumed copy), mark the failure: the weight (kTmaMr) or the
    // tiles this warp did not compute become NaN.  A copy can still be
    // outstanding when the warp leaves only if this second wait also runs out.
    for (int q = 0; q < (NSEG ? NSEG : STAGES); ++q)
      if ((pending >> q) & 1u) mbar_wait(&mbar[warp][q], (phase >> q) & 1u);
    if (lane == 0) {
      atomicExch(err, 1);
      s_fail = 1;
    }
    if constexpr (MODE != kTmaMr) {
      const C<T> nan = mk<T>((T)NAN, (T)NAN);
      for (; t < ntiles; t += stride) {
        const int64_t j = t * 32 + lane;
        if (j < g.N) {
          out[j] = nan;
          if constexpr (MODE == kTmaResid) out2[j] = nan;
        }
      }
    }
  }
  if constexpr (MODE == kTmaArnoldi) {
    // Every warp is past its tiles: the tile buffers are scratch from here on.
    // The warps' running sums go to shared memory and one thread per value
    // adds them in warp order (float64).
    const int nv = kd + 1;
    __shared__ double2 s_dots[kMaxArnoldiDots];
    __syncthreads();
    C<T>* wsum = reinterpret_cast<C<T>*>(tma_smem);   // [WARPS][64]
    wsum[warp * 64 + lane] = facc0;
    wsum[warp * 64 + 32 + lane] = facc1;
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
      for (int w = 0; w < WARPS; ++w) {
        const C<T> v = wsum[w * 64 + i];
        acc.x += (double)v.x;
        acc.y += (double)v.y;
      }
      s_dots[i] = acc;
    }
    __syncthreads();
    if (last_block_rt(nv, s_dots, partial, ticket, alpha, sh)) {   // uniform over the block
      if (threadIdx.x == 0 && (*(volatile int*)err != 0 || s_fail))
        for (int i = 0; i < nv; ++i) alpha[i] = make_double2(NAN, NAN);
      __syncthreads();
      const ArnoldiState ast = arnoldi_at(tail.st, blockIdx.y);
      constexpr size_t kScratch = (size_t)WARPS * tile_buffers(STAGES) * W * 32 * sizeof(C<T>);   // dynamic smem
      constexpr size_t kSums = (size_t)WARPS * 64 * sizeof(C<T>);
      if (kSums + (size_t)arnoldi_stage_words(ast.m, kd) * sizeof(double2) <= kScratch) {
        double2* stage = reinterpret_cast<double2*>(tma_smem + kSums);
        coarse_select_block(alpha, tail.hb, kd, tail.eta2, ast, tail.j, tail.finish, tail.nrm2, stage);
      } else if (threadIdx.x == 0) {   // a long basis on a 2D level: the state does not fit beside the sums
        coarse_select_dev(alpha, tail.hb, kd, tail.eta2, ast, tail.j, tail.finish, tail.nrm2);
      }
    }
  }
  if constexpr (MODE == kTmaMr) {
    double2 mine[2], tot[2];
    block_sum_t<T, 2>(sacc, sh, mine);
    if (last_block_total<2>(mine, partial, ticket, tot, sh) && threadIdx.x == 0) {
      const double den = tot[1].x;
      const bool bad = *(volatile int*)err != 0 || s_fail;
      *alpha = bad ? make_double2(NAN, NAN)
                   : (den > 0.0 ? make_double2(tot[0].x / den, tot[0].y / den) : make_double2(0.0, 0.0));
    }
  }
}

template <int DIM, int WARPS, int STAGES> constexpr size_t tma_smem_bytes() {
  return (size_t)WARPS * tile_buffers(STAGES) * Split<DIM>::W * 32 * sizeof(float2);
}
template <int DIM, int WARPS, int STAGES, int MODE> static bool tma_attr_mode() {
  constexpr int bytes = (int)tma_smem_bytes<DIM, WARPS, STAGES>();
  return cudaFuncSetAttribute(k_stencil_tma<DIM, float, false, WARPS, STAGES, MODE>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&
         cudaFuncSetAttribute(k_stencil_tma<DIM, float, true, WARPS, STAGES, MODE>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
}
template <int DIM, int WARPS, int STAGES> static bool tma_attr() {
  return tma_attr_mode<DIM, WARPS, STAGES, kTmaMr>() && tma_attr_mode<DIM, WARPS, STAGES, kTmaApply>() &&
         tma_attr_mode<DIM, WARPS, STAGES, kTmaResid>() && tma_attr_mode<DIM, WARPS, STAGES, kTmaArnoldi>();
}

// Opts the kernels into their dynamic shared memory (call outside capture);
// returns false if the device cannot give it.
bool prepare_stencil_tma() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if ((size_t)optin < tma_smem_bytes<3, 16, 1>() + 2048 || (size_t)optin < tma_smem_bytes<3, 8, 2>() + 2048) return false;
  const bool ok = tma_attr<3, 8, 2>() && tma_attr<2, 8, 2>() && tma_attr<3, 16, 1>() && tma_attr<2, 16, 1>() &&
                  tma_attr<3, 16, kHalves>() && tma_attr<2, 16, kHalves>() && tma_attr<3, 16, kQuarters>() &&
                  tma_attr<2, 16, kQuarters>();
  cudaGetLastError();
  return ok;
}

template <int DIM, int WARPS, int STAGES, int MODE>
static void launch_tma(const Dims& g, const float2* A, const float2* x, const float2* aux, float2* out,
                       const float2* dinv, float2* out2, double2* partial, unsigned* ticket, double2* alpha, int* err,
                       int blocks, cudaStream_t st, const float2* V = nullptr, int64_t ld = 0, int kd = 0,
                       ArnoldiTail tail = ArnoldiTail{}) {
  const int64_t ntiles = (g.N + 31) >> 5;
  int64_t nb = (ntiles + WARPS - 1) / WARPS;
  if (nb > blocks) nb = blocks;
  if (nb < 1) nb = 1;
  const dim3 grid((unsigned)nb, g.B);
  constexpr size_t smem = tma_smem_bytes<DIM, WARPS, STAGES>();
  count_launches(1), (g.B > 1 ? k_stencil_tma<DIM, float, true, WARPS, STAGES, MODE>
                              : k_stencil_tma<DIM, float, false, WARPS, STAGES, MODE>)
                         <<<grid, WARPS * 32, smem, st>>>(g, A, x, aux, out, dinv, out2, partial, ticket, alpha, err, V,
                                                          ld, kd, tail);
}

template <int MODE>
static void launch_variant(const Dims& g, const float2* A, const float2* x, const float2* aux, float2* out,
                           const float2* dinv, float2* out2, double2* partial, unsigned* ticket, double2* alpha,
                           int* err, int blocks, int variant, cudaStream_t st, const float2* V = nullptr, int64_t ld = 0,
                           int kd = 0, ArnoldiTail tail = ArnoldiTail{}) {
  if (variant == 2) {
    if (g.dim == 2)
      launch_tma<2, 8, 2, MODE>(g, A, x, aux, out, dinv, out2, partial, ticket, alpha, err, blocks, st, V, ld, kd, tail);
    else
      launch_tma<3, 8, 2, MODE>(g, A, x, aux, out, dinv, out2, partial, ticket, alpha, err, blocks, st, V, ld, kd, tail);
  } else if (variant == 4) {
    if (g.dim == 2)
      launch_tma<2, 16, kQuarters, MODE>(g, A, x, aux, out, dinv, out2, partial, ticket, alpha, err, blocks, st, V, ld,
                                         kd, tail);
    else
      launch_tma<3, 16, kQuarters, MODE>(g, A, x, aux, out, dinv, out2, partial, ticket, alpha, err, blocks, st, V, ld,
                                         kd, tail);
  } else if (variant == 3) {
    if (g.dim == 2)
      launch_tma<2, 16, kHalves, MODE>(g, A, x, aux, out, dinv, out2, partial, ticket, alpha, err, blocks, st, V, ld, kd,
                                       tail);
    else
      launch_tma<3, 16, kHalves, MODE>(g, A, x, aux, out, dinv, out2, partial, ticket, alpha, err, blocks, st, V, ld, kd,
                                       tail);
  } else {
    if (g.dim == 2)
      launch_tma<2, 16, 1, MODE>(g, A, x, aux, out, dinv, out2, partial, ticket, alpha, err, blocks, st, V, ld, kd, tail);
    else
      launch_tma<3, 16, 1, MODE>(g, A, x, aux, out, dinv, out2, partial, ticket, alpha, err, blocks, st, V, ld, kd, tail);
  }
}

// variant 1: 16 warps per block, one tile buffer each (96 us per level-1
// relaxation launch of the 257x257x129 workload); variant 2: 8 warps, two
// buffers each (98 us); variant 3: 16 warps, one buffer each refilled in
// halves, the box half reissued for the next tile before the two-point half
// is consumed (92 us; the library default); the plain-load kernel takes 115 us.
void launch_stencil_mr_apply_tma(const Dims& g, const float2* A, const float2* z, const float2* r, float2* w,
                                 double2* partial, unsigned* ticket, double2* alpha, int* err, int blocks, int variant,
                                 cudaStream_t st) {
  launch_variant<kTmaMr>(g, A, z, r, w, nullptr, nullptr, partial, ticket, alpha, err, blocks, variant, st);
}
void launch_stencil_apply_tma(const Dims& g, const float2* A, const float2* x, float2* y, int* err, int blocks,
                              int variant, cudaStream_t st) {
  launch_variant<kTmaApply>(g, A, x, x, y, nullptr, nullptr, nullptr, nullptr, nullptr, err, blocks, variant, st);
}
void launch_stencil_arnoldi_tma(const Dims& g, const float2* A, const float2* z, float2* w, const float2* V, int64_t ld,
                                int kd, const KrylovScratch& s, const ArnoldiState& st, int j, int finish, double eta,
                                int* err, int blocks, int variant, cudaStream_t stream) {
  ArnoldiTail tail{st, s.hb, s.nrm2, j, finish, eta * eta};
  // whole tiles on the coarsest grid: a warp there takes one or two tiles, too
  // few for the refill in halves to pay (386 against 376 us per coarsest solve)
  launch_variant<kTmaArnoldi>(g, A, z, z, w, nullptr, nullptr, s.partial, s.ticket, s.ha, err, blocks,
                              variant >= 3 ? 1 : variant, stream, V, ld, kd, tail);
}
void launch_stencil_residual_dinv_tma(const Dims& g, const float2* A, const float2* b, const float2* x,
                                      const float2* dinv, float2* r, float2* z, int* err, int blocks, int variant,
                                      cudaStream_t st) {
  launch_variant<kTmaResid>(g, A, x, b, r, dinv, z, nullptr, nullptr, nullptr, err, blocks, variant, st);
}

}  // namespace adr
