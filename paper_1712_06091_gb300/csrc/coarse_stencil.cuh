// Apply of a stored Galerkin stencil at one node (shared by the coarse-level
// kernels and the cluster coarsest-grid solver).
#pragma once

#include <utility>

#include "adr_common.cuh"

namespace adr {

// Pattern offsets as compile-time constants (for the unrolled loop below).
struct PatternConst {
  static constexpr PatternTables t = make_pattern_tables();
};
template <int DIM, int P> struct Off {
  static constexpr int o0 = DIM == 2 ? PatternConst::t.off2[P][0] : PatternConst::t.off3[P][0];
  static constexpr int o1 = DIM == 2 ? PatternConst::t.off2[P][1] : PatternConst::t.off3[P][1];
  static constexpr int o2 = DIM == 2 ? 0 : PatternConst::t.off3[P][2];
};

// Bit (o + 2) of the returned mask is set when offset o in [-2, 2] stays on
// an axis of n nodes from index i.
__device__ __forceinline__ unsigned axis_mask(int i, int n) {
  unsigned m = 0;
#pragma unroll
  for (int o = -2; o <= 2; ++o) m |= ((unsigned)(i + o) < (unsigned)n) ? (1u << (o + 2)) : 0u;
  return m;
}

// Layout of a stored stencil: nodes are grouped in tiles of 32 (one warp);
// a tile keeps its S points' coefficients together, point-major inside the
// tile, so a warp streams one contiguous 32*S-entry segment (locality in the
// DRAM pages instead of S scattered streams).  Entry (p, j) lives at
// ((j / 32) * S + p) * 32 + j % 32; arrays hold S * round_up(N, 32) entries.
__host__ __device__ __forceinline__ int64_t stencil_index(int p, int64_t j, int S) {
  return (((j >> 5) * S + p) << 5) + (j & 31);
}
__host__ __device__ __forceinline__ int64_t stencil_entries(int64_t N, int S) { return ((N + 31) >> 5) * 32 * S; }

// sum_p A[p][j] x[j + o_p], unrolled over the pattern with compile-time
// offsets and no branch: a neighbour off the grid is replaced by node j
// itself, whose product with the (exactly zero) Galerkin coefficient of that
// point adds nothing.  All loads can be issued back to back; four partial
// sums break the dependent FMA chain.
// x loads: read-only path (__ldg) when x is constant for the whole kernel;
// COH (x rewritten by other blocks or CTAs of the same launch between
// barriers): ordinary coherent loads, which the acquire side of those
// barriers orders after the writers' release (no read-only path).
template <bool COH, typename V> __device__ __forceinline__ V load_x(const V* p) {
  if constexpr (COH) return *p;
  else return __ldg(p);
}

template <int DIM, typename T, bool COH, int... P>
__device__ __forceinline__ C<T> stencil_dot_seq(const C<T>* __restrict__ A, const C<T>* __restrict__ x, int64_t j,
                                                int64_t N, int64_t s1, int64_t s2, unsigned m0, unsigned m1, unsigned m2,
                                                std::integer_sequence<int, P...>) {
  C<T> acc[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
  const C<T>* Aj = A + stencil_index(0, j, (int)sizeof...(P));
  ((acc[P & 3] = cfma(__ldg(Aj + P * 32),
                      load_x<COH>(x + ((((m0 >> (Off<DIM, P>::o0 + 2)) & (m1 >> (Off<DIM, P>::o1 + 2)) &
                                         (m2 >> (Off<DIM, P>::o2 + 2))) & 1u)
                                           ? j + Off<DIM, P>::o0 + Off<DIM, P>::o1 * s1 + Off<DIM, P>::o2 * s2
                                           : j)),
                      acc[P & 3])),
   ...);
  return cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
}

template <int DIM, typename T, bool COH = false>
__device__ __forceinline__ C<T> stencil_dot(const Dims& g, const C<T>* __restrict__ A, const C<T>* __restrict__ x,
                                            int64_t j, int i0, int i1, int i2) {
  constexpr int S = PatternSize<DIM>::value;
  const unsigned m0 = axis_mask(i0, g.n[0]), m1 = axis_mask(i1, g.n[1]), m2 = DIM > 2 ? axis_mask(i2, g.n[2]) : 4u;
  return stencil_dot_seq<DIM, T, COH>(A, x, j, g.N, g.s1, g.s2, m0, m1, m2, std::make_integer_sequence<int, S>{});
}

}  // namespace adr
