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

// Layout of a stored stencil.  The Galerkin entries at the "two-points" (an
// offset of +-2 along one axis) are purely imaginary: they arise only from
// the fine second-order upwind entries at +-2, which are i * real (Eq.
// londUpwindDiff), through the real weights of P (an entry at coarse offset
// +-2 needs a fine offset of +-2), and so on down the hierarchy.  Only their
// imaginary parts are stored: per node NB complex box entries (|o| <= 1) and
// NT reals, 54 complex-sized words per node in 3D instead of 81 (15 for 21
// in 2D).
//
// Nodes are grouped in tiles of 32 (one warp), point-major inside the tile,
// so a warp streams one contiguous segment: in units of C<T>, tile t starts
// at t * W * 32; box entry b of lane l at + b * 32 + l; the reals follow the
// box entries (two-point q of lane l at real offset 2 * NB * 32 + q * 32 + l
// from the tile start, in units of T).
template <int DIM> struct Split {
  static constexpr int S = PatternSize<DIM>::value;
  static constexpr int NB = DIM == 2 ? 9 : 27;
  static constexpr int NT = S - NB;
  static constexpr int W = NB + NT / 2;
  static_assert(NT % 2 == 0, "two-point reals fill whole complex words");
};
static_assert(Split<2>::W == 15 && Split<3>::W == 54, "stencil_words");
__host__ __device__ __forceinline__ int64_t stencil_entries(int64_t N, int S) {
  return ((N + 31) >> 5) * 32 * (S == kPattern2 ? Split<2>::W : Split<3>::W);
}

// Entry p (pattern order) of node j, and its store (the real part of a
// two-point, exactly zero, is not kept).
template <int DIM, typename T> __device__ __forceinline__ C<T> stencil_get(const C<T>* A, int p, int64_t j) {
  const C<T>* tile = A + (j >> 5) * (int64_t)Split<DIM>::W * 32;
  const int lane = (int)(j & 31);
  if (!pattern_two<DIM>(p)) return tile[pattern_part<DIM>(p) * 32 + lane];
  const T* re = reinterpret_cast<const T*>(tile + Split<DIM>::NB * 32);
  return mk<T>(T(0), re[pattern_part<DIM>(p) * 32 + lane]);
}
template <int DIM, typename T> __device__ __forceinline__ void stencil_put(C<T>* A, int p, int64_t j, C<T> v) {
  C<T>* tile = A + (j >> 5) * (int64_t)Split<DIM>::W * 32;
  const int lane = (int)(j & 31);
  if (!pattern_two<DIM>(p)) {
    tile[pattern_part<DIM>(p) * 32 + lane] = v;
  } else {
    T* re = reinterpret_cast<T*>(tile + Split<DIM>::NB * 32);
    re[pattern_part<DIM>(p) * 32 + lane] = v.y;
  }
}

// x loads: read-only path (__ldg) when x is constant for the whole kernel;
// COH (x rewritten by other blocks or CTAs of the same launch between
// barriers): ordinary coherent loads, which the acquire side of those
// barriers orders after the writers' release (no read-only path).
template <bool COH, typename V> __device__ __forceinline__ V load_x(const V* p) {
  if constexpr (COH) return *p;
  else return __ldg(p);
}

template <int DIM, int P> struct PointKind {
  static constexpr bool two = DIM == 2 ? PatternConst::t.two2[P] != 0 : PatternConst::t.two3[P] != 0;
  static constexpr int part = DIM == 2 ? PatternConst::t.part2[P] : PatternConst::t.part3[P];
};

// One point's term: box points a complex product, two-points (0 + i a) x.
template <int DIM, typename T, bool COH, int P>
__device__ __forceinline__ void stencil_term(const C<T>* __restrict__ Ab, const T* __restrict__ Rb, const C<T>* __restrict__ x,
                                             int64_t j, int64_t s1, int64_t s2, unsigned m0, unsigned m1, unsigned m2,
                                             C<T>& acc) {
  const bool in = ((m0 >> (Off<DIM, P>::o0 + 2)) & (m1 >> (Off<DIM, P>::o1 + 2)) & (m2 >> (Off<DIM, P>::o2 + 2))) & 1u;
  const C<T> xv = load_x<COH>(x + (in ? j + Off<DIM, P>::o0 + Off<DIM, P>::o1 * s1 + Off<DIM, P>::o2 * s2 : j));
  if constexpr (PointKind<DIM, P>::two) {
    const T a = __ldg(Rb + PointKind<DIM, P>::part * 32);
    acc.x = fma(-a, xv.y, acc.x);
    acc.y = fma(a, xv.x, acc.y);
  } else {
    acc = cfma(__ldg(Ab + PointKind<DIM, P>::part * 32), xv, acc);
  }
}

// sum_p A[p][j] x[j + o_p], unrolled over the pattern with compile-time
// offsets and no branch: a neighbour off the grid is replaced by node j
// itself, whose product with the (exactly zero) Galerkin coefficient of that
// point adds nothing.  All loads can be issued back to back; four partial
// sums break the dependent FMA chain.
template <int DIM, typename T, bool COH, int... P>
__device__ __forceinline__ C<T> stencil_dot_seq(const C<T>* __restrict__ A, const C<T>* __restrict__ x, int64_t j,
                                                int64_t N, int64_t s1, int64_t s2, unsigned m0, unsigned m1, unsigned m2,
                                                std::integer_sequence<int, P...>) {
  C<T> acc[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
  const C<T>* tile = A + (j >> 5) * (int64_t)Split<DIM>::W * 32;
  const int lane = (int)(j & 31);
  const C<T>* Ab = tile + lane;
  const T* Rb = reinterpret_cast<const T*>(tile + Split<DIM>::NB * 32) + lane;
  (stencil_term<DIM, T, COH, P>(Ab, Rb, x, j, s1, s2, m0, m1, m2, acc[P & 3]), ...);
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
