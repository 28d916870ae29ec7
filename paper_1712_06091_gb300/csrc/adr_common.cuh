// Internal declarations shared by the CUDA translation units of libadr.
//
// Data layout in device memory (one arena per operator):
//   * complex vectors: interleaved (re, im) of T = double or float, i.e.
//     double2 / float2 per node, node j = i0 + n0*(i1 + n1*i2);
//   * fine-level coefficients (matrix-free level): structure of arrays
//     g[d][N] = d_d tau, t[d][N] = d_dd tau, rho[N] (complex reaction);
//   * Galerkin levels: point-major stencils A[p][N] (p over the 21 / 81
//     offsets of the coarse pattern), plus the inverse diagonal dinv[N].
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

#include "adr.h"

namespace adr {

// ---------------------------------------------------------------------------
// Complex helpers on double2 / float2
// ---------------------------------------------------------------------------
template <typename T> struct cvec;
template <> struct cvec<double> { using type = double2; };
template <> struct cvec<float> { using type = float2; };
template <typename T> using C = typename cvec<T>::type;

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T re, T im) {
  C<T> z; z.x = re; z.y = im; return z;
}
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) {
  V z; z.x = a.x + b.x; z.y = a.y + b.y; return z;
}
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) {
  V z; z.x = a.x - b.x; z.y = a.y - b.y; return z;
}
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
  V z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
// acc + a * b
template <typename V> __host__ __device__ __forceinline__ V cfma(V a, V b, V acc) {
  V z;
  z.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  z.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
  return z;
}
// acc + conj(a) * b
template <typename V> __host__ __device__ __forceinline__ V cfma_conj(V a, V b, V acc) {
  V z;
  z.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  z.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
  return z;
}
template <typename V, typename T> __host__ __device__ __forceinline__ V cscale(V a, T s) {
  V z; z.x = a.x * s; z.y = a.y * s; return z;
}
template <typename V> __host__ __device__ __forceinline__ V cinv(V a) {
  // 1 / a, scaled to avoid overflow in |a|^2
  auto m = fabs(a.x) > fabs(a.y) ? fabs(a.x) : fabs(a.y);
  V b; b.x = a.x / m; b.y = a.y / m;
  auto d = (b.x * b.x + b.y * b.y) * m;
  V z; z.x = b.x / d; z.y = -b.y / d; return z;
}
template <typename T> __host__ __device__ __forceinline__ C<T> czero() { return mk<T>(T(0), T(0)); }

template <typename Dst, typename Src> __host__ __device__ __forceinline__ Dst ccast(Src a) {
  Dst z; z.x = a.x; z.y = a.y; return z;
}

// ---------------------------------------------------------------------------
// Grid descriptor
// ---------------------------------------------------------------------------
// One problem's grid inside a batch whose problems have grids (and spacings)
// of their own: its shape, the index-division constants, where its entries
// start in the batch's node arrays and in its stored stencils, its spacing.
struct ProblemDims {
  int n[3];
  int64_t N, s1, s2;
  unsigned mul0, mul1;
  int shr0, shr1;
  int64_t off;     // first node entry: the earlier problems' N summed
  int64_t soff;    // first stored-stencil entry: the earlier problems' stencil entries summed
  double h[3];
};

struct Dims {
  int dim;
  int n[3];
  int64_t N;       // nodes of one problem; for per-problem grids (pd) the largest, which sizes launches
  int64_t s1, s2;  // strides of axes 1 and 2
  int B;           // problems in a batched launch (grid.y)
  int mrcap;       // largest grid of the relaxation applies (0: kMaxMrBlocks)
  unsigned mul0, mul1;  // division by n[0], n[1] as a multiply and a shift (fast_div_params)
  int shr0, shr1;
  const ProblemDims* pd;  // device table of per-problem grids; nullptr: every problem has this grid
  const int* skip;        // per problem: nonzero = frozen, its blocks return at once (nullptr: none)
  int64_t total;          // node entries of one vector over all problems
  int64_t off, soff;      // after resolve(): the block's problem's first node / stencil entry
};

// Entries of a stored Galerkin stencil for N nodes (32-node tiles of W words
// of the element type: 27 complex + 54 imaginary-only reals in 3D, 9 + 12 in 2D).
__host__ __device__ __forceinline__ int64_t stencil_words(int dim) { return dim == 2 ? 15 : 54; }
__host__ __device__ __forceinline__ int64_t stencil_entries_dim(int64_t N, int dim) {
  return ((N + 31) >> 5) * 32 * stencil_words(dim);
}

// The grid of the calling block's problem (blockIdx.y): its shape and the
// first entries of its slices of the batch's arrays.  Every kernel calls it
// before using g and returns at once when it answers true: the problem is
// frozen (a batch member that already met its tolerance), so the whole
// block, and every block of that problem, skips the launch.
__device__ __forceinline__ bool resolve(Dims& g) {
  const int p = blockIdx.y;
  if (g.skip && g.skip[p]) return true;
  if (g.pd == nullptr) {
    g.off = (int64_t)p * g.N;
    g.soff = (int64_t)p * stencil_entries_dim(g.N, g.dim);
    return false;
  }
  const ProblemDims& q = g.pd[p];
  g.n[0] = q.n[0]; g.n[1] = q.n[1]; g.n[2] = q.n[2];
  g.N = q.N; g.s1 = q.s1; g.s2 = q.s2;
  g.mul0 = q.mul0; g.mul1 = q.mul1; g.shr0 = q.shr0; g.shr1 = q.shr1;
  g.off = q.off;
  g.soff = q.soff;
  return false;
}
// resolve() for a batch known to share one grid (no table): only the skip
// test and the offsets, so the shape stays in the launch parameters.
__device__ __forceinline__ bool resolve_uniform(Dims& g) {
  const int p = blockIdx.y;
  if (g.skip && g.skip[p]) return true;
  g.off = (int64_t)p * g.N;
  g.soff = (int64_t)p * stencil_entries_dim(g.N, g.dim);
  return false;
}

// Pointers moved to the block's problem's slice (node arrays, node arrays of
// `k` entries per node, stored stencils); the _opt forms leave nullptr alone.
template <typename... P> __device__ __forceinline__ void shift_nodes(const Dims& g, P&... p) { ((p += g.off), ...); }
template <typename... P> __device__ __forceinline__ void shift_nodes_opt(const Dims& g, P&... p) {
  ((p = (p != nullptr) ? p + g.off : p), ...);
}
template <typename... P> __device__ __forceinline__ void shift_scaled(const Dims& g, int64_t k, P&... p) {
  ((p += k * g.off), ...);
}
template <typename... P> __device__ __forceinline__ void shift_stencil(const Dims& g, P&... p) { ((p += g.soff), ...); }

// Division of a 31-bit unsigned x by an invariant d >= 1 without a divide
// instruction (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994, round-up method): with l = ceil(log2 d),
// m = ceil(2^(31+l) / d) < 2^32 and x < 2^31,
//   floor(x / d) = floor(x m / 2^(31+l)) = umulhi(x, m) >> (l - 1),
// because x m / 2^(31+l) = x / d + delta with 0 <= delta < 2^-l <= 1/d.
// d = 1 is the identity (shr = -1).
inline void fast_div_params(unsigned d, unsigned& mul, int& shr) {
  if (d <= 1u) {
    mul = 0u;
    shr = -1;
    return;
  }
  int l = 0;
  while ((1ull << l) < (unsigned long long)d) ++l;
  mul = (unsigned)(((1ull << (31 + l)) + d - 1) / d);
  shr = l - 1;
}
__host__ __device__ __forceinline__ unsigned fast_div(unsigned x, unsigned mul, int shr) {
#ifdef __CUDA_ARCH__
  const unsigned hi = __umulhi(x, mul);
#else
  const unsigned hi = (unsigned)(((unsigned long long)x * mul) >> 32);
#endif
  return shr < 0 ? x : (hi >> shr);
}

inline Dims make_dims(int dim, const int* n) {
  Dims g;
  g.dim = dim;
  g.n[0] = n[0];
  g.n[1] = dim > 1 ? n[1] : 1;
  g.n[2] = dim > 2 ? n[2] : 1;
  g.s1 = g.n[0];
  g.s2 = (int64_t)g.n[0] * g.n[1];
  g.N = g.s2 * g.n[2];
  g.B = 1;
  g.mrcap = 0;
  fast_div_params((unsigned)g.n[0], g.mul0, g.shr0);
  fast_div_params((unsigned)g.n[1], g.mul1, g.shr1);
  g.pd = nullptr;
  g.skip = nullptr;
  g.total = g.N;
  g.off = g.soff = 0;
  return g;
}

// Batched launches: problem blockIdx.y, whose slice of every per-problem
// array starts `stride` entries after the previous problem's.
template <typename... P>
__device__ __forceinline__ void batch_shift(int64_t stride, P&... p) {
  const int64_t o = (int64_t)blockIdx.y * stride;
  ((p += o), ...);
}
// The same for pointers that may be null (they stay null).
template <typename... P>
__device__ __forceinline__ void batch_shift_opt(int64_t stride, P&... p) {
  const int64_t o = (int64_t)blockIdx.y * stride;
  ((p = (p != nullptr) ? p + o : p), ...);
}

// Per-problem partial sums of the last-block reductions.
constexpr int64_t kPartialStride = 20480;
// Per-problem stride of the Gram-Schmidt coefficient arrays (KrylovScratch ha / hb).
constexpr int kMaxArnoldiDots = 66;

__device__ __forceinline__ void unravel(const Dims& g, int64_t j, int& i0, int& i1, int& i2) {
  if (j >= 0 && j <= 0x7fffffffLL) {   // every grid of the solver: two multiply-shift divisions
    const unsigned u = (unsigned)j;
    const unsigned q = fast_div(u, g.mul0, g.shr0);
    i0 = (int)(u - q * (unsigned)g.n[0]);
    const unsigned q2 = fast_div(q, g.mul1, g.shr1);
    i1 = (int)(q - q2 * (unsigned)g.n[1]);
    i2 = (int)q2;
    return;
  }
  i0 = (int)(j % g.n[0]);
  int64_t q = j / g.n[0];
  i1 = (int)(q % g.n[1]);
  i2 = (int)(q / g.n[1]);
}

// ---------------------------------------------------------------------------
// Galerkin stencil pattern: offsets in [-2,2]^dim with at most one |o_d| = 2
// (21 points in 2D, 81 in 3D), enumerated with axis 0 fastest.
// ---------------------------------------------------------------------------
constexpr int kPattern2 = 21;
constexpr int kPattern3 = 81;
template <int DIM> struct PatternSize { static constexpr int value = DIM == 2 ? kPattern2 : kPattern3; };

// Offsets of each pattern point (third component 0 in 2D) and the inverse map
// from (o0+2) + 5 (o1+2) + 25 (o2+2) to the point index (-1 outside).
// two*[p] = 1 for the points with an offset of +-2 (their Galerkin entries
// are purely imaginary, see coarse_stencil.cuh); part*[p] = index of p among
// the points of its kind (box points |o| <= 1 or two-points).
struct PatternTables {
  int8_t off2[kPattern2][3];
  int8_t off3[kPattern3][3];
  int8_t slot2[25];
  int8_t slot3[125];
  int8_t two2[kPattern2], part2[kPattern2];
  int8_t two3[kPattern3], part3[kPattern3];
};

constexpr PatternTables make_pattern_tables() {
  PatternTables t{};
  for (int k = 0; k < 25; ++k) t.slot2[k] = -1;
  for (int k = 0; k < 125; ++k) t.slot3[k] = -1;
  int p = 0;
  for (int o1 = -2; o1 <= 2; ++o1)
    for (int o0 = -2; o0 <= 2; ++o0) {
      const int twos = (o0 == 2 || o0 == -2) + (o1 == 2 || o1 == -2);
      if (twos > 1) continue;
      t.off2[p][0] = (int8_t)o0; t.off2[p][1] = (int8_t)o1; t.off2[p][2] = 0;
      t.slot2[(o0 + 2) + 5 * (o1 + 2)] = (int8_t)p;
      ++p;
    }
  p = 0;
  for (int o2 = -2; o2 <= 2; ++o2)
    for (int o1 = -2; o1 <= 2; ++o1)
      for (int o0 = -2; o0 <= 2; ++o0) {
        const int twos = (o0 == 2 || o0 == -2) + (o1 == 2 || o1 == -2) + (o2 == 2 || o2 == -2);
        if (twos > 1) continue;
        t.off3[p][0] = (int8_t)o0; t.off3[p][1] = (int8_t)o1; t.off3[p][2] = (int8_t)o2;
        t.slot3[(o0 + 2) + 5 * (o1 + 2) + 25 * (o2 + 2)] = (int8_t)p;
        ++p;
      }
  {
    int nb = 0, nt = 0;
    for (int q = 0; q < kPattern2; ++q) {
      const bool two = t.off2[q][0] == 2 || t.off2[q][0] == -2 || t.off2[q][1] == 2 || t.off2[q][1] == -2;
      t.two2[q] = two ? 1 : 0;
      t.part2[q] = (int8_t)(two ? nt++ : nb++);
    }
    nb = 0; nt = 0;
    for (int q = 0; q < kPattern3; ++q) {
      bool two = false;
      for (int d = 0; d < 3; ++d) two = two || t.off3[q][d] == 2 || t.off3[q][d] == -2;
      t.two3[q] = two ? 1 : 0;
      t.part3[q] = (int8_t)(two ? nt++ : nb++);
    }
  }
  return t;
}

// One copy per translation unit (internal linkage), so no device linking is needed.
static __constant__ PatternTables c_pattern = make_pattern_tables();

template <int DIM> __device__ __forceinline__ const int8_t* pattern_offset(int p) {
  return DIM == 2 ? c_pattern.off2[p] : c_pattern.off3[p];
}
template <int DIM> __device__ __forceinline__ bool pattern_two(int p) {
  return DIM == 2 ? c_pattern.two2[p] != 0 : c_pattern.two3[p] != 0;
}
template <int DIM> __device__ __forceinline__ int pattern_part(int p) {
  return DIM == 2 ? c_pattern.part2[p] : c_pattern.part3[p];
}
template <int DIM> __device__ __forceinline__ int pattern_slot(int o0, int o1, int o2) {
  return DIM == 2 ? c_pattern.slot2[(o0 + 2) + 5 * (o1 + 2)]
                  : c_pattern.slot3[(o0 + 2) + 5 * (o1 + 2) + 25 * (o2 + 2)];
}

// ---------------------------------------------------------------------------
// Fine (matrix-free) level
// ---------------------------------------------------------------------------
// Row of the fine operator in "cross" form: entry 0 is the centre, entry
// 1 + 4 d + {0,1,2,3} the neighbour at offset {-1,+1,-2,+2} along axis d.
constexpr int kCross2 = 9;
constexpr int kCross3 = 13;
template <int DIM> struct CrossSize { static constexpr int value = 1 + 4 * DIM; };

// Per-source values read by the fine-level kernels from device memory, so a
// captured CUDA graph stays valid when the operator is rebuilt for another
// source or frequency.
struct FineDyn {
  double omega;
  int src[3];
  int64_t src_index;
};

template <typename T> struct FineOp {
  const FineDyn* dyn;  // omega and the source (device)
  const T* g[3];     // d_d tau
  const T* t[3];     // d_dd tau
  const C<T>* rho;   // w^2 (kappa^2 - |grad tau|^2) - i w gamma kappa^2
  const C<T>* src_row;    // row of M^{-1} H M at the source (cross form, device)
  T h[3];
  T ih2[3];          // 1 / h^2
  T ih[3];           // 1 / h
  T hih[3];          // 1 / (2 h)
  T w2, w1;          // weights of the second- and first-order upwind differences
  int central;       // 1: central ADR scheme (upwind only on boundary nodes)
  int near;          // Chebyshev radius around the source with central advection
  const C<T>* rows;  // if set: stored cross rows (entry q of node j at q * N + j) used
                     // instead of building the row (the conjugate-transposed operator)
  const T* packed;   // if set: the row's varying parts, stored once per setup (see fine_row)
};


// The block's problem's grid, and for per-problem grids the spacing
// constants of f (computed as the host computes them for a single grid).
template <typename T> __device__ __forceinline__ void problem_spacing(const Dims& g, FineOp<T>& f);
template <typename T> __device__ __forceinline__ bool resolve(Dims& g, FineOp<T>& f) {
  if (resolve(g)) return true;
  if (g.pd != nullptr) problem_spacing(g, f);
  return false;
}
// The spacing constants of the block's problem (per-problem grids).
template <typename T> __device__ __forceinline__ void problem_spacing(const Dims& g, FineOp<T>& f) {
  const ProblemDims& q = g.pd[blockIdx.y];
#pragma unroll
  for (int d = 0; d < 3; ++d) {   // compile-time indices keep f out of local memory
    if (d < g.dim) {
      const double h = q.h[d];
      f.h[d] = (T)h;
      f.ih2[d] = (T)(1.0 / (h * h));
      f.ih[d] = (T)(1.0 / h);
      f.hih[d] = (T)(0.5 / h);
    }
  }
}

// Scheme -> upwind weights.
template <typename T> inline void set_scheme(FineOp<T>& f, int scheme, double beta) {
  f.central = 0;
  if (scheme == ADR_SCHEME_2UP) { f.w2 = T(1); f.w1 = T(0); }
  else if (scheme == ADR_SCHEME_1UP) { f.w2 = T(0); f.w1 = T(1); }
  else if (scheme == ADR_SCHEME_PREC) { f.w2 = T(1.0 - beta); f.w1 = T(beta); }
  else { f.w2 = T(1); f.w1 = T(0); f.central = 1; }
}

// ---------------------------------------------------------------------------
// Launchers (all asynchronous on `st`)
// ---------------------------------------------------------------------------
struct FineInputs {
  const double* kappa;
  const double* tau1;   // tau1 of tau = |x - x0| tau1, or tau itself when plain != 0
  const double* gamma;
  int src[3];
  double omega;
  double h[3];
  double ih[3];   // 1 / h
  int plain;      // 1: tau1 holds plain tau, differentiated by finite differences
};

// Fine coefficients in float64 (g, t, rho, tau) and the source row.
void launch_coefficients(const Dims& g, const FineInputs& in, double* const gd[3], double* const td[3],
                         double2* rho, double* tau, double2* src_row, cudaStream_t st);
// float64 -> float32 copy of n reals.
void launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t st);
// diag(M) = exp(-i w tau) per node of every problem (Eq. matrix_rescaling).
void launch_phase(const Dims& g, const double* tau, const FineDyn* dyn, double2* phase, cudaStream_t st);
// Stored cross rows A -> M A M^{-1}: entry (i, i + o) times m_i conj(m_{i+o}).
template <typename T> void launch_rows_rescale(const Dims& g, C<T>* rows, const double2* phase, cudaStream_t st);
// dst = (Td)(src * m) or, with conj, (Td)(src * conj(m)), m = phase (whole arrays of n entries).
template <typename Ts, typename Td>
void launch_phase_cast(const C<Ts>* src, const double2* phase, bool conj, C<Td>* dst, int64_t n, cudaStream_t st);
// The cycle's coefficients under the complex shift of Eq. shift: rho_s = rho -
// i alpha w^2 kappa^2 per node and the source row with the same diagonal change.
void launch_shift(const Dims& g, const FineInputs& in, double alpha, const double2* rho, const double2* src_row,
                  double2* rho_s, double2* src_row_s, cudaStream_t st);

// Level-0 operations; x, y, b complex of T.
template <typename T> void launch_fine_apply(const Dims& g, const FineOp<T>& f, const C<T>* x, C<T>* y, cudaStream_t st);
template <typename T> void launch_fine_residual(const Dims& g, const FineOp<T>& f, const C<T>* b, const C<T>* x, C<T>* r, cudaStream_t st);
// xout = xin + w D^{-1} (b - A xin); xin may be null (zero guess).
template <typename T> void launch_fine_jacobi(const Dims& g, const FineOp<T>& f, const C<T>* b, const C<T>* xin, C<T>* xout, T w, cudaStream_t st);
// z = D^{-1} v, or z = diag(A)^{-1} itself when v is null
template <typename T> void launch_fine_dinv(const Dims& g, const FineOp<T>& f, const C<T>* v, C<T>* z, cudaStream_t st);
// Fused minimal-residual sweep pieces: w = A z with alpha = (w^H r)/(w^H w)
// reduced by the last block; r = b - A x with z = D^{-1} r.
template <typename T> void launch_fine_mr_apply(const Dims& g, const FineOp<T>& f, const C<T>* z, const C<T>* r, C<T>* w,
                                                double2* partial, unsigned* ticket, double2* alpha, cudaStream_t st);
template <typename T> void launch_fine_residual_dinv(const Dims& g, const FineOp<T>& f, const C<T>* b, const C<T>* x,
                                                     const C<T>* dinv, C<T>* r, C<T>* z, cudaStream_t st);
// Stored float64 cross rows (point-major, (1 + 4 dim) x N) of a fine operator,
// and the plain stencil apply / residual with them.
void launch_fine_store_rows(const Dims& g, const FineOp<double>& f, double2* rows, cudaStream_t st);
void launch_fine_store_rows(const Dims& g, const FineOp<float>& f, float2* rows, cudaStream_t st);
// Packed rows of f ((2 + 4 dim) reals per node and problem), for FineOp::packed.
template <typename T> void launch_fine_pack(const Dims& g, const FineOp<T>& f, T* packed, cudaStream_t st);
// rowsT = conjugate transpose of the stored cross rows (same layout).
template <typename T> void launch_rows_adjoint(const Dims& g, const C<T>* rows, C<T>* rowsT, cudaStream_t st);
void launch_rows_apply(const Dims& g, const double2* rows, const double2* x, double2* y, cudaStream_t st);
void launch_rows_residual(const Dims& g, const double2* rows, const double2* b, const double2* x, double2* r, cudaStream_t st);
// the outer float64 operator from packed rows (f.packed set; see k_fine_pack)
void launch_packed_apply(const Dims& g, const FineOp<double>& f, const double2* x, double2* y, cudaStream_t st);
void launch_packed_residual(const Dims& g, const FineOp<double>& f, const double2* b, const double2* x, double2* r,
                            cudaStream_t st);
// Writes the per-source values read by the fine kernels.
void launch_set_dyn(FineDyn* d, const FineDyn& v, cudaStream_t st);
// Galerkin product of the fine operator into the stored stencil of level 1.
template <typename T> void launch_galerkin_fine(const Dims& gf, const Dims& gc, const FineOp<T>& f, C<T>* stencil, C<T>* dinv, cudaStream_t st);

// Stored-stencil levels.
template <typename T> void launch_stencil_apply(const Dims& g, const C<T>* A, const C<T>* x, C<T>* y, cudaStream_t st);
template <typename T> void launch_stencil_residual(const Dims& g, const C<T>* A, const C<T>* b, const C<T>* x, C<T>* r, cudaStream_t st);
template <typename T> void launch_stencil_jacobi(const Dims& g, const C<T>* A, const C<T>* dinv, const C<T>* b, const C<T>* xin, C<T>* xout, T w, cudaStream_t st);
template <typename T> void launch_stencil_mr_apply(const Dims& g, const C<T>* A, const C<T>* z, const C<T>* r, C<T>* w,
                                                   double2* partial, unsigned* ticket, double2* alpha, cudaStream_t st);
template <typename T> void launch_stencil_residual_dinv(const Dims& g, const C<T>* A, const C<T>* b, const C<T>* x,
                                                        const C<T>* dinv, C<T>* r, C<T>* z, cudaStream_t st);
// The minimal-residual apply with the coefficient tiles streamed into shared
// memory by bulk copies (float32 only); err: per-problem error words (a
// bounded wait that ran out sets it and the weight to NaN).  blocks: grid
// size per problem.  prepare_stencil_tma opts the kernel into its shared
// memory; call it outside capture, false if unavailable.
bool prepare_stencil_tma();
void launch_stencil_mr_apply_tma(const Dims& g, const float2* A, const float2* z, const float2* r, float2* w,
                                 double2* partial, unsigned* ticket, double2* alpha, int* err, int blocks, int variant,
                                 cudaStream_t st);
// y = A x and r = b - A x, z = dinv .* r with the same streaming (NaN output on a failed wait).
void launch_stencil_apply_tma(const Dims& g, const float2* A, const float2* x, float2* y, int* err, int blocks,
                              int variant, cudaStream_t st);
void launch_stencil_residual_dinv_tma(const Dims& g, const float2* A, const float2* b, const float2* x,
                                      const float2* dinv, float2* r, float2* z, int* err, int blocks, int variant,
                                      cudaStream_t st);

template <typename T> void launch_stencil_export(const Dims& g, const C<T>* A, C<T>* out, int S, cudaStream_t st);
template <typename T> void launch_galerkin_stored(const Dims& gf, const Dims& gc, const C<T>* Af, C<T>* Ac, C<T>* dinv, cudaStream_t st);

// Transfers.
template <typename T> void launch_restrict(const Dims& gf, const Dims& gc, const C<T>* rf, C<T>* rc, cudaStream_t st);
template <typename T> void launch_prolong_add(const Dims& gf, const Dims& gc, const C<T>* ec, C<T>* xf, cudaStream_t st);

// Largest grid of the fused relaxation kernels (grid-stride beyond): about
// sixteen 256-thread blocks per SM keeps every SM busy while bounding the
// number of blocks that meet at the ticket of the last-block reduction (a
// full one-node-per-thread grid spent more time on that atomic than on the
// stencil).  Also sizes their partial sums.
constexpr int kMaxMrBlocks = 2432;

// Counts kernel launches issued by the library (all threads).
void count_launches(int n);

// Records msg as the calling thread's adr_last_error text; returns code.
int set_last_error(int code, const char* msg);

// The outer float64 operator on a vector of float32 values in double-float
// arithmetic (see fine.cu): pk2 are the packed rows split into float32
// (hi, lo) pairs by launch_split_df (n reals).  y = A x as double-float planes
// (high parts at y, low parts at y + ylo); x is also copied to zcopy when
// that is not null.
struct DfLaplacian { float hi[3], lo[3]; };
void launch_split_df(const double* src, float2* dst, int64_t n, cudaStream_t st);
void launch_packed_apply_df(const Dims& g, const FineOp<double>& f, const float2* pk2, const float2* x, float2* y,
                            int64_t ylo, float2* zcopy, cudaStream_t st);

// Vector kernels.
template <typename T> void launch_cmul_vec(const C<T>* a, const C<T>* b, C<T>* out, int64_t n, cudaStream_t st);  // out = a .* b
template <typename Ts, typename Td> void launch_ccast(const C<Ts>* src, C<Td>* dst, int64_t n, cudaStream_t st);

// q = value at each problem's source node (dyn[p].src_index), zero elsewhere.
void launch_rhs_point(const Dims& g, double2* q, const FineDyn* dyn, double value, cudaStream_t st);
// Receiver residuals res = R u - d, rhs += M^H R^T res, out = (sum |res|^2, bad indices).
void launch_receivers(int64_t N, int nrec, const int64_t* rec, const double2* d, const double2* u, const double* tau,
                      double omega, double2* res, double2* rhs, double2* out, cudaStream_t st);
// grad -= Re(conj(lambda) (2 w^2 kappa - 2 i w gamma kappa) a), elementwise.
void launch_kappa_gradient(int64_t N, double omega, const double* kappa, const double* gamma, const double2* a,
                           const double2* lambda, double* grad, cudaStream_t st);
// u = a exp(-i w tau) with each problem's w from dyn.
void launch_reconstruct(const Dims& g, const double2* a, const double* tau, const FineDyn* dyn, double2* u, cudaStream_t st);
void launch_pack_coefficients(const Dims& g, const double* const gd[3], const double* const td[3], const double2* rho,
                              const double* tau, double* out, cudaStream_t st);

}  // namespace adr
