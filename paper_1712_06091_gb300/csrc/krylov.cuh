// Krylov building blocks (see krylov.cu).
//
// Batched launches: a level of B problems on one grid runs every kernel once
// with grid.y = B (problem = blockIdx.y).  Vectors of a level are packed
// problem-major (problem p's n entries at p * n); a Krylov basis keeps its
// vectors at stride ld = B * n, so vector i of problem p starts at
// V + i * ld + p * n.  Per-problem scalars (Arnoldi state, reduction scratch)
// are packed problem-major too, see arnoldi_at / scratch_at.
#pragma once

#include "adr_common.cuh"

namespace adr {

constexpr int kMaxReduceBlocks = 304;  // 2 x 152 SMs: per-block partials of a reduction
constexpr int kMaxKrylov = 64;         // largest restart / inner Krylov dimension
constexpr int kMaxDots = kMaxKrylov + 2;
static_assert(kMaxDots == kMaxArnoldiDots, "stride of ha / hb per problem");
static_assert(kPartialStride >= (int64_t)kMaxReduceBlocks * kMaxDots, "partial sums of the Gram-Schmidt passes");
static_assert(kPartialStride >= (int64_t)kMaxMrBlocks * 2, "partial sums of the relaxation apply");

// Device-resident Arnoldi state of one (F)GMRES instance with restart m.
//   scal: beta, Givens estimate |g_{j+1}|, last h_{j+1,j}, last |w|^2, and the
//         convergence target (estimate <= target freezes the instance; 0 = never)
//   iscal: exact-breakdown column (-1: none), convergence column (-1: none)
enum { kScalBeta = 0, kScalEst = 1, kScalHn = 2, kScalNrm2 = 3, kScalTarget = 4, kNumScal = 5 };
enum { kIScalStop = 0, kIScalConv = 1, kNumIScal = 2 };
struct ArnoldiState {
  int m;
  double2* H;      // (m+1) x m, column-major
  double* cs;      // m
  double2* sn;     // m
  double2* g;      // m+1
  double2* y;      // m
  double* scal;    // kNumScal
  int* iscal;      // kNumIScal
};

// Problem pb's state in an allocation of B states packed problem-major.
__host__ __device__ inline ArnoldiState arnoldi_at(ArnoldiState s, int pb) {
  const int64_t m = s.m;
  s.H += pb * (m + 1) * m;
  s.cs += pb * m;
  s.sn += pb * m;
  s.g += pb * (m + 1);
  s.y += pb * m;
  s.scal += (int64_t)pb * kNumScal;
  s.iscal += (int64_t)pb * kNumIScal;
  return s;
}

int reduction_blocks(int64_t n, int values);

// Scratch shared by the fused reductions (all launches on one stream).
struct KrylovScratch {
  double2* partial;   // per-block partials, kPartialStride per problem
  unsigned* ticket;   // arrival counter of the last-block reductions (kept at 0 between launches)
  double2* ha;        // first Gram-Schmidt coefficients (kMaxDots per problem)
  double2* hb;        // second Gram-Schmidt coefficients (kMaxDots per problem)
  double2* nrm2;      // squared norm (x) and reciprocal norm (y)
  double2* alpha;     // minimal-residual weight
};

__host__ __device__ inline KrylovScratch scratch_at(KrylovScratch s, int pb) {
  s.partial += (int64_t)pb * kPartialStride;
  s.ticket += pb;
  s.ha += (int64_t)pb * kMaxDots;
  s.hb += (int64_t)pb * kMaxDots;
  s.nrm2 += pb;
  s.alpha += pb;
  return s;
}

// In the launchers below n is the length of one problem's vectors and B the
// number of problems (grid.y); V/Z bases have stride ld between vectors.

// CGS2 step j: w <- w - V (V^H w) twice, |w|^2, Arnoldi column j and Givens
// rotation in st (three launches).
template <typename T>
void launch_cgs2(const C<T>* V, int64_t ld, int k, C<T>* w, const Dims& g, const KrylovScratch& s, const ArnoldiState& st, int j,
                 cudaStream_t stream);
// Gram-Schmidt step j with the second pass only when the first one cancelled
// |w| below eta |w| (four launches; eta >= 1 is launch_cgs2).
template <typename T>
void launch_cgs_selective(const C<T>* V, int64_t ld, int k, C<T>* w, const Dims& g, const KrylovScratch& s,
                          const ArnoldiState& st, int j, double eta, cudaStream_t stream);
// The Jacobi-preconditioned GMRES step of the coarsest grid with the
// selective second Gram-Schmidt pass (at most three launches; the column's
// norm from Pythagoras, see coarse_select_dev / coarse_reorth_dev):
//   launch_cgs_dots_sel: ha = V^H w, |w|^2, and the decision (when the apply
//     does not fuse the first pass);
//   launch_cgs_reorth: the second pass where the first cancelled (returns at
//     once otherwise);
//   launch_cgs_next: V_next = (w - V c) / h_{j+1,j}, z = dinv .* V_next.
// finish > 0 on the last step: the least-squares solve over `finish` columns.
template <typename T>
void launch_cgs_dots_sel(const C<T>* V, int64_t ld, int k, const C<T>* w, const Dims& g, const KrylovScratch& s,
                         const ArnoldiState& st, int j, int finish, double eta, cudaStream_t stream);
template <typename T>
void launch_cgs_reorth(const C<T>* V, int64_t ld, int k, C<T>* w, const Dims& g, const KrylovScratch& s,
                       const ArnoldiState& st, int j, int finish, cudaStream_t stream);
template <typename T>
void launch_cgs_next(const C<T>* V, int64_t ld, int k, const C<T>* w, const Dims& g, const KrylovScratch& s, C<T>* Vnext,
                     const C<T>* dinv, C<T>* z, cudaStream_t stream);
// The coarsest step's apply w = A z fused with its first Gram-Schmidt pass
// (float32 stencil levels, coefficient tiles streamed by bulk copies):
// ha = V^H w over the kd <= 63 basis vectors V_i = V + i ld, |w|^2, and the
// selective decision of launch_cgs_dots_sel in the last block (eta: the
// threshold; finish as there).  NaN coefficients on a failed wait.
void launch_stencil_arnoldi_tma(const Dims& g, const float2* A, const float2* z, float2* w, const float2* V, int64_t ld,
                                int kd, const KrylovScratch& s, const ArnoldiState& st, int j, int finish, double eta,
                                int* err, int blocks, int variant, cudaStream_t stream);
// x = dinv .* sum_{i<k} V_i y_i (the coarsest solution from its basis).
template <typename T>
void launch_combine_dinv(C<T>* x, const C<T>* V, int64_t ld, int k, const ArnoldiState& st, const C<T>* dinv, const Dims& g,
                         cudaStream_t stream);
// |b|^2 into s.nrm2; with st, also starts an Arnoldi cycle with beta = |b|
// (rel_target >= 0: the cycle's convergence target becomes rel_target * beta;
// < 0: the stored target is kept).
template <typename T>
void launch_norm_start(const C<T>* b, const Dims& g, const KrylovScratch& s, const ArnoldiState* st, cudaStream_t stream, double rel_target = -1.0);
// x = (assign ? 0 : x) + sum_{i<k} Z_i y_i with y from st.
template <typename T>
void launch_combine(C<T>* x, const C<T>* Z, int64_t ld, int k, const ArnoldiState& st, bool assign, const Dims& g,
                    cudaStream_t stream);
// x = (x_zero ? 0 : x) + alpha z ; r_dst = r_src - alpha w ; znext = dinv .* r_dst (if not null)
template <typename T>
void launch_mr_update2(C<T>* x, const C<T>* z, const C<T>* r_src, C<T>* r_dst, const C<T>* w, const double2* alpha,
                       const C<T>* dinv, C<T>* znext, bool x_zero, const Dims& g, cudaStream_t stream);
// out = w * (1 / |w|) with the reciprocal norm from s.nrm2 (per problem).
template <typename T> void launch_scale_inv_norm(const C<T>* w, C<T>* out, const double2* nrm2, const Dims& g, cudaStream_t st);
// out = w * (1 / |w|) and z = dinv .* out (per problem).
template <typename T> void launch_scale_dinv(const C<T>* w, C<T>* out, const C<T>* dinv, C<T>* z, const double2* nrm2,
                                             const Dims& g, cudaStream_t st);
// Whole-array elementwise operations (n = all problems' entries).
template <typename T> void launch_copy(const C<T>* a, C<T>* b, int64_t n, cudaStream_t st);
template <typename T> void launch_zero(C<T>* a, int64_t n, cudaStream_t st);
// y = R^{-1} g for the leading block of each problem's rotated Hessenberg
// matrix, k cut to its breakdown or convergence column.
void launch_backsolve(const ArnoldiState& s, int k, cudaStream_t st, int B = 1);
// Convergence targets: st.scal[kScalTarget] = tol * sqrt(nrm2.x) per problem.
void launch_set_target(const ArnoldiState& s, const double2* nrm2, double tol, cudaStream_t st, int B = 1);

// The same solve on one thread-block cluster (cluster = 16 or 8 CTAs), for
// Krylov dimensions up to kClusterKMax.  prepare_coarse_cluster returns the
// cluster size the device can schedule (0 if none); call it outside capture.
constexpr int kClusterKMax = 32;
int prepare_coarse_cluster(int dim, bool f32);
template <typename T>
void launch_coarse_gmres_cluster(const Dims& g, const C<T>* A, const C<T>* dinv, const C<T>* b, C<T>* x, C<T>* V, C<T>* z,
                                 int k, const ArnoldiState& s, int cluster, cudaStream_t st);

// The same solve as one persistent cooperative launch: gs.nblk co-resident
// blocks per problem meeting at grid barriers (bounded spins; on a timeout
// the problem's error word is raised and x is set to NaN).
// prepare_coarse_grid returns how many such blocks the device holds at once
// (0: no cooperative launch); call it outside capture.
constexpr int kGridMaxK = 32;
struct GridScratch {
  double2* part;   // per problem: 2 x nblk x (kGridMaxK + 1) partial sums
  double2* tot;    // per problem: kGridMaxK + 1 totals of the last reduction
  unsigned* bar;   // per problem: arrival count, generation
  int* err;        // per problem: barrier timeout flag (sticky)
  int nblk;        // blocks per problem
};
int prepare_coarse_grid(int dim, bool f32);
template <typename T>
void launch_coarse_gmres_grid(const Dims& g, const C<T>* A, const C<T>* dinv, const C<T>* b, C<T>* x, C<T>* V, C<T>* z,
                              int k, const GridScratch& gs, double eta, cudaStream_t st);

// Whole fixed-count Jacobi-preconditioned GMRES of a small stored-stencil
// level in one block of 1024 threads per problem (V: basis of stride B n,
// z: scratch vector).
template <typename T>
void launch_coarse_gmres_cta(const Dims& g, const C<T>* A, const C<T>* dinv, const C<T>* b, C<T>* x, C<T>* V, C<T>* z, int k,
                             const ArnoldiState& s, cudaStream_t st);

}  // namespace adr
