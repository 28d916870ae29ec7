// Krylov building blocks (see krylov.cu).
#pragma once

#include "adr_common.cuh"

namespace adr {

constexpr int kMaxReduceBlocks = 304;  // 2 x 152 SMs: per-block partials of a reduction
constexpr int kMaxKrylov = 64;         // largest restart / inner Krylov dimension

// Device-resident Arnoldi state of one (F)GMRES instance with restart m.
enum { kScalBeta = 0, kScalEst = 1, kScalHn = 2, kScalNrm2 = 3, kNumScal = 4 };
enum { kIScalStop = 0, kNumIScal = 2 };
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

int reduction_blocks(int64_t n);

// Scratch shared by the fused reductions (all launches on one stream).
struct KrylovScratch {
  double2* partial;   // per-block partials (>= blocks x values of the largest launch)
  unsigned* ticket;   // arrival counter of the last-block reductions (kept at 0 between launches)
  double2* ha;        // first Gram-Schmidt coefficients
  double2* hb;        // second Gram-Schmidt coefficients
  double2* nrm2;      // squared norm
  double2* alpha;     // minimal-residual weight
};

// CGS2 step j: w <- w - V (V^H w) twice, |w|^2, Arnoldi column j and Givens
// rotation in st (three launches).
template <typename T>
void launch_cgs2(const C<T>* V, int64_t ld, int k, C<T>* w, int64_t n, const KrylovScratch& s, const ArnoldiState& st, int j,
                 cudaStream_t stream);
// Gram-Schmidt step j with the second pass only when the first one cancelled
// |w| below eta |w| (four launches; eta >= 1 is launch_cgs2).
template <typename T>
void launch_cgs_selective(const C<T>* V, int64_t ld, int k, C<T>* w, int64_t n, const KrylovScratch& s,
                          const ArnoldiState& st, int j, double eta, cudaStream_t stream);
// |b|^2 into s.nrm2; with st, also starts an Arnoldi cycle with beta = |b|.
template <typename T>
void launch_norm_start(const C<T>* b, int64_t n, const KrylovScratch& s, const ArnoldiState* st, cudaStream_t stream);
// x = (assign ? 0 : x) + sum_{i<k} Z_i y_i with y from st.
template <typename T>
void launch_combine(C<T>* x, const C<T>* Z, int64_t ld, int k, const ArnoldiState& st, bool assign, int64_t n, cudaStream_t stream);
// x = (x_zero ? 0 : x) + alpha z ; r_dst = r_src - alpha w ; znext = dinv .* r_dst (if not null)
template <typename T>
void launch_mr_update2(C<T>* x, const C<T>* z, const C<T>* r_src, C<T>* r_dst, const C<T>* w, const double2* alpha,
                       const C<T>* dinv, C<T>* znext, bool x_zero, int64_t n, cudaStream_t stream);

template <typename T>
void launch_dots(const C<T>* V, int64_t ld, int k, const C<T>* w, int64_t n, double2* partial, double2* out,
                 cudaStream_t st, bool accumulate = false);
template <typename T>
void launch_dot2(const C<T>* a, const C<T>* b, const C<T>* c, int64_t n, double2* partial, double2* out, cudaStream_t st);
template <typename T>
void launch_axpy_multi(C<T>* w, const C<T>* V, int64_t ld, int k, const double2* coef, double sign, int64_t n, cudaStream_t st);
template <typename T> void launch_scale_inv_norm(const C<T>* w, C<T>* out, const double2* nrm2, int64_t n, cudaStream_t st);
template <typename T> void launch_copy(const C<T>* a, C<T>* b, int64_t n, cudaStream_t st);
template <typename T> void launch_zero(C<T>* a, int64_t n, cudaStream_t st);
template <typename T>
void launch_mr_update(C<T>* x, const C<T>* z, C<T>* r, const C<T>* w, const double2* alpha, const C<T>* dinv, C<T>* znext,
                      int64_t n, cudaStream_t st);

// The same solve on one thread-block cluster (cluster = 16 or 8 CTAs), for
// Krylov dimensions up to kClusterKMax.  prepare_coarse_cluster returns the
// cluster size the device can schedule (0 if none); call it outside capture.
constexpr int kClusterKMax = 32;
int prepare_coarse_cluster(int dim, bool f32);
template <typename T>
void launch_coarse_gmres_cluster(const Dims& g, const C<T>* A, const C<T>* dinv, const C<T>* b, C<T>* x, C<T>* V, C<T>* z,
                                 int k, const ArnoldiState& s, int cluster, cudaStream_t st);

// Whole fixed-count Jacobi-preconditioned GMRES of a small stored-stencil
// level in one block of 1024 threads (V: (k+1) n scratch, z: n scratch).
template <typename T>
void launch_coarse_gmres_cta(const Dims& g, const C<T>* A, const C<T>* dinv, const C<T>* b, C<T>* x, C<T>* V, C<T>* z, int k,
                             const ArnoldiState& s, cudaStream_t st);

void launch_cycle_start(const ArnoldiState& s, const double2* nrm2, cudaStream_t st);
void launch_arnoldi_column(const ArnoldiState& s, int j, const double2* ha, const double2* hb, const double2* nrm2, cudaStream_t st);
void launch_backsolve(const ArnoldiState& s, int k, cudaStream_t st);
void launch_mr_alpha(const double2* d, double2* alpha, cudaStream_t st);

}  // namespace adr
