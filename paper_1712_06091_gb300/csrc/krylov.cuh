// Krylov building blocks (see krylov.cu).
#pragma once

#include "adr_common.cuh"

namespace adr {

constexpr int kMaxReduceBlocks = 304;  // 2 x 152 SMs: per-block partials of a reduction

// Device-resident Arnoldi state of one (F)GMRES instance with restart m.
enum { kScalBeta = 0, kScalEst = 1, kScalHn = 2, kNumScal = 4 };
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

void launch_cycle_start(const ArnoldiState& s, const double2* nrm2, cudaStream_t st);
void launch_arnoldi_column(const ArnoldiState& s, int j, const double2* ha, const double2* hb, const double2* nrm2, cudaStream_t st);
void launch_backsolve(const ArnoldiState& s, int k, cudaStream_t st);
void launch_mr_alpha(const double2* d, double2* alpha, cudaStream_t st);

}  // namespace adr
