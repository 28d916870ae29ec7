// Double-float outer Krylov passes (krylov_df.cu).  A double-float vector is
// two float32 planes of complex values: high parts at v, low parts at v + lo
// (float2 units); basis vector i at V + i ld.  Batches and per-problem grids
// as in krylov.cuh (Dims; grid.y = problems).
#pragma once

#include "krylov.cuh"

namespace adr {

// Gram-Schmidt step j of the outer FGMRES on the double-float basis V (k
// vectors) and the new vector w: the selective passes (the decision from
// Pythagoras after the first pass's dots; eta >= 1: the second pass always),
// the Arnoldi column and its Givens rotation in st, |w|^2 and 1/|w| in
// s.nrm2, and w normalised in place with its high plane in cyc (may be null).
void launch_df_selective(const float2* V, int64_t ld, int64_t lo, int k, float2* w, float2* cyc, const Dims& g,
                         const KrylovScratch& s, const ArnoldiState& st, int j, double eta, cudaStream_t stream);
// out = r / |r| from a float64 r (1/|r| from nrm2->y per problem); the high
// plane also into cyc (may be null).
void launch_df_from_double(const double2* r, float2* out, int64_t lo, const double2* nrm2, float2* cyc, const Dims& g,
                           cudaStream_t st);
// x += sum_{i<k} Z_i y_i: float32 vectors Z_i at stride ld, y from st, the
// sum in double-float, x float64.
void launch_df_combine(double2* x, const float2* Z, int64_t ld, int k, const ArnoldiState& st, const Dims& g,
                       cudaStream_t stream);

}  // namespace adr
