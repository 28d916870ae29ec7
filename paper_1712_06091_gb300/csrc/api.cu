// C ABI, operator lifetime and the solver drivers of libadr.
//
//  * adr_operator_create: fine coefficients (Eq. travel_time_coeff), the
//    multigrid hierarchy with Galerkin coarse operators of the blend
//    (1 - beta) H_2up + beta H_1up (Eqs. precADRup, coarseGridMatrix).
//  * the cycle: Alg. TwoGrid applied recursively (V) or with an inner
//    flexible GMRES on every coarse level but the last (Alg. Kcycle);
//    relaxation by damped Jacobi or by one Jacobi-preconditioned GMRES step
//    (Sec. 3.1); fixed-count Jacobi-preconditioned GMRES on the coarsest
//    level (Sec. 3.1, Sec. 4.2).
//  * adr_solve: right-preconditioned flexible GMRES(m) in float64 on H_2up,
//    classical Gram-Schmidt applied twice, Givens rotations on the device.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "krylov.cuh"
#include "krylov_df.cuh"
#include "coarse_stencil.cuh"

namespace adr {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
int set_last_error(int code, const char* msg) { return fail(code, msg); }

#define ADR_CUDA(call)                                                                            \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(ADR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define ADR_TRY(expr)              \
  do {                             \
    int rc_ = (expr);              \
    if (rc_ != ADR_OK) return rc_; \
  } while (0)

static int check_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ADR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return ADR_OK;
}

// ---------------------------------------------------------------------------
// Arena: one device allocation carved into 256-byte aligned pieces.  The
// layout is computed twice: once with a null base to size it, once for real.
// ---------------------------------------------------------------------------
struct Arena {
  char* base = nullptr;
  size_t used = 0;
  template <typename X> X* take(size_t count) {
    used = (used + 255) & ~size_t(255);
    X* p = base ? reinterpret_cast<X*>(base + used) : nullptr;
    used += count * sizeof(X);
    return p;
  }
};

// ---------------------------------------------------------------------------
// Hierarchy in one precision
// ---------------------------------------------------------------------------
template <typename T> struct Level {
  Dims g;
  C<T>* A = nullptr;     // Galerkin stencil (levels >= 1)
  C<T>* dinv = nullptr;  // inverse diagonal
  C<T>* b = nullptr;     // right-hand side handed down by restriction
  C<T>* x = nullptr;     // correction handed up to prolongation
  C<T>* r = nullptr;     // residual
  C<T>* t = nullptr;     // scratch: Jacobi ping-pong, A z of the MR step, Krylov w
  C<T>* z = nullptr;     // MR search direction / preconditioned vector
  C<T>* KV = nullptr;    // Krylov basis (K-cycle or coarsest GMRES)
  C<T>* KZ = nullptr;    // K-cycle preconditioned basis
  int kdim = 0;          // Krylov dimension used on this level
  ArnoldiState ks{};
};

constexpr int64_t kSmallCoarse = 8192;      // one-block coarsest solve up to this size (no cluster)
constexpr int64_t kClusterCoarse = 32768;   // cluster coarsest solve up to this size

// B Arnoldi states packed problem-major (see arnoldi_at).
static void take_arnoldi(Arena& a, ArnoldiState& s, int m, int B) {
  s.m = m;
  s.H = a.take<double2>((size_t)(m + 1) * m * B);
  s.cs = a.take<double>((size_t)m * B);
  s.sn = a.take<double2>((size_t)m * B);
  s.g = a.take<double2>((size_t)(m + 1) * B);
  s.y = a.take<double2>((size_t)m * B);
  s.scal = a.take<double>((size_t)kNumScal * B);
  s.iscal = a.take<int>((size_t)kNumIScal * B);
}

template <typename T> struct Hier {
  int L = 0;
  T* packed = nullptr;   // packed rows of the level-0 operator (2 + 4 dim reals per node); with
                         // params.rescale its full rows M A M^{-1} (1 + 4 dim complex per node)
  Level<T> lv[ADR_MAX_LEVELS];
  GridScratch gs{};   // persistent coarsest-grid solve (nblk = 0: not planned)
  FineOp<T> prec{};   // level-0 operator of the cycle (params.prec_scheme, shift, rescale)
};

struct Op {
  int dim = 0;
  int B = 1;                        // problems of the batch (own source, frequency, medium; own grid if hetero)
  Dims g0{};                        // the finest level (largest grid, totals over the batch)
  // Batches of unequal grids (adr_batch_create_grids): per problem its nodes
  // and spacing, per level a table of the problems' grids (host, and its copy
  // in the arena that the kernels read); every level's Dims, fixed at creation.
  bool hetero = false;
  std::vector<int> pn;              // 3 per problem
  std::vector<double> ph;           // 3 per problem
  int nlev = 0;
  Dims lvg[ADR_MAX_LEVELS]{};
  std::vector<ProblemDims> tab[ADR_MAX_LEVELS];
  ProblemDims* dtab[ADR_MAX_LEVELS] = {};
  // Batches: per problem 1 while it is frozen inside adr_solve (the kernels
  // of the cycle and of the iteration skip it), 0 otherwise; the host's
  // pinned copy it is uploaded from.
  int* skip = nullptr;
  int* host_skip = nullptr;         // kSkipSlots rings of B ints inside the pinned host_scal block
  int skip_slot = 0;
  adr_params_t p{};
  cudaStream_t st = nullptr;
  double omega = 0;                 // problem 0 (the only one when B = 1)
  double h[3] = {0, 0, 0};
  int src[3] = {0, 0, 0};
  int64_t src_index = 0;
  std::vector<double> omegas;       // per problem
  std::vector<int> srcs;            // 3 per problem
  // fine coefficients
  double* gd[3] = {nullptr, nullptr, nullptr};
  double* td[3] = {nullptr, nullptr, nullptr};
  double2* rho = nullptr;
  double* tau = nullptr;
  double2* srow = nullptr;
  float* srowf = nullptr;  // float2 view
  float* gf[3] = {nullptr, nullptr, nullptr};
  float* tf[3] = {nullptr, nullptr, nullptr};
  float* rhof = nullptr;  // float2 view
  // shifted copies for the cycle (Eq. shift; only when params.shift != 0)
  double2* rhos = nullptr;
  float* rhosf = nullptr;
  double2* srows = nullptr;
  float* srowsf = nullptr;
  // diag(M) = exp(-i w tau) per node (only when params.rescale != 0)
  double2* phase = nullptr;
  Hier<double> h64;
  Hier<float> h32;
  // outer FGMRES
  double2* V = nullptr;
  double2* Z = nullptr;
  double2* b = nullptr;  // point-source right-hand side
  double2* r = nullptr;
  double* packed_out = nullptr; // packed float64 rows of the outer system (k_fine_pack layout)
  float2* packed_df = nullptr;  // the same rows split into float32 (hi, lo) pairs (float32 cycle, not rescaled)
  double2* rows_out = nullptr;  // stored float64 rows of the outer system (adjoint operators only)
  ArnoldiState ost{};
  KrylovScratch ks{};
  FineDyn* dyn = nullptr;           // omega and the source, read by the fine kernels
  // the cycle below the float64 Krylov loop, captured once and replayed
  cudaStream_t cap = nullptr;
  cudaGraphExec_t cycle_exec = nullptr;
  long long cycle_kernels = 0;
  // conjugate-transposed operator (params.adjoint): H_2up^H rows for the outer
  // iteration and a hierarchy on A^H sharing the forward one's work vectors
  double2* rows_outT = nullptr;
  void* rows0 = nullptr;            // stored rows of the cycle's fine operator (setup scratch)
  void* rows0T = nullptr;           // their conjugate transpose
  Hier<double> a64;
  Hier<float> a32;
  cudaGraphExec_t cycle_exec_adj = nullptr;
  long long cycle_kernels_adj = 0;
  bool prof_off = false;            // the adjoint cycle is never timed
  bool use_graph = true;
  int cluster_size = 0;             // CTAs of the coarsest-grid cluster solver (0: not available)
  int grid_coresident = 0;          // co-resident blocks of the persistent coarsest solve (0: not available)
  bool tma_ok = false;              // bulk-copy relaxation apply available (and enabled by params.tma)
  int num_sms = 0;
  int plain_tau = 0;                // 1: the travel-time input is plain tau (adr_operator_create_tau)
  int* tma_err = nullptr;           // per problem: error words of the bulk-copy kernels
  // instrumentation (adr_profile_kernel): event pairs 2k, 2k+1 of prof_pool
  int prof_class = ADR_PROF_NONE;
  std::vector<cudaEvent_t> prof_pool;
  int prof_graph_pairs = 0;         // pairs recorded inside the captured cycle
  int prof_stream_pairs = 0;        // pairs recorded on the stream since the last collection
  bool prof_graph_fresh = false;    // the cycle was replayed since the last collection
  bool capturing = false;
  long long prof_count = 0;
  double prof_ms = 0.0;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  double* host_scal = nullptr;  // pinned: the per-problem scalars read by the solve
  size_t host_scal_count = 0;
};

constexpr int kProfPairs = 256;
// Pinned slots of the frozen-problem flags: uploads between two stream
// synchronisations of adr_solve (at most three) never reuse a slot in flight.
constexpr int kSkipSlots = 4;

// Uploads per-problem skip flags (batches only; ordered before the next launch).
static int upload_skip(Op& op, const std::vector<int>& frozen) {
  if (!op.skip) return ADR_OK;
  int* slot = op.host_skip + (size_t)op.skip_slot * op.B;
  op.skip_slot = (op.skip_slot + 1) % kSkipSlots;
  for (int pb = 0; pb < op.B; ++pb) slot[pb] = frozen[pb] ? 1 : 0;
  const cudaError_t e = cudaMemcpyAsync(op.skip, slot, sizeof(int) * (size_t)op.B, cudaMemcpyHostToDevice, op.st);
  if (e != cudaSuccess) {
    g_last_error = std::string("skip flags: ") + cudaGetErrorString(e);
    return ADR_ERR_CUDA;
  }
  return ADR_OK;
}

// Starts timing one launch of class cls on stream s; returns the pair index or -1.
static int prof_begin(Op& op, int cls, cudaStream_t s) {
  if (op.prof_class != cls || op.prof_pool.empty() || op.prof_off) return -1;
  int k;
  if (op.capturing) {
    if (op.prof_graph_pairs >= kProfPairs / 2) return -1;
    k = op.prof_graph_pairs++;
  } else {
    if (kProfPairs / 2 + op.prof_stream_pairs >= kProfPairs) return -1;
    k = kProfPairs / 2 + op.prof_stream_pairs++;
  }
  // Inside stream capture a plain record only marks a dependency; the external
  // flag turns it into an event-record node of the graph.
  cudaEventRecordWithFlags(op.prof_pool[2 * k], s, op.capturing ? cudaEventRecordExternal : 0);
  return k;
}
static void prof_end(Op& op, int k, cudaStream_t s) {
  if (k >= 0) cudaEventRecordWithFlags(op.prof_pool[2 * k + 1], s, op.capturing ? cudaEventRecordExternal : 0);
}
// Adds the completed pairs to the totals (call after a stream synchronisation).
static void prof_collect(Op& op) {
  if (op.prof_class == ADR_PROF_NONE || op.prof_pool.empty()) return;
  auto add = [&](int k) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, op.prof_pool[2 * k], op.prof_pool[2 * k + 1]) == cudaSuccess) {
      op.prof_ms += ms;
      op.prof_count += 1;
    }
  };
  if (op.prof_graph_fresh)
    for (int k = 0; k < op.prof_graph_pairs; ++k) add(k);
  for (int k = 0; k < op.prof_stream_pairs; ++k) add(kProfPairs / 2 + k);
  op.prof_graph_fresh = false;
  op.prof_stream_pairs = 0;
  cudaGetLastError();
}

static bool can_coarsen(const Dims& g) {
  for (int d = 0; d < g.dim; ++d)
    if (g.n[d] % 2 == 0 || g.n[d] < 5) return false;
  return true;
}

// One problem's grid record from its nodes and spacing.
static ProblemDims problem_dims(int dim, const int* n, const double* h) {
  const Dims d = make_dims(dim, n);
  ProblemDims q{};
  for (int k = 0; k < 3; ++k) { q.n[k] = d.n[k]; q.h[k] = k < dim ? h[k] : 1.0; }
  q.N = d.N; q.s1 = d.s1; q.s2 = d.s2;
  q.mul0 = d.mul0; q.mul1 = d.mul1; q.shr0 = d.shr0; q.shr1 = d.shr1;
  return q;
}

// The grids of every level (op.lvg[0..nlev), op.tab for unequal grids): a
// level exists while every problem's grid coarsens (reading M1), up to
// params.levels.  Fixed at creation; the tables' device copies are set by plan().
static void plan_levels(Op& op) {
  op.nlev = 0;
  for (int l = 0; l < op.p.levels; ++l) {
    Dims g;
    if (!op.hetero) {
      if (l == 0) {
        g = op.g0;
      } else {
        if (!can_coarsen(op.lvg[l - 1])) break;
        int nc[3];
        for (int d = 0; d < 3; ++d) nc[d] = (op.lvg[l - 1].n[d] - 1) / 2 + 1;
        g = make_dims(op.dim, nc);
      }
    } else {
      std::vector<ProblemDims> t(op.B);
      bool ok = true;
      for (int pb = 0; pb < op.B && ok; ++pb) {
        int nn[3];
        double hh[3];
        for (int d = 0; d < 3; ++d) {
          nn[d] = l == 0 ? op.pn[3 * pb + d] : (op.tab[l - 1][pb].n[d] - 1) / 2 + 1;
          hh[d] = l == 0 ? op.ph[3 * pb + d] : 2.0 * op.tab[l - 1][pb].h[d];
        }
        if (l > 0) ok = can_coarsen(make_dims(op.dim, op.tab[l - 1][pb].n));
        t[pb] = problem_dims(op.dim, nn, hh);
      }
      if (!ok) break;
      int64_t off = 0, soff = 0;
      int big = 0;
      for (int pb = 0; pb < op.B; ++pb) {
        t[pb].off = off;
        t[pb].soff = soff;
        off += t[pb].N;
        soff += stencil_entries_dim(t[pb].N, op.dim);
        if (t[pb].N > t[big].N) big = pb;
      }
      g = make_dims(op.dim, t[big].n);   // the largest grid sizes the launches
      g.total = off;
      op.tab[l] = t;
    }
    g.B = op.B;
    g.mrcap = op.p.relax_blocks;
    if (!op.hetero) g.total = g.N * op.B;
    op.lvg[l] = g;
    op.nlev = l + 1;
  }
}

// Stored-stencil entries of level l over the batch.
static int64_t stencil_total(const Op& op, int l) {
  if (!op.hetero) return stencil_entries_dim(op.lvg[l].N, op.dim) * op.B;
  const ProblemDims& q = op.tab[l].back();
  return q.soff + stencil_entries_dim(q.N, op.dim);
}

template <typename T> static void plan_hierarchy(Op& op, Hier<T>& H, Arena& a) {
  const adr_params_t& p = op.p;
  H.L = op.nlev;
  for (int l = 0; l < H.L; ++l) {
    H.lv[l].g = op.lvg[l];
    H.lv[l].g.pd = op.dtab[l];
    H.lv[l].g.skip = op.skip;
  }
  const size_t row_reals = op.p.rescale ? (size_t)2 * (1 + 4 * op.dim) : (size_t)(2 + 4 * op.dim);
  H.packed = a.take<T>(row_reals * (size_t)op.g0.total);
  for (int l = 0; l < H.L; ++l) {
    Level<T>& L = H.lv[l];
    const size_t NB = (size_t)L.g.total;
    L.A = l > 0 ? a.take<C<T>>((size_t)stencil_total(op, l)) : nullptr;
    L.dinv = a.take<C<T>>(NB);
    L.b = a.take<C<T>>(NB);
    L.x = a.take<C<T>>(NB);
    L.r = a.take<C<T>>(NB);
    L.t = a.take<C<T>>(NB);
    L.z = a.take<C<T>>(NB);
    L.kdim = 0;
    if (l == H.L - 1) L.kdim = p.coarse_iterations;
    else if (p.cycle == ADR_CYCLE_K && l > 0) L.kdim = p.kcycle_iterations;
    if (L.kdim > 0) {
      L.KV = a.take<C<T>>((size_t)(L.kdim + 1) * NB);
      L.KZ = (l == H.L - 1) ? nullptr : a.take<C<T>>((size_t)L.kdim * NB);
      take_arnoldi(a, L.ks, L.kdim, op.B);
    }
  }
  const size_t B = (size_t)op.B;
  // persistent coarsest solve: one block per 1024 nodes, all problems co-resident
  H.gs = GridScratch{};
  const int per_problem = op.grid_coresident / op.B;
  const Level<T>& Lc = H.lv[H.L - 1];
  if (H.L > 1 && per_problem > 0 && Lc.kdim <= kGridMaxK) {
    const int64_t want = (Lc.g.N + 1023) / 1024;
    H.gs.nblk = (int)(want < per_problem ? want : per_problem);
    H.gs.part = a.take<double2>((size_t)2 * H.gs.nblk * (kGridMaxK + 1) * B);
    H.gs.tot = a.take<double2>((size_t)(kGridMaxK + 1) * B);
    H.gs.bar = a.take<unsigned>(2 * B);
    H.gs.err = a.take<int>(B);
  }
}

// The adjoint hierarchy: its own operators (stencils and inverse diagonals)
// on the forward hierarchy's grids and work vectors.
template <typename T> static void plan_adjoint(const Hier<T>& H, Hier<T>& HT, Arena& a, int dim) {
  const int S = dim == 2 ? kPattern2 : kPattern3;
  HT.L = H.L;
  for (int l = 0; l < H.L; ++l) {
    HT.lv[l] = H.lv[l];
    const size_t N = (size_t)H.lv[l].g.N;
    HT.lv[l].A = l > 0 ? a.take<C<T>>((size_t)stencil_entries((int64_t)N, S)) : nullptr;
    HT.lv[l].dinv = a.take<C<T>>(N);
  }
  HT.gs = H.gs;   // the two cycles never run at the same time
}

static void plan(Op& op, Arena& a) {
  const size_t B = (size_t)op.B;
  const size_t N = (size_t)op.g0.N;
  const size_t NB = (size_t)op.g0.total;
  for (int l = 0; l < op.nlev; ++l) op.dtab[l] = op.hetero ? a.take<ProblemDims>(B) : nullptr;
  op.skip = op.B > 1 ? a.take<int>(B) : nullptr;
  op.g0.pd = op.dtab[0];
  op.g0.skip = op.skip;
  for (int d = 0; d < op.dim; ++d) {
    op.gd[d] = a.take<double>(NB);
    op.td[d] = a.take<double>(NB);
    op.gf[d] = a.take<float>(NB);
    op.tf[d] = a.take<float>(NB);
  }
  op.rho = a.take<double2>(NB);
  op.rhof = a.take<float>(2 * NB);
  op.tau = a.take<double>(NB);
  op.srow = a.take<double2>(kCross3 * B);
  op.srowf = a.take<float>(2 * kCross3 * B);
  if (op.p.shift != 0.0) {
    op.rhos = a.take<double2>(NB);
    op.rhosf = a.take<float>(2 * NB);
    op.srows = a.take<double2>(kCross3 * B);
    op.srowsf = a.take<float>(2 * kCross3 * B);
  }
  if (op.p.rescale) op.phase = a.take<double2>(NB);
  if (op.p.precond_precision == ADR_F64) plan_hierarchy(op, op.h64, a);
  else plan_hierarchy(op, op.h32, a);
  const int m = op.p.restart;
  op.V = a.take<double2>((size_t)(m + 1) * NB);
  op.Z = a.take<double2>((size_t)m * NB);
  op.b = a.take<double2>(NB);
  op.r = a.take<double2>(NB);
  op.packed_out = a.take<double>((size_t)(2 + 4 * op.dim) * NB);
  if (op.p.outer_df && op.p.precond_precision == ADR_F32 && !op.p.rescale)
    op.packed_df = a.take<float2>((size_t)(2 + 4 * op.dim) * NB);
  take_arnoldi(a, op.ost, m, op.B);
  op.ks.partial = a.take<double2>((size_t)kPartialStride * B);
  op.ks.ticket = a.take<unsigned>(B);
  op.ks.ha = a.take<double2>((size_t)kMaxDots * B);
  op.ks.hb = a.take<double2>((size_t)kMaxDots * B);
  op.ks.nrm2 = a.take<double2>(B);
  op.ks.alpha = a.take<double2>(B);
  op.dyn = a.take<FineDyn>(B);
  op.tma_err = a.take<int>(B);
  if (op.p.adjoint) {
    const size_t cross = (size_t)(1 + 4 * op.dim) * N;
    const size_t cbytes = op.p.precond_precision == ADR_F64 ? sizeof(double2) : sizeof(float2);
    op.rows_out = a.take<double2>(cross);
    op.rows_outT = a.take<double2>(cross);
    op.rows0 = a.take<char>(cross * cbytes);
    op.rows0T = a.take<char>(cross * cbytes);
    if (op.p.precond_precision == ADR_F64) plan_adjoint(op.h64, op.a64, a, op.dim);
    else plan_adjoint(op.h32, op.a32, a, op.dim);
  }
}

// The finest-grid operator of `scheme`; cycle = true gives the cycle's version
// (Eq. shift applied when params.shift != 0).
template <typename T> static FineOp<T> make_fine(const Op& op, int scheme, bool f32, bool cycle = false) {
  FineOp<T> f{};
  for (int d = 0; d < 3; ++d) {
    if (d < op.dim) {
      f.g[d] = f32 ? (const T*)(const void*)op.gf[d] : (const T*)(const void*)op.gd[d];
      f.t[d] = f32 ? (const T*)(const void*)op.tf[d] : (const T*)(const void*)op.td[d];
      f.h[d] = (T)op.h[d];
      f.ih2[d] = (T)(1.0 / (op.h[d] * op.h[d]));
      f.ih[d] = (T)(1.0 / op.h[d]);
      f.hih[d] = (T)(0.5 / op.h[d]);
    } else {
      f.g[d] = nullptr; f.t[d] = nullptr; f.h[d] = T(1); f.ih2[d] = T(0); f.ih[d] = T(0); f.hih[d] = T(0);
    }
  }
  f.dyn = op.dyn;
  const bool shifted = cycle && op.rhos;   // Eq. shift applies to the cycle's operator only
  if (shifted) {
    f.rho = f32 ? (const C<T>*)(const void*)op.rhosf : (const C<T>*)(const void*)op.rhos;
    f.src_row = f32 ? (const C<T>*)(const void*)op.srowsf : (const C<T>*)(const void*)op.srows;
  } else {
    f.rho = f32 ? (const C<T>*)(const void*)op.rhof : (const C<T>*)(const void*)op.rho;
    f.src_row = f32 ? (const C<T>*)(const void*)op.srowf : (const C<T>*)(const void*)op.srow;
  }
  f.near = op.p.near_source;
  set_scheme(f, scheme, op.p.beta);
  return f;
}

// The outer iteration's float64 operator (params.scheme, unshifted), read
// from the packed rows written at setup.
static FineOp<double> outer_op(const Op& op) {
  FineOp<double> f = make_fine<double>(op, op.p.scheme, false);
  f.packed = op.packed_out;
  return f;
}

// Grid of the bulk-copy relaxation applies: one block per SM, or
// params.relax_blocks when that is smaller (every warp then walks several
// tiles; a launch shape only).
static int tma_blocks(const Op& op) {
  return op.p.relax_blocks > 0 && op.p.relax_blocks < op.num_sms ? op.p.relax_blocks : op.num_sms;
}

// ---------------------------------------------------------------------------
// Level operations
// ---------------------------------------------------------------------------
template <typename T> struct Cycle {
  Op& op;
  Hier<T>& H;
  cudaStream_t st;

  void apply(int l, const C<T>* x, C<T>* y) {
    if (l == 0) {
      launch_fine_apply<T>(H.lv[0].g, H.prec, x, y, st);
    } else if constexpr (sizeof(T) == 4) {
      if (op.tma_ok) launch_stencil_apply_tma(H.lv[l].g, H.lv[l].A, x, y, op.tma_err, tma_blocks(op), op.p.tma, st);
      else launch_stencil_apply<T>(H.lv[l].g, H.lv[l].A, x, y, st);
    } else {
      launch_stencil_apply<T>(H.lv[l].g, H.lv[l].A, x, y, st);
    }
  }
  void residual(int l, const C<T>* b, const C<T>* x, C<T>* r) {
    if (l == 0) launch_fine_residual<T>(H.lv[0].g, H.prec, b, x, r, st);
    else launch_stencil_residual<T>(H.lv[l].g, H.lv[l].A, b, x, r, st);
  }
  void jacobi(int l, const C<T>* b, const C<T>* xin, C<T>* xout, T w) {
    if (l == 0) launch_fine_jacobi<T>(H.lv[0].g, H.prec, b, xin, xout, w, st);
    else launch_stencil_jacobi<T>(H.lv[l].g, H.lv[l].A, H.lv[l].dinv, b, xin, xout, w, st);
  }
  void residual_dinv(int l, const C<T>* b, const C<T>* x, C<T>* r, C<T>* z) {
    if (l == 0) {
      launch_fine_residual_dinv<T>(H.lv[0].g, H.prec, b, x, H.lv[0].dinv, r, z, st);
    } else if constexpr (sizeof(T) == 4) {
      if (op.tma_ok)
        launch_stencil_residual_dinv_tma(H.lv[l].g, H.lv[l].A, b, x, H.lv[l].dinv, r, z, op.tma_err, tma_blocks(op),
                                         op.p.tma, st);
      else
        launch_stencil_residual_dinv<T>(H.lv[l].g, H.lv[l].A, b, x, H.lv[l].dinv, r, z, st);
    } else {
      launch_stencil_residual_dinv<T>(H.lv[l].g, H.lv[l].A, b, x, H.lv[l].dinv, r, z, st);
    }
  }
  void mr_apply(int l, const C<T>* z, const C<T>* r, C<T>* w) {
    const int pk = prof_begin(op, l == 0 ? ADR_PROF_FINE_RELAX : (l == 1 ? ADR_PROF_LEVEL1_RELAX : -1), st);
    if (l == 0) {
      launch_fine_mr_apply<T>(H.lv[0].g, H.prec, z, r, w, op.ks.partial, op.ks.ticket, op.ks.alpha, st);
    } else if constexpr (sizeof(T) == 4) {
      if (op.tma_ok)
        launch_stencil_mr_apply_tma(H.lv[l].g, H.lv[l].A, z, r, w, op.ks.partial, op.ks.ticket, op.ks.alpha, op.tma_err,
                                    tma_blocks(op), op.p.tma, st);
      else
        launch_stencil_mr_apply<T>(H.lv[l].g, H.lv[l].A, z, r, w, op.ks.partial, op.ks.ticket, op.ks.alpha, st);
    } else {
      launch_stencil_mr_apply<T>(H.lv[l].g, H.lv[l].A, z, r, w, op.ks.partial, op.ks.ticket, op.ks.alpha, st);
    }
    prof_end(op, pk, st);
  }

  // `sweeps` relaxations on A_l x = b; x_zero says x holds zero on entry.
  // Returns true when L.r holds b - A x afterwards.
  bool relax(int l, const C<T>* b, C<T>* x, int sweeps, bool& x_zero) {
    Level<T>& L = H.lv[l];
    const int64_t n = L.g.N;
    if (sweeps <= 0) return false;
    if (op.p.relax == ADR_RELAX_JACOBI) {
      const T w = (T)op.p.jacobi_weight[l];
      C<T>* cur = x;
      C<T>* oth = L.t;
      for (int s = 0; s < sweeps; ++s) {
        jacobi(l, b, x_zero ? nullptr : cur, oth, w);
        x_zero = false;
        C<T>* tmp = cur; cur = oth; oth = tmp;
      }
      if (cur != x) launch_copy<T>(cur, x, L.g.total, st);
      return false;
    }
    // Minimal-residual Jacobi: z = D^{-1} r, w = A z, alpha = (w^H r)/(w^H w),
    // x += alpha z, r -= alpha w (two launches per sweep).
    const C<T>* rsrc;
    if (x_zero) {
      launch_cmul_vec<T>(L.dinv, b, L.z, L.g.total, st);
      rsrc = b;
    } else {
      residual_dinv(l, b, x, L.r, L.z);
      rsrc = L.r;
    }
    for (int s = 0; s < sweeps; ++s) {
      mr_apply(l, L.z, rsrc, L.t);
      launch_mr_update2<T>(x, L.z, rsrc, L.r, L.t, op.ks.alpha, L.dinv, s + 1 < sweeps ? L.z : nullptr, x_zero && s == 0,
                           L.g, st);
      rsrc = L.r;
    }
    x_zero = false;
    return true;
  }

  // Arnoldi step j: w (holding A z_j) orthogonalised against V_0..V_j by CGS2,
  // Hessenberg column and rotation updated; V_{j+1} = w / |w| if store_next.
  // Vb holds the basis at stride ld = B n (vector-major over the batch).
  void arnoldi(ArnoldiState& ks, C<T>* Vb, int64_t ld, int j, C<T>* w, const Dims& g, bool store_next) {
    launch_cgs2<T>(Vb, ld, j + 1, w, g, op.ks, ks, j, st);
    if (store_next) launch_scale_inv_norm<T>(w, Vb + (int64_t)(j + 1) * ld, op.ks.nrm2, g, st);
  }

  // Fixed-count GMRES from zero, right-preconditioned by D^{-1} (coarsest level).
  void coarse_solve(int l, const C<T>* b, C<T>* x) {
    const int pk = prof_begin(op, ADR_PROF_COARSEST, st);
    coarse_solve_impl(l, b, x);
    prof_end(op, pk, st);
  }
  void coarse_solve_impl(int l, const C<T>* b, C<T>* x) {
    Level<T>& L = H.lv[l];
    const int64_t n = L.g.N;
    const int k = L.kdim;
    const int form = op.p.coarse_solver;
    const bool cluster_ok = l > 0 && op.cluster_size > 0 && k <= kClusterKMax;
    const bool grid_ok = l > 0 && H.gs.nblk > 0 && k <= kGridMaxK && !op.hetero;
    if (form == ADR_COARSE_CLUSTER || (form == ADR_COARSE_AUTO && n <= kClusterCoarse)) {
      if (cluster_ok) {
        launch_coarse_gmres_cluster<T>(L.g, L.A, L.dinv, b, x, L.KV, L.z, k, L.ks, op.cluster_size, st);
        return;
      }
    }
    if (l > 0 && (form == ADR_COARSE_CTA || (form == ADR_COARSE_AUTO && n <= kSmallCoarse))) {
      launch_coarse_gmres_cta<T>(L.g, L.A, L.dinv, b, x, L.KV, L.z, k, L.ks, st);
      return;
    }
    // The persistent form is opt-in: on the 65x65x33 coarsest grid of the
    // 257x257x129 workload it takes about 0.92 ms per solve against 0.59 ms
    // for the per-step launches (four grid barriers per GMRES step; the whole
    // ADR solve 455 against 409 ms).
    if (grid_ok && form == ADR_COARSE_GRID) {
      launch_coarse_gmres_grid<T>(L.g, L.A, L.dinv, b, x, L.KV, L.z, k, H.gs, op.p.reorth_eta, st);
      return;
    }
    // Per step: the apply fused with the first Gram-Schmidt pass and the
    // selective decision (or the two launches), the second pass where the
    // first cancelled (reading M2, eta = params.reorth_eta; it returns at once
    // otherwise), and the next basis vector with its Jacobi-scaled direction;
    // the last step's column also solves the least-squares problem.
    const int64_t ld = L.g.total;
    const double eta = op.p.reorth_eta;
    launch_norm_start<T>(b, L.g, op.ks, &L.ks, st);
    launch_scale_dinv<T>(b, L.KV, L.dinv, L.z, op.ks.nrm2, L.g, st);   // V_0 and z = D^{-1} V_0
    for (int j = 0; j < k; ++j) {
      const int finish = j + 1 == k ? k : 0;
      bool fused = false;
      if constexpr (sizeof(T) == 4) {
        if (op.tma_ok && k < kMaxArnoldiDots - 2) {
          launch_stencil_arnoldi_tma(L.g, L.A, L.z, L.t, L.KV, ld, j + 1, op.ks, L.ks, j, finish, eta, op.tma_err,
                                     tma_blocks(op), op.p.tma, st);
          fused = true;
        }
      }
      if (!fused) {
        apply(l, L.z, L.t);
        launch_cgs_dots_sel<T>(L.KV, ld, j + 1, L.t, L.g, op.ks, L.ks, j, finish, eta, st);
      }
      launch_cgs_reorth<T>(L.KV, ld, j + 1, L.t, L.g, op.ks, L.ks, j, finish, st);
      if (j + 1 < k) launch_cgs_next<T>(L.KV, ld, j + 1, L.t, L.g, op.ks, L.KV + (int64_t)(j + 1) * ld, L.dinv, L.z, st);
    }
    launch_combine_dinv<T>(x, L.KV, ld, k, L.ks, L.dinv, L.g, st);
  }

  // Inner flexible GMRES of the K-cycle on level l, from zero: kdim steps,
  // or fewer when params.kcycle_threshold > 0 (Alg. Kcycle's early exit:
  // the instance's convergence target is that fraction of |b|, and the back
  // substitution stops at the column that met it).
  void kcycle(int l, const C<T>* b, C<T>* x) {
    Level<T>& L = H.lv[l];
    const int64_t n = L.g.N;
    const int k = L.kdim;
    const int64_t ld = L.g.total;
    launch_norm_start<T>(b, L.g, op.ks, &L.ks, st, op.p.kcycle_threshold);
    launch_scale_inv_norm<T>(b, L.KV, op.ks.nrm2, L.g, st);
    for (int j = 0; j < k; ++j) {
      C<T>* zj = L.KZ + (int64_t)j * ld;
      cycle(l, L.KV + (int64_t)j * ld, zj);
      apply(l, zj, L.t);
      arnoldi(L.ks, L.KV, ld, j, L.t, L.g, j + 1 < k);
    }
    launch_backsolve(L.ks, k, st, L.g.B);
    launch_combine<T>(x, L.KZ, ld, k, L.ks, true, L.g, st);
  }

  // x = B_l^{-1} b, zero initial guess (Alg. TwoGrid / Alg. Kcycle).
  void cycle(int l, const C<T>* b, C<T>* x) {
    if (l == H.L - 1) { coarse_solve(l, b, x); return; }
    Level<T>& L = H.lv[l];
    Level<T>& Lc = H.lv[l + 1];
    const int64_t n = L.g.N;
    bool x_zero = true;
    const bool rvalid = relax(l, b, x, op.p.pre_sweeps[l], x_zero);
    if (x_zero) {
      launch_restrict<T>(L.g, Lc.g, b, Lc.b, st);
    } else {
      if (!rvalid) residual(l, b, x, L.r);
      launch_restrict<T>(L.g, Lc.g, L.r, Lc.b, st);
    }
    if (op.p.cycle == ADR_CYCLE_K && l + 1 < H.L - 1) kcycle(l + 1, Lc.b, Lc.x);
    else cycle(l + 1, Lc.b, Lc.x);
    if (x_zero) { launch_zero<T>(x, L.g.total, st); x_zero = false; }
    launch_prolong_add<T>(L.g, Lc.g, Lc.x, x, st);
    relax(l, b, x, op.p.post_sweeps[l], x_zero);
  }
};

template <typename T> static int build_hierarchy(Op& op, Hier<T>& H) {
  const bool f32 = sizeof(T) == 4;
  H.prec = make_fine<T>(op, op.p.prec_scheme, f32, true);
  if (op.p.rescale) {
    // Alg. ADRlong, stage 2: the cycle acts on M A M^{-1}, stored as rows
    C<T>* rows = (C<T>*)(void*)H.packed;
    launch_fine_store_rows(H.lv[0].g, H.prec, rows, op.st);
    launch_rows_rescale<T>(H.lv[0].g, rows, op.phase, op.st);
    H.prec.rows = rows;
  } else {
    launch_fine_pack<T>(H.lv[0].g, H.prec, H.packed, op.st);   // the cycle reads the packed rows from here on
    H.prec.packed = H.packed;
  }
  Level<T>& L0 = H.lv[0];
  launch_fine_dinv<T>(L0.g, H.prec, nullptr, L0.dinv, op.st);
  for (int l = 1; l < H.L; ++l) {
    if (l == 1) launch_galerkin_fine<T>(H.lv[0].g, H.lv[1].g, H.prec, H.lv[1].A, H.lv[1].dinv, op.st);
    else launch_galerkin_stored<T>(H.lv[l - 1].g, H.lv[l].g, H.lv[l - 1].A, H.lv[l].A, H.lv[l].dinv, op.st);
  }
  return check_launch("hierarchy setup");
}

// Hierarchy on A^H: the cycle's fine operator stored as rows, conjugate-
// transposed, and the Galerkin products P^T A^H P of its levels (the same
// kernels as the forward hierarchy, reading the stored rows).
template <typename T> static int build_adjoint(Op& op, Hier<T>& H, Hier<T>& HT) {
  launch_fine_store_rows(H.lv[0].g, H.prec, (C<T>*)op.rows0, op.st);
  launch_rows_adjoint<T>(H.lv[0].g, (const C<T>*)op.rows0, (C<T>*)op.rows0T, op.st);
  HT.prec = H.prec;
  HT.prec.rows = (const C<T>*)op.rows0T;
  launch_fine_dinv<T>(HT.lv[0].g, HT.prec, nullptr, HT.lv[0].dinv, op.st);
  for (int l = 1; l < HT.L; ++l) {
    if (l == 1) launch_galerkin_fine<T>(HT.lv[0].g, HT.lv[1].g, HT.prec, HT.lv[1].A, HT.lv[1].dinv, op.st);
    else launch_galerkin_stored<T>(HT.lv[l - 1].g, HT.lv[l].g, HT.lv[l - 1].A, HT.lv[l].A, HT.lv[l].dinv, op.st);
  }
  return check_launch("adjoint hierarchy setup");
}

// Coefficients, their float32 copies and the Galerkin hierarchy for the
// current source / frequency, written into the operator's arena (no sync).
static int setup(Op& op, const double* kappa, const double* tau1, const double* gamma) {
  const int64_t N = op.g0.N;
  const int64_t NB = op.g0.total;
  for (int pb = 0; pb < op.B; ++pb) {   // per-problem coefficients (setup, not the cycle)
    // this problem alone: its grid, where its entries start, its spacing
    const ProblemDims* q = op.hetero ? &op.tab[0][pb] : nullptr;
    const Dims g1 = make_dims(op.dim, q ? q->n : op.g0.n);
    const int64_t o = q ? q->off : (int64_t)pb * N;
    const double* hp = q ? q->h : op.h;
    FineDyn dyn{};
    dyn.omega = op.omegas[pb];
    for (int d = 0; d < 3; ++d) dyn.src[d] = op.srcs[3 * pb + d];
    dyn.src_index = dyn.src[0] + g1.s1 * dyn.src[1] + g1.s2 * dyn.src[2];
    launch_set_dyn(op.dyn + pb, dyn, op.st);
    FineInputs in{};
    in.kappa = kappa + o; in.tau1 = tau1 + o; in.gamma = gamma + o;
    for (int d = 0; d < 3; ++d) { in.src[d] = dyn.src[d]; in.h[d] = hp[d]; in.ih[d] = 1.0 / hp[d]; }
    in.omega = dyn.omega;
    in.plain = op.plain_tau;
    double* gd[3] = {nullptr, nullptr, nullptr};
    double* td[3] = {nullptr, nullptr, nullptr};
    for (int d = 0; d < op.dim; ++d) { gd[d] = op.gd[d] + o; td[d] = op.td[d] + o; }
    launch_coefficients(g1, in, gd, td, op.rho + o, op.tau + o, op.srow + (int64_t)pb * kCross3, op.st);
    if (op.rhos)
      launch_shift(g1, in, op.p.shift, op.rho + o, op.srow + (int64_t)pb * kCross3, op.rhos + o,
                   op.srows + (int64_t)pb * kCross3, op.st);
  }
  for (int d = 0; d < op.dim; ++d) {
    launch_to_f32(op.gd[d], op.gf[d], NB, op.st);
    launch_to_f32(op.td[d], op.tf[d], NB, op.st);
  }
  launch_to_f32((const double*)op.rho, op.rhof, 2 * NB, op.st);
  launch_to_f32((const double*)op.srow, op.srowf, 2 * kCross3 * op.B, op.st);
  if (op.rhos) {
    launch_to_f32((const double*)op.rhos, op.rhosf, 2 * NB, op.st);
    launch_to_f32((const double*)op.srows, op.srowsf, 2 * kCross3 * op.B, op.st);
  }
  if (op.phase) launch_phase(op.g0, op.tau, op.dyn, op.phase, op.st);
  launch_fine_pack<double>(op.g0, make_fine<double>(op, op.p.scheme, false), op.packed_out, op.st);
  if (op.packed_df) launch_split_df(op.packed_out, op.packed_df, (int64_t)(2 + 4 * op.dim) * NB, op.st);
  ADR_TRY(check_launch("coefficients"));
  ADR_TRY(op.p.precond_precision == ADR_F64 ? build_hierarchy(op, op.h64) : build_hierarchy(op, op.h32));
  if (!op.p.adjoint) return ADR_OK;
  launch_fine_store_rows(op.g0, make_fine<double>(op, op.p.scheme, false), op.rows_out, op.st);
  launch_rows_adjoint<double>(op.g0, op.rows_out, op.rows_outT, op.st);
  return op.p.precond_precision == ADR_F64 ? build_adjoint(op, op.h64, op.a64) : build_adjoint(op, op.h32, op.a32);
}

// Runs the cycle of level 0 from H.lv[0].b into H.lv[0].x: captured into a
// CUDA graph on first use (every pointer and parameter it touches is fixed
// for the operator's lifetime, per-source values live in device memory) and
// replayed on the operator's stream.
template <typename T> static int run_cycle(Op& op, Hier<T>& H, bool adj = false) {
  Level<T>& L0 = H.lv[0];
  op.prof_off = adj;
  if (!op.use_graph) {
    const int pk = adj ? -1 : prof_begin(op, ADR_PROF_CYCLE, op.st);
    Cycle<T> c{op, H, op.st};
    c.cycle(0, L0.b, L0.x);
    prof_end(op, pk, op.st);
    op.prof_off = false;
    return check_launch("cycle");
  }
  cudaGraphExec_t& exec = adj ? op.cycle_exec_adj : op.cycle_exec;
  long long& kernels = adj ? op.cycle_kernels_adj : op.cycle_kernels;
  if (!exec) {
    const long long before = g_launches.load(std::memory_order_relaxed);
    ADR_CUDA(cudaStreamBeginCapture(op.cap, cudaStreamCaptureModeThreadLocal));
    if (!adj) op.prof_graph_pairs = 0;
    op.capturing = true;
    Cycle<T> c{op, H, op.cap};
    c.cycle(0, L0.b, L0.x);
    op.capturing = false;
    op.prof_off = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(op.cap, &graph);
    if (e != cudaSuccess) return fail(ADR_ERR_CUDA, std::string("cycle capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      exec = nullptr;
      return fail(ADR_ERR_CUDA, std::string("cycle graph instantiation: ") + cudaGetErrorString(e));
    }
    kernels = g_launches.load(std::memory_order_relaxed) - before;
    count_launches((int)-kernels);  // capture launched nothing; replays are counted below
  }
  op.prof_off = false;
  const int pk = adj ? -1 : prof_begin(op, ADR_PROF_CYCLE, op.st);
  ADR_CUDA(cudaGraphLaunch(exec, op.st));
  prof_end(op, pk, op.st);
  count_launches((int)kernels);
  if (!adj) op.prof_graph_fresh = true;
  return ADR_OK;
}

// One preconditioner application on float64 vectors (casting for a float32
// cycle); adj selects the cycle on A^H.
// z = K v with K the cycle; with params.rescale, z = M^{-1} K (M v) (the
// cycle works on the rescaled variables, Alg. ADRlong; the same form for the
// adjoint since M is unitary).
static int precondition(Op& op, const double2* v, double2* z, bool adj = false) {
  const int64_t NB = op.g0.total;
  if (op.p.precond_precision == ADR_F64) {
    Hier<double>& H = adj ? op.a64 : op.h64;
    if (op.phase) launch_phase_cast<double, double>(v, op.phase, false, H.lv[0].b, NB, op.st);
    else launch_copy<double>(v, H.lv[0].b, NB, op.st);
    ADR_TRY(run_cycle(op, H, adj));
    if (op.phase) launch_phase_cast<double, double>(H.lv[0].x, op.phase, true, z, NB, op.st);
    else launch_copy<double>(H.lv[0].x, z, NB, op.st);
  } else {
    Hier<float>& H = adj ? op.a32 : op.h32;
    if (op.phase) launch_phase_cast<double, float>(v, op.phase, false, H.lv[0].b, NB, op.st);
    else launch_ccast<double, float>(v, H.lv[0].b, NB, op.st);
    ADR_TRY(run_cycle(op, H, adj));
    if (op.phase) launch_phase_cast<float, double>(H.lv[0].x, op.phase, true, z, NB, op.st);
    else launch_ccast<float, double>(H.lv[0].x, z, NB, op.st);
  }
  return ADR_OK;
}

static int read_scalars(Op& op, const double* dev, int count) {
  if ((size_t)count > op.host_scal_count) return fail(ADR_ERR_STATE, "scalar read larger than the host buffer");
  ADR_CUDA(cudaMemcpyAsync(op.host_scal, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, op.st));
  ADR_CUDA(cudaStreamSynchronize(op.st));
  prof_collect(op);
  return ADR_OK;
}

static int validate_params(const adr_params_t& p) {
  if (p.levels < 1 || p.levels > ADR_MAX_LEVELS) return fail(ADR_ERR_ARG, "levels must be in [1, 8]");
  if (!(p.beta >= 0.0 && p.beta <= 1.0)) return fail(ADR_ERR_ARG, "beta must be in [0, 1]");
  if (p.cycle != ADR_CYCLE_V && p.cycle != ADR_CYCLE_K) return fail(ADR_ERR_ARG, "unknown cycle");
  if (p.relax != ADR_RELAX_JACOBI && p.relax != ADR_RELAX_MR) return fail(ADR_ERR_ARG, "unknown relaxation");
  if (p.coarse_iterations < 1 || p.coarse_iterations > 64) return fail(ADR_ERR_ARG, "coarse_iterations must be in [1, 64]");
  if (p.kcycle_iterations < 1 || p.kcycle_iterations > 16) return fail(ADR_ERR_ARG, "kcycle_iterations must be in [1, 16]");
  if (p.restart < 1 || p.restart > 64) return fail(ADR_ERR_ARG, "restart must be in [1, 64]");
  if (p.precond_precision != ADR_F64 && p.precond_precision != ADR_F32) return fail(ADR_ERR_ARG, "unknown precision");
  if (p.near_source < 1 || p.near_source > 4) return fail(ADR_ERR_ARG, "near_source must be in [1, 4]");
  if (!(p.reorth_eta >= 0.0 && p.reorth_eta <= 1e6)) return fail(ADR_ERR_ARG, "reorth_eta must be in [0, 1e6]");
  if (p.adjoint != 0 && p.adjoint != 1) return fail(ADR_ERR_ARG, "adjoint must be 0 or 1");
  if (p.relax_blocks < 0 || (int64_t)p.relax_blocks * 2 > kPartialStride)
    return fail(ADR_ERR_ARG, "relax_blocks must be in [0, 10240]");
  if (p.coarse_solver < ADR_COARSE_AUTO || p.coarse_solver > ADR_COARSE_GRID)
    return fail(ADR_ERR_ARG, "unknown coarse_solver");
  if (p.tma < 0 || p.tma > 4) return fail(ADR_ERR_ARG, "tma must be 0, 1, 2, 3 or 4");
  if (!(p.shift >= 0.0 && p.shift <= 100.0)) return fail(ADR_ERR_ARG, "shift must be in [0, 100]");
  if (p.scheme != ADR_SCHEME_2UP && p.scheme != ADR_SCHEME_1UP && p.scheme != ADR_SCHEME_CEN)
    return fail(ADR_ERR_ARG, "scheme must be ADR_SCHEME_2UP, ADR_SCHEME_1UP or ADR_SCHEME_CEN");
  if (p.prec_scheme < ADR_SCHEME_2UP || p.prec_scheme > ADR_SCHEME_PREC) return fail(ADR_ERR_ARG, "unknown prec_scheme");
  if (p.rescale != 0 && p.rescale != 1) return fail(ADR_ERR_ARG, "rescale must be 0 or 1");
  if (!(p.kcycle_threshold >= 0.0 && p.kcycle_threshold <= 1e6))
    return fail(ADR_ERR_ARG, "kcycle_threshold must be in [0, 1e6]");
  if (p.outer_df != 0 && p.outer_df != 1) return fail(ADR_ERR_ARG, "outer_df must be 0 or 1");
  for (int l = 0; l < ADR_MAX_LEVELS; ++l) {
    if (p.pre_sweeps[l] < 0 || p.pre_sweeps[l] > 16 || p.post_sweeps[l] < 0 || p.post_sweeps[l] > 16)
      return fail(ADR_ERR_ARG, "sweeps must be in [0, 16]");
    if (!(p.jacobi_weight[l] > 0.0 && p.jacobi_weight[l] <= 2.0)) return fail(ADR_ERR_ARG, "jacobi_weight must be in (0, 2]");
  }
  return ADR_OK;
}

}  // namespace adr

using namespace adr;

struct adr_op_s {
  Op op;
};

extern "C" {

const char* adr_last_error(void) { return g_last_error.c_str(); }
const char* adr_version(void) { return "0.1.0"; }

int adr_params_default(adr_params_t* p) {
  if (!p) return fail(ADR_ERR_ARG, "params is null");
  std::memset(p, 0, sizeof(*p));
  p->levels = 5;
  p->beta = 0.25;
  p->cycle = ADR_CYCLE_K;
  p->relax = ADR_RELAX_MR;
  for (int l = 0; l < ADR_MAX_LEVELS; ++l) {
    p->pre_sweeps[l] = l + 2;   // level l+1 in the paper's numbering gets l+2 relaxations
    p->post_sweeps[l] = l + 2;
    p->jacobi_weight[l] = 0.5;
  }
  p->coarse_iterations = 10;
  p->kcycle_iterations = 2;
  p->restart = 20;
  p->precond_precision = ADR_F32;
  p->near_source = 1;
  p->reorth_eta = 0.1;
  p->tma = 3;
  p->scheme = ADR_SCHEME_2UP;
  p->prec_scheme = ADR_SCHEME_PREC;
  p->outer_df = 1;
  return ADR_OK;
}

// pn, ph (batches of unequal grids): 3 node counts and 3 spacings per
// problem, in place of n and h.
static int create_impl(int dim, const int* n, const double* h, int B, const int* src, const double* omega,
                       const double* kappa, const double* tau1, const double* gamma, const adr_params_t* params,
                       void* stream, adr_op_t* out, int plain_tau = 0, const int* pn = nullptr,
                       const double* ph = nullptr) {
  if (!out) return fail(ADR_ERR_ARG, "out is null");
  *out = nullptr;
  if (dim != 2 && dim != 3) return fail(ADR_ERR_ARG, "dim must be 2 or 3");
  if (B < 1 || B > 65535) return fail(ADR_ERR_ARG, "problems must be in [1, 65535]");
  const bool hetero = pn != nullptr;
  if ((hetero ? (!ph) : (!n || !h)) || !src || !omega || !kappa || !tau1 || !gamma)
    return fail(ADR_ERR_ARG, "null argument");
  int64_t total = 0;
  for (int pb = 0; pb < (hetero ? B : 1); ++pb) {
    const int* np = hetero ? pn + 3 * pb : n;
    const double* hp = hetero ? ph + 3 * pb : h;
    for (int d = 0; d < dim; ++d) {
      if (np[d] < 4) return fail(ADR_ERR_ARG, "every axis needs at least 4 nodes");
      if (!(hp[d] > 0.0)) return fail(ADR_ERR_ARG, "spacings must be positive");
    }
    const int64_t Np = (int64_t)np[0] * np[1] * (dim > 2 ? np[2] : 1);
    total += hetero ? Np : Np * B;
  }
  for (int pb = 0; pb < B; ++pb) {
    if (!(omega[pb] > 0.0)) return fail(ADR_ERR_ARG, "omega must be positive");
    const int* np = hetero ? pn + 3 * pb : n;
    for (int d = 0; d < dim; ++d)
      if (src[3 * pb + d] < 0 || src[3 * pb + d] >= np[d]) return fail(ADR_ERR_ARG, "source outside the grid");
  }
  adr_params_t p;
  if (params) p = *params;
  else adr_params_default(&p);
  ADR_TRY(validate_params(p));
  if (p.adjoint && B > 1) return fail(ADR_ERR_ARG, "the adjoint operator is built for one problem at a time");
  if (total > ((int64_t)1 << 31) - 1) return fail(ADR_ERR_ARG, "grid too large (more than 2^31 - 1 nodes)");

  adr_op_s* h_ = new (std::nothrow) adr_op_s();
  if (!h_) return fail(ADR_ERR_OOM, "host allocation failed");
  Op& op = h_->op;
  op.dim = dim;
  op.B = B;
  op.plain_tau = plain_tau;
  op.p = p;
  op.st = (cudaStream_t)stream;
  op.hetero = hetero;
  if (hetero) {
    op.pn.assign(3 * (size_t)B, 1);
    op.ph.assign(3 * (size_t)B, 1.0);
    for (int pb = 0; pb < B; ++pb)
      for (int d = 0; d < dim; ++d) { op.pn[3 * pb + d] = pn[3 * pb + d]; op.ph[3 * pb + d] = ph[3 * pb + d]; }
  } else {
    op.g0 = make_dims(dim, n);
  }
  plan_levels(op);
  op.g0 = op.lvg[0];
  for (int d = 0; d < 3; ++d) op.h[d] = hetero ? op.ph[d] : (d < dim ? h[d] : 1.0);
  op.omegas.assign(omega, omega + B);
  op.srcs.assign(3 * (size_t)B, 0);
  for (int pb = 0; pb < B; ++pb)
    for (int d = 0; d < dim; ++d) op.srcs[3 * pb + d] = src[3 * pb + d];
  op.omega = op.omegas[0];
  for (int d = 0; d < 3; ++d) op.src[d] = op.srcs[d];
  {
    const Dims g1 = hetero ? make_dims(dim, op.tab[0][0].n) : op.g0;
    op.src_index = op.src[0] + g1.s1 * op.src[1] + g1.s2 * op.src[2];
  }

  op.grid_coresident = prepare_coarse_grid(dim, p.precond_precision == ADR_F32);
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&op.num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
  }
  op.tma_ok = p.tma && p.precond_precision == ADR_F32 && op.num_sms > 0 && prepare_stencil_tma();
  Arena sizing;
  plan(op, sizing);
  op.arena_bytes = sizing.used + 256;
  cudaError_t e = cudaMalloc(&op.arena, op.arena_bytes);
  if (e != cudaSuccess) {
    delete h_;
    cudaGetLastError();
    return fail(ADR_ERR_OOM, std::string("cudaMalloc of the operator arena failed: ") + cudaGetErrorString(e));
  }
  op.host_scal_count = std::max<size_t>(16, (size_t)B * (kNumScal > 2 ? kNumScal : 2));
  const size_t skip_doubles = ((size_t)kSkipSlots * B * sizeof(int) + sizeof(double) - 1) / sizeof(double);
  e = cudaMallocHost(&op.host_scal, (op.host_scal_count + skip_doubles) * sizeof(double));
  if (e == cudaSuccess) op.host_skip = reinterpret_cast<int*>(op.host_scal + op.host_scal_count);
  if (e != cudaSuccess) {
    cudaFree(op.arena);
    delete h_;
    return fail(ADR_ERR_OOM, "pinned host allocation failed");
  }
  Arena real;
  real.base = (char*)op.arena;
  plan(op, real);
  op.cluster_size = prepare_coarse_cluster(dim, p.precond_precision == ADR_F32);
  e = cudaStreamCreateWithFlags(&op.cap, cudaStreamNonBlocking);
  // all of the arena starts at zero: reduction tickets, convergence targets of
  // the inner Krylov instances (0 = never frozen)
  if (e == cudaSuccess) e = cudaMemsetAsync(op.arena, 0, op.arena_bytes, op.st);
  for (int l = 0; e == cudaSuccess && hetero && l < op.nlev; ++l)   // the per-problem grid tables
    e = cudaMemcpyAsync(op.dtab[l], op.tab[l].data(), sizeof(ProblemDims) * (size_t)B, cudaMemcpyHostToDevice, op.st);
  if (e != cudaSuccess) {
    if (op.cap) cudaStreamDestroy(op.cap);
    cudaFree(op.arena);
    cudaFreeHost(op.host_scal);
    delete h_;
    return fail(ADR_ERR_CUDA, std::string("operator streams: ") + cudaGetErrorString(e));
  }

  int rc = setup(op, kappa, tau1, gamma);
  if (rc != ADR_OK) {
    cudaStreamSynchronize(op.st);
    cudaStreamDestroy(op.cap);
    cudaFree(op.arena);
    cudaFreeHost(op.host_scal);
    delete h_;
    return rc;
  }
  *out = h_;
  return ADR_OK;
}

int adr_operator_create(int dim, const int* n, const double* h, const int* src, double omega, const double* kappa,
                        const double* tau1, const double* gamma, const adr_params_t* params, void* stream, adr_op_t* out) {
  if (!src) return fail(ADR_ERR_ARG, "null argument");
  const int s3[3] = {src[0], dim > 1 ? src[1] : 0, dim > 2 ? src[2] : 0};
  return create_impl(dim, n, h, 1, s3, &omega, kappa, tau1, gamma, params, stream, out);
}

int adr_operator_create_tau(int dim, const int* n, const double* h, const int* src, double omega, const double* kappa,
                            const double* tau, const double* gamma, const adr_params_t* params, void* stream,
                            adr_op_t* out) {
  if (!src) return fail(ADR_ERR_ARG, "null argument");
  const int s3[3] = {src[0], dim > 1 ? src[1] : 0, dim > 2 ? src[2] : 0};
  return create_impl(dim, n, h, 1, s3, &omega, kappa, tau, gamma, params, stream, out, 1);
}

int adr_batch_create(int dim, const int* n, const double* h, int problems, const int* src, const double* omega,
                     const double* kappa, const double* tau1, const double* gamma, const adr_params_t* params,
                     void* stream, adr_op_t* out) {
  return create_impl(dim, n, h, problems, src, omega, kappa, tau1, gamma, params, stream, out);
}

int adr_batch_create_grids(int dim, int problems, const int* n, const double* h, const int* src, const double* omega,
                           const double* kappa, const double* tau1, const double* gamma, const adr_params_t* params,
                           void* stream, adr_op_t* out) {
  if (!n || !h) return fail(ADR_ERR_ARG, "null argument");
  return create_impl(dim, nullptr, nullptr, problems, src, omega, kappa, tau1, gamma, params, stream, out, 0, n, h);
}

static int update_impl(Op& op, const int* src, const double* omega, const double* kappa, const double* tau1,
                       const double* gamma) {
  if (!src || !omega || !kappa || !tau1 || !gamma) return fail(ADR_ERR_ARG, "null argument");
  for (int pb = 0; pb < op.B; ++pb) {
    if (!(omega[pb] > 0.0)) return fail(ADR_ERR_ARG, "omega must be positive");
    const int* np = op.hetero ? op.tab[0][pb].n : op.g0.n;
    for (int d = 0; d < op.dim; ++d)
      if (src[3 * pb + d] < 0 || src[3 * pb + d] >= np[d]) return fail(ADR_ERR_ARG, "source outside the grid");
  }
  for (int pb = 0; pb < op.B; ++pb) {
    op.omegas[pb] = omega[pb];
    for (int d = 0; d < 3; ++d) op.srcs[3 * pb + d] = d < op.dim ? src[3 * pb + d] : 0;
  }
  op.omega = op.omegas[0];
  for (int d = 0; d < 3; ++d) op.src[d] = op.srcs[d];
  const Dims g1 = op.hetero ? make_dims(op.dim, op.tab[0][0].n) : op.g0;
  op.src_index = op.src[0] + g1.s1 * op.src[1] + g1.s2 * op.src[2];
  return setup(op, kappa, tau1, gamma);
}

int adr_operator_update(adr_op_t h, const int* src, double omega, const double* kappa, const double* tau1,
                        const double* gamma) {
  if (!h || !src) return fail(ADR_ERR_ARG, "null argument");
  Op& op = h->op;
  if (op.B != 1) return fail(ADR_ERR_STATE, "batched operator: use adr_batch_update");
  const int s3[3] = {src[0], op.dim > 1 ? src[1] : 0, op.dim > 2 ? src[2] : 0};
  return update_impl(op, s3, &omega, kappa, tau1, gamma);
}

int adr_batch_update(adr_op_t h, const int* src, const double* omega, const double* kappa, const double* tau1,
                     const double* gamma) {
  if (!h) return fail(ADR_ERR_ARG, "null argument");
  return update_impl(h->op, src, omega, kappa, tau1, gamma);
}

long long adr_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int adr_profile_kernel(adr_op_t h, int kernel_class) {
  if (!h) return fail(ADR_ERR_ARG, "null argument");
  if (kernel_class < ADR_PROF_NONE || kernel_class > ADR_PROF_CYCLE) return fail(ADR_ERR_ARG, "unknown kernel class");
  Op& op = h->op;
  ADR_CUDA(cudaStreamSynchronize(op.st));
  if (kernel_class != ADR_PROF_NONE && op.prof_pool.empty()) {
    op.prof_pool.resize(2 * kProfPairs, nullptr);
    for (auto& ev : op.prof_pool) ADR_CUDA(cudaEventCreate(&ev));
  }
  if (kernel_class != op.prof_class && op.cycle_exec) {  // the event nodes live in the captured cycle
    cudaGraphExecDestroy(op.cycle_exec);
    op.cycle_exec = nullptr;
    op.prof_graph_pairs = 0;
  }
  op.prof_class = kernel_class;
  op.prof_stream_pairs = 0;
  op.prof_graph_fresh = false;
  op.prof_count = 0;
  op.prof_ms = 0.0;
  return ADR_OK;
}

int adr_profile_read(adr_op_t h, long long* launches, double* total_ms) {
  if (!h || !launches || !total_ms) return fail(ADR_ERR_ARG, "null argument");
  Op& op = h->op;
  ADR_CUDA(cudaStreamSynchronize(op.st));
  prof_collect(op);
  *launches = op.prof_count;
  *total_ms = op.prof_ms;
  return ADR_OK;
}

int adr_operator_destroy(adr_op_t h) {
  if (!h) return ADR_OK;
  Op& op = h->op;
  cudaStreamSynchronize(op.st);
  if (op.cycle_exec) cudaGraphExecDestroy(op.cycle_exec);
  if (op.cycle_exec_adj) cudaGraphExecDestroy(op.cycle_exec_adj);
  if (op.cap) cudaStreamDestroy(op.cap);
  for (cudaEvent_t ev : op.prof_pool) cudaEventDestroy(ev);
  cudaError_t e1 = cudaFree(op.arena);
  cudaError_t e2 = cudaFreeHost(op.host_scal);
  delete h;
  if (e1 != cudaSuccess) return fail(ADR_ERR_CUDA, std::string("cudaFree: ") + cudaGetErrorString(e1));
  if (e2 != cudaSuccess) return fail(ADR_ERR_CUDA, std::string("cudaFreeHost: ") + cudaGetErrorString(e2));
  return ADR_OK;
}

int adr_operator_info(adr_op_t h, adr_op_info_t* info) {
  if (!h || !info) return fail(ADR_ERR_ARG, "null argument");
  Op& op = h->op;
  std::memset(info, 0, sizeof(*info));
  info->dim = op.dim;
  const int L = op.p.precond_precision == ADR_F64 ? op.h64.L : op.h32.L;
  info->levels = L;
  for (int l = 0; l < L; ++l) {
    const Dims& g = op.p.precond_precision == ADR_F64 ? op.h64.lv[l].g : op.h32.lv[l].g;
    for (int d = 0; d < 3; ++d) info->level[l].n[d] = g.n[d];
    info->level[l].nodes = g.N;
    info->level[l].stencil_points = l == 0 ? 0 : (op.dim == 2 ? kPattern2 : kPattern3);
  }
  info->arena_bytes = (int64_t)op.arena_bytes;
  info->problems = op.B;
  return ADR_OK;
}

int adr_coefficients(adr_op_t h, double* out) {
  if (!h || !out) return fail(ADR_ERR_ARG, "null argument");
  Op& op = h->op;
  launch_pack_coefficients(op.g0, op.gd, op.td, op.rho, op.tau, out, op.st);
  return check_launch("adr_coefficients");
}

int adr_apply(adr_op_t h, int scheme, int precision, const void* x, void* y) {
  if (!h || !x || !y) return fail(ADR_ERR_ARG, "null argument");
  if (scheme < ADR_SCHEME_2UP || scheme > ADR_SCHEME_PREC) return fail(ADR_ERR_ARG, "unknown scheme");
  Op& op = h->op;
  if (precision != ADR_F64 && precision != ADR_F32) return fail(ADR_ERR_ARG, "unknown precision");
  if (scheme == ADR_SCHEME_PREC && precision == op.p.precond_precision) {
    // the cycle's finest-grid operator exactly as the cycle applies it
    if (precision == ADR_F64) launch_fine_apply<double>(op.g0, op.h64.prec, (const double2*)x, (double2*)y, op.st);
    else launch_fine_apply<float>(op.g0, op.h32.prec, (const float2*)x, (float2*)y, op.st);
  } else if (scheme == ADR_SCHEME_PREC && op.p.rescale) {
    return fail(ADR_ERR_ARG, "with rescale the cycle's operator exists in the cycle's precision only");
  } else if (scheme == ADR_SCHEME_PREC) {
    if (precision == ADR_F64) {
      FineOp<double> f = make_fine<double>(op, op.p.prec_scheme, false, true);
      launch_fine_apply<double>(op.g0, f, (const double2*)x, (double2*)y, op.st);
    } else {
      FineOp<float> f = make_fine<float>(op, op.p.prec_scheme, true, true);
      launch_fine_apply<float>(op.g0, f, (const float2*)x, (float2*)y, op.st);
    }
  } else if (precision == ADR_F64 && scheme == op.p.scheme) {
    launch_packed_apply(op.g0, outer_op(op), (const double2*)x, (double2*)y, op.st);   // the outer iteration's operator
  } else if (precision == ADR_F64) {
    FineOp<double> f = make_fine<double>(op, scheme, false);
    launch_fine_apply<double>(op.g0, f, (const double2*)x, (double2*)y, op.st);
  } else if (precision == ADR_F32) {
    FineOp<float> f = make_fine<float>(op, scheme, true);
    launch_fine_apply<float>(op.g0, f, (const float2*)x, (float2*)y, op.st);
  }
  return check_launch("adr_apply");
}

int adr_level_stencil(adr_op_t h, int level, void* out) {
  if (!h || !out) return fail(ADR_ERR_ARG, "null argument");
  Op& op = h->op;
  const int L = op.p.precond_precision == ADR_F64 ? op.h64.L : op.h32.L;
  if (level < 1 || level >= L) return fail(ADR_ERR_ARG, "level must be in [1, levels)");
  const int S = op.dim == 2 ? kPattern2 : kPattern3;
  if (op.p.precond_precision == ADR_F64)
    launch_stencil_export<double>(op.h64.lv[level].g, op.h64.lv[level].A, (double2*)out, S, op.st);
  else
    launch_stencil_export<float>(op.h32.lv[level].g, op.h32.lv[level].A, (float2*)out, S, op.st);
  ADR_TRY(check_launch("adr_level_stencil"));
  return ADR_OK;
}

int adr_vcycle(adr_op_t h, const void* r, void* z) {
  if (!h || !r || !z) return fail(ADR_ERR_ARG, "null argument");
  if (r == z) return fail(ADR_ERR_ARG, "z may not alias r");
  Op& op = h->op;
  const int64_t N = op.g0.total;
  if (op.p.precond_precision == ADR_F64) {
    launch_copy<double>((const double2*)r, op.h64.lv[0].b, N, op.st);
    ADR_TRY(run_cycle(op, op.h64));
    launch_copy<double>(op.h64.lv[0].x, (double2*)z, N, op.st);
  } else {
    launch_copy<float>((const float2*)r, op.h32.lv[0].b, N, op.st);
    ADR_TRY(run_cycle(op, op.h32));
    launch_copy<float>(op.h32.lv[0].x, (float2*)z, N, op.st);
  }
  return check_launch("adr_vcycle");
}

int adr_point_source_rhs(adr_op_t h, void* q) {
  if (!h || !q) return fail(ADR_ERR_ARG, "null argument");
  Op& op = h->op;
  double vol = 1.0;
  for (int d = 0; d < op.dim; ++d) vol *= op.h[d];
  launch_rhs_point(op.g0, (double2*)q, op.dyn, 1.0 / vol, op.st);
  return check_launch("adr_point_source_rhs");
}

int adr_reconstruct(adr_op_t h, const void* a, void* u) {
  if (!h || !a || !u) return fail(ADR_ERR_ARG, "null argument");
  Op& op = h->op;
  launch_reconstruct(op.g0, (const double2*)a, op.tau, op.dyn, (double2*)u, op.st);
  return check_launch("adr_reconstruct");
}

// Flexible GMRES(m) on H_2up (adj: on H_2up^H with the cycle on A^H),
// right-preconditioned, float64 (Sec. 3.1; readings K1-K4).  The B problems of
// a batch iterate in lockstep, one launch per step for all of them; a problem
// whose estimate meets its tolerance is frozen on the device (its later
// columns are ignored by the back substitution), and a restart cycle ends
// when every problem is frozen, broken down or the budget is spent.  info
// receives B entries.
static int fgmres(Op& op, bool adj, const double2* b, double2* a, int use_x0, double tol, int maxit, adr_solve_info_t* info) {
  cudaStream_t st = op.st;
  const int B = op.B;
  const int64_t NB = op.g0.total;
  const int m = op.p.restart;
  // the outer operator: packed rows, or the stored conjugate-transposed rows;
  // A z_j with a float32 cycle reads z_j as the cycle left it (float32
  // values) and sums in double-float arithmetic
  const FineOp<double> fo = outer_op(op);
  auto outer_apply = [&](const double2* x, double2* y) {
    if (adj) launch_rows_apply(op.g0, op.rows_outT, x, y, st);
    else launch_packed_apply(op.g0, fo, x, y, st);
  };
  // The double-float outer iteration (params.outer_df with the float32
  // cycle): basis vector j as two float32 planes at Vf + 2 j NB (low parts NB
  // further), z_j as the cycle's float32 output at Zf + j NB, and the cycle's
  // input written by the kernel that normalises the basis vector.  The
  // solution and the restart residual stay float64.
  const bool dfk = op.packed_df != nullptr && !adj;
  float2* const Vf = (float2*)op.V;
  float2* const Zf = (float2*)op.Z;
  float2* const cyc = op.h32.lv[0].b;
  auto outer_residual = [&](const double2* bb, const double2* x, double2* r) {
    if (adj) launch_rows_residual(op.g0, op.rows_outT, bb, x, r, st);
    else launch_packed_residual(op.g0, fo, bb, x, r, st);
  };
  const double* hs = op.host_scal;

  launch_norm_start<double>(b, op.g0, op.ks, nullptr, st);
  launch_set_target(op.ost, op.ks.nrm2, tol, st, B);
  ADR_TRY(read_scalars(op, (const double*)op.ks.nrm2, 2 * B));
  std::vector<double> bnorm(B), beta(B), est(B);
  std::vector<int> its_p(B, 0), status(B, ADR_OK), done(B, 0);
  for (int pb = 0; pb < B; ++pb) bnorm[pb] = sqrt(hs[2 * pb]);
  if (use_x0) {
    outer_residual(b, a, op.r);
  } else {
    launch_zero<double>(a, NB, st);
    launch_copy<double>(b, op.r, NB, st);
  }
  launch_norm_start<double>(op.r, op.g0, op.ks, &op.ost, st);
  ADR_TRY(read_scalars(op, (const double*)op.ks.nrm2, 2 * B));
  int active = 0;
  for (int pb = 0; pb < B; ++pb) {
    beta[pb] = sqrt(hs[2 * pb]);
    est[pb] = bnorm[pb] > 0.0 ? beta[pb] / bnorm[pb] : 0.0;
    done[pb] = bnorm[pb] == 0.0 || beta[pb] <= tol * bnorm[pb];
    active += !done[pb];
  }
  int its = 0, cycles = 0;
  bool nan = false;
  std::vector<int> frozen(B), none(B, 0);
  // Batches: a frozen problem's blocks skip every launch of the iteration and
  // of the cycle (op.skip), until the restart's combination and explicit
  // residual, which run for every problem.
  while (active > 0 && its < maxit) {
    // op.ks.nrm2 holds |r|^2 and op.ost fresh cycles here
    for (int pb = 0; pb < B; ++pb) frozen[pb] = done[pb];
    ADR_TRY(upload_skip(op, frozen));
    if (dfk) launch_df_from_double(op.r, Vf, NB, op.ks.nrm2, cyc, op.g0, st);
    else launch_scale_inv_norm<double>(op.r, op.V, op.ks.nrm2, op.g0, st);
    int k = 0;
    for (int j = 0; j < m; ++j) {
      if (dfk) {
        float2* w = Vf + (int64_t)(j + 1) * 2 * NB;   // A z_j, orthogonalised and normalised in place
        ADR_TRY(run_cycle(op, op.h32));
        const int pk = prof_begin(op, ADR_PROF_OUTER_APPLY, st);
        launch_packed_apply_df(op.g0, fo, op.packed_df, op.h32.lv[0].x, w, NB, Zf + (int64_t)j * NB, st);
        prof_end(op, pk, st);
        launch_df_selective(Vf, 2 * NB, NB, j + 1, w, j + 1 < m ? cyc : nullptr, op.g0, op.ks, op.ost, j,
                            op.p.reorth_eta, st);
      } else {
        double2* vj = op.V + (int64_t)j * NB;
        double2* zj = op.Z + (int64_t)j * NB;
        double2* w = op.V + (int64_t)(j + 1) * NB;  // A z_j, orthogonalised and normalised in place
        ADR_TRY(precondition(op, vj, zj, adj));
        {
          const int pk = adj ? -1 : prof_begin(op, ADR_PROF_OUTER_APPLY, st);
          outer_apply(zj, w);
          prof_end(op, pk, st);
        }
        launch_cgs_selective<double>(op.V, NB, j + 1, w, op.g0, op.ks, op.ost, j, op.p.reorth_eta, st);
        launch_scale_inv_norm<double>(w, w, op.ks.nrm2, op.g0, st);
      }
      ADR_TRY(check_launch("adr_solve iteration"));
      ADR_TRY(read_scalars(op, op.ost.scal, kNumScal * B));
      ++its;
      k = j + 1;
      int open = 0, newly = 0;
      for (int pb = 0; pb < B; ++pb) {
        if (frozen[pb]) continue;
        const double* sc = hs + (size_t)pb * kNumScal;
        ++its_p[pb];
        est[pb] = sc[kScalEst] / bnorm[pb];
        if (!std::isfinite(est[pb]) || !std::isfinite(sc[kScalHn])) { nan = true; status[pb] = ADR_ERR_NAN; }
        if (sc[kScalHn] == 0.0 || sc[kScalEst] <= sc[kScalTarget]) { frozen[pb] = 1; ++newly; }
        else ++open;
      }
      if (nan || open == 0 || its >= maxit) break;
      if (newly) ADR_TRY(upload_skip(op, frozen));
    }
    if (nan) break;
    ADR_TRY(upload_skip(op, none));
    launch_backsolve(op.ost, k, st, B);
    if (dfk) launch_df_combine(a, Zf, NB, k, op.ost, op.g0, st);
    else launch_combine<double>(a, op.Z, NB, k, op.ost, false, op.g0, st);
    outer_residual(b, a, op.r);
    launch_norm_start<double>(op.r, op.g0, op.ks, &op.ost, st);
    ADR_TRY(read_scalars(op, (const double*)op.ks.nrm2, 2 * B));
    ++cycles;
    active = 0;
    for (int pb = 0; pb < B; ++pb) {
      if (done[pb]) continue;
      beta[pb] = sqrt(hs[2 * pb]);
      if (!std::isfinite(beta[pb])) { nan = true; status[pb] = ADR_ERR_NAN; continue; }
      done[pb] = beta[pb] <= tol * bnorm[pb];
      active += !done[pb];
    }
    if (nan) break;
  }
  ADR_TRY(upload_skip(op, none));
  for (int pb = 0; pb < B; ++pb) {   // zero right-hand side: a = 0
    if (bnorm[pb] != 0.0) continue;
    if (op.hetero) launch_zero<double>(a + op.tab[0][pb].off, op.tab[0][pb].N, st);
    else launch_zero<double>(a + (int64_t)pb * op.g0.N, op.g0.N, st);
  }
  ADR_TRY(check_launch("adr_solve"));
  bool all_ok = true;
  for (int pb = 0; pb < B; ++pb) {
    adr_solve_info_t res{};
    res.iterations = its_p[pb];
    res.restarts = cycles;
    res.rel_residual = bnorm[pb] > 0.0 ? beta[pb] / bnorm[pb] : 0.0;
    res.rel_estimate = est[pb];
    if (status[pb] == ADR_OK && !done[pb]) status[pb] = ADR_ERR_NOT_CONVERGED;
    res.status = status[pb];
    all_ok = all_ok && status[pb] == ADR_OK;
    if (info) info[pb] = res;
  }
  if (nan) return fail(ADR_ERR_NAN, "NaN or Inf in the Krylov iteration");
  if (!all_ok) return fail(ADR_ERR_NOT_CONVERGED, "iteration budget spent above the tolerance");
  return ADR_OK;
}

int adr_solve(adr_op_t h, const void* rhs_in, void* a_out, int use_x0, double tol, int maxit, adr_solve_info_t* info) {
  if (!h || !a_out) return fail(ADR_ERR_ARG, "null argument");
  if (!(tol >= 0.0) || maxit < 0) return fail(ADR_ERR_ARG, "tol must be >= 0 and maxit >= 0");
  Op& op = h->op;
  const double2* b = (const double2*)rhs_in;
  if (!b) {
    ADR_TRY(adr_point_source_rhs(h, op.b));
    b = op.b;
  }
  return fgmres(op, false, b, (double2*)a_out, use_x0, tol, maxit, info);
}

int adr_solve_two_stage(adr_op_t s1, adr_op_t s2, const void* rhs, void* a, double tol1, int maxit1, double tol,
                        int maxit, adr_solve_info_t* info) {
  if (!s1 || !s2 || !a) return fail(ADR_ERR_ARG, "null argument");
  if (s1 == s2) return fail(ADR_ERR_ARG, "the two stages need their own operators");
  if (!(tol1 >= 0.0) || maxit1 < 0 || !(tol >= 0.0) || maxit < 0)
    return fail(ADR_ERR_ARG, "tolerances must be >= 0 and iteration counts >= 0");
  const Op& o1 = s1->op;
  const Op& o2 = s2->op;
  bool same = o1.dim == o2.dim && o1.B == o2.B && o1.omegas == o2.omegas && o1.srcs == o2.srcs;
  for (int d = 0; d < 3; ++d) same = same && o1.g0.n[d] == o2.g0.n[d] && o1.h[d] == o2.h[d];
  if (!same) return fail(ADR_ERR_ARG, "the two stages must share grid, spacing, problems, sources and frequencies");
  const int rc1 = adr_solve(s1, rhs, a, 0, tol1, maxit1, info);
  if (rc1 != ADR_OK && rc1 != ADR_ERR_NOT_CONVERGED) return rc1;
  if (o1.st != o2.st) ADR_CUDA(cudaStreamSynchronize(o1.st));   // stage 2 reads stage 1's iterate
  return adr_solve(s2, rhs, a, 1, tol, maxit, info ? info + o1.B : nullptr);
}

int adr_adjoint_solve(adr_op_t h, const void* rhs, void* lambda, int use_x0, double tol, int maxit,
                      adr_solve_info_t* info) {
  if (!h || !rhs || !lambda) return fail(ADR_ERR_ARG, "null argument");
  if (!(tol >= 0.0) || maxit < 0) return fail(ADR_ERR_ARG, "tol must be >= 0 and maxit >= 0");
  if (rhs == lambda) return fail(ADR_ERR_ARG, "lambda may not alias rhs");
  Op& op = h->op;
  if (!op.p.adjoint) return fail(ADR_ERR_STATE, "operator created without params.adjoint");
  return fgmres(op, true, (const double2*)rhs, (double2*)lambda, use_x0, tol, maxit, info);
}

int adr_apply_adjoint(adr_op_t h, const void* x, void* y) {
  if (!h || !x || !y) return fail(ADR_ERR_ARG, "null argument");
  Op& op = h->op;
  if (!op.p.adjoint) return fail(ADR_ERR_STATE, "operator created without params.adjoint");
  launch_rows_apply(op.g0, op.rows_outT, (const double2*)x, (double2*)y, op.st);
  return check_launch("adr_apply_adjoint");
}

int adr_vcycle_adjoint(adr_op_t h, const void* r, void* z) {
  if (!h || !r || !z) return fail(ADR_ERR_ARG, "null argument");
  if (r == z) return fail(ADR_ERR_ARG, "z may not alias r");
  Op& op = h->op;
  if (!op.p.adjoint) return fail(ADR_ERR_STATE, "operator created without params.adjoint");
  const int64_t N = op.g0.N;
  if (op.p.precond_precision == ADR_F64) {
    launch_copy<double>((const double2*)r, op.a64.lv[0].b, N, op.st);
    ADR_TRY(run_cycle(op, op.a64, true));
    launch_copy<double>(op.a64.lv[0].x, (double2*)z, N, op.st);
  } else {
    launch_copy<float>((const float2*)r, op.a32.lv[0].b, N, op.st);
    ADR_TRY(run_cycle(op, op.a32, true));
    launch_copy<float>(op.a32.lv[0].x, (float2*)z, N, op.st);
  }
  return check_launch("adr_vcycle_adjoint");
}

int adr_receivers(adr_op_t h, int nrec, const int64_t* rec, const void* d, const void* u, void* res, void* rhs,
                  double* misfit) {
  if (!h || nrec < 0 || (nrec > 0 && (!rec || !d || !u))) return fail(ADR_ERR_ARG, "null argument");
  Op& op = h->op;
  if (op.B != 1) return fail(ADR_ERR_STATE, "receivers are sampled for one problem at a time");
  if (rhs) launch_zero<double>((double2*)rhs, op.g0.N, op.st);
  if (nrec == 0) {
    if (misfit) *misfit = 0.0;
    return check_launch("adr_receivers");
  }
  launch_receivers(op.g0.N, nrec, rec, (const double2*)d, (const double2*)u, op.tau, op.omega, (double2*)res,
                   (double2*)rhs, op.ks.nrm2, op.st);
  ADR_TRY(check_launch("adr_receivers"));
  if (misfit) {
    ADR_TRY(read_scalars(op, (const double*)op.ks.nrm2, 2));
    if (op.host_scal[1] != 0.0) return fail(ADR_ERR_ARG, "receiver index outside the grid");
    *misfit = 0.5 * op.host_scal[0];
  }
  return ADR_OK;
}

int adr_kappa_gradient(adr_op_t h, const double* kappa, const double* gamma, const void* a, const void* lambda,
                       double* grad) {
  if (!h || !kappa || !gamma || !a || !lambda || !grad) return fail(ADR_ERR_ARG, "null argument");
  Op& op = h->op;
  if (op.B != 1) return fail(ADR_ERR_STATE, "the gradient is accumulated for one problem at a time");
  launch_kappa_gradient(op.g0.N, op.omega, kappa, gamma, (const double2*)a, (const double2*)lambda, grad, op.st);
  return check_launch("adr_kappa_gradient");
}

int adr_solve_host(int dim, const int* n, const double* h, const int* src, double omega, const double* kappa,
                   const double* tau1, const double* gamma, const adr_params_t* params, double tol, int maxit,
                   void* stream, double* u_host, double* a_host, adr_solve_info_t* info) {
  if (!n || !kappa || !tau1 || !gamma || !u_host) return fail(ADR_ERR_ARG, "null argument");
  if (dim != 2 && dim != 3) return fail(ADR_ERR_ARG, "dim must be 2 or 3");
  int64_t N = 1;
  for (int d = 0; d < dim; ++d) {
    if (n[d] < 4) return fail(ADR_ERR_ARG, "every axis needs at least 4 nodes");
    N *= n[d];
  }
  cudaStream_t st = (cudaStream_t)stream;
  // one allocation, each piece on a 256-byte boundary (complex pieces are read as double2)
  const size_t real_bytes = sizeof(double) * (size_t)N;
  const size_t real_slot = (real_bytes + 255) & ~size_t(255);
  const size_t cplx_slot = (2 * real_bytes + 255) & ~size_t(255);
  char* dev = nullptr;
  ADR_CUDA(cudaMalloc(&dev, 3 * real_slot + 2 * cplx_slot));
  double* dk = (double*)(dev);
  double* dt = (double*)(dev + real_slot);
  double* dg = (double*)(dev + 2 * real_slot);
  double* da = (double*)(dev + 3 * real_slot);
  double* du = (double*)(dev + 3 * real_slot + cplx_slot);
  int rc = ADR_OK;
  cudaError_t e = cudaMemcpyAsync(dk, kappa, real_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dt, tau1, real_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dg, gamma, real_bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) rc = fail(ADR_ERR_CUDA, std::string("host to device copy: ") + cudaGetErrorString(e));
  adr_op_t op = nullptr;
  if (rc == ADR_OK) rc = adr_operator_create(dim, n, h, src, omega, dk, dt, dg, params, stream, &op);
  adr_solve_info_t res{};
  int solve_rc = ADR_OK;
  if (rc == ADR_OK) {
    solve_rc = adr_solve(op, nullptr, da, 0, tol, maxit, &res);
    if (solve_rc == ADR_OK || solve_rc == ADR_ERR_NOT_CONVERGED) {
      rc = adr_reconstruct(op, da, du);
      if (rc == ADR_OK) {
        e = cudaMemcpyAsync(u_host, du, 2 * real_bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && a_host) e = cudaMemcpyAsync(a_host, da, 2 * real_bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(ADR_ERR_CUDA, std::string("device to host copy: ") + cudaGetErrorString(e));
      }
    } else {
      rc = solve_rc;
    }
  }
  if (op) adr_operator_destroy(op);
  cudaStreamSynchronize(st);
  cudaFree(dev);
  if (info) *info = res;
  if (rc != ADR_OK) return rc;
  return solve_rc;
}

}  // extern "C"
