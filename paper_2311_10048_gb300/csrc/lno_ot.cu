// Host driver of the C ABI declared in include/lno_ot.h.
//
// One domain (eq cim_pt_energy, spin cases aaa, aab, abb, bbb):
//  1. stage: validate, lay the DF factors out as K-contiguous blocks
//     (occ-occ, occ-vir, vir-vir rows, Q fastest), assemble (ia|jb);
//  2. per spin s: assemble the DF integrals and build the K-concatenated
//     contraction operands AT, BT (same spin) and A1, BG, BF, AT2 (mixed,
//     spin s twice and the other spin once), see pack.cu;
//  3. per group of triplets: one grouped contraction launch writes X (same
//     spin) or Y and Z' (mixed) per triplet, one energy launch assembles W,
//     V and sums W (W + V) / D per triplet (energy.cu);
//  4. per-triplet sums -> per-case compensated sums -> host.
// Precision FP64 runs every contraction on the CUDA cores in float64; the
// BF16X3 / BF16X6 precisions run them on the tensor cores on exact BF16
// slices (tc_gemm.cu), with float64 kept for orbital energies and sums.
#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"

namespace lno {
// gemm_f64.cu
cudaError_t launch_gemm_f64(const ProbF64* probs_dev, int nprob, int M, int N, int ldo,
                            cudaStream_t st);
// energy.cu
cudaError_t launch_energy(const EnergyArgs& a, const void* X, const void* Z, bool f64, int ntrip,
                          int nchunks, cudaStream_t st);
cudaError_t launch_energy_f32(const EnergyArgs& a, const float* X, const float* Z, float* vtab,
                              int64_t vt_stride, int pv, int pvt, int ntrip, int nchunks,
                              cudaStream_t st);
cudaError_t launch_energy_f32_fused(const EnergyArgs& a, const float* X, const float* Z,
                                   float* vtab, int64_t vt_half, int pv, int pvt, int ntrip,
                                   int nchunks, cudaStream_t st);
cudaError_t launch_reduce_partials(const double* partial, int np, const double* partial2,
                                   int ntrip, double* e_trip, cudaStream_t st);
cudaError_t launch_orbital_partition(const OrbPartArgs& A, cudaStream_t st);
cudaError_t launch_neumaier_sum(const double* e, int64_t n, double* out, cudaStream_t st);
cudaError_t energy_timeout_selftest(long long wait_cycles, int nsm, int* code, cudaStream_t st);
// pack.cu
template <class St>
cudaError_t launch_transpose_block(const double*, int, int, int, int, int, int, int, St,
                                   cudaStream_t);
template <class St>
cudaError_t launch_pack_at_same(const int2*, int, int, int, int, int, const double*, const double*,
                                St, cudaStream_t);
template <class St>
cudaError_t launch_pack_bt_same(int, int, int, int, int, int, const double*, const double*, St,
                                cudaStream_t);
template <class St>
cudaError_t launch_pack_a1(const int2*, int, int, int, int, int, int, int, const double*,
                           const double*, St, cudaStream_t);
template <class St>
cudaError_t launch_pack_bg(int, int, int, int, int, int, int, int, const double*, const double*,
                           St, cudaStream_t);
template <class St>
cudaError_t launch_pack_bf(int, int, int, int, int, int, int, int, const double*, const double*,
                           St, cudaStream_t);
template <class St>
cudaError_t launch_pack_at2(const int2*, int, int, int, int, int, int, int, const double*,
                            const double*, St, cudaStream_t);
cudaError_t launch_transpose_t2ab(const double*, int, int, int, int, double*, cudaStream_t);
cudaError_t launch_absmax(const double*, int64_t, unsigned long long*, cudaStream_t);
cudaError_t launch_view_absmax(const double* in, int64_t rs, int64_t ks, int rows, int K,
                               unsigned long long* out, cudaStream_t s);
cudaError_t launch_sum_partials(const double* part, int nsp, int M, int N, double* C,
                                int64_t ldc, bool accum, cudaStream_t s);
template <int S>
cudaError_t launch_view_slices(const double* in, int64_t rs, int64_t ks, int rows, int K,
                               int Kp, __nv_bfloat16* out, int64_t slice_stride, double inv,
                               cudaStream_t s);
cudaError_t launch_t2ab_flip_mismatch(const double* t2ab, int n, int v, double tol,
                                     unsigned int* count, cudaStream_t s);
cudaError_t launch_gather_rows(const void* src, void* dst, const int* list, int nlist,
                               int64_t row_bytes, int nslice, int64_t src_slice_bytes,
                               int64_t dst_slice_bytes, cudaStream_t s);
cudaError_t launch_scatter_add_rows(const double* src, double* dst, const int* list, int nlist,
                                    int64_t row, cudaStream_t s);
// naf.cu
int jacobi_eigh(double* A, double* V, int n, double2* cs, double* norms, cudaStream_t st,
                int max_sweeps);
cudaError_t launch_pack_pairs(const double* B, int naux, int n, double* J, cudaStream_t st);
cudaError_t launch_transpose_x(const double* B, int naux, int64_t n2, double* Bt,
                               cudaStream_t st);
cudaError_t launch_get_diag(const double* A, int n, double* d, cudaStream_t st);
cudaError_t launch_gather_cols(const double* V, int n, const int* cols, int nk, double* Vt,
                               cudaStream_t st);
// backward.cu
struct GemmS {
  const double* A;
  const double* B;
  double* C;
  int M, N, K;
  int atomic;
  int64_t sam, sak, sbk, sbn, scm, scn;
  double alpha;
};
cudaError_t launch_gemm_strided(const GemmS* probs_dev, int nprob, int maxM, int maxN,
                                cudaStream_t st);
cudaError_t launch_energy_backward(const EnergyArgs& a, const double* X, const double* Z,
                                   double* dX, double* dZ, double* dt1s, double* dt1t,
                                   double* dov_ss, double* dov_ts, double* deps_s,
                                   double* deps_t, double gscale, int ntrip, int nchunks,
                                   cudaStream_t st);
cudaError_t launch_adj_at_same(const int2*, int, int, int, int, const double*, double*, double*,
                               cudaStream_t);
cudaError_t launch_adj_bt_same(int, int, int, int, int, const double*, double*, double*,
                               cudaStream_t);
cudaError_t launch_adj_a1(const int2*, int, int, int, int, int, int, const double*, double*,
                          double*, cudaStream_t);
cudaError_t launch_adj_bg(int, int, int, int, int, int, int, const double*, double*, double*,
                          cudaStream_t);
cudaError_t launch_adj_bf(int, int, int, int, int, int, int, const double*, double*, double*,
                          cudaStream_t);
cudaError_t launch_adj_at2(const int2*, int, int, int, int, int, int, const double*, double*,
                           double*, cudaStream_t);
cudaError_t launch_adj_transpose_block(const double*, int, int, int, int, int, int, int, double*,
                                       cudaStream_t);
cudaError_t launch_sym_project(const double*, int, int, double, double*, cudaStream_t);
cudaError_t launch_antisym_project(const double*, int, int, double, double*, cudaStream_t);
cudaError_t launch_adj_transpose_t2ab(const double*, int, int, int, int, double*, cudaStream_t);
cudaError_t launch_scale_copy(const double*, int64_t, double, double*, cudaStream_t);
cudaError_t launch_sym_inplace(double*, int, int, cudaStream_t);
cudaError_t launch_antisym_inplace(double*, int, int, cudaStream_t);
}  // namespace lno

using namespace lno;

// ----------------------------------------------------------------------------
static thread_local std::string g_last_error;

void lno_set_last_error(const char* what, cudaError_t e, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_last_error = buf;
}

struct lno_ot_ctx {
  int device = 0;
  int prec = LNO_OT_FP64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t ws_limit = 0;
  int nsm = 152;
  // tuning table: per virtual-space size bucket (rows of the contraction,
  // ascending vmax) the contraction tile width (0 = the precision's default)
  // and the triplet-group cap
  struct TuneRow {
    int vmax, bn, group_cap;
  };
  std::vector<TuneRow> tune;
  const TuneRow* tune_for(int v) const {
    for (const TuneRow& r : tune)
      if (v <= r.vmax) return &r;
    return tune.empty() ? nullptr : &tune.back();
  }
  int* d_flag = nullptr;               // device error flag (bounded waits)
  unsigned long long* d_amax = nullptr;
  double* d_sums = nullptr;            // [8]
  lno_ot_stats stats{};
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  // prepared operands of the last domain (options.keep_operands)
  bool keep = false;
  struct DomainCache* cache = nullptr;
};

void destroy_cache(DomainCache* c);

namespace {

#define TRY(expr)                       \
  do {                                  \
    int rc__ = (expr);                  \
    if (rc__ != LNO_OT_OK) return rc__; \
  } while (0)

// Stream-ordered device allocations released at scope exit.
struct Arena {
  cudaStream_t st;
  size_t limit, used = 0;
  std::vector<void*> ptrs;
  Arena(cudaStream_t s, size_t lim) : st(s), limit(lim) {}
  ~Arena() { release(); }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    ptrs.clear();
    used = 0;
  }
  template <typename T>
  int get(T** out, size_t n) {
    size_t bytes = std::max<size_t>(n * sizeof(T), 256);
    bytes = (bytes + 255) / 256 * 256;
    if (limit && used + bytes > limit) return LNO_OT_ENOMEM;
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return LNO_OT_ENOMEM;
    }
    ptrs.push_back(p);
    used += bytes;
    *out = static_cast<T*>(p);
    return LNO_OT_OK;
  }
  void drop(void* p) {
    for (auto& q : ptrs)
      if (q == p) {
        cudaFreeAsync(q, st);
        q = ptrs.back();
        ptrs.pop_back();
        return;
      }
  }
};

int cuda_rc(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LNO_OT_OK;
  lno_set_last_error(what, e, __FILE__, __LINE__);
  cudaGetLastError();
  return LNO_OT_ECUDA;
}
#define CU(...) TRY(cuda_rc((__VA_ARGS__), #__VA_ARGS__))

int64_t pow2ceil_exp(double x) {  // smallest e with 2^e >= x (x > 0)
  int e;
  double m = std::frexp(x, &e);    // x = m 2^e, m in [0.5, 1)
  return (m == 0.5) ? e - 1 : e;
}

double pow2_scale(double amax) {
  if (!(amax > 0.0) || !std::isfinite(amax)) return 1.0;
  return std::ldexp(1.0, (int)pow2ceil_exp(amax));
}

// K-concatenated operand tensor: nslot slots of `rows` rows, pitch Kp.
struct Operand {
  int nslot = 0;
  int64_t rows = 0;  // rows per slot
  int K = 0, Kp = 0;
  double* f64 = nullptr;
  __nv_bfloat16* bf = nullptr;   // BF16 slices
  float* f32 = nullptr;          // TF32 slices (stored as float)
  int esz = 2;                   // bytes per slice element
  int S = 0;
  int64_t slice_stride = 0;
  CUtensorMap map128, map256, map96, map64;  // TMA maps with boxes of 128 (A role, B of BN 128), 256, 96, 64 rows
  int64_t total_rows() const { return (int64_t)nslot * rows; }
};

// Tile width of the W contraction for S slices: the tuned value when it is
// one the build has (S * BN <= 512 TMEM columns), else the default.
int contract_bn(int S, int bn) {
  switch (S) {
    case 2: return bn == 128 ? 128 : 256;
    case 3: return bn == 64 ? 64 : 128;
    case 4: return bn == 64 ? 64 : bn == 96 ? 96 : 128;
    default: return 64;
  }
}

const CUtensorMap& map_for(const Operand& op, int box) {
  return box == 256 ? op.map256 : box == 96 ? op.map96 : box == 64 ? op.map64 : op.map128;
}

// One grouped W-contraction launch with float32 output XT[n][m] (pitch ldo)
// = sum_seg A_seg[m] . B_seg[n], m < M the virtual index of the A operands, n
// < N the (pair) rows of the B operands.  The kernel runs it row-major with
// the roles exchanged: its 128-row tiles run over the N rows (a long
// dimension, so they are full) and its n-tiles over the M rows, the last one
// only as wide as needed (M rounded up to 16).  seg_tc stores the segments
// with the roles already exchanged.
cudaError_t launch_contract(int S, bool tf, int bn_req, const Operand& A0, const Operand& A1,
                            const Operand& B0, const Operand& B1, const TcProb* dpt, int nprob,
                            int M, int N, int ldo, double scale, int* flag, int nsm,
                            cudaStream_t st, TcOut lay) {
  const int bn = contract_bn(S, bn_req);
  CUtensorMap mA[2] = {B0.map128, B1.map128};
  CUtensorMap mB[2] = {map_for(A0, bn), map_for(A1, bn)};
  const TcDiag dg = tc_normal();
  std::swap(M, N);
#define LNO_CALL(SS, BB)                                                                      \
  launch_tc_gemm<SS, BB, float, false, true>(mA, mB, dpt, nprob, M, N, ldo, scale, flag, nullptr, \
                                             nsm, st, dg, lay)
  if (tf)
    return bn == 128
               ? launch_tc_gemm<2, 128, float, true, true>(mA, mB, dpt, nprob, M, N, ldo, scale,
                                                           flag, nullptr, nsm, st, dg, lay)
               : launch_tc_gemm<2, 256, float, true, true>(mA, mB, dpt, nprob, M, N, ldo, scale,
                                                           flag, nullptr, nsm, st, dg, lay);
  if (S == 2) return bn == 128 ? LNO_CALL(2, 128) : LNO_CALL(2, 256);
  if (S == 3) return bn == 64 ? LNO_CALL(3, 64) : LNO_CALL(3, 128);
  if (S == 4) return bn == 64 ? LNO_CALL(4, 64) : bn == 96 ? LNO_CALL(4, 96) : LNO_CALL(4, 128);
  return LNO_CALL(5, 64);
#undef LNO_CALL
}

// Strided float64 view: element (r, k) at p[r rs + k ks].
struct View {
  const double* p;
  int64_t rs, ks;
};
constexpr int64_t kMaxSplit = 64;   // K chunks of one tc_matmul
struct Run;
int tc_matmul(Run& R, Arena& A, int M, int N, int K, View a, View b, double* C, int64_t ldc,
              double alpha, bool accum, bool b_const = false);

// Slices of a read-only view kept by tc_matmul for the rest of a Run (the DF
// factor blocks that every slot's DF adjoint multiplies).
struct SliceCacheEntry {
  const double* p;
  int64_t rs, ks;
  int rows, K, Kc, nsp;
  __nv_bfloat16* q;
  double sigma;
};

struct Run {
  lno_ot_ctx* ctx;
  const lno_ot_domain* dom;
  cudaStream_t st;
  Arena arena;
  bool f64;
  bool tf32 = false;  // W contraction operands as TF32 slices (precision TF32)
  bool tc_adjoint = false;  // adjoint: its contractions on the tensor cores (tc_matmul)
  int S = 0;          // slices of the W contraction operands
  int Sdf = 4;        // slices of the DF factors
  double sigT = 1, sigI = 1, sigB = 1;
  bool amax_pass = false;  // true while measuring integral magnitudes
  double amax_int = 0.0;
  int nbas, naux, no[2], nv[2];
  // orbitals per spin: nbas, or nbas + P for a spin that carries P central
  // pseudo-orbitals (set before stage(); 0 = nbas)
  int nbs[2] = {0, 0};
  // occupied orbitals the internal (summed) indices run over: no[s] unless
  // pseudo-orbitals (central LMOs, Sec. 3.7) follow the real ones
  int noi[2] = {-1, -1};
  // Laplace quadrature point of the central-LMO pass (lap_w = 0: 1/D)
  double lap_s = 0.0, lap_w = 0.0;
  // DF factor blocks per spin (rows, K = naux); Boo rows are [internal][external]
  Operand Boo[2], Bov[2], Bvv[2];
  const double* fov[2] = {nullptr, nullptr};  // f_ov blocks (both or none)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> contract_ev, energy_ev;
  std::vector<SliceCacheEntry> slice_cache;   // tc_matmul, read-only B views
  lno_ot_stats* stats;

  Run(lno_ot_ctx* c, const lno_ot_domain* d)
      : ctx(c), dom(d), st(c->stream), arena(c->stream, c->ws_limit), stats(&c->stats) {}

  cudaEvent_t event() {
    if (ctx->ev_used == ctx->ev_pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      ctx->ev_pool.push_back(e);
    }
    return ctx->ev_pool[ctx->ev_used++];
  }

  // ---- operand allocation -------------------------------------------------
  int alloc_operand(Operand& op, int nslot, int64_t rows, int K, int S_) {
    return alloc_operand(arena, op, nslot, rows, K, S_);
  }
  // tf: TF32 slices (the W operands of precision TF32); DF blocks are BF16
  int alloc_operand(Arena& ar, Operand& op, int nslot, int64_t rows, int K, int S_,
                    bool tf = false) {
    op.nslot = nslot;
    op.rows = rows;
    op.K = K;
    op.Kp = (int)round_up(std::max(K, 1), 8);
    op.S = f64 ? 0 : S_;
    const int64_t n = std::max<int64_t>((int64_t)nslot * rows * op.Kp, 8);
    if (f64) {
      TRY(ar.get(&op.f64, (size_t)n));
    } else {
      op.slice_stride = round_up(n, 8);
      void* base;
      if (tf) {
        op.esz = 4;
        TRY(ar.get(&op.f32, (size_t)(op.slice_stride * op.S)));
        base = op.f32;
      } else {
        op.esz = 2;
        TRY(ar.get(&op.bf, (size_t)(op.slice_stride * op.S)));
        base = op.bf;
      }
      const int64_t rows_ = std::max<int64_t>(op.total_rows(), 1);
      TRY(make_operand_map(&op.map128, base, op.Kp, rows_, op.S, op.slice_stride, 128, op.esz));
      TRY(make_operand_map(&op.map256, base, op.Kp, rows_, op.S, op.slice_stride, 256, op.esz));
      TRY(make_operand_map(&op.map64, base, op.Kp, rows_, op.S, op.slice_stride, 64, op.esz));
      TRY(make_operand_map(&op.map96, base, op.Kp, rows_, op.S, op.slice_stride, 96, op.esz));
    }
    return LNO_OT_OK;
  }

  // Store functor for an operand (amplitude scale sigT, integral scale sigI).
  template <int SS>
  StoreSlices<SS> slices(const Operand& op) const {
    return StoreSlices<SS>{op.bf, op.slice_stride, 128.0 / sigT, 128.0 / sigI};
  }
  StoreTF32<2> tf32_slices(const Operand& op) const {
    return StoreTF32<2>{op.f32, op.slice_stride, 1024.0 / sigT, 1024.0 / sigI};
  }

  // ---- DF integrals: out[n][m] = sum_Q L[m][Q] R[n][Q] (float64) ------------
  // L rows [l0, l0+M) of operand Lo, R rows [r0, r0+N) of Ro.
  int df(const Operand& Lo, int64_t l0, int M, const Operand& Ro, int64_t r0, int N, double* out,
         int ldo) {
    if (M <= 0 || N <= 0) return LNO_OT_OK;
    stats->other_launches++;
    if (f64 && tc_adjoint)   // adjoint of a tensor-core precision: float64 blocks, TC product
      return tc_matmul(*this, arena, N, M, naux, View{Ro.f64 + r0 * Ro.Kp, Ro.Kp, 1},
                       View{Lo.f64 + l0 * Lo.Kp, Lo.Kp, 1}, out, ldo, 1.0, false);
    if (f64) {
      ProbF64 p{};
      p.nseg = 1;
      p.seg[0] = SegF64{Lo.f64 + l0 * Lo.Kp, Ro.f64 + r0 * Ro.Kp, naux, Lo.Kp, Ro.Kp, 1.0};
      p.XT = out;
      ProbF64* dp;
      TRY(arena.get(&dp, 1));
      CU(cudaMemcpyAsync(dp, &p, sizeof p, cudaMemcpyHostToDevice, st));
      CU(launch_gemm_f64(dp, 1, M, N, ldo, st));
      return LNO_OT_OK;
    }
    TcProb p{};
    p.nseg = 1;
    p.seg[0] = TcSeg{0, 0, (int)l0, (int)r0, naux, 0};
    p.out = amax_pass ? nullptr : out;
    TcProb* dp;
    TRY(arena.get(&dp, 1));
    CU(cudaMemcpyAsync(dp, &p, sizeof p, cudaMemcpyHostToDevice, st));
    const double scale = sigB * sigB * std::ldexp(1.0, -14);
    unsigned long long* am = amax_pass ? ctx->d_amax : nullptr;
    if (Sdf == 5) {
      CUtensorMap mA[2] = {Lo.map128, Lo.map128}, mB[2] = {Ro.map64, Ro.map64};
      CU(launch_tc_gemm<5, 64, double>(mA, mB, dp, 1, M, N, ldo, scale, ctx->d_flag, am,
                                       ctx->nsm, st, tc_normal()));
    } else {
      CUtensorMap mA[2] = {Lo.map128, Lo.map128}, mB[2] = {Ro.map128, Ro.map128};
      CU(launch_tc_gemm<4, 128, double>(mA, mB, dp, 1, M, N, ldo, scale, ctx->d_flag, am,
                                        ctx->nsm, st, tc_normal()));
    }
    return LNO_OT_OK;
  }

  // ---- stage ----------------------------------------------------------------
  int stage() {
    nbas = dom->nbas;
    naux = dom->naux;
    for (int s = 0; s < 2; ++s) {
      if (nbs[s] <= 0) nbs[s] = nbas;
      no[s] = dom->nocc[s];
      nv[s] = nbs[s] - no[s];
      if (noi[s] < 0 || noi[s] > no[s]) noi[s] = no[s];
    }
    if (!f64) {  // global scales of B and T2
      CU(cudaMemsetAsync(ctx->d_amax, 0, sizeof(unsigned long long), st));
      for (int s = 0; s < 2; ++s)
        CU(launch_absmax(dom->B[s], (int64_t)naux * nbs[s] * nbs[s], ctx->d_amax, st));
      unsigned long long h;
      CU(cudaMemcpyAsync(&h, ctx->d_amax, sizeof h, cudaMemcpyDeviceToHost, st));
      CU(cudaMemsetAsync(ctx->d_amax, 0, sizeof(unsigned long long), st));
      CU(launch_absmax(dom->t2aa, (int64_t)no[0] * no[0] * nv[0] * nv[0], ctx->d_amax, st));
      CU(launch_absmax(dom->t2bb, (int64_t)no[1] * no[1] * nv[1] * nv[1], ctx->d_amax, st));
      CU(launch_absmax(dom->t2ab, (int64_t)no[0] * no[1] * nv[0] * nv[1], ctx->d_amax, st));
      unsigned long long ht;
      CU(cudaMemcpyAsync(&ht, ctx->d_amax, sizeof ht, cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      double mb, mt;
      std::memcpy(&mb, &h, 8);
      std::memcpy(&mt, &ht, 8);
      sigB = pow2_scale(mb);
      sigT = pow2_scale(mt);
      stats->other_launches += 5;
    }
    if (dom->fov[0] || dom->fov[1]) {  // a missing spin block is zero
      for (int s = 0; s < 2; ++s) {
        if (dom->fov[s]) {
          fov[s] = dom->fov[s];
        } else {
          double* z;
          const size_t n = std::max<size_t>((size_t)no[s] * nv[s], 1);
          TRY(arena.get(&z, n));
          CU(cudaMemsetAsync(z, 0, n * sizeof(double), st));
          fov[s] = z;
        }
      }
    }
    for (int s = 0; s < 2; ++s) {
      const int o = no[s], oi = noi[s], v = nv[s];
      TRY(alloc_operand(Boo[s], 1, (int64_t)oi * o, naux, Sdf));
      TRY(alloc_operand(Bov[s], 1, (int64_t)o * v, naux, Sdf));
      TRY(alloc_operand(Bvv[s], 1, (int64_t)v * v, naux, Sdf));
      struct Blk {
        Operand* op;
        int p0, np, q0, nq;
      } blks[3] = {{&Boo[s], 0, oi, 0, o}, {&Bov[s], 0, o, o, v}, {&Bvv[s], o, v, o, v}};
      for (auto& b : blks) {
        stats->other_launches++;
        if (f64)
          CU(launch_transpose_block(dom->B[s], naux, nbs[s], b.p0, b.np, b.q0, b.nq, b.op->Kp,
                                    StoreF64{b.op->f64}, st));
        else if (Sdf == 5)
          CU(launch_transpose_block(
              dom->B[s], naux, nbs[s], b.p0, b.np, b.q0, b.nq, b.op->Kp,
              StoreSlices<5>{b.op->bf, b.op->slice_stride, 128.0 / sigB, 128.0 / sigB}, st));
        else
          CU(launch_transpose_block(
              dom->B[s], naux, nbs[s], b.p0, b.np, b.q0, b.nq, b.op->Kp,
              StoreSlices<4>{b.op->bf, b.op->slice_stride, 128.0 / sigB, 128.0 / sigB}, st));
      }
    }
    return LNO_OT_OK;
  }

  // dst slot q = src rows [dlist[q] * rows, (dlist[q] + 1) * rows): a DF block
  // restricted to some occupied orbitals (same slicing and scales as src)
  int gather_operand(Arena& ar, const Operand& src, const int* dlist, int nlist, int64_t rows,
                     Operand& dst) {
    TRY(alloc_operand(ar, dst, nlist, rows, src.K, Sdf));
    if (nlist == 0 || rows == 0) return LNO_OT_OK;
    stats->other_launches++;
    if (f64)
      CU(launch_gather_rows(src.f64, dst.f64, dlist, nlist, rows * src.Kp * 8, 1, 0, 0, st));
    else
      CU(launch_gather_rows(src.bf, dst.bf, dlist, nlist, rows * src.Kp * 2, src.S,
                            src.slice_stride * 2, dst.slice_stride * 2, st));
    return LNO_OT_OK;
  }
};

// Spin-case triplet selection.
struct CaseSel {
  std::vector<Trip> trips;   // triplets to compute, in output order
  int64_t ntot = 0;          // all restricted triplets of the case
};

int64_t c2(int64_t n) { return n * (n - 1) / 2; }
int64_t c3(int64_t n) { return n * (n - 1) * (n - 2) / 6; }

Trip decode_triplet(int c, int64_t q, int na, int nb) {
  // lexicographic enumeration as in the header
  auto same = [](int64_t q, int n) {
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) {
        int64_t cnt = n - j - 1;
        if (q < cnt) return Trip{i, j, (int)(j + 1 + q)};
        q -= cnt;
      }
    return Trip{-1, -1, -1};
  };
  auto mixed = [](int64_t q, int n2, int n1) {
    int64_t pairi = q / n1;
    int k = (int)(q % n1);
    for (int i = 0; i < n2; ++i) {
      int64_t cnt = n2 - i - 1;
      if (pairi < cnt) return Trip{i, (int)(i + 1 + pairi), k};
      pairi -= cnt;
    }
    return Trip{-1, -1, -1};
  };
  switch (c) {
    case 0: return same(q, na);
    case 3: return same(q, nb);
    case 1: return mixed(q, na, nb);
    default: return mixed(q, nb, na);
  }
}

int select_case(const lno_ot_domain* d, int c, CaseSel& cs) {
  const int na = d->nocc[0], nb = d->nocc[1];
  cs.ntot = c == 0 ? c3(na) : c == 3 ? c3(nb) : c == 1 ? c2(na) * nb : c2(nb) * na;
  cs.trips.clear();
  if (d->trip_sel[c]) {
    if (d->n_sel[c] < 0) return LNO_OT_EINVAL;
    cs.trips.reserve((size_t)d->n_sel[c]);
    for (int64_t q = 0; q < d->n_sel[c]; ++q) {
      int64_t id = d->trip_sel[c][q];
      if (id < 0 || id >= cs.ntot) return LNO_OT_EINVAL;
      cs.trips.push_back(decode_triplet(c, id, na, nb));
    }
  } else {
    // enumerate directly (fast path)
    if (c == 0 || c == 3) {
      const int n = c == 0 ? na : nb;
      for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
          for (int k = j + 1; k < n; ++k) cs.trips.push_back(Trip{i, j, k});
    } else {
      const int n2 = c == 1 ? na : nb, n1 = c == 1 ? nb : na;
      for (int i = 0; i < n2; ++i)
        for (int j = i + 1; j < n2; ++j)
          for (int k = 0; k < n1; ++k) cs.trips.push_back(Trip{i, j, k});
    }
  }
  return LNO_OT_OK;
}

double flops_alg_same(double v, double o) { return 3.0 * (2 * v * v * v * v + 2 * v * v * v * o); }
double flops_alg_mixed(double vs, double vt, double os, double ot) {
  return 4 * vs * vs * vt * vt + 6 * vs * vs * vs * vt + 4 * vs * vs * vt * ot + 6 * os * vs * vs * vt;
}
double kpad16(double k) { return std::ceil(k / 16.0) * 16.0; }

// ----------------------------------------------------------------------------
// Per spin s: same-spin case (sss) and the mixed case with two s orbitals.
struct SpinPass {
  Run& R;
  int s, t;
  int o, v, ot, vt;
  int oi, oti;  // internal occupied ranges (== o, ot without pseudo-orbitals)
  CaseSel& same;   // case s==0 ? aaa : bbb
  CaseSel& mixed;  // case s==0 ? aab : abb
  double* e_same;  // per-triplet outputs (device)
  double* e_mixed;

  Operand AT, BT, A1, BG, BF, AT2;
  std::vector<int> slotAT, slotBT, slotA1, slotBG, slotBF, slotAT2;  // -1 = unused
  std::vector<int2> listAT, listA1, listAT2;
  std::vector<int> listBT, listBG, listBF;
  int bn = 0;                // contraction tile width of the current case (0 = default)
  int group_cap = 64;        // triplets per group (upper bound)
  double* t2st = nullptr;    // [os][ot][vs][vt]
  const double* t2ss = nullptr;
  // V-term integrals over the occupied orbitals in use: spin-s slots are those
  // of listBT (every i, j, k of a computed triplet), spin-t slots those of
  // listBF (every K of a mixed triplet)
  Operand BsS, BsT;          // Bov rows of the slots, [slot][vir] x naux
  double* ovss = nullptr;    // (ia|jb) as [nS][vs][nS][vs]
  double* ovts = nullptr;    // (jb|KC) as [nT][vt][nS][vs]
  int* d_slot_s = nullptr;   // occupied index -> slot (-1 absent), spin s [os]
  int* d_slot_t = nullptr;   // spin t [ot]
  int* d_list_s = nullptr;   // slot -> occupied index
  int* d_list_t = nullptr;

  Arena own;  // operands and temporaries of this spin pass

  SpinPass(Run& r, int s_, CaseSel& sm, CaseSel& mx, double* es, double* em)
      : R(r), s(s_), t(1 - s_), same(sm), mixed(mx), e_same(es), e_mixed(em),
        own(r.st, 0) {
    o = R.no[s];
    v = R.nv[s];
    ot = R.no[t];
    vt = R.nv[t];
    oi = R.noi[s];
    oti = R.noi[t];
  }

  void plan() {
    listAT.clear();
    listA1.clear();
    listAT2.clear();
    listBT.clear();
    listBG.clear();
    listBF.clear();
    slotAT.assign((size_t)o * o, -1);
    slotBT.assign(o, -1);
    slotA1.assign((size_t)o * ot, -1);
    slotBG.assign(o, -1);
    slotBF.assign(ot, -1);
    slotAT2.assign((size_t)o * ot, -1);
    auto need_pair = [&](std::vector<int>& slot, std::vector<int2>& list, int p, int q, int w) {
      int& sl = slot[(size_t)p * w + q];
      if (sl < 0) {
        sl = (int)list.size();
        list.push_back(make_int2(p, q));
      }
    };
    auto need_one = [&](std::vector<int>& slot, std::vector<int>& list, int x) {
      if (slot[x] < 0) {
        slot[x] = (int)list.size();
        list.push_back(x);
      }
    };
    for (const Trip& tr : same.trips) {
      need_pair(slotAT, listAT, tr.j, tr.k, o);
      need_pair(slotAT, listAT, tr.k, tr.i, o);
      need_pair(slotAT, listAT, tr.i, tr.j, o);
      need_one(slotBT, listBT, tr.i);
      need_one(slotBT, listBT, tr.j);
      need_one(slotBT, listBT, tr.k);
    }
    for (const Trip& tr : mixed.trips) {
      need_pair(slotA1, listA1, tr.j, tr.k, ot);
      need_pair(slotA1, listA1, tr.i, tr.k, ot);
      need_one(slotBG, listBG, tr.i);
      need_one(slotBG, listBG, tr.j);
      need_pair(slotAT, listAT, tr.i, tr.j, o);
      need_one(slotBF, listBF, tr.k);
      need_pair(slotAT2, listAT2, tr.j, tr.k, ot);
      need_pair(slotAT2, listAT2, tr.i, tr.k, ot);
      need_one(slotBT, listBT, tr.i);
      need_one(slotBT, listBT, tr.j);
    }
  }

  template <class St>
  int pack_all(St stAT, St stBT, St stA1, St stBG, St stBF, St stAT2) {
    Arena& A = own;
    cudaStream_t st = R.st;
    // ---- same-spin operands -------------------------------------------------
    if (!listAT.empty()) {
      double* oovoT;
      TRY(A.get(&oovoT, (size_t)o * v * oi * o));
      TRY(R.df(R.Boo[s], 0, oi * o, R.Bov[s], 0, o * v, oovoT, oi * o));
      if (!R.amax_pass) {
        int2* dl;
        TRY(A.get(&dl, listAT.size()));
        CU(cudaMemcpyAsync(dl, listAT.data(), listAT.size() * sizeof(int2),
                           cudaMemcpyHostToDevice, st));
        R.stats->other_launches++;
        CU(launch_pack_at_same(dl, (int)listAT.size(), o, oi, v, AT.Kp, t2ss, oovoT, stAT, st));
      }
      A.drop(oovoT);
    }
    if (!listBT.empty()) {
      double* vvovT;
      TRY(A.get(&vvovT, (size_t)v * v * v));
      for (size_t q = 0; q < listBT.size(); ++q) {
        const int x = listBT[q];
        TRY(R.df(R.Bvv[s], 0, v * v, R.Bov[s], (int64_t)x * v, v, vvovT, v * v));
        if (!R.amax_pass) {
          R.stats->other_launches++;
          CU(launch_pack_bt_same((int)q, x, o, oi, v, BT.Kp, vvovT, t2ss, stBT, st));
        }
      }
      A.drop(vvovT);
    }
    // ---- mixed operands -----------------------------------------------------
    if (!listA1.empty()) {
      double* jT;
      TRY(A.get(&jT, (size_t)o * v * oti * ot));
      TRY(R.df(R.Bov[s], 0, o * v, R.Boo[t], 0, oti * ot, jT, o * v));
      if (!R.amax_pass) {
        int2* dl;
        TRY(A.get(&dl, listA1.size()));
        CU(cudaMemcpyAsync(dl, listA1.data(), listA1.size() * sizeof(int2),
                           cudaMemcpyHostToDevice, st));
        R.stats->other_launches++;
        CU(launch_pack_a1(dl, (int)listA1.size(), o, v, ot, oti, vt, A1.Kp, t2st, jT, stA1, st));
      }
      A.drop(jT);
    }
    if (!listBG.empty()) {
      double* gT;
      TRY(A.get(&gT, (size_t)v * vt * vt));
      for (size_t q = 0; q < listBG.size(); ++q) {
        const int x = listBG[q];
        TRY(R.df(R.Bvv[t], 0, vt * vt, R.Bov[s], (int64_t)x * v, v, gT, vt * vt));
        if (!R.amax_pass) {
          R.stats->other_launches++;
          CU(launch_pack_bg((int)q, x, o, v, ot, oti, vt, BG.Kp, gT, t2st, stBG, st));
        }
      }
      A.drop(gT);
    }
    if (!listBF.empty()) {
      double* fT;
      TRY(A.get(&fT, (size_t)vt * v * v));
      for (size_t q = 0; q < listBF.size(); ++q) {
        const int K = listBF[q];
        TRY(R.df(R.Bvv[s], 0, v * v, R.Bov[t], (int64_t)K * vt, vt, fT, v * v));
        if (!R.amax_pass) {
          R.stats->other_launches++;
          CU(launch_pack_bf((int)q, K, o, oi, v, ot, vt, BF.Kp, fT, t2st, stBF, st));
        }
      }
      A.drop(fT);
    }
    if (!listAT2.empty()) {
      double* lT;
      TRY(A.get(&lT, (size_t)ot * vt * oi * o));
      TRY(R.df(R.Boo[s], 0, oi * o, R.Bov[t], 0, ot * vt, lT, oi * o));
      if (!R.amax_pass) {
        int2* dl;
        TRY(A.get(&dl, listAT2.size()));
        CU(cudaMemcpyAsync(dl, listAT2.data(), listAT2.size() * sizeof(int2),
                           cudaMemcpyHostToDevice, st));
        R.stats->other_launches++;
        CU(launch_pack_at2(dl, (int)listAT2.size(), o, oi, v, ot, vt, AT2.Kp, t2st, lT, stAT2,
                           st));
      }
      A.drop(lT);
    }
    return LNO_OT_OK;
  }

  int upload_ints(const std::vector<int>& h, int** d) {
    TRY(own.get(d, std::max<size_t>(h.size(), 1)));
    if (!h.empty())
      CU(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, R.st));
    return LNO_OT_OK;
  }

  int build_v_blocks() {
    const int nS = (int)listBT.size(), nT = (int)listBF.size();
    TRY(upload_ints(slotBT, &d_slot_s));
    TRY(upload_ints(slotBF, &d_slot_t));
    TRY(upload_ints(listBT, &d_list_s));
    TRY(upload_ints(listBF, &d_list_t));
    const int64_t ns = (int64_t)nS * v;
    TRY(R.gather_operand(own, R.Bov[s], d_list_s, nS, v, BsS));
    TRY(own.get(&ovss, (size_t)std::max<int64_t>(ns * ns, 1)));
    TRY(R.df(BsS, 0, (int)ns, BsS, 0, (int)ns, ovss, (int)ns));
    if (!mixed.trips.empty()) {
      const int64_t nt = (int64_t)nT * vt;
      TRY(R.gather_operand(own, R.Bov[t], d_list_t, nT, vt, BsT));
      TRY(own.get(&ovts, (size_t)std::max<int64_t>(nt * ns, 1)));
      TRY(R.df(BsS, 0, (int)ns, BsT, 0, (int)nt, ovts, (int)ns));
    }
    return LNO_OT_OK;
  }

  void set_v_args(EnergyArgs& ea, bool is_mixed) const {
    ea.ovov_ss = ovss;
    ea.ovov_ts = ovts;
    ea.oslot_s = d_slot_s;
    ea.oslot_t = is_mixed ? d_slot_t : d_slot_s;
    ea.ns_c = (int)listBT.size();
    ea.nt_c = is_mixed ? (int)listBF.size() : ea.ns_c;
  }

  int prepare_inputs() {
    t2ss = s == 0 ? R.dom->t2aa : R.dom->t2bb;
    if (!mixed.trips.empty() && t2st == nullptr) {
      if (s == 0) {
        t2st = const_cast<double*>(R.dom->t2ab);
      } else {
        TRY(own.get(&t2st, (size_t)std::max<int64_t>((int64_t)o * ot * v * vt, 1)));
        R.stats->other_launches++;
        CU(launch_transpose_t2ab(R.dom->t2ab, ot, o, vt, v, t2st, R.st));
      }
    }
    return LNO_OT_OK;
  }

  // measure integral magnitudes (sliced path, first pass)
  int measure() {
    if (listAT.empty() && listBT.empty() && listA1.empty() && listBG.empty() && listBF.empty() &&
        listAT2.empty())
      return LNO_OT_OK;
    R.amax_pass = true;
    StoreF64 dummy{nullptr};
    int rc = pack_all(dummy, dummy, dummy, dummy, dummy, dummy);
    R.amax_pass = false;
    return rc;
  }

  int build() {
    const bool tf = R.tf32;
    TRY(R.alloc_operand(own, AT, (int)listAT.size(), v, v + oi, R.S, tf));
    TRY(R.alloc_operand(own, BT, (int)listBT.size(), npairs(v), v + oi, R.S, tf));
    TRY(R.alloc_operand(own, A1, (int)listA1.size(), v, vt + oti, R.S, tf));
    TRY(R.alloc_operand(own, BG, (int)listBG.size(), (int64_t)v * vt, vt + oti, R.S, tf));
    TRY(R.alloc_operand(own, BF, (int)listBF.size(), (int64_t)v * vt, v + oi, R.S, tf));
    TRY(R.alloc_operand(own, AT2, (int)listAT2.size(), vt, v + oi, R.S, tf));
    if (R.f64) return pack_all(StoreF64{AT.f64}, StoreF64{BT.f64}, StoreF64{A1.f64},
                               StoreF64{BG.f64}, StoreF64{BF.f64}, StoreF64{AT2.f64});
    if (tf)
      return pack_all(R.tf32_slices(AT), R.tf32_slices(BT), R.tf32_slices(A1),
                      R.tf32_slices(BG), R.tf32_slices(BF), R.tf32_slices(AT2));
    if (R.S == 2)
      return pack_all(R.slices<2>(AT), R.slices<2>(BT), R.slices<2>(A1), R.slices<2>(BG),
                      R.slices<2>(BF), R.slices<2>(AT2));
    if (R.S == 4)
      return pack_all(R.slices<4>(AT), R.slices<4>(BT), R.slices<4>(A1), R.slices<4>(BG),
                      R.slices<4>(BF), R.slices<4>(AT2));
    if (R.S == 5)
      return pack_all(R.slices<5>(AT), R.slices<5>(BT), R.slices<5>(A1), R.slices<5>(BG),
                      R.slices<5>(BF), R.slices<5>(AT2));
    return pack_all(R.slices<3>(AT), R.slices<3>(BT), R.slices<3>(A1), R.slices<3>(BG),
                    R.slices<3>(BF), R.slices<3>(AT2));
  }

  // ---- contraction launches -------------------------------------------------
  int contract(int nprob, int M, int N, int ldo, const Operand& opA0, const Operand& opA1,
               const Operand& opB0, const Operand& opB1, const std::vector<ProbF64>& pf,
               const std::vector<TcProb>& pt, ProbF64* dpf, TcProb* dpt,
               TcOut lay = TcOut{kOutRows, 0, 0, 0}) {
    cudaEvent_t e0 = R.event(), e1 = R.event();
    if (e0) cudaEventRecord(e0, R.st);
    if (R.f64) {
      CU(cudaMemcpyAsync(dpf, pf.data(), nprob * sizeof(ProbF64), cudaMemcpyHostToDevice, R.st));
      CU(launch_gemm_f64(dpf, nprob, M, N, ldo, R.st));
    } else {
      CU(cudaMemcpyAsync(dpt, pt.data(), nprob * sizeof(TcProb), cudaMemcpyHostToDevice, R.st));
      const double scale = R.sigT * R.sigI * std::ldexp(1.0, R.tf32 ? -20 : -14);
      CU(launch_contract(R.S, R.tf32, bn, opA0, opA1, opB0, opB1, dpt, nprob, M, N, ldo, scale,
                         R.ctx->d_flag, R.ctx->nsm, R.st, lay));
    }
    if (e1) cudaEventRecord(e1, R.st);
    if (e0 && e1) R.contract_ev.push_back({e0, e1});
    R.stats->contract_launches++;
    return LNO_OT_OK;
  }

  void seg_f64(SegF64& sg, const Operand& A, int64_t arow, const Operand& B, int64_t brow,
               double sign) {
    sg = SegF64{A.f64 + arow * A.Kp, B.f64 + brow * B.Kp, A.K, A.Kp, B.Kp, sign};
  }
  // roles exchanged for the row-major launch (launch_contract): the kernel's
  // A is the pair operand B, its B the virtual operand A
  void seg_tc(TcSeg& sg, int amap, const Operand& A, int64_t arow, int bmap, const Operand& B,
              int64_t brow, int neg) {
    sg = TcSeg{bmap, amap, (int)brow, (int)arow, A.K, neg};
  }

  int run_case(bool is_mixed) {
    CaseSel& cs = is_mixed ? mixed : same;
    const int ntrip = (int)cs.trips.size();
    if (ntrip == 0) return LNO_OT_OK;
    Arena A(R.st, 0);  // per-case buffers
    const bool f64 = R.f64;
    const size_t esz = f64 ? 8 : 4;
    // output layouts
    const int M1 = v;                                       // rows a
    const int64_t N1 = is_mixed ? (int64_t)v * vt : npairs(v);
    const int P1 = (int)round_up(std::max(M1, 1), 16);
    const int M2 = vt;                                      // mixed Z': rows C
    const int64_t N2 = is_mixed ? npairs(v) : 0;
    const int P2 = (int)round_up(std::max(M2, 1), 16);
    const int nbs = (v + 15) / 16, nbt = (vt + 15) / 16;
    // mixed spin on the tensor cores without f_ov: Y and Z' as 16^3 tiles (the
    // TMA-staged energy kernel reads each sub-cube with one bulk copy);
    // otherwise rows [pair][a] of pitch P1 (P2)
    const bool fov = R.fov[0] != nullptr;   // restricted open-shell f_ov term
    const bool tiled = !f64 && is_mixed && !fov;
    const int64_t xs = tiled ? (int64_t)nbs * nbt * nbs * kTile : N1 * P1;   // per triplet
    const int64_t zs = tiled ? (int64_t)nbs * (nbs + 1) / 2 * nbt * kTile : N2 * P2;
    const TcOut lay1 = tiled ? TcOut{kOutYTile, vt, nbs, nbt} : TcOut{kOutRows, 0, 0, 0};
    const TcOut lay2 = tiled ? TcOut{kOutZTile, 0, nbs, nbt} : TcOut{kOutRows, 0, 0, 0};
    const int64_t per_trip = (xs + zs) * (int64_t)esz;
    const int64_t budget = (int64_t)6 << 30;
    bn = 0;
    group_cap = 64;
    if (const auto* row = R.ctx->tune_for(v)) {
      bn = row->bn;
      group_cap = std::max(1, row->group_cap);
    }
    int G = (int)std::max<int64_t>(
        1, std::min<int64_t>(group_cap, budget / std::max<int64_t>(per_trip, 1)));
    // energy chunks per triplet from the domain's shape only, so that a
    // triplet's partial sums (and its e_t, bit for bit) do not depend on
    // which other triplets the call selects
    const int Gshape = G;
    G = std::min(G, ntrip);
    char *X = nullptr, *Z = nullptr;
    TRY(A.get(&X, (size_t)(G * xs * esz) + 64));
    if (is_mixed) TRY(A.get(&Z, (size_t)(G * zs * esz) + 64));
    CU(cudaMemsetAsync(X, 0, (size_t)(G * xs * esz), R.st));
    if (is_mixed) CU(cudaMemsetAsync(Z, 0, (size_t)(G * zs * esz), R.st));
    // cube tiles
    std::vector<int3> blocks;
    if (!is_mixed) {
      for (int a = 0; a < nbs; ++a)
        for (int b = a; b < nbs; ++b)
          for (int c = b; c < nbs; ++c) blocks.push_back(make_int3(a, b, c));
    } else {
      for (int a = 0; a < nbs; ++a)
        for (int b = a; b < nbs; ++b)
          for (int c = 0; c < nbt; ++c) blocks.push_back(make_int3(a, b, c));
    }
    if (blocks.empty()) {  // no virtual orbitals in this case: every W is empty
      CU(cudaMemsetAsync(is_mixed ? e_mixed : e_same, 0, (size_t)ntrip * sizeof(double), R.st));
      return LNO_OT_OK;
    }
    int3* dblocks;
    TRY(A.get(&dblocks, blocks.size()));
    CU(cudaMemcpyAsync(dblocks, blocks.data(), blocks.size() * sizeof(int3),
                       cudaMemcpyHostToDevice, R.st));
    Trip* dtrips;
    TRY(A.get(&dtrips, (size_t)ntrip));
    CU(cudaMemcpyAsync(dtrips, cs.trips.data(), ntrip * sizeof(Trip), cudaMemcpyHostToDevice,
                       R.st));
    // float64 path: P chunks per triplet, one CTA each.  Float32 path: P
    // items per triplet on a persistent grid, about 32 items per resident CTA
    // in a full group (so the last round of items is a small fraction), one
    // partial per warp and item.
    const int P = f64 ? std::max(1, std::min((int)blocks.size(), R.ctx->nsm * 6 / Gshape + 1))
                      : std::max(1, std::min((int)blocks.size(),
                                             (64 * R.ctx->nsm + Gshape - 1) / Gshape));
    const int npart = f64 ? P : 8 * P;   // partials per triplet
    double* partial;
    TRY(A.get(&partial, (size_t)G * npart * (fov ? 2 : 1)));
    // float32 V tables of the tensor-core path, per triplet
    const int pv = (int)round_up(std::max(v, 1), 16), pvt = (int)round_up(std::max(vt, 1), 16);
    const int64_t vt_stride = is_mixed ? round_up(2LL * v * pvt + (int64_t)v * pv, 16)
                                       : 3LL * v * pv;
    // mixed spin on the tensor-core path takes the f_ov term in the same pass
    // (T1 and f_ov planes side by side in the V table); elsewhere a second pass
    const bool fuse = fov && !f64 && is_mixed;
    float* vtab = nullptr;
    if (!f64) TRY(A.get(&vtab, (size_t)(G * vt_stride * (fuse ? 2 : 1))));
    ProbF64* dpf = nullptr;
    TcProb* dpt = nullptr;
    if (f64) {
      TRY(A.get(&dpf, (size_t)G));
    } else {
      TRY(A.get(&dpt, (size_t)G));
    }
    std::vector<ProbF64> pf(G), pf2(G);
    std::vector<TcProb> pt(G), pt2(G);
    double* eout = is_mixed ? e_mixed : e_same;

    EnergyArgs ea{};
    ea.kind = is_mixed ? MIXED : SAME;
    ea.nvs = v;
    ea.nvt = is_mixed ? vt : v;
    ea.nos = o;
    ea.not_ = is_mixed ? ot : o;
    ea.eps_s = R.dom->eps[s];
    ea.eps_t = R.dom->eps[is_mixed ? t : s];
    ea.t1s = R.dom->t1[s];
    ea.t1t = R.dom->t1[is_mixed ? t : s];
    set_v_args(ea, is_mixed);
    ea.blocks = dblocks;
    ea.nblocks = (int)blocks.size();
    ea.pitch_x = P1;
    ea.pitch_z = P2;
    ea.x_stride = xs;
    ea.z_stride = zs;
    ea.tiled = tiled ? 1 : 0;
    ea.lap_s = R.lap_s;
    ea.lap_w = R.lap_w;
    ea.nsm = R.ctx->nsm;
    ea.flag = R.ctx->d_flag;

    // stats
    const double dv = v, dvt = vt;
    const double alg = is_mixed ? flops_alg_mixed(dv, dvt, (double)oi, (double)oti)
                                : flops_alg_same(dv, (double)oi);
    const double doi = oi, doti = oti;   // K of the hole parts: the internal ranges
    const double exe = is_mixed ? 2.0 * dv * (dv * dvt) * (2 * (dvt + doti) + dv + doi) +
                                      2.0 * dvt * (double)npairs(v) * 2 * (dv + doi)
                                : 2.0 * dv * (double)npairs(v) * 3 * (dv + doi);
    const double tens = is_mixed ? 2.0 * dv * (dv * dvt) * (2 * kpad16(dvt + doti) + kpad16(dv + doi)) +
                                       2.0 * dvt * (double)npairs(v) * 2 * kpad16(dv + doi)
                                 : 2.0 * dv * (double)npairs(v) * 3 * kpad16(dv + doi);
    R.stats->flops_algorithmic += alg * ntrip;
    R.stats->flops_executed += exe * ntrip;
    if (!f64) R.stats->tensor_flops += tens * ntrip * (R.S * (R.S + 1) / 2);
    R.stats->triplets += ntrip;
    R.stats->elements += (int64_t)ntrip *
                         (is_mixed ? npairs(v) * vt : (int64_t)v * (v - 1) * (v - 2) / 6);

    for (int g0 = 0; g0 < ntrip; g0 += G) {
      const int ng = std::min(G, ntrip - g0);
      for (int g = 0; g < ng; ++g) {
        const Trip tr = cs.trips[g0 + g];
        const int i = tr.i, j = tr.j, k = tr.k;
        char* Xg = X + (size_t)g * xs * esz;
        if (!is_mixed) {
          const int64_t r_jk = (int64_t)slotAT[(size_t)j * o + k] * v;
          const int64_t r_ki = (int64_t)slotAT[(size_t)k * o + i] * v;
          const int64_t r_ij = (int64_t)slotAT[(size_t)i * o + j] * v;
          const int64_t b_i = slotBT[i] * npairs(v), b_j = slotBT[j] * npairs(v),
                        b_k = slotBT[k] * npairs(v);
          if (f64) {
            ProbF64& p = pf[g];
            p.nseg = 3;
            seg_f64(p.seg[0], AT, r_jk, BT, b_i, 1.0);
            seg_f64(p.seg[1], AT, r_ki, BT, b_j, 1.0);
            seg_f64(p.seg[2], AT, r_ij, BT, b_k, 1.0);
            p.XT = reinterpret_cast<double*>(Xg);
          } else {
            TcProb& p = pt[g];
            p.nseg = 3;
            seg_tc(p.seg[0], 0, AT, r_jk, 0, BT, b_i, 0);
            seg_tc(p.seg[1], 0, AT, r_ki, 0, BT, b_j, 0);
            seg_tc(p.seg[2], 0, AT, r_ij, 0, BT, b_k, 0);
            p.out = Xg;
          }
        } else {
          const int K = k;
          const int64_t a1_jK = (int64_t)slotA1[(size_t)j * ot + K] * v;
          const int64_t a1_iK = (int64_t)slotA1[(size_t)i * ot + K] * v;
          const int64_t at_ij = (int64_t)slotAT[(size_t)i * o + j] * v;
          const int64_t bg_i = (int64_t)slotBG[i] * v * vt, bg_j = (int64_t)slotBG[j] * v * vt;
          const int64_t bf_K = (int64_t)slotBF[K] * v * vt;
          const int64_t a2_jK = (int64_t)slotAT2[(size_t)j * ot + K] * vt;
          const int64_t a2_iK = (int64_t)slotAT2[(size_t)i * ot + K] * vt;
          const int64_t bt_i = slotBT[i] * npairs(v), bt_j = slotBT[j] * npairs(v);
          char* Zg = Z + (size_t)g * zs * esz;
          if (f64) {
            ProbF64& p = pf[g];
            p.nseg = 3;
            seg_f64(p.seg[0], A1, a1_jK, BG, bg_i, 1.0);
            seg_f64(p.seg[1], A1, a1_iK, BG, bg_j, -1.0);
            seg_f64(p.seg[2], AT, at_ij, BF, bf_K, 1.0);
            p.XT = reinterpret_cast<double*>(Xg);
            ProbF64& q = pf2[g];
            q.nseg = 2;
            seg_f64(q.seg[0], AT2, a2_jK, BT, bt_i, -1.0);
            seg_f64(q.seg[1], AT2, a2_iK, BT, bt_j, 1.0);
            q.XT = reinterpret_cast<double*>(Zg);
          } else {
            TcProb& p = pt[g];
            p.nseg = 3;
            seg_tc(p.seg[0], 0, A1, a1_jK, 0, BG, bg_i, 0);
            seg_tc(p.seg[1], 0, A1, a1_iK, 0, BG, bg_j, 1);
            seg_tc(p.seg[2], 1, AT, at_ij, 1, BF, bf_K, 0);
            p.out = Xg;
            TcProb& q = pt2[g];
            q.nseg = 2;
            seg_tc(q.seg[0], 0, AT2, a2_jK, 0, BT, bt_i, 1);
            seg_tc(q.seg[1], 0, AT2, a2_iK, 0, BT, bt_j, 0);
            q.out = Zg;
          }
        }
      }
      if (!is_mixed) {
        TRY(contract(ng, M1, (int)N1, P1, AT, AT, BT, BT, pf, pt, dpf, dpt));
      } else {
        TRY(contract(ng, M1, (int)N1, P1, A1, AT, BG, BF, pf, pt, dpf, dpt, lay1));
        ProbF64* dpf2 = nullptr;
        TcProb* dpt2 = nullptr;
        // second problem list uses its own device array (the first may still be read)
        if (f64) {
          TRY(A.get(&dpf2, (size_t)ng));
        } else {
          TRY(A.get(&dpt2, (size_t)ng));
        }
        TRY(contract(ng, M2, (int)N2, P2, AT2, AT2, BT, BT, pf2, pt2, dpf2, dpt2, lay2));
        A.drop(f64 ? (void*)dpf2 : (void*)dpt2);
      }
      // energy
      ea.trips = dtrips + g0;
      ea.partial = partial;
      cudaEvent_t e0 = R.event(), e1 = R.event();
      if (e0) cudaEventRecord(e0, R.st);
      if (f64) {
        CU(launch_energy(ea, X, Z, f64, ng, P, R.st));
      } else if (fuse) {
        EnergyArgs ef = ea;
        ef.fs = R.fov[s];
        ef.ft = R.fov[t];
        ef.t2ss = t2ss;
        ef.t2st = t2st;
        CU(launch_energy_f32_fused(ef, reinterpret_cast<const float*>(X),
                                   reinterpret_cast<const float*>(Z), vtab, vt_stride, pv, pvt,
                                   ng, P, R.st));
        R.stats->energy_launches += 1;
      } else {
        CU(launch_energy_f32(ea, reinterpret_cast<const float*>(X),
                             reinterpret_cast<const float*>(Z), vtab, vt_stride, pv, pvt, ng, P,
                             R.st));
      }
      double* partial2 = nullptr;
      if (fov && !fuse) {
        // the f_ov part of V in a second pass over the same X (and Z'):
        // sum W V_f / D with V_f built like the T1 term from f_ov and T2
        EnergyArgs ef = ea;
        ef.vmode = 1;
        ef.t1s = R.fov[s];
        ef.t1t = R.fov[is_mixed ? t : s];
        ef.t2ss = t2ss;
        ef.t2st = t2st;
        ef.partial = partial2 = partial + (size_t)G * npart;
        if (f64)
          CU(launch_energy(ef, X, Z, f64, ng, P, R.st));
        else
          CU(launch_energy_f32(ef, reinterpret_cast<const float*>(X),
                               reinterpret_cast<const float*>(Z), vtab, vt_stride, pv, pvt, ng,
                               P, R.st));
        R.stats->energy_launches += 2;
      }
      CU(launch_reduce_partials(partial, npart, partial2, ng, eout + g0, R.st));
      if (e1) cudaEventRecord(e1, R.st);
      if (e0 && e1) R.energy_ev.push_back({e0, e1});
      R.stats->energy_launches += 2;
      // no host sync: the next group's descriptors overwrite pf/pt only after
      // cudaMemcpyAsync has staged this group's (pageable source), and the
      // device array is reused in stream order after this group's kernels
    }
    return LNO_OT_OK;
  }

  // operands for the current selections (the whole domain when cached)
  int prepare() {
    plan();
    TRY(prepare_inputs());
    TRY(build_v_blocks());
    TRY(build());
    return LNO_OT_OK;
  }
  int compute() {
    TRY(run_case(false));
    TRY(run_case(true));
    return LNO_OT_OK;
  }
  int run() {
    if (same.trips.empty() && mixed.trips.empty()) return LNO_OT_OK;
    TRY(prepare());
    return compute();
  }
};

int check_ptr(const lno_ot_ctx* ctx, const void* p, bool required) {
  if (!p) return required ? LNO_OT_EINVAL : LNO_OT_OK;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return LNO_OT_EDEVICE;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return LNO_OT_EDEVICE;
  if (at.device != ctx->device) return LNO_OT_EDEVICE;
  return LNO_OT_OK;
}

int validate(const lno_ot_ctx* ctx, const lno_ot_domain* d) {
  if (!d) return LNO_OT_EINVAL;
  if (d->nbas <= 0 || d->naux <= 0) return LNO_OT_EINVAL;
  if (d->nocc[1] < 0 || d->nocc[1] > d->nocc[0] || d->nocc[0] > d->nbas) return LNO_OT_EINVAL;
  if ((int64_t)d->nbas * d->nbas * d->naux > ((int64_t)1 << 40)) return LNO_OT_EINVAL;
  for (int s = 0; s < 2; ++s) {
    TRY(check_ptr(ctx, d->B[s], true));
    TRY(check_ptr(ctx, d->eps[s], true));
    const bool need_t1 = d->nocc[s] > 0 && d->nocc[s] < d->nbas;
    TRY(check_ptr(ctx, d->t1[s], need_t1));
  }
  const bool va = d->nocc[0] < d->nbas, vb = d->nocc[1] < d->nbas;
  TRY(check_ptr(ctx, d->t2aa, d->nocc[0] > 0 && va));
  TRY(check_ptr(ctx, d->t2bb, d->nocc[1] > 0 && vb));
  TRY(check_ptr(ctx, d->t2ab, d->nocc[0] > 0 && d->nocc[1] > 0 && va && vb));
  for (int c = 0; c < 4; ++c) TRY(check_ptr(ctx, d->e_trip[c], false));
  for (int s = 0; s < 2; ++s) {
    const bool has = d->nocc[s] > 0 && d->nocc[s] < d->nbas;
    TRY(check_ptr(ctx, d->fov[s], false));
    if (d->fov[s] && !has) return LNO_OT_EINVAL;   // nothing to hold
    TRY(check_ptr(ctx, d->e_orb[s], false));
  }
  return LNO_OT_OK;
}

// Per-case sums, per-triplet and orbital outputs, results and stats of one
// call (after the spin passes have filled e_int).
int finish_call(lno_ot_ctx* ctx, Run& R, Arena& A, const lno_ot_domain* dom, const CaseSel* cs,
                double* const* e_int, bool thirds, cudaEvent_t t0, cudaEvent_t t1,
                cudaEvent_t t2, lno_ot_result* out) {
  // per-case sums
  for (int c = 0; c < 4; ++c) {
    if (cs[c].trips.empty()) {
      CU(cudaMemsetAsync(ctx->d_sums + c, 0, sizeof(double), R.st));
    } else {
      CU(launch_neumaier_sum(e_int[c], (int64_t)cs[c].trips.size(), ctx->d_sums + c, R.st));
      R.stats->other_launches++;
      if (dom->e_trip[c])
        CU(cudaMemcpyAsync(dom->e_trip[c], e_int[c], cs[c].trips.size() * sizeof(double),
                           cudaMemcpyDeviceToDevice, R.st));
    }
  }
  // orbital contributions (eq cim_pt_energy) of the computed triplets
  if (dom->e_orb[0] || dom->e_orb[1]) {
    OrbPartArgs oa{};
    oa.na = dom->nocc[0];
    oa.nb = dom->nocc[1];
    oa.thirds = thirds;
    oa.out[0] = dom->e_orb[0];
    oa.out[1] = dom->e_orb[1];
    for (int c = 0; c < 4; ++c) {
      oa.e[c] = e_int[c];
      oa.n[c] = (int64_t)cs[c].trips.size();
      Trip* dt;
      TRY(A.get(&dt, std::max<size_t>(cs[c].trips.size(), 1)));
      if (!cs[c].trips.empty())
        CU(cudaMemcpyAsync(dt, cs[c].trips.data(), cs[c].trips.size() * sizeof(Trip),
                           cudaMemcpyHostToDevice, R.st));
      oa.trips[c] = dt;
    }
    CU(launch_orbital_partition(oa, R.st));
    R.stats->other_launches++;
  }
  double hs[4];
  CU(cudaMemcpyAsync(hs, ctx->d_sums, sizeof hs, cudaMemcpyDeviceToHost, R.st));
  if (t2) cudaEventRecord(t2, R.st);
  CU(cudaStreamSynchronize(R.st));
  int flag = 0;
  CU(cudaMemcpy(&flag, ctx->d_flag, sizeof flag, cudaMemcpyDeviceToHost));
  if (flag) return LNO_OT_ETIMEOUT;
  // stats
  float ms = 0;
  if (t0 && t2 && cudaEventElapsedTime(&ms, t0, t2) == cudaSuccess) ctx->stats.ms_total = ms;
  if (t0 && t1 && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess) ctx->stats.ms_stage = ms;
  double acc = 0;
  for (auto& p : R.contract_ev)
    if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) acc += ms;
  ctx->stats.ms_contract = acc;
  acc = 0;
  for (auto& p : R.energy_ev)
    if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) acc += ms;
  ctx->stats.ms_energy = acc;
  // order: aaa, aab, abb, bbb, total (Neumaier on the host for the last 4)
  double S = 0, Cc = 0;
  for (int c = 0; c < 4; ++c) {
    out->e[c] = hs[c];
    double x = hs[c], tt = S + x;
    Cc += std::fabs(S) >= std::fabs(x) ? (S - tt) + x : (x - tt) + S;
    S = tt;
  }
  out->e[4] = S + Cc;
  return LNO_OT_OK;
}

}  // namespace

// Whole-domain operands kept between calls (options.keep_operands): the DF
// blocks and scales of the Run and the operand tensors of both spin passes,
// built for every triplet of the domain.  A later call on the same arrays
// (another triplet selection) only runs the contractions and energy kernels.
struct DomainCache {
  lno_ot_domain key{};      // arrays and sizes the operands were built from
  int prec = 0;
  std::unique_ptr<Run> R;
  CaseSel cs[4];            // full selections at build time, the call's afterwards
  std::unique_ptr<SpinPass> pa, pb;
  bool has_a = false, has_b = false;

  bool matches(const lno_ot_domain* d, int p) const {
    if (p != prec || d->nbas != key.nbas || d->naux != key.naux) return false;
    for (int s = 0; s < 2; ++s)
      if (d->nocc[s] != key.nocc[s] || d->B[s] != key.B[s] || d->eps[s] != key.eps[s] ||
          d->t1[s] != key.t1[s] || d->fov[s] != key.fov[s])
        return false;
    return d->t2aa == key.t2aa && d->t2bb == key.t2bb && d->t2ab == key.t2ab;
  }
};

void destroy_cache(DomainCache* c) {
  if (!c) return;
  c->pa.reset();  // spin-pass operands first, then the Run's DF blocks
  c->pb.reset();
  c->R.reset();
  delete c;
}

namespace {

// Settings of an internal energy pass over an augmented domain (the central
// LMOs of the Laplace form): explicit triplet lists, per-spin orbital counts,
// internal occupied ranges, one quadrature point and eq local_pt's partition.
struct PassSpec {
  const CaseSel* cs;   // [4]
  int nbs[2];
  int noi[2];
  double lap_s, lap_w;
};

void set_precision(Run& R, int prec) {
  R.f64 = prec == LNO_OT_FP64;
  R.tf32 = prec == LNO_OT_TF32;
  R.S = prec == LNO_OT_BF16X6    ? 3
        : prec == LNO_OT_BF16X10 ? 4
        : prec == LNO_OT_BF16X15 ? 5
                                 : 2;
  R.Sdf = prec == LNO_OT_BF16X15 ? 5 : 4;
}

// Integral scale of the sliced path: one pass over every DF block the two
// spin passes need (their current selections).
int measure_sigI(lno_ot_ctx* ctx, Run& R, SpinPass* pa, SpinPass* pb) {
  if (R.f64) return LNO_OT_OK;
  if (pa) pa->plan();
  if (pb) pb->plan();
  if (pa) TRY(pa->prepare_inputs());
  if (pb) TRY(pb->prepare_inputs());
  CU(cudaMemsetAsync(ctx->d_amax, 0, sizeof(unsigned long long), R.st));
  if (pa) TRY(pa->measure());
  if (pb) TRY(pb->measure());
  unsigned long long h;
  CU(cudaMemcpyAsync(&h, ctx->d_amax, sizeof h, cudaMemcpyDeviceToHost, R.st));
  CU(cudaStreamSynchronize(R.st));
  double m;
  std::memcpy(&m, &h, 8);
  R.sigI = pow2_scale(2.0 * m);  // antisymmetrised combinations are <= 2 max
  return LNO_OT_OK;
}

// Builds ctx->cache for dom (every triplet of the domain).
int build_cache(lno_ot_ctx* ctx, const lno_ot_domain* dom) {
  destroy_cache(ctx->cache);
  ctx->cache = nullptr;
  std::unique_ptr<DomainCache> C(new DomainCache());
  C->key = *dom;
  for (int c = 0; c < 4; ++c) {
    C->key.e_trip[c] = nullptr;
    C->key.trip_sel[c] = nullptr;
    C->key.n_sel[c] = 0;
  }
  C->key.e_orb[0] = C->key.e_orb[1] = nullptr;
  C->prec = ctx->prec;
  C->R.reset(new Run(ctx, &C->key));
  Run& R = *C->R;
  set_precision(R, ctx->prec);
  for (int c = 0; c < 4; ++c) TRY(select_case(&C->key, c, C->cs[c]));
  TRY(R.stage());
  C->has_a = !C->cs[0].trips.empty() || !C->cs[1].trips.empty();
  C->has_b = !C->cs[3].trips.empty() || !C->cs[2].trips.empty();
  C->pa.reset(new SpinPass(R, 0, C->cs[0], C->cs[1], nullptr, nullptr));
  C->pb.reset(new SpinPass(R, 1, C->cs[3], C->cs[2], nullptr, nullptr));
  TRY(measure_sigI(ctx, R, C->has_a ? C->pa.get() : nullptr, C->has_b ? C->pb.get() : nullptr));
  if (C->has_a) TRY(C->pa->prepare());
  if (C->has_b) TRY(C->pb->prepare());
  CU(cudaStreamSynchronize(R.st));
  ctx->cache = C.release();
  return LNO_OT_OK;
}

// One call through the cache (built on a miss).  Returns LNO_OT_ENOMEM when
// the whole-domain operands do not fit; the caller then runs uncached.
int cached_energy(lno_ot_ctx* ctx, const lno_ot_domain* dom, lno_ot_result* out) {
  ctx->stats = lno_ot_stats{};
  ctx->ev_used = 0;
  CU(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
  cudaEvent_t t0 = nullptr, t1 = nullptr, t2 = nullptr;
  const bool hit = ctx->cache && ctx->cache->matches(dom, ctx->prec);
  {
    // events from the pool (the Run may not exist yet)
    for (cudaEvent_t* e : {&t0, &t1, &t2}) {
      if (ctx->ev_used == ctx->ev_pool.size()) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) {
          cudaGetLastError();
          break;
        }
        ctx->ev_pool.push_back(ev);
      }
      *e = ctx->ev_pool[ctx->ev_used++];
    }
  }
  if (t0) cudaEventRecord(t0, ctx->stream);
  if (!hit) {
    const int rc = build_cache(ctx, dom);
    if (rc != LNO_OT_OK) {
      destroy_cache(ctx->cache);
      ctx->cache = nullptr;
      cudaGetLastError();
      return rc;
    }
  }
  DomainCache* C = ctx->cache;
  Run& R = *C->R;
  R.dom = dom;
  R.contract_ev.clear();
  R.energy_ev.clear();
  if (t1) cudaEventRecord(t1, R.st);
  CaseSel sel[4];
  for (int c = 0; c < 4; ++c) {
    TRY(select_case(dom, c, sel[c]));
    C->cs[c].trips.swap(sel[c].trips);
    C->cs[c].ntot = sel[c].ntot;
  }
  Arena A(R.st, ctx->ws_limit);
  double* e_int[4];
  for (int c = 0; c < 4; ++c)
    TRY(A.get(&e_int[c], std::max<size_t>(C->cs[c].trips.size(), 1)));
  C->pa->e_same = e_int[0];
  C->pa->e_mixed = e_int[1];
  C->pb->e_same = e_int[3];
  C->pb->e_mixed = e_int[2];
  if (C->has_a) TRY(C->pa->compute());
  if (C->has_b) TRY(C->pb->compute());
  return finish_call(ctx, R, A, dom, C->cs, e_int, false, t0, t1, t2, out);
}

bool flip_candidate(const lno_ot_domain* dom) {
  bool flip = dom->nocc[0] == dom->nocc[1] && dom->B[0] == dom->B[1] &&
              dom->eps[0] == dom->eps[1] && dom->t1[0] == dom->t1[1] &&
              dom->t2aa == dom->t2bb && dom->fov[0] == dom->fov[1];
  for (int c = 0; c < 4; ++c) flip = flip && dom->trip_sel[c] == nullptr;
  return flip;
}

int energy_impl(lno_ot_ctx* ctx, const lno_ot_domain* dom, lno_ot_result* out,
                const PassSpec* spec = nullptr) {
  if (!spec) TRY(validate(ctx, dom));
  CU(cudaSetDevice(ctx->device));
  if (!spec && ctx->keep && !flip_candidate(dom)) {
    const int rc = cached_energy(ctx, dom, out);
    if (rc != LNO_OT_ENOMEM) return rc;   // the whole domain did not fit: run uncached
  }
  if (!spec) ctx->stats = lno_ot_stats{};
  ctx->ev_used = 0;
  Run R(ctx, dom);
  if (spec) {
    for (int s = 0; s < 2; ++s) {
      R.nbs[s] = spec->nbs[s];
      R.noi[s] = spec->noi[s];
    }
    R.lap_s = spec->lap_s;
    R.lap_w = spec->lap_w;
  }
  set_precision(R, ctx->prec);
  CU(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
  cudaEvent_t t0 = R.event(), t1 = R.event(), t2 = R.event();
  if (t0) cudaEventRecord(t0, R.st);

  CaseSel cs[4];
  for (int c = 0; c < 4; ++c) {
    if (spec)
      cs[c] = spec->cs[c];
    else
      TRY(select_case(dom, c, cs[c]));
  }
  double* e_int[4];
  for (int c = 0; c < 4; ++c)
    TRY(R.arena.get(&e_int[c], std::max<size_t>(cs[c].trips.size(), 1)));
  // Closed-shell domain (both spins given by the same arrays, spin-flip
  // symmetric mixed amplitudes): bbb and abb are the spin-flip images of aaa
  // and aab, with identical values, so only the spin-up pass runs.
  bool flip = flip_candidate(dom) && spec == nullptr;
  if (flip && dom->nocc[0] > 0 && dom->nocc[0] < dom->nbas) {
    // symmetric to within 1e-12 of the largest amplitude: amplitudes from a
    // closed-shell calculation agree with their spin-flip images to rounding
    const int n = dom->nocc[0], v = dom->nbas - dom->nocc[0];
    CU(cudaMemsetAsync(ctx->d_amax, 0, sizeof(unsigned long long), R.st));
    CU(launch_absmax(dom->t2ab, (int64_t)n * n * v * v, ctx->d_amax, R.st));
    unsigned long long hm = 0;
    CU(cudaMemcpyAsync(&hm, ctx->d_amax, sizeof hm, cudaMemcpyDeviceToHost, R.st));
    CU(cudaStreamSynchronize(R.st));
    double amax;
    std::memcpy(&amax, &hm, 8);
    unsigned int* cnt;
    TRY(R.arena.get(&cnt, 1));
    CU(cudaMemsetAsync(cnt, 0, sizeof(unsigned int), R.st));
    CU(launch_t2ab_flip_mismatch(dom->t2ab, n, v, 1e-12 * amax, cnt, R.st));
    unsigned int h = 1;
    CU(cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, R.st));
    CU(cudaStreamSynchronize(R.st));
    R.stats->other_launches += 2;
    flip = h == 0;
  }
  TRY(R.stage());
  {
    SpinPass pa(R, 0, cs[0], cs[1], e_int[0], e_int[1]);
    SpinPass pb(R, 1, cs[3], cs[2], e_int[3], e_int[2]);
    // integral scale: first pass over every DF block both spins need
    TRY(measure_sigI(ctx, R, &pa, flip ? nullptr : &pb));
    if (t1) cudaEventRecord(t1, R.st);
    TRY(pa.run());
    pa.own.release();
    if (!flip) {
      TRY(pb.run());
    } else {  // spin-flip images: bbb = aaa, abb = aab, triplet for triplet
      if (!cs[3].trips.empty())
        CU(cudaMemcpyAsync(e_int[3], e_int[0], cs[3].trips.size() * sizeof(double),
                           cudaMemcpyDeviceToDevice, R.st));
      if (!cs[2].trips.empty())
        CU(cudaMemcpyAsync(e_int[2], e_int[1], cs[2].trips.size() * sizeof(double),
                           cudaMemcpyDeviceToDevice, R.st));
    }
  }
  return finish_call(ctx, R, R.arena, dom, cs, e_int, spec != nullptr, t0, t1, t2, out);
}

// ---------------------------------------------------------------------------
// Natural auxiliary functions (Sec. 3.6, eq naf_w), float64 (naf.cu).
int naf_impl(lno_ot_ctx* ctx, const lno_ot_domain* dom, double eps, double* const* Bout,
             int* naux_out, double* lam_host) {
  if (!dom || !Bout || !naux_out || !(eps >= 0.0) || !std::isfinite(eps)) return LNO_OT_EINVAL;
  if (dom->nbas <= 0 || dom->naux <= 0) return LNO_OT_EINVAL;
  if ((int64_t)dom->nbas * dom->nbas * dom->naux > ((int64_t)1 << 40)) return LNO_OT_EINVAL;
  for (int s = 0; s < 2; ++s) {
    TRY(check_ptr(ctx, dom->B[s], true));
    TRY(check_ptr(ctx, Bout[s], true));
  }
  CU(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const int n = dom->naux, nb = dom->nbas;
  const int64_t npair = (int64_t)nb * (nb + 1) / 2, n2 = (int64_t)nb * nb;
  Arena A(st, ctx->ws_limit);
  double *J[2], *W, *V, *d, *norms;
  double2* cs;
  ProbF64* dp;
  for (int s = 0; s < 2; ++s) {
    TRY(A.get(&J[s], (size_t)(n * npair)));
    CU(launch_pack_pairs(dom->B[s], n, nb, J[s], st));
  }
  TRY(A.get(&W, (size_t)n * n));
  TRY(A.get(&dp, 2));
  {  // W = (J^up J^up^T + J^down J^down^T) / 2
    ProbF64 p{};
    p.nseg = 2;
    p.seg[0] = SegF64{J[0], J[0], (int)npair, (int)npair, (int)npair, 0.5};
    p.seg[1] = SegF64{J[1], J[1], (int)npair, (int)npair, (int)npair, 0.5};
    p.XT = W;
    CU(cudaMemcpyAsync(dp, &p, sizeof p, cudaMemcpyHostToDevice, st));
    CU(launch_gemm_f64(dp, 1, n, n, n, st));
    CU(cudaStreamSynchronize(st));
  }
  A.drop(J[0]);
  A.drop(J[1]);
  TRY(A.get(&V, (size_t)n * n));
  TRY(A.get(&cs, (size_t)(n / 2 + 1)));
  TRY(A.get(&norms, 2));
  TRY(A.get(&d, (size_t)n));
  const int sweeps = jacobi_eigh(W, V, n, cs, norms, st, 40);
  if (sweeps < 0) return sweeps;
  CU(launch_get_diag(W, n, d, st));
  std::vector<double> lam(n);
  CU(cudaMemcpyAsync(lam.data(), d, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] > lam[b]; });
  int nk = 0;
  while (nk < n && lam[order[nk]] > eps) ++nk;
  if (lam_host)
    for (int i = 0; i < n; ++i) lam_host[i] = lam[order[i]];
  *naux_out = nk;
  if (nk > 0) {
    int* cols;
    double *Vt, *Bt;
    TRY(A.get(&cols, (size_t)nk));
    CU(cudaMemcpyAsync(cols, order.data(), (size_t)nk * sizeof(int), cudaMemcpyHostToDevice, st));
    TRY(A.get(&Vt, (size_t)nk * n));
    CU(launch_gather_cols(V, n, cols, nk, Vt, st));
    TRY(A.get(&Bt, (size_t)(n2 * n)));
    for (int s = 0; s < 2; ++s) {   // B'[X'][pq] = sum_X V[X][X'] B[X][pq]
      CU(launch_transpose_x(dom->B[s], n, n2, Bt, st));
      ProbF64 p{};
      p.nseg = 1;
      p.seg[0] = SegF64{Bt, Vt, n, n, n, 1.0};
      p.XT = Bout[s];
      CU(cudaMemcpyAsync(dp + s, &p, sizeof p, cudaMemcpyHostToDevice, st));
      CU(launch_gemm_f64(dp + s, 1, (int)n2, nk, (int)n2, st));
      CU(cudaStreamSynchronize(st));
    }
  }
  CU(cudaStreamSynchronize(st));
  return LNO_OT_OK;
}

// ---------------------------------------------------------------------------
// Central-LMO share in the Laplace form (Sec. 3.7, eqs laplace_transform and
// local_pt): per quadrature point, an augmented domain with one pseudo-orbital
// per central orbital (central.cu), the triplets that hold exactly one of
// them, the element weight -w_q exp(s_q D), and eq local_pt's 1/3 of each
// triplet to the pseudo-orbital; the quadrature points are summed on the host.
int central_impl(lno_ot_ctx* ctx, const lno_ot_domain* dom, const lno_ot_central* c) {
  if (!c) return LNO_OT_EINVAL;
  TRY(validate(ctx, dom));
  if (c->nq < 1 || c->nq > 256 || !c->s || !c->w || c->spin < 0 || c->spin > 1 || c->nlmo < 0)
    return LNO_OT_EINVAL;
  if (c->nlmo > 0 && !c->dE) return LNO_OT_EINVAL;
  for (int q = 0; q < c->nq; ++q)
    if (!(c->s[q] > 0.0) || !std::isfinite(c->s[q]) || !std::isfinite(c->w[q]))
      return LNO_OT_EINVAL;
  const int sg = c->spin, tg = 1 - sg, P = c->nlmo;
  const int nbas = dom->nbas, naux = dom->naux;
  const int na = dom->nocc[0], nb = dom->nocc[1], o = dom->nocc[sg];
  const int v = nbas - o;
  for (int l = 0; l < P; ++l) c->dE[l] = 0.0;
  if (P == 0) return LNO_OT_OK;
  if (o == 0) return LNO_OT_EINVAL;
  TRY(check_ptr(ctx, c->U, true));
  CU(cudaSetDevice(ctx->device));
  ctx->stats = lno_ot_stats{};
  cudaStream_t st = ctx->stream;
  Arena A(st, ctx->ws_limit);
  // augmented arrays of spin sg
  const int nb2 = nbas + P, o2 = o + P;
  AugmentArgs ag{};
  ag.spin = sg;
  ag.P = P;
  ag.nbas = nbas;
  ag.naux = naux;
  ag.nocc[0] = na;
  ag.nocc[1] = nb;
  ag.U = c->U;
  ag.B_in = dom->B[sg];
  ag.eps_in = dom->eps[sg];
  ag.t1_in = dom->t1[sg];
  ag.fov_in = dom->fov[sg];
  ag.t2ss_in = sg == 0 ? dom->t2aa : dom->t2bb;
  ag.t2ab_in = dom->t2ab;
  const int va = nbas - na, vb = nbas - nb;
  TRY(A.get(&ag.coef, (size_t)P * o));
  TRY(A.get(&ag.B_out, (size_t)naux * nb2 * nb2));
  TRY(A.get(&ag.eps_out, (size_t)nb2));
  TRY(A.get(&ag.t1_out, (size_t)std::max(o2 * v, 1)));
  if (ag.fov_in) TRY(A.get(&ag.fov_out, (size_t)std::max(o2 * v, 1)));
  TRY(A.get(&ag.t2ss_out, (size_t)std::max<int64_t>((int64_t)o2 * o2 * v * v, 1)));
  TRY(A.get(&ag.t2ab_out, (size_t)std::max<int64_t>(
                              (int64_t)(sg == 0 ? o2 : na) * (sg == 0 ? nb : o2) * va * vb, 1)));
  double* eorb;
  TRY(A.get(&eorb, (size_t)o2));
  // triplets holding exactly one pseudo-orbital (augmented indices o + p)
  CaseSel cs[4];
  const int ot = dom->nocc[tg];
  for (int p = 0; p < P; ++p) {
    const int u = o + p;
    for (int j = 0; j < o; ++j)      // same spin: (j, k, u), j < k < u
      for (int k = j + 1; k < o; ++k) cs[sg == 0 ? 0 : 3].trips.push_back(Trip{j, k, u});
    for (int j = 0; j < o; ++j)      // u and j of spin sg, K of the other: (j, u; K)
      for (int K = 0; K < ot; ++K) cs[sg == 0 ? 1 : 2].trips.push_back(Trip{j, u, K});
    for (int J = 0; J < ot; ++J)     // J < K of the other spin, u the single: (J, K; u)
      for (int K = J + 1; K < ot; ++K) cs[sg == 0 ? 2 : 1].trips.push_back(Trip{J, K, u});
  }
  lno_ot_domain ad = *dom;
  ad.nocc[sg] = o2;
  ad.B[sg] = ag.B_out;
  ad.eps[sg] = ag.eps_out;
  ad.t1[sg] = ag.t1_out;
  if (ag.fov_in) ad.fov[sg] = ag.fov_out;
  if (sg == 0)
    ad.t2aa = ag.t2ss_out;
  else
    ad.t2bb = ag.t2ss_out;
  ad.t2ab = ag.t2ab_out;
  for (int k = 0; k < 4; ++k) {
    ad.e_trip[k] = nullptr;
    ad.trip_sel[k] = nullptr;
    ad.n_sel[k] = 0;
  }
  ad.e_orb[sg] = eorb;
  ad.e_orb[tg] = nullptr;
  PassSpec spec{};
  spec.cs = cs;
  spec.nbs[sg] = nb2;
  spec.nbs[tg] = nbas;
  spec.noi[0] = na;
  spec.noi[1] = nb;
  std::vector<double> acc(P, 0.0), comp(P, 0.0), part(P);
  double ms[4] = {0, 0, 0, 0};
  for (int q = 0; q < c->nq; ++q) {
    ag.s = c->s[q];
    CU(launch_lmo_augment(ag, st));
    ctx->stats.other_launches += 7;
    spec.lap_s = c->s[q];
    spec.lap_w = c->w[q];
    lno_ot_result r;
    TRY(energy_impl(ctx, &ad, &r, &spec));
    ms[0] += ctx->stats.ms_total;
    ms[1] += ctx->stats.ms_stage;
    ms[2] += ctx->stats.ms_contract;
    ms[3] += ctx->stats.ms_energy;
    CU(cudaMemcpyAsync(part.data(), eorb + o, (size_t)P * sizeof(double), cudaMemcpyDeviceToHost,
                       st));
    CU(cudaStreamSynchronize(st));
    for (int l = 0; l < P; ++l) {   // Neumaier over the quadrature points, in order
      const double x = part[l], t = acc[l] + x;
      comp[l] += std::fabs(acc[l]) >= std::fabs(x) ? (acc[l] - t) + x : (x - t) + acc[l];
      acc[l] = t;
    }
  }
  for (int l = 0; l < P; ++l) c->dE[l] = acc[l] + comp[l];
  ctx->stats.ms_total = ms[0];
  ctx->stats.ms_stage = ms[1];
  ctx->stats.ms_contract = ms[2];
  ctx->stats.ms_energy = ms[3];
  return LNO_OT_OK;
}

// ---------------------------------------------------------------------------
// Adjoint (float64).  Gradient accumulators of one domain (raw, unprojected).
struct GradAcc {
  Operand dBoo[2], dBov[2], dBvv[2];  // same layout as the DF blocks
  double* dt1[2];
  double* deps[2];
  double* dfov[2];                    // f_ov gradients (when the domain has f_ov)
  double* dt2aa;
  double* dt2bb;
  double* dt2ab;
};

int zeros(Arena& A, double** p, int64_t n, cudaStream_t st) {
  TRY(A.get(p, (size_t)std::max<int64_t>(n, 1)));
  CU(cudaMemsetAsync(*p, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(double), st));
  return LNO_OT_OK;
}

int zero_operand_like(Arena& A, const Operand& src, Operand& d, cudaStream_t st) {
  d = src;
  const int64_t n = std::max<int64_t>((int64_t)src.nslot * src.rows * src.Kp, 8);
  return zeros(A, &d.f64, n, st);
}

// C[m ldc + n] (+)= alpha sum_k a(m, k) b(n, k) on the tensor cores: both views
// are cut into 4 exact BF16 slices with power-of-two scales (the DF assembly's
// representation, 10 slice products, float64 output of the exact class sums).
// Used by the adjoint of the tensor-core precisions.
int tc_matmul(Run& R, Arena& A, int M, int N, int K, View a, View b, double* C, int64_t ldc,
              double alpha, bool accum, bool b_const) {
  if (M <= 0 || N <= 0 || K <= 0) return LNO_OT_OK;
  constexpr int S = 4;
  cudaStream_t st = R.st;
  cudaEvent_t e0 = R.event(), e1 = R.event();
  if (e0) cudaEventRecord(e0, st);
  // Split K when the output has few 128 x 128 tiles (a long contraction onto a
  // short output: the contraction adjoints over the pair rows, the DF adjoints
  // over v^2 rows): chunk c is problem c of one launch, writing its own float64
  // partial; the partials are added into C in chunk order.
  const int64_t tiles = (int64_t)ceil_div(N, 128) * ceil_div(M, 128);
  int nsp = 1;
  if (tiles < 2 * R.ctx->nsm && K >= 4096)
    nsp = (int)std::max<int64_t>(1, std::min<int64_t>({ceil_div(4 * R.ctx->nsm, tiles),
                                                       K / 2048, kMaxSplit}));
  const int Kc = (int)round_up(ceil_div(K, nsp), 32);
  nsp = ceil_div(K, Kc);
  const int64_t Kp = round_up(Kc, 8);
  // a read-only B view sliced before with the same chunking
  const SliceCacheEntry* hit = nullptr;
  if (b_const)
    for (const auto& e : R.slice_cache)
      if (e.p == b.p && e.rs == b.rs && e.ks == b.ks && e.rows == N && e.K == K && e.Kc == Kc &&
          e.nsp == nsp)
        hit = &e;
  unsigned long long* am = R.ctx->d_amax;
  CU(cudaMemsetAsync(am, 0, 2 * sizeof(unsigned long long), st));
  CU(launch_view_absmax(a.p, a.rs, a.ks, M, K, am, st));
  if (!hit) CU(launch_view_absmax(b.p, b.rs, b.ks, N, K, am + 1, st));
  unsigned long long hb[2];
  CU(cudaMemcpyAsync(hb, am, sizeof hb, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  double amax[2];
  std::memcpy(amax, hb, sizeof amax);
  if (hit) amax[1] = hit->sigma;
  if (!std::isfinite(amax[0]) || !std::isfinite(amax[1])) return LNO_OT_EINVAL;
  if (amax[0] == 0.0 || amax[1] == 0.0) {   // a zero operand: nothing to add
    if (!accum)
      for (int m = 0; m < M; ++m)
        CU(cudaMemsetAsync(C + (int64_t)m * ldc, 0, (size_t)N * sizeof(double), st));
    return LNO_OT_OK;
  }
  auto pow2_at_least = [](double x) {
    int e;
    const double f = std::frexp(x, &e);
    return std::ldexp(1.0, f == 0.5 ? e - 1 : e);
  };
  const double sa = pow2_at_least(amax[0]), sb = hit ? hit->sigma : pow2_at_least(amax[1]);
  __nv_bfloat16 *qa, *qb = hit ? hit->q : nullptr;
  TRY(A.get(&qa, (size_t)(S * nsp * M * Kp)));
  if (!qb) {
    if (b_const)
      TRY(R.arena.get(&qb, (size_t)(S * nsp * N * Kp)));
    else
      TRY(A.get(&qb, (size_t)(S * nsp * N * Kp)));
  }
  for (int c = 0; c < nsp; ++c) {
    const int k0 = c * Kc, kc = std::min(Kc, K - k0);
    CU(launch_view_slices<S>(a.p + k0 * a.ks, a.rs, a.ks, M, kc, (int)Kp, qa + c * M * Kp,
                             (int64_t)nsp * M * Kp, 128.0 / sa, st));
    if (!hit)
      CU(launch_view_slices<S>(b.p + k0 * b.ks, b.rs, b.ks, N, kc, (int)Kp, qb + c * N * Kp,
                               (int64_t)nsp * N * Kp, 128.0 / sb, st));
  }
  if (b_const && !hit) R.slice_cache.push_back({b.p, b.rs, b.ks, N, K, Kc, nsp, qb, sb});
  // the kernel writes its output transposed: its rows (A role) are n, its
  // columns (B role) m, so out[m ldc + n]
  CUtensorMap mA[2], mB[2];
  TRY(make_operand_map(&mA[0], qb, Kp, (int64_t)nsp * N, S, (int64_t)nsp * N * Kp, 128));
  TRY(make_operand_map(&mB[0], qa, Kp, (int64_t)nsp * M, S, (int64_t)nsp * M * Kp, 128));
  mA[1] = mA[0];
  mB[1] = mB[0];
  double* part = nullptr;
  if (nsp > 1) TRY(A.get(&part, (size_t)nsp * M * N));
  // the float32 rest scales in float32: |alpha| must be a power of two (the
  // adjoint's products use +-1)
  int ex;
  if (std::frexp(std::fabs(alpha), &ex) != 0.5) return LNO_OT_EINVAL;
  const double scale = sa * sb * std::ldexp(1.0, -14) * std::fabs(alpha);
  // products of the class sums with the scale stay normal floats
  const bool float_rest = scale >= std::ldexp(1.0, -100) && scale <= std::ldexp(1.0, 100);
  std::vector<TcProb> pv(nsp);
  for (int c = 0; c < nsp; ++c) {
    TcProb& p = pv[c];
    p.nseg = 1;
    p.seg[0] = TcSeg{0, 0, c * N, c * M, std::min(Kc, K - c * Kc), alpha < 0 ? 1 : 0};
    p.flags = (float_rest ? kTcFloatRest : 0) | (nsp == 1 && accum ? kTcAccum : 0);
    p.out = nsp == 1 ? C : part + (int64_t)c * M * N;
  }
  TcProb* dp;
  TRY(A.get(&dp, (size_t)nsp));
  CU(cudaMemcpyAsync(dp, pv.data(), nsp * sizeof(TcProb), cudaMemcpyHostToDevice, st));
  CU((launch_tc_gemm<4, 128, double, false, false>(mA, mB, dp, nsp, N, M,
                                                   nsp == 1 ? (int)ldc : N, scale,
                                                   R.ctx->d_flag, nullptr, R.ctx->nsm, st,
                                                   tc_normal())));
  if (nsp > 1) CU(launch_sum_partials(part, nsp, M, N, C, ldc, accum, st));
  if (e1) cudaEventRecord(e1, st);
  if (e0 && e1) R.contract_ev.push_back({e0, e1});
  R.stats->contract_launches++;
  R.stats->other_launches += 3 + 2 * nsp;
  A.drop(qa);
  if (!b_const) A.drop(qb);
  A.drop(dp);
  if (part) A.drop(part);
  return LNO_OT_OK;
}

// DF adjoint: out[n][m] = sum_Q L[l0+m][Q] R[r0+n][Q]  ->  dL, dR (+=)
int df_adjoint(Run& R, Arena& A, const Operand& Lo, Operand& dL, int64_t l0, int M,
               const Operand& Ro, Operand& dR, int64_t r0, int N, const double* dout, int ldo) {
  if (M <= 0 || N <= 0) return LNO_OT_OK;
  const int64_t Qp = Lo.Kp;
  if (R.tc_adjoint) {
    // dL[l0+m][Q] += sum_n dout[n][m] R[r0+n][Q];  dR[r0+n][Q] += sum_m dout[n][m] L[l0+m][Q]
    TRY(tc_matmul(R, A, M, R.naux, N, View{dout, 1, ldo}, View{Ro.f64 + r0 * Qp, 1, Qp},
                  dL.f64 + l0 * Qp, Qp, 1.0, true, true));
    TRY(tc_matmul(R, A, N, R.naux, M, View{dout, ldo, 1}, View{Lo.f64 + l0 * Qp, 1, Qp},
                  dR.f64 + r0 * Qp, Qp, 1.0, true, true));
    return LNO_OT_OK;
  }
  GemmS g[2];
  g[0] = GemmS{dout, Ro.f64 + r0 * Qp, dL.f64 + l0 * Qp, M, R.naux, N, 0,
               1, ldo, Qp, 1, Qp, 1, 1.0};
  g[1] = GemmS{dout, Lo.f64 + l0 * Qp, dR.f64 + r0 * Qp, N, R.naux, M, 0,
               ldo, 1, Qp, 1, Qp, 1, 1.0};
  GemmS* dg;
  TRY(A.get(&dg, 2));
  CU(cudaMemcpyAsync(dg, g, sizeof g, cudaMemcpyHostToDevice, R.st));
  CU(launch_gemm_strided(dg, 1, M, R.naux, R.st));
  CU(launch_gemm_strided(dg + 1, 1, N, R.naux, R.st));
  R.stats->other_launches += 2;
  CU(cudaStreamSynchronize(R.st));  // g lives on the host stack
  A.drop(dg);
  return LNO_OT_OK;
}

int backward_spin(SpinPass& P, GradAcc& G, double gE) {
  Run& R = P.R;
  cudaStream_t st = R.st;
  Arena A(st, 0);
  const int o = P.o, v = P.v, ot = P.ot, vt = P.vt, s = P.s, t = P.t;
  Operand dAT, dBT, dA1, dBG, dBF, dAT2;
  TRY(zero_operand_like(A, P.AT, dAT, st));
  TRY(zero_operand_like(A, P.BT, dBT, st));
  TRY(zero_operand_like(A, P.A1, dA1, st));
  TRY(zero_operand_like(A, P.BG, dBG, st));
  TRY(zero_operand_like(A, P.BF, dBF, st));
  TRY(zero_operand_like(A, P.AT2, dAT2, st));
  // gradients of the slot-compacted V-term blocks
  const int nS = (int)P.listBT.size(), nT = (int)P.listBF.size();
  const int64_t ns = (int64_t)nS * v, nt = (int64_t)nT * vt;
  double* dovss = nullptr;
  double* dovts = nullptr;
  TRY(zeros(A, &dovss, ns * ns, st));
  if (!P.mixed.trips.empty()) TRY(zeros(A, &dovts, nt * ns, st));
  double* dt2ss = s == 0 ? G.dt2aa : G.dt2bb;
  double* dt2st = G.dt2ab;
  if (s == 1 && !P.mixed.trips.empty()) TRY(zeros(A, &dt2st, (int64_t)o * ot * v * vt, st));

  // ---- per case: recompute, energy adjoint, contraction adjoint ------------
  for (int im = 0; im < 2; ++im) {
    const bool is_mixed = im == 1;
    CaseSel& cs = is_mixed ? P.mixed : P.same;
    const int ntrip = (int)cs.trips.size();
    if (ntrip == 0) continue;
    if (v == 0 || (is_mixed && vt == 0)) continue;
    const int M1 = v;
    const int64_t N1 = is_mixed ? (int64_t)v * vt : npairs(v);
    const int P1 = (int)round_up(std::max(M1, 1), 16);
    const int M2 = vt;
    const int64_t N2 = is_mixed ? npairs(v) : 0;
    const int P2 = (int)round_up(std::max(M2, 1), 16);
    const int64_t per = (N1 * P1 + N2 * P2) * 8 * 2;
    int Gn = (int)std::max<int64_t>(1, std::min<int64_t>(32, ((int64_t)4 << 30) / std::max<int64_t>(per, 1)));
    Gn = std::min(Gn, ntrip);
    double *X, *Z = nullptr, *dX, *dZ = nullptr;
    TRY(A.get(&X, (size_t)(Gn * N1 * P1) + 8));
    TRY(A.get(&dX, (size_t)(Gn * N1 * P1) + 8));
    if (is_mixed) {
      TRY(A.get(&Z, (size_t)(Gn * N2 * P2) + 8));
      TRY(A.get(&dZ, (size_t)(Gn * N2 * P2) + 8));
    }
    std::vector<int3> blocks;
    const int nbs = (v + 15) / 16, nbt = (vt + 15) / 16;
    for (int a = 0; a < nbs; ++a)
      for (int b = a; b < nbs; ++b)
        if (!is_mixed) {
          for (int c = b; c < nbs; ++c) blocks.push_back(make_int3(a, b, c));
        } else {
          for (int c = 0; c < nbt; ++c) blocks.push_back(make_int3(a, b, c));
        }
    int3* dblocks;
    TRY(A.get(&dblocks, blocks.size()));
    CU(cudaMemcpyAsync(dblocks, blocks.data(), blocks.size() * sizeof(int3),
                       cudaMemcpyHostToDevice, st));
    Trip* dtrips;
    TRY(A.get(&dtrips, (size_t)ntrip));
    CU(cudaMemcpyAsync(dtrips, cs.trips.data(), ntrip * sizeof(Trip), cudaMemcpyHostToDevice,
                       st));
    const int Pch = std::max(1, std::min((int)blocks.size(), R.ctx->nsm * 4 / Gn + 1));
    EnergyArgs ea{};
    ea.kind = is_mixed ? MIXED : SAME;
    ea.nvs = v;
    ea.nvt = is_mixed ? vt : v;
    ea.nos = o;
    ea.not_ = is_mixed ? ot : o;
    ea.eps_s = R.dom->eps[s];
    ea.eps_t = R.dom->eps[is_mixed ? t : s];
    ea.t1s = R.dom->t1[s];
    ea.t1t = R.dom->t1[is_mixed ? t : s];
    P.set_v_args(ea, is_mixed);
    ea.blocks = dblocks;
    ea.nblocks = (int)blocks.size();
    ea.pitch_x = P1;
    ea.pitch_z = P2;
    ea.x_stride = N1 * P1;
    ea.z_stride = N2 * P2;
    ProbF64* dpf;
    ProbF64* dpf2;
    GemmS* dgs;
    TRY(A.get(&dpf, (size_t)Gn));
    TRY(A.get(&dpf2, (size_t)Gn));
    TRY(A.get(&dgs, (size_t)Gn * 6));
    std::vector<ProbF64> pf(Gn), pf2(Gn);
    struct SegRef {
      const Operand* A;
      Operand* dA;
      int64_t arow;
      const Operand* B;
      Operand* dB;
      int64_t brow;
      double sign;
    };
    for (int g0 = 0; g0 < ntrip; g0 += Gn) {
      const int ng = std::min(Gn, ntrip - g0);
      std::vector<std::vector<SegRef>> segs1(ng), segs2(ng);
      for (int g = 0; g < ng; ++g) {
        const Trip tr = cs.trips[g0 + g];
        const int i = tr.i, j = tr.j, k = tr.k;
        if (!is_mixed) {
          const int64_t bp = npairs(v);
          segs1[g] = {{&P.AT, &dAT, (int64_t)P.slotAT[(size_t)j * o + k] * v, &P.BT, &dBT, P.slotBT[i] * bp, 1.0},
                      {&P.AT, &dAT, (int64_t)P.slotAT[(size_t)k * o + i] * v, &P.BT, &dBT, P.slotBT[j] * bp, 1.0},
                      {&P.AT, &dAT, (int64_t)P.slotAT[(size_t)i * o + j] * v, &P.BT, &dBT, P.slotBT[k] * bp, 1.0}};
        } else {
          const int K = k;
          const int64_t bp = npairs(v), bgr = (int64_t)v * vt;
          segs1[g] = {{&P.A1, &dA1, (int64_t)P.slotA1[(size_t)j * ot + K] * v, &P.BG, &dBG, P.slotBG[i] * bgr, 1.0},
                      {&P.A1, &dA1, (int64_t)P.slotA1[(size_t)i * ot + K] * v, &P.BG, &dBG, P.slotBG[j] * bgr, -1.0},
                      {&P.AT, &dAT, (int64_t)P.slotAT[(size_t)i * o + j] * v, &P.BF, &dBF, P.slotBF[K] * bgr, 1.0}};
          segs2[g] = {{&P.AT2, &dAT2, (int64_t)P.slotAT2[(size_t)j * ot + K] * vt, &P.BT, &dBT, P.slotBT[i] * bp, -1.0},
                      {&P.AT2, &dAT2, (int64_t)P.slotAT2[(size_t)i * ot + K] * vt, &P.BT, &dBT, P.slotBT[j] * bp, 1.0}};
        }
        auto fill = [&](ProbF64& pr, const std::vector<SegRef>& sg, double* out) {
          pr.nseg = (int)sg.size();
          for (size_t q = 0; q < sg.size(); ++q)
            pr.seg[q] = SegF64{sg[q].A->f64 + sg[q].arow * sg[q].A->Kp,
                               sg[q].B->f64 + sg[q].brow * sg[q].B->Kp, sg[q].A->K, sg[q].A->Kp,
                               sg[q].B->Kp, sg[q].sign};
          pr.XT = out;
        };
        fill(pf[g], segs1[g], X + (size_t)g * N1 * P1);
        if (is_mixed) fill(pf2[g], segs2[g], Z + (size_t)g * N2 * P2);
      }
      // recompute X (and Z')
      if (R.tc_adjoint) {
        // XT[n][m] = sum_seg sign A[arow+m][:] . B[brow+n][:], one tensor-core
        // product per segment, the later ones added
        auto recompute = [&](const std::vector<std::vector<SegRef>>& segs, double* Xb, int64_t Nn,
                             int Mm, int ldo) -> int {
          for (int g = 0; g < ng; ++g)
            for (size_t q = 0; q < segs[g].size(); ++q) {
              const SegRef& r = segs[g][q];
              TRY(tc_matmul(R, A, (int)Nn, Mm, r.A->K,
                            View{r.B->f64 + r.brow * r.B->Kp, r.B->Kp, 1},
                            View{r.A->f64 + r.arow * r.A->Kp, r.A->Kp, 1},
                            Xb + (size_t)g * Nn * ldo, ldo, r.sign, q > 0));
            }
          return LNO_OT_OK;
        };
        TRY(recompute(segs1, X, N1, M1, P1));
        if (is_mixed) TRY(recompute(segs2, Z, N2, M2, P2));
      } else {
        CU(cudaMemcpyAsync(dpf, pf.data(), ng * sizeof(ProbF64), cudaMemcpyHostToDevice, st));
        CU(launch_gemm_f64(dpf, ng, M1, (int)N1, P1, st));
        if (is_mixed) {
          CU(cudaMemcpyAsync(dpf2, pf2.data(), ng * sizeof(ProbF64), cudaMemcpyHostToDevice, st));
          CU(launch_gemm_f64(dpf2, ng, M2, (int)N2, P2, st));
        }
      }
      // energy adjoint -> dX, dT1, deps, V-integral gradients
      CU(cudaMemsetAsync(dX, 0, (size_t)ng * N1 * P1 * sizeof(double), st));
      if (is_mixed) CU(cudaMemsetAsync(dZ, 0, (size_t)ng * N2 * P2 * sizeof(double), st));
      ea.trips = dtrips + g0;
      cudaEvent_t ee0 = R.event(), ee1 = R.event();
      if (ee0) cudaEventRecord(ee0, st);
      CU(launch_energy_backward(ea, X, Z, dX, dZ, G.dt1[s], G.dt1[is_mixed ? t : s], dovss,
                                dovts, G.deps[s], G.deps[is_mixed ? t : s], gE, ng, Pch, st));
      if (ee1) cudaEventRecord(ee1, st);
      if (ee0 && ee1) R.energy_ev.push_back({ee0, ee1});
      if (R.fov[0]) {  // the f_ov part: planes are T2 amplitudes, coefficients f_ov
        EnergyArgs ef = ea;
        ef.vmode = 1;
        ef.t1s = R.fov[s];
        ef.t1t = R.fov[is_mixed ? t : s];
        ef.t2ss = P.t2ss;
        ef.t2st = P.t2st;
        CU(launch_energy_backward(ef, X, Z, dX, dZ, G.dfov[s], G.dfov[is_mixed ? t : s], dt2ss,
                                  dt2st, G.deps[s], G.deps[is_mixed ? t : s], gE, ng, Pch, st));
        R.stats->energy_launches += 1;
      }
      // contraction adjoint: dA += sign dX.B, dB += sign dX^T.A
      auto adj = [&](const std::vector<std::vector<SegRef>>& segs, const double* dXb, int64_t Nn,
                     int Mm, int ldo) -> int {
        if (R.tc_adjoint) {
          // dA[arow+m][k] += s sum_n dX[n][m] B[brow+n][k]
          // dB[brow+n][k] += s sum_m dX[n][m] A[arow+m][k]
          for (int g = 0; g < ng; ++g)
            for (const SegRef& r : segs[g]) {
              const double* dxg = dXb + (size_t)g * Nn * ldo;
              const int K = r.A->K;
              TRY(tc_matmul(R, A, Mm, K, (int)Nn, View{dxg, 1, ldo},
                            View{r.B->f64 + r.brow * r.B->Kp, 1, r.B->Kp},
                            r.dA->f64 + r.arow * r.A->Kp, r.A->Kp, r.sign, true));
              TRY(tc_matmul(R, A, (int)Nn, K, Mm, View{dxg, ldo, 1},
                            View{r.A->f64 + r.arow * r.A->Kp, 1, r.A->Kp},
                            r.dB->f64 + r.brow * r.B->Kp, r.B->Kp, r.sign, true));
            }
          return LNO_OT_OK;
        }
        for (int q = 0; q < 3; ++q) {  // one launch per segment position
          std::vector<GemmS> ga, gb;
          int maxKa = 0;
          for (int g = 0; g < ng; ++g) {
            if ((int)segs[g].size() <= q) continue;
            const SegRef& r = segs[g][q];
            const double* dxg = dXb + (size_t)g * Nn * ldo;
            const int K = r.A->K;
            maxKa = std::max(maxKa, K);
            ga.push_back(GemmS{dxg, r.B->f64 + r.brow * r.B->Kp, r.dA->f64 + r.arow * r.A->Kp,
                               Mm, K, (int)Nn, 1, 1, ldo, r.B->Kp, 1, r.A->Kp, 1, r.sign});
            gb.push_back(GemmS{dxg, r.A->f64 + r.arow * r.A->Kp, r.dB->f64 + r.brow * r.B->Kp,
                               (int)Nn, K, Mm, 1, ldo, 1, r.A->Kp, 1, r.B->Kp, 1, r.sign});
          }
          if (ga.empty()) continue;
          const int n = (int)ga.size();
          CU(cudaMemcpyAsync(dgs, ga.data(), n * sizeof(GemmS), cudaMemcpyHostToDevice, st));
          CU(launch_gemm_strided(dgs, n, Mm, maxKa, st));
          CU(cudaMemcpyAsync(dgs + Gn * 3, gb.data(), n * sizeof(GemmS), cudaMemcpyHostToDevice,
                             st));
          CU(launch_gemm_strided(dgs + Gn * 3, n, (int)Nn, maxKa, st));
          CU(cudaStreamSynchronize(st));
        }
        return LNO_OT_OK;
      };
      TRY(adj(segs1, dX, N1, M1, P1));
      if (is_mixed) TRY(adj(segs2, dZ, N2, M2, P2));
      CU(cudaStreamSynchronize(st));
      R.stats->contract_launches += is_mixed ? 2 : 1;
      R.stats->energy_launches += 1;
    }
  }

  // ---- layout adjoints and DF adjoints ---------------------------------------
  auto upload_pairs = [&](const std::vector<int2>& l, int2** d) -> int {
    TRY(A.get(d, std::max<size_t>(l.size(), 1)));
    if (!l.empty())
      CU(cudaMemcpyAsync(*d, l.data(), l.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    return LNO_OT_OK;
  };
  if (!P.listAT.empty()) {
    double* doovoT;
    TRY(zeros(A, &doovoT, (int64_t)o * v * o * o, st));
    int2* dl;
    TRY(upload_pairs(P.listAT, &dl));
    CU(launch_adj_at_same(dl, (int)P.listAT.size(), o, v, dAT.Kp, dAT.f64, dt2ss, doovoT, st));
    TRY(df_adjoint(R, A, R.Boo[s], G.dBoo[s], 0, o * o, R.Bov[s], G.dBov[s], 0, o * v, doovoT,
                   o * o));
    A.drop(doovoT);
  }
  if (!P.listBT.empty()) {
    double* dvv;
    TRY(A.get(&dvv, (size_t)v * v * v));
    for (size_t q = 0; q < P.listBT.size(); ++q) {
      const int x = P.listBT[q];
      CU(cudaMemsetAsync(dvv, 0, (size_t)v * v * v * sizeof(double), st));
      CU(launch_adj_bt_same((int)q, x, o, v, dBT.Kp, dBT.f64, dvv, dt2ss, st));
      TRY(df_adjoint(R, A, R.Bvv[s], G.dBvv[s], 0, v * v, R.Bov[s], G.dBov[s], (int64_t)x * v, v,
                     dvv, v * v));
    }
    A.drop(dvv);
  }
  if (!P.listA1.empty()) {
    double* djT;
    TRY(zeros(A, &djT, (int64_t)o * v * ot * ot, st));
    int2* dl;
    TRY(upload_pairs(P.listA1, &dl));
    CU(launch_adj_a1(dl, (int)P.listA1.size(), o, v, ot, vt, dA1.Kp, dA1.f64, dt2st, djT, st));
    TRY(df_adjoint(R, A, R.Bov[s], G.dBov[s], 0, o * v, R.Boo[t], G.dBoo[t], 0, ot * ot, djT,
                   o * v));
    A.drop(djT);
  }
  if (!P.listBG.empty()) {
    double* dgT;
    TRY(A.get(&dgT, (size_t)v * vt * vt));
    for (size_t q = 0; q < P.listBG.size(); ++q) {
      const int x = P.listBG[q];
      CU(cudaMemsetAsync(dgT, 0, (size_t)v * vt * vt * sizeof(double), st));
      CU(launch_adj_bg((int)q, x, o, v, ot, vt, dBG.Kp, dBG.f64, dgT, dt2st, st));
      TRY(df_adjoint(R, A, R.Bvv[t], G.dBvv[t], 0, vt * vt, R.Bov[s], G.dBov[s], (int64_t)x * v, v,
                     dgT, vt * vt));
    }
    A.drop(dgT);
  }
  if (!P.listBF.empty()) {
    double* dfT;
    TRY(A.get(&dfT, (size_t)vt * v * v));
    for (size_t q = 0; q < P.listBF.size(); ++q) {
      const int K = P.listBF[q];
      CU(cudaMemsetAsync(dfT, 0, (size_t)vt * v * v * sizeof(double), st));
      CU(launch_adj_bf((int)q, K, o, v, ot, vt, dBF.Kp, dBF.f64, dfT, dt2st, st));
      TRY(df_adjoint(R, A, R.Bvv[s], G.dBvv[s], 0, v * v, R.Bov[t], G.dBov[t], (int64_t)K * vt, vt,
                     dfT, v * v));
    }
    A.drop(dfT);
  }
  if (!P.listAT2.empty()) {
    double* dlT;
    TRY(zeros(A, &dlT, (int64_t)ot * vt * o * o, st));
    int2* dl;
    TRY(upload_pairs(P.listAT2, &dl));
    CU(launch_adj_at2(dl, (int)P.listAT2.size(), o, v, ot, vt, dAT2.Kp, dAT2.f64, dt2st, dlT, st));
    TRY(df_adjoint(R, A, R.Boo[s], G.dBoo[s], 0, o * o, R.Bov[t], G.dBov[t], 0, ot * vt, dlT,
                   o * o));
    A.drop(dlT);
  }
  // V-term blocks over the gathered rows, then added back into the Bov rows:
  // (ia|jb): L = R = BsS; (jb|KC): L = BsS rows (j,b), R = BsT rows (K,C)
  if (nS > 0) {
    Operand dBsS;
    TRY(zero_operand_like(A, P.BsS, dBsS, st));
    TRY(df_adjoint(R, A, P.BsS, dBsS, 0, (int)ns, P.BsS, dBsS, 0, (int)ns, dovss, (int)ns));
    if (dovts && nT > 0) {
      Operand dBsT;
      TRY(zero_operand_like(A, P.BsT, dBsT, st));
      TRY(df_adjoint(R, A, P.BsS, dBsS, 0, (int)ns, P.BsT, dBsT, 0, (int)nt, dovts, (int)ns));
      CU(launch_scatter_add_rows(dBsT.f64, G.dBov[t].f64, P.d_list_t, nT, (int64_t)vt * dBsT.Kp,
                                 st));
      R.stats->other_launches++;
    }
    CU(launch_scatter_add_rows(dBsS.f64, G.dBov[s].f64, P.d_list_s, nS, (int64_t)v * dBsS.Kp, st));
    R.stats->other_launches++;
  }
  if (s == 1 && !P.mixed.trips.empty())
    CU(launch_adj_transpose_t2ab(dt2st, ot, o, vt, v, G.dt2ab, st));
  CU(cudaStreamSynchronize(st));
  return LNO_OT_OK;
}

int backward_impl(lno_ot_ctx* ctx, const lno_ot_domain* dom, double gE, lno_ot_grad* g) {
  TRY(validate(ctx, dom));
  const int nbas = dom->nbas, naux = dom->naux;
  const int na = dom->nocc[0], nb = dom->nocc[1];
  const int va = nbas - na, vb = nbas - nb;
  const int64_t nB = (int64_t)naux * nbas * nbas;
  const int64_t n1[2] = {(int64_t)na * va, (int64_t)nb * vb};
  const int64_t naa = (int64_t)na * na * va * va, nbb = (int64_t)nb * nb * vb * vb,
                nab = (int64_t)na * nb * va * vb;
  for (int s = 0; s < 2; ++s) {
    TRY(check_ptr(ctx, g->dB[s], false));
    TRY(check_ptr(ctx, g->deps[s], false));
    TRY(check_ptr(ctx, g->dt1[s], false));
    TRY(check_ptr(ctx, g->dfov[s], false));
  }
  TRY(check_ptr(ctx, g->dt2aa, false));
  TRY(check_ptr(ctx, g->dt2bb, false));
  TRY(check_ptr(ctx, g->dt2ab, false));
  CU(cudaSetDevice(ctx->device));
  ctx->stats = lno_ot_stats{};
  ctx->ev_used = 0;
  Run R(ctx, dom);
  R.f64 = true;
  R.S = 0;
  // float64 operands and energy adjoint; with a tensor-core precision the
  // contractions (X recompute, contraction and DF adjoints) run on the tensor
  // cores through tc_matmul
  R.tc_adjoint = ctx->prec != LNO_OT_FP64;
  CU(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
  // wall-clock phases (the stream is synchronised at each boundary)
  using clk = std::chrono::steady_clock;
  const auto w0 = clk::now();
  double wbuild = 0.0;
  CaseSel cs[4];
  for (int c = 0; c < 4; ++c) TRY(select_case(dom, c, cs[c]));
  TRY(R.stage());
  CU(cudaStreamSynchronize(R.st));
  const double wstage = std::chrono::duration<double, std::milli>(clk::now() - w0).count();
  if (!R.fov[0] && (g->dfov[0] || g->dfov[1])) {
    // dE/df_ov at f_ov = 0 (E is affine in f_ov): run the f_ov pass on zeros
    for (int s = 0; s < 2; ++s) {
      double* z;
      TRY(zeros(R.arena, &z, n1[s], R.st));
      R.fov[s] = z;
    }
  }
  Arena GA(R.st, 0);
  GradAcc G{};
  for (int s = 0; s < 2; ++s) {
    TRY(zero_operand_like(GA, R.Boo[s], G.dBoo[s], R.st));
    TRY(zero_operand_like(GA, R.Bov[s], G.dBov[s], R.st));
    TRY(zero_operand_like(GA, R.Bvv[s], G.dBvv[s], R.st));
    TRY(zeros(GA, &G.dt1[s], n1[s], R.st));
    G.dfov[s] = nullptr;
    if (R.fov[0]) TRY(zeros(GA, &G.dfov[s], n1[s], R.st));
    TRY(zeros(GA, &G.deps[s], nbas, R.st));
  }
  // T2 gradients accumulate in the caller's buffers when given (projected in
  // place at the end), else in scratch
  auto acc_buf = [&](double* user, int64_t n, double** out) -> int {
    if (user) {
      CU(cudaMemsetAsync(user, 0, (size_t)std::max<int64_t>(n, 1) * sizeof(double), R.st));
      *out = user;
      return LNO_OT_OK;
    }
    return zeros(GA, out, n, R.st);
  };
  TRY(acc_buf(g->dt2aa, naa, &G.dt2aa));
  TRY(acc_buf(g->dt2bb, nbb, &G.dt2bb));
  TRY(acc_buf(g->dt2ab, nab, &G.dt2ab));
  double* e_dummy[4];
  for (int c = 0; c < 4; ++c)
    TRY(GA.get(&e_dummy[c], std::max<size_t>(cs[c].trips.size(), 1)));
  for (int s = 0; s < 2; ++s) {
    SpinPass P(R, s, s == 0 ? cs[0] : cs[3], s == 0 ? cs[1] : cs[2], e_dummy[s == 0 ? 0 : 3],
               e_dummy[s == 0 ? 1 : 2]);
    if (P.same.trips.empty() && P.mixed.trips.empty()) continue;
    const auto b0 = clk::now();
    P.plan();
    TRY(P.prepare_inputs());
    TRY(P.build_v_blocks());
    TRY(P.build());
    CU(cudaStreamSynchronize(R.st));
    wbuild += std::chrono::duration<double, std::milli>(clk::now() - b0).count();
    TRY(backward_spin(P, G, gE));
    CU(cudaStreamSynchronize(R.st));
  }
  // outputs: dB (symmetrised), deps, dt1, dt2 (antisymmetrised same-spin)
  for (int s = 0; s < 2; ++s) {
    const int o = dom->nocc[s], v = nbas - o;
    if (g->dB[s]) {  // raw gradient into the caller's buffer, symmetrised in place
      double* raw = g->dB[s];
      CU(cudaMemsetAsync(raw, 0, (size_t)nB * sizeof(double), R.st));
      CU(launch_adj_transpose_block(G.dBoo[s].f64, naux, nbas, 0, o, 0, o, G.dBoo[s].Kp, raw, R.st));
      CU(launch_adj_transpose_block(G.dBov[s].f64, naux, nbas, 0, o, o, v, G.dBov[s].Kp, raw, R.st));
      CU(launch_adj_transpose_block(G.dBvv[s].f64, naux, nbas, o, v, o, v, G.dBvv[s].Kp, raw, R.st));
      CU(launch_sym_inplace(raw, naux, nbas, R.st));
    }
    if (g->deps[s]) CU(launch_scale_copy(G.deps[s], nbas, 1.0, g->deps[s], R.st));
    if (g->dt1[s]) CU(launch_scale_copy(G.dt1[s], n1[s], 1.0, g->dt1[s], R.st));
    if (g->dfov[s]) CU(launch_scale_copy(G.dfov[s], n1[s], 1.0, g->dfov[s], R.st));
  }
  if (g->dt2aa) CU(launch_antisym_inplace(g->dt2aa, na, va, R.st));
  if (g->dt2bb) CU(launch_antisym_inplace(g->dt2bb, nb, vb, R.st));
  CU(cudaStreamSynchronize(R.st));
  int flag = 0;
  CU(cudaMemcpy(&flag, ctx->d_flag, sizeof flag, cudaMemcpyDeviceToHost));
  if (flag) return LNO_OT_ETIMEOUT;
  // stats of the adjoint: ms_total wall clock, ms_stage the staging plus the
  // operand and V-block builds (their DF assembly), ms_contract the event time
  // of its contractions (tensor-core products or float64 GEMMs), ms_energy the
  // energy adjoint kernels
  ctx->stats.ms_total = std::chrono::duration<double, std::milli>(clk::now() - w0).count();
  ctx->stats.ms_stage = wstage + wbuild;
  float ms = 0;
  double acc = 0;
  for (auto& p : R.contract_ev)
    if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) acc += ms;
  ctx->stats.ms_contract = acc;
  acc = 0;
  for (auto& p : R.energy_ev)
    if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) acc += ms;
  ctx->stats.ms_energy = acc;
  return LNO_OT_OK;
}

}  // namespace

// ============================================================================
extern "C" {

int lno_ot_init(lno_ot_ctx** ctx, const lno_ot_options* opt) {
  if (!ctx || !opt) return LNO_OT_EINVAL;
  if (opt->precision < 0 || opt->precision > LNO_OT_BF16X15) return LNO_OT_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return LNO_OT_ECUDA;
  }
  if (opt->device < 0 || opt->device >= ndev) return LNO_OT_EDEVICE;
  CU(cudaSetDevice(opt->device));
  cudaDeviceProp prop;
  CU(cudaGetDeviceProperties(&prop, opt->device));
  if (opt->precision != LNO_OT_FP64 && !(prop.major == 10 && prop.minor == 3))
    return LNO_OT_EUNSUPPORTED;  // the tensor-core path is built for sm_103a only
  lno_ot_ctx* c = new lno_ot_ctx();
  c->device = opt->device;
  c->prec = opt->precision;
  c->ws_limit = opt->workspace_bytes;
  c->nsm = prop.multiProcessorCount;
  if (opt->tune_cache && opt->tune_cache[0]) {  // "vmax bn group_cap" per line
    FILE* f = fopen(opt->tune_cache, "r");
    if (!f) {
      lno_ot_destroy(c);
      return LNO_OT_EINVAL;
    }
    char line[256];
    while (fgets(line, sizeof line, f)) {
      if (line[0] == '#') continue;
      lno_ot_ctx::TuneRow r;
      if (sscanf(line, "%d %d %d", &r.vmax, &r.bn, &r.group_cap) == 3 && r.vmax > 0)
        c->tune.push_back(r);
    }
    fclose(f);
    std::sort(c->tune.begin(), c->tune.end(),
              [](const lno_ot_ctx::TuneRow& a, const lno_ot_ctx::TuneRow& b) { return a.vmax < b.vmax; });
  }
  c->keep = opt->keep_operands != 0;
  // NULL = the legacy default stream (ordered with every blocking stream)
  c->stream = static_cast<cudaStream_t>(opt->stream);
  c->own_stream = false;
  // keep freed stream-ordered memory in the pool between calls
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (cudaMalloc(&c->d_flag, 256) != cudaSuccess || cudaMalloc(&c->d_amax, 256) != cudaSuccess ||
      cudaMalloc(&c->d_sums, 256) != cudaSuccess) {
    cudaGetLastError();
    lno_ot_destroy(c);
    return LNO_OT_ENOMEM;
  }
  *ctx = c;
  return LNO_OT_OK;
}

void lno_ot_destroy(lno_ot_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  destroy_cache(c->cache);
  c->cache = nullptr;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  cudaFree(c->d_flag);
  cudaFree(c->d_amax);
  cudaFree(c->d_sums);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

int lno_ot_energy(lno_ot_ctx* ctx, const lno_ot_domain* dom, lno_ot_result* out) {
  if (!ctx || !out) return LNO_OT_EINVAL;
  int rc = energy_impl(ctx, dom, out);
  out->status = rc;
  if (rc != LNO_OT_OK)
    for (double& e : out->e) e = 0.0;
  return rc;
}

int lno_ot_energy_batched(lno_ot_ctx* ctx, int ndom, const lno_ot_domain* doms,
                          lno_ot_result* out) {
  if (!ctx || ndom < 0 || (ndom > 0 && (!doms || !out))) return LNO_OT_EINVAL;
  int first = LNO_OT_OK;
  lno_ot_stats tot{};
  for (int d = 0; d < ndom; ++d) {
    int rc = lno_ot_energy(ctx, doms + d, out + d);
    if (rc != LNO_OT_OK && first == LNO_OT_OK) first = rc;
    const lno_ot_stats& s = ctx->stats;
    tot.ms_total += s.ms_total;
    tot.ms_stage += s.ms_stage;
    tot.ms_contract += s.ms_contract;
    tot.ms_energy += s.ms_energy;
    tot.flops_algorithmic += s.flops_algorithmic;
    tot.flops_executed += s.flops_executed;
    tot.tensor_flops += s.tensor_flops;
    tot.contract_launches += s.contract_launches;
    tot.energy_launches += s.energy_launches;
    tot.other_launches += s.other_launches;
    tot.triplets += s.triplets;
    tot.elements += s.elements;
  }
  ctx->stats = tot;
  return first;
}

int lno_ot_backward(lno_ot_ctx* ctx, const lno_ot_domain* dom, double gE, lno_ot_grad* g) {
  if (!ctx || !dom || !g) return LNO_OT_EINVAL;
  if (!std::isfinite(gE)) return LNO_OT_EINVAL;
  return backward_impl(ctx, dom, gE, g);
}

int lno_ot_energy_central(lno_ot_ctx* ctx, const lno_ot_domain* dom, const lno_ot_central* c) {
  if (!ctx) return LNO_OT_EINVAL;
  return central_impl(ctx, dom, c);
}

int lno_ot_naf(lno_ot_ctx* ctx, const lno_ot_domain* dom, double eps_naf, double* B_out[2],
               int* naux_out, double* eigenvalues) {
  if (!ctx) return LNO_OT_EINVAL;
  return naf_impl(ctx, dom, eps_naf, B_out, naux_out, eigenvalues);
}

int lno_ot_laplace_quadrature(double xmin, double xmax, double tol, int nmax, double* s,
                              double* w, int* nq) {
  return laplace_quadrature(xmin, xmax, tol, nmax, s, w, nq);
}

int lno_ot_release(lno_ot_ctx* ctx) {
  if (!ctx) return LNO_OT_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return LNO_OT_ECUDA;
  }
  destroy_cache(ctx->cache);
  ctx->cache = nullptr;
  CU(cudaStreamSynchronize(ctx->stream));
  return LNO_OT_OK;
}

int lno_ot_last_stats(const lno_ot_ctx* ctx, lno_ot_stats* st) {
  if (!ctx || !st) return LNO_OT_EINVAL;
  *st = ctx->stats;
  return LNO_OT_OK;
}

const char* lno_ot_strerror(int code) {
  switch (code) {
    case LNO_OT_OK: return "ok";
    case LNO_OT_EINVAL: return "invalid argument (sizes, null pointer, nocc[1] > nocc[0])";
    case LNO_OT_EDEVICE: return "pointer is not device memory of the context's device";
    case LNO_OT_ENOMEM: return "device workspace allocation failed";
    case LNO_OT_ECUDA: return "CUDA call failed";
    case LNO_OT_ETIMEOUT: return "bounded device wait gave up";
    case LNO_OT_EUNSUPPORTED: return "unsupported option or input";
    default: return "unknown status";
  }
}

const char* lno_ot_version(void) { return "lno_ot 0.1 sm_103a"; }

int lno_ot_selftest_gemm(int device, int S, int M, int N, int K, const double* A, const double* B,
                         double* Cout, void* stream) {
  if (S < 1 || S > 5 || M <= 0 || N <= 0 || K <= 0 || !A || !B || !Cout) return LNO_OT_EINVAL;
  CU(cudaSetDevice(device));
  cudaDeviceProp prop;
  CU(cudaGetDeviceProperties(&prop, device));
  if (!(prop.major == 10 && prop.minor == 3)) return LNO_OT_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Arena ar(st, 0);
  unsigned long long* amax;
  int* flag;
  TRY(ar.get(&amax, 2));
  TRY(ar.get(&flag, 1));
  CU(cudaMemsetAsync(amax, 0, 16, st));
  CU(cudaMemsetAsync(flag, 0, 4, st));
  CU(launch_absmax(A, (int64_t)M * K, amax, st));
  CU(launch_absmax(B, (int64_t)N * K, amax + 1, st));
  unsigned long long h[2];
  CU(cudaMemcpyAsync(h, amax, 16, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  double ma, mb;
  std::memcpy(&ma, &h[0], 8);
  std::memcpy(&mb, &h[1], 8);
  const double sa = pow2_scale(ma), sb = pow2_scale(mb);
  const int Kp = (int)round_up(K, 8);
  const int64_t na = round_up((int64_t)M * Kp, 8), nb = round_up((int64_t)N * Kp, 8);
  __nv_bfloat16 *a16, *b16;
  TRY(ar.get(&a16, (size_t)(na * S)));
  TRY(ar.get(&b16, (size_t)(nb * S)));
  // slice on the host (diagnostic path only; the product path slices on the GPU)
  std::vector<double> ha((size_t)M * K), hb((size_t)N * K);
  CU(cudaMemcpyAsync(ha.data(), A, ha.size() * 8, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(hb.data(), B, hb.size() * 8, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  std::vector<uint16_t> sa16((size_t)na * S, 0), sb16((size_t)nb * S, 0);
  auto host_slices = [&](const std::vector<double>& src, int rows, std::vector<uint16_t>& dst,
                         int64_t stride, double sc) {
    for (int r = 0; r < rows; ++r)
      for (int k = 0; k < K; ++k) {
        double x = src[(size_t)r * K + k] * (128.0 / sc), w = 1.0;
        for (int q = 0; q < S; ++q) {
          double v = std::nearbyint(x * w) / w;
          x -= v;
          float f = (float)v;  // exact: at most 8 significant bits
          uint32_t u;
          std::memcpy(&u, &f, 4);
          dst[(size_t)q * stride + (size_t)r * Kp + k] = (uint16_t)(u >> 16);
          w *= 256.0;
        }
      }
  };
  host_slices(ha, M, sa16, na, sa);
  host_slices(hb, N, sb16, nb, sb);
  CU(cudaMemcpyAsync(a16, sa16.data(), sa16.size() * 2, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(b16, sb16.data(), sb16.size() * 2, cudaMemcpyHostToDevice, st));
  CUtensorMap mA[2], mB[2];
  TRY(make_operand_map(&mA[0], a16, Kp, M, S, na, 128));
  TRY(make_operand_map(&mB[0], b16, Kp, N, S, nb, sliced_product_bn(S)));
  mA[1] = mA[0];
  mB[1] = mB[0];
  TcProb p{};
  p.nseg = 1;
  p.seg[0] = TcSeg{0, 0, 0, 0, K, 0};
  p.out = Cout;
  TcProb* dp;
  TRY(ar.get(&dp, 1));
  CU(cudaMemcpyAsync(dp, &p, sizeof p, cudaMemcpyHostToDevice, st));
  const double scale = sa * sb * std::ldexp(1.0, -14);
  CU(launch_sliced_product(S, mA, mB, dp, M, N, scale, flag, prop.multiProcessorCount, st,
                           tc_normal()));
  int hflag = 0;
  CU(cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return hflag ? LNO_OT_ETIMEOUT : LNO_OT_OK;
}

int lno_ot_selftest_timeout(int device, long long wait_cycles, int* code, void* stream) {
  if (wait_cycles < 1000 || wait_cycles > tc_default_wait_cycles()) return LNO_OT_EINVAL;
  if (code) *code = 0;
  CU(cudaSetDevice(device));
  cudaDeviceProp prop;
  CU(cudaGetDeviceProperties(&prop, device));
  if (!(prop.major == 10 && prop.minor == 3)) return LNO_OT_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // one 128 x 256 tile of a 2-slice product, K = 64: grid of one CTA
  constexpr int S = 2, M = 128, N = 256, K = 64;
  Arena ar(st, 0);
  int* flag;
  __nv_bfloat16 *a16, *b16;
  double* out;
  TcProb* dp;
  TRY(ar.get(&flag, 1));
  TRY(ar.get(&a16, (size_t)S * M * K));
  TRY(ar.get(&b16, (size_t)S * N * K));
  TRY(ar.get(&out, (size_t)M * N));
  TRY(ar.get(&dp, 1));
  CU(cudaMemsetAsync(flag, 0, 4, st));
  CU(cudaMemsetAsync(a16, 0, (size_t)S * M * K * 2, st));
  CU(cudaMemsetAsync(b16, 0, (size_t)S * N * K * 2, st));
  CUtensorMap mA[2], mB[2];
  TRY(make_operand_map(&mA[0], a16, K, M, S, (int64_t)M * K, 128));
  TRY(make_operand_map(&mB[0], b16, K, N, S, (int64_t)N * K, sliced_product_bn(S)));
  mA[1] = mA[0];
  mB[1] = mB[0];
  TcProb p{};
  p.nseg = 1;
  p.seg[0] = TcSeg{0, 0, 0, 0, K, 0};
  p.out = out;
  CU(cudaMemcpyAsync(dp, &p, sizeof p, cudaMemcpyHostToDevice, st));
  CU(launch_sliced_product(S, mA, mB, dp, M, N, 1.0, flag, 1, st, TcDiag{wait_cycles, 1}));
  int hflag = 0;
  CU(cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (code) *code = hflag;
  return hflag ? LNO_OT_ETIMEOUT : LNO_OT_OK;
}

int lno_ot_selftest_energy_timeout(int device, long long wait_cycles, int* code, void* stream) {
  if (wait_cycles < 1000 || wait_cycles > tc_default_wait_cycles()) return LNO_OT_EINVAL;
  if (code) *code = 0;
  CU(cudaSetDevice(device));
  cudaDeviceProp prop;
  CU(cudaGetDeviceProperties(&prop, device));
  if (!(prop.major == 10 && prop.minor == 3)) return LNO_OT_EUNSUPPORTED;
  int h = 0;
  CU(energy_timeout_selftest(wait_cycles, prop.multiProcessorCount, &h,
                             static_cast<cudaStream_t>(stream)));
  if (code) *code = h;
  return h ? LNO_OT_ETIMEOUT : LNO_OT_OK;
}

const char* lno_ot_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
