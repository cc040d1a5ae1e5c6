// Internal helpers shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>

#include "lno_ot.h"

namespace lno {

// Spin-case kinds of one triplet group.
enum CaseKind { SAME = 0, MIXED = 1 };

// One K-segment of a per-triplet contraction in float64:
//   XT[n][m] += sign * sum_k A[m][k] * B[n][k],  k < K.
struct SegF64 {
  const double* A;  // row m at A + m * lda
  const double* B;  // row n at B + n * ldb
  int K;
  int lda, ldb;
  double sign;
};

constexpr int kMaxSeg = 3;

// Problem of a grouped float64 contraction: output XT [N][ldo] (column m < M).
struct ProbF64 {
  SegF64 seg[kMaxSeg];
  int nseg;
  double* XT;
};

// Triplet descriptor for the energy kernels.
struct Trip {
  int i, j, k;   // same spin: i<j<k; mixed: i<j (spin s), k = K (spin t)
};

// Energy-kernel arguments of one triplet group.
struct EnergyArgs {
  int kind;            // SAME or MIXED
  int nvs, nvt;        // virtual counts (same spin: nvt == nvs)
  int nos, not_;       // occupied counts
  const double* eps_s; // [nbas] orbital energies of spin s (occ then vir)
  const double* eps_t; // [nbas] spin t
  const double* t1s;   // [nos][nvs]
  const double* t1t;   // [not][nvt]
  // V-term integral blocks, stored only for the occupied orbitals the computed
  // triplets use (occupied index -> slot through oslot_s / oslot_t, -1 = absent):
  // (ia|jb) spin s-s as [slot i][a][slot j][b], i.e. [ns_c][nvs][ns_c][nvs]
  const double* ovov_ss;
  // mixed: (jb|KC) as [slot K][C][slot j][b], i.e. [nt_c][nvt][ns_c][nvs]
  const double* ovov_ts;
  const int* oslot_s;  // [nos]
  const int* oslot_t;  // [not] (same spin: equal to oslot_s)
  int ns_c, nt_c;      // number of slots
  // Source of V.  vmode 0: coefficients t1s/t1t, planes from the integral
  // blocks above, the kernels sum W (W + V) / D.  vmode 1 (the restricted
  // open-shell f_ov term): t1s/t1t point at the f_ov blocks, the planes are
  // the doubles amplitudes of the same indices, and the kernels sum W V / D.
  int vmode;
  const double* t2ss;  // [nos][nos][nvs][nvs] t^{xy}_{pr} (vmode 1)
  const double* t2st;  // [nos][not][nvs][nvt] t^{xC}_{pK} (vmode 1, mixed)
  const double* fs;    // [nos][nvs] f_ov of spin s (fused mixed pass only)
  const double* ft;    // [not][nvt] f_ov of spin t (fused mixed pass only)
  const int3* blocks;  // cube tiles (A,B,C) of 16-blocks
  int nblocks;
  int pitch_x;         // row pitch (elements) of XT / YT (same: a; mixed: a)
  int pitch_z;         // row pitch of ZT (mixed: C)
  int64_t x_stride;    // elements between consecutive triplets' XT (or YT)
  int64_t z_stride;    // between consecutive ZT
  const Trip* trips;   // [ntrip]
  double* partial;     // float64 path: [ntrip][gridDim.x]; float32 path: [ntrip][nchunk][8]
  // float32 path: the tiles of a triplet are split into nchunk items
  // (chunk c: tiles c, c + nchunk, ...); nitems = ntrip * nchunk items run on a
  // persistent grid of at most (resident CTAs per SM) * nsm CTAs
  int nchunk, nitems, nsm;
  int* flag;           // device error flag (bounded waits of the TMA-staged variant)
  // bounded-wait test hook of the TMA-staged variant: stage waits give up after
  // wait_cycles (0: the normal 4e9); starve = 1 issues no copy at all
  long long wait_cycles;
  int starve;
  // mixed spin: Y and Z' stored as 16^3 tiles (kOutYTile / kOutZTile, strides
  // in floats per triplet above); selects the TMA-staged kernel
  int tiled;
  // Laplace form (Sec. 3.7, eq laplace_transform): with lap_w != 0 the
  // kernels weight each element by -lap_w exp(lap_s D) instead of 1/D (one
  // quadrature point of 1/D = -sum_q w_q exp(s_q D), D < 0)
  double lap_s, lap_w;
};

// (px|ry) of spin s in the slot-compacted [ns][nvs][ns][nvs] block
__device__ __forceinline__ int64_t ovss_idx(const EnergyArgs& a, int p, int x, int r, int y) {
  return (((int64_t)a.oslot_s[p] * a.nvs + x) * a.ns_c + a.oslot_s[r]) * a.nvs + y;
}
// (px|KC) with p of spin s, K of spin t: [nt][nvt][ns][nvs]
__device__ __forceinline__ int64_t ovts_idx(const EnergyArgs& a, int K, int C, int p, int x) {
  return (((int64_t)a.oslot_t[K] * a.nvt + C) * a.ns_c + a.oslot_s[p]) * a.nvs + x;
}

// Inputs of the orbital partition: per-case triplets and contributions.
struct OrbPartArgs {
  const double* e[4];   // per-triplet contributions of cases aaa, aab, abb, bbb
  const Trip* trips[4];
  int64_t n[4];
  int na, nb;
  double* out[2];       // [na], [nb] (either may be NULL)
  // 0: the prefactors of eq cim_pt_energy (mixed triplet 1/4, 1/4, 1/2);
  // 1: eq local_pt's 1/3 of every triplet to each of its orbitals
  int thirds;
};

// V plane on two spin-s virtuals: vmode 0 <pr||xy> = (px|ry) - (py|rx),
// vmode 1 t^{xy}_{pr}
__device__ __forceinline__ double vplane_ss(const EnergyArgs& a, int p, int x, int r, int y) {
  if (a.vmode) return a.t2ss[(((int64_t)p * a.nos + r) * a.nvs + x) * a.nvs + y];
  return a.ovov_ss[ovss_idx(a, p, x, r, y)] - a.ovov_ss[ovss_idx(a, p, y, r, x)];
}
// V plane on a spin-s and a spin-t virtual: vmode 0 (px|KC), vmode 1 t^{xC}_{pK}
__device__ __forceinline__ double vplane_ts(const EnergyArgs& a, int K, int C, int p, int x) {
  if (a.vmode) return a.t2st[(((int64_t)p * a.not_ + K) * a.nvs + x) * a.nvt + C];
  return a.ovov_ts[ovts_idx(a, K, C, p, x)];
}

// Tensor-core contraction problem: up to kMaxSeg K-segments, each a row block
// of a sliced operand tensor addressed through a TMA map (index 0 or 1).
struct TcSeg {
  int amap, bmap;   // tensor map index (0/1) for A and B
  int a_row, b_row; // first row of the A / B operand block in its tensor
  int K;            // contraction length (k < K is real data)
  int neg;          // 1: subtract this segment
};

// TcProb.flags: kTcAccum adds the result to out instead of storing it;
// kTcFloatRest forms the float64 result as HI + the float32 sum of the lower
// weight classes, scaled in float32 (the scale must be a power of two): two
// float64 operations per element instead of six, ~2^-32 relative instead of
// the exact class sums (used by the adjoint's products)
constexpr int kTcAccum = 1, kTcFloatRest = 2;

struct TcProb {
  TcSeg seg[kMaxSeg];
  int nseg;
  int flags;        // float64 transposed output only: kTcAccum, kTcFloatRest
  void* out;        // output of this problem: [N][ldo] (transposed) or [M][ldo] (row-major)
};

// Output layout of a row-major (RM) float32 contraction launch.
//   kOutRows:  out[m][n], pitch ldo.
//   kOutYTile: mixed-spin Y, rows m = b nvt + C, columns a, stored as 16^3
//              tiles (b/16, C/16, a/16), tile index (B nbt + C') nbs + A; in a
//              tile, row r = (b%16) 16 + C%16 holds 16 floats of a with its four
//              16-byte chunks permuted (chunk ^ ((r >> 1) & 3)).
//   kOutZTile: mixed-spin Z', rows m = pair(a, b) (a < b), columns C, stored as
//              tiles (a/16 <= b/16, C/16), tile index (B(B+1)/2 + A) nbt + C';
//              row r = (a%16) 16 + b%16 sits at row r ^ ((r >> 1) & 1) of the
//              tile.
// The energy kernel reads each 16^3 sub-cube of the tiled layouts with one
// 16 KB bulk copy, in the shared-memory layout its element loops index.
constexpr int kOutRows = 0, kOutYTile = 1, kOutZTile = 2;
struct TcOut {
  int mode;
  int nvt;    // kOutYTile: C count per b
  int nbs;    // 16-blocks of a (and b)
  int nbt;    // 16-blocks of C
};
constexpr int kTile = 4096;   // floats of one 16^3 tile

// Bounded-wait settings of one contraction launch: wait_cycles limits every
// wait for work; starve = 1 is the timeout test hook (no copy is issued, so
// the first wait for data runs out).  Library calls use tc_normal().
struct TcDiag {
  long long wait_cycles;
  int starve;
  // mixed spin: Y and Z' stored as 16^3 tiles (kOutYTile / kOutZTile, strides
  // in floats per triplet above); selects the TMA-staged kernel
  int tiled;
};

// tc_gemm.cu: grouped sliced contraction.  mA: maps with 128-row boxes,
// mB: maps with BN-row boxes; instances (S, BN, OutT, TF, RM) are listed there
// (RM: row-major output out[m][n], else the transposed out[n][m]).
template <int S, int BN, typename OutT, bool TF = false, bool RM = false>
cudaError_t launch_tc_gemm(const CUtensorMap* mA, const CUtensorMap* mB, const TcProb* probs_dev,
                           int nprob, int M, int N, int ldo, double scale, int* flag,
                           unsigned long long* amax, int nsm, cudaStream_t st, TcDiag diag,
                           TcOut lay = TcOut{kOutRows, 0, 0, 0});
long long tc_default_wait_cycles();
inline TcDiag tc_normal() { return TcDiag{tc_default_wait_cycles(), 0}; }
int make_operand_map(CUtensorMap* map, const void* base, int64_t Kp, int64_t rows, int S,
                     int64_t slice_stride, int box_rows, int esz = 2);
int sliced_product_bn(int S);
cudaError_t launch_sliced_product(int S, const CUtensorMap* mA, const CUtensorMap* mB,
                                  const TcProb* dp, int M, int N, double scale, int* flag,
                                  int nsm, cudaStream_t st, TcDiag dg);

// Augmented domain of the central-LMO pass (central.cu): P pseudo-orbitals
// appended after the occupied orbitals of spin `spin`, for quadrature point s.
struct AugmentArgs {
  int spin, P, nbas, naux, nocc[2];
  double s;
  const double* U;        // [P][nocc[spin]] LMO coefficients
  const double* B_in;     // [naux][nbas][nbas] of `spin`
  const double* eps_in;   // [nbas]
  const double* t1_in;    // [nocc][nvir]
  const double* fov_in;   // [nocc][nvir] or NULL
  const double* t2ss_in;  // same-spin doubles of `spin`
  const double* t2ab_in;  // [na][nb][va][vb]
  double* coef;           // [P][nocc[spin]]
  double *B_out, *eps_out, *t1_out, *fov_out, *t2ss_out, *t2ab_out;
};
cudaError_t launch_lmo_augment(const AugmentArgs& A, cudaStream_t st);
int laplace_quadrature(double xmin, double xmax, double tol, int nmax, double* s, double* w,
                       int* nq);

// Operand stores used by the layout kernels.  `part` says whether the value
// is an amplitude (0) or an integral (1): the two have separate scales.
struct StoreF64 {
  double* p;
  __device__ __forceinline__ void operator()(int64_t idx, double v, int) const { p[idx] = v; }
};

// Exact BF16 slices: value = scale 2^-7 (s_0 + ... + s_{S-1}), s_0 an integer
// in [-128,128], s_q a multiple of 2^(-8q) with |s_q| <= 2^(-8q+7), every
// step rounded to nearest (ties to even) in float64.
template <int S>
struct StoreSlices {
  __nv_bfloat16* p;
  int64_t slice_stride;  // elements between slices
  double inv_t;          // 2^7 / amplitude scale
  double inv_i;          // 2^7 / integral scale
  __device__ __forceinline__ void operator()(int64_t idx, double v, int part) const {
    double x = v * (part ? inv_i : inv_t);
    double w = 1.0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      double q = rint(x * w) / w;   // w = 2^(8s): exact scaling
      x -= q;                        // exact
      p[s * slice_stride + idx] = __double2bfloat16(q);
      w *= 256.0;
    }
  }
};

// Exact TF32 slices (stored as float): value = scale 2^-10 (s_0 + ... +
// s_{S-1}), s_0 an integer in [-1024, 1024], s_q a multiple of 2^(-11q): 11
// significant bits each, what one TF32 operand holds.
template <int S>
struct StoreTF32 {
  float* p;
  int64_t slice_stride;
  double inv_t;          // 2^10 / amplitude scale
  double inv_i;          // 2^10 / integral scale
  __device__ __forceinline__ void operator()(int64_t idx, double v, int part) const {
    double x = v * (part ? inv_i : inv_t);
    double w = 1.0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      double q = rint(x * w) / w;   // w = 2^(11s): exact scaling
      x -= q;
      p[s * slice_stride + idx] = (float)q;
      w *= 2048.0;
    }
  }
};

__host__ __device__ inline int64_t pair_index(int p, int q) {  // p < q
  return (int64_t)q * (q - 1) / 2 + p;
}
__host__ __device__ inline int64_t npairs(int n) { return (int64_t)n * (n - 1) / 2; }

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace lno

#define LNO_CUDA_TRY(expr)                                                   \
  do {                                                                       \
    cudaError_t e__ = (expr);                                                \
    if (e__ != cudaSuccess) {                                                \
      lno_set_last_error(#expr, e__, __FILE__, __LINE__);                    \
      return LNO_OT_ECUDA;                                                   \
    }                                                                        \
  } while (0)

void lno_set_last_error(const char* what, cudaError_t e, const char* file, int line);
