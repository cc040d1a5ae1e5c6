// Tensor-core contraction for sm_103a: tcgen05.mma (BF16 x BF16 -> FP32 in
// TMEM) fed by TMA, on exactly sliced float64 operands.
//
// Each float64 operand value is stored as S BF16 slices with a power-of-two
// scale sigma (StoreSlices in common.cuh):
//     x = sigma 2^-7 (s_0 + s_1 + ... + s_{S-1}),
// s_0 an integer in [-128,128], s_1 a multiple of 2^-8 in [-1/2,1/2], ...
// For C[m][n] = sum_k A[m][k] B[n][k] the kernel issues, per 16-wide k step,
// the slice products (p,q) with p + q <= S-1 and accumulates each weight
// class g = p + q in its own TMEM accumulator.  Every term of class g is an
// integer multiple of 2^(-8g) no larger than 2^(14-8g), so each class sum is
// exact (no rounding at all) while it needs at most 24 significant bits:
// always for k <= 1024, and for random-sign data far beyond.  (Measured on sm_103a: a single FP32
// accumulator shared by classes of different weight drifts by ~2^-17 of its
// value over a few hundred MMAs, because each MMA rounds the running sum at
// its own magnitude.)  The epilogue adds the classes from the smallest up in
// float32 (the lower classes are ~2^-8 of the next, so this is one rounding
// of the final sum) and scales by the power of two sigma_A sigma_B 2^-14.
// Float64 output (the DF assembly) adds the exact class sums in float64.  No float64
// arithmetic runs per element: this GPU's FP64 rate is ~1/64 of FP32.  No
// systematic bias enters the sum of ~1e12 positive-definite energy terms.
//
// A problem is XT[n][m] = sum_seg (+/-) A_seg[m][:] . B_seg[n][:]: up to 3
// K-segments from different operand tensors (the three occupied
// permutations of P(i/jk), or the mixed-spin terms); the sign is applied with
// the instruction descriptor's negate-A bit.  Operand tensors are 3-D TMA
// maps (k, row, slice); k beyond the tensor and rows beyond the last row
// arrive as zeros.
//
// Kernel structure (one CTA per SM, persistent over tiles of 128 x BN):
//   warp 0      TMA producer (one thread), STAGES-deep smem ring
//   warp 1      TMEM allocator and MMA issuer (one thread); S accumulators
//               of 128 x BN FP32 (S * BN <= 512 TMEM columns: BN = 256 or 128
//               for S = 2, 128 or 64 for S = 3, 128, 96 or 64 for S = 4, and 64
//               for S = 5)
//   warps 2..5  epilogue: tcgen05.ld -> scale -> coalesced stores along m; when
//               TMEM has room ((S + 1) BN <= 512) the combined tile is parked in
//               spare columns so the next tile's MMAs overlap the stores
// Tiles are visited m fastest: the CTAs that run at the same time share the
// B tile of one n-tile (read from HBM once, the other m-tiles hit L2), and the
// small A operand of a problem stays resident in L2.
// Every mbarrier wait is bounded; on a timeout the kernel records an error
// code, drains its own TMA copies and MMAs, frees TMEM and returns.
#include "common.cuh"
#include "ptx.cuh"

namespace lno {

namespace {

constexpr int BM = 128;
constexpr int BK = 32;                     // BF16 elements per 64-byte row, SWIZZLE_64B
constexpr long long kWaitCycles = 4000000000LL;
constexpr int kSmemBudget = 227 * 1024;

// Wait for phase `parity` of `bar`; false if another role raised the error
// flag (abortable) or `limit` cycles passed (then records `code`).  Waits for
// work use the launch's limit; the drain waits before TMEM and shared memory
// are released always use the long kWaitCycles.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* flag, int code,
                                       bool abortable, long long limit = kWaitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0) {
      if (abortable && *(volatile int*)flag != 0) return false;
      if (clock64() - t0 > limit) {
        atomicCAS(flag, 0, code);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

// The same MMAs with a collector-buffer usage for A: consecutive MMAs that
// share one A operand (slice pa against the slices pb of B) read it from shared
// memory once (fill), then from the collector (use, lastuse).
#define LNO_UMMA_C(NAME, KIND, COLL)                                                        \
  __device__ __forceinline__ void NAME(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,     \
                                       uint32_t idesc, uint32_t accum) {                    \
    asm volatile("{\n\t.reg .pred p;\n\t"                                                   \
                 "setp.ne.b32 p, %4, 0;\n\t"                                               \
                 "tcgen05.mma.cta_group::1.kind::" KIND ".collector::a::" COLL                \
                 " [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),                                 \
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)                             \
                 : "memory");                                                               \
  }
LNO_UMMA_C(umma_bf16_fill, "f16", "fill")
LNO_UMMA_C(umma_bf16_use, "f16", "use")
LNO_UMMA_C(umma_bf16_last, "f16", "lastuse")
LNO_UMMA_C(umma_tf32_fill, "tf32", "fill")
LNO_UMMA_C(umma_tf32_use, "tf32", "use")
LNO_UMMA_C(umma_tf32_last, "tf32", "lastuse")
#undef LNO_UMMA_C

// mode 0: no collector, 1: fill, 2: use, 3: last use
template <bool TF>
__device__ __forceinline__ void umma_any(int mode, uint32_t d, uint64_t a, uint64_t b,
                                         uint32_t id, uint32_t acc) {
  if constexpr (TF) {
    if (mode == 1) umma_tf32_fill(d, a, b, id, acc);
    else if (mode == 2) umma_tf32_use(d, a, b, id, acc);
    else if (mode == 3) umma_tf32_last(d, a, b, id, acc);
    else umma_tf32(d, a, b, id, acc);
  } else {
    if (mode == 1) umma_bf16_fill(d, a, b, id, acc);
    else if (mode == 2) umma_bf16_use(d, a, b, id, acc);
    else if (mode == 3) umma_bf16_last(d, a, b, id, acc);
    else umma_bf16(d, a, b, id, acc);
  }
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32"
      " [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, rows of 64 B in
// groups of 8 (stride 512 B between groups).
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused when swizzled)
  d |= (uint64_t)(512 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
  d |= (uint64_t)4 << 61;            // SWIZZLE_64B
  return d;
}

// Instruction descriptor: D FP32, A/B K-major of format 1 (BF16, kind::f16)
// or 2 (TF32, kind::tf32), M=128, N=n (a multiple of 16, 16..256).
template <bool TF>
__device__ __forceinline__ uint32_t idesc_mma(int neg, int n) {
  constexpr uint32_t fmt = TF ? 2u : 1u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)neg << 13) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// 16 consecutive floats of one output row; `left` columns remain in the row
// (the rest of the 16 are not written).  16-byte aligned when left >= 16.
__device__ __forceinline__ void store_row16(float* p, const uint32_t (&v)[16], int left) {
  if (left >= 16) {
    float4* p4 = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      p4[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                          __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < left) p[j] = __uint_as_float(v[j]);
  }
}

// One 16-float row chunk (columns n0 .. n0+15 of output row m) of a
// row-major launch, in the launch's output layout; `left` = columns remaining
// in the row (only those are written).
__device__ __forceinline__ void store_out16(float* out, const TcOut& lay, int ldo, int m, int n0,
                                            const uint32_t (&v)[16], int left) {
  if (lay.mode == kOutRows) {
    store_row16(out + (int64_t)m * ldo + n0, v, left);
  } else if (lay.mode == kOutYTile) {
    const int b = m / lay.nvt, c = m - b * lay.nvt;
    const int r = ((b & 15) << 4) | (c & 15), sw = (r >> 1) & 3;
    float* row = out + ((int64_t)((b >> 4) * lay.nbt + (c >> 4)) * lay.nbs + (n0 >> 4)) * kTile +
                 r * 16;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float* d = row + ((q ^ sw) << 2);
      if (left >= 4 * q + 4) {
        *reinterpret_cast<float4*>(d) =
            make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                        __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * q + j < left) d[j] = __uint_as_float(v[4 * q + j]);
      }
    }
  } else {   // kOutZTile: m = pair(a, b) = b (b - 1) / 2 + a
    int b = (int)((1.0 + sqrt(1.0 + 8.0 * (double)m)) * 0.5);
    while ((int64_t)b * (b - 1) / 2 > m) --b;
    while ((int64_t)(b + 1) * b / 2 <= m) ++b;
    const int a = m - (int)((int64_t)b * (b - 1) / 2);
    const int A = a >> 4, B = b >> 4;
    const int r = ((a & 15) << 4) | (b & 15), slot = r ^ ((r >> 1) & 1);
    store_row16(out + ((int64_t)(B * (B + 1) / 2 + A) * lay.nbt + (n0 >> 4)) * kTile + slot * 16,
                v, left);
  }
}

template <int S, int BN>
struct Cfg {
  static constexpr int kABytes = BM * BK * 2;          // one slice of A
  static constexpr int kBBytes = BN * BK * 2;          // one slice of B
  static constexpr int kStage = S * (kABytes + kBBytes);
  static constexpr int kStages = (kSmemBudget - 2048) / kStage;
  static constexpr int kSmem = kStages * kStage + 1024 + 256;
  static_assert(kStages >= 2, "pipeline needs two stages");
  static_assert(S * BN <= 512, "one TMEM accumulator per weight class");
};

// One CTA per SM, persistent over the (problem, n-tile, m-tile) units.
// `diag` is the bounded-wait test hook: wait_cycles limits every wait for work
// (kWaitCycles in normal launches); starve = 1 makes the producer issue no copy
// at all, so the MMA thread's first wait (on a full barrier nothing will
// complete) runs out after wait_cycles and the kernel takes its error exit
// with nothing in flight.  Library calls always pass {kWaitCycles, 0}.
// TF: TF32 slices (32-bit elements, 16 per 64-byte row, K 8 per MMA) instead
// of BF16 ones (32 per row, K 16 per MMA); the shared-memory layout, the
// descriptors and the MMAs per row are the same in bytes.
// RM: row-major output out[m][n] (pitch ldo), n-tiles fastest; otherwise the
// transposed out[n][m], m-tiles fastest.  The last n-tile's MMAs are only as
// wide as its columns (rounded up to 16), so a narrow n costs little.
template <int S, int BN, typename OutT, bool TF, bool RM>
__global__ void __launch_bounds__(192, 1)
tc_gemm_sliced(const __grid_constant__ CUtensorMap mapA0, const __grid_constant__ CUtensorMap mapA1,
               const __grid_constant__ CUtensorMap mapB0, const __grid_constant__ CUtensorMap mapB1,
               const TcProb* __restrict__ probs, int nprob, int M, int N, int ldo, double scale,
               int* __restrict__ flag, unsigned long long* __restrict__ amax, TcDiag diag,
               TcOut lay) {
  using C = Cfg<S, BN>;
  constexpr int BKE = TF ? BK / 2 : BK;   // elements per 64-byte row
  constexpr int KM = TF ? 8 : 16;         // K of one MMA
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kStages * C::kStage);
  // bars[0..st): full, [st..2st): empty, [2st]: tmem_full, [2st+1]: tmem_empty, [2st+2]: drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * C::kStages + 3);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nM = (M + BM - 1) / BM, nN = (N + BN - 1) / BN;
  const long long nunits = (long long)nprob * nM * nN;
  const long long wlim = diag.wait_cycles;
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + C::kStages + s); };
  const uint32_t tfull = smem_u32(bars + 2 * C::kStages);
  const uint32_t tempty = smem_u32(bars + 2 * C::kStages + 1);
  const uint32_t drain = smem_u32(bars + 2 * C::kStages + 2);
  auto a_addr = [&](int st, int sl) { return smem_u32(smem + st * C::kStage + sl * C::kABytes); };
  auto b_addr = [&](int st, int sl) {
    return smem_u32(smem + st * C::kStage + S * C::kABytes + sl * C::kBBytes);
  };
  // unit -> (problem, m-tile, n-tile): m fastest (transposed output: the
  // concurrent CTAs share one n-tile of B), n fastest for RM (they share one
  // m-tile of A)
  auto decode = [&](long long u, int& mt, int& nt, long long& pr) {
    if constexpr (RM) {
      nt = (int)(u % nN);
      const long long r = u / nN;
      mt = (int)(r % nM);
      pr = r / nM;
    } else {
      mt = (int)(u % nM);
      const long long r = u / nM;
      nt = (int)(r % nN);
      pr = r / nN;
    }
  };
  // MMA width of n-tile nt: its columns rounded up to 16
  auto ntile_w = [&](int nt) { return min(BN, (N - nt * BN + 15) & ~15); };

  if (warp == 0 && lane == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 128);
    mbar_init(drain, 1);
    mbar_init_fence();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------ producer -------------------------------
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, last_phase = 0;
      bool ok = diag.starve == 0;
      for (long long u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int mt, nt;
        long long pr;
        decode(u, mt, nt, pr);
        const TcProb& P = probs[pr];
        for (int sg = 0; sg < P.nseg && ok; ++sg) {
          const TcSeg seg = P.seg[sg];
          const CUtensorMap* ma = seg.amap ? &mapA1 : &mapA0;
          const CUtensorMap* mb = seg.bmap ? &mapB1 : &mapB0;
          for (int k0 = 0; k0 < seg.K; k0 += BKE) {
            if (!mbar_wait(empty_bar(stage), phase ^ 1u, flag, 1, true, wlim)) {
              ok = false;
              break;
            }
            mbar_expect_tx(full_bar(stage), (uint32_t)C::kStage);
#pragma unroll
            for (int sl = 0; sl < S; ++sl)
              tma_load_3d(a_addr(stage, sl), ma, full_bar(stage), k0, seg.a_row + mt * BM, sl);
#pragma unroll
            for (int sl = 0; sl < S; ++sl)
              tma_load_3d(b_addr(stage, sl), mb, full_bar(stage), k0, seg.b_row + nt * BN, sl);
            issued_mask |= 1u << stage;
            last_phase = (last_phase & ~(1u << stage)) | (phase << stage);
            if (++stage == C::kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      // every copy this thread issued must have landed before smem goes away
      for (int s = 0; s < C::kStages; ++s)
        if (issued_mask & (1u << s)) mbar_wait(full_bar(s), (last_phase >> s) & 1u, flag, 4, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // -------------------------------- MMA ----------------------------------
      int stage = 0;
      uint32_t phase = 0, tile_it = 0;
      bool ok = true, any = false;
      for (long long u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++tile_it) {
        int mt, nt;
        long long pr;
        decode(u, mt, nt, pr);
        const TcProb& P = probs[pr];
        if (tile_it > 0 && !mbar_wait(tempty, (tile_it - 1) & 1u, flag, 2, true, wlim)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t cls_on = 0;  // bit g: accumulator of class g already written
        const int nw = ntile_w(nt);
        for (int sg = 0; sg < P.nseg && ok; ++sg) {
          const TcSeg seg = P.seg[sg];
          const uint32_t idesc = idesc_mma<TF>(seg.neg, nw);
          for (int k0 = 0; k0 < seg.K; k0 += BKE) {
            if (!mbar_wait(full_bar(stage), phase, flag, 3, true, wlim)) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {   // two 32-byte MMA steps per 64-byte row
              if (k0 + ks * KM < seg.K) {
#pragma unroll
                for (int pa = 0; pa < S; ++pa) {
                  const uint64_t ad = sdesc_sw64(a_addr(stage, pa) + ks * 32);
#pragma unroll
                  for (int pb = 0; pb + pa < S; ++pb) {
                    const uint64_t bd = sdesc_sw64(b_addr(stage, pb) + ks * 32);
                    const int g = pa + pb;
                    // A slice pa meets S - pa slices of B in a row: read it once
                    const int last = S - 1 - pa;
                    const int mode = last == 0 ? 0 : pb == 0 ? 1 : pb == last ? 3 : 2;
                    umma_any<TF>(mode, tmem + g * BN, ad, bd, idesc, (cls_on >> g) & 1u);
                    cls_on |= 1u << g;
                    any = true;
                  }
                }
              }
            }
            umma_commit(empty_bar(stage));
            if (++stage == C::kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (ok) umma_commit(tfull);
      }
      if (!ok && any) {  // drain this thread's MMAs before TMEM is released
        umma_commit(drain);
        mbar_wait(drain, 0, flag, 5, false);
      }
    }
  } else {
    // ------------------------------- epilogue ---------------------------------
    const int q = warp & 3;
    const int row = q * 32 + lane;
    uint32_t tile_it = 0;
    float lmax = 0.f;
    // scale = sigma_A sigma_B 2^-14 is a power of two: exact in float
    const float fscale = (float)scale;
    for (long long u = blockIdx.x; u < nunits; u += gridDim.x, ++tile_it) {
      int mt, nt;
      long long pr;
      decode(u, mt, nt, pr);
      const TcProb& P = probs[pr];
      if (!mbar_wait(tfull, tile_it & 1u, flag, 6, true, wlim)) break;
      tc_fence_after();
      const int m = mt * BM + row;
      OutT* out = reinterpret_cast<OutT*>(P.out);
      const bool mok = m < M && out != nullptr;
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16);
      if constexpr ((S + 1) * BN <= 512 && sizeof(OutT) == 4) {
        // combine the classes into the spare TMEM columns, free the class
        // accumulators for the next tile's MMAs, then store from the spare copy
        const uint32_t spare = tbase + S * BN;
        const int nch = ntile_w(nt) / 16;
#pragma unroll 1
        for (int c = 0; c < nch; ++c) {
          uint32_t acc[S][16];
#pragma unroll
          for (int g = 0; g < S; ++g) tmem_ld16(tbase + g * BN + c * 16, acc[g]);
          tmem_ld_wait();
          uint32_t v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float lo = 0.f;
#pragma unroll
            for (int g = S - 1; g >= 1; --g) lo = __fadd_rn(lo, __uint_as_float(acc[g][j]));
            v[j] = __float_as_uint(__fmul_rn(__fadd_rn(__uint_as_float(acc[0][j]), lo), fscale));
          }
          tmem_st16(spare + c * 16, v);
        }
        tmem_st_wait();
        tc_fence_before();
        mbar_arrive(tempty);
#pragma unroll 1
        for (int c = 0; c < nch; ++c) {
          uint32_t v[16];
          tmem_ld16(spare + c * 16, v);
          tmem_ld_wait();
          const int n0 = nt * BN + c * 16;
          if constexpr (RM) {
            if (mok) store_out16(reinterpret_cast<float*>(out), lay, ldo, m, n0, v, N - n0);
          } else {
            OutT* op = out + (int64_t)n0 * ldo + m;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float x = __uint_as_float(v[j]);
              if (mok && n0 + j < N) op[(int64_t)j * ldo] = x;
              if (amax != nullptr && m < M && n0 + j < N) lmax = fmaxf(lmax, fabsf(x));
            }
          }
        }
      } else if constexpr (RM && BN <= 128) {
        // the class accumulators fill TMEM: combine the whole row into
        // registers, free TMEM for the next tile's MMAs, then store
        static_assert(sizeof(OutT) == 4, "row-major output is float32");
        const int nch = ntile_w(nt) / 16;
        uint32_t v[BN];
#pragma unroll
        for (int c = 0; c < BN / 16; ++c) {
          if (c < nch) {
            uint32_t acc[S][16];
#pragma unroll
            for (int g = 0; g < S; ++g) tmem_ld16(tbase + g * BN + c * 16, acc[g]);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float lo = 0.f;
#pragma unroll
              for (int g = S - 1; g >= 1; --g) lo = __fadd_rn(lo, __uint_as_float(acc[g][j]));
              v[c * 16 + j] =
                  __float_as_uint(__fmul_rn(__fadd_rn(__uint_as_float(acc[0][j]), lo), fscale));
            }
          }
        }
        tc_fence_before();
        mbar_arrive(tempty);
        if (mok) {
#pragma unroll
          for (int c = 0; c < BN / 16; ++c) {
            if (c < nch) {
              uint32_t w[16];
#pragma unroll
              for (int j = 0; j < 16; ++j) w[j] = v[c * 16 + j];
              const int n0 = nt * BN + c * 16;
              store_out16(reinterpret_cast<float*>(out), lay, ldo, m, n0, w, N - n0);
            }
          }
        }
      } else {
        const int nch = ntile_w(nt) / 16;
#pragma unroll 1
        for (int c = 0; c < nch; ++c) {
          uint32_t acc[S][16];
#pragma unroll
          for (int g = 0; g < S; ++g) tmem_ld16(tbase + g * BN + c * 16, acc[g]);
          tmem_ld_wait();
          const int n0 = nt * BN + c * 16;
          if constexpr (RM) {
            static_assert(sizeof(OutT) == 4, "row-major output is float32");
            uint32_t v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float lo = 0.f;
#pragma unroll
              for (int g = S - 1; g >= 1; --g) lo = __fadd_rn(lo, __uint_as_float(acc[g][j]));
              v[j] = __float_as_uint(__fmul_rn(__fadd_rn(__uint_as_float(acc[0][j]), lo), fscale));
            }
            if (mok) store_out16(reinterpret_cast<float*>(out), lay, ldo, m, n0, v, N - n0);
            continue;
          }
          OutT* op = out + (int64_t)n0 * ldo + m;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            // lower classes first (each exact), then one rounding against HI
            float lo = 0.f;
#pragma unroll
            for (int g = S - 1; g >= 1; --g) lo = __fadd_rn(lo, __uint_as_float(acc[g][j]));
            const float hi = __uint_as_float(acc[0][j]);
            if constexpr (sizeof(OutT) == 4) {
              const float v = __fmul_rn(__fadd_rn(hi, lo), fscale);
              if (mok && n0 + j < N) op[(int64_t)j * ldo] = v;
              if (amax != nullptr && m < M && n0 + j < N) lmax = fmaxf(lmax, fabsf(v));
            } else {
              // float64 output: the exact class sums added in float64 (smallest
              // first), so the output keeps ~53 bits instead of HI + a float32 rest
              if (mok && n0 + j < N) {
                double r;
                if (P.flags & kTcFloatRest) {
                  r = (double)__fmul_rn(hi, fscale) + (double)__fmul_rn(lo, fscale);
                } else {
                  double v = 0.0;
#pragma unroll
                  for (int g = S - 1; g >= 1; --g) v += (double)__uint_as_float(acc[g][j]);
                  r = ((double)hi + v) * scale;
                }
                double* o = &op[(int64_t)j * ldo];
                *o = (P.flags & kTcAccum) ? *o + r : r;
              }
              if (amax != nullptr && m < M && n0 + j < N)
                lmax = fmaxf(lmax, fabsf(__fmul_rn(__fadd_rn(hi, lo), fscale)));
            }
          }
        }
        tc_fence_before();
        mbar_arrive(tempty);
      }
    }
    if (amax != nullptr)
      atomicMax(amax, (unsigned long long)__double_as_longlong((double)lmax));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
  }
}

}  // namespace

// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3-D map over a sliced operand tensor: (k < Kp, row < rows, slice < S) of
// esz-byte elements (2: BF16, 4: TF32 values stored as float).
// Box: one 64-byte row of k x box_rows rows x 1 slice, 64-byte swizzle, zero fill.
int make_operand_map(CUtensorMap* map, const void* base, int64_t Kp, int64_t rows, int S,
                     int64_t slice_stride, int box_rows, int esz) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return LNO_OT_ECUDA;
  if ((esz != 2 && esz != 4) || Kp % 8 || slice_stride % 8 ||
      (reinterpret_cast<uintptr_t>(base) & 15))
    return LNO_OT_EINVAL;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)S};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * esz), (cuuint64_t)(slice_stride * esz)};
  cuuint32_t box[3] = {(cuuint32_t)(64 / esz), (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(map, esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   3, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? LNO_OT_OK : LNO_OT_ECUDA;
}

// mB must be maps with boxes of BN rows; mA boxes of 128 rows.
template <int S, int BN, typename OutT, bool TF, bool RM>
cudaError_t launch_tc_gemm(const CUtensorMap* mA, const CUtensorMap* mB, const TcProb* probs_dev,
                           int nprob, int M, int N, int ldo, double scale, int* flag,
                           unsigned long long* amax, int nsm, cudaStream_t st, TcDiag diag,
                           TcOut lay) {
  using C = Cfg<S, BN>;
  if (nprob <= 0 || M <= 0 || N <= 0) return cudaSuccess;
  if (RM && lay.mode == kOutRows && (ldo % 4 != 0 || ldo < ((N + 15) & ~15)))
    return cudaErrorInvalidValue;
  if (lay.mode != kOutRows &&
      (!RM || lay.nbs < 1 || lay.nbt < 1 || (lay.mode == kOutYTile && lay.nvt < 1)))
    return cudaErrorInvalidValue;
  auto k = tc_gemm_sliced<S, BN, OutT, TF, RM>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  if (e != cudaSuccess) return e;
  const long long ntiles = (long long)nprob * ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  const int grid = (int)(ntiles < nsm ? ntiles : nsm);
  k<<<grid, 192, C::kSmem, st>>>(mA[0], mA[1], mB[0], mB[1], probs_dev, nprob, M, N, ldo, scale,
                                 flag, amax, diag, lay);
  return cudaGetLastError();
}

int tc_products(int S) { return S * (S + 1) / 2; }

// Tile width of the single-product diagnostics for S slices.
int sliced_product_bn(int S) { return S <= 2 ? 256 : S <= 4 ? 128 : 64; }

// One plain product C[n][m] = sum_k A[m][k] B[n][k] (float64 output) on
// sliced operands already in device memory; mB boxes of sliced_product_bn(S) rows.
cudaError_t launch_sliced_product(int S, const CUtensorMap* mA, const CUtensorMap* mB,
                                  const TcProb* dp, int M, int N, double scale, int* flag,
                                  int nsm, cudaStream_t st, TcDiag dg) {
  switch (S) {
    case 1: return launch_tc_gemm<1, 256, double, false, false>(mA, mB, dp, 1, M, N, M, scale, flag, nullptr, nsm, st, dg);
    case 2: return launch_tc_gemm<2, 256, double, false, false>(mA, mB, dp, 1, M, N, M, scale, flag, nullptr, nsm, st, dg);
    case 3: return launch_tc_gemm<3, 128, double, false, false>(mA, mB, dp, 1, M, N, M, scale, flag, nullptr, nsm, st, dg);
    case 4: return launch_tc_gemm<4, 128, double, false, false>(mA, mB, dp, 1, M, N, M, scale, flag, nullptr, nsm, st, dg);
    case 5: return launch_tc_gemm<5, 64, double, false, false>(mA, mB, dp, 1, M, N, M, scale, flag, nullptr, nsm, st, dg);
    default: return cudaErrorInvalidValue;
  }
}
long long tc_default_wait_cycles() { return kWaitCycles; }

#define LNO_TC_INST(S, BN, T, TF, RM)                                                        \
  template cudaError_t launch_tc_gemm<S, BN, T, TF, RM>(                                     \
      const CUtensorMap*, const CUtensorMap*, const TcProb*, int, int, int, int, double, int*, \
      unsigned long long*, int, cudaStream_t, TcDiag, TcOut);
// W contractions (float32 row-major output): slices x tile width
LNO_TC_INST(2, 256, float, false, true)
LNO_TC_INST(2, 128, float, false, true)
LNO_TC_INST(3, 128, float, false, true)
LNO_TC_INST(3, 64, float, false, true)
LNO_TC_INST(4, 128, float, false, true)
LNO_TC_INST(4, 96, float, false, true)
LNO_TC_INST(4, 64, float, false, true)
LNO_TC_INST(5, 64, float, false, true)
// TF32 W contractions (2 TF32 slices, 3 products)
LNO_TC_INST(2, 256, float, true, true)
LNO_TC_INST(2, 128, float, true, true)
// DF assembly and the diagnostics (float64 transposed output)
LNO_TC_INST(1, 256, double, false, false)
LNO_TC_INST(2, 256, double, false, false)
LNO_TC_INST(3, 128, double, false, false)
LNO_TC_INST(4, 128, double, false, false)
LNO_TC_INST(5, 64, double, false, false)
#undef LNO_TC_INST

}  // namespace lno
