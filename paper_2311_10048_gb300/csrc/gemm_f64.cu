// Plain float64 contractions on the CUDA cores (the FP64 comparator path).
//
// One launch evaluates a group of independent problems, each
//   XT[n][m] = sum_seg sign_seg * sum_{k < K_seg} A_seg[m][k] * B_seg[n][k]
// (both operands K-contiguous, output stored transposed so that the m index
// is contiguous).  This is the per-triplet W contraction of eq cim_pt_energy
// with the particle and hole sums of one occupied permutation concatenated
// along k, and also the DF assembly (pq|rs) = sum_Q B^Q_pq B^Q_rs.
#include "common.cuh"

namespace lno {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256)
gemm_f64_grouped(const ProbF64* __restrict__ probs, int M, int N, int ldo) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const ProbF64& P = probs[blockIdx.z];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x;
  const int tm = tid % 16, tn = tid / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  const int lr = tid / 4, lk = (tid % 4) * 4;  // loader: row, first k
  for (int s = 0; s < P.nseg; ++s) {
    const SegF64 sg = P.seg[s];
    for (int k0 = 0; k0 < sg.K; k0 += BK) {
      {
        const int m = m0 + lr;
        const double* src = sg.A + (int64_t)m * sg.lda + k0 + lk;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int k = k0 + lk + q;
          As[lk + q][lr] = (m < M && k < sg.K) ? sg.sign * src[q] : 0.0;
        }
        const int n = n0 + lr;
        const double* srb = sg.B + (int64_t)n * sg.ldb + k0 + lk;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int k = k0 + lk + q;
          Bs[lk + q][lr] = (n < N && k < sg.K) ? srb[q] : 0.0;
        }
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[kk][tm * 4 + a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tn * 4 + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int n = n0 + tn * 4 + b;
    if (n >= N) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int m = m0 + tm * 4 + a;
      if (m < M) P.XT[(int64_t)n * ldo + m] = acc[a][b];
    }
  }
}

}  // namespace

// probs: device array of nprob problems sharing M, N and the output pitch.
cudaError_t launch_gemm_f64(const ProbF64* probs_dev, int nprob, int M, int N,
                            int ldo, cudaStream_t st) {
  if (nprob <= 0 || M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid(ceil_div(N, BN), ceil_div(M, BM), nprob);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  gemm_f64_grouped<<<grid, 256, 0, st>>>(probs_dev, M, N, ldo);
  return cudaGetLastError();
}

}  // namespace lno
