// Natural auxiliary functions of a domain (arXiv 2311.10048, Sec. 3.6, eq
// naf_w), in float64 on the CUDA cores:
//   1. J^s[X][(p<=q)] = B^X_pq (pair-packed factors of each spin);
//   2. W = (J^up J^up^T + J^down J^down^T) / 2, one grouped contraction;
//   3. eigenvectors of W by cyclic Jacobi rotations in the round-robin order
//      (n/2 disjoint rotations per round, n - 1 rounds per sweep; one sweep
//      is one CUDA graph of 3 (n - 1) launches, replayed until the
//      off-diagonal norm is below 1e-14 of the Frobenius norm);
//   4. the eigenvectors with eigenvalues above eps_naf, in descending order;
//   5. B'^s[X'][pq] = sum_X V[X][X'] B^s[X][pq] (one contraction per spin).
// The eigen-decomposition runs on the device; only the n eigenvalues and the
// convergence measure come back to the host (to sort and to stop).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace lno {

cudaError_t launch_gemm_f64(const ProbF64* probs_dev, int nprob, int M, int N, int ldo,
                            cudaStream_t st);

namespace {

inline int grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

// J[X][pair] = B[X][p][q] for p <= q (pair = q (q + 1) / 2 + p)
__global__ void pack_pairs(const double* __restrict__ B, int naux, int n,
                           double* __restrict__ J) {
  const int64_t np = (int64_t)n * (n + 1) / 2;
  const int64_t total = (int64_t)naux * np;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = idx % np;
    const int X = (int)(idx / np);
    int q = (int)((sqrt(8.0 * (double)pr + 1.0) - 1.0) * 0.5);
    while ((int64_t)q * (q + 1) / 2 > pr) --q;
    while ((int64_t)(q + 1) * (q + 2) / 2 <= pr) ++q;
    const int p = (int)(pr - (int64_t)q * (q + 1) / 2);
    J[idx] = B[((int64_t)X * n + p) * n + q];
  }
}

// Bt[pq][X] = B[X][pq]
__global__ void transpose_x(const double* __restrict__ B, int naux, int64_t n2,
                            double* __restrict__ Bt) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int X0 = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int X = X0 + yy;
    const int64_t r = r0 + threadIdx.x;
    tile[yy][threadIdx.x] = (X < naux && r < n2) ? B[(int64_t)X * n2 + r] : 0.0;
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t r = r0 + yy;
    const int X = X0 + threadIdx.x;
    if (r < n2 && X < naux) Bt[r * naux + X] = tile[threadIdx.x][yy];
  }
}

// Round-robin pair k of round r over m = np / 2 pairs of np (even) indices:
// pair 0 is (r, np - 1), pair k > 0 is ((r + k) mod (np-1), (r - k) mod (np-1)).
__device__ __forceinline__ void rr_pair(int r, int k, int np, int& p, int& q) {
  const int L = np - 1;
  if (k == 0) {
    p = r;
    q = L;
  } else {
    p = (r + k) % L;
    q = (r - k + L) % L;
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// rotation of pair k: zeroes A[p][q]; indices >= n are padding (no rotation)
__global__ void jac_angles(const double* __restrict__ A, int n, int np, int r,
                           double2* __restrict__ cs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np / 2) return;
  int p, q;
  rr_pair(r, k, np, p, q);
  double c = 1.0, s = 0.0;
  if (q < n) {
    const double apq = A[(int64_t)p * n + q];
    if (apq != 0.0) {
      const double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
      const double tau = (aqq - app) / (2.0 * apq);
      const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      c = 1.0 / sqrt(1.0 + t * t);
      s = t * c;
    }
  }
  cs[k] = make_double2(c, s);
}

// rows p, q of A (and nothing else): A <- J^T A for all pairs of the round
__global__ void jac_rows(double* __restrict__ A, int n, int np, int r,
                         const double2* __restrict__ cs) {
  const int m = np / 2;
  const int64_t total = (int64_t)m * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx % n), k = (int)(idx / n);
    int p, q;
    rr_pair(r, k, np, p, q);
    if (q >= n) continue;
    const double2 g = cs[k];
    const double ap = A[(int64_t)p * n + j], aq = A[(int64_t)q * n + j];
    A[(int64_t)p * n + j] = g.x * ap - g.y * aq;
    A[(int64_t)q * n + j] = g.y * ap + g.x * aq;
  }
}

// columns p, q of A and of V: A <- A J, V <- V J
__global__ void jac_cols(double* __restrict__ A, double* __restrict__ V, int n, int np, int r,
                         const double2* __restrict__ cs) {
  const int m = np / 2;
  const int64_t total = (int64_t)m * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), k = (int)(idx / n);
    int p, q;
    rr_pair(r, k, np, p, q);
    if (q >= n) continue;
    const double2 g = cs[k];
    double ap = A[(int64_t)i * n + p], aq = A[(int64_t)i * n + q];
    A[(int64_t)i * n + p] = g.x * ap - g.y * aq;
    A[(int64_t)i * n + q] = g.y * ap + g.x * aq;
    ap = V[(int64_t)i * n + p];
    aq = V[(int64_t)i * n + q];
    V[(int64_t)i * n + p] = g.x * ap - g.y * aq;
    V[(int64_t)i * n + q] = g.y * ap + g.x * aq;
  }
}

// out[0] = sum of squares of the off-diagonal elements, out[1] = of all
__global__ void jac_norms(const double* __restrict__ A, int n, double* __restrict__ out) {
  __shared__ double so[256], sa[256];
  double o = 0.0, a = 0.0;
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += blockDim.x) {
    const double x = A[idx];
    a += x * x;
    if (idx / n != idx % n) o += x * x;
  }
  so[threadIdx.x] = o;
  sa[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      so[threadIdx.x] += so[threadIdx.x + w];
      sa[threadIdx.x] += sa[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = so[0];
    out[1] = sa[0];
  }
}

__global__ void set_identity(double* __restrict__ V, int n) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * n;
       idx += (int64_t)gridDim.x * blockDim.x)
    V[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

__global__ void get_diag(const double* __restrict__ A, int n, double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    d[i] = A[(int64_t)i * n + i];
}

// Vt[c][X] = V[X][cols[c]]  (kept eigenvectors as rows)
__global__ void gather_cols(const double* __restrict__ V, int n, const int* __restrict__ cols,
                            int nk, double* __restrict__ Vt) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)nk * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int X = (int)(idx % n), c = (int)(idx / n);
    Vt[idx] = V[(int64_t)X * n + cols[c]];
  }
}

}  // namespace

// Symmetric eigen-decomposition of A (n x n, device, destroyed: its diagonal
// ends up holding the eigenvalues) with eigenvectors in the columns of V.
// Returns the number of sweeps, or a negative lno_ot_status.
int jacobi_eigh(double* A, double* V, int n, double2* cs, double* norms, cudaStream_t st,
                int max_sweeps) {
  if (n <= 0) return 0;
  set_identity<<<grid_n((int64_t)n * n), 256, 0, st>>>(V, n);
  if (n == 1) return 0;
  const int np = n + (n & 1);
  const int m = np / 2;
  // one sweep as a graph
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return LNO_OT_ECUDA;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = LNO_OT_OK;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    rc = LNO_OT_ECUDA;
  } else {
    for (int r = 0; r < np - 1; ++r) {
      jac_angles<<<(m + 127) / 128, 128, 0, cap>>>(A, n, np, r, cs);
      jac_rows<<<grid_n((int64_t)m * n), 256, 0, cap>>>(A, n, np, r, cs);
      jac_cols<<<grid_n((int64_t)m * n), 256, 0, cap>>>(A, V, n, np, r, cs);
    }
    if (cudaStreamEndCapture(cap, &graph) != cudaSuccess ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
      rc = LNO_OT_ECUDA;
  }
  int sweeps = 0;
  if (rc == LNO_OT_OK) {
    double h[2];
    for (; sweeps < max_sweeps; ++sweeps) {
      jac_norms<<<1, 256, 0, st>>>(A, n, norms);
      if (cudaMemcpyAsync(h, norms, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        rc = LNO_OT_ECUDA;
        break;
      }
      if (!(h[0] > 1e-28 * h[1])) break;   // off-diagonal norm < 1e-14 of the whole
      if (cudaGraphLaunch(exec, st) != cudaSuccess) {
        rc = LNO_OT_ECUDA;
        break;
      }
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  if (rc != LNO_OT_OK) {
    cudaGetLastError();
    return rc;
  }
  return sweeps;
}

cudaError_t launch_pack_pairs(const double* B, int naux, int n, double* J, cudaStream_t st) {
  pack_pairs<<<grid_n((int64_t)naux * n * (n + 1) / 2), 256, 0, st>>>(B, naux, n, J);
  return cudaGetLastError();
}

cudaError_t launch_transpose_x(const double* B, int naux, int64_t n2, double* Bt,
                               cudaStream_t st) {
  dim3 grid((unsigned)((n2 + 31) / 32), (unsigned)((naux + 31) / 32));
  transpose_x<<<grid, dim3(32, 8), 0, st>>>(B, naux, n2, Bt);
  return cudaGetLastError();
}

cudaError_t launch_get_diag(const double* A, int n, double* d, cudaStream_t st) {
  get_diag<<<grid_n(n), 256, 0, st>>>(A, n, d);
  return cudaGetLastError();
}

cudaError_t launch_gather_cols(const double* V, int n, const int* cols, int nk, double* Vt,
                               cudaStream_t st) {
  if (nk <= 0) return cudaSuccess;
  gather_cols<<<grid_n((int64_t)nk * n), 256, 0, st>>>(V, n, cols, nk, Vt);
  return cudaGetLastError();
}

}  // namespace lno
