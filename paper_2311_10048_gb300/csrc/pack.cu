// Layout kernels: DF factor blocks and the K-concatenated operands of the
// per-triplet W contractions (eq cim_pt_energy, connected triples).
//
// Same spin s (o occupied, v virtual, Kx = v + o):
//   AT[p][q][a][kk] = t^{ae}_{pq}            (kk = e < v)
//                   = <ma||qp> = H_qp[m][a]  (kk = v + m), H_xy[m][a] = (mx|ay)-(my|ax)
//   BT[x][(b<c)][kk] = <ex||bc> = (eb|xc)-(ec|xb)   (kk = e)
//                    = t^{bc}_{xm}                   (kk = v + m)
//   X_{ijk}[a,(bc)] = AT[j][k].BT[i] + AT[k][i].BT[j] + AT[i][j].BT[k]
//   (= P(i/jk) of the particle and hole terms; the signs are absorbed by
//   t^{ae}_{pq} = -t^{ae}_{qp} and H_qp = -H_pq).
// Mixed (i<j spin s, K spin t):
//   A1[p][K][a][kk]  = -t^{aE}_{pK} (kk=E<vt),  (pa|MK) (kk = vt+M)
//   BG[x][(b,C)][kk] = (xb|EC)      (kk=E),     t^{bC}_{xM} (kk = vt+M)
//   BF[K][(b,C)][kk] = (be|KC)      (kk=e<vs),  -t^{bC}_{mK} (kk = vs+m)
//   AT2[p][K][C][kk] = t^{eC}_{pK}  (kk=e),     (mp|CK) (kk = vs+m)
//   Y[a,(bC)]   = A1[j][K].BG[i] - A1[i][K].BG[j] + AT[i][j].BF[K]
//   Z'[C,(a<b)] = -AT2[j][K].BT[i] + AT2[i][K].BT[j]
// Rows are padded with zeros to a pitch Kp (multiple of 8).
// Occupied indices come in two ranges: the summed (internal) m, M run over the
// first oi (oti) orbitals, the external ones over all o (ot) the arrays hold.
// The two differ only when pseudo-orbitals (the central LMOs of the Laplace
// form, Sec. 3.7) are appended after the real occupied orbitals; the DF
// blocks with one internal occupied index are laid out [internal][external].
//
// Every pack kernel is templated on its store: float64, or the exact
// BF16 slices of the tensor-core path (value = scale 2^-7 (s1 + s2 + s3),
// s1 an integer in [-128, 128], s2 a multiple of 2^-8 in [-1/2, 1/2], ...,
// each step rounded to nearest).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace lno {

namespace {

// B[s] [naux][nbas][nbas] -> out[p'][q'][Q] = B[Q][p0+p'][q0+q'] (p' < np, q' < nq)
template <class St>
__global__ void transpose_block(const double* __restrict__ B, int naux, int nbas, int p0, int np,
                                int q0, int nq, int Qp, St st) {
  __shared__ double tile[32][33];
  const int64_t nrows = (int64_t)np * nq;
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int Q0 = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int Q = Q0 + yy;
    const int64_t r = r0 + threadIdx.x;
    double v = 0.0;
    if (Q < naux && r < nrows) {
      const int p = (int)(r / nq), q = (int)(r % nq);
      v = B[((int64_t)Q * nbas + p0 + p) * nbas + q0 + q];
    }
    tile[yy][threadIdx.x] = v;
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t r = r0 + yy;
    const int Q = Q0 + threadIdx.x;
    if (r < nrows && Q < Qp) st(r * Qp + Q, Q < naux ? tile[threadIdx.x][yy] : 0.0, 1);
  }
}

// AT[slot][a][kk] for same-spin pair (p,q) = pairs[slot]
template <class St>
__global__ void pack_at_same(const int2* __restrict__ pairs, int nslot, int o, int oi, int v,
                             int Kp, const double* __restrict__ t2ss,
                             const double* __restrict__ oovoT, St st) {
  const int64_t total = (int64_t)nslot * v * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const int64_t r = idx / Kp;
    const int a = (int)(r % v);
    const int slot = (int)(r / v);
    const int2 pq = pairs[slot];
    double val = 0.0;
    if (kk < v) {
      val = t2ss[(((int64_t)pq.x * o + pq.y) * v + a) * v + kk];
    } else if (kk < v + oi) {
      const int m = kk - v;
      const int64_t oo = (int64_t)oi * o;
      // H_qp[m][a] = (mq|ap) - (mp|aq);  oovoT[(y*v+a)][(m*o+x)] = (mx|ya)
      val = oovoT[((int64_t)pq.x * v + a) * oo + m * o + pq.y] -
            oovoT[((int64_t)pq.y * v + a) * oo + m * o + pq.x];
    }
    st(idx, val, kk >= v);
  }
}

// BT[slot][pair(b<c)][kk] for occupied x; vvovT[c][(e*v+b)] = (eb|xc)
template <class St>
__global__ void pack_bt_same(int slot, int x, int o, int oi, int v, int Kp,
                             const double* __restrict__ vvovT, const double* __restrict__ t2ss,
                             St st) {
  const int64_t np = npairs(v);
  const int64_t total = np * Kp;
  const int64_t base = (int64_t)slot * np * Kp;
  const int64_t vv = (int64_t)v * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const int64_t pr = idx / Kp;
    // decode pair index pr = c(c-1)/2 + b
    int c = (int)((1.0 + sqrt(1.0 + 8.0 * (double)pr)) * 0.5);
    while ((int64_t)c * (c - 1) / 2 > pr) --c;
    while ((int64_t)(c + 1) * c / 2 <= pr) ++c;
    const int b = (int)(pr - (int64_t)c * (c - 1) / 2);
    double val = 0.0;
    if (kk < v) {
      val = vvovT[(int64_t)c * vv + (int64_t)kk * v + b] - vvovT[(int64_t)b * vv + (int64_t)kk * v + c];
    } else if (kk < v + oi) {
      const int m = kk - v;
      val = t2ss[(((int64_t)x * o + m) * v + b) * v + c];
    }
    st(base + idx, val, kk < v);
  }
}

// A1[slot][a][kk] for mixed pair (p,K) = pk[slot]; jT[(M*ot+K)][(p*vs+a)] = (pa|MK)
template <class St>
__global__ void pack_a1(const int2* __restrict__ pk, int nslot, int os, int vs, int ot, int oti,
                        int vt, int Kp, const double* __restrict__ t2st,
                        const double* __restrict__ jT, St st) {
  const int64_t total = (int64_t)nslot * vs * Kp;
  const int64_t ld = (int64_t)os * vs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const int64_t r = idx / Kp;
    const int a = (int)(r % vs);
    const int2 p = pk[r / vs];
    double val = 0.0;
    if (kk < vt) {
      val = -t2st[(((int64_t)p.x * ot + p.y) * vs + a) * vt + kk];
    } else if (kk < vt + oti) {
      const int M = kk - vt;
      val = jT[((int64_t)M * ot + p.y) * ld + (int64_t)p.x * vs + a];
    }
    st(idx, val, kk >= vt);
  }
}

// BG[slot][(b*vt+C)][kk] for occupied x (spin s); gT[b][(E*vt+C)] = (xb|EC)
template <class St>
__global__ void pack_bg(int slot, int x, int os, int vs, int ot, int oti, int vt, int Kp,
                        const double* __restrict__ gT, const double* __restrict__ t2st, St st) {
  const int64_t rows = (int64_t)vs * vt;
  const int64_t total = rows * Kp;
  const int64_t base = (int64_t)slot * total;
  const int64_t vv = (int64_t)vt * vt;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const int64_t r = idx / Kp;
    const int b = (int)(r / vt), C = (int)(r % vt);
    double val = 0.0;
    if (kk < vt) {
      val = gT[(int64_t)b * vv + (int64_t)kk * vt + C];
    } else if (kk < vt + oti) {
      const int M = kk - vt;
      val = t2st[(((int64_t)x * ot + M) * vs + b) * vt + C];
    }
    st(base + idx, val, kk < vt);
  }
}

// BF[slot][(b*vt+C)][kk] for occupied K (spin t); fT[C][(b*vs+e)] = (be|KC)
template <class St>
__global__ void pack_bf(int slot, int K, int os, int osi, int vs, int ot, int vt, int Kp,
                        const double* __restrict__ fT, const double* __restrict__ t2st, St st) {
  const int64_t rows = (int64_t)vs * vt;
  const int64_t total = rows * Kp;
  const int64_t base = (int64_t)slot * total;
  const int64_t vv = (int64_t)vs * vs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const int64_t r = idx / Kp;
    const int b = (int)(r / vt), C = (int)(r % vt);
    double val = 0.0;
    if (kk < vs) {
      val = fT[(int64_t)C * vv + (int64_t)b * vs + kk];
    } else if (kk < vs + osi) {
      const int m = kk - vs;
      val = -t2st[(((int64_t)m * ot + K) * vs + b) * vt + C];
    }
    st(base + idx, val, kk < vs);
  }
}

// AT2[slot][C][kk] for (p,K) = pk[slot]; lT[(K*vt+C)][(m*os+p)] = (mp|KC)
template <class St>
__global__ void pack_at2(const int2* __restrict__ pk, int nslot, int os, int osi, int vs, int ot,
                         int vt, int Kp, const double* __restrict__ t2st,
                         const double* __restrict__ lT, St st) {
  const int64_t total = (int64_t)nslot * vt * Kp;
  const int64_t ld = (int64_t)osi * os;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const int64_t r = idx / Kp;
    const int C = (int)(r % vt);
    const int2 p = pk[r / vt];
    double val = 0.0;
    if (kk < vs) {
      val = t2st[(((int64_t)p.x * ot + p.y) * vs + kk) * vt + C];
    } else if (kk < vs + osi) {
      const int m = kk - vs;
      val = lT[((int64_t)p.y * vt + C) * ld + (int64_t)m * os + p.x];
    }
    st(idx, val, kk >= vs);
  }
}

// t2ba[I][k][A][c] = t2ab[k][I][c][A]
__global__ void transpose_t2ab(const double* __restrict__ t2ab, int na, int nb, int va, int vb,
                               double* __restrict__ out) {
  const int64_t total = (int64_t)na * nb * va * vb;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    // out index (I, k, A, c)
    int c = (int)(idx % va);
    int64_t r = idx / va;
    int A = (int)(r % vb);
    r /= vb;
    int k = (int)(r % na);
    int I = (int)(r / na);
    out[idx] = t2ab[(((int64_t)k * nb + I) * va + c) * vb + A];
  }
}

// Strided float64 views for the tensor-core adjoint: element (r, k) of a
// rows x K view sits at in[r rs + k ks].  Work goes in 32 x 32 tiles whose
// loads run along the view's unit-stride index (k when ks == 1, else r), so
// they coalesce either way.
__device__ __forceinline__ double view_at(const double* in, int64_t rs, int64_t ks, int rows,
                                          int K, int r, int k) {
  return (r < rows && k < K) ? in[(int64_t)r * rs + (int64_t)k * ks] : 0.0;
}

// max |x| over the view (bits of a non-negative double, atomicMax into *out)
__global__ void view_absmax(const double* __restrict__ in, int64_t rs, int64_t ks, int rows,
                            int K, unsigned long long* __restrict__ out) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool rfast = ks != 1 && rs == 1;
  double m = 0.0;
  for (int r0 = blockIdx.y * 32; r0 < rows; r0 += gridDim.y * 32) {
    const int k0 = blockIdx.x * 32;
    for (int i = ty; i < 32; i += 8) {
      const double x = rfast ? view_at(in, rs, ks, rows, K, r0 + tx, k0 + i)
                             : view_at(in, rs, ks, rows, K, r0 + i, k0 + tx);
      m = fmax(m, fabs(x));
    }
  }
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((tx & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// round(v 2^e2) to nearest (ties to even) from the bits of v, in integer
// arithmetic (this GPU's float64 rate is 1/64 of its float32 rate); |v 2^e2|
// must stay below 2^62, v finite.
__device__ __forceinline__ int64_t round_scaled(double v, int e2) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  uint64_t m = b & ((1ull << 52) - 1);
  if (ex != 0) m |= 1ull << 52;
  const int sh = (ex == 0 ? 1 : ex) - 1075 + e2;   // |v| 2^e2 = m 2^sh
  uint64_t q;
  if (m == 0) {
    q = 0;
  } else if (sh >= 0) {
    q = m << sh;
  } else if (-sh > 54) {
    q = 0;                                        // m 2^sh < 1/2
  } else {
    const int r = -sh;
    const uint64_t rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
    q = m >> r;
    if (rem > half || (rem == half && (q & 1))) ++q;
  }
  return (b >> 63) ? -(int64_t)q : (int64_t)q;
}

// The same exact slices as StoreSlices, from one rounding of the scaled value
// to S * 8 - 1 fractional bits followed by integer digit extraction (base 256,
// each digit rounded half up, so |s_0| <= 128 and |s_q 2^(8q)| <= 128):
// value = 2^-e7 (s_0 + ... + s_{S-1}), e7 = e2 - 8 (S - 1), e2 passed in.
template <int S>
struct StoreSlicesInt {
  __nv_bfloat16* p;
  int64_t slice_stride;
  int e2;   // log2(2^7 / scale) + 8 (S - 1)
  __device__ __forceinline__ void operator()(int64_t idx, double v) const {
    int64_t R = round_scaled(v, e2);
#pragma unroll
    for (int q = 0; q < S; ++q) {
      const int sh = 8 * (S - 1 - q);
      const int64_t d = sh ? (R + (1ll << (sh - 1))) >> sh : R;
      R -= d << sh;
      p[q * slice_stride + idx] = __float2bfloat16_rn(ldexpf((float)d, -8 * q));
    }
  }
};

// view -> S BF16 slices [s][r][Kp] (k-contiguous rows, zero for k >= K)
template <int S>
__global__ void view_slices(const double* __restrict__ in, int64_t rs, int64_t ks, int rows,
                            int K, int Kp, StoreSlicesInt<S> st) {
  __shared__ double t[32][33];   // [k][r]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool rfast = ks != 1 && rs == 1;
  const int k0 = blockIdx.x * 32;
  for (int r0 = blockIdx.y * 32; r0 < rows; r0 += gridDim.y * 32) {
    for (int i = ty; i < 32; i += 8) {
      if (rfast)
        t[i][tx] = view_at(in, rs, ks, rows, K, r0 + tx, k0 + i);
      else
        t[tx][i] = view_at(in, rs, ks, rows, K, r0 + i, k0 + tx);
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
      const int r = r0 + i, k = k0 + tx;
      if (r < rows && k < Kp) st((int64_t)r * Kp + k, t[tx][i]);
    }
    __syncthreads();
  }
}

// C[m ldc + n] = (accum ? C : 0) + sum over c of part[c][m][n], in chunk order.
__global__ void sum_partials(const double* __restrict__ part, int nsp, int M, int N,
                             double* __restrict__ C, int64_t ldc, int accum) {
  const int64_t n_all = (int64_t)M * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_all;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = i / N, n = i - m * N;
    double v = 0.0;
    for (int c = 0; c < nsp; ++c) v += part[(int64_t)c * n_all + i];
    double* o = C + m * ldc + n;
    *o = accum ? *o + v : v;
  }
}

// max |x| over n doubles, as the bits of a non-negative double in *out (atomicMax).
__global__ void absmax_kernel(const double* __restrict__ x, int64_t n,
                              unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// Row-block gather: dst slot q <- src slot list[q], each slot `row16` 16-byte
// words, repeated over `nslice` slices (bf16 slices of one operand, or one
// float64 plane).  Used to keep only the occupied orbitals a triplet set uses.
__global__ void gather_rows_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                   const int* __restrict__ list, int nlist, int64_t row16,
                                   int nslice, int64_t src_slice16, int64_t dst_slice16) {
  const int64_t per = (int64_t)nlist * row16, n = per * nslice;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = e / per, r = e - sl * per;
    const int64_t q = r / row16, w = r - q * row16;
    dst[sl * dst_slice16 + r] = src[sl * src_slice16 + (int64_t)list[q] * row16 + w];
  }
}

// dst slot list[q] += src slot q (float64; slots of `row` elements, list
// entries distinct, so no two threads touch one element).
__global__ void scatter_add_rows_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                        const int* __restrict__ list, int nlist, int64_t row) {
  const int64_t n = (int64_t)nlist * row;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / row, w = e - q * row;
    dst[(int64_t)list[q] * row + w] += src[e];
  }
}

// Number of elements with |t2ab[i][J][a][B] - t2ab[J][i][B][a]| > tol (n
// occupied and v virtual of each spin); zero means the mixed amplitudes are
// spin-flip symmetric to within tol.
__global__ void t2ab_flip_mismatch(const double* __restrict__ t2ab, int n, int v, double tol,
                                   unsigned int* __restrict__ count) {
  const int64_t total = (int64_t)n * n * v * v;
  unsigned int bad = 0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int B = (int)(idx % v);
    int64_t r = idx / v;
    const int a = (int)(r % v);
    r /= v;
    const int J = (int)(r % n), i = (int)(r / n);
    if (!(fabs(t2ab[idx] - t2ab[(((int64_t)J * n + i) * v + B) * v + a]) <= tol)) ++bad;
  }
  if (bad) atomicAdd(count, bad);
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers (templated store: F64 or slices)
// ---------------------------------------------------------------------------
template <class St>
cudaError_t launch_transpose_block(const double* B, int naux, int nbas, int p0, int np, int q0,
                                   int nq, int Qp, St st, cudaStream_t s) {
  int64_t rows = (int64_t)np * nq;
  if (rows == 0) return cudaSuccess;
  dim3 grid(ceil_div(rows, 32), ceil_div(Qp, 32));
  transpose_block<<<grid, dim3(32, 8), 0, s>>>(B, naux, nbas, p0, np, q0, nq, Qp, st);
  return cudaGetLastError();
}

template <class St>
cudaError_t launch_pack_at_same(const int2* pairs, int nslot, int o, int oi, int v, int Kp,
                                const double* t2ss, const double* oovoT, St st, cudaStream_t s) {
  int64_t n = (int64_t)nslot * v * Kp;
  if (n == 0) return cudaSuccess;
  pack_at_same<<<grid_for(n), 256, 0, s>>>(pairs, nslot, o, oi, v, Kp, t2ss, oovoT, st);
  return cudaGetLastError();
}

template <class St>
cudaError_t launch_pack_bt_same(int slot, int x, int o, int oi, int v, int Kp,
                                const double* vvovT, const double* t2ss, St st, cudaStream_t s) {
  int64_t n = npairs(v) * Kp;
  if (n == 0) return cudaSuccess;
  pack_bt_same<<<grid_for(n), 256, 0, s>>>(slot, x, o, oi, v, Kp, vvovT, t2ss, st);
  return cudaGetLastError();
}

template <class St>
cudaError_t launch_pack_a1(const int2* pk, int nslot, int os, int vs, int ot, int oti, int vt,
                           int Kp, const double* t2st, const double* jT, St st, cudaStream_t s) {
  int64_t n = (int64_t)nslot * vs * Kp;
  if (n == 0) return cudaSuccess;
  pack_a1<<<grid_for(n), 256, 0, s>>>(pk, nslot, os, vs, ot, oti, vt, Kp, t2st, jT, st);
  return cudaGetLastError();
}

template <class St>
cudaError_t launch_pack_bg(int slot, int x, int os, int vs, int ot, int oti, int vt, int Kp,
                           const double* gT, const double* t2st, St st, cudaStream_t s) {
  int64_t n = (int64_t)vs * vt * Kp;
  if (n == 0) return cudaSuccess;
  pack_bg<<<grid_for(n), 256, 0, s>>>(slot, x, os, vs, ot, oti, vt, Kp, gT, t2st, st);
  return cudaGetLastError();
}

template <class St>
cudaError_t launch_pack_bf(int slot, int K, int os, int osi, int vs, int ot, int vt, int Kp,
                           const double* fT, const double* t2st, St st, cudaStream_t s) {
  int64_t n = (int64_t)vs * vt * Kp;
  if (n == 0) return cudaSuccess;
  pack_bf<<<grid_for(n), 256, 0, s>>>(slot, K, os, osi, vs, ot, vt, Kp, fT, t2st, st);
  return cudaGetLastError();
}

template <class St>
cudaError_t launch_pack_at2(const int2* pk, int nslot, int os, int osi, int vs, int ot, int vt,
                            int Kp, const double* t2st, const double* lT, St st,
                            cudaStream_t s) {
  int64_t n = (int64_t)nslot * vt * Kp;
  if (n == 0) return cudaSuccess;
  pack_at2<<<grid_for(n), 256, 0, s>>>(pk, nslot, os, osi, vs, ot, vt, Kp, t2st, lT, st);
  return cudaGetLastError();
}

cudaError_t launch_transpose_t2ab(const double* t2ab, int na, int nb, int va, int vb, double* out,
                                  cudaStream_t s) {
  int64_t n = (int64_t)na * nb * va * vb;
  if (n == 0) return cudaSuccess;
  transpose_t2ab<<<grid_for(n), 256, 0, s>>>(t2ab, na, nb, va, vb, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const void* src, void* dst, const int* list, int nlist,
                               int64_t row_bytes, int nslice, int64_t src_slice_bytes,
                               int64_t dst_slice_bytes, cudaStream_t s) {
  if (nlist == 0 || row_bytes == 0 || nslice == 0) return cudaSuccess;
  if (row_bytes % 16 || src_slice_bytes % 16 || dst_slice_bytes % 16 ||
      reinterpret_cast<uintptr_t>(src) % 16 || reinterpret_cast<uintptr_t>(dst) % 16)
    return cudaErrorInvalidValue;
  const int64_t n = (int64_t)nlist * (row_bytes / 16) * nslice;
  gather_rows_kernel<<<grid_for(n), 256, 0, s>>>(
      static_cast<const uint4*>(src), static_cast<uint4*>(dst), list, nlist, row_bytes / 16,
      nslice, src_slice_bytes / 16, dst_slice_bytes / 16);
  return cudaGetLastError();
}

cudaError_t launch_scatter_add_rows(const double* src, double* dst, const int* list, int nlist,
                                    int64_t row, cudaStream_t s) {
  const int64_t n = (int64_t)nlist * row;
  if (n == 0) return cudaSuccess;
  scatter_add_rows_kernel<<<grid_for(n), 256, 0, s>>>(src, dst, list, nlist, row);
  return cudaGetLastError();
}

cudaError_t launch_t2ab_flip_mismatch(const double* t2ab, int n, int v, double tol,
                                     unsigned int* count, cudaStream_t s) {
  const int64_t total = (int64_t)n * n * v * v;
  if (total == 0) return cudaSuccess;
  t2ab_flip_mismatch<<<grid_for(total), 256, 0, s>>>(t2ab, n, v, tol, count);
  return cudaGetLastError();
}

cudaError_t launch_absmax(const double* x, int64_t n, unsigned long long* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  absmax_kernel<<<grid_for(n), 256, 0, s>>>(x, n, out);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* part, int nsp, int M, int N, double* C,
                                int64_t ldc, bool accum, cudaStream_t s) {
  const int64_t n = (int64_t)M * N;
  if (n <= 0) return cudaSuccess;
  sum_partials<<<grid_for(n), 256, 0, s>>>(part, nsp, M, N, C, ldc, accum ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_view_absmax(const double* in, int64_t rs, int64_t ks, int rows, int K,
                               unsigned long long* out, cudaStream_t s) {
  if (rows <= 0 || K <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((K + 31) / 32), (unsigned)std::min((rows + 31) / 32, 4096));
  view_absmax<<<grid, dim3(32, 8), 0, s>>>(in, rs, ks, rows, K, out);
  return cudaGetLastError();
}

// inv = 2^7 / scale, a power of two
template <int S>
cudaError_t launch_view_slices(const double* in, int64_t rs, int64_t ks, int rows, int K,
                               int Kp, __nv_bfloat16* out, int64_t slice_stride, double inv,
                               cudaStream_t s) {
  if (rows <= 0 || Kp <= 0) return cudaSuccess;
  int e;
  if (!(inv > 0) || std::frexp(inv, &e) != 0.5) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((Kp + 31) / 32), (unsigned)std::min((rows + 31) / 32, 4096));
  view_slices<S><<<grid, dim3(32, 8), 0, s>>>(
      in, rs, ks, rows, K, Kp, StoreSlicesInt<S>{out, slice_stride, (e - 1) + 8 * (S - 1)});
  return cudaGetLastError();
}
template cudaError_t launch_view_slices<4>(const double*, int64_t, int64_t, int, int, int,
                                           __nv_bfloat16*, int64_t, double, cudaStream_t);
template cudaError_t launch_view_slices<5>(const double*, int64_t, int64_t, int, int, int,
                                           __nv_bfloat16*, int64_t, double, cudaStream_t);

#define LNO_INST(St)                                                                           \
  template cudaError_t launch_transpose_block<St>(const double*, int, int, int, int, int, int,  \
                                                  int, St, cudaStream_t);                       \
  template cudaError_t launch_pack_at_same<St>(const int2*, int, int, int, int, int,           \
                                               const double*, const double*, St, cudaStream_t); \
  template cudaError_t launch_pack_bt_same<St>(int, int, int, int, int, int, const double*,     \
                                               const double*, St, cudaStream_t);               \
  template cudaError_t launch_pack_a1<St>(const int2*, int, int, int, int, int, int, int,      \
                                          const double*, const double*, St, cudaStream_t);     \
  template cudaError_t launch_pack_bg<St>(int, int, int, int, int, int, int, int,               \
                                          const double*, const double*, St, cudaStream_t);     \
  template cudaError_t launch_pack_bf<St>(int, int, int, int, int, int, int, int,               \
                                          const double*, const double*, St, cudaStream_t);     \
  template cudaError_t launch_pack_at2<St>(const int2*, int, int, int, int, int, int, int,     \
                                           const double*, const double*, St, cudaStream_t);

LNO_INST(StoreF64)
LNO_INST(StoreSlices<2>)
LNO_INST(StoreSlices<3>)
LNO_INST(StoreSlices<4>)
LNO_INST(StoreSlices<5>)
LNO_INST(StoreTF32<2>)
#undef LNO_INST

}  // namespace lno
