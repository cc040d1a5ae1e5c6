// Adjoint of the domain (T) energy (float64): gradient of
//   E = sum_t sum_{restricted abc} W (W + V) / D       (eq cim_pt_energy)
// with respect to B, eps, T1 and T2, W recomputed per triplet (never stored).
//
// Per element: g_W = (2W + V)/D, g_V = W/D, g_D = -W (W + V)/D^2.
//   W = X[a,(bc)] - X[b,(ac)] + X[c,(ab)]   -> dX entries +g_W, -g_W, +g_W
//   V = sum of t1 x (pq|rs) products         -> dT1 and d(ia|jb) / d(jb|KC)
//   D = e_i + e_j + e_k - e_a - e_b - e_c    -> deps
// Each X entry with distinct virtual labels belongs to exactly one
// restricted element, so dX is written with plain stores (the caller zeroes
// it first).  Per-tile sums of dT1, deps and the V-integral gradients are
// reduced in shared memory and added to global memory with atomics.
//
// Contraction adjoint (grouped strided GEMM, atomically accumulated):
//   X^T[n][m] = sum_seg s A[m][:] . B[n][:]  ->  dA += s dX.B,  dB += s dX^T.A
// Layout adjoints of the pack kernels scatter operand gradients back to T2
// and to the DF intermediates, whose adjoint GEMMs give dB.
#include "common.cuh"

namespace lno {

// C(m,n) (+)= alpha sum_k A(m,k) B(k,n); strides in elements.
struct GemmS {
  const double* A;
  const double* B;
  double* C;
  int M, N, K;
  int atomic;
  int64_t sam, sak, sbk, sbn, scm, scn;
  double alpha;
};

namespace {

constexpr int TB = 16;
constexpr int GBM = 64, GBN = 64, GBK = 16;

__global__ void __launch_bounds__(256) gemm_f64_strided(const GemmS* __restrict__ probs) {
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  const GemmS P = probs[blockIdx.z];
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  if (m0 >= P.M || n0 >= P.N) return;
  const int tid = threadIdx.x;
  const int tm = tid % 16, tn = tid / 16;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < P.K; k0 += GBK) {
    for (int e = tid; e < GBK * GBM; e += 256) {
      // coalesce along whichever index is contiguous in memory
      int kk, mm;
      if (P.sam == 1) { mm = e % GBM; kk = e / GBM; } else { kk = e % GBK; mm = e / GBK; }
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < P.M && k < P.K) ? P.A[(int64_t)m * P.sam + (int64_t)k * P.sak] : 0.0;
    }
    for (int e = tid; e < GBK * GBN; e += 256) {
      int kk, nn;
      if (P.sbn == 1) { nn = e % GBN; kk = e / GBN; } else { kk = e % GBK; nn = e / GBK; }
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < P.N && k < P.K) ? P.B[(int64_t)k * P.sbk + (int64_t)n * P.sbn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
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
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int m = m0 + tm * 4 + a;
    if (m >= P.M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int n = n0 + tn * 4 + b;
      if (n >= P.N) continue;
      double* c = P.C + (int64_t)m * P.scm + (int64_t)n * P.scn;
      const double v = P.alpha * acc[a][b];
      if (P.atomic) atomicAdd(c, v); else *c += v;
    }
  }
}

// Energy adjoint of one triplet group (float64 X).  Gradient outputs:
//   dX (same layout as X, zeroed by the caller), dt1s/dt1t [n][nv],
//   dov_ss (same layout as ovov_ss), dov_ts (as ovov_ts), deps_s/deps_t [nbas].
// FM (a.vmode 1, the f_ov part sum W V_f / D): dX is added to, dt1s/dt1t are
// the f_ov gradients and dov_ss/dov_ts the raw T2 gradients (t2ss / t2st
// layouts), since the planes are then the amplitudes themselves.
template <bool MIXED, bool FM>
__global__ void __launch_bounds__(256)
energy_backward(EnergyArgs a, const double* __restrict__ X, const double* __restrict__ Z,
                double* __restrict__ dX, double* __restrict__ dZ, double* __restrict__ dt1s,
                double* __restrict__ dt1t, double* __restrict__ dov_ss,
                double* __restrict__ dov_ts, double* __restrict__ deps_s,
                double* __restrict__ deps_t, double gscale) {
  __shared__ double vt[9][TB][TB];   // V integral tables (as in the forward)
  __shared__ double gvt[9][TB][TB];  // their gradients
  __shared__ double t1s[9][TB], gt1[9][TB];
  __shared__ double ev[3][TB], gev[3][TB];
  __shared__ double gocc;
  const int g = blockIdx.y;
  const Trip tr = a.trips[g];
  const double* Xg = X + (int64_t)g * a.x_stride;
  const double* Zg = MIXED ? Z + (int64_t)g * a.z_stride : nullptr;
  double* dXg = dX + (int64_t)g * a.x_stride;
  double* dZg = MIXED ? dZ + (int64_t)g * a.z_stride : nullptr;
  const int tid = threadIdx.x, r1 = tid / TB, r2 = tid % TB;
  const int nvs = a.nvs, nvt = a.nvt, nos = a.nos;
  const double eocc = MIXED ? a.eps_s[tr.i] + a.eps_s[tr.j] + a.eps_t[tr.k]
                            : a.eps_s[tr.i] + a.eps_s[tr.j] + a.eps_s[tr.k];
  if (tid == 0) gocc = 0.0;
  for (int q = blockIdx.x; q < a.nblocks; q += gridDim.x) {
    const int3 blk = a.blocks[q];
    const int a0 = blk.x * TB, b0 = blk.y * TB, c0 = blk.z * TB;
    // ---- V tables and t1 / eps of the tile (as in the forward) -------------
    if (!MIXED) {
      const int occ3[3][2] = {{tr.j, tr.k}, {tr.k, tr.i}, {tr.i, tr.j}};
      const int offs[3][2] = {{b0, c0}, {a0, c0}, {a0, b0}};
      for (int pl = 0; pl < 3; ++pl) {
        const int x = offs[pl][0] + r1, y = offs[pl][1] + r2;
        for (int o = 0; o < 3; ++o) {
          double v = 0.0;
          if (x < nvs && y < nvs) v = vplane_ss(a, occ3[o][0], x, occ3[o][1], y);
          vt[pl * 3 + o][r1][r2] = v;
          gvt[pl * 3 + o][r1][r2] = 0.0;
        }
      }
    } else {
      const int offs[2] = {b0, a0};
      for (int pl = 0; pl < 2; ++pl) {
        const int x = offs[pl] + r1, y = c0 + r2;
        for (int o = 0; o < 2; ++o) {
          double v = 0.0;
          if (x < nvs && y < nvt) v = vplane_ts(a, tr.k, y, o == 0 ? tr.j : tr.i, x);
          vt[pl * 2 + o][r1][r2] = v;
          gvt[pl * 2 + o][r1][r2] = 0.0;
        }
      }
      const int x = a0 + r1, y = b0 + r2;
      double v = 0.0;
      if (x < nvs && y < nvs) v = vplane_ss(a, tr.i, x, tr.j, y);
      vt[4][r1][r2] = v;
      gvt[4][r1][r2] = 0.0;
    }
    if (tid < 3 * TB) {
      const int bl = tid / TB, l = tid % TB;
      const int base = bl == 0 ? a0 : (bl == 1 ? b0 : c0);
      const int x = base + l;
      const bool tblock = MIXED && bl == 2;
      const int nv = tblock ? nvt : nvs;
      if (!MIXED) {
        const int occ[3] = {tr.i, tr.j, tr.k};
        for (int o = 0; o < 3; ++o)
          t1s[bl * 3 + o][l] = x < nvs ? a.t1s[(int64_t)occ[o] * nvs + x] : 0.0;
      } else if (!tblock) {
        t1s[bl * 3 + 0][l] = x < nvs ? a.t1s[(int64_t)tr.i * nvs + x] : 0.0;
        t1s[bl * 3 + 1][l] = x < nvs ? a.t1s[(int64_t)tr.j * nvs + x] : 0.0;
        t1s[bl * 3 + 2][l] = 0.0;
      } else {
        t1s[bl * 3 + 0][l] = x < nvt ? a.t1t[(int64_t)tr.k * nvt + x] : 0.0;
        t1s[bl * 3 + 1][l] = t1s[bl * 3 + 2][l] = 0.0;
      }
      for (int o = 0; o < 3; ++o) gt1[bl * 3 + o][l] = 0.0;
      const double* e = tblock ? a.eps_t : a.eps_s;
      const int no = tblock ? a.not_ : a.nos;
      ev[bl][l] = x < nv ? e[no + x] : 0.0;
      gev[bl][l] = 0.0;
    }
    __syncthreads();
    // ---- elements: thread (b, c), loop over a ------------------------------
    {
      const int bl = r1, cl = r2;
      const int b = b0 + bl, c = c0 + cl;
      const bool rowok = MIXED ? (b < nvs && c < nvt) : (b < c && c < nvs);
      if (rowok) {
        const int na = min(b, a0 + TB) - a0;
        double gb_e = 0.0, gc_e = 0.0, gocc_t = 0.0;
        double gk_bc[3] = {0.0, 0.0, 0.0}, gtb[3] = {0.0, 0.0, 0.0}, gtc[3] = {0.0, 0.0, 0.0};
        for (int al = 0; al < na; ++al) {
          const int aa = a0 + al;
          int64_t i1, i2, i3;
          double x1, x2, x3;
          if (!MIXED) {
            i1 = pair_index(b, c) * a.pitch_x + aa;
            i2 = pair_index(aa, c) * a.pitch_x + b;
            i3 = pair_index(aa, b) * a.pitch_x + c;
            x1 = Xg[i1]; x2 = Xg[i2]; x3 = Xg[i3];
          } else {
            i1 = ((int64_t)b * nvt + c) * a.pitch_x + aa;
            i2 = ((int64_t)aa * nvt + c) * a.pitch_x + b;
            i3 = pair_index(aa, b) * a.pitch_z + c;
            x1 = Xg[i1]; x2 = Xg[i2]; x3 = Zg[i3];
          }
          const double w = x1 - x2 + x3;
          double v;
          if (!MIXED) {
            const double ya = t1s[0][al] * vt[0][bl][cl] + t1s[1][al] * vt[1][bl][cl] +
                              t1s[2][al] * vt[2][bl][cl];
            const double yb = t1s[3][bl] * vt[3][al][cl] + t1s[4][bl] * vt[4][al][cl] +
                              t1s[5][bl] * vt[5][al][cl];
            const double yc = t1s[6][cl] * vt[6][al][bl] + t1s[7][cl] * vt[7][al][bl] +
                              t1s[8][cl] * vt[8][al][bl];
            v = ya - yb + yc;
          } else {
            v = t1s[0][al] * vt[0][bl][cl] - t1s[1][al] * vt[1][bl][cl] -
                t1s[3][bl] * vt[2][al][cl] + t1s[4][bl] * vt[3][al][cl] +
                t1s[6][cl] * vt[4][al][bl];
          }
          const double D = eocc - ev[0][al] - ev[1][bl] - ev[2][cl];
          // E = W (W + V) / D, or W V / D for the f_ov part
          const double gw = gscale * (FM ? v : 2.0 * w + v) / D;
          const double gv = gscale * w / D;
          const double gd = -gscale * w * (FM ? v : w + v) / (D * D);
          if (!MIXED) {
            if (FM) {
              dXg[i1] += gw; dXg[i2] -= gw; dXg[i3] += gw;
            } else {
              dXg[i1] = gw; dXg[i2] = -gw; dXg[i3] = gw;
            }
            for (int o = 0; o < 3; ++o) {
              gk_bc[o] += gv * t1s[o][al];
              atomicAdd(&gt1[o][al], gv * vt[o][bl][cl]);
              gtb[o] -= gv * vt[3 + o][al][cl];
              atomicAdd(&gvt[3 + o][al][cl], -gv * t1s[3 + o][bl]);
              gtc[o] += gv * vt[6 + o][al][bl];
              atomicAdd(&gvt[6 + o][al][bl], gv * t1s[6 + o][cl]);
            }
          } else {
            if (FM) {
              dXg[i1] += gw; dXg[i2] -= gw; dZg[i3] += gw;
            } else {
              dXg[i1] = gw; dXg[i2] = -gw; dZg[i3] = gw;
            }
            gk_bc[0] += gv * t1s[0][al];             // (jb|KC)
            gk_bc[1] -= gv * t1s[1][al];             // (ib|KC)
            atomicAdd(&gt1[0][al], gv * vt[0][bl][cl]);
            atomicAdd(&gt1[1][al], -gv * vt[1][bl][cl]);
            gtb[0] -= gv * vt[2][al][cl];            // t^b_i
            gtb[1] += gv * vt[3][al][cl];            // t^b_j
            atomicAdd(&gvt[2][al][cl], -gv * t1s[3][bl]);
            atomicAdd(&gvt[3][al][cl], gv * t1s[4][bl]);
            gtc[0] += gv * vt[4][al][bl];            // t^C_K
            atomicAdd(&gvt[4][al][bl], gv * t1s[6][cl]);
          }
          gocc_t += gd;
          atomicAdd(&gev[0][al], -gd);
          gb_e -= gd;
          gc_e -= gd;
        }
        const int nk = MIXED ? 2 : 3;
        for (int o = 0; o < nk; ++o) atomicAdd(&gvt[o][bl][cl], gk_bc[o]);
        for (int o = 0; o < 3; ++o) {
          atomicAdd(&gt1[3 + o][bl], gtb[o]);
          atomicAdd(&gt1[6 + o][cl], gtc[o]);
        }
        atomicAdd(&gev[1][bl], gb_e);
        atomicAdd(&gev[2][cl], gc_e);
        atomicAdd(&gocc, gocc_t);
      }
    }
    __syncthreads();
    // ---- flush tile gradients ----------------------------------------------
    if (!MIXED) {
      const int occ3[3][2] = {{tr.j, tr.k}, {tr.k, tr.i}, {tr.i, tr.j}};
      const int offs[3][2] = {{b0, c0}, {a0, c0}, {a0, b0}};
      for (int pl = 0; pl < 3; ++pl) {
        const int x = offs[pl][0] + r1, y = offs[pl][1] + r2;
        if (x >= nvs || y >= nvs) continue;
        for (int o = 0; o < 3; ++o) {
          const double gk = gvt[pl * 3 + o][r1][r2];
          if (gk == 0.0) continue;
          const int p = occ3[o][0], r = occ3[o][1];
          if (FM) {
            atomicAdd(&dov_ss[(((int64_t)p * nos + r) * nvs + x) * nvs + y], gk);
          } else {
            atomicAdd(&dov_ss[ovss_idx(a, p, x, r, y)], gk);
            atomicAdd(&dov_ss[ovss_idx(a, p, y, r, x)], -gk);
          }
        }
      }
    } else {
      const int offs[2] = {b0, a0};
      for (int pl = 0; pl < 2; ++pl) {
        const int x = offs[pl] + r1, y = c0 + r2;
        if (x >= nvs || y >= nvt) continue;
        for (int o = 0; o < 2; ++o) {
          const double gk = gvt[pl * 2 + o][r1][r2];
          if (gk == 0.0) continue;
          const int p = o == 0 ? tr.j : tr.i;
          if (FM)
            atomicAdd(&dov_ts[(((int64_t)p * a.not_ + tr.k) * nvs + x) * nvt + y], gk);
          else
            atomicAdd(&dov_ts[ovts_idx(a, tr.k, y, p, x)], gk);
        }
      }
      const int x = a0 + r1, y = b0 + r2;
      const double gk = gvt[4][r1][r2];
      if (x < nvs && y < nvs && gk != 0.0) {
        if (FM) {
          atomicAdd(&dov_ss[(((int64_t)tr.i * nos + tr.j) * nvs + x) * nvs + y], gk);
        } else {
          atomicAdd(&dov_ss[ovss_idx(a, tr.i, x, tr.j, y)], gk);
          atomicAdd(&dov_ss[ovss_idx(a, tr.i, y, tr.j, x)], -gk);
        }
      }
    }
    if (tid < 3 * TB) {
      const int bl = tid / TB, l = tid % TB;
      const int base = bl == 0 ? a0 : (bl == 1 ? b0 : c0);
      const int x = base + l;
      const bool tblock = MIXED && bl == 2;
      const int nv = tblock ? nvt : nvs;
      if (x < nv) {
        if (!MIXED) {
          const int occ[3] = {tr.i, tr.j, tr.k};
          for (int o = 0; o < 3; ++o)
            if (gt1[bl * 3 + o][l] != 0.0)
              atomicAdd(&dt1s[(int64_t)occ[o] * nvs + x], gt1[bl * 3 + o][l]);
        } else if (!tblock) {
          atomicAdd(&dt1s[(int64_t)tr.i * nvs + x], gt1[bl * 3 + 0][l]);
          atomicAdd(&dt1s[(int64_t)tr.j * nvs + x], gt1[bl * 3 + 1][l]);
        } else {
          atomicAdd(&dt1t[(int64_t)tr.k * nvt + x], gt1[bl * 3 + 0][l]);
        }
        double* de = tblock ? deps_t : deps_s;
        const int no = tblock ? a.not_ : a.nos;
        if (gev[bl][l] != 0.0) atomicAdd(&de[no + x], gev[bl][l]);
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    atomicAdd(&deps_s[tr.i], gocc);
    atomicAdd(&deps_s[tr.j], gocc);
    atomicAdd(MIXED ? &deps_t[tr.k] : &deps_s[tr.k], gocc);
  }
}

// ---- layout adjoints (mirror the pack kernels; atomically accumulated) -----
__global__ void adj_at_same(const int2* __restrict__ pairs, int nslot, int o, int v, int Kp,
                            const double* __restrict__ dAT, double* __restrict__ dt2ss,
                            double* __restrict__ doovoT) {
  const int64_t total = (int64_t)nslot * v * Kp;
  const int64_t oo = (int64_t)o * o;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const int64_t r = idx / Kp;
    const int a = (int)(r % v);
    const int2 pq = pairs[r / v];
    const double gd = dAT[idx];
    if (gd == 0.0 || kk >= v + o) continue;
    if (kk < v) {
      atomicAdd(&dt2ss[(((int64_t)pq.x * o + pq.y) * v + a) * v + kk], gd);
    } else {
      const int m = kk - v;
      atomicAdd(&doovoT[((int64_t)pq.x * v + a) * oo + m * o + pq.y], gd);
      atomicAdd(&doovoT[((int64_t)pq.y * v + a) * oo + m * o + pq.x], -gd);
    }
  }
}

__global__ void adj_bt_same(int slot, int x, int o, int v, int Kp, const double* __restrict__ dBT,
                            double* __restrict__ dvvovT, double* __restrict__ dt2ss) {
  const int64_t np = npairs(v);
  const int64_t total = np * Kp;
  const int64_t base = (int64_t)slot * np * Kp;
  const int64_t vv = (int64_t)v * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const double gd = dBT[base + idx];
    if (gd == 0.0 || kk >= v + o) continue;
    const int64_t pr = idx / Kp;
    int c = (int)((1.0 + sqrt(1.0 + 8.0 * (double)pr)) * 0.5);
    while ((int64_t)c * (c - 1) / 2 > pr) --c;
    while ((int64_t)(c + 1) * c / 2 <= pr) ++c;
    const int b = (int)(pr - (int64_t)c * (c - 1) / 2);
    if (kk < v) {
      atomicAdd(&dvvovT[(int64_t)c * vv + (int64_t)kk * v + b], gd);
      atomicAdd(&dvvovT[(int64_t)b * vv + (int64_t)kk * v + c], -gd);
    } else {
      atomicAdd(&dt2ss[(((int64_t)x * o + (kk - v)) * v + b) * v + c], gd);
    }
  }
}

__global__ void adj_a1(const int2* __restrict__ pk, int nslot, int os, int vs, int ot, int vt,
                       int Kp, const double* __restrict__ dA1, double* __restrict__ dt2st,
                       double* __restrict__ djT) {
  const int64_t total = (int64_t)nslot * vs * Kp;
  const int64_t ld = (int64_t)os * vs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const double gd = dA1[idx];
    if (gd == 0.0 || kk >= vt + ot) continue;
    const int64_t r = idx / Kp;
    const int a = (int)(r % vs);
    const int2 p = pk[r / vs];
    if (kk < vt)
      atomicAdd(&dt2st[(((int64_t)p.x * ot + p.y) * vs + a) * vt + kk], -gd);
    else
      atomicAdd(&djT[((int64_t)(kk - vt) * ot + p.y) * ld + (int64_t)p.x * vs + a], gd);
  }
}

__global__ void adj_bg(int slot, int x, int os, int vs, int ot, int vt, int Kp,
                       const double* __restrict__ dBG, double* __restrict__ dgT,
                       double* __restrict__ dt2st) {
  const int64_t rows = (int64_t)vs * vt;
  const int64_t total = rows * Kp;
  const int64_t base = (int64_t)slot * total;
  const int64_t vv = (int64_t)vt * vt;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const double gd = dBG[base + idx];
    if (gd == 0.0 || kk >= vt + ot) continue;
    const int64_t r = idx / Kp;
    const int b = (int)(r / vt), C = (int)(r % vt);
    if (kk < vt)
      atomicAdd(&dgT[(int64_t)b * vv + (int64_t)kk * vt + C], gd);
    else
      atomicAdd(&dt2st[(((int64_t)x * ot + (kk - vt)) * vs + b) * vt + C], gd);
  }
}

__global__ void adj_bf(int slot, int K, int os, int vs, int ot, int vt, int Kp,
                       const double* __restrict__ dBF, double* __restrict__ dfT,
                       double* __restrict__ dt2st) {
  const int64_t rows = (int64_t)vs * vt;
  const int64_t total = rows * Kp;
  const int64_t base = (int64_t)slot * total;
  const int64_t vv = (int64_t)vs * vs;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const double gd = dBF[base + idx];
    if (gd == 0.0 || kk >= vs + os) continue;
    const int64_t r = idx / Kp;
    const int b = (int)(r / vt), C = (int)(r % vt);
    if (kk < vs)
      atomicAdd(&dfT[(int64_t)C * vv + (int64_t)b * vs + kk], gd);
    else
      atomicAdd(&dt2st[(((int64_t)(kk - vs) * ot + K) * vs + b) * vt + C], -gd);
  }
}

__global__ void adj_at2(const int2* __restrict__ pk, int nslot, int os, int vs, int ot, int vt,
                        int Kp, const double* __restrict__ dAT2, double* __restrict__ dt2st,
                        double* __restrict__ dlT) {
  const int64_t total = (int64_t)nslot * vt * Kp;
  const int64_t ld = (int64_t)os * os;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % Kp);
    const double gd = dAT2[idx];
    if (gd == 0.0 || kk >= vs + os) continue;
    const int64_t r = idx / Kp;
    const int C = (int)(r % vt);
    const int2 p = pk[r / vt];
    if (kk < vs)
      atomicAdd(&dt2st[(((int64_t)p.x * ot + p.y) * vs + kk) * vt + C], gd);
    else
      atomicAdd(&dlT[((int64_t)p.y * vt + C) * ld + (int64_t)(kk - vs) * os + p.x], gd);
  }
}

// dB[Q][p0+p][q0+q] += dblk[(p*nq+q)][Q]  (inverse of transpose_block)
__global__ void adj_transpose_block(const double* __restrict__ dblk, int naux, int nbas, int p0,
                                    int np, int q0, int nq, int Qp, double* __restrict__ dB) {
  const int64_t total = (int64_t)np * nq * naux;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx % ((int64_t)np * nq);
    const int Q = (int)(idx / ((int64_t)np * nq));
    const int p = (int)(r / nq), q = (int)(r % nq);
    dB[((int64_t)Q * nbas + p0 + p) * nbas + q0 + q] += dblk[r * Qp + Q];
  }
}

// out = scale * (G + G^T)/2 over the last two indices of [naux][n][n]
__global__ void sym_project(const double* __restrict__ G, int naux, int n, double scale,
                            double* __restrict__ out) {
  const int64_t total = (int64_t)naux * n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx % n);
    const int64_t r = idx / n;
    const int p = (int)(r % n);
    const int64_t Q = r / n;
    out[idx] = 0.5 * scale * (G[idx] + G[(Q * n + q) * n + p]);
  }
}

// out[i][j][a][b] = scale (G - G_ji - G_ba + G_jiba)/4
__global__ void antisym_project(const double* __restrict__ G, int o, int v, double scale,
                                double* __restrict__ out) {
  const int64_t total = (int64_t)o * o * v * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx % v);
    int64_t r = idx / v;
    const int a = (int)(r % v);
    r /= v;
    const int j = (int)(r % o);
    const int i = (int)(r / o);
    auto at = [&](int ii, int jj, int aa, int bb) {
      return G[(((int64_t)ii * o + jj) * v + aa) * v + bb];
    };
    out[idx] = 0.25 * scale * (at(i, j, a, b) - at(j, i, a, b) - at(i, j, b, a) + at(j, i, b, a));
  }
}

// In place: G[Q][p][q], G[Q][q][p] <- (G[Q][p][q] + G[Q][q][p]) / 2
__global__ void sym_inplace(double* __restrict__ G, int naux, int n) {
  const int64_t np = (int64_t)n * (n - 1) / 2;
  const int64_t total = (int64_t)naux * np;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t Q = idx / np, pr = idx % np;
    int q = (int)((1.0 + sqrt(1.0 + 8.0 * (double)pr)) * 0.5);
    while ((int64_t)q * (q - 1) / 2 > pr) --q;
    while ((int64_t)(q + 1) * q / 2 <= pr) ++q;
    const int p = (int)(pr - (int64_t)q * (q - 1) / 2);
    double* x = G + (Q * n + p) * n + q;
    double* y = G + (Q * n + q) * n + p;
    const double m = 0.5 * (*x + *y);
    *x = m;
    *y = m;
  }
}

// In place over one index pair of [o][o][v][v]: first (i,j), then (a,b):
// X <- (X - X^T)/2 (diagonal -> 0).  Both passes give (G-G_ji-G_ba+G_jiba)/4.
__global__ void antisym_inplace_occ(double* __restrict__ G, int o, int v) {
  const int64_t vv = (int64_t)v * v;
  const int64_t total = (int64_t)o * o * vv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ab = idx % vv, ij = idx / vv;
    const int i = (int)(ij / o), j = (int)(ij % o);
    if (i > j) continue;
    double* x = G + ((int64_t)i * o + j) * vv + ab;
    if (i == j) { *x = 0.0; continue; }
    double* y = G + ((int64_t)j * o + i) * vv + ab;
    const double d = 0.5 * (*x - *y);
    *x = d;
    *y = -d;
  }
}
__global__ void antisym_inplace_vir(double* __restrict__ G, int o, int v) {
  const int64_t vv = (int64_t)v * v;
  const int64_t total = (int64_t)o * o * vv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ij = idx / vv, ab = idx % vv;
    const int a = (int)(ab / v), b = (int)(ab % v);
    if (a > b) continue;
    double* x = G + ij * vv + (int64_t)a * v + b;
    if (a == b) { *x = 0.0; continue; }
    double* y = G + ij * vv + (int64_t)b * v + a;
    const double d = 0.5 * (*x - *y);
    *x = d;
    *y = -d;
  }
}

// dt2ab[k][I][c][A] += dt2ba[I][k][A][c]
__global__ void adj_transpose_t2ab(const double* __restrict__ dt2ba, int na, int nb, int va, int vb,
                                   double* __restrict__ dt2ab) {
  const int64_t total = (int64_t)na * nb * va * vb;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(idx % va);
    int64_t r = idx / va;
    int A = (int)(r % vb);
    r /= vb;
    int k = (int)(r % na);
    int I = (int)(r / na);
    dt2ab[(((int64_t)k * nb + I) * va + c) * vb + A] += dt2ba[idx];
  }
}

__global__ void scale_copy(const double* __restrict__ in, int64_t n, double s,
                           double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = s * in[i];
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

}  // namespace

// ---------------------------------------------------------------------------
cudaError_t launch_gemm_strided(const GemmS* probs_dev, int nprob, int maxM, int maxN,
                                cudaStream_t st) {
  if (nprob <= 0 || maxM <= 0 || maxN <= 0) return cudaSuccess;
  dim3 grid(ceil_div(maxN, GBN), ceil_div(maxM, GBM), nprob);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  gemm_f64_strided<<<grid, 256, 0, st>>>(probs_dev);
  return cudaGetLastError();
}

cudaError_t launch_energy_backward(const EnergyArgs& a, const double* X, const double* Z,
                                   double* dX, double* dZ, double* dt1s, double* dt1t,
                                   double* dov_ss, double* dov_ts, double* deps_s,
                                   double* deps_t, double gscale, int ntrip, int nchunks,
                                   cudaStream_t st) {
  if (ntrip <= 0) return cudaSuccess;
  dim3 grid(nchunks, ntrip);
  const bool fm = a.vmode != 0;
  if (a.kind == SAME) {
    if (fm)
      energy_backward<false, true><<<grid, 256, 0, st>>>(a, X, Z, dX, dZ, dt1s, dt1t, dov_ss,
                                                         dov_ts, deps_s, deps_t, gscale);
    else
      energy_backward<false, false><<<grid, 256, 0, st>>>(a, X, Z, dX, dZ, dt1s, dt1t, dov_ss,
                                                          dov_ts, deps_s, deps_t, gscale);
  } else {
    if (fm)
      energy_backward<true, true><<<grid, 256, 0, st>>>(a, X, Z, dX, dZ, dt1s, dt1t, dov_ss,
                                                        dov_ts, deps_s, deps_t, gscale);
    else
      energy_backward<true, false><<<grid, 256, 0, st>>>(a, X, Z, dX, dZ, dt1s, dt1t, dov_ss,
                                                         dov_ts, deps_s, deps_t, gscale);
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_at_same(const int2* pairs, int nslot, int o, int v, int Kp,
                               const double* dAT, double* dt2ss, double* doovoT, cudaStream_t st) {
  int64_t n = (int64_t)nslot * v * Kp;
  if (n == 0) return cudaSuccess;
  adj_at_same<<<grid_for(n), 256, 0, st>>>(pairs, nslot, o, v, Kp, dAT, dt2ss, doovoT);
  return cudaGetLastError();
}
cudaError_t launch_adj_bt_same(int slot, int x, int o, int v, int Kp, const double* dBT,
                               double* dvvovT, double* dt2ss, cudaStream_t st) {
  int64_t n = npairs(v) * Kp;
  if (n == 0) return cudaSuccess;
  adj_bt_same<<<grid_for(n), 256, 0, st>>>(slot, x, o, v, Kp, dBT, dvvovT, dt2ss);
  return cudaGetLastError();
}
cudaError_t launch_adj_a1(const int2* pk, int nslot, int os, int vs, int ot, int vt, int Kp,
                          const double* dA1, double* dt2st, double* djT, cudaStream_t st) {
  int64_t n = (int64_t)nslot * vs * Kp;
  if (n == 0) return cudaSuccess;
  adj_a1<<<grid_for(n), 256, 0, st>>>(pk, nslot, os, vs, ot, vt, Kp, dA1, dt2st, djT);
  return cudaGetLastError();
}
cudaError_t launch_adj_bg(int slot, int x, int os, int vs, int ot, int vt, int Kp,
                          const double* dBG, double* dgT, double* dt2st, cudaStream_t st) {
  int64_t n = (int64_t)vs * vt * Kp;
  if (n == 0) return cudaSuccess;
  adj_bg<<<grid_for(n), 256, 0, st>>>(slot, x, os, vs, ot, vt, Kp, dBG, dgT, dt2st);
  return cudaGetLastError();
}
cudaError_t launch_adj_bf(int slot, int K, int os, int vs, int ot, int vt, int Kp,
                          const double* dBF, double* dfT, double* dt2st, cudaStream_t st) {
  int64_t n = (int64_t)vs * vt * Kp;
  if (n == 0) return cudaSuccess;
  adj_bf<<<grid_for(n), 256, 0, st>>>(slot, K, os, vs, ot, vt, Kp, dBF, dfT, dt2st);
  return cudaGetLastError();
}
cudaError_t launch_adj_at2(const int2* pk, int nslot, int os, int vs, int ot, int vt, int Kp,
                           const double* dAT2, double* dt2st, double* dlT, cudaStream_t st) {
  int64_t n = (int64_t)nslot * vt * Kp;
  if (n == 0) return cudaSuccess;
  adj_at2<<<grid_for(n), 256, 0, st>>>(pk, nslot, os, vs, ot, vt, Kp, dAT2, dt2st, dlT);
  return cudaGetLastError();
}
cudaError_t launch_adj_transpose_block(const double* dblk, int naux, int nbas, int p0, int np,
                                       int q0, int nq, int Qp, double* dB, cudaStream_t st) {
  int64_t n = (int64_t)np * nq * naux;
  if (n == 0) return cudaSuccess;
  adj_transpose_block<<<grid_for(n), 256, 0, st>>>(dblk, naux, nbas, p0, np, q0, nq, Qp, dB);
  return cudaGetLastError();
}
cudaError_t launch_sym_project(const double* G, int naux, int n, double scale, double* out,
                               cudaStream_t st) {
  int64_t m = (int64_t)naux * n * n;
  if (m == 0) return cudaSuccess;
  sym_project<<<grid_for(m), 256, 0, st>>>(G, naux, n, scale, out);
  return cudaGetLastError();
}
cudaError_t launch_antisym_project(const double* G, int o, int v, double scale, double* out,
                                   cudaStream_t st) {
  int64_t m = (int64_t)o * o * v * v;
  if (m == 0) return cudaSuccess;
  antisym_project<<<grid_for(m), 256, 0, st>>>(G, o, v, scale, out);
  return cudaGetLastError();
}
cudaError_t launch_sym_inplace(double* G, int naux, int n, cudaStream_t st) {
  int64_t m = (int64_t)naux * n * (n - 1) / 2;
  if (m == 0) return cudaSuccess;
  sym_inplace<<<grid_for(m), 256, 0, st>>>(G, naux, n);
  return cudaGetLastError();
}
cudaError_t launch_antisym_inplace(double* G, int o, int v, cudaStream_t st) {
  int64_t m = (int64_t)o * o * v * v;
  if (m == 0) return cudaSuccess;
  antisym_inplace_occ<<<grid_for(m), 256, 0, st>>>(G, o, v);
  antisym_inplace_vir<<<grid_for(m), 256, 0, st>>>(G, o, v);
  return cudaGetLastError();
}
cudaError_t launch_adj_transpose_t2ab(const double* dt2ba, int na, int nb, int va, int vb,
                                      double* dt2ab, cudaStream_t st) {
  int64_t m = (int64_t)na * nb * va * vb;
  if (m == 0) return cudaSuccess;
  adj_transpose_t2ab<<<grid_for(m), 256, 0, st>>>(dt2ba, na, nb, va, vb, dt2ab);
  return cudaGetLastError();
}
cudaError_t launch_scale_copy(const double* in, int64_t n, double s, double* out,
                              cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  scale_copy<<<grid_for(n), 256, 0, st>>>(in, n, s, out);
  return cudaGetLastError();
}

}  // namespace lno
