/*
 * lno_ot.h -- C ABI of the GB300 (sm_103a) open-shell LNO domain (T) library.
 *
 * The library computes the perturbative triples energy E(T) of one local
 * natural orbital domain (one "local interacting subspace", LIS) from
 * semicanonical high-spin orbitals: arXiv 2311.10048, Sec. 2.1, eq
 * cim_pt_energy, evaluated over restricted occupied triplets in the four spin
 * cases aaa, aab, abb, bbb, with the disconnected term V:
 *
 *   E(T) = sum_cases sum_{restricted ijk} sum_{restricted abc} W (W + V) / D,
 *   W = t D (connected triples times denominator), V from T1 and <jk||bc>
 *   (plus f_ia and the doubles when the domain carries an f_ov block),
 *   D = e_i + e_j + e_k - e_a - e_b - e_c.
 *
 * Restricted ranges: aaa/bbb i<j<k and a<b<c; aab i<j (alpha), K (beta),
 * a<b (alpha), C (beta); abb I<J (beta), k (alpha), A<B (beta), c (alpha).
 * The four-index integrals are assembled from density-fitted three-centre
 * factors, (pq|rs) = sum_Q B^Q_pq B^Q_rs (Sec. 3.3, eqs ed_eri/ed_df_int with
 * B = I L^-T already applied), one auxiliary index shared by both spins as the
 * mixed-spin integrals require (Sec. 3.6).
 *
 * General conventions
 *  - Every function returns LNO_OT_OK (0) or a negative lno_ot_status code;
 *    lno_ot_strerror() names it.  Nothing is thrown and nothing aborts.
 *  - Domain arrays are DEVICE memory on the context's device, owned by the
 *    caller, read only (except gradient outputs), never freed by the library.
 *  - All work is ordered on the context's stream.  The energy calls return
 *    after the results have reached host memory.
 *  - Not thread safe per context: one context must not be used by two host
 *    threads at once.  Different contexts are independent.
 */
#ifndef LNO_OT_H
#define LNO_OT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LNO_OT_API __attribute__((visibility("default")))
#else
#define LNO_OT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LNO_OT_OK = 0,
  LNO_OT_EINVAL = -1,       /* bad sizes, null required pointer, nocc[1] > nocc[0] */
  LNO_OT_EDEVICE = -2,      /* a pointer is not device memory of the context's device */
  LNO_OT_ENOMEM = -3,       /* device workspace could not be allocated */
  LNO_OT_ECUDA = -4,        /* a CUDA runtime/driver call failed */
  LNO_OT_ETIMEOUT = -5,     /* a bounded device-side wait gave up */
  LNO_OT_EUNSUPPORTED = -6  /* option or input not supported by this build */
} lno_ot_status;

/* Arithmetic of the W contractions (Sec. 3.7, the (T) step).
 *  FP64    plain float64 on the CUDA cores for everything (comparator path).
 *  BF16X3  tensor cores (tcgen05, BF16 inputs, FP32 accumulate): every
 *          float64 operand is split into 2 BF16 slices with an exact power of
 *          two scale; 3 slice products per multiply.  FP64 is kept for the
 *          denominators' orbital energies and the compensated energy sum.
 *  BF16X6  as BF16X3 with 3 slices per operand and 6 slice products (about
 *          8 more significant bits per operand).
 *  BF16X10 4 slices per operand and 10 slice products (8 bits more again):
 *          the accurate mode for large domains, where the BF16X6 truncation
 *          adds up over ~1e5 triplets; about 1.7x the contraction time.
 *  BF16X15 5 slices per operand and 15 slice products, with the DF assembly
 *          on 5 slices too: 8 bits more again than BF16X10 in both steps, at
 *          about 1.5x its contraction time.  The reference mode against which
 *          the domain-total error of the faster modes is measured when a
 *          float64 run of a whole domain is too slow.
 *  TF32    tensor cores on their TF32 path (kind::tf32): every float64
 *          operand split into 2 TF32 slices of 11 significant bits with an
 *          exact power-of-two scale, 3 slice products per multiply, one FP32
 *          accumulator per weight class.  Unlike the BF16 modes the class
 *          sums are not exact (11-bit x 11-bit products overflow the FP32
 *          significand after a few terms), so the accumulation rounds; it is
 *          about as fast as BF16X6 (TF32 runs at half the BF16 rate) and less
 *          accurate: provided for comparison, with its error measured. */
typedef enum {
  LNO_OT_FP64 = 0,
  LNO_OT_BF16X3 = 1,
  LNO_OT_TF32 = 2,
  LNO_OT_BF16X6 = 3,
  LNO_OT_BF16X10 = 4,
  LNO_OT_BF16X15 = 5
} lno_ot_precision;

typedef struct lno_ot_ctx lno_ot_ctx; /* opaque: device, stream, workspace */

typedef struct {
  int device;             /* CUDA device ordinal */
  int precision;          /* lno_ot_precision */
  void* stream;           /* cudaStream_t to order all work on; NULL = the
                             legacy default stream */
  size_t workspace_bytes; /* upper bound on device workspace; 0 = no bound */
  const char* tune_cache; /* NULL, or a tuning table written by the autotuner
                             (paper_2311_10048_gb300/tune.py): text lines
                             "vmax bn group_cap" giving, per bucket of
                             virtual-space size, the tile width of the W
                             contraction (64, 96, 128 or 256 where the
                             precision has that variant; 0 = its default) and
                             the cap
                             on triplets per contraction launch.  Lines
                             starting with '#' are comments.  Unreadable
                             file: lno_ot_init returns LNO_OT_EINVAL. */
  int keep_operands;      /* 0: every lno_ot_energy call builds and frees its
                             own DF blocks and contraction operands.  1: the
                             context keeps those of the last domain, built for
                             ALL its triplets, and a later lno_ot_energy on the
                             same arrays (same pointers, sizes and precision;
                             e.g. another trip_sel block) only runs the
                             contractions and the energy kernels.  The caller
                             must not change the arrays' contents while they
                             are kept (lno_ot_release frees them).  Costs the
                             whole domain's operands in device memory; if they
                             do not fit the call runs uncached.  Closed-shell
                             calls (spin-flip images) are never cached. */
} lno_ot_options;

/* One domain.  Orbitals of each spin are ordered occupied first (ascending
 * energy) then virtual; nvir[s] = nbas - nocc[s].  All pointers are device
 * float64 arrays in C order:
 *   B[s]    [naux][nbas][nbas]   symmetric in (p,q)
 *   eps[s]  [nbas]               semicanonical orbital energies (Eh)
 *   t1[s]   [nocc[s]][nvir[s]]   t^a_i
 *   t2aa    [na][na][nva][nva]   t^{ab}_{ij}, antisymmetric in (i,j), (a,b)
 *   t2bb    [nb][nb][nvb][nvb]   t^{AB}_{IJ}
 *   t2ab    [na][nb][nva][nvb]   t2ab[i][J][a][B] = t^{aB}_{iJ}
 * High spin: 0 <= nocc[1] <= nocc[0] <= nbas.
 *
 * Closed-shell domains (no singly occupied orbital): when both spins are given
 * by the same arrays (B[0] == B[1], eps[0] == eps[1], t1[0] == t1[1],
 * t2aa == t2bb, fov[0] == fov[1] as pointers, nocc[0] == nocc[1]), no
 * trip_sel is set, and t2ab[i][J][a][B] equals t2ab[J][i][B][a] to within
 * 1e-12 of the largest |t2ab| for every element (checked on the device), E_bbb
 * and E_abb are the spin-flip images of E_aaa and E_aab, triplet for triplet;
 * only the spin-up cases are computed and the others are copies.  Otherwise
 * all four cases run.
 *
 * Optional:
 *   fov[s]        [nocc[s]][nvir[s]] f_ia: the occupied-virtual block of the
 *                 Fock matrix in the semicanonical basis, non-zero for a
 *                 restricted open-shell reference (Sec. 3.3, eq
 *                 off_diagonal_fock).  It adds the disconnected term
 *                 P(i/jk) P(a/bc) f_ia t^{bc}_{jk} to V (the T1 term with
 *                 f_ia for t^a_i and the doubles amplitude for <jk||bc>).
 *                 NULL for both spins = no such term; a NULL spin next to a
 *                 non-NULL one counts as zero.
 *   e_trip[c]     device float64 output, one value per computed triplet of
 *                 case c (0 aaa, 1 aab, 2 abb, 3 bbb): the triplet's
 *                 contribution sum_{restricted abc} W (W + V) / D.  NULL = not
 *                 requested.
 *   trip_sel[c]   HOST int64 array of n_sel[c] triplet indices (into the
 *                 lexicographic order of the restricted triplets of case c:
 *                 aaa (i,j,k), aab (i,j,K), abb (I,J,k), bbb (I,J,K));
 *                 NULL = all triplets.  Only the selected triplets are
 *                 computed and summed; e_trip[c][q] belongs to trip_sel[c][q].
 *   n_sel[c]      length of trip_sel[c] (ignored when it is NULL).
 *   e_orb[s]      device float64 output [nocc[s]]: the orbital contributions
 *                 dE_i / dE_I of eq cim_pt_energy (E(T) = sum_i dE_i +
 *                 sum_I dE_I), i.e. 1/3 of each same-spin triplet to each of
 *                 its orbitals, and of each mixed triplet 1/4 to each of its
 *                 two same-spin orbitals and 1/2 to the third; over the
 *                 computed (selected) triplets only.  NULL = not requested. */
typedef struct {
  int nbas, naux, nocc[2];
  const double* B[2];
  const double* eps[2];
  const double* t1[2];
  const double* t2aa;
  const double* t2bb;
  const double* t2ab;
  const double* fov[2];
  double* e_trip[4];
  const int64_t* trip_sel[4];
  int64_t n_sel[4];
  double* e_orb[2];
} lno_ot_domain;

/* e = {aaa, aab, abb, bbb, total} in Eh; status as lno_ot_status. */
typedef struct {
  double e[5];
  int status;
} lno_ot_result;

/* Gradient outputs g = gE * dE/d(input), device float64, caller owned, same
 * layouts as the inputs, overwritten.  A NULL member skips that gradient.
 * Gradients of inputs with symmetry are projected onto it: dB symmetric in
 * (p,q), dt2aa/dt2bb antisymmetric in (i,j) and in (a,b), so that
 * sum g * delta is the directional derivative for any symmetry-respecting
 * perturbation delta.  dfov[s] [nocc[s]][nvir[s]] is the gradient with
 * respect to the f_ov block; it is defined (and returned) also when the
 * domain has no f_ov block, as the derivative at f_ov = 0. */
typedef struct {
  double* dB[2];
  double* deps[2];
  double* dt1[2];
  double* dt2aa;
  double* dt2bb;
  double* dt2ab;
  double* dfov[2];
} lno_ot_grad;

/* Timings and work counts of the last lno_ot_energy call on a context. */
typedef struct {
  double ms_total;          /* call wall time on the stream (CUDA events) */
  double ms_stage;          /* input checks, layout and DF integral assembly */
  double ms_contract;       /* W contraction kernels (sum of launches) */
  double ms_energy;         /* W/V assembly + energy reduction kernels */
  double flops_algorithmic; /* W contraction flops over the computed triplets,
                               counting every (b,c) output (full n_v^2) */
  double flops_executed;    /* method flops the kernels execute (antisymmetric
                               outputs computed once), one product each */
  double tensor_flops;      /* tensor-core flops issued incl. slice products */
  int64_t contract_launches;/* W contraction kernel launches */
  int64_t energy_launches;  /* energy kernel launches */
  int64_t other_launches;   /* all other kernel launches */
  int64_t triplets;         /* triplets computed */
  int64_t elements;         /* restricted (abc) elements summed */
} lno_ot_stats;

/* Create a context on opt->device.  *ctx is set only on success. */
LNO_OT_API int lno_ot_init(lno_ot_ctx** ctx, const lno_ot_options* opt);

/* Release the context and its device buffers (after its stream drained). */
LNO_OT_API void lno_ot_destroy(lno_ot_ctx* ctx);

/* Free the operands kept by options.keep_operands (no-op when none are
 * kept); the next lno_ot_energy builds them again. */
LNO_OT_API int lno_ot_release(lno_ot_ctx* ctx);

/* E(T) of one domain (eq cim_pt_energy, all occupied orbitals of the
 * domain).  out: host memory; out->status mirrors the return value. */
LNO_OT_API int lno_ot_energy(lno_ot_ctx* ctx, const lno_ot_domain* dom, lno_ot_result* out);

/* E(T) of ndom independent domains (the per-LMO domains of Sec. 3, eq
 * lno_ccsdpt_energy sums them).  out[d] gets domain d; per-domain status in
 * out[d].status; returns the first error (or LNO_OT_OK). */
LNO_OT_API int lno_ot_energy_batched(lno_ot_ctx* ctx, int ndom, const lno_ot_domain* doms,
                          lno_ot_result* out);

/* Adjoint of lno_ot_energy: g = gE * dE(T)/d(B, eps, T1, T2), W recomputed
 * per triplet (never stored).  Operands, energy adjoint and layout adjoints
 * run in float64; the contractions (the DF assembly, the X recompute, the
 * contraction and DF adjoints) run in float64 in an LNO_OT_FP64 context and on
 * the tensor cores otherwise (4 exact BF16 slices of each float64 operand with
 * a power-of-two scale, float64 output of the exact class sums).  Stats of the
 * call (lno_ot_last_stats): ms_total wall clock, ms_stage staging and operand
 * builds, ms_contract the contraction kernels (tensor-core context), ms_energy
 * the energy adjoint kernels. */
LNO_OT_API int lno_ot_backward(lno_ot_ctx* ctx, const lno_ot_domain* dom, double gE,
                    lno_ot_grad* g);

/* Central-LMO share of E(T) in the Laplace form (Sec. 3.7, eqs
 * laplace_transform and local_pt).  The denominators are replaced by the
 * quadrature 1/Delta ~ sum_q w_q exp(-Delta s_q) (Delta = -D > 0), after
 * which the sum over the first occupied index is a trace and can be taken in
 * a basis of localized orbitals.  For each central orbital u (row l of U: its
 * coefficients in the semicanonical occupied orbitals of spin `spin`) the
 * call returns
 *
 *   dE[l] = -(1/3) sum_q w_q [ sum_{j<k, a<b<c} Wbar (Wbar + Vbar)_{u j k}
 *                             + sum_{j, K, a<b, C} ... + sum_{J<K, A<B, c} ... ]
 *
 * the i' (spin 0) or I' (spin 1) terms of eq local_pt: every triplet that
 * holds u, with 1/3 of it to u, and the bars exp(+e_p s_q/2) per occupied and
 * exp(-e_x s_q/2) per virtual index.  The share of a spatial LMO is
 * dE of its spin-up part plus dE of its spin-down part.  Over a complete
 * orthonormal set of central orbitals of both spins the shares add up to the
 * Laplace-quadrature E(T) of the domain, which tends to E(T) as the
 * quadrature gets accurate.  Cost O(nq no^2 nv^4) per central orbital.  The
 * domain's trip_sel, e_trip and e_orb members are ignored.  Runs in the
 * context's precision; results in host memory on return. */
typedef struct {
  int nq;                 /* quadrature points, 1..256 */
  const double* s;        /* HOST [nq] points s_q > 0 (1/Eh) */
  const double* w;        /* HOST [nq] weights w_q */
  int spin;               /* 0: central orbitals of spin up, 1: spin down */
  int nlmo;               /* number of central orbitals (>= 0) */
  const double* U;        /* DEVICE [nlmo][nocc[spin]] coefficients (rows) */
  double* dE;             /* HOST out [nlmo] (Eh) */
} lno_ot_central;

LNO_OT_API int lno_ot_energy_central(lno_ot_ctx* ctx, const lno_ot_domain* dom,
                                     const lno_ot_central* c);

/* Quadrature for the Laplace form (host only, no device work): the fewest
 * points n <= nmax (<= 32) whose sum_q w_q exp(-x s_q) approximates 1/x with a
 * largest relative error <= tol on [xmin, xmax] (0 < xmin < xmax; the range of
 * Delta over the domain's triples).  The paper fixes the tolerance (laptol =
 * 1e-2, Table thresholds, giving 3-4 points) but not the construction: here a
 * least-squares fit of the relative error, reweighted towards the minimax
 * fit, from a trapezoid start.  s, w: HOST [nmax]; *nq = n.  Returns
 * LNO_OT_EUNSUPPORTED if nmax points do not reach tol. */
LNO_OT_API int lno_ot_laplace_quadrature(double xmin, double xmax, double tol, int nmax,
                                         double* s, double* w, int* nq);

/* Natural auxiliary functions (Sec. 3.6, eq naf_w): compresses the shared
 * auxiliary index of the DF factors before the integrals are assembled.
 *   W^s_XY = sum_{p<=q} B^X_pq B^Y_pq  (s = up, down),  W = (W^up + W^down)/2,
 * the eigenvectors of W with eigenvalue > eps_naf (the paper's default is
 * 1e-2 Eh) become the NAFs, in descending eigenvalue order, and
 *   B_out[s][X'][p][q] = sum_X V[X][X'] B[s][X][p][q]
 * for the *naux_out kept X'.  One auxiliary basis serves both spins, as the
 * mixed-spin integrals need.  Uses dom->nbas, naux and B only.  B_out[s]:
 * DEVICE [naux][nbas][nbas] caller-owned (the first *naux_out blocks are
 * written; may be dom->B[s] itself).  eigenvalues: HOST [naux] (all
 * eigenvalues of W, descending) or NULL.  Runs in float64 on the CUDA cores
 * (pair-packed contraction, cyclic Jacobi rotations replayed as a CUDA
 * graph, contraction), whatever the context's precision; synchronous. */
LNO_OT_API int lno_ot_naf(lno_ot_ctx* ctx, const lno_ot_domain* dom, double eps_naf,
                          double* B_out[2], int* naux_out, double* eigenvalues);

/* Stats of the last lno_ot_energy on this context. */
LNO_OT_API int lno_ot_last_stats(const lno_ot_ctx* ctx, lno_ot_stats* st);

/* Static description of a status code (never NULL). */
LNO_OT_API const char* lno_ot_strerror(int code);

/* Diagnostic (no counterpart in the paper): the tensor-core contraction
 * kernel of the W step on one plain product, C[n][m] = sum_k A[m][k] B[n][k]
 * for device float64 A [M][K], B [N][K], C [N][M] (C written), with S BF16
 * slices per operand (S = 1..5; the W step uses S = 2..5, the DF assembly
 * S = 4 or 5).  Synchronous on `stream` (cudaStream_t, NULL = legacy default).
 * Returns LNO_OT_EUNSUPPORTED on devices other than sm_103. */
LNO_OT_API int lno_ot_selftest_gemm(int device, int S, int M, int N, int K, const double* A,
                                    const double* B, double* C, void* stream);

/* Diagnostic (no counterpart in the paper): checks the bounded device waits
 * of the contraction kernel.  Runs one 128 x 256 tile with the kernel's test
 * hook that issues no copy, so its first wait for operand data can only end
 * by the time limit `wait_cycles` (1000 .. the library's normal limit of
 * 4e9 cycles); the kernel then records which wait gave up, releases its TMEM
 * and returns, and the context stays usable.  Returns LNO_OT_ETIMEOUT when
 * the bounded wait behaved as designed (*code, if not NULL, = the kernel's
 * code of the wait that gave up: 3 MMA thread, 6 epilogue), LNO_OT_OK if no
 * wait gave up, another status on a CUDA failure or bad argument.  Allocates
 * its own small scratch; synchronous on `stream`. */
LNO_OT_API int lno_ot_selftest_timeout(int device, long long wait_cycles, int* code,
                                       void* stream);

/* Diagnostic (no counterpart in the paper): the same check for the energy
 * kernel's TMA staging (mixed spin).  One 16^3 tile of zeros with the kernel's
 * test hook that issues no copy, so its first stage wait can only end by the
 * limit `wait_cycles` (1000 .. 4e9); the kernel records code 7 and leaves with
 * nothing in flight.  Returns LNO_OT_ETIMEOUT when the wait gave up as
 * designed (*code = 7), LNO_OT_OK if it did not, another status on a CUDA
 * failure or bad argument.  Allocates its own scratch; synchronous on
 * `stream`. */
LNO_OT_API int lno_ot_selftest_energy_timeout(int device, long long wait_cycles, int* code,
                                              void* stream);

/* The same product as lno_ot_selftest_gemm (same slicing, same kernel, same
 * result) for callers that must not allocate device memory: programs whose
 * HBM is owned by their own pool or arena, or code paths where a cudaMalloc
 * would synchronise the device or is not permitted.  No counterpart in the
 * paper.  It calls no cudaMalloc/cudaFree or allocating library routine; its
 * scratch is one static device array of 64 MiB held by every GPU that loads
 * the library.  Operands must fit: 256 B + sum over A and B of
 * S * ceil8(rows * ceil8(K)) * 2 bytes (each part rounded up to 256 B)
 * <= 64 MiB, else LNO_OT_EINVAL (lno_ot_last_error() says how much is needed).
 * A, B and C must be device (or managed) memory of `device`, else
 * LNO_OT_EDEVICE before anything runs; the caller's current device is restored
 * on return.  The first call on a device looks up the array's address and the
 * device's properties (make it before any stream capture).  Every call reuses the array and clears what must
 * start at zero; calls that overlap on the GPU race on it.  Synchronous on
 * `stream` (NULL = legacy default stream). */
LNO_OT_API int lno_ot_gemm_sliced_noalloc(int device, int S, int M, int N, int K, const double* A,
                                          const double* B, double* C, void* stream);

/* Text of the last CUDA failure seen by this host thread ("" if none). */
LNO_OT_API const char* lno_ot_last_error(void);

/* Library version string, e.g. "lno_ot 0.1 sm_103a". */
LNO_OT_API const char* lno_ot_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LNO_OT_H */
