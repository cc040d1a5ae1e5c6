// lno_ot_gemm_sliced_noalloc: the tensor-core contraction of lno_ot_selftest_gemm
// for callers that must not allocate device memory.
//
// Who needs it: host programs whose device memory is owned by their own pool
// or arena (a serving process that reserves HBM up front, a framework whose
// allocator must see every byte), and code paths where a cudaMalloc would
// synchronise the device or is simply not permitted.  This entry point calls
// no cudaMalloc, cudaFree or allocating library routine: its scratch (the
// BF16 slices of both operands, the magnitude reduction, the error flag and
// the problem descriptor) lives in one file-scope device array of
// kScratchBytes, which every GPU that loads the library holds until exit.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress and the device's SM count
// and compute capability, and caches them; make that first call before any
// stream capture.  Every call shares the array and leaves its contents
// behind: the reduction and the flag are cleared at the start of each call,
// and two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it.
//
// Arguments are checked before anything is launched: A, B and C must be
// device (or managed) memory of `device` (else LNO_OT_EDEVICE), and the
// caller's current device is restored on every return.
#include <cstring>
#include <mutex>
#include <string>

#include "common.cuh"

namespace lno {
cudaError_t launch_absmax(const double*, int64_t, unsigned long long*, cudaStream_t);
}  // namespace lno

using namespace lno;

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr size_t kHeader = 256;                     // amax[2], flag, descriptor
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Per-device set-up, done once with the device current.
struct DeviceSetup {
  void* scratch = nullptr;  // device address of g_scratch
  int nsm = 0;
  int cc = 0;               // 10 * major + minor
};
std::mutex g_mu;
DeviceSetup g_setup[kMaxDevices];

int device_setup(int device, DeviceSetup* out) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceSetup& d = g_setup[device];
  if (!d.scratch) {
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
      lno_set_last_error("cudaGetDeviceProperties", e, __FILE__, __LINE__);
      cudaGetLastError();
      return LNO_OT_ECUDA;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
      lno_set_last_error("cudaGetSymbolAddress(g_scratch)", e, __FILE__, __LINE__);
      cudaGetLastError();
      return LNO_OT_ECUDA;
    }
    d.nsm = prop.multiProcessorCount;
    d.cc = 10 * prop.major + prop.minor;
    d.scratch = p;
  }
  *out = d;
  return LNO_OT_OK;
}

// LNO_OT_OK if p is device or managed memory of `device`.
int check_device_ptr(const void* p, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return LNO_OT_EDEVICE;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return LNO_OT_EDEVICE;
  return at.device == device ? LNO_OT_OK : LNO_OT_EDEVICE;
}

// Restores the caller's current device when the call returns.
struct DeviceGuard {
  int prev = -1;
  DeviceGuard() {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// rows x K float64 (row-major) -> S BF16 slices [s][row][Kp], zero for k >= K.
template <int S>
__global__ void slice_rows(const double* __restrict__ in, int rows, int K, int Kp,
                           StoreSlices<S> st) {
  const int64_t n = (int64_t)rows * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % Kp);
    const int64_t r = idx / Kp;
    st(idx, k < K ? in[r * K + k] : 0.0, 1);
  }
}

double pow2_scale_of(double amax) {  // smallest power of two >= amax (1 if amax is 0)
  if (!(amax > 0.0) || !std::isfinite(amax)) return 1.0;
  int e;
  const double m = std::frexp(amax, &e);
  return std::ldexp(1.0, m == 0.5 ? e - 1 : e);
}

template <int S>
cudaError_t launch_slices(const double* in, int rows, int K, int Kp, __nv_bfloat16* out,
                          int64_t stride, double inv, cudaStream_t st) {
  const int64_t n = (int64_t)rows * Kp;
  const int64_t b = (n + 255) / 256;
  const int grid = (int)(b < 4864 ? (b < 1 ? 1 : b) : 4864);
  slice_rows<S><<<grid, 256, 0, st>>>(in, rows, K, Kp, StoreSlices<S>{out, stride, inv, inv});
  return cudaGetLastError();
}

int64_t round_up8(int64_t x) { return (x + 7) / 8 * 8; }
size_t round_up256(size_t x) { return (x + 255) / 256 * 256; }

#define NA_CU(...)                                                              \
  do {                                                                          \
    cudaError_t e__ = (__VA_ARGS__);                                            \
    if (e__ != cudaSuccess) {                                                   \
      lno_set_last_error(#__VA_ARGS__, e__, __FILE__, __LINE__);                \
      cudaGetLastError();                                                       \
      return LNO_OT_ECUDA;                                                      \
    }                                                                           \
  } while (0)

}  // namespace

extern "C" LNO_OT_API int lno_ot_gemm_sliced_noalloc(int device, int S, int M, int N, int K,
                                                     const double* A, const double* B,
                                                     double* Cout, void* stream) {
  if (S < 1 || S > 4 || M <= 0 || N <= 0 || K <= 0 || !A || !B || !Cout) return LNO_OT_EINVAL;
  if (device < 0 || device >= kMaxDevices) return LNO_OT_EDEVICE;
  const int64_t Kp = round_up8(K);
  const int64_t sa = round_up8((int64_t)M * Kp), sb = round_up8((int64_t)N * Kp);
  const size_t abytes = round_up256((size_t)(sa * S) * 2), bbytes = round_up256((size_t)(sb * S) * 2);
  if (kHeader + abytes + bbytes > kScratchBytes) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "lno_ot_gemm_sliced_noalloc: needs %zu bytes of scratch, limit is %zu",
             kHeader + abytes + bbytes, kScratchBytes);
    lno_set_last_error(msg, cudaSuccess, __FILE__, __LINE__);
    return LNO_OT_EINVAL;
  }
  int ndev = 0;
  NA_CU(cudaGetDeviceCount(&ndev));
  if (device >= ndev) return LNO_OT_EDEVICE;
  DeviceGuard guard;
  NA_CU(cudaSetDevice(device));
  for (const void* p : {(const void*)A, (const void*)B, (const void*)Cout}) {
    const int rc = check_device_ptr(p, device);
    if (rc != LNO_OT_OK) return rc;
  }
  DeviceSetup ds;
  {
    const int rc = device_setup(device, &ds);
    if (rc != LNO_OT_OK) return rc;
  }
  if (ds.cc != 103) return LNO_OT_EUNSUPPORTED;
  unsigned char* base = static_cast<unsigned char*>(ds.scratch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long* amax = reinterpret_cast<unsigned long long*>(base);
  int* flag = reinterpret_cast<int*>(base + 16);
  TcProb* desc = reinterpret_cast<TcProb*>(base + 64);
  __nv_bfloat16* a16 = reinterpret_cast<__nv_bfloat16*>(base + kHeader);
  __nv_bfloat16* b16 = reinterpret_cast<__nv_bfloat16*>(base + kHeader + abytes);

  // magnitudes -> power-of-two scales (the array keeps the last call's contents)
  NA_CU(cudaMemsetAsync(base, 0, 64, st));
  NA_CU(launch_absmax(A, (int64_t)M * K, amax, st));
  NA_CU(launch_absmax(B, (int64_t)N * K, amax + 1, st));
  unsigned long long h[2];
  NA_CU(cudaMemcpyAsync(h, amax, sizeof h, cudaMemcpyDeviceToHost, st));
  NA_CU(cudaStreamSynchronize(st));
  double ma, mb;
  std::memcpy(&ma, &h[0], 8);
  std::memcpy(&mb, &h[1], 8);
  const double sca = pow2_scale_of(ma), scb = pow2_scale_of(mb);

  switch (S) {
    case 1:
      NA_CU(launch_slices<1>(A, M, K, (int)Kp, a16, sa, 128.0 / sca, st));
      NA_CU(launch_slices<1>(B, N, K, (int)Kp, b16, sb, 128.0 / scb, st));
      break;
    case 2:
      NA_CU(launch_slices<2>(A, M, K, (int)Kp, a16, sa, 128.0 / sca, st));
      NA_CU(launch_slices<2>(B, N, K, (int)Kp, b16, sb, 128.0 / scb, st));
      break;
    case 3:
      NA_CU(launch_slices<3>(A, M, K, (int)Kp, a16, sa, 128.0 / sca, st));
      NA_CU(launch_slices<3>(B, N, K, (int)Kp, b16, sb, 128.0 / scb, st));
      break;
    default:
      NA_CU(launch_slices<4>(A, M, K, (int)Kp, a16, sa, 128.0 / sca, st));
      NA_CU(launch_slices<4>(B, N, K, (int)Kp, b16, sb, 128.0 / scb, st));
  }
  CUtensorMap mA[2], mB[2];
  int rc = make_operand_map(&mA[0], a16, Kp, M, S, sa, 128);
  if (rc == LNO_OT_OK) rc = make_operand_map(&mB[0], b16, Kp, N, S, sb, sliced_product_bn(S));
  if (rc != LNO_OT_OK) return rc;
  mA[1] = mA[0];
  mB[1] = mB[0];
  TcProb p{};
  p.nseg = 1;
  p.seg[0] = TcSeg{0, 0, 0, 0, K, 0};
  p.out = Cout;
  NA_CU(cudaMemcpyAsync(desc, &p, sizeof p, cudaMemcpyHostToDevice, st));
  const double scale = sca * scb * std::ldexp(1.0, -14);
  NA_CU(launch_sliced_product(S, mA, mB, desc, M, N, scale, flag, ds.nsm, st, tc_normal()));
  int hflag = 0;
  NA_CU(cudaMemcpyAsync(&hflag, flag, sizeof hflag, cudaMemcpyDeviceToHost, st));
  NA_CU(cudaStreamSynchronize(st));
  return hflag ? LNO_OT_ETIMEOUT : LNO_OT_OK;
}
