// norm_static.cu -- residual norms without any device allocation.
//
// For callers that cannot allocate device memory at all, e.g. code running
// inside a memory pool it does not own, a process whose allocator is locked
// after start-up, or an embedded host that forbids cudaMalloc once it has
// started: mg_residual_norm_static() computes the same defect norms as the
// solver's own reduction from caller-owned arrays only.  Its scratch (one
// partial sum and one partial maximum per interior grid row) lives in the
// file-scope device array below, sized for at most MAX_ROWS interior rows.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "mg_internal.h"

namespace tmg {

namespace {

constexpr int MAX_ROWS = 16384;  // interior rows the scratch holds (ny - 1 <= MAX_ROWS)
constexpr int MAX_DEVICES = 64;
constexpr int THREADS = 256;

// Per-row partials: [0, MAX_ROWS) sums of squares of f - L u, [MAX_ROWS,
// 2 MAX_ROWS) their maxima, then the same two for f.  Shared by every call on
// a device; every entry a call reads was written earlier in that same call.
static __device__ __align__(256) double g_row_scratch[4 * MAX_ROWS];

// Device address of g_row_scratch per device: looked up by every call made
// outside a stream capture (so that a context re-created after
// cudaDeviceReset gets its own address), and taken from this cache by calls
// made while their stream is being captured.
std::mutex g_addr_mutex;
double *g_addr[MAX_DEVICES] = {};

// max that propagates NaN (fmax would drop it): once a NaN has entered m it
// stays, so a non-finite residual shows in the max norms as in the sums.
__device__ __forceinline__ double max_nan(double m, double v) { return (v > m || v != v) ? v : m; }

__device__ __forceinline__ void reduce2(double &s, double &m) {
  __shared__ double ss[THREADS], sm[THREADS];
  ss[threadIdx.x] = s; sm[threadIdx.x] = m;
  __syncthreads();
  for (int h = THREADS / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      ss[threadIdx.x] += ss[threadIdx.x + h];
      sm[threadIdx.x] = max_nan(sm[threadIdx.x], sm[threadIdx.x + h]);
    }
    __syncthreads();
  }
  s = ss[0]; m = sm[0];
  __syncthreads();
}

// One CTA per interior row j: sums of r^2 and f^2 and maxima of |r|, |f|
// over the row, r = f - L u.
__global__ void __launch_bounds__(THREADS) row_norms(int nx, const double *__restrict__ W,
                                                     const double *__restrict__ E, const double *__restrict__ S,
                                                     const double *__restrict__ N, const double *__restrict__ u,
                                                     const double *__restrict__ f, double *__restrict__ scratch) {
  const int j = blockIdx.x + 1, nx1 = nx + 1;
  double rs = 0.0, rm = 0.0, fs = 0.0, fm = 0.0;
  for (int i = threadIdx.x + 1; i < nx; i += THREADS) {
    const size_t p = (size_t)j * nx1 + i;
    const double w = W[i], e = E[i], s = S[j], n = N[j];
    const double lu = w * u[p - 1] + e * u[p + 1] + s * u[p - nx1] + n * u[p + nx1] - ((w + e) + (s + n)) * u[p];
    const double r = f[p] - lu;
    rs += r * r; rm = max_nan(rm, fabs(r));
    fs += f[p] * f[p]; fm = max_nan(fm, fabs(f[p]));
  }
  reduce2(rs, rm);
  reduce2(fs, fm);
  if (threadIdx.x == 0) {
    scratch[blockIdx.x] = rs;
    scratch[MAX_ROWS + blockIdx.x] = rm;
    scratch[2 * MAX_ROWS + blockIdx.x] = fs;
    scratch[3 * MAX_ROWS + blockIdx.x] = fm;
  }
}

// One CTA: the rows in index order (deterministic), then the four results.
__global__ void __launch_bounds__(THREADS) rows_total(int rows, const double *__restrict__ scratch,
                                                      double *__restrict__ out) {
  double rs = 0.0, rm = 0.0, fs = 0.0, fm = 0.0;
  for (int k = threadIdx.x; k < rows; k += THREADS) {
    rs += scratch[k]; rm = max_nan(rm, scratch[MAX_ROWS + k]);
    fs += scratch[2 * MAX_ROWS + k]; fm = max_nan(fm, scratch[3 * MAX_ROWS + k]);
  }
  reduce2(rs, rm);
  reduce2(fs, fm);
  if (threadIdx.x == 0) { out[0] = rs; out[1] = rm; out[2] = fs; out[3] = fm; }
}

}  // namespace
}  // namespace tmg

using namespace tmg;

extern "C" mg_status mg_residual_norm_static(int64_t nx, int64_t ny, const double *W, const double *E,
                                             const double *S, const double *N, const double *u, const double *f,
                                             double *out, void *stream) {
  if (!W || !E || !S || !N || !u || !f || !out) return MG_ERR_INVALID_ARG;
  if (nx < 2 || ny < 2 || nx > 1048576) return MG_ERR_SIZE;
  if (ny - 1 > MAX_ROWS) {
    char msg[160];
    std::snprintf(msg, sizeof(msg), "mg_residual_norm_static: %lld interior rows exceed the static scratch (%d rows)",
                  (long long)(ny - 1), MAX_ROWS);
    set_error_text(msg);
    return MG_ERR_SIZE;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_error("cudaGetDevice", e); return MG_ERR_CUDA; }
  if (dev < 0 || dev >= MAX_DEVICES) return MG_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) { set_error("cudaStreamIsCapturing", e); return MG_ERR_CUDA; }
  double *scratch;
  {
    // set-up, with the device current: the host-side name g_row_scratch is
    // only a stand-in, the kernels need its device address.  Looked up on
    // every call outside a capture; a captured call uses the address an
    // earlier uncaptured call on this device found.
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_row_scratch);
      if (e != cudaSuccess) { set_error("cudaGetSymbolAddress(row scratch)", e); return MG_ERR_CUDA; }
      g_addr[dev] = static_cast<double *>(p);
    } else if (!g_addr[dev]) {
      set_error_text("mg_residual_norm_static: the first call on a device must come before any stream capture");
      return MG_ERR_INVALID_ARG;
    }
    scratch = g_addr[dev];
  }
  const int rows = (int)(ny - 1);
  row_norms<<<rows, THREADS, 0, s>>>((int)nx, W, E, S, N, u, f, scratch);
  rows_total<<<1, THREADS, 0, s>>>(rows, scratch, out);
  count_launch(2);
  e = cudaGetLastError();
  if (e != cudaSuccess) { set_error("residual norm (static scratch)", e); return MG_ERR_CUDA; }
  return MG_OK;
}
