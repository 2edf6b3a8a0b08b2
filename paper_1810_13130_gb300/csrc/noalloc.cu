// Allocation-free dipole reduction: tdks_dipole_noalloc.
//
// For callers that cannot allocate device memory: programs whose device memory
// is owned by another allocator with a fixed budget, and code paths where an
// allocation is not allowed once running, such as a real-time propagation loop
// after start-up.  It needs no context.  Every call synchronizes its stream.
//
// Its scratch -- the per-block partial sums, the 3 results, and copies of the
// breakpoints and the Gauss rule -- lives in one file-scope __device__ array of
// fixed size that every GPU loading this library keeps until the process exits.
// Nothing in the array is read before the same call has written it, so it needs
// no clearing; every call shares it, so calls that overlap on the GPU (other
// streams, other host threads) race and must be serialized by the caller.
#include <cmath>
#include <mutex>

#include "tdks_internal.h"

namespace {

constexpr int kNB = 608;          // reduction blocks (4 x 152 SMs)
constexpr int kThreads = 256;
constexpr int kMaxDoubles = 16384;
constexpr int kOffRes = 3 * kNB;  // 3 results after the partials
constexpr int kOffData = 3 * kNB + 8;

static __device__ __align__(256) double g_noalloc_scratch[kMaxDoubles];

std::mutex g_setup_mutex;
// Device address of the array, per device ordinal, looked up by the first call on
// that device and kept for the life of the process (stale after cudaDeviceReset).
double* g_scratch_ptr[128] = {nullptr};

// Gauss-Legendre rule with 2 <= n <= 9 points in fixed-size storage (Newton on
// the Legendre three-term recurrence, long double).
void legendre_n(int n, long double t, long double* P, long double* dP) {
  long double p0 = 1.0L, p1 = t;
  for (int k = 1; k < n; ++k) {
    const long double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = n * (p0 - t * p1) / (1.0L - t * t);
}

void gauss_rule(int n, double* x, double* w) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    long double t = -cosl(pi * (i + 0.75L) / (n + 0.5L)), P, dP;
    for (int it = 0; it < 100; ++it) {
      legendre_n(n, t, &P, &dP);
      const long double step = P / dP;
      t -= step;
      if (fabsl(step) < 1e-30L) break;
    }
    legendre_n(n, t, &P, &dP);
    x[i] = (double)t;
    w[i] = (double)(2.0L / ((1.0L - t * t) * dP * dP));
  }
}

// Same reduction as the context's dipole kernel, with geometry read from scratch.
__global__ void k_dipole_noalloc(double* scratch, int nx, int ny, int nz, int P1,
                                 const double* __restrict__ rho, long long n) {
  __shared__ double red[3][kThreads / 32];
  const double* X = scratch + kOffData;
  const double* Y = X + nx + 1;
  const double* Z = Y + ny + 1;
  const double* eta = Z + nz + 1;
  const double* w = eta + P1;
  const int P2 = P1 * P1, P3 = P2 * P1;
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / P3;
    const int q = (int)(i - e * P3);
    const int qx = q % P1, qy = (q / P1) % P1, qz = q / P2;
    const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((long long)nx * ny));
    const double hx = X[ex + 1] - X[ex], hy = Y[ey + 1] - Y[ey], hz = Z[ez + 1] - Z[ez];
    const double m = 0.125 * hx * hy * hz * w[qx] * w[qy] * w[qz] * rho[i];
    acc[0] += m * (X[ex] + 0.5 * (eta[qx] + 1.0) * hx);
    acc[1] += m * (Y[ey] + 0.5 * (eta[qy] + 1.0) * hy);
    acc[2] += m * (Z[ez] + 0.5 * (eta[qz] + 1.0) * hz);
  }
  for (int d = 0; d < 3; ++d) {
    double v = acc[d];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[d][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s += red[threadIdx.x][k];
    scratch[threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_dipole_noalloc_sum(double* scratch, int nb) {
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += scratch[threadIdx.x * nb + k];
    scratch[kOffRes + threadIdx.x] = s;
  }
}

}  // namespace

extern "C" tdks_status tdks_dipole_noalloc(const double* rho_q_dev, int nx, int ny, int nz,
                                           const double* X, const double* Y, const double* Z,
                                           int p, void* stream, double d_host[3]) {
  if (!rho_q_dev || !X || !Y || !Z || !d_host) return TDKS_ERR_ARG;
  if (nx < 1 || ny < 1 || nz < 1 || p < 1 || p > TDKS_MAX_P1 - 1) return TDKS_ERR_ARG;
  const int P1 = p + 1;
  const long long need = (long long)kOffData + (nx + 1) + (ny + 1) + (nz + 1) + 2 * P1;
  if (need > kMaxDoubles) return TDKS_ERR_ARG;   // nx + ny + nz larger than the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return TDKS_ERR_CUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return TDKS_ERR_CUDA;
      }
      g_scratch_ptr[dev] = static_cast<double*>(ptr);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  double rule[2 * TDKS_MAX_P1];
  gauss_rule(P1, rule, rule + P1);
  double* data = scratch + kOffData;
  if (cudaMemcpyAsync(data, X, (nx + 1) * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(data + nx + 1, Y, (ny + 1) * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(data + nx + ny + 2, Z, (nz + 1) * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(data + nx + ny + nz + 3, rule, 2 * P1 * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return TDKS_ERR_CUDA;
  const long long n = (long long)nx * ny * nz * P1 * P1 * P1;
  long long nb = (n + kThreads - 1) / kThreads;
  nb = nb < kNB ? (nb < 1 ? 1 : nb) : kNB;
  k_dipole_noalloc<<<(int)nb, kThreads, 0, s>>>(scratch, nx, ny, nz, P1, rho_q_dev, n);
  k_dipole_noalloc_sum<<<1, 32, 0, s>>>(scratch, (int)nb);
  if (cudaGetLastError() != cudaSuccess) return TDKS_ERR_CUDA;
  if (cudaMemcpyAsync(d_host, scratch + kOffRes, 3 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return TDKS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TDKS_ERR_CUDA;
  return TDKS_OK;
}
