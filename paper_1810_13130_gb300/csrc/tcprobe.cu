// One-dimensional contraction stage of the element kernels (Sec. VI.A sum
// factorization) in four arithmetic forms, for measuring which one the element
// kernels should use.  Each line of P1 values (a 1-D line of an element's nodal or
// Gauss-point values) is multiplied by a P1 x P1 operator M (B, B^T or Kq of the
// element kernels) `reps` times in a row, all in shared memory, so the measured time
// is that of the arithmetic and the shared-memory traffic of the stage:
//   0  CUDA cores, FP32 fused multiply-adds
//   1  CUDA cores, double-float (two-product and two-sum; ~48-bit results)
//   2  tensor cores, BF16 operands with FP32 accumulation (mma.sync m16n8k16): the
//      operand rounding of a BF16 tensor-core contraction
//   3  tensor cores, three TF32 products per product (hi*hi + hi*lo + lo*hi, mma.sync
//      m16n8k8): FP32-level products, FP32 accumulation
// The tensor-core forms take a tile of 16 lines as the M dimension, the P1 inputs as
// K (padded with zeros to 16 or 8) and the P1 outputs as N (padded to 8).
#include <cuda_bf16.h>

#include <cstring>

#include "df64.cuh"
#include "tdks_internal.h"

namespace {

using tdks::Df;

constexpr int kThreads = 128;   // four warps
constexpr int kLines = 512;     // lines per CTA (each warp owns 128 = 8 tiles of 16)
constexpr int kMaxP1 = 8;

struct Op {
  double m[kMaxP1 * kMaxP1];    // M[q][i], row-major
};

__device__ __forceinline__ Df d2df(double x) {
  const float h = __double2float_rn(x);
  return Df{h, __double2float_rn(x - (double)h)};
}

// ---- 0: FP32 CUDA cores: stride 9 words per line (odd: conflict-free) --------------
template <int P1>
__global__ void __launch_bounds__(kThreads) k_stage_f32(Op op, const double* __restrict__ x,
                                                      double* __restrict__ y, int reps) {
  constexpr int S = 9;
  __shared__ float sx[kLines * S];
  const long long base = (long long)blockIdx.x * kLines * P1;
  float m[P1 * P1];
#pragma unroll
  for (int k = 0; k < P1 * P1; ++k) m[k] = (float)op.m[k];
  for (int k = threadIdx.x; k < kLines * P1; k += kThreads) sx[(k / P1) * S + k % P1] = (float)x[base + k];
  __syncthreads();
  for (int r = 0; r < reps; ++r) {
    for (int l = threadIdx.x; l < kLines; l += kThreads) {
      float v[P1], o[P1];
#pragma unroll
      for (int i = 0; i < P1; ++i) v[i] = sx[l * S + i];
#pragma unroll
      for (int q = 0; q < P1; ++q) {
        float a = 0.f;
#pragma unroll
        for (int i = 0; i < P1; ++i) a = fmaf(m[q * P1 + i], v[i], a);
        o[q] = a;
      }
#pragma unroll
      for (int q = 0; q < P1; ++q) sx[l * S + q] = o[q];
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kLines * P1; k += kThreads) y[base + k] = (double)sx[(k / P1) * S + k % P1];
}

// ---- 1: double-float CUDA cores (operator in shared memory) -----------------------
template <int P1>
__global__ void __launch_bounds__(kThreads) k_stage_df(Op op, const double* __restrict__ x,
                                                     double* __restrict__ y, int reps) {
  constexpr int S = 9;
  __shared__ Df sx[kLines * S];
  __shared__ Df sm[P1 * P1];
  const long long base = (long long)blockIdx.x * kLines * P1;
  for (int k = threadIdx.x; k < P1 * P1; k += kThreads) sm[k] = d2df(op.m[k]);
  for (int k = threadIdx.x; k < kLines * P1; k += kThreads) sx[(k / P1) * S + k % P1] = d2df(x[base + k]);
  __syncthreads();
  for (int r = 0; r < reps; ++r) {
    for (int l = threadIdx.x; l < kLines; l += kThreads) {
      Df v[P1], o[P1];
#pragma unroll
      for (int i = 0; i < P1; ++i) v[i] = sx[l * S + i];
#pragma unroll
      for (int q = 0; q < P1; ++q) {
        Df acc{0.f, 0.f};
#pragma unroll
        for (int i = 0; i < P1; ++i) tdks::df_madd(acc, sm[q * P1 + i], v[i]);
        o[q] = acc;
      }
#pragma unroll
      for (int q = 0; q < P1; ++q) sx[l * S + q] = o[q];
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kLines * P1; k += kThreads) {
    const Df v = sx[(k / P1) * S + k % P1];
    y[base + k] = (double)v.hi + (double)v.lo;
  }
}

// ---- tensor-core forms ------------------------------------------------------------
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low 16 bits) = lo
  unsigned u;
  memcpy(&u, &v, 4);
  return u;
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ unsigned tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 2: BF16 operands.  Lines as rows of 16 bf16 (K padded with zeros), stored as 32-bit
// pairs with a row stride of 12 words (bank-conflict-free fragment loads).  Fragments of
// m16n8k16: A a0 = (row g, cols 2t, 2t+1), a1 = row g+8, a2/a3 = cols + 8; B b0 = (k = 2t,
// 2t+1; n = g), b1 = k + 8; C c0, c1 = (row g, cols 2t, 2t+1), c2, c3 = row g+8
// (g = lane / 4, t = lane % 4).
template <int P1>
__global__ void __launch_bounds__(kThreads) k_stage_bf16(Op op, const double* __restrict__ x,
                                                       double* __restrict__ y, int reps) {
  constexpr int SW = 12;   // 32-bit words per row (8 used: 16 bf16)
  __shared__ unsigned sx[kLines * SW];
  const long long base = (long long)blockIdx.x * kLines * P1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  for (int k = threadIdx.x; k < kLines * 8; k += kThreads) {
    const int l = k >> 3, w = k & 7, i0 = 2 * w;
    const float v0 = i0 < P1 ? (float)x[base + (long long)l * P1 + i0] : 0.f;
    const float v1 = i0 + 1 < P1 ? (float)x[base + (long long)l * P1 + i0 + 1] : 0.f;
    sx[l * SW + w] = pack_bf16(v0, v1);
  }
  auto mq = [&](int n, int k) -> float { return (n < P1 && k < P1) ? (float)op.m[n * P1 + k] : 0.f; };
  const unsigned b[2] = {pack_bf16(mq(gid, 2 * tig), mq(gid, 2 * tig + 1)),
                         pack_bf16(mq(gid, 2 * tig + 8), mq(gid, 2 * tig + 9))};
  __syncthreads();
  for (int r = 0; r < reps; ++r) {
#pragma unroll 1
    for (int t = 0; t < kLines / 64; ++t) {
      const int row0 = warp * (kLines / 4) + t * 16;
      const unsigned a[4] = {sx[(row0 + gid) * SW + tig], sx[(row0 + gid + 8) * SW + tig],
                             sx[(row0 + gid) * SW + tig + 4], sx[(row0 + gid + 8) * SW + tig + 4]};
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(d, a, b);
      __syncwarp();
      sx[(row0 + gid) * SW + tig] = pack_bf16(d[0], d[1]);
      sx[(row0 + gid + 8) * SW + tig] = pack_bf16(d[2], d[3]);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kLines * P1; k += kThreads) {
    const int l = k / P1, i = k % P1;
    const unsigned w = sx[l * SW + (i >> 1)];
    const unsigned h = (i & 1) ? (w >> 16) : (w & 0xffffu);
    y[base + k] = (double)__uint_as_float(h << 16);
  }
}

// 3: three TF32 products per product.  Lines as rows of 8 floats (K padded), row stride
// 12 words.  Fragments of m16n8k8: A a0 = (g, t), a1 = (g+8, t), a2 = (g, t+4),
// a3 = (g+8, t+4); B b0 = (k = t, n = g), b1 = (k = t+4, n = g); C as above.
template <int P1>
__global__ void __launch_bounds__(kThreads) k_stage_tf32x3(Op op, const double* __restrict__ x,
                                                         double* __restrict__ y, int reps) {
  constexpr int SW = 12;
  __shared__ float sx[kLines * SW];
  const long long base = (long long)blockIdx.x * kLines * P1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  for (int k = threadIdx.x; k < kLines * 8; k += kThreads) {
    const int l = k >> 3, i = k & 7;
    sx[l * SW + i] = i < P1 ? (float)x[base + (long long)l * P1 + i] : 0.f;
  }
  auto mq = [&](int n, int k) -> float { return (n < P1 && k < P1) ? (float)op.m[n * P1 + k] : 0.f; };
  const float bf[2] = {mq(gid, tig), mq(gid, tig + 4)};
  unsigned bh[2], bl[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    bh[k] = tf32(bf[k]);
    bl[k] = tf32(bf[k] - __uint_as_float(bh[k]));
  }
  __syncthreads();
  for (int r = 0; r < reps; ++r) {
#pragma unroll 1
    for (int t = 0; t < kLines / 64; ++t) {
      const int row0 = warp * (kLines / 4) + t * 16;
      const float af[4] = {sx[(row0 + gid) * SW + tig], sx[(row0 + gid + 8) * SW + tig],
                           sx[(row0 + gid) * SW + tig + 4], sx[(row0 + gid + 8) * SW + tig + 4]};
      unsigned ah[4], al[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ah[k] = tf32(af[k]);
        al[k] = tf32(af[k] - __uint_as_float(ah[k]));
      }
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      mma_tf32(d, al, bh);
      mma_tf32(d, ah, bl);
      mma_tf32(d, ah, bh);
      __syncwarp();
      sx[(row0 + gid) * SW + 2 * tig] = d[0];
      sx[(row0 + gid) * SW + 2 * tig + 1] = d[1];
      sx[(row0 + gid + 8) * SW + 2 * tig] = d[2];
      sx[(row0 + gid + 8) * SW + 2 * tig + 1] = d[3];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kLines * P1; k += kThreads) y[base + k] = (double)sx[(k / P1) * SW + k % P1];
}

template <int P1>
void launch_stage(int variant, int grid, cudaStream_t st, const Op& op, const double* x, double* y,
                  int reps) {
  switch (variant) {
    case 0: k_stage_f32<P1><<<grid, kThreads, 0, st>>>(op, x, y, reps); break;
    case 1: k_stage_df<P1><<<grid, kThreads, 0, st>>>(op, x, y, reps); break;
    case 2: k_stage_bf16<P1><<<grid, kThreads, 0, st>>>(op, x, y, reps); break;
    default: k_stage_tf32x3<P1><<<grid, kThreads, 0, st>>>(op, x, y, reps); break;
  }
}

}  // namespace

extern "C" tdks_status tdks_contraction_probe(int variant, int P1, const double* op_host,
                                              const double* x_dev, double* y_dev, int64_t n_lines,
                                              int reps, void* stream, double* ms_host) {
  if (variant < 0 || variant > 3 || P1 < 2 || P1 > kMaxP1 || !op_host || !x_dev || !y_dev || reps < 1 ||
      n_lines < kLines || n_lines % kLines != 0 || n_lines / kLines > (1 << 30))
    return TDKS_ERR_ARG;
  Op op;
  std::memset(&op, 0, sizeof(op));
  std::memcpy(op.m, op_host, (size_t)P1 * P1 * sizeof(double));
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = (int)(n_lines / kLines);
  auto launch = [&]() {
    switch (P1) {
      case 2: launch_stage<2>(variant, grid, st, op, x_dev, y_dev, reps); break;
      case 3: launch_stage<3>(variant, grid, st, op, x_dev, y_dev, reps); break;
      case 4: launch_stage<4>(variant, grid, st, op, x_dev, y_dev, reps); break;
      case 5: launch_stage<5>(variant, grid, st, op, x_dev, y_dev, reps); break;
      case 6: launch_stage<6>(variant, grid, st, op, x_dev, y_dev, reps); break;
      case 7: launch_stage<7>(variant, grid, st, op, x_dev, y_dev, reps); break;
      default: launch_stage<8>(variant, grid, st, op, x_dev, y_dev, reps); break;
    }
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return TDKS_ERR_CUDA;
  }
  launch();   // warm-up
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  float ms = 0.f;
  const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return TDKS_ERR_CUDA;
  if (ms_host) *ms_host = ms;
  return TDKS_OK;
}
