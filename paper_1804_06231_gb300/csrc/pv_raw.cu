// pv_raw.cu -- raw interaction throughput: every particle of one set against
// every particle of another, all lanes busy, with no window, no mask and no
// cut-off test.  The GPU counterpart of the paper's first experiment (Section
// 4: one particle against 2560, scalar against SIMD): it measures the cost of
// the interaction arithmetic of the density sweep on its own, the ceiling
// that the sorted sweeps are compared with.
#include <cuda_runtime.h>

#include "pv_internal.cuh"

namespace pv {
namespace {

constexpr int kRawThreads = 256;
constexpr int kRawTile = 1024;

// One thread per i; the j set is staged in tiles of kRawTile.  The per-pair
// arithmetic is that of the sweep's evaluation pass: r^2, q by approximate
// square root, the half-scaled kernel terms and two accumulations.
__global__ void __launch_bounds__(kRawThreads) k_raw_density(const float4* __restrict__ xi,
                                                             int ni,
                                                             const float4* __restrict__ xj,
                                                             int nj, float Hinv2, int reps,
                                                             float2* __restrict__ out) {
  pdl_enter();
  __shared__ float4 s[kRawTile];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float4 x = i < ni ? xi[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  float rho = 0.0f, D = 0.0f;
  for (int rep = 0; rep < reps; rep++) {
    for (int j0 = 0; j0 < nj; j0 += kRawTile) {
      const int len = min(kRawTile, nj - j0);
      __syncthreads();
      for (int e = threadIdx.x; e < len; e += blockDim.x) s[e] = xj[j0 + e];
      __syncthreads();
#pragma unroll 4
      for (int e = 0; e < len; e++) {
        const float4 q = s[e];
        const float dx = x.x - q.x, dy = x.y - q.y, dz = x.z - q.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        float wh, th;
        spline_half(sqrt_approx(r2 * Hinv2), wh, th);
        rho = fmaf(q.w, wh, rho);
        D = fmaf(q.w, th, D);
      }
    }
  }
  if (i < ni) out[i] = make_float2(rho, D);
}

// FP32 throughput probe: every thread runs kProbeChains independent chains
// a <- a b + c (b just below 1, so the values stay bounded), as scalar FFMA or
// as packed fma.rn.f32x2 pairs, and writes their sum so nothing is dropped.
constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 4;

template <bool Packed>
__global__ void __launch_bounds__(256) k_fp32_probe(int iters, float* __restrict__ sink) {
  pdl_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const float b = 0.99999994f, c = 1.0e-7f;
  float acc = 0.0f;
  if (Packed) {
    float2 a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; k++) a[k] = make_float2(t * 1e-9f + k, t * 1e-9f - k);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int it = 0; it < iters; it++) {
#pragma unroll
      for (int u = 0; u < kProbeUnroll; u++)
#pragma unroll
        for (int k = 0; k < kProbeChains; k++) a[k] = __ffma2_rn(a[k], b2, c2);
    }
#pragma unroll
    for (int k = 0; k < kProbeChains; k++) acc += a[k].x + a[k].y;
  } else {
    float a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; k++) a[k] = t * 1e-9f + k;
    for (int it = 0; it < iters; it++) {
#pragma unroll
      for (int u = 0; u < kProbeUnroll; u++)
#pragma unroll
        for (int k = 0; k < kProbeChains; k++) a[k] = fmaf(a[k], b, c);
    }
#pragma unroll
    for (int k = 0; k < kProbeChains; k++) acc += a[k];
  }
  sink[t] = acc;
}

}  // namespace

cudaError_t launch_fp32_probe(int packed, int iters, float* sink, int64_t threads,
                              double* flops, cudaStream_t st) {
  const int blocks = (int)(threads / 256);
  *flops = 2.0 * (packed ? 2.0 : 1.0) * kProbeChains * kProbeUnroll * (double)iters *
           (double)blocks * 256.0;
  if (blocks == 0) return cudaSuccess;
  if (packed)
    k_fp32_probe<true><<<blocks, 256, 0, st>>>(iters, sink);
  else
    k_fp32_probe<false><<<blocks, 256, 0, st>>>(iters, sink);
  return cudaGetLastError();
}

cudaError_t launch_raw_density(const float4* xi, int ni, const float4* xj, int nj, float H,
                               int reps, float2* out, cudaStream_t st) {
  if (ni == 0) return cudaSuccess;
  k_raw_density<<<(ni + kRawThreads - 1) / kRawThreads, kRawThreads, 0, st>>>(
      xi, ni, xj, nj, 1.0f / (H * H), reps, out);
  return cudaGetLastError();
}

}  // namespace pv
