// pv_backward.cu -- adjoint of the density gather.
//
// With g_i = dL/drho_i, k_i = dL/d(drho/dh)_i, W_r = dW/dr and W_hr =
// d2W/dh dr:
//   dL/dh_i = g_i drho/dh_i + k_i sum_j m_j d2W/dh2(r_ij, h_i)
//   dL/dx_i = sum_{j!=i} (x_i - x_j)/r_ij [ m_j (g_i W_r(r,H_i) + k_i W_hr(r,h_i)) [r<H_i]
//                                          + m_i (g_j W_r(r,H_j) + k_j W_hr(r,h_j)) [r<H_j] ]
// Both terms are gathered for particle i while sweeping the same sorted cell
// pairs as the forward pass (the second, "transposed" term is the scatter of
// the pair's symmetric position derivative, done as a gather), with the
// window widened to max(H_i, H_max of the other cell).
//
// Half-scaled shape functions (w, w', w'' of the workload's spline, divided
// by 16/pi; s = 1 - q):
//   th = (3w + q w')            q<1/2: 3/2 + q^2 (18q - 15)    else s^2 (3 - 6q)
//   uh = (12w + 8q w' + q^2 w'') q<1/2: 6 + q^2 (126q - 90)    else 6 s (7s^2 - 6s + 1)
//   vr = w'/q                   q<1/2: -6 + 9q                 else -3 s^2 / q
//   vh = (4w' + q w'')/q        q<1/2: -30 + 54q               else -12 s^2/q + 6 s
// so that dW/dh = -(16/pi) th/(h H^3), d2W/dh2 = (16/pi) uh/(h^2 H^3),
// W_r/r = (16/pi) vr/H^5 and W_hr/r = -(16/pi) vh/(h H^5).  With
// G = g/H^5 and K = k/(h H^5) per particle:
//   dL/dx_i = (16/pi) sum_j (x_i-x_j) [ m_j (G_i vr_i - K_i vh_i) + m_i (G_j vr_j - K_j vh_j) ]
//   dL/dh_i = (16/pi)/(h_i H_i^3) [ -g_i sum_j m_j th_i + (k_i/h_i) sum_j m_j uh_i ]
#include <cuda_runtime.h>

#include "pv_internal.cuh"

namespace pv {

namespace {

constexpr int kBlkI = 128;   // must match the plan kernel
constexpr int kTileJ = 512;

struct TaskB {
  int a, o, p0, p1, j0, j1;
};

__device__ __forceinline__ TaskB decode_b(int4 t) {
  TaskB r;
  r.a = t.x;
  r.o = t.y;
  r.p0 = t.z & 0xffff;
  r.p1 = (int)((unsigned)t.z >> 16);
  r.j0 = t.w & 0xffff;
  r.j1 = (int)((unsigned)t.w >> 16);
  return r;
}

// Upstream gradients to cell order, with the per-particle constants of the
// sweep: gk = {G = g/H^5, K = k/(h H^5), H^2 + guard, H^2 - guard},
// ghh = {1/H, H}.
__global__ void k_bwd_prep(GridDev g, const float* __restrict__ g_rho,
                           const float* __restrict__ g_D) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.n || *g.flags) return;
  const int i = g.orig[s];
  const BoxDev& B = g.boxes[g.cell_box[g.pcell[i]]];
  const float h = g.hs[s];
  const float H = g.gamma * h;
  const double Hd = (double)H;
  const double H5 = Hd * Hd * Hd * Hd * Hd;
  const float gi = g_rho[i];
  const float ki = g_D ? g_D[i] : 0.0f;
  const float gb = guard_band(H, B.edge_f);
  g.gk[s] = make_float4((float)((double)gi / H5), (float)((double)ki / ((double)h * H5)),
                        H * H + gb, H * H - gb);
  g.ghh[s] = make_float2(1.0f / H, H);
}

__device__ __forceinline__ void spline_bwd(float q, float qinv, float& th, float& uh, float& vr,
                                           float& vh) {
  const float q2 = q * q;
  const float s = fmaxf(1.0f - q, 0.0f);
  const float s2 = s * s;
  if (q < 0.5f) {
    th = fmaf(q2, fmaf(18.0f, q, -15.0f), 1.5f);
    uh = fmaf(q2, fmaf(126.0f, q, -90.0f), 6.0f);
    vr = fmaf(9.0f, q, -6.0f);
    vh = fmaf(54.0f, q, -30.0f);
  } else {
    th = s2 * fmaf(-6.0f, q, 3.0f);
    uh = 6.0f * s * fmaf(7.0f * s, s, fmaf(-6.0f, s, 1.0f));
    vr = -3.0f * s2 * qinv;
    vh = fmaf(-12.0f * s2, qinv, 6.0f * s);
  }
}

__device__ __forceinline__ void spline_bwd_v(float q, float qinv, float& vr, float& vh) {
  const float s = fmaxf(1.0f - q, 0.0f);
  const float s2 = s * s;
  if (q < 0.5f) {
    vr = fmaf(9.0f, q, -6.0f);
    vh = fmaf(54.0f, q, -30.0f);
  } else {
    vr = -3.0f * s2 * qinv;
    vh = fmaf(-12.0f * s2, qinv, 6.0f * s);
  }
}

__global__ void __launch_bounds__(kBlkI) k_backward_tasks(GridDev g) {
  __shared__ float4 s_x[kTileJ];
  __shared__ float4 s_a[kTileJ];
  __shared__ float2 s_h[kTileJ];
  __shared__ float s_d[kTileJ];
  __shared__ int s_j[kTileJ];
  __shared__ int s_task;
  if (*g.flags) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntask = *g.ntask;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(g.task_next, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= ntask) break;
    const TaskB tk = decode_b(g.tasks[t]);
    const int a = tk.a, o = tk.o;
    const int b = neighbour_cell(g, a, o);
    const int na = g.cell_count[a], nb = g.cell_count[b];
    const int ca = g.cell_start[a], cb = g.cell_start[b];
    const BoxDev B = g.boxes[g.cell_box[a]];
    const Slot sl = slot_info(o);
    const float off = sl.v2 ? vnorm(sl.v2) * B.edge_f : 0.0f;
    const size_t kbase = (size_t)sl.k * g.n;
    const float Hmax_b = g.cell_Hmax[b];

    const int p = tk.p0 + warp * 32 + lane;
    const bool valid = p < tk.p1;
    float xi = 0.f, yi = 0.f, zi = 0.f, mi = 0.f, Gi = 0.f, Ki = 0.f;
    float Hsq_hi = -1.f, Hsq_lo = -1.f, Hinv = 0.f, Hi = 0.f;
    double Hd = 0.0;
    int si = 0;
    float d_lo = 3.0e38f, d_hi = -3.0e38f;
    if (valid) {
      const int pos_i = (o == kSelfSlot) ? p : order_pos(sl.s, na - 1 - p, na);
      si = ca + g.perm[kbase + ca + pos_i];
      const float4 x = g.xm[si];
      const float4 ak = g.gk[si];
      const float2 hh = g.ghh[si];
      xi = x.x - sl.ox * B.edge_f;
      yi = x.y - sl.oy * B.edge_f;
      zi = x.z - sl.oz * B.edge_f;
      mi = x.w;
      Gi = ak.x; Ki = ak.y; Hsq_hi = ak.z; Hsq_lo = ak.w;
      Hinv = hh.x; Hi = hh.y;
      Hd = g.gamma_d * (double)g.hs[si];
      const float di = sl.s * g.dist[kbase + ca + pos_i];
      const float reach = fmaxf(Hi, Hmax_b) + B.pad;
      d_lo = di - reach;
      d_hi = di + reach;
    }
    float w_lo = d_lo, w_hi = d_hi;
    for (int s = 16; s > 0; s >>= 1) {
      w_lo = fminf(w_lo, __shfl_xor_sync(0xffffffffu, w_lo, s));
      w_hi = fmaxf(w_hi, __shfl_xor_sync(0xffffffffu, w_hi, s));
    }
    float Sth = 0.f, Suh = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    for (int j0 = tk.j0; j0 < tk.j1; j0 += kTileJ) {
      const int len = min(kTileJ, tk.j1 - j0);
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const int pos_j = order_pos(sl.s, j0 + e, nb);
        const int sj = cb + g.perm[kbase + cb + pos_j];
        s_x[e] = g.xm[sj];
        s_a[e] = g.gk[sj];
        s_h[e] = g.ghh[sj];
        s_d[e] = sl.s * g.dist[kbase + cb + pos_j] + off;
        s_j[e] = sj;
      }
      __syncthreads();
      if (w_hi > w_lo) {
        const int lo = (o == kSelfSlot) ? upper_bound_f(s_d, len, w_lo) : 0;
        const int hi = lower_bound_f(s_d, len, w_hi);
        for (int e = lo; e < hi; e++) {
          const float4 xj = s_x[e];
          const float dx = xi - xj.x, dy = yi - xj.y, dz = zi - xj.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const float4 aj = s_a[e];
          bool own = r2 < Hsq_hi;
          bool trans = valid && r2 < aj.z;
          if (own || trans) {
            if (own && r2 >= Hsq_lo) own = guard_inside(g.pos64, si, s_j[e], B.L, B.inv_L, Hd);
            if (trans && r2 >= aj.w)
              trans = guard_inside(g.pos64, si, s_j[e], B.L, B.inv_L,
                                   g.gamma_d * (double)g.hs[s_j[e]]);
            const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
            const float r = r2 * rinv;
            float c = 0.0f;
            if (own) {
              float th, uh, vr, vh;
              spline_bwd(r * Hinv, Hi * rinv, th, uh, vr, vh);
              Sth = fmaf(xj.w, th, Sth);
              Suh = fmaf(xj.w, uh, Suh);
              c = xj.w * fmaf(Gi, vr, -Ki * vh);
            }
            if (trans) {
              const float2 hj = s_h[e];
              float vr, vh;
              spline_bwd_v(r * hj.x, hj.y * rinv, vr, vh);
              c = fmaf(mi, fmaf(aj.x, vr, -aj.y * vh), c);
            }
            gx = fmaf(c, dx, gx);
            gy = fmaf(c, dy, gy);
            gz = fmaf(c, dz, gz);
          }
        }
      }
      __syncthreads();
    }
    if (valid) {
      double* acc = reinterpret_cast<double*>(g.gacc);
      const size_t N = (size_t)g.n;
      if (Sth != 0.f || Suh != 0.f) {
        atomicAdd(&acc[si], (double)Sth);
        atomicAdd(&acc[N + si], (double)Suh);
      }
      if (gx != 0.f || gy != 0.f || gz != 0.f) {
        atomicAdd(&acc[2 * N + si], (double)gx);
        atomicAdd(&acc[3 * N + si], (double)gy);
        atomicAdd(&acc[4 * N + si], (double)gz);
      }
    }
  }
}

__global__ void k_bwd_finalize(GridDev g, const float* __restrict__ g_rho,
                               const float* __restrict__ g_D, float* __restrict__ g_pos,
                               float* __restrict__ g_h) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.n) return;
  double* acc = reinterpret_cast<double*>(g.gacc);
  const size_t N = (size_t)g.n;
  if (!*g.flags) {
    const int i = g.orig[s];
    const double h = (double)g.hs[s];
    const double H = g.gamma_d * h;
    const double c = (16.0 / 3.14159265358979323846) * (double)*g.m_max;
    const double gi = g_rho[i];
    const double ki = g_D ? (double)g_D[i] : 0.0;
    g_pos[3 * (size_t)i + 0] = (float)(c * acc[2 * N + s]);
    g_pos[3 * (size_t)i + 1] = (float)(c * acc[3 * N + s]);
    g_pos[3 * (size_t)i + 2] = (float)(c * acc[4 * N + s]);
    if (g_h) g_h[i] = (float)(c / (h * H * H * H) * (-gi * acc[s] + (ki / h) * acc[N + s]));
  }
  for (int q = 0; q < 5; q++) acc[q * N + s] = 0.0;
}

}  // namespace

cudaError_t launch_backward(const GridDev& g, const float* g_rho, const float* g_drho_dh,
                            float* g_pos, float* g_h, int num_sms, cudaStream_t st) {
  if (g.n == 0) return cudaSuccess;
  const int nb = (g.n + 255) / 256;
  k_bwd_prep<<<nb, 256, 0, st>>>(g, g_rho, g_drho_dh);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = launch_plan(g, 1, 0, 1, 1, st)) != cudaSuccess) return e;  // all cells as tasks
  k_backward_tasks<<<num_sms * 8, kBlkI, 0, st>>>(g);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_bwd_finalize<<<nb, 256, 0, st>>>(g, g_rho, g_drho_dh, g_pos, g_h);
  return cudaGetLastError();
}

}  // namespace pv
